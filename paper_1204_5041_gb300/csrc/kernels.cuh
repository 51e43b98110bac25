// Launchers of the library's kernels (one translation unit each), called by the C ABI layer.
#pragma once

#include "isw_internal.cuh"

namespace isw {

// api.cu: number of work chunks along the streamed axis for ntiles tiles of the other axis, nst
// streamed tiles and `slots` resident CTAs (near-equal waves; at least two streamed tiles per
// chunk; at most max_split chunks)
int choose_split(int64_t ntiles, int64_t nst, int slots, int max_split, int min_items = 0, int min_chunk = 256);
constexpr int kMapItemsPerSlot = 64;   // work items per CTA slot that the map's chunk count aims at
constexpr int kAdjItemsPerSlot = 64;   // the same for the adjoint's pixel chunks,
constexpr int kAdjMinChunk = 32;       // each chunk keeping at least this many pixel tiles

// probe.cu: FMA-pipe throughput (flop/s, FMA = 2) of the FP32 or FP64 pipe; sink is never written
int fma_probe(bool f64, int num_sms, double *sink, double *flops, cudaStream_t s);

// healpix.cu
int launch_pix2vec(int64_t N, int64_t pix0, int64_t npix, const int64_t *pix_list, double *out, int64_t ld,
                   DevStatus *st, cudaStream_t s);
void launch_pixel_table(int64_t N, int mode, int64_t pix0, int64_t npix, const int64_t *pix_list, int tx, int ty,
                        int64_t ntiles, double *nv, int64_t ldn, int64_t *outidx, float4 *caps, DevStatus *st,
                        cudaStream_t s);

// A gnomonic patch: orthonormal frame (e1, e2, e3) with e3 the centre, M x M pixels of
// coordinate pitch width / M; pixel (i, j) at (xi, eta) = ((i + 1/2 - M/2), (j + 1/2 - M/2)) * pitch,
// direction (xi e1 + eta e2 + e3) / norm, output slot j M + i.
struct PatchSpec {
    double frame[9];
    int64_t M;
    double width;
};
// patch pixel table: compact tx x ty blocks of the M x M grid (caps as for the sphere)
void launch_patch_table(const PatchSpec &p, int tx, int ty, int64_t ntiles, double *nv, int64_t ldn,
                        int64_t *outidx, float4 *caps, cudaStream_t s);

// flat.cu: flat-sky patch map (pixel tiles 32 x flat_ty() of the patch table)
int flat_seg_tile();
int flat_tx();
int flat_ty();
size_t flat_record_bytes();   // FP32 + FP64 record bytes per sample
int flat_slots(bool f64, int num_sms);
void launch_flat_pack(const double *S, int64_t n, int64_t ld, const PatchSpec &p, double xo0, double xo1, double xo2,
                      double GU, int64_t n_pad, void *r32, void *r64, cudaStream_t s);
void launch_map_flat(bool f64, const void *r32, const void *r64, const int64_t *outidx, int64_t ntiles, int64_t nst,
                     int split, int64_t M, double pitch, double *theta, double *partial, int accumulate,
                     DevStatus *st, unsigned long long *queue, uint32_t wait_polls, int grid, cudaStream_t s);

// cl.cu: angular power spectrum (F: double[2][4N-1][lmax+1] workspace; alm: double[2][lmax+1][lmax+1])
int cl_max_nside();
void launch_map_cl(int64_t N, const double *map, int64_t lmax, double *F, double *alm, double *cl, cudaStream_t s);

// lightcone.cu
void launch_lightcone(int mode, const double *nodes, int64_t n, int64_t ld, const double *P, int64_t nloops,
                      int64_t ldp, double t_box, double xo0, double xo1, double xo2, double t_obs, double tol,
                      int max_iter, double *out, int64_t ld_out, double *tau, int32_t *status, DevStatus *st,
                      cudaStream_t s);
// one launch over many shells: per-node shell lookup through shell_off (device copies)
void launch_lightcone_shells(const double *nodes, int64_t n, int64_t ld, const int64_t *shell_off, int64_t nshell,
                             const double *t_box, const int32_t *mode, const double *P, int64_t nloops, int64_t ldp,
                             double xo0, double xo1, double xo2, double t_obs, double tol, double *out,
                             int64_t ld_out, DevStatus *st, cudaStream_t s);

// lcadj.cu: adjoint of the light-cone solve.  runs (int[nloops], zeroed by the caller), first,
// last (int64[nloops]) are workspace of the Burden per-loop reduction; gl may be NULL in LINEAR mode.
void launch_lightcone_adjoint(int mode, const double *nodes, int64_t n, int64_t ld, const double *P, int64_t nloops,
                              int64_t ldp, double t_box, double xo0, double xo1, double xo2, const double *tau,
                              const double *gs, int64_t ldgs, int ngs, double *gn, int64_t ldgn, double *gl,
                              int64_t ldgl, int *runs, int64_t *first, int64_t *last, DevStatus *st, cudaStream_t s);

// cone.cu: stacking with HEALPix cones
void launch_vec2pix(int64_t N, const double *v, int64_t n, int64_t ld, int64_t *pix, DevStatus *st, cudaStream_t s);
void launch_box_place(const double *nodes, int64_t ld, const int64_t *off_out, const int64_t *src_start,
                      int64_t nshell, const double *place, double *out, int64_t ld_out, int64_t n_out,
                      cudaStream_t s);
// scratch: incl int32[n], block_tot int64[cone_cut_scratch_blocks(n) + 1]
int64_t cone_cut_scratch_blocks(int64_t n);
void launch_cone_cut(const double *S, int64_t ld, int64_t n, const int64_t *off, int64_t nshell, int64_t nside_hz,
                     const int64_t *cone_pix, const double *r_lo, const double *r_hi, double xo0, double xo1,
                     double xo2, int32_t *incl, int64_t *block_tot, double *out, int64_t ld_out, int64_t *off_out,
                     int64_t *count, cudaStream_t s);

// sort.cu: spatial order of the samples (stable radix sort of the Morton code of Xhat); returns the
// device array perm[n] (record s holds sample perm[s]), inside scratch of sort_scratch_bytes(n)
size_t sort_scratch_bytes(int64_t n);
const uint32_t *launch_spatial_order(const double *S, int64_t n, int64_t ld, double xo0, double xo1, double xo2,
                                     void *scratch, cudaStream_t s);
int spatial_order_launches();

// pack.cu: per-sample records of the map kernels and per-tile caps
// perm (may be NULL): record s is built from sample perm[s] (else from sample s)
// far (may be NULL): far-field records for the FP32 pair kernel, pair-interleaved (n_pad even)
// mid (may be NULL): mid-range records for the FP32 near-field pass
// far64 (may be NULL): far-field records for the FP64 kernel
void launch_pack(const double *samples, int64_t n, int64_t ld, double xo0, double xo1, double xo2, double GU,
                 double theta_pix, double near_k, int64_t n_pad, const uint32_t *perm, Seg32 *s32, Seg64 *s64,
                 Far2 *far, Mid2 *mid, Far64 *far64, DevStatus *st, cudaStream_t s);
void launch_seg_caps(const Seg32 *s32, const Seg64 *s64, int64_t n, int64_t n_pad, int seg_tile, float b_min,
                     SegCap *caps, cudaStream_t s);

// map.cu
struct MapArgs {
    const double *nv;        // pixel table directions [3][ldn]
    int64_t ldn;
    const int64_t *outidx;   // pixel table output indices
    const float4 *pcaps;     // pixel tile caps
    int64_t ntiles;          // pixel tiles
    const Seg32 *s32;
    const Seg64 *s64;
    const Far2 *far;         // far-field records of sample pairs (FP32 kernels)
    const Mid2 *mid;         // mid-range records of samples (FP32 near-field pass)
    const Far64 *far64;      // far-field records of samples (FP64 kernel)
    const SegCap *scaps;
    int64_t nst;             // segment tiles
    int split;               // segment chunks
    float b_min;
    float d_far;             // tile pairs at least this chord apart use the far-field form
    double *theta;           // output (RING or list order)
    double *partial;         // [split][ntiles*tile] when split > 1
    int accumulate;
    DevStatus *st;
    int64_t tile_stride;     // 1; > 1 only when timing variants: every tile_stride-th pixel tile
    unsigned long long *queue;   // work counters (far pass or FP64 kernel, near pass), zero at launch
    uint32_t wait_polls;     // limit of the consumer waits (kWaitPolls by default)
};
struct Variant {
    int threads, ppt, seg_tile, tx, ty;
};
int num_f32_variants();
Variant f32_variant(int idx);
int f64_seg_tile();
Variant f64_variant();
// slots = resident CTAs on the whole GPU for the variant
int map_f32c_slots(int idx, int num_sms);
int map_f64_slots(int num_sms);
void launch_map_f32c(int idx, const MapArgs &a, int grid, cudaStream_t s);
void launch_map_f32c_near(int idx, const MapArgs &a, int num_sms, cudaStream_t s);
void launch_map_f64(const MapArgs &a, int grid, cudaStream_t s);
void launch_reduce_partials(const MapArgs &a, int tile_sz, cudaStream_t s);

// adjoint.cu
struct AdjArgs {
    const Pix32 *p32;        // pixel records in tile order
    const Pix64 *p64;
    const PixF2 *pf2;        // far-field records of pixel pairs (FP32 kernel)
    const float4 *pcaps;     // pixel tile caps
    int64_t npix_tiles;
    const Seg32 *s32;
    const Seg64 *s64;
    const SegCap *scaps;     // caps of the adjoint's sample tiles
    int64_t nseg_tiles;
    int64_t n, n_pad;
    int split;               // pixel chunks
    int ngrad;               // 6 or 9
    float b_min, d_far;
    double *grad;            // [ngrad][ld_g]
    int64_t ld_g;
    double *partial;         // [split][ngrad][n_pad] when split > 1
    DevStatus *st;
    unsigned long long *queue;   // work counter, zero at launch
    uint32_t wait_polls;     // limit of the consumer waits (kWaitPolls by default)
};
int adj_seg_tile(int prec);
int adj_pix_tile(int prec);
int adj_slots(int prec, int ngrad, int num_sms);
void launch_pack_pixels(const double *nv, int64_t ldn, const int64_t *outidx, const double *g, int64_t tot,
                        Pix32 *p32, Pix64 *p64, PixF2 *pf2, cudaStream_t s);
void launch_adjoint(int prec, const AdjArgs &a, int grid, cudaStream_t s);

}  // namespace isw
