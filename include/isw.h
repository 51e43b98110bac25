/*
 * isw.h -- C ABI of the GB300 (sm_103a) full-sky string ISW map library (libisw.so).
 *
 * The library evaluates the all-sky integrated Sachs-Wolfe temperature shift sourced by
 * Nambu-Goto strings on the observer's past light cone, Eq. (1)-(2) of Ringeval & Bouchet,
 * "All sky CMB map from cosmic strings integrated Sachs-Wolfe effect" (arXiv:1204.5041):
 *
 *   Theta(n) = -4 GU  sum_s  u.D / D^2  eps_s dsigma_s,    D = X n - X_s,  X = |X_s - x_obs|,
 *   u = Xdot - (n.X') X' / (1 + n.Xdot),                 eps^2 = X'^2 / (1 - Xdot^2),
 *
 * for every HEALPix RING pixel direction n (Sec. II.D), summed over every string sample s
 * on the light cone (Sec. II.A, Sec. III.A: no segment is cut).
 *
 * Units and conventions: flat conformal coordinates, c = 1; the observer sits at x_obs at
 * conformal time t_obs (horizon units: x_obs = 0, t_obs = 1).  GU is the string tension in
 * Planck units; maps scale linearly with it.
 *
 * Memory: every array argument is a DEVICE pointer owned by the caller (for example a
 * PyTorch CUDA tensor's data pointer), except where marked (host).  Device arrays must live on
 * the context's GPU (or be managed memory); a pointer to host memory or to another GPU's memory
 * is rejected with ISW_EINVAL before anything is enqueued.  Arrays of several rows
 * are row-major "double[rows][ld]": element (r, k) sits at base[r * ld + k].  The library
 * allocates only its own workspace, held in the context and freed by isw_destroy.
 *
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).  Every compute
 * call only enqueues work on it and returns; results are ready when the stream is.
 *
 * Errors: every call returns an isw_status.  Argument errors (ISW_EINVAL) are found on the
 * host before anything is enqueued.  Conditions found on the device (a sample with
 * |Xdot| >= 1, a light-cone iteration that did not converge, a bounded wait that ran out)
 * are recorded in a device status word and returned by isw_check_status, which
 * synchronises the stream.  The message of the last error is available from
 * isw_last_error.  No C++ exception crosses this interface.
 *
 * Threads: a context may be used by one host thread at a time; use one context per
 * thread (they may share a device).
 */
#ifndef ISW_H
#define ISW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct isw_ctx isw_ctx;

typedef enum {
    ISW_OK = 0,
    ISW_EINVAL = 1,   /* bad argument: null pointer, host pointer where a device one is due, bad size */
    ISW_ECUDA = 2,    /* a CUDA runtime call failed (message in isw_last_error) */
    ISW_EDOMAIN = 3,  /* a sample with 1 - Xdot^2 <= 0 or a non-finite weight (skipped) */
    ISW_ENOCONV = 4,  /* a light-cone solve hit its iteration cap */
    ISW_ETIMEOUT = 5, /* a bounded device-side wait ran out (the kernel returned early) */
    ISW_ENOMEM = 6    /* workspace allocation failed */
} isw_status;

/* precision of the pair arithmetic */
enum { ISW_F64 = 0, ISW_F32C = 1 };
/* light-cone solve mode */
enum { ISW_LINEAR = 0, ISW_BURDEN = 1 };
/* patch maps: full-sky formula or the flat-sky / small-angle approximation */
enum { ISW_FULLSKY = 0, ISW_FLATSKY = 1 };
/* isw_map_batched flags */
enum { ISW_SKIP_LIGHTCONE = 1, ISW_GRAPH = 2, ISW_AUTOTUNE = 4 };
/* isw_set_param keys */
enum {
    ISW_PARAM_NEAR_K = 0,
    ISW_PARAM_B_MIN = 1,
    ISW_PARAM_SPLIT = 2,
    ISW_PARAM_VARIANT = 3,
    ISW_PARAM_TIMING = 4,
    ISW_PARAM_D_FAR = 5,
    ISW_PARAM_NUM_VARIANTS = 6,  /* read-only (isw_get_param): number of FP32 kernel variants */
    ISW_PARAM_WAIT_POLLS = 7
};

/* Create a context bound to CUDA device `device`.  Allocates a small device status block.
 * Returns ISW_EINVAL for a bad device index, ISW_ECUDA / ISW_ENOMEM on CUDA failures. */
int isw_create(isw_ctx **ctx, int device);

/* Free the context and its workspace (synchronises the device first). */
int isw_destroy(isw_ctx *ctx);

/* Message of the last error on this context ("" when none).  Owned by the context. */
const char *isw_last_error(const isw_ctx *ctx);

/* Synchronise `stream`, then return and clear the device status: ISW_ETIMEOUT, ISW_ENOCONV
 * or ISW_EDOMAIN (in that order of precedence) if any kernel recorded one since the last
 * call, else ISW_OK.  counts (host, may be NULL) receives 3 counters accumulated since the
 * last call: pairs with D = 0 exactly (zero term), skipped samples (|Xdot| >= 1 or
 * non-finite weight), pairs that the FP32 path evaluated in FP64 (near field). */
int isw_check_status(isw_ctx *ctx, void *stream, int64_t *counts);

/* Tunables: ISW_PARAM_NEAR_K (default 2): a pair is "near" when the chord |n - Xhat| is
 * below near_k * max(pixel size, angular length of the sample's segment); ISW_PARAM_B_MIN
 * (default 0.01): a pair with 1 + n.Xdot below b_min is evaluated in FP64 by the FP32 path;
 * ISW_PARAM_SPLIT: number of segment chunks of the forward maps (0 = automatic: enough
 * (pixel tile, chunk) work items to fill every resident CTA in near-equal waves and at least 64
 * per resident CTA, while each chunk keeps 256 segment tiles; chunk partials cost 8 bytes per
 * pixel and chunk of device memory);
 * ISW_PARAM_VARIANT: FP32 kernel variant (-1 = automatic); ISW_PARAM_D_FAR (default 0.25):
 * segment tiles whose every pair is at least this chord apart from the pixel tile use the
 * FP32 far-field form (d.d = 2 (1 - n.Xhat), Xdot.d and X'.d from per-sample constants);
 * 4 disables it; ISW_PARAM_TIMING (default 0):
 * when 1, every launch of the pair kernel (the all-pairs sum of isw_map and
 * isw_map_batched: the FP32 far- and near-field passes and the chunk reduction between them, or
 * the FP64 kernel and its reduction) is bracketed by CUDA events on its stream, read by
 * isw_get_timing.  ISW_PARAM_WAIT_POLLS (default 2^22; a negative value restores it): the
 * limit, in mbarrier try_wait polls, of every wait of the pair kernels (isw_map, isw_map_batched,
 * isw_map_adjoint, isw_map_patch) for a stage of records to land in shared memory.  A wait that
 * runs out stops its block: the block waits for its own copies still in flight (a separate limit
 * of 2^26 polls), records ISW_ETIMEOUT and returns, so the output is incomplete and
 * isw_check_status returns ISW_ETIMEOUT.  0 makes every wait give up at once, which exercises
 * this failure path without a fault. */
int isw_set_param(isw_ctx *ctx, int key, double value);

/* Read a tunable into *value (host pointer).  For ISW_PARAM_VARIANT the value is the FP32
 * kernel variant the last FP32 map of this context used (the override, the autotuner's pick or
 * the default), or -1 before any FP32 map. */
int isw_get_param(const isw_ctx *ctx, int key, double *value);

/* Timing of the pair kernel (ISW_PARAM_TIMING = 1): synchronises the recorded events and
 * returns in *ms the summed device time of the pair-kernel launches recorded since the last
 * reset, in *pair_launches their number and in *all_launches the number of kernels of any
 * kind this context launched in that interval (counted whether or not timing is on).  All
 * three are host pointers and may be NULL.  reset = 1 clears the record.  At most 4096
 * pair-kernel launches are timed between resets (later ones are counted, not timed). */
int isw_get_timing(isw_ctx *ctx, double *ms, int64_t *pair_launches, int64_t *all_launches, int reset);

/* Measured throughput of the GPU's fused multiply-add pipe, the peak against which the pair
 * kernels' FP32 (prec = ISW_F32C) or FP64 (prec = ISW_F64) arithmetic is stated (the paper has no
 * counterpart: it times CPU cores).  A calibration kernel runs independent FMA chains on every
 * SM; *flop_per_s (host) receives the best of three timed launches, an FMA counting two flops.
 * Synchronises `stream`; takes a few milliseconds (FP32) to tens of milliseconds (FP64). */
int isw_fma_rate(isw_ctx *ctx, int prec, double *flop_per_s, void *stream);

/* Pixel centres, HEALPix RING scheme (Sec. II.D; Gorski et al. 2005 geometry).
 *   nside    : resolution N >= 1 (N_pix = 12 N^2), N <= 2^24
 *   pix_list : device int64[npix] of RING indices, or NULL for the range pix0 .. pix0+npix-1
 *   vec_out  : device double[3][ld_out] receiving (x, y, z) of each pixel, ld_out >= npix
 * The directions are bit-identical to the published specification of this library: exact
 * integer ring arithmetic, IEEE-rounded z and sin(theta), and an own sin/cos series.
 * Indices outside [0, N_pix) write NaN and set ISW_EINVAL in the device status. */
int hp_pix2vec_ring(isw_ctx *ctx, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list,
                    double *vec_out, int64_t ld_out, void *stream);

/* RING pixel of arbitrary directions (the inverse of hp_pix2vec_ring; Gorski et al. 2005 rules).
 *   vec     : device double[3][ld] directions (any positive length), ld >= n
 *   pix_out : device int64[n]
 * phi comes from the library's own atan2 series and every step is an IEEE operation in a fixed
 * order, so the pixel decided for a direction is reproducible.  A zero or non-finite
 * direction writes -1 and sets ISW_EINVAL in the device status. */
int hp_vec2pix_ring(isw_ctx *ctx, int64_t nside, const double *vec, int64_t n, int64_t ld, int64_t *pix_out,
                    void *stream);

/* Past-light-cone intersection (Eq. 1: the string points X with X cap x_gamma; Sec. II.B:
 * X' and Xdot are recorded at the crossing).
 *   mode = ISW_LINEAR: nodes_in is double[10][ld]: X(3), Xdot(3), X'(3), dsigma at box time
 *          t_box; the worldline X + Xdot*D meets |X - x_obs| = t_obs - tau at the past root
 *          D = tau - t_box (closed form); Xdot, X', dsigma are carried unchanged.
 *   mode = ISW_BURDEN: nodes_in rows 0, 1 are (loop id, sigma) and row 9 dsigma; loop_params
 *          is double[17][ldp] per loop: centre (3), rotation (9, row-major), L, m, n, psi,
 *          t0; the sample is the analytic Burden worldsheet at the retarded time, found by
 *          safeguarded Newton iteration (at most 60 steps, residual <= 4 ulp of t_obs).
 *   x_obs    : host double[3]; t_obs: observer time (> t_box for LINEAR)
 *   samples_out : device double[10][ld_out] (X, Xdot, X', dsigma on the cone)
 *   tau_out  : device double[n] retarded times (may be NULL)
 *   status   : device int32[n] per-node status (ISW_OK, ISW_EDOMAIN, ISW_ENOCONV, ISW_EINVAL),
 *              may be NULL; any non-OK node is also recorded in the context status.
 * The arithmetic is IEEE double without contraction, reproducible operation by operation. */
int lightcone_intersect(isw_ctx *ctx, int mode, const double *nodes_in, int64_t n, int64_t ld,
                        const double *loop_params, int64_t nloops, int64_t ldp, double t_box,
                        const double *x_obs, double t_obs, double *samples_out, int64_t ld_out,
                        double *tau_out, int32_t *status, void *stream);

/* lightcone_intersect for many shells in one launch (the solve isw_map_batched runs):
 *   nodes        : device double[10][ld] of all shells; shell_off host int64[nshell+1]
 *                  (shell_off[0] = 0), t_box host double[nshell], mode host int32[nshell]
 *   loop_params  : as in lightcone_intersect (required when a shell is ISW_BURDEN)
 *   samples_out  : device double[10][ld_out], ld_out >= shell_off[nshell]
 * Non-OK nodes are recorded in the context status (read with isw_check_status). */
int lightcone_intersect_shells(isw_ctx *ctx, const double *nodes, int64_t ld, const int64_t *shell_off,
                               int64_t nshell, const double *t_box, const int32_t *mode, const double *loop_params,
                               int64_t nloops, int64_t ldp, const double *x_obs, double t_obs,
                               double *samples_out, int64_t ld_out, void *stream);

/* Stacking with HEALPix cones (Sec. III.B, Fig. 1: the comoving volume is voxelised by the
 * cones of a coarse HEALPix grid, each filled from a simulation box rotated to face the
 * observer; one box serves several cones).
 *
 * box_place: shell k takes the nodes of box shell_box[k] and maps X -> R_k X + T_k,
 * Xdot -> R_k Xdot, X' -> R_k X' (dsigma unchanged).
 *   nodes_box     : device double[10][ld_box] of all boxes, box_off host int64[nbox+1]
 *   shell_box     : host int64[nshell], the box of each shell (a box may serve many shells)
 *   place         : device double[nshell][12]: R_k row-major (9), then T_k (3)
 *   nodes_out     : device double[10][ld_out], ld_out >= the total node count
 *   shell_off_out : host int64[nshell+1], written on return (before the kernel runs)
 * (R x)_i is evaluated as (R_i0 x_0 + R_i1 x_1) + R_i2 x_2 in IEEE double (reproducible). */
int box_place(isw_ctx *ctx, const double *nodes_box, int64_t ld_box, const int64_t *box_off, int64_t nbox,
              const int64_t *shell_box, int64_t nshell, const double *place, double *nodes_out, int64_t ld_out,
              int64_t *shell_off_out, void *stream);

/* cone_cut: keep a light-cone sample of shell k when the direction of X - x_obs lies in RING
 * pixel cone_pix[k] of resolution nside_hz and r_lo[k] <= |X - x_obs| < r_hi[k]; kept samples
 * are compacted in input order (a stable, deterministic stream compaction).
 *   samples       : device double[10][ld]; shell_off host int64[nshell+1]
 *   cone_pix, r_lo, r_hi : device arrays of nshell
 *   samples_out   : device double[10][ld_out], ld_out >= shell_off[nshell]
 *   shell_off_out : device int64[nshell+1], kept-sample offsets of the shells
 *   count         : host int64* or NULL; when given, the call synchronises the stream and
 *                   writes the number of kept samples (what isw_map needs as n) */
int cone_cut(isw_ctx *ctx, const double *samples, int64_t ld, const int64_t *shell_off, int64_t nshell,
             int64_t nside_hz, const int64_t *cone_pix, const double *r_lo, const double *r_hi,
             const double *x_obs, double *samples_out, int64_t ld_out, int64_t *shell_off_out, int64_t *count,
             void *stream);

/* The map of Eq. (1)-(2) (Sec. III.A: every pixel sums every sample, none cut).
 *   nside, pix0, npix, pix_list : pixels as in hp_pix2vec_ring; npix = 12 N^2 with
 *              pix0 = 0 and pix_list = NULL selects the full sky (processed in compact tiles)
 *   samples  : device double[10][ld] on the light cone (output of lightcone_intersect)
 *   x_obs    : host double[3] (NULL = origin); GU: tension
 *   prec     : ISW_F32C (FP32 pair arithmetic with per-pixel compensated sums; near-field
 *              pairs and pairs with 1 + n.Xdot < b_min in FP64) or ISW_F64 (all FP64)
 *   accumulate : 0 writes theta_out, 1 adds to it
 *   theta_out: device double[npix] in the order of the selected pixels
 * A pair with D = 0 contributes zero; a sample with |Xdot| >= 1 contributes nothing (both
 * counted in the device status).  The result is deterministic (fixed reduction order). */
int isw_map(isw_ctx *ctx, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list,
            const double *samples, int64_t n, int64_t ld, const double *x_obs, double GU, int prec,
            int accumulate, double *theta_out, void *stream);

/* A gnomonic patch map (Sec. IV, Fig. 3: full sky against the flat-sky / small-angle
 * approximation on the same patch).
 *   frame    : host double[9], orthonormal e1, e2, e3 (e3 = patch centre)
 *   M, width : M x M pixels of gnomonic coordinates xi, eta in [-width/2, width/2]; pixel
 *              (i, j) is centred at xi = (i + 1/2 - M/2) width/M, eta likewise, and stored at
 *              theta_out[j M + i] (device double[M*M])
 *   approx   : ISW_FULLSKY: the map of Eq. (1)-(2) at the directions (xi e1 + eta e2 + e3)/norm
 *              (the isw_map kernels, prec as there); ISW_FLATSKY: the limit X n -> X with
 *              parallel photon paths (Sec. II.A): a sample at depth Z = (X - x_obs).e3 > 0 sits
 *              at ((X - x_obs).e1, (X - x_obs).e2)/Z and contributes
 *              -4 GU eps dsigma / Z (u_perp . d)/|d|^2 with u = Xdot - (e3.X')X'/(1 + e3.Xdot),
 *              u_perp its e1, e2 components and d the coordinate separation; samples with Z <= 0
 *              contribute nothing, d = 0 gives 0.  ISW_F32C forms d from float-pair positions and
 *              sums with compensation; ISW_F64 is plain FP64.
 *   accumulate : 0 writes theta_out, 1 adds to it
 * ISW_EINVAL for a frame that is not orthonormal (to 1e-9), M outside [1, 2^20] or width <= 0. */
int isw_map_patch(isw_ctx *ctx, const double *frame, int64_t M, double width, const double *samples, int64_t n,
                  int64_t ld, const double *x_obs, double GU, int prec, int approx, int accumulate,
                  double *theta_out, void *stream);

/* Angular power spectrum of a full-sky RING map (Sec. IV, Fig. 4): spherical-harmonic analysis
 * with uniform pixel weights, a_lm = (4 pi / N_pix) sum_p Theta_p conj(Y_lm(n_p)) (Condon-Shortley
 * phase), C_l = (|a_l0|^2 + 2 sum_{m>=1} |a_lm|^2) / (2l + 1).
 *   theta : device double[12 nside^2], RING order; nside <= 1024
 *   lmax  : 0 .. 4 nside (m runs to lmax)
 *   alm   : device double[2][lmax+1][lmax+1] (real plane, then imaginary; entry [m][l], zero for
 *           l < m) or NULL (kept in the context's workspace)
 *   cl    : device double[lmax+1]
 * Per-ring Fourier sums cost N_pix (lmax + 1) complex products (no FFT); the sums over rings
 * have a fixed order (deterministic). */
int isw_map_cl(isw_ctx *ctx, int64_t nside, const double *theta, int64_t lmax, double *alm, double *cl,
               void *stream);

/* Adjoint of isw_map with respect to the samples (an extension of the method: the
 * derivative of Eq. (1)-(2)).  Given g = dL/dTheta (device double[npix], same pixel
 * selection), writes grad_out = device double[ngrad][ld_g] with rows dL/dX (3), dL/dXdot (3),
 * then dL/dX' (3) when ngrad >= 9 and dL/ddsigma when ngrad = 10 (ngrad is 6, 9 or 10), for
 * every sample.  Pair terms are recomputed, not stored; the reduction over pixels has a fixed
 * order (deterministic).  A skipped sample (|Xdot| >= 1) gets zero rows. */
int isw_map_adjoint(isw_ctx *ctx, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list,
                    const double *samples, int64_t n, int64_t ld, const double *x_obs, double GU, int prec,
                    const double *dL_dtheta, double *grad_out, int64_t ld_g, int ngrad, void *stream);

/* Adjoint of lightcone_intersect (an extension of the method: the derivative of the crossing
 * condition X cap x_gamma of Eq. (1), with X', Xdot taken at the crossing as in Sec. II.B).
 * The retarded time tau solves |X(tau) - x_obs| = t_obs - tau, so by the implicit-function
 * theorem dtau/dq = -(rhat . dX/dq) / (1 + rhat . Xdot) for every parameter q of the node.
 *   mode, nodes_in, n, ld, loop_params, nloops, ldp, t_box, x_obs : as given to
 *              lightcone_intersect (x_obs host double[3], NULL = origin)
 *   tau      : device double[n], the tau_out of that call
 *   grad_samples : device double[ngrad][ld_gs], dL/d(samples): rows X (3), Xdot (3), then
 *              X' (3) and dsigma when ngrad is 9 or 10 (the rows isw_map_adjoint writes);
 *              rows not given count as zero
 *   grad_nodes : device double[10][ld_gn].  LINEAR: dL/d(box-time X, Xdot, X', dsigma).
 *              BURDEN: row 1 = dL/dsigma, row 9 = dL/ddsigma, other rows 0.
 *   grad_loops : BURDEN only (ignored for LINEAR, may be NULL): device double[17][ld_gl],
 *              ld_gl >= nloops: dL/d(centre (3), rotation (9 entries, each taken as a free
 *              parameter), L, m, n, psi, t0) summed over the loop's nodes; the m and n rows are
 *              0 (integer harmonic numbers).  The nodes of one loop must be contiguous in
 *              nodes_in: a loop whose nodes form several runs gets NaN rows and ISW_EINVAL in
 *              the device status.  The per-loop sum has a fixed order (deterministic).
 * A node with an out-of-range loop id gets zero rows (ISW_EINVAL in the device status); one
 * where 1 + rhat . Xdot <= 0 gets zero rows (ISW_EDOMAIN).  ISW_EINVAL on the host for bad
 * sizes, modes or pointers. */
int lightcone_adjoint(isw_ctx *ctx, int mode, const double *nodes_in, int64_t n, int64_t ld,
                      const double *loop_params, int64_t nloops, int64_t ldp, double t_box,
                      const double *x_obs, const double *tau, const double *grad_samples, int64_t ld_gs,
                      int ngrad, double *grad_nodes, int64_t ld_gn, double *grad_loops, int64_t ld_gl,
                      void *stream);

/* Many shells into one full-sky map (Sec. III.A: the final map is the sum of maps sourced
 * by subsets of the simulation cones).  nodes: device double[10][ld] of all shells
 * concatenated; shell_off: host int64[nshell+1] offsets; t_box, mode: host arrays of
 * nshell; loop_params as in lightcone_intersect.  The light-cone solve of every shell and
 * one map over all samples are enqueued (flags: ISW_SKIP_LIGHTCONE when nodes are already
 * samples on the cone; ISW_GRAPH to capture the sequence in a CUDA graph that later calls
 * with the same arguments replay; ISW_AUTOTUNE to pick the FP32 kernel variant by timing).
 * theta_out: device double[12 N^2] (RING), written or accumulated as in isw_map. */
int isw_map_batched(isw_ctx *ctx, int64_t nside, const double *nodes, int64_t ld, const int64_t *shell_off,
                    int64_t nshell, const double *t_box, const int32_t *mode, const double *loop_params,
                    int64_t nloops, int64_t ldp, const double *x_obs, double t_obs, double GU, int prec,
                    int flags, int accumulate, double *theta_out, void *stream);

/* The FP32-compensated map of isw_map (full sky, or the RING range pix0 .. pix0+npix-1)
 * for callers that may not allocate device memory: code running inside a host framework
 * that owns all device memory through its own pool, or a latency-critical loop that cannot
 * take the implicit device synchronisation of cudaMalloc / cudaFree.  The paper has no
 * counterpart; this is a deployment variant of isw_map.
 *   - Needs no isw_ctx and calls no cudaMalloc, cudaFree or allocating library routine.
 *     Its scratch is a static device array of 64 MiB that every GPU loading the library
 *     holds until the process exits; a problem whose scratch does not fit (roughly
 *     32 bytes per padded pixel + 420 bytes per padded sample, plus 8 bytes per padded pixel
 *     per segment chunk: a full Nside=256 sky fits with 8 x 10^4 samples, not with 10^5) is
 *     rejected with ISW_EINVAL before anything is enqueued.
 *   - The first call on a device, with that device current, looks up the array's device
 *     address (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents; each call clears
 *     what must start at zero.  Calls that overlap on the GPU (for example on two streams
 *     without ordering) race on the array and produce wrong maps.
 *   - Arguments as in isw_map (device samples double[10][ld] and theta_out double[npix] on the
 *     current device, host x_obs or NULL); kernel variant, segment chunks, near-field and b_min
 *     settings are those of isw_map with default settings (the chunk count capped by the
 *     scratch), so the map equals isw_map's.
 *   - status_out (host, may be NULL): when given, the call waits for `stream` and stores the
 *     status the kernels recorded: ISW_OK, ISW_EDOMAIN (a sample with |Xdot| >= 1 or a
 *     non-finite weight was skipped) or ISW_ETIMEOUT (a bounded device wait ran out: the map is
 *     incomplete).  Without it the call does not synchronise and such conditions go unreported.
 *     The return value is the host-side status (argument checks and launches). */
int isw_map_f32c_noalloc(int64_t nside, int64_t pix0, int64_t npix, const double *samples, int64_t n, int64_t ld,
                         const double *x_obs, double GU, double *theta_out, int32_t *status_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ISW_H */
