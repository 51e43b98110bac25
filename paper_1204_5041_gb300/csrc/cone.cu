// Stacking with HEALPix cones (Sec. III.B, Fig. 1 of the paper): the comoving volume between
// two radii is voxelised by the cones that subtend the pixels of a coarse HEALPix grid
// (N_side^hz); each cone is filled from a simulation box rotated to face the observer (one box
// serves several cones), and only the strings inside the cone are kept.  Kernels here:
//   k_vec2pix      RING pixel of arbitrary directions (reproducible operation by operation)
//   k_box_place    shell k takes the nodes of box b_k and maps X -> R X + T, Xdot -> R Xdot,
//                  X' -> R X' (a gather: one box read by many shells)
//   cone cut       per-sample keep flag (direction in pixel cone_pix[k] of N_side^hz and
//                  r_lo[k] <= |X - x_obs| < r_hi[k]), block scan, carry scan, scatter: a
//                  stable stream compaction (kept samples in input order, deterministic)
#include "isw_internal.cuh"
#include "kernels.cuh"

namespace isw {

constexpr int kScanBlock = 1024;

__global__ void k_vec2pix(int64_t N, const double *__restrict__ v, int64_t n, int64_t ld, int64_t *__restrict__ pix,
                          DevStatus *st)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double x = v[k], y = v[ld + k], z = v[2 * ld + k];
        if (!(x * x + y * y + z * z > 0.0) || !isfinite(x + y + z)) {
            pix[k] = -1;
            atomicOr(&st->bits, kStatBadIndex);
        } else {
            pix[k] = vec2pix_ring(N, x, y, z);
        }
    }
}

// shell of output index o: off[k] <= o < off[k+1] (binary search over nshell + 1 offsets)
__device__ __forceinline__ int64_t find_shell(const int64_t *__restrict__ off, int64_t nshell, int64_t o)
{
    int64_t lo = 0, hi = nshell;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= o) lo = mid; else hi = mid;
    }
    return lo;
}

// place: [nshell][12] (R row-major, then T); src_start[k] = first node of shell k's box;
// (R x)_i = (R_i0 x_0 + R_i1 x_1) + R_i2 x_2 in IEEE double without contraction
__global__ void k_box_place(const double *__restrict__ nodes, int64_t ld, const int64_t *__restrict__ off_out,
                            const int64_t *__restrict__ src_start, int64_t nshell, const double *__restrict__ place,
                            double *__restrict__ out, int64_t ld_out, int64_t n_out)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_out; o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = find_shell(off_out, nshell, o);
        const int64_t s = src_start[k] + (o - off_out[k]);
        const double *R = place + 12 * k;
#pragma unroll
        for (int blk = 0; blk < 3; ++blk) {
            const double x0 = nodes[(3 * blk) * ld + s], x1 = nodes[(3 * blk + 1) * ld + s],
                         x2 = nodes[(3 * blk + 2) * ld + s];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double y = dadd(dadd(dmul(R[3 * i], x0), dmul(R[3 * i + 1], x1)), dmul(R[3 * i + 2], x2));
                out[(3 * blk + i) * ld_out + o] = blk == 0 ? dadd(y, R[9 + i]) : y;
            }
        }
        out[9 * ld_out + o] = nodes[9 * ld + s];
    }
}

// Keep flag of every sample and a per-block inclusive scan of the flags (block totals out).
__global__ void __launch_bounds__(kScanBlock) k_cut_flags(const double *__restrict__ S, int64_t ld, int64_t n,
                                                          const int64_t *__restrict__ off, int64_t nshell,
                                                          int64_t nside_hz, const int64_t *__restrict__ cone_pix,
                                                          const double *__restrict__ r_lo,
                                                          const double *__restrict__ r_hi, double xo0, double xo1,
                                                          double xo2, int32_t *__restrict__ incl,
                                                          int64_t *__restrict__ block_tot)
{
    __shared__ int32_t warp_tot[kScanBlock / 32];
    const int64_t s = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    int32_t f = 0;
    if (s < n) {
        const int64_t k = find_shell(off, nshell, s);
        const double dx = dsub(S[s], xo0), dy = dsub(S[ld + s], xo1), dz = dsub(S[2 * ld + s], xo2);
        const double r = dsqrt(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
        if (r >= r_lo[k] && r < r_hi[k] && r > 0.0) f = vec2pix_ring(nside_hz, dx, dy, dz) == cone_pix[k] ? 1 : 0;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    const int32_t before = w > 0 ? warp_tot[w - 1] : 0;
    if (s < n) incl[s] = before + x;
    if (threadIdx.x == 0) block_tot[blockIdx.x] = warp_tot[kScanBlock / 32 - 1];
}

// Exclusive scan of the block totals in place (one block, chunks of kScanBlock with a carry);
// block_tot[nb] receives the grand total.
__global__ void __launch_bounds__(kScanBlock) k_scan_totals(int64_t *__restrict__ block_tot, int64_t nb)
{
    __shared__ int64_t warp_tot[kScanBlock / 32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nb ? block_tot[i] : 0;
        int64_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const int64_t incl = (w > 0 ? warp_tot[w - 1] : 0) + x;
        if (i < nb) block_tot[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[kScanBlock / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_tot[nb] = carry;
}

// Scatter kept samples to their compacted position; per-shell output offsets.
__global__ void __launch_bounds__(kScanBlock) k_cut_scatter(const double *__restrict__ S, int64_t ld, int64_t n,
                                                            const int32_t *__restrict__ incl,
                                                            const int64_t *__restrict__ block_pre,
                                                            double *__restrict__ out, int64_t ld_out)
{
    const int64_t s = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (s >= n) return;
    const int32_t prev = threadIdx.x > 0 ? incl[s - 1] : 0;
    if (incl[s] == prev) return;                      // not kept
    const int64_t pos = block_pre[blockIdx.x] + prev;
#pragma unroll
    for (int q = 0; q < 10; ++q) out[q * ld_out + pos] = S[q * ld + s];
}

// off_out[k] = number of kept samples before shell k's first sample (exclusive prefix)
__global__ void k_cut_offsets(const int64_t *__restrict__ off, int64_t nshell, int64_t n,
                              const int32_t *__restrict__ incl, const int64_t *__restrict__ block_pre,
                              int64_t *__restrict__ off_out, int64_t *__restrict__ count)
{
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= nshell; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = off[k];
        int64_t v;
        if (s >= n) {
            v = block_pre[nb];
        } else {
            const int64_t b = s / kScanBlock;
            v = block_pre[b] + ((s % kScanBlock) > 0 ? incl[s - 1] : 0);
        }
        off_out[k] = v;
        if (k == nshell && count) *count = v;
    }
}

static unsigned grid1(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

void launch_vec2pix(int64_t N, const double *v, int64_t n, int64_t ld, int64_t *pix, DevStatus *st, cudaStream_t s)
{
    if (n > 0) k_vec2pix<<<grid1(n, 256), 256, 0, s>>>(N, v, n, ld, pix, st);
}

void launch_box_place(const double *nodes, int64_t ld, const int64_t *off_out, const int64_t *src_start,
                      int64_t nshell, const double *place, double *out, int64_t ld_out, int64_t n_out,
                      cudaStream_t s)
{
    if (n_out > 0)
        k_box_place<<<grid1(n_out, 256), 256, 0, s>>>(nodes, ld, off_out, src_start, nshell, place, out, ld_out,
                                                       n_out);
}

int64_t cone_cut_scratch_blocks(int64_t n) { return (n + kScanBlock - 1) / kScanBlock; }

void launch_cone_cut(const double *S, int64_t ld, int64_t n, const int64_t *off, int64_t nshell, int64_t nside_hz,
                     const int64_t *cone_pix, const double *r_lo, const double *r_hi, double xo0, double xo1,
                     double xo2, int32_t *incl, int64_t *block_tot, double *out, int64_t ld_out, int64_t *off_out,
                     int64_t *count, cudaStream_t s)
{
    const int64_t nb = cone_cut_scratch_blocks(n);
    if (n > 0) {
        k_cut_flags<<<(unsigned)nb, kScanBlock, 0, s>>>(S, ld, n, off, nshell, nside_hz, cone_pix, r_lo, r_hi, xo0,
                                                         xo1, xo2, incl, block_tot);
    }
    k_scan_totals<<<1, kScanBlock, 0, s>>>(block_tot, nb);
    if (n > 0) k_cut_scatter<<<(unsigned)nb, kScanBlock, 0, s>>>(S, ld, n, incl, block_tot, out, ld_out);
    k_cut_offsets<<<grid1(nshell + 1, 256), 256, 0, s>>>(off, nshell, n, incl, block_tot, off_out, count);
}

}  // namespace isw
