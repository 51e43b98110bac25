// Spatial order of the samples for the FP32 map.  The sum of Eq. (1)-(2) does not depend on the
// order of the samples, but the tiling does: a segment tile of consecutive samples gets a
// bounding cap, and only tile pairs whose caps are far apart take the far-field form.  Samples
// that are adjacent in the input need not be adjacent on the sky (a string whose nodes are moved
// to the light cone with velocities of random direction scatters), so the records are written in
// the order of a 3-D Morton code of the unit vector Xhat quantised to 8 bits per axis.  The sort
// is a stable least-significant-digit radix sort of (key, index) in three passes of 8 bits, so
// the order, and with it the rounding of the map's sums, is reproducible.
//   k_sort_keys     key = Morton code of Xhat (invalid samples last), index = input position
//   k_sort_hist     per block of 1024 elements, the 256-bin histogram of the pass's digit
//   k_sort_scan     exclusive scan of the histograms in (digit, block) order: each block's first
//                   output position for each digit
//   k_sort_scatter  the block's elements in input order, ranked within their digit by a warp
//                   match and per-warp counts, written to their positions (stable)
#include "isw_internal.cuh"
#include "kernels.cuh"

namespace isw {

namespace {
constexpr int kSortThreads = 256, kSortBlock = 1024, kRadix = 256, kSortWarps = kSortThreads / 32;
constexpr uint32_t kInvalidKey = 0xffffffu;

__device__ __forceinline__ uint32_t spread3(uint32_t x)   // bits b0..b7 -> positions 0, 3, 6, ...
{
    x &= 0xffu;
    x = (x | (x << 8)) & 0x00f00fu;
    x = (x | (x << 4)) & 0x0c30c3u;
    x = (x | (x << 2)) & 0x249249u;
    return x;
}

__global__ void k_sort_keys(const double *__restrict__ S, int64_t n, int64_t ld, double xo0, double xo1, double xo2,
                            uint32_t *__restrict__ key, uint32_t *__restrict__ idx)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const double r[3] = {S[s] - xo0, S[ld + s] - xo1, S[2 * ld + s] - xo2};
        const double nrm = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        uint32_t k = kInvalidKey;
        if (nrm > 0.0 && isfinite(nrm)) {
            uint32_t q[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double u = floor((r[c] / nrm + 1.0) * 128.0);
                q[c] = (uint32_t)(u < 0.0 ? 0.0 : (u > 255.0 ? 255.0 : u));
            }
            k = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
        }
        key[s] = k;
        idx[s] = (uint32_t)s;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t *__restrict__ key, int64_t n, int shift,
                                                            uint32_t *__restrict__ hist, int nblocks)
{
    __shared__ uint32_t h[kRadix];
    const int tid = threadIdx.x;
    const int64_t b = blockIdx.x;
    h[tid] = 0;
    __syncthreads();
    for (int i = tid; i < kSortBlock; i += kSortThreads) {
        const int64_t e = b * kSortBlock + i;
        if (e < n) atomicAdd(&h[(key[e] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)tid * nblocks + b] = h[tid];
}

// One block of 1024 threads: each thread scans a contiguous run serially, then the run totals
// are scanned across the block.
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t *__restrict__ hist, int64_t total)
{
    __shared__ uint32_t part[1024];
    const int tid = threadIdx.x;
    const int64_t per = (total + 1023) / 1024;
    const int64_t a = tid * per, e = a + per < total ? a + per : total;
    uint32_t s = 0;
    for (int64_t i = a; i < e; ++i) s += hist[i];
    part[tid] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan of the run totals
        const uint32_t v = tid >= o ? part[tid - o] : 0u;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    uint32_t run = tid > 0 ? part[tid - 1] : 0u;
    for (int64_t i = a; i < e; ++i) {
        const uint32_t h = hist[i];
        hist[i] = run;
        run += h;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t *__restrict__ key_in,
                                                               const uint32_t *__restrict__ idx_in, int64_t n,
                                                               int shift, const uint32_t *__restrict__ offs,
                                                               int nblocks, uint32_t *__restrict__ key_out,
                                                               uint32_t *__restrict__ idx_out)
{
    __shared__ uint32_t base[kRadix];                // next output position of each digit
    __shared__ uint32_t wcnt[kSortWarps][kRadix];    // elements of each digit per warp, this round
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t b = blockIdx.x;
    base[tid] = offs[(int64_t)tid * nblocks + b];
    for (int r = 0; r < kSortBlock / kSortThreads; ++r) {
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wcnt[w][tid] = 0u;
        __syncthreads();
        const int64_t e = b * kSortBlock + (int64_t)r * kSortThreads + tid;
        const bool valid = e < n;
        const uint32_t k = valid ? key_in[e] : 0u;
        const uint32_t d = valid ? (k >> shift) & (kRadix - 1) : (uint32_t)kRadix;   // sentinel never written
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned below = peers & ((1u << lane) - 1u);
        if (valid && below == 0u) wcnt[wid][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = base[d] + (uint32_t)__popc(below);
            for (int w = 0; w < wid; ++w) pos += wcnt[w][d];
            key_out[pos] = k;
            idx_out[pos] = idx_in[e];
        }
        __syncthreads();
        uint32_t add = 0u;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) add += wcnt[w][tid];
        base[tid] += add;
        __syncthreads();
    }
}
}  // namespace

size_t sort_scratch_bytes(int64_t n)
{
    const int64_t nblocks = (n + kSortBlock - 1) / kSortBlock;
    return (size_t)4 * n * sizeof(uint32_t) + (size_t)kRadix * nblocks * sizeof(uint32_t) + 4 * 256;
}

const uint32_t *launch_spatial_order(const double *S, int64_t n, int64_t ld, double xo0, double xo1, double xo2,
                                     void *scratch, cudaStream_t s)
{
    if (n <= 0) return nullptr;
    const int64_t nblocks = (n + kSortBlock - 1) / kSortBlock;
    uint32_t *p = reinterpret_cast<uint32_t *>(scratch);
    uint32_t *key[2] = {p, p + n}, *idx[2] = {p + 2 * n, p + 3 * n};
    uint32_t *hist = p + 4 * n;
    int64_t kb = (n + 255) / 256;
    if (kb > 152 * 32) kb = 152 * 32;
    k_sort_keys<<<(unsigned)kb, 256, 0, s>>>(S, n, ld, xo0, xo1, xo2, key[0], idx[0]);
    int cur = 0;
    for (int shift = 0; shift < 24; shift += 8) {
        k_sort_hist<<<(unsigned)nblocks, kSortThreads, 0, s>>>(key[cur], n, shift, hist, (int)nblocks);
        k_sort_scan<<<1, 1024, 0, s>>>(hist, (int64_t)kRadix * nblocks);
        k_sort_scatter<<<(unsigned)nblocks, kSortThreads, 0, s>>>(key[cur], idx[cur], n, shift, hist, (int)nblocks,
                                                                    key[cur ^ 1], idx[cur ^ 1]);
        cur ^= 1;
    }
    return idx[cur];
}

int spatial_order_launches() { return 1 + 3 * 3; }

}  // namespace isw
