// The all-pairs line-of-sight sum of Eq. (1)-(2) (Sec. III.A: every pixel sums every sample).
//
// Work items are (pixel tile, segment chunk).  A CTA holds the directions of its pixel tile
// in registers (P pixels per thread, compact tx x ty face patch for full-sky maps) and
// streams the chunk's segment records through a ring of shared-memory stages filled by 1-D
// bulk copies (TMA engine, mbarrier completion); every warp reads every record (broadcast).
// Per pixel the sum is kept in registers: FP32 partials per segment tile folded into a
// compensated (hi, lo) pair, plus an FP64 accumulator for near-field pairs.
//
// Per pair (d = n - Xhat as a float pair, see pack.cu):
//   t = c [ B (Xdot.d) - A (X'.d) ] / [ B (d.d) ],  A = n.X',  B = 1 + n.Xdot.
// A segment tile is checked pair by pair only when its bounding cap comes within the near
// radius of the pixel tile's cap, or when it holds a sample with 1 - |Xdot| < b_min; checked
// pairs with |d| < rho (rho = near_k * max(pixel size, segment angle)) or B < b_min are
// evaluated in FP64 from the FP64 records.
#include "isw_internal.cuh"
#include "kernels.cuh"
#include "pipeline.cuh"

namespace isw {

template <int NT, int P, int S>
__global__ void __launch_bounds__(NT, (P >= 8 ? 1 : (NT >= 256 ? 2 : 4))) k_map_f32c(MapArgs a)
{
    constexpr int TILE = NT * P;
    extern __shared__ __align__(128) unsigned char smem[];
    Seg32 *sbuf = reinterpret_cast<Seg32 *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * S * sizeof(Seg32));
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    unsigned nearcnt = 0, zerocnt = 0;
    uint32_t g = 0;
    const int64_t n_items = a.ntiles * a.split;
    const int64_t tot = a.ntiles * TILE;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t tile = item / a.split;
        const int kc = (int)(item - tile * a.split);
        const int64_t j0 = a.nst * kc / a.split, j1 = a.nst * (kc + 1) / a.split;
        const int nt = (int)(j1 - j0);

        float nh[P][3], nl[P][3], ahi[P], alo[P];
        double a64[P];
        unsigned valid = 0;  // padding slots are computed but neither written nor counted
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
            if (a.outidx[k] >= 0) valid |= 1u << q;
            const double v[3] = {a.nv[k], a.nv[a.ldn + k], a.nv[2 * a.ldn + k]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                nh[q][c] = __double2float_rn(v[c]);
                nl[q][c] = __double2float_rn(v[c] - (double)nh[q][c]);
            }
            ahi[q] = 0.f;
            alo[q] = 0.f;
            a64[q] = 0.0;
        }
        const float4 pc = a.pcaps[tile];

        if (tid == 0) {
            const int pro = nt < kStages ? nt : kStages;
            for (int i = 0; i < pro; ++i) issue_tile<Seg32, S>(sbuf, bars, a.s32, j0 + i, g + i);
        }
        int i = 0;
        for (; i < nt; ++i) {
            const uint32_t gi = g + i;
            const int buf = gi % kStages;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[buf], (gi / kStages) & 1))) {
                s_abort = 1;
            } else {
                const int64_t j = j0 + i;
                const SegCap sc = a.scaps[j];
                const float ex = pc.x - sc.c.x, ey = pc.y - sc.c.y, ez = pc.z - sc.c.z;
                const float gap = sqrtf(ex * ex + ey * ey + ez * ez) - pc.w - sc.c.w;  // lower bound of |d|
                // B = 1 + n.Xdot >= b_min for every pair unless the pixel cap meets the tile's beam cap
                const float bx = pc.x - sc.b.x, by = pc.y - sc.b.y, bz = pc.z - sc.b.z;
                const bool fast_b = sc.b.w < 0.f || sqrtf(bx * bx + by * by + bz * bz) > pc.w + sc.b.w;
                const bool near = (gap < sc.r.x) || !fast_b;
                const bool far = fast_b && (gap >= a.d_far);
                const Seg32 *sb = sbuf + buf * S;
                float part[P];
#pragma unroll
                for (int q = 0; q < P; ++q) part[q] = 0.f;
                if (far) {
                    // |d| >= d_far for every pair: d.d/2 = 1 - n.Xhat, Xdot.d = B - e, X'.d = A - f
#pragma unroll 2
                    for (int s = 0; s < S; ++s) {
                        const float4 ra = sb[s].a, rd = sb[s].d, re = sb[s].e;
                        const float ch = 0.5f * ra.w;
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const float h = fmaf(-nh[q][2], ra.z, fmaf(-nh[q][1], ra.y, fmaf(-nh[q][0], ra.x, 1.f)));
                            const float A = fmaf(nh[q][2], re.z, fmaf(nh[q][1], re.y, nh[q][0] * re.x));
                            const float B = fmaf(nh[q][2], rd.z, fmaf(nh[q][1], rd.y, fmaf(nh[q][0], rd.x, 1.f)));
                            const float Pd = B - rd.w;
                            const float Qd = A - re.w;
                            const float num = fmaf(B, Pd, -A * Qd);
                            const float r = rcp_approx(B * h);
                            part[q] = fmaf(ch * num, r, part[q]);
                        }
                    }
                } else if (!near) {
#pragma unroll 2
                    for (int s = 0; s < S; ++s) {
                        const float4 ra = sb[s].a, rb = sb[s].b, rd = sb[s].d, re = sb[s].e;
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const float dx = (nh[q][0] - ra.x) + (nl[q][0] - rb.x);
                            const float dy = (nh[q][1] - ra.y) + (nl[q][1] - rb.y);
                            const float dz = (nh[q][2] - ra.z) + (nl[q][2] - rb.z);
                            const float Q = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            const float Pd = fmaf(rd.z, dz, fmaf(rd.y, dy, rd.x * dx));
                            const float Qd = fmaf(re.z, dz, fmaf(re.y, dy, re.x * dx));
                            const float A = fmaf(nh[q][2], re.z, fmaf(nh[q][1], re.y, nh[q][0] * re.x));
                            const float B = fmaf(nh[q][2], rd.z, fmaf(nh[q][1], rd.y, fmaf(nh[q][0], rd.x, 1.f)));
                            const float num = fmaf(B, Pd, -A * Qd);
                            const float r = rcp_approx(B * Q);
                            part[q] = fmaf(ra.w * num, r, part[q]);
                        }
                    }
                } else {
                    // checked loop: two-float d, B formed without cancellation near -Xdot/|Xdot|;
                    // pairs with |d| < rho or B < b_min/1000 go to FP64
                    const float b_tiny = a.b_min * 1e-3f;
                    for (int s = 0; s < S; ++s) {
                        const float4 ra = sb[s].a, rb = sb[s].b, rd = sb[s].d, re = sb[s].e, rk = sb[s].k;
                        const float hv = fmaf(-0.5f, rk.w, 0.5f);   // |Xdot| / 2
                        unsigned mask = 0;
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const float dx = (nh[q][0] - ra.x) + (nl[q][0] - rb.x);
                            const float dy = (nh[q][1] - ra.y) + (nl[q][1] - rb.y);
                            const float dz = (nh[q][2] - ra.z) + (nl[q][2] - rb.z);
                            const float Q = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            const float Pd = fmaf(rd.z, dz, fmaf(rd.y, dy, rd.x * dx));
                            const float Qd = fmaf(re.z, dz, fmaf(re.y, dy, re.x * dx));
                            const float A = fmaf(nh[q][2], re.z, fmaf(nh[q][1], re.y, nh[q][0] * re.x));
                            const float wx = nh[q][0] + rk.x, wy = nh[q][1] + rk.y, wz = nh[q][2] + rk.z;
                            const float B = fmaf(hv, fmaf(wz, wz, fmaf(wy, wy, wx * wx)), rk.w);
                            if (Q < rb.w || B < b_tiny) {
                                mask |= 1u << q;
                            } else {
                                const float num = fmaf(B, Pd, -A * Qd);
                                const float r = rcp_approx(B * Q);
                                part[q] = fmaf(ra.w * num, r, part[q]);
                            }
                        }
                        if (__any_sync(0xffffffffu, mask != 0)) {
                            const Seg64 g64 = a.s64[j * S + s];
#pragma unroll
                            for (int q = 0; q < P; ++q) {
                                if (mask & (1u << q)) {
                                    const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
                                    unsigned z = 0;
                                    a64[q] += pair64(a.nv[k], a.nv[a.ldn + k], a.nv[2 * a.ldn + k], g64, z);
                                    if (valid & (1u << q)) {
                                        zerocnt += z;
                                        ++nearcnt;
                                    }
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < P; ++q) fold(ahi[q], alo[q], part[q]);
            }
            __syncthreads();
            if (s_abort) break;
            if (tid == 0 && i + kStages < nt) issue_tile<Seg32, S>(sbuf, bars, a.s32, j0 + i + kStages, gi + kStages);
        }
        if (s_abort) {
            if (tid == 0) {
                atomicOr(&a.st->bits, kStatTimeout);
                drain<S>(bars, g, i, nt);
            }
            return;
        }
        g += nt;

#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
            const double v = ((double)ahi[q] + (double)alo[q]) + a64[q];
            if (a.split == 1) {
                const int64_t oi = a.outidx[k];
                if (oi >= 0) a.theta[oi] = a.accumulate ? a.theta[oi] + v : v;
            } else {
                a.partial[(int64_t)kc * tot + k] = v;
            }
        }
    }
    // per-warp counters
    for (int o = 16; o > 0; o >>= 1) {
        nearcnt += __shfl_xor_sync(0xffffffffu, nearcnt, o);
        zerocnt += __shfl_xor_sync(0xffffffffu, zerocnt, o);
    }
    if (lane == 0 && (nearcnt | zerocnt)) {
        atomicAdd(&a.st->near_pairs, (unsigned long long)nearcnt);
        atomicAdd(&a.st->zero_pairs, (unsigned long long)zerocnt);
    }
}

// Plain FP64 path: every pair in FP64, same tiling.
template <int NT, int P, int S>
__global__ void __launch_bounds__(NT) k_map_f64(MapArgs a)
{
    constexpr int TILE = NT * P;
    extern __shared__ __align__(128) unsigned char smem[];
    Seg64 *sbuf = reinterpret_cast<Seg64 *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * S * sizeof(Seg64));
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    unsigned zerocnt = 0;
    uint32_t g = 0;
    const int64_t n_items = a.ntiles * a.split;
    const int64_t tot = a.ntiles * TILE;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int64_t tile = item / a.split;
        const int kc = (int)(item - tile * a.split);
        const int64_t j0 = a.nst * kc / a.split, j1 = a.nst * (kc + 1) / a.split;
        const int nt = (int)(j1 - j0);
        double nv[P][3], hi[P], lo[P];
        unsigned valid = 0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
            if (a.outidx[k] >= 0) valid |= 1u << q;
            nv[q][0] = a.nv[k];
            nv[q][1] = a.nv[a.ldn + k];
            nv[q][2] = a.nv[2 * a.ldn + k];
            hi[q] = 0.0;
            lo[q] = 0.0;
        }
        if (tid == 0) {
            const int pro = nt < kStages ? nt : kStages;
            for (int i = 0; i < pro; ++i) issue_tile<Seg64, S>(sbuf, bars, a.s64, j0 + i, g + i);
        }
        int i = 0;
        for (; i < nt; ++i) {
            const uint32_t gi = g + i;
            const int buf = gi % kStages;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[buf], (gi / kStages) & 1))) {
                s_abort = 1;
            } else {
                const Seg64 *sb = sbuf + buf * S;
                double part[P];
#pragma unroll
                for (int q = 0; q < P; ++q) part[q] = 0.0;
                unsigned z[P];
#pragma unroll
                for (int q = 0; q < P; ++q) z[q] = 0;
                for (int s = 0; s < S; ++s) {
                    const Seg64 g64 = sb[s];
#pragma unroll
                    for (int q = 0; q < P; ++q) part[q] += pair64(nv[q][0], nv[q][1], nv[q][2], g64, z[q]);
                }
#pragma unroll
                for (int q = 0; q < P; ++q)
                    if (valid & (1u << q)) zerocnt += z[q];
#pragma unroll
                for (int q = 0; q < P; ++q) fold64(hi[q], lo[q], part[q]);
            }
            __syncthreads();
            if (s_abort) break;
            if (tid == 0 && i + kStages < nt) issue_tile<Seg64, S>(sbuf, bars, a.s64, j0 + i + kStages, gi + kStages);
        }
        if (s_abort) {
            if (tid == 0) {
                atomicOr(&a.st->bits, kStatTimeout);
                drain<S>(bars, g, i, nt);
            }
            return;
        }
        g += nt;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
            const double v = hi[q] + lo[q];
            if (a.split == 1) {
                const int64_t oi = a.outidx[k];
                if (oi >= 0) a.theta[oi] = a.accumulate ? a.theta[oi] + v : v;
            } else {
                a.partial[(int64_t)kc * tot + k] = v;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) zerocnt += __shfl_xor_sync(0xffffffffu, zerocnt, o);
    if (lane == 0 && zerocnt) atomicAdd(&a.st->zero_pairs, (unsigned long long)zerocnt);
}

// theta[out(k)] (=|+=) sum over chunks c = 0..split-1 of partial[c][k], fixed order, compensated.
__global__ void k_reduce_partials(const double *__restrict__ partial, int64_t tot, int split,
                                  const int64_t *__restrict__ outidx, double *__restrict__ theta, int accumulate)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t oi = outidx[k];
        if (oi < 0) continue;
        double hi = 0.0, lo = 0.0;
        for (int c = 0; c < split; ++c) fold64(hi, lo, partial[(int64_t)c * tot + k]);
        const double v = hi + lo;
        theta[oi] = accumulate ? theta[oi] + v : v;
    }
}

// ------------------------------------------------------------------------------------
// Variant table and launchers
// ------------------------------------------------------------------------------------
#define ISW_F32_VARIANTS(X) \
    X(256, 4, 64)           \
    X(256, 2, 64)           \
    X(128, 4, 64)           \
    X(256, 8, 32)           \
    X(128, 8, 32)

namespace {
struct VEntry {
    Variant v;
    const void *fn;
};
#define ISW_ENTRY(NT, P, S) {{NT, P, S, 32, (NT / 32) * P}, (const void *)&k_map_f32c<NT, P, S>},
const VEntry kF32[] = {ISW_F32_VARIANTS(ISW_ENTRY)};
#undef ISW_ENTRY
constexpr int kF64NT = 128, kF64P = 2, kF64S = 32;

size_t smem_f32(int S) { return kStages * S * sizeof(Seg32) + kStages * sizeof(uint64_t); }
size_t smem_f64(int S) { return kStages * S * sizeof(Seg64) + kStages * sizeof(uint64_t); }
}  // namespace

int num_f32_variants() { return (int)(sizeof(kF32) / sizeof(kF32[0])); }
Variant f32_variant(int idx) { return kF32[idx].v; }
int f64_seg_tile() { return kF64S; }
Variant f64_variant() { return Variant{kF64NT, kF64P, kF64S, 32, (kF64NT / 32) * kF64P}; }

int map_f32c_slots(int idx, int num_sms)
{
    int nb = 0;
    const Variant v = kF32[idx].v;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kF32[idx].fn, v.threads, smem_f32(v.seg_tile));
    return (nb > 0 ? nb : 1) * num_sms;
}

int map_f64_slots(int num_sms)
{
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)&k_map_f64<kF64NT, kF64P, kF64S>, kF64NT,
                                                  smem_f64(kF64S));
    return (nb > 0 ? nb : 1) * num_sms;
}

void launch_map_f32c(int idx, const MapArgs &a, int grid, cudaStream_t s)
{
    const Variant v = kF32[idx].v;
    void *args[] = {(void *)&a};
    cudaLaunchKernel(kF32[idx].fn, dim3(grid), dim3(v.threads), args, smem_f32(v.seg_tile), s);
}

void launch_map_f64(const MapArgs &a, int grid, cudaStream_t s)
{
    k_map_f64<kF64NT, kF64P, kF64S><<<grid, kF64NT, smem_f64(kF64S), s>>>(a);
}

void launch_reduce_partials(const MapArgs &a, int tile_sz, cudaStream_t s)
{
    const int64_t tot = a.ntiles * tile_sz;
    int64_t blocks = (tot + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_reduce_partials<<<(unsigned)blocks, 256, 0, s>>>(a.partial, tot, a.split, a.outidx, a.theta, a.accumulate);
}

}  // namespace isw
