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

// Segment tiles per far-pass stage (each classified and copied on its own).
constexpr int kFarGroup = 2;

// Tile classes of the FP32 kernel: far-field form, mid-range float-pair form, checked loop.
enum : int { kFar = 0, kMid = 1, kChecked = 2 };

__device__ __forceinline__ int classify(const float4 &pc, const SegCap &sc, float d_far)
{
    const float ex = pc.x - sc.c.x, ey = pc.y - sc.c.y, ez = pc.z - sc.c.z;
    const float gap = sqrtf(ex * ex + ey * ey + ez * ez) - pc.w - sc.c.w;  // lower bound of |d| over the tile pair
    // B = 1 + n.Xdot >= b_min for every pair unless the pixel cap meets the tile's beam cap
    const float bx = pc.x - sc.b.x, by = pc.y - sc.b.y, bz = pc.z - sc.b.z;
    const bool fast_b = sc.b.w < 0.f || sqrtf(bx * bx + by * by + bz * bz) > pc.w + sc.b.w;
    if (!fast_b || gap < sc.r.x) return kChecked;
    return gap >= d_far ? kFar : kMid;
}

// Far-field pass: every segment tile whose class is kFar, in the completed-square form with
// the numerator factored, t = [(B2 - A2)(B2 + A2) + K] / (B hs), two samples at a time in packed
// f32x2 arithmetic (Far2 records: 7 f32x2 instructions + 1 rcp per pair); other tiles are
// skipped here and summed by the near-field pass.  A stage holds kFarGroup segment tiles, each
// classified and copied on its own (one block barrier per group: 320 vs 325 ms per bench step
// with 2, 332 with 4); a stage with no far tile completes its mbarrier phase with a zero-byte
// arrive.
template <int NT, int P, int S, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_map_f32c(MapArgs a)
{
    constexpr int TILE = NT * P;
    extern __shared__ __align__(128) unsigned char smem[];
    static_assert(S % 2 == 0, "segment tiles hold whole sample pairs");
    constexpr int S2 = S / 2, G = kFarGroup;
    Far2 *sbuf = reinterpret_cast<Far2 *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * G * S2 * sizeof(Far2));
    __shared__ int s_abort;
    __shared__ int s_cls[kStages];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint64_t one2 = f2_pack(1.f, 1.f);
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    uint32_t g = 0;
    __shared__ int64_t s_item;
    const int64_t n_items = (a.ntiles + a.tile_stride - 1) / a.tile_stride * a.split;
    const int64_t tot = a.ntiles * TILE;
    for (int64_t item = next_item(&a.queue[0], &s_item); item < n_items; item = next_item(&a.queue[0], &s_item)) {
        const int64_t tile = item / a.split * a.tile_stride;
        const int kc = (int)(item % a.split);
        const int64_t j0 = a.nst * kc / a.split, j1 = a.nst * (kc + 1) / a.split;
        const int nt = (int)(j1 - j0), ns = (nt + G - 1) / G;

        uint64_t n2[P][3];   // pixel direction, each component duplicated into both halves
        float ahi[P], alo[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = __double2float_rn(a.nv[c * a.ldn + k]);
                n2[q][c] = f2_pack(v, v);
            }
            ahi[q] = 0.f;
            alo[q] = 0.f;
        }
        const float4 pc = a.pcaps[tile];
        auto issue = [&](int ig, uint32_t gi) {
            const int b = gi % kStages;
            int mask = 0;
            uint32_t bytes = 0;
#pragma unroll
            for (int t = 0; t < G; ++t) {
                const int64_t j = j0 + (int64_t)ig * G + t;
                if (j < j1 && classify(pc, a.scaps[j], a.d_far) == kFar) {
                    mask |= 1 << t;
                    bytes += (uint32_t)(S2 * sizeof(Far2));
                }
            }
            s_cls[b] = mask;
            mbar_arrive_expect_tx(&bars[b], bytes);
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (mask & (1 << t))
                    bulk_g2s(sbuf + ((size_t)b * G + t) * S2, a.far + (j0 + (int64_t)ig * G + t) * S2,
                             (uint32_t)(S2 * sizeof(Far2)), &bars[b]);
        };
        if (tid == 0) {
            const int pro = ns < kStages ? ns : kStages;
            for (int i = 0; i < pro; ++i) issue(i, g + i);
        }
        int i = 0;
        for (; i < ns; ++i) {
            const uint32_t gi = g + i;
            const int buf = gi % kStages;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[buf], (gi / kStages) & 1, a.wait_polls))) {
                s_abort = 1;
            } else {
                const int mask = s_cls[buf];
                for (int t = 0; t < G; ++t) {
                    if (!(mask & (1 << t))) continue;
                    const ulonglong2 *fr = reinterpret_cast<const ulonglong2 *>(sbuf + ((size_t)buf * G + t) * S2);
                    uint64_t part[P];
#pragma unroll
                    for (int q = 0; q < P; ++q) part[q] = 0ull;   // (+0, +0)
#pragma unroll 1
                    for (int s = 0; s < S2; ++s) {
                        // (a.x, a.y) (a.z, a.w) (b.x, b.y) (b.z, b.w) (c.x, c.y) (c.z, c.w) (d.x, d.y),
                        // every entry a pair over the two samples
                        const ulonglong2 r0 = fr[7 * s], r1 = fr[7 * s + 1], r2 = fr[7 * s + 2], r3 = fr[7 * s + 3];
                        const ulonglong2 r4 = fr[7 * s + 4], r5 = fr[7 * s + 5], r6 = fr[7 * s + 6];
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const uint64_t hs = f2_fma(n2[q][2], r1.x, f2_fma(n2[q][1], r0.y, f2_fma(n2[q][0], r0.x, r1.y)));
                            const uint64_t B = f2_fma(n2[q][2], r3.x, f2_fma(n2[q][1], r2.y, f2_fma(n2[q][0], r2.x, one2)));
                            const uint64_t A2 = f2_fma(n2[q][2], r5.x, f2_fma(n2[q][1], r4.y, f2_fma(n2[q][0], r4.x, r5.y)));
                            const uint64_t B2 = f2_fma(r6.x, B, r3.y);
                            const uint64_t num = f2_fma(f2_sub(B2, A2), f2_add(B2, A2), r6.y);
                            float d0, d1;
                            f2_unpack(f2_mul(B, hs), d0, d1);
                            part[q] = f2_fma(num, f2_pack(rcp_approx(d0), rcp_approx(d1)), part[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < P; ++q) {
                        float lo, hi;
                        f2_unpack(part[q], lo, hi);
                        fold(ahi[q], alo[q], lo + hi);
                    }
                }
            }
            __syncthreads();
            if (s_abort) break;
            if (tid == 0 && i + kStages < ns) issue(i + kStages, gi + kStages);
        }
        if (s_abort) {
            if (tid == 0) drain(bars, g, i, i + kStages < ns ? i + kStages : ns, a.st);
            return;
        }
        g += ns;

#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
            const double v = (double)ahi[q] + (double)alo[q];
            if (a.split == 1) {
                const int64_t oi = a.outidx[k];
                if (oi >= 0) a.theta[oi] = a.accumulate ? a.theta[oi] + v : v;
            } else {
                a.partial[(int64_t)kc * tot + k] = v;
            }
        }
    }
}

// Near-field pass: per (pixel tile, segment chunk) item, the segment tiles that the far pass
// skipped (class kMid or kChecked), found by a warp-wide scan of the tile classes; the result
// is added to the chunk's partial (or to theta when there is one chunk) after the far pass.
// Pixels are held as pairs (pixels q and q + 1 of the thread) so that the loops run in packed
// f32x2 arithmetic over two pixels, reading each sample's constants from duplicated (Mid2)
// records.  In checked tiles a sample whose warp has a pair within the near radius or with
// B < b_min is redone one pixel at a time: B without cancellation, FP64 for pairs with
// |d| < rho or B < b_min/1000.
template <int NT, int P, int S>
__global__ void __launch_bounds__(NT, (P <= 4 ? 512 : 256) / NT) k_map_f32c_near(MapArgs a)
{
    constexpr int TILE = NT * P, P2 = P / 2;
    static_assert(P % 2 == 0, "pixels are held in pairs");
    constexpr size_t kStageBytes = S * sizeof(Mid2);
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sbuf = smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    __shared__ int s_abort;
    __shared__ int s_cls[kStages];
    __shared__ int64_t s_j[kStages];
    __shared__ int64_t s_first;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint64_t one2 = f2_pack(1.f, 1.f), half2 = f2_pack(0.5f, 0.5f);
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    unsigned nearcnt = 0, zerocnt = 0;
    uint32_t g = 0;
    __shared__ int64_t s_item;
    const int64_t n_items = (a.ntiles + a.tile_stride - 1) / a.tile_stride * a.split;
    const int64_t tot = a.ntiles * TILE;
    for (int64_t item = next_item(&a.queue[1], &s_item); item < n_items; item = next_item(&a.queue[1], &s_item)) {
        const int64_t tile = item / a.split * a.tile_stride;
        const int kc = (int)(item % a.split);
        const int64_t j0 = a.nst * kc / a.split, j1 = a.nst * (kc + 1) / a.split;
        const float4 pc = a.pcaps[tile];
        // warp 0 finds the chunk's first segment tile that is not far; an item without one is
        // skipped before its pixels are loaded (most items: strings cover little of the sky)
        if (w == 0) {
            int64_t first = -1;
            for (int64_t p0 = j0; p0 < j1 && first < 0; p0 += 32) {
                const int64_t jj = p0 + lane;
                const int c = jj < j1 ? classify(pc, a.scaps[jj], a.d_far) : kFar;
                const unsigned m = __ballot_sync(0xffffffffu, c != kFar);
                if (m) first = p0 + __ffs(m) - 1;
            }
            if (lane == 0) s_first = first;
        }
        __syncthreads();
        const int64_t first = s_first;
        if (first < 0) continue;   // next_item's barriers order the next write of s_first
        // pixel direction as a float pair (hi, lo), pixels 2pp and 2pp + 1 in the two halves
        uint64_t nh2[P2][3], nl2[P2][3];
        float ahi[P], alo[P];
        double a64[P];
        unsigned valid = 0;
#pragma unroll
        for (int pp = 0; pp < P2; ++pp) {
            float h[2][3], l[2][3];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int q = 2 * pp + u;
                const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
                if (a.outidx[k] >= 0) valid |= 1u << q;
                const double v[3] = {a.nv[k], a.nv[a.ldn + k], a.nv[2 * a.ldn + k]};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    h[u][c] = __double2float_rn(v[c]);
                    l[u][c] = __double2float_rn(v[c] - (double)h[u][c]);
                }
                ahi[q] = 0.f;
                alo[q] = 0.f;
                a64[q] = 0.0;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                nh2[pp][c] = f2_pack(h[0][c], h[1][c]);
                nl2[pp][c] = f2_pack(l[0][c], l[1][c]);
            }
        }
        // the scalar (hi or lo) component c of pixel q
        auto pix = [&](const uint64_t (&v)[P2][3], int q, int c) -> float {
            float lo, hi;
            f2_unpack(v[q >> 1][c], lo, hi);
            return (q & 1) ? hi : lo;
        };
        // warp 0 finds the next segment tile of this chunk at or after `pos` that is not far;
        // lane 0 issues the copy of its Mid2 records
        int64_t pos = first;
        auto issue_next = [&](uint32_t gi) {
            int64_t found = -1;
            int cls = kFar;
            while (pos < j1) {
                const int64_t jj = pos + lane;
                const int c = jj < j1 ? classify(pc, a.scaps[jj], a.d_far) : kFar;
                const unsigned m = __ballot_sync(0xffffffffu, c != kFar);
                if (m) {
                    const int l = __ffs(m) - 1;
                    found = pos + l;
                    cls = __shfl_sync(0xffffffffu, c, l);
                    pos = found + 1;
                    break;
                }
                pos += 32;
            }
            if (lane == 0) {
                const int b = gi % kStages;
                s_j[b] = found;
                s_cls[b] = cls;
                unsigned char *dst = sbuf + (size_t)b * kStageBytes;
                if (found >= 0) {
                    mbar_arrive_expect_tx(&bars[b], (uint32_t)(S * sizeof(Mid2)));
                    bulk_g2s(dst, a.mid + found * S, (uint32_t)(S * sizeof(Mid2)), &bars[b]);
                } else {
                    mbar_arrive_expect_tx(&bars[b], 0u);
                }
            }
        };
        if (w == 0)
            for (int i = 0; i < kStages; ++i) issue_next(g + i);
        int i = 0;
        for (;; ++i) {
            const uint32_t gi = g + i;
            const int buf = gi % kStages;
            // the stage's tile index is read before the barrier: warp 0 rewrites the slot after it
            int64_t j = -1;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[buf], (gi / kStages) & 1, a.wait_polls))) {
                s_abort = 1;
            } else {
                j = s_j[buf];
                if (j >= 0) {
                    const int cls = s_cls[buf];
                    float part[P];
#pragma unroll
                    for (int q = 0; q < P; ++q) part[q] = 0.f;
                    if (cls == kMid) {
                        // Mid2 record: (Xh.x, Xh.y) (Xh.z, Xl.x) (Xl.y, Xl.z) (Xd.x, Xd.y) (Xd.z, -X'.x)
                        // (-X'.y, -X'.z) (c, e) (f, -f), every entry a (v, v) pair.
                        // Per warp and sample: when every pair of the warp has h = 1 - n.Xhat >= d_far^2/2
                        // (with a margin for its FP32 rounding), the direct far-field form
                        // t = (c/2) [B (B - e) - A (A - f)] / [B h]; else d = n - Xhat as a float pair and
                        // t = c [B Xdot.d - A X'.d] / [B d.d] with B = Xdot.d + e, A = X'.d + f.
                        const ulonglong2 *mr = reinterpret_cast<const ulonglong2 *>(sbuf + (size_t)buf * kStageBytes);
                        const float hmin = 0.5f * a.d_far * a.d_far * 1.001f + 1e-6f;
                        uint64_t part2[P2];
#pragma unroll
                        for (int pp = 0; pp < P2; ++pp) part2[pp] = 0ull;
                        for (int s = 0; s < S; ++s) {
                            const ulonglong2 r0 = mr[8 * s], r1 = mr[8 * s + 1];
                            uint64_t h[P2];
                            bool ok = true;
#pragma unroll
                            for (int pp = 0; pp < P2; ++pp) {
                                h[pp] = f2_sub(one2, f2_fma(nh2[pp][2], r1.x, f2_fma(nh2[pp][1], r0.y, f2_mul(nh2[pp][0], r0.x))));
                                float h0, h1;
                                f2_unpack(h[pp], h0, h1);
                                ok = ok && (h0 >= hmin) && (h1 >= hmin);
                            }
                            const ulonglong2 r3 = mr[8 * s + 3], r4 = mr[8 * s + 4], r5 = mr[8 * s + 5];
                            const ulonglong2 r6 = mr[8 * s + 6], r7 = mr[8 * s + 7];
                            if (__all_sync(0xffffffffu, ok)) {
                                const uint64_t ch = f2_mul(r6.x, half2);
#pragma unroll
                                for (int pp = 0; pp < P2; ++pp) {
                                    const uint64_t B = f2_fma(nh2[pp][2], r4.x, f2_fma(nh2[pp][1], r3.y, f2_fma(nh2[pp][0], r3.x, one2)));
                                    const uint64_t An = f2_fma(nh2[pp][2], r5.y, f2_fma(nh2[pp][1], r5.x, f2_mul(nh2[pp][0], r4.y)));
                                    const uint64_t num = f2_fma(An, f2_sub(r7.y, An), f2_mul(B, f2_sub(B, r6.y)));
                                    float d0, d1;
                                    f2_unpack(f2_mul(B, h[pp]), d0, d1);
                                    part2[pp] = f2_fma(f2_mul(ch, num), f2_pack(rcp_approx(d0), rcp_approx(d1)), part2[pp]);
                                }
                                continue;
                            }
                            const ulonglong2 r2 = mr[8 * s + 2];
#pragma unroll
                            for (int pp = 0; pp < P2; ++pp) {
                                const uint64_t dx = f2_add(f2_sub(nh2[pp][0], r0.x), f2_sub(nl2[pp][0], r1.y));
                                const uint64_t dy = f2_add(f2_sub(nh2[pp][1], r0.y), f2_sub(nl2[pp][1], r2.x));
                                const uint64_t dz = f2_add(f2_sub(nh2[pp][2], r1.x), f2_sub(nl2[pp][2], r2.y));
                                const uint64_t Q = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
                                const uint64_t Pd = f2_fma(r4.x, dz, f2_fma(r3.y, dy, f2_mul(r3.x, dx)));
                                const uint64_t Qdn = f2_fma(r5.y, dz, f2_fma(r5.x, dy, f2_mul(r4.y, dx)));
                                const uint64_t B = f2_add(Pd, r6.y);
                                const uint64_t A = f2_sub(r7.x, Qdn);
                                const uint64_t num = f2_fma(A, Qdn, f2_mul(B, Pd));
                                float d0, d1;
                                f2_unpack(f2_mul(B, Q), d0, d1);
                                part2[pp] = f2_fma(f2_mul(r6.x, num), f2_pack(rcp_approx(d0), rcp_approx(d1)), part2[pp]);
                            }
                        }
#pragma unroll
                        for (int pp = 0; pp < P2; ++pp) f2_unpack(part2[pp], part[2 * pp], part[2 * pp + 1]);
                    } else {
                        // checked tile: per sample, the packed float-pair form for every pixel pair; kept
                        // when no pair of the warp is within the tile's largest near radius and every
                        // B is at least b_min (as in a mid tile), else the sample is redone one pixel at a
                        // time from its Seg32 record: B without cancellation, FP64 for |d| < rho or
                        // B < b_min / 1000
                        const ulonglong2 *mr = reinterpret_cast<const ulonglong2 *>(sbuf + (size_t)buf * kStageBytes);
                        const float rmax = a.scaps[j].r.x, rho2 = rmax * rmax, b_safe = a.b_min;
                        const float b_tiny = a.b_min * 1e-3f;
                        uint64_t part2[P2];
#pragma unroll
                        for (int pp = 0; pp < P2; ++pp) part2[pp] = 0ull;
                        for (int s = 0; s < S; ++s) {
                            const ulonglong2 r0 = mr[8 * s], r1 = mr[8 * s + 1], r2 = mr[8 * s + 2], r3 = mr[8 * s + 3];
                            const ulonglong2 r4 = mr[8 * s + 4], r5 = mr[8 * s + 5], r6 = mr[8 * s + 6], r7 = mr[8 * s + 7];
                            uint64_t t2[P2];
                            bool ok = true;
#pragma unroll
                            for (int pp = 0; pp < P2; ++pp) {
                                const uint64_t dx = f2_add(f2_sub(nh2[pp][0], r0.x), f2_sub(nl2[pp][0], r1.y));
                                const uint64_t dy = f2_add(f2_sub(nh2[pp][1], r0.y), f2_sub(nl2[pp][1], r2.x));
                                const uint64_t dz = f2_add(f2_sub(nh2[pp][2], r1.x), f2_sub(nl2[pp][2], r2.y));
                                const uint64_t Q = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
                                const uint64_t Pd = f2_fma(r4.x, dz, f2_fma(r3.y, dy, f2_mul(r3.x, dx)));
                                const uint64_t Qdn = f2_fma(r5.y, dz, f2_fma(r5.x, dy, f2_mul(r4.y, dx)));
                                const uint64_t B = f2_add(Pd, r6.y);
                                const uint64_t A = f2_sub(r7.x, Qdn);
                                const uint64_t num = f2_fma(A, Qdn, f2_mul(B, Pd));
                                float q0, q1, b0, b1, d0, d1;
                                f2_unpack(Q, q0, q1);
                                f2_unpack(B, b0, b1);
                                ok = ok && (q0 >= rho2) && (q1 >= rho2) && (b0 >= b_safe) && (b1 >= b_safe);
                                f2_unpack(f2_mul(B, Q), d0, d1);
                                t2[pp] = f2_mul(f2_mul(r6.x, num), f2_pack(rcp_approx(d0), rcp_approx(d1)));
                            }
                            if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
                                for (int pp = 0; pp < P2; ++pp) part2[pp] = f2_add(part2[pp], t2[pp]);
                                continue;
                            }
                            const Seg32 rec = a.s32[j * S + s];
                            const float4 ra = rec.a, rb = rec.b, rd = rec.d, re = rec.e, rk = rec.k;
                            const float hv = fmaf(-0.5f, rk.w, 0.5f);   // |Xdot| / 2
                            unsigned mask = 0;
#pragma unroll
                            for (int q = 0; q < P; ++q) {
                                const float nx = pix(nh2, q, 0), ny = pix(nh2, q, 1), nz = pix(nh2, q, 2);
                                const float dx = (nx - ra.x) + (pix(nl2, q, 0) - rb.x);
                                const float dy = (ny - ra.y) + (pix(nl2, q, 1) - rb.y);
                                const float dz = (nz - ra.z) + (pix(nl2, q, 2) - rb.z);
                                const float Q = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                                const float Pd = fmaf(rd.z, dz, fmaf(rd.y, dy, rd.x * dx));
                                const float Qd = fmaf(re.z, dz, fmaf(re.y, dy, re.x * dx));
                                const float A = fmaf(nz, re.z, fmaf(ny, re.y, nx * re.x));
                                const float wx = nx + rk.x, wy = ny + rk.y, wz = nz + rk.z;
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
#pragma unroll
                        for (int pp = 0; pp < P2; ++pp) {
                            float lo, hi;
                            f2_unpack(part2[pp], lo, hi);
                            part[2 * pp] += lo;
                            part[2 * pp + 1] += hi;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < P; ++q) fold(ahi[q], alo[q], part[q]);
                }
            }
            __syncthreads();
            if (s_abort || j < 0) break;
            if (w == 0) issue_next(gi + kStages);
        }
        if (s_abort) {
            // stages i .. i + kStages - 1 are issued: copies or zero-byte arrives
            if (tid == 0) drain(bars, g, i, i + kStages, a.st);
            return;
        }
        // stages issued after the end marker are zero-byte arrives, made before the last barrier:
        // their phases are complete; consume them
        for (int m = i + 1; m < i + kStages; ++m) {
            const uint32_t gm = g + m;
            (void)__all_sync(0xffffffffu, mbar_wait_bounded(&bars[gm % kStages], (gm / kStages) & 1, kDrainPolls));
        }
        __syncthreads();
        g += i + kStages;

        // added after the far pass of the same chunk: into the chunk's partial, or into theta
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
            const double v = ((double)ahi[q] + (double)alo[q]) + a64[q];
            if (v != 0.0) {
                if (a.split == 1) {
                    const int64_t oi = a.outidx[k];
                    if (oi >= 0) a.theta[oi] += v;
                } else {
                    a.partial[(int64_t)kc * tot + k] += v;
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        nearcnt += __shfl_xor_sync(0xffffffffu, nearcnt, o);
        zerocnt += __shfl_xor_sync(0xffffffffu, zerocnt, o);
    }
    if (lane == 0 && (nearcnt | zerocnt)) {
        atomicAdd(&a.st->near_pairs, (unsigned long long)nearcnt);
        atomicAdd(&a.st->zero_pairs, (unsigned long long)zerocnt);
    }
}

// Plain FP64 path: every pair in FP64, same tiling.  Segment tiles whose cap is at least d_far
// from the pixel tile's cap are evaluated in the FP64 far-field form
// t = (c/2) [B (B - e) - A (A - f)] / [B (1 - n.Xhat)], written with completed squares scaled by
// sqrt(|c|/2) (Far64 records: 17 FP64 operations per pair; the cancellation in 1 - n.Xhat costs
// at most a factor 2/d_far^2 = 32 of the 1e-16 rounding); the others pair by pair from
// d = n - Xhat formed from the double-double Xhat, with the IEEE division.
template <int NT, int P, int S>
__global__ void __launch_bounds__(NT) k_map_f64(MapArgs a)
{
    constexpr int TILE = NT * P;
    constexpr size_t kStageBytes = S * sizeof(Seg64);
    static_assert(sizeof(Far64) <= sizeof(Seg64), "stage layout");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sbuf = smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    __shared__ int s_abort;
    __shared__ int s_far[kStages];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    unsigned zerocnt = 0;
    uint32_t g = 0;
    __shared__ int64_t s_item;
    const int64_t n_items = a.ntiles * a.split;
    const int64_t tot = a.ntiles * TILE;
    for (int64_t item = next_item(&a.queue[0], &s_item); item < n_items; item = next_item(&a.queue[0], &s_item)) {
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
        const float4 pc = a.pcaps[tile];
        auto issue = [&](int64_t j, uint32_t gi) {
            const int b = gi % kStages;
            const SegCap sc = a.scaps[j];
            const float ex = pc.x - sc.c.x, ey = pc.y - sc.c.y, ez = pc.z - sc.c.z;
            const bool far = sqrtf(ex * ex + ey * ey + ez * ez) - pc.w - sc.c.w >= a.d_far;
            s_far[b] = far;
            unsigned char *dst = sbuf + (size_t)b * kStageBytes;
            if (far) {
                mbar_arrive_expect_tx(&bars[b], (uint32_t)(S * sizeof(Far64)));
                bulk_g2s(dst, a.far64 + j * S, (uint32_t)(S * sizeof(Far64)), &bars[b]);
            } else {
                mbar_arrive_expect_tx(&bars[b], (uint32_t)(S * sizeof(Seg64)));
                bulk_g2s(dst, a.s64 + j * S, (uint32_t)(S * sizeof(Seg64)), &bars[b]);
            }
        };
        if (tid == 0) {
            const int pro = nt < kStages ? nt : kStages;
            for (int i = 0; i < pro; ++i) issue(j0 + i, g + i);
        }
        int i = 0;
        for (; i < nt; ++i) {
            const uint32_t gi = g + i;
            const int buf = gi % kStages;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[buf], (gi / kStages) & 1, a.wait_polls))) {
                s_abort = 1;
            } else {
                double part[P];
#pragma unroll
                for (int q = 0; q < P; ++q) part[q] = 0.0;
                if (s_far[buf]) {
                    const Far64 *fb = reinterpret_cast<const Far64 *>(sbuf + (size_t)buf * kStageBytes);
                    for (int s = 0; s < S; ++s) {
                        const Far64 r = fb[s];
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const double hs = fma(nv[q][2], r.mxh[2], fma(nv[q][1], r.mxh[1], fma(nv[q][0], r.mxh[0], r.sg)));
                            const double B = fma(nv[q][2], r.xd[2], fma(nv[q][1], r.xd[1], fma(nv[q][0], r.xd[0], 1.0)));
                            const double A2 = fma(nv[q][2], r.xp[2], fma(nv[q][1], r.xp[1], fma(nv[q][0], r.xp[0], r.af)));
                            const double B2 = fma(r.sx, B, r.be);
                            const double num = fma(-A2, A2, fma(B2, B2, -r.K));
                            part[q] = fma(num, rcp64(B * hs), part[q]);
                        }
                    }
                } else {
                    const Seg64 *sb = reinterpret_cast<const Seg64 *>(sbuf + (size_t)buf * kStageBytes);
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
                }
#pragma unroll
                for (int q = 0; q < P; ++q) fold64(hi[q], lo[q], part[q]);
            }
            __syncthreads();
            if (s_abort) break;
            if (tid == 0 && i + kStages < nt) issue(j0 + i + kStages, gi + kStages);
        }
        if (s_abort) {
            if (tid == 0) drain(bars, g, i, i + kStages < nt ? i + kStages : nt, a.st);
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
// (threads, pixels per thread, segments per stage, minimum resident CTAs per SM)
#define ISW_F32_VARIANTS(X) \
    X(256, 4, 64, 2)        \
    X(256, 2, 64, 2)        \
    X(128, 4, 64, 4)        \
    X(256, 8, 32, 1)        \
    X(128, 8, 32, 1)        \
    X(256, 4, 64, 3)        \
    X(128, 4, 64, 6)        \
    X(128, 4, 32, 5)        \
    X(128, 4, 128, 4)       \
    X(128, 8, 64, 3)        \
    X(256, 8, 64, 2)

namespace {
struct VEntry {
    Variant v;
    const void *fn;       // far-field pass
    const void *near_fn;  // near-field pass with the same tiling
};
#define ISW_ENTRY(NT, P, S, MB)                                                                                   \
    {{NT, P, S, 32, (NT / 32) * P}, (const void *)&k_map_f32c<NT, P, S, MB>, (const void *)&k_map_f32c_near<NT, P, S>},
const VEntry kF32[] = {ISW_F32_VARIANTS(ISW_ENTRY)};
#undef ISW_ENTRY
constexpr int kF64NT = 128, kF64P = 2, kF64S = 32;

size_t smem_f32(int S) { return kStages * kFarGroup * (S / 2) * sizeof(Far2) + kStages * sizeof(uint64_t); }
// Stages above the default 48 KB of dynamic shared memory need the opt-in attribute.
void allow_smem(const void *fn, size_t bytes)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
size_t smem_near(int S) { return kStages * S * sizeof(Mid2) + kStages * sizeof(uint64_t); }
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
    allow_smem(kF32[idx].fn, smem_f32(v.seg_tile));
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
    allow_smem(kF32[idx].fn, smem_f32(v.seg_tile));
    cudaLaunchKernel(kF32[idx].fn, dim3(grid), dim3(v.threads), args, smem_f32(v.seg_tile), s);
}

// The near-field pass runs the same pixel tiling and segment tiles as the far pass.
void launch_map_f32c_near(int idx, const MapArgs &a, int num_sms, cudaStream_t s)
{
    const Variant v = kF32[idx].v;
    void *args[] = {(void *)&a};
    const void *fn = kF32[idx].near_fn;
    const size_t sm = smem_near(v.seg_tile);
    allow_smem(fn, sm);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, v.threads, sm);
    const int64_t slots = (int64_t)(nb > 0 ? nb : 1) * num_sms;
    const int64_t items = (a.ntiles + a.tile_stride - 1) / a.tile_stride * a.split;
    const int grid = (int)(items < slots ? items : slots);
    cudaLaunchKernel(fn, dim3(grid), dim3(v.threads), args, sm, s);
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
