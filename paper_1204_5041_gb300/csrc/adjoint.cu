// Adjoint of the map (an extension of the method): for a per-pixel g = dL/dTheta, the
// gradient of L with respect to every sample's X, Xdot (and X'), by differentiating the pair
// term of Eq. (1)-(2) and recomputing it pair by pair (nothing is stored per pair).
//
// With d = n - Xhat, Q = d.d, A = n.X', B = 1 + n.Xdot, u = Xdot - (A/B) X', c = -4GU eps dsig/X
// and the pair term t = c T, T = (u.d)/Q, the derivatives of t are combinations of the
// sample's own vectors Xhat, Xdot, X' and of n:
//   dt/dX     = (c/X) [ alpha Xhat - Xdot/Q + (A/(BQ)) X' + eta n ],
//                eta = 2 (u.d)/Q^2,  alpha = (u.Xhat)/Q - eta,
//   dt/dXdot  = c [ T/(1 - Xdot^2) Xdot - Xhat/Q + (1 + A (X'.d)/B^2)/Q n ],
//   dt/dX'    = c [ T/X'^2 X' + (A/(BQ)) Xhat - (X'.d + A)/(BQ) n ],
// so a sample only accumulates four scalars and three n-weighted vectors over the pixels:
//   S1 = sum g alpha, S2 = sum g/Q, S3 = sum g A/(BQ), S4 = sum g T,
//   V1 = sum g eta n, V2 = sum g (1 + A (X'.d)/B^2)/Q n, V3 = sum g (X'.d + A)/(BQ) n,
// and its gradient is assembled once, in FP64, from these sums and its FP64 record.
//
// Work items are (tile of NT samples, chunk of pixel tiles): one thread per sample, pixel
// records of a tile staged in shared memory by 1-D bulk copies and read by every thread.
// FP32 kernel: a pixel tile whose bounding cap is at least d_far from the sample tile's cap (and
// outside its beam cap) is staged as pixel-pair records and summed by a packed f32x2 loop, two
// pixels per instruction, from the far-field form of the sums (adj_far_stage: 30 FP32 lane
// operations and two reciprocals per pair); other tiles go through the checked loop (float-pair
// d, cancellation-free B, FP64 for near pairs).  FP64 kernel: the same sums in FP64 from Pix64
// records, far tiles in the far-field form with Newton-refined reciprocals (rcp64), the others
// pair by pair in the d form with IEEE divisions.  Per-chunk gradients are reduced over chunks in
// a fixed order (deterministic).
#include "isw_internal.cuh"
#include "kernels.cuh"
#include "pipeline.cuh"

namespace isw {

constexpr int kAcc = 13;

// Per-pair derivative sums.  With d = n - Xhat, Q = d.d, u = Xdot - (A/B) X', T = u.d / Q and
// eta = 2T/Q, the n-dependent parts of the three gradients are accumulated as vectors along d
// (and n where d does not appear): sums along n and Xhat separately differ by O(1/|d|) from their
// combination and lose that factor of precision for pixels close to the sample.
//   acc[0] = sum g uX/Q (uX = u.Xhat)   acc[1] = sum g/Q   acc[2] = sum g A/(BQ)   acc[3] = sum g T
//   acc[4..6]   = sum g eta d
//   acc[7..9]   = sum g/Q (d + (A Qd/B^2) n)
//   acc[10..12] = sum g/(BQ) (A d + Qd n)       (Qd = X'.d, Pd = Xdot.d)
// FP64 version (the FP64 kernel and the FP32 kernel's near field)
__device__ __forceinline__ void adj_pair64(double nx, double ny, double nz, double g, const Seg64 &s, int ngrad,
                                           double *acc, unsigned &zero)
{
    const double dx = (nx - s.xh[0]) - s.xl[0];
    const double dy = (ny - s.xh[1]) - s.xl[1];
    const double dz = (nz - s.xh[2]) - s.xl[2];
    const double Q = dx * dx + dy * dy + dz * dz;
    if (Q == 0.0) {
        ++zero;
        return;
    }
    const double A = nx * s.xp[0] + ny * s.xp[1] + nz * s.xp[2];
    const double B = 1.0 + (nx * s.xd[0] + ny * s.xd[1] + nz * s.xd[2]);
    const double Pd = s.xd[0] * dx + s.xd[1] * dy + s.xd[2] * dz;
    const double Qd = s.xp[0] * dx + s.xp[1] * dy + s.xp[2] * dz;
    const double iQ = 1.0 / Q, iB = 1.0 / B;
    const double AB = A * iB;
    const double uX = (s.xd[0] * s.xh[0] + s.xd[1] * s.xh[1] + s.xd[2] * s.xh[2]) -
                      AB * (s.xp[0] * s.xh[0] + s.xp[1] * s.xh[1] + s.xp[2] * s.xh[2]);
    const double T = (Pd - AB * Qd) * iQ;
    const double gq = g * iQ;
    acc[0] += gq * uX;
    acc[1] += gq;
    acc[2] += gq * AB;
    acc[3] += g * T;
    const double ge = 2.0 * g * T * iQ;
    acc[4] += ge * dx;
    acc[5] += ge * dy;
    acc[6] += ge * dz;
    const double v = gq * AB * Qd * iB;
    acc[7] += gq * dx + v * nx;
    acc[8] += gq * dy + v * ny;
    acc[9] += gq * dz + v * nz;
    if (ngrad >= 9) {
        const double gb = gq * iB;
        const double ga = gb * A, gd = gb * Qd;
        acc[10] += ga * dx + gd * nx;
        acc[11] += ga * dy + gd * ny;
        acc[12] += ga * dz + gd * nz;
    }
}

// FP32 version from the pair quantities (shared by the far and checked loops); em1 = Xdot.Xhat,
// f = X'.Xhat
template <bool NG9>
__device__ __forceinline__ void adj_pair32(float dx, float dy, float dz, float Q, float A, float B, float Pd,
                                           float Qd, float em1, float f, float g, float nx, float ny, float nz,
                                           float *p)
{
    const float iQ = rcp_approx(Q), iB = rcp_approx(B);
    const float AB = A * iB;
    const float T = fmaf(-AB, Qd, Pd) * iQ;
    const float gq = g * iQ;
    p[0] = fmaf(gq, fmaf(-AB, f, em1), p[0]);
    p[1] += gq;
    p[2] = fmaf(gq, AB, p[2]);
    p[3] = fmaf(g, T, p[3]);
    const float ge = 2.f * (g * T) * iQ;
    p[4] = fmaf(ge, dx, p[4]);
    p[5] = fmaf(ge, dy, p[5]);
    p[6] = fmaf(ge, dz, p[6]);
    const float v = gq * (AB * Qd * iB);
    p[7] = fmaf(gq, dx, fmaf(v, nx, p[7]));
    p[8] = fmaf(gq, dy, fmaf(v, ny, p[8]));
    p[9] = fmaf(gq, dz, fmaf(v, nz, p[9]));
    if (NG9) {
        const float gb = gq * iB;
        const float ga = gb * A, gd = gb * Qd;
        p[10] = fmaf(ga, dx, fmaf(gd, nx, p[10]));
        p[11] = fmaf(ga, dy, fmaf(gd, ny, p[11]));
        p[12] = fmaf(ga, dz, fmaf(gd, nz, p[12]));
    }
}

// Gradient rows of one sample from its sums (FP64).  With c = -4 GU eps dsigma / |X| and
// eps = sqrt(X'^2 / (1 - Xdot^2)):
//   dTheta/dX     = (c/|X|) [eta d - (u - Xhat uX)/Q]    (c/|X| from dc/dX and the projection
//                                                          of d(Xhat)/dX; the Xhat T terms cancel)
//   dTheta/dXdot  = c [T Xdot / (1 - Xdot^2) + (d + (A Qd/B^2) n)/Q]
//   dTheta/dX'    = c [T X' / X'^2 - (A d + Qd n)/(BQ)]
//   dTheta/ddsigma = (c / dsigma) T = cu T                  (the term is linear in dsigma)
// Rows: X (3), Xdot (3), then X' (3) when ngrad >= 9 and dsigma when ngrad == 10.
__device__ __forceinline__ void adj_assemble(const Seg64 &s, const double *acc, int ngrad, double *out)
{
    const double cX = s.c / s.X;
    const double om2 = s.om * (2.0 - s.om);   // 1 - |Xdot|^2 = (1 - v)(1 + v)
    const double xp2 = s.xp[0] * s.xp[0] + s.xp[1] * s.xp[1] + s.xp[2] * s.xp[2];
    for (int k = 0; k < 3; ++k) {
        const double xh = s.xh[k] + s.xl[k];
        out[k] = cX * (acc[0] * xh - acc[1] * s.xd[k] + acc[2] * s.xp[k] + acc[4 + k]);
        out[3 + k] = s.c * (acc[3] / om2 * s.xd[k] + acc[7 + k]);
        if (ngrad >= 9) out[6 + k] = s.c * ((xp2 > 0.0 ? acc[3] / xp2 : 0.0) * s.xp[k] - acc[10 + k]);
    }
    if (ngrad == 10) out[9] = s.cu * acc[3];
}

__global__ void k_pack_pixels(const double *__restrict__ nv, int64_t ldn, const int64_t *__restrict__ outidx,
                              const double *__restrict__ g, int64_t tot, Pix32 *__restrict__ p32,
                              Pix64 *__restrict__ p64, PixF2 *__restrict__ pf2)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < tot; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t oi = outidx[k];
        Pix64 d;
        Pix32 f;
        if (oi >= 0) {
            for (int c = 0; c < 3; ++c) d.n[c] = nv[c * ldn + k];
            d.g = g[oi];
        } else {
            d.n[0] = d.n[1] = d.n[2] = 0.0;
            d.g = 0.0;
        }
        float hi[3], lo[3];
        for (int c = 0; c < 3; ++c) {
            hi[c] = __double2float_rn(d.n[c]);
            lo[c] = __double2float_rn(d.n[c] - (double)hi[c]);
        }
        const float gf = __double2float_rn(d.g);
        f.a = make_float4(hi[0], hi[1], hi[2], gf);
        f.b = make_float4(lo[0], lo[1], lo[2], 0.f);
        p32[k] = f;
        p64[k] = d;
        // pixel k is half (k & 1) of pair k / 2
        float *fp = reinterpret_cast<float *>(pf2 + k / 2) + (k & 1);
        fp[0] = hi[0];
        fp[2] = hi[1];
        fp[4] = hi[2];
        fp[6] = gf;
    }
}

// Far-field loop of the FP32 adjoint over one stage of pixel-pair records (|d| >= d_far and
// B >= b_min for every pair of the tile pair), two pixels per packed f32x2 operation.  Per pair,
// with d = n - Xhat, Q = d.d, A = n.X', B = 1 + n.Xdot, Xdot.d = B - e and X'.d = A - f
// (e = 1 + Xdot.Xhat, f = X'.Xhat from the sample record) and N = B Xdot.d - A X'.d (so that
// the pair's T = N / (BQ)):
//   gq = g/Q,  ga = gq A/B,  gT = g N/(BQ),  ge = gT/Q,  w = gq + ga (X'.d)/B,  [u = ga + gq (X'.d)/B]
// and the partial sums  S2 = sum gq, S3 = sum ga, S4 = sum gT, V1n = sum ge n, G = sum ge,
// V2 = sum w n [V3 = sum u n]; the signs of N, gT, ge are carried negated so that every step is
// a plain packed multiply or multiply-add.  Q is formed as 2 - 2 n.Xhat and d never appears
// (the sums along n and Xhat replace sum ge d): 30 FP32 lane operations and two reciprocals per
// pair (ngrad 6), against 32 with d (3% faster; gradient errors unchanged at ~1e-7 of the block
// maximum).  Per window of 32 pixel pairs the partials are converted into the accumulator
// layout of the checked loop (adj_pair32): acc0 += (e - 1) S2 - f S3, acc1 += S2, acc2 += S3,
// acc3 += S4, acc4..6 += 2 (V1n - G Xhat), acc7..9 += V2 - S2 Xhat, acc10..12 += V3 - S3 Xhat
// (|d| >= d_far bounds the cancellation of the last three by 1/d_far), and folded into the
// compensated (hi, lo) pairs.
template <int TP, bool NG9>
__device__ __forceinline__ void adj_far_stage(const ulonglong2 *__restrict__ fr, const Seg32 &r, float *ahi,
                                              float *alo)
{
    constexpr int kWin = 32, NP = NG9 ? 13 : 10, kG = NP - 1;
    const uint64_t one2 = f2_pack(1.f, 1.f), two2 = f2_pack(2.f, 2.f);
    const uint64_t cx = f2_pack(-2.f * r.a.x, -2.f * r.a.x), cy = f2_pack(-2.f * r.a.y, -2.f * r.a.y),
                   cz = f2_pack(-2.f * r.a.z, -2.f * r.a.z);
    const uint64_t dx0 = f2_pack(r.d.x, r.d.x), dy0 = f2_pack(r.d.y, r.d.y), dz0 = f2_pack(r.d.z, r.d.z);
    const uint64_t px0 = f2_pack(r.e.x, r.e.x), py0 = f2_pack(r.e.y, r.e.y), pz0 = f2_pack(r.e.z, r.e.z);
    const uint64_t ce = f2_pack(r.d.w, r.d.w), cf = f2_pack(r.e.w, r.e.w);
    for (int w0 = 0; w0 < TP / 2; w0 += kWin) {
        uint64_t ps[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) ps[k] = 0ull;
#pragma unroll 4
        for (int q = w0; q < w0 + kWin; ++q) {
            const ulonglong2 ra = fr[2 * q], rb = fr[2 * q + 1];
            const uint64_t nx = ra.x, ny = ra.y, nz = rb.x, g = rb.y;
            const uint64_t Q = f2_fma(nz, cz, f2_fma(ny, cy, f2_fma(nx, cx, two2)));   // 2 - 2 n.Xhat
            const uint64_t A = f2_fma(nz, pz0, f2_fma(ny, py0, f2_mul(nx, px0)));
            const uint64_t B = f2_fma(nz, dz0, f2_fma(ny, dy0, f2_fma(nx, dx0, one2)));
            const uint64_t Qd = f2_sub(A, cf);                             // X'.d
            const uint64_t Nn = f2_fma(B, f2_sub(ce, B), f2_mul(A, Qd));   // -N
            float q0, q1, b0, b1;
            f2_unpack(Q, q0, q1);
            f2_unpack(B, b0, b1);
            const uint64_t iQ = f2_pack(rcp_approx(q0), rcp_approx(q1));
            const uint64_t iB = f2_pack(rcp_approx(b0), rcp_approx(b1));
            const uint64_t gq = f2_mul(g, iQ);
            const uint64_t gqb = f2_mul(gq, iB);                           // g/(BQ)
            const uint64_t ga = f2_mul(gqb, A);
            const uint64_t gTn = f2_mul(gqb, Nn);                          // -gT
            const uint64_t gen = f2_mul(gTn, iQ);                          // -ge
            const uint64_t t1 = f2_mul(Qd, iB);
            const uint64_t w = f2_fma(ga, t1, gq);
            ps[0] = f2_add(ps[0], gq);
            ps[1] = f2_add(ps[1], ga);
            ps[2] = f2_add(ps[2], gTn);
            ps[3] = f2_fma(gen, nx, ps[3]);
            ps[4] = f2_fma(gen, ny, ps[4]);
            ps[5] = f2_fma(gen, nz, ps[5]);
            ps[kG] = f2_add(ps[kG], gen);
            ps[6] = f2_fma(w, nx, ps[6]);
            ps[7] = f2_fma(w, ny, ps[7]);
            ps[8] = f2_fma(w, nz, ps[8]);
            if (NG9) {
                const uint64_t u = f2_fma(gq, t1, ga);
                ps[9] = f2_fma(u, nx, ps[9]);
                ps[10] = f2_fma(u, ny, ps[10]);
                ps[11] = f2_fma(u, nz, ps[11]);
            }
        }
        float v[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            float lo, hi;
            f2_unpack(ps[k], lo, hi);
            v[k] = lo + hi;
        }
        const float xh[3] = {r.a.x, r.a.y, r.a.z};
        fold(ahi[0], alo[0], fmaf(r.d.w - 1.f, v[0], -r.e.w * v[1]));
        fold(ahi[1], alo[1], v[0]);
        fold(ahi[2], alo[2], v[1]);
        fold(ahi[3], alo[3], -v[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            fold(ahi[4 + c], alo[4 + c], -2.f * fmaf(-v[kG], xh[c], v[3 + c]));
            fold(ahi[7 + c], alo[7 + c], fmaf(-v[0], xh[c], v[6 + c]));
            if (NG9) fold(ahi[10 + c], alo[10 + c], fmaf(-v[1], xh[c], v[9 + c]));
        }
    }
}

// Checked loop of the FP32 adjoint over one stage of Pix32 records: d as a float pair, B formed
// without cancellation, pairs with |d| < rho or B < b_min / 1000 in FP64 from the FP64 records.
template <int TP, bool NG9>
__device__ __forceinline__ void adj_checked_stage(const Pix32 *__restrict__ sp, const Seg32 &r, const AdjArgs &a,
                                                  int64_t pt, int64_t s, int NG, float *ahi, float *alo,
                                                  unsigned &nearcnt, unsigned &zerocnt)
{
    const float em1 = r.d.w - 1.f;   // Xdot.Xhat
    const float hv = fmaf(-0.5f, r.k.w, 0.5f);
    const float b_tiny = a.b_min * 1e-3f;
    // FP32 partial sums over windows of 32 pixels, folded into compensated (hi, lo) pairs
    for (int w0 = 0; w0 < TP; w0 += 32) {
        float part[kAcc];
#pragma unroll
        for (int k = 0; k < kAcc; ++k) part[k] = 0.f;
        for (int q = w0; q < w0 + 32; ++q) {
            const float4 pa = sp[q].a, pb = sp[q].b;
            const float dx = (pa.x - r.a.x) + (pb.x - r.b.x);
            const float dy = (pa.y - r.a.y) + (pb.y - r.b.y);
            const float dz = (pa.z - r.a.z) + (pb.z - r.b.z);
            const float Q = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float Pd = fmaf(r.d.z, dz, fmaf(r.d.y, dy, r.d.x * dx));
            const float Qd = fmaf(r.e.z, dz, fmaf(r.e.y, dy, r.e.x * dx));
            const float A = fmaf(pa.z, r.e.z, fmaf(pa.y, r.e.y, pa.x * r.e.x));
            const float wx = pa.x + r.k.x, wy = pa.y + r.k.y, wz = pa.z + r.k.z;
            const float B = fmaf(hv, fmaf(wz, wz, fmaf(wy, wy, wx * wx)), r.k.w);
            if (Q < r.b.w || B < b_tiny) {
                const Pix64 px = a.p64[pt * TP + q];
                if (px.g != 0.0) {
                    double t64[kAcc];
#pragma unroll
                    for (int k = 0; k < kAcc; ++k) t64[k] = 0.0;
                    const Seg64 s64 = a.s64[s];
                    adj_pair64(px.n[0], px.n[1], px.n[2], px.g, s64, NG, t64, zerocnt);
                    ++nearcnt;
#pragma unroll
                    for (int k = 0; k < kAcc; ++k) {
                        const float th = __double2float_rn(t64[k]);
                        fold(ahi[k], alo[k], th);
                        alo[k] += __double2float_rn(t64[k] - (double)th);
                    }
                }
            } else {
                adj_pair32<NG9>(dx, dy, dz, Q, A, B, Pd, Qd, em1, r.e.w, pa.w, pa.x, pa.y, pa.z, part);
            }
        }
#pragma unroll
        for (int k = 0; k < kAcc; ++k) fold(ahi[k], alo[k], part[k]);
    }
}

// One thread per sample.  Per stage the producer classifies the pixel tile against the CTA's
// sample-tile cap and copies the pixel-pair far records (far tile) or the full Pix32 records.
template <int NT, int TP, bool NG9>
__global__ void __launch_bounds__(NT, 3) k_adj_f32c(AdjArgs a)
{
    constexpr size_t kStageBytes = TP * sizeof(Pix32);
    static_assert(TP % 32 == 0 && (TP / 2) * sizeof(PixF2) <= kStageBytes, "stage layout");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sbuf = smem;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    __shared__ int s_abort;
    __shared__ int s_far[kStages];
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    const int NG = a.ngrad;   // 6, or 9 / 10 with NG9
    unsigned nearcnt = 0, zerocnt = 0;
    uint32_t gl = 0;
    __shared__ int64_t s_item;
    const int64_t n_items = a.nseg_tiles * a.split;
    for (int64_t item = next_item(a.queue, &s_item); item < n_items; item = next_item(a.queue, &s_item)) {
        const int64_t st = item / a.split;
        const int kc = (int)(item - st * a.split);
        const int64_t p0 = a.npix_tiles * kc / a.split, p1 = a.npix_tiles * (kc + 1) / a.split;
        const int nt = (int)(p1 - p0);
        const int64_t s = st * NT + tid;
        const Seg32 r = a.s32[s];
        float ahi[kAcc], alo[kAcc];
#pragma unroll
        for (int k = 0; k < kAcc; ++k) ahi[k] = alo[k] = 0.f;

        auto issue = [&](int64_t pt, uint32_t gi) {
            const int b = gi % kStages;
            const SegCap sc = a.scaps[st];
            const float4 pc = a.pcaps[pt];
            const float ex = pc.x - sc.c.x, ey = pc.y - sc.c.y, ez = pc.z - sc.c.z;
            const float gap = sqrtf(ex * ex + ey * ey + ez * ez) - pc.w - sc.c.w;
            const float bx = pc.x - sc.b.x, by = pc.y - sc.b.y, bz = pc.z - sc.b.z;
            const bool fast_b = sc.b.w < 0.f || sqrtf(bx * bx + by * by + bz * bz) > pc.w + sc.b.w;
            const bool far = fast_b && (gap >= a.d_far);
            s_far[b] = far;
            unsigned char *dst = sbuf + (size_t)b * kStageBytes;
            if (far) {
                const uint32_t bytes = (uint32_t)((TP / 2) * sizeof(PixF2));
                mbar_arrive_expect_tx(&bars[b], bytes);
                bulk_g2s(dst, a.pf2 + pt * (TP / 2), bytes, &bars[b]);
            } else {
                const uint32_t bytes = (uint32_t)(TP * sizeof(Pix32));
                mbar_arrive_expect_tx(&bars[b], bytes);
                bulk_g2s(dst, a.p32 + pt * TP, bytes, &bars[b]);
            }
        };
        if (tid == 0) {
            const int pro = nt < kStages ? nt : kStages;
            for (int i = 0; i < pro; ++i) issue(p0 + i, gl + i);
        }
        int i = 0;
        for (; i < nt; ++i) {
            const uint32_t gi = gl + i;
            const int buf = gi % kStages;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[buf], (gi / kStages) & 1, a.wait_polls))) {
                s_abort = 1;
            } else {
                const unsigned char *stage = sbuf + (size_t)buf * kStageBytes;
                if (s_far[buf]) {
                    adj_far_stage<TP, NG9>(reinterpret_cast<const ulonglong2 *>(stage), r, ahi, alo);
                } else {
                    adj_checked_stage<TP, NG9>(reinterpret_cast<const Pix32 *>(stage), r, a, p0 + i, s, NG, ahi,
                                               alo, nearcnt, zerocnt);
                }
            }
            __syncthreads();
            if (s_abort) break;
            if (tid == 0 && i + kStages < nt) issue(p0 + i + kStages, gi + kStages);
        }
        if (s_abort) {
            if (tid == 0) drain(bars, gl, i, i + kStages < nt ? i + kStages : nt, a.st);
            return;
        }
        gl += nt;
        if (s < a.n) {
            const Seg64 s64 = a.s64[s];
            double acc[kAcc], out[10];
#pragma unroll
            for (int k = 0; k < kAcc; ++k) acc[k] = (double)ahi[k] + (double)alo[k];
            adj_assemble(s64, acc, NG, out);
            if (a.split == 1) {
                for (int k = 0; k < NG; ++k) a.grad[k * a.ld_g + s] = out[k];
            } else {
                for (int k = 0; k < NG; ++k) a.partial[((int64_t)kc * NG + k) * a.n_pad + s] = out[k];
            }
        }
    }
    const int lane = tid & 31;
    for (int o = 16; o > 0; o >>= 1) {
        nearcnt += __shfl_xor_sync(0xffffffffu, nearcnt, o);
        zerocnt += __shfl_xor_sync(0xffffffffu, zerocnt, o);
    }
    if (lane == 0 && (nearcnt | zerocnt)) {
        atomicAdd(&a.st->near_pairs, (unsigned long long)nearcnt);
        atomicAdd(&a.st->zero_pairs, (unsigned long long)zerocnt);
    }
}

template <int NT, int TP>
__global__ void __launch_bounds__(NT) k_adj_f64(AdjArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Pix64 *sbuf = reinterpret_cast<Pix64 *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * TP * sizeof(Pix64));
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    const int NG = a.ngrad;
    unsigned zerocnt = 0;
    uint32_t gl = 0;
    __shared__ int64_t s_item;
    const int64_t n_items = a.nseg_tiles * a.split;
    for (int64_t item = next_item(a.queue, &s_item); item < n_items; item = next_item(a.queue, &s_item)) {
        const int64_t st = item / a.split;
        const int kc = (int)(item - st * a.split);
        const int64_t p0 = a.npix_tiles * kc / a.split, p1 = a.npix_tiles * (kc + 1) / a.split;
        const int nt = (int)(p1 - p0);
        const int64_t s = st * NT + tid;
        const Seg64 s64 = a.s64[s];
        const SegCap sc = a.scaps[st];
        const double xh[3] = {s64.xh[0] + s64.xl[0], s64.xh[1] + s64.xl[1], s64.xh[2] + s64.xl[2]};
        const double e1 = 1.0 + (s64.xd[0] * xh[0] + s64.xd[1] * xh[1] + s64.xd[2] * xh[2]);   // 1 + Xdot.Xhat
        const double f1 = s64.xp[0] * xh[0] + s64.xp[1] * xh[1] + s64.xp[2] * xh[2];           // X'.Xhat
        double acc[kAcc];
        for (int k = 0; k < kAcc; ++k) acc[k] = 0.0;
        if (tid == 0) {
            const int pro = nt < kStages ? nt : kStages;
            for (int i = 0; i < pro; ++i) issue_tile<Pix64, TP>(sbuf, bars, a.p64, p0 + i, gl + i);
        }
        int i = 0;
        for (; i < nt; ++i) {
            const uint32_t gi = gl + i;
            const int buf = gi % kStages;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[buf], (gi / kStages) & 1, a.wait_polls))) {
                s_abort = 1;
            } else {
                const Pix64 *sp = sbuf + buf * TP;
                double part[kAcc];
                for (int k = 0; k < kAcc; ++k) part[k] = 0.0;
                // far pixel tile (cap gap >= d_far): the far-field sums of adj_far_stage in FP64
                const float4 pc = a.pcaps[p0 + i];
                const float ex = pc.x - sc.c.x, ey = pc.y - sc.c.y, ez = pc.z - sc.c.z;
                if (sqrtf(ex * ex + ey * ey + ez * ez) - pc.w - sc.c.w >= a.d_far) {
                    double S2 = 0.0, S3 = 0.0, S4 = 0.0, V1[3] = {0.0, 0.0, 0.0}, V2[3] = {0.0, 0.0, 0.0},
                           V3[3] = {0.0, 0.0, 0.0};
                    for (int q = 0; q < TP; ++q) {
                        const Pix64 px = sp[q];
                        const double dx = px.n[0] - xh[0], dy = px.n[1] - xh[1], dz = px.n[2] - xh[2];
                        const double Q = fma(dz, dz, fma(dy, dy, dx * dx));
                        const double A = fma(px.n[2], s64.xp[2], fma(px.n[1], s64.xp[1], px.n[0] * s64.xp[0]));
                        const double B = fma(px.n[2], s64.xd[2], fma(px.n[1], s64.xd[1], fma(px.n[0], s64.xd[0], 1.0)));
                        const double Qd = A - f1;
                        const double Nn = fma(B, e1 - B, A * Qd);   // -(B Xdot.d - A X'.d)
                        const double iBQ = rcp64(B * Q), iQ = B * iBQ, iB = Q * iBQ;
                        const double gq = px.g * iQ, gqb = px.g * iBQ;
                        const double ga = gqb * A, gTn = gqb * Nn, gen = gTn * iQ;
                        const double t1 = Qd * iB, w = fma(ga, t1, gq);
                        S2 += gq;
                        S3 += ga;
                        S4 += gTn;
                        V1[0] = fma(gen, dx, V1[0]);
                        V1[1] = fma(gen, dy, V1[1]);
                        V1[2] = fma(gen, dz, V1[2]);
                        for (int c = 0; c < 3; ++c) V2[c] = fma(w, px.n[c], V2[c]);
                        if (NG >= 9) {
                            const double u = fma(gq, t1, ga);
                            for (int c = 0; c < 3; ++c) V3[c] = fma(u, px.n[c], V3[c]);
                        }
                    }
                    part[0] = (e1 - 1.0) * S2 - f1 * S3;
                    part[1] = S2;
                    part[2] = S3;
                    part[3] = -S4;
                    for (int c = 0; c < 3; ++c) {
                        part[4 + c] = -2.0 * V1[c];
                        part[7 + c] = V2[c] - S2 * xh[c];
                        part[10 + c] = V3[c] - S3 * xh[c];
                    }
                } else {
                    unsigned z = 0;
                    for (int q = 0; q < TP; ++q) {
                        const Pix64 px = sp[q];
                        if (px.g != 0.0) adj_pair64(px.n[0], px.n[1], px.n[2], px.g, s64, NG, part, z);
                    }
                    if (s < a.n) zerocnt += z;
                }
                for (int k = 0; k < kAcc; ++k) acc[k] += part[k];
            }
            __syncthreads();
            if (s_abort) break;
            if (tid == 0 && i + kStages < nt) issue_tile<Pix64, TP>(sbuf, bars, a.p64, p0 + i + kStages, gi + kStages);
        }
        if (s_abort) {
            if (tid == 0) drain(bars, gl, i, i + kStages < nt ? i + kStages : nt, a.st);
            return;
        }
        gl += nt;
        if (s < a.n) {
            double out[10];
            adj_assemble(s64, acc, NG, out);
            if (a.split == 1) {
                for (int k = 0; k < NG; ++k) a.grad[k * a.ld_g + s] = out[k];
            } else {
                for (int k = 0; k < NG; ++k) a.partial[((int64_t)kc * NG + k) * a.n_pad + s] = out[k];
            }
        }
    }
    const int lane = tid & 31;
    for (int o = 16; o > 0; o >>= 1) zerocnt += __shfl_xor_sync(0xffffffffu, zerocnt, o);
    if (lane == 0 && zerocnt) atomicAdd(&a.st->zero_pairs, (unsigned long long)zerocnt);
}

// grad[k][s] = sum over chunks c = 0..split-1 of partial[c][k][s], fixed order, compensated
__global__ void k_adj_reduce(const double *__restrict__ partial, int split, int ngrad, int64_t n, int64_t n_pad,
                             double *__restrict__ grad, int64_t ld_g)
{
    const int64_t tot = (int64_t)ngrad * n;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx / n, s = idx - k * n;
        double hi = 0.0, lo = 0.0;
        for (int c = 0; c < split; ++c) fold64(hi, lo, partial[((int64_t)c * ngrad + k) * n_pad + s]);
        grad[k * ld_g + s] = hi + lo;
    }
}

namespace {
constexpr int kAdjNT = 128, kAdjTP = 256, kAdj64NT = 128, kAdj64TP = 128;
size_t smem_adj32() { return kStages * kAdjTP * sizeof(Pix32) + kStages * sizeof(uint64_t); }
size_t smem_adj64() { return kStages * kAdj64TP * sizeof(Pix64) + kStages * sizeof(uint64_t); }
}  // namespace

int adj_seg_tile(int prec) { return prec == ISW_F32C ? kAdjNT : kAdj64NT; }
int adj_pix_tile(int prec) { return prec == ISW_F32C ? kAdjTP : kAdj64TP; }

int adj_slots(int prec, int ngrad, int num_sms)
{
    int nb = 0;
    if (prec == ISW_F32C) {
        const void *fn = ngrad >= 9 ? (const void *)&k_adj_f32c<kAdjNT, kAdjTP, true>
                                    : (const void *)&k_adj_f32c<kAdjNT, kAdjTP, false>;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kAdjNT, smem_adj32());
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)&k_adj_f64<kAdj64NT, kAdj64TP>, kAdj64NT,
                                                      smem_adj64());
    }
    return (nb > 0 ? nb : 1) * num_sms;
}

void launch_pack_pixels(const double *nv, int64_t ldn, const int64_t *outidx, const double *g, int64_t tot,
                        Pix32 *p32, Pix64 *p64, PixF2 *pf2, cudaStream_t s)
{
    int64_t blocks = (tot + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    k_pack_pixels<<<(unsigned)blocks, 256, 0, s>>>(nv, ldn, outidx, g, tot, p32, p64, pf2);
}

void launch_adjoint(int prec, const AdjArgs &a, int grid, cudaStream_t s)
{
    void *args[] = {(void *)&a};
    if (prec == ISW_F32C) {
        const void *fn = a.ngrad >= 9 ? (const void *)&k_adj_f32c<kAdjNT, kAdjTP, true>
                                      : (const void *)&k_adj_f32c<kAdjNT, kAdjTP, false>;
        cudaLaunchKernel(fn, dim3(grid), dim3(kAdjNT), args, smem_adj32(), s);
    } else {
        cudaLaunchKernel((const void *)&k_adj_f64<kAdj64NT, kAdj64TP>, dim3(grid), dim3(kAdj64NT), args,
                         smem_adj64(), s);
    }
    if (a.split > 1) {
        const int64_t tot = (int64_t)a.ngrad * a.n;
        int64_t blocks = (tot + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        k_adj_reduce<<<(unsigned)blocks, 256, 0, s>>>(a.partial, a.split, a.ngrad, a.n, a.n_pad, a.grad, a.ld_g);
    }
}

}  // namespace isw
