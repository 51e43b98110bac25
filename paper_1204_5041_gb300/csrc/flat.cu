// Flat-sky / small-angle map of a gnomonic patch (Sec. II.A: the limit X n -> X with parallel
// photon paths; Fig. 3 compares it with the full-sky map of the same patch).  A sample at depth
// Z = (X - x_obs).e3 > 0 sits at (xi_s, eta_s) = ((X - x_obs).e1, (X - x_obs).e2) / Z of the patch
// and contributes
//     t = -4 GU eps dsigma / Z * (u_perp . d) / |d|^2,   d = (xi - xi_s, eta - eta_s),
// with u = Xdot - (e3.X') X' / (1 + e3.Xdot) and u_perp = (u.e1, u.e2).  Per sample the record
// holds (xi_s, eta_s) and w = (-4 GU eps dsigma / Z) u_perp, so a pair costs d, |d|^2, w.d and
// one reciprocal.  FP32 records keep the positions as float pairs (hi + lo): d is formed to
// ~1e-15 absolute before the FP32 arithmetic, and the per-pixel sums are compensated.  Samples
// behind the patch plane (Z <= 0) get zero weight; d = 0 contributes zero.
#include <type_traits>

#include "isw_internal.cuh"
#include "kernels.cuh"
#include "pipeline.cuh"

namespace isw {

struct __align__(16) Flat32 {
    float4 a;   // xi_s hi, eta_s hi, xi_s lo, eta_s lo
    float4 b;   // w1, w2, 0, 0
};
struct __align__(16) Flat64 {
    double xs, ys, w1, w2;
};

constexpr int kFlatNT = 128, kFlatP = 4, kFlatS = 128;

__global__ void k_flat_pack(const double *__restrict__ S, int64_t n, int64_t ld, PatchSpec p, double xo0, double xo1,
                            double xo2, double GU, int64_t n_pad, Flat32 *__restrict__ r32, Flat64 *__restrict__ r64)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
        double xs = 1e3, ys = 1e3, w1 = 0.0, w2 = 0.0;   // zero weight, far from the patch
        if (s < n) {
            // IEEE operations in a fixed order (no contraction): the positions are specified
            // exactly, because the 1/|d| term amplifies their rounding near a pixel centre
            auto dot = [](const double *x, const double *y) {
                return dadd(dadd(dmul(x[0], y[0]), dmul(x[1], y[1])), dmul(x[2], y[2]));
            };
            const double r[3] = {dsub(S[s], xo0), dsub(S[ld + s], xo1), dsub(S[2 * ld + s], xo2)};
            const double Xd[3] = {S[3 * ld + s], S[4 * ld + s], S[5 * ld + s]};
            const double Xp[3] = {S[6 * ld + s], S[7 * ld + s], S[8 * ld + s]};
            const double *e1 = p.frame, *e2 = p.frame + 3, *e3 = p.frame + 6;
            const double Z = dot(r, e3);
            const double om = dsub(1.0, dot(Xd, Xd));
            const double eps = dsqrt(ddiv(dot(Xp, Xp), om));
            const double Bz = dadd(1.0, dot(e3, Xd)), Az = dot(e3, Xp);
            const double kd = ddiv(dmul(dmul(-4.0, GU), dmul(eps, S[9 * ld + s])), Z);
            if (Z > 0.0 && om > 0.0 && Bz > 0.0 && isfinite(kd)) {
                double u[3];
                for (int k = 0; k < 3; ++k) u[k] = dsub(Xd[k], ddiv(dmul(Az, Xp[k]), Bz));
                xs = ddiv(dot(r, e1), Z);
                ys = ddiv(dot(r, e2), Z);
                w1 = dmul(kd, dot(u, e1));
                w2 = dmul(kd, dot(u, e2));
            }
        }
        const float xh = __double2float_rn(xs), yh = __double2float_rn(ys);
        Flat32 f;
        f.a = make_float4(xh, yh, __double2float_rn(xs - (double)xh), __double2float_rn(ys - (double)yh));
        f.b = make_float4(__double2float_rn(w1), __double2float_rn(w2), 0.f, 0.f);
        r32[s] = f;
        Flat64 g;
        g.xs = xs;
        g.ys = ys;
        g.w1 = w1;
        g.w2 = w2;
        r64[s] = g;
    }
}

struct FlatArgs {
    const Flat32 *r32;
    const Flat64 *r64;
    const int64_t *outidx;   // patch table output slots (-1 padding)
    int64_t ntiles;
    int64_t nst;             // sample tiles
    int split;
    int64_t M;
    double pitch;
    double *theta;
    double *partial;
    int accumulate;
    DevStatus *st;
    unsigned long long *queue;
    uint32_t wait_polls;
};

template <bool F64>
__global__ void __launch_bounds__(kFlatNT) k_map_flat(FlatArgs a)
{
    using Rec = typename std::conditional<F64, Flat64, Flat32>::type;
    constexpr int NT = kFlatNT, P = kFlatP, S = kFlatS, TILE = NT * P;
    extern __shared__ __align__(128) unsigned char smem[];
    Rec *sbuf = reinterpret_cast<Rec *>(smem);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * S * sizeof(Rec));
    __shared__ int s_abort;
    __shared__ int64_t s_item;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    const Rec *src = F64 ? reinterpret_cast<const Rec *>(a.r64) : reinterpret_cast<const Rec *>(a.r32);
    uint32_t g = 0;
    const int64_t n_items = a.ntiles * a.split;
    const int64_t tot = a.ntiles * TILE;
    for (int64_t item = next_item(a.queue, &s_item); item < n_items; item = next_item(a.queue, &s_item)) {
        const int64_t tile = item / a.split;
        const int kc = (int)(item - tile * a.split);
        const int64_t j0 = a.nst * kc / a.split, j1 = a.nst * (kc + 1) / a.split;
        const int nt = (int)(j1 - j0);
        // pixel coordinates from the patch slot; padding slots sit far away with no output
        double px[P], py[P];
        float xh[P], yh[P], xl[P], yl[P], ahi[P], alo[P];
        double s64[P], s64lo[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
            const int64_t oi = a.outidx[k];
            const int64_t i = oi >= 0 ? oi % a.M : 0, j = oi >= 0 ? oi / a.M : 0;
            px[q] = dmul(dsub(dadd((double)i, 0.5), dmul(0.5, (double)a.M)), a.pitch);
            py[q] = dmul(dsub(dadd((double)j, 0.5), dmul(0.5, (double)a.M)), a.pitch);
            xh[q] = __double2float_rn(px[q]);
            yh[q] = __double2float_rn(py[q]);
            xl[q] = __double2float_rn(px[q] - (double)xh[q]);
            yl[q] = __double2float_rn(py[q] - (double)yh[q]);
            ahi[q] = alo[q] = 0.f;
            s64[q] = s64lo[q] = 0.0;
        }
        if (tid == 0) {
            const int pro = nt < kStages ? nt : kStages;
            for (int i = 0; i < pro; ++i) issue_tile<Rec, S>(sbuf, bars, src, j0 + i, g + i);
        }
        int i = 0;
        for (; i < nt; ++i) {
            const uint32_t gi = g + i;
            const int buf = gi % kStages;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[buf], (gi / kStages) & 1, a.wait_polls))) {
                s_abort = 1;
            } else {
                const Rec *sb = sbuf + buf * S;
                if constexpr (F64) {
                    double part[P];
#pragma unroll
                    for (int q = 0; q < P; ++q) part[q] = 0.0;
#pragma unroll 2
                    for (int s = 0; s < S; ++s) {
                        const Flat64 r = sb[s];
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const double dx = dsub(px[q], r.xs), dy = dsub(py[q], r.ys);
                            const double Q = dadd(dmul(dx, dx), dmul(dy, dy));
                            part[q] += Q > 0.0 ? ddiv(dadd(dmul(r.w1, dx), dmul(r.w2, dy)), Q) : 0.0;
                        }
                    }
                    // per-tile partials folded into compensated (hi, lo) pairs: the terms of
                    // strings on either side of a pixel cancel
#pragma unroll
                    for (int q = 0; q < P; ++q) fold64(s64[q], s64lo[q], part[q]);
                } else {
                    float part[P];
#pragma unroll
                    for (int q = 0; q < P; ++q) part[q] = 0.f;
#pragma unroll 4
                    for (int s = 0; s < S; ++s) {
                        const float4 ra = sb[s].a, rb = sb[s].b;
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            const float dx = (xh[q] - ra.x) + (xl[q] - ra.z);
                            const float dy = (yh[q] - ra.y) + (yl[q] - ra.w);
                            // d = 0 exactly makes the numerator 0: the floor keeps 0 * (1/Q) finite
                            const float Q = fmaxf(fmaf(dy, dy, dx * dx), 1e-30f);
                            part[q] = fmaf(fmaf(rb.y, dy, rb.x * dx), rcp_approx(Q), part[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < P; ++q) fold(ahi[q], alo[q], part[q]);
                }
            }
            __syncthreads();
            if (s_abort) break;
            if (tid == 0 && i + kStages < nt) issue_tile<Rec, S>(sbuf, bars, src, j0 + i + kStages, gi + kStages);
        }
        if (s_abort) {
            if (tid == 0) drain(bars, g, i, i + kStages < nt ? i + kStages : nt, a.st);
            return;
        }
        g += nt;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int64_t k = tile * TILE + (w * P + q) * 32 + lane;
            const double v = F64 ? s64[q] + s64lo[q] : (double)ahi[q] + (double)alo[q];
            if (a.split == 1) {
                const int64_t oi = a.outidx[k];
                if (oi >= 0) a.theta[oi] = a.accumulate ? a.theta[oi] + v : v;
            } else {
                a.partial[(int64_t)kc * tot + k] = v;
            }
        }
    }
}

int flat_seg_tile() { return kFlatS; }
int flat_tx() { return 32; }
int flat_ty() { return kFlatNT / 32 * kFlatP; }

void launch_flat_pack(const double *S, int64_t n, int64_t ld, const PatchSpec &p, double xo0, double xo1, double xo2,
                      double GU, int64_t n_pad, void *r32, void *r64, cudaStream_t s)
{
    int64_t b = (n_pad + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    k_flat_pack<<<(unsigned)b, 256, 0, s>>>(S, n, ld, p, xo0, xo1, xo2, GU, n_pad, (Flat32 *)r32, (Flat64 *)r64);
}

size_t flat_record_bytes() { return sizeof(Flat32) + sizeof(Flat64); }

int flat_slots(bool f64, int num_sms)
{
    const void *fn = f64 ? (const void *)&k_map_flat<true> : (const void *)&k_map_flat<false>;
    const size_t sm = kStages * kFlatS * (f64 ? sizeof(Flat64) : sizeof(Flat32)) + kStages * sizeof(uint64_t);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kFlatNT, sm);
    return (nb > 0 ? nb : 1) * num_sms;
}

void launch_map_flat(bool f64, const void *r32, const void *r64, const int64_t *outidx, int64_t ntiles, int64_t nst,
                     int split, int64_t M, double pitch, double *theta, double *partial, int accumulate,
                     DevStatus *st, unsigned long long *queue, uint32_t wait_polls, int grid, cudaStream_t s)
{
    FlatArgs a;
    a.r32 = (const Flat32 *)r32;
    a.r64 = (const Flat64 *)r64;
    a.outidx = outidx;
    a.ntiles = ntiles;
    a.nst = nst;
    a.split = split;
    a.M = M;
    a.pitch = pitch;
    a.theta = theta;
    a.partial = partial;
    a.accumulate = accumulate;
    a.st = st;
    a.queue = queue;
    a.wait_polls = wait_polls;
    const size_t sm = kStages * kFlatS * (f64 ? sizeof(Flat64) : sizeof(Flat32)) + kStages * sizeof(uint64_t);
    if (f64) k_map_flat<true><<<grid, kFlatNT, sm, s>>>(a);
    else k_map_flat<false><<<grid, kFlatNT, sm, s>>>(a);
}

}  // namespace isw
