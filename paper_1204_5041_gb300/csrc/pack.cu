// Per-sample records of the map kernels (FP64 in, FP32 + FP64 out) and per-tile caps.
//
// With D = X n - X_s = X (n - Xhat), X = |X_s - x_obs|, Eq. (1)-(2) per pair become
//   t = c [ B (Xdot.d) - A (X'.d) ] / [ B (d.d) ],  d = n - Xhat,  A = n.X',  B = 1 + n.Xdot,
//   c = -4 GU eps dsigma / X,  eps^2 = X'^2 / (1 - Xdot^2)  (text after Eq. 1).
// Xhat is formed in double-double so that d keeps full relative accuracy when n is close
// to Xhat (near a string d cancels); the FP32 record carries it as a float pair (hi, lo).
#include "isw_internal.cuh"
#include "kernels.cuh"

namespace isw {

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    const double x = dadd(a, b);
    const double bb = dsub(x, a);
    e = dadd(dsub(a, dsub(x, bb)), dsub(b, bb));
    s = x;
}

// exact product: p + e = a * b
__device__ __forceinline__ void two_prod(double a, double b, double &p, double &e)
{
    p = dmul(a, b);
    e = __fma_rn(a, b, -p);
}

// r / |r| as hi + lo per component, and |r|
__device__ __forceinline__ void unit_dd(const double r[3], double hi[3], double lo[3], double &norm)
{
    double sh = 0.0, sl = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double p, pe, s, se;
        two_prod(r[k], r[k], p, pe);
        two_sum(sh, p, s, se);
        sl = dadd(sl, dadd(se, pe));
        two_sum(s, sl, sh, sl);
    }
    const double q = dsqrt(sh);
    double qq, qqe;
    two_prod(q, q, qq, qqe);
    const double ql = ddiv(dadd(dsub(dsub(sh, qq), qqe), sl), dmul(2.0, q));
    double nh, nl;
    two_sum(q, ql, nh, nl);
    norm = nh;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double q1 = ddiv(r[k], nh);
        double p, pe;
        two_prod(q1, nh, p, pe);
        const double rem = dsub(dsub(dsub(r[k], p), pe), dmul(q1, nl));
        const double q2 = ddiv(rem, nh);
        two_sum(q1, q2, hi[k], lo[k]);
    }
}

__global__ void k_pack(const double *__restrict__ S, int64_t n, int64_t ld, double xo0, double xo1, double xo2,
                       double GU, double theta_pix, double near_k, int64_t n_pad, const uint32_t *__restrict__ perm,
                       Seg32 *__restrict__ s32, Seg64 *__restrict__ s64, Far2 *__restrict__ far,
                       Mid2 *__restrict__ mid, Far64 *__restrict__ far64, DevStatus *ds)
{
    unsigned long long bad = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad; s += (int64_t)gridDim.x * blockDim.x) {
        Seg64 g;
        Seg32 f;
        if (s < n) {
            const int64_t src = perm ? (int64_t)perm[s] : s;   // record s holds sample perm[s]
            const double r[3] = {dsub(S[src], xo0), dsub(S[ld + src], xo1), dsub(S[2 * ld + src], xo2)};
            double X;
            unit_dd(r, g.xh, g.xl, X);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                g.xd[k] = S[(3 + k) * ld + src];
                g.xp[k] = S[(6 + k) * ld + src];
            }
            const double dsig = S[9 * ld + src];
            const double v2 = dadd(dadd(dmul(g.xd[0], g.xd[0]), dmul(g.xd[1], g.xd[1])), dmul(g.xd[2], g.xd[2]));
            const double xp2 = dadd(dadd(dmul(g.xp[0], g.xp[0]), dmul(g.xp[1], g.xp[1])), dmul(g.xp[2], g.xp[2]));
            const double om2 = dsub(1.0, v2);
            const double eps = dsqrt(ddiv(xp2, om2));
            const double w = dmul(eps, dsig);
            double c = ddiv(dmul(-4.0 * GU, w), X);
            const bool ok = (om2 > 0.0) && (X > 0.0) && isfinite(c);
            if (!ok) {
                c = 0.0;
                ++bad;
            }
            g.c = c;
            g.cu = ok ? ddiv(dmul(-4.0 * GU, eps), X) : 0.0;
            g.om = ok ? dsub(1.0, dsqrt(v2)) : 1.0;
            g.X = ok ? X : 1.0;
            // near-field chord radius: near_k * max(pixel size, angular length of the segment)
            double ang = ok ? ddiv(w, X) : 0.0;
            if (!(ang < 1.0)) ang = 1.0;
            const double rho = near_k * fmax(theta_pix, ang);
            float hi32[3], lo32[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                hi32[k] = __double2float_rn(g.xh[k]);
                lo32[k] = __double2float_rn(dadd(dsub(g.xh[k], (double)hi32[k]), g.xl[k]));
            }
            f.a = make_float4(hi32[0], hi32[1], hi32[2], __double2float_rn(c));
            f.b = make_float4(lo32[0], lo32[1], lo32[2], ok ? __double2float_rn(rho * rho) : -1.0f);
            // far-field constants: Xdot.d = B - e and X'.d = A - f with d = n - Xhat
            const double e1 = dadd(1.0, dadd(dadd(dmul(g.xd[0], g.xh[0]), dmul(g.xd[1], g.xh[1])), dmul(g.xd[2], g.xh[2])));
            const double f1 = dadd(dadd(dmul(g.xp[0], g.xh[0]), dmul(g.xp[1], g.xh[1])), dmul(g.xp[2], g.xh[2]));
            f.d = make_float4(__double2float_rn(g.xd[0]), __double2float_rn(g.xd[1]), __double2float_rn(g.xd[2]),
                              __double2float_rn(e1));
            f.e = make_float4(__double2float_rn(g.xp[0]), __double2float_rn(g.xp[1]), __double2float_rn(g.xp[2]),
                              __double2float_rn(f1));
            {
                const double v = dsqrt(v2);
                const double iv = v > 0.0 ? ddiv(1.0, v) : 0.0;
                f.k = make_float4(__double2float_rn(dmul(g.xd[0], iv)), __double2float_rn(dmul(g.xd[1], iv)),
                                  __double2float_rn(dmul(g.xd[2], iv)), __double2float_rn(g.om));
            }
            if (!ok) {
                // skipped sample: zero weight, moved to Xhat = 0 so every pair stays finite
                f.k = make_float4(0.f, 0.f, 0.f, 1.f);
                f.a = make_float4(0.f, 0.f, 0.f, 0.f);
                f.b = make_float4(0.f, 0.f, 0.f, -1.f);
                f.d = make_float4(0.f, 0.f, 0.f, 1.f);
                f.e = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int k = 0; k < 3; ++k) g.xh[k] = g.xl[k] = g.xd[k] = g.xp[k] = 0.0;
                g.om = 1.0;
                g.X = 1.0;
                g.cu = 0.0;
            }
        } else {
            // padding: zero weight at Xhat = 0 (so d = n, d.d = 1), never near, B = 1
            for (int k = 0; k < 3; ++k) g.xh[k] = g.xl[k] = g.xd[k] = g.xp[k] = 0.0;
            g.c = 0.0;
            g.cu = 0.0;
            g.om = 1.0;
            g.X = 1.0;
            f.a = make_float4(0.f, 0.f, 0.f, 0.f);
            f.b = make_float4(0.f, 0.f, 0.f, -1.f);
            f.d = make_float4(0.f, 0.f, 0.f, 1.f);
            f.e = make_float4(0.f, 0.f, 0.f, 0.f);
            f.k = make_float4(0.f, 0.f, 0.f, 1.f);
        }
        s32[s] = f;
        s64[s] = g;
        if (mid) {
            // from the FP32 record (a skipped or padding sample has c = 0: its terms are zero)
            const float v[kMidConsts] = {f.a.x, f.a.y, f.a.z, f.b.x, f.b.y, f.b.z, f.d.x, f.d.y, f.d.z,
                                         -f.e.x, -f.e.y, -f.e.z, f.a.w, f.d.w, f.e.w, -f.e.w};
            float4 *dst = mid[s].v;
#pragma unroll
            for (int k = 0; k < kMidConsts / 2; ++k) dst[k] = make_float4(v[2 * k], v[2 * k], v[2 * k + 1], v[2 * k + 1]);
        }
        if (far64) {
            Far64 r;
            const double xh[3] = {g.xh[0] + g.xl[0], g.xh[1] + g.xl[1], g.xh[2] + g.xl[2]};
            const double ch = 0.5 * g.c;
            const double sg = ch < 0.0 ? -1.0 : 1.0, sq = sqrt(fabs(ch));
            const double e1 = 1.0 + (g.xd[0] * xh[0] + g.xd[1] * xh[1] + g.xd[2] * xh[2]);
            const double f1 = g.xp[0] * xh[0] + g.xp[1] * xh[1] + g.xp[2] * xh[2];
            for (int k = 0; k < 3; ++k) {
                r.mxh[k] = -sg * xh[k];
                r.xd[k] = g.xd[k];
                r.xp[k] = sq * g.xp[k];
            }
            r.sg = sg;
            r.sx = sq;
            r.be = -0.5 * sq * e1;
            r.af = -0.5 * sq * f1;
            r.K = fabs(ch) * 0.25 * (e1 * e1 - f1 * f1);
            far64[s] = r;
        }
        if (far) {
            // far-field constants from the FP64 record (zero weight gives a zero record with sigma = 1)
            const double ch = 0.5 * g.c;
            const double sg = ch < 0.0 ? -1.0 : 1.0;
            const double sq = sqrt(fabs(ch));
            const double xh[3] = {g.xh[0] + g.xl[0], g.xh[1] + g.xl[1], g.xh[2] + g.xl[2]};
            const double e1 = 1.0 + (g.xd[0] * xh[0] + g.xd[1] * xh[1] + g.xd[2] * xh[2]);
            const double f1 = g.xp[0] * xh[0] + g.xp[1] * xh[1] + g.xp[2] * xh[2];
            const float v[kFarConsts] = {(float)(-sg * xh[0]), (float)(-sg * xh[1]), (float)(-sg * xh[2]), (float)sg,
                                         (float)g.xd[0], (float)g.xd[1], (float)g.xd[2], (float)(-0.5 * sq * e1),
                                         (float)(sq * g.xp[0]), (float)(sq * g.xp[1]), (float)(sq * g.xp[2]),
                                         (float)(-0.5 * sq * f1), (float)sq,
                                         (float)(fabs(ch) * 0.25 * (f1 * f1 - e1 * e1))};
            float *dst = reinterpret_cast<float *>(far + (s >> 1)) + (s & 1);
#pragma unroll
            for (int k = 0; k < kFarConsts; ++k) dst[2 * k] = v[k];
        }
    }
    if (bad) {
        atomicAdd(&ds->domain_segs, bad);
        atomicOr(&ds->bits, kStatDomain);
    }
}

// One warp per segment tile: centre of the Xhat directions, largest chord to it, largest
// near radius and smallest 1 - |Xdot| over the tile's real samples.
__global__ void k_seg_caps(const Seg32 *__restrict__ s32, const Seg64 *__restrict__ s64, int64_t n, int64_t n_pad,
                           int seg_tile, float b_min, SegCap *__restrict__ caps)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t ntile = n_pad / seg_tile;
    if (warp >= ntile) return;
    const int64_t base = warp * seg_tile;
    float sx = 0.f, sy = 0.f, sz = 0.f, rho2 = 0.f, om = 1.f;
    for (int l = lane; l < seg_tile; l += 32) {
        const int64_t s = base + l;
        const float4 b = s32[s < n ? s : 0].b;
        if (s < n && b.w >= 0.f) {
            const float4 a = s32[s].a;
            sx += a.x;
            sy += a.y;
            sz += a.z;
            rho2 = fmaxf(rho2, b.w);
            om = fminf(om, (float)s64[s].om);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        rho2 = fmaxf(rho2, __shfl_xor_sync(0xffffffffu, rho2, o));
        om = fminf(om, __shfl_xor_sync(0xffffffffu, om, o));
    }
    const float nrm = sqrtf(sx * sx + sy * sy + sz * sz);
    float cx = 0.f, cy = 0.f, cz = 1.f;
    if (nrm > 0.f) {
        cx = sx / nrm;
        cy = sy / nrm;
        cz = sz / nrm;
    }
    float r = 0.f;
    for (int l = lane; l < seg_tile; l += 32) {
        const int64_t s = base + l;
        if (s < n && s32[s].b.w >= 0.f) {
            const float4 a = s32[s].a;
            const float dx = a.x - cx, dy = a.y - cy, dz = a.z - cz;
            r = fmaxf(r, sqrtf(dx * dx + dy * dy + dz * dz));
        }
    }
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    // beam cap: directions n with B = 1 + n.Xdot < b_min lie within chord sqrt(2 b_min / |Xdot|)
    // of -Xdot/|Xdot|, and only samples with 1 - |Xdot| < b_min have any
    float bx = 0.f, by = 0.f, bz = 0.f;
    int nb = 0;
    for (int l = lane; l < seg_tile; l += 32) {
        const int64_t s = base + l;
        if (s < n && s32[s].b.w >= 0.f && s64[s].om < (double)b_min) {
            const float4 k = s32[s].k;
            bx -= k.x;
            by -= k.y;
            bz -= k.z;
            ++nb;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        bx += __shfl_xor_sync(0xffffffffu, bx, o);
        by += __shfl_xor_sync(0xffffffffu, by, o);
        bz += __shfl_xor_sync(0xffffffffu, bz, o);
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    float4 beam = make_float4(0.f, 0.f, 1.f, -1.f);
    if (nb > 0) {
        const float bn = sqrtf(bx * bx + by * by + bz * bz);
        if (bn > 0.f) {
            bx /= bn;
            by /= bn;
            bz /= bn;
        } else {
            bx = 0.f;
            by = 0.f;
            bz = 1.f;
        }
        float rb = 0.f;
        for (int l = lane; l < seg_tile; l += 32) {
            const int64_t s = base + l;
            if (s < n && s32[s].b.w >= 0.f && s64[s].om < (double)b_min) {
                const float4 k = s32[s].k;
                const float dx = -k.x - bx, dy = -k.y - by, dz = -k.z - bz;
                rb = fmaxf(rb, sqrtf(dx * dx + dy * dy + dz * dz));
            }
        }
        for (int o = 16; o > 0; o >>= 1) rb = fmaxf(rb, __shfl_xor_sync(0xffffffffu, rb, o));
        // |Xdot| > 1 - b_min for these samples; margin for FP32 rounding
        const float cone = sqrtf(2.f * b_min / (1.f - b_min)) * 1.001f + 1e-5f;
        beam = make_float4(bx, by, bz, rb * 1.0001f + cone);
    }
    if (lane == 0) {
        SegCap c;
        c.c = make_float4(cx, cy, cz, r * 1.0001f + 1e-6f);
        c.r = make_float4(sqrtf(rho2) * 1.0001f + 1e-6f, om, 0.f, 0.f);
        c.b = beam;
        caps[warp] = c;
    }
}

void launch_pack(const double *samples, int64_t n, int64_t ld, double xo0, double xo1, double xo2, double GU,
                 double theta_pix, double near_k, int64_t n_pad, const uint32_t *perm, Seg32 *s32, Seg64 *s64,
                 Far2 *far, Mid2 *mid, Far64 *far64, DevStatus *st, cudaStream_t s)
{
    if (n_pad <= 0) return;
    int64_t blocks = (n_pad + 127) / 128;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_pack<<<(unsigned)blocks, 128, 0, s>>>(samples, n, ld, xo0, xo1, xo2, GU, theta_pix, near_k, n_pad, perm, s32,
                                             s64, far, mid, far64, st);
}

void launch_seg_caps(const Seg32 *s32, const Seg64 *s64, int64_t n, int64_t n_pad, int seg_tile, float b_min,
                     SegCap *caps, cudaStream_t s)
{
    const int64_t ntile = n_pad / seg_tile;
    if (ntile <= 0) return;
    const int64_t threads = ntile * 32;
    k_seg_caps<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(s32, s64, n, n_pad, seg_tile, b_min, caps);
}

}  // namespace isw
