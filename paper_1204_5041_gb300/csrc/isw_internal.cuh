// Internal declarations of the GB300 string-ISW library: device helpers shared by the
// kernels (IEEE-explicit FP64 arithmetic, the angle routines, the HEALPix RING geometry,
// mbarrier / bulk-copy wrappers) and the host-side context.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/isw.h"

namespace isw {

// ------------------------------------------------------------------------------------
// FP64 with explicit IEEE rounding (no contraction into FMA): the pixel directions and the
// light-cone solve are specified operation by operation so that they are reproducible.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }

// pi rounded to the nearest double
constexpr double kPi = 3.14159265358979323846264338327950288;

// sin and cos of x = f * pi/4, f in [0, 1]: Taylor series, ten terms after the first, each
// term obtained from the previous one by (term * x^2) / ((2k)(2k+1)) (sin) or
// / ((2k-1)(2k)) (cos), summed from the smallest term up.
__device__ __forceinline__ void sincos_octant(double f, double &s, double &c)
{
    const double quarter_pi = kPi * 0.25;
    const double x = dmul(f, quarter_pi);
    const double x2 = dmul(x, x);
    double st[11], ct[11];
    st[0] = x;
    ct[0] = 1.0;
#pragma unroll
    for (int k = 1; k <= 10; ++k) {
        st[k] = ddiv(dmul(st[k - 1], x2), (double)((2 * k) * (2 * k + 1)));
        ct[k] = ddiv(dmul(ct[k - 1], x2), (double)((2 * k - 1) * (2 * k)));
    }
    double S = 0.0, C = 0.0;
#pragma unroll
    for (int k = 10; k >= 0; --k) {
        if (k & 1) {
            S = dsub(S, st[k]);
            C = dsub(C, ct[k]);
        } else {
            S = dadd(S, st[k]);
            C = dadd(C, ct[k]);
        }
    }
    s = S;
    c = C;
}

// (sin, cos) of k*pi/4 + the folded octant angle
__device__ __forceinline__ void octant_unfold(int k, double sf, double cf, double &s, double &c)
{
    switch (k & 7) {
    case 0: s = sf;  c = cf;  break;
    case 1: s = cf;  c = sf;  break;
    case 2: s = cf;  c = -sf; break;
    case 3: s = sf;  c = -cf; break;
    case 4: s = -sf; c = -cf; break;
    case 5: s = -cf; c = -sf; break;
    case 6: s = -cf; c = sf;  break;
    default: s = -sf; c = cf; break;
    }
}

// sin and cos of pi*a/b, b > 0, with the angle reduced exactly in integers
__device__ __forceinline__ void sincospi_frac(int64_t a, int64_t b, double &s, double &c)
{
    const int64_t m = 8 * b;
    int64_t A = (4 * a) % m;
    if (A < 0) A += m;
    const int64_t k = A / b;
    const int64_t r = A - k * b;
    const double f = (k & 1) ? ddiv((double)(b - r), (double)b) : ddiv((double)r, (double)b);
    double sf, cf;
    sincos_octant(f, sf, cf);
    octant_unfold((int)k, sf, cf, s, c);
}

// sin and cos of 2*pi*w, reduced in turns (exact for |w| < 2^52)
__device__ __forceinline__ void sincos_turns(double w, double &s, double &c)
{
    double wr = dsub(w, floor(w));
    if (wr >= 1.0) wr = 0.0;
    const double e = dmul(wr, 8.0);
    const double kd = floor(e);
    const double r = dsub(e, kd);
    const int k = (int)kd;
    const double f = (k & 1) ? dsub(1.0, r) : r;
    double sf, cf;
    sincos_octant(f, sf, cf);
    octant_unfold(k, sf, cf, s, c);
}

__device__ __forceinline__ int64_t isqrt64(int64_t v)
{
    int64_t r = (int64_t)sqrt((double)v);
    while (r > 0 && r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

// Centre of RING pixel p at resolution N (the pixel-centre relations of Gorski et al. 2005,
// Sec. 4): rings i = 1..4N-1 from the north; the polar caps hold 4i pixels at
// z = +-(1 - i^2/(3N^2)), phi = (pi/(2i)) (j - 1/2); the belt holds 4N pixels at
// z = 4/3 - 2i/(3N), phi = (pi/(2N)) (j - s/2), s = 2 when i + N is odd, 1 when even.
__device__ __forceinline__ void pix2vec_ring(int64_t N, int64_t p, double &x, double &y, double &z)
{
    const int64_t npix = 12 * N * N;
    const int64_t ncap = 2 * N * (N - 1);
    int64_t i, j, a, b;
    double st;
    if (p < ncap) {
        i = (1 + isqrt64(1 + 2 * p)) / 2;
        j = p - 2 * i * (i - 1) + 1;
        z = ddiv((double)(3 * N * N - i * i), (double)(3 * N * N));
        st = ddiv(dmul((double)i, dsqrt((double)(6 * N * N - i * i))), (double)(3 * N * N));
        a = 2 * j - 1;
        b = 4 * i;
    } else if (p < npix - ncap) {
        const int64_t q = p - ncap;
        i = q / (4 * N) + N;
        j = q % (4 * N) + 1;
        const int64_t s = ((i + N) & 1) ? 2 : 1;
        z = ddiv((double)(4 * N - 2 * i), (double)(3 * N));
        st = ddiv(dsqrt((double)((2 * i - N) * (7 * N - 2 * i))), (double)(3 * N));
        a = 2 * j - s;
        b = 4 * N;
    } else {
        const int64_t q = npix - p;
        i = (1 + isqrt64(2 * q - 1)) / 2;
        j = 4 * i + 1 - (q - 2 * i * (i - 1));
        z = -ddiv((double)(3 * N * N - i * i), (double)(3 * N * N));
        st = ddiv(dmul((double)i, dsqrt((double)(6 * N * N - i * i))), (double)(3 * N * N));
        a = 2 * j - 1;
        b = 4 * i;
    }
    double sp, cp;
    sincospi_frac(a, b, sp, cp);
    x = dmul(st, cp);
    y = dmul(st, sp);
}

// atan2(y, x) in quarter turns, in [0, 4): a = min/max of |x|, |y|; a > tan(pi/8) is moved to
// (a - 1)/(a + 1) with pi/4 added back; one half-angle step atan(a) = 2 atan(a/(1 + sqrt(1 + a^2)))
// leaves |v| <= 0.2 for the Taylor series v (1 - v^2/3 + v^4/5 - ...), 13 terms summed from the
// smallest; the octant is unfolded exactly.  IEEE operations in a fixed order, so the result
// (and every HEALPix pixel decided from it) is reproducible operation by operation.
__device__ __forceinline__ double atan2_quarter(double y, double x)
{
    const double tan_pi_8 = 0.41421356237309504880;
    const double two_over_pi = 0.63661977236758134308;
    const double ax = fabs(x), ay = fabs(y);
    if (ax == 0.0 && ay == 0.0) return 0.0;
    const bool swap = ay > ax;
    double a = swap ? ddiv(ax, ay) : ddiv(ay, ax);
    double base = 0.0;
    if (a > tan_pi_8) {
        a = ddiv(dsub(a, 1.0), dadd(a, 1.0));
        base = 0.5;
    }
    const double v = ddiv(a, dadd(1.0, dsqrt(dadd(1.0, dmul(a, a)))));
    const double w = dmul(v, v);
    double s = 0.0;
    for (int k = 12; k >= 0; --k) {
        const double ck = ddiv(1.0, (double)(2 * k + 1));
        s = (k & 1) ? dsub(dmul(s, w), ck) : dadd(dmul(s, w), ck);
    }
    double q = dadd(base, dmul(dmul(2.0, dmul(v, s)), two_over_pi));
    if (swap) q = dsub(1.0, q);
    if (x < 0.0) q = dsub(2.0, q);
    if (y < 0.0) q = dsub(4.0, q);
    if (q >= 4.0) q = dsub(q, 4.0);
    return q;
}

// RING pixel of direction v (not necessarily unit, not zero), with z = cos(theta) and
// t = phi/(pi/2) in [0, 4).  The pixel boundaries of Gorski et al. (2005, Sec. 4) are two
// families of curves: in the equatorial zone the lines z = 2/3 - 4k/(3N) +- 8 phi/(3 pi), in
// the polar caps z = 1 - (k/N)^2 (pi/(2 phi_t))^2 / 3 and z = 1 - (k/N)^2 (pi/(2 phi_t - pi))^2 / 3
// with phi_t = phi mod pi/2.  Solved for k at the direction, each family gives how many of its
// curves lie below it: jp = floor(N (1/2 + t - 3z/4)), jm = floor(N (1/2 + t + 3z/4)) in the
// belt, jp = floor(t_p h), jm = floor((1 - t_p) h) with t_p = frac(t), h = N sqrt(3 (1 - |z|))
// in a cap.  The ring is then N + 1 + jp - jm (belt) or jp + jm + 1 (counted from the nearer
// pole), and the position in it (jp + jm - N + kshift + 1)/2 or floor(t * ring).
__device__ __forceinline__ int64_t vec2pix_ring(int64_t N, double vx, double vy, double vz)
{
    const double r = dsqrt(dadd(dadd(dmul(vx, vx), dmul(vy, vy)), dmul(vz, vz)));
    const double z = ddiv(vz, r);
    const double za = fabs(z);
    const double t = atan2_quarter(vy, vx);
    const double Nd = (double)N;
    if (za <= 2.0 / 3.0) {
        const double t1 = dmul(Nd, dadd(0.5, t));
        const double t2 = dmul(Nd, dmul(z, 0.75));
        const int64_t jp = (int64_t)floor(dsub(t1, t2));
        const int64_t jm = (int64_t)floor(dadd(t1, t2));
        const int64_t ir = N + 1 + jp - jm;
        const int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - N + kshift + 1) / 2;
        ip = ((ip % (4 * N)) + 4 * N) % (4 * N);
        return 2 * N * (N - 1) + (ir - 1) * 4 * N + ip;
    }
    const double tp = dsub(t, floor(t));
    const double h = dmul(Nd, dsqrt(dmul(3.0, dsub(1.0, za))));
    const int64_t jp = (int64_t)floor(dmul(tp, h));
    const int64_t jm = (int64_t)floor(dmul(dsub(1.0, tp), h));
    const int64_t ir = jp + jm + 1;
    int64_t ip = (int64_t)floor(dmul(t, (double)ir));
    ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
    if (z > 0.0) return 2 * ir * (ir - 1) + ip;
    return 12 * N * N - 2 * ir * (ir + 1) + ip;
}

// RING index of the pixel at (ix, iy) of base face f (0..11).  The twelve base pixels of
// Gorski et al. (2005, Sec. 4) are rhombi in three rings of four: face f is centred on ring
// jr(f) * N, jr = 2 (north faces 0-3), 3 (equatorial faces 4-7), 4 (south faces 8-11), with its
// corner at longitude jp(f) * pi/4; inside a face, ring number falls by one per step of ix + iy
// and the position in the ring rises by one per two steps of ix - iy (plus the half-pixel
// shift kshift of alternate belt rings).  Used only to order pixels in compact 2-D tiles; any
// bijection gives the same map.
__device__ __forceinline__ int64_t xyf2ring(int64_t N, int f, int64_t ix, int64_t iy)
{
    const int jr_face = (f < 4) ? 2 : (f < 8 ? 3 : 4);
    const int jp_face = (f < 4) ? 2 * f + 1 : (f < 8 ? 2 * (f - 4) : 2 * (f - 8) + 1);
    const int64_t jr = (int64_t)jr_face * N - ix - iy - 1;
    const int64_t npix = 12 * N * N;
    const int64_t ncap = 2 * N * (N - 1);
    int64_t nr, before, kshift;
    if (jr < N) {
        nr = jr;
        before = 2 * nr * (nr - 1);
        kshift = 0;
    } else if (jr > 3 * N) {
        nr = 4 * N - jr;
        before = npix - 2 * nr * (nr + 1);
        kshift = 0;
    } else {
        nr = N;
        before = ncap + (jr - N) * 4 * N;
        kshift = (jr - N) & 1;
    }
    // floor division: the numerator is negative on face 4 (corner at longitude 0), so shift it
    // by 8 nr (even) before dividing
    int64_t jp = ((int64_t)jp_face * nr + ix - iy + 1 + kshift + 8 * nr) / 2 - 4 * nr;
    if (jp > 4 * nr) jp -= 4 * nr;
    if (jp < 1) jp += 4 * nr;
    return before + jp - 1;
}

// ------------------------------------------------------------------------------------
// mbarrier + 1-D bulk copy (TMA engine) wrappers.  Waits are bounded: a wait that runs
// out returns false and the caller reports ISW_ETIMEOUT instead of spinning forever.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Limits of the bounded waits, in try_wait polls (each try_wait itself suspends the thread for
// a hardware-defined interval while the phase is incomplete).  A consumer wait (a stage of
// records or pixels the CTA is about to read) gives up after kWaitPolls by default
// (ISW_PARAM_WAIT_POLLS overrides it); after a consumer wait ran out, the CTA waits for the
// bulk copies it still has in flight with the separate, much longer kDrainPolls, so that it
// does not exit while a copy into its shared memory is outstanding.
constexpr uint32_t kWaitPolls = 1u << 22;
constexpr uint32_t kDrainPolls = 1u << 26;

// Bounded wait on phase `parity`: at most `polls` polls, then false (polls = 0 gives up at once).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t polls)
{
    for (uint32_t it = 0; it < polls; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    return false;
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completion signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Device-side error reporting: status bits OR-ed into a word the host reads on demand.
enum : uint32_t {
    kStatDomain = 1u << 0,   // a segment with 1 - Xdot^2 <= 0 or a non-finite weight
    kStatTimeout = 1u << 1,  // a bounded wait ran out
    kStatNoConv = 1u << 2,   // light-cone Newton iteration cap reached
    kStatBadIndex = 1u << 3, // a loop id or pixel index out of range
    kStatDrain = 1u << 4,    // after a time-out, the wait for a CTA's copies in flight ran out too
};

struct DevStatus {
    uint32_t bits;
    uint32_t pad;
    unsigned long long zero_pairs;   // D = 0 pairs (zero contribution)
    unsigned long long domain_segs;  // skipped segments
    unsigned long long near_pairs;   // pairs evaluated in FP64 by the FP32 path
};

// ------------------------------------------------------------------------------------
// Packed segment records.
// FP32 record (80 B): Xhat hi (3), c | Xhat lo (3), rho^2 | Xdot (3), e | X' (3), f |
// Xdot/|Xdot| (3), 1 - |Xdot|, with c = -4 GU eps dsigma / |X|, rho = near-field chord
// radius, e = 1 + Xdot.Xhat, f = X'.Xhat (so that Xdot.d = B - e and X'.d = A - f for
// d = n - Xhat); the last four give B = (1 - |Xdot|) + |Xdot| |n + Xdot/|Xdot||^2 / 2
// without cancellation when n approaches -Xdot/|Xdot|.
// FP64 record (128 B): Xhat hi (3), Xhat lo (3), Xdot (3), X' (3), c, 1 - |Xdot|, |X - x_obs|,
// cu = c / dsigma = -4 GU eps / |X| (the weight per unit dsigma, for the dsigma gradient).
// Segment tile cap (48 B): centre (3), chord radius, max rho, min (1 - |Xdot|), beam cap (4).
// Pixel tile cap (16 B): centre (3), chord radius.
// ------------------------------------------------------------------------------------
struct __align__(16) Seg32 {
    float4 a, b, d, e, k;
};
// Far-field constants of one sample, with sigma = sign(c), s = sqrt(|c|/2):
//   a = (-sigma Xhat, sigma), b = (Xdot, -s e/2), c = (s X', -s f/2), d = (s, K),
//   K = (|c|/2) (f^2 - e^2)/4, so that for |d| >= d_far the pair term is
//   t = [(s B - s e/2)^2 - (s A - s f/2)^2 + K] / [B sigma (1 - n.Xhat)]   (completed squares of
//   c/2 [B (B - e) - A (A - f)] / [B (1 - n.Xhat)]).
// The far pass stores them for samples 2i and 2i+1 interleaved (112 B per pair): the 14
// constants (a.xyzw, b.xyzw, c.xyzw, d.x, d.y) in that order, each as a float pair (sample 2i,
// sample 2i+1), so that one packed f32x2 instruction serves both samples.
struct __align__(16) Far2 {
    float4 v[7];
};
constexpr int kFarConsts = 14;
// Mid-range constants of one sample for the packed near-field loop, each value stored twice so
// that one 8-byte load gives the (v, v) operand of an f32x2 instruction over two pixels:
// Xhat hi (3), Xhat lo (3), Xdot (3), -X' (3), c, e = 1 + Xdot.Xhat, f = X'.Xhat, -f.
struct __align__(16) Mid2 {
    float4 v[8];
};
constexpr int kMidConsts = 16;

// Packed FP32 pairs (f32x2, sm_100 and later): two IEEE single operations per instruction,
// round to nearest; a 64-bit register holds (lo, hi).
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

struct __align__(16) Seg64 {
    double xh[3], xl[3], xd[3], xp[3], c, om, X, cu;   // X = |X_s - x_obs|
};
// Far-field constants of one sample for the FP64 kernel, the completed-square form of the FP32
// far pass in FP64 (sigma = sign(c), s = sqrt(|c|/2), e = 1 + Xdot.Xhat, f = X'.Xhat):
// mxh = -sigma Xhat, sg = sigma, xd = Xdot, sx = s, be = -s e/2, xp = s X', af = -s f/2,
// K = (|c|/2) (e^2 - f^2)/4, so that for |d| >= d_far the pair term is
// t = [(s B - s e/2)^2 - (s A - s f/2)^2 - K] / [B sigma (1 - n.Xhat)]
//   = (c/2) [B (B - e) - A (A - f)] / [B (1 - n.Xhat)]  (d.d = 2 (1 - n.Xhat), Xdot.d = B - e,
// X'.d = A - f).  A zero-weight sample has s = 0 and K = 0: its terms are exactly zero.
struct __align__(16) Far64 {
    double mxh[3], sg, xd[3], sx, be, xp[3], af, K;
};
// Pixel records of the adjoint: FP32 (n hi, g | n lo, 0) and FP64 (n, g); padding slots
// hold n = 0, g = 0 so that every pair stays finite and contributes nothing.
struct __align__(16) Pix32 {
    float4 a, b;
};
struct __align__(16) Pix64 {
    double n[3], g;
};
// Far-field pixel records of the FP32 adjoint, one per pixel pair (pixels 2i, 2i+1 of the tile
// order): a = (nx, nx', ny, ny'), b = (nz, nz', g, g') with the primed entries those of the second
// pixel, so that each float pair is one packed f32x2 operand over the two pixels.
struct __align__(16) PixF2 {
    float4 a, b;
};
struct __align__(16) SegCap {
    float4 c;   // centre xyz, chord radius
    float4 r;   // rho_max, om_min, -, -
    float4 b;   // beam cap of the samples with 1 - |Xdot| < b_min: centre of -Xdot/|Xdot| (xyz) and
                // chord radius enlarged by the B < b_min cone; radius < 0 when there is no such sample
};

// Default tunables of the FP32 map (isw_map and the allocation-free entry point use the same):
// near-field radius in units of max(pixel size, segment angle) (2: four pixel radii; 4 measured
// 318.5 against 312.8 ms per bench step with the same largest error, 7.3e-7 of the rms on the
// pixels nearest the strings), the 1 + n.Xdot below which a pair goes to FP64, and the tile-cap
// gap beyond which the far-field form is used.
constexpr double kNearK = 2.0;
constexpr double kBMin = 0.01;
constexpr double kDFar = 0.25;

struct Tunables {
    int threads;    // threads per CTA (FP32 map)
    int ppt;        // pixels per thread
    int seg_tile;   // segments per shared-memory tile
    int split;      // segment chunks (0 = automatic)
};

}  // namespace isw

// ------------------------------------------------------------------------------------
// Host-side context
// ------------------------------------------------------------------------------------
// workspace slots of a context (device buffers grown on demand)
constexpr int kMaxWorkspaces = 32;

struct isw_ctx {
    int device;
    int num_sms;
    char last_error[512];
    isw::DevStatus *d_status;     // device status word + counters
    // workspace buffers (grown on demand, never shrunk)
    void *ws[kMaxWorkspaces];
    size_t ws_size[kMaxWorkspaces];
    // tunables
    double near_k;      // near-field radius in units of max(pixel size, segment angle)
    double b_min;       // 1 + n.Xdot below this goes to FP64
    double d_far;       // segment tiles this chord away from the pixel tile use the far-field form
    int split_override; // segment chunks for the forward maps (0 = automatic)
    int tile_override;  // FP32 kernel variant index (-1 = automatic)
    uint32_t wait_polls; // limit of the kernels' consumer waits (ISW_PARAM_WAIT_POLLS)
    // pair-kernel timing (ISW_PARAM_TIMING)
    int timing;
    int n_timed;
    int64_t n_pair;     // pair-kernel launches since the last reset
    int64_t n_launch;   // all kernel launches since the last reset
    cudaEvent_t *ev;    // 2 * kMaxTimed events, created on first use
    // FP32 variant picked by the autotuner for (tuned_nside, tuned_n); used when no override
    int auto_variant;
    int last_variant;   // FP32 variant used by the last FP32 map
    int64_t tuned_nside, tuned_n;
    // batched path: shell metadata last uploaded, and one captured graph
    uint64_t meta_hash;
    int64_t meta_nshell;
    int capturing;
    cudaStream_t cap_stream;
    uint64_t graph_key;
    cudaGraph_t graph;
    cudaGraphExec_t graph_exec;
    int64_t graph_kernels, graph_pairs;  // kernel / pair-kernel launches inside the captured graph
};
constexpr int kMaxTimed = 4096;
