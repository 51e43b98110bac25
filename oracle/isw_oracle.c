/*
 * Oracle for the all-sky string ISW map -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of what the GPU library computes,
 * written from the paper (Ringeval & Bouchet, "All sky CMB map from cosmic strings
 * integrated Sachs-Wolfe effect", arXiv:1204.5041) and from the published HEALPix
 * geometry (Gorski et al. 2005).  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product path never does.  It shares no code,
 * header or constant with the CUDA library.
 *
 * Built with -O2 -ffp-contract=off: every expression below is evaluated as written,
 * with IEEE double rounding of each operation and no fused multiply-add.
 *
 * Contents
 *   1. sincos of an angle given as an exact fraction of a turn (own series, no libm trig)
 *   2. HEALPix RING pix2vec (Sec. II.D; Gorski et al. 2005 ring geometry)
 *   3. retarded-time (past light cone) solve, LINEAR and BURDEN modes (Eq. 1: X cap x_gamma)
 *   4. per-segment weight eps*dsigma (text after Eq. 1) and the pair term of Eq. (1)-(2)
 *   5. the discrete line-of-sight sum per pixel, Neumaier-compensated, input order
 *   6. the analytic adjoint of the sum with respect to X and Xdot (optionally X', dsigma)
 *   7. the adjoint of the light-cone solve (implicit-function theorem on the crossing
 *      condition): gradients of LINEAR box-time nodes and of BURDEN loop parameters
 *   8. stacking with HEALPix cones (Sec. III.B): own atan2, RING vec2pix, box placement,
 *      cone cut
 *   9. patch maps: full sky on a gnomonic patch and the flat-sky approximation (Sec. II.A,
 *      Fig. 3)
 *  10. angular power spectrum of a RING map (Fig. 4): ring Fourier sums, normalised
 *      Legendre recursion with exponent tracking, C_l
 *
 * Pins (tests/test_oracle_*.py) tie each part to something other than itself; see the
 * header comment of each section for what pins it.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>

/* pi rounded to the nearest double */
static const double PI = 3.14159265358979323846264338327950288;

#define OR_OK 0
#define OR_EINVAL 1
#define OR_EDOMAIN 3
#define OR_ENOCONV 4

/* ------------------------------------------------------------------------------------
 * 1. sin/cos on [0, pi/4] by the Taylor series, and exact octant reduction.
 *
 * For x = f*pi/4 with f in [0, 1]: x2 = x*x, term_0 = x (sin) or 1 (cos), each next
 * term = (previous * x2) / (2k(2k+1)) for sin and / ((2k-1)2k) for cos, k = 1..10, and
 * the alternating series is summed from the smallest term (k = 10) down to k = 0.
 * The angle is reduced exactly: to octant k and a fraction f of it, folding odd octants
 * so the series always sees x in [0, pi/4].  Pinned against mpmath (test_oracle_sincos).
 * ---------------------------------------------------------------------------------- */
#define NTERMS 10

static void sincos_octant(double f, double *s, double *c)
{
    const double quarter_pi = PI * 0.25;
    double x = f * quarter_pi;
    double x2 = x * x;
    double st[NTERMS + 1], ct[NTERMS + 1];
    st[0] = x;
    ct[0] = 1.0;
    for (int k = 1; k <= NTERMS; ++k) {
        st[k] = (st[k - 1] * x2) / (double)((2 * k) * (2 * k + 1));
        ct[k] = (ct[k - 1] * x2) / (double)((2 * k - 1) * (2 * k));
    }
    double S = 0.0, C = 0.0;
    for (int k = NTERMS; k >= 0; --k) {
        if (k & 1) {
            S = S - st[k];
            C = C - ct[k];
        } else {
            S = S + st[k];
            C = C + ct[k];
        }
    }
    *s = S;
    *c = C;
}

/* Map (sin, cos) of the folded octant angle back to the full angle (k*pi/4 + ...). */
static void octant_unfold(int k, double sf, double cf, double *s, double *c)
{
    switch (k & 7) {
    case 0: *s = sf;  *c = cf;  break;
    case 1: *s = cf;  *c = sf;  break;
    case 2: *s = cf;  *c = -sf; break;
    case 3: *s = sf;  *c = -cf; break;
    case 4: *s = -sf; *c = -cf; break;
    case 5: *s = -cf; *c = -sf; break;
    case 6: *s = -cf; *c = sf;  break;
    default: *s = -sf; *c = cf; break;
    }
}

/* sin and cos of pi*a/b for integers a, b > 0 (exact integer reduction). */
void or_sincospi_frac(int64_t a, int64_t b, double *s, double *c)
{
    int64_t m = 8 * b;
    int64_t A = (4 * a) % m;
    if (A < 0) A += m;
    int64_t k = A / b;
    int64_t r = A - k * b;
    double f = (k & 1) ? (double)(b - r) / (double)b : (double)r / (double)b;
    double sf, cf;
    sincos_octant(f, &sf, &cf);
    octant_unfold((int)k, sf, cf, s, c);
}

/* sin and cos of 2*pi*w for a double w (reduction in turns: exact for |w| < 2^52). */
void or_sincos_turns(double w, double *s, double *c)
{
    double wr = w - floor(w);
    if (wr >= 1.0) wr = 0.0;
    double e = wr * 8.0;
    double kd = floor(e);
    double r = e - kd;
    int k = (int)kd;
    double f = (k & 1) ? 1.0 - r : r;
    double sf, cf;
    sincos_octant(f, &sf, &cf);
    octant_unfold(k, sf, cf, s, c);
}

/* ------------------------------------------------------------------------------------
 * 2. HEALPix RING pixel centres (Sec. II.D of the paper; the pixel-centre relations of
 * Gorski et al. 2005, Sec. 4).
 *
 * Rings are numbered 1..4N-1 from the north pole.  North polar cap: ring i < N holds 4i
 * pixels, z = 1 - i^2/(3N^2), phi = (pi/(2i)) (j - 1/2).  Equatorial belt N <= i <= 3N: 4N
 * pixels, z = 4/3 - 2i/(3N), phi = (pi/(2N)) (j - s/2) with s = 2 when i + N is odd and
 * s = 1 when it is even (rings alternate between a pixel centred on phi = 0 and a half-pixel
 * offset; the first pixel of a ring is the one at or just after phi = 0).  South cap
 * mirrors the north.  z and sin(theta) are formed from exact integers with one division:
 *   caps:    z = +-(3N^2 - i^2) / (3N^2),  sin(theta) = i * sqrt(6N^2 - i^2) / (3N^2)
 *   belt:    z = (4N - 2i) / (3N),         sin(theta) = sqrt((2i - N)(7N - 2i)) / (3N)
 * Pinned by brute-force ring enumeration, exact rational z, the equal-area identity and
 * reflection / rotation symmetries (test_oracle_pix2vec).
 * ---------------------------------------------------------------------------------- */
static int64_t isqrt64(int64_t v)
{
    int64_t r = (int64_t)sqrt((double)v);
    while (r > 0 && r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return r;
}

int or_pix2vec_ring_one(int64_t nside, int64_t p, int64_t *ring, int64_t *jpix, double vec[3])
{
    const int64_t N = nside;
    const int64_t npix = 12 * N * N;
    const int64_t ncap = 2 * N * (N - 1);
    if (N < 1 || p < 0 || p >= npix) return OR_EINVAL;
    int64_t i, j, a, b;
    double z, st;
    if (p < ncap) {
        i = (1 + isqrt64(1 + 2 * p)) / 2;
        j = p - 2 * i * (i - 1) + 1;
        z = (double)(3 * N * N - i * i) / (double)(3 * N * N);
        st = ((double)i * sqrt((double)(6 * N * N - i * i))) / (double)(3 * N * N);
        a = 2 * j - 1;
        b = 4 * i;
        *ring = i;
    } else if (p < npix - ncap) {
        int64_t q = p - ncap;
        i = q / (4 * N) + N;
        j = q % (4 * N) + 1;
        int64_t s = ((i + N) & 1) ? 2 : 1;
        z = (double)(4 * N - 2 * i) / (double)(3 * N);
        st = sqrt((double)((2 * i - N) * (7 * N - 2 * i))) / (double)(3 * N);
        a = 2 * j - s;
        b = 4 * N;
        *ring = i;
    } else {
        int64_t q = npix - p;
        i = (1 + isqrt64(2 * q - 1)) / 2;
        j = 4 * i + 1 - (q - 2 * i * (i - 1));
        z = -((double)(3 * N * N - i * i) / (double)(3 * N * N));
        st = ((double)i * sqrt((double)(6 * N * N - i * i))) / (double)(3 * N * N);
        a = 2 * j - 1;
        b = 4 * i;
        *ring = 4 * N - i;
    }
    *jpix = j;
    double sp, cp;
    or_sincospi_frac(a, b, &sp, &cp);
    vec[0] = st * cp;
    vec[1] = st * sp;
    vec[2] = z;
    return OR_OK;
}

/* n pixels, ring indices in pix (or pix0 + k when pix == NULL); out double[3][ld]. */
int or_pix2vec_ring(int64_t nside, int64_t pix0, int64_t n, const int64_t *pix,
                    double *vec, int64_t ld, int64_t *ring, int64_t *jpix)
{
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = pix ? pix[k] : pix0 + k;
        int64_t ri, ji;
        double v[3];
        int st = or_pix2vec_ring_one(nside, p, &ri, &ji, v);
        if (st) return st;
        vec[k] = v[0];
        vec[ld + k] = v[1];
        vec[2 * ld + k] = v[2];
        if (ring) ring[k] = ri;
        if (jpix) jpix[k] = ji;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------
 * 3. Past-light-cone solve: the integral of Eq. (1) runs over the string points X that
 * intercept the photon path x_gamma, i.e. |X(tau) - x_obs| = t_obs - tau (flat conformal
 * coordinates, c = 1).  The paper records X', Xdot at the crossing (Sec. II.B).
 *
 * LINEAR: straight worldline X + Xdot*Delta from box time t_box.  With r0 = X - x_obs,
 * T = t_obs - t_box: (v^2 - 1) D^2 + 2 (r0.Xdot + T) D + (|r0|^2 - T^2) = 0; the past root
 * is D = -c / (b + sqrt(b^2 + (1 - v^2) c)) with b = r0.Xdot + T, c = (|r0| - T)(|r0| + T).
 * Xdot, X', dsigma are carried unchanged.  Pinned by closed forms (static node; radial
 * motion) and the light-cone residual (test_oracle_lightcone).
 *
 * BURDEN: analytic loop X(s,t) = c + R (a(s - (t - t0)) + b(s + (t - t0)))/2 with
 * a(u) = L/(2 pi m) (sin 2 pi m u/L, -cos 2 pi m u/L, 0) and
 * b(v) = L/(2 pi n) (sin 2 pi n v/L, -cos(psi) cos 2 pi n v/L, -sin(psi) cos 2 pi n v/L).
 * f(t) = |X(s,t) - x_obs| - (t_obs - t) is increasing; safeguarded Newton on the bracket
 * [t_obs - d - L/2, t_obs - d + L/2] (d = |c - x_obs|): a bisection replaces the Newton step
 * when it leaves the bracket or is longer than half the step two iterations back; stop when
 * |f| <= tol.
 * ---------------------------------------------------------------------------------- */
static void burden_eval(const double *P, int64_t ldp, int64_t id, double sigma, double t,
                        double X[3], double Xd[3], double Xp[3])
{
    const double two_pi = 2.0 * PI;
    double c[3], R[9];
    for (int k = 0; k < 3; ++k) c[k] = P[k * ldp + id];
    for (int k = 0; k < 9; ++k) R[k] = P[(3 + k) * ldp + id];
    double L = P[12 * ldp + id], m = P[13 * ldp + id], n = P[14 * ldp + id];
    double psi = P[15 * ldp + id], t0 = P[16 * ldp + id];
    double dt = t - t0;
    double u = sigma - dt, v = sigma + dt;
    double sa, ca, sb, cb, sp, cp;
    or_sincos_turns((m * u) / L, &sa, &ca);
    or_sincos_turns((n * v) / L, &sb, &cb);
    or_sincos_turns(psi / two_pi, &sp, &cp);
    double ra = L / (two_pi * m), rb = L / (two_pi * n);
    double a[3] = {ra * sa, -(ra * ca), 0.0};
    double b[3] = {rb * sb, -(rb * (cp * cb)), -(rb * (sp * cb))};
    double ap[3] = {ca, sa, 0.0};
    double bp[3] = {cb, cp * sb, sp * sb};
    double h[3], hd[3], hp[3];
    for (int k = 0; k < 3; ++k) {
        h[k] = 0.5 * (a[k] + b[k]);
        hd[k] = 0.5 * (bp[k] - ap[k]);
        hp[k] = 0.5 * (ap[k] + bp[k]);
    }
    for (int k = 0; k < 3; ++k) {
        X[k] = c[k] + ((R[3 * k] * h[0] + R[3 * k + 1] * h[1]) + R[3 * k + 2] * h[2]);
        Xd[k] = (R[3 * k] * hd[0] + R[3 * k + 1] * hd[1]) + R[3 * k + 2] * hd[2];
        Xp[k] = (R[3 * k] * hp[0] + R[3 * k + 1] * hp[1]) + R[3 * k + 2] * hp[2];
    }
}

/* Burden worldsheet at (sigma, t) for loop id (exposed for tests). */
void or_burden_eval(const double *P, int64_t ldp, int64_t id, double sigma, double t,
                    double *out9)
{
    burden_eval(P, ldp, id, sigma, t, out9, out9 + 3, out9 + 6);
}

int or_lightcone(int mode, const double *nodes, int64_t n, int64_t ld,
                 const double *P, int64_t nloops, int64_t ldp, double t_box,
                 const double x_obs[3], double t_obs, double tol, int max_iter,
                 double *out, double *tau, int32_t *status)
{
    int worst = OR_OK;
    for (int64_t s = 0; s < n; ++s) {
        int st = OR_OK;
        double X[3], Xd[3], Xp[3], t = t_obs;
        if (mode == 0) {
            double r0[3];
            for (int k = 0; k < 3; ++k) {
                X[k] = nodes[k * ld + s];
                Xd[k] = nodes[(3 + k) * ld + s];
                Xp[k] = nodes[(6 + k) * ld + s];
                r0[k] = X[k] - x_obs[k];
            }
            double R = sqrt((r0[0] * r0[0] + r0[1] * r0[1]) + r0[2] * r0[2]);
            double T = t_obs - t_box;
            double v2 = (Xd[0] * Xd[0] + Xd[1] * Xd[1]) + Xd[2] * Xd[2];
            double om = 1.0 - v2;
            if (!(om > 0.0) || !(R == R)) {
                st = OR_EDOMAIN;
                t = t_box;
            } else {
                double c = (R - T) * (R + T);
                double bh = ((r0[0] * Xd[0] + r0[1] * Xd[1]) + r0[2] * Xd[2]) + T;
                double disc = bh * bh + om * c;
                if (disc < 0.0) disc = 0.0;
                double D = -c / (bh + sqrt(disc));
                t = t_box + D;
                for (int k = 0; k < 3; ++k) X[k] = X[k] + Xd[k] * D;
            }
        } else {
            int64_t id = (int64_t)nodes[s];
            double sigma = nodes[ld + s];
            if (id < 0 || id >= nloops) {
                st = OR_EINVAL;
                for (int k = 0; k < 3; ++k) X[k] = Xd[k] = Xp[k] = 0.0;
            } else {
                double cx = P[0 * ldp + id] - x_obs[0];
                double cy = P[1 * ldp + id] - x_obs[1];
                double cz = P[2 * ldp + id] - x_obs[2];
                double d = sqrt((cx * cx + cy * cy) + cz * cz);
                double halfL = 0.5 * P[12 * ldp + id];
                double lo = (t_obs - d) - halfL, hi = (t_obs - d) + halfL;
                double step1 = hi - lo, step2 = hi - lo;   /* last two step lengths */
                t = t_obs - d;
                st = OR_ENOCONV;
                for (int it = 0; it < max_iter; ++it) {
                    burden_eval(P, ldp, id, sigma, t, X, Xd, Xp);
                    double r[3] = {X[0] - x_obs[0], X[1] - x_obs[1], X[2] - x_obs[2]};
                    double rn = sqrt((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]);
                    double f = rn - (t_obs - t);
                    if (fabs(f) <= tol) {
                        st = OR_OK;
                        break;
                    }
                    if (!(rn > 0.0)) {
                        st = OR_EDOMAIN;
                        break;
                    }
                    if (f < 0.0) lo = t; else hi = t;
                    double fp = 1.0 + ((r[0] * Xd[0] + r[1] * Xd[1]) + r[2] * Xd[2]) / rn;
                    double tn = t - f / fp;
                    /* bisect when Newton leaves the bracket or does not at least halve the step
                       taken two iterations earlier (stops two-cycles between the bracket ends) */
                    if (!(tn > lo && tn < hi) || fabs(tn - t) > 0.5 * step2) tn = 0.5 * (lo + hi);
                    step2 = step1;
                    step1 = fabs(tn - t);
                    if (it + 1 < max_iter) t = tn;
                }
            }
        }
        for (int k = 0; k < 3; ++k) {
            out[k * ld + s] = X[k];
            out[(3 + k) * ld + s] = Xd[k];
            out[(6 + k) * ld + s] = Xp[k];
        }
        out[9 * ld + s] = nodes[9 * ld + s];
        if (tau) tau[s] = t;
        if (status) status[s] = st;
        if (st > worst) worst = st;
    }
    return worst;
}

/* ------------------------------------------------------------------------------------
 * 4. The pair term of Eq. (1)-(2).
 *
 *   Theta(n) = -4 GU sum_s u.D / D^2 * eps_s dsigma_s,  D = X n - X_s,  X = |X_s - x_obs|,
 *   u = Xdot - (n.X') X' / (1 + n.Xdot),  eps^2 = X'^2 / (1 - Xdot^2).
 *
 * D is formed as X * (n - Xhat) with the unit vector Xhat = (X_s - x_obs)/X carried in
 * double-double (hi + lo): near a string n - Xhat cancels, and an FP64-rounded Xhat would
 * leave D with a relative error of ~1e-16 / |n - Xhat|.  D = 0 exactly gives a zero term
 * (counted); a segment with 1 - Xdot^2 <= 0 or a non-finite weight contributes nothing
 * (counted).  Pinned by an independent mpmath evaluation of Eq. (1)-(2), the Kaiser-
 * Stebbins step of a straight moving string and brute-force quadrature (tests).
 * ---------------------------------------------------------------------------------- */

/* Error-free transformations (Knuth two-sum, Dekker split product: no FMA needed). */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bb = x - a;
    *e = (a - (x - bb)) + (b - bb);
    *s = x;
}

static void split(double a, double *hi, double *lo)
{
    const double factor = 134217729.0; /* 2^27 + 1 */
    double t = factor * a;
    *hi = t - (t - a);
    *lo = a - *hi;
}

static void two_prod(double a, double b, double *p, double *e)
{
    double ah, al, bh, bl;
    double x = a * b;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    *e = ((ah * bh - x) + ah * bl + al * bh) + al * bl;
    *p = x;
}

/* Unit vector r/|r| with each component as hi + lo (relative accuracy ~1e-30). */
static void unit_dd(const double r[3], double hi[3], double lo[3], double *norm)
{
    /* |r|^2 in double-double */
    double sh = 0.0, sl = 0.0;
    for (int k = 0; k < 3; ++k) {
        double p, pe, s, se;
        two_prod(r[k], r[k], &p, &pe);
        two_sum(sh, p, &s, &se);
        sl = sl + (se + pe);
        two_sum(s, sl, &sh, &sl);
    }
    /* |r| = sqrt in double-double: one Newton correction of the double root */
    double q = sqrt(sh);
    double qq, qqe;
    two_prod(q, q, &qq, &qqe);
    double ql = (((sh - qq) - qqe) + sl) / (2.0 * q);
    double nh, nl;
    two_sum(q, ql, &nh, &nl);
    *norm = nh;
    /* r_k / (nh + nl) in double-double: quotient, remainder, correction */
    for (int k = 0; k < 3; ++k) {
        double q1 = r[k] / nh;
        double p, pe;
        two_prod(q1, nh, &p, &pe);
        double rem = ((r[k] - p) - pe) - q1 * nl;
        double q2 = rem / nh;
        two_sum(q1, q2, &hi[k], &lo[k]);
    }
}

typedef struct {
    double xh[3], xl[3]; /* Xhat as double-double */
    double X;            /* |X_s - x_obs| */
    double xd[3], xp[3]; /* Xdot, X' */
    double kappa;        /* -4 GU eps dsigma */
    double kd;           /* -4 GU eps: kappa per unit dsigma */
    double om;           /* 1 - Xdot^2 */
    double xp2;          /* X'^2 */
    int ok;
} seg_t;

static void seg_prepare(const double *samples, int64_t ld, int64_t s, const double x_obs[3],
                        double GU, seg_t *g)
{
    double r[3];
    for (int k = 0; k < 3; ++k) {
        r[k] = samples[k * ld + s] - x_obs[k];
        g->xd[k] = samples[(3 + k) * ld + s];
        g->xp[k] = samples[(6 + k) * ld + s];
    }
    double dsig = samples[9 * ld + s];
    unit_dd(r, g->xh, g->xl, &g->X);
    double v2 = (g->xd[0] * g->xd[0] + g->xd[1] * g->xd[1]) + g->xd[2] * g->xd[2];
    g->om = 1.0 - v2;
    g->xp2 = (g->xp[0] * g->xp[0] + g->xp[1] * g->xp[1]) + g->xp[2] * g->xp[2];
    double eps = sqrt(g->xp2 / g->om);
    g->kappa = -4.0 * GU * (eps * dsig);
    g->kd = -4.0 * GU * eps;
    g->ok = (g->om > 0.0) && (g->X > 0.0) && isfinite(g->kappa);
}

/* u.D / D^2 pieces for one (pixel, segment) pair; returns 0 when D = 0 exactly. */
typedef struct {
    double D[3], D2, A, B, u[3], uD, XpD;
} pair_t;

static int pair_eval(const double n[3], const seg_t *g, pair_t *q)
{
    for (int k = 0; k < 3; ++k) q->D[k] = g->X * ((n[k] - g->xh[k]) - g->xl[k]);
    q->D2 = (q->D[0] * q->D[0] + q->D[1] * q->D[1]) + q->D[2] * q->D[2];
    if (q->D2 == 0.0) return 0;
    q->A = (n[0] * g->xp[0] + n[1] * g->xp[1]) + n[2] * g->xp[2];
    q->B = 1.0 + ((n[0] * g->xd[0] + n[1] * g->xd[1]) + n[2] * g->xd[2]);
    for (int k = 0; k < 3; ++k) q->u[k] = g->xd[k] - (q->A * g->xp[k]) / q->B;
    q->uD = (q->u[0] * q->D[0] + q->u[1] * q->D[1]) + q->u[2] * q->D[2];
    q->XpD = (g->xp[0] * q->D[0] + g->xp[1] * q->D[1]) + g->xp[2] * q->D[2];
    return 1;
}

/* One pair term (for pins): n[3], one sample (10 doubles, row stride 1). */
double or_pair_term(const double n[3], const double sample10[10], const double x_obs[3],
                    double GU)
{
    seg_t g;
    pair_t q;
    seg_prepare(sample10, 1, 0, x_obs, GU, &g);
    if (!g.ok) return 0.0;
    if (!pair_eval(n, &g, &q)) return 0.0;
    return g.kappa * (q.uD / q.D2);
}

/* ------------------------------------------------------------------------------------
 * 5. The map: for every requested pixel, the sum over all samples in input order with
 * Neumaier compensation (the discrete form of Eq. (1), Sec. III.A: no segment is cut).
 * Pixels are RING indices pix[k] (or pix0 + k).  stats (optional, int64[2]): number of
 * D = 0 pairs, number of samples skipped for 1 - Xdot^2 <= 0.
 * ---------------------------------------------------------------------------------- */
int or_isw_map(int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix,
               const double *samples, int64_t n, int64_t ld, const double x_obs[3], double GU,
               double *theta, int64_t *stats)
{
    int64_t zero_pairs = 0, bad = 0;
    seg_t *segs = (seg_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(seg_t));
    if (!segs) return OR_EINVAL;
    for (int64_t s = 0; s < n; ++s) {
        seg_prepare(samples, ld, s, x_obs, GU, &segs[s]);
        if (!segs[s].ok) ++bad;
    }
    for (int64_t k = 0; k < npix; ++k) {
        int64_t p = pix ? pix[k] : pix0 + k, ri, ji;
        double nv[3];
        int st = or_pix2vec_ring_one(nside, p, &ri, &ji, nv);
        if (st) {
            free(segs);
            return st;
        }
        double sum = 0.0, comp = 0.0;
        for (int64_t s = 0; s < n; ++s) {
            pair_t q;
            if (!segs[s].ok) continue;
            if (!pair_eval(nv, &segs[s], &q)) {
                ++zero_pairs;
                continue;
            }
            double t = segs[s].kappa * (q.uD / q.D2);
            double x = sum + t;
            if (fabs(sum) >= fabs(t)) comp += (sum - x) + t;
            else comp += (t - x) + sum;
            sum = x;
        }
        theta[k] = sum + comp;
    }
    free(segs);
    if (stats) {
        stats[0] = zero_pairs;
        stats[1] = bad;
    }
    return OR_OK;
}

/* Same sum for explicit unit directions dirs[3][ld_dir] (for pins off the HEALPix grid). */
int or_isw_sum_dirs(int64_t ndir, const double *dirs, int64_t ld_dir, const double *samples,
                    int64_t n, int64_t ld, const double x_obs[3], double GU, double *theta)
{
    seg_t *segs = (seg_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(seg_t));
    if (!segs) return OR_EINVAL;
    for (int64_t s = 0; s < n; ++s) seg_prepare(samples, ld, s, x_obs, GU, &segs[s]);
    for (int64_t k = 0; k < ndir; ++k) {
        double nv[3] = {dirs[k], dirs[ld_dir + k], dirs[2 * ld_dir + k]};
        double sum = 0.0, comp = 0.0;
        for (int64_t s = 0; s < n; ++s) {
            pair_t q;
            if (!segs[s].ok || !pair_eval(nv, &segs[s], &q)) continue;
            double t = segs[s].kappa * (q.uD / q.D2);
            double x = sum + t;
            if (fabs(sum) >= fabs(t)) comp += (sum - x) + t;
            else comp += (t - x) + sum;
            sum = x;
        }
        theta[k] = sum + comp;
    }
    free(segs);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------
 * 6. Adjoint.  With t = kappa (u.D)/D^2, kappa = -4 GU eps dsigma:
 *   dt/dX_s    = kappa [ (h.n) Xhat - h ],  h = u/D^2 - 2 (u.D) D / D^4   (dD/dX_s = n Xhat^T - I)
 *   dt/dXdot   = t Xdot/(1 - Xdot^2) + kappa [ D + A (X'.D) n / B^2 ] / D^2
 *   dt/dX'     = t X'/X'^2 - kappa [ (X'.D) n + A D ] / (B D^2)
 *   dt/ddsigma = t / dsigma = -4 GU eps (u.D)/D^2            (t is linear in dsigma)
 * and dL/dq_s = sum_p g_p dt_ps/dq_s.  grad is double[ngrad][ldg] with rows X(3), Xdot(3),
 * then X'(3) when ngrad >= 9 and dsigma when ngrad == 10.  Pinned by central finite
 * differences of the oracle map and, for dsigma, by the linearity of the map in dsigma.
 * ---------------------------------------------------------------------------------- */
int or_isw_map_adjoint(int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix,
                       const double *samples, int64_t n, int64_t ld, const double x_obs[3],
                       double GU, const double *g_pix, double *grad, int64_t ldg, int ngrad)
{
    double *nvs = (double *)malloc((size_t)(npix > 0 ? npix : 1) * 3 * sizeof(double));
    if (!nvs) return OR_EINVAL;
    for (int64_t k = 0; k < npix; ++k) {
        int64_t p = pix ? pix[k] : pix0 + k, ri, ji;
        int st = or_pix2vec_ring_one(nside, p, &ri, &ji, nvs + 3 * k);
        if (st) {
            free(nvs);
            return st;
        }
    }
    for (int64_t s = 0; s < n; ++s) {
        seg_t g;
        seg_prepare(samples, ld, s, x_obs, GU, &g);
        double acc[10] = {0}, cmp[10] = {0};
        for (int64_t k = 0; k < npix && g.ok; ++k) {
            const double *nv = nvs + 3 * k;
            pair_t q;
            if (!pair_eval(nv, &g, &q)) continue;
            double gp = g_pix[k];
            double t = g.kappa * (q.uD / q.D2);
            double inv = 1.0 / q.D2;
            double h[3];
            for (int c = 0; c < 3; ++c) h[c] = q.u[c] * inv - 2.0 * q.uD * q.D[c] * inv * inv;
            double hn = (h[0] * nv[0] + h[1] * nv[1]) + h[2] * nv[2];
            double xhat[3] = {g.xh[0] + g.xl[0], g.xh[1] + g.xl[1], g.xh[2] + g.xl[2]};
            double d[10];
            double B2 = q.B * q.B;
            for (int c = 0; c < 3; ++c) {
                d[c] = g.kappa * (hn * xhat[c] - h[c]);
                d[3 + c] = t * g.xd[c] / g.om + g.kappa * (q.D[c] + q.A * q.XpD * nv[c] / B2) * inv;
                d[6 + c] = t * g.xp[c] / g.xp2 - g.kappa * (q.XpD * nv[c] + q.A * q.D[c]) / (q.B * q.D2);
            }
            d[9] = g.kd * (q.uD / q.D2);
            for (int c = 0; c < ngrad; ++c) {
                double tt = gp * d[c];
                double x = acc[c] + tt;
                if (fabs(acc[c]) >= fabs(tt)) cmp[c] += (acc[c] - x) + tt;
                else cmp[c] += (tt - x) + acc[c];
                acc[c] = x;
            }
        }
        for (int c = 0; c < ngrad; ++c) grad[c * ldg + s] = acc[c] + cmp[c];
    }
    free(nvs);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------
 * 7. Adjoint of the light-cone solve (an extension of the method: the derivative of the
 * crossing condition X cap x_gamma of Eq. (1), with X', Xdot recorded at the crossing as in
 * Sec. II.B).  A sample's X, Xdot, X' are the worldsheet at the retarded time tau, the root
 * of F(tau) = |X(tau) - x_obs| - (t_obs - tau) = 0.  By the implicit-function theorem
 *   dtau/dq = -(rhat . dX/dq|_t) / (1 + rhat . Xdot),   rhat = (X - x_obs) / |X - x_obs|,
 * so with g_X, g_Xd, g_Xp = dL/d(sample X, Xdot, X') and the time derivatives of the three,
 *   lambda = (g_X . dX/dt + g_Xd . dXdot/dt + g_Xp . dX'/dt) / (1 + rhat . Xdot),
 *   gamma  = g_X - lambda rhat,
 *   dL/dq  = gamma . dX/dq|_t + g_Xd . dXdot/dq|_t + g_Xp . dX'/dq|_t.
 * LINEAR (straight worldline X = X_b + Xdot (tau - t_box); Xdot, X' constant):
 *   dL/dX_b = gamma, dL/dXdot_b = g_Xd + (tau - t_box) gamma, dL/dX'_b = g_Xp,
 *   dL/ddsigma_b = g_dsigma.
 * BURDEN (X = c + R h, h = (a(u) + b(v))/2, u = sigma - (t - t0), v = sigma + (t - t0)):
 *   dX/dt = R hd, hd = (b' - a')/2;  dXdot/dt = R hdd, hdd = (a'' + b'')/2;
 *   dX'/dt = dXdot/dsigma = R hdp, hdp = (b'' - a'')/2;  dX/dsigma = X' = R hp, hp = (a' + b')/2,
 *   dX'/dsigma = R hdd.  Per loop, summed over its samples in input order:
 *   dL/dc = gamma;  dL/dR_kj = gamma_k h_j + g_Xd,k hd_j + g_Xp,k hp_j;
 *   dL/dt0 = -(gamma . R hd + g_Xd . R hdd + g_Xp . R hdp)       (d/dt0 = -d/dt at fixed sigma);
 *   dL/dL, dL/dpsi from da/dL = a/L - (u/L) a', da'/dL = -(u/L) a'' (b alike with v) and
 *   db/dpsi, db'/dpsi.  Per sample: dL/dsigma = gamma . R hp + g_Xd . R hdp + g_Xp . R hdd
 *   (node row 1) and dL/ddsigma (node row 9).  m and n are integer harmonic numbers: their
 *   rows stay zero.  Pinned by central finite differences of the oracle's light-cone solve
 *   followed by the oracle map.
 * ---------------------------------------------------------------------------------- */
typedef struct {
    double h[3], hd[3], hp[3], hdd[3], hdp[3];  /* h and its t / sigma derivatives */
    double hL[3], hdL[3], hpL[3];               /* d/dL of h, hd, hp at fixed (sigma, t) */
    double hs[3], hds[3], hps[3];               /* d/dpsi of h, hd, hp */
} burden_jet_t;

static void burden_jet(const double *P, int64_t ldp, int64_t id, double sigma, double t,
                       burden_jet_t *J)
{
    const double two_pi = 2.0 * PI;
    double L = P[12 * ldp + id], m = P[13 * ldp + id], n = P[14 * ldp + id];
    double psi = P[15 * ldp + id], t0 = P[16 * ldp + id];
    double dt = t - t0;
    double u = sigma - dt, v = sigma + dt;
    double sa, ca, sb, cb, sp, cp;
    or_sincos_turns((m * u) / L, &sa, &ca);
    or_sincos_turns((n * v) / L, &sb, &cb);
    or_sincos_turns(psi / two_pi, &sp, &cp);
    double ra = L / (two_pi * m), rb = L / (two_pi * n);
    double ka = (two_pi * m) / L, kb = (two_pi * n) / L;
    double a[3] = {ra * sa, -(ra * ca), 0.0};
    double ap[3] = {ca, sa, 0.0};
    double app[3] = {-(ka * sa), ka * ca, 0.0};
    double b[3] = {rb * sb, -(rb * (cp * cb)), -(rb * (sp * cb))};
    double bp[3] = {cb, cp * sb, sp * sb};
    double bpp[3] = {-(kb * sb), kb * (cp * cb), kb * (sp * cb)};
    double bs[3] = {0.0, rb * (sp * cb), -(rb * (cp * cb))};
    double bps[3] = {0.0, -(sp * sb), cp * sb};
    for (int k = 0; k < 3; ++k) {
        double aL = a[k] / L - (u / L) * ap[k], bL = b[k] / L - (v / L) * bp[k];
        double apL = -(u / L) * app[k], bpL = -(v / L) * bpp[k];
        J->h[k] = 0.5 * (a[k] + b[k]);
        J->hd[k] = 0.5 * (bp[k] - ap[k]);
        J->hp[k] = 0.5 * (ap[k] + bp[k]);
        J->hdd[k] = 0.5 * (app[k] + bpp[k]);
        J->hdp[k] = 0.5 * (bpp[k] - app[k]);
        J->hL[k] = 0.5 * (aL + bL);
        J->hdL[k] = 0.5 * (bpL - apL);
        J->hpL[k] = 0.5 * (apL + bpL);
        J->hs[k] = 0.5 * bs[k];
        J->hds[k] = 0.5 * bps[k];
        J->hps[k] = 0.5 * bps[k];
    }
}

static void mat_vec(const double R[9], const double x[3], double y[3])
{
    for (int k = 0; k < 3; ++k) y[k] = (R[3 * k] * x[0] + R[3 * k + 1] * x[1]) + R[3 * k + 2] * x[2];
}

static double dot3(const double *a, const double *b)
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

static void neumaier(double *acc, double *cmp, double t)
{
    double x = *acc + t;
    if (fabs(*acc) >= fabs(t)) *cmp += (*acc - x) + t;
    else *cmp += (t - x) + *acc;
    *acc = x;
}

int or_lightcone_adjoint(int mode, const double *nodes, int64_t n, int64_t ld,
                         const double *P, int64_t nloops, int64_t ldp, double t_box,
                         const double x_obs[3], const double *tau, const double *gs, int64_t ldgs,
                         int ngs, double *gn, int64_t ldgn, double *gP, int64_t ldgP)
{
    int worst = OR_OK;
    double *cmp = NULL;
    if (mode != 0) {
        if (!gP) return OR_EINVAL;
        cmp = (double *)calloc((size_t)(nloops > 0 ? nloops : 1) * 17, sizeof(double));
        if (!cmp) return OR_EINVAL;
        for (int r = 0; r < 17; ++r)
            for (int64_t l = 0; l < nloops; ++l) gP[r * ldgP + l] = 0.0;
    }
    for (int64_t s = 0; s < n; ++s) {
        double gX[3], gXd[3], gXp[3] = {0.0, 0.0, 0.0}, gsig = 0.0;
        for (int k = 0; k < 3; ++k) {
            gX[k] = gs[k * ldgs + s];
            gXd[k] = gs[(3 + k) * ldgs + s];
            if (ngs >= 9) gXp[k] = gs[(6 + k) * ldgs + s];
        }
        if (ngs >= 10) gsig = gs[9 * ldgs + s];
        double out[10] = {0};
        out[9] = gsig;
        double t = tau[s];
        if (mode == 0) {
            double X[3], Xd[3], r[3];
            double D = t - t_box;
            for (int k = 0; k < 3; ++k) {
                Xd[k] = nodes[(3 + k) * ld + s];
                X[k] = nodes[k * ld + s] + Xd[k] * D;
                r[k] = X[k] - x_obs[k];
            }
            double rn = sqrt(dot3(r, r));
            double den = 1.0 + dot3(r, Xd) / rn;
            if (!(rn > 0.0) || !(den > 0.0)) {
                worst = OR_EDOMAIN > worst ? OR_EDOMAIN : worst;
            } else {
                double lam = dot3(gX, Xd) / den;
                for (int k = 0; k < 3; ++k) {
                    double gam = gX[k] - lam * (r[k] / rn);
                    out[k] = gam;
                    out[3 + k] = gXd[k] + D * gam;
                    out[6 + k] = gXp[k];
                }
            }
        } else {
            int64_t id = (int64_t)nodes[s];
            double sigma = nodes[ld + s];
            if (id < 0 || id >= nloops) {
                worst = OR_EINVAL > worst ? OR_EINVAL : worst;
            } else {
                double R[9], c[3];
                for (int k = 0; k < 3; ++k) c[k] = P[k * ldp + id];
                for (int k = 0; k < 9; ++k) R[k] = P[(3 + k) * ldp + id];
                burden_jet_t J;
                burden_jet(P, ldp, id, sigma, t, &J);
                double Rh[3], Xd[3], Xp[3], Xdd[3], Xdp[3], r[3];
                mat_vec(R, J.h, Rh);
                mat_vec(R, J.hd, Xd);
                mat_vec(R, J.hp, Xp);
                mat_vec(R, J.hdd, Xdd);
                mat_vec(R, J.hdp, Xdp);
                for (int k = 0; k < 3; ++k) r[k] = (c[k] + Rh[k]) - x_obs[k];
                double rn = sqrt(dot3(r, r));
                double den = 1.0 + dot3(r, Xd) / rn;
                if (!(rn > 0.0) || !(den > 0.0)) {
                    worst = OR_EDOMAIN > worst ? OR_EDOMAIN : worst;
                } else {
                    double lam = (dot3(gX, Xd) + dot3(gXd, Xdd) + dot3(gXp, Xdp)) / den;
                    double gam[3];
                    for (int k = 0; k < 3; ++k) gam[k] = gX[k] - lam * (r[k] / rn);
                    out[1] = (dot3(gam, Xp) + dot3(gXd, Xdp)) + dot3(gXp, Xdd);
                    double contrib[17] = {0};
                    for (int k = 0; k < 3; ++k) contrib[k] = gam[k];
                    for (int k = 0; k < 3; ++k)
                        for (int j = 0; j < 3; ++j)
                            contrib[3 + 3 * k + j] = (gam[k] * J.h[j] + gXd[k] * J.hd[j]) + gXp[k] * J.hp[j];
                    double v1[3], v2[3], v3[3];
                    mat_vec(R, J.hL, v1);
                    mat_vec(R, J.hdL, v2);
                    mat_vec(R, J.hpL, v3);
                    contrib[12] = (dot3(gam, v1) + dot3(gXd, v2)) + dot3(gXp, v3);
                    mat_vec(R, J.hs, v1);
                    mat_vec(R, J.hds, v2);
                    mat_vec(R, J.hps, v3);
                    contrib[15] = (dot3(gam, v1) + dot3(gXd, v2)) + dot3(gXp, v3);
                    contrib[16] = -((dot3(gam, Xd) + dot3(gXd, Xdd)) + dot3(gXp, Xdp));
                    for (int q = 0; q < 17; ++q)
                        neumaier(&gP[q * ldgP + id], &cmp[q * nloops + id], contrib[q]);
                }
            }
        }
        for (int q = 0; q < 10; ++q) gn[q * ldgn + s] = out[q];
    }
    if (cmp) {
        for (int q = 0; q < 17; ++q)
            for (int64_t l = 0; l < nloops; ++l) gP[q * ldgP + l] += cmp[q * nloops + l];
        free(cmp);
    }
    return worst;
}

/* ------------------------------------------------------------------------------------
 * 8. Stacking with HEALPix cones (Sec. III.B, Fig. 1): the comoving volume is voxelised by
 * the cones that subtend the pixels of a coarse HEALPix grid (N_side^hz); each cone is
 * filled from a simulation box rotated to face the observer, one box serving several cones
 * (the paper reuses each run three times), and only the strings inside the cone between
 * two radii are kept.
 *
 * (a) atan2 in quarter turns, own series: reduce to a = min/max of |x|, |y| in [0, 1];
 *     a > tan(pi/8) goes to (a - 1)/(a + 1) with pi/4 added back; one half-angle step
 *     atan(a) = 2 atan(a / (1 + sqrt(1 + a^2))) leaves |v| <= 0.2; atan(v) by its Taylor
 *     series v (1 - v^2/3 + v^4/5 - ...), 13 terms summed from the smallest; the octant is
 *     unfolded exactly.  Pinned against mpmath (<= 4 ulp).
 * (b) RING vec2pix, from the pixel-boundary curves of Gorski et al. (2005, Sec. 4): with
 *     z = cos(theta), t = phi / (pi/2) in [0, 4), the equatorial-zone boundaries are the lines
 *     z = 2/3 - 4k/(3N) +- 8 phi/(3 pi) and the polar-cap boundaries the curves
 *     z = 1 - (k/N)^2 (pi/(2 phi_t))^2 / 3 and z = 1 - (k/N)^2 (pi/(2 phi_t - pi))^2 / 3,
 *     phi_t = phi mod pi/2.  Solving each family for k at the direction counts the curves below
 *     it: in the belt |z| <= 2/3, jp = floor(N (1/2 + t - 3z/4)), jm = floor(N (1/2 + t + 3z/4)),
 *     ring N + 1 + jp - jm and position (jp + jm - N + kshift + 1)/2; in a cap, with
 *     tp = frac(t) and h = N sqrt(3 (1 - |z|)), jp = floor(tp h), jm = floor((1 - tp) h), ring
 *     jp + jm + 1 counted from the pole and position floor(t * ring).  Pinned by
 *     vec2pix(pix2vec(p)) = p, by an independent numpy statement of the same rules away from
 *     pixel edges, and by equal-area counts.
 * (c) box placement: shell k takes the nodes of box b_k and maps X -> R X + T, Xdot -> R Xdot,
 *     X' -> R X' (R row-major, (R x)_i = (R_i0 x_0 + R_i1 x_1) + R_i2 x_2), dsigma unchanged.
 * (d) cone cut: a light-cone sample of shell k is kept when the direction of X - x_obs lies
 *     in RING pixel cone_pix[k] of N_side^hz and r_lo[k] <= |X - x_obs| < r_hi[k]; kept
 *     samples keep their input order.
 * ---------------------------------------------------------------------------------- */
#define ATAN_TERMS 13

double or_atan2_quarter(double y, double x)
{
    const double tan_pi_8 = 0.41421356237309504880;  /* tan(pi/8) */
    const double two_over_pi = 0.63661977236758134308;
    double ax = fabs(x), ay = fabs(y);
    if (ax == 0.0 && ay == 0.0) return 0.0;
    int swap = ay > ax;
    double a = swap ? ax / ay : ay / ax;
    double base = 0.0;  /* quarter turns */
    if (a > tan_pi_8) {
        a = (a - 1.0) / (a + 1.0);
        base = 0.5;
    }
    double v = a / (1.0 + sqrt(1.0 + a * a));
    double w = v * v;
    double s = 0.0;
    for (int k = ATAN_TERMS - 1; k >= 0; --k) {
        double ck = 1.0 / (double)(2 * k + 1);
        s = (k & 1) ? s * w - ck : s * w + ck;
    }
    /* s = 1 - w/3 + w^2/5 - ... (Horner: the sign of each coefficient alternates) */
    double q = base + (2.0 * (v * s)) * two_over_pi;
    if (swap) q = 1.0 - q;
    if (x < 0.0) q = 2.0 - q;
    if (y < 0.0) q = 4.0 - q;
    if (q >= 4.0) q = q - 4.0;
    return q;
}

int64_t or_vec2pix_ring_one(int64_t N, const double v[3])
{
    double r = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    double z = v[2] / r;
    double za = fabs(z);
    double t = or_atan2_quarter(v[1], v[0]);
    double Nd = (double)N;
    int64_t npix = 12 * N * N, ncap = 2 * N * (N - 1);
    if (za <= 2.0 / 3.0) {
        double t1 = Nd * (0.5 + t);
        double t2 = Nd * (z * 0.75);
        int64_t jp = (int64_t)floor(t1 - t2);
        int64_t jm = (int64_t)floor(t1 + t2);
        int64_t ir = N + 1 + jp - jm;              /* 1 .. 2N+1, from z = 2/3 down */
        int64_t kshift = 1 - (ir & 1);
        int64_t ip = (jp + jm - N + kshift + 1) / 2;
        ip = ((ip % (4 * N)) + 4 * N) % (4 * N);
        return ncap + (ir - 1) * 4 * N + ip;
    }
    double tp = t - floor(t);
    double h = Nd * sqrt(3.0 * (1.0 - za));
    int64_t jp = (int64_t)floor(tp * h);
    int64_t jm = (int64_t)floor((1.0 - tp) * h);
    int64_t ir = jp + jm + 1;                      /* ring from the nearer pole */
    int64_t ip = (int64_t)floor(t * (double)ir);
    ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
    if (z > 0.0) return 2 * ir * (ir - 1) + ip;
    return npix - 2 * ir * (ir + 1) + ip;
}

/* vec: double[3][ld] (need not be normalised, not zero); pix: int64[n] */
void or_vec2pix_ring(int64_t N, const double *vec, int64_t n, int64_t ld, int64_t *pix)
{
    for (int64_t k = 0; k < n; ++k) {
        double v[3] = {vec[k], vec[ld + k], vec[2 * ld + k]};
        pix[k] = or_vec2pix_ring_one(N, v);
    }
}

/* nodes_box: double[10][ldb]; box_off[nbox+1]; shell_box[nshell]; place: double[nshell][12]
 * (R row-major, then T); out: double[10][ldo]; shell_off_out[nshell+1] (host) */
int or_box_place(const double *nodes_box, int64_t ldb, const int64_t *box_off, int64_t nbox,
                 int64_t nshell, const int64_t *shell_box, const double *place, double *out,
                 int64_t ldo, int64_t *shell_off_out)
{
    int64_t o = 0;
    shell_off_out[0] = 0;
    for (int64_t k = 0; k < nshell; ++k) {
        int64_t b = shell_box[k];
        if (b < 0 || b >= nbox) return OR_EINVAL;
        const double *R = place + 12 * k, *T = place + 12 * k + 9;
        for (int64_t s = box_off[b]; s < box_off[b + 1]; ++s, ++o) {
            if (o >= ldo) return OR_EINVAL;
            for (int blk = 0; blk < 3; ++blk) {
                double x[3];
                for (int c = 0; c < 3; ++c) x[c] = nodes_box[(3 * blk + c) * ldb + s];
                for (int i = 0; i < 3; ++i) {
                    double y = (R[3 * i] * x[0] + R[3 * i + 1] * x[1]) + R[3 * i + 2] * x[2];
                    out[(3 * blk + i) * ldo + o] = blk == 0 ? y + T[i] : y;
                }
            }
            out[9 * ldo + o] = nodes_box[9 * ldb + s];
        }
        shell_off_out[k + 1] = o;
    }
    return OR_OK;
}

/* samples: double[10][ld], shell_off[nshell+1]; cone_pix, r_lo, r_hi per shell; out:
 * double[10][ldo] kept samples in input order; shell_off_out[nshell+1]; returns the count
 * (or -1 on a bad argument). */
int64_t or_cone_cut(const double *samples, int64_t ld, const int64_t *shell_off, int64_t nshell,
                    int64_t nside_hz, const int64_t *cone_pix, const double *r_lo,
                    const double *r_hi, const double x_obs[3], double *out, int64_t ldo,
                    int64_t *shell_off_out)
{
    int64_t o = 0;
    shell_off_out[0] = 0;
    for (int64_t k = 0; k < nshell; ++k) {
        for (int64_t s = shell_off[k]; s < shell_off[k + 1]; ++s) {
            double d[3] = {samples[s] - x_obs[0], samples[ld + s] - x_obs[1],
                           samples[2 * ld + s] - x_obs[2]};
            double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
            if (!(r >= r_lo[k] && r < r_hi[k]) || !(r > 0.0)) continue;
            if (or_vec2pix_ring_one(nside_hz, d) != cone_pix[k]) continue;
            if (o >= ldo) return -1;
            for (int q = 0; q < 10; ++q) out[q * ldo + o] = samples[q * ld + s];
            ++o;
        }
        shell_off_out[k + 1] = o;
    }
    return o;
}

/* ------------------------------------------------------------------------------------
 * 9. Patch maps: full sky vs the flat-sky / small-angle approximation (Sec. II.A: the limit
 * X n -> X with parallel photon paths; Sec. IV, Fig. 3: a gnomonic patch of the full-sky map
 * against the flat-sky map of the same strings).
 *
 * Patch: orthonormal frame (e1, e2, e3) with e3 the patch centre; an M x M grid of gnomonic
 * coordinates xi_i = (i + 1/2 - M/2) w/M, eta_j likewise (w the coordinate width); pixel
 * (i, j) is stored at theta[j M + i].
 *   full sky: the discrete Eq. (1) sum at n = (xi e1 + eta e2 + e3) / |xi e1 + eta e2 + e3|;
 *   flat sky: every sample at depth Z = (X - x_obs).e3 > 0 sits at (xi_s, eta_s) =
 *     ((X - x_obs).e1, (X - x_obs).e2) / Z and contributes
 *       -4 GU eps dsigma / Z * (u_perp . d) / |d|^2,   d = (xi - xi_s, eta - eta_s),
 *     with u = Xdot - (e3.X') X' / (1 + e3.Xdot) (the photon direction fixed to e3) and
 *     u_perp = (u.e1, u.e2); samples with Z <= 0 are skipped, d = 0 gives 0.
 * Neumaier sums in input order.  Pinned by the flat-sky Kaiser-Stebbins step of a straight
 * moving segment, -8 GU gamma v atan(Lambda / eta) at its midpoint, and by the approach of the
 * full-sky patch to the flat-sky one at the centre of a small patch.
 * ---------------------------------------------------------------------------------- */
static void patch_dir(const double frame[9], int64_t M, double width, int64_t i, int64_t j,
                      double *xi, double *eta, double n[3])
{
    double h = width / (double)M;
    *xi = ((double)i + 0.5 - 0.5 * (double)M) * h;
    *eta = ((double)j + 0.5 - 0.5 * (double)M) * h;
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = (*xi * frame[k] + *eta * frame[3 + k]) + frame[6 + k];
    double r = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    for (int k = 0; k < 3; ++k) n[k] = v[k] / r;
}

/* rows j0 .. j1-1 of the patch; approx 0 = full sky, 1 = flat sky */
int or_isw_map_patch(const double frame[9], int64_t M, double width, int64_t j0, int64_t j1,
                     const double *samples, int64_t n, int64_t ld, const double x_obs[3], double GU,
                     int approx, double *theta)
{
    if (M < 1 || !(width > 0.0) || j0 < 0 || j1 > M) return OR_EINVAL;
    if (approx == 0) {
        seg_t *segs = (seg_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(seg_t));
        if (!segs) return OR_EINVAL;
        for (int64_t s = 0; s < n; ++s) seg_prepare(samples, ld, s, x_obs, GU, &segs[s]);
        for (int64_t j = j0; j < j1; ++j)
            for (int64_t i = 0; i < M; ++i) {
                double xi, eta, nv[3];
                patch_dir(frame, M, width, i, j, &xi, &eta, nv);
                double sum = 0.0, comp = 0.0;
                for (int64_t s = 0; s < n; ++s) {
                    pair_t q;
                    if (!segs[s].ok || !pair_eval(nv, &segs[s], &q)) continue;
                    neumaier(&sum, &comp, segs[s].kappa * (q.uD / q.D2));
                }
                theta[j * M + i] = sum + comp;
            }
        free(segs);
        return OR_OK;
    }
    /* flat sky: per-sample position in the patch and weight */
    double *rec = (double *)malloc((size_t)(n > 0 ? n : 1) * 5 * sizeof(double));
    int *ok = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    if (!rec || !ok) {
        free(rec);
        free(ok);
        return OR_EINVAL;
    }
    for (int64_t s = 0; s < n; ++s) {
        double r[3], Xd[3], Xp[3];
        for (int k = 0; k < 3; ++k) {
            r[k] = samples[k * ld + s] - x_obs[k];
            Xd[k] = samples[(3 + k) * ld + s];
            Xp[k] = samples[(6 + k) * ld + s];
        }
        double Z = dot3(r, frame + 6);
        double v2 = dot3(Xd, Xd), xp2 = dot3(Xp, Xp);
        double om = 1.0 - v2;
        double eps = sqrt(xp2 / om);
        double Bz = 1.0 + dot3(frame + 6, Xd), Az = dot3(frame + 6, Xp);
        double u[3];
        for (int k = 0; k < 3; ++k) u[k] = Xd[k] - (Az * Xp[k]) / Bz;
        double kd = -4.0 * GU * (eps * samples[9 * ld + s]) / Z;
        ok[s] = Z > 0.0 && om > 0.0 && Bz > 0.0 && isfinite(kd);
        rec[5 * s + 0] = dot3(r, frame) / Z;
        rec[5 * s + 1] = dot3(r, frame + 3) / Z;
        rec[5 * s + 2] = kd * dot3(u, frame);
        rec[5 * s + 3] = kd * dot3(u, frame + 3);
        rec[5 * s + 4] = kd;
    }
    for (int64_t j = j0; j < j1; ++j)
        for (int64_t i = 0; i < M; ++i) {
            double xi, eta, nv[3];
            patch_dir(frame, M, width, i, j, &xi, &eta, nv);
            double sum = 0.0, comp = 0.0;
            for (int64_t s = 0; s < n; ++s) {
                if (!ok[s]) continue;
                double dx = xi - rec[5 * s], dy = eta - rec[5 * s + 1];
                double Q = dx * dx + dy * dy;
                if (Q == 0.0) continue;
                neumaier(&sum, &comp, (rec[5 * s + 2] * dx + rec[5 * s + 3] * dy) / Q);
            }
            theta[j * M + i] = sum + comp;
        }
    free(rec);
    free(ok);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------
 * 10. Angular power spectrum of a full-sky RING map (Sec. IV, Fig. 4): spherical-harmonic
 * analysis with uniform pixel weights, a_lm = (4 pi / N_pix) sum_p Theta_p Y*_lm(n_p), and
 * C_l = (|a_l0|^2 + 2 sum_{m >= 1} |a_lm|^2) / (2l + 1).
 *   per ring r (z_r, n_r pixels at phi_rj = phi_r0 + 2 pi j / n_r):
 *     F_r(m) = sum_j Theta_rj exp(-i m phi_rj)        (each exponential from its own angle)
 *   per (l, m): a_lm = (4 pi / N_pix) sum_r lambda_lm(z_r) F_r(m),
 *     lambda_lm(z) = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(z) (Condon-Shortley phase), from
 *     lambda_mm = (-1)^m sqrt((2m+1)/(4 pi) prod_{k<=m} (2k-1)/(2k)) (1 - z^2)^(m/2),
 *     lambda_{m+1,m} = z sqrt(2m+3) lambda_mm and
 *     lambda_lm = z a_lm lambda_{l-1,m} - b_lm lambda_{l-2,m},
 *     a_lm = sqrt((4l^2 - 1)/(l^2 - m^2)), b_lm = sqrt(((2l+1)(l+m-1)(l-m-1)) / ((2l-3)(l^2 - m^2))).
 *     Values are carried as (mantissa, power of 2^256) so that lambda_mm near the poles does
 *     not underflow; a term counts once its scale is back to 1.
 * Pinned against mpmath's associated Legendre functions, by the analysis of band-limited maps
 * synthesised with scipy's spherical harmonics, and by exact symmetries of ring maps.
 * ---------------------------------------------------------------------------------- */
static const double LSCALE = 1.157920892373162e77;   /* 2^256 */

/* ring i (1..4N-1): z, number of pixels, first pixel index, phase phi_0 / (2 pi) in turns */
static void ring_info(int64_t N, int64_t i, double *z, int64_t *np, int64_t *p0, double *t0)
{
    double N3 = 3.0 * (double)N * (double)N;
    if (i < N) {
        *z = 1.0 - ((double)i * (double)i) / N3;
        *np = 4 * i;
        *p0 = 2 * i * (i - 1);
        *t0 = 1.0 / (8.0 * (double)i);
    } else if (i <= 3 * N) {
        *z = (4.0 * (double)N - 2.0 * (double)i) / (3.0 * (double)N);
        *np = 4 * N;
        *p0 = 2 * N * (N - 1) + (i - N) * 4 * N;
        *t0 = ((i + N) & 1) ? 0.0 : 1.0 / (8.0 * (double)N);
    } else {
        int64_t k = 4 * N - i;
        *z = -(1.0 - ((double)k * (double)k) / N3);
        *np = 4 * k;
        *p0 = 12 * N * N - 2 * k * (k + 1);
        *t0 = 1.0 / (8.0 * (double)k);
    }
}

/* lambda_lm(z) for l = m .. lmax into out[l] (out[l] = 0 for l < m and while the value is below
 * the double range): the recursion of this section with (mantissa, power of 2^256) scaling */
static void legendre_column(double z, int64_t m, int64_t lmax, double *out)
{
    for (int64_t l = 0; l < m && l <= lmax; ++l) out[l] = 0.0;
    if (m > lmax) return;
    double sth = sqrt((1.0 - z) * (1.0 + z));
    double lam = sqrt(1.0 / (4.0 * PI));
    int sc = 0;
    for (int64_t k = 1; k <= m; ++k) {
        lam = lam * (sqrt((2.0 * k - 1.0) / (2.0 * k)) * sth);
        if (fabs(lam) < 1.0 / LSCALE && lam != 0.0) {
            lam *= LSCALE;
            --sc;
        }
    }
    lam = lam * sqrt(2.0 * m + 1.0);
    if (m & 1) lam = -lam;
    double lprev = 0.0, lcur = lam;
    for (int64_t l = m; l <= lmax; ++l) {
        if (l > m) {
            double lnext;
            if (l == m + 1) {
                lnext = z * sqrt(2.0 * m + 3.0) * lcur;
            } else {
                double ll = (double)l, mm = (double)m;
                double a = sqrt((4.0 * ll * ll - 1.0) / (ll * ll - mm * mm));
                double b = sqrt(((2.0 * ll + 1.0) * (ll + mm - 1.0) * (ll - mm - 1.0)) /
                                ((2.0 * ll - 3.0) * (ll * ll - mm * mm)));
                lnext = z * a * lcur - b * lprev;
            }
            lprev = lcur;
            lcur = lnext;
            if (sc < 0 && fabs(lcur) > 1.0) {
                lcur /= LSCALE;
                lprev /= LSCALE;
                ++sc;
            }
        }
        out[l] = sc == 0 ? lcur : 0.0;
    }
}

void or_legendre_column(double z, int64_t m, int64_t lmax, double *out)
{
    legendre_column(z, m, lmax, out);
}

void or_ring_info(int64_t N, int64_t i, double *z, int64_t *np, int64_t *p0, double *t0)
{
    ring_info(N, i, z, np, p0, t0);
}

/* a_lm of one m, l = 0 .. lmax, into re[l], im[l] (zero for l < m): the Fourier sum of every
 * ring at this m (Neumaier, exact phase reduction), then the Legendre sum over the rings in
 * ring order.  Independent m give independent coefficients, so callers may split m freely. */
int or_map_alm_m(int64_t N, const double *map, int64_t lmax, int64_t m, double *re, double *im)
{
    if (N < 1 || lmax < 0 || m < 0 || m > lmax) return OR_EINVAL;
    int64_t nring = 4 * N - 1, npix = 12 * N * N;
    size_t L1 = (size_t)(lmax + 1);
    double *lam = (double *)malloc(L1 * sizeof(double));
    if (!lam) return OR_EINVAL;
    for (size_t l = 0; l < L1; ++l) re[l] = im[l] = 0.0;
    const double omega = 4.0 * PI / (double)npix;
    for (int64_t r = 0; r < nring; ++r) {
        double z, t0;
        int64_t np, p0;
        ring_info(N, r + 1, &z, &np, &p0, &t0);
        double sr = 0.0, cr = 0.0, si = 0.0, ci = 0.0;
        for (int64_t j = 0; j < np; ++j) {
            /* m phi / (2 pi) = m (t0 + j/np), reduced exactly: (m j mod np) / np + m t0 */
            double w = (double)((m * j) % np) / (double)np + (double)m * t0;
            double s, c;
            or_sincos_turns(w, &s, &c);
            double v = map[p0 + j];
            neumaier(&sr, &cr, v * c);
            neumaier(&si, &ci, -(v * s));
        }
        const double Fre = sr + cr, Fim = si + ci;
        legendre_column(z, m, lmax, lam);
        for (int64_t l = m; l <= lmax; ++l) {
            re[l] += omega * (lam[l] * Fre);
            im[l] += omega * (lam[l] * Fim);
        }
    }
    free(lam);
    return OR_OK;
}

/* C_l = (|a_l0|^2 + 2 sum_{m>=1} |a_lm|^2) / (2l + 1) from alm: double[2][lmax+1][lmax+1] */
void or_cl_from_alm(int64_t lmax, const double *alm, double *cl)
{
    size_t L1 = (size_t)(lmax + 1), M1 = L1;
    for (int64_t l = 0; l <= lmax; ++l) {
        double s = 0.0;
        for (int64_t m = 0; m <= l; ++m) {
            size_t q = (size_t)m * L1 + (size_t)l;
            double p = alm[q] * alm[q] + alm[M1 * L1 + q] * alm[M1 * L1 + q];
            s += m == 0 ? p : 2.0 * p;
        }
        cl[l] = s / (2.0 * l + 1.0);
    }
}

/* alm: double[2][mmax+1][lmax+1] (re then im), only l >= m filled; cl: double[lmax+1] */
int or_map_alm_cl(int64_t N, const double *map, int64_t lmax, double *alm, double *cl)
{
    if (N < 1 || lmax < 0) return OR_EINVAL;
    size_t L1 = (size_t)(lmax + 1), M1 = L1;
    for (int64_t m = 0; m <= lmax; ++m) {
        int r = or_map_alm_m(N, map, lmax, m, alm + (size_t)m * L1, alm + M1 * L1 + (size_t)m * L1);
        if (r) return r;
    }
    or_cl_from_alm(lmax, alm, cl);
    return OR_OK;
}
