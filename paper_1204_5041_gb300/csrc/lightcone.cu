// Past-light-cone intersection of string nodes (Eq. 1: the samples are the string points
// X with X cap x_gamma; Sec. II.B: X' and Xdot are recorded at the crossing).  One thread
// per node, IEEE double without contraction so that the result is reproducible operation
// by operation (flat conformal coordinates, c = 1).
#include "isw_internal.cuh"
#include "kernels.cuh"

namespace isw {

// Burden loop X(s, t) = c + R (a(s - (t - t0)) + b(s + (t - t0))) / 2 with
//   a(u) = L/(2 pi m) (sin 2 pi m u/L, -cos 2 pi m u/L, 0),
//   b(v) = L/(2 pi n) (sin 2 pi n v/L, -cos psi cos 2 pi n v/L, -sin psi cos 2 pi n v/L);
// Xdot = R (b' - a')/2, X' = R (a' + b')/2.  P is double[17][ldp]: c(3) R(9) L m n psi t0.
__device__ __forceinline__ void burden_worldsheet(const double *__restrict__ P, int64_t ldp, int64_t id, double sigma,
                                                  double t, double X[3], double Xd[3], double Xp[3])
{
    const double two_pi = 2.0 * kPi;
    const double L = P[12 * ldp + id], m = P[13 * ldp + id], n = P[14 * ldp + id];
    const double psi = P[15 * ldp + id], t0 = P[16 * ldp + id];
    const double dt = dsub(t, t0);
    const double u = dsub(sigma, dt), v = dadd(sigma, dt);
    double sa, ca, sb, cb, sp, cp;
    sincos_turns(ddiv(dmul(m, u), L), sa, ca);
    sincos_turns(ddiv(dmul(n, v), L), sb, cb);
    sincos_turns(ddiv(psi, two_pi), sp, cp);
    const double ra = ddiv(L, dmul(two_pi, m)), rb = ddiv(L, dmul(two_pi, n));
    const double a[3] = {dmul(ra, sa), -dmul(ra, ca), 0.0};
    const double b[3] = {dmul(rb, sb), -dmul(rb, dmul(cp, cb)), -dmul(rb, dmul(sp, cb))};
    const double ap[3] = {ca, sa, 0.0};
    const double bp[3] = {cb, dmul(cp, sb), dmul(sp, sb)};
    double h[3], hd[3], hp[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        h[k] = dmul(0.5, dadd(a[k], b[k]));
        hd[k] = dmul(0.5, dsub(bp[k], ap[k]));
        hp[k] = dmul(0.5, dadd(ap[k], bp[k]));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double r0 = P[(3 + 3 * k) * ldp + id], r1 = P[(4 + 3 * k) * ldp + id], r2 = P[(5 + 3 * k) * ldp + id];
        X[k] = dadd(P[k * ldp + id], dadd(dadd(dmul(r0, h[0]), dmul(r1, h[1])), dmul(r2, h[2])));
        Xd[k] = dadd(dadd(dmul(r0, hd[0]), dmul(r1, hd[1])), dmul(r2, hd[2]));
        Xp[k] = dadd(dadd(dmul(r0, hp[0]), dmul(r1, hp[1])), dmul(r2, hp[2]));
    }
}

__device__ __forceinline__ int solve_node(int mode, const double *__restrict__ nodes, int64_t ld, int64_t s,
                                          const double *__restrict__ P, int64_t nloops, int64_t ldp, double t_box,
                                          double xo0, double xo1, double xo2, double t_obs, double tol, int max_iter,
                                          double X[3], double Xd[3], double Xp[3], double &t)
{
    const double xo[3] = {xo0, xo1, xo2};
    int st = ISW_OK;
    if (mode == ISW_LINEAR) {
        double r0[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            X[k] = nodes[k * ld + s];
            Xd[k] = nodes[(3 + k) * ld + s];
            Xp[k] = nodes[(6 + k) * ld + s];
            r0[k] = dsub(X[k], xo[k]);
        }
        const double R = dsqrt(dadd(dadd(dmul(r0[0], r0[0]), dmul(r0[1], r0[1])), dmul(r0[2], r0[2])));
        const double T = dsub(t_obs, t_box);
        const double v2 = dadd(dadd(dmul(Xd[0], Xd[0]), dmul(Xd[1], Xd[1])), dmul(Xd[2], Xd[2]));
        const double om = dsub(1.0, v2);
        t = t_box;
        if (!(om > 0.0) || !(R == R)) {
            st = ISW_EDOMAIN;
        } else {
            // (v^2 - 1) D^2 + 2 (r0.Xdot + T) D + (|r0|^2 - T^2) = 0, past root without cancellation
            const double c = dmul(dsub(R, T), dadd(R, T));
            const double bh = dadd(dadd(dadd(dmul(r0[0], Xd[0]), dmul(r0[1], Xd[1])), dmul(r0[2], Xd[2])), T);
            double disc = dadd(dmul(bh, bh), dmul(om, c));
            if (disc < 0.0) disc = 0.0;
            const double D = ddiv(-c, dadd(bh, dsqrt(disc)));
            t = dadd(t_box, D);
#pragma unroll
            for (int k = 0; k < 3; ++k) X[k] = dadd(X[k], dmul(Xd[k], D));
        }
    } else {
        const int64_t id = (int64_t)nodes[s];
        const double sigma = nodes[ld + s];
        t = t_obs;
        if (id < 0 || id >= nloops) {
#pragma unroll
            for (int k = 0; k < 3; ++k) X[k] = Xd[k] = Xp[k] = 0.0;
            st = ISW_EINVAL;
        } else {
            const double cx = dsub(P[0 * ldp + id], xo0), cy = dsub(P[1 * ldp + id], xo1),
                         cz = dsub(P[2 * ldp + id], xo2);
            const double d = dsqrt(dadd(dadd(dmul(cx, cx), dmul(cy, cy)), dmul(cz, cz)));
            const double halfL = dmul(0.5, P[12 * ldp + id]);
            double lo = dsub(dsub(t_obs, d), halfL), hi = dadd(dsub(t_obs, d), halfL);
            double step1 = dsub(hi, lo), step2 = dsub(hi, lo);   // last two step lengths
            t = dsub(t_obs, d);
            st = ISW_ENOCONV;
            // f(t) = |X(s, t) - x_obs| - (t_obs - t) is increasing (f' = 1 + rhat.Xdot > 0):
            // Newton steps, replaced by bisection when they leave the bracket or fail to halve
            // the step taken two iterations earlier
            for (int it = 0; it < max_iter; ++it) {
                burden_worldsheet(P, ldp, id, sigma, t, X, Xd, Xp);
                const double r[3] = {dsub(X[0], xo0), dsub(X[1], xo1), dsub(X[2], xo2)};
                const double rn = dsqrt(dadd(dadd(dmul(r[0], r[0]), dmul(r[1], r[1])), dmul(r[2], r[2])));
                const double f = dsub(rn, dsub(t_obs, t));
                if (fabs(f) <= tol) {
                    st = ISW_OK;
                    break;
                }
                if (!(rn > 0.0)) {
                    st = ISW_EDOMAIN;
                    break;
                }
                if (f < 0.0) lo = t; else hi = t;
                const double fp = dadd(1.0, ddiv(dadd(dadd(dmul(r[0], Xd[0]), dmul(r[1], Xd[1])), dmul(r[2], Xd[2])), rn));
                double tn = dsub(t, ddiv(f, fp));
                // bisect when Newton leaves the bracket or does not at least halve the step taken
                // two iterations earlier (stops two-cycles between the bracket ends)
                if (!(tn > lo && tn < hi) || fabs(dsub(tn, t)) > dmul(0.5, step2)) tn = dmul(0.5, dadd(lo, hi));
                step2 = step1;
                step1 = fabs(dsub(tn, t));
                if (it + 1 < max_iter) t = tn;
            }
        }
    }
    return st;
}

__device__ __forceinline__ void record_status(int st, DevStatus *ds)
{
    if (st == ISW_ENOCONV) atomicOr(&ds->bits, kStatNoConv);
    else if (st == ISW_EDOMAIN) atomicOr(&ds->bits, kStatDomain);
    else if (st == ISW_EINVAL) atomicOr(&ds->bits, kStatBadIndex);
}

__global__ void k_lightcone(int mode, const double *__restrict__ nodes, int64_t n, int64_t ld,
                            const double *__restrict__ P, int64_t nloops, int64_t ldp, double t_box, double xo0,
                            double xo1, double xo2, double t_obs, double tol, int max_iter, double *__restrict__ out,
                            int64_t ld_out, double *__restrict__ tau, int32_t *__restrict__ status, DevStatus *ds)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        double X[3], Xd[3], Xp[3], t;
        const int st = solve_node(mode, nodes, ld, s, P, nloops, ldp, t_box, xo0, xo1, xo2, t_obs, tol, max_iter, X,
                                  Xd, Xp, t);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            out[k * ld_out + s] = X[k];
            out[(3 + k) * ld_out + s] = Xd[k];
            out[(6 + k) * ld_out + s] = Xp[k];
        }
        out[9 * ld_out + s] = nodes[9 * ld + s];
        if (tau) tau[s] = t;
        if (status) status[s] = st;
        if (st != ISW_OK) record_status(st, ds);
    }
}

// Many shells in one launch: node s belongs to the shell k with off[k] <= s < off[k+1].
__global__ void k_lightcone_shells(const double *__restrict__ nodes, int64_t n, int64_t ld,
                                   const int64_t *__restrict__ off, int64_t nshell, const double *__restrict__ t_box,
                                   const int32_t *__restrict__ mode, const double *__restrict__ P, int64_t nloops,
                                   int64_t ldp, double xo0, double xo1, double xo2, double t_obs, double tol,
                                   double *__restrict__ out, int64_t ld_out, DevStatus *ds)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nshell;  // find k with off[k] <= s < off[k+1]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (off[mid] <= s) lo = mid; else hi = mid;
        }
        double X[3], Xd[3], Xp[3], t;
        const int st = solve_node(mode[lo], nodes, ld, s, P, nloops, ldp, t_box[lo], xo0, xo1, xo2, t_obs, tol, 60, X,
                                  Xd, Xp, t);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            out[k * ld_out + s] = X[k];
            out[(3 + k) * ld_out + s] = Xd[k];
            out[(6 + k) * ld_out + s] = Xp[k];
        }
        out[9 * ld_out + s] = nodes[9 * ld + s];
        if (st != ISW_OK) record_status(st, ds);
    }
}

static unsigned grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

void launch_lightcone(int mode, const double *nodes, int64_t n, int64_t ld, const double *P, int64_t nloops,
                      int64_t ldp, double t_box, double xo0, double xo1, double xo2, double t_obs, double tol,
                      int max_iter, double *out, int64_t ld_out, double *tau, int32_t *status, DevStatus *st,
                      cudaStream_t s)
{
    if (n <= 0) return;
    k_lightcone<<<grid_for(n, 128), 128, 0, s>>>(mode, nodes, n, ld, P, nloops, ldp, t_box, xo0, xo1, xo2, t_obs, tol,
                                                  max_iter, out, ld_out, tau, status, st);
}

void launch_lightcone_shells(const double *nodes, int64_t n, int64_t ld, const int64_t *shell_off, int64_t nshell,
                             const double *t_box, const int32_t *mode, const double *P, int64_t nloops, int64_t ldp,
                             double xo0, double xo1, double xo2, double t_obs, double tol, double *out,
                             int64_t ld_out, DevStatus *st, cudaStream_t s)
{
    if (n <= 0) return;
    k_lightcone_shells<<<grid_for(n, 128), 128, 0, s>>>(nodes, n, ld, shell_off, nshell, t_box, mode, P, nloops, ldp,
                                                         xo0, xo1, xo2, t_obs, tol, out, ld_out, st);
}

}  // namespace isw
