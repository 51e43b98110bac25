// Adjoint of the past-light-cone intersection: an extension of the method that
// differentiates the crossing condition X cap x_gamma of Eq. (1) (X' and Xdot recorded at
// the crossing, Sec. II.B).  A sample is the worldsheet at the retarded time tau, the root of
// F = |X(tau) - x_obs| - (t_obs - tau); by the implicit-function theorem
//   dtau/dq = -(rhat . dX/dq|_t) / (1 + rhat . Xdot),  rhat = (X - x_obs)/|X - x_obs|,
// so with g_X, g_Xd, g_Xp the gradients of the sample's X, Xdot, X' and
//   lambda = (g_X . dX/dt + g_Xd . dXdot/dt + g_Xp . dX'/dt) / (1 + rhat . Xdot),
//   gamma = g_X - lambda rhat,
// dL/dq = gamma . dX/dq|_t + g_Xd . dXdot/dq|_t + g_Xp . dX'/dq|_t for every parameter q.
// One thread per node writes the node gradients; for Burden loops one warp per loop sums the
// loop-parameter gradients over the loop's samples in a fixed order (deterministic).
#include "isw_internal.cuh"
#include "kernels.cuh"

namespace isw {

// Burden worldsheet h = (a(u) + b(v))/2 (X = c + R h) and the derivatives the adjoint needs,
// at fixed (sigma, t): hd = dh/dt, hp = dh/dsigma, hdd = d2h/dt2 (= d2h/dsigma2 by the wave
// equation), hdp = d2h/dt dsigma, and d/dL, d/dpsi of h, hd, hp (dhp/dpsi = dhd/dpsi).
struct BurdenJet {
    double h[3], hd[3], hp[3], hdd[3], hdp[3];
    double hL[3], hdL[3], hpL[3], hs[3], hds[3];
};

__device__ __forceinline__ void burden_jet(const double *__restrict__ P, int64_t ldp, int64_t id, double sigma,
                                           double t, BurdenJet &J)
{
    const double two_pi = 2.0 * kPi;
    const double L = P[12 * ldp + id], m = P[13 * ldp + id], n = P[14 * ldp + id];
    const double psi = P[15 * ldp + id], t0 = P[16 * ldp + id];
    const double dt = t - t0;
    const double u = sigma - dt, v = sigma + dt;
    double sa, ca, sb, cb, sp, cp;
    sincos_turns(m * u / L, sa, ca);
    sincos_turns(n * v / L, sb, cb);
    sincos_turns(psi / two_pi, sp, cp);
    const double ra = L / (two_pi * m), rb = L / (two_pi * n);
    const double ka = two_pi * m / L, kb = two_pi * n / L;
    const double iL = 1.0 / L;
    // a, a', a'' and b, b', b'' (derivatives in their own argument), db/dpsi, db'/dpsi
    const double a[3] = {ra * sa, -ra * ca, 0.0}, ap[3] = {ca, sa, 0.0}, app[3] = {-ka * sa, ka * ca, 0.0};
    const double b[3] = {rb * sb, -rb * cp * cb, -rb * sp * cb}, bp[3] = {cb, cp * sb, sp * sb};
    const double bpp[3] = {-kb * sb, kb * cp * cb, kb * sp * cb};
    const double bs[3] = {0.0, rb * sp * cb, -rb * cp * cb}, bps[3] = {0.0, -sp * sb, cp * sb};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // d/dL at fixed argument: a/L - (u/L) a',  a' -> -(u/L) a''  (b alike with v)
        const double aL = (a[k] - u * ap[k]) * iL, bL = (b[k] - v * bp[k]) * iL;
        const double apL = -u * iL * app[k], bpL = -v * iL * bpp[k];
        J.h[k] = 0.5 * (a[k] + b[k]);
        J.hd[k] = 0.5 * (bp[k] - ap[k]);
        J.hp[k] = 0.5 * (ap[k] + bp[k]);
        J.hdd[k] = 0.5 * (app[k] + bpp[k]);
        J.hdp[k] = 0.5 * (bpp[k] - app[k]);
        J.hL[k] = 0.5 * (aL + bL);
        J.hdL[k] = 0.5 * (bpL - apL);
        J.hpL[k] = 0.5 * (apL + bpL);
        J.hs[k] = 0.5 * bs[k];
        J.hds[k] = 0.5 * bps[k];
    }
}

__device__ __forceinline__ void rot(const double *R, const double *x, double *y)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) y[k] = R[3 * k] * x[0] + R[3 * k + 1] * x[1] + R[3 * k + 2] * x[2];
}

__device__ __forceinline__ double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Sample gradients of node s (missing rows of grad_samples count as zero)
__device__ __forceinline__ void load_gs(const double *__restrict__ gs, int64_t ldgs, int ngs, int64_t s, double gX[3],
                                        double gXd[3], double gXp[3], double &gsig)
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gX[k] = gs[k * ldgs + s];
        gXd[k] = gs[(3 + k) * ldgs + s];
        gXp[k] = ngs >= 9 ? gs[(6 + k) * ldgs + s] : 0.0;
    }
    gsig = ngs >= 10 ? gs[9 * ldgs + s] : 0.0;
}

// One Burden sample: gamma-weighted derivatives.  Returns false when rhat is undefined or
// 1 + rhat.Xdot <= 0.  contrib (optional): centre (3), rotation (9), L, psi, t0.
__device__ __forceinline__ bool burden_sample(const double *__restrict__ P, int64_t ldp, int64_t id, double sigma,
                                              double t, const double xo[3], const double gX[3], const double gXd[3],
                                              const double gXp[3], double &g_sigma, double *contrib)
{
    double R[9], c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = P[k * ldp + id];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = P[(3 + k) * ldp + id];
    BurdenJet J;
    burden_jet(P, ldp, id, sigma, t, J);
    double Rh[3], Xd[3], Xp[3], Xdd[3], Xdp[3], r[3];
    rot(R, J.h, Rh);
    rot(R, J.hd, Xd);
    rot(R, J.hp, Xp);
    rot(R, J.hdd, Xdd);
    rot(R, J.hdp, Xdp);
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = c[k] + Rh[k] - xo[k];
    const double rn = sqrt(dot3(r, r));
    const double den = 1.0 + dot3(r, Xd) / rn;
    if (!(rn > 0.0) || !(den > 0.0)) return false;
    const double lam = (dot3(gX, Xd) + dot3(gXd, Xdd) + dot3(gXp, Xdp)) / den;
    double gam[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) gam[k] = gX[k] - lam * (r[k] / rn);
    g_sigma = dot3(gam, Xp) + dot3(gXd, Xdp) + dot3(gXp, Xdd);
    if (contrib) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            contrib[k] = gam[k];
#pragma unroll
            for (int j = 0; j < 3; ++j) contrib[3 + 3 * k + j] = gam[k] * J.h[j] + gXd[k] * J.hd[j] + gXp[k] * J.hp[j];
        }
        double v1[3], v2[3], v3[3];
        rot(R, J.hL, v1);
        rot(R, J.hdL, v2);
        rot(R, J.hpL, v3);
        contrib[12] = dot3(gam, v1) + dot3(gXd, v2) + dot3(gXp, v3);
        rot(R, J.hs, v1);
        rot(R, J.hds, v2);
        contrib[13] = dot3(gam, v1) + dot3(gXd, v2) + dot3(gXp, v2);
        contrib[14] = -(dot3(gam, Xd) + dot3(gXd, Xdd) + dot3(gXp, Xdp));
    }
    return true;
}

// loop id of node s as the light-cone solve reads it (truncated), -1 when out of range
__device__ __forceinline__ int64_t loop_id(const double *__restrict__ nodes, int64_t s, int64_t nloops)
{
    const int64_t id = (int64_t)nodes[s];
    return (id >= 0 && id < nloops) ? id : -1;
}

// Node gradients; Burden mode also marks the first and one-past-last sample of every run of
// equal loop ids (runs[l] counts the runs of loop l: 1 when its samples are contiguous).
__global__ void k_lcadj_nodes(int mode, const double *__restrict__ nodes, int64_t n, int64_t ld,
                              const double *__restrict__ P, int64_t nloops, int64_t ldp, double t_box, double xo0,
                              double xo1, double xo2, const double *__restrict__ tau, const double *__restrict__ gs,
                              int64_t ldgs, int ngs, double *__restrict__ gn, int64_t ldgn, int *__restrict__ runs,
                              int64_t *__restrict__ first, int64_t *__restrict__ last, DevStatus *ds)
{
    const double xo[3] = {xo0, xo1, xo2};
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        double gX[3], gXd[3], gXp[3], gsig;
        load_gs(gs, ldgs, ngs, s, gX, gXd, gXp, gsig);
        double out[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) out[k] = 0.0;
        out[9] = gsig;
        const double t = tau[s];
        if (mode == ISW_LINEAR) {
            const double D = t - t_box;
            double Xd[3], r[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Xd[k] = nodes[(3 + k) * ld + s];
                r[k] = nodes[k * ld + s] + Xd[k] * D - xo[k];
            }
            const double rn = sqrt(dot3(r, r));
            const double den = 1.0 + dot3(r, Xd) / rn;
            if (!(rn > 0.0) || !(den > 0.0)) {
                atomicOr(&ds->bits, kStatDomain);
            } else {
                const double lam = dot3(gX, Xd) / den;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double gam = gX[k] - lam * (r[k] / rn);
                    out[k] = gam;
                    out[3 + k] = gXd[k] + D * gam;
                    out[6 + k] = gXp[k];
                }
            }
        } else {
            const int64_t id = loop_id(nodes, s, nloops);
            if (id < 0) {
                atomicOr(&ds->bits, kStatBadIndex);
            } else {
                double gsigma = 0.0;
                if (burden_sample(P, ldp, id, nodes[ld + s], t, xo, gX, gXd, gXp, gsigma, nullptr)) out[1] = gsigma;
                else atomicOr(&ds->bits, kStatDomain);
                if (s == 0 || loop_id(nodes, s - 1, nloops) != id) {
                    atomicAdd(&runs[id], 1);
                    first[id] = s;
                }
                if (s == n - 1 || loop_id(nodes, s + 1, nloops) != id) last[id] = s + 1;
            }
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) gn[k * ldgn + s] = out[k];
    }
}

// Loop-parameter gradients: one warp per loop, lanes stride over the loop's samples, fixed
// butterfly reduction.  Rows: centre (3), rotation (9), L, m (0), n (0), psi, t0.
__global__ void k_lcadj_loops(const double *__restrict__ nodes, int64_t ld, const double *__restrict__ P,
                              int64_t nloops, int64_t ldp, double xo0, double xo1, double xo2,
                              const double *__restrict__ tau, const double *__restrict__ gs, int64_t ldgs, int ngs,
                              const int *__restrict__ runs, const int64_t *__restrict__ first,
                              const int64_t *__restrict__ last, double *__restrict__ gl, int64_t ldgl, DevStatus *ds)
{
    const double xo[3] = {xo0, xo1, xo2};
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t l = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); l < nloops; l += warps) {
        const int nr = runs[l];
        double acc[15];
#pragma unroll
        for (int q = 0; q < 15; ++q) acc[q] = 0.0;
        if (nr == 1) {
            for (int64_t s = first[l] + lane; s < last[l]; s += 32) {
                double gX[3], gXd[3], gXp[3], gsig, gsigma, contrib[15];
                load_gs(gs, ldgs, ngs, s, gX, gXd, gXp, gsig);
                if (burden_sample(P, ldp, l, nodes[ld + s], tau[s], xo, gX, gXd, gXp, gsigma, contrib)) {
#pragma unroll
                    for (int q = 0; q < 15; ++q) acc[q] += contrib[q];
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 15; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
        }
        if (nr > 1) {
            // the loop's samples are not contiguous: its gradient is undefined here
            if (lane == 0) atomicOr(&ds->bits, kStatBadIndex);
#pragma unroll
            for (int q = 0; q < 15; ++q) acc[q] = __longlong_as_double(0x7ff8000000000000ll);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 13; ++q) gl[q * ldgl + l] = acc[q];
            gl[13 * ldgl + l] = 0.0;
            gl[14 * ldgl + l] = 0.0;
            gl[15 * ldgl + l] = acc[13];
            gl[16 * ldgl + l] = acc[14];
        }
    }
}

void launch_lightcone_adjoint(int mode, const double *nodes, int64_t n, int64_t ld, const double *P, int64_t nloops,
                              int64_t ldp, double t_box, double xo0, double xo1, double xo2, const double *tau,
                              const double *gs, int64_t ldgs, int ngs, double *gn, int64_t ldgn, double *gl,
                              int64_t ldgl, int *runs, int64_t *first, int64_t *last, DevStatus *st, cudaStream_t s)
{
    if (n > 0) {
        int64_t b = (n + 127) / 128;
        if (b > 152 * 32) b = 152 * 32;
        k_lcadj_nodes<<<(unsigned)b, 128, 0, s>>>(mode, nodes, n, ld, P, nloops, ldp, t_box, xo0, xo1, xo2, tau, gs,
                                                  ldgs, ngs, gn, ldgn, runs, first, last, st);
    }
    if (mode == ISW_BURDEN && nloops > 0) {
        int64_t b = (nloops + 3) / 4;   // 4 warps per block
        if (b > 152 * 16) b = 152 * 16;
        k_lcadj_loops<<<(unsigned)b, 128, 0, s>>>(nodes, ld, P, nloops, ldp, xo0, xo1, xo2, tau, gs, ldgs, ngs, runs,
                                                  first, last, gl, ldgl, st);
    }
}

}  // namespace isw
