// Angular power spectrum of a full-sky RING map (Sec. IV, Fig. 4 of the paper): spherical-
// harmonic analysis with uniform pixel weights, a_lm = (4 pi / N_pix) sum_p Theta_p Y*_lm(n_p),
// then C_l = (|a_l0|^2 + 2 sum_{m>=1} |a_lm|^2) / (2l + 1).
//   k_ring_dft   F_r(m) = sum_j Theta_rj exp(-i m phi_rj): one block per ring, one thread per m;
//                the phase advances by a complex rotation per pixel and is re-seeded from the
//                library's own sin/cos every 32 pixels (error stays at a few ulp)
//   k_alm        a_lm = (4 pi / N_pix) sum_r lambda_lm(z_r) F_r(m): one block per m, each thread a
//                few north/south ring pairs (lambda_lm(-z) = (-1)^(l+m) lambda_lm(z)), the
//                normalised Legendre recursion in l with (mantissa, 2^256 power) scaling so that
//                lambda_mm near the poles does not underflow; the sum over rings is a fixed-
//                order block reduction per l (deterministic)
//   k_cl         one thread per l, fixed order over m
// Cost: N_pix (l_max + 1) complex products for the ring sums (no FFT) and
// 2N (l_max + 1)^2 / 2 recursion steps.
#include "isw_internal.cuh"
#include "kernels.cuh"

namespace isw {

constexpr double kLScale = 1.157920892373162e77;   // 2^256
constexpr int kAlmThreads = 256, kAlmPairs = 8, kCoefChunk = 512;

struct RingGeom {
    double z, t0;   // z and the first pixel's phase in turns
    int64_t np, p0;
};

__device__ __forceinline__ RingGeom ring_geom(int64_t N, int64_t i)
{
    RingGeom g;
    const double N3 = 3.0 * (double)N * (double)N;
    if (i < N) {
        g.z = 1.0 - ((double)i * (double)i) / N3;
        g.np = 4 * i;
        g.p0 = 2 * i * (i - 1);
        g.t0 = 1.0 / (8.0 * (double)i);
    } else if (i <= 3 * N) {
        g.z = (4.0 * (double)N - 2.0 * (double)i) / (3.0 * (double)N);
        g.np = 4 * N;
        g.p0 = 2 * N * (N - 1) + (i - N) * 4 * N;
        g.t0 = ((i + N) & 1) ? 0.0 : 1.0 / (8.0 * (double)N);
    } else {
        const int64_t k = 4 * N - i;
        g.z = -(1.0 - ((double)k * (double)k) / N3);
        g.np = 4 * k;
        g.p0 = 12 * N * N - 2 * k * (k + 1);
        g.t0 = 1.0 / (8.0 * (double)k);
    }
    return g;
}

// F: double[2][nring][mmax+1] (re plane, im plane)
__global__ void k_ring_dft(int64_t N, const double *__restrict__ map, int64_t mmax, double *__restrict__ F)
{
    const int64_t nring = 4 * N - 1;
    const int64_t r = blockIdx.x;
    const RingGeom g = ring_geom(N, r + 1);
    const int64_t M1 = mmax + 1;
    for (int64_t m = threadIdx.x; m <= mmax; m += blockDim.x) {
        double sr = 0.0, si = 0.0;
        double s1, c1;   // exp(-i m 2 pi / np) per pixel step
        sincos_turns((double)(m % g.np) / (double)g.np, s1, c1);
        double c = 1.0, s = 0.0;
        for (int64_t j = 0; j < g.np; ++j) {
            if ((j & 31) == 0) {   // exact phase m (t0 + j/np), reduced by whole turns
                sincos_turns((double)((m * j) % g.np) / (double)g.np + (double)m * g.t0, s, c);
            }
            const double v = map[g.p0 + j];
            sr += v * c;
            si -= v * s;
            const double cn = c * c1 - s * s1, sn = s * c1 + c * s1;
            c = cn;
            s = sn;
        }
        F[r * M1 + m] = sr;
        F[(nring + r) * M1 + m] = si;
    }
}

// value * 2^(256 sc), normalised so that |value| stays in range
struct Scaled {
    double v;
    int sc;
};

// sin(theta)^m as a scaled value (repeated squaring with rescaling)
__device__ __forceinline__ Scaled pow_scaled(double x, int64_t m)
{
    Scaled r{1.0, 0}, b{x, 0};
    while (m > 0) {
        if (m & 1) {
            r.v *= b.v;
            r.sc += b.sc;
            while (r.v != 0.0 && fabs(r.v) < 1.0 / kLScale) { r.v *= kLScale; --r.sc; }
        }
        m >>= 1;
        if (m) {
            b.v *= b.v;
            b.sc *= 2;
            while (b.v != 0.0 && fabs(b.v) < 1.0 / kLScale) { b.v *= kLScale; --b.sc; }
        }
    }
    return r;
}

// alm: double[2][mmax+1][lmax+1]; one block per m
__global__ void __launch_bounds__(kAlmThreads) k_alm(int64_t N, const double *__restrict__ F, int64_t lmax,
                                                    double omega, double *__restrict__ alm)
{
    __shared__ double coef_a[kCoefChunk], coef_b[kCoefChunk];
    __shared__ double red[2][kAlmThreads / 32];
    const int64_t m = blockIdx.x, mmax = lmax, M1 = mmax + 1, L1 = lmax + 1;
    const int64_t nring = 4 * N - 1, npair = 2 * N;   // pairs (i, 4N - i), i = 1..2N; i = 2N alone
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // c_m = sqrt((2m+1)/(4 pi) prod_{k<=m} (2k-1)/(2k)) (no underflow: ~ m^(-1/4))
    double cm = sqrt(1.0 / (4.0 * kPi));
    for (int64_t k = 1; k <= m; ++k) cm *= sqrt((2.0 * k - 1.0) / (2.0 * k));
    cm *= sqrt(2.0 * m + 1.0);
    if (m & 1) cm = -cm;
    // per-thread ring pairs: state of the recursion
    double lp[kAlmPairs], lc[kAlmPairs], zz[kAlmPairs];
    int scp[kAlmPairs];
    double fsr[kAlmPairs], fsi[kAlmPairs], fdr[kAlmPairs], fdi[kAlmPairs];
#pragma unroll
    for (int q = 0; q < kAlmPairs; ++q) {
        const int64_t pidx = tid + (int64_t)q * kAlmThreads;
        lp[q] = lc[q] = 0.0;
        zz[q] = 0.0;
        scp[q] = 1;   // > 0: unused slot, contributes nothing
        fsr[q] = fsi[q] = fdr[q] = fdi[q] = 0.0;
        if (pidx < npair) {
            const int64_t i = pidx + 1;   // north ring (z >= 0)
            const int64_t rn = i - 1, rs = nring - i;
            const RingGeom g = ring_geom(N, i);
            zz[q] = g.z;
            const double an = F[rn * M1 + m], bn = F[(nring + rn) * M1 + m];
            double as = 0.0, bs = 0.0;
            if (rs != rn) {
                as = F[rs * M1 + m];
                bs = F[(nring + rs) * M1 + m];
            }
            fsr[q] = an + as;
            fsi[q] = bn + bs;
            fdr[q] = an - as;
            fdi[q] = bn - bs;
            const Scaled sm = pow_scaled(sqrt((1.0 - g.z) * (1.0 + g.z)), m);
            lc[q] = cm * sm.v;
            scp[q] = sm.sc;
            while (lc[q] != 0.0 && fabs(lc[q]) < 1.0 / kLScale) { lc[q] *= kLScale; --scp[q]; }
        }
    }
    for (int64_t l0 = m; l0 <= lmax; l0 += kCoefChunk) {
        __syncthreads();
        for (int k = tid; k < kCoefChunk; k += kAlmThreads) {
            const double ll = (double)(l0 + k), mm = (double)m;
            coef_a[k] = sqrt((4.0 * ll * ll - 1.0) / (ll * ll - mm * mm));
            coef_b[k] = sqrt(((2.0 * ll + 1.0) * (ll + mm - 1.0) * (ll - mm - 1.0)) /
                             ((2.0 * ll - 3.0) * (ll * ll - mm * mm)));
        }
        __syncthreads();
        const int64_t l1 = l0 + kCoefChunk <= lmax + 1 ? l0 + kCoefChunk : lmax + 1;
        for (int64_t l = l0; l < l1; ++l) {
            const bool even = ((l + m) & 1) == 0;
            double sr = 0.0, si = 0.0;
#pragma unroll
            for (int q = 0; q < kAlmPairs; ++q) {
                if (l > m) {
                    double ln;
                    if (l == m + 1) ln = zz[q] * sqrt(2.0 * m + 3.0) * lc[q];
                    else ln = zz[q] * coef_a[l - l0] * lc[q] - coef_b[l - l0] * lp[q];
                    lp[q] = lc[q];
                    lc[q] = ln;
                    if (scp[q] < 0 && fabs(lc[q]) > 1.0) {
                        lc[q] /= kLScale;
                        lp[q] /= kLScale;
                        ++scp[q];
                    }
                }
                if (scp[q] == 0) {
                    sr += lc[q] * (even ? fsr[q] : fdr[q]);
                    si += lc[q] * (even ? fsi[q] : fdi[q]);
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) {
                red[0][wid] = sr;
                red[1][wid] = si;
            }
            __syncthreads();
            if (tid == 0) {
                double tr = 0.0, ti = 0.0;
                for (int w = 0; w < kAlmThreads / 32; ++w) {
                    tr += red[0][w];
                    ti += red[1][w];
                }
                alm[m * L1 + l] = omega * tr;
                alm[M1 * L1 + m * L1 + l] = omega * ti;
            }
            __syncthreads();
        }
    }
}

__global__ void k_cl(const double *__restrict__ alm, int64_t lmax, double *__restrict__ cl)
{
    const int64_t L1 = lmax + 1, M1 = lmax + 1;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l <= lmax; l += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t m = 0; m <= l; ++m) {
            const double re = alm[m * L1 + l], im = alm[M1 * L1 + m * L1 + l];
            const double p = re * re + im * im;
            s += m == 0 ? p : 2.0 * p;
        }
        cl[l] = s / (2.0 * l + 1.0);
    }
}

int cl_max_nside() { return kAlmPairs * kAlmThreads / 2; }

void launch_map_cl(int64_t N, const double *map, int64_t lmax, double *F, double *alm, double *cl, cudaStream_t s)
{
    const int64_t nring = 4 * N - 1;
    k_ring_dft<<<(unsigned)nring, 256, 0, s>>>(N, map, lmax, F);
    // only l >= m is written: clear the plane so the unused triangle reads as zero
    cudaMemsetAsync(alm, 0, (size_t)2 * (lmax + 1) * (lmax + 1) * sizeof(double), s);
    k_alm<<<(unsigned)(lmax + 1), kAlmThreads, 0, s>>>(N, F, lmax, 4.0 * kPi / (12.0 * (double)N * (double)N), alm);
    int64_t b = (lmax + 256) / 256;
    k_cl<<<(unsigned)b, 256, 0, s>>>(alm, lmax, cl);
}

}  // namespace isw
