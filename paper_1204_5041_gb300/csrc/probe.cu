// Throughput of the FP32 and FP64 fused multiply-add pipes of the context's GPU: the peaks the
// pair kernels are measured against.  Every thread runs eight independent chains
// x <- x * a + b (0 < a < 1, so the chains stay finite and normal) for `iters` steps; the result
// is stored only when `flag` is set, which it never is, so every FMA is kept and nothing is
// written.  One FMA counts two flops.
#include "isw_internal.cuh"
#include "kernels.cuh"

namespace isw {

namespace {
constexpr int kProbeThreads = 256, kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T a, T b, double *sink, int flag)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (flag) *sink = (double)s;
}
}  // namespace

// Best of `reps` timed launches (after one untimed launch), in flop/s.
int fma_probe(bool f64, int num_sms, double *sink, double *flops, cudaStream_t s)
{
    const void *fn = f64 ? (const void *)&k_fma_probe<double> : (const void *)&k_fma_probe<float>;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kProbeThreads, 0) != cudaSuccess || nb < 1) nb = 1;
    const int grid = nb * num_sms;
    // about 4 ms per launch at the nominal rates (FP32 ~40e12, FP64 ~0.6e12 FMA/s)
    const int iters = f64 ? 1024 : 65536;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ISW_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ISW_ECUDA;
    }
    double best = 0.0;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        if (f64) k_fma_probe<double><<<grid, kProbeThreads, 0, s>>>(iters, 0.999999, 1e-3, sink, 0);
        else k_fma_probe<float><<<grid, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-3f, sink, 0);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms > 0.f) {
            const double fl = 2.0 * (double)grid * kProbeThreads * (double)iters * kChains;
            const double r = fl / (ms * 1e-3);
            if (r > best) best = r;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return ISW_ECUDA;
    *flops = best;
    return ISW_OK;
}

}  // namespace isw
