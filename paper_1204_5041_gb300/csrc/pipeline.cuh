// Device helpers shared by the pair kernels (map.cu, adjoint.cu): the FP64 pair term, the
// compensated folds, and the shared-memory stage ring fed by 1-D bulk copies.
#pragma once

#include "isw_internal.cuh"

namespace isw {

constexpr int kStages = 4;

// FP64 pair term (d = (n - Xhat_hi) - Xhat_lo keeps full relative accuracy near the string)
__device__ __forceinline__ double pair64(double nx, double ny, double nz, const Seg64 &g, unsigned &zero)
{
    const double dx = (nx - g.xh[0]) - g.xl[0];
    const double dy = (ny - g.xh[1]) - g.xl[1];
    const double dz = (nz - g.xh[2]) - g.xl[2];
    const double Q = dx * dx + dy * dy + dz * dz;
    if (Q == 0.0) {
        ++zero;
        return 0.0;
    }
    const double A = nx * g.xp[0] + ny * g.xp[1] + nz * g.xp[2];
    const double B = 1.0 + (nx * g.xd[0] + ny * g.xd[1] + nz * g.xd[2]);
    const double Pd = g.xd[0] * dx + g.xd[1] * dy + g.xd[2] * dz;
    const double Qd = g.xp[0] * dx + g.xp[1] * dy + g.xp[2] * dz;
    return g.c * (B * Pd - A * Qd) / (B * Q);
}

// 1/x for a nonzero normal double of either sign within the float range: the FP32 estimate r
// (relative error e = 1 - x r below ~2^-22) refined by one third-order step of the iteration for
// 1/x, r (1 + e + e^2) (error e^3 < 2^-66, below an ulp): three FP64 FMAs and two conversions
// instead of the IEEE division's longer sequence.
__device__ __forceinline__ double rcp64(double x)
{
    const double r = (double)rcp_approx((float)x);
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

__device__ __forceinline__ void fold(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

__device__ __forceinline__ void fold64(double &hi, double &lo, double x)
{
    const double s = hi + x;
    const double bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

// Issue the bulk copy of segment tile j into stage (load index gi) -- one thread.
template <typename Rec, int S>
__device__ __forceinline__ void issue_tile(Rec *sbuf, uint64_t *bars, const Rec *src, int64_t j, uint32_t gi)
{
    const int b = gi % kStages;
    mbar_arrive_expect_tx(&bars[b], (uint32_t)(S * sizeof(Rec)));
    bulk_g2s(sbuf + b * S, src + j * S, (uint32_t)(S * sizeof(Rec)), &bars[b]);
}

// After a consumer wait ran out (one thread): record the time-out, then wait for the stages
// i .. last-1 of this item, issued and not yet consumed, so that no bulk copy into this CTA's
// shared memory is still in flight when it exits.  These waits have their own limit
// (kDrainPolls), independent of the consumer limit; if one runs out as well, kStatDrain is
// recorded (the host reports it as a time-out with a copy possibly outstanding).  Kept out of
// line: the path is cold, and inlined into the pair kernels it slowed their loops by ~5%.
static __device__ __noinline__ void drain(uint64_t *bars, uint32_t g, int i, int last, DevStatus *st)
{
    atomicOr(&st->bits, kStatTimeout);
    for (int m = i; m < last; ++m) {
        const uint32_t gm = g + m;
        if (!mbar_wait_bounded(&bars[gm % kStages], (gm / kStages) & 1, kDrainPolls)) {
            atomicOr(&st->bits, kStatDrain);
            return;
        }
    }
}

// Dynamic work distribution: block-wide fetch of the next work item from
// a global counter.  Each item's arithmetic and output slots do not depend on which block takes
// it, so the result is the same as with a static assignment; only the load balance changes
// (near-field work is concentrated where pixels and strings are close).
__device__ __forceinline__ int64_t next_item(unsigned long long *counter, int64_t *slot)
{
    if (threadIdx.x == 0) *slot = (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t item = *slot;
    __syncthreads();
    return item;
}

}  // namespace isw
