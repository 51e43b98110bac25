// isw_map_f32c_noalloc: the FP32-compensated full map without any device allocation.
//
// Who needs it: callers that may not call cudaMalloc / cudaFree at all -- for example code
// embedded in a host framework that owns all device memory through its own pool and forbids
// raw CUDA allocations, or a latency-critical loop that cannot afford the implicit device
// synchronisation cudaMalloc and cudaFree may perform.  isw_map needs an isw_ctx, whose
// creation and workspace growth allocate; this entry point needs neither.
//
// Its scratch (pixel table, spatial sort of the samples, sample records, far- and mid-range records, tile caps,
// segment-chunk partials and the device status word) lives in one file-scope __device__ array of kStaticScratchBytes.
// Every GPU that loads the library holds that array until the process exits.  All calls
// share it and it keeps the previous call's contents: each call clears the status word and
// overwrites every other byte it reads, and two calls that overlap on the GPU (different
// streams, no ordering between them) race on it and give wrong maps.  The launch sequence,
// kernel variant and segment-chunk rule are those of isw_map with default settings (the chunk
// count is capped by the scratch left), so within that cap the map equals isw_map's bit for bit.
// A caller that passes status_out gets the status the kernels recorded (skipped samples, a
// bounded wait that ran out), read back after a stream synchronisation.
#include <cmath>
#include <mutex>

#include "isw_internal.cuh"
#include "kernels.cuh"

using namespace isw;

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB per device
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];  // device address of g_scratch, per device
int g_num_sms[kMaxDevices];

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Device memory of GPU `dev` (the current device), or managed memory: the kernels of this call
// run on `dev` and would fault on a host pointer or on another GPU's memory.
bool device_ptr(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Device-side conditions recorded in the status word, as a status code (time-outs first).
int status_code(const DevStatus &h)
{
    if (h.bits & (kStatTimeout | kStatDrain)) return ISW_ETIMEOUT;
    if (h.bits & kStatBadIndex) return ISW_EINVAL;
    if (h.bits & kStatDomain) return ISW_EDOMAIN;
    return ISW_OK;
}

// One-time set-up per device (the device must be current): the device address of the
// static array.  In host code g_scratch names a host-side stand-in, never the device memory.
int scratch_address(int dev, void **addr, int *sms)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return ISW_ECUDA;
        }
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return ISW_ECUDA;
        g_num_sms[dev] = n;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return ISW_OK;
}

}  // namespace

extern "C" int isw_map_f32c_noalloc(int64_t nside, int64_t pix0, int64_t npix, const double *samples, int64_t n,
                                    int64_t ld, const double *x_obs, double GU, double *theta_out, int32_t *status_out,
                                    void *stream)
{
    if (status_out) *status_out = ISW_OK;
    // ---- host-side checks (nothing is enqueued when they fail)
    if (nside < 1 || nside > (1 << 24)) return ISW_EINVAL;
    const int64_t all = 12 * nside * nside;
    if (pix0 < 0 || pix0 > all || npix < 0 || npix > all - pix0 || n < 0 || (n > 0 && ld < n)) return ISW_EINVAL;
    if (npix == 0) return ISW_OK;
    if (!theta_out || (n > 0 && !samples)) return ISW_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return ISW_ECUDA;
    }
    if (!device_ptr(theta_out, dev) || (n > 0 && !device_ptr(samples, dev))) return ISW_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(theta_out, 0, (size_t)npix * sizeof(double), s) == cudaSuccess ? ISW_OK
                                                                                                         : ISW_ECUDA;

    // ---- scratch layout for the FP32 pair kernel's first variant (the one isw_map uses by default)
    const Variant v = f32_variant(0);
    const int S = v.seg_tile, tile = v.tx * v.ty;
    const bool full = (pix0 == 0 && npix == all);
    const int64_t ntiles = full ? 12 * ((nside + v.tx - 1) / v.tx) * ((nside + v.ty - 1) / v.ty)
                                : (npix + tile - 1) / tile;
    const int64_t tot = ntiles * tile;
    const int64_t n_pad = (n + S - 1) / S * S, nst = n_pad / S;
    size_t off[8];
    size_t at = 0;
    off[0] = at; at += up256(sizeof(DevStatus));
    const size_t off_queue = at; at += up256(2 * sizeof(unsigned long long));
    off[1] = at; at += up256((size_t)tot * 3 * sizeof(double));
    off[2] = at; at += up256((size_t)tot * sizeof(int64_t));
    off[3] = at; at += up256((size_t)ntiles * sizeof(float4));
    off[4] = at; at += up256((size_t)n_pad * sizeof(Seg32));
    off[5] = at; at += up256((size_t)n_pad * sizeof(Seg64));
    off[6] = at; at += up256((size_t)nst * sizeof(SegCap));
    const size_t off_far = at; at += up256((size_t)(n_pad / 2) * sizeof(Far2));
    const size_t off_mid = at; at += up256((size_t)n_pad * sizeof(Mid2));
    const size_t off_sort = at; at += up256(sort_scratch_bytes(n));
    off[7] = at;
    if (at > kStaticScratchBytes) return ISW_EINVAL;  // problem too large for the static scratch
    // segment-chunk partials fit for at most `room` chunks
    const int64_t room = (int64_t)((kStaticScratchBytes - at) / ((size_t)tot * sizeof(double)));

    void *base = nullptr;
    int sms = 0;
    int r = scratch_address(dev, &base, &sms);
    if (r) return r;

    // segment chunks: the rule isw_map uses, capped by the scratch left
    const int slots = map_f32c_slots(0, sms);
    const int split = choose_split(ntiles, nst, slots, (int)(room < 64 ? room : 64), kMapItemsPerSlot);
    unsigned char *b = (unsigned char *)base;
    DevStatus *st = (DevStatus *)(b + off[0]);
    double *nv = (double *)(b + off[1]);
    int64_t *outidx = (int64_t *)(b + off[2]);
    float4 *pcaps = (float4 *)(b + off[3]);
    Seg32 *s32 = (Seg32 *)(b + off[4]);
    Seg64 *s64 = (Seg64 *)(b + off[5]);
    SegCap *scaps = (SegCap *)(b + off[6]);
    double *partial = (double *)(b + off[7]);

    // the status word and the two work counters are the only scratch read before it is written
    // in this call
    unsigned long long *queue = (unsigned long long *)(b + off_queue);
    if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) return ISW_ECUDA;
    if (cudaMemsetAsync(queue, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) return ISW_ECUDA;
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};
    const double theta_pix = std::sqrt(4.0 * M_PI / (12.0 * (double)nside * (double)nside));
    launch_pixel_table(nside, full ? 0 : 1, pix0, npix, nullptr, v.tx, v.ty, ntiles, nv, tot, outidx, pcaps, st, s);
    Far2 *far = (Far2 *)(b + off_far);
    const uint32_t *perm = launch_spatial_order(samples, n, ld, xo[0], xo[1], xo[2], b + off_sort, s);
    Mid2 *mid = (Mid2 *)(b + off_mid);
    launch_pack(samples, n, ld, xo[0], xo[1], xo[2], GU, theta_pix, kNearK, n_pad, perm, s32, s64, far, mid, nullptr, st,
                s);
    launch_seg_caps(s32, s64, n, n_pad, S, (float)kBMin, scaps, s);
    MapArgs a;
    a.nv = nv;
    a.ldn = tot;
    a.outidx = outidx;
    a.pcaps = pcaps;
    a.ntiles = ntiles;
    a.s32 = s32;
    a.s64 = s64;
    a.far = far;
    a.mid = mid;
    a.far64 = nullptr;
    a.scaps = scaps;
    a.nst = nst;
    a.split = split;
    a.b_min = (float)kBMin;
    a.d_far = (float)kDFar;
    a.theta = theta_out;
    a.partial = split > 1 ? partial : nullptr;
    a.accumulate = 0;
    a.st = st;
    a.tile_stride = 1;
    a.queue = queue;
    a.wait_polls = kWaitPolls;
    const int64_t items = ntiles * split;
    launch_map_f32c(0, a, (int)(items < slots ? items : slots), s);
    launch_map_f32c_near(0, a, sms, s);
    if (split > 1) launch_reduce_partials(a, tile, s);
    if (cudaGetLastError() != cudaSuccess) return ISW_ECUDA;
    if (status_out) {
        // what the kernels recorded: wait for them, then read the status word (no allocation)
        DevStatus h;
        if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return ISW_ECUDA;
        }
        *status_out = status_code(h);
    }
    return ISW_OK;
}
