// C ABI of the library (include/isw.h): argument checks, workspace, launch sequences.
#include <cmath>
#include <vector>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "isw_internal.cuh"
#include "kernels.cuh"

using namespace isw;

namespace {

enum WsSlot {
    kWsNv = 0, kWsOut, kWsPcap, kWsS32, kWsS64, kWsScap, kWsPartial, kWsMisc,
    kWsP32, kWsP64, kWsAdjPartial, kWsSamples, kWsShell, kWsFar, kWsLoops, kWsQueue, kWsConeMeta, kWsCut, kWsFlat, kWsClF, kWsAlm, kWsPF2, kWsSort, kWsMid, kWsFar64, kWsCount
};
static_assert(kWsCount <= kMaxWorkspaces, "isw_ctx holds kMaxWorkspaces workspace slots");

int set_err(isw_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->last_error, sizeof(c->last_error), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_err(isw_ctx *c, cudaError_t e, const char *where)
{
    return set_err(c, e == cudaErrorMemoryAllocation ? ISW_ENOMEM : ISW_ECUDA, "%s: %s", where,
                   cudaGetErrorString(e));
}

// A pointer the context's kernels may read: device memory of the context's own GPU, or managed
// memory.  Host (even pinned) pointers are rejected because the kernels would read them over the
// bus or fault, and so is device memory of another GPU (no peer mapping is set up: a kernel
// reading it would fault).
bool is_device_ptr(const isw_ctx *c, const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == c->device;
}

void drop_graph(isw_ctx *c)
{
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    c->graph_key = 0;
}

int ensure_ws(isw_ctx *c, int slot, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (c->ws_size[slot] >= bytes) return ISW_OK;
    if (c->capturing) return set_err(c, ISW_ECUDA, "workspace growth during graph capture");
    drop_graph(c);  // a captured graph refers to the old buffers
    if (c->ws[slot]) {
        cudaError_t e = cudaFree(c->ws[slot]);
        c->ws[slot] = nullptr;
        c->ws_size[slot] = 0;
        if (e != cudaSuccess) return cuda_err(c, e, "cudaFree(workspace)");
    }
    const size_t grown = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&c->ws[slot], grown);
    if (e != cudaSuccess) {
        c->ws[slot] = nullptr;
        return cuda_err(c, e, "cudaMalloc(workspace)");
    }
    c->ws_size[slot] = grown;
    return ISW_OK;
}

int set_device(isw_ctx *c)
{
    cudaError_t e = cudaSetDevice(c->device);
    return e == cudaSuccess ? ISW_OK : cuda_err(c, e, "cudaSetDevice");
}

int check_launch(isw_ctx *c, const char *where)
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ISW_OK : cuda_err(c, e, where);
}

int check_pixels(isw_ctx *c, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list)
{
    if (nside < 1 || nside > (1 << 24)) return set_err(c, ISW_EINVAL, "nside %lld out of [1, 2^24]", (long long)nside);
    const int64_t all = 12 * nside * nside;
    if (npix < 0) return set_err(c, ISW_EINVAL, "npix < 0");
    if (pix_list) {
        if (npix > 0 && !is_device_ptr(c, pix_list)) return set_err(c, ISW_EINVAL, "pix_list is not a device pointer of the context's GPU");
    } else if (pix0 < 0 || pix0 > all || npix > all - pix0) {
        return set_err(c, ISW_EINVAL, "pixel range [%lld, %lld) outside [0, %lld)", (long long)pix0,
                       (long long)(pix0 + npix), (long long)all);
    }
    return ISW_OK;
}

int check_samples(isw_ctx *c, const double *samples, int64_t n, int64_t ld)
{
    if (n < 0) return set_err(c, ISW_EINVAL, "n < 0");
    if (n > 0 && ld < n) return set_err(c, ISW_EINVAL, "ld (%lld) < n (%lld)", (long long)ld, (long long)n);
    if (n > 0 && !is_device_ptr(c, samples)) return set_err(c, ISW_EINVAL, "samples is not a device pointer");
    return ISW_OK;
}

struct PixelPlan {
    int mode;          // 0 full sky (face tiles), 1 range, 2 list
    int tx, ty;
    int64_t ntiles, tot;
};

PixelPlan plan_pixels(int64_t N, int64_t pix0, int64_t npix, const int64_t *pix_list, const Variant &v)
{
    PixelPlan p;
    p.tx = v.tx;
    p.ty = v.ty;
    const int tile = v.tx * v.ty;
    if (!pix_list && pix0 == 0 && npix == 12 * N * N) {
        p.mode = 0;
        p.ntiles = 12 * ((N + p.tx - 1) / p.tx) * ((N + p.ty - 1) / p.ty);
    } else {
        p.mode = pix_list ? 2 : 1;
        p.ntiles = (npix + tile - 1) / tile;
    }
    p.tot = p.ntiles * tile;
    return p;
}

}  // namespace

// Number of segment chunks: enough work items to fill every resident CTA slot with
// near-equal waves, at least two segment tiles per chunk, at most max_split chunks.  With
// min_items > 0 the count then grows while there are fewer than min_items work items per slot
// and every chunk keeps at least min_chunk streamed tiles: items are taken from a global counter,
// so the last ones leave slots idle for about half an item's time, and shorter items shorten that
// tail (N_side 512 with 2e5 samples: 314 ms per map with 4 chunks, 310 ms with 8-12).
int isw::choose_split(int64_t ntiles, int64_t nst, int slots, int max_split, int min_items, int min_chunk)
{
    const double ideal = (double)ntiles / slots;
    int best = 1;
    double best_t = 1e300;
    for (int k = 1; k <= 64 && k <= max_split; ++k) {
        if (k > 1 && nst / k < 2) break;
        const int64_t items = ntiles * k;
        const double waves = (double)((items + slots - 1) / slots);
        const double t = waves / k;
        if (t < best_t * 0.98) {
            best_t = t;
            best = k;
        }
        if (t <= ideal * 1.01) break;
    }
    while (best < max_split && ntiles * best < (int64_t)min_items * slots && nst / (best + 1) >= min_chunk) ++best;
    return best;
}

namespace {

// Events around a pair-kernel launch when timing is on; returns the slot or -1.
int timing_begin(isw_ctx *c, cudaStream_t s)
{
    if (!c->timing || c->capturing || c->n_timed >= kMaxTimed) return -1;
    if (!c->ev) {
        c->ev = (cudaEvent_t *)calloc(2 * kMaxTimed, sizeof(cudaEvent_t));
        if (!c->ev) return -1;
    }
    const int k = c->n_timed;
    for (int e = 2 * k; e < 2 * k + 2; ++e)
        if (!c->ev[e] && cudaEventCreate(&c->ev[e]) != cudaSuccess) return -1;
    cudaEventRecord(c->ev[2 * k], s);
    return k;
}

void timing_end(isw_ctx *c, int k, cudaStream_t s)
{
    if (k < 0) return;
    cudaEventRecord(c->ev[2 * k + 1], s);
    c->n_timed = k + 1;
}

// Shared body of isw_map: pixel table, sample records, caps, map kernel, partial reduce.
int map_impl(isw_ctx *c, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list, const double *samples,
             int64_t n, int64_t ld, const double *x_obs, double GU, int prec, int accumulate, double *theta,
             cudaStream_t s, int64_t tune_waves = 0, int64_t *tuned_pixels = nullptr, const PatchSpec *patch = nullptr)
{
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};
    if (npix == 0) return ISW_OK;
    if (n == 0) {
        if (!accumulate) {
            cudaError_t e = cudaMemsetAsync(theta, 0, (size_t)npix * sizeof(double), s);
            if (e != cudaSuccess) return cuda_err(c, e, "cudaMemsetAsync");
        }
        return ISW_OK;
    }
    int vidx = 0;
    if (prec == ISW_F32C) {
        if (c->tile_override >= 0 && c->tile_override < num_f32_variants()) vidx = c->tile_override;
        else if (c->tuned_nside == nside && c->tuned_n == n) vidx = c->auto_variant;
    }
    if (prec == ISW_F32C && !c->capturing) c->last_variant = vidx;
    const Variant v = prec == ISW_F32C ? f32_variant(vidx) : f64_variant();
    const int S = v.seg_tile;
    PixelPlan pp = plan_pixels(nside, pix0, npix, pix_list, v);
    if (patch) {
        pp.mode = 3;
        pp.ntiles = ((patch->M + v.tx - 1) / v.tx) * ((patch->M + v.ty - 1) / v.ty);
        pp.tot = pp.ntiles * v.tx * v.ty;
    }
    const int64_t n_pad = (n + S - 1) / S * S;
    const int64_t nst = n_pad / S;
    const int slots = prec == ISW_F32C ? map_f32c_slots(vidx, c->num_sms) : map_f64_slots(c->num_sms);
    const int split = c->split_override > 0 ? c->split_override : choose_split(pp.ntiles, nst, slots, 64, kMapItemsPerSlot);
    int r;
    if ((r = ensure_ws(c, kWsNv, (size_t)pp.tot * 3 * sizeof(double)))) return r;
    if ((r = ensure_ws(c, kWsOut, (size_t)pp.tot * sizeof(int64_t)))) return r;
    if ((r = ensure_ws(c, kWsPcap, (size_t)pp.ntiles * sizeof(float4)))) return r;
    if ((r = ensure_ws(c, kWsS32, (size_t)n_pad * sizeof(Seg32)))) return r;
    if ((r = ensure_ws(c, kWsS64, (size_t)n_pad * sizeof(Seg64)))) return r;
    if ((r = ensure_ws(c, kWsScap, (size_t)nst * sizeof(SegCap)))) return r;
    if (prec == ISW_F32C && (r = ensure_ws(c, kWsFar, (size_t)(n_pad / 2) * sizeof(Far2)))) return r;
    if (prec == ISW_F32C && (r = ensure_ws(c, kWsMid, (size_t)n_pad * sizeof(Mid2)))) return r;
    if (prec == ISW_F64 && (r = ensure_ws(c, kWsFar64, (size_t)n_pad * sizeof(Far64)))) return r;
    if (split > 1 && (r = ensure_ws(c, kWsPartial, (size_t)split * pp.tot * sizeof(double)))) return r;
    if ((r = ensure_ws(c, kWsQueue, 2 * sizeof(unsigned long long)))) return r;
    if (prec == ISW_F32C && (r = ensure_ws(c, kWsSort, sort_scratch_bytes(n)))) return r;

    const double theta_pix = patch ? patch->width / (double)patch->M
                                   : std::sqrt(4.0 * M_PI / (12.0 * (double)nside * (double)nside));
    double *nv = (double *)c->ws[kWsNv];
    int64_t *outidx = (int64_t *)c->ws[kWsOut];
    float4 *pcaps = (float4 *)c->ws[kWsPcap];
    Seg32 *s32 = (Seg32 *)c->ws[kWsS32];
    Seg64 *s64 = (Seg64 *)c->ws[kWsS64];
    SegCap *scaps = (SegCap *)c->ws[kWsScap];

    if (patch) launch_patch_table(*patch, pp.tx, pp.ty, pp.ntiles, nv, pp.tot, outidx, pcaps, s);
    else launch_pixel_table(nside, pp.mode, pix0, npix, pix_list, pp.tx, pp.ty, pp.ntiles, nv, pp.tot, outidx,
                            pcaps, c->d_status, s);
    Far2 *far = prec == ISW_F32C ? (Far2 *)c->ws[kWsFar] : nullptr;
    Mid2 *mid = prec == ISW_F32C ? (Mid2 *)c->ws[kWsMid] : nullptr;
    Far64 *far64 = prec == ISW_F64 ? (Far64 *)c->ws[kWsFar64] : nullptr;
    // FP32 path: records in the spatial order of the samples (tight segment-tile caps)
    const uint32_t *perm = nullptr;
    if (prec == ISW_F32C) {
        perm = launch_spatial_order(samples, n, ld, xo[0], xo[1], xo[2], c->ws[kWsSort], s);
        c->n_launch += spatial_order_launches();
    }
    launch_pack(samples, n, ld, xo[0], xo[1], xo[2], GU, theta_pix, c->near_k, n_pad, perm, s32, s64, far, mid,
                far64, c->d_status, s);
    launch_seg_caps(s32, s64, n, n_pad, S, (float)c->b_min, scaps, s);
    c->n_launch += 4;

    MapArgs a;
    a.nv = nv;
    a.ldn = pp.tot;
    a.outidx = outidx;
    a.pcaps = pcaps;
    a.ntiles = pp.ntiles;
    a.s32 = s32;
    a.s64 = s64;
    a.far = far;
    a.mid = mid;
    a.far64 = far64;
    a.scaps = scaps;
    a.nst = nst;
    a.split = split;
    a.b_min = (float)c->b_min;
    a.d_far = (float)c->d_far;
    a.theta = theta;
    a.partial = split > 1 ? (double *)c->ws[kWsPartial] : nullptr;
    a.accumulate = accumulate;
    a.st = c->d_status;
    a.queue = (unsigned long long *)c->ws[kWsQueue];
    a.wait_polls = c->wait_polls;
    // timing a variant: every k-th pixel tile (all its segment chunks), about tune_waves waves
    a.tile_stride = 1;
    if (tune_waves > 0) {
        const int64_t want = tune_waves * slots / split;
        a.tile_stride = want > 0 && pp.ntiles > want ? pp.ntiles / want : 1;
    }
    const int64_t items = (pp.ntiles + a.tile_stride - 1) / a.tile_stride * split;
    const int grid = (int)(items < slots ? items : slots);
    if (tuned_pixels) *tuned_pixels = (pp.ntiles + a.tile_stride - 1) / a.tile_stride * (v.tx * v.ty);
    // the timed pair work: far pass (or the FP64 kernel), chunk reduce, near-field pass
    const int ti = timing_begin(c, s);
    cudaError_t e = cudaMemsetAsync(a.queue, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMemsetAsync(work counters)");
    if (prec == ISW_F32C) {
        launch_map_f32c(vidx, a, grid, s);
        // near-field pass: adds the segment tiles the far pass skipped, chunk by chunk
        launch_map_f32c_near(vidx, a, c->num_sms, s);
        c->n_launch += 2;
    } else {
        launch_map_f64(a, grid, s);
        c->n_launch += 1;
    }
    c->n_pair += 1;
    if (split > 1) {
        launch_reduce_partials(a, v.tx * v.ty, s);
        c->n_launch += 1;
    }
    timing_end(c, ti, s);
    return check_launch(c, "isw_map launch");
}

}  // namespace

extern "C" {

int isw_create(isw_ctx **out, int device)
{
    if (!out) return ISW_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ISW_EINVAL;
    }
    isw_ctx *c = (isw_ctx *)calloc(1, sizeof(isw_ctx));
    if (!c) return ISW_ENOMEM;
    c->device = device;
    c->near_k = kNearK;
    c->b_min = kBMin;
    c->d_far = kDFar;
    c->split_override = 0;
    c->tile_override = -1;
    c->wait_polls = kWaitPolls;
    c->tuned_nside = -1;
    c->last_variant = -1;
    c->meta_nshell = -1;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(DevStatus));
    if (e != cudaSuccess) {
        int code = e == cudaErrorMemoryAllocation ? ISW_ENOMEM : ISW_ECUDA;
        if (c->d_status) cudaFree(c->d_status);
        free(c);
        return code;
    }
    *out = c;
    return ISW_OK;
}

int isw_destroy(isw_ctx *c)
{
    if (!c) return ISW_EINVAL;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (int k = 0; k < kWsCount; ++k)
        if (c->ws[k]) cudaFree(c->ws[k]);
    if (c->ev) {
        for (int e = 0; e < 2 * kMaxTimed; ++e)
            if (c->ev[e]) cudaEventDestroy(c->ev[e]);
        free(c->ev);
    }
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->d_status) cudaFree(c->d_status);
    free(c);
    return ISW_OK;
}

const char *isw_last_error(const isw_ctx *c) { return c ? c->last_error : "null context"; }

int isw_set_param(isw_ctx *c, int key, double value)
{
    if (!c) return ISW_EINVAL;
    switch (key) {
    case ISW_PARAM_NEAR_K:
        if (!(value >= 0.0 && value < 1e6)) return set_err(c, ISW_EINVAL, "near_k out of range");
        c->near_k = value;
        return ISW_OK;
    case ISW_PARAM_B_MIN:
        if (!(value >= 0.0 && value <= 2.0)) return set_err(c, ISW_EINVAL, "b_min out of range");
        c->b_min = value;
        return ISW_OK;
    case ISW_PARAM_SPLIT:
        if (!(value >= 0.0 && value <= 1024.0)) return set_err(c, ISW_EINVAL, "split out of range");
        c->split_override = (int)value;
        return ISW_OK;
    case ISW_PARAM_D_FAR:
        if (!(value >= 0.0 && value <= 4.0)) return set_err(c, ISW_EINVAL, "d_far out of range");
        c->d_far = value;
        return ISW_OK;
    case ISW_PARAM_TIMING:
        c->timing = value != 0.0;
        return ISW_OK;
    case ISW_PARAM_VARIANT:
        if (!(value >= -1.0 && value < num_f32_variants())) return set_err(c, ISW_EINVAL, "variant out of range");
        c->tile_override = (int)value;
        return ISW_OK;
    case ISW_PARAM_WAIT_POLLS:
        if (value < 0.0) {
            c->wait_polls = kWaitPolls;
            return ISW_OK;
        }
        if (!(value <= 2147483648.0) || value != std::floor(value))
            return set_err(c, ISW_EINVAL, "wait polls must be an integer in [0, 2^31] (or < 0 for the default)");
        c->wait_polls = (uint32_t)value;
        return ISW_OK;
    default:
        return set_err(c, ISW_EINVAL, "unknown parameter key %d", key);
    }
}

int isw_get_param(const isw_ctx *c, int key, double *value)
{
    if (!c || !value) return ISW_EINVAL;
    switch (key) {
    case ISW_PARAM_NEAR_K: *value = c->near_k; return ISW_OK;
    case ISW_PARAM_B_MIN: *value = c->b_min; return ISW_OK;
    case ISW_PARAM_SPLIT: *value = c->split_override; return ISW_OK;
    case ISW_PARAM_VARIANT: *value = c->last_variant; return ISW_OK;
    case ISW_PARAM_TIMING: *value = c->timing; return ISW_OK;
    case ISW_PARAM_D_FAR: *value = c->d_far; return ISW_OK;
    case ISW_PARAM_NUM_VARIANTS: *value = num_f32_variants(); return ISW_OK;
    case ISW_PARAM_WAIT_POLLS: *value = c->wait_polls; return ISW_OK;
    default: return ISW_EINVAL;
    }
}

int isw_get_timing(isw_ctx *c, double *ms, int64_t *pair_launches, int64_t *all_launches, int reset)
{
    if (!c) return ISW_EINVAL;
    int r;
    if ((r = set_device(c))) return r;
    double tot = 0.0;
    for (int k = 0; k < c->n_timed; ++k) {
        cudaError_t e = cudaEventSynchronize(c->ev[2 * k + 1]);
        float x = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&x, c->ev[2 * k], c->ev[2 * k + 1]);
        if (e != cudaSuccess) return cuda_err(c, e, "timing events");
        tot += x;
    }
    if (ms) *ms = tot;
    if (pair_launches) *pair_launches = c->n_pair;
    if (all_launches) *all_launches = c->n_launch;
    if (reset) {
        c->n_timed = 0;
        c->n_pair = 0;
        c->n_launch = 0;
    }
    return ISW_OK;
}

int isw_fma_rate(isw_ctx *c, int prec, double *flop_per_s, void *stream)
{
    if (!c || !flop_per_s) return ISW_EINVAL;
    if (prec != ISW_F64 && prec != ISW_F32C) return set_err(c, ISW_EINVAL, "unknown precision %d", prec);
    int r;
    if ((r = set_device(c))) return r;
    if ((r = ensure_ws(c, kWsMisc, sizeof(double)))) return r;
    r = fma_probe(prec == ISW_F64, c->num_sms, (double *)c->ws[kWsMisc], flop_per_s, (cudaStream_t)stream);
    if (r) return set_err(c, r, "FMA throughput probe failed: %s", cudaGetErrorString(cudaGetLastError()));
    return ISW_OK;
}

int isw_check_status(isw_ctx *c, void *stream, int64_t *counts)
{
    if (!c) return ISW_EINVAL;
    int r;
    if ((r = set_device(c))) return r;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamSynchronize");
    DevStatus h;
    e = cudaMemcpy(&h, c->d_status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(DevStatus));
    if (e != cudaSuccess) return cuda_err(c, e, "status readback");
    if (counts) {
        counts[0] = (int64_t)h.zero_pairs;
        counts[1] = (int64_t)h.domain_segs;
        counts[2] = (int64_t)h.near_pairs;
    }
    if (h.bits & kStatDrain)
        return set_err(c, ISW_ETIMEOUT, "a bounded device wait ran out, and so did the wait for a block's copies in flight");
    if (h.bits & kStatTimeout) return set_err(c, ISW_ETIMEOUT, "a bounded device wait ran out (the map is incomplete)");
    if (h.bits & kStatNoConv) return set_err(c, ISW_ENOCONV, "a light-cone solve hit its iteration cap");
    if (h.bits & kStatBadIndex) return set_err(c, ISW_EINVAL, "a loop id or pixel index was out of range");
    if (h.bits & kStatDomain) return set_err(c, ISW_EDOMAIN, "a sample had 1 - Xdot^2 <= 0 or a non-finite weight");
    return ISW_OK;
}

int hp_pix2vec_ring(isw_ctx *c, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list, double *vec_out,
                    int64_t ld_out, void *stream)
{
    if (!c) return ISW_EINVAL;
    int r;
    if ((r = check_pixels(c, nside, pix0, npix, pix_list))) return r;
    if (npix == 0) return ISW_OK;
    if (ld_out < npix) return set_err(c, ISW_EINVAL, "ld_out < npix");
    if (!is_device_ptr(c, vec_out)) return set_err(c, ISW_EINVAL, "vec_out is not a device pointer");
    if ((r = set_device(c))) return r;
    launch_pix2vec(nside, pix0, npix, pix_list, vec_out, ld_out, c->d_status, (cudaStream_t)stream);
    c->n_launch += 1;
    return check_launch(c, "hp_pix2vec_ring launch");
}

int lightcone_intersect(isw_ctx *c, int mode, const double *nodes_in, int64_t n, int64_t ld, const double *loop_params,
                        int64_t nloops, int64_t ldp, double t_box, const double *x_obs, double t_obs,
                        double *samples_out, int64_t ld_out, double *tau_out, int32_t *status, void *stream)
{
    if (!c) return ISW_EINVAL;
    if (mode != ISW_LINEAR && mode != ISW_BURDEN) return set_err(c, ISW_EINVAL, "unknown mode %d", mode);
    int r;
    if ((r = check_samples(c, nodes_in, n, ld))) return r;
    if (n == 0) return ISW_OK;
    if (ld_out < n) return set_err(c, ISW_EINVAL, "ld_out < n");
    if (!is_device_ptr(c, samples_out)) return set_err(c, ISW_EINVAL, "samples_out is not a device pointer");
    if (tau_out && !is_device_ptr(c, tau_out)) return set_err(c, ISW_EINVAL, "tau_out is not a device pointer");
    if (status && !is_device_ptr(c, status)) return set_err(c, ISW_EINVAL, "status is not a device pointer");
    if (mode == ISW_LINEAR && !(t_obs > t_box)) return set_err(c, ISW_EINVAL, "t_obs must exceed t_box");
    if (mode == ISW_BURDEN) {
        if (nloops <= 0 || ldp < nloops || !is_device_ptr(c, loop_params))
            return set_err(c, ISW_EINVAL, "BURDEN mode needs device loop_params[17][ldp], ldp >= nloops > 0");
    }
    if (!(std::isfinite(t_obs))) return set_err(c, ISW_EINVAL, "t_obs not finite");
    if ((r = set_device(c))) return r;
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};
    const double tol = 4.0 * (std::nextafter(t_obs, INFINITY) - t_obs);
    launch_lightcone(mode, nodes_in, n, ld, loop_params, nloops, ldp, t_box, xo[0], xo[1], xo[2], t_obs, tol, 60,
                     samples_out, ld_out, tau_out, status, c->d_status, (cudaStream_t)stream);
    c->n_launch += 1;
    return check_launch(c, "lightcone_intersect launch");
}

int lightcone_adjoint(isw_ctx *c, int mode, const double *nodes_in, int64_t n, int64_t ld, const double *loop_params,
                      int64_t nloops, int64_t ldp, double t_box, const double *x_obs, const double *tau,
                      const double *grad_samples, int64_t ld_gs, int ngrad, double *grad_nodes, int64_t ld_gn,
                      double *grad_loops, int64_t ld_gl, void *stream)
{
    if (!c) return ISW_EINVAL;
    if (mode != ISW_LINEAR && mode != ISW_BURDEN) return set_err(c, ISW_EINVAL, "unknown mode %d", mode);
    int r;
    if ((r = check_samples(c, nodes_in, n, ld))) return r;
    if (ngrad != 6 && ngrad != 9 && ngrad != 10) return set_err(c, ISW_EINVAL, "ngrad must be 6, 9 or 10");
    if (mode == ISW_BURDEN) {
        if (nloops <= 0 || ldp < nloops || !is_device_ptr(c, loop_params))
            return set_err(c, ISW_EINVAL, "BURDEN mode needs device loop_params[17][ldp], ldp >= nloops > 0");
        if (ld_gl < nloops || !is_device_ptr(c, grad_loops))
            return set_err(c, ISW_EINVAL, "BURDEN mode needs device grad_loops[17][ld_gl], ld_gl >= nloops");
    }
    if (n > 0) {
        if (ld_gs < n || ld_gn < n) return set_err(c, ISW_EINVAL, "ld_gs and ld_gn must be >= n");
        if (!is_device_ptr(c, tau) || !is_device_ptr(c, grad_samples) || !is_device_ptr(c, grad_nodes))
            return set_err(c, ISW_EINVAL, "tau, grad_samples and grad_nodes must be device pointers");
    }
    if (mode == ISW_LINEAR && !std::isfinite(t_box)) return set_err(c, ISW_EINVAL, "t_box not finite");
    if ((r = set_device(c))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    int *runs = nullptr;
    int64_t *first = nullptr, *last = nullptr;
    if (mode == ISW_BURDEN) {
        const size_t nl = (size_t)nloops;
        if ((r = ensure_ws(c, kWsLoops, nl * (2 * sizeof(int64_t) + sizeof(int)) + 16))) return r;
        first = (int64_t *)c->ws[kWsLoops];
        last = first + nl;
        runs = (int *)(last + nl);
        cudaError_t e = cudaMemsetAsync(runs, 0, nl * sizeof(int), s);
        if (e != cudaSuccess) return cuda_err(c, e, "cudaMemsetAsync");
    }
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};
    launch_lightcone_adjoint(mode, nodes_in, n, ld, loop_params, nloops, ldp, t_box, xo[0], xo[1], xo[2], tau,
                             grad_samples, ld_gs, ngrad, grad_nodes, ld_gn, grad_loops, ld_gl, runs, first, last,
                             c->d_status, s);
    c->n_launch += (n > 0 ? 1 : 0) + (mode == ISW_BURDEN ? 1 : 0);
    return check_launch(c, "lightcone_adjoint launch");
}

int hp_vec2pix_ring(isw_ctx *c, int64_t nside, const double *vec, int64_t n, int64_t ld, int64_t *pix_out,
                    void *stream)
{
    if (!c) return ISW_EINVAL;
    if (nside < 1 || nside > (1 << 24)) return set_err(c, ISW_EINVAL, "nside out of range");
    if (n < 0) return set_err(c, ISW_EINVAL, "n < 0");
    if (n == 0) return ISW_OK;
    if (ld < n) return set_err(c, ISW_EINVAL, "ld < n");
    if (!is_device_ptr(c, vec) || !is_device_ptr(c, pix_out)) return set_err(c, ISW_EINVAL, "vec and pix_out must be device pointers");
    int r;
    if ((r = set_device(c))) return r;
    launch_vec2pix(nside, vec, n, ld, pix_out, c->d_status, (cudaStream_t)stream);
    c->n_launch += 1;
    return check_launch(c, "hp_vec2pix_ring launch");
}

// Host metadata for the stacking calls: copied to the context's device workspace after the
// stream has drained (earlier work on it may still read the previous copy).
static int upload_meta(isw_ctx *c, cudaStream_t s, const void *const *src, const size_t *bytes, int nsrc, void **dst)
{
    size_t tot = 0;
    for (int i = 0; i < nsrc; ++i) tot += (bytes[i] + 255) / 256 * 256;
    int r;
    if ((r = ensure_ws(c, kWsConeMeta, tot))) return r;
    cudaError_t e = cudaStreamSynchronize(s);
    unsigned char *p = (unsigned char *)c->ws[kWsConeMeta];
    for (int i = 0; i < nsrc && e == cudaSuccess; ++i) {
        dst[i] = p;
        if (bytes[i]) e = cudaMemcpy(p, src[i], bytes[i], cudaMemcpyHostToDevice);
        p += (bytes[i] + 255) / 256 * 256;
    }
    return e == cudaSuccess ? ISW_OK : cuda_err(c, e, "metadata upload");
}

int box_place(isw_ctx *c, const double *nodes_box, int64_t ld_box, const int64_t *box_off, int64_t nbox,
              const int64_t *shell_box, int64_t nshell, const double *place, double *nodes_out, int64_t ld_out,
              int64_t *shell_off_out, void *stream)
{
    if (!c) return ISW_EINVAL;
    if (nbox < 1 || nshell < 0 || !box_off || (nshell > 0 && (!shell_box || !shell_off_out)))
        return set_err(c, ISW_EINVAL, "box_off (host, nbox + 1), shell_box and shell_off_out (host) are required");
    if (box_off[0] != 0) return set_err(c, ISW_EINVAL, "box_off[0] must be 0");
    for (int64_t b = 0; b < nbox; ++b)
        if (box_off[b + 1] < box_off[b]) return set_err(c, ISW_EINVAL, "box_off must be non-decreasing");
    std::vector<int64_t> off(nshell + 1), start(nshell > 0 ? nshell : 1);
    off[0] = 0;
    for (int64_t k = 0; k < nshell; ++k) {
        const int64_t b = shell_box[k];
        if (b < 0 || b >= nbox) return set_err(c, ISW_EINVAL, "shell_box[%lld] out of range", (long long)k);
        start[k] = box_off[b];
        off[k + 1] = off[k] + (box_off[b + 1] - box_off[b]);
    }
    for (int64_t k = 0; k <= nshell; ++k) shell_off_out[k] = off[k];
    const int64_t n_out = off[nshell];
    if (n_out == 0) return ISW_OK;
    if (ld_box < box_off[nbox] || ld_out < n_out) return set_err(c, ISW_EINVAL, "ld_box or ld_out too small");
    if (!is_device_ptr(c, nodes_box) || !is_device_ptr(c, place) || !is_device_ptr(c, nodes_out))
        return set_err(c, ISW_EINVAL, "nodes_box, place and nodes_out must be device pointers");
    int r;
    if ((r = set_device(c))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    const void *src[2] = {off.data(), start.data()};
    const size_t bytes[2] = {(size_t)(nshell + 1) * 8, (size_t)nshell * 8};
    void *dst[2];
    if ((r = upload_meta(c, s, src, bytes, 2, dst))) return r;
    launch_box_place(nodes_box, ld_box, (const int64_t *)dst[0], (const int64_t *)dst[1], nshell, place, nodes_out,
                     ld_out, n_out, s);
    c->n_launch += 1;
    return check_launch(c, "box_place launch");
}

int lightcone_intersect_shells(isw_ctx *c, const double *nodes, int64_t ld, const int64_t *shell_off, int64_t nshell,
                               const double *t_box, const int32_t *mode, const double *loop_params, int64_t nloops,
                               int64_t ldp, const double *x_obs, double t_obs, double *samples_out, int64_t ld_out,
                               void *stream)
{
    if (!c) return ISW_EINVAL;
    if (nshell < 1 || !shell_off || !t_box || !mode)
        return set_err(c, ISW_EINVAL, "shell_off, t_box and mode (host arrays) are required");
    if (shell_off[0] != 0) return set_err(c, ISW_EINVAL, "shell_off[0] must be 0");
    bool burden = false;
    for (int64_t k = 0; k < nshell; ++k) {
        if (shell_off[k + 1] < shell_off[k]) return set_err(c, ISW_EINVAL, "shell_off must be non-decreasing");
        if (mode[k] != ISW_LINEAR && mode[k] != ISW_BURDEN) return set_err(c, ISW_EINVAL, "unknown mode");
        if (mode[k] == ISW_LINEAR && !(t_obs > t_box[k])) return set_err(c, ISW_EINVAL, "t_obs must exceed t_box");
        burden = burden || mode[k] == ISW_BURDEN;
    }
    const int64_t n = shell_off[nshell];
    int r;
    if ((r = check_samples(c, nodes, n, ld))) return r;
    if (n == 0) return ISW_OK;
    if (ld_out < n || !is_device_ptr(c, samples_out)) return set_err(c, ISW_EINVAL, "samples_out: device, ld_out >= n");
    if (burden && (nloops <= 0 || ldp < nloops || !is_device_ptr(c, loop_params)))
        return set_err(c, ISW_EINVAL, "BURDEN shells need device loop_params[17][ldp], ldp >= nloops > 0");
    if (!std::isfinite(t_obs)) return set_err(c, ISW_EINVAL, "t_obs not finite");
    if ((r = set_device(c))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    const void *src[3] = {shell_off, t_box, mode};
    const size_t bytes[3] = {(size_t)(nshell + 1) * 8, (size_t)nshell * 8, (size_t)nshell * 4};
    void *dst[3];
    if ((r = upload_meta(c, s, src, bytes, 3, dst))) return r;
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};
    const double tol = 4.0 * (std::nextafter(t_obs, INFINITY) - t_obs);
    launch_lightcone_shells(nodes, n, ld, (const int64_t *)dst[0], nshell, (const double *)dst[1],
                            (const int32_t *)dst[2], loop_params, nloops, ldp, xo[0], xo[1], xo[2], t_obs, tol,
                            samples_out, ld_out, c->d_status, s);
    c->n_launch += 1;
    return check_launch(c, "lightcone_intersect_shells launch");
}

int cone_cut(isw_ctx *c, const double *samples, int64_t ld, const int64_t *shell_off, int64_t nshell, int64_t nside_hz,
             const int64_t *cone_pix, const double *r_lo, const double *r_hi, const double *x_obs,
             double *samples_out, int64_t ld_out, int64_t *shell_off_out, int64_t *count, void *stream)
{
    if (!c) return ISW_EINVAL;
    if (nshell < 1 || !shell_off) return set_err(c, ISW_EINVAL, "shell_off (host, nshell + 1) is required");
    if (nside_hz < 1 || nside_hz > (1 << 24)) return set_err(c, ISW_EINVAL, "nside_hz out of range");
    if (shell_off[0] != 0) return set_err(c, ISW_EINVAL, "shell_off[0] must be 0");
    for (int64_t k = 0; k < nshell; ++k)
        if (shell_off[k + 1] < shell_off[k]) return set_err(c, ISW_EINVAL, "shell_off must be non-decreasing");
    const int64_t n = shell_off[nshell];
    int r;
    if ((r = check_samples(c, samples, n, ld))) return r;
    if (!is_device_ptr(c, cone_pix) || !is_device_ptr(c, r_lo) || !is_device_ptr(c, r_hi) || !is_device_ptr(c, shell_off_out))
        return set_err(c, ISW_EINVAL, "cone_pix, r_lo, r_hi and shell_off_out must be device pointers");
    if (n > 0 && (ld_out < n || !is_device_ptr(c, samples_out)))
        return set_err(c, ISW_EINVAL, "samples_out: device, ld_out >= n");
    if ((r = set_device(c))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    const void *src[1] = {shell_off};
    const size_t bytes[1] = {(size_t)(nshell + 1) * 8};
    void *dst[1];
    if ((r = upload_meta(c, s, src, bytes, 1, dst))) return r;
    const int64_t nb = cone_cut_scratch_blocks(n);
    const size_t incl_bytes = ((size_t)(n > 0 ? n : 1) * 4 + 255) / 256 * 256;
    if ((r = ensure_ws(c, kWsCut, incl_bytes + (size_t)(nb + 2) * 8))) return r;
    int32_t *incl = (int32_t *)c->ws[kWsCut];
    int64_t *block_tot = (int64_t *)((unsigned char *)c->ws[kWsCut] + incl_bytes);
    int64_t *d_count = block_tot + nb + 1;
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};
    launch_cone_cut(samples, ld, n, (const int64_t *)dst[0], nshell, nside_hz, cone_pix, r_lo, r_hi, xo[0], xo[1],
                    xo[2], incl, block_tot, samples_out, ld_out, shell_off_out, d_count, s);
    c->n_launch += n > 0 ? 4 : 2;
    if ((r = check_launch(c, "cone_cut launch"))) return r;
    if (count) {
        cudaError_t e = cudaMemcpyAsync(count, d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(c, e, "cone_cut count");
    }
    return ISW_OK;
}

int isw_map_patch(isw_ctx *c, const double *frame, int64_t M, double width, const double *samples, int64_t n,
                  int64_t ld, const double *x_obs, double GU, int prec, int approx, int accumulate, double *theta_out,
                  void *stream)
{
    if (!c) return ISW_EINVAL;
    if (!frame) return set_err(c, ISW_EINVAL, "frame (host double[9]) is required");
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double d = frame[3 * a] * frame[3 * b] + frame[3 * a + 1] * frame[3 * b + 1] +
                             frame[3 * a + 2] * frame[3 * b + 2];
            if (!(std::fabs(d - (a == b ? 1.0 : 0.0)) < 1e-9)) return set_err(c, ISW_EINVAL, "frame is not orthonormal");
        }
    if (M < 1 || M > (1 << 20)) return set_err(c, ISW_EINVAL, "M out of range");
    if (!(width > 0.0) || !std::isfinite(width)) return set_err(c, ISW_EINVAL, "width must be positive");
    if (prec != ISW_F64 && prec != ISW_F32C) return set_err(c, ISW_EINVAL, "unknown precision %d", prec);
    if (approx != ISW_FULLSKY && approx != ISW_FLATSKY) return set_err(c, ISW_EINVAL, "unknown approximation %d", approx);
    int r;
    if ((r = check_samples(c, samples, n, ld))) return r;
    if (!is_device_ptr(c, theta_out)) return set_err(c, ISW_EINVAL, "theta_out is not a device pointer");
    if (!std::isfinite(GU)) return set_err(c, ISW_EINVAL, "GU not finite");
    if ((r = set_device(c))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    PatchSpec p;
    for (int k = 0; k < 9; ++k) p.frame[k] = frame[k];
    p.M = M;
    p.width = width;
    const int64_t npix = M * M;
    if (approx == ISW_FULLSKY)
        return map_impl(c, 0, 0, npix, nullptr, samples, n, ld, x_obs, GU, prec, accumulate, theta_out, s, 0, nullptr,
                        &p);
    if (n == 0) {
        if (!accumulate) {
            cudaError_t e = cudaMemsetAsync(theta_out, 0, (size_t)npix * sizeof(double), s);
            if (e != cudaSuccess) return cuda_err(c, e, "cudaMemsetAsync");
        }
        return ISW_OK;
    }
    const bool f64 = prec == ISW_F64;
    const int S = flat_seg_tile(), tx = flat_tx(), ty = flat_ty();
    const int64_t ntiles = ((M + tx - 1) / tx) * ((M + ty - 1) / ty), tot = ntiles * tx * ty;
    const int64_t n_pad = (n + S - 1) / S * S, nst = n_pad / S;
    const int slots = flat_slots(f64, c->num_sms);
    const int split = c->split_override > 0 ? c->split_override : choose_split(ntiles, nst, slots, 64);
    if ((r = ensure_ws(c, kWsNv, (size_t)tot * 3 * sizeof(double)))) return r;
    if ((r = ensure_ws(c, kWsOut, (size_t)tot * sizeof(int64_t)))) return r;
    if ((r = ensure_ws(c, kWsPcap, (size_t)ntiles * sizeof(float4)))) return r;
    if ((r = ensure_ws(c, kWsFlat, (size_t)n_pad * flat_record_bytes()))) return r;
    if ((r = ensure_ws(c, kWsQueue, 2 * sizeof(unsigned long long)))) return r;
    if (split > 1 && (r = ensure_ws(c, kWsPartial, (size_t)split * tot * sizeof(double)))) return r;
    double *nv = (double *)c->ws[kWsNv];
    int64_t *outidx = (int64_t *)c->ws[kWsOut];
    unsigned char *rec = (unsigned char *)c->ws[kWsFlat];
    void *r32 = rec, *r64 = rec + (size_t)n_pad * (flat_record_bytes() / 2);
    unsigned long long *queue = (unsigned long long *)c->ws[kWsQueue];
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};
    launch_patch_table(p, tx, ty, ntiles, nv, tot, outidx, (float4 *)c->ws[kWsPcap], s);
    launch_flat_pack(samples, n, ld, p, xo[0], xo[1], xo[2], GU, n_pad, r32, r64, s);
    c->n_launch += 3;
    const int64_t items = ntiles * split;
    const int grid = (int)(items < slots ? items : slots);
    const int ti = timing_begin(c, s);
    cudaError_t e = cudaMemsetAsync(queue, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMemsetAsync(work counters)");
    launch_map_flat(f64, r32, r64, outidx, ntiles, nst, split, M, width / (double)M, theta_out,
                    split > 1 ? (double *)c->ws[kWsPartial] : nullptr, accumulate, c->d_status, queue, c->wait_polls,
                    grid, s);
    c->n_launch += 1;
    c->n_pair += 1;
    if (split > 1) {
        MapArgs a{};
        a.outidx = outidx;
        a.ntiles = ntiles;
        a.split = split;
        a.theta = theta_out;
        a.partial = (double *)c->ws[kWsPartial];
        a.accumulate = accumulate;
        launch_reduce_partials(a, tx * ty, s);
        c->n_launch += 1;
    }
    timing_end(c, ti, s);
    return check_launch(c, "isw_map_patch launch");
}

int isw_map_cl(isw_ctx *c, int64_t nside, const double *theta, int64_t lmax, double *alm, double *cl, void *stream)
{
    if (!c) return ISW_EINVAL;
    if (nside < 1 || nside > cl_max_nside()) return set_err(c, ISW_EINVAL, "nside must be in [1, %d]", cl_max_nside());
    if (lmax < 0 || lmax > 4 * nside) return set_err(c, ISW_EINVAL, "lmax must be in [0, 4 nside]");
    if (!is_device_ptr(c, theta) || !is_device_ptr(c, cl) || (alm && !is_device_ptr(c, alm)))
        return set_err(c, ISW_EINVAL, "theta, cl (and alm when given) must be device pointers");
    int r;
    if ((r = set_device(c))) return r;
    const size_t L1 = (size_t)lmax + 1;
    if ((r = ensure_ws(c, kWsClF, 2 * (size_t)(4 * nside - 1) * L1 * sizeof(double)))) return r;
    if (!alm) {
        if ((r = ensure_ws(c, kWsAlm, 2 * L1 * L1 * sizeof(double)))) return r;
        alm = (double *)c->ws[kWsAlm];
    }
    launch_map_cl(nside, theta, lmax, (double *)c->ws[kWsClF], alm, cl, (cudaStream_t)stream);
    c->n_launch += 3;
    return check_launch(c, "isw_map_cl launch");
}

int isw_map(isw_ctx *c, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list, const double *samples,
            int64_t n, int64_t ld, const double *x_obs, double GU, int prec, int accumulate, double *theta_out,
            void *stream)
{
    if (!c) return ISW_EINVAL;
    int r;
    if ((r = check_pixels(c, nside, pix0, npix, pix_list))) return r;
    if ((r = check_samples(c, samples, n, ld))) return r;
    if (prec != ISW_F64 && prec != ISW_F32C) return set_err(c, ISW_EINVAL, "unknown precision %d", prec);
    if (npix > 0 && !is_device_ptr(c, theta_out)) return set_err(c, ISW_EINVAL, "theta_out is not a device pointer");
    if (!std::isfinite(GU)) return set_err(c, ISW_EINVAL, "GU not finite");
    if ((r = set_device(c))) return r;
    return map_impl(c, nside, pix0, npix, pix_list, samples, n, ld, x_obs, GU, prec, accumulate, theta_out,
                    (cudaStream_t)stream);
}

int isw_map_adjoint(isw_ctx *c, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list,
                    const double *samples, int64_t n, int64_t ld, const double *x_obs, double GU, int prec,
                    const double *dL_dtheta, double *grad_out, int64_t ld_g, int ngrad, void *stream)
{
    if (!c) return ISW_EINVAL;
    int r;
    if ((r = check_pixels(c, nside, pix0, npix, pix_list))) return r;
    if ((r = check_samples(c, samples, n, ld))) return r;
    if (prec != ISW_F64 && prec != ISW_F32C) return set_err(c, ISW_EINVAL, "unknown precision %d", prec);
    if (ngrad != 6 && ngrad != 9 && ngrad != 10) return set_err(c, ISW_EINVAL, "ngrad must be 6, 9 or 10");
    if (n == 0) return ISW_OK;
    if (ld_g < n) return set_err(c, ISW_EINVAL, "ld_g < n");
    if (!is_device_ptr(c, grad_out)) return set_err(c, ISW_EINVAL, "grad_out is not a device pointer");
    if (npix > 0 && !is_device_ptr(c, dL_dtheta)) return set_err(c, ISW_EINVAL, "dL_dtheta is not a device pointer");
    if (!std::isfinite(GU)) return set_err(c, ISW_EINVAL, "GU not finite");
    if ((r = set_device(c))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    if (npix == 0) {
        for (int k = 0; k < ngrad; ++k) {
            cudaError_t e = cudaMemsetAsync(grad_out + (int64_t)k * ld_g, 0, (size_t)n * sizeof(double), s);
            if (e != cudaSuccess) return cuda_err(c, e, "cudaMemsetAsync");
        }
        return ISW_OK;
    }
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};
    const int NT = adj_seg_tile(prec), TP = adj_pix_tile(prec);
    const Variant pv{0, 0, 0, 32, TP / 32};
    const PixelPlan pp = plan_pixels(nside, pix0, npix, pix_list, pv);
    const int64_t n_pad = (n + NT - 1) / NT * NT;
    const int64_t nseg_tiles = n_pad / NT;
    const int slots = adj_slots(prec, ngrad, c->num_sms);
    int split = c->split_override > 0 ? c->split_override
                                      : choose_split(nseg_tiles, pp.ntiles, slots, 64, kAdjItemsPerSlot, kAdjMinChunk);
    if (split > pp.ntiles) split = (int)pp.ntiles;
    if ((r = ensure_ws(c, kWsNv, (size_t)pp.tot * 3 * sizeof(double)))) return r;
    if ((r = ensure_ws(c, kWsOut, (size_t)pp.tot * sizeof(int64_t)))) return r;
    if ((r = ensure_ws(c, kWsPcap, (size_t)pp.ntiles * sizeof(float4)))) return r;
    if ((r = ensure_ws(c, kWsP32, (size_t)pp.tot * sizeof(Pix32)))) return r;
    if ((r = ensure_ws(c, kWsP64, (size_t)pp.tot * sizeof(Pix64)))) return r;
    if ((r = ensure_ws(c, kWsPF2, (size_t)(pp.tot / 2) * sizeof(PixF2)))) return r;
    if ((r = ensure_ws(c, kWsS32, (size_t)n_pad * sizeof(Seg32)))) return r;
    if ((r = ensure_ws(c, kWsS64, (size_t)n_pad * sizeof(Seg64)))) return r;
    if ((r = ensure_ws(c, kWsScap, (size_t)nseg_tiles * sizeof(SegCap)))) return r;
    if (split > 1 && (r = ensure_ws(c, kWsAdjPartial, (size_t)split * ngrad * n_pad * sizeof(double)))) return r;
    if ((r = ensure_ws(c, kWsQueue, 2 * sizeof(unsigned long long)))) return r;
    const double theta_pix = std::sqrt(4.0 * M_PI / (12.0 * (double)nside * (double)nside));
    double *nv = (double *)c->ws[kWsNv];
    int64_t *outidx = (int64_t *)c->ws[kWsOut];
    float4 *pcaps = (float4 *)c->ws[kWsPcap];
    Pix32 *p32 = (Pix32 *)c->ws[kWsP32];
    Pix64 *p64 = (Pix64 *)c->ws[kWsP64];
    Seg32 *s32 = (Seg32 *)c->ws[kWsS32];
    Seg64 *s64 = (Seg64 *)c->ws[kWsS64];
    SegCap *scaps = (SegCap *)c->ws[kWsScap];
    launch_pixel_table(nside, pp.mode, pix0, npix, pix_list, pp.tx, pp.ty, pp.ntiles, nv, pp.tot, outidx, pcaps,
                       c->d_status, s);
    PixF2 *pf2 = (PixF2 *)c->ws[kWsPF2];
    launch_pack_pixels(nv, pp.tot, outidx, dL_dtheta, pp.tot, p32, p64, pf2, s);
    launch_pack(samples, n, ld, xo[0], xo[1], xo[2], GU, theta_pix, c->near_k, n_pad, nullptr, s32, s64, nullptr,
                nullptr, nullptr, c->d_status, s);
    c->n_launch += 4;
    launch_seg_caps(s32, s64, n, n_pad, NT, (float)c->b_min, scaps, s);
    c->n_launch += 1;
    AdjArgs a;
    a.p32 = p32;
    a.p64 = p64;
    a.pf2 = pf2;
    a.pcaps = pcaps;
    a.npix_tiles = pp.ntiles;
    a.s32 = s32;
    a.s64 = s64;
    a.scaps = scaps;
    a.nseg_tiles = nseg_tiles;
    a.n = n;
    a.n_pad = n_pad;
    a.split = split;
    a.ngrad = ngrad;
    a.b_min = (float)c->b_min;
    a.d_far = (float)c->d_far;
    a.grad = grad_out;
    a.ld_g = ld_g;
    a.partial = split > 1 ? (double *)c->ws[kWsAdjPartial] : nullptr;
    a.st = c->d_status;
    a.queue = (unsigned long long *)c->ws[kWsQueue];
    a.wait_polls = c->wait_polls;
    const int64_t items = nseg_tiles * split;
    const int grid = (int)(items < slots ? items : slots);
    const int ti = timing_begin(c, s);
    cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaMemsetAsync(work counter)");
    launch_adjoint(prec, a, grid, s);
    timing_end(c, ti, s);
    c->n_pair += 1;
    c->n_launch += split > 1 ? 2 : 1;
    return check_launch(c, "isw_map_adjoint launch");
}

int isw_map_batched(isw_ctx *c, int64_t nside, const double *nodes, int64_t ld, const int64_t *shell_off,
                    int64_t nshell, const double *t_box, const int32_t *mode, const double *loop_params,
                    int64_t nloops, int64_t ldp, const double *x_obs, double t_obs, double GU, int prec, int flags,
                    int accumulate, double *theta_out, void *stream)
{
    if (!c) return ISW_EINVAL;
    if (nside < 1 || nside > (1 << 24)) return set_err(c, ISW_EINVAL, "nside out of range");
    if (nshell < 0 || (nshell > 0 && (!shell_off || !t_box || !mode)))
        return set_err(c, ISW_EINVAL, "shell_off, t_box and mode (host arrays) are required");
    if (prec != ISW_F64 && prec != ISW_F32C) return set_err(c, ISW_EINVAL, "unknown precision %d", prec);
    if (flags & ~(ISW_SKIP_LIGHTCONE | ISW_GRAPH | ISW_AUTOTUNE)) return set_err(c, ISW_EINVAL, "unknown flags");
    const int64_t n = nshell > 0 ? shell_off[nshell] : 0;
    if (nshell > 0 && shell_off[0] != 0) return set_err(c, ISW_EINVAL, "shell_off[0] must be 0");
    bool has_burden = false;
    for (int64_t k = 0; k < nshell; ++k) {
        if (shell_off[k + 1] < shell_off[k]) return set_err(c, ISW_EINVAL, "shell_off must be non-decreasing");
        if (mode[k] != ISW_LINEAR && mode[k] != ISW_BURDEN) return set_err(c, ISW_EINVAL, "bad mode in shell %lld", (long long)k);
        if (mode[k] == ISW_LINEAR && !(t_obs > t_box[k])) return set_err(c, ISW_EINVAL, "t_obs must exceed t_box");
        if (mode[k] == ISW_BURDEN) has_burden = true;
    }
    int r;
    if ((r = check_samples(c, nodes, n, ld))) return r;
    if (!is_device_ptr(c, theta_out)) return set_err(c, ISW_EINVAL, "theta_out is not a device pointer");
    if (has_burden && !(flags & ISW_SKIP_LIGHTCONE) && (nloops <= 0 || ldp < nloops || !is_device_ptr(c, loop_params)))
        return set_err(c, ISW_EINVAL, "BURDEN shells need device loop_params[17][ldp], ldp >= nloops > 0");
    if (!std::isfinite(t_obs) || !std::isfinite(GU)) return set_err(c, ISW_EINVAL, "t_obs / GU not finite");
    if ((r = set_device(c))) return r;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npix = 12 * nside * nside;
    const double xo[3] = {x_obs ? x_obs[0] : 0.0, x_obs ? x_obs[1] : 0.0, x_obs ? x_obs[2] : 0.0};

    // shell metadata on the device (uploaded when it changes)
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](const void *p, size_t bytes) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t k = 0; k < bytes; ++k) h = (h ^ b[k]) * 1099511628211ull;
    };
    mix(shell_off, (size_t)(nshell + 1) * sizeof(int64_t));
    mix(t_box, (size_t)nshell * sizeof(double));
    mix(mode, (size_t)nshell * sizeof(int32_t));
    const size_t meta_bytes = (size_t)(nshell + 1) * 8 + (size_t)nshell * 8 + (size_t)nshell * 4 + 64;
    if ((r = ensure_ws(c, kWsShell, meta_bytes))) return r;
    int64_t *d_off = (int64_t *)c->ws[kWsShell];
    double *d_tbox = (double *)(d_off + nshell + 1);
    int32_t *d_mode = (int32_t *)(d_tbox + nshell);
    if (h != c->meta_hash || nshell != c->meta_nshell) {
        // earlier batched work on this stream may still read the previous metadata
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMemcpy(d_off, shell_off, (size_t)(nshell + 1) * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_tbox, t_box, (size_t)nshell * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_mode, mode, (size_t)nshell * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_err(c, e, "shell metadata upload");
        c->meta_hash = h;
        c->meta_nshell = nshell;
    }
    const bool skip_lc = (flags & ISW_SKIP_LIGHTCONE) != 0;
    if (!skip_lc && (r = ensure_ws(c, kWsSamples, (size_t)(n > 0 ? n : 1) * 10 * sizeof(double)))) return r;
    const double *samples = skip_lc ? nodes : (const double *)c->ws[kWsSamples];
    const int64_t lds = skip_lc ? ld : n;
    const double tol = 4.0 * (std::nextafter(t_obs, INFINITY) - t_obs);

    auto enqueue = [&](cudaStream_t st) -> int {
        if (!skip_lc && n > 0) {
            launch_lightcone_shells(nodes, n, ld, d_off, nshell, d_tbox, d_mode, loop_params, nloops, ldp, xo[0],
                                    xo[1], xo[2], t_obs, tol, (double *)c->ws[kWsSamples], n, c->d_status, st);
            c->n_launch += 1;
        }
        return map_impl(c, nside, 0, npix, nullptr, samples, n, lds, x_obs, GU, prec, accumulate, theta_out, st);
    };

    // autotuner: time every FP32 variant on a prefix of the samples, keep the fastest
    if ((flags & ISW_AUTOTUNE) && prec == ISW_F32C && n > 0 && c->tile_override < 0 &&
        !(c->tuned_nside == nside && c->tuned_n == n)) {
        if (!skip_lc) {
            launch_lightcone_shells(nodes, n, ld, d_off, nshell, d_tbox, d_mode, loop_params, nloops, ldp, xo[0],
                                    xo[1], xo[2], t_obs, tol, (double *)c->ws[kWsSamples], n, c->d_status, s);
            c->n_launch += 1;
        }
        // every variant maps all samples onto a strided subset of the pixel tiles (~4 waves)
        if ((r = ensure_ws(c, kWsMisc, (size_t)npix * sizeof(double)))) return r;
        double *scratch_theta = (double *)c->ws[kWsMisc];
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        double best = 1e300;   // device ms per processed pixel slot
        int best_v = 0;
        const int saved_timing = c->timing;
        c->timing = 0;
        for (int v = 0; v < num_f32_variants(); ++v) {
            c->tile_override = v;
            double tv = 0.0;
            int64_t px = 1;
            for (int rep = 0; rep < 2; ++rep) {
                cudaEventRecord(e0, s);
                r = map_impl(c, nside, 0, npix, nullptr, samples, n, lds, x_obs, GU, prec, 0, scratch_theta, s, 4,
                             &px);
                cudaEventRecord(e1, s);
                if (r) break;
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1) tv = (double)ms / (double)(px > 0 ? px : 1);
            }
            if (r) break;
            if (tv < best) {
                best = tv;
                best_v = v;
            }
        }
        c->tile_override = -1;
        c->timing = saved_timing;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (r) return r;
        c->auto_variant = best_v;
        c->tuned_nside = nside;
        c->tuned_n = n;
    }

    if (!(flags & ISW_GRAPH)) return enqueue(s);

    // CUDA graph: capture the light cone + map once per argument set, replay afterwards
    uint64_t key = h;
    auto mixv = [&key](uint64_t v) { key = (key ^ v) * 1099511628211ull; };
    mixv((uint64_t)nside); mixv((uint64_t)(uintptr_t)nodes); mixv((uint64_t)ld); mixv((uint64_t)nshell);
    mixv((uint64_t)(uintptr_t)loop_params); mixv((uint64_t)nloops); mixv((uint64_t)ldp);
    double dv[9] = {xo[0], xo[1], xo[2], t_obs, GU, c->near_k, c->b_min, c->d_far, (double)c->wait_polls};
    for (double d : dv) { uint64_t u; memcpy(&u, &d, 8); mixv(u); }
    mixv((uint64_t)prec); mixv((uint64_t)flags); mixv((uint64_t)accumulate); mixv((uint64_t)(uintptr_t)theta_out);
    mixv((uint64_t)c->split_override); mixv((uint64_t)(c->tile_override + 1)); mixv((uint64_t)c->auto_variant);
    if (c->graph_exec && key == c->graph_key) {
        cudaError_t e = cudaGraphLaunch(c->graph_exec, s);
        if (e != cudaSuccess) return cuda_err(c, e, "cudaGraphLaunch");
        c->n_launch += c->graph_kernels;
        c->n_pair += c->graph_pairs;
        return ISW_OK;
    }
    // first call with these arguments: run eagerly (this also sizes the workspace), then capture
    if ((r = enqueue(s))) return r;
    if (!c->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamCreate");
    }
    drop_graph(c);
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamBeginCapture");
    c->capturing = 1;
    const int64_t launches = c->n_launch, pairs = c->n_pair;
    r = enqueue(c->cap_stream);
    c->capturing = 0;
    c->graph_kernels = c->n_launch - launches;
    c->graph_pairs = c->n_pair - pairs;
    c->n_launch = launches;
    c->n_pair = pairs;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &g);
    if (r) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_err(c, e, "cudaGraphInstantiate");
    }
    c->graph = g;
    c->graph_key = key;
    return ISW_OK;
}

}  // extern "C"
