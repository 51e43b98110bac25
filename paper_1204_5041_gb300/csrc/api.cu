// C ABI of the library (include/isw.h): argument checks, workspace, launch sequences.
#include <cmath>
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
    kWsP32, kWsP64, kWsAdjPartial, kWsCount
};

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

// A device-accessible pointer: device or managed memory.  Host (even pinned) pointers are
// rejected because the kernels would read them over the bus or fault.
bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ensure_ws(isw_ctx *c, int slot, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (c->ws_size[slot] >= bytes) return ISW_OK;
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
        if (npix > 0 && !is_device_ptr(pix_list)) return set_err(c, ISW_EINVAL, "pix_list is not a device pointer");
    } else if (pix0 < 0 || pix0 + npix > all) {
        return set_err(c, ISW_EINVAL, "pixel range [%lld, %lld) outside [0, %lld)", (long long)pix0,
                       (long long)(pix0 + npix), (long long)all);
    }
    return ISW_OK;
}

int check_samples(isw_ctx *c, const double *samples, int64_t n, int64_t ld)
{
    if (n < 0) return set_err(c, ISW_EINVAL, "n < 0");
    if (n > 0 && ld < n) return set_err(c, ISW_EINVAL, "ld (%lld) < n (%lld)", (long long)ld, (long long)n);
    if (n > 0 && !is_device_ptr(samples)) return set_err(c, ISW_EINVAL, "samples is not a device pointer");
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

// Number of segment chunks: enough work items to fill every resident CTA slot with
// near-equal waves, at least two segment tiles per chunk.
int choose_split(int64_t ntiles, int64_t nst, int slots)
{
    const double ideal = (double)ntiles / slots;
    int best = 1;
    double best_t = 1e300;
    for (int k = 1; k <= 64; ++k) {
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
    return best;
}

// Events around a pair-kernel launch when timing is on; returns the slot or -1.
int timing_begin(isw_ctx *c, cudaStream_t s)
{
    if (!c->timing || c->n_timed >= kMaxTimed) return -1;
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
             cudaStream_t s)
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
        vidx = c->tile_override >= 0 && c->tile_override < num_f32_variants() ? c->tile_override : 0;
    }
    const Variant v = prec == ISW_F32C ? f32_variant(vidx) : f64_variant();
    const int S = v.seg_tile;
    const PixelPlan pp = plan_pixels(nside, pix0, npix, pix_list, v);
    const int64_t n_pad = (n + S - 1) / S * S;
    const int64_t nst = n_pad / S;
    const int slots = prec == ISW_F32C ? map_f32c_slots(vidx, c->num_sms) : map_f64_slots(c->num_sms);
    const int split = c->split_override > 0 ? c->split_override : choose_split(pp.ntiles, nst, slots);
    int r;
    if ((r = ensure_ws(c, kWsNv, (size_t)pp.tot * 3 * sizeof(double)))) return r;
    if ((r = ensure_ws(c, kWsOut, (size_t)pp.tot * sizeof(int64_t)))) return r;
    if ((r = ensure_ws(c, kWsPcap, (size_t)pp.ntiles * sizeof(float4)))) return r;
    if ((r = ensure_ws(c, kWsS32, (size_t)n_pad * sizeof(Seg32)))) return r;
    if ((r = ensure_ws(c, kWsS64, (size_t)n_pad * sizeof(Seg64)))) return r;
    if ((r = ensure_ws(c, kWsScap, (size_t)nst * sizeof(SegCap)))) return r;
    if (split > 1 && (r = ensure_ws(c, kWsPartial, (size_t)split * pp.tot * sizeof(double)))) return r;

    const double theta_pix = std::sqrt(4.0 * M_PI / (12.0 * (double)nside * (double)nside));
    double *nv = (double *)c->ws[kWsNv];
    int64_t *outidx = (int64_t *)c->ws[kWsOut];
    float4 *pcaps = (float4 *)c->ws[kWsPcap];
    Seg32 *s32 = (Seg32 *)c->ws[kWsS32];
    Seg64 *s64 = (Seg64 *)c->ws[kWsS64];
    SegCap *scaps = (SegCap *)c->ws[kWsScap];

    launch_pixel_table(nside, pp.mode, pix0, npix, pix_list, pp.tx, pp.ty, pp.ntiles, nv, pp.tot, outidx, pcaps,
                       c->d_status, s);
    launch_pack(samples, n, ld, xo[0], xo[1], xo[2], GU, theta_pix, c->near_k, n_pad, s32, s64, c->d_status, s);
    c->n_launch += 3;
    if (prec == ISW_F32C) {
        launch_seg_caps(s32, s64, n, n_pad, S, (float)c->b_min, scaps, s);
        c->n_launch += 1;
    }

    MapArgs a;
    a.nv = nv;
    a.ldn = pp.tot;
    a.outidx = outidx;
    a.pcaps = pcaps;
    a.ntiles = pp.ntiles;
    a.s32 = s32;
    a.s64 = s64;
    a.scaps = scaps;
    a.nst = nst;
    a.split = split;
    a.b_min = (float)c->b_min;
    a.d_far = (float)c->d_far;
    a.theta = theta;
    a.partial = split > 1 ? (double *)c->ws[kWsPartial] : nullptr;
    a.accumulate = accumulate;
    a.st = c->d_status;
    const int64_t items = pp.ntiles * split;
    const int grid = (int)(items < slots ? items : slots);
    const int ti = timing_begin(c, s);
    if (prec == ISW_F32C) launch_map_f32c(vidx, a, grid, s);
    else launch_map_f64(a, grid, s);
    timing_end(c, ti, s);
    c->n_pair += 1;
    c->n_launch += 1;
    if (split > 1) {
        launch_reduce_partials(a, v.tx * v.ty, s);
        c->n_launch += 1;
    }
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
    c->near_k = 4.0;
    c->b_min = 0.01;
    c->d_far = 0.4;
    c->split_override = 0;
    c->tile_override = -1;
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
    default:
        return set_err(c, ISW_EINVAL, "unknown parameter key %d", key);
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
    if (h.bits & kStatTimeout) return set_err(c, ISW_ETIMEOUT, "a bounded device wait ran out");
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
    if (!is_device_ptr(vec_out)) return set_err(c, ISW_EINVAL, "vec_out is not a device pointer");
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
    if (!is_device_ptr(samples_out)) return set_err(c, ISW_EINVAL, "samples_out is not a device pointer");
    if (tau_out && !is_device_ptr(tau_out)) return set_err(c, ISW_EINVAL, "tau_out is not a device pointer");
    if (status && !is_device_ptr(status)) return set_err(c, ISW_EINVAL, "status is not a device pointer");
    if (mode == ISW_LINEAR && !(t_obs > t_box)) return set_err(c, ISW_EINVAL, "t_obs must exceed t_box");
    if (mode == ISW_BURDEN) {
        if (nloops <= 0 || ldp < nloops || !is_device_ptr(loop_params))
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

int isw_map(isw_ctx *c, int64_t nside, int64_t pix0, int64_t npix, const int64_t *pix_list, const double *samples,
            int64_t n, int64_t ld, const double *x_obs, double GU, int prec, int accumulate, double *theta_out,
            void *stream)
{
    if (!c) return ISW_EINVAL;
    int r;
    if ((r = check_pixels(c, nside, pix0, npix, pix_list))) return r;
    if ((r = check_samples(c, samples, n, ld))) return r;
    if (prec != ISW_F64 && prec != ISW_F32C) return set_err(c, ISW_EINVAL, "unknown precision %d", prec);
    if (npix > 0 && !is_device_ptr(theta_out)) return set_err(c, ISW_EINVAL, "theta_out is not a device pointer");
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
    if (ngrad != 6 && ngrad != 9) return set_err(c, ISW_EINVAL, "ngrad must be 6 or 9");
    if (n == 0) return ISW_OK;
    if (ld_g < n) return set_err(c, ISW_EINVAL, "ld_g < n");
    if (!is_device_ptr(grad_out)) return set_err(c, ISW_EINVAL, "grad_out is not a device pointer");
    if (npix > 0 && !is_device_ptr(dL_dtheta)) return set_err(c, ISW_EINVAL, "dL_dtheta is not a device pointer");
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
    int split = c->split_override > 0 ? c->split_override : choose_split(nseg_tiles, pp.ntiles, slots);
    if (split > pp.ntiles) split = (int)pp.ntiles;
    if ((r = ensure_ws(c, kWsNv, (size_t)pp.tot * 3 * sizeof(double)))) return r;
    if ((r = ensure_ws(c, kWsOut, (size_t)pp.tot * sizeof(int64_t)))) return r;
    if ((r = ensure_ws(c, kWsPcap, (size_t)pp.ntiles * sizeof(float4)))) return r;
    if ((r = ensure_ws(c, kWsP32, (size_t)pp.tot * sizeof(Pix32)))) return r;
    if ((r = ensure_ws(c, kWsP64, (size_t)pp.tot * sizeof(Pix64)))) return r;
    if ((r = ensure_ws(c, kWsS32, (size_t)n_pad * sizeof(Seg32)))) return r;
    if ((r = ensure_ws(c, kWsS64, (size_t)n_pad * sizeof(Seg64)))) return r;
    if ((r = ensure_ws(c, kWsScap, (size_t)nseg_tiles * sizeof(SegCap)))) return r;
    if (split > 1 && (r = ensure_ws(c, kWsAdjPartial, (size_t)split * ngrad * n_pad * sizeof(double)))) return r;
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
    launch_pack_pixels(nv, pp.tot, outidx, dL_dtheta, pp.tot, p32, p64, s);
    launch_pack(samples, n, ld, xo[0], xo[1], xo[2], GU, theta_pix, c->near_k, n_pad, s32, s64, c->d_status, s);
    c->n_launch += 4;
    if (prec == ISW_F32C) {
        launch_seg_caps(s32, s64, n, n_pad, NT, (float)c->b_min, scaps, s);
        c->n_launch += 1;
    }
    AdjArgs a;
    a.p32 = p32;
    a.p64 = p64;
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
    const int64_t items = nseg_tiles * split;
    const int grid = (int)(items < slots ? items : slots);
    const int ti = timing_begin(c, s);
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
    (void)nside; (void)nodes; (void)ld; (void)shell_off; (void)nshell; (void)t_box; (void)mode;
    (void)loop_params; (void)nloops; (void)ldp; (void)x_obs; (void)t_obs; (void)GU; (void)prec; (void)flags;
    (void)accumulate; (void)theta_out; (void)stream;
    return set_err(c, ISW_EINVAL, "isw_map_batched: not built yet");
}

}  // extern "C"
