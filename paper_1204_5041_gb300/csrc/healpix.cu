// HEALPix RING pixel centres (Sec. II.D) and the tile-ordered pixel tables of the map kernels.
#include "isw_internal.cuh"
#include "kernels.cuh"

namespace isw {

// Public pix2vec: one thread per requested pixel, RING order in, SoA (x, y, z) out.
__global__ void k_pix2vec(int64_t N, int64_t pix0, int64_t npix, const int64_t *__restrict__ pix_list,
                          double *__restrict__ out, int64_t ld, DevStatus *st)
{
    const int64_t npix_all = 12 * N * N;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < npix; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = pix_list ? pix_list[k] : pix0 + k;
        double x, y, z;
        if (p < 0 || p >= npix_all) {
            x = y = z = __longlong_as_double(0x7ff8000000000000LL);
            atomicOr(&st->bits, kStatBadIndex);
        } else {
            pix2vec_ring(N, p, x, y, z);
        }
        out[k] = x;
        out[ld + k] = y;
        out[2 * ld + k] = z;
    }
}

// Position (lx, ly) in a tx x ty block of the slot-th pixel when the block is enumerated by
// anti-diagonals lx + ly from the largest down, lx ascending along each.  On a HEALPix base face
// the ring number falls as ix + iy grows and the index within a ring grows with ix - iy, so this
// order follows RING order: consecutive slots hold consecutive RING indices along each ring, and
// the map kernels' per-slot stores of a warp land on a few contiguous runs of the output.
__device__ __forceinline__ void diag_slot(int l, int tx, int ty, int &lx, int &ly)
{
    for (int s = tx + ty - 2; s >= 0; --s) {
        const int lo = s - (ty - 1) > 0 ? s - (ty - 1) : 0, hi = s < tx - 1 ? s : tx - 1;
        const int cnt = hi - lo + 1;
        if (l < cnt) {
            lx = lo + l;
            ly = s - lx;
            return;
        }
        l -= cnt;
    }
    lx = ly = 0;
}

// Pixel table in tile order.  Slot l of tile t holds the direction of one pixel and the
// index its value is written to (RING index for full-sky maps, list position otherwise),
// or -1 for padding.  Full-sky tiles are tx x ty blocks of face coordinates (compact
// patches) with their slots in anti-diagonal (RING-following) order; range / list tiles are
// consecutive chunks of tx*ty pixels.
__global__ void k_pixel_table(int64_t N, int mode, int64_t pix0, int64_t npix, const int64_t *__restrict__ pix_list,
                              int tx, int ty, int64_t ntiles, double *__restrict__ nv, int64_t ldn,
                              int64_t *__restrict__ outidx, DevStatus *st)
{
    const int tile_sz = tx * ty;
    const int64_t total = ntiles * tile_sz;
    const int64_t nbx = (N + tx - 1) / tx, nby = (N + ty - 1) / ty;
    const int64_t npix_all = 12 * N * N;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = k / tile_sz;
        const int l = (int)(k - t * tile_sz);
        int64_t ring = -1, oi = -1;
        if (mode == 0) {
            const int64_t f = t / (nbx * nby);
            const int64_t rem = t - f * nbx * nby;
            const int64_t by = rem / nbx, bx = rem - by * nbx;
            int lx, ly;
            diag_slot(l, tx, ty, lx, ly);
            const int64_t ix = bx * tx + lx, iy = by * ty + ly;
            if (ix < N && iy < N) {
                ring = xyf2ring(N, (int)f, ix, iy);
                oi = ring;
            }
        } else if (k < npix) {
            ring = (mode == 2) ? pix_list[k] : pix0 + k;
            oi = k;
            if (ring < 0 || ring >= npix_all) {
                atomicOr(&st->bits, kStatBadIndex);
                ring = -1;
                oi = -1;
            }
        }
        double x = 0.0, y = 0.0, z = 1.0;
        if (ring >= 0) pix2vec_ring(N, ring, x, y, z);
        nv[k] = x;
        nv[ldn + k] = y;
        nv[2 * ldn + k] = z;
        outidx[k] = oi;
    }
}

// Bounding cap of each pixel tile: centre = normalised mean direction, radius = largest
// chord from the centre (valid pixels only).  One block of 256 threads per tile.
__global__ void k_pixel_caps(const double *__restrict__ nv, int64_t ldn, const int64_t *__restrict__ outidx,
                             int tile_sz, float4 *__restrict__ caps)
{
    __shared__ float red[3][32];
    __shared__ float cen[3];
    const int64_t t = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    float s[3] = {0.f, 0.f, 0.f};
    for (int l = tid; l < tile_sz; l += blockDim.x) {
        const int64_t k = t * tile_sz + l;
        if (outidx[k] >= 0)
            for (int c = 0; c < 3; ++c) s[c] += (float)nv[c * ldn + k];
    }
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
        if (lane == 0) red[c][wid] = s[c];
    }
    __syncthreads();
    if (tid == 0) {
        float a[3] = {0.f, 0.f, 0.f};
        for (int w = 0; w < nw; ++w)
            for (int c = 0; c < 3; ++c) a[c] += red[c][w];
        const float nrm = sqrtf(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        if (nrm > 0.f) {
            for (int c = 0; c < 3; ++c) cen[c] = a[c] / nrm;
        } else {
            cen[0] = 0.f; cen[1] = 0.f; cen[2] = 1.f;
        }
    }
    __syncthreads();
    float r = 0.f;
    for (int l = tid; l < tile_sz; l += blockDim.x) {
        const int64_t k = t * tile_sz + l;
        if (outidx[k] >= 0) {
            const float dx = (float)nv[k] - cen[0], dy = (float)nv[ldn + k] - cen[1], dz = (float)nv[2 * ldn + k] - cen[2];
            r = fmaxf(r, sqrtf(dx * dx + dy * dy + dz * dz));
        }
    }
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    __syncthreads();
    if (lane == 0) red[0][wid] = r;
    __syncthreads();
    if (tid == 0) {
        float m = 0.f;
        for (int w = 0; w < nw; ++w) m = fmaxf(m, red[0][w]);
        // margin for the FP32 rounding of the directions and of the centre
        caps[t] = make_float4(cen[0], cen[1], cen[2], m * 1.0001f + 1e-6f);
    }
}

// Patch table: tile t is block (t mod ntx, t / ntx) of tx x ty pixels of the M x M grid;
// padding slots hold the patch centre with output index -1.
__global__ void k_patch_table(PatchSpec p, int tx, int ty, int64_t ntiles, double *__restrict__ nv, int64_t ldn,
                              int64_t *__restrict__ outidx)
{
    const int tile_sz = tx * ty;
    const int64_t total = ntiles * tile_sz;
    const int64_t ntx = (p.M + tx - 1) / tx;
    const double h = p.width / (double)p.M;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = k / tile_sz;
        const int l = (int)(k - t * tile_sz);
        const int64_t i = (t % ntx) * tx + (l % tx), j = (t / ntx) * ty + (l / tx);
        double v[3] = {p.frame[6], p.frame[7], p.frame[8]};
        int64_t oi = -1;
        if (i < p.M && j < p.M) {
            const double xi = ((double)i + 0.5 - 0.5 * (double)p.M) * h;
            const double eta = ((double)j + 0.5 - 0.5 * (double)p.M) * h;
            for (int c = 0; c < 3; ++c) v[c] = xi * p.frame[c] + eta * p.frame[3 + c] + p.frame[6 + c];
            const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            for (int c = 0; c < 3; ++c) v[c] /= r;
            oi = j * p.M + i;
        }
        nv[k] = v[0];
        nv[ldn + k] = v[1];
        nv[2 * ldn + k] = v[2];
        outidx[k] = oi;
    }
}

void launch_patch_table(const PatchSpec &p, int tx, int ty, int64_t ntiles, double *nv, int64_t ldn,
                        int64_t *outidx, float4 *caps, cudaStream_t s)
{
    const int64_t total = ntiles * tx * ty;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_patch_table<<<(unsigned)blocks, 256, 0, s>>>(p, tx, ty, ntiles, nv, ldn, outidx);
    k_pixel_caps<<<(unsigned)ntiles, 256, 0, s>>>(nv, ldn, outidx, tx * ty, caps);
}

int launch_pix2vec(int64_t N, int64_t pix0, int64_t npix, const int64_t *pix_list, double *out, int64_t ld,
                   DevStatus *st, cudaStream_t s)
{
    if (npix == 0) return 0;
    const int threads = 256;
    const int64_t blocks = (npix + threads - 1) / threads;
    k_pix2vec<<<(unsigned)(blocks < 65535 * 8 ? blocks : 65535 * 8), threads, 0, s>>>(N, pix0, npix, pix_list, out,
                                                                                         ld, st);
    return 0;
}

void launch_pixel_table(int64_t N, int mode, int64_t pix0, int64_t npix, const int64_t *pix_list, int tx, int ty,
                        int64_t ntiles, double *nv, int64_t ldn, int64_t *outidx, float4 *caps, DevStatus *st,
                        cudaStream_t s)
{
    const int64_t total = ntiles * tx * ty;
    const int threads = 256;
    int64_t blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_pixel_table<<<(unsigned)blocks, threads, 0, s>>>(N, mode, pix0, npix, pix_list, tx, ty, ntiles, nv, ldn, outidx,
                                                       st);
    k_pixel_caps<<<(unsigned)ntiles, 256, 0, s>>>(nv, ldn, outidx, tx * ty, caps);
}

}  // namespace isw
