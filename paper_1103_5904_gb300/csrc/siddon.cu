// Siddon traversal: forward projection P, transpose P^T, segment count.
//
// Definition (Section 3.3.1, Eq. lo): pixel k of image n receives
// y_k = g_n * sum_j P_{k,j} x_j, with P_{k,j} the length of the pixel's line
// of sight inside voxel j (Siddon's algorithm, cited in Section 3.1).  P^T
// spreads g_n y_k back over the same voxels with the same lengths.
//
// GPU design: one thread per line of sight; a CTA covers a tile of pixels
// of one image, each warp a compact sub-tile (warp_u x 32/warp_u), so the
// 32 rays of a warp leave one observer through neighbouring pixels and walk
// neighbouring voxels at the same time: their gathers coalesce in L1 and L2.
// Pixel-major output makes the stores of a warp contiguous runs.
//
// The walk itself (walk.cuh) is shared with the batched kernels.
#include <math.h>

#include "walk.cuh"

namespace tomo {

namespace {

// One pixel of the forward projection: the masked, gained line integral.
template <typename CubeT, bool kTime>
__device__ __forceinline__ void forward_pixel(
    const RayRec *__restrict__ rays, const ImgParam *__restrict__ prm,
    const CubeT *__restrict__ cube, int64_t frame_stride,
    const uint8_t *__restrict__ mask, float *__restrict__ out, int nu, int nv,
    int nx, int nxny, int img, int iu, int iv)
{
    const int64_t id = ((int64_t)img * nv + iv) * nu + iu;
    float y = 0.0f;
    if (mask == nullptr || mask[id] == 0) {
        const RayRec r = load_ray(rays + id);
        if (r.chord > 0.0f) {
            const ImgParam q = prm[img];
            if (kTime) {
                GatherTimeOp<CubeT> op;
                op.c0 = cube + (int64_t)img_frame(q) * frame_stride;
                op.c1 = op.c0 + frame_stride;
                op.w0 = q.w0;
                op.w1 = q.w;
                op.acc = 0.0f;
                siddon_gather(r, nx, nxny, op);
                y = q.gain * op.acc;
            } else {
                GatherOp<CubeT> op;
                op.c = cube;
                op.acc = 0.0f;
                siddon_gather(r, nx, nxny, op);
                y = q.gain * op.acc;
            }
        }
    }
    out[id] = y;
}

// One CTA per pixel tile of one image; with skip_plane_images the CTAs of
// images whose hint selects the plane forward return at once.
template <typename CubeT, bool kTime>
__global__ void __launch_bounds__(512)
k_forward(const RayRec *__restrict__ rays, const ImgParam *__restrict__ prm,
          const CubeT *__restrict__ cube, int64_t frame_stride,
          const uint8_t *__restrict__ mask, float *__restrict__ out, int nu,
          int nv, int nx, int nxny, Tiling tl, const double *__restrict__ done,
          bool skip_plane_images)
{
    if (done != nullptr && *done != 0.0) return;
    if (skip_plane_images && (prm[blockIdx.z].pad & kPlaneFwdBit)) return;
    int iu, iv;
    if (!pixel_of_thread(tl, blockIdx.x, blockIdx.y, nu, nv, iu, iv)) return;
    forward_pixel<CubeT, kTime>(rays, prm, cube, frame_stride, mask, out, nu,
                                nv, nx, nxny, blockIdx.z, iu, iv);
}

// The images listed in listed = { count, image indices ... }: a grid of
// about one wave of CTAs deals the (listed image, tile) units out in turn.
// With an empty list (every image taken by the plane-synchronous forward)
// the launch costs one wave of CTAs that read the count and return, not one
// CTA per tile of every image.
template <typename CubeT, bool kTime>
__global__ void __launch_bounds__(512)
k_forward_listed(const RayRec *__restrict__ rays,
                 const ImgParam *__restrict__ prm,
                 const CubeT *__restrict__ cube, int64_t frame_stride,
                 const uint8_t *__restrict__ mask, float *__restrict__ out,
                 int nu, int nv, int nx, int nxny, Tiling tl,
                 const double *__restrict__ done,
                 const unsigned *__restrict__ listed, unsigned tiles_u,
                 unsigned tiles)
{
    if (done != nullptr && *done != 0.0) return;
    // units + gridDim.x < 2^32: the launcher checks it
    const unsigned units = listed[0] * tiles;
    for (unsigned w = blockIdx.x; w < units; w += gridDim.x) {
        const int img = (int)listed[1 + w / tiles];
        const unsigned t = w % tiles;
        int iu, iv;
        if (pixel_of_thread(tl, (int)(t % tiles_u), (int)(t / tiles_u), nu,
                            nv, iu, iv))
            forward_pixel<CubeT, kTime>(rays, prm, cube, frame_stride, mask,
                                        out, nu, nv, nx, nxny, img, iu, iv);
    }
}

template <bool kTime>
__global__ void __launch_bounds__(512)
k_adjoint(const RayRec *__restrict__ rays, const ImgParam *__restrict__ prm,
          const float *__restrict__ images, const uint8_t *__restrict__ mask,
          float *cube, int64_t frame_stride, int nu, int nv, int nx, int nxny,
          Tiling tl, const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    int iu, iv;
    if (!pixel_of_thread(tl, blockIdx.x, blockIdx.y, nu, nv, iu, iv)) return;
    const int img = blockIdx.z;
    const int64_t id = ((int64_t)img * nv + iv) * nu + iu;
    if (mask != nullptr && mask[id] != 0) return;
    const ImgParam q = prm[img];
    const float yv = q.gain * images[id];
    if (yv == 0.0f) return;
    const RayRec r = load_ray(rays + id);
    if (!(r.chord > 0.0f)) return;
    if (kTime) {
        ScatterTimeOp op;
        op.c0 = cube + (int64_t)img_frame(q) * frame_stride;
        op.c1 = op.c0 + frame_stride;
        op.y0 = yv * q.w0;
        op.y1 = yv * q.w;
        siddon_walk(r, nx, nxny, op);
    } else {
        ScatterOp op;
        op.c = cube;
        op.y = yv;
        siddon_walk(r, nx, nxny, op);
    }
}

__global__ void __launch_bounds__(512)
k_count(const RayRec *__restrict__ rays, const uint8_t *__restrict__ mask,
        int nu, int nv, Tiling tl, unsigned long long *count)
{
    int iu, iv;
    unsigned int n = 0;
    if (pixel_of_thread(tl, blockIdx.x, blockIdx.y, nu, nv, iu, iv)) {
        const int64_t id = ((int64_t)blockIdx.z * nv + iv) * nu + iu;
        if (mask == nullptr || mask[id] == 0) {
            const RayRec r = load_ray(rays + id);
            if (r.chord > 0.0f) {
                CountOp op;
                op.n = 0;
                // the walk's index arithmetic is not used by CountOp
                siddon_walk(r, 1, 1, op);
                n = op.n;
            }
        }
    }
    n = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(count, (unsigned long long)n);
}

dim3 grid_of(int nu, int nv, int n_img, Tiling t)
{
    return dim3((unsigned)((nu + t.tile_u - 1) / t.tile_u),
                (unsigned)((nv + t.tile_v - 1) / t.tile_v), (unsigned)n_img);
}

template <typename CubeT, bool kTime>
cudaError_t forward_kernel(const RayRec *rays, const ImgParam *prm,
                           const CubeT *cube, int64_t frame_stride,
                           const uint8_t *mask, float *out, int32_t n_img,
                           int32_t nu, int32_t nv, int32_t nx, int32_t nxny,
                           Tiling t, const double *done, cudaStream_t s,
                           bool skip, const unsigned *listed, int num_sms)
{
    const dim3 grid = grid_of(nu, nv, n_img, t);
    const int block = t.tile_u * t.tile_v;
    if (!skip || listed == nullptr) {
        k_forward<CubeT, kTime><<<grid, block, 0, s>>>(
            rays, prm, cube, frame_stride, mask, out, nu, nv, nx, nxny, t, done,
            skip);
        return cudaGetLastError();
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_forward_listed<CubeT, kTime>, block, 0);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (int64_t)grid.x * grid.y;
    const int64_t units = tiles * n_img;
    int64_t ctas = (int64_t)(per_sm > 0 ? per_sm : 1) * (num_sms > 0 ? num_sms : 1);
    if (ctas > units) ctas = units;
    // the unit counter w < units steps by ctas without wrapping
    if (units + ctas >= ((int64_t)1 << 32)) return cudaErrorInvalidValue;
    k_forward_listed<CubeT, kTime><<<(unsigned)ctas, block, 0, s>>>(
        rays, prm, cube, frame_stride, mask, out, nu, nv, nx, nxny, t, done,
        listed, grid.x, (unsigned)tiles);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_forward(const RayRec *rays, const ImgParam *prm,
                           const void *cube, tomo_dtype dtype,
                           int64_t frame_stride, bool time_interp,
                           const uint8_t *mask, float *out, int32_t n_img,
                           int32_t nu, int32_t nv, int32_t nx, int32_t nxny,
                           Tiling t, const double *done, cudaStream_t s,
                           bool skip_plane_images, const unsigned *listed,
                           int num_sms)
{
    if (n_img <= 0) return cudaSuccess;
    const bool sk = skip_plane_images;
    if (dtype == TOMO_BF16) {
        const uint16_t *c = static_cast<const uint16_t *>(cube);
        return time_interp
                   ? forward_kernel<uint16_t, true>(rays, prm, c, frame_stride,
                                                    mask, out, n_img, nu, nv,
                                                    nx, nxny, t, done, s, sk,
                                                    listed, num_sms)
                   : forward_kernel<uint16_t, false>(rays, prm, c, frame_stride,
                                                     mask, out, n_img, nu, nv,
                                                     nx, nxny, t, done, s, sk,
                                                     listed, num_sms);
    }
    const float *c = static_cast<const float *>(cube);
    return time_interp
               ? forward_kernel<float, true>(rays, prm, c, frame_stride, mask,
                                             out, n_img, nu, nv, nx, nxny, t,
                                             done, s, sk, listed, num_sms)
               : forward_kernel<float, false>(rays, prm, c, frame_stride, mask,
                                              out, n_img, nu, nv, nx, nxny, t,
                                              done, s, sk, listed, num_sms);
}

cudaError_t launch_adjoint(const RayRec *rays, const ImgParam *prm,
                           const float *images, const uint8_t *mask,
                           float *cube, int64_t frame_stride,
                           bool time_interp, int32_t n_img, int32_t nu,
                           int32_t nv, int32_t nx, int32_t nxny, Tiling t,
                           const double *done, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid = grid_of(nu, nv, n_img, t);
    const int block = t.tile_u * t.tile_v;
    if (time_interp)
        k_adjoint<true><<<grid, block, 0, s>>>(rays, prm, images, mask, cube,
                                               frame_stride, nu, nv, nx, nxny,
                                               t, done);
    else
        k_adjoint<false><<<grid, block, 0, s>>>(rays, prm, images, mask, cube,
                                                frame_stride, nu, nv, nx, nxny,
                                                t, done);
    return cudaGetLastError();
}

cudaError_t launch_count(const RayRec *rays, const uint8_t *mask,
                         int32_t n_img, int32_t nu, int32_t nv, Tiling t,
                         unsigned long long *count, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid = grid_of(nu, nv, n_img, t);
    k_count<<<grid, t.tile_u * t.tile_v, 0, s>>>(rays, mask, nu, nv, t, count);
    return cudaGetLastError();
}

}  // namespace tomo
