// tomo_project_noalloc: the forward projection with its scratch in a fixed
// array of this library instead of context workspace (see include/tomo.h
// for who needs this and for the limits).
//
// The array is a file-scope __device__ variable.  Host code cannot use its
// name as an address (on the host the name denotes a stand-in object, not
// device memory), so the first call on each device looks the device address
// up with cudaGetSymbolAddress while that device is current, and every call
// passes that address to the ray-setup kernels and the per-ray forward
// kernel that tomo_project also launches.
#include <mutex>

#include "host.h"

using namespace tomo;
using namespace tomo::host;

namespace {

static __device__ __align__(256) unsigned char
    g_noalloc_scratch[TOMO_NOALLOC_SCRATCH_BYTES];

static_assert(sizeof(tomo_pointing) == 96 && sizeof(Frame) == 96 &&
                  sizeof(ImgParam) == 16 && sizeof(RayRec) == 32,
              "the scratch formula in tomo.h assumes these record sizes");

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_dev[kMaxDevices] = { nullptr };

size_t round256(size_t n)
{
    return (n + 255) & ~(size_t)255;
}

// Device address of the scratch array on the current device, looked up once
// per device and kept for the process (the header forbids calls after a
// cudaDeviceReset, which would move the array).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_dev[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" tomo_status
tomo_project_noalloc(const tomo_cube_geom *cube, int32_t n_frames,
                     const void *cube_dev, tomo_dtype dtype,
                     const tomo_image_geom *img,
                     const tomo_pointing *pointing_host,
                     const uint8_t *mask_dev, float *images_dev, void *stream)
{
    tomo_status st;
    if ((st = check_cube(nullptr, cube, n_frames)) ||
        (st = check_img(nullptr, img)) ||
        (st = check_pointing(nullptr, pointing_host, img, n_frames)))
        return st;
    if (dtype != TOMO_F32 && dtype != TOMO_BF16) return TOMO_ERR_ARG;
    if (img->kind != TOMO_KIND_EMISSION) return TOMO_ERR_UNSUPPORTED;
    if (img->n_img == 0) return TOMO_OK;
    if (!cube_dev || !images_dev) return TOMO_ERR_ARG;
    if (!aligned(cube_dev, dtype == TOMO_F32 ? 4 : 2) || !aligned(images_dev, 4))
        return TOMO_ERR_ARG;

    const size_t n_img = (size_t)img->n_img;
    const size_t npix = n_img * img->nu * img->nv;
    const size_t off_ptg = 0;
    const size_t off_frames = off_ptg + round256(sizeof(tomo_pointing) * n_img);
    const size_t off_params = off_frames + round256(sizeof(Frame) * n_img);
    const size_t off_tan_u = off_params + round256(sizeof(ImgParam) * n_img);
    const size_t off_tan_v = off_tan_u + round256(sizeof(double) * n_img * img->nu);
    const size_t off_rays = off_tan_v + round256(sizeof(double) * n_img * img->nv);
    const size_t need = off_rays + round256(sizeof(RayRec) * npix);
    if (need > TOMO_NOALLOC_SCRATCH_BYTES) return TOMO_ERR_UNSUPPORTED;

    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        cudaGetLastError();
        return TOMO_ERR_CUDA;
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    tomo_pointing *ptg = reinterpret_cast<tomo_pointing *>(b + off_ptg);
    Frame *frames = reinterpret_cast<Frame *>(b + off_frames);
    ImgParam *params = reinterpret_cast<ImgParam *>(b + off_params);
    double *tan_u = reinterpret_cast<double *>(b + off_tan_u);
    double *tan_v = reinterpret_cast<double *>(b + off_tan_v);
    RayRec *rays = reinterpret_cast<RayRec *>(b + off_rays);
    cudaStream_t s = (cudaStream_t)stream;
    const Tiling tl = { 32, 8, 8 };

    if (cudaMemcpyAsync(ptg, pointing_host, sizeof(tomo_pointing) * n_img,
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        launch_frames(ptg, img->n_img, img->nu, img->nv, n_frames, frames,
                      tan_u, tan_v, params,
                      make_double3(cube->dx, cube->dy, cube->dz), nullptr,
                      nullptr, default_plane_rules(), s) != cudaSuccess ||
        launch_ray_setup(frames, tan_u, tan_v, tomo::host::cube_dev(cube),
                         img->n_img,
                         img->nu, img->nv, rays, s) != cudaSuccess ||
        launch_forward(rays, params, cube_dev, dtype,
                       (int64_t)cube->nx * cube->ny * cube->nz, n_frames > 1,
                       mask_dev, images_dev, img->n_img, img->nu, img->nv,
                       cube->nx, cube->nx * cube->ny, tl, nullptr,
                       s) != cudaSuccess) {
        cudaGetLastError();
        return TOMO_ERR_CUDA;
    }
    return TOMO_OK;
}
