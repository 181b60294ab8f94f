// Map mask: voxels excluded from the reconstruction (uint8 [nz][ny][nx],
// nonzero = excluded; Section 4 names masks of the data and of the map).
//
// Reading of the operation: an excluded voxel is not an unknown.  The
// projector reads it as 0 (P K x, K = diag(1 - mask)), the transpose gives
// it nothing (K P^T y), and the solver works on the system restricted to the
// other voxels.  These element-wise kernels apply K around the walks; the
// walks themselves are unchanged.  With T > 1 frames the same mask applies
// to every frame.
//
// Each is one pass over the cube, HBM-bound (mask byte + one or two floats
// per voxel and frame), grid-stride over voxels with the frames in an inner
// loop so the mask byte is read once.
#include <stdint.h>

#include <cuda_runtime.h>

namespace tomo {

namespace {

constexpr int kThreads = 256;

unsigned int grid_for(int64_t n)
{
    const int64_t g = (n + kThreads - 1) / kThreads;
    return (unsigned int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

// dst = K src; E is float or the raw bits of bfloat16 (0 is +0.0 in both)
template <typename E>
__global__ void k_map_keep_copy(const E *__restrict__ src, E *__restrict__ dst,
                                const uint8_t *__restrict__ mm, int64_t n,
                                int32_t frames)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool out = mm[i] != 0;
        for (int32_t t = 0; t < frames; ++t) {
            const int64_t j = (int64_t)t * n + i;
            dst[j] = out ? E(0) : src[j];
        }
    }
}

// x = K x (writes only the excluded voxels)
__global__ void k_map_zero(float *__restrict__ x,
                           const uint8_t *__restrict__ mm, int64_t n,
                           int32_t frames)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (mm[i] == 0) continue;
        for (int32_t t = 0; t < frames; ++t) x[(int64_t)t * n + i] = 0.0f;
    }
}

// dst += K src
__global__ void k_map_keep_add(float *__restrict__ dst,
                               const float *__restrict__ src,
                               const uint8_t *__restrict__ mm, int64_t n,
                               int32_t frames)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (mm[i] != 0) continue;
        for (int32_t t = 0; t < frames; ++t) {
            const int64_t j = (int64_t)t * n + i;
            dst[j] += src[j];
        }
    }
}

}  // namespace

cudaError_t launch_map_keep_copy(const void *src, void *dst, bool bf16,
                                 const uint8_t *mm, int64_t n, int32_t frames,
                                 cudaStream_t s)
{
    if (n <= 0 || frames <= 0) return cudaSuccess;
    if (bf16)
        k_map_keep_copy<uint16_t><<<grid_for(n), kThreads, 0, s>>>(
            (const uint16_t *)src, (uint16_t *)dst, mm, n, frames);
    else
        k_map_keep_copy<float><<<grid_for(n), kThreads, 0, s>>>(
            (const float *)src, (float *)dst, mm, n, frames);
    return cudaGetLastError();
}

cudaError_t launch_map_zero(float *x, const uint8_t *mm, int64_t n,
                            int32_t frames, cudaStream_t s)
{
    if (n <= 0 || frames <= 0) return cudaSuccess;
    k_map_zero<<<grid_for(n), kThreads, 0, s>>>(x, mm, n, frames);
    return cudaGetLastError();
}

cudaError_t launch_map_keep_add(float *dst, const float *src,
                                const uint8_t *mm, int64_t n, int32_t frames,
                                cudaStream_t s)
{
    if (n <= 0 || frames <= 0) return cudaSuccess;
    k_map_keep_add<<<grid_for(n), kThreads, 0, s>>>(dst, src, mm, n, frames);
    return cudaGetLastError();
}

}  // namespace tomo
