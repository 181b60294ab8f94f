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
// The walk is the incremental form of Siddon's method (Amanatides-Woo
// ordering): at every step the axis whose next voxel plane is nearest is
// crossed.  Crossing parameters are evaluated as t0 + k dt with one fused
// multiply-add (never accumulated), so every crossing carries a single
// float rounding relative to the entry point, and segment lengths, being
// differences of consecutive crossings, telescope to the chord.
#include <math.h>

#include "tomo_internal.cuh"

namespace tomo {

namespace {

__device__ __forceinline__ RayRec load_ray(const RayRec *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    RayRec r;
    r.t0x = a.x;
    r.t0y = a.y;
    r.t0z = a.z;
    r.chord = a.w;
    r.dtx = b.x;
    r.dty = b.y;
    r.dtz = b.z;
    r.idx0 = __float_as_int(b.w);
    return r;
}

// Map this thread to a pixel of the CTA's tile; false past the image edge.
__device__ __forceinline__ bool pixel_of_thread(const Tiling t, int nu, int nv,
                                                int &iu, int &iv)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows = 32 / t.warp_u;
    const int warps_u = t.tile_u / t.warp_u;
    iu = blockIdx.x * t.tile_u + (warp % warps_u) * t.warp_u + (lane % t.warp_u);
    iv = blockIdx.y * t.tile_v + (warp / warps_u) * rows + (lane / t.warp_u);
    return iu < nu && iv < nv;
}

// Walk one ray; op(idx, len) is called for every step, including steps of
// zero length at ties (two planes crossed at the same parameter).  The loop
// ends after at most (#planes inside the cube + 1) steps: each step that does
// not end the walk advances one axis, and no axis can advance past its last
// in-cube plane because the setup kernel capped the chord there.
template <class Op>
__device__ __forceinline__ void siddon_walk(const RayRec &r, int nx, int nxny,
                                            Op &op)
{
    const float chord = r.chord;
    const float ax = fabsf(r.dtx), ay = fabsf(r.dty), az = fabsf(r.dtz);
    const int sx = signbit(r.dtx) ? -1 : 1;
    const int sy = signbit(r.dty) ? -nx : nx;
    const int sz = signbit(r.dtz) ? -nxny : nxny;
    float kx = 0.0f, ky = 0.0f, kz = 0.0f;
    float tx = r.t0x, ty = r.t0y, tz = r.t0z;
    float t = 0.0f;
    int idx = r.idx0;
    for (;;) {
        const float tm = fminf(tx, fminf(ty, tz));
        const float te = fminf(tm, chord);
        op(idx, te - t);
        if (te >= chord) break;
        t = te;
        if (tx == tm) {
            kx += 1.0f;
            tx = fmaf(kx, ax, r.t0x);
            idx += sx;
        } else if (ty == tm) {
            ky += 1.0f;
            ty = fmaf(ky, ay, r.t0y);
            idx += sy;
        } else {
            kz += 1.0f;
            tz = fmaf(kz, az, r.t0z);
            idx += sz;
        }
    }
}

__device__ __forceinline__ float load_voxel(const float *c, int idx)
{
    return __ldg(c + idx);
}

__device__ __forceinline__ float load_voxel(const uint16_t *c, int idx)
{
    // bfloat16 -> float32 is exact: the bf16 bits are the top half
    return __uint_as_float(((uint32_t)__ldg(c + idx)) << 16);
}

template <typename CubeT>
struct GatherOp {
    const CubeT *c;
    float acc;
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        acc = fmaf(len, load_voxel(c, idx), acc);
    }
};

template <typename CubeT>
struct GatherTimeOp {
    const CubeT *c0;
    const CubeT *c1;
    float w0, w1, acc;
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        const float v = fmaf(w0, load_voxel(c0, idx), w1 * load_voxel(c1, idx));
        acc = fmaf(len, v, acc);
    }
};

struct ScatterOp {
    float *c;
    float y;
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        if (len > 0.0f) atomicAdd(c + idx, len * y);
    }
};

struct ScatterTimeOp {
    float *c0;
    float *c1;
    float y0, y1;
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        if (len > 0.0f) {
            atomicAdd(c0 + idx, len * y0);
            atomicAdd(c1 + idx, len * y1);
        }
    }
};

struct CountOp {
    unsigned int n;
    __device__ __forceinline__ void operator()(int, float len)
    {
        n += (len > 0.0f) ? 1u : 0u;
    }
};

template <typename CubeT, bool kTime>
__global__ void __launch_bounds__(512)
k_forward(const RayRec *__restrict__ rays, const ImgParam *__restrict__ prm,
          const CubeT *__restrict__ cube, int64_t frame_stride,
          const uint8_t *__restrict__ mask, float *__restrict__ out, int nu,
          int nv, int nx, int nxny, Tiling tl, const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    int iu, iv;
    if (!pixel_of_thread(tl, nu, nv, iu, iv)) return;
    const int img = blockIdx.z;
    const int64_t id = ((int64_t)img * nv + iv) * nu + iu;
    float y = 0.0f;
    if (mask == nullptr || mask[id] == 0) {
        const RayRec r = load_ray(rays + id);
        if (r.chord > 0.0f) {
            const ImgParam q = prm[img];
            if (kTime) {
                GatherTimeOp<CubeT> op;
                op.c0 = cube + (int64_t)q.frame * frame_stride;
                op.c1 = op.c0 + frame_stride;
                op.w0 = 1.0f - q.w;
                op.w1 = q.w;
                op.acc = 0.0f;
                siddon_walk(r, nx, nxny, op);
                y = q.gain * op.acc;
            } else {
                GatherOp<CubeT> op;
                op.c = cube;
                op.acc = 0.0f;
                siddon_walk(r, nx, nxny, op);
                y = q.gain * op.acc;
            }
        }
    }
    out[id] = y;
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
    if (!pixel_of_thread(tl, nu, nv, iu, iv)) return;
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
        op.c0 = cube + (int64_t)q.frame * frame_stride;
        op.c1 = op.c0 + frame_stride;
        op.y0 = yv * (1.0f - q.w);
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
    if (pixel_of_thread(tl, nu, nv, iu, iv)) {
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

}  // namespace

cudaError_t launch_forward(const RayRec *rays, const ImgParam *prm,
                           const void *cube, tomo_dtype dtype,
                           int64_t frame_stride, bool time_interp,
                           const uint8_t *mask, float *out, int32_t n_img,
                           int32_t nu, int32_t nv, int32_t nx, int32_t nxny,
                           Tiling t, const double *done, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid = grid_of(nu, nv, n_img, t);
    const int block = t.tile_u * t.tile_v;
    if (dtype == TOMO_BF16) {
        const uint16_t *c = static_cast<const uint16_t *>(cube);
        if (time_interp)
            k_forward<uint16_t, true><<<grid, block, 0, s>>>(
                rays, prm, c, frame_stride, mask, out, nu, nv, nx, nxny, t, done);
        else
            k_forward<uint16_t, false><<<grid, block, 0, s>>>(
                rays, prm, c, frame_stride, mask, out, nu, nv, nx, nxny, t, done);
    } else {
        const float *c = static_cast<const float *>(cube);
        if (time_interp)
            k_forward<float, true><<<grid, block, 0, s>>>(
                rays, prm, c, frame_stride, mask, out, nu, nv, nx, nxny, t, done);
        else
            k_forward<float, false><<<grid, block, 0, s>>>(
                rays, prm, c, frame_stride, mask, out, nu, nv, nx, nxny, t, done);
    }
    return cudaGetLastError();
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
