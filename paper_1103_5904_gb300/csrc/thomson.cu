// Thomson-scattering operators for white-light images (Section 3.5):
//     T_pB = O P M ,    T_B = P M' - O P M ,
// O = diag(rho_k^2) over pixels (rho = impact parameter of the line of
// sight), M = diag(m_j), M' = diag(m'_j) over voxels (Eq. thomson_lo,
// Eq. brightness, Eq. thomson_direct).  The walks are the plain projector's;
// these kernels are the diagonal factors around them.
//
// Readings (Eq. 4C and Eq. thomson_lo are garbled in places):
// sin(Omega) = 1/r; C4 carries +1/8 (with -1/8 the tangential intensity of a
// limb-darkened Sun would be negative; the coefficients are disk integrals
// of positive quantities); m_j = ((1-u) C1 + u C2) / r^4 and
// m'_j = 2 ((1-u) C3 + u C4) / r^2 as in Eq. brightness; no scattering
// inside the photosphere (r <= 1: m = m' = 0); the constant pi sigma I0 / 2
// is left to the per-image gains.
//
// The per-voxel factors are computed once per (cube geometry, u) in FP64
// (a log and square roots near r = 1, cancellation in C2 and C4 at large r)
// and stored as float2 (m, m'); rho^2 is computed per pixel in FP64 from the
// observer frame during the ray setup and stored as float.  The other
// kernels are element-wise passes (HBM-bound).
#include <math.h>

#include "tomo_internal.cuh"

namespace tomo {

namespace {

constexpr int kThreads = 256;

unsigned int grid_for(int64_t n)
{
    const int64_t g = (n + kThreads - 1) / kThreads;
    return (unsigned int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

__device__ __forceinline__ bool is_done(const double *done)
{
    return done != nullptr && *done != 0.0;
}

__global__ void k_thomson_factors(CubeDev c, double u, float2 *__restrict__ mf)
{
    const int64_t n = (int64_t)c.nx * c.ny * c.nz;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(v % c.nx);
        const int64_t rest = v / c.nx;
        const int j = (int)(rest % c.ny), k = (int)(rest / c.ny);
        const double px = c.lo[0] + (i + 0.5) * c.d[0];
        const double py = c.lo[1] + (j + 0.5) * c.d[1];
        const double pz = c.lo[2] + (k + 0.5) * c.d[2];
        const double r = sqrt(px * px + py * py + pz * pz);
        float2 out = make_float2(0.0f, 0.0f);
        if (r > 1.0) {
            const double s = 1.0 / r;
            const double s2 = s * s;
            const double cs = sqrt(1.0 - s2);
            // (cos^2 Omega / sin Omega) ln((1 + sin Omega) / cos Omega)
            const double g = cs > 0.0 ? cs * cs / s * log((1.0 + s) / cs) : 0.0;
            const double c1 = cs * s2;
            const double c2 = -0.125 * (1.0 - 3.0 * s2 - g * (1.0 + 3.0 * s2));
            const double c3 = 4.0 / 3.0 - cs - cs * cs * cs / 3.0;
            const double c4 = 0.125 * (5.0 + s2 - g * (5.0 - s2));
            const double r2 = r * r;
            out.x = (float)(((1.0 - u) * c1 + u * c2) / (r2 * r2));
            out.y = (float)(2.0 * ((1.0 - u) * c3 + u * c4) / r2);
        }
        mf[v] = out;
    }
}

// rho^2 = |o x u|^2 per pixel, u the unit direction of the pixel's ray (the
// ray setup's construction), in FP64.
__global__ void k_impact2(const Frame *__restrict__ frames,
                          const double *__restrict__ tan_u,
                          const double *__restrict__ tan_v, int32_t nu,
                          int32_t nv, float *__restrict__ rho2)
{
    const int img = blockIdx.y;
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (int64_t)nu * nv) return;
    const int iu = (int)(pix % nu), iv = (int)(pix / nu);
    const Frame &f = frames[img];
    const double tu = tan_u[(int64_t)img * nu + iu];
    const double tv = tan_v[(int64_t)img * nv + iv];
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = f.w[a] + tu * f.e1[a] + tv * f.e2[a];
    const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double cx = f.o[1] * d[2] - f.o[2] * d[1];
    const double cy = f.o[2] * d[0] - f.o[0] * d[2];
    const double cz = f.o[0] * d[1] - f.o[1] * d[0];
    rho2[(int64_t)img * nu * nv + pix] =
        (float)((cx * cx + cy * cy + cz * cz) / dd);
}

// dst = f K src over frames (f = m or m' of the voxel); src float or bf16
template <bool kBf16>
__global__ void k_thomson_weight(const void *__restrict__ src,
                                 const float2 *__restrict__ mf, int which,
                                 const uint8_t *__restrict__ mm, int64_t n,
                                 int32_t frames, float *__restrict__ dst,
                                 const double *__restrict__ done)
{
    if (is_done(done)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 m = mf[i];
        const float f = (mm != nullptr && mm[i] != 0) ? 0.0f
                                                        : (which ? m.y : m.x);
        for (int32_t t = 0; t < frames; ++t) {
            const int64_t j = (int64_t)t * n + i;
            float x;
            if (kBf16)
                x = __uint_as_float((unsigned)((const uint16_t *)src)[j] << 16);
            else
                x = ((const float *)src)[j];
            dst[j] = f * x;
        }
    }
}

// dst += K (m a) (b == NULL, pB) or K (m' a - m b) (B)
__global__ void k_thomson_add(float *__restrict__ dst,
                              const float *__restrict__ a,
                              const float *__restrict__ b,
                              const float2 *__restrict__ mf,
                              const uint8_t *__restrict__ mm, int64_t n,
                              int32_t frames, const double *__restrict__ done)
{
    if (is_done(done)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (mm != nullptr && mm[i] != 0) continue;
        const float2 m = mf[i];
        for (int32_t t = 0; t < frames; ++t) {
            const int64_t j = (int64_t)t * n + i;
            dst[j] += b == nullptr ? m.x * a[j] : fmaf(m.y, a[j], -m.x * b[j]);
        }
    }
}

// dst[v] = (m' K src, m K src) for one frame (src float or bf16): the pair
// the single-walk B forward gathers
template <bool kBf16>
__global__ void k_thomson_weight2(const void *__restrict__ src,
                                  const float2 *__restrict__ mf,
                                  const uint8_t *__restrict__ mm, int64_t n,
                                  float2 *__restrict__ dst,
                                  const double *__restrict__ done)
{
    if (is_done(done)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool out = mm != nullptr && mm[i] != 0;
        const float2 m = mf[i];
        float x;
        if (kBf16)
            x = __uint_as_float((unsigned)((const uint16_t *)src)[i] << 16);
        else
            x = ((const float *)src)[i];
        dst[i] = out ? make_float2(0.0f, 0.0f) : make_float2(m.y * x, m.x * x);
    }
}

// dst += K (m' a.x - m a.y) for one frame (a: the single-walk B transpose's
// pair accumulator)
__global__ void k_thomson_add2(float *__restrict__ dst,
                               const float2 *__restrict__ a,
                               const float2 *__restrict__ mf,
                               const uint8_t *__restrict__ mm, int64_t n,
                               const double *__restrict__ done)
{
    if (is_done(done)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (mm != nullptr && mm[i] != 0) continue;
        const float2 m = mf[i];
        const float2 v = a[i];
        dst[i] += fmaf(m.y, v.x, -m.x * v.y);
    }
}

// out = rho^2 y (t == NULL; out may be y), or out = y - rho^2 t
__global__ void k_rho2_apply(const float *__restrict__ rho2, const float *y,
                             const float *__restrict__ t, float *out,
                             int64_t n, const double *__restrict__ done)
{
    if (is_done(done)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = t == nullptr ? rho2[i] * y[i] : fmaf(-rho2[i], t[i], y[i]);
}

}  // namespace

cudaError_t launch_thomson_factors(CubeDev c, double limb_u, float2 *mf,
                                   cudaStream_t s)
{
    const int64_t n = (int64_t)c.nx * c.ny * c.nz;
    if (n <= 0) return cudaSuccess;
    k_thomson_factors<<<grid_for(n), kThreads, 0, s>>>(c, limb_u, mf);
    return cudaGetLastError();
}

cudaError_t launch_impact2(const Frame *frames, const double *tan_u,
                           const double *tan_v, int32_t n_img, int32_t nu,
                           int32_t nv, float *rho2, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    const int64_t npix = (int64_t)nu * nv;
    dim3 grid((unsigned)((npix + 255) / 256), (unsigned)n_img);
    k_impact2<<<grid, 256, 0, s>>>(frames, tan_u, tan_v, nu, nv, rho2);
    return cudaGetLastError();
}

cudaError_t launch_thomson_weight(const void *src, bool bf16, const float2 *mf,
                                  int which, const uint8_t *mm, int64_t n,
                                  int32_t frames, float *dst,
                                  const double *done, cudaStream_t s)
{
    if (n <= 0 || frames <= 0) return cudaSuccess;
    if (bf16)
        k_thomson_weight<true><<<grid_for(n), kThreads, 0, s>>>(
            src, mf, which, mm, n, frames, dst, done);
    else
        k_thomson_weight<false><<<grid_for(n), kThreads, 0, s>>>(
            src, mf, which, mm, n, frames, dst, done);
    return cudaGetLastError();
}

cudaError_t launch_thomson_add(float *dst, const float *a, const float *b,
                               const float2 *mf, const uint8_t *mm, int64_t n,
                               int32_t frames, const double *done,
                               cudaStream_t s)
{
    if (n <= 0 || frames <= 0) return cudaSuccess;
    k_thomson_add<<<grid_for(n), kThreads, 0, s>>>(dst, a, b, mf, mm, n, frames,
                                                   done);
    return cudaGetLastError();
}

cudaError_t launch_thomson_weight2(const void *src, bool bf16,
                                   const float2 *mf, const uint8_t *mm,
                                   int64_t n, float2 *dst, const double *done,
                                   cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (bf16)
        k_thomson_weight2<true><<<grid_for(n), kThreads, 0, s>>>(src, mf, mm, n,
                                                                 dst, done);
    else
        k_thomson_weight2<false><<<grid_for(n), kThreads, 0, s>>>(src, mf, mm, n,
                                                                  dst, done);
    return cudaGetLastError();
}

cudaError_t launch_thomson_add2(float *dst, const float2 *a, const float2 *mf,
                                const uint8_t *mm, int64_t n,
                                const double *done, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_thomson_add2<<<grid_for(n), kThreads, 0, s>>>(dst, a, mf, mm, n, done);
    return cudaGetLastError();
}

cudaError_t launch_rho2_apply(const float *rho2, const float *y, const float *t,
                              float *out, int64_t n, const double *done,
                              cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_rho2_apply<<<grid_for(n), kThreads, 0, s>>>(rho2, y, t, out, n, done);
    return cudaGetLastError();
}

}  // namespace tomo
