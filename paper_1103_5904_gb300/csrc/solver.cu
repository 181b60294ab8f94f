// Conjugate-gradient building blocks: the finite-difference prior D^T D and
// the vector updates of CG with FP64 reductions.
//
// The criterion (Section 2.2, Eq. criterion) is ||M (y - P x)||^2 +
// lambda ||D x||^2 with D the finite differences along each axis of the map
// (Section 3.3.1).  Reading where the paper is silent: forward differences
// x[i+1] - x[i] along x, y and z without wrap-around, one lambda for all
// axes.  Then D^T D is, on every line, the path-graph Laplacian: a 7-point
// stencil whose end points see only their one neighbour.
//
// CG scalars (alpha, beta, r.r, p.q, the criterion) live in device memory in
// FP64, so the iteration loop needs no host round trip.  Every dot product
// sums its elements per thread in compensated float pairs (SumF2, as
// accurate as FP64 for a thread's share) and then in a two-stage FP64
// reduction: each CTA writes its FP64 partial sum, and the
// last CTA to finish (found with one atomic counter, no waiting) adds the
// partials in a fixed order, which makes the result deterministic, and then
// applies the scalar update of that CG step.  A "done" flag in the same slot
// array lets every later kernel of the loop return at once after
// convergence or a breakdown.
#include <cuda_bf16.h>
#include <math.h>

#include "reduce.cuh"

namespace tomo {

namespace {

constexpr int kThreads = 256;

// Two-stage reduction of K values.  Returns true in the last CTA, where
// total[] (valid in thread 0) holds the grid-wide sums.
template <int K>
__device__ bool grid_sum(double (&v)[K], double *partials,
                         unsigned int *counter, double (&total)[K])
{
    __shared__ double sm[32];
    __shared__ bool last;
    for (int k = 0; k < K; ++k) v[k] = block_sum(v[k], sm);
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) partials[blockIdx.x * K + k] = v[k];
        __threadfence();
        const unsigned int prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x)
            s += __ldcg(partials + i * K + k);
        total[k] = block_sum(s, sm);
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// Stores one element of the CG direction.  With a bf16 copy (p16 != NULL)
// the direction itself is rounded to bf16 (round to nearest even) and the
// float copy keeps exactly that value, so the projector (which gathers the
// bf16 copy), the prior and the vector updates all use the same p, and CG
// stays an exact line search along a slightly perturbed direction.
__device__ __forceinline__ float direction_store(float v, uint16_t *p16,
                                                 int64_t i)
{
    if (p16 == nullptr) return v;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    p16[i] = __bfloat16_as_ushort(h);
    return __bfloat162float(h);
}

__global__ void k_prior(int nx, int ny, int nz, const float *__restrict__ x,
                        const float *__restrict__ w, float *__restrict__ q,
                        float lam, bool accumulate,
                        const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const int64_t v = ((int64_t)k * ny + j) * nx + i;
    const float val = prior_at(x, w, v, i, j, k, nx, ny, nz, lam);
    q[v] = accumulate ? q[v] + val : val;
}

// q += lambda_t D_t^T D_t x over T frames of n voxels (temporal prior of the
// block-diagonal smooth temporal model): frame t gets
// (x[t] - x[t-1]) for t > 0 plus (x[t] - x[t+1]) for t < T - 1.
__global__ void k_prior_time(const float *__restrict__ x, float *__restrict__ q,
                             float lam_t, int64_t n, int32_t T,
                             const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int32_t t = 0; t < T; ++t) {
            const int64_t j = (int64_t)t * n + i;
            const float xc = x[j];
            float s = 0.0f;
            if (t > 0) s += xc - x[j - n];
            if (t < T - 1) s += xc - x[j + n];
            q[j] += lam_t * s;
        }
    }
}

__global__ void k_fill_f32(float *p, float v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_fill_f64(double *p, double v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_masked_sumsq(const float *__restrict__ y,
                               const uint8_t *__restrict__ mask, int64_t n,
                               double *partials, unsigned int *counter,
                               double *S)
{
    SumF2 a;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (mask == nullptr || mask[i] == 0) {
            const float yi = y[i];
            a.add_prod(yi, yi);
        }
    }
    double v[1] = { a.value() };
    double tot[1];
    if (grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0)
        S[S_YMY] = tot[0];
}

// With a map mask (mm != NULL, mm_n voxels per frame, the same mask for
// every frame) b, r and p are set to 0 on the excluded voxels, so every
// later iterate stays in the restricted space.  Masked vectors are walked
// voxel by voxel with the frames in an inner loop, so each mask byte is read
// once and no index needs a division.
struct CgInitElem {
    float *b;
    const float *q, *x;
    float *r, *p;
    uint16_t *p16;
    __device__ __forceinline__ void operator()(int64_t i, bool out,
                                               SumF2 v[2]) const
    {
        if (out) b[i] = 0.0f;
        const float bi = out ? 0.0f : b[i];
        const float ri = out ? 0.0f : ((q != nullptr) ? bi - q[i] : bi);
        r[i] = ri;
        p[i] = direction_store(ri, p16, i);
        v[0].add_prod(ri, ri);
        if (x != nullptr) v[1].add_prod_sum(x[i], ri, bi);
    }
};

// Calls f(i, excluded, v) for every element of n = frames * mm_n (mm_n = n
// without a mask) in a grid-stride order.
template <class F>
__device__ __forceinline__ void masked_elements(const uint8_t *__restrict__ mm,
                                                int64_t mm_n, int64_t n,
                                                const F &f, SumF2 v[2])
{
    const int64_t start = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (mm == nullptr) {
        for (int64_t i = start; i < n; i += stride) f(i, false, v);
        return;
    }
    for (int64_t i = start; i < mm_n; i += stride) {
        const bool out = mm[i] != 0;
        for (int64_t j = i; j < n; j += mm_n) f(j, out, v);
    }
}

__global__ void k_cg_init(float *__restrict__ b, const float *__restrict__ q,
                          const float *__restrict__ x, float *__restrict__ r,
                          float *__restrict__ p, uint16_t *__restrict__ p16,
                          const uint8_t *__restrict__ mm, int64_t mm_n,
                          int64_t n, double tol2, double *partials,
                          unsigned int *counter, double *S, double *report)
{
    SumF2 a[2];
    const CgInitElem f = { b, q, x, r, p, p16 };
    masked_elements(mm, mm_n, n, f, a);
    double v[2] = { a[0].value(), a[1].value() };
    double tot[2];
    if (grid_sum<2>(v, partials, counter, tot) && threadIdx.x == 0)
        cg_finalize_init(S, report, tot[0], tot[1], tol2);
}

__global__ void k_cg_pq(const float *__restrict__ p, const float *__restrict__ q,
                        int64_t n, double *partials, unsigned int *counter,
                        double *S)
{
    if (S[S_DONE] != 0.0) return;
    SumF2 a;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a.add_prod(p[i], q[i]);
    double v[1] = { a.value() };
    double tot[1];
    if (grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0)
        cg_finalize_pq(S, tot[0]);
}

// With a map mask the residual stays 0 on the excluded voxels (q there is
// the unrestricted operator's value; p, x and b are already 0).
struct CgUpdateElem {
    float *x, *r;
    const float *p, *q, *b;
    float alpha;
    __device__ __forceinline__ void operator()(int64_t i, bool out,
                                               SumF2 v[2]) const
    {
        const float xi = fmaf(alpha, p[i], x[i]);
        const float ri = out ? 0.0f : fmaf(-alpha, q[i], r[i]);
        x[i] = xi;
        r[i] = ri;
        v[0].add_prod(ri, ri);
        v[1].add_prod_sum(xi, ri, b[i]);
    }
};

__global__ void k_cg_update(float *__restrict__ x, float *__restrict__ r,
                            const float *__restrict__ p,
                            const float *__restrict__ q,
                            const float *__restrict__ b,
                            const uint8_t *__restrict__ mm, int64_t mm_n,
                            int64_t n, double *partials,
                            unsigned int *counter, double *S, double *report)
{
    if (S[S_DONE] != 0.0) return;
    SumF2 a[2];
    const CgUpdateElem f = { x, r, p, q, b, (float)S[S_ALPHA] };
    masked_elements(mm, mm_n, n, f, a);
    double v[2] = { a[0].value(), a[1].value() };
    double tot[2];
    if (grid_sum<2>(v, partials, counter, tot) && threadIdx.x == 0)
        cg_finalize_update(S, report, tot[0], tot[1]);
}

__global__ void k_cg_direction(const float *__restrict__ r, float *p,
                               uint16_t *__restrict__ p16, int64_t n,
                               const double *__restrict__ S)
{
    if (S[S_DONE] != 0.0) return;
    const float beta = (float)S[S_BETA];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        p[i] = direction_store(fmaf(beta, p[i], r[i]), p16, i);
    }
}

unsigned int fill_grid(int64_t n)
{
    const int64_t g = (n + kThreads - 1) / kThreads;
    return (unsigned int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

cudaError_t launch_prior(CubeDev c, const float *x, const float *w, float *q,
                         float lam, bool accumulate, const double *done,
                         cudaStream_t s)
{
    const dim3 block(32, 8);
    const dim3 grid((unsigned)((c.nx + 31) / 32), (unsigned)((c.ny + 7) / 8),
                    (unsigned)c.nz);
    k_prior<<<grid, block, 0, s>>>(c.nx, c.ny, c.nz, x, w, q, lam, accumulate,
                                   done);
    return cudaGetLastError();
}

cudaError_t launch_prior_time(const float *x, float *q, float lam_t,
                              int64_t n, int32_t T, const double *done,
                              cudaStream_t s)
{
    if (n <= 0 || T <= 1) return cudaSuccess;
    k_prior_time<<<fill_grid(n), kThreads, 0, s>>>(x, q, lam_t, n, T, done);
    return cudaGetLastError();
}

cudaError_t launch_fill_f32(float *p, float v, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_fill_f32<<<fill_grid(n), kThreads, 0, s>>>(p, v, n);
    return cudaGetLastError();
}

cudaError_t launch_fill_f64(double *p, double v, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_fill_f64<<<fill_grid(n), kThreads, 0, s>>>(p, v, n);
    return cudaGetLastError();
}

cudaError_t launch_masked_sumsq(const float *y, const uint8_t *mask,
                                int64_t n, double *partials,
                                unsigned int *counter, double *S, int grid,
                                cudaStream_t s)
{
    k_masked_sumsq<<<grid, kThreads, 0, s>>>(y, mask, n, partials, counter, S);
    return cudaGetLastError();
}

cudaError_t launch_cg_init(float *b, const float *q, const float *x,
                           float *r, float *p, uint16_t *p16,
                           const uint8_t *map_mask, int64_t mm_n, int64_t n,
                           double tol2, double *partials,
                           unsigned int *counter, double *S, double *report,
                           int grid, cudaStream_t s)
{
    k_cg_init<<<grid, kThreads, 0, s>>>(b, q, x, r, p, p16, map_mask,
                                        mm_n > 0 ? mm_n : 1, n, tol2,
                                        partials, counter, S, report);
    return cudaGetLastError();
}

cudaError_t launch_cg_pq(const float *p, const float *q, int64_t n,
                         double *partials, unsigned int *counter, double *S,
                         int grid, cudaStream_t s)
{
    k_cg_pq<<<grid, kThreads, 0, s>>>(p, q, n, partials, counter, S);
    return cudaGetLastError();
}

cudaError_t launch_cg_update(float *x, float *r, const float *p,
                             const float *q, const float *b,
                             const uint8_t *map_mask, int64_t mm_n, int64_t n,
                             double *partials, unsigned int *counter,
                             double *S, double *report, int grid,
                             cudaStream_t s)
{
    k_cg_update<<<grid, kThreads, 0, s>>>(x, r, p, q, b, map_mask,
                                          mm_n > 0 ? mm_n : 1, n, partials,
                                          counter, S, report);
    return cudaGetLastError();
}

cudaError_t launch_cg_direction(const float *r, float *p, uint16_t *p16,
                                int64_t n, const double *S, int grid,
                                cudaStream_t s)
{
    k_cg_direction<<<grid, kThreads, 0, s>>>(r, p, p16, n, S);
    return cudaGetLastError();
}

}  // namespace tomo
