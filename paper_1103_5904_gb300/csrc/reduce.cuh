// FP64 block reductions and the scalar steps of conjugate gradients, shared
// by the single-problem and the batched solvers.
//
// CG on (P^T M P + lambda D^T D) x = P^T M y (Eq. criterion, normal
// equations), textbook Hestenes-Stiefel form:
//   alpha = r.r / p.q;  x += alpha p;  r -= alpha q;
//   beta = r'.r' / r.r; p = r' + beta p.
// The criterion is reported through J = y^T M y - x^T (r + b), exact for
// every CG iterate (b = P^T M y, r = b - A x).
#pragma once

#include <math.h>

#include "tomo_internal.cuh"

namespace tomo {

// A per-thread partial sum kept as a compensated pair of floats.  A product
// of two floats is split exactly into p + e (p = fl(a b) with an unfused
// multiply, e = fmaf(a, b, -p): the FMA-based TwoProduct), and every term
// is added with Knuth's TwoSum, whose rounding error goes to the second
// float.  For the few dozen terms of one thread this is as accurate as FP64
// accumulation of the exact products (the error is of order u^2 times the
// sum of magnitudes), and it runs on the FP32 pipes: GB300 issues FP64 at a
// small fraction of its FP32 rate, and converting every element to FP64
// made the CG vector passes FP64-bound at a third of their memory rate.
// The pairs are summed across threads in FP64.
struct SumF2 {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float a)
    {
        const float s = __fadd_rn(hi, a);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)),
                                  __fsub_rn(a, bb));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        add(p);
        lo = __fadd_rn(lo, e);
    }
    // adds a (b + c), with b + c split exactly by TwoSum first
    __device__ __forceinline__ void add_prod_sum(float a, float b, float c)
    {
        const float s = __fadd_rn(b, c);
        const float bb = __fsub_rn(s, b);
        const float es = __fadd_rn(__fsub_rn(b, __fsub_rn(s, bb)),
                                   __fsub_rn(c, bb));
        add_prod(a, s);
        lo = __fadd_rn(lo, __fmul_rn(a, es));
    }
    __device__ __forceinline__ double value() const
    {
        return (double)hi + (double)lo;
    }
};

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA; valid in thread 0.  Ends with a barrier so `sm` (32
// doubles of shared memory) can be reused by the next call.
__device__ __forceinline__ double block_sum(double v, double *sm)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sm[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sm[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    __syncthreads();
    return v;
}

// Scalar steps; called by one thread with the grid-wide sums.

__device__ __forceinline__ void cg_finalize_init(double *S, double *report,
                                                 double rr, double xrb,
                                                 double tol2)
{
    S[S_RR] = rr;
    S[S_RR0] = rr;
    S[S_TOL2] = tol2;
    S[S_ITERS] = 0.0;
    S[S_ERR] = 0.0;
    S[S_DONE] = (rr == 0.0) ? 1.0 : 0.0;
    if (report != nullptr) {
        report[0] = S[S_YMY] - xrb;
        report[1] = rr;
    }
}

__device__ __forceinline__ void cg_finalize_pq(double *S, double pq)
{
    S[S_PQ] = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
        S[S_DONE] = 1.0;
        S[S_ERR] = 1.0;
    } else {
        S[S_ALPHA] = S[S_RR] / pq;
    }
}

__device__ __forceinline__ void cg_finalize_update(double *S, double *report,
                                                   double rr_new, double xrb)
{
    const int k = (int)S[S_ITERS];
    S[S_BETA] = rr_new / S[S_RR];
    S[S_RR] = rr_new;
    S[S_ITERS] = k + 1;
    if (report != nullptr) {
        report[2 * (k + 1)] = S[S_YMY] - xrb;
        report[2 * (k + 1) + 1] = rr_new;
    }
    if (!isfinite(rr_new)) {
        S[S_DONE] = 1.0;
        S[S_ERR] = 1.0;
    } else if (rr_new <= S[S_TOL2] * S[S_RR0]) {
        S[S_DONE] = 1.0;
    }
}

// The 7-point stencil of lambda D^T D at voxel (i, j, k) of x, or with a
// diagonal weight w (nullable) the stencil of lambda R D^T D R, R = diag(w)
// (the height-weighted prior ||D R x||^2 of Eq. srt_inversion): the
// differences are taken of w x and the result is scaled by w at (i, j, k).
__device__ __forceinline__ float prior_at(const float *__restrict__ x,
                                          const float *__restrict__ w,
                                          int64_t v, int i, int j, int k,
                                          int nx, int ny, int nz, float lam)
{
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    if (w == nullptr) {
        const float xc = x[v];
        float s = 0.0f;
        if (i > 0) s += xc - x[v - 1];
        if (i < nx - 1) s += xc - x[v + 1];
        if (j > 0) s += xc - x[v - sy];
        if (j < ny - 1) s += xc - x[v + sy];
        if (k > 0) s += xc - x[v - sz];
        if (k < nz - 1) s += xc - x[v + sz];
        return lam * s;
    }
    const float wc = w[v];
    const float xc = wc * x[v];
    float s = 0.0f;
    if (i > 0) s += xc - w[v - 1] * x[v - 1];
    if (i < nx - 1) s += xc - w[v + 1] * x[v + 1];
    if (j > 0) s += xc - w[v - sy] * x[v - sy];
    if (j < ny - 1) s += xc - w[v + sy] * x[v + sy];
    if (k > 0) s += xc - w[v - sz] * x[v - sz];
    if (k < nz - 1) s += xc - w[v + sz] * x[v + sz];
    return lam * wc * s;
}

}  // namespace tomo
