// Batched projector, transpose and CG over many independent problems of
// uneven sizes (cube side, image count and image size differ per problem).
//
// Ray kernels are persistent: one grid of (SM count x resident CTAs) CTAs
// strides over the work list until it is exhausted.  A work unit is one warp
// tile (32 pixels) of one pixel tile of one image of one problem; the
// schedule deals groups of kSchedGroup tiles round-robin over the problems,
// so every warp's share mixes all problems evenly, and the transposes of all
// problems run side by side with their float atomics spread over every cube
// instead of piling onto one small cube at a time.  Each problem carries its own tile shape (256
// threads per CTA for all of them), chosen by the autotuner.  The walk is the same
// Siddon walk as the single-problem kernels (walk.cuh).
//
// Vector kernels run over (problem, chunk of kChunk elements) items: a CTA
// handles one chunk, writes its FP64 partial sums, and a finalize kernel
// with one CTA per problem adds that problem's partials in a fixed order and
// applies the CG scalar step (reduce.cuh).  Every problem has its own FP64
// slots and "done" flag, so problems that converge early stop working while
// the others continue.
#include <cuda_bf16.h>

#include "batch.cuh"
#include "plane.cuh"
#include "reduce.cuh"
#include "walk.cuh"

namespace tomo {

namespace {

constexpr int kThreads = 256;

// Problem owning `item`: the largest p with prefix[p] <= item.
__device__ __forceinline__ int owner(const int64_t *__restrict__ prefix,
                                     int n_probs, int64_t item)
{
    int lo = 0, hi = n_probs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <bool kAdjoint>
__global__ void __launch_bounds__(kThreads, 6)
k_walk_batched(const WalkDesc *__restrict__ descs,
               const int64_t *__restrict__ prefix,
               const int2 *__restrict__ sched, int64_t n_chunks,
               unsigned long long *next_item)
{
    // CTAs take tiles from a work queue (one atomic counter); warp w of the
    // CTA walks warp tile w of the tile, and a barrier per tile keeps the
    // CTA's warps together: their rays are neighbours that sweep the same
    // voxels at the same depth, which is what the L1 reuses (measured:
    // without the barrier, or with static striding, the walks run slower).
    // The fetch of the next tile is issued when the current one starts and
    // read after its walk: in the transpose the counter shares the L2 atomic
    // units with every segment's reduction, and a fetch waited for at the
    // barrier would park the whole CTA in that queue.
    __shared__ long long s_item;
    const int lane = threadIdx.x & 31;
    const int wt = threadIdx.x >> 5;  // warp tile in the tile
    const int64_t n_items = n_chunks * kSchedGroup;
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(next_item, 1ull);
    __syncthreads();
    int64_t item = s_item;
    while (item < n_items) {
        unsigned long long ahead = 0;
        if (threadIdx.x == 0) ahead = atomicAdd(next_item, 1ull);
        do {
            const int2 ch = sched[item / kSchedGroup];
            const int p = ch.x;
            const int t = ch.y + (int)(item % kSchedGroup);
            if (t >= (int)(prefix[p + 1] - prefix[p])) continue;
            const WalkDesc d = descs[p];
            if (d.done != nullptr && *d.done != 0.0) continue;
            const int tu = t % d.tiles_u;
            const int rest = t / d.tiles_u;
            const int tv = rest % d.tiles_v;
            const int img = rest / d.tiles_v;
            // the pixel of this lane: warp tile wt of tile (tu, tv), laid out as
            // in the single-problem kernels
            const int rows = 32 / d.tl.warp_u;
            const int warps_u = d.tl.tile_u / d.tl.warp_u;
            const int iu = tu * d.tl.tile_u + (wt % warps_u) * d.tl.warp_u +
                           (lane % d.tl.warp_u);
            const int iv = tv * d.tl.tile_v + (wt / warps_u) * rows +
                           (lane / d.tl.warp_u);
            if (iu >= d.nu || iv >= d.nv) continue;
            const int64_t id = ((int64_t)img * d.nv + iv) * d.nu + iu;
            const bool masked = d.mask != nullptr && d.mask[id] != 0;
            const float gain = d.prm[img].gain;
            if (!kAdjoint) {
                float y = 0.0f;
                if (!masked) {
                    const RayRec r = load_ray(d.rays + id);
                    if (r.chord > 0.0f) {
                        GatherOp<float> op;
                        op.c = d.src;
                        op.acc = 0.0f;
                        siddon_gather(r, d.nx, d.nxny, op);
                        y = gain * op.acc;
                    }
                }
                d.dst[id] = y;
            } else if (!masked) {
                const float yv = gain * d.src[id];
                if (yv != 0.0f) {
                    const RayRec r = load_ray(d.rays + id);
                    if (r.chord > 0.0f) {
                        ScatterOp op;
                        op.c = d.dst;
                        op.y = yv;
                        siddon_walk(r, d.nx, d.nxny, op);
                    }
                }
            }
        } while (false);
        __syncthreads();  // every thread has read s_item
        if (threadIdx.x == 0) s_item = (long long)ahead;
        __syncthreads();
        item = s_item;
    }
}

// Plane-synchronous transpose over the plane tiles of every problem, with
// the work queue of k_walk_batched.  All lanes of a warp take part in the
// plane walk's votes, so lanes outside the image only vote.
__global__ void __launch_bounds__(kThreads, 5)
k_adjoint_plane_batched(const WalkDesc *__restrict__ descs,
                        const int64_t *__restrict__ prefix,
                        const int2 *__restrict__ sched, int64_t n_chunks,
                        unsigned long long *next_item)
{
    __shared__ long long s_item;
    const int lane = threadIdx.x & 31;
    const int wt = threadIdx.x >> 5;  // image row of the tile
    const int64_t n_items = n_chunks * kSchedGroup;
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(next_item, 1ull);
    __syncthreads();
    int64_t item = s_item;
    while (item < n_items) {
        unsigned long long ahead = 0;
        if (threadIdx.x == 0) ahead = atomicAdd(next_item, 1ull);
        const int2 ch = sched[item / kSchedGroup];
        const int p = ch.x;
        const int t = ch.y + (int)(item % kSchedGroup);
        // t, p and the done flag are the same for every thread of the CTA
        if (t < (int)(prefix[p + 1] - prefix[p])) {
            const WalkDesc d = descs[p];
            if (d.done == nullptr || *d.done == 0.0) {
                const int tiles_u = (d.nu + kPlaneTileU - 1) / kPlaneTileU;
                const int tiles_v = (d.nv + kPlaneTileV - 1) / kPlaneTileV;
                const int tu = t % tiles_u;
                const int rest = t / tiles_u;
                const int tv = rest % tiles_v;
                const int img = rest / tiles_v;
                const int iu = tu * kPlaneTileU + lane;
                const int iv = tv * kPlaneTileV + wt;
                const bool in_img = iu < d.nu && iv < d.nv;
                const int64_t id = ((int64_t)img * d.nv + iv) * d.nu + iu;
                const ImgParam q = d.prm[img];
                RayRec r;
                r.chord = -1.0f;
                float yv = 0.0f;
                if (in_img && (d.mask == nullptr || d.mask[id] == 0)) {
                    yv = q.gain * d.src[id];
                    if (yv != 0.0f) r = load_ray(d.rays + id);
                }
                const bool live = r.chord > 0.0f;
                PlaneRay pr;
                const bool regular =
                    live && plane_ray(r, q.pad, d.nx, d.ny, d.nz, pr,
                                         sizeof(float));
                const int L = (q.pad >> 2) & 3;
                PlaneScatterOp op;
                op.c = L == 1 ? d.lay1 : (L == 2 ? d.lay2 : d.dst);
                op.y = yv;
                plane_walk_for(q.pad, pr, regular, op);
                if (live && !regular) {
                    ScatterOp op2;
                    op2.c = d.dst;
                    op2.y = yv;
                    siddon_walk(r, d.nx, d.nxny, op2);
                }
            }
        }
        __syncthreads();  // every thread has read s_item
        if (threadIdx.x == 0) s_item = (long long)ahead;
        __syncthreads();
        item = s_item;
    }
}

// Layout accumulators back into the native cubes: one CTA per 32 x 32 tile
// of (x, b) at one c, reading the accumulator along b and adding into the
// cube along x (both coalesced, the additions atomic); the accumulator is
// zeroed as it is read.
__global__ void __launch_bounds__(kThreads)
k_add_from_layout_batched(const LayoutJob *__restrict__ jobs,
                          const int64_t *__restrict__ prefix, int n_jobs)
{
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t n_items = prefix[n_jobs];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int j = owner(prefix, n_jobs, item);
        const LayoutJob J = jobs[j];
        // the same for every thread of the CTA
        if (!(*J.used & J.bit) || (J.done != nullptr && *J.done != 0.0))
            continue;
        const int64_t k = item - prefix[j];
        const int x0 = (int)(k % J.tiles_x) * 32;
        const int64_t r = k / J.tiles_x;
        const int b0 = (int)(r % J.tiles_b) * 32;
        const int c = (int)(r / J.tiles_b);
        for (int i = ty; i < 32; i += 8) {
            const int x = x0 + i, b = b0 + tx;
            if (b < J.nb && x < J.nx) {
                const int64_t a = b + (int64_t)J.nb * (x + (int64_t)J.nx * c);
                tile[tx][i] = J.acc[a];
                J.acc[a] = 0.0f;
            }
        }
        __syncthreads();
        // the jobs of layouts 1 and 2 of one problem run in this same launch
        // and add into the same cube: the additions must be atomic
        for (int i = ty; i < 32; i += 8) {
            const int b = b0 + i, x = x0 + tx;
            if (b < J.nb && x < J.nx) red_add(J.cube + x + J.sb * b + J.sc * c, tile[i][tx]);
        }
        __syncthreads();
    }
}

// The problems' cubes into their layout copies (the inverse tile move of
// k_add_from_layout_batched: read along x, write along b).
__global__ void __launch_bounds__(kThreads)
k_to_layout_batched(const LayoutJob *__restrict__ jobs,
                    const int64_t *__restrict__ prefix, int n_jobs)
{
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t n_items = prefix[n_jobs];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int j = owner(prefix, n_jobs, item);
        const LayoutJob J = jobs[j];
        // the same for every thread of the CTA
        if (!(*J.used & J.bit) || (J.done != nullptr && *J.done != 0.0))
            continue;
        const int64_t k = item - prefix[j];
        const int x0 = (int)(k % J.tiles_x) * 32;
        const int64_t r = k / J.tiles_x;
        const int b0 = (int)(r % J.tiles_b) * 32;
        const int c = (int)(r / J.tiles_b);
        for (int i = ty; i < 32; i += 8) {
            const int b = b0 + i, x = x0 + tx;
            if (b < J.nb && x < J.nx) tile[i][tx] = J.cube[x + J.sb * b + J.sc * c];
        }
        __syncthreads();
        for (int i = ty; i < 32; i += 8) {
            const int x = x0 + i, b = b0 + tx;
            if (b < J.nb && x < J.nx)
                J.acc[b + (int64_t)J.nb * (x + (int64_t)J.nx * c)] = tile[tx][i];
        }
        __syncthreads();
    }
}

// Forward projection over the plane tiles of every problem: one CTA per
// tile, tiles taken problem by problem (a CTA finds its problem by a binary
// search of the tile prefix), so the CTAs resident at one time gather from
// one problem's cube and layout copies.  A CTA covers 32 x 8 pixels of one
// image; when the image's hint selects the plane forward the warps walk
// plane by plane on the layout copies, with the gather bodies free of slot
// predicates and six slabs of loads in flight as in the single-problem
// forward (irregular lanes per ray on the native cube), otherwise every
// lane walks its own ray.  Measured on the 32-problem workload: 10.34 ms
// per projection against 11.0 for a persistent work-queue kernel (whose
// loop state left no registers for the predicate-free bodies) and 10.29
// for the single-problem calls one after another.
__global__ void __launch_bounds__(kThreads, 4)
k_forward_plane_batched(const WalkDesc *__restrict__ descs,
                        const int64_t *__restrict__ prefix, int n_probs)
{
    const int lane = threadIdx.x & 31;
    const int wt = threadIdx.x >> 5;  // image row of the tile
    const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (tile >= prefix[n_probs]) return;
    int lo = 0, hi = n_probs;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= tile) lo = mid;
        else hi = mid;
    }
    const int p = lo;
    const int t = (int)(tile - prefix[p]);
    const WalkDesc &d = descs[p];
    if (d.done != nullptr && *d.done != 0.0) return;
    const int tiles_u = (d.nu + kPlaneTileU - 1) / kPlaneTileU;
    const int tiles_v = (d.nv + kPlaneTileV - 1) / kPlaneTileV;
    const int tu = t % tiles_u;
    const int rest = t / tiles_u;
    const int tv = rest % tiles_v;
    const int img = rest / tiles_v;
    const int iu = tu * kPlaneTileU + lane;
    const int iv = tv * kPlaneTileV + wt;
    const bool in_img = iu < d.nu && iv < d.nv;
    const int64_t id = ((int64_t)img * d.nv + iv) * d.nu + iu;
    const ImgParam q = d.prm[img];
    RayRec r;
    r.chord = -1.0f;
    if (in_img && (d.mask == nullptr || d.mask[id] == 0))
        r = load_ray(d.rays + id);
    const bool live = r.chord > 0.0f;
    float acc = 0.0f;
    if (q.pad & kPlaneFwdBit) {
        PlaneRay pr;
        const bool regular =
            live && plane_ray(r, q.pad, d.nx, d.ny, d.nz, pr, sizeof(float));
        const int L = (q.pad >> 2) & 3;
        PlaneGatherOp<float> op;
        op.c = L == 1 ? d.lay1 : (L == 2 ? d.lay2 : d.src);
        op.acc = 0.0f;
        plane_walk_for<6>(q.pad, pr, regular, op);
        acc = op.acc;
        if (live && !regular) {
            GatherOp<float> op2;
            op2.c = d.src;
            op2.acc = 0.0f;
            siddon_gather(r, d.nx, d.nxny, op2);
            acc = op2.acc;
        }
    } else if (live) {
        GatherOp<float> op2;
        op2.c = d.src;
        op2.acc = 0.0f;
        siddon_gather(r, d.nx, d.nxny, op2);
        acc = op2.acc;
    }
    if (in_img) d.dst[id] = q.gain * acc;
}

// Operation codes (batch.cuh): what one vector pass does.
constexpr int V_SUMSQ = BV_SUMSQ, V_ZERO = BV_ZERO, V_INIT = BV_INIT,
              V_PRIOR = BV_PRIOR, V_PQ = BV_PQ, V_UPDATE = BV_UPDATE,
              V_DIR = BV_DIR, V_PRIOR_X = BV_PRIOR_X;

__global__ void __launch_bounds__(kThreads)
k_vec_batched(int op, const VecDesc *__restrict__ descs,
              const int64_t *__restrict__ prefix, int n_probs, bool warm,
              double *partials)
{
    __shared__ double sm[32];
    const int64_t n_items = prefix[n_probs];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int p = owner(prefix, n_probs, item);
        const VecDesc d = descs[p];  // a copy: stores below cannot alias it
        const int64_t len = (op == V_SUMSQ) ? d.m : d.n;
        // this item's chunk of its problem: elements [c.c0, c.c1)
        struct { int64_t c0, c1; } c;
        c.c0 = (item - prefix[p]) * kChunk;
        c.c1 = c.c0 + kChunk < len ? c.c0 + kChunk : len;
        // per-thread sums in compensated float pairs (SumF2), then FP64
        SumF2 a0, a1;
        const bool done = d.S[S_DONE] != 0.0;
        if (op == V_SUMSQ) {
            for (int64_t i = c.c0 + threadIdx.x; i < c.c1; i += blockDim.x)
                if (d.mask == nullptr || d.mask[i] == 0) {
                    const float yi = d.y[i];
                    a0.add_prod(yi, yi);
                }
        } else if (op == V_ZERO) {
            for (int64_t i = c.c0 + threadIdx.x; i < c.c1; i += blockDim.x) {
                d.b[i] = 0.0f;
                if (!warm || (d.mm != nullptr && d.mm[i] != 0)) d.x[i] = 0.0f;
            }
        } else if (op == V_INIT) {
            // map mask: b, r, p are 0 on the excluded voxels, so every
            // iterate stays in the restricted space
            for (int64_t i = c.c0 + threadIdx.x; i < c.c1; i += blockDim.x) {
                const bool out = d.mm != nullptr && d.mm[i] != 0;
                if (out) d.b[i] = 0.0f;
                const float bi = out ? 0.0f : d.b[i];
                const float ri = out ? 0.0f : (warm ? bi - d.q[i] : bi);
                d.r[i] = ri;
                d.p[i] = ri;
                a0.add_prod(ri, ri);
                if (warm) a1.add_prod_sum(d.x[i], ri, bi);
            }
        } else if (op == V_PRIOR || op == V_PRIOR_X) {
            if (!done) {
                const float *src = (op == V_PRIOR_X) ? d.x : d.p;
                const int nx = d.nx, ny = d.ny, nz = d.nz;
                for (int64_t v = c.c0 + threadIdx.x; v < c.c1; v += blockDim.x) {
                    const int i = (int)(v % nx);
                    const int64_t r = v / nx;
                    const int j = (int)(r % ny), k = (int)(r / ny);
                    d.q[v] = prior_at(src, d.w, v, i, j, k, nx, ny, nz, d.lam);
                }
            }
        } else if (op == V_PQ) {
            if (!done)
                for (int64_t i = c.c0 + threadIdx.x; i < c.c1; i += blockDim.x)
                    a0.add_prod(d.p[i], d.q[i]);
        } else if (op == V_UPDATE) {
            if (!done) {
                const float alpha = (float)d.S[S_ALPHA];
                for (int64_t i = c.c0 + threadIdx.x; i < c.c1; i += blockDim.x) {
                    const float xi = fmaf(alpha, d.p[i], d.x[i]);
                    const float ri = (d.mm != nullptr && d.mm[i] != 0)
                                         ? 0.0f
                                         : fmaf(-alpha, d.q[i], d.r[i]);
                    d.x[i] = xi;
                    d.r[i] = ri;
                    a0.add_prod(ri, ri);
                    a1.add_prod_sum(xi, ri, d.b[i]);
                }
            }
        } else if (op == V_DIR) {
            if (!done) {
                const float beta = (float)d.S[S_BETA];
                for (int64_t i = c.c0 + threadIdx.x; i < c.c1; i += blockDim.x)
                    d.p[i] = fmaf(beta, d.p[i], d.r[i]);
            }
        }
        if (op == V_SUMSQ || op == V_INIT || op == V_PQ || op == V_UPDATE) {
            const double s0 = block_sum(a0.value(), sm);
            const double s1 = block_sum(a1.value(), sm);
            if (threadIdx.x == 0) {
                partials[2 * item] = s0;
                partials[2 * item + 1] = s1;
            }
        }
    }
}

// One CTA per problem: add its partials in item order, apply the step.
__global__ void __launch_bounds__(kThreads)
k_finalize_batched(int op, const VecDesc *__restrict__ descs,
                   const int64_t *__restrict__ prefix, int n_probs,
                   double tol2, const double *__restrict__ partials)
{
    __shared__ double sm[32];
    for (int p = blockIdx.x; p < n_probs; p += gridDim.x) {
        const VecDesc d = descs[p];
        if ((op == V_PQ || op == V_UPDATE) && d.S[S_DONE] != 0.0) continue;
        double s0 = 0.0, s1 = 0.0;
        for (int64_t i = prefix[p] + threadIdx.x; i < prefix[p + 1];
             i += blockDim.x) {
            s0 += partials[2 * i];
            s1 += partials[2 * i + 1];
        }
        s0 = block_sum(s0, sm);
        s1 = block_sum(s1, sm);
        if (threadIdx.x != 0) continue;
        if (op == V_SUMSQ)
            d.S[S_YMY] = s0;
        else if (op == V_INIT)
            cg_finalize_init(d.S, d.report, s0, s1, tol2);
        else if (op == V_PQ)
            cg_finalize_pq(d.S, s0);
        else if (op == V_UPDATE)
            cg_finalize_update(d.S, d.report, s0, s1);
    }
}

}  // namespace

int walk_batched_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, k_walk_batched<false>, kThreads, 0) != cudaSuccess)
        return 1;
    int m = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &m, k_walk_batched<true>, kThreads, 0) != cudaSuccess)
        return 1;
    return n < m ? (n > 0 ? n : 1) : (m > 0 ? m : 1);
}

int plane_batched_blocks_per_sm()
{
    int q = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &q, k_adjoint_plane_batched, kThreads, 0) != cudaSuccess)
        return 1;
    return q > 0 ? q : 1;
}

cudaError_t launch_walk_batched(bool adjoint, const WalkDesc *descs,
                                const int64_t *prefix, const int2 *sched,
                                int64_t n_chunks, unsigned long long *next_item,
                                int grid, cudaStream_t s)
{
    if (adjoint)
        k_walk_batched<true><<<grid, kThreads, 0, s>>>(descs, prefix, sched,
                                                        n_chunks, next_item);
    else
        k_walk_batched<false><<<grid, kThreads, 0, s>>>(descs, prefix, sched,
                                                         n_chunks, next_item);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_plane_batched(const WalkDesc *descs,
                                         const int64_t *prefix,
                                         const int2 *sched, int64_t n_chunks,
                                         unsigned long long *next_item,
                                         int grid, cudaStream_t s)
{
    k_adjoint_plane_batched<<<grid, kThreads, 0, s>>>(descs, prefix, sched,
                                                      n_chunks, next_item);
    return cudaGetLastError();
}

cudaError_t launch_add_from_layout_batched(const LayoutJob *jobs,
                                           const int64_t *prefix, int n_jobs,
                                           int grid, cudaStream_t s)
{
    if (n_jobs <= 0) return cudaSuccess;
    k_add_from_layout_batched<<<grid, kThreads, 0, s>>>(jobs, prefix, n_jobs);
    return cudaGetLastError();
}

cudaError_t launch_to_layout_batched(const LayoutJob *jobs,
                                     const int64_t *prefix, int n_jobs,
                                     int grid, cudaStream_t s)
{
    if (n_jobs <= 0) return cudaSuccess;
    k_to_layout_batched<<<grid, kThreads, 0, s>>>(jobs, prefix, n_jobs);
    return cudaGetLastError();
}

cudaError_t launch_forward_plane_batched(const WalkDesc *descs,
                                         const int64_t *prefix, int n_probs,
                                         int64_t n_tiles, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    const int64_t gx = n_tiles < 65536 ? n_tiles : 65536;
    const dim3 grid((unsigned)gx, (unsigned)((n_tiles + gx - 1) / gx));
    k_forward_plane_batched<<<grid, kThreads, 0, s>>>(descs, prefix, n_probs);
    return cudaGetLastError();
}

cudaError_t launch_vec_batched(int op, const VecDesc *descs,
                               const int64_t *prefix, int n_probs, bool warm,
                               double *partials, int grid, cudaStream_t s)
{
    k_vec_batched<<<grid, kThreads, 0, s>>>(op, descs, prefix, n_probs, warm,
                                            partials);
    return cudaGetLastError();
}

cudaError_t launch_finalize_batched(int op, const VecDesc *descs,
                                    const int64_t *prefix, int n_probs,
                                    double tol2, const double *partials,
                                    cudaStream_t s)
{
    const int grid = n_probs < 1024 ? n_probs : 1024;
    k_finalize_batched<<<grid, kThreads, 0, s>>>(op, descs, prefix, n_probs,
                                                 tol2, partials);
    return cudaGetLastError();
}

}  // namespace tomo
