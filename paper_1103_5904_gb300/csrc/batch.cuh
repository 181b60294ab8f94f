// Descriptors and launchers of the batched kernels (batch.cu).
#pragma once

#include "tomo_internal.cuh"

namespace tomo {

constexpr int64_t kChunk = 16384;  // elements per vector work item
constexpr int kSchedGroup = 4;     // tiles per walk schedule entry

// One problem as seen by a persistent walk kernel.  Forward: gathers `src`
// (cube) into `dst` (images).  Adjoint: scatters `src` (images) into `dst`
// (cube).  Tiles per image row / column follow the problem's tile shape.
struct WalkDesc {
    const RayRec *rays;
    const ImgParam *prm;
    const uint8_t *mask;
    const float *src;
    float *dst;
    const double *done;
    int32_t nu, nv, nx, nxny;
    int32_t tiles_u, tiles_v;
    Tiling tl;
    int32_t pad;
};

// One problem as seen by the batched vector kernels.
struct VecDesc {
    float *x, *r, *p, *q, *b;
    const float *y;
    const uint8_t *mask;
    double *S;       // the problem's FP64 slots (S_*)
    double *report;  // (n_iter + 1) x 2: J, r.r
    int64_t n, m;    // voxels, pixels
    int32_t nx, ny, nz;
    float lam;
};

int walk_batched_blocks_per_sm();
// sched[c] = (problem, first tile) of chunk c: kSchedGroup consecutive
// tiles of one problem (tiles past the problem's count are skipped)
cudaError_t launch_walk_batched(bool adjoint, const WalkDesc *descs,
                                const int64_t *prefix, const int2 *sched,
                                int64_t n_chunks, unsigned long long *next_item,
                                int grid, cudaStream_t s);
cudaError_t launch_vec_batched(int op, const VecDesc *descs,
                               const int64_t *prefix, int n_probs, bool warm,
                               double *partials, int grid, cudaStream_t s);
cudaError_t launch_finalize_batched(int op, const VecDesc *descs,
                                    const int64_t *prefix, int n_probs,
                                    double tol2, const double *partials,
                                    cudaStream_t s);

// operation codes of launch_vec_batched / launch_finalize_batched
enum : int {
    BV_SUMSQ = 0, BV_ZERO = 1, BV_INIT = 2, BV_PRIOR = 3, BV_PQ = 4,
    BV_UPDATE = 5, BV_DIR = 6, BV_PRIOR_X = 7
};

}  // namespace tomo
