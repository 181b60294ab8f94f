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
    int32_t ny, nz;
    // plane-synchronous transpose: accumulators of layouts 1 and 2 (zero
    // between transposes; k_add_from_layout_batched adds them to dst and
    // zeroes them again)
    float *lay1, *lay2;
};

// Plane-synchronous batched transpose tiles: 32 x 8 pixels, one image row of
// 32 pixels per warp.
constexpr int kPlaneTileU = 32, kPlaneTileV = 8;

// One layout buffer of one problem and that problem's native cube, moved in
// 32 x 32 tiles of (x, b) per value of c (layout L: b = y (L = 1) or z
// (L = 2), c = the remaining axis): added into the cube by the batched
// combine kernel (transpose accumulators), or copied from the cube by the
// batched layout-copy kernel (forward).
struct LayoutJob {
    float *acc;
    float *cube;
    const unsigned *used;  // the job runs when (*used & bit) != 0
    const double *done;    // may be NULL
    int32_t L, nx, nb, nc;
    int64_t sb, sc;        // native strides of b and c
    int32_t tiles_x, tiles_b;
    unsigned bit;
    int32_t pad;
};

// One problem as seen by the batched vector kernels.
struct VecDesc {
    float *x, *r, *p, *q, *b;
    const float *y;
    const uint8_t *mask;
    const uint8_t *mm;  // map mask (nullable): restricts b, r, p, x0
    const float *w;     // prior weight R (nullable): lambda R D^T D R
    double *S;       // the problem's FP64 slots (S_*)
    double *report;  // (n_iter + 1) x 2: J, r.r
    int64_t n, m;    // voxels, pixels
    int32_t nx, ny, nz;
    float lam;
};

int walk_batched_blocks_per_sm();
int plane_batched_blocks_per_sm();  // the persistent plane transpose
// sched[c] = (problem, first tile) of chunk c: kSchedGroup consecutive
// tiles of one problem (tiles past the problem's count are skipped)
cudaError_t launch_walk_batched(bool adjoint, const WalkDesc *descs,
                                const int64_t *prefix, const int2 *sched,
                                int64_t n_chunks, unsigned long long *next_item,
                                int grid, cudaStream_t s);
// Plane-synchronous transpose of every problem (work list over plane
// tiles, same schedule format as launch_walk_batched).
cudaError_t launch_adjoint_plane_batched(const WalkDesc *descs,
                                         const int64_t *prefix,
                                         const int2 *sched, int64_t n_chunks,
                                         unsigned long long *next_item,
                                         int grid, cudaStream_t s);
// cube += acc, acc = 0 for every job; prefix[j] = first tile item of job j
cudaError_t launch_add_from_layout_batched(const LayoutJob *jobs,
                                           const int64_t *prefix, int n_jobs,
                                           int grid, cudaStream_t s);
// acc = the cube in layout L, for every job
cudaError_t launch_to_layout_batched(const LayoutJob *jobs,
                                     const int64_t *prefix, int n_jobs,
                                     int grid, cudaStream_t s);
// Forward projection of every problem over the plane tiles (prefix[p]:
// first tile of problem p, prefix[n_probs] = n_tiles), one CTA per tile:
// images whose hint selects the plane forward walk plane-synchronously (on
// the layout copies in descs[p].lay1 / lay2, made by
// launch_to_layout_batched), the others per ray.
cudaError_t launch_forward_plane_batched(const WalkDesc *descs,
                                         const int64_t *prefix, int n_probs,
                                         int64_t n_tiles, cudaStream_t s);
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
