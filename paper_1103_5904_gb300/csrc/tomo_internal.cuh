// Internal declarations of libtomo (not part of the C ABI).
//
// Data layout in device memory
//   RayRec  one 32-byte record per pixel, [n_img][nv][nu]: the Siddon walk of
//           that pixel's line of sight, re-based to its entry point into the
//           cube (built in FP64 by the setup kernel, walked in FP32).
//   ImgParam one 16-byte record per image: gain, time weight, frame index.
//   Frame   per-image FP64 observer frame (o, w, e1, e2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tomo.h"

namespace tomo {

// Walk of one line of sight, relative to its entry point into the cube.
// t is the distance travelled from the entry point.  The walk crosses the
// k-th plane (k = 0, 1, ...) of axis a at t = fmaf(k, |dt_a|, t0_a); the sign
// bit of dt_a is the step direction along a.  The walk ends at t = chord,
// which the setup kernel has already lowered, in the walk's own float
// arithmetic, to the last in-cube plane of every axis, so the voxel index
// never leaves the cube.  chord <= 0 marks a ray that misses the cube.
struct __align__(16) RayRec {
    float t0x, t0y, t0z, chord;
    float dtx, dty, dtz;
    int32_t idx0;  // linear index (within one frame) of the entry voxel
};
static_assert(sizeof(RayRec) == 32, "RayRec must stay 32 bytes");

struct __align__(16) ImgParam {
    float gain;     // image gain g_n
    float w;        // weight w of frame k + 1
    float w0;       // weight 1 - w of frame k (formed in FP64: a float
                    // 1 - w would lose the digits of a w close to 1)
    int32_t pad;    // bits 0-7 plane-walk hint: bits 0-1 major axis M,
                    // bits 2-3 lateral axis L (the layout), bit 4 M
                    // direction < 0, bit 5 set when the hint is valid, bit 6
                    // set when the plane forward is chosen (kPlaneFwdBit),
                    // bit 7 every-slab variant (kPlaneGeneralBit); bits
                    // 8-30 the frame index k (0 when T == 1)
};

__host__ __device__ __forceinline__ int32_t img_frame(const ImgParam &q)
{
    return q.pad >> 8;
}

constexpr int32_t kPlaneHintValid = 32;
constexpr int32_t kPlaneMaxSide = 16384;
// Below this pixel pitch (in voxels of the lateral axis, at the distance of
// Sun centre) a row of 32 rays covers only a few voxels; the per-ray walk,
// which sums the contributions of lanes in the same voxel before its float
// atomic, is faster there (measured crossover between 0.13 and 0.20).
constexpr double kPlaneMinPitch = 0.16;
// Hint bits chosen by measurement (GB300, 24 views of 512^2 around a 256^3
// cube, latitude 0-25 degrees; 64 views of 256^2 for the pixel pitch).
// "lo" is the less steep minor direction component of the image's central
// line of sight over the major one.
//  * kPlaneGeneralBit (lo >= kPlaneGeneralRatio): the plane walks take the
//    general three-segment body on every slab.  The lanes of a warp cross
//    the a2 planes in different slabs once lo is more than about 0.02 (a
//    row's rays differ slightly in slope, and the observer is ~200 cube
//    widths away), so the counted fast loop keeps stopping; the transpose
//    with the counted loop takes 0.46x the per-ray time at lo = 0 and 0.63x
//    at lo = 0.035, where the every-slab variant takes 0.63x.
//  * kPlaneFwdBit: the plane forward is the faster one: with the counted
//    loop when lo < kPlaneFwdMaxRatio (0.81x the per-ray forward at lo = 0,
//    0.94x at 0.017, 1.04x at 0.026), and whenever the pixels are at least
//    kPlaneFwdMinPitch voxels apart, where the per-ray warps share few L1
//    lines (1.22 against 2.14 ms at 1.07 voxel).
constexpr int32_t kPlaneFwdBit = 64;
constexpr double kPlaneFwdMinPitch = 0.75;
constexpr double kPlaneFwdMaxRatio = 0.02;
constexpr int32_t kPlaneGeneralBit = 128;
constexpr double kPlaneGeneralRatio = 0.035;
// The thresholds above as walk rules (the default of every size bucket that
// tomo_autotune or tomo_set_plane_rules has not set).
inline tomo_plane_rules default_plane_rules()
{
    tomo_plane_rules r;
    r.min_pitch = kPlaneMinPitch;
    r.fwd_min_pitch = kPlaneFwdMinPitch;
    r.fwd_max_ratio = kPlaneFwdMaxRatio;
    r.general_ratio = kPlaneGeneralRatio;
    r.fwd_group = 0.0;
    r.adj_group = 0.0;
    return r;
}

// Cube pointers per layout (0 = native x-fastest, 1 = y-fastest,
// 2 = z-fastest) for the plane-synchronous walk (plane.cu).
struct PlaneCubes {
    const void *c[3];
};
struct PlaneAcc {
    float *c[3];
};

struct Frame {
    double o[3], w[3], e1[3], e2[3];
};

struct CubeDev {
    int32_t nx, ny, nz;
    double lo[3], d[3];
    double hi[3];     // lo + n d: the upper faces
    double inv_d[3];  // 1 / d
    double r_obs;     // opaque sphere at the origin (0: none)
};

struct Tiling {
    int32_t tile_u, tile_v, warp_u;
};

// Device-side scalar slots of the CG solver (FP64).
enum : int {
    S_RR = 0,     // r.r of the current residual
    S_PQ = 1,     // p.q
    S_ALPHA = 2,  // step length
    S_BETA = 3,   // direction update
    S_YMY = 4,    // y^T M y
    S_RR0 = 5,    // r0.r0
    S_DONE = 6,   // nonzero: stop (converged or breakdown)
    S_ITERS = 7,  // iterations done
    S_ERR = 8,    // nonzero: numerical breakdown
    S_TOL2 = 9,   // tol^2
    S_NSLOTS = 16
};

constexpr int kMaxReduceBlocks = 2048;

// ---- setup.cu
// vox: voxel size per axis (for the plane-walk hint's pixel-pitch test);
// layout_used (may be NULL): bit L is or-ed in for every image whose plane
// hint is valid and names layout L, bit 8 + L if its hint also selects the
// plane forward.  per_ray_fwd (may be NULL; 1 + n_img words, word 0 zeroed
// by the caller): the images whose hint leaves them to the per-ray forward
// are appended, per_ray_fwd[0] = their count, then their indices in no
// fixed order.
cudaError_t launch_frames(const tomo_pointing *ptg_dev, int32_t n_img,
                          int32_t nu, int32_t nv, int32_t n_frames,
                          Frame *frames, double *tan_u, double *tan_v,
                          ImgParam *params, double3 vox, unsigned *layout_used,
                          unsigned *per_ray_fwd, const tomo_plane_rules &rules,
                          cudaStream_t s);
cudaError_t launch_ray_setup(const Frame *frames, const double *tan_u,
                             const double *tan_v, CubeDev cube, int32_t n_img,
                             int32_t nu, int32_t nv, RayRec *rays,
                             cudaStream_t s);

// ---- siddon.cu
// skip_plane_images: leave the images whose hint has kPlaneFwdBit to the
// plane-synchronous forward (launched with only_marked).  With listed (a
// per_ray_fwd list built by launch_frames) the skipping launch takes about
// one wave of CTAs (num_sms x resident CTAs per SM) that deal out the
// listed images' tiles instead of one CTA per tile of every image: far
// cheaper when the list is short or empty, at a few more registers per
// thread.  A pixel gets the same value from every form.
cudaError_t launch_forward(const RayRec *rays, const ImgParam *prm,
                           const void *cube, tomo_dtype dtype,
                           int64_t frame_stride, bool time_interp,
                           const uint8_t *mask, float *out, int32_t n_img,
                           int32_t nu, int32_t nv, int32_t nx, int32_t nxny,
                           Tiling t, const double *done, cudaStream_t s,
                           bool skip_plane_images = false,
                           const unsigned *listed = nullptr, int num_sms = 0);
cudaError_t launch_adjoint(const RayRec *rays, const ImgParam *prm,
                           const float *images, const uint8_t *mask,
                           float *cube, int64_t frame_stride,
                           bool time_interp, int32_t n_img, int32_t nu,
                           int32_t nv, int32_t nx, int32_t nxny, Tiling t,
                           const double *done, cudaStream_t s);
// plane.cu: plane-synchronous walk on lateral-axis-fastest cube copies.
// The walk kernels use their own tiling: CTAs of 32 x 8 pixels, one image
// row of 32 pixels per warp.  Layout kernels return at once unless bit L of
// *used is set.
// esize: bytes per voxel of the buffers the plane walk addresses (4 for
// float or bf16 cubes, 8 for the two-value pair buffers)
bool plane_supported(const tomo_cube_geom *c, int esize);
// Images per group of the plane walks' CTA order (plane_cta in plane.cuh),
// clamped to [1, n_img] and to the grid's y extent (tiles_v tile rows).
int plane_group_clamp(int group, int n_img, int tiles_v);
// (copies for the forward: runs when bit `bit` of *used is set)
cudaError_t launch_to_layout(const void *cube, tomo_dtype dtype, void *out,
                             int L, const tomo_cube_geom *c, int32_t n_frames,
                             const unsigned *used, unsigned bit,
                             const double *done, cudaStream_t s);
cudaError_t launch_add_from_layout(const float *acc, float *cube, int L,
                                   const tomo_cube_geom *c, int32_t n_frames,
                                   const unsigned *used, const double *done,
                                   cudaStream_t s);
cudaError_t launch_zero_layout(float *acc, int L, int64_t n,
                               const unsigned *used, const double *done,
                               int num_sms, cudaStream_t s);
cudaError_t launch_forward_plane(const RayRec *rays, const ImgParam *prm,
                                 PlaneCubes cubes, tomo_dtype dtype,
                                 int64_t frame_stride, bool time_interp,
                                 const uint8_t *mask, float *out,
                                 int32_t n_img, int32_t nu, int32_t nv,
                                 const tomo_cube_geom *c, const double *done,
                                 cudaStream_t s, bool only_marked, int group);
cudaError_t launch_adjoint_plane(const RayRec *rays, const ImgParam *prm,
                                 const float *images, const uint8_t *mask,
                                 PlaneAcc acc, int64_t frame_stride,
                                 bool time_interp, int32_t n_img, int32_t nu,
                                 int32_t nv, const tomo_cube_geom *c,
                                 const double *done, cudaStream_t s,
                                 int group);
cudaError_t launch_count(const RayRec *rays, const uint8_t *mask,
                         int32_t n_img, int32_t nu, int32_t nv, Tiling t,
                         unsigned long long *count, cudaStream_t s);

// ---- solver.cu
// q = lambda D^T D x, or lambda R D^T D R x with R = diag(w) (w nullable)
cudaError_t launch_prior(CubeDev cube, const float *x, const float *w,
                         float *q, float lam, bool accumulate,
                         const double *done, cudaStream_t s);
// q += lambda_t D_t^T D_t x over T frames of n voxels
cudaError_t launch_prior_time(const float *x, float *q, float lam_t,
                              int64_t n, int32_t T, const double *done,
                              cudaStream_t s);
cudaError_t launch_fill_f32(float *p, float v, int64_t n, cudaStream_t s);
cudaError_t launch_fill_f64(double *p, double v, int64_t n, cudaStream_t s);
// S[S_YMY] = sum over unmasked pixels of y^2
cudaError_t launch_masked_sumsq(const float *y, const uint8_t *mask,
                                int64_t n, double *partials,
                                unsigned int *counter, double *S,
                                int grid, cudaStream_t s);
// r = b - q (or r = b if q == NULL); p = r (+ bf16 copy); S[RR], S[RR0],
// report row 0 from r.r and x.(r + b).  map_mask (nullable, mm_n voxels
// per frame): b, r, p set to 0 on the excluded voxels of every frame.
cudaError_t launch_cg_init(float *b, const float *q, const float *x,
                           float *r, float *p, uint16_t *p16,
                           const uint8_t *map_mask, int64_t mm_n, int64_t n,
                           double tol2,
                           double *partials, unsigned int *counter, double *S,
                           double *report, int grid, cudaStream_t s);
// S[S_PQ] = p.q, S[S_ALPHA] = rr / pq
cudaError_t launch_cg_pq(const float *p, const float *q, int64_t n,
                         double *partials, unsigned int *counter, double *S,
                         int grid, cudaStream_t s);
// x += alpha p; r -= alpha q (r = 0 on voxels excluded by map_mask);
// S[RR] <- r.r, beta, report row
cudaError_t launch_cg_update(float *x, float *r, const float *p,
                             const float *q, const float *b,
                             const uint8_t *map_mask, int64_t mm_n, int64_t n,
                             double *partials, unsigned int *counter,
                             double *S, double *report, int grid,
                             cudaStream_t s);
// p = r + beta p (+ bf16 copy)
cudaError_t launch_cg_direction(const float *r, float *p, uint16_t *p16,
                                int64_t n, const double *S, int grid,
                                cudaStream_t s);

// ---- thomson.cu (T_pB = O P M, T_B = P M' - O P M; Section 3.5)
// per-voxel (m, m') in FP64, stored as float2 [nz][ny][nx]
cudaError_t launch_thomson_factors(CubeDev c, double limb_u, float2 *mf,
                                   cudaStream_t s);
// rho^2 = |o x u|^2 per pixel, [n_img][nv][nu]
cudaError_t launch_impact2(const Frame *frames, const double *tan_u,
                           const double *tan_v, int32_t n_img, int32_t nu,
                           int32_t nv, float *rho2, cudaStream_t s);
// dst = (which ? m' : m) K src over frames (src float32 or bf16 bits)
cudaError_t launch_thomson_weight(const void *src, bool bf16, const float2 *mf,
                                  int which, const uint8_t *mm, int64_t n,
                                  int32_t frames, float *dst,
                                  const double *done, cudaStream_t s);
// dst += K (m a) (b == NULL) or K (m' a - m b)
cudaError_t launch_thomson_add(float *dst, const float *a, const float *b,
                               const float2 *mf, const uint8_t *mm, int64_t n,
                               int32_t frames, const double *done,
                               cudaStream_t s);
// out = rho^2 y (t == NULL), or out = y - rho^2 t
cudaError_t launch_rho2_apply(const float *rho2, const float *y, const float *t,
                              float *out, int64_t n, const double *done,
                              cudaStream_t s);

// dst[v] = (m' K src, m K src), one frame (the single-walk B forward's pairs)
cudaError_t launch_thomson_weight2(const void *src, bool bf16,
                                   const float2 *mf, const uint8_t *mm,
                                   int64_t n, float2 *dst, const double *done,
                                   cudaStream_t s);
// dst += K (m' a.x - m a.y), one frame
cudaError_t launch_thomson_add2(float *dst, const float2 *a, const float2 *mf,
                                const uint8_t *mm, int64_t n,
                                const double *done, cudaStream_t s);

// ---- plane2.cu: two-value plane walks (frame pairs; Thomson B pairs).
// Pair buffers hold two floats per voxel (8 bytes; a bf16 frame pair packs
// into 4 bytes), T - 1 frame pairs or one B pair of n voxels, in layout L.
// Layout passes return at once unless bit `bit` (or bit L) of *used is set.
cudaError_t launch_to_pairs(const void *cube, tomo_dtype dtype, void *out,
                            int L, const tomo_cube_geom *c, int32_t n_frames,
                            const unsigned *used, unsigned bit,
                            const double *done, int num_sms, cudaStream_t s);
// frames += pair accumulators of layout L (frame f: pair f's first value and
// pair f - 1's second)
cudaError_t launch_add_pairs(const void *acc, float *cube, int L,
                             const tomo_cube_geom *c, int32_t n_frames,
                             const unsigned *used, const double *done,
                             int num_sms, cudaStream_t s);
// float2 native buffer -> layout L (1 or 2), and native += layout L
cudaError_t launch_b_to_layout(const void *in, void *out, int L,
                               const tomo_cube_geom *c, const unsigned *used,
                               unsigned bit, const double *done,
                               cudaStream_t s);
cudaError_t launch_add_b_layout(const void *acc, void *out, int L,
                                const tomo_cube_geom *c, const unsigned *used,
                                const double *done, cudaStream_t s);
cudaError_t launch_forward_plane_pair(const RayRec *rays, const ImgParam *prm,
                                      PlaneCubes pairs, const void *native,
                                      tomo_dtype dtype, int64_t fstride,
                                      const uint8_t *mask, float *out,
                                      int32_t n_img, int32_t nu, int32_t nv,
                                      const tomo_cube_geom *c,
                                      const double *done, cudaStream_t s,
                                      bool only_marked, int group);
cudaError_t launch_adjoint_plane_pair(const RayRec *rays, const ImgParam *prm,
                                      const float *images, const uint8_t *mask,
                                      PlaneAcc acc, float *cube,
                                      int64_t fstride, int32_t n_img,
                                      int32_t nu, int32_t nv,
                                      const tomo_cube_geom *c,
                                      const double *done, cudaStream_t s,
                                      int group);
// plane_mode: 0 every image per ray, 1 the images whose hint has the
// plane-forward bit, 2 every image plane by plane (where the hint allows)
cudaError_t launch_forward_b(const RayRec *rays, const ImgParam *prm,
                             PlaneCubes pairs, const float *rho2,
                             const uint8_t *mask, float *out, int32_t n_img,
                             int32_t nu, int32_t nv, const tomo_cube_geom *c,
                             const double *done, int plane_mode,
                             cudaStream_t s, int group);
// plane_on false: every image per ray into acc.c[0]
cudaError_t launch_adjoint_b(const RayRec *rays, const ImgParam *prm,
                             const float *images, const float *rho2,
                             const uint8_t *mask, PlaneAcc acc, int32_t n_img,
                             int32_t nu, int32_t nv, const tomo_cube_geom *c,
                             const double *done, bool plane_on,
                             cudaStream_t s, int group);

// ---- mapmask.cu (map mask K = diag(1 - mask), same mask for every frame)
// dst = K src over `frames` frames of n voxels (float32 or bf16 bits)
cudaError_t launch_map_keep_copy(const void *src, void *dst, bool bf16,
                                 const uint8_t *mm, int64_t n, int32_t frames,
                                 cudaStream_t s);
// x = K x
cudaError_t launch_map_zero(float *x, const uint8_t *mm, int64_t n,
                            int32_t frames, cudaStream_t s);
// dst += K src
cudaError_t launch_map_keep_add(float *dst, const float *src,
                                const uint8_t *mm, int64_t n, int32_t frames,
                                cudaStream_t s);

}  // namespace tomo
