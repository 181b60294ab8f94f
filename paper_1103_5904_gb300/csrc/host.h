// Host-side internals of libtomo shared by the C ABI translation units:
// the context, argument checks, workspace growth, launch accounting.
#pragma once

#include <stdarg.h>
#include <stdint.h>

#include <vector>

#include <cuda_runtime.h>

#include "tomo_internal.cuh"

namespace tomo {
namespace host {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// The schedule of one size bucket (cube voxel counts, image size): the
// per-ray tile shape and the walk rules, set by the autotuner (or the
// rules by tomo_set_plane_rules).
struct Tuned {
    int32_t nx, ny, nz, nu, nv;
    Tiling tl;
    float fwd_ms, adj_ms;
    tomo_plane_rules rules;
};

struct BatchPlan;  // batch_api.cu

}  // namespace host
}  // namespace tomo

struct tomo_ctx {
    int device = 0;
    int num_sms = 0;
    int64_t l2_bytes = 0;
    // images per group of the plane walks' CTA order (TOMO_OPT_GROUP_FWD /
    // TOMO_OPT_GROUP_ADJ); 0: chosen from the bytes a walk touches
    int group_fwd = 0, group_adj = 0;
    char err[512] = { 0 };
    bool ray_cache = true;
    // bit 0: P^T plane-synchronous; bit 1: P plane-synchronous for every
    // image; bit 2: P plane-synchronous for the images whose hint marks it
    // as the faster walk (coarse pixels), per ray for the others
    int plane_sync = 5;
    // bit 0: time-interpolated plane walks on frame pairs stored side by
    // side; bit 1: Thomson B in one walk on (m' x, m x) pairs
    int channels = 3;
    tomo::Tiling tiling = { 32, 8, 8 };
    // walk rules of size buckets without their own
    tomo_plane_rules rules = tomo::default_plane_rules();
    // geometry cache
    bool key_valid = false;
    uint64_t key = 0;       // geometry of the cached ray records
    uint64_t hint_key = 0;  // geometry and walk rules of the cached hints
    int32_t cached_n_img = 0;  // images of the cached geometry
    tomo_cube_geom cached_cube = {};  // cube of the cached geometry
    cudaEvent_t setup_done = nullptr;
    // per-geometry buffers
    tomo::host::DevBuf ptg, frames, tan_u, tan_v, params, rays;
    // bit L set: some image of the cached geometry walks in layout L
    tomo::host::DevBuf layout_used;
    // { count, image indices }: the images of the cached geometry whose hint
    // leaves them to the per-ray forward
    tomo::host::DevBuf per_ray_fwd;
    // some image of the cached geometry may select the plane forward (a
    // host-side upper bound of the device's per-image pixel-pitch test)
    bool fwd_plane_possible = true;
    // every image of the cached geometry may select the plane forward (the
    // same estimate): the per-ray forward then runs in its listed form
    bool fwd_plane_all = false;
    // some image of the cached geometry may have a valid plane hint (the
    // same kind of estimate; when false the per-ray transpose runs)
    bool plane_possible = true;
    // cube copies (forward) / accumulators (transpose) in layouts 1 and 2
    tomo::host::DevBuf lay1, lay2;
    // two-value buffers (8 bytes per voxel) in layouts 0, 1, 2: frame pairs
    // of the time-interpolated plane walks, (m' x, m x) pairs of the
    // single-walk Thomson B operator
    tomo::host::DevBuf pr[3];
    // solver workspace
    tomo::host::DevBuf b, r, p, q, t, p16, S, partials, counter, count64;
    // map-masked cube copy (forward) / transpose scratch (accumulate)
    tomo::host::DevBuf mcube;
    // Thomson operators: rho^2 per pixel (computed with the ray records),
    // (m, m') per voxel (keyed by cube geometry and u), two cube and one
    // image scratch buffers
    tomo::host::DevBuf rho2, thf, th1, th2, thimg;
    uint64_t thf_key = 0;
    bool thf_valid = false;
    // tuned tile shapes per problem size, and the cached batch plan
    std::vector<tomo::host::Tuned> tuned;
    tomo::host::BatchPlan *plan = nullptr;
    cudaStream_t capture_stream = nullptr;
    // launch counts and optional per-launch event timing
    bool profile = false;
    int64_t launches[TOMO_K_COUNT] = { 0 };
    double ms[TOMO_K_COUNT] = { 0 };
    std::vector<cudaEvent_t> ev_start, ev_stop;  // event pool (pairs)
    std::vector<int> ev_free;                    // free pair slots
    std::vector<int> ev_pending_slot, ev_pending_kind;
};

namespace tomo {
namespace host {

tomo_status fail(tomo_ctx *ctx, tomo_status st, const char *fmt, ...);
tomo_status ensure(tomo_ctx *ctx, DevBuf &b, size_t bytes);
tomo_status check_cube(tomo_ctx *ctx, const tomo_cube_geom *c, int32_t n_frames);
tomo_status check_img(tomo_ctx *ctx, const tomo_image_geom *g);
tomo_status check_pointing(tomo_ctx *ctx, const tomo_pointing *p,
                           const tomo_image_geom *g, int32_t n_frames);
tomo_status check_tiling(tomo_ctx *ctx, Tiling t);
bool aligned(const void *p, size_t a);
uint64_t fnv1a(uint64_t h, const void *data, size_t n);
CubeDev cube_dev(const tomo_cube_geom *c);
int reduce_grid(const tomo_ctx *ctx, int64_t n);
// Tile shape for a problem: the tuned one for its size if any, else the
// context's option.
Tiling tiling_for(const tomo_ctx *ctx, const tomo_cube_geom *c,
                  const tomo_image_geom *g);
// Walk rules for a problem: its size bucket's, else the context's.
tomo_plane_rules rules_for(const tomo_ctx *ctx, const tomo_cube_geom *c,
                           const tomo_image_geom *g);
void free_plan(tomo_ctx *ctx);
// Single-problem P and P^T with the context's walk: plane-synchronous
// (layout copies + plane kernels) when enabled and supported, else the
// per-ray kernels.  ensure_plane must have succeeded for the problem first.
bool use_plane(const tomo_ctx *ctx, const tomo_cube_geom *c, Tiling t,
               bool forward);
tomo_status ensure_plane(tomo_ctx *ctx, const tomo_cube_geom *c,
                         int32_t n_frames, Tiling t);
tomo_status forward_one(tomo_ctx *ctx, const void *cube_dev, tomo_dtype dtype,
                        int32_t n_frames, const uint8_t *mask, float *out,
                        const tomo_cube_geom *c, const tomo_image_geom *g,
                        Tiling t, const double *done, cudaStream_t s);
tomo_status ensure_thomson(tomo_ctx *ctx, const tomo_cube_geom *c, double u,
                           cudaStream_t s);
tomo_status op_forward(tomo_ctx *ctx, const void *src, tomo_dtype dtype,
                       int32_t n_frames, const uint8_t *mask,
                       const uint8_t *mm, float *out, const tomo_cube_geom *c,
                       const tomo_image_geom *g, Tiling t, const double *done,
                       cudaStream_t s);
tomo_status op_adjoint(tomo_ctx *ctx, const float *images, const uint8_t *mask,
                       const uint8_t *mm, float *dst, const tomo_cube_geom *c,
                       int32_t n_frames, const tomo_image_geom *g, Tiling t,
                       const double *done, cudaStream_t s);
tomo_status adjoint_one(tomo_ctx *ctx, const float *images,
                        const uint8_t *mask, float *cube,
                        const tomo_cube_geom *c, int32_t n_frames,
                        const tomo_image_geom *g, Tiling t,
                        const double *done, cudaStream_t s);
// Builds (or reuses) the context's ray records for one geometry on `s`.
// Host estimates of the device's per-image plane-walk rules (setup.cu) from
// the boresight: whether an image may get a valid hint, and whether it may
// select the plane forward.  Only speed depends on them: the kernel that
// runs when an estimate says no walks every ray per ray.
bool plane_estimate(const tomo_pointing &p, const tomo_cube_geom *c,
                    const tomo_plane_rules &r);
bool plane_forward_estimate(const tomo_pointing &p, const tomo_cube_geom *c,
                            const tomo_plane_rules &r);
tomo_status prepare_rays(tomo_ctx *ctx, const tomo_cube_geom *c,
                         int32_t n_frames, const tomo_image_geom *g,
                         const tomo_pointing *ptg, cudaStream_t s);

#define CUDA_TRY(ctx, call)                                                  \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess)                                               \
            return fail((ctx), e_ == cudaErrorMemoryAllocation               \
                                   ? TOMO_ERR_OOM : TOMO_ERR_CUDA,           \
                        "%s: %s", #call, cudaGetErrorString(e_));            \
    } while (0)

// Launch a kernel through its host launcher `call`, counted and (optionally)
// timed as class `kind` on stream `s`.
#define LAUNCH(ctx, kind, s, call)                                           \
    do {                                                                     \
        Launch L_((ctx), (kind), (s));                                       \
        CUDA_TRY((ctx), (call));                                             \
    } while (0)

// Makes the context's device current for the call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Counts one kernel launch of class `kind`; with profiling on, brackets it
// with a pair of CUDA events on the launching stream.
struct Launch {
    tomo_ctx *ctx;
    int kind;
    cudaStream_t s;
    int slot = -1;
    Launch(tomo_ctx *c, int k, cudaStream_t st) : ctx(c), kind(k), s(st)
    {
        ctx->launches[kind] += 1;
        if (!ctx->profile) return;
        if (ctx->ev_free.empty()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess) return;
            if (cudaEventCreate(&b) != cudaSuccess) {
                cudaEventDestroy(a);
                return;
            }
            ctx->ev_start.push_back(a);
            ctx->ev_stop.push_back(b);
            ctx->ev_free.push_back((int)ctx->ev_start.size() - 1);
        }
        slot = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        cudaEventRecord(ctx->ev_start[slot], s);
    }
    ~Launch()
    {
        if (slot < 0) return;
        cudaEventRecord(ctx->ev_stop[slot], s);
        ctx->ev_pending_slot.push_back(slot);
        ctx->ev_pending_kind.push_back(kind);
    }
};

}  // namespace host
}  // namespace tomo
