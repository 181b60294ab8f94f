// C ABI of the batched projector, transpose and solver, and of the tile-shape
// autotuner (kernels in batch.cu and siddon.cu).
//
// A batch plan holds, for one set of problem geometries, the ray records of
// every problem back to back, the descriptors of the persistent kernels and,
// for the solver, one CUDA graph with the whole CG run (initialisation and
// every iteration).  Replaying the plan for the same geometries and buffers
// costs one graph launch.
#include <math.h>
#include <string.h>

#include <vector>

#include "batch.cuh"
#include "host.h"

using namespace tomo;
using namespace tomo::host;

namespace tomo {
namespace host {

struct BatchPlan {
    uint64_t geom_key = 0;
    uint64_t graph_key = 0;
    int32_t n = 0;
    // geometry of every problem, back to back
    DevBuf ptg, frames, tan_u, tan_v, params, rays;
    std::vector<int64_t> ray_off, img_off, tu_off, tv_off;
    std::vector<Tiling> tl;
    std::vector<int64_t> tile_prefix;  // n + 1
    DevBuf tpre_dev, sched_dev;        // tile prefix, walk schedule
    int64_t n_chunks = 0;
    // plane-synchronous transpose: plane-tile prefix and schedule, voxel
    // offsets, per-problem layout masks, accumulators of layouts 1 and 2
    // (2 x voxels per problem, zero between transposes), combine-job tile
    // prefix (jobs: problem i, layout 1 / 2 at 2 i, 2 i + 1)
    std::vector<int64_t> ptile_prefix, vox_off, job_prefix;
    DevBuf ptpre_dev, psched_dev, lay, lay_used, jpre_dev;
    // with the plane walks on, problems whose pixels are too dense for them
    // (host estimate) walk per ray with their own tile shapes: tile prefix
    // and schedule of those problems only (the plane prefix holds the rest)
    std::vector<int64_t> rtile_prefix;
    DevBuf rtpre_dev, rsched_dev;
    int64_t rn_chunks = 0;
    DevBuf flay;  // layout copies of the forward's source cubes (2 x voxels)
    DevBuf mcube;  // map-masked cubes / transpose scratch (1 x voxels)
    int64_t pn_chunks = 0;
    bool lay_dirty = false;
    cudaEvent_t ready = nullptr;
    // per-call descriptors of the projector / transpose entry points
    DevBuf call_desc, call_counter, call_jobs, call_fjobs;
    // solver workspace and graph
    DevBuf vec, timg, S, partials, counters, walk_desc, vec_desc, prefixes,
        solve_jobs, solve_fjobs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_launches[TOMO_K_COUNT] = { 0 };
    int32_t n_iter = 0;
    size_t report_stride = 0;
};

void free_plan(tomo_ctx *ctx)
{
    BatchPlan *p = ctx->plan;
    if (!p) return;
    DevBuf *bufs[] = { &p->ptg, &p->frames, &p->tan_u, &p->tan_v, &p->params,
                       &p->rays, &p->tpre_dev, &p->sched_dev,
                       &p->ptpre_dev, &p->psched_dev, &p->rtpre_dev,
                       &p->rsched_dev, &p->lay, &p->lay_used,
                       &p->jpre_dev, &p->flay, &p->call_desc,
                       &p->call_counter, &p->call_jobs, &p->call_fjobs,
                       &p->vec, &p->timg, &p->S, &p->partials, &p->counters,
                       &p->walk_desc, &p->vec_desc, &p->prefixes,
                       &p->solve_jobs, &p->solve_fjobs, &p->mcube };
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->ready) cudaEventDestroy(p->ready);
    delete p;
    ctx->plan = nullptr;
}

}  // namespace host
}  // namespace tomo

namespace {

constexpr int kBatchThreads = 256;

const Tiling kDefaultTiling = { 32, 8, 8 };

// Tile shapes the autotuner tries: all 256 threads, so the batched
// persistent kernel can mix them.
const Tiling kCandidates[] = {
    { 32, 8, 8 }, { 16, 16, 8 }, { 16, 16, 4 }, { 64, 4, 16 },
    { 32, 8, 32 }, { 128, 2, 32 }, { 16, 16, 16 }, { 8, 32, 4 },
    { 32, 8, 16 }, { 64, 4, 32 } };

bool is_batch_tiling(Tiling t)
{
    return t.tile_u * t.tile_v == kBatchThreads;
}

tomo_status check_problem(tomo_ctx *ctx, const tomo_problem *p, int32_t i,
                          bool need_cube, bool need_images)
{
    tomo_status st;
    if ((st = check_cube(ctx, &p->cube, 1)) || (st = check_img(ctx, &p->img)) ||
        (st = check_pointing(ctx, p->pointing_host, &p->img, 1)))
        return fail(ctx, st, "problem %d: %s", i, ctx->err);
    if (p->reserved != 0)
        return fail(ctx, TOMO_ERR_ARG, "problem %d: reserved must be 0", i);
    if (p->img.kind != TOMO_KIND_EMISSION)
        return fail(ctx, TOMO_ERR_UNSUPPORTED,
                    "problem %d: the batched entry points take emission "
                    "images only", i);
    if (need_cube && (!p->cube_dev || !aligned(p->cube_dev, 4)))
        return fail(ctx, TOMO_ERR_ARG, "problem %d: cube_dev NULL or misaligned", i);
    if (need_images && p->img.n_img > 0 &&
        (!p->images_dev || !aligned(p->images_dev, 4)))
        return fail(ctx, TOMO_ERR_ARG,
                    "problem %d: images_dev NULL or misaligned", i);
    if (!isfinite(p->lambda) || p->lambda < 0)
        return fail(ctx, TOMO_ERR_ARG, "problem %d: lambda must be >= 0", i);
    if (!aligned(p->prior_weight_dev, 4))
        return fail(ctx, TOMO_ERR_ARG, "problem %d: misaligned prior_weight_dev", i);
    return TOMO_OK;
}

Tiling batch_tiling(const tomo_ctx *ctx, const tomo_problem *p)
{
    const Tiling t = tiling_for(ctx, &p->cube, &p->img);
    return is_batch_tiling(t) ? t : kDefaultTiling;
}

tomo_status upload(tomo_ctx *ctx, DevBuf &b, const void *src, size_t bytes,
                   cudaStream_t s)
{
    tomo_status st = ensure(ctx, b, bytes);
    if (st) return st;
    CUDA_TRY(ctx, cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s));
    return TOMO_OK;
}

// Ray records of every problem (FP64 setup kernels, one pair per problem),
// kept while the geometries do not change.
tomo_status prepare_batch(tomo_ctx *ctx, int32_t n, const tomo_problem *probs,
                          cudaStream_t s)
{
    uint64_t h = 1469598103934665603ull;
    h = fnv1a(h, &n, sizeof(n));
    for (int32_t i = 0; i < n; ++i) {
        const tomo_problem &p = probs[i];
        h = fnv1a(h, &p.cube, sizeof(p.cube));
        h = fnv1a(h, &p.img, sizeof(p.img));
        h = fnv1a(h, p.pointing_host, sizeof(tomo_pointing) * (size_t)p.img.n_img);
        const Tiling t = batch_tiling(ctx, &p);
        h = fnv1a(h, &t, sizeof(t));
        const tomo_plane_rules r = rules_for(ctx, &p.cube, &p.img);
        h = fnv1a(h, &r, sizeof(r));
    }
    if (!ctx->plan) {
        ctx->plan = new BatchPlan();
        CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->plan->ready,
                                               cudaEventDisableTiming));
    }
    BatchPlan *P = ctx->plan;
    if (P->geom_key == h && P->n == n) {
        CUDA_TRY(ctx, cudaStreamWaitEvent(s, P->ready, 0));
        return TOMO_OK;
    }
    P->geom_key = 0;
    P->graph_key = 0;
    P->n = n;
    P->ray_off.assign(n + 1, 0);
    P->img_off.assign(n + 1, 0);
    P->tu_off.assign(n + 1, 0);
    P->tv_off.assign(n + 1, 0);
    P->tile_prefix.assign(n + 1, 0);
    P->ptile_prefix.assign(n + 1, 0);
    P->rtile_prefix.assign(n + 1, 0);
    P->vox_off.assign(n + 1, 0);
    P->job_prefix.assign(2 * (size_t)n + 1, 0);
    P->tl.assign(n, kDefaultTiling);
    for (int32_t i = 0; i < n; ++i) {
        const tomo_image_geom &g = probs[i].img;
        P->tl[i] = batch_tiling(ctx, &probs[i]);
        P->ray_off[i + 1] = P->ray_off[i] + (int64_t)g.n_img * g.nu * g.nv;
        P->img_off[i + 1] = P->img_off[i] + g.n_img;
        P->tu_off[i + 1] = P->tu_off[i] + (int64_t)g.n_img * g.nu;
        P->tv_off[i + 1] = P->tv_off[i] + (int64_t)g.n_img * g.nv;
        const int64_t tiles = (int64_t)g.n_img *
                              ((g.nu + P->tl[i].tile_u - 1) / P->tl[i].tile_u) *
                              ((g.nv + P->tl[i].tile_v - 1) / P->tl[i].tile_v);
        P->tile_prefix[i + 1] = P->tile_prefix[i] + tiles;
        bool plane_ok = false;
        const tomo_plane_rules rules = rules_for(ctx, &probs[i].cube, &g);
        for (int32_t k = 0; k < g.n_img; ++k)
            plane_ok |= plane_estimate(probs[i].pointing_host[k],
                                       &probs[i].cube, rules);
        P->ptile_prefix[i + 1] =
            P->ptile_prefix[i] + (plane_ok ? (int64_t)g.n_img *
                                     ((g.nu + kPlaneTileU - 1) / kPlaneTileU) *
                                     ((g.nv + kPlaneTileV - 1) / kPlaneTileV) : 0);
        P->rtile_prefix[i + 1] = P->rtile_prefix[i] + (plane_ok ? 0 : tiles);
        const tomo_cube_geom &c = probs[i].cube;
        P->vox_off[i + 1] = P->vox_off[i] + (int64_t)c.nx * c.ny * c.nz;
        for (int L = 1; L <= 2; ++L) {
            const int64_t nb = L == 1 ? c.ny : c.nz, nc = L == 1 ? c.nz : c.ny;
            const size_t j = 2 * (size_t)i + (L - 1);
            P->job_prefix[j + 1] = P->job_prefix[j] + ((c.nx + 31) / 32) *
                                                          ((nb + 31) / 32) * nc;
        }
    }
    const int64_t n_img = P->img_off[n];
    tomo_status st;
    if ((st = ensure(ctx, P->ptg, sizeof(tomo_pointing) * n_img)) ||
        (st = ensure(ctx, P->frames, sizeof(Frame) * n_img)) ||
        (st = ensure(ctx, P->params, sizeof(ImgParam) * n_img)) ||
        (st = ensure(ctx, P->tan_u, sizeof(double) * P->tu_off[n])) ||
        (st = ensure(ctx, P->tan_v, sizeof(double) * P->tv_off[n])) ||
        (st = ensure(ctx, P->rays, sizeof(RayRec) * P->ray_off[n])) ||
        (st = ensure(ctx, P->lay, sizeof(float) * 2 * (P->vox_off[n] > 0 ? P->vox_off[n] : 1))) ||
        (st = ensure(ctx, P->flay, sizeof(float) * 2 * (P->vox_off[n] > 0 ? P->vox_off[n] : 1))) ||
        (st = ensure(ctx, P->lay_used, sizeof(unsigned) * n)))
        return st;
    CUDA_TRY(ctx, cudaMemsetAsync(P->lay.p, 0, sizeof(float) * 2 * P->vox_off[n], s));
    CUDA_TRY(ctx, cudaMemsetAsync(P->lay_used.p, 0, sizeof(unsigned) * n, s));
    P->lay_dirty = false;
    std::vector<tomo_pointing> all((size_t)n_img);
    for (int32_t i = 0; i < n; ++i)
        if (probs[i].img.n_img > 0)
            memcpy(&all[P->img_off[i]], probs[i].pointing_host,
                   sizeof(tomo_pointing) * probs[i].img.n_img);
    if (n_img > 0)
        CUDA_TRY(ctx, cudaMemcpyAsync(P->ptg.p, all.data(),
                                      sizeof(tomo_pointing) * n_img,
                                      cudaMemcpyHostToDevice, s));
    for (int32_t i = 0; i < n; ++i) {
        const tomo_problem &p = probs[i];
        if (p.img.n_img == 0) continue;
        Frame *fr = (Frame *)P->frames.p + P->img_off[i];
        ImgParam *pr = (ImgParam *)P->params.p + P->img_off[i];
        double *tu = (double *)P->tan_u.p + P->tu_off[i];
        double *tv = (double *)P->tan_v.p + P->tv_off[i];
        LAUNCH(ctx, TOMO_K_SETUP, s,
               launch_frames((const tomo_pointing *)P->ptg.p + P->img_off[i],
                             p.img.n_img, p.img.nu, p.img.nv, 1, fr, tu, tv, pr,
                             make_double3(p.cube.dx, p.cube.dy, p.cube.dz),
                             (unsigned *)P->lay_used.p + i, nullptr,
                             rules_for(ctx, &p.cube, &p.img), s));
        LAUNCH(ctx, TOMO_K_SETUP, s,
               launch_ray_setup(fr, tu, tv, cube_dev(&p.cube), p.img.n_img,
                                p.img.nu, p.img.nv,
                                (RayRec *)P->rays.p + P->ray_off[i], s));
    }
    // walk schedules: groups of kSchedGroup tiles of one problem, dealt
    // round-robin over the problems (all problems per ray; the plane-walk
    // problems in plane tiles; the others per ray)
    auto deal = [n](const std::vector<int64_t> &pre) {
        std::vector<int2> out;
        std::vector<int64_t> next(n, 0);
        for (bool any = true; any;) {
            any = false;
            for (int32_t i = 0; i < n; ++i) {
                if (next[i] < pre[i + 1] - pre[i]) {
                    out.push_back(make_int2(i, (int)next[i]));
                    next[i] += kSchedGroup;
                    any = true;
                }
            }
        }
        return out;
    };
    std::vector<int2> sched = deal(P->tile_prefix);
    std::vector<int2> psched = deal(P->ptile_prefix);
    std::vector<int2> rsched = deal(P->rtile_prefix);
    P->n_chunks = (int64_t)sched.size();
    P->pn_chunks = (int64_t)psched.size();
    P->rn_chunks = (int64_t)rsched.size();
    // an empty schedule still gets a (never read) element to upload
    for (std::vector<int2> *v : { &sched, &psched, &rsched })
        if (v->empty()) v->push_back(make_int2(0, 0));
    if ((st = upload(ctx, P->tpre_dev, P->tile_prefix.data(),
                     sizeof(int64_t) * (n + 1), s)) ||
        (st = upload(ctx, P->sched_dev, sched.data(),
                     sizeof(int2) * sched.size(), s)) ||
        (st = upload(ctx, P->ptpre_dev, P->ptile_prefix.data(),
                     sizeof(int64_t) * (n + 1), s)) ||
        (st = upload(ctx, P->psched_dev, psched.data(),
                     sizeof(int2) * psched.size(), s)) ||
        (st = upload(ctx, P->rtpre_dev, P->rtile_prefix.data(),
                     sizeof(int64_t) * (n + 1), s)) ||
        (st = upload(ctx, P->rsched_dev, rsched.data(),
                     sizeof(int2) * rsched.size(), s)) ||
        (st = upload(ctx, P->jpre_dev, P->job_prefix.data(),
                     sizeof(int64_t) * P->job_prefix.size(), s)))
        return st;
    CUDA_TRY(ctx, cudaEventRecord(P->ready, s));
    P->geom_key = h;
    return TOMO_OK;
}

// forward: the layout buffers are the forward's copies (flay), else the
// transpose's accumulators (lay)
WalkDesc walk_desc(const BatchPlan *P, const tomo_problem &p, int32_t i,
                   const float *src, float *dst, const double *done,
                   bool forward)
{
    WalkDesc d;
    d.rays = (const RayRec *)P->rays.p + P->ray_off[i];
    d.prm = (const ImgParam *)P->params.p + P->img_off[i];
    d.mask = p.mask_dev;
    d.src = src;
    d.dst = dst;
    d.done = done;
    d.nu = p.img.nu;
    d.nv = p.img.nv;
    d.nx = p.cube.nx;
    d.nxny = p.cube.nx * p.cube.ny;
    d.tl = P->tl[i];
    d.tiles_u = (p.img.nu + d.tl.tile_u - 1) / d.tl.tile_u;
    d.tiles_v = (p.img.nv + d.tl.tile_v - 1) / d.tl.tile_v;
    d.ny = p.cube.ny;
    d.nz = p.cube.nz;
    d.lay1 = (float *)(forward ? P->flay.p : P->lay.p) + 2 * P->vox_off[i];
    d.lay2 = d.lay1 + (P->vox_off[i + 1] - P->vox_off[i]);
    return d;
}

// Combine jobs of every problem (layouts 1 and 2) into the cubes cube[i].
// forward: copy jobs into the forward's layout copies (run when some image
// of the problem takes the plane forward in layout L), else combine jobs of
// the transpose's accumulators (run when some image walks in layout L)
std::vector<LayoutJob> layout_jobs(const BatchPlan *P, int32_t n,
                                   const tomo_problem *probs,
                                   float *const *cubes, const double *const *done,
                                   bool forward = false)
{
    std::vector<LayoutJob> jobs(2 * (size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        const tomo_cube_geom &c = probs[i].cube;
        float *lay1 = (float *)(forward ? P->flay.p : P->lay.p) + 2 * P->vox_off[i];
        for (int L = 1; L <= 2; ++L) {
            LayoutJob &J = jobs[2 * (size_t)i + (L - 1)];
            J.acc = L == 1 ? lay1 : lay1 + (P->vox_off[i + 1] - P->vox_off[i]);
            J.cube = cubes[i];
            J.used = (const unsigned *)P->lay_used.p + i;
            J.done = done ? done[i] : nullptr;
            J.L = L;
            J.nx = c.nx;
            J.nb = L == 1 ? c.ny : c.nz;
            J.nc = L == 1 ? c.nz : c.ny;
            J.sb = L == 1 ? (int64_t)c.nx : (int64_t)c.nx * c.ny;
            J.sc = L == 1 ? (int64_t)c.nx * c.ny : (int64_t)c.nx;
            J.tiles_x = (c.nx + 31) / 32;
            J.tiles_b = (J.nb + 31) / 32;
            J.bit = forward ? 1u << (8 + L) : 1u << L;
            J.pad = 0;
        }
    }
    return jobs;
}

// Plane-synchronous transposes for this batch: enabled for P^T
// atomics mode, and every cube within the plane walk's limits.
bool batch_plane(const tomo_ctx *ctx, int32_t n, const tomo_problem *probs)
{
    if (!(ctx->plane_sync & 1)) return false;
    for (int32_t i = 0; i < n; ++i)
        if (!plane_supported(&probs[i].cube, 4)) return false;
    return true;
}

// Batched forward over plane tiles, each image taking the walk its hint
// selects (TOMO_OPT_PLANE_SYNC bit 1 or 2; the batched path follows the
// per-image choice in both cases).
bool batch_plane_forward(const tomo_ctx *ctx, int32_t n, const tomo_problem *probs)
{
    if (!(ctx->plane_sync & (2 | 4))) return false;
    for (int32_t i = 0; i < n; ++i)
        if (!plane_supported(&probs[i].cube, 4)) return false;
    return true;
}

int plane_walk_grid(const tomo_ctx *ctx)
{
    return (ctx->num_sms > 0 ? ctx->num_sms : 152) *
           plane_batched_blocks_per_sm();
}

int combine_grid(const tomo_ctx *ctx)
{
    return 8 * (ctx->num_sms > 0 ? ctx->num_sms : 152);
}

int walk_grid(const tomo_ctx *ctx)
{
    return (ctx->num_sms > 0 ? ctx->num_sms : 152) * walk_batched_blocks_per_sm();
}

// The walks of one batched projection or transpose; cubes[i] is the cube
// that problem i's walk reads (forward) or accumulates into (transpose).
tomo_status batched_walk_core(tomo_ctx *ctx, int32_t n,
                              const tomo_problem *probs, bool adjoint,
                              float *const *cubes, cudaStream_t s)
{
    tomo_status st;
    BatchPlan *P = ctx->plan;
    std::vector<WalkDesc> d(n);
    for (int32_t i = 0; i < n; ++i)
        d[i] = adjoint ? walk_desc(P, probs[i], i, probs[i].images_dev,
                                   cubes[i], nullptr, false)
                       : walk_desc(P, probs[i], i, cubes[i],
                                   probs[i].images_dev, nullptr, true);
    // two queue counters: the plane-tile walk and the per-ray walk of the
    // problems too dense for it
    if ((st = upload(ctx, P->call_desc, d.data(), sizeof(WalkDesc) * n, s)) ||
        (st = ensure(ctx, P->call_counter, 2 * sizeof(unsigned long long))))
        return st;
    CUDA_TRY(ctx, cudaMemsetAsync(P->call_counter.p, 0,
                                  2 * sizeof(unsigned long long), s));
    unsigned long long *ctr2 = (unsigned long long *)P->call_counter.p;
    if (adjoint && batch_plane(ctx, n, probs)) {
        if (P->lay_dirty)
            CUDA_TRY(ctx, cudaMemsetAsync(P->lay.p, 0,
                                          sizeof(float) * 2 * P->vox_off[n], s));
        const std::vector<LayoutJob> jobs = layout_jobs(P, n, probs, cubes, nullptr);
        if ((st = upload(ctx, P->call_jobs, jobs.data(), sizeof(LayoutJob) * jobs.size(), s)))
            return st;
        P->lay_dirty = true;
        if (P->pn_chunks > 0)
            LAUNCH(ctx, TOMO_K_ADJOINT, s,
                   launch_adjoint_plane_batched((const WalkDesc *)P->call_desc.p,
                                                (const int64_t *)P->ptpre_dev.p,
                                                (const int2 *)P->psched_dev.p,
                                                P->pn_chunks, ctr2,
                                                plane_walk_grid(ctx), s));
        if (P->rn_chunks > 0)
            LAUNCH(ctx, TOMO_K_ADJOINT, s,
                   launch_walk_batched(true, (const WalkDesc *)P->call_desc.p,
                                       (const int64_t *)P->rtpre_dev.p,
                                       (const int2 *)P->rsched_dev.p,
                                       P->rn_chunks, ctr2 + 1, walk_grid(ctx), s));
        LAUNCH(ctx, TOMO_K_LAYOUT, s,
               launch_add_from_layout_batched((const LayoutJob *)P->call_jobs.p,
                                              (const int64_t *)P->jpre_dev.p,
                                              2 * n, combine_grid(ctx), s));
        P->lay_dirty = false;
        return TOMO_OK;
    }
    if (!adjoint && batch_plane_forward(ctx, n, probs)) {
        const std::vector<LayoutJob> jobs =
            layout_jobs(P, n, probs, cubes, nullptr, true);
        if ((st = upload(ctx, P->call_fjobs, jobs.data(), sizeof(LayoutJob) * jobs.size(), s)))
            return st;
        LAUNCH(ctx, TOMO_K_LAYOUT, s,
               launch_to_layout_batched((const LayoutJob *)P->call_fjobs.p,
                                        (const int64_t *)P->jpre_dev.p, 2 * n,
                                        combine_grid(ctx), s));
        if (P->pn_chunks > 0)
            LAUNCH(ctx, TOMO_K_FORWARD, s,
                   launch_forward_plane_batched((const WalkDesc *)P->call_desc.p,
                                                (const int64_t *)P->ptpre_dev.p,
                                                n, P->ptile_prefix[n], s));
        if (P->rn_chunks > 0)
            LAUNCH(ctx, TOMO_K_FORWARD, s,
                   launch_walk_batched(false, (const WalkDesc *)P->call_desc.p,
                                       (const int64_t *)P->rtpre_dev.p,
                                       (const int2 *)P->rsched_dev.p,
                                       P->rn_chunks, ctr2 + 1, walk_grid(ctx), s));
        return TOMO_OK;
    }
    LAUNCH(ctx, adjoint ? TOMO_K_ADJOINT : TOMO_K_FORWARD, s,
           launch_walk_batched(adjoint, (const WalkDesc *)P->call_desc.p,
                               (const int64_t *)P->tpre_dev.p,
                               (const int2 *)P->sched_dev.p, P->n_chunks,
                               (unsigned long long *)P->call_counter.p,
                               walk_grid(ctx), s));
    return TOMO_OK;
}

// Map masks (tomo_problem.map_mask_dev): the forward walks a copy of K x
// (scratch), the transpose is followed by x = K x, or with ACCUMULATE runs
// into zeroed scratch whose kept voxels are then added.
tomo_status batched_walk(tomo_ctx *ctx, int32_t n, const tomo_problem *probs,
                         bool adjoint, uint32_t flags, cudaStream_t s)
{
    tomo_status st;
    for (int32_t i = 0; i < n; ++i)
        if ((st = check_problem(ctx, &probs[i], i, true, true))) return st;
    if ((st = prepare_batch(ctx, n, probs, s))) return st;
    BatchPlan *P = ctx->plan;
    const bool accumulate = (flags & TOMO_ACCUMULATE) != 0;
    bool scratch = false;
    for (int32_t i = 0; i < n; ++i)
        scratch |= probs[i].map_mask_dev != nullptr && (!adjoint || accumulate);
    if (scratch &&
        (st = ensure(ctx, P->mcube, sizeof(float) * (P->vox_off[n] > 0 ? P->vox_off[n] : 1))))
        return st;
    std::vector<float *> cubes(n);
    for (int32_t i = 0; i < n; ++i) {
        const int64_t nvox = P->vox_off[i + 1] - P->vox_off[i];
        const uint8_t *mm = probs[i].map_mask_dev;
        float *tmp = (float *)P->mcube.p + P->vox_off[i];
        cubes[i] = probs[i].cube_dev;
        if (!adjoint && mm) {
            LAUNCH(ctx, TOMO_K_VECTOR, s,
                   launch_map_keep_copy(probs[i].cube_dev, tmp, false, mm,
                                        nvox, 1, s));
            cubes[i] = tmp;
        } else if (adjoint && mm && accumulate) {
            CUDA_TRY(ctx, cudaMemsetAsync(tmp, 0, sizeof(float) * nvox, s));
            cubes[i] = tmp;
        } else if (adjoint && !accumulate) {
            CUDA_TRY(ctx, cudaMemsetAsync(cubes[i], 0, sizeof(float) * nvox, s));
        }
    }
    if (P->tile_prefix[n] == 0) return TOMO_OK;
    if ((st = batched_walk_core(ctx, n, probs, adjoint, cubes.data(), s)))
        return st;
    if (adjoint)
        for (int32_t i = 0; i < n; ++i) {
            const uint8_t *mm = probs[i].map_mask_dev;
            if (!mm) continue;
            const int64_t nvox = P->vox_off[i + 1] - P->vox_off[i];
            if (accumulate)
                LAUNCH(ctx, TOMO_K_VECTOR, s,
                       launch_map_keep_add(probs[i].cube_dev, cubes[i], mm,
                                           nvox, 1, s));
            else
                LAUNCH(ctx, TOMO_K_VECTOR, s,
                       launch_map_zero(probs[i].cube_dev, mm, nvox, 1, s));
        }
    return TOMO_OK;
}

// Times the forward and transpose of one problem under tile shape t.
tomo_status time_tiling(tomo_ctx *ctx, const tomo_problem *p, Tiling t,
                        float *images_tmp, float *cube_tmp, cudaStream_t s,
                        float *fwd_ms, float *adj_ms)
{
    cudaEvent_t e[3];
    for (int k = 0; k < 3; ++k)
        CUDA_TRY(ctx, cudaEventCreate(&e[k]));
    const int64_t nvox = (int64_t)p->cube.nx * p->cube.ny * p->cube.nz;
    float best_f = INFINITY, best_a = INFINITY;
    tomo_status st = TOMO_OK;
    for (int rep = 0; rep < 3 && st == TOMO_OK; ++rep) {
        cudaError_t err = cudaEventRecord(e[0], s);
        if (err == cudaSuccess)
            err = launch_forward((const RayRec *)ctx->rays.p,
                                 (const ImgParam *)ctx->params.p, p->cube_dev,
                                 TOMO_F32, nvox, false, p->mask_dev,
                                 images_tmp, p->img.n_img, p->img.nu,
                                 p->img.nv, p->cube.nx,
                                 p->cube.nx * p->cube.ny, t, nullptr, s);
        if (err == cudaSuccess) err = cudaEventRecord(e[1], s);
        if (err == cudaSuccess) {
            // the transpose the single-problem calls would run (the plane
            // walk ignores t, the per-ray walk uses it)
            st = adjoint_one(ctx, p->images_dev, p->mask_dev, cube_tmp, &p->cube,
                             1, &p->img, t, nullptr, s);
            if (st) break;
        }
        if (err == cudaSuccess) err = cudaEventRecord(e[2], s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e[2]);
        float f = 0, a = 0;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&f, e[0], e[1]);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&a, e[1], e[2]);
        if (err != cudaSuccess) {
            st = fail(ctx, TOMO_ERR_CUDA, "autotune: %s", cudaGetErrorString(err));
            break;
        }
        if (rep > 0) {  // the first repetition warms caches
            best_f = f < best_f ? f : best_f;
            best_a = a < best_a ? a : best_a;
        }
    }
    for (int k = 0; k < 3; ++k) cudaEventDestroy(e[k]);
    *fwd_ms = best_f;
    *adj_ms = best_a;
    return st;
}

// Times P and P^T of one problem as the single-problem calls run them
// (walks chosen per image by the bucket's current rules, layout copies and
// combines included); best of the last two of three repetitions.
tomo_status time_schedule(tomo_ctx *ctx, const tomo_problem *p, Tiling t,
                          float *images_tmp, float *cube_tmp, cudaStream_t s,
                          float *fwd_ms, float *adj_ms)
{
    tomo_status st;
    if ((st = prepare_rays(ctx, &p->cube, 1, &p->img, p->pointing_host, s)))
        return st;
    cudaEvent_t e[3];
    for (int k = 0; k < 3; ++k)
        CUDA_TRY(ctx, cudaEventCreate(&e[k]));
    float best_f = INFINITY, best_a = INFINITY;
    for (int rep = 0; rep < 3 && st == TOMO_OK; ++rep) {
        cudaError_t err = cudaEventRecord(e[0], s);
        if (err == cudaSuccess &&
            (st = forward_one(ctx, p->cube_dev, TOMO_F32, 1, p->mask_dev,
                              images_tmp, &p->cube, &p->img, t, nullptr, s)))
            break;
        if (err == cudaSuccess) err = cudaEventRecord(e[1], s);
        if (err == cudaSuccess &&
            (st = adjoint_one(ctx, p->images_dev, p->mask_dev, cube_tmp,
                              &p->cube, 1, &p->img, t, nullptr, s)))
            break;
        if (err == cudaSuccess) err = cudaEventRecord(e[2], s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e[2]);
        float f = 0, a = 0;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&f, e[0], e[1]);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&a, e[1], e[2]);
        if (err != cudaSuccess) {
            st = fail(ctx, TOMO_ERR_CUDA, "autotune: %s", cudaGetErrorString(err));
            break;
        }
        if (rep > 0) {
            best_f = f < best_f ? f : best_f;
            best_a = a < best_a ? a : best_a;
        }
    }
    for (int k = 0; k < 3; ++k) cudaEventDestroy(e[k]);
    *fwd_ms = best_f;
    *adj_ms = best_a;
    return st;
}

Tuned *bucket_of(tomo_ctx *ctx, const tomo_cube_geom *c,
                 const tomo_image_geom *g)
{
    for (Tuned &e : ctx->tuned)
        if (e.nx == c->nx && e.ny == c->ny && e.nz == c->nz && e.nu == g->nu &&
            e.nv == g->nv)
            return &e;
    return nullptr;
}

}  // namespace

extern "C" {

tomo_status tomo_autotune(tomo_ctx *ctx, const tomo_problem *prob,
                          tomo_tiling *best_out, void *stream)
{
    if (!ctx || !prob) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    tomo_status st = check_problem(ctx, prob, 0, true, true);
    if (st) return st;
    if (prob->img.n_img == 0)
        return fail(ctx, TOMO_ERR_ARG, "autotune needs at least one image");
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_plane(ctx, &prob->cube, 1, kDefaultTiling)) ||
        (st = prepare_rays(ctx, &prob->cube, 1, &prob->img,
                           prob->pointing_host, s)))
        return st;
    const int64_t nvox = (int64_t)prob->cube.nx * prob->cube.ny * prob->cube.nz;
    const int64_t npix = (int64_t)prob->img.n_img * prob->img.nu * prob->img.nv;
    if ((st = ensure(ctx, ctx->t, sizeof(float) * npix)) ||
        (st = ensure(ctx, ctx->q, sizeof(float) * nvox)))
        return st;
    Tuned best;
    best.nx = prob->cube.nx;
    best.ny = prob->cube.ny;
    best.nz = prob->cube.nz;
    best.nu = prob->img.nu;
    best.nv = prob->img.nv;
    best.tl = kDefaultTiling;
    best.fwd_ms = best.adj_ms = INFINITY;
    for (const Tiling &t : kCandidates) {
        float f, a;
        if ((st = time_tiling(ctx, prob, t, (float *)ctx->t.p,
                              (float *)ctx->q.p, s, &f, &a)))
            return st;
        if (f + a < best.fwd_ms + best.adj_ms) {
            best.tl = t;
            best.fwd_ms = f;
            best.adj_ms = a;
        }
    }
    best.rules = rules_for(ctx, &prob->cube, &prob->img);
    Tuned *entry = bucket_of(ctx, &prob->cube, &prob->img);
    if (entry)
        *entry = best;
    else {
        ctx->tuned.push_back(best);
        entry = &ctx->tuned.back();
    }

    // Walk rules, one threshold at a time, each candidate timed on P and
    // P^T as the single-problem calls run them (the winner of one search
    // is kept for the next).  A candidate replaces the current rules only
    // when it is more than 1 % faster (timing noise).
    const double never = 1e30;
    float cur_f, cur_a;
    if ((st = time_schedule(ctx, prob, entry->tl, (float *)ctx->t.p,
                            (float *)ctx->q.p, s, &cur_f, &cur_a)))
        return st;
    struct Search {
        int field;          // 0 min_pitch, 1 general_ratio, 2 fwd_max_ratio,
                            // 3 fwd_min_pitch, 4 fwd_group, 5 adj_group
        bool forward_only;  // compare P alone (else P + P^T)
        double cand[5];
        int n;
    };
    // group candidates: automatic, image after image, 8 and 32 images, one
    // group of every image
    const double all = 65535.0;
    const Search searches[] = {
        { 0, false, { never, 0.10, 0.16, 0.25, 0.40 }, 5 },
        { 1, false, { 0.0, 0.02, 0.035, 0.06, never }, 5 },
        { 2, true, { 0.0, 0.01, 0.02, 0.04, never }, 5 },
        { 3, true, { 0.5, 0.75, 1.0, never, never }, 4 },
        { 4, true, { 0.0, 1.0, 8.0, 32.0, all }, 5 },
        { 5, false, { 0.0, 1.0, 8.0, 32.0, all }, 5 },
    };
    for (const Search &q : searches) {
        for (int k = 0; k < q.n; ++k) {
            tomo_plane_rules r = entry->rules;
            double *fld = q.field == 0 ? &r.min_pitch
                          : q.field == 1 ? &r.general_ratio
                          : q.field == 2 ? &r.fwd_max_ratio
                          : q.field == 3 ? &r.fwd_min_pitch
                          : q.field == 4 ? &r.fwd_group
                                         : &r.adj_group;
            if (*fld == q.cand[k]) continue;
            *fld = q.cand[k];
            const tomo_plane_rules keep = entry->rules;
            entry->rules = r;
            float f, a;
            if ((st = time_schedule(ctx, prob, entry->tl, (float *)ctx->t.p,
                                    (float *)ctx->q.p, s, &f, &a)))
                return st;
            const float now = q.forward_only ? f : f + a;
            const float was = q.forward_only ? cur_f : cur_f + cur_a;
            if (now < 0.99f * was) {
                cur_f = f;
                cur_a = a;
            } else {
                entry->rules = keep;
            }
        }
    }
    entry->fwd_ms = cur_f;
    entry->adj_ms = cur_a;
    // leave the cached hints on the winning rules
    if ((st = prepare_rays(ctx, &prob->cube, 1, &prob->img,
                           prob->pointing_host, s)))
        return st;
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (best_out) {
        best_out->tile_u = entry->tl.tile_u;
        best_out->tile_v = entry->tl.tile_v;
        best_out->warp_u = entry->tl.warp_u;
        best_out->fwd_ms = entry->fwd_ms;
        best_out->adj_ms = entry->adj_ms;
        best_out->rules = entry->rules;
    }
    return TOMO_OK;
}

tomo_status tomo_set_plane_rules(tomo_ctx *ctx, const tomo_cube_geom *cube,
                                 const tomo_image_geom *img,
                                 const tomo_plane_rules *rules)
{
    if (!ctx) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    if ((cube == nullptr) != (img == nullptr))
        return fail(ctx, TOMO_ERR_ARG, "cube and img must both be given or "
                                       "both be NULL");
    const tomo_plane_rules r = rules ? *rules : default_plane_rules();
    const double v[6] = { r.min_pitch, r.fwd_min_pitch, r.fwd_max_ratio,
                          r.general_ratio, r.fwd_group, r.adj_group };
    for (double x : v)
        if (!(x >= 0.0) || isnan(x))
            return fail(ctx, TOMO_ERR_ARG, "plane rules must be >= 0");
    if (!cube) {
        ctx->rules = r;
        return TOMO_OK;
    }
    tomo_status st;
    if ((st = check_cube(ctx, cube, 1)) || (st = check_img(ctx, img)))
        return st;
    Tuned *e = bucket_of(ctx, cube, img);
    if (!e) {
        Tuned t;
        t.nx = cube->nx;
        t.ny = cube->ny;
        t.nz = cube->nz;
        t.nu = img->nu;
        t.nv = img->nv;
        t.tl = ctx->tiling;
        t.fwd_ms = t.adj_ms = INFINITY;
        ctx->tuned.push_back(t);
        e = &ctx->tuned.back();
    }
    e->rules = r;
    return TOMO_OK;
}

tomo_status tomo_project_batched(tomo_ctx *ctx, int32_t n,
                                 const tomo_problem *probs, void *stream)
{
    if (!ctx || n < 0 || (n > 0 && !probs)) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    if (n == 0) return TOMO_OK;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    return batched_walk(ctx, n, probs, false, 0, (cudaStream_t)stream);
}

tomo_status tomo_backproject_batched(tomo_ctx *ctx, int32_t n,
                                     const tomo_problem *probs, uint32_t flags,
                                     void *stream)
{
    if (!ctx || n < 0 || (n > 0 && !probs)) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    if (flags & ~TOMO_ACCUMULATE)
        return fail(ctx, TOMO_ERR_ARG, "unknown flags 0x%x", flags);
    if (n == 0) return TOMO_OK;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    return batched_walk(ctx, n, probs, true, flags, (cudaStream_t)stream);
}

tomo_status tomo_solve_batched(tomo_ctx *ctx, int32_t n,
                               const tomo_problem *probs, int32_t n_iter,
                               uint32_t flags, double *report_host,
                               int32_t *iters_host, void *stream)
{
    if (!ctx || n < 0 || (n > 0 && !probs)) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    if (flags & ~(TOMO_SOLVE_X0 | TOMO_BATCH_AUTOTUNE))
        return fail(ctx, TOMO_ERR_ARG, "unknown flags 0x%x", flags);
    if (n_iter < 0 || n_iter > 100000)
        return fail(ctx, TOMO_ERR_ARG, "n_iter must be in [0, 1e5]");
    if (n == 0) return TOMO_OK;
    tomo_status st;
    for (int32_t i = 0; i < n; ++i)
        if ((st = check_problem(ctx, &probs[i], i, true, true))) return st;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    cudaStream_t s = (cudaStream_t)stream;
    const bool warm = (flags & TOMO_SOLVE_X0) != 0;

    if (flags & TOMO_BATCH_AUTOTUNE) {
        for (int32_t i = 0; i < n; ++i) {
            const tomo_problem &p = probs[i];
            bool known = p.img.n_img == 0;
            for (const Tuned &e : ctx->tuned)
                known |= e.nx == p.cube.nx && e.ny == p.cube.ny &&
                         e.nz == p.cube.nz && e.nu == p.img.nu &&
                         e.nv == p.img.nv;
            if (!known && (st = tomo_autotune(ctx, &p, nullptr, stream)))
                return st;
        }
    }
    if ((st = prepare_batch(ctx, n, probs, s))) return st;
    BatchPlan *P = ctx->plan;

    // graph key: geometry plan + caller buffers + lambdas + run shape
    uint64_t h = P->geom_key;
    for (int32_t i = 0; i < n; ++i) {
        const void *ptrs[5] = { probs[i].images_dev, probs[i].cube_dev,
                                probs[i].mask_dev, probs[i].map_mask_dev,
                                probs[i].prior_weight_dev };
        h = fnv1a(h, ptrs, sizeof(ptrs));
        h = fnv1a(h, &probs[i].lambda, sizeof(double));
    }
    h = fnv1a(h, &n_iter, sizeof(n_iter));
    h = fnv1a(h, &flags, sizeof(flags));
    const bool plane = batch_plane(ctx, n, probs);
    const bool plane_fwd = batch_plane_forward(ctx, n, probs);
    h = fnv1a(h, &plane, sizeof(plane));
    h = fnv1a(h, &plane_fwd, sizeof(plane_fwd));
    const size_t stride = 2 * ((size_t)n_iter + 1);

    if (!(P->exec && P->graph_key == h)) {
        P->graph_key = 0;
        if (P->exec) cudaGraphExecDestroy(P->exec);
        if (P->graph) cudaGraphDestroy(P->graph);
        P->exec = nullptr;
        P->graph = nullptr;
        // workspace: b, r, p, q per problem (voxels), t per problem (pixels)
        std::vector<int64_t> voff(n + 1, 0), poff(n + 1, 0), vitems(n + 1, 0),
            pitems(n + 1, 0);
        for (int32_t i = 0; i < n; ++i) {
            const int64_t nv = (int64_t)probs[i].cube.nx * probs[i].cube.ny *
                               probs[i].cube.nz;
            const int64_t np = P->ray_off[i + 1] - P->ray_off[i];
            voff[i + 1] = voff[i] + nv;
            poff[i + 1] = poff[i] + np;
            vitems[i + 1] = vitems[i] + (nv + kChunk - 1) / kChunk;
            pitems[i + 1] = pitems[i] + (np + kChunk - 1) / kChunk;
        }
        const int64_t NV = voff[n];
        const int64_t max_items = vitems[n] > pitems[n] ? vitems[n] : pitems[n];
        // queue counters: up to two walks (plane tiles, dense problems per
        // ray) per projection
        const int n_walks = 2 * (1 + (warm ? 2 : 0) + 2 * n_iter);
        if ((st = ensure(ctx, P->vec, sizeof(float) * 4 * NV)) ||
            (st = ensure(ctx, P->timg, sizeof(float) * (poff[n] > 0 ? poff[n] : 1))) ||
            (st = ensure(ctx, P->S, sizeof(double) * n * (S_NSLOTS + stride))) ||
            (st = ensure(ctx, P->partials, sizeof(double) * 2 * max_items)) ||
            (st = ensure(ctx, P->counters, sizeof(unsigned long long) * n_walks)))
            return st;
        float *vb = (float *)P->vec.p, *vr = vb + NV, *vp = vr + NV, *vq = vp + NV;
        float *tim = (float *)P->timg.p;
        double *S = (double *)P->S.p;
        double *rep = S + (size_t)n * S_NSLOTS;
        // descriptors: walks [b, fwd_x, adj_x, fwd, adj] x n, then vectors
        std::vector<WalkDesc> wd(5 * (size_t)n);
        std::vector<VecDesc> vd(n);
        for (int32_t i = 0; i < n; ++i) {
            const tomo_problem &p = probs[i];
            double *Si = S + (size_t)i * S_NSLOTS;
            const double *done = Si + S_DONE;
            float *bi = vb + voff[i], *ri = vr + voff[i], *pi = vp + voff[i],
                  *qi = vq + voff[i], *ti = tim + poff[i];
            wd[0 * n + i] = walk_desc(P, p, i, p.images_dev, bi, nullptr, false);
            wd[1 * n + i] = walk_desc(P, p, i, p.cube_dev, ti, nullptr, true);
            wd[2 * n + i] = walk_desc(P, p, i, ti, qi, nullptr, false);
            wd[3 * n + i] = walk_desc(P, p, i, pi, ti, done, true);
            wd[4 * n + i] = walk_desc(P, p, i, ti, qi, done, false);
            VecDesc &v = vd[i];
            v.x = p.cube_dev;
            v.r = ri;
            v.p = pi;
            v.q = qi;
            v.b = bi;
            v.y = p.images_dev;
            v.mask = p.mask_dev;
            v.mm = p.map_mask_dev;
            v.w = p.prior_weight_dev;
            v.S = Si;
            v.report = rep + (size_t)i * stride;
            v.n = voff[i + 1] - voff[i];
            v.m = poff[i + 1] - poff[i];
            v.nx = p.cube.nx;
            v.ny = p.cube.ny;
            v.nz = p.cube.nz;
            v.lam = (float)p.lambda;
        }
        // combine jobs of the plane-synchronous transposes: into b, into q,
        // into q skipping problems that are done
        std::vector<float *> bs(n), qs(n);
        std::vector<const double *> dn(n);
        for (int32_t i = 0; i < n; ++i) {
            bs[i] = vb + voff[i];
            qs[i] = vq + voff[i];
            dn[i] = S + (size_t)i * S_NSLOTS + S_DONE;
        }
        std::vector<LayoutJob> jobs = layout_jobs(P, n, probs, bs.data(), nullptr);
        const std::vector<LayoutJob> jq = layout_jobs(P, n, probs, qs.data(), nullptr);
        const std::vector<LayoutJob> jqd = layout_jobs(P, n, probs, qs.data(), dn.data());
        jobs.insert(jobs.end(), jq.begin(), jq.end());
        jobs.insert(jobs.end(), jqd.begin(), jqd.end());
        if ((st = upload(ctx, P->solve_jobs, jobs.data(), sizeof(LayoutJob) * jobs.size(), s)))
            return st;
        // copy jobs of the plane forwards: from x (warm start), from p
        std::vector<float *> xs(n), ps(n);
        for (int32_t i = 0; i < n; ++i) {
            xs[i] = probs[i].cube_dev;
            ps[i] = vp + voff[i];
        }
        std::vector<LayoutJob> fj = layout_jobs(P, n, probs, xs.data(), nullptr, true);
        const std::vector<LayoutJob> fp = layout_jobs(P, n, probs, ps.data(), dn.data(), true);
        fj.insert(fj.end(), fp.begin(), fp.end());
        if ((st = upload(ctx, P->solve_fjobs, fj.data(), sizeof(LayoutJob) * fj.size(), s)))
            return st;
        if (P->lay_dirty)
            CUDA_TRY(ctx, cudaMemsetAsync(P->lay.p, 0,
                                          sizeof(float) * 2 * P->vox_off[n], s));
        P->lay_dirty = false;
        std::vector<int64_t> pre;  // tile, voxel-item, pixel-item prefixes
        pre.insert(pre.end(), P->tile_prefix.begin(), P->tile_prefix.end());
        pre.insert(pre.end(), vitems.begin(), vitems.end());
        pre.insert(pre.end(), pitems.begin(), pitems.end());
        if ((st = upload(ctx, P->walk_desc, wd.data(), sizeof(WalkDesc) * wd.size(), s)) ||
            (st = upload(ctx, P->vec_desc, vd.data(), sizeof(VecDesc) * n, s)) ||
            (st = upload(ctx, P->prefixes, pre.data(), sizeof(int64_t) * pre.size(), s)))
            return st;
        CUDA_TRY(ctx, cudaStreamSynchronize(s));  // uploads done before capture

        if (!ctx->capture_stream)
            CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream,
                                                    cudaStreamNonBlocking));
        cudaStream_t c = ctx->capture_stream;
        const WalkDesc *W = (const WalkDesc *)P->walk_desc.p;
        const VecDesc *V = (const VecDesc *)P->vec_desc.p;
        const int64_t *tile_pre = (const int64_t *)P->prefixes.p;
        const int64_t *vox_pre = tile_pre + (n + 1);
        const int64_t *pix_pre = vox_pre + (n + 1);
        unsigned long long *ctr = (unsigned long long *)P->counters.p;
        int next_ctr = 0;
        const int2 *sch = (const int2 *)P->sched_dev.p;
        const int64_t nch = P->n_chunks;
        double *part = (double *)P->partials.p;
        const int wgrid = walk_grid(ctx);
        const int vgrid = (int)(max_items < 4 * walk_grid(ctx) ? max_items
                                                               : 4 * walk_grid(ctx));
        int64_t counts[TOMO_K_COUNT] = { 0 };
        cudaError_t e = cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess)
            return fail(ctx, TOMO_ERR_CUDA, "begin capture: %s",
                        cudaGetErrorString(e));
#define CAP(kind, call)                                                      \
    do {                                                                     \
        if (e == cudaSuccess) e = (call);                                    \
        counts[kind] += 1;                                                   \
    } while (0)
        // transpose of walk-descriptor set `ws` (combine-job set `js` for
        // the plane-synchronous walk)
        const LayoutJob *JB = (const LayoutJob *)P->solve_jobs.p;
        const int64_t *jpre = (const int64_t *)P->jpre_dev.p;
        const int64_t *ptile_pre = (const int64_t *)P->ptpre_dev.p;
        const int2 *psch = (const int2 *)P->psched_dev.p;
        const int cgrid = combine_grid(ctx);
        const int pgrid = plane_walk_grid(ctx);
        const LayoutJob *FJ = (const LayoutJob *)P->solve_fjobs.p;
        const int64_t *rtile_pre = (const int64_t *)P->rtpre_dev.p;
        const int2 *rsch = (const int2 *)P->rsched_dev.p;
        // forward of walk-descriptor set `ws` (copy-job set `js` for the
        // plane forward; problems too dense for the plane walks per ray)
#define CAP_FWD(ws, js)                                                      \
    do {                                                                     \
        if (plane_fwd) {                                                     \
            CAP(TOMO_K_LAYOUT,                                               \
                launch_to_layout_batched(FJ + (js) * 2 * n, jpre, 2 * n,     \
                                         cgrid, c));                         \
            if (P->pn_chunks > 0)                                            \
                CAP(TOMO_K_FORWARD,                                          \
                    launch_forward_plane_batched(W + (ws) * n, ptile_pre,    \
                                                 n, P->ptile_prefix[n], c)); \
            if (P->rn_chunks > 0)                                            \
                CAP(TOMO_K_FORWARD,                                          \
                    launch_walk_batched(false, W + (ws) * n, rtile_pre, rsch, \
                                        P->rn_chunks, ctr + next_ctr++,      \
                                        wgrid, c));                          \
        } else {                                                             \
            CAP(TOMO_K_FORWARD,                                              \
                launch_walk_batched(false, W + (ws) * n, tile_pre, sch, nch, \
                                    ctr + next_ctr++, wgrid, c));            \
        }                                                                    \
    } while (0)
#define CAP_ADJ(ws, js)                                                      \
    do {                                                                     \
        if (plane) {                                                         \
            if (P->pn_chunks > 0)                                            \
                CAP(TOMO_K_ADJOINT,                                          \
                    launch_adjoint_plane_batched(W + (ws) * n, ptile_pre,    \
                                                 psch, P->pn_chunks,         \
                                                 ctr + next_ctr++, pgrid, c)); \
            if (P->rn_chunks > 0)                                            \
                CAP(TOMO_K_ADJOINT,                                          \
                    launch_walk_batched(true, W + (ws) * n, rtile_pre, rsch, \
                                        P->rn_chunks, ctr + next_ctr++,      \
                                        wgrid, c));                          \
            CAP(TOMO_K_LAYOUT,                                               \
                launch_add_from_layout_batched(JB + (js) * 2 * n, jpre,      \
                                               2 * n, cgrid, c));            \
        } else {                                                             \
            CAP(TOMO_K_ADJOINT,                                              \
                launch_walk_batched(true, W + (ws) * n, tile_pre, sch, nch,  \
                                    ctr + next_ctr++, wgrid, c));            \
        }                                                                    \
    } while (0)
        e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * n_walks, c);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(S, 0, sizeof(double) * n * S_NSLOTS, c);
        CAP(TOMO_K_VECTOR, launch_fill_f64(rep, NAN, (int64_t)(n * stride), c));
        CAP(TOMO_K_VECTOR, launch_vec_batched(BV_SUMSQ, V, pix_pre, n, warm, part,
                                              vgrid, c));
        CAP(TOMO_K_VECTOR, launch_finalize_batched(BV_SUMSQ, V, pix_pre, n, 0.0,
                                                   part, c));
        CAP(TOMO_K_VECTOR, launch_vec_batched(BV_ZERO, V, vox_pre, n, warm, part,
                                              vgrid, c));
        CAP_ADJ(0, 0);
        if (warm) {
            CAP(TOMO_K_PRIOR, launch_vec_batched(BV_PRIOR_X, V, vox_pre, n, warm,
                                                 part, vgrid, c));
            CAP_FWD(1, 0);
            CAP_ADJ(2, 1);
        }
        CAP(TOMO_K_VECTOR, launch_vec_batched(BV_INIT, V, vox_pre, n, warm, part,
                                              vgrid, c));
        CAP(TOMO_K_VECTOR, launch_finalize_batched(BV_INIT, V, vox_pre, n, 0.0,
                                                   part, c));
        for (int32_t k = 0; k < n_iter; ++k) {
            CAP_FWD(3, 1);
            CAP(TOMO_K_PRIOR, launch_vec_batched(BV_PRIOR, V, vox_pre, n, warm,
                                                 part, vgrid, c));
            CAP_ADJ(4, 2);
            CAP(TOMO_K_VECTOR, launch_vec_batched(BV_PQ, V, vox_pre, n, warm,
                                                  part, vgrid, c));
            CAP(TOMO_K_VECTOR, launch_finalize_batched(BV_PQ, V, vox_pre, n, 0.0,
                                                       part, c));
            CAP(TOMO_K_VECTOR, launch_vec_batched(BV_UPDATE, V, vox_pre, n, warm,
                                                  part, vgrid, c));
            CAP(TOMO_K_VECTOR, launch_finalize_batched(BV_UPDATE, V, vox_pre, n,
                                                       0.0, part, c));
            CAP(TOMO_K_VECTOR, launch_vec_batched(BV_DIR, V, vox_pre, n, warm,
                                                  part, vgrid, c));
        }
#undef CAP_ADJ
#undef CAP_FWD
#undef CAP
        cudaGraph_t g = nullptr;
        const cudaError_t e_end = cudaStreamEndCapture(c, &g);
        if (e != cudaSuccess || e_end != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(ctx, TOMO_ERR_CUDA, "graph capture: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e_end));
        }
        P->graph = g;
        CUDA_TRY(ctx, cudaGraphInstantiate(&P->exec, g, 0));
        for (int k = 0; k < TOMO_K_COUNT; ++k) P->graph_launches[k] = counts[k];
        P->graph_key = h;
        P->n_iter = n_iter;
        P->report_stride = stride;
    }
    // the initial-residual step reads lambda from the descriptors; the
    // tolerance is not used by the batched solver (fixed iteration count)
    CUDA_TRY(ctx, cudaGraphLaunch(P->exec, s));
    for (int k = 0; k < TOMO_K_COUNT; ++k) ctx->launches[k] += P->graph_launches[k];
    if (report_host || iters_host) {
        std::vector<double> slots((size_t)n * S_NSLOTS);
        CUDA_TRY(ctx, cudaMemcpyAsync(slots.data(), P->S.p,
                                      sizeof(double) * slots.size(),
                                      cudaMemcpyDeviceToHost, s));
        if (report_host)
            CUDA_TRY(ctx, cudaMemcpyAsync(
                              report_host, (double *)P->S.p + (size_t)n * S_NSLOTS,
                              sizeof(double) * n * P->report_stride,
                              cudaMemcpyDeviceToHost, s));
        CUDA_TRY(ctx, cudaStreamSynchronize(s));
        for (int32_t i = 0; i < n; ++i) {
            if (iters_host) iters_host[i] = (int32_t)slots[(size_t)i * S_NSLOTS + S_ITERS];
            if (slots[(size_t)i * S_NSLOTS + S_ERR] != 0.0)
                return fail(ctx, TOMO_ERR_NUMERIC, "problem %d: CG breakdown", i);
        }
    }
    return TOMO_OK;
}

}  // extern "C"
