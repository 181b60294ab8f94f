// C ABI of libtomo: argument validation, workspace, ray-record cache and the
// orchestration of the projector and of the CG solver.  Declarations and the
// contract of every entry point are in include/tomo.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include <cuda_runtime.h>

#include "host.h"

using namespace tomo;
using namespace tomo::host;

namespace tomo {
namespace host {

tomo_status fail(tomo_ctx *ctx, tomo_status st, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return st;
}


tomo_status ensure(tomo_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return TOMO_OK;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess)
            return fail(ctx, TOMO_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(ctx, TOMO_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes,
                    cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return TOMO_OK;
}

bool finite_all(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(v[i])) return false;
    return true;
}

tomo_status check_cube(tomo_ctx *ctx, const tomo_cube_geom *c, int32_t n_frames)
{
    if (!c) return fail(ctx, TOMO_ERR_ARG, "cube geometry is NULL");
    if (c->nx < 1 || c->ny < 1 || c->nz < 1)
        return fail(ctx, TOMO_ERR_ARG, "cube counts must be >= 1 (got %d %d %d)",
                    c->nx, c->ny, c->nz);
    if (c->reserved != 0)
        return fail(ctx, TOMO_ERR_ARG, "cube geometry: reserved must be 0");
    const double v[7] = { c->x0, c->y0, c->z0, c->dx, c->dy, c->dz, c->r_obs };
    if (!finite_all(v, 7) || !(c->dx > 0) || !(c->dy > 0) || !(c->dz > 0))
        return fail(ctx, TOMO_ERR_ARG, "cube corner/voxel size/r_obs must be "
                                       "finite, voxel size > 0");
    if (c->r_obs < 0)
        return fail(ctx, TOMO_ERR_ARG, "r_obs must be >= 0");
    const int64_t nvox = (int64_t)c->nx * c->ny * c->nz;
    if (nvox > INT32_MAX)
        return fail(ctx, TOMO_ERR_UNSUPPORTED,
                    "cube of %lld voxels exceeds 2^31-1 per frame",
                    (long long)nvox);
    if (n_frames < 1 || n_frames > 65535)
        return fail(ctx, TOMO_ERR_ARG, "n_frames must be in [1, 65535]");
    if (c->nz > 65535)
        return fail(ctx, TOMO_ERR_UNSUPPORTED, "nz > 65535");
    return TOMO_OK;
}

tomo_status check_img(tomo_ctx *ctx, const tomo_image_geom *g)
{
    if (!g) return fail(ctx, TOMO_ERR_ARG, "image geometry is NULL");
    if (g->n_img < 0 || g->n_img > 65535)
        return fail(ctx, TOMO_ERR_ARG, "n_img must be in [0, 65535]");
    if (g->n_img > 0 && (g->nu < 1 || g->nv < 1 || g->nu > 1 << 20 ||
                         g->nv > 1 << 19))
        return fail(ctx, TOMO_ERR_ARG, "image size out of range (%d x %d)",
                    g->nu, g->nv);
    if (g->kind < TOMO_KIND_EMISSION || g->kind > TOMO_KIND_B)
        return fail(ctx, TOMO_ERR_ARG, "unknown image kind %d", g->kind);
    if (g->kind != TOMO_KIND_EMISSION &&
        !(isfinite(g->limb_u) && g->limb_u >= 0.0 && g->limb_u <= 1.0))
        return fail(ctx, TOMO_ERR_ARG, "limb_u must be in [0, 1]");
    return TOMO_OK;
}

tomo_status check_pointing(tomo_ctx *ctx, const tomo_pointing *p,
                           const tomo_image_geom *g, int32_t n_frames)
{
    if (g->n_img == 0) return TOMO_OK;
    if (!p) return fail(ctx, TOMO_ERR_ARG, "pointing table is NULL");
    const double half_pi = 1.5707963267948966;
    for (int32_t n = 0; n < g->n_img; ++n) {
        const tomo_pointing &q = p[n];
        if (!finite_all(&q.d_obs, 12))
            return fail(ctx, TOMO_ERR_ARG, "pointing %d: non-finite field", n);
        if (!(q.d_obs > 0))
            return fail(ctx, TOMO_ERR_ARG, "pointing %d: d_obs must be > 0", n);
        if (!(fabs(cos(q.lat)) > 1e-9))
            return fail(ctx, TOMO_ERR_ARG,
                        "pointing %d: |lat| = 90 deg leaves the frame undefined", n);
        const double th[4] = {
            (0 - q.crpix_u) * q.cdelt_u + q.crval_u,
            (g->nu - 1 - q.crpix_u) * q.cdelt_u + q.crval_u,
            (0 - q.crpix_v) * q.cdelt_v + q.crval_v,
            (g->nv - 1 - q.crpix_v) * q.cdelt_v + q.crval_v };
        for (int i = 0; i < 4; ++i)
            if (!(fabs(th[i]) < half_pi - 1e-6))
                return fail(ctx, TOMO_ERR_ARG,
                            "pointing %d: pixel angle reaches 90 deg", n);
        if (n_frames > 1 && !(q.time >= 0.0 && q.time <= n_frames - 1))
            return fail(ctx, TOMO_ERR_ARG,
                        "pointing %d: time %g outside [0, %d]", n, q.time,
                        n_frames - 1);
    }
    return TOMO_OK;
}

tomo_status check_tiling(tomo_ctx *ctx, Tiling t)
{
    const int wu = t.warp_u;
    if (wu < 1 || wu > 32 || (wu & (wu - 1)) != 0)
        return fail(ctx, TOMO_ERR_ARG, "warp_u must be a power of 2 in [1, 32]");
    if (t.tile_u < 1 || t.tile_v < 1 || t.tile_u % wu != 0 ||
        t.tile_v % (32 / wu) != 0 || t.tile_u * t.tile_v > 512)
        return fail(ctx, TOMO_ERR_ARG,
                    "tile %dx%d incompatible with warp_u %d (<= 512 threads)",
                    t.tile_u, t.tile_v, wu);
    return TOMO_OK;
}

bool aligned(const void *p, size_t a)
{
    return ((uintptr_t)p % a) == 0;
}

uint64_t fnv1a(uint64_t h, const void *data, size_t n)
{
    const unsigned char *c = (const unsigned char *)data;
    for (size_t i = 0; i < n; ++i) {
        h ^= c[i];
        h *= 1099511628211ull;
    }
    return h;
}

CubeDev cube_dev(const tomo_cube_geom *c)
{
    CubeDev d;
    d.nx = c->nx;
    d.ny = c->ny;
    d.nz = c->nz;
    d.lo[0] = c->x0;
    d.lo[1] = c->y0;
    d.lo[2] = c->z0;
    d.r_obs = c->r_obs;
    d.d[0] = c->dx;
    d.d[1] = c->dy;
    d.d[2] = c->dz;
    const int32_t n[3] = { c->nx, c->ny, c->nz };
    for (int k = 0; k < 3; ++k) {
        d.inv_d[k] = 1.0 / d.d[k];
        d.hi[k] = d.lo[k] + n[k] * d.d[k];
    }
    return d;
}

// Builds (or reuses) the ray records and image parameters of a geometry on
// `s`.  On return, work on `s` is ordered after the records are complete.
tomo_status prepare_rays(tomo_ctx *ctx, const tomo_cube_geom *c,
                         int32_t n_frames, const tomo_image_geom *g,
                         const tomo_pointing *ptg, cudaStream_t s)
{
    uint64_t h = 1469598103934665603ull;
    const int32_t cn[4] = { c->nx, c->ny, c->nz, n_frames };
    const double cv[7] = { c->x0, c->y0, c->z0, c->dx, c->dy, c->dz, c->r_obs };
    h = fnv1a(h, cn, sizeof(cn));
    h = fnv1a(h, cv, sizeof(cv));
    h = fnv1a(h, g, sizeof(*g));
    h = fnv1a(h, ptg, sizeof(tomo_pointing) * (size_t)g->n_img);
    const tomo_plane_rules rules = rules_for(ctx, c, g);
    const uint64_t hh = fnv1a(h, &rules, sizeof(rules));
    tomo_status st;
    if ((st = ensure(ctx, ctx->layout_used, sizeof(unsigned))) ||
        (st = ensure(ctx, ctx->per_ray_fwd,
                     sizeof(unsigned) * (1 + (size_t)g->n_img))))
        return st;
    if (ctx->ray_cache && ctx->key_valid && ctx->key == h) {
        if (ctx->hint_key == hh) {
            CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->setup_done, 0));
            return TOMO_OK;
        }
        // same rays, other walk rules: only the per-image hints change
        CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->setup_done, 0));
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->layout_used.p, 0, sizeof(unsigned), s));
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->per_ray_fwd.p, 0, sizeof(unsigned), s));
        ctx->fwd_plane_possible = false;
        ctx->fwd_plane_all = true;
        ctx->plane_possible = false;
        for (int32_t i = 0; i < g->n_img; ++i) {
            const bool f = plane_forward_estimate(ptg[i], c, rules);
            ctx->plane_possible |= plane_estimate(ptg[i], c, rules);
            ctx->fwd_plane_possible |= f;
            ctx->fwd_plane_all &= f;
        }
        LAUNCH(ctx, TOMO_K_SETUP, s,
               launch_frames((const tomo_pointing *)ctx->ptg.p, g->n_img, g->nu,
                             g->nv, n_frames, (Frame *)ctx->frames.p,
                             (double *)ctx->tan_u.p, (double *)ctx->tan_v.p,
                             (ImgParam *)ctx->params.p,
                             make_double3(c->dx, c->dy, c->dz),
                             (unsigned *)ctx->layout_used.p,
                             (unsigned *)ctx->per_ray_fwd.p, rules, s));
        CUDA_TRY(ctx, cudaEventRecord(ctx->setup_done, s));
        ctx->hint_key = hh;
        return TOMO_OK;
    }
    ctx->key_valid = false;
    const size_t n_img = (size_t)g->n_img;
    const size_t npix = n_img * g->nu * g->nv;
    if ((st = ensure(ctx, ctx->ptg, sizeof(tomo_pointing) * n_img)) ||
        (st = ensure(ctx, ctx->frames, sizeof(Frame) * n_img)) ||
        (st = ensure(ctx, ctx->tan_u, sizeof(double) * n_img * g->nu)) ||
        (st = ensure(ctx, ctx->tan_v, sizeof(double) * n_img * g->nv)) ||
        (st = ensure(ctx, ctx->params, sizeof(ImgParam) * n_img)) ||
        (st = ensure(ctx, ctx->rays, sizeof(RayRec) * npix)))
        return st;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ptg.p, ptg, sizeof(tomo_pointing) * n_img,
                                  cudaMemcpyHostToDevice, s));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->layout_used.p, 0, sizeof(unsigned), s));
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->per_ray_fwd.p, 0, sizeof(unsigned), s));
    ctx->fwd_plane_possible = false;
    ctx->fwd_plane_all = true;
    ctx->plane_possible = false;
    for (size_t i = 0; i < n_img; ++i) {
        const bool f = plane_forward_estimate(ptg[i], c, rules);
        ctx->plane_possible |= plane_estimate(ptg[i], c, rules);
        ctx->fwd_plane_possible |= f;
        ctx->fwd_plane_all &= f;
    }
    LAUNCH(ctx, TOMO_K_SETUP, s,
           launch_frames((const tomo_pointing *)ctx->ptg.p, g->n_img, g->nu,
                         g->nv, n_frames, (Frame *)ctx->frames.p,
                         (double *)ctx->tan_u.p, (double *)ctx->tan_v.p,
                         (ImgParam *)ctx->params.p,
                         make_double3(c->dx, c->dy, c->dz),
                         (unsigned *)ctx->layout_used.p,
                         (unsigned *)ctx->per_ray_fwd.p, rules, s));
    LAUNCH(ctx, TOMO_K_SETUP, s,
           launch_ray_setup((const Frame *)ctx->frames.p,
                            (const double *)ctx->tan_u.p,
                            (const double *)ctx->tan_v.p, cube_dev(c),
                            g->n_img, g->nu, g->nv, (RayRec *)ctx->rays.p, s));
    if (g->kind != TOMO_KIND_EMISSION) {
        if ((st = ensure(ctx, ctx->rho2, sizeof(float) * (npix > 0 ? npix : 1))))
            return st;
        LAUNCH(ctx, TOMO_K_SETUP, s,
               launch_impact2((const Frame *)ctx->frames.p,
                              (const double *)ctx->tan_u.p,
                              (const double *)ctx->tan_v.p, g->n_img, g->nu,
                              g->nv, (float *)ctx->rho2.p, s));
    }
    CUDA_TRY(ctx, cudaEventRecord(ctx->setup_done, s));
    ctx->key = h;
    ctx->hint_key = hh;
    ctx->cached_n_img = g->n_img;
    ctx->cached_cube = *c;
    ctx->key_valid = true;
    return TOMO_OK;
}

tomo_status common_checks(tomo_ctx *ctx, const tomo_cube_geom *c,
                          int32_t n_frames, const tomo_image_geom *g,
                          const tomo_pointing *ptg)
{
    tomo_status st;
    if ((st = check_cube(ctx, c, n_frames)) || (st = check_img(ctx, g)) ||
        (st = check_pointing(ctx, ptg, g, n_frames)) ||
        (st = check_tiling(ctx, tiling_for(ctx, c, g))))
        return st;
    return TOMO_OK;
}

Tiling tiling_for(const tomo_ctx *ctx, const tomo_cube_geom *c,
                  const tomo_image_geom *g)
{
    for (const Tuned &t : ctx->tuned)
        if (t.nx == c->nx && t.ny == c->ny && t.nz == c->nz && t.nu == g->nu &&
            t.nv == g->nv)
            return t.tl;
    return ctx->tiling;
}

tomo_plane_rules rules_for(const tomo_ctx *ctx, const tomo_cube_geom *c,
                           const tomo_image_geom *g)
{
    for (const Tuned &t : ctx->tuned)
        if (t.nx == c->nx && t.ny == c->ny && t.nz == c->nz && t.nu == g->nu &&
            t.nv == g->nv)
            return t.rules;
    return ctx->rules;
}

// The device's rules (setup.cu) evaluated from the boresight, with margins
// towards "may"; the pixel pitch with the smallest voxel side.
bool plane_estimate(const tomo_pointing &p, const tomo_cube_geom *c,
                    const tomo_plane_rules &r)
{
    const double dmin = fmin(c->dx, fmin(c->dy, c->dz));
    return p.d_obs * fabs(tan(p.cdelt_u)) / dmin >= 0.9 * r.min_pitch;
}

bool plane_forward_estimate(const tomo_pointing &p, const tomo_cube_geom *c,
                            const tomo_plane_rules &r)
{
    if (!plane_estimate(p, c, r)) return false;
    const double cl = cos(p.lat);
    const double w[3] = { fabs(cl * cos(p.lon)), fabs(cl * sin(p.lon)),
                          fabs(sin(p.lat)) };
    const double hi = fmax(w[0], fmax(w[1], w[2]));
    const double lo = fmin(w[0], fmin(w[1], w[2])) / hi;
    const double dmin = fmin(c->dx, fmin(c->dy, c->dz));
    const double pitch = p.d_obs * fabs(tan(p.cdelt_u)) / dmin;
    return pitch >= 0.9 * r.fwd_min_pitch || lo < 1.5 * r.fwd_max_ratio;
}

bool use_plane(const tomo_ctx *ctx, const tomo_cube_geom *c, Tiling t,
               bool forward)
{
    const int bits = forward ? (2 | 4) : 1;
    (void)t;
    return (ctx->plane_sync & bits) != 0 && plane_supported(c, 4);
}

tomo_status ensure_plane(tomo_ctx *ctx, const tomo_cube_geom *c,
                         int32_t n_frames, Tiling t)
{
    if (!use_plane(ctx, c, t, true) && !use_plane(ctx, c, t, false))
        return TOMO_OK;
    const size_t bytes =
        sizeof(float) * (size_t)c->nx * c->ny * c->nz * (size_t)n_frames;
    tomo_status st;
    if ((st = ensure(ctx, ctx->lay1, bytes)) || (st = ensure(ctx, ctx->lay2, bytes)))
        return st;
    return TOMO_OK;
}

// Two-value buffers for layouts 0, 1, 2: T - 1 frame pairs (or one pair)
// of 8 bytes per voxel.
tomo_status ensure_pairs(tomo_ctx *ctx, const tomo_cube_geom *c,
                         int32_t n_frames)
{
    const size_t npairs = n_frames > 1 ? (size_t)(n_frames - 1) : 1;
    const size_t bytes = 8 * (size_t)c->nx * c->ny * c->nz * npairs;
    tomo_status st;
    for (int L = 0; L < 3; ++L)
        if ((st = ensure(ctx, ctx->pr[L], bytes))) return st;
    return TOMO_OK;
}

// Images per group of a plane walk's CTA order (plane_cta): the option if
// set, else chosen from the bytes of the buffers the walk gathers from or
// adds into (all frames or frame pairs of one layout) against L2, as
// measured on GB300 (times against image-after-image order):
//  - P: every image in one group once the cube reaches a quarter of L2
//    (256^3 cube -3 %, 512^3 -10 %, 8 frame pairs -22 %, Thomson B pairs
//    -17 %; a 128^3 cube +4 %);
//  - P^T: image after image while the accumulators fit twice in L2 (one
//    group of every image: 256^3 +7 %, B pairs +2 %: the CTAs of many images
//    then add into the same lines), else groups of 8 images into a single
//    accumulator (512^3: -7 %; 32 images -6 %, every image -5 %) and one
//    group of every image when the images spread over several frame or
//    frame-pair accumulators (8 frames, 7 pairs: -14 %; 32 images -13 %,
//    8 images -8 %).
int plane_group(const tomo_ctx *ctx, const tomo_cube_geom *c,
                const tomo_image_geom *g, bool adjoint, int64_t walked_bytes,
                int n_acc)
{
    const int32_t n_img = g->n_img;
    const int opt = adjoint ? ctx->group_adj : ctx->group_fwd;
    if (opt > 0) return opt;
    const tomo_plane_rules r = rules_for(ctx, c, g);
    const double rg = adjoint ? r.adj_group : r.fwd_group;
    if (rg >= 1.0) return rg >= 65535.0 ? 65535 : (int)rg;
    const int64_t l2 = ctx->l2_bytes > 0 ? ctx->l2_bytes : (int64_t)126 << 20;
    if (!adjoint) return walked_bytes >= l2 / 4 ? n_img : 1;
    if (walked_bytes <= 2 * l2) return 1;
    return n_acc > 1 ? n_img : 8;
}

bool use_time_pairs(const tomo_ctx *ctx, const tomo_cube_geom *c,
                    int32_t n_frames)
{
    return n_frames > 1 && (ctx->channels & 1) && plane_supported(c, 8);
}

// The per-ray forward's image list when the host estimate says every image
// may take the plane forward (the list is then short or empty), else NULL:
// images certain to need the per-ray walk keep its one-CTA-per-tile grid.
const unsigned *per_ray_list(const tomo_ctx *ctx)
{
    return ctx->fwd_plane_all ? (const unsigned *)ctx->per_ray_fwd.p : nullptr;
}

tomo_status forward_one(tomo_ctx *ctx, const void *cube_dev, tomo_dtype dtype,
                        int32_t n_frames, const uint8_t *mask, float *out,
                        const tomo_cube_geom *c, const tomo_image_geom *g,
                        Tiling t, const double *done, cudaStream_t s)
{
    const RayRec *rays = (const RayRec *)ctx->rays.p;
    const ImgParam *prm = (const ImgParam *)ctx->params.p;
    const int64_t fstride = (int64_t)c->nx * c->ny * c->nz;
    // bit 1: every image plane-synchronous; else (bit 2) the images whose
    // hint marks the plane forward as faster, the rest per ray
    const bool all = (ctx->plane_sync & 2) != 0;
    if (use_plane(ctx, c, t, true) && (all || ctx->fwd_plane_possible) &&
        use_time_pairs(ctx, c, n_frames)) {
        // frame pairs side by side in every layout in use (layout 0 too)
        tomo_status st;
        if ((st = ensure_pairs(ctx, c, n_frames))) return st;
        const unsigned *used = (const unsigned *)ctx->layout_used.p;
        for (int L = 0; L <= 2; ++L)
            LAUNCH(ctx, TOMO_K_LAYOUT, s,
                   launch_to_pairs(cube_dev, dtype, ctx->pr[L].p, L, c,
                                   n_frames, used,
                                   all ? 1u << L : 1u << (8 + L), done,
                                   ctx->num_sms, s));
        PlaneCubes pc = { { ctx->pr[0].p, ctx->pr[1].p, ctx->pr[2].p } };
        if (!all)
            LAUNCH(ctx, TOMO_K_FORWARD, s,
                   launch_forward(rays, prm, cube_dev, dtype, fstride, true,
                                  mask, out, g->n_img, g->nu, g->nv, c->nx,
                                  c->nx * c->ny, t, done, s, true,
                                  per_ray_list(ctx), ctx->num_sms));
        LAUNCH(ctx, TOMO_K_FORWARD, s,
               launch_forward_plane_pair(
                   rays, prm, pc, cube_dev, dtype, fstride, mask, out,
                   g->n_img, g->nu, g->nv, c, done, s, !all,
                   plane_group(ctx, c, g, false, 8 * fstride * (n_frames - 1),
                               n_frames - 1)));
        return TOMO_OK;
    }
    if (use_plane(ctx, c, t, true) && (all || ctx->fwd_plane_possible)) {
        const unsigned *used = (const unsigned *)ctx->layout_used.p;
        for (int L = 1; L <= 2; ++L)
            LAUNCH(ctx, TOMO_K_LAYOUT, s,
                   launch_to_layout(cube_dev, dtype, L == 1 ? ctx->lay1.p : ctx->lay2.p,
                                    L, c, n_frames, used,
                                    all ? 1u << L : 1u << (8 + L), done, s));
        PlaneCubes pc = { { cube_dev, ctx->lay1.p, ctx->lay2.p } };
        if (!all)
            LAUNCH(ctx, TOMO_K_FORWARD, s,
                   launch_forward(rays, prm, cube_dev, dtype, fstride,
                                  n_frames > 1, mask, out, g->n_img, g->nu,
                                  g->nv, c->nx, c->nx * c->ny, t, done, s,
                                  true, per_ray_list(ctx), ctx->num_sms));
        LAUNCH(ctx, TOMO_K_FORWARD, s,
               launch_forward_plane(
                   rays, prm, pc, dtype, fstride, n_frames > 1, mask, out,
                   g->n_img, g->nu, g->nv, c, done, s, !all,
                   plane_group(ctx, c, g, false,
                               (dtype == TOMO_BF16 ? 2 : 4) * fstride * n_frames,
                               n_frames)));
        return TOMO_OK;
    }
    LAUNCH(ctx, TOMO_K_FORWARD, s,
           launch_forward(rays, prm, cube_dev, dtype, fstride, n_frames > 1,
                          mask, out, g->n_img, g->nu, g->nv, c->nx,
                          c->nx * c->ny, t, done, s));
    return TOMO_OK;
}

tomo_status adjoint_one(tomo_ctx *ctx, const float *images,
                        const uint8_t *mask, float *cube,
                        const tomo_cube_geom *c, int32_t n_frames,
                        const tomo_image_geom *g, Tiling t,
                        const double *done, cudaStream_t s)
{
    const RayRec *rays = (const RayRec *)ctx->rays.p;
    const ImgParam *prm = (const ImgParam *)ctx->params.p;
    if (use_plane(ctx, c, t, false) && ctx->plane_possible &&
        use_time_pairs(ctx, c, n_frames)) {
        // frame-pair accumulators in every layout in use, added into the
        // frames after the walk
        tomo_status st;
        if ((st = ensure_pairs(ctx, c, n_frames))) return st;
        const int64_t fstride = (int64_t)c->nx * c->ny * c->nz;
        const unsigned *used = (const unsigned *)ctx->layout_used.p;
        for (int L = 0; L <= 2; ++L)
            LAUNCH(ctx, TOMO_K_LAYOUT, s,
                   launch_zero_layout((float *)ctx->pr[L].p, L,
                                      2 * fstride * (n_frames - 1), used,
                                      done, ctx->num_sms, s));
        PlaneAcc pa = { { (float *)ctx->pr[0].p, (float *)ctx->pr[1].p,
                          (float *)ctx->pr[2].p } };
        LAUNCH(ctx, TOMO_K_ADJOINT, s,
               launch_adjoint_plane_pair(
                   rays, prm, images, mask, pa, cube, fstride, g->n_img,
                   g->nu, g->nv, c, done, s,
                   plane_group(ctx, c, g, true, 8 * fstride * (n_frames - 1),
                               n_frames - 1)));
        for (int L = 0; L <= 2; ++L)
            LAUNCH(ctx, TOMO_K_LAYOUT, s,
                   launch_add_pairs(ctx->pr[L].p, cube, L, c, n_frames, used,
                                    done, ctx->num_sms, s));
        return TOMO_OK;
    }
    if (use_plane(ctx, c, t, false) && ctx->plane_possible) {
        const int64_t fstride = (int64_t)c->nx * c->ny * c->nz;
        const unsigned *used = (const unsigned *)ctx->layout_used.p;
        float *a1 = (float *)ctx->lay1.p, *a2 = (float *)ctx->lay2.p;
        LAUNCH(ctx, TOMO_K_LAYOUT, s,
               launch_zero_layout(a1, 1, fstride * n_frames, used, done,
                                  ctx->num_sms, s));
        LAUNCH(ctx, TOMO_K_LAYOUT, s,
               launch_zero_layout(a2, 2, fstride * n_frames, used, done,
                                  ctx->num_sms, s));
        PlaneAcc pa = { { cube, a1, a2 } };
        LAUNCH(ctx, TOMO_K_ADJOINT, s,
               launch_adjoint_plane(
                   rays, prm, images, mask, pa, fstride, n_frames > 1,
                   g->n_img, g->nu, g->nv, c, done, s,
                   plane_group(ctx, c, g, true, 4 * fstride * n_frames,
                               n_frames)));
        LAUNCH(ctx, TOMO_K_LAYOUT, s,
               launch_add_from_layout(a1, cube, 1, c, n_frames, used, done, s));
        LAUNCH(ctx, TOMO_K_LAYOUT, s,
               launch_add_from_layout(a2, cube, 2, c, n_frames, used, done, s));
        return TOMO_OK;
    }
    const int64_t fstride = (int64_t)c->nx * c->ny * c->nz;
    LAUNCH(ctx, TOMO_K_ADJOINT, s,
           launch_adjoint(rays, prm, images, mask, cube, fstride, n_frames > 1,
                          g->n_img, g->nu, g->nv, c->nx, c->nx * c->ny, t,
                          done, s));
    return TOMO_OK;
}

// (m, m') per voxel for the cube geometry and limb darkening, cached.
tomo_status ensure_thomson(tomo_ctx *ctx, const tomo_cube_geom *c, double u,
                           cudaStream_t s)
{
    uint64_t h = 1469598103934665603ull;
    const int32_t cn[3] = { c->nx, c->ny, c->nz };
    const double cv[7] = { c->x0, c->y0, c->z0, c->dx, c->dy, c->dz, u };
    h = fnv1a(h, cn, sizeof(cn));
    h = fnv1a(h, cv, sizeof(cv));
    if (ctx->thf_valid && ctx->thf_key == h) return TOMO_OK;
    ctx->thf_valid = false;
    const int64_t n = (int64_t)c->nx * c->ny * c->nz;
    tomo_status st;
    if ((st = ensure(ctx, ctx->thf, sizeof(float2) * n))) return st;
    LAUNCH(ctx, TOMO_K_SETUP, s,
           launch_thomson_factors(cube_dev(c), u, (float2 *)ctx->thf.p, s));
    ctx->thf_key = h;
    ctx->thf_valid = true;
    return TOMO_OK;
}

// y = T x for the image kind: P (emission), O P M x (pB) or
// P M' x - O P M x (B).  mm (map mask) is applied by the Thomson prologue
// only; the emission path leaves it to the caller.
tomo_status op_forward(tomo_ctx *ctx, const void *src, tomo_dtype dtype,
                       int32_t n_frames, const uint8_t *mask,
                       const uint8_t *mm, float *out, const tomo_cube_geom *c,
                       const tomo_image_geom *g, Tiling t, const double *done,
                       cudaStream_t s)
{
    if (g->kind == TOMO_KIND_EMISSION)
        return forward_one(ctx, src, dtype, n_frames, mask, out, c, g, t,
                           done, s);
    const int64_t n = (int64_t)c->nx * c->ny * c->nz;
    const int64_t npix = (int64_t)g->n_img * g->nu * g->nv;
    tomo_status st;
    const float2 *mf = (const float2 *)ctx->thf.p;
    const float *rho2 = (const float *)ctx->rho2.p;
    const bool bf16 = dtype == TOMO_BF16;
    if (g->kind == TOMO_KIND_B && n_frames == 1 && (ctx->channels & 2)) {
        // one walk on (m' K x, m K x) pairs: y = g s' - rho^2 g s
        if ((st = ensure_pairs(ctx, c, 1))) return st;
        LAUNCH(ctx, TOMO_K_VECTOR, s,
               launch_thomson_weight2(src, bf16, mf, mm, n,
                                      (float2 *)ctx->pr[0].p, done, s));
        const bool all = (ctx->plane_sync & 2) != 0;
        const bool plane = use_plane(ctx, c, t, true) &&
                           plane_supported(c, 8) &&
                           (all || ctx->fwd_plane_possible);
        if (plane) {
            const unsigned *used = (const unsigned *)ctx->layout_used.p;
            for (int L = 1; L <= 2; ++L)
                LAUNCH(ctx, TOMO_K_LAYOUT, s,
                       launch_b_to_layout(ctx->pr[0].p, ctx->pr[L].p, L, c,
                                          used, all ? 1u << L : 1u << (8 + L),
                                          done, s));
        }
        PlaneCubes pc = { { ctx->pr[0].p, ctx->pr[1].p, ctx->pr[2].p } };
        LAUNCH(ctx, TOMO_K_FORWARD, s,
               launch_forward_b((const RayRec *)ctx->rays.p,
                                (const ImgParam *)ctx->params.p, pc, rho2,
                                mask, out, g->n_img, g->nu, g->nv, c, done,
                                plane ? (all ? 2 : 1) : 0, s,
                                plane_group(ctx, c, g, false, 8 * n, 1)));
        return TOMO_OK;
    }
    if ((st = ensure(ctx, ctx->th1, sizeof(float) * n * n_frames)) ||
        (g->kind == TOMO_KIND_B &&
         (st = ensure(ctx, ctx->thimg, sizeof(float) * (npix > 0 ? npix : 1)))))
        return st;
    float *c1 = (float *)ctx->th1.p;
    // pB: M x; B: first M' x, then M x (the scratch is reused in order)
    LAUNCH(ctx, TOMO_K_VECTOR, s,
           launch_thomson_weight(src, bf16, mf, g->kind == TOMO_KIND_B ? 1 : 0,
                                 mm, n, n_frames, c1, done, s));
    if ((st = forward_one(ctx, c1, TOMO_F32, n_frames, mask, out, c, g, t,
                          done, s)))
        return st;
    if (g->kind == TOMO_KIND_PB) {
        LAUNCH(ctx, TOMO_K_VECTOR, s,
               launch_rho2_apply(rho2, out, nullptr, out, npix, done, s));
        return TOMO_OK;
    }
    float *ti = (float *)ctx->thimg.p;
    LAUNCH(ctx, TOMO_K_VECTOR, s,
           launch_thomson_weight(src, bf16, mf, 0, mm, n, n_frames, c1, done, s));
    if ((st = forward_one(ctx, c1, TOMO_F32, n_frames, mask, ti, c, g, t,
                          done, s)))
        return st;
    LAUNCH(ctx, TOMO_K_VECTOR, s,
           launch_rho2_apply(rho2, out, ti, out, npix, done, s));
    return TOMO_OK;
}

// dst += T^T y: P^T y (emission), M P^T O y (pB) or M' P^T y - M P^T O y
// (B); the Thomson epilogue applies the map mask mm.
tomo_status op_adjoint(tomo_ctx *ctx, const float *images, const uint8_t *mask,
                       const uint8_t *mm, float *dst, const tomo_cube_geom *c,
                       int32_t n_frames, const tomo_image_geom *g, Tiling t,
                       const double *done, cudaStream_t s)
{
    if (g->kind == TOMO_KIND_EMISSION)
        return adjoint_one(ctx, images, mask, dst, c, n_frames, g, t, done, s);
    const int64_t n = (int64_t)c->nx * c->ny * c->nz;
    const int64_t npix = (int64_t)g->n_img * g->nu * g->nv;
    const bool b = g->kind == TOMO_KIND_B;
    tomo_status st;
    const float2 *mf = (const float2 *)ctx->thf.p;
    const float *rho2 = (const float *)ctx->rho2.p;
    if (b && n_frames == 1 && (ctx->channels & 2)) {
        // one walk scattering (g y, rho^2 g y) into pair accumulators, then
        // dst += K (m' a - m b)
        if ((st = ensure_pairs(ctx, c, 1))) return st;
        const bool plane = use_plane(ctx, c, t, false) &&
                           plane_supported(c, 8) && ctx->plane_possible;
        const unsigned *used = (const unsigned *)ctx->layout_used.p;
        CUDA_TRY(ctx, cudaMemsetAsync(ctx->pr[0].p, 0, 8 * (size_t)n, s));
        if (plane)
            for (int L = 1; L <= 2; ++L)
                LAUNCH(ctx, TOMO_K_LAYOUT, s,
                       launch_zero_layout((float *)ctx->pr[L].p, L, 2 * n,
                                          used, done, ctx->num_sms, s));
        PlaneAcc pa = { { (float *)ctx->pr[0].p, (float *)ctx->pr[1].p,
                          (float *)ctx->pr[2].p } };
        LAUNCH(ctx, TOMO_K_ADJOINT, s,
               launch_adjoint_b((const RayRec *)ctx->rays.p,
                                (const ImgParam *)ctx->params.p, images, rho2,
                                mask, pa, g->n_img, g->nu, g->nv, c, done,
                                plane, s,
                                plane_group(ctx, c, g, true, 8 * n, 1)));
        if (plane)
            for (int L = 1; L <= 2; ++L)
                LAUNCH(ctx, TOMO_K_LAYOUT, s,
                       launch_add_b_layout(ctx->pr[L].p, ctx->pr[0].p, L, c,
                                           used, done, s));
        LAUNCH(ctx, TOMO_K_VECTOR, s,
               launch_thomson_add2(dst, (const float2 *)ctx->pr[0].p, mf, mm,
                                   n, done, s));
        return TOMO_OK;
    }
    if ((st = ensure(ctx, ctx->th1, sizeof(float) * n * n_frames)) ||
        (b && (st = ensure(ctx, ctx->th2, sizeof(float) * n * n_frames))) ||
        (st = ensure(ctx, ctx->thimg, sizeof(float) * (npix > 0 ? npix : 1))))
        return st;
    float *c1 = (float *)ctx->th1.p, *c2 = (float *)ctx->th2.p;
    float *ti = (float *)ctx->thimg.p;
    LAUNCH(ctx, TOMO_K_VECTOR, s,
           launch_rho2_apply(rho2, images, nullptr, ti, npix, done, s));
    CUDA_TRY(ctx, cudaMemsetAsync(c1, 0, sizeof(float) * n * n_frames, s));
    if (!b) {
        if ((st = adjoint_one(ctx, ti, mask, c1, c, n_frames, g, t, done, s)))
            return st;
        LAUNCH(ctx, TOMO_K_VECTOR, s,
               launch_thomson_add(dst, c1, nullptr, mf, mm, n, n_frames, done, s));
        return TOMO_OK;
    }
    CUDA_TRY(ctx, cudaMemsetAsync(c2, 0, sizeof(float) * n * n_frames, s));
    if ((st = adjoint_one(ctx, images, mask, c1, c, n_frames, g, t, done, s)) ||
        (st = adjoint_one(ctx, ti, mask, c2, c, n_frames, g, t, done, s)))
        return st;
    LAUNCH(ctx, TOMO_K_VECTOR, s,
           launch_thomson_add(dst, c1, c2, mf, mm, n, n_frames, done, s));
    return TOMO_OK;
}

// q = lambda R D^T D R x per frame (+ lambda_t D_t^T D_t x over frames).
tomo_status apply_prior(tomo_ctx *ctx, const tomo_cube_geom *c, const float *x,
                        const float *w, float *q, float lam, float lam_t,
                        int32_t n_frames, const double *done, cudaStream_t s)
{
    const int64_t nvox = (int64_t)c->nx * c->ny * c->nz;
    const CubeDev cd = cube_dev(c);
    for (int32_t f = 0; f < n_frames; ++f)
        LAUNCH(ctx, TOMO_K_PRIOR, s,
               launch_prior(cd, x + f * nvox, w, q + f * nvox, lam, false,
                            done, s));
    if (n_frames > 1 && lam_t != 0.0f)
        LAUNCH(ctx, TOMO_K_PRIOR, s,
               launch_prior_time(x, q, lam_t, nvox, n_frames, done, s));
    return TOMO_OK;
}

int reduce_grid(const tomo_ctx *ctx, int64_t n)
{
    int64_t g = (n + 255) / 256;
    int64_t cap = 4LL * (ctx->num_sms > 0 ? ctx->num_sms : 152);
    if (cap > kMaxReduceBlocks) cap = kMaxReduceBlocks;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}


}  // namespace host
}  // namespace tomo

extern "C" {

const char *tomo_status_string(tomo_status s)
{
    switch (s) {
    case TOMO_OK: return "ok";
    case TOMO_ERR_ARG: return "invalid argument";
    case TOMO_ERR_CUDA: return "CUDA error";
    case TOMO_ERR_UNSUPPORTED: return "unsupported";
    case TOMO_ERR_OOM: return "out of device memory";
    case TOMO_ERR_TIMEOUT: return "device wait timed out";
    case TOMO_ERR_NUMERIC: return "numerical breakdown";
    }
    return "unknown status";
}

const char *tomo_last_error(const tomo_ctx *ctx)
{
    return ctx ? ctx->err : "";
}

tomo_status tomo_create(tomo_ctx **out, int32_t device)
{
    if (!out) return TOMO_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 ||
        device >= count) {
        cudaGetLastError();
        return TOMO_ERR_ARG;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess)
        return TOMO_ERR_CUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return TOMO_ERR_UNSUPPORTED;
    DeviceGuard guard(device);
    if (!guard.ok) return TOMO_ERR_CUDA;
    tomo_ctx *ctx = new tomo_ctx();
    ctx->device = device;
    ctx->num_sms = prop.multiProcessorCount;
    ctx->l2_bytes = prop.l2CacheSize;
    if (cudaEventCreateWithFlags(&ctx->setup_done, cudaEventDisableTiming) !=
        cudaSuccess) {
        delete ctx;
        return TOMO_ERR_CUDA;
    }
    *out = ctx;
    return TOMO_OK;
}

void tomo_destroy(tomo_ctx *ctx)
{
    if (!ctx) return;
    DeviceGuard guard(ctx->device);
    DevBuf *bufs[] = { &ctx->ptg, &ctx->frames, &ctx->tan_u, &ctx->tan_v,
                       &ctx->params, &ctx->rays, &ctx->b, &ctx->r, &ctx->p,
                       &ctx->q, &ctx->t, &ctx->p16, &ctx->S, &ctx->partials,
                       &ctx->counter, &ctx->count64, &ctx->layout_used,
                       &ctx->per_ray_fwd,
                       &ctx->lay1, &ctx->lay2, &ctx->mcube, &ctx->rho2,
                       &ctx->thf, &ctx->th1, &ctx->th2, &ctx->thimg,
                       &ctx->pr[0], &ctx->pr[1], &ctx->pr[2] };
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    free_plan(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->setup_done) cudaEventDestroy(ctx->setup_done);
    for (cudaEvent_t e : ctx->ev_start) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->ev_stop) cudaEventDestroy(e);
    delete ctx;
}

tomo_status tomo_set_option(tomo_ctx *ctx, int32_t option, int64_t value)
{
    if (!ctx) return TOMO_ERR_ARG;
    switch (option) {
    case TOMO_OPT_RAY_CACHE:
        ctx->ray_cache = value != 0;
        if (!ctx->ray_cache) ctx->key_valid = false;
        return TOMO_OK;
    case TOMO_OPT_TILE_U:
        if (value < 1 || value > 512) break;
        ctx->tiling.tile_u = (int32_t)value;
        return TOMO_OK;
    case TOMO_OPT_TILE_V:
        if (value < 1 || value > 512) break;
        ctx->tiling.tile_v = (int32_t)value;
        return TOMO_OK;
    case TOMO_OPT_WARP_U:
        if (value < 1 || value > 32) break;
        ctx->tiling.warp_u = (int32_t)value;
        return TOMO_OK;
    case TOMO_OPT_PROFILE:
        ctx->profile = value != 0;
        return TOMO_OK;
    case TOMO_OPT_PLANE_SYNC:
        if (value < 0 || value > 7) break;
        ctx->plane_sync = (int)value;
        return TOMO_OK;
    case TOMO_OPT_CHANNELS:
        if (value < 0 || value > 3) break;
        ctx->channels = (int)value;
        return TOMO_OK;
    case TOMO_OPT_GROUP_FWD:
    case TOMO_OPT_GROUP_ADJ:
        if (value < 0 || value > 65535) break;
        (option == TOMO_OPT_GROUP_FWD ? ctx->group_fwd : ctx->group_adj) =
            (int)value;
        return TOMO_OK;
    default:
        return fail(ctx, TOMO_ERR_ARG, "unknown option %d", option);
    }
    return fail(ctx, TOMO_ERR_ARG, "option %d: value %lld out of range", option,
                (long long)value);
}

tomo_status tomo_walk_plan(tomo_ctx *ctx, int32_t n_img, int32_t *codes_host)
{
    if (!ctx) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    if (!ctx->key_valid)
        return fail(ctx, TOMO_ERR_ARG, "no geometry has been set up yet");
    if (n_img != ctx->cached_n_img || (n_img > 0 && !codes_host))
        return fail(ctx, TOMO_ERR_ARG, "n_img does not match the geometry");
    if (n_img == 0) return TOMO_OK;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    std::vector<ImgParam> prm((size_t)n_img);
    CUDA_TRY(ctx, cudaStreamWaitEvent(0, ctx->setup_done, 0));
    CUDA_TRY(ctx, cudaMemcpy(prm.data(), ctx->params.p,
                             sizeof(ImgParam) * (size_t)n_img,
                             cudaMemcpyDeviceToHost));
    // what the single-value walks of P and P^T run (Section 3.3.1): the
    // device hint, gated as the host gates the launches (option bits, the
    // host estimates, the plane walk's buffer-size bound)
    const bool fits = plane_supported(&ctx->cached_cube, 4);
    const bool adj_on = fits && (ctx->plane_sync & 1) && ctx->plane_possible;
    const bool all = (ctx->plane_sync & 2) != 0;
    const bool fwd_on = fits && (ctx->plane_sync & (2 | 4)) &&
                        (all || ctx->fwd_plane_possible);
    for (int32_t i = 0; i < n_img; ++i) {
        const int32_t h = prm[i].pad;
        const bool valid = (h & kPlaneHintValid) != 0;
        const bool fwd = valid && fwd_on && (all || (h & kPlaneFwdBit));
        codes_host[i] = ((valid && adj_on) ? 1 : 0) | (fwd ? 2 : 0) |
                        ((h & kPlaneGeneralBit) ? 4 : 0) | ((h & 3) << 3) |
                        (((h >> 2) & 3) << 5);
    }
    return TOMO_OK;
}

tomo_status tomo_clear_cache(tomo_ctx *ctx)
{
    if (!ctx) return TOMO_ERR_ARG;
    ctx->key_valid = false;
    return TOMO_OK;
}

tomo_status tomo_profile_read(tomo_ctx *ctx, tomo_profile *out, int32_t reset)
{
    if (!ctx) return TOMO_ERR_ARG;
    DeviceGuard guard(ctx->device);
    tomo_status st = TOMO_OK;
    for (size_t i = 0; i < ctx->ev_pending_slot.size(); ++i) {
        const int slot = ctx->ev_pending_slot[i];
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(ctx->ev_stop[slot]);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, ctx->ev_start[slot], ctx->ev_stop[slot]);
        if (e != cudaSuccess && st == TOMO_OK)
            st = fail(ctx, TOMO_ERR_CUDA, "profile events: %s",
                      cudaGetErrorString(e));
        ctx->ms[ctx->ev_pending_kind[i]] += ms;
        ctx->ev_free.push_back(slot);
    }
    ctx->ev_pending_slot.clear();
    ctx->ev_pending_kind.clear();
    if (out) {
        for (int k = 0; k < TOMO_K_COUNT; ++k) {
            out->launches[k] = ctx->launches[k];
            out->ms[k] = ctx->ms[k];
        }
    }
    if (reset) {
        for (int k = 0; k < TOMO_K_COUNT; ++k) {
            ctx->launches[k] = 0;
            ctx->ms[k] = 0.0;
        }
    }
    return st;
}

tomo_status tomo_project(tomo_ctx *ctx, const tomo_cube_geom *cube,
                         int32_t n_frames, const void *cube_dev,
                         tomo_dtype dtype, const tomo_image_geom *img,
                         const tomo_pointing *pointing_host,
                         const uint8_t *mask_dev, const uint8_t *map_mask_dev,
                         float *images_dev, void *stream)
{
    if (!ctx) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    tomo_status st = common_checks(ctx, cube, n_frames, img, pointing_host);
    if (st) return st;
    if (dtype != TOMO_F32 && dtype != TOMO_BF16)
        return fail(ctx, TOMO_ERR_ARG, "unknown dtype %d", (int)dtype);
    if (img->n_img == 0) return TOMO_OK;
    if (!cube_dev || !images_dev)
        return fail(ctx, TOMO_ERR_ARG, "cube_dev / images_dev is NULL");
    if (!aligned(cube_dev, dtype == TOMO_F32 ? 4 : 2) || !aligned(images_dev, 4))
        return fail(ctx, TOMO_ERR_ARG, "misaligned cube_dev / images_dev");
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    cudaStream_t s = (cudaStream_t)stream;
    const Tiling tl = tiling_for(ctx, cube, img);
    if ((st = ensure_plane(ctx, cube, n_frames, tl)) ||
        (st = prepare_rays(ctx, cube, n_frames, img, pointing_host, s)))
        return st;
    if (img->kind != TOMO_KIND_EMISSION) {
        // the Thomson prologue applies the map mask with M or M'
        if ((st = ensure_thomson(ctx, cube, img->limb_u, s))) return st;
        return op_forward(ctx, cube_dev, dtype, n_frames, mask_dev,
                          map_mask_dev, images_dev, cube, img, tl, nullptr, s);
    }
    if (map_mask_dev) {
        // P K x: the walks read a copy with the excluded voxels at 0
        const int64_t nvox = (int64_t)cube->nx * cube->ny * cube->nz;
        const size_t esz = dtype == TOMO_F32 ? 4 : 2;
        if ((st = ensure(ctx, ctx->mcube, esz * nvox * n_frames))) return st;
        LAUNCH(ctx, TOMO_K_VECTOR, s,
               launch_map_keep_copy(cube_dev, ctx->mcube.p, dtype == TOMO_BF16,
                                    map_mask_dev, nvox, n_frames, s));
        cube_dev = ctx->mcube.p;
    }
    return forward_one(ctx, cube_dev, dtype, n_frames, mask_dev, images_dev,
                       cube, img, tl, nullptr, s);
}

tomo_status tomo_backproject(tomo_ctx *ctx, const tomo_cube_geom *cube,
                             int32_t n_frames, const tomo_image_geom *img,
                             const tomo_pointing *pointing_host,
                             const uint8_t *mask_dev,
                             const uint8_t *map_mask_dev,
                             const float *images_dev, float *cube_dev,
                             uint32_t flags, void *stream)
{
    if (!ctx) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    tomo_status st = common_checks(ctx, cube, n_frames, img, pointing_host);
    if (st) return st;
    if (flags & ~TOMO_ACCUMULATE)
        return fail(ctx, TOMO_ERR_ARG, "unknown flags 0x%x", flags);
    if (!cube_dev) return fail(ctx, TOMO_ERR_ARG, "cube_dev is NULL");
    if (!aligned(cube_dev, 4))
        return fail(ctx, TOMO_ERR_ARG, "misaligned cube_dev");
    if (img->n_img > 0 && (!images_dev || !aligned(images_dev, 4)))
        return fail(ctx, TOMO_ERR_ARG, "images_dev NULL or misaligned");
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t fstride = (int64_t)cube->nx * cube->ny * cube->nz;
    if (!(flags & TOMO_ACCUMULATE))
        CUDA_TRY(ctx, cudaMemsetAsync(cube_dev, 0,
                                      sizeof(float) * fstride * n_frames, s));
    if (img->n_img == 0) return TOMO_OK;
    const Tiling tl = tiling_for(ctx, cube, img);
    if ((st = ensure_plane(ctx, cube, n_frames, tl)) ||
        (st = prepare_rays(ctx, cube, n_frames, img, pointing_host, s)))
        return st;
    if (img->kind != TOMO_KIND_EMISSION) {
        // dst += K T^T y: the Thomson epilogue skips the excluded voxels
        if ((st = ensure_thomson(ctx, cube, img->limb_u, s))) return st;
        return op_adjoint(ctx, images_dev, mask_dev, map_mask_dev, cube_dev,
                          cube, n_frames, img, tl, nullptr, s);
    }
    if (map_mask_dev && (flags & TOMO_ACCUMULATE)) {
        // cube += K P^T y: transpose into scratch, add the kept voxels
        const size_t bytes = sizeof(float) * fstride * n_frames;
        if ((st = ensure(ctx, ctx->mcube, bytes))) return st;
        float *tmp = (float *)ctx->mcube.p;
        CUDA_TRY(ctx, cudaMemsetAsync(tmp, 0, bytes, s));
        if ((st = adjoint_one(ctx, images_dev, mask_dev, tmp, cube, n_frames,
                              img, tl, nullptr, s)))
            return st;
        LAUNCH(ctx, TOMO_K_VECTOR, s,
               launch_map_keep_add(cube_dev, tmp, map_mask_dev, fstride,
                                   n_frames, s));
        return TOMO_OK;
    }
    if ((st = adjoint_one(ctx, images_dev, mask_dev, cube_dev, cube, n_frames,
                          img, tl, nullptr, s)))
        return st;
    if (map_mask_dev)  // cube = K P^T y
        LAUNCH(ctx, TOMO_K_VECTOR, s,
               launch_map_zero(cube_dev, map_mask_dev, fstride, n_frames, s));
    return TOMO_OK;
}

tomo_status tomo_prior_apply(tomo_ctx *ctx, const tomo_cube_geom *cube,
                             const float *x_dev,
                             const float *prior_weight_dev, float *q_dev,
                             double lambda, uint32_t flags, void *stream)
{
    if (!ctx) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    tomo_status st = check_cube(ctx, cube, 1);
    if (st) return st;
    if (flags & ~TOMO_ACCUMULATE)
        return fail(ctx, TOMO_ERR_ARG, "unknown flags 0x%x", flags);
    if (!x_dev || !q_dev || !aligned(x_dev, 4) || !aligned(q_dev, 4))
        return fail(ctx, TOMO_ERR_ARG, "x_dev / q_dev NULL or misaligned");
    if (!aligned(prior_weight_dev, 4))
        return fail(ctx, TOMO_ERR_ARG, "misaligned prior_weight_dev");
    if (!isfinite(lambda) || lambda < 0)
        return fail(ctx, TOMO_ERR_ARG, "lambda must be finite and >= 0");
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    cudaStream_t s = (cudaStream_t)stream;
    LAUNCH(ctx, TOMO_K_PRIOR, s,
           launch_prior(cube_dev(cube), x_dev, prior_weight_dev, q_dev,
                        (float)lambda,
                        (flags & TOMO_ACCUMULATE) != 0, nullptr, s));
    return TOMO_OK;
}

tomo_status tomo_count_segments(tomo_ctx *ctx, const tomo_cube_geom *cube,
                                const tomo_image_geom *img,
                                const tomo_pointing *pointing_host,
                                const uint8_t *mask_dev, int64_t *count_host,
                                void *stream)
{
    if (!ctx) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    tomo_status st = common_checks(ctx, cube, 1, img, pointing_host);
    if (st) return st;
    if (!count_host) return fail(ctx, TOMO_ERR_ARG, "count_host is NULL");
    *count_host = 0;
    if (img->n_img == 0) return TOMO_OK;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = prepare_rays(ctx, cube, 1, img, pointing_host, s))) return st;
    if ((st = ensure(ctx, ctx->count64, sizeof(unsigned long long)))) return st;
    CUDA_TRY(ctx, cudaMemsetAsync(ctx->count64.p, 0, sizeof(unsigned long long), s));
    LAUNCH(ctx, TOMO_K_FORWARD, s, launch_count((const RayRec *)ctx->rays.p, mask_dev, img->n_img,
                               img->nu, img->nv, tiling_for(ctx, cube, img),
                               (unsigned long long *)ctx->count64.p, s));
    unsigned long long n = 0;
    CUDA_TRY(ctx, cudaMemcpyAsync(&n, ctx->count64.p, sizeof(n),
                                  cudaMemcpyDeviceToHost, s));
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    *count_host = (int64_t)n;
    return TOMO_OK;
}

tomo_status tomo_solve(tomo_ctx *ctx, const tomo_cube_geom *cube,
                       int32_t n_frames, const tomo_image_geom *img,
                       const tomo_pointing *pointing_host,
                       const uint8_t *mask_dev, const uint8_t *map_mask_dev,
                       const float *prior_weight_dev, const float *y_dev,
                       float *x_dev, double lambda, double lambda_t,
                       int32_t max_iter, double tol, uint32_t flags,
                       double *report_host, int32_t *iters_host, void *stream)
{
    if (!ctx) return TOMO_ERR_ARG;
    ctx->err[0] = 0;
    tomo_status st = common_checks(ctx, cube, n_frames, img, pointing_host);
    if (st) return st;
    if (!isfinite(lambda_t) || lambda_t < 0)
        return fail(ctx, TOMO_ERR_ARG, "lambda_t must be finite and >= 0");

    if (flags & ~(TOMO_SOLVE_X0 | TOMO_SOLVE_BF16))
        return fail(ctx, TOMO_ERR_ARG, "unknown flags 0x%x", flags);
    if (!isfinite(lambda) || lambda < 0)
        return fail(ctx, TOMO_ERR_ARG, "lambda must be finite and >= 0");
    if (max_iter < 0 || max_iter > 1000000)
        return fail(ctx, TOMO_ERR_ARG, "max_iter must be in [0, 1e6]");
    if (!isfinite(tol) || tol < 0)
        return fail(ctx, TOMO_ERR_ARG, "tol must be finite and >= 0");
    if (!x_dev || !aligned(x_dev, 4))
        return fail(ctx, TOMO_ERR_ARG, "x_dev NULL or misaligned");
    if (!aligned(prior_weight_dev, 4))
        return fail(ctx, TOMO_ERR_ARG, "misaligned prior_weight_dev");
    if (img->n_img > 0 && (!y_dev || !aligned(y_dev, 4)))
        return fail(ctx, TOMO_ERR_ARG, "y_dev NULL or misaligned");
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, TOMO_ERR_CUDA, "cannot select device");
    cudaStream_t s = (cudaStream_t)stream;

    // all frames' voxels are one CG vector
    const int64_t nvox = (int64_t)cube->nx * cube->ny * cube->nz;
    const int64_t n = nvox * n_frames;
    const int64_t m = (int64_t)img->n_img * img->nu * img->nv;
    const bool bf16 = (flags & TOMO_SOLVE_BF16) != 0;
    const size_t n_report = 2 * ((size_t)max_iter + 1);
    if ((st = ensure(ctx, ctx->b, sizeof(float) * n)) ||
        (st = ensure(ctx, ctx->r, sizeof(float) * n)) ||
        (st = ensure(ctx, ctx->p, sizeof(float) * n)) ||
        (st = ensure(ctx, ctx->q, sizeof(float) * n)) ||
        (st = ensure(ctx, ctx->t, sizeof(float) * (m > 0 ? m : 1))) ||
        (bf16 && (st = ensure(ctx, ctx->p16, sizeof(uint16_t) * n))) ||
        (st = ensure(ctx, ctx->S, sizeof(double) * (S_NSLOTS + n_report))) ||
        (st = ensure(ctx, ctx->partials, sizeof(double) * 2 * kMaxReduceBlocks)) ||
        (st = ensure(ctx, ctx->counter, sizeof(unsigned int))))
        return st;
    const Tiling tl = tiling_for(ctx, cube, img);
    if (img->n_img > 0 &&
        ((st = ensure_plane(ctx, cube, n_frames, tl)) ||
         (st = prepare_rays(ctx, cube, n_frames, img, pointing_host, s)) ||
         (img->kind != TOMO_KIND_EMISSION &&
          (st = ensure_thomson(ctx, cube, img->limb_u, s)))))
        return st;

    float *b = (float *)ctx->b.p, *r = (float *)ctx->r.p;
    float *p = (float *)ctx->p.p, *q = (float *)ctx->q.p;
    float *t = (float *)ctx->t.p;
    uint16_t *p16 = bf16 ? (uint16_t *)ctx->p16.p : nullptr;
    double *S = (double *)ctx->S.p;
    double *report = S + S_NSLOTS;
    double *partials = (double *)ctx->partials.p;
    unsigned int *counter = (unsigned int *)ctx->counter.p;
    const double *done = S + S_DONE;
    const RayRec *rays = (const RayRec *)ctx->rays.p;
    const ImgParam *prm = (const ImgParam *)ctx->params.p;
    const Frame *frames = (const Frame *)ctx->frames.p;
    const tomo_pointing *ptgd = (const tomo_pointing *)ctx->ptg.p;
    const CubeDev cd = cube_dev(cube);
    const int nxny = cube->nx * cube->ny;
    const float lam = (float)lambda, lam_t = (float)lambda_t;
    const int grid = reduce_grid(ctx, n > m ? n : m);

    CUDA_TRY(ctx, cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
    CUDA_TRY(ctx, cudaMemsetAsync(S, 0, sizeof(double) * S_NSLOTS, s));
    LAUNCH(ctx, TOMO_K_VECTOR, s, launch_fill_f64(report, NAN, (int64_t)n_report, s));
    // y^T M y and b = P^T M y
    if (m > 0) {
        LAUNCH(ctx, TOMO_K_VECTOR, s, launch_masked_sumsq(y_dev, mask_dev, m, partials, counter,
                                          S, grid, s));
    }
    CUDA_TRY(ctx, cudaMemsetAsync(b, 0, sizeof(float) * n, s));
    if (m > 0 &&
        (st = op_adjoint(ctx, y_dev, mask_dev, nullptr, b, cube, n_frames, img,
                         tl, nullptr, s)))
        return st;
    // with a map mask, b, r and p are restricted by the init and update
    // kernels, and x0 here, so every iterate has 0 on the excluded voxels
    // and the forward walks of p need no masked copy
    const uint8_t *mm = map_mask_dev;
    if (flags & TOMO_SOLVE_X0) {
        // r0 = b - (P^T M P + lambda D^T D) x0
        if (mm)
            LAUNCH(ctx, TOMO_K_VECTOR, s, launch_map_zero(x_dev, mm, nvox, n_frames, s));
        if ((st = apply_prior(ctx, cube, x_dev, prior_weight_dev, q, lam, lam_t,
                              n_frames, nullptr, s)))
            return st;
        if (m > 0 &&
            ((st = op_forward(ctx, x_dev, TOMO_F32, n_frames, mask_dev, nullptr,
                              t, cube, img, tl, nullptr, s)) ||
             (st = op_adjoint(ctx, t, mask_dev, nullptr, q, cube, n_frames, img,
                              tl, nullptr, s))))
            return st;
        LAUNCH(ctx, TOMO_K_VECTOR, s, launch_cg_init(b, q, x_dev, r, p, p16, mm, nvox, n, tol * tol,
                                     partials, counter, S, report, grid, s));
    } else {
        CUDA_TRY(ctx, cudaMemsetAsync(x_dev, 0, sizeof(float) * n, s));
        LAUNCH(ctx, TOMO_K_VECTOR, s, launch_cg_init(b, nullptr, nullptr, r, p, p16, mm, nvox, n,
                                     tol * tol, partials, counter, S, report,
                                     grid, s));
    }
    const void *p_gather = bf16 ? (const void *)p16 : (const void *)p;
    const tomo_dtype p_dtype = bf16 ? TOMO_BF16 : TOMO_F32;
    for (int32_t k = 0; k < max_iter; ++k) {
        // q = (P^T M P + lambda D^T D) p
        if (m > 0 &&
            (st = op_forward(ctx, p_gather, p_dtype, n_frames, mask_dev, nullptr,
                             t, cube, img, tl, done, s)))
            return st;
        if ((st = apply_prior(ctx, cube, p, prior_weight_dev, q, lam, lam_t,
                              n_frames, done, s)))
            return st;
        if (m > 0 &&
            (st = op_adjoint(ctx, t, mask_dev, nullptr, q, cube, n_frames, img,
                             tl, done, s)))
            return st;
        LAUNCH(ctx, TOMO_K_VECTOR, s, launch_cg_pq(p, q, n, partials, counter, S, grid, s));
        LAUNCH(ctx, TOMO_K_VECTOR, s, launch_cg_update(x_dev, r, p, q, b, mm, nvox, n, partials, counter,
                                       S, report, grid, s));
        LAUNCH(ctx, TOMO_K_VECTOR, s, launch_cg_direction(r, p, p16, n, S, grid, s));
    }
    if (report_host || iters_host) {
        double host_S[S_NSLOTS];
        CUDA_TRY(ctx, cudaMemcpyAsync(host_S, S, sizeof(host_S),
                                      cudaMemcpyDeviceToHost, s));
        if (report_host)
            CUDA_TRY(ctx, cudaMemcpyAsync(report_host, report,
                                          sizeof(double) * n_report,
                                          cudaMemcpyDeviceToHost, s));
        CUDA_TRY(ctx, cudaStreamSynchronize(s));
        if (iters_host) *iters_host = (int32_t)host_S[S_ITERS];
        if (host_S[S_ERR] != 0.0)
            return fail(ctx, TOMO_ERR_NUMERIC,
                        "CG breakdown after %d iterations (p.q = %g)",
                        (int)host_S[S_ITERS], host_S[S_PQ]);
    }
    return TOMO_OK;
}

}  // extern "C"
