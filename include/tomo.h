/*
 * tomo.h — C ABI of the GB300 solar-tomography projector library (libtomo).
 *
 * The library implements the line-of-sight projector P of TomograPy
 * (Barbey, Guennou & Auchere; Section 3.3.1, Eq. lo), its exact transpose
 * P^T, and a conjugate-gradient inversion of the regularised least-squares
 * criterion built on them (Section 2.2, Eq. criterion), on one NVIDIA GB300
 * (sm_103a).  Every step runs in the library's own CUDA kernels.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Cube: identical rectangular voxels (Section 3.3.1: required by Siddon),
 *    laid out [nz][ny][nx] with x fastest; with n_frames = T > 1 the frames
 *    are stacked as [T][nz][ny][nx].
 *  - Images: [n_img][nv][nu] float32, u fastest; one pointing record per image.
 *  - Pointing (Section 3.2, WCS keywords): Sun-centred frame, z = solar
 *    rotation axis, x at longitude 0; observer o = d (cos lat cos lon,
 *    cos lat sin lon, sin lat); boresight w = -o/|o|; e1 = unit(w x z),
 *    e2 = e1 x w, both turned by `roll` about w; gnomonic (TAN) pixels:
 *    theta_u = (i_u - crpix_u) cdelt_u + crval_u (likewise v), ray direction
 *    unit(w + tan(theta_u) e1 + tan(theta_v) e2).  Angles in radians,
 *    distances in the cube's length unit.  The paper names the keywords but
 *    not these formulas; this is the library's reading.
 *  - Voxels are half-open, [x0 + i dx, x0 + (i+1) dx): a ray lying exactly on
 *    a face is charged to the voxel above it.
 *  - Masks: uint8 [n_img][nv][nu], nonzero = excluded (Section 4: the
 *    projector skips masked pixels).  P writes 0 there, P^T ignores them.
 *  - Map masks: uint8 [nz][ny][nx], nonzero = voxel excluded from the map
 *    (Section 4 names masks of the data and of the map; the paper gives no
 *    formula).  Reading: an excluded voxel is not an unknown.  P reads it as
 *    0 (P K x, K = diag(1 - map mask)), P^T leaves it 0 (K P^T y), and the
 *    solver works on the system restricted to the other voxels.  With
 *    T > 1 frames the one mask applies to every frame.  Always nullable.
 *  - Gains: each image is scaled by its record's gain (Eq. two_spacecraft,
 *    Eq. lin2space).
 *  - Time (Section 3.3.3, a parameterised temporal evolution): with T > 1
 *    frames an image with time stamp tau in [0, T-1] sees
 *    (1 - w) X[k] + w X[k+1], k = min(floor(tau), T-2), w = tau - k.
 *  - Pointers named *_dev are device pointers, *_host host pointers.  All
 *    buffers belong to the caller; the library keeps no pointer to them
 *    after a call returns.  The library allocates only its own workspace
 *    (ray records, solver vectors), owned by the context.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless stated.
 *  - Errors: every entry point validates its arguments before any launch
 *    and returns a tomo_status; it never aborts.  tomo_last_error() gives a
 *    one-line message.  A context must not be used by two host threads at
 *    once.
 */
#ifndef TOMO_H
#define TOMO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TOMO_OK = 0,
    TOMO_ERR_ARG = -1,         /* invalid argument (pointer, size, geometry) */
    TOMO_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    TOMO_ERR_UNSUPPORTED = -3, /* valid but not supported (e.g. no sm_103a) */
    TOMO_ERR_OOM = -4,         /* workspace allocation failed */
    TOMO_ERR_TIMEOUT = -5,     /* a bounded device wait gave up */
    TOMO_ERR_NUMERIC = -6      /* solver breakdown (non-positive or NaN p.q) */
} tomo_status;

typedef enum {
    TOMO_F32 = 0,  /* float32 cube */
    TOMO_BF16 = 1  /* bfloat16 cube, widened to float32 on load */
} tomo_dtype;

/* Cube geometry: voxel counts, minimum corner (x0, y0, z0) and voxel size
 * (dx, dy, dz > 0).  `reserved` must be 0. */
typedef struct {
    int32_t nx, ny, nz, reserved;
    double x0, y0, z0;
    double dx, dy, dz;
    /* Radius of an opaque sphere centred at the frame origin (the
     * photosphere, in the cube's units), or 0 for none.  Lines of sight end
     * where they first reach it (the paper ends the line-of-sight
     * integration at the photosphere, Section 4); a line of sight from an
     * observer inside the sphere integrates nothing.  Must be finite and
     * >= 0. */
    double r_obs;
} tomo_cube_geom;

/* What the images measure (Section 3.5; tomo_image_geom.kind). */
#define TOMO_KIND_EMISSION 0 /* line-of-sight integral y = P x (EUV, Eq. srt) */
#define TOMO_KIND_PB 1       /* polarised brightness, y = O P M x */
#define TOMO_KIND_B 2        /* total brightness, y = P M' x - O P M x */

/* Image stack geometry: n_img images of nv rows by nu columns, and what
 * they measure.  With kind PB or B the single-problem entry points apply
 * the Thomson operator instead of P (its transpose instead of P^T, in the
 * solver too): O = diag(rho_k^2), rho = impact parameter of the pixel's line
 * of sight; M = diag(m_j), M' = diag(m'_j) at the voxel centre's distance r
 * from Sun centre, with sin(Omega) = 1/r and the coefficients C1..C4 of
 * Eq. 4C:
 *     m_j  = ((1 - u) C1 + u C2) / r^4 ,
 *     m'_j = 2 ((1 - u) C3 + u C4) / r^2      (Eq. brightness),
 * 0 for r <= 1 (inside the photosphere).  Readings: C4 takes +1/8 (the
 * printed -1/8 makes the scattered intensity of a limb-darkened Sun
 * negative), m_j keeps the u on C2 and m'_j the factor 2 of Eq. brightness,
 * and the constant pi sigma I0 / 2 is left to the per-image gains.
 * limb_u: limb-darkening coefficient u in [0, 1] (ignored for EMISSION).
 * The batched and allocation-free entry points accept EMISSION only. */
typedef struct {
    int32_t n_img, nu, nv;
    int32_t kind;
    double limb_u;
} tomo_image_geom;

/* One pointing record (96 bytes; the 12 doubles of one row of a float64
 * (n_img, 12) table, in this order). */
typedef struct {
    double d_obs, lon, lat, roll;
    double cdelt_u, cdelt_v, crpix_u, crpix_v, crval_u, crval_v;
    double gain, time;
} tomo_pointing;

typedef struct tomo_ctx tomo_ctx;

/* Flags */
#define TOMO_ACCUMULATE   1u  /* backproject: add into cube_dev (else overwrite) */
#define TOMO_SOLVE_X0     2u  /* solve: start from x_dev (else from 0) */
#define TOMO_SOLVE_BF16   4u  /* solve: gather the CG direction from a bf16 copy */

/* Options for tomo_set_option */
#define TOMO_OPT_RAY_CACHE  1  /* 1 (default): keep ray records per geometry */
#define TOMO_OPT_TILE_U     2  /* pixel tile width of one CTA (default 32) */
#define TOMO_OPT_TILE_V     3  /* pixel tile height of one CTA (default 8) */
#define TOMO_OPT_WARP_U     4  /* pixel tile width of one warp (default 8) */
#define TOMO_OPT_PROFILE    5  /* 1: time every kernel launch with CUDA events */
/* (option 6 is not used: it chose among transpose kernels that were
 * measured slower and removed) */
#define TOMO_OPT_PLANE_SYNC 7  /* bit mask (default 5) choosing the Siddon
                                  walk of single-problem calls: bit 0 for
                                  P^T; bit 1 for P
                                  on every image; bit 2 for P on the images
                                  where it measured faster: views within
                                  ~1 degree of a cube-axis plane, or pixels
                                  at least 0.75 voxel apart (per ray on the
                                  others).  A set bit
                                  makes the rays of a warp walk the cube one
                                  plane of the image's major axis at a time,
                                  on a copy of the cube stored with the
                                  image's lateral axis fastest, so the voxels
                                  a warp touches at once fall in few 32-byte
                                  sectors; a clear bit makes every lane walk
                                  its own ray one segment per step.  Same
                                  segments either way: P is bit-identical,
                                  P^T differs only by the order of float
                                  additions.  Images whose pixels are less
                                  than 0.16 voxel apart always take the
                                  per-ray walk.  The plane walk uses its own
                                  tiling (32 x 8 pixels per CTA, one image
                                  row per warp) whatever the tile options
                                  say.  Needs cubes of at most 16384 voxels
                                  per side and 2^32 bytes as float32 (it
                                  addresses voxels by 32-bit byte offsets),
                                  else the per-ray walk is used.  Costs two
                                  cube-sized float buffers (times the
                                  frames) of workspace. */
#define TOMO_OPT_CHANNELS   8  /* bit mask (default 3) of the two-value
                                  plane walks: bit 0, time-interpolated P
                                  and P^T walk frame pairs (X[k], X[k+1])
                                  stored side by side (one 8-byte load or
                                  vector reduction per segment instead of
                                  two 4-byte ones a cube apart; P stays
                                  bit-identical); bit 1, the Thomson B
                                  operator of a single frame runs one walk
                                  on (m' x, m x) pairs instead of two walks.
                                  Costs three buffers of 8 bytes per voxel
                                  (times T - 1 frame pairs) of workspace.
                                  Above 2^29 voxels (pair buffers of more
                                  than 2^32 bytes) time interpolation walks
                                  separate frames and the B pairs are walked
                                  per ray. */

#define TOMO_OPT_GROUP_FWD  9  /* CTA order of the plane-synchronous P: 0
                                  (default) chosen from the bytes the walk
                                  gathers from; n >= 1: images are taken in
                                  groups of n, and inside a group the CTAs of
                                  one 8-pixel row band of every image run
                                  before the next band (1: image after
                                  image), so that the CTAs resident at once
                                  read one band of the cube.  Same results
                                  whatever the order (P bit-identical). */
#define TOMO_OPT_GROUP_ADJ  10 /* the same for the plane-synchronous P^T
                                  (results differ only by the order of
                                  float additions) */

/* Kernel classes of tomo_profile */
enum {
    TOMO_K_SETUP = 0,   /* pointing -> ray records (FP64) */
    TOMO_K_FORWARD = 1, /* Siddon gather, P */
    TOMO_K_ADJOINT = 2, /* Siddon scatter, P^T */
    TOMO_K_PRIOR = 3,   /* D^T D stencil */
    TOMO_K_VECTOR = 4,  /* CG vector updates and reductions */
    TOMO_K_LAYOUT = 5,  /* cube layout copies of the plane-synchronous walk */
    TOMO_K_COUNT = 6
};

/* Per kernel class: launches since the last reset and, with
 * TOMO_OPT_PROFILE on, their summed device time in milliseconds (CUDA events
 * recorded on the launching stream around each launch). */
typedef struct {
    int64_t launches[TOMO_K_COUNT];
    double ms[TOMO_K_COUNT];
} tomo_profile;

/* Create a context on CUDA device `device` (made current for the call).
 * Returns TOMO_ERR_UNSUPPORTED if the device is not sm_103. */
tomo_status tomo_create(tomo_ctx **ctx_out, int32_t device);

/* Free the context and its workspace.  NULL is accepted.  The caller makes
 * sure no work of the context is still running. */
void tomo_destroy(tomo_ctx *ctx);

/* Static text of a status code. */
const char *tomo_status_string(tomo_status status);

/* Message of the context's last error ("" if none).  Valid until the next
 * call on the context. */
const char *tomo_last_error(const tomo_ctx *ctx);

/* Set an option (see TOMO_OPT_*).  Tile options must satisfy
 * tile_u * tile_v <= 512, tile_u % warp_u == 0, tile_v % (32 / warp_u) == 0;
 * they are checked at the next launch. */
tomo_status tomo_set_option(tomo_ctx *ctx, int32_t option, int64_t value);

/* Drop the cached ray records (the memory stays with the context). */
tomo_status tomo_clear_cache(tomo_ctx *ctx);

/* Read the launch counts and timings gathered so far (waits for the pending
 * timing events), then zero them if `reset` is nonzero. */
tomo_status tomo_profile_read(tomo_ctx *ctx, tomo_profile *out, int32_t reset);

/* Forward projection y = P x (Eq. lo for one image, stacked over images as in
 * Eq. srt; gains per Eq. lin2space; time interpolation per Section 3.3.3).
 *   cube:          geometry of one frame
 *   n_frames:      T >= 1 frames in cube_dev
 *   cube_dev:      [T][nz][ny][nx] of `dtype` (4- or 2-byte aligned)
 *   img:           image stack geometry
 *   pointing_host: n_img records (copied during the call)
 *   mask_dev:      nullable; nonzero pixels are written as 0
 *   map_mask_dev:  nullable; excluded voxels are read as 0 (the call copies
 *                  the masked cube into context workspace; cube_dev is not
 *                  modified)
 *   images_dev:    [n_img][nv][nu] float32, overwritten
 * Ray records are computed in FP64 by a setup kernel and cached in the
 * context, keyed by (cube, img, pointing) contents. */
tomo_status tomo_project(tomo_ctx *ctx, const tomo_cube_geom *cube,
                         int32_t n_frames, const void *cube_dev,
                         tomo_dtype dtype, const tomo_image_geom *img,
                         const tomo_pointing *pointing_host,
                         const uint8_t *mask_dev, const uint8_t *map_mask_dev,
                         float *images_dev, void *stream);

/* Backprojection x = P^T y: the exact transpose of tomo_project with the
 * same arguments (same segments, lengths, mask, gains and time weights).
 *   images_dev:   [n_img][nv][nu] float32 input
 *   map_mask_dev: nullable; excluded voxels receive 0 (with
 *                 TOMO_ACCUMULATE they keep their value)
 *   cube_dev:     [T][nz][ny][nx] float32 output; overwritten unless
 *                 flags has TOMO_ACCUMULATE
 * Results are accumulated with float32 atomics, so the summation order and
 * the last bits vary from run to run. */
tomo_status tomo_backproject(tomo_ctx *ctx, const tomo_cube_geom *cube,
                             int32_t n_frames, const tomo_image_geom *img,
                             const tomo_pointing *pointing_host,
                             const uint8_t *mask_dev,
                             const uint8_t *map_mask_dev,
                             const float *images_dev, float *cube_dev,
                             uint32_t flags, void *stream);

/* Regularised least squares (Eq. criterion with A = M P, B = D, or
 * B = D R for the height-weighted prior of Eq. srt_inversion):
 *     x = argmin ||M (y - P x)||^2 + lambda ||D R x||^2 ,
 * D = forward differences along x, y, z without wrap (Section 3.3.1: finite
 * differences along each axis of the map), R = diag(prior weight) or
 * the identity, by conjugate gradients on
 * (P^T M P + lambda R D^T D R) x = P^T M y, one static frame, FP32 vectors
 * and FP64 scalars (alpha, beta, residual norms, J).
 *   y_dev:       [n_img][nv][nu] float32 data
 *   map_mask_dev: nullable; restricts the unknowns to the other voxels:
 *                the criterion becomes ||M (y - P K x)||^2 +
 *                lambda ||D K x||^2 and CG runs on K (P^T M P +
 *                lambda D^T D) K x = K P^T M y; the excluded voxels of the
 *                result (and of the initial guess, in place) are 0
 *   prior_weight_dev: nullable; [nz][ny][nx] float32, the diagonal of R
 *                (Eq. srt_inversion puts the voxels' height there; the
 *                caller chooses which height), 4-byte aligned
 *   x_dev:       [nz][ny][nx] float32; initial guess if flags has
 *                TOMO_SOLVE_X0 (else start from 0); receives the result
 *   lambda:      >= 0
 *   max_iter:    >= 0 iterations
 *   tol:         stop once ||r_k|| <= tol ||r_0|| (0 = run max_iter)
 *   flags:       TOMO_SOLVE_X0, TOMO_SOLVE_BF16
 *   report_host: nullable; (max_iter + 1) x 2 doubles: for every iterate k,
 *                J(x_k) (through J = y^T M y - x^T (r + b), b = P^T M y) and
 *                ||r_k||^2.  Rows past the last iteration are NaN.
 *   iters_host:  nullable; receives the number of iterations done
 * No host synchronisation happens inside the loop.  If report_host or
 * iters_host is given, the call synchronises `stream` before returning. */
/* Several frames (n_frames = T > 1; the smooth temporal model of Section
 * 3.3.3, block-diagonal for integer time stamps as in Eq. srt_t / stsrt):
 * x_dev is [T][nz][ny][nx], each image sees its frames through its time
 * stamp, the spatial prior applies to every frame, and lambda_t >= 0 adds
 * lambda_t ||D_t x||^2 with D_t the difference x[t+1] - x[t] of consecutive
 * frames (normal operator + lambda_t D_t^T D_t).  A map mask applies to
 * every frame. */
tomo_status tomo_solve(tomo_ctx *ctx, const tomo_cube_geom *cube,
                       int32_t n_frames, const tomo_image_geom *img,
                       const tomo_pointing *pointing_host,
                       const uint8_t *mask_dev, const uint8_t *map_mask_dev,
                       const float *prior_weight_dev, const float *y_dev,
                       float *x_dev, double lambda, double lambda_t,
                       int32_t max_iter, double tol, uint32_t flags,
                       double *report_host, int32_t *iters_host, void *stream);

/* q = lambda D^T D x (+ q if flags has TOMO_ACCUMULATE), the gradient of the
 * prior term lambda ||D x||^2 / 2 (Section 3.3.1); with prior_weight_dev
 * (nullable, the diagonal of R) q = lambda R D^T D R x, the gradient of
 * lambda ||D R x||^2 / 2 (Eq. srt_inversion).  x, q, weight: [nz][ny][nx]
 * f32. */
tomo_status tomo_prior_apply(tomo_ctx *ctx, const tomo_cube_geom *cube,
                             const float *x_dev,
                             const float *prior_weight_dev, float *q_dev,
                             double lambda, uint32_t flags, void *stream);

/* Number of positive-length voxel intersections (Siddon segments) of the
 * unmasked rays, counted on the device with the projector's own walk. */
tomo_status tomo_count_segments(tomo_ctx *ctx, const tomo_cube_geom *cube,
                                const tomo_image_geom *img,
                                const tomo_pointing *pointing_host,
                                const uint8_t *mask_dev, int64_t *count_host,
                                void *stream);

/* ---------------------------------------------------------------------
 * Batches of independent problems (uneven cube and image sizes).
 *
 * One persistent kernel launch walks the rays of every problem: a grid of
 * (SM count x resident CTAs) CTAs takes (problem, pixel tile) work items from
 * an atomic counter; each problem may use its own tile shape (256 threads),
 * taken from the autotuner's table.  The solver captures its whole run
 * (initial residual and every iteration, for every problem) in one CUDA
 * graph that is replayed while geometries, buffers, lambdas and the
 * iteration count stay the same.
 *
 * Each problem is described by a tomo_problem (all buffers belong to the
 * caller):
 *   cube, img, pointing_host  geometry as for tomo_project (one frame)
 *   mask_dev                  nullable
 *   images_dev                project: output; backproject: input;
 *                             solve: the data y
 *   cube_dev                  project: input; backproject: output;
 *                             solve: the solution (initial guess with
 *                             TOMO_SOLVE_X0)
 *   lambda                    solve: prior weight (>= 0)
 *   reserved                  must be 0
 *   map_mask_dev              nullable; the map mask of the single-problem
 *                             calls (project: excluded voxels read as 0;
 *                             backproject: they receive 0; solve: the
 *                             restricted system)
 *   prior_weight_dev          nullable; solve: the diagonal of R of the
 *                             height-weighted prior, as for tomo_solve
 */
typedef struct {
    tomo_cube_geom cube;
    tomo_image_geom img;
    int32_t reserved;
    const tomo_pointing *pointing_host;
    const uint8_t *mask_dev;
    float *images_dev;
    float *cube_dev;
    double lambda;
    const uint8_t *map_mask_dev;
    const float *prior_weight_dev;
} tomo_problem;

/* Thresholds that choose, per image, which Siddon walk P and P^T run.
 * "pitch": the image's pixel spacing at the distance of Sun centre, in
 * voxels of the axis along which a row of pixels moves; "ratio": the less
 * steep minor direction component of the image's central line of sight
 * over its major component.  Only speed depends on them: every walk gives
 * the same segments (P bit-identical, P^T up to the order of float
 * additions).  Values >= 1e30 stand for "never". */
typedef struct {
    double min_pitch;      /* plane-synchronous walks when pitch >= this,
                              per-ray walks below (default 0.16) */
    double fwd_min_pitch;  /* P plane-synchronous when pitch >= this ... */
    double fwd_max_ratio;  /* ... or ratio < this (defaults 0.75, 0.02; P
                              per ray otherwise) */
    double general_ratio;  /* plane walks cross every slab with the general
                              three-segment body when ratio >= this, else
                              they count the slabs to the next crossing of
                              the rarer minor axis (default 0.035) */
    double fwd_group;      /* images per group of the plane P's CTA order
                              (TOMO_OPT_GROUP_FWD, which overrides it when
                              set); 0 (default): chosen from the bytes the
                              walk gathers from */
    double adj_group;      /* the same for the plane P^T
                              (TOMO_OPT_GROUP_ADJ) */
} tomo_plane_rules;

/* A tile shape, walk rules and measured times (tomo_autotune): the
 * per-ray tile and the rules the problem's size bucket uses, and the time
 * of its P and P^T with them. */
typedef struct {
    int32_t tile_u, tile_v, warp_u;
    float fwd_ms, adj_ms;
    tomo_plane_rules rules;
} tomo_tiling;

#define TOMO_BATCH_AUTOTUNE 8u /* solve_batched: tune unseen problem sizes */

/* Tunes the schedule of one problem's size bucket (cube voxel counts and
 * image size): times the per-ray forward and transpose kernels for a fixed
 * list of 256-thread tile shapes and keeps the fastest; then, with that
 * tile, times P and P^T as the single-problem calls run them under
 * candidate walk rules (tomo_plane_rules: per-ray or plane-synchronous
 * walks by pixel pitch, counted or every-slab plane walks by direction
 * ratio, the plane forward by pitch and ratio, the CTA order of the plane
 * P and P^T), searching one rule at a time and keeping the fastest P + P^T
 * (P alone for the rules that concern only P).  The batched calls use the
 * bucket's walk rules but keep their own work order (the group sizes do
 * not apply to them).  The problem's cube_dev and
 * images_dev are read, not written.  The winners are kept in the context
 * for the bucket and returned in best_out (nullable); later single and
 * batched calls on problems of the same size use them.  Synchronises
 * `stream`. */
tomo_status tomo_autotune(tomo_ctx *ctx, const tomo_problem *prob,
                          tomo_tiling *best_out, void *stream);

/* Sets the walk rules of a size bucket (cube voxel counts and image size,
 * both non-NULL), or the context's default for buckets without their own
 * (cube and img NULL).  rules NULL: the built-in defaults.  Takes effect at
 * the next call on a geometry of that bucket.  A schedule control with no
 * counterpart in the paper: every walk it selects computes the same
 * operator (Section 3.3.1, Eq. lo).  Returns TOMO_ERR_ARG for a negative or
 * NaN threshold, or for only one of cube / img given. */
tomo_status tomo_set_plane_rules(tomo_ctx *ctx, const tomo_cube_geom *cube,
                                 const tomo_image_geom *img,
                                 const tomo_plane_rules *rules);

/* The walk chosen for each image of the most recent single-problem
 * geometry by the single-value P and P^T (a report of the schedule, no
 * counterpart in the paper; synchronises the legacy default stream).  It
 * follows the per-image hints and the context's TOMO_OPT_PLANE_SYNC, and
 * reports per-ray walks for a cube of more than 2^32 bytes, which the plane
 * walk does not address:
 *   bit 0: P^T walks plane by plane (else per ray)
 *   bit 1: P walks plane by plane
 *   bit 2: the plane walks cross every slab with the general body
 *   bits 3-4: the major axis (0 x, 1 y, 2 z); bits 5-6: the lateral axis
 * codes_host: n_img entries; n_img must equal the geometry's image count. */
tomo_status tomo_walk_plan(tomo_ctx *ctx, int32_t n_img, int32_t *codes_host);

/* images = P cube for every problem, in one persistent launch (plus the FP64
 * ray setup of every problem when the set of geometries changes). */
tomo_status tomo_project_batched(tomo_ctx *ctx, int32_t n,
                                 const tomo_problem *probs, void *stream);

/* cube = P^T images for every problem (overwritten unless TOMO_ACCUMULATE),
 * in one persistent launch. */
tomo_status tomo_backproject_batched(tomo_ctx *ctx, int32_t n,
                                     const tomo_problem *probs, uint32_t flags,
                                     void *stream);

/* n_iter CG iterations of tomo_solve for every problem at once (one CUDA
 * graph replay).  flags: TOMO_SOLVE_X0, TOMO_BATCH_AUTOTUNE.
 *   report_host: nullable; n x (n_iter + 1) x 2 doubles (J, r.r per
 *                iterate, as tomo_solve)
 *   iters_host:  nullable; n iteration counts
 * Synchronises `stream` when report_host or iters_host is given. */
tomo_status tomo_solve_batched(tomo_ctx *ctx, int32_t n,
                               const tomo_problem *probs, int32_t n_iter,
                               uint32_t flags, double *report_host,
                               int32_t *iters_host, void *stream);

/* ---------------------------------------------------------------------
 * Forward projection without any device allocation.
 *
 * The paper has no counterpart to this entry point: it exists for callers
 * that cannot let a library allocate device memory.  tomo_project keeps its
 * ray records and per-image tables in workspace that the context allocates
 * with cudaMalloc on first use; some programs cannot accept that: programs
 * that reserve the device memory they may use up front and hand out pieces
 * of it themselves (a framework's caching allocator, a fixed memory budget
 * shared with other jobs), and latency-critical loops in which a cudaMalloc
 * or cudaFree, which can wait for work already queued on the device, would
 * stall other streams.  tomo_project_noalloc computes the same images as
 * tomo_project, bit for bit, with its scratch in a fixed array that is part
 * of the library image.  It always runs the per-ray forward walk; the
 * plane-synchronous walk that tomo_project picks for many images gives the
 * same sums in the same order, but can be faster, so this call may take
 * longer than tomo_project on the same input.
 *
 * Scratch: one array of TOMO_NOALLOC_SCRATCH_BYTES per device, compiled into
 * the library and therefore held by every device on which this entry point
 * has been called, until the process exits.  A call needs, each part
 * rounded up to 256 bytes,
 *     96 n_img + 96 n_img + 16 n_img + 8 n_img nu + 8 n_img nv
 *     + 32 n_img nu nv   bytes
 * (pointing copy, observer frames, image parameters, tangent tables, one
 * 32-byte ray record per pixel); a call that needs more returns
 * TOMO_ERR_UNSUPPORTED before launching anything.
 *
 * Every call uses the same array and leaves its contents behind; each call
 * rewrites all of the scratch it reads, so nothing has to start at zero.
 * Calls whose work overlaps on the GPU (other streams, or other host
 * threads) race on the array: order them on one stream, or wait for one to
 * finish before the next starts.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and remembers it for the
 * rest of the process; make that first call before any stream capture.  A
 * cudaDeviceReset reloads the library's device code at another address, so
 * this entry point must not be called on a device after that device has
 * been reset in the same process.
 *
 * Arguments are those of tomo_project without the context and without the
 * map mask (a masked copy of the cube would need cube-sized scratch; apply
 * the mask to the cube before the call): the current device is used, the stream is a cudaStream_t passed as void* (NULL = the
 * legacy default stream), and the call is asynchronous on it.  The
 * pointing table is copied to the array by a cudaMemcpyAsync queued on the
 * stream: a table in page-locked (pinned) host memory is read only when the
 * stream reaches that copy and must stay unchanged until then; a table in
 * pageable memory may be reused as soon as the call returns.  No
 * cudaMalloc, cudaFree or other allocating routine is called. */
#define TOMO_NOALLOC_SCRATCH_BYTES (16u << 20)

tomo_status tomo_project_noalloc(const tomo_cube_geom *cube, int32_t n_frames,
                                 const void *cube_dev, tomo_dtype dtype,
                                 const tomo_image_geom *img,
                                 const tomo_pointing *pointing_host,
                                 const uint8_t *mask_dev, float *images_dev,
                                 void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TOMO_H */
