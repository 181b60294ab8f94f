// Plane-synchronous Siddon walk: P and P^T with the 32 rays of a warp
// crossing the cube one plane of the image's major axis at a time, on a copy
// of the cube stored with the image's lateral axis fastest.
//
// The operator is the one of siddon.cu (Section 3.3.1, Eq. lo: pixel k
// receives g sum_j P_{k,j} x_j, P_{k,j} the length of its line of sight in
// voxel j; P^T spreads g y_k back with the same lengths).  Only the order in
// which the lanes of a warp visit their segments differs.
//
// Why: in the per-ray walk the lanes of a warp advance one segment per
// iteration.  Neighbouring rays cross the planes of the two minor axes at
// different iterations, so after a few voxels they sit at different depths
// along the line of sight and their voxels fall in different 32-byte
// sectors.  L2 float reductions are processed per sector (a warp reducing
// into eight consecutive floats per sector runs about six times faster on
// GB300 than one reducing into scattered floats), and L1 serves gathers one
// sector per wavefront, so both directions of the projector pay per sector.
//
// Here the lanes of a warp hold one row of pixels of one image.  The warp
// walks all its rays through the same plane of the image's major axis M (the
// axis along which the central line of sight advances fastest) in the same
// iteration: iteration i handles, for every lane, the slab between the
// (i-1)-th and i-th M planes counted from the warp's first plane.  Inside a
// slab a ray whose M component is strictly the largest crosses each minor
// axis at most once, so a slab holds one to three segments, handled
// branch-free.  At a fixed M plane, neighbouring pixels of a row sit at
// neighbouring voxels along one lateral axis L; with the cube copied so that
// L is the fastest axis, the 32 segments of a warp iteration fall in two or
// three sectors.
//
// Exactness: every crossing parameter is computed as in the per-ray walk,
// fmaf(k, |dt_a|, t0_a), and ends at the chord the setup kernel capped to
// the last in-cube plane of every axis; each segment is the difference of
// two consecutive crossings, so segment lengths equal the per-ray walk's.
// Only a zero-length segment at an exact tie may be charged to an adjacent
// voxel, which changes no sum.  Rays that do not fit the scheme take the
// per-ray walk on the native layout: rays of an image without a plane hint,
// rays whose M direction differs from the image's, and rays for which a
// minor axis is as steep as M within rounding (two of its crossings could
// then fall in one slab).
//
// Cube layouts (index of voxel (x, y, z); n? = voxel counts):
//   0  x fastest (native):  x + nx (y + ny z)
//   1  y fastest:           y + ny (x + nx z)
//   2  z fastest:           z + nz (x + nx y)
#include "plane.cuh"

namespace tomo {

namespace {

// Slabs per iteration of the middle range (plane_walk) and resident CTAs per
// SM the register allocation targets, measured on GB300 (256^3 cube, 240
// views of 512^2; 512^3 cube, 360 views of 1024^2): the static forward keeps
// the loads of six slabs in flight (7.49 / 114.8 ms; four slabs 7.72 /
// 129.9, seven 7.60 / 129.0, eight 7.53 / 124.1, twelve 7.44 / 122.7, all at
// four CTAs; three slabs 7.78, five 8.09, two at five CTAs 10.5 on the 256^3
// cube); the transpose, bound by the rate at which an SM sends reduction
// sectors to L2, walks one slab per iteration at six CTAs (9.19 ms; five
// CTAs 9.31, two slabs per iteration 9.52).
constexpr int kFwdUnroll = 6;
// bf16 cubes: eight slabs (7.97 / 109.4 ms against 8.11 / 112.0 at six; the
// predicated slot bodies 9.01 / 125.0)
constexpr int kFwdBf16Unroll = 8;
constexpr int kFwdTimeUnroll = 1;
constexpr int kFwdMinBlocks = 4;
constexpr int kAdjUnroll = 1;
constexpr int kAdjMinBlocks = 6;
constexpr int kAdjTimeMinBlocks = 5;

template <typename CubeT, bool kTime>
__global__ void __launch_bounds__(256, kFwdMinBlocks)
k_forward_plane(const RayRec *__restrict__ rays,
                const ImgParam *__restrict__ prm, PlaneCubes cubes,
                int64_t frame_stride, const uint8_t *__restrict__ mask,
                float *__restrict__ out, int nu, int nv, int nx, int ny,
                int nz, Tiling tl, const double *__restrict__ done,
                bool only_marked, int n_img, int group)
{
    if (done != nullptr && *done != 0.0) return;
    int img, tile_v;
    if (!plane_cta(n_img, group, img, tile_v)) return;
    const ImgParam q = prm[img];
    // the whole CTA covers one image: this return is uniform
    if (only_marked && !(q.pad & kPlaneFwdBit)) return;
    int iu, iv;
    const bool in_img = pixel_of_thread(tl, blockIdx.x, tile_v, nu, nv, iu, iv);
    const int64_t id = ((int64_t)img * nv + iv) * nu + iu;
    RayRec r;
    r.chord = -1.0f;
    if (in_img && (mask == nullptr || mask[id] == 0)) r = load_ray(rays + id);
    const bool live = r.chord > 0.0f;
    PlaneRay p;
    const bool regular = live && plane_ray(r, q.pad, nx, ny, nz, p, sizeof(CubeT));
    const int L = (q.pad >> 2) & 3;
    const CubeT *native = static_cast<const CubeT *>(cubes.c[0]);
    const CubeT *lay = static_cast<const CubeT *>(
        L == 1 ? cubes.c[1] : (L == 2 ? cubes.c[2] : cubes.c[0]));
    const int64_t f0 = kTime ? (int64_t)img_frame(q) * frame_stride : 0;
    float acc = 0.0f;
    if (kTime) {
        PlaneGatherTimeOp<CubeT> op;
        op.c0 = lay + f0;
        op.c1 = op.c0 + frame_stride;
        op.w0 = q.w0;
        op.w1 = q.w;
        op.acc = 0.0f;
        plane_walk_for<kFwdTimeUnroll>(q.pad, p, regular, op);
        acc = op.acc;
        if (live && !regular) {
            GatherTimeOp<CubeT> op2;
            op2.c0 = native + f0;
            op2.c1 = op2.c0 + frame_stride;
            op2.w0 = op.w0;
            op2.w1 = op.w1;
            op2.acc = 0.0f;
            siddon_gather(r, nx, nx * ny, op2);
            acc = op2.acc;
        }
    } else {
        PlaneGatherOp<CubeT> op;
        op.c = lay;
        op.acc = 0.0f;
        constexpr int kU = sizeof(CubeT) == 2 ? kFwdBf16Unroll : kFwdUnroll;
        plane_walk_for<kU>(q.pad, p, regular, op);
        acc = op.acc;
        if (live && !regular) {
            GatherOp<CubeT> op2;
            op2.c = native;
            op2.acc = 0.0f;
            siddon_gather(r, nx, nx * ny, op2);
            acc = op2.acc;
        }
    }
    if (in_img) out[id] = q.gain * acc;
}

template <bool kTime>
__global__ void __launch_bounds__(256, kTime ? kAdjTimeMinBlocks : kAdjMinBlocks)
k_adjoint_plane(const RayRec *__restrict__ rays,
                const ImgParam *__restrict__ prm,
                const float *__restrict__ images,
                const uint8_t *__restrict__ mask, PlaneAcc acc,
                int64_t frame_stride, int nu, int nv, int nx, int ny, int nz,
                Tiling tl, const double *__restrict__ done, int n_img,
                int group)
{
    if (done != nullptr && *done != 0.0) return;
    int img, tile_v;
    if (!plane_cta(n_img, group, img, tile_v)) return;
    int iu, iv;
    const bool in_img = pixel_of_thread(tl, blockIdx.x, tile_v, nu, nv, iu, iv);
    const int64_t id = ((int64_t)img * nv + iv) * nu + iu;
    const ImgParam q = prm[img];
    RayRec r;
    r.chord = -1.0f;
    float yv = 0.0f;
    if (in_img && (mask == nullptr || mask[id] == 0)) {
        yv = q.gain * images[id];
        if (yv != 0.0f) r = load_ray(rays + id);
    }
    const bool live = r.chord > 0.0f;
    PlaneRay p;
    const bool regular = live && plane_ray(r, q.pad, nx, ny, nz, p, sizeof(float));
    const int L = (q.pad >> 2) & 3;
    float *lay = L == 1 ? acc.c[1] : (L == 2 ? acc.c[2] : acc.c[0]);
    const int64_t f0 = kTime ? (int64_t)img_frame(q) * frame_stride : 0;
    if (kTime) {
        PlaneScatterTimeOp op;
        op.c0 = lay + f0;
        op.c1 = op.c0 + frame_stride;
        op.y0 = yv * q.w0;
        op.y1 = yv * q.w;
        plane_walk_for<kAdjUnroll>(q.pad, p, regular, op);
        if (live && !regular) {
            ScatterTimeOp op2;
            op2.c0 = acc.c[0] + f0;
            op2.c1 = op2.c0 + frame_stride;
            op2.y0 = op.y0;
            op2.y1 = op.y1;
            siddon_walk(r, nx, nx * ny, op2);
        }
    } else {
        PlaneScatterOp op;
        op.c = lay;
        op.y = yv;
        plane_walk_for<kAdjUnroll>(q.pad, p, regular, op);
        if (live && !regular) {
            ScatterOp op2;
            op2.c = acc.c[0];
            op2.y = yv;
            siddon_walk(r, nx, nx * ny, op2);
        }
    }
}

// Layout copies.  Layout L (1 or 2) makes axis b (y or z) the fastest; c is
// the remaining axis (z or y).  Native index: x + sb b + sc c; layout index:
// b + nb (x + nx c).  One CTA moves a 32 x 32 (x, b) tile through shared
// memory so that both the native reads (along x) and the layout writes
// (along b) are coalesced.
struct LayoutMap {
    int nx, nb, nc;
    int64_t sb, sc;
};

LayoutMap layout_map(int L, int nx, int ny, int nz)
{
    LayoutMap m;
    m.nx = nx;
    if (L == 1) {
        m.nb = ny;
        m.nc = nz;
        m.sb = nx;
        m.sc = (int64_t)nx * ny;
    } else {
        m.nb = nz;
        m.nc = ny;
        m.sb = (int64_t)nx * ny;
        m.sc = nx;
    }
    return m;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_to_layout(const T *__restrict__ in, T *__restrict__ out, LayoutMap m,
            int n_frames, int64_t fstride, const unsigned *__restrict__ used,
            unsigned bit, const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    __shared__ T tile[32][33];
    const int x0 = blockIdx.x * 32, b0 = blockIdx.y * 32, c = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int f = 0; f < n_frames; ++f) {
        const T *src = in + f * fstride;
        T *dst = out + f * fstride;
        for (int k = ty; k < 32; k += 8) {
            const int b = b0 + k, x = x0 + tx;
            if (b < m.nb && x < m.nx) tile[k][tx] = src[x + m.sb * b + m.sc * c];
        }
        __syncthreads();
        for (int k = ty; k < 32; k += 8) {
            const int x = x0 + k, b = b0 + tx;
            if (b < m.nb && x < m.nx)
                dst[b + (int64_t)m.nb * (x + (int64_t)m.nx * c)] = tile[tx][k];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
k_add_from_layout(const float *__restrict__ acc, float *__restrict__ out,
                  LayoutMap m, int n_frames, int64_t fstride,
                  const unsigned *__restrict__ used, unsigned bit,
                  const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    __shared__ float tile[32][33];
    const int x0 = blockIdx.x * 32, b0 = blockIdx.y * 32, c = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int f = 0; f < n_frames; ++f) {
        const float *src = acc + f * fstride;
        float *dst = out + f * fstride;
        for (int k = ty; k < 32; k += 8) {
            const int x = x0 + k, b = b0 + tx;
            if (b < m.nb && x < m.nx)
                tile[tx][k] = src[b + (int64_t)m.nb * (x + (int64_t)m.nx * c)];
        }
        __syncthreads();
        for (int k = ty; k < 32; k += 8) {
            const int b = b0 + k, x = x0 + tx;
            if (b < m.nb && x < m.nx) dst[x + m.sb * b + m.sc * c] += tile[k][tx];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
k_zero_layout(float *__restrict__ p, int64_t n, const unsigned *__restrict__ used,
              unsigned bit, const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        p[i] = 0.0f;
}

// 32 x 8 pixels per CTA, one row of 32 pixels per warp
constexpr Tiling kPlaneTiling = { 32, 8, 32 };

dim3 plane_grid(int nu, int nv, int n_img, int group)
{
    const Tiling t = kPlaneTiling;
    const int tiles_v = (nv + t.tile_v - 1) / t.tile_v;
    return dim3((unsigned)((nu + t.tile_u - 1) / t.tile_u),
                (unsigned)(tiles_v * group),
                (unsigned)((n_img + group - 1) / group));
}

dim3 layout_grid(const LayoutMap &m)
{
    return dim3((unsigned)((m.nx + 31) / 32), (unsigned)((m.nb + 31) / 32),
                (unsigned)m.nc);
}

}  // namespace

int plane_group_clamp(int group, int n_img, int tiles_v)
{
    // the grid's y extent (tile rows x group) stays within 65535
    const int cap = tiles_v > 0 ? 65535 / tiles_v : 1;
    if (group > n_img) group = n_img;
    if (group > cap) group = cap;
    return group < 1 ? 1 : group;
}

bool plane_supported(const tomo_cube_geom *c, int esize)
{
    // layout copies index (x, b) tiles with a grid of at most 65535 in y and
    // z; the walk addresses one buffer of esize-byte voxels with 32-bit byte
    // offsets
    const uint64_t bytes = (uint64_t)c->nx * c->ny * c->nz * (uint64_t)esize;
    return c->nx <= kPlaneMaxSide && c->ny <= kPlaneMaxSide &&
           c->nz <= kPlaneMaxSide && bytes <= (1ull << 32);
}

cudaError_t launch_to_layout(const void *cube, tomo_dtype dtype, void *out,
                             int L, const tomo_cube_geom *c, int32_t n_frames,
                             const unsigned *used, unsigned bit,
                             const double *done, cudaStream_t s)
{
    const LayoutMap m = layout_map(L, c->nx, c->ny, c->nz);
    const int64_t fstride = (int64_t)c->nx * c->ny * c->nz;
    if (dtype == TOMO_BF16)
        k_to_layout<uint16_t><<<layout_grid(m), 256, 0, s>>>(
            static_cast<const uint16_t *>(cube), static_cast<uint16_t *>(out),
            m, n_frames, fstride, used, bit, done);
    else
        k_to_layout<float><<<layout_grid(m), 256, 0, s>>>(
            static_cast<const float *>(cube), static_cast<float *>(out), m,
            n_frames, fstride, used, bit, done);
    return cudaGetLastError();
}

cudaError_t launch_add_from_layout(const float *acc, float *cube, int L,
                                   const tomo_cube_geom *c, int32_t n_frames,
                                   const unsigned *used, const double *done,
                                   cudaStream_t s)
{
    const LayoutMap m = layout_map(L, c->nx, c->ny, c->nz);
    const int64_t fstride = (int64_t)c->nx * c->ny * c->nz;
    k_add_from_layout<<<layout_grid(m), 256, 0, s>>>(acc, cube, m, n_frames,
                                                     fstride, used, 1u << L,
                                                     done);
    return cudaGetLastError();
}

cudaError_t launch_zero_layout(float *acc, int L, int64_t n,
                               const unsigned *used, const double *done,
                               int num_sms, cudaStream_t s)
{
    int64_t g = (n + 255) / 256;
    const int64_t cap = 8LL * (num_sms > 0 ? num_sms : 152);
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    k_zero_layout<<<(unsigned)g, 256, 0, s>>>(acc, n, used, 1u << L, done);
    return cudaGetLastError();
}

cudaError_t launch_forward_plane(const RayRec *rays, const ImgParam *prm,
                                 PlaneCubes cubes, tomo_dtype dtype,
                                 int64_t frame_stride, bool time_interp,
                                 const uint8_t *mask, float *out,
                                 int32_t n_img, int32_t nu, int32_t nv,
                                 const tomo_cube_geom *c, const double *done,
                                 cudaStream_t s, bool only_marked, int group)
{
    if (n_img <= 0) return cudaSuccess;
    const Tiling t = kPlaneTiling;
    group = plane_group_clamp(group, n_img, (nv + t.tile_v - 1) / t.tile_v);
    const dim3 grid = plane_grid(nu, nv, n_img, group);
    const int block = t.tile_u * t.tile_v;
    const bool om = only_marked;
    if (dtype == TOMO_BF16) {
        if (time_interp)
            k_forward_plane<uint16_t, true><<<grid, block, 0, s>>>(
                rays, prm, cubes, frame_stride, mask, out, nu, nv, c->nx,
                c->ny, c->nz, t, done, om, n_img, group);
        else
            k_forward_plane<uint16_t, false><<<grid, block, 0, s>>>(
                rays, prm, cubes, frame_stride, mask, out, nu, nv, c->nx,
                c->ny, c->nz, t, done, om, n_img, group);
    } else {
        if (time_interp)
            k_forward_plane<float, true><<<grid, block, 0, s>>>(
                rays, prm, cubes, frame_stride, mask, out, nu, nv, c->nx,
                c->ny, c->nz, t, done, om, n_img, group);
        else
            k_forward_plane<float, false><<<grid, block, 0, s>>>(
                rays, prm, cubes, frame_stride, mask, out, nu, nv, c->nx,
                c->ny, c->nz, t, done, om, n_img, group);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_plane(const RayRec *rays, const ImgParam *prm,
                                 const float *images, const uint8_t *mask,
                                 PlaneAcc acc, int64_t frame_stride,
                                 bool time_interp, int32_t n_img, int32_t nu,
                                 int32_t nv, const tomo_cube_geom *c,
                                 const double *done, cudaStream_t s, int group)
{
    if (n_img <= 0) return cudaSuccess;
    const Tiling t = kPlaneTiling;
    group = plane_group_clamp(group, n_img, (nv + t.tile_v - 1) / t.tile_v);
    const dim3 grid = plane_grid(nu, nv, n_img, group);
    const int block = t.tile_u * t.tile_v;
    if (time_interp)
        k_adjoint_plane<true><<<grid, block, 0, s>>>(
            rays, prm, images, mask, acc, frame_stride, nu, nv, c->nx, c->ny,
            c->nz, t, done, n_img, group);
    else
        k_adjoint_plane<false><<<grid, block, 0, s>>>(
            rays, prm, images, mask, acc, frame_stride, nu, nv, c->nx, c->ny,
            c->nz, t, done, n_img, group);
    return cudaGetLastError();
}

}  // namespace tomo
