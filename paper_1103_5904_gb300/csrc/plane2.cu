// Two-value plane-synchronous walks: every voxel of the walked buffer holds
// two floats side by side, gathered with one 8-byte load and scattered with
// one 8-byte vector reduction per segment.
//
// Time interpolation (Section 3.3.3; image i sees (1 - w) X[k] + w X[k+1],
// k and w from its time stamp): the walks read and write frame pairs
// (X[k], X[k+1]) stored side by side, k = 0 .. T-2, in the image's layout.
// The forward gathers both frames of a voxel with one load and forms
// fmaf(1 - w, X[k], w X[k+1]) as the separate-frame walk does, so its images
// are bit-identical to it; the transpose adds (len (1 - w) g y, len w g y)
// into the pair accumulator of frame pair k with one red.global.add.v2, and
// a combine pass adds pair k's first value into frame k and its second into
// frame k + 1.  With separate frames the two reductions of a segment land
// one frame (a cube) apart, in two sectors; side by side they are one 8-byte
// operation in one sector.
//
// Thomson total brightness (Section 3.5, Eq. thomson_direct): T_B x =
// P M' x - O P M x needs two projections of the same rays.  One walk gathers
// the pair (m' x, m x) of every voxel and gives both sums; the pixel is
// g (s' - rho^2 s).  The transpose scatters (len g y, len rho^2 g y) into
// one pair accumulator, and T_B^T y = m' a - m b is formed per voxel
// afterwards.
//
// Rays that do not fit the plane walk take the per-ray walk on the native
// layout, with the caller's separate frames (time interpolation) or the
// native pair buffer (Thomson B).
#include "plane.cuh"

namespace tomo {

namespace {

// Slabs per iteration of the forward's middle range (loads in flight), as
// measured on GB300: 8-frame 256^3 temporal P 22.7 ms at 2 slabs, 16.6 ms
// at 4, 18.6 ms at 6, 20.7 ms at 8 (3 CTAs per SM); Thomson B forward on
// the 256^3 cube 14.8, 11.6, 12.5, 13.2 ms.  At 4 CTAs per SM with byte
// offsets: temporal 15.9 ms at 4 slabs, 17.1 at 6, 15.7 at 8; B 10.9, 12.1,
// 11.3 ms.
constexpr int kPairFwdUnroll = 4;
constexpr int kPairFwdMinBlocks = 4;
constexpr int kPairAdjMinBlocks = 5;

__device__ __forceinline__ float2 load_pair(const float2 *c, int idx)
{
    return __ldg(c + idx);
}

// bf16 pair: the first value in the low half, the second in the high half
__device__ __forceinline__ float2 load_pair(const uint32_t *c, int idx)
{
    const uint32_t e = __ldg(c + idx);
    return make_float2(__uint_as_float(e << 16), __uint_as_float(e & 0xffff0000u));
}

// Fire-and-forget addition of two adjacent floats (8-byte aligned) in
// global memory, one vector reduction, under a predicate (see red_add_if).
__device__ __forceinline__ void red_add2_if(bool on, float2 *p, float a,
                                            float b)
{
    asm volatile("{\n\t.reg .pred q;\n\t"
                 "setp.ne.b32 q, %3, 0;\n\t"
                 "@q red.global.add.v2.f32 [%0], {%1, %2};\n\t}"
                 :
                 : "l"(__cvta_generic_to_global(p)), "f"(a), "f"(b),
                   "r"((int)on)
                 : "memory");
}

// Buffer of layout L, chosen by selects (indexing the kernel parameter's
// array with a run-time L would copy it to local memory).
__device__ __forceinline__ const void *pick(const PlaneCubes &c, int L)
{
    return L == 1 ? c.c[1] : (L == 2 ? c.c[2] : c.c[0]);
}

__device__ __forceinline__ float *pick(const PlaneAcc &c, int L)
{
    return L == 1 ? c.c[1] : (L == 2 ? c.c[2] : c.c[0]);
}

// Plane ops (byte offsets, see plane.cuh)
template <typename PairT>
struct PlaneGatherPairOp {
    const PairT *c;
    float w0, w1, acc;
    using Val = float2;
    static constexpr bool kAllSlots = true;
    __device__ __forceinline__ void clear() { acc = 0.0f; }
    __device__ __forceinline__ float2 fetch(bool on, uint32_t off) const
    {
        return on ? load_pair(byte_at(c, off), 0) : make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ void apply(bool on, uint32_t, float len, float2 v)
    {
        if (on) acc = fmaf(len, fmaf(w0, v.x, w1 * v.y), acc);
    }
    __device__ __forceinline__ void operator()(bool on, uint32_t off, float len)
    {
        apply(on, off, len, fetch(on, off));
    }
};

struct PlaneGatherBOp {
    const float2 *c;
    float s1, s2;
    using Val = float2;
    // two sums per slot: the predicated bodies measured faster (11.0
    // against 12.9 ms on the 256^3 cube)
    static constexpr bool kAllSlots = false;
    __device__ __forceinline__ void clear()
    {
        s1 = 0.0f;
        s2 = 0.0f;
    }
    __device__ __forceinline__ float2 fetch(bool on, uint32_t off) const
    {
        return on ? load_pair(byte_at(c, off), 0) : make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ void apply(bool on, uint32_t, float len, float2 v)
    {
        if (on) {
            s1 = fmaf(len, v.x, s1);
            s2 = fmaf(len, v.y, s2);
        }
    }
    __device__ __forceinline__ void operator()(bool on, uint32_t off, float len)
    {
        apply(on, off, len, fetch(on, off));
    }
};

// per-ray form of PlaneGatherBOp (walk.cuh's op signature)
struct GatherBOp {
    const float2 *c;
    float s1, s2;
    using Val = float2;
    __device__ __forceinline__ float2 fetch(int idx) const
    {
        return load_pair(c, idx);
    }
    __device__ __forceinline__ void apply(float len, float2 v)
    {
        s1 = fmaf(len, v.x, s1);
        s2 = fmaf(len, v.y, s2);
    }
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        const float2 v = load_pair(c, idx);
        s1 = fmaf(len, v.x, s1);
        s2 = fmaf(len, v.y, s2);
    }
};

struct PlaneScatterPairOp {
    float2 *c;
    float y0, y1;
    using Val = NoVal;
    static constexpr bool kAllSlots = false;
    __device__ __forceinline__ NoVal fetch(bool, uint32_t) const { return NoVal(); }
    __device__ __forceinline__ void apply(bool on, uint32_t off, float len, NoVal)
    {
        red_add2_if(on, byte_at(c, off), len * y0, len * y1);
    }
    __device__ __forceinline__ void operator()(bool on, uint32_t off, float len)
    {
        apply(on, off, len, NoVal());
    }
};

struct ScatterPairOp {
    float2 *c;
    float y0, y1;
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        red_add2_if(len > 0.0f, c + idx, len * y0, len * y1);
    }
};

// ---------------------------------------------------------------- forward

// Time-interpolated forward on frame pairs.  pairs.c[L]: pair buffer of
// layout L, T - 1 pairs of n voxels; native: the caller's frames (for rays
// outside the plane walk).
template <typename CubeT, typename PairT>
__global__ void __launch_bounds__(256, kPairFwdMinBlocks)
k_forward_plane_pair(const RayRec *__restrict__ rays,
                     const ImgParam *__restrict__ prm, PlaneCubes pairs,
                     const CubeT *__restrict__ native, int64_t fstride,
                     const uint8_t *__restrict__ mask, float *__restrict__ out,
                     int nu, int nv, int nx, int ny, int nz, Tiling tl,
                     const double *__restrict__ done, bool only_marked,
                     int n_img, int group)
{
    if (done != nullptr && *done != 0.0) return;
    int img, tile_v;
    if (!plane_cta(n_img, group, img, tile_v)) return;
    const ImgParam q = prm[img];
    if (only_marked && !(q.pad & kPlaneFwdBit)) return;  // uniform per CTA
    int iu, iv;
    const bool in_img = pixel_of_thread(tl, blockIdx.x, tile_v, nu, nv, iu, iv);
    const int64_t id = ((int64_t)img * nv + iv) * nu + iu;
    RayRec r;
    r.chord = -1.0f;
    if (in_img && (mask == nullptr || mask[id] == 0)) r = load_ray(rays + id);
    const bool live = r.chord > 0.0f;
    PlaneRay p;
    const bool regular = live && plane_ray(r, q.pad, nx, ny, nz, p, sizeof(PairT));
    const int L = (q.pad >> 2) & 3;
    const int64_t f0 = (int64_t)img_frame(q) * fstride;
    PlaneGatherPairOp<PairT> op;
    op.c = static_cast<const PairT *>(pick(pairs, L)) + f0;
    op.w0 = q.w0;
    op.w1 = q.w;
    op.acc = 0.0f;
    plane_walk_for<kPairFwdUnroll>(q.pad, p, regular, op);
    float acc = op.acc;
    if (live && !regular) {
        GatherTimeOp<CubeT> op2;
        op2.c0 = native + f0;
        op2.c1 = op2.c0 + fstride;
        op2.w0 = op.w0;
        op2.w1 = op.w1;
        op2.acc = 0.0f;
        siddon_gather(r, nx, nx * ny, op2);
        acc = op2.acc;
    }
    if (in_img) out[id] = q.gain * acc;
}

// Thomson B forward on (m' x, m x) pairs: y = g s' - rho^2 (g s).
// pairs.c[L]: the pair buffer in layout L (c[0]: native).  plane_mode 2
// walks every image plane by plane, 1 the images whose hint has the
// plane-forward bit, 0 none; the other images (and the rays that do not fit
// the plane walk) walk per ray on the native pairs.
__global__ void __launch_bounds__(256, kPairFwdMinBlocks)
k_forward_b(const RayRec *__restrict__ rays, const ImgParam *__restrict__ prm,
            PlaneCubes pairs, const float *__restrict__ rho2,
            const uint8_t *__restrict__ mask, float *__restrict__ out, int nu,
            int nv, int nx, int ny, int nz, Tiling tl,
            const double *__restrict__ done, int plane_mode, int n_img,
            int group)
{
    if (done != nullptr && *done != 0.0) return;
    int img, tile_v;
    if (!plane_cta(n_img, group, img, tile_v)) return;
    const ImgParam q = prm[img];
    // uniform per CTA
    const bool plane = plane_mode == 2 || (plane_mode == 1 && (q.pad & kPlaneFwdBit));
    int iu, iv;
    const bool in_img = pixel_of_thread(tl, blockIdx.x, tile_v, nu, nv, iu, iv);
    const int64_t id = ((int64_t)img * nv + iv) * nu + iu;
    RayRec r;
    r.chord = -1.0f;
    if (in_img && (mask == nullptr || mask[id] == 0)) r = load_ray(rays + id);
    const bool live = r.chord > 0.0f;
    PlaneRay p;
    const bool regular =
        plane && live && plane_ray(r, q.pad, nx, ny, nz, p, sizeof(float2));
    const int L = (q.pad >> 2) & 3;
    float s1 = 0.0f, s2 = 0.0f;
    if (plane) {
        PlaneGatherBOp op;
        op.c = static_cast<const float2 *>(pick(pairs, L));
        op.s1 = 0.0f;
        op.s2 = 0.0f;
        plane_walk_for<kPairFwdUnroll>(q.pad, p, regular, op);
        s1 = op.s1;
        s2 = op.s2;
    }
    if (live && !regular) {
        GatherBOp op2;
        op2.c = static_cast<const float2 *>(pairs.c[0]);
        op2.s1 = 0.0f;
        op2.s2 = 0.0f;
        siddon_gather(r, nx, nx * ny, op2);
        s1 = op2.s1;
        s2 = op2.s2;
    }
    if (in_img) out[id] = fmaf(-rho2[id], q.gain * s2, q.gain * s1);
}

// -------------------------------------------------------------- transpose

// Time-interpolated transpose into frame-pair accumulators.  acc.c[L]:
// pair accumulator of layout L (float2, T - 1 pairs of n voxels); cube: the
// caller's frames, which rays outside the plane walk add into directly.
__global__ void __launch_bounds__(256, kPairAdjMinBlocks)
k_adjoint_plane_pair(const RayRec *__restrict__ rays,
                     const ImgParam *__restrict__ prm,
                     const float *__restrict__ images,
                     const uint8_t *__restrict__ mask, PlaneAcc acc,
                     float *cube, int64_t fstride, int nu, int nv, int nx,
                     int ny, int nz, Tiling tl, const double *__restrict__ done,
                     int n_img, int group)
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
    const bool regular = live && plane_ray(r, q.pad, nx, ny, nz, p, sizeof(float2));
    const int L = (q.pad >> 2) & 3;
    const int64_t f0 = (int64_t)img_frame(q) * fstride;
    PlaneScatterPairOp op;
    op.c = reinterpret_cast<float2 *>(pick(acc, L)) + f0;
    op.y0 = yv * q.w0;
    op.y1 = yv * q.w;
    plane_walk_for<1>(q.pad, p, regular, op);
    if (live && !regular) {
        ScatterTimeOp op2;
        op2.c0 = cube + f0;
        op2.c1 = op2.c0 + fstride;
        op2.y0 = op.y0;
        op2.y1 = op.y1;
        siddon_walk(r, nx, nx * ny, op2);
    }
}

// Thomson B transpose into one (a, b) pair accumulator per layout:
// a += len g y, b += len rho^2 g y.  acc.c[0] is the native accumulator,
// which rays outside the plane walk (and, with plane_on false, every ray)
// use.
__global__ void __launch_bounds__(256, kPairAdjMinBlocks)
k_adjoint_b(const RayRec *__restrict__ rays, const ImgParam *__restrict__ prm,
            const float *__restrict__ images, const float *__restrict__ rho2,
            const uint8_t *__restrict__ mask, PlaneAcc acc, int nu, int nv,
            int nx, int ny, int nz, Tiling tl, const double *__restrict__ done,
            bool plane_on, int n_img, int group)
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
    float yv = 0.0f, rv = 0.0f;
    if (in_img && (mask == nullptr || mask[id] == 0)) {
        yv = q.gain * images[id];
        rv = rho2[id] * yv;
        if (yv != 0.0f) r = load_ray(rays + id);
    }
    const bool live = r.chord > 0.0f;
    PlaneRay p;
    const bool regular =
        plane_on && live && plane_ray(r, q.pad, nx, ny, nz, p, sizeof(float2));
    const int L = (q.pad >> 2) & 3;
    PlaneScatterPairOp op;
    op.c = reinterpret_cast<float2 *>(pick(acc, L));
    op.y0 = yv;
    op.y1 = rv;
    plane_walk_for<1>(q.pad, p, regular, op);
    if (live && !regular) {
        ScatterPairOp op2;
        op2.c = reinterpret_cast<float2 *>(acc.c[0]);
        op2.y0 = yv;
        op2.y1 = rv;
        siddon_walk(r, nx, nx * ny, op2);
    }
}

// ---------------------------------------------------------- layout passes

// Layout L (1 or 2) makes axis b (y or z) the fastest; c is the remaining
// axis.  Native index: x + sb b + sc c; layout index: b + nb (x + nx c).
struct PairMap {
    int nx, nb, nc;
    int64_t sb, sc;
};

PairMap pair_map(int L, int nx, int ny, int nz)
{
    PairMap m;
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

__device__ __forceinline__ float2 make_pair(float a, float b)
{
    return make_float2(a, b);
}

__device__ __forceinline__ uint32_t make_pair(uint16_t a, uint16_t b)
{
    return (uint32_t)a | ((uint32_t)b << 16);
}

// Native-order frame pairs: out[k][v] = (src[k][v], src[k + 1][v]).
template <typename T, typename PairT>
__global__ void __launch_bounds__(256)
k_pairs_native(const T *__restrict__ src, PairT *__restrict__ out, int64_t n,
               int T_frames, const unsigned *__restrict__ used, unsigned bit,
               const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        T prev = src[v];
        for (int k = 0; k + 1 < T_frames; ++k) {
            const T cur = src[(int64_t)(k + 1) * n + v];
            out[(int64_t)k * n + v] = make_pair(prev, cur);
            prev = cur;
        }
    }
}

// Frame pairs in layout L: one CTA moves 32 x 32 (x, b) tiles of every frame
// through shared memory (reads along x, writes along b coalesced), keeping
// the previous frame's tile to form the pairs.
template <typename T, typename PairT>
__global__ void __launch_bounds__(256)
k_pairs_layout(const T *__restrict__ src, PairT *__restrict__ out, PairMap m,
               int T_frames, int64_t n, const unsigned *__restrict__ used,
               unsigned bit, const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    __shared__ T tile[2][32][33];
    const int x0 = blockIdx.x * 32, b0 = blockIdx.y * 32, c = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int f = 0; f < T_frames; ++f) {
        const T *s = src + (int64_t)f * n;
        const int cur = f & 1;
        for (int k = ty; k < 32; k += 8) {
            const int b = b0 + k, x = x0 + tx;
            if (b < m.nb && x < m.nx) tile[cur][k][tx] = s[x + m.sb * b + m.sc * c];
        }
        __syncthreads();
        if (f > 0) {
            PairT *o = out + (int64_t)(f - 1) * n;
            for (int k = ty; k < 32; k += 8) {
                const int x = x0 + k, b = b0 + tx;
                if (b < m.nb && x < m.nx)
                    o[b + (int64_t)m.nb * (x + (int64_t)m.nx * c)] =
                        make_pair(tile[cur ^ 1][tx][k], tile[cur][tx][k]);
            }
        }
        __syncthreads();
    }
}

// Frames += pair accumulators (native order): frame f receives the first
// value of pair f and the second value of pair f - 1.
__global__ void __launch_bounds__(256)
k_add_pairs_native(const float2 *__restrict__ acc, float *__restrict__ cube,
                   int64_t n, int T_frames, const unsigned *__restrict__ used,
                   unsigned bit, const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        float carry = 0.0f;
        for (int f = 0; f < T_frames; ++f) {
            const float2 a = f + 1 < T_frames ? acc[(int64_t)f * n + v]
                                              : make_float2(0.0f, 0.0f);
            cube[(int64_t)f * n + v] += a.x + carry;
            carry = a.y;
        }
    }
}

// The same from layout L, through 32 x 32 shared-memory tiles.
__global__ void __launch_bounds__(256)
k_add_pairs_layout(const float2 *__restrict__ acc, float *__restrict__ cube,
                   PairMap m, int T_frames, int64_t n,
                   const unsigned *__restrict__ used, unsigned bit,
                   const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    __shared__ float2 tile[32][33];
    const int x0 = blockIdx.x * 32, b0 = blockIdx.y * 32, c = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float carry[4] = { 0.0f, 0.0f, 0.0f, 0.0f };
    for (int f = 0; f < T_frames; ++f) {
        if (f + 1 < T_frames) {
            const float2 *a = acc + (int64_t)f * n;
            for (int k = ty; k < 32; k += 8) {
                const int x = x0 + k, b = b0 + tx;
                if (b < m.nb && x < m.nx)
                    tile[tx][k] = a[b + (int64_t)m.nb * (x + (int64_t)m.nx * c)];
            }
        }
        __syncthreads();
        float *dst = cube + (int64_t)f * n;
        for (int k = ty, e = 0; k < 32; k += 8, ++e) {
            const int b = b0 + k, x = x0 + tx;
            const float2 a = f + 1 < T_frames ? tile[k][tx] : make_float2(0.0f, 0.0f);
            if (b < m.nb && x < m.nx) dst[x + m.sb * b + m.sc * c] += a.x + carry[e];
            carry[e] = a.y;
        }
        __syncthreads();
    }
}

// Native float2 buffer += layout-L float2 accumulator (Thomson B pairs).
__global__ void __launch_bounds__(256)
k_add_b_layout(const float2 *__restrict__ acc, float2 *__restrict__ out,
               PairMap m, const unsigned *__restrict__ used, unsigned bit,
               const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    __shared__ float2 tile[32][33];
    const int x0 = blockIdx.x * 32, b0 = blockIdx.y * 32, c = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const int x = x0 + k, b = b0 + tx;
        if (b < m.nb && x < m.nx)
            tile[tx][k] = acc[b + (int64_t)m.nb * (x + (int64_t)m.nx * c)];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int b = b0 + k, x = x0 + tx;
        if (b < m.nb && x < m.nx) {
            float2 &d = out[x + m.sb * b + m.sc * c];
            const float2 a = tile[k][tx];
            d = make_float2(d.x + a.x, d.y + a.y);
        }
    }
}

// Copy of a native float2 buffer in layout L (Thomson B forward).
__global__ void __launch_bounds__(256)
k_b_to_layout(const float2 *__restrict__ in, float2 *__restrict__ out,
              PairMap m, const unsigned *__restrict__ used, unsigned bit,
              const double *__restrict__ done)
{
    if (done != nullptr && *done != 0.0) return;
    if (!(*used & bit)) return;
    __shared__ float2 tile[32][33];
    const int x0 = blockIdx.x * 32, b0 = blockIdx.y * 32, c = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const int b = b0 + k, x = x0 + tx;
        if (b < m.nb && x < m.nx) tile[k][tx] = in[x + m.sb * b + m.sc * c];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int x = x0 + k, b = b0 + tx;
        if (b < m.nb && x < m.nx)
            out[b + (int64_t)m.nb * (x + (int64_t)m.nx * c)] = tile[tx][k];
    }
}

constexpr Tiling kPlaneTiling2 = { 32, 8, 32 };

dim3 plane_grid2(int nu, int nv, int n_img, int &group)
{
    const int tiles_v = (nv + 7) / 8;
    group = plane_group_clamp(group, n_img, tiles_v);
    return dim3((unsigned)((nu + 31) / 32), (unsigned)(tiles_v * group),
                (unsigned)((n_img + group - 1) / group));
}

dim3 pair_grid(const PairMap &m)
{
    return dim3((unsigned)((m.nx + 31) / 32), (unsigned)((m.nb + 31) / 32),
                (unsigned)m.nc);
}

unsigned flat_grid(int64_t n, int num_sms)
{
    int64_t g = (n + 255) / 256;
    const int64_t cap = 8LL * (num_sms > 0 ? num_sms : 152);
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_to_pairs(const void *cube, tomo_dtype dtype, void *out,
                            int L, const tomo_cube_geom *c, int32_t n_frames,
                            const unsigned *used, unsigned bit,
                            const double *done, int num_sms, cudaStream_t s)
{
    if (n_frames < 2) return cudaSuccess;
    const int64_t n = (int64_t)c->nx * c->ny * c->nz;
    const bool bf = dtype == TOMO_BF16;
    if (L == 0) {
        if (bf)
            k_pairs_native<uint16_t, uint32_t><<<flat_grid(n, num_sms), 256, 0, s>>>(
                static_cast<const uint16_t *>(cube), static_cast<uint32_t *>(out),
                n, n_frames, used, bit, done);
        else
            k_pairs_native<float, float2><<<flat_grid(n, num_sms), 256, 0, s>>>(
                static_cast<const float *>(cube), static_cast<float2 *>(out), n,
                n_frames, used, bit, done);
        return cudaGetLastError();
    }
    const PairMap m = pair_map(L, c->nx, c->ny, c->nz);
    if (bf)
        k_pairs_layout<uint16_t, uint32_t><<<pair_grid(m), 256, 0, s>>>(
            static_cast<const uint16_t *>(cube), static_cast<uint32_t *>(out), m,
            n_frames, n, used, bit, done);
    else
        k_pairs_layout<float, float2><<<pair_grid(m), 256, 0, s>>>(
            static_cast<const float *>(cube), static_cast<float2 *>(out), m,
            n_frames, n, used, bit, done);
    return cudaGetLastError();
}

cudaError_t launch_add_pairs(const void *acc, float *cube, int L,
                             const tomo_cube_geom *c, int32_t n_frames,
                             const unsigned *used, const double *done,
                             int num_sms, cudaStream_t s)
{
    const int64_t n = (int64_t)c->nx * c->ny * c->nz;
    const float2 *a = static_cast<const float2 *>(acc);
    if (L == 0) {
        k_add_pairs_native<<<flat_grid(n, num_sms), 256, 0, s>>>(
            a, cube, n, n_frames, used, 1u << L, done);
        return cudaGetLastError();
    }
    const PairMap m = pair_map(L, c->nx, c->ny, c->nz);
    k_add_pairs_layout<<<pair_grid(m), 256, 0, s>>>(a, cube, m, n_frames, n,
                                                    used, 1u << L, done);
    return cudaGetLastError();
}

cudaError_t launch_b_to_layout(const void *in, void *out, int L,
                               const tomo_cube_geom *c, const unsigned *used,
                               unsigned bit, const double *done,
                               cudaStream_t s)
{
    const PairMap m = pair_map(L, c->nx, c->ny, c->nz);
    k_b_to_layout<<<pair_grid(m), 256, 0, s>>>(
        static_cast<const float2 *>(in), static_cast<float2 *>(out), m, used,
        bit, done);
    return cudaGetLastError();
}

cudaError_t launch_add_b_layout(const void *acc, void *out, int L,
                                const tomo_cube_geom *c, const unsigned *used,
                                const double *done, cudaStream_t s)
{
    const PairMap m = pair_map(L, c->nx, c->ny, c->nz);
    k_add_b_layout<<<pair_grid(m), 256, 0, s>>>(
        static_cast<const float2 *>(acc), static_cast<float2 *>(out), m, used,
        1u << L, done);
    return cudaGetLastError();
}

cudaError_t launch_forward_plane_pair(const RayRec *rays, const ImgParam *prm,
                                      PlaneCubes pairs, const void *native,
                                      tomo_dtype dtype, int64_t fstride,
                                      const uint8_t *mask, float *out,
                                      int32_t n_img, int32_t nu, int32_t nv,
                                      const tomo_cube_geom *c,
                                      const double *done, cudaStream_t s,
                                      bool only_marked, int group)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid = plane_grid2(nu, nv, n_img, group);
    if (dtype == TOMO_BF16)
        k_forward_plane_pair<uint16_t, uint32_t><<<grid, 256, 0, s>>>(
            rays, prm, pairs, static_cast<const uint16_t *>(native), fstride,
            mask, out, nu, nv, c->nx, c->ny, c->nz, kPlaneTiling2, done,
            only_marked, n_img, group);
    else
        k_forward_plane_pair<float, float2><<<grid, 256, 0, s>>>(
            rays, prm, pairs, static_cast<const float *>(native), fstride,
            mask, out, nu, nv, c->nx, c->ny, c->nz, kPlaneTiling2, done,
            only_marked, n_img, group);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_plane_pair(const RayRec *rays, const ImgParam *prm,
                                      const float *images, const uint8_t *mask,
                                      PlaneAcc acc, float *cube,
                                      int64_t fstride, int32_t n_img,
                                      int32_t nu, int32_t nv,
                                      const tomo_cube_geom *c,
                                      const double *done, cudaStream_t s,
                                      int group)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid = plane_grid2(nu, nv, n_img, group);
    k_adjoint_plane_pair<<<grid, 256, 0, s>>>(
        rays, prm, images, mask, acc, cube, fstride, nu, nv, c->nx, c->ny,
        c->nz, kPlaneTiling2, done, n_img, group);
    return cudaGetLastError();
}

cudaError_t launch_forward_b(const RayRec *rays, const ImgParam *prm,
                             PlaneCubes pairs, const float *rho2,
                             const uint8_t *mask, float *out, int32_t n_img,
                             int32_t nu, int32_t nv, const tomo_cube_geom *c,
                             const double *done, int plane_mode,
                             cudaStream_t s, int group)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid = plane_grid2(nu, nv, n_img, group);
    k_forward_b<<<grid, 256, 0, s>>>(
        rays, prm, pairs, rho2, mask, out, nu, nv, c->nx, c->ny, c->nz,
        kPlaneTiling2, done, plane_mode, n_img, group);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_b(const RayRec *rays, const ImgParam *prm,
                             const float *images, const float *rho2,
                             const uint8_t *mask, PlaneAcc acc, int32_t n_img,
                             int32_t nu, int32_t nv, const tomo_cube_geom *c,
                             const double *done, bool plane_on,
                             cudaStream_t s, int group)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid = plane_grid2(nu, nv, n_img, group);
    k_adjoint_b<<<grid, 256, 0, s>>>(
        rays, prm, images, rho2, mask, acc, nu, nv, c->nx, c->ny, c->nz,
        kPlaneTiling2, done, plane_on, n_img, group);
    return cudaGetLastError();
}

}  // namespace tomo
