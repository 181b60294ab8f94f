// Plane-synchronous Siddon walk: per-ray setup, the warp-wide walk and its
// segment operations, shared by the single-problem kernels (plane.cu) and
// the batched transpose (batch.cu).  The design and its exactness argument
// are described at the top of plane.cu.
#pragma once

#include <limits.h>
#include <math.h>

#include <type_traits>

#include "walk.cuh"

namespace tomo {

// The CTA's image and pixel-tile row.  The grid is (tile columns, tile rows
// x group, image groups): inside a group of `group` consecutive images the
// CTAs of one tile row of every image run before those of the next row, so
// the CTAs resident at one time gather from or add into one band of the
// cube (the rays of one pixel row of views taken near a common plane cross
// few planes of the cube) rather than the whole cube of one image.  Returns
// false for the padding images of the last group (uniform over the CTA).
__device__ __forceinline__ bool plane_cta(int n_img, int group, int &img,
                                          int &tile_v)
{
    tile_v = (int)blockIdx.y / group;
    img = (int)blockIdx.z * group + (int)blockIdx.y % group;
    return img < n_img;
}

// One ray, re-expressed for the plane walk: M first, then the two minor
// axes, a1 the one with the smaller crossing spacing (crossed more often).
// Voxel positions are byte offsets from the walked buffer's base, held as
// unsigned 32-bit numbers (a step in the negative direction adds the
// stride's two's complement, which wraps to the right offset); a gather or
// reduction then needs no 64-bit index arithmetic, only the base plus a
// 32-bit offset.  The walked buffer (one cube or one frame pair of it) must
// therefore span at most 2^32 bytes: plane_supported() checks that.
struct PlaneRay {
    float t0M, t01, t02;  // first crossings
    float AM, A1, A2;     // crossing spacings
    float chord;
    uint32_t sM, s1, s2;  // signed strides in the image's layout, in bytes
    uint32_t idx;         // entry voxel in the image's layout, in bytes
    int key;              // entry M coordinate, signed by the M direction
};

// base + off bytes (off: a plane-walk voxel offset)
template <typename T>
__device__ __forceinline__ T *byte_at(T *base, uint32_t off)
{
    using B = typename std::conditional<std::is_const<T>::value, const char,
                                        char>::type;
    return reinterpret_cast<T *>(reinterpret_cast<B *>(base) + off);
}

__device__ __forceinline__ void layout_strides(int L, int nx, int ny, int nz,
                                               int &stx, int &sty, int &stz)
{
    if (L == 1) {
        stx = ny;
        sty = 1;
        stz = nx * ny;
    } else if (L == 2) {
        stx = nz;
        sty = nx * nz;
        stz = 1;
    } else {
        stx = 1;
        sty = nx;
        stz = nx * ny;
    }
}

// Fills p and returns true when the ray fits the plane walk of its image;
// esize is the size in bytes of one voxel of the walked buffer.
__device__ __forceinline__ bool plane_ray(const RayRec &r, int hint, int nx,
                                          int ny, int nz, PlaneRay &p,
                                          uint32_t esize)
{
    if (!(hint & kPlaneHintValid)) return false;
    const int M = hint & 3, L = (hint >> 2) & 3;
    const bool neg = (hint >> 4) & 1;
    const int cx = r.idx0 % nx;
    const int rest = r.idx0 / nx;
    const int cy = rest % ny, cz = rest / ny;
    int lx, ly, lz;
    layout_strides(L, nx, ny, nz, lx, ly, lz);
    const uint32_t stx = (uint32_t)lx * esize, sty = (uint32_t)ly * esize,
                   stz = (uint32_t)lz * esize;
    const uint32_t gx = signbit(r.dtx) ? 0u - stx : stx;
    const uint32_t gy = signbit(r.dty) ? 0u - sty : sty;
    const uint32_t gz = signbit(r.dtz) ? 0u - stz : stz;
    const float dM = M == 0 ? r.dtx : (M == 1 ? r.dty : r.dtz);
    p.t0M = M == 0 ? r.t0x : (M == 1 ? r.t0y : r.t0z);
    p.t01 = M == 0 ? r.t0y : r.t0x;
    p.t02 = M == 2 ? r.t0y : r.t0z;
    p.AM = fabsf(dM);
    p.A1 = fabsf(M == 0 ? r.dty : r.dtx);
    p.A2 = fabsf(M == 2 ? r.dty : r.dtz);
    p.sM = M == 0 ? gx : (M == 1 ? gy : gz);
    p.s1 = M == 0 ? gy : gx;
    p.s2 = M == 2 ? gy : gz;
    // a1 = the minor axis crossed more often (spacing 0: never crossed)
    if (p.A2 != 0.0f && (p.A1 == 0.0f || p.A2 < p.A1)) {
        float f = p.t01;
        p.t01 = p.t02;
        p.t02 = f;
        f = p.A1;
        p.A1 = p.A2;
        p.A2 = f;
        const uint32_t g = p.s1;
        p.s1 = p.s2;
        p.s2 = g;
    }
    p.chord = r.chord;
    p.idx = (uint32_t)cx * stx + (uint32_t)cy * sty + (uint32_t)cz * stz;
    const int cM = M == 0 ? cx : (M == 1 ? cy : cz);
    p.key = neg ? -cM : cM;
    // Two crossings of a minor axis in one slab need its crossing spacing,
    // less rounding of two crossing parameters (each <= 2^-24 of a value of
    // at most chord + spacing), below the slab length plus the same: the
    // margin below is eight times that bound.
    const float margin = ldexpf(p.chord + fmaxf(p.A1, p.A2) + p.AM, -19);
    const bool ok1 = p.A1 == 0.0f || p.A1 > p.AM + margin;
    const bool ok2 = p.A2 == 0.0f || p.A2 > p.AM + margin;
    return p.AM > 0.0f && (signbit(dM) != 0) == neg && ok1 && ok2;
}

// First slab j >= 0 whose far plane fmaf(j, AM, t0M) lies beyond x (at or
// beyond x when `reach`).  The far planes are the walk's own float values,
// so the answer agrees with every comparison the walk makes; the quotient
// only gives the starting point, the two loops make it exact.
__device__ __forceinline__ int slab_past(float AM, float t0M, float x, bool reach)
{
    int j = (int)fmaxf(ceilf((x - t0M) / AM), 0.0f);
    for (;;) {
        if (j == 0) break;
        const float f = fmaf((float)(j - 1), AM, t0M);
        if (reach ? f < x : f <= x) break;
        --j;
    }
    for (;;) {
        const float f = fmaf((float)j, AM, t0M);
        if (reach ? f >= x : f > x) break;
        ++j;
    }
    return j;
}

// Per-lane state of the plane walk: distance travelled t, next crossings
// t1, t2 of the two minor axes and their crossing counts, current voxel.
struct PlaneState {
    float t, t1, t2, k1, k2;
    uint32_t idx;
};

// The fast slab body: at most one crossing, of a1, inside the slab that ends
// at te.  Emits two segment slots; `go` says whether the lane walks this slab.
__device__ __forceinline__ void slab_fast(const PlaneRay &p, uint32_t sM,
                                          PlaneState &s, bool go, float te,
                                          bool *o, uint32_t *id, float *ln)
{
    const bool c1 = go && s.t1 < te;
    o[0] = go;
    id[0] = s.idx;
    ln[0] = fminf(s.t1, te) - s.t;
    o[1] = c1;
    id[1] = s.idx + p.s1;
    ln[1] = te - s.t1;
    s.k1 = c1 ? s.k1 + 1.0f : s.k1;
    s.t1 = c1 ? fmaf(s.k1, p.A1, p.t01) : s.t1;
    s.idx += (c1 ? p.s1 : 0u) + (go ? sM : 0u);
    s.t = go ? te : s.t;
}

// The general slab body: up to one crossing of each minor axis, in either
// order.  Emits three segment slots.
__device__ __forceinline__ void slab_general(const PlaneRay &p, uint32_t sM,
                                             PlaneState &s, bool go, float te,
                                             bool *o, uint32_t *id, float *ln)
{
    const bool first1 = s.t1 <= s.t2;
    const float ta = first1 ? s.t1 : s.t2;
    const float tb = first1 ? s.t2 : s.t1;
    const uint32_t sa = first1 ? p.s1 : p.s2;
    o[0] = go;
    id[0] = s.idx;
    ln[0] = fminf(ta, te) - s.t;
    o[1] = go && ta < te;
    id[1] = s.idx + sa;
    ln[1] = fminf(tb, te) - ta;
    o[2] = go && tb < te;
    id[2] = s.idx + p.s1 + p.s2;
    ln[2] = te - tb;
    const bool c1 = go && s.t1 < te, c2 = go && s.t2 < te;
    s.k1 = c1 ? s.k1 + 1.0f : s.k1;
    s.k2 = c2 ? s.k2 + 1.0f : s.k2;
    s.t1 = c1 ? fmaf(s.k1, p.A1, p.t01) : s.t1;
    s.t2 = c2 ? fmaf(s.k2, p.A2, p.t02) : s.t2;
    s.idx += (c1 ? p.s1 : 0u) + (c2 ? p.s2 : 0u) + (go ? sM : 0u);
    s.t = go ? te : s.t;
}

// Gather forms of the two bodies, used inside the middle range, where every
// regular lane walks the slab.  Every slot is on: a slot without its
// crossing in this slab reads the lane's current voxel (in the cube) with
// length max(..., 0) = 0, so gathers and their additions need no per-slot
// predicate (keeping up to eight slot predicates live across the fetches of
// four slabs measured 5.5 % slower).  The lengths of the crossed slots are
// the general forms' values, so sums keep their bits for finite cubes (a
// zero length times an infinite voxel gives NaN where the per-ray walk
// gives the infinity).  Lanes that are not regular walk safe_plane_ray().
__device__ __forceinline__ void slab_fast_g(const PlaneRay &p, uint32_t sM,
                                            PlaneState &s, bool go, float te,
                                            bool *o, uint32_t *id, float *ln)
{
    const bool c1 = go && s.t1 < te;
    const uint32_t d1 = c1 ? p.s1 : 0u;
    o[0] = true;
    id[0] = s.idx;
    ln[0] = fminf(s.t1, te) - s.t;
    o[1] = true;
    id[1] = s.idx + d1;
    ln[1] = fmaxf(te - s.t1, 0.0f);
    s.k1 = c1 ? s.k1 + 1.0f : s.k1;
    s.t1 = c1 ? fmaf(s.k1, p.A1, p.t01) : s.t1;
    s.idx += d1 + (go ? sM : 0u);
    s.t = go ? te : s.t;
}

__device__ __forceinline__ void slab_general_g(const PlaneRay &p, uint32_t sM,
                                               PlaneState &s, bool go,
                                               float te, bool *o,
                                               uint32_t *id, float *ln)
{
    const bool first1 = s.t1 <= s.t2;
    const float ta = first1 ? s.t1 : s.t2;
    const float tb = first1 ? s.t2 : s.t1;
    const uint32_t sa = first1 ? p.s1 : p.s2;
    const bool ca = go && ta < te, cb = go && tb < te;
    o[0] = true;
    id[0] = s.idx;
    ln[0] = fminf(ta, te) - s.t;
    o[1] = true;
    id[1] = s.idx + (ca ? sa : 0u);
    ln[1] = fmaxf(fminf(tb, te) - ta, 0.0f);
    o[2] = true;
    id[2] = s.idx + (cb ? p.s1 + p.s2 : 0u);
    ln[2] = fmaxf(te - tb, 0.0f);
    const bool c1 = go && s.t1 < te, c2 = go && s.t2 < te;
    s.k1 = c1 ? s.k1 + 1.0f : s.k1;
    s.k2 = c2 ? s.k2 + 1.0f : s.k2;
    s.t1 = c1 ? fmaf(s.k1, p.A1, p.t01) : s.t1;
    s.t2 = c2 ? fmaf(s.k2, p.A2, p.t02) : s.t2;
    s.idx += (c1 ? p.s1 : 0u) + (c2 ? p.s2 : 0u) + (go ? sM : 0u);
    s.t = go ? te : s.t;
}

// The ray a gathering lane that is not regular walks: offset 0 (inside the
// buffer), no steps, zero lengths (its plane-walk result is discarded).
__device__ __forceinline__ PlaneRay safe_plane_ray()
{
    PlaneRay p;
    p.t0M = 0.0f;
    p.t01 = INFINITY;
    p.t02 = INFINITY;
    p.AM = 0.0f;
    p.A1 = 0.0f;
    p.A2 = 0.0f;
    p.chord = 0.0f;
    p.sM = 0u;
    p.s1 = 0u;
    p.s2 = 0u;
    p.idx = 0u;
    p.key = 0;
    return p;
}

// Value type of the scatter ops, which fetch nothing.
struct NoVal {};

// Walks the regular lanes of the warp plane by plane; op(on, off, len) is
// called for every segment with on == true (len may be 0 at ties, which adds
// an exact zero) and, with on == false, for slots without a segment (off
// then may lie outside the cube and must not be touched).  For an op with
// kAllSlots set, the middle range calls it with on == true for every slot,
// a slot without a segment giving the lane's current voxel and length 0.
// Every lane of the warp must call this (it uses warp-wide reductions);
// lanes with regular == false only take part in those.
//
// Warp iteration i handles slab j = i - j0 of every lane (j0: how many M
// planes after the warp's first one the lane enters).  Each lane knows how
// many slabs it walks (jend) and in which slab its next crossing of the less
// steep minor axis a2 falls (j2); the warp runs a fast body, which allows at
// most one crossing (of a1) per slab, in a counted loop up to the first slab
// in which any lane crosses a2, runs the general three-segment body for that
// slab, and recomputes the bound.  For views near the ecliptic a2 is z and
// is crossed every few tens of slabs, so almost every slab takes the fast
// body with no warp-wide vote.  Both bodies give the same segments.
//
// With kEveryGeneral, every slab takes the general body and nothing is
// tracked: for views whose a2 component is large enough that some lane of
// the warp crosses a2 in most slabs (the lanes' a2 crossings spread over
// many slabs, since a row's rays differ slightly in slope and the observer
// is ~200 cube widths away), the votes and bound updates would cost more
// than they save.
//
// Inside the slabs that every regular lane walks and that end before every
// regular lane's last slab ([lo_all, hi_all)), no lane needs the "does it
// walk this slab" test nor the cap of the slab's far plane at the chord
// (that plane lies below the chord there, in the walk's own float values),
// and the slab index is carried as an exact float counter.  That middle
// range runs U slabs per iteration: the segment slots of U slabs are
// computed first and op is called on them afterwards, in slab order, so a
// gathering op can have all of its loads in flight at once while the sums
// keep their order (and their bits).
template <bool kEveryGeneral, int U, class Op>
__device__ __forceinline__ void plane_walk(const PlaneRay &p, bool regular,
                                           Op &op)
{
    constexpr int kSlots = kEveryGeneral ? 3 : 2;
    const unsigned full = 0xffffffffu;
    const int kmin = __reduce_min_sync(full, regular ? p.key : INT_MAX);
    const int j0 = regular ? p.key - kmin : 0;
    // the walk ends in the first slab whose far plane reaches the chord
    const int jend = regular ? 1 + slab_past(p.AM, p.t0M, p.chord, true) : 0;
    const int i_end = __reduce_max_sync(full, regular ? j0 + jend : 0);
    const int lo_all = __reduce_max_sync(full, regular ? j0 : 0);
    const int hi_all = __reduce_min_sync(full, regular ? j0 + jend - 1 : INT_MAX);
    // Scatters take a copy of the middle loop for warps whose lanes are all
    // regular: a reduction under a per-lane predicate costs about three more
    // instructions than an unconditional one (ptxas branches around it), and
    // the first slot of every middle slab is then unconditional (P^T on the
    // 256^3 cube: 7.5 % fewer instructions, 1.5 % less time).  Gathers keep
    // one copy: their unrolled loop is larger, and two copies measured 6 %
    // (256^3) to 30 % (512^3) slower.
    constexpr bool kSplit = std::is_same<typename Op::Val, NoVal>::value;
    const bool all_regular = kSplit && __all_sync(full, regular);
    // non-regular lanes never advance (their slots are all off)
    const uint32_t sM = regular ? p.sM : 0u;
    PlaneState s;
    s.t = 0.0f;
    s.k1 = 0.0f;
    s.k2 = 0.0f;
    s.t1 = p.t01;
    s.t2 = p.t02;
    s.idx = p.idx;

    // one slab with the lane tests (outside the middle range)
    auto edge = [&](int i, bool general) {
        const int j = i - j0;
        const bool go = (unsigned)j < (unsigned)jend;
        const float te = fminf(fmaf((float)j, p.AM, p.t0M), p.chord);
        bool o[3];
        uint32_t id[3];
        float ln[3];
        if (general) {
            slab_general(p, sM, s, go, te, o, id, ln);
            op(o[0], id[0], ln[0]);
            op(o[1], id[1], ln[1]);
            op(o[2], id[2], ln[2]);
        } else {
            slab_fast(p, sM, s, go, te, o, id, ln);
            op(o[0], id[0], ln[0]);
            op(o[1], id[1], ln[1]);
        }
    };
    // slabs [i, m_end) inside the middle range, kSlots-segment body; `all`
    // (warp-uniform): every lane of the warp is regular, so no slot needs the
    // lane's own test and the first slot's operation is unconditional
    auto middle = [&](int &i, int m_end, auto all) {
        constexpr bool kAll = decltype(all)::value;
        const bool reg = kAll ? true : regular;
        float jf = (float)(i - j0);
        for (; i + U <= m_end; i += U) {
            bool o[U * kSlots];
            uint32_t id[U * kSlots];
            float ln[U * kSlots];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float te = fmaf(jf, p.AM, p.t0M);
                jf += 1.0f;
                if constexpr (kEveryGeneral && !Op::kAllSlots)
                    slab_general(p, sM, s, reg, te, o + u * kSlots,
                                 id + u * kSlots, ln + u * kSlots);
                else if constexpr (kEveryGeneral)
                    slab_general_g(p, sM, s, reg, te, o + u * kSlots,
                                   id + u * kSlots, ln + u * kSlots);
                else if constexpr (!Op::kAllSlots)
                    slab_fast(p, sM, s, reg, te, o + u * kSlots,
                              id + u * kSlots, ln + u * kSlots);
                else
                    slab_fast_g(p, sM, s, reg, te, o + u * kSlots,
                                id + u * kSlots, ln + u * kSlots);
            }
            // all loads of the U slabs first, then the additions in order
            typename Op::Val v[U * kSlots];
#pragma unroll
            for (int k = 0; k < U * kSlots; ++k) v[k] = op.fetch(o[k], id[k]);
#pragma unroll
            for (int k = 0; k < U * kSlots; ++k) op.apply(o[k], id[k], ln[k], v[k]);
        }
        for (; i < m_end; ++i) {
            bool o[kSlots];
            uint32_t id[kSlots];
            float ln[kSlots];
            const float te = fmaf(jf, p.AM, p.t0M);
            jf += 1.0f;
            if constexpr (kEveryGeneral && !Op::kAllSlots)
                slab_general(p, sM, s, reg, te, o, id, ln);
            else if constexpr (kEveryGeneral)
                slab_general_g(p, sM, s, reg, te, o, id, ln);
            else if constexpr (!Op::kAllSlots)
                slab_fast(p, sM, s, reg, te, o, id, ln);
            else
                slab_fast_g(p, sM, s, reg, te, o, id, ln);
#pragma unroll
            for (int k = 0; k < kSlots; ++k) op(o[k], id[k], ln[k]);
        }
    };
    // slabs [i, stop) with the kSlots-segment body
    auto run = [&](int &i, int stop) {
        const int e1 = stop < lo_all ? stop : lo_all;
        for (; i < e1; ++i) edge(i, kEveryGeneral);
        const int m_end = stop < hi_all ? stop : hi_all;
        if (i < m_end) {
            if (kSplit && all_regular)
                middle(i, m_end, std::true_type());
            else
                middle(i, m_end, std::false_type());
        }
        for (; i < stop; ++i) edge(i, kEveryGeneral);
    };

    int i = 0;
    if constexpr (kEveryGeneral) {
        run(i, i_end);
        return;
    }
    // slab of the next a2 crossing (the first whose far plane lies beyond it)
    int j2 = (regular && s.t2 < p.chord) ? slab_past(p.AM, p.t0M, s.t2, false) : INT_MAX;
    int next = __reduce_min_sync(full, j2 < jend ? j0 + j2 : INT_MAX);
    while (i < i_end) {
        run(i, next < i_end ? next : i_end);
        if (i >= i_end) break;
        // slab i holds a crossing of a2 for at least one lane
        const int j = i - j0;
        const bool go = (unsigned)j < (unsigned)jend;
        const float te = fminf(fmaf((float)j, p.AM, p.t0M), p.chord);
        const bool c2 = go && s.t2 < te;
        bool o[3];
        uint32_t id[3];
        float ln[3];
        slab_general(p, sM, s, go, te, o, id, ln);
        op(o[0], id[0], ln[0]);
        op(o[1], id[1], ln[1]);
        op(o[2], id[2], ln[2]);
        if (c2) j2 = s.t2 < p.chord ? slab_past(p.AM, p.t0M, s.t2, false) : INT_MAX;
        ++i;
        next = __reduce_min_sync(full, j2 < jend ? j0 + j2 : INT_MAX);
    }
}

// The walk variant the image's hint selects (the hint is the same for the
// whole CTA, so every lane of a warp takes the same branch).  With an op
// whose kAllSlots is set (a gather that takes the bodies without slot
// predicates), a lane that is not regular walks safe_plane_ray() and its op
// is cleared afterwards (its sums stay 0).
template <int U = 1, class Op>
__device__ __forceinline__ void plane_walk_for(int hint, const PlaneRay &p_in,
                                               bool regular, Op &op)
{
    constexpr bool kAll = Op::kAllSlots;
    const PlaneRay p = (kAll && !regular) ? safe_plane_ray() : p_in;
    if (hint & kPlaneGeneralBit)
        plane_walk<true, U>(p, regular, op);
    else
        plane_walk<false, U>(p, regular, op);
    if constexpr (kAll)
        if (!regular) op.clear();
}

// Plane ops: fetch(on, off) loads what the segment needs (nothing for the
// scatters), apply(on, off, len, v) adds it; the walk's middle range issues
// the fetches of several slabs before their applies.  op(on, off, len) does
// both at once.  off is the voxel's byte offset from the op's buffer.

template <typename CubeT, bool kAll = true>
struct PlaneGatherOp {
    const CubeT *c;
    float acc;
    using Val = float;
    static constexpr bool kAllSlots = kAll;
    __device__ __forceinline__ void clear() { acc = 0.0f; }
    __device__ __forceinline__ float fetch(bool on, uint32_t off) const
    {
        return on ? load_voxel(byte_at(c, off), 0) : 0.0f;
    }
    __device__ __forceinline__ void apply(bool on, uint32_t, float len, float v)
    {
        if (on) acc = fmaf(len, v, acc);
    }
    __device__ __forceinline__ void operator()(bool on, uint32_t off, float len)
    {
        apply(on, off, len, fetch(on, off));
    }
};

template <typename CubeT>
struct PlaneGatherTimeOp {
    const CubeT *c0;
    const CubeT *c1;
    float w0, w1, acc;
    using Val = float2;
    // two loads a frame apart per slot, one slab per iteration: the
    // predicated bodies measured faster (22.9 against 29.7 ms, 8 frames)
    static constexpr bool kAllSlots = false;
    __device__ __forceinline__ void clear() { acc = 0.0f; }
    __device__ __forceinline__ float2 fetch(bool on, uint32_t off) const
    {
        return on ? make_float2(load_voxel(byte_at(c0, off), 0),
                                load_voxel(byte_at(c1, off), 0))
                  : make_float2(0.0f, 0.0f);
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

struct PlaneScatterOp {
    float *c;
    float y;
    using Val = NoVal;
    static constexpr bool kAllSlots = false;
    __device__ __forceinline__ NoVal fetch(bool, uint32_t) const { return NoVal(); }
    __device__ __forceinline__ void apply(bool on, uint32_t off, float len, NoVal)
    {
        red_add_if(on, byte_at(c, off), len * y);
    }
    __device__ __forceinline__ void operator()(bool on, uint32_t off, float len)
    {
        apply(on, off, len, NoVal());
    }
};

struct PlaneScatterTimeOp {
    float *c0;
    float *c1;
    float y0, y1;
    using Val = NoVal;
    static constexpr bool kAllSlots = false;
    __device__ __forceinline__ NoVal fetch(bool, uint32_t) const { return NoVal(); }
    __device__ __forceinline__ void apply(bool on, uint32_t off, float len, NoVal)
    {
        red_add_if(on, byte_at(c0, off), len * y0);
        red_add_if(on, byte_at(c1, off), len * y1);
    }
    __device__ __forceinline__ void operator()(bool on, uint32_t off, float len)
    {
        apply(on, off, len, NoVal());
    }
};

}  // namespace tomo
