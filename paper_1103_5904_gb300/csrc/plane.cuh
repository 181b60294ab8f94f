// Plane-synchronous Siddon walk: per-ray setup, the warp-wide walk and its
// segment operations, shared by the single-problem kernels (plane.cu) and
// the batched transpose (batch.cu).  The design and its exactness argument
// are described at the top of plane.cu.
#pragma once

#include <limits.h>
#include <math.h>

#include "walk.cuh"

namespace tomo {

// One ray, re-expressed for the plane walk: M first, then the two minor
// axes, a1 the one with the smaller crossing spacing (crossed more often).
struct PlaneRay {
    float t0M, t01, t02;  // first crossings
    float AM, A1, A2;     // crossing spacings
    float chord;
    int sM, s1, s2;       // signed strides in the image's layout
    int idx;              // entry voxel in the image's layout
    int key;              // entry M coordinate, signed by the M direction
};

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

// Fills p and returns true when the ray fits the plane walk of its image.
__device__ __forceinline__ bool plane_ray(const RayRec &r, int hint, int nx,
                                          int ny, int nz, PlaneRay &p)
{
    if (!(hint & kPlaneHintValid)) return false;
    const int M = hint & 3, L = (hint >> 2) & 3;
    const bool neg = (hint >> 4) & 1;
    const int cx = r.idx0 % nx;
    const int rest = r.idx0 / nx;
    const int cy = rest % ny, cz = rest / ny;
    int stx, sty, stz;
    layout_strides(L, nx, ny, nz, stx, sty, stz);
    const int gx = signbit(r.dtx) ? -stx : stx;
    const int gy = signbit(r.dty) ? -sty : sty;
    const int gz = signbit(r.dtz) ? -stz : stz;
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
        const int g = p.s1;
        p.s1 = p.s2;
        p.s2 = g;
    }
    p.chord = r.chord;
    p.idx = cx * stx + cy * sty + cz * stz;
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

// Walks the regular lanes of the warp plane by plane; op(on, idx, len) is
// called for every segment with on == true (len may be 0 at ties, which adds
// an exact zero) and, with on == false, for slots without a segment (idx
// then may lie outside the cube and must not be touched).  Every lane of the
// warp must call this (it uses warp-wide reductions); lanes with regular ==
// false only take part in those.
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
template <bool kEveryGeneral, class Op>
__device__ __forceinline__ void plane_walk(const PlaneRay &p, bool regular,
                                           Op &op)
{
    const unsigned full = 0xffffffffu;
    const int kmin = __reduce_min_sync(full, regular ? p.key : INT_MAX);
    const int j0 = regular ? p.key - kmin : 0;
    // the walk ends in the first slab whose far plane reaches the chord
    const int jend = regular ? 1 + slab_past(p.AM, p.t0M, p.chord, true) : 0;
    const int i_end = __reduce_max_sync(full, regular ? j0 + jend : 0);
    float t = 0.0f, k1 = 0.0f, k2 = 0.0f;
    float t1 = p.t01, t2 = p.t02;
    int idx = p.idx;
    if (kEveryGeneral) {
        for (int i = 0; i < i_end; ++i) {
            const int j = i - j0;
            const bool go = (unsigned)j < (unsigned)jend;
            const float te = fminf(fmaf((float)j, p.AM, p.t0M), p.chord);
            const bool first1 = t1 <= t2;
            const float ta = first1 ? t1 : t2;
            const float tb = first1 ? t2 : t1;
            const int sa = first1 ? p.s1 : p.s2;
            op(go, idx, fminf(ta, te) - t);
            op(go && ta < te, idx + sa, fminf(tb, te) - ta);
            op(go && tb < te, idx + p.s1 + p.s2, te - tb);
            const bool c1 = go && t1 < te, c2 = go && t2 < te;
            k1 = c1 ? k1 + 1.0f : k1;
            k2 = c2 ? k2 + 1.0f : k2;
            t1 = c1 ? fmaf(k1, p.A1, p.t01) : t1;
            t2 = c2 ? fmaf(k2, p.A2, p.t02) : t2;
            idx += (c1 ? p.s1 : 0) + (c2 ? p.s2 : 0) + (go ? p.sM : 0);
            t = go ? te : t;
        }
        return;
    }
    // slab of the next a2 crossing (the first whose far plane lies beyond it)
    int j2 = (regular && t2 < p.chord) ? slab_past(p.AM, p.t0M, t2, false) : INT_MAX;
    int next = __reduce_min_sync(full, j2 < jend ? j0 + j2 : INT_MAX);
    int i = 0;
    while (i < i_end) {
        const int stop = next < i_end ? next : i_end;
        for (; i < stop; ++i) {
            const int j = i - j0;
            const bool go = (unsigned)j < (unsigned)jend;
            const float te = fminf(fmaf((float)j, p.AM, p.t0M), p.chord);
            const bool c1 = go && t1 < te;
            op(go, idx, fminf(t1, te) - t);
            op(c1, idx + p.s1, te - t1);
            k1 = c1 ? k1 + 1.0f : k1;
            t1 = c1 ? fmaf(k1, p.A1, p.t01) : t1;
            idx += (c1 ? p.s1 : 0) + (go ? p.sM : 0);
            t = go ? te : t;
        }
        if (i >= i_end) break;
        // slab i holds a crossing of a2 for at least one lane
        const int j = i - j0;
        const bool go = (unsigned)j < (unsigned)jend;
        const float te = fminf(fmaf((float)j, p.AM, p.t0M), p.chord);
        const bool first1 = t1 <= t2;
        const float ta = first1 ? t1 : t2;
        const float tb = first1 ? t2 : t1;
        const int sa = first1 ? p.s1 : p.s2;
        op(go, idx, fminf(ta, te) - t);
        op(go && ta < te, idx + sa, fminf(tb, te) - ta);
        op(go && tb < te, idx + p.s1 + p.s2, te - tb);
        const bool c1 = go && t1 < te, c2 = go && t2 < te;
        k1 = c1 ? k1 + 1.0f : k1;
        k2 = c2 ? k2 + 1.0f : k2;
        t1 = c1 ? fmaf(k1, p.A1, p.t01) : t1;
        t2 = c2 ? fmaf(k2, p.A2, p.t02) : t2;
        idx += (c1 ? p.s1 : 0) + (c2 ? p.s2 : 0) + (go ? p.sM : 0);
        t = go ? te : t;
        if (c2) j2 = t2 < p.chord ? slab_past(p.AM, p.t0M, t2, false) : INT_MAX;
        ++i;
        next = __reduce_min_sync(full, j2 < jend ? j0 + j2 : INT_MAX);
    }
}

// The walk variant the image's hint selects (the hint is the same for the
// whole CTA, so every lane of a warp takes the same branch).
template <class Op>
__device__ __forceinline__ void plane_walk_for(int hint, const PlaneRay &p,
                                               bool regular, Op &op)
{
    if (hint & kPlaneGeneralBit)
        plane_walk<true>(p, regular, op);
    else
        plane_walk<false>(p, regular, op);
}

template <typename CubeT>
struct PlaneGatherOp {
    const CubeT *c;
    float acc;
    __device__ __forceinline__ void operator()(bool on, int idx, float len)
    {
        if (on) acc = fmaf(len, load_voxel(c, idx), acc);
    }
};

template <typename CubeT>
struct PlaneGatherTimeOp {
    const CubeT *c0;
    const CubeT *c1;
    float w0, w1, acc;
    __device__ __forceinline__ void operator()(bool on, int idx, float len)
    {
        if (on) {
            const float v = fmaf(w0, load_voxel(c0, idx), w1 * load_voxel(c1, idx));
            acc = fmaf(len, v, acc);
        }
    }
};

struct PlaneScatterOp {
    float *c;
    float y;
    __device__ __forceinline__ void operator()(bool on, int idx, float len)
    {
        if (on) red_add(c + idx, len * y);
    }
};

struct PlaneScatterTimeOp {
    float *c0;
    float *c1;
    float y0, y1;
    __device__ __forceinline__ void operator()(bool on, int idx, float len)
    {
        if (on) {
            red_add(c0 + idx, len * y0);
            red_add(c1 + idx, len * y1);
        }
    }
};

}  // namespace tomo
