// Device-side Siddon walk shared by the single-problem and batched kernels.
//
// The walk is the incremental form of Siddon's method (Amanatides-Woo
// ordering): at every step the axis whose next voxel plane is nearest is
// crossed.  Crossing parameters are evaluated as t0 + k dt with one fused
// multiply-add (never accumulated), so every crossing carries a single
// float rounding relative to the entry point, and segment lengths, being
// differences of consecutive crossings, telescope to the chord.
#pragma once

#include "tomo_internal.cuh"

namespace tomo {

__device__ __forceinline__ RayRec load_ray(const RayRec *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    RayRec r;
    r.t0x = a.x;
    r.t0y = a.y;
    r.t0z = a.z;
    r.chord = a.w;
    r.dtx = b.x;
    r.dty = b.y;
    r.dtz = b.z;
    r.idx0 = __float_as_int(b.w);
    return r;
}

// Map this thread to a pixel of tile (tu, tv) of an image; false past the
// image edge.  A warp covers warp_u x (32 / warp_u) pixels.
__device__ __forceinline__ bool pixel_of_thread(const Tiling t, int tu, int tv,
                                                int nu, int nv, int &iu,
                                                int &iv)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows = 32 / t.warp_u;
    const int warps_u = t.tile_u / t.warp_u;
    iu = tu * t.tile_u + (warp % warps_u) * t.warp_u + (lane % t.warp_u);
    iv = tv * t.tile_v + (warp / warps_u) * rows + (lane / t.warp_u);
    return iu < nu && iv < nv;
}

// Walk one ray; op(idx, len) is called for every step, including steps of
// zero length at ties (two planes crossed at the same parameter).  The loop
// ends after at most (#planes inside the cube + 1) steps: each step that does
// not end the walk advances one axis, and no axis can advance past its last
// in-cube plane because the setup kernel capped the chord there.
template <class Op>
__device__ __forceinline__ void siddon_walk(const RayRec &r, int nx, int nxny,
                                            Op &op)
{
    const float chord = r.chord;
    const float ax = fabsf(r.dtx), ay = fabsf(r.dty), az = fabsf(r.dtz);
    const int sx = signbit(r.dtx) ? -1 : 1;
    const int sy = signbit(r.dty) ? -nx : nx;
    const int sz = signbit(r.dtz) ? -nxny : nxny;
    float kx = 0.0f, ky = 0.0f, kz = 0.0f;
    float tx = r.t0x, ty = r.t0y, tz = r.t0z;
    float t = 0.0f;
    int idx = r.idx0;
    for (;;) {
        const float tm = fminf(tx, fminf(ty, tz));
        const float te = fminf(tm, chord);
        op(idx, te - t);
        if (te >= chord) break;
        t = te;
        if (tx == tm) {
            kx += 1.0f;
            tx = fmaf(kx, ax, r.t0x);
            idx += sx;
        } else if (ty == tm) {
            ky += 1.0f;
            ty = fmaf(ky, ay, r.t0y);
            idx += sy;
        } else {
            kz += 1.0f;
            tz = fmaf(kz, az, r.t0z);
            idx += sz;
        }
    }
}

// siddon_walk for gathering ops, with the load of each segment's voxel
// issued before the previous segment's product is added: op.fetch(idx)
// loads, op.apply(len, v) adds.  Same segments and the same order of
// additions as siddon_walk (so the same sums, bit for bit); one load is
// always in flight while the walk computes the next crossing.
template <class Op>
__device__ __forceinline__ void siddon_gather(const RayRec &r, int nx, int nxny,
                                              Op &op)
{
    const float chord = r.chord;
    const float ax = fabsf(r.dtx), ay = fabsf(r.dty), az = fabsf(r.dtz);
    const int sx = signbit(r.dtx) ? -1 : 1;
    const int sy = signbit(r.dty) ? -nx : nx;
    const int sz = signbit(r.dtz) ? -nxny : nxny;
    float kx = 0.0f, ky = 0.0f, kz = 0.0f;
    float tx = r.t0x, ty = r.t0y, tz = r.t0z;
    int idx = r.idx0;
    float tm = fminf(tx, fminf(ty, tz));
    float te = fminf(tm, chord);
    typename Op::Val v = op.fetch(idx);
    float len = te;
    while (te < chord) {
        const float t = te;
        if (tx == tm) {
            kx += 1.0f;
            tx = fmaf(kx, ax, r.t0x);
            idx += sx;
        } else if (ty == tm) {
            ky += 1.0f;
            ty = fmaf(ky, ay, r.t0y);
            idx += sy;
        } else {
            kz += 1.0f;
            tz = fmaf(kz, az, r.t0z);
            idx += sz;
        }
        tm = fminf(tx, fminf(ty, tz));
        te = fminf(tm, chord);
        const typename Op::Val vn = op.fetch(idx);
        op.apply(len, v);
        v = vn;
        len = te - t;
    }
    op.apply(len, v);
}

// Fire-and-forget float addition into global memory (PTX red.global).
// atomicAdd through a pointer whose address space the compiler cannot infer
// (one read from a descriptor in global memory, as in the batched kernels)
// compiles to a generic atomic that returns the old value; measured on
// GB300 that made the batched transposes wait on every addition.  The
// pointer must point to global memory (every caller passes a cube or
// accumulator allocated with cudaMalloc).
__device__ __forceinline__ void red_add(float *p, float v)
{
    asm volatile("red.global.add.f32 [%0], %1;"
                 :
                 : "l"(__cvta_generic_to_global(p)), "f"(v)
                 : "memory");
}

// red_add under a predicate, as one predicated instruction: a lane-varying
// `if (on) red_add(...)` compiles to a divergent branch around the
// reduction, which the plane walks would pay for every segment slot.
__device__ __forceinline__ void red_add_if(bool on, float *p, float v)
{
    asm volatile("{\n\t.reg .pred q;\n\t"
                 "setp.ne.b32 q, %2, 0;\n\t"
                 "@q red.global.add.f32 [%0], %1;\n\t}"
                 :
                 : "l"(__cvta_generic_to_global(p)), "f"(v), "r"((int)on)
                 : "memory");
}

__device__ __forceinline__ float load_voxel(const float *c, int idx)
{
    return __ldg(c + idx);
}

__device__ __forceinline__ float load_voxel(const uint16_t *c, int idx)
{
    // bfloat16 -> float32 is exact: the bf16 bits are the top half
    return __uint_as_float(((uint32_t)__ldg(c + idx)) << 16);
}

template <typename CubeT>
struct GatherOp {
    const CubeT *c;
    float acc;
    using Val = float;
    __device__ __forceinline__ float fetch(int idx) const
    {
        return load_voxel(c, idx);
    }
    __device__ __forceinline__ void apply(float len, float v)
    {
        acc = fmaf(len, v, acc);
    }
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        acc = fmaf(len, load_voxel(c, idx), acc);
    }
};

template <typename CubeT>
struct GatherTimeOp {
    const CubeT *c0;
    const CubeT *c1;
    float w0, w1, acc;
    using Val = float2;
    __device__ __forceinline__ float2 fetch(int idx) const
    {
        return make_float2(load_voxel(c0, idx), load_voxel(c1, idx));
    }
    __device__ __forceinline__ void apply(float len, float2 v)
    {
        acc = fmaf(len, fmaf(w0, v.x, w1 * v.y), acc);
    }
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        const float v = fmaf(w0, load_voxel(c0, idx), w1 * load_voxel(c1, idx));
        acc = fmaf(len, v, acc);
    }
};

// Scatter of one segment, len * y, into voxel idx.  Neighbouring lanes walk
// neighbouring rays of one observer and are often in the same voxel at the
// same step; before the float atomic, contributions of lanes that hold the
// same voxel are summed along a small shuffle tree (partner lanes at lane
// distance 1, 2 and 8: neighbours along u, and the next pixel row for the
// default 8 x 4 warp tile), so one lane issues the atomic for the group.
// The equality test makes it correct for any lane layout; it only pays when
// neighbours coincide.  The sum is the same up to the order of additions.
struct ScatterOp {
    float *c;
    float y;
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        float v = (len > 0.0f) ? len * y : 0.0f;
        const unsigned act = __activemask();
        const int lane = threadIdx.x & 31;
        int key = (len > 0.0f) ? idx : -1 - lane;  // idle lanes never match
#pragma unroll
        for (int lvl = 0; lvl < 3; ++lvl) {
            const int o = lvl == 0 ? 1 : (lvl == 1 ? 2 : 8);
            const bool partner_active = (act >> (lane ^ o)) & 1u;
            const int pk = __shfl_xor_sync(act, key, o);
            const float pv = __shfl_xor_sync(act, v, o);
            if (partner_active && pk == key) {
                if (lane & o) {
                    v = 0.0f;
                    key = -1 - lane;
                } else {
                    v += pv;
                }
            }
        }
        red_add_if(v != 0.0f, c + idx, v);
    }
};

struct ScatterTimeOp {
    float *c0;
    float *c1;
    float y0, y1;
    __device__ __forceinline__ void operator()(int idx, float len)
    {
        red_add_if(len > 0.0f, c0 + idx, len * y0);
        red_add_if(len > 0.0f, c1 + idx, len * y1);
    }
};

struct CountOp {
    unsigned int n;
    __device__ __forceinline__ void operator()(int, float len)
    {
        n += (len > 0.0f) ? 1u : 0u;
    }
};

}  // namespace tomo
