// Ray setup: pointing records -> per-pixel Siddon walk records, in FP64.
//
// The observer sits ~215 solar radii from a cube a few radii wide, so the
// entry parameter of a ray is ~215 while a voxel is ~0.01: in float32 the
// entry point would be off by a sizeable fraction of a voxel.  Everything up
// to and including the entry point is therefore computed in double; the walk
// itself is then re-based to the entry point (t = 0 there), where float32
// keeps ~1e-7 relative precision over the whole chord.
//
// Geometry reading (the paper names the WCS keywords, Section 3.2, but gives
// no formulas): Sun-centred frame with z along the rotation axis; observer
// o = d (cos lat cos lon, cos lat sin lon, sin lat); boresight w = -o/|o|;
// e1 = unit(w x z), e2 = e1 x w, turned by the roll angle about w; gnomonic
// (TAN) pixel angles theta = (i - crpix) cdelt + crval per axis; ray
// direction unit(w + tan(theta_u) e1 + tan(theta_v) e2).
#include <math.h>

#include "tomo_internal.cuh"

namespace tomo {

namespace {

// Hint for the plane-synchronous walk of one image: M = the axis along
// which the line of sight of the image centre advances fastest, its
// direction, and L = the axis (other than M) along which neighbouring pixels
// of a row move at a fixed M plane.  Moving along the row turns the
// direction by ~e1; at a fixed M plane the ray through u + e1 d is displaced
// along e1 - u e1_M / u_M.  The hint is marked valid only when neighbouring
// pixels are at least rules.min_pitch voxels of L apart at the distance of
// Sun centre; the forward and walk-variant bits follow the other rules
// (defaults: the measured thresholds in tomo_internal.cuh; tomo_autotune
// can tune them per size bucket).  Only the walks' speed depends on the
// hint.
__device__ int32_t plane_hint(const tomo_pointing &p, const Frame &f, int nu,
                              int nv, double3 vox, const tomo_plane_rules &rules)
{
    const double tu = tan((0.5 * (nu - 1) - p.crpix_u) * p.cdelt_u + p.crval_u);
    const double tv = tan((0.5 * (nv - 1) - p.crpix_v) * p.cdelt_v + p.crval_v);
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = f.w[a] + tu * f.e1[a] + tv * f.e2[a];
    int M = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(u[a]) > fabs(u[M])) M = a;
    int L = -1;
    double best = -1.0;
    for (int a = 0; a < 3; ++a) {
        if (a == M) continue;
        const double lat = fabs(f.e1[a] - u[a] * f.e1[M] / u[M]);
        if (lat > best) {
            best = lat;
            L = a;
        }
    }
    const double dL = L == 0 ? vox.x : (L == 1 ? vox.y : vox.z);
    const double pitch = p.d_obs * fabs(tan(p.cdelt_u)) / dL;
    const bool valid = pitch >= rules.min_pitch;
    double lo = INFINITY;  // the less steep minor component
    for (int a = 0; a < 3; ++a)
        if (a != M) lo = fmin(lo, fabs(u[a]));
    lo /= fabs(u[M]);
    const bool general = lo >= rules.general_ratio;
    const bool fwd = valid && (pitch >= rules.fwd_min_pitch || lo < rules.fwd_max_ratio);
    return (valid ? kPlaneHintValid : 0) | (fwd ? kPlaneFwdBit : 0) |
           (general ? kPlaneGeneralBit : 0) | M | (L << 2) |
           ((u[M] < 0.0) ? 16 : 0);
}

// One block per image: the FP64 frame, the image parameters and the tangent
// tables tan(theta_u), tan(theta_v) (one value per column / row).
__global__ void k_frames(const tomo_pointing *__restrict__ ptg, int32_t nu,
                         int32_t nv, int32_t n_frames, Frame *frames,
                         double *tan_u, double *tan_v, ImgParam *params,
                         double3 vox, unsigned *layout_used,
                         unsigned *per_ray_fwd, tomo_plane_rules rules)
{
    const int img = blockIdx.x;
    const tomo_pointing p = ptg[img];
    if (threadIdx.x == 0) {
        Frame f;
        const double cl = cos(p.lat), sl = sin(p.lat);
        const double co = cos(p.lon), so = sin(p.lon);
        f.o[0] = p.d_obs * cl * co;
        f.o[1] = p.d_obs * cl * so;
        f.o[2] = p.d_obs * sl;
        f.w[0] = -cl * co;
        f.w[1] = -cl * so;
        f.w[2] = -sl;
        // w x z = (w_y, -w_x, 0), of length cos(lat)
        const double n1 = sqrt(f.w[0] * f.w[0] + f.w[1] * f.w[1]);
        const double a1[3] = { f.w[1] / n1, -f.w[0] / n1, 0.0 };
        const double a2[3] = { a1[1] * f.w[2] - a1[2] * f.w[1],
                               a1[2] * f.w[0] - a1[0] * f.w[2],
                               a1[0] * f.w[1] - a1[1] * f.w[0] };
        const double cr = cos(p.roll), sr = sin(p.roll);
        for (int a = 0; a < 3; ++a) {
            f.e1[a] = cr * a1[a] + sr * a2[a];
            f.e2[a] = -sr * a1[a] + cr * a2[a];
        }
        frames[img] = f;
        ImgParam q;
        q.gain = (float)p.gain;
        q.pad = plane_hint(p, f, nu, nv, vox, rules);
        if (layout_used && (q.pad & kPlaneHintValid)) {
            // bit L: a plane transpose uses layout L; bit 8 + L: so does a
            // plane forward
            const int L = (q.pad >> 2) & 3;
            atomicOr(layout_used, (1u << L) |
                                      ((q.pad & kPlaneFwdBit) ? 1u << (8 + L) : 0u));
        }
        if (per_ray_fwd && !(q.pad & kPlaneFwdBit))
            per_ray_fwd[1 + atomicAdd(per_ray_fwd, 1u)] = (unsigned)img;
        if (n_frames > 1) {
            int k = (int)floor(p.time);
            if (k > n_frames - 2) k = n_frames - 2;
            if (k < 0) k = 0;
            const double w = p.time - k;
            q.pad |= k << 8;
            q.w = (float)w;
            q.w0 = (float)(1.0 - w);
        } else {
            q.w = 0.0f;
            q.w0 = 1.0f;
        }
        params[img] = q;
    }
    for (int i = threadIdx.x; i < nu; i += blockDim.x)
        tan_u[(int64_t)img * nu + i] = tan((i - p.crpix_u) * p.cdelt_u + p.crval_u);
    for (int i = threadIdx.x; i < nv; i += blockDim.x)
        tan_v[(int64_t)img * nv + i] = tan((i - p.crpix_v) * p.cdelt_v + p.crval_v);
}

// Sign, zero and order tests of doubles on their bits.  This GPU's FP64
// pipe completes about two operations per clock per SM, and a double compare
// (also the one inside fmin / fmax) takes a slot of it like an FMA; the ray
// setup is bound by that pipe, while its integer pipe is nearly idle.  The
// tests below give the IEEE answer for every non-NaN input.
__device__ __forceinline__ bool d_sign(double x)  // sign bit (also -0.0)
{
    return __double2hiint(x) < 0;
}

__device__ __forceinline__ bool d_zero(double x)  // x == 0.0
{
    return (__double_as_longlong(x) << 1) == 0;
}

// An integer ordered like the doubles: a < b  <=>  d_key(a) < d_key(b), and
// -0.0 and +0.0 share a key.
__device__ __forceinline__ long long d_key(double x)
{
    const long long b = __double_as_longlong(x);
    return b < 0 ? -(b & 0x7fffffffffffffffLL) : b;
}

// One thread per pixel.  Slab clip of the half-line o + a u (a >= 0) in FP64,
// entry voxel by the half-open rule, then per-axis first crossing and
// crossing spacing relative to the entry point.
__global__ void k_ray_setup(const Frame *__restrict__ frames,
                            const double *__restrict__ tan_u,
                            const double *__restrict__ tan_v, CubeDev c,
                            int32_t nu, int32_t nv, RayRec *rays)
{
    const int img = blockIdx.y;
    const Frame &f = frames[img];
    // o - lo and o - hi, constants of the image: once per block
    __shared__ double s_olo[3], s_ohi[3];
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            s_olo[a] = f.o[a] - c.lo[a];
            s_ohi[a] = f.o[a] - c.hi[a];
        }
    }
    __syncthreads();
    const int64_t pix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (int64_t)nu * nv) return;
    const int iu = (int)(pix % nu), iv = (int)(pix / nu);
    const double tu = tan_u[(int64_t)img * nu + iu];
    const double tv = tan_v[(int64_t)img * nv + iv];
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = f.w[a] + tu * f.e1[a] + tv * f.e2[a];
    const double inv = rsqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < 3; ++a) u[a] *= inv;

    const int n[3] = { c.nx, c.ny, c.nz };
    bool zero[3], neg[3];  // u_a == 0, u_a < 0
    for (int a = 0; a < 3; ++a) {
        zero[a] = d_zero(u[a]);
        neg[a] = d_sign(u[a]) && !zero[a];
    }
    // one FP64 reciprocal per axis serves the clip and the crossing spacing
    double ru[3];
    for (int a = 0; a < 3; ++a) ru[a] = zero[a] ? 0.0 : 1.0 / u[a];
    // amin = max(0, near faces), amax = min(far faces), with their keys; the
    // near face of an axis is the lower one when u_a > 0 (lo < hi and the
    // rounded difference and product keep that order)
    double amin = 0.0, amax = INFINITY;
    long long kmin = d_key(amin), kmax = d_key(amax);
    bool hit = true;
    for (int a = 0; a < 3; ++a) {
        if (zero[a]) {
            const long long ko = d_key(f.o[a]);
            if (ko < d_key(c.lo[a]) || ko >= d_key(c.hi[a])) hit = false;
        } else {
            // (lo - o) ru, with lo - o = -(o - lo) exactly
            const double a0 = -(s_olo[a] * ru[a]);
            const double a1 = -(s_ohi[a] * ru[a]);
            const double near = neg[a] ? a1 : a0, far = neg[a] ? a0 : a1;
            const long long kn = d_key(near), kf = d_key(far);
            if (kn > kmin) {
                amin = near;
                kmin = kn;
            }
            if (kf < kmax) {
                amax = far;
                kmax = kf;
            }
        }
    }
    // Opaque sphere of radius r_obs at the origin (the photosphere): the
    // line of sight ends at its first point on the sphere (the paper stops
    // the integration there, Section 4).  Roots of |o + a u| = r: with p the
    // point of closest approach to the origin, a = -(o.u) -+ sqrt(r^2 -
    // |p|^2); |p|^2 is summed from p's components, which keeps the ~200-radii
    // observer distance out of the difference.  An observer inside the
    // sphere sees nothing.
    if (hit && c.r_obs > 0.0) {
        const double r2 = c.r_obs * c.r_obs;
        const double ou = f.o[0] * u[0] + f.o[1] * u[1] + f.o[2] * u[2];
        double oo = 0.0, pp = 0.0;
        for (int a = 0; a < 3; ++a) {
            oo += f.o[a] * f.o[a];
            const double pa = f.o[a] - ou * u[a];
            pp += pa * pa;
        }
        if (oo <= r2) {
            hit = false;
        } else if (pp < r2) {
            const double first = -ou - sqrt(r2 - pp);
            const long long kf = d_key(first);
            if (kf > 0 && kf < kmax) {
                amax = first;
                kmax = kf;
            }
        }
    }
    RayRec r;
    r.t0x = r.t0y = r.t0z = 0.0f;
    r.dtx = r.dty = r.dtz = 0.0f;
    r.idx0 = 0;
    r.chord = -1.0f;
    if (hit && kmin < kmax) {
        float chord = (float)(amax - amin);
        int idx[3];
        float t0f[3], dtf[3];
        for (int a = 0; a < 3; ++a) {
            // voxel coordinate of the entry point o + amin u
            const double g = fma(amin, u[a], s_olo[a]) * c.inv_d[a];
            // half-open voxels: floor(g), or ceil(g) - 1 walking down
            int ia = neg[a] ? __double2int_ru(g) - 1 : __double2int_rd(g);
            ia = ia < 0 ? 0 : (ia > n[a] - 1 ? n[a] - 1 : ia);
            idx[a] = ia;
            if (!zero[a]) {
                const bool pos = !neg[a];
                const double plane = (double)(pos ? ia + 1 : ia);
                const double dr = c.d[a] * ru[a];  // d_a / u_a
                const double t0 = (plane - g) * dr;
                const float dt = (float)fabs(dr);
                const int rem = pos ? n[a] - 1 - ia : ia;
                t0f[a] = d_sign(t0) ? 0.0f : (float)t0;
                // last in-cube plane of this axis, in the walk's arithmetic
                chord = fminf(chord, fmaf((float)rem, dt, t0f[a]));
                dtf[a] = pos ? dt : -dt;
            } else {
                t0f[a] = 1e30f;
                dtf[a] = 0.0f;
            }
        }
        if (chord > 0.0f) {
            r.t0x = t0f[0];
            r.t0y = t0f[1];
            r.t0z = t0f[2];
            r.dtx = dtf[0];
            r.dty = dtf[1];
            r.dtz = dtf[2];
            r.chord = chord;
            r.idx0 = (idx[2] * c.ny + idx[1]) * c.nx + idx[0];
        }
    }
    rays[(int64_t)img * nu * nv + pix] = r;
}

}  // namespace

cudaError_t launch_frames(const tomo_pointing *ptg_dev, int32_t n_img,
                          int32_t nu, int32_t nv, int32_t n_frames,
                          Frame *frames, double *tan_u, double *tan_v,
                          ImgParam *params, double3 vox,
                          unsigned *layout_used, unsigned *per_ray_fwd,
                          const tomo_plane_rules &rules, cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    k_frames<<<n_img, 128, 0, s>>>(ptg_dev, nu, nv, n_frames, frames, tan_u,
                                   tan_v, params, vox, layout_used,
                                   per_ray_fwd, rules);
    return cudaGetLastError();
}

cudaError_t launch_ray_setup(const Frame *frames, const double *tan_u,
                             const double *tan_v, CubeDev cube, int32_t n_img,
                             int32_t nu, int32_t nv, RayRec *rays,
                             cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    const int64_t npix = (int64_t)nu * nv;
    dim3 grid((unsigned)((npix + 255) / 256), (unsigned)n_img);
    k_ray_setup<<<grid, 256, 0, s>>>(frames, tan_u, tan_v, cube, nu, nv, rays);
    return cudaGetLastError();
}

}  // namespace tomo
