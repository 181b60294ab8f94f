// Transpose P^T driven by cube tiles: no global atomics.
//
// x_j = sum_k g_k y_k P_{k,j} (Eq. lo transposed).  A CTA owns one tile of
// kTile^3 voxels and accumulates it in shared memory over every image:
// for image n it projects the tile's eight corners into the image (central
// projection keeps the box's image convex, and the pixel grid is uniform in
// angle, so the corners' angle ranges give the exact pixel bounding box; one
// pixel of margin absorbs rounding), and for every pixel in that box it
// walks the pixel's ray through the tile only.
//
// The walk restarts at the ray's entry into the tile with the crossing
// counts it would have there in the full walk: crossing k of axis a is at
// fmaf(k, |dt_a|, t0_a) in both, so every segment length is bitwise the one
// the forward projection uses and the result is its exact transpose (up to
// the order of the float additions).  Each voxel belongs to one CTA, which
// adds its total to the cube with one plain read-modify-write.
#include <math.h>

#include "walk.cuh"

namespace tomo {

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 16;

// Tile slab of one axis, in crossing counts: the ray's index along the axis
// is inside [I0, I1) for crossing counts m in [m_lo, m_hi].  Returns false
// if the ray never enters the slab.  t_lo / t_hi bound the slab in t.
__device__ __forceinline__ bool slab(int i0, int s, float a, float t0, int I0,
                                     int I1, int &m_lo, int &m_hi, float &t_lo,
                                     float &t_hi)
{
    if (!(a > 0.0f)) {  // parallel to this axis' planes: index fixed
        m_lo = 0;
        m_hi = 0;
        t_lo = 0.0f;
        t_hi = INFINITY;
        return i0 >= I0 && i0 < I1;
    }
    if (s > 0) {
        m_lo = I0 - i0;
        m_hi = I1 - 1 - i0;
    } else {
        m_lo = i0 - (I1 - 1);
        m_hi = i0 - I0;
    }
    if (m_hi < 0) return false;
    if (m_lo < 0) m_lo = 0;
    t_lo = (m_lo == 0) ? 0.0f : fmaf((float)(m_lo - 1), a, t0);
    t_hi = fmaf((float)m_hi, a, t0);
    return true;
}

// Number of crossings of one axis at or before T (in [m_lo, m_hi + 1]).
__device__ __forceinline__ int crossings_done(float a, float t0, int m_lo,
                                              int m_hi, float T)
{
    if (!(a > 0.0f)) return 0;
    int k = m_lo;
    const float est = floorf((T - t0) / a) + 1.0f;
    if (est > (float)k) k = est < (float)(m_hi + 1) ? (int)est : m_hi + 1;
    while (k > m_lo && fmaf((float)(k - 1), a, t0) > T) --k;
    while (k <= m_hi && fmaf((float)k, a, t0) <= T) ++k;
    return k;
}

__global__ void __launch_bounds__(kThreads)
k_adjoint_tiled(const RayRec *__restrict__ rays,
                const ImgParam *__restrict__ prm,
                const Frame *__restrict__ frames,
                const tomo_pointing *__restrict__ ptg,
                const float *__restrict__ images,
                const uint8_t *__restrict__ mask, float *__restrict__ cube,
                CubeDev c, int n_img, int nu, int nv,
                const double *__restrict__ done)
{
    __shared__ float acc[kTile * kTile * kTile];
    __shared__ float s_u[8], s_v[8];
    __shared__ int s_fail;
    __shared__ int s_box[4];
    if (done != nullptr && *done != 0.0) return;
    const int tid = threadIdx.x;
    const int nx = c.nx, ny = c.ny, nz = c.nz, nxny = nx * ny;
    const int I0x = blockIdx.x * kTile, I0y = blockIdx.y * kTile,
              I0z = blockIdx.z * kTile;
    const int I1x = min(I0x + kTile, nx), I1y = min(I0y + kTile, ny),
              I1z = min(I0z + kTile, nz);
    const int tx_ = I1x - I0x, ty_ = I1y - I0y;  // local extents (x, y)
    for (int i = tid; i < kTile * kTile * kTile; i += kThreads) acc[i] = 0.0f;

    for (int n = 0; n < n_img; ++n) {
        if (tid == 0) s_fail = 0;
        __syncthreads();  // previous image's pixels are all done
        if (tid < 8) {
            const Frame &f = frames[n];
            const double px = c.lo[0] + ((tid & 1) ? I1x : I0x) * c.d[0];
            const double py = c.lo[1] + ((tid & 2) ? I1y : I0y) * c.d[1];
            const double pz = c.lo[2] + ((tid & 4) ? I1z : I0z) * c.d[2];
            const double dx = px - f.o[0], dy = py - f.o[1], dz = pz - f.o[2];
            const double xw = dx * f.w[0] + dy * f.w[1] + dz * f.w[2];
            const double x1 = dx * f.e1[0] + dy * f.e1[1] + dz * f.e1[2];
            const double x2 = dx * f.e2[0] + dy * f.e2[1] + dz * f.e2[2];
            if (!(xw > 1e-9 * (fabs(x1) + fabs(x2) + 1e-30))) {
                s_fail = 1;  // corner at or behind the observer
            } else {
                const tomo_pointing p = ptg[n];
                s_u[tid] = (float)((atan(x1 / xw) - p.crval_u) / p.cdelt_u + p.crpix_u);
                s_v[tid] = (float)((atan(x2 / xw) - p.crval_v) / p.cdelt_v + p.crpix_v);
            }
        }
        __syncthreads();
        if (tid == 0) {
            int u0 = 0, u1 = nu - 1, v0 = 0, v1 = nv - 1;
            if (!s_fail) {
                float umin = s_u[0], umax = s_u[0], vmin = s_v[0], vmax = s_v[0];
                for (int k = 1; k < 8; ++k) {
                    umin = fminf(umin, s_u[k]);
                    umax = fmaxf(umax, s_u[k]);
                    vmin = fminf(vmin, s_v[k]);
                    vmax = fmaxf(vmax, s_v[k]);
                }
                // clamp in float first: the box may lie far outside the image
                umin = fmaxf(floorf(umin) - 1.0f, 0.0f);
                vmin = fmaxf(floorf(vmin) - 1.0f, 0.0f);
                umax = fminf(ceilf(umax) + 1.0f, (float)(nu - 1));
                vmax = fminf(ceilf(vmax) + 1.0f, (float)(nv - 1));
                u0 = (int)umin;
                v0 = (int)vmin;
                u1 = umax >= umin ? (int)umax : u0 - 1;
                v1 = vmax >= vmin ? (int)vmax : v0 - 1;
            }
            s_box[0] = u0;
            s_box[1] = u1;
            s_box[2] = v0;
            s_box[3] = v1;
        }
        __syncthreads();
        const int u0 = s_box[0], v0 = s_box[2];
        const int bw = s_box[1] - u0 + 1, bh = s_box[3] - v0 + 1;
        if (bw <= 0 || bh <= 0) continue;
        const float gain = prm[n].gain;
        const int npx = bw * bh;
        for (int q = tid; q < npx; q += kThreads) {
            const int iu = u0 + q % bw, iv = v0 + q / bw;
            const int64_t id = ((int64_t)n * nv + iv) * nu + iu;
            if (mask != nullptr && mask[id] != 0) continue;
            const float yv = gain * images[id];
            if (yv == 0.0f) continue;
            const RayRec r = load_ray(rays + id);
            if (!(r.chord > 0.0f)) continue;
            const float ax = fabsf(r.dtx), ay = fabsf(r.dty), az = fabsf(r.dtz);
            const int sx = signbit(r.dtx) ? -1 : 1, sy = signbit(r.dty) ? -1 : 1,
                      sz = signbit(r.dtz) ? -1 : 1;
            const int i0x = r.idx0 % nx, i0y = (r.idx0 / nx) % ny,
                      i0z = r.idx0 / nxny;
            int mlx, mhx, mly, mhy, mlz, mhz;
            float tlx, thx, tly, thy, tlz, thz;
            if (!slab(i0x, sx, ax, r.t0x, I0x, I1x, mlx, mhx, tlx, thx) ||
                !slab(i0y, sy, ay, r.t0y, I0y, I1y, mly, mhy, tly, thy) ||
                !slab(i0z, sz, az, r.t0z, I0z, I1z, mlz, mhz, tlz, thz))
                continue;
            const float T_in = fmaxf(tlx, fmaxf(tly, tlz));
            const float T_out = fminf(r.chord, fminf(thx, fminf(thy, thz)));
            if (!(T_in < T_out)) continue;
            // walk state at T_in: every crossing at or before T_in is done
            float kx = (float)crossings_done(ax, r.t0x, mlx, mhx, T_in);
            float ky = (float)crossings_done(ay, r.t0y, mly, mhy, T_in);
            float kz = (float)crossings_done(az, r.t0z, mlz, mhz, T_in);
            const int lx = i0x + sx * (int)kx - I0x;
            const int ly = i0y + sy * (int)ky - I0y;
            const int lz = i0z + sz * (int)kz - I0z;
            if ((unsigned)lx >= (unsigned)(I1x - I0x) ||
                (unsigned)ly >= (unsigned)(I1y - I0y) ||
                (unsigned)lz >= (unsigned)(I1z - I0z))
                continue;  // cannot happen: kept as a guard of the index
            int li = (lz * ty_ + ly) * tx_ + lx;
            const int stx = sx, sty = sy * tx_, stz = sz * tx_ * ty_;
            float tnx = ax > 0.0f ? fmaf(kx, ax, r.t0x) : INFINITY;
            float tny = ay > 0.0f ? fmaf(ky, ay, r.t0y) : INFINITY;
            float tnz = az > 0.0f ? fmaf(kz, az, r.t0z) : INFINITY;
            float t = T_in;
            for (;;) {
                const float tm = fminf(tnx, fminf(tny, tnz));
                const float te = fminf(tm, T_out);
                const float len = te - t;
                if (len > 0.0f) atomicAdd(&acc[li], len * yv);
                if (te >= T_out) break;
                t = te;
                if (tnx == tm) {
                    kx += 1.0f;
                    tnx = fmaf(kx, ax, r.t0x);
                    li += stx;
                } else if (tny == tm) {
                    ky += 1.0f;
                    tny = fmaf(ky, ay, r.t0y);
                    li += sty;
                } else {
                    kz += 1.0f;
                    tnz = fmaf(kz, az, r.t0z);
                    li += stz;
                }
            }
        }
    }
    __syncthreads();
    const int nloc = tx_ * ty_ * (I1z - I0z);
    for (int i = tid; i < nloc; i += kThreads) {
        const int lx = i % tx_, ly = (i / tx_) % ty_, lz = i / (tx_ * ty_);
        const float v = acc[i];
        if (v != 0.0f) {
            float *dst = cube + ((int64_t)(I0z + lz) * ny + (I0y + ly)) * nx + I0x + lx;
            *dst += v;
        }
    }
}

}  // namespace

cudaError_t launch_adjoint_tiled(const RayRec *rays, const ImgParam *prm,
                                 const Frame *frames, const tomo_pointing *ptg,
                                 const float *images, const uint8_t *mask,
                                 float *cube, CubeDev c, int32_t n_img,
                                 int32_t nu, int32_t nv, const double *done,
                                 cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((c.nx + kTile - 1) / kTile),
                    (unsigned)((c.ny + kTile - 1) / kTile),
                    (unsigned)((c.nz + kTile - 1) / kTile));
    k_adjoint_tiled<<<grid, kThreads, 0, s>>>(rays, prm, frames, ptg, images,
                                              mask, cube, c, n_img, nu, nv,
                                              done);
    return cudaGetLastError();
}

}  // namespace tomo
