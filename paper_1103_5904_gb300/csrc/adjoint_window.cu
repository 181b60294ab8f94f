// Transpose P^T with per-bundle shared-memory accumulation.
//
// P^T spreads g y_k over the voxels crossed by ray k, weighted by the
// segment lengths (the exact transpose of Eq. lo).  Done with one float atomic
// per segment into the cube, the L2 atomic units are the bottleneck: a voxel
// is crossed by several neighbouring rays of the same image, and each of
// their updates is a separate read-modify-write in L2.
//
// Here a CTA walks a bundle of rays that leave one observer through a
// compact pixel tile.  Their walks are cut into chunks of kDepth voxel planes
// along the bundle's major axis.  For every chunk the CTA bounds the voxels
// its rays can reach (from each ray's current voxel and the ratio of its
// plane spacings), accumulates the chunk's segments into a window of shared
// memory with shared-memory atomics, and then adds only the nonzero window
// entries to the cube, row by row.  A segment that falls outside the window,
// a window larger than shared memory, and rays that do not advance along the
// major axis in the bundle's direction all fall back to a global atomic, so
// the result never depends on the bound being tight.  Segment lengths are
// computed exactly as in the plain walk; only the order of the additions
// changes.
#include <limits.h>
#include <math.h>

#include "walk.cuh"

namespace tomo {

namespace {

constexpr int kThreads = 256;
constexpr int kDepth = 16;    // major-axis planes per chunk
constexpr int kWinCap = 8192; // floats of shared memory per window (32 KB)

__device__ __forceinline__ int crossings_within(float dist, float a, int n)
{
    // planes of spacing a met within distance dist from any start point
    if (!(a > 0.0f)) return 0;
    const float c = ceilf(dist / a) + 1.0f;
    return c < (float)n ? (int)c : n;
}

__global__ void __launch_bounds__(kThreads)
k_adjoint_window(const RayRec *__restrict__ rays,
                 const ImgParam *__restrict__ prm,
                 const float *__restrict__ images,
                 const uint8_t *__restrict__ mask, float *__restrict__ cube,
                 int nu, int nv, int nx, int ny, int nz, Tiling tl,
                 const double *__restrict__ done)
{
    __shared__ float win[kWinCap];
    __shared__ int s_lo[3], s_hi[3];
    __shared__ int s_major, s_chunk;
    if (done != nullptr && *done != 0.0) return;
    const int tid = threadIdx.x;
    if (tid == 0) s_major = -1;
    __syncthreads();

    int iu, iv;
    const bool in_img = pixel_of_thread(tl, blockIdx.x, blockIdx.y, nu, nv, iu, iv);
    const int img = blockIdx.z;
    bool active = false;
    float yv = 0.0f;
    RayRec r;
    r.chord = -1.0f;
    if (in_img) {
        const int64_t id = ((int64_t)img * nv + iv) * nu + iu;
        if (mask == nullptr || mask[id] == 0) {
            yv = prm[img].gain * images[id];
            if (yv != 0.0f) {
                r = load_ray(rays + id);
                active = r.chord > 0.0f;
            }
        }
    }
    const int nxny = nx * ny;
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
    int sx = 1, sy = 1, sz = 1;
    int ix = 0, iy = 0, iz = 0, idx = 0;
    float kx = 0.0f, ky = 0.0f, kz = 0.0f, t = 0.0f;
    float tx = 0.0f, ty = 0.0f, tz = 0.0f;
    if (active) {
        ax = fabsf(r.dtx);
        ay = fabsf(r.dty);
        az = fabsf(r.dtz);
        sx = signbit(r.dtx) ? -1 : 1;
        sy = signbit(r.dty) ? -1 : 1;
        sz = signbit(r.dtz) ? -1 : 1;
        idx = r.idx0;
        ix = idx % nx;
        iy = (idx / nx) % ny;
        iz = idx / nxny;
        tx = r.t0x;
        ty = r.t0y;
        tz = r.t0z;
        // dominant axis of this ray (smallest plane spacing) and direction
        int dom = 0;
        float best = ax > 0.0f ? ax : INFINITY;
        if (ay > 0.0f && ay < best) { dom = 1; best = ay; }
        if (az > 0.0f && az < best) dom = 2;
        const int sd = dom == 0 ? sx : (dom == 1 ? sy : sz);
        atomicCAS(&s_major, -1, 2 * dom + (sd > 0 ? 1 : 0));
    }
    __syncthreads();
    const int code = s_major;
    if (code < 0) return;  // no live ray in this CTA (uniform)
    const int M = code >> 1;
    const int dirM = (code & 1) ? 1 : -1;
    const int nM = M == 0 ? nx : (M == 1 ? ny : nz);
    const float aM = M == 0 ? ax : (M == 1 ? ay : az);
    const int sM = M == 0 ? sx : (M == 1 ? sy : sz);

    // One step of the walk: the segment in the current voxel, then the
    // crossing of the nearest plane.  Returns false when the ray has ended.
    auto step = [&](bool use_win, int lx, int ly, int lz, int wx, int wy,
                    int wz, int &mp) -> bool {
        const float tm = fminf(tx, fminf(ty, tz));
        const float te = fminf(tm, r.chord);
        const float len = te - t;
        if (len > 0.0f) {
            const float v = len * yv;
            const unsigned ux = (unsigned)(ix - lx), uy = (unsigned)(iy - ly),
                           uz = (unsigned)(iz - lz);
            if (use_win && ux < (unsigned)wx && uy < (unsigned)wy &&
                uz < (unsigned)wz)
                atomicAdd(&win[((int)uz * wy + (int)uy) * wx + (int)ux], v);
            else
                atomicAdd(cube + idx, v);
        }
        if (te >= r.chord) return false;
        t = te;
        if (tx == tm) {
            kx += 1.0f;
            tx = fmaf(kx, ax, r.t0x);
            ix += sx;
            idx += sx;
            if (M == 0) ++mp;
        } else if (ty == tm) {
            ky += 1.0f;
            ty = fmaf(ky, ay, r.t0y);
            iy += sy;
            idx += sy * nx;
            if (M == 1) ++mp;
        } else {
            kz += 1.0f;
            tz = fmaf(kz, az, r.t0z);
            iz += sz;
            idx += sz * nxny;
            if (M == 2) ++mp;
        }
        return true;
    };

    // rays that do not advance along the major axis in the bundle's
    // direction are walked at once with global atomics
    int mp = 0;  // major coordinate in the bundle's travel order
    if (active) {
        const int iM = M == 0 ? ix : (M == 1 ? iy : iz);
        mp = dirM > 0 ? iM : nM - 1 - iM;
        if (!(aM > 0.0f) || sM != dirM) {
            int dummy = 0;
            while (step(false, 0, 0, 0, 0, 0, 0, dummy)) {
            }
            active = false;
        }
    }

    for (;;) {
        if (tid == 0) s_chunk = INT_MAX;
        if (tid < 3) {
            s_lo[tid] = INT_MAX;
            s_hi[tid] = INT_MIN;
        }
        __syncthreads();
        if (active) atomicMin(&s_chunk, mp / kDepth);
        __syncthreads();
        const int chunk = s_chunk;
        if (chunk == INT_MAX) break;  // every ray has ended (uniform)
        const int cend = (chunk + 1) * kDepth;
        const bool part = active && mp < cend;
        if (part) {
            // the ray leaves the chunk within (cend - mp) major spacings
            const float dist = (float)(cend - mp) * aM;
            const int cxn = crossings_within(dist, ax, nx);
            const int cyn = crossings_within(dist, ay, ny);
            const int czn = crossings_within(dist, az, nz);
            atomicMin(&s_lo[0], sx > 0 ? ix : max(ix - cxn, 0));
            atomicMax(&s_hi[0], sx > 0 ? min(ix + cxn, nx - 1) : ix);
            atomicMin(&s_lo[1], sy > 0 ? iy : max(iy - cyn, 0));
            atomicMax(&s_hi[1], sy > 0 ? min(iy + cyn, ny - 1) : iy);
            atomicMin(&s_lo[2], sz > 0 ? iz : max(iz - czn, 0));
            atomicMax(&s_hi[2], sz > 0 ? min(iz + czn, nz - 1) : iz);
        }
        __syncthreads();
        const int lx = s_lo[0], ly = s_lo[1], lz = s_lo[2];
        const int wx = s_hi[0] - lx + 1, wy = s_hi[1] - ly + 1,
                  wz = s_hi[2] - lz + 1;
        const bool use_win = lx <= s_hi[0] && ly <= s_hi[1] && lz <= s_hi[2] &&
                             (int64_t)wx * wy * wz <= kWinCap;
        const int wn = use_win ? wx * wy * wz : 0;
        for (int w = tid; w < wn; w += kThreads) win[w] = 0.0f;
        __syncthreads();
        if (part) {
            while (mp < cend) {
                if (!step(use_win, lx, ly, lz, wx, wy, wz, mp)) {
                    active = false;
                    break;
                }
            }
        }
        __syncthreads();
        if (use_win) {
            const int warp = tid >> 5, lane = tid & 31;
            for (int row = warp; row < wy * wz; row += kThreads / 32) {
                const int yy = row % wy, zz = row / wy;
                float *dst = cube + ((int64_t)(lz + zz) * ny + (ly + yy)) * nx + lx;
                const float *src = win + row * wx;
                for (int xx = lane; xx < wx; xx += 32) {
                    const float v = src[xx];
                    if (v != 0.0f) atomicAdd(dst + xx, v);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

bool adjoint_window_supported(Tiling t)
{
    return t.tile_u * t.tile_v == kThreads;
}

cudaError_t launch_adjoint_window(const RayRec *rays, const ImgParam *prm,
                                  const float *images, const uint8_t *mask,
                                  float *cube, int32_t n_img, int32_t nu,
                                  int32_t nv, int32_t nx, int32_t ny,
                                  int32_t nz, Tiling t, const double *done,
                                  cudaStream_t s)
{
    if (n_img <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((nu + t.tile_u - 1) / t.tile_u),
                    (unsigned)((nv + t.tile_v - 1) / t.tile_v), (unsigned)n_img);
    k_adjoint_window<<<grid, kThreads, 0, s>>>(rays, prm, images, mask, cube,
                                               nu, nv, nx, ny, nz, t, done);
    return cudaGetLastError();
}

}  // namespace tomo
