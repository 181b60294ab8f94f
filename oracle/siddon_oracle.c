/*
 * FP64 CPU oracle of the solar-tomography projector.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled and called by the test
 * suite, by the package smoke check and by the CPU-baseline leg of the
 * benchmark; nothing on the product path may link or call it.  It shares no
 * code, header or table with the CUDA implementation.
 *
 * What it computes (Barbey, Guennou & Auchere, "TomograPy", Section 3.3.1,
 * Eq. lo): for every detector pixel k,
 *
 *     y_k = g_n * sum_j P_{k,j} e_j ,
 *
 * where P_{k,j} is the length of the line of sight of pixel k inside voxel j
 * and g_n the gain of the image n holding pixel k (Eq. two_spacecraft).  The
 * paper's index letters are garbled (the voxel index of Eq. lo is written
 * with two different letters); this file
 * reads k as the pixel and j as the voxel.  Masked pixels project to 0 and are
 * ignored by the transpose (Section 4: the projector skips masked pixels).
 * The transpose is the exact matrix transpose of the same P.
 *
 * Siddon's algorithm is cited by the paper (Section 3.1) but not restated.
 * The enumeration below is the textbook merge form: all voxel-plane crossing
 * parameters inside the cube are merged into one ascending list, and every
 * positive-length interval between consecutive crossings is charged to the
 * voxel that holds its midpoint.  Voxels are half-open, [lo + i d, lo + (i+1) d),
 * which settles rays that run along a voxel face.  It is not the incremental
 * walk the CUDA path uses: both reach the same definition by different steps.
 *
 * Readings where the paper is silent (it names the WCS keywords, Section 3.2,
 * but gives no formulas):
 *   - Sun-centred frame, z = rotation axis, x at longitude 0.  Observer
 *     o = d (cos lat cos lon, cos lat sin lon, sin lat).
 *   - Boresight w = -o/|o|; e1 = unit(w x z), e2 = e1 x w; the pair (e1, e2)
 *     is turned by the roll angle about w: e1' = cos r e1 + sin r e2,
 *     e2' = -sin r e1 + cos r e2.
 *   - Gnomonic (TAN) pixels: theta_u = (i_u - crpix_u) cdelt_u + crval_u,
 *     likewise v; direction u = unit(w + tan(theta_u) e1' + tan(theta_v) e2').
 *   - |lat| = 90 degrees leaves e1 undefined and is rejected.
 *   - Smooth temporal model (Section 3.3.3, "parameterization of the temporal
 *     evolution"): image n with time stamp tau sees the map
 *     (1 - w) X[k] + w X[k+1], k = min(floor(tau), T - 2), w = tau - k;
 *     tau must lie in [0, T - 1].  With one frame tau is ignored.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Cube of identical voxels: counts (nx, ny, nz), minimum corner, voxel size.
 * Arrays are [nz][ny][nx], x fastest.  r_obs > 0: radius of an opaque sphere
 * centred at the frame origin (the photosphere); 0: no obstacle. */
typedef struct {
    int32_t n[3];
    double lo[3];
    double d[3];
    double r_obs;
} orc_cube;

/* Column order of one pointing record. */
enum {
    C_DOBS = 0, C_LON, C_LAT, C_ROLL, C_CDELT_U, C_CDELT_V, C_CRPIX_U,
    C_CRPIX_V, C_CRVAL_U, C_CRVAL_V, C_GAIN, C_TIME, C_NCOL
};

/* ---------------------------------------------------------------- threads */

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------ ray (WCS) */

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double a[3])
{
    return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
}

/* Observer position o and unit direction u of the line of sight of pixel
 * (iu, iv) (Section 3.2, with the readings in the header).  Returns 0, or -1
 * for a pointing whose frame is undefined. */
int orc_ray(const double *p, int32_t iu, int32_t iv, double o[3], double u[3])
{
    double d = p[C_DOBS], lon = p[C_LON], lat = p[C_LAT], roll = p[C_ROLL];
    if (!(d > 0.0) || !(fabs(cos(lat)) > 1e-12)) return -1;
    o[0] = d * cos(lat) * cos(lon);
    o[1] = d * cos(lat) * sin(lon);
    o[2] = d * sin(lat);
    double w[3] = { -o[0] / d, -o[1] / d, -o[2] / d };
    const double zhat[3] = { 0.0, 0.0, 1.0 };
    double e1[3], e2[3];
    cross3(w, zhat, e1);
    double n1 = norm3(e1);
    for (int a = 0; a < 3; ++a) e1[a] /= n1;
    cross3(e1, w, e2);
    double cr = cos(roll), sr = sin(roll);
    double f1[3], f2[3];
    for (int a = 0; a < 3; ++a) {
        f1[a] = cr * e1[a] + sr * e2[a];
        f2[a] = -sr * e1[a] + cr * e2[a];
    }
    double tu = tan((iu - p[C_CRPIX_U]) * p[C_CDELT_U] + p[C_CRVAL_U]);
    double tv = tan((iv - p[C_CRPIX_V]) * p[C_CDELT_V] + p[C_CRVAL_V]);
    double dir[3];
    for (int a = 0; a < 3; ++a) dir[a] = w[a] + tu * f1[a] + tv * f2[a];
    double nd = norm3(dir);
    for (int a = 0; a < 3; ++a) u[a] = dir[a] / nd;
    return 0;
}

/* ---------------------------------------------------------- slab clip */

/* Parameter interval [amin, amax] of the half-line o + a u, a >= 0, inside the
 * cube.  An axis with u_a = 0 is dropped; the ray then misses unless o_a lies
 * in [lo_a, lo_a + n_a d_a).  Returns 1 on a hit of positive length. */
/* The part of the half-line o + a u (a >= 0, u a unit vector) that the line
 * of sight integrates: the slab clip against the cube, ended where the ray
 * first meets the opaque sphere if there is one.  The paper ends the
 * integration at the photosphere (Section 4) and gives no formula; reading: the first root a of |o + a u| = r_obs ends the
 * interval, a ray from an observer inside (or on) the sphere integrates
 * nothing, and a ray that misses or only grazes the sphere is unchanged. */
int orc_clip(const orc_cube *c, const double o[3], const double u[3],
             double *amin, double *amax)
{
    double lo = 0.0, hi = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double p0 = c->lo[a], p1 = c->lo[a] + c->n[a] * c->d[a];
        if (u[a] == 0.0) {
            if (o[a] < p0 || o[a] >= p1) return 0;
            continue;
        }
        double a0 = (p0 - o[a]) / u[a], a1 = (p1 - o[a]) / u[a];
        lo = fmax(lo, fmin(a0, a1));
        hi = fmin(hi, fmax(a0, a1));
    }
    if (c->r_obs > 0.0) {
        /* |o + a u|^2 = r^2.  With q = o - (o.u) u, the point of closest
         * approach, the roots are a = -(o.u) -+ sqrt(r^2 - |q|^2); forming
         * r^2 - |q|^2 from q avoids subtracting |o|^2 ~ (o.u)^2 from each
         * other (the observer is ~200 radii away). */
        double r2 = c->r_obs * c->r_obs;
        double oo = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
        if (oo <= r2) return 0; /* observer inside the sphere */
        double ou = o[0] * u[0] + o[1] * u[1] + o[2] * u[2];
        double q2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double q = o[a] - ou * u[a];
            q2 += q * q;
        }
        double disc = r2 - q2;
        if (disc > 0.0) {
            double first = -ou - sqrt(disc);
            if (first > 0.0) hi = fmin(hi, first);
        }
    }
    if (!(lo < hi)) return 0;
    *amin = lo;
    *amax = hi;
    return 1;
}

/* ------------------------------------------------------ merge-form Siddon */

/* Crossing parameters of the planes of axis a that lie strictly inside
 * (amin, amax), in ascending order.  Returns their number. */
static int32_t axis_crossings(const orc_cube *c, int a, const double o[3],
                              const double u[3], double amin, double amax,
                              double *out)
{
    int32_t m = 0;
    if (u[a] == 0.0) return 0;
    int32_t n = c->n[a];
    for (int32_t j = 0; j <= n; ++j) {
        int32_t k = (u[a] > 0.0) ? j : n - j; /* ascending parameter order */
        double al = (c->lo[a] + k * c->d[a] - o[a]) / u[a];
        if (al > amin && al < amax) out[m++] = al;
    }
    return m;
}

/* Largest number of segments one ray can produce in cube c. */
int64_t orc_max_segments(const orc_cube *c)
{
    return (int64_t)c->n[0] + c->n[1] + c->n[2] + 4;
}

/* Siddon segments of the ray o + a u through cube c: linear voxel indices and
 * lengths (|u| times the parameter interval), in order along the ray.  The
 * caller provides room for orc_max_segments(c) entries.  Returns the count
 * (0 for a miss) and, if amin_out is not NULL, the clip interval. */
int64_t orc_segments(const orc_cube *c, const double o[3], const double u[3],
                     int64_t *idx, double *len, double *amin_out,
                     double *amax_out)
{
    double amin, amax;
    if (amin_out) { *amin_out = 0.0; *amax_out = 0.0; }
    if (!orc_clip(c, o, u, &amin, &amax)) return 0;
    if (amin_out) { *amin_out = amin; *amax_out = amax; }

    int32_t cap = c->n[0] + c->n[1] + c->n[2] + 3;
    double *buf = (double *)malloc(sizeof(double) * (size_t)(2 * cap + 2));
    double *lists[3];
    int32_t cnt[3];
    double *w = buf;
    for (int a = 0; a < 3; ++a) {
        lists[a] = w;
        cnt[a] = axis_crossings(c, a, o, u, amin, amax, w);
        w += cnt[a];
    }
    /* merge the three ascending lists between amin and amax */
    double *merged = w;
    int32_t m = 0, h[3] = { 0, 0, 0 };
    merged[m++] = amin;
    for (;;) {
        int best = -1;
        for (int a = 0; a < 3; ++a)
            if (h[a] < cnt[a] &&
                (best < 0 || lists[a][h[a]] < lists[best][h[best]]))
                best = a;
        if (best < 0) break;
        merged[m++] = lists[best][h[best]++];
    }
    merged[m++] = amax;

    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    int64_t s = 0;
    for (int32_t q = 0; q + 1 < m; ++q) {
        double da = merged[q + 1] - merged[q];
        if (!(da > 0.0)) continue; /* zero-length interval: no voxel */
        double mid = 0.5 * (merged[q] + merged[q + 1]);
        int32_t i[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            double x = (o[a] + mid * u[a] - c->lo[a]) / c->d[a];
            i[a] = (int32_t)floor(x);
            if (i[a] < 0 || i[a] >= c->n[a]) inside = 0;
        }
        if (!inside) continue;
        idx[s] = ((int64_t)i[2] * c->n[1] + i[1]) * c->n[0] + i[0];
        len[s] = da * un;
        ++s;
    }
    free(buf);
    return s;
}

/* ------------------------------------------------------ time interpolation */

/* Frame index k and weight w of an image with time stamp tau over n_frames
 * frames (header).  Returns -1 when tau is outside [0, T - 1]. */
static int time_weights(int32_t n_frames, double tau, int32_t *k, double *w)
{
    if (n_frames <= 1) { *k = 0; *w = 0.0; return 0; }
    if (!(tau >= 0.0 && tau <= (double)(n_frames - 1))) return -1;
    int32_t kk = (int32_t)floor(tau);
    if (kk > n_frames - 2) kk = n_frames - 2;
    *k = kk;
    *w = tau - kk;
    return 0;
}

/* Validate the pointing table: every frame defined, every tau in range. */
static int check_pointing(int32_t n_frames, int32_t n_img, const double *ptg)
{
    for (int32_t n = 0; n < n_img; ++n) {
        const double *p = ptg + (size_t)n * C_NCOL;
        double o[3], u[3];
        int32_t k;
        double w;
        if (orc_ray(p, 0, 0, o, u) != 0) return -1;
        if (time_weights(n_frames, p[C_TIME], &k, &w) != 0) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------ projector P */

/* y = P x over all pixels (ray_ids == NULL) or over the listed pixels
 * (ray id = (n * nv + iv) * nu + iu; out[r] is the value of ray_ids[r]).
 * cube is [T][nz][ny][nx] FP64.  mask (nullable) is [n_img][nv][nu], nonzero =
 * excluded.  Returns 0, or -1 on an invalid pointing / time stamp. */
int orc_project(const orc_cube *c, int32_t n_frames, const double *cube,
                int32_t n_img, int32_t nu, int32_t nv, const double *pointing,
                const uint8_t *mask, int64_t n_rays, const int64_t *ray_ids,
                double *out)
{
    if (check_pointing(n_frames, n_img, pointing) != 0) return -1;
    int64_t n_all = (int64_t)n_img * nv * nu;
    int64_t total = ray_ids ? n_rays : n_all;
    int64_t nvox = (int64_t)c->n[0] * c->n[1] * c->n[2];
    int64_t cap = orc_max_segments(c);
#pragma omp parallel
    {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < total; ++r) {
            int64_t id = ray_ids ? ray_ids[r] : r;
            int32_t n = (int32_t)(id / ((int64_t)nv * nu));
            int32_t iv = (int32_t)((id / nu) % nv);
            int32_t iu = (int32_t)(id % nu);
            const double *p = pointing + (size_t)n * C_NCOL;
            if (mask && mask[id]) { out[r] = 0.0; continue; }
            double o[3], u[3];
            orc_ray(p, iu, iv, o, u);
            int32_t k;
            double w;
            time_weights(n_frames, p[C_TIME], &k, &w);
            int64_t s = orc_segments(c, o, u, idx, len, NULL, NULL);
            double acc = 0.0;
            for (int64_t q = 0; q < s; ++q) {
                double v;
                if (n_frames <= 1)
                    v = cube[idx[q]];
                else
                    v = (1.0 - w) * cube[(int64_t)k * nvox + idx[q]] +
                        w * cube[(int64_t)(k + 1) * nvox + idx[q]];
                acc += len[q] * v;
            }
            out[r] = p[C_GAIN] * acc;
        }
        free(idx);
        free(len);
    }
    return 0;
}

/* ------------------------------------------------------------ transpose P^T */

/* x = P^T y: cube_out ([T][nz][ny][nx] FP64) is overwritten with the
 * transpose of orc_project applied to images ([n_img][nv][nu]), restricted to
 * the listed rays when ray_ids is not NULL (images is then indexed by ray
 * id as a full image stack).  Masked pixels contribute nothing. */
static int backproject_impl(const orc_cube *c, int32_t n_frames,
                            int32_t n_img, int32_t nu, int32_t nv,
                            const double *pointing, const uint8_t *mask,
                            const double *images, int64_t n_rays,
                            const int64_t *ray_ids, double *cube_out,
                            int crossing_weights)
{
    if (check_pointing(n_frames, n_img, pointing) != 0) return -1;
    int64_t n_all = (int64_t)n_img * nv * nu;
    int64_t total = ray_ids ? n_rays : n_all;
    int64_t nvox = (int64_t)c->n[0] * c->n[1] * c->n[2];
    int64_t cap = orc_max_segments(c);
    memset(cube_out, 0, sizeof(double) * (size_t)(nvox * (n_frames > 1 ? n_frames : 1)));
#pragma omp parallel
    {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < total; ++r) {
            int64_t id = ray_ids ? ray_ids[r] : r;
            int32_t n = (int32_t)(id / ((int64_t)nv * nu));
            int32_t iv = (int32_t)((id / nu) % nv);
            int32_t iu = (int32_t)(id % nu);
            const double *p = pointing + (size_t)n * C_NCOL;
            if (mask && mask[id]) continue;
            double yk = p[C_GAIN] * images[id];
            if (crossing_weights) yk = fabs(yk);
            if (yk == 0.0) continue;
            double o[3], u[3];
            orc_ray(p, iu, iv, o, u);
            int32_t k;
            double w;
            time_weights(n_frames, p[C_TIME], &k, &w);
            int64_t s = orc_segments(c, o, u, idx, len, NULL, NULL);
            for (int64_t q = 0; q < s; ++q) {
                if (crossing_weights) len[q] = 1.0;
                if (n_frames <= 1) {
#pragma omp atomic
                    cube_out[idx[q]] += len[q] * yk;
                } else {
                    double a0 = (1.0 - w) * len[q] * yk, a1 = w * len[q] * yk;
#pragma omp atomic
                    cube_out[(int64_t)k * nvox + idx[q]] += a0;
#pragma omp atomic
                    cube_out[(int64_t)(k + 1) * nvox + idx[q]] += a1;
                }
            }
        }
        free(idx);
        free(len);
    }
    return 0;
}

/* x = P^T y (header: Eq. lo transposed). */
int orc_backproject(const orc_cube *c, int32_t n_frames, int32_t n_img,
                    int32_t nu, int32_t nv, const double *pointing,
                    const uint8_t *mask, const double *images, int64_t n_rays,
                    const int64_t *ray_ids, double *cube_out)
{
    return backproject_impl(c, n_frames, n_img, nu, nv, pointing, mask,
                            images, n_rays, ray_ids, cube_out, 0);
}

/* Crossing weights C_j = sum over the rays k with a positive-length segment
 * in voxel j of |g_k y_k| (time-weighted like the transpose): the transpose
 * with every length replaced by 1 and every pixel value by its magnitude.
 * It scales the error bound of a transpose whose segment lengths carry an
 * absolute rounding error independent of their length. */
int orc_crossing_weights(const orc_cube *c, int32_t n_frames, int32_t n_img,
                         int32_t nu, int32_t nv, const double *pointing,
                         const uint8_t *mask, const double *images,
                         int64_t n_rays, const int64_t *ray_ids,
                         double *cube_out)
{
    return backproject_impl(c, n_frames, n_img, nu, nv, pointing, mask,
                            images, n_rays, ray_ids, cube_out, 1);
}

/* Total number of Siddon segments (positive-length voxel intersections) of
 * the listed rays, or of all unmasked rays when ray_ids is NULL. */
int64_t orc_count_segments(const orc_cube *c, int32_t n_img, int32_t nu,
                           int32_t nv, const double *pointing,
                           const uint8_t *mask, int64_t n_rays,
                           const int64_t *ray_ids)
{
    int64_t n_all = (int64_t)n_img * nv * nu;
    int64_t total = ray_ids ? n_rays : n_all;
    int64_t cap = orc_max_segments(c);
    int64_t sum = 0;
#pragma omp parallel reduction(+ : sum)
    {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < total; ++r) {
            int64_t id = ray_ids ? ray_ids[r] : r;
            int32_t n = (int32_t)(id / ((int64_t)nv * nu));
            int32_t iv = (int32_t)((id / nu) % nv);
            int32_t iu = (int32_t)(id % nu);
            if (mask && mask[id]) continue;
            double o[3], u[3];
            if (orc_ray(pointing + (size_t)n * C_NCOL, iu, iv, o, u) != 0)
                continue;
            sum += orc_segments(c, o, u, idx, len, NULL, NULL);
        }
        free(idx);
        free(len);
    }
    return sum;
}

/* ------------------------------------------------- impact parameter */

/* Squared impact parameter of every pixel's line of sight: rho^2 = |o x u|^2,
 * the squared distance from Sun centre to the line (Section 3.5: the pB
 * operator's per-pixel diagonal o_k = rho_k^2, Eq. thomson_lo).  out is
 * [n_img][nv][nu].  Returns 0, or -1 on an undefined pointing frame. */
int orc_impact2(int32_t n_img, int32_t nu, int32_t nv, const double *pointing,
                double *out)
{
    for (int32_t n = 0; n < n_img; ++n)
        for (int32_t iv = 0; iv < nv; ++iv)
            for (int32_t iu = 0; iu < nu; ++iu) {
                double o[3], u[3], c[3];
                if (orc_ray(pointing + (size_t)n * C_NCOL, iu, iv, o, u) != 0)
                    return -1;
                cross3(o, u, c);
                out[((size_t)n * nv + iv) * nu + iu] =
                    c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
            }
    return 0;
}
