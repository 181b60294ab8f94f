"""Pins of the FP64 oracle against geometry, closed forms and brute force.

None of these checks re-types the oracle's own formulas: each compares it
with something the geometry or the mathematics fixes independently, chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails at
least one of them.
"""

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import checks, siddon, solver


def _geom(n, lo, d):
    nx, ny, nz = n
    return {"nx": nx, "ny": ny, "nz": nz, "x0": lo[0], "y0": lo[1],
            "z0": lo[2], "dx": d[0], "dy": d[1], "dz": d[2]}


def _dense(geom, o, u):
    idx, ln, _, _ = siddon.segments(geom, o, u)
    out = np.zeros(geom["nx"] * geom["ny"] * geom["nz"])
    np.add.at(out, idx, ln)
    return out


# --------------------------------------------------------------- hand cases

def test_hand_derived_cases(golden_dir):
    """Hand-derived integrals through a 2x2x2 cube, incl. the half-open tie
    rule, a corner-to-corner diagonal and an observer inside the cube."""
    g = _geom((2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    k, j, i = np.meshgrid(np.arange(2), np.arange(2), np.arange(2),
                          indexing="ij")
    cube = (1 + i + 2 * j + 4 * k).astype(np.float64).reshape(-1)
    rows = [ln.split() for ln in open(os.path.join(golden_dir,
                                                   "siddon_hand_cases.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 8
    for name, *vals in rows:
        ox, oy, oz, ux, uy, uz, want = map(float, vals)
        idx, ln, _, _ = siddon.segments(g, [ox, oy, oz], [ux, uy, uz])
        got = float(np.sum(ln * cube[idx]))
        assert got == pytest.approx(want, rel=1e-14, abs=1e-14), name


# ------------------------------------------------------ exact rational pins

def _exact_lengths(n, o, u):
    """Parameter length (in units of |u|) of o + a u, a >= 0, inside every
    half-open unit voxel of [0, n)^3, in exact rational arithmetic."""
    out = {}
    for kk in range(n):
        for jj in range(n):
            for ii in range(n):
                b0 = (ii, jj, kk)
                t_in, t_out = Fraction(0), None
                ok = True
                for a in range(3):
                    if u[a] == 0:
                        if not (b0[a] <= o[a] < b0[a] + 1):
                            ok = False
                        continue
                    ta = (Fraction(b0[a]) - o[a]) / u[a]
                    tb = (Fraction(b0[a] + 1) - o[a]) / u[a]
                    lo_, hi_ = min(ta, tb), max(ta, tb)
                    t_in = max(t_in, lo_)
                    t_out = hi_ if t_out is None else min(t_out, hi_)
                if ok and t_out is not None and t_out > t_in:
                    out[(kk * n + jj) * n + ii] = t_out - t_in
    return out


@pytest.mark.parametrize("o,u", [
    ((Fraction(-1), Fraction(-1), Fraction(-1)), (1, 1, 1)),          # corners
    ((Fraction(-1), Fraction(1, 2), Fraction(-2)), (2, 0, 3)),        # edges
    ((Fraction(5), Fraction(3, 7), Fraction(9, 4)), (-3, 1, -1)),
    ((Fraction(-2), Fraction(-3), Fraction(1)), (1, 2, 0)),           # face z=1
    ((Fraction(1, 3), Fraction(4, 3), Fraction(7, 5)), (1, -1, 2)),   # inside
    ((Fraction(-1), Fraction(2), Fraction(2)), (1, -1, -1)),          # edges
])
def test_exact_rational_brute_force(o, u):
    """Every per-voxel length equals the exact rational slab clip, including
    rays through voxel corners, along edges and lying in faces."""
    n = 3
    g = _geom((n, n, n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    exact = _exact_lengths(n, o, u)
    un = math.sqrt(sum(c * c for c in u))
    want = np.zeros(n ** 3)
    for j, v in exact.items():
        want[j] = float(v) * un
    got = _dense(g, [float(c) for c in o], [float(c) for c in u])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


# ------------------------------------------------------------ brute force O2

def test_brute_force_random_rays():
    """Merge-form Siddon equals the per-voxel slab clip on small anisotropic
    cubes for random rays (random origins inside and outside the cube)."""
    rng = np.random.default_rng(7)
    g = _geom((5, 4, 6), (-0.7, 0.2, -1.1), (0.3, 0.45, 0.25))
    for _ in range(60):
        o = rng.uniform(-3, 3, 3)
        u = rng.standard_normal(3)
        np.testing.assert_allclose(_dense(g, o, u),
                                   checks.brute_force_ray(g, o, u),
                                   rtol=0, atol=1e-12)


def test_brute_force_wcs_rays():
    """Same pin on rays built from pointing records (far observer)."""
    g = synth.cube_geom(6, 1.5)
    ptg = synth.pointing_table([17.0, 133.0], [3.0, -11.0], 215.0, 9, 7, 3.2,
                               roll_deg=[0.0, 25.0][1])
    for n in range(2):
        for iu, iv in [(0, 0), (4, 3), (8, 6), (2, 5)]:
            o, u = siddon.ray(ptg[n], iu, iv)
            np.testing.assert_allclose(_dense(g, o, u),
                                       checks.brute_force_ray(g, o, u),
                                       rtol=0, atol=1e-11)


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("seed", range(5))
def test_chord_through_centre_closed_form(seed):
    """A line through the centre of a cube of half-width h along unit u has
    chord 2 h / max|u_a|; a uniform cube c integrates to c times the chord,
    and the segment lengths sum to the chord."""
    rng = np.random.default_rng(seed)
    h = 1.3
    n = int(rng.integers(3, 12))
    g = synth.cube_geom(n, h)
    u = rng.standard_normal(3)
    u /= np.linalg.norm(u)
    o = -200.0 * u  # far observer, line through the centre
    idx, ln, a0, a1 = siddon.segments(g, o, u)
    chord = 2 * h / np.max(np.abs(u))
    assert np.sum(ln) == pytest.approx(chord, rel=1e-12)
    cube = np.full(n ** 3, 2.5)
    assert np.sum(ln * cube[idx]) == pytest.approx(2.5 * chord, rel=1e-12)


def test_axis_aligned_column_sums():
    """Axis-aligned rays through voxel centres return dx times the exact
    column sums, along x, y and z and in both directions."""
    rng = np.random.default_rng(3)
    g = _geom((7, 5, 4), (-1.0, -0.5, 0.25), (0.2, 0.3, 0.4))
    x = rng.random((4, 5, 7))
    flat = x.reshape(-1)
    for (k, j) in [(0, 0), (3, 4), (2, 1)]:
        yc = g["y0"] + (j + 0.5) * g["dy"]
        zc = g["z0"] + (k + 0.5) * g["dz"]
        for sgn in (1, -1):
            o = [-5.0 * sgn, yc, zc]
            idx, ln, _, _ = siddon.segments(g, o, [sgn * 1.0, 0, 0])
            assert np.sum(ln * flat[idx]) == pytest.approx(
                g["dx"] * x[k, j, :].sum(), rel=1e-13)
    for (k, i) in [(1, 6), (0, 0)]:
        xc = g["x0"] + (i + 0.5) * g["dx"]
        zc = g["z0"] + (k + 0.5) * g["dz"]
        idx, ln, _, _ = siddon.segments(g, [xc, 9.0, zc], [0, -2.0, 0])
        assert np.sum(ln * flat[idx]) == pytest.approx(
            g["dy"] * x[k, :, i].sum(), rel=1e-13)
    for (j, i) in [(2, 3), (4, 6)]:
        xc = g["x0"] + (i + 0.5) * g["dx"]
        yc = g["y0"] + (j + 0.5) * g["dy"]
        idx, ln, _, _ = siddon.segments(g, [xc, yc, -3.0], [0, 0, 0.5])
        assert np.sum(ln * flat[idx]) == pytest.approx(
            g["dz"] * x[:, j, i].sum(), rel=1e-13)


def test_rays_in_the_boundary_faces():
    """Half-open voxels [lo + i d, lo + (i + 1) d): a ray lying in a lower
    face of the cube runs inside the first layer of voxels and integrates
    that layer's row; the same ray in the upper face lies in no voxel and
    integrates nothing.  Rays along x in the faces z = z0 and z = z0 + nz dz,
    along y in x = x0 and x = x0 + nx dx, along z in y = y0 and y = y0 + ny dy
    (the coordinates chosen exactly representable)."""
    rng = np.random.default_rng(11)
    g = _geom((7, 5, 4), (-1.0, -0.5, 0.25), (0.25, 0.5, 0.125))
    x = rng.random((4, 5, 7))
    flat = x.reshape(-1)
    hi = [g["x0"] + 7 * g["dx"], g["y0"] + 5 * g["dy"], g["z0"] + 4 * g["dz"]]
    j, k, i = 2, 1, 3
    yc = g["y0"] + (j + 0.5) * g["dy"]
    zc = g["z0"] + (k + 0.5) * g["dz"]
    xc = g["x0"] + (i + 0.5) * g["dx"]
    cases = [
        ([-5.0, yc, g["z0"]], [1.0, 0, 0], g["dx"] * x[0, j, :].sum()),
        ([-5.0, yc, hi[2]], [1.0, 0, 0], 0.0),
        ([g["x0"], 9.0, zc], [0, -1.0, 0], g["dy"] * x[k, :, 0].sum()),
        ([hi[0], 9.0, zc], [0, -1.0, 0], 0.0),
        ([xc, g["y0"], -3.0], [0, 0, 1.0], g["dz"] * x[:, 0, i].sum()),
        ([xc, hi[1], -3.0], [0, 0, 1.0], 0.0),
    ]
    for o, u, want in cases:
        idx, ln, _, _ = siddon.segments(g, o, u)
        got = float(np.sum(ln * flat[idx])) if len(idx) else 0.0
        assert got == pytest.approx(want, rel=1e-13, abs=0.0), (o, u)


def test_fine_sampling_converges():
    """Midpoint sampling with step h stays within (S + 2) h max|x| of the
    Siddon integral (S = number of segments), and the error shrinks with h."""
    rng = np.random.default_rng(11)
    g = synth.cube_geom(8, 1.0)
    x = rng.random((8, 8, 8))
    flat = x.reshape(-1)
    for _ in range(4):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        o = rng.uniform(-0.3, 0.3, 3) - 5.0 * u
        idx, ln, _, _ = siddon.segments(g, o, u)
        exact = float(np.sum(ln * flat[idx]))
        errs = []
        for h in (1e-2, 1e-3, 1e-4):
            approx = checks.sampled_ray(g, x, o, u, h, 5.0 + 2 * np.sqrt(3))
            err = abs(approx - exact)
            assert err <= (len(idx) + 2) * h * x.max()
            errs.append(err)
        assert errs[-1] < 1e-2 * (len(idx) + 2) * x.max() * 1e-2 + 1e-12


# --------------------------------------------------------- WCS ray reading

def test_wcs_reference_pixel_hits_sun_centre():
    """With crval = 0 the reference pixel looks at Sun centre: the impact
    parameter |o x u| is 0 and u = -o/|o|."""
    ptg = synth.pointing_table([0.0, 57.0, 211.0], [0.0, 12.0, -30.0], 215.0,
                               5, 9, 3.2, roll_deg=17.0)
    for n in range(3):
        o, u = siddon.ray(ptg[n], 2, 4)  # crpix = (2, 4)
        assert np.linalg.norm(np.cross(o, u)) < 1e-12
        np.testing.assert_allclose(u, -o / np.linalg.norm(o), atol=1e-15)
        lon, lat = np.deg2rad([0.0, 57.0, 211.0][n]), np.deg2rad(
            [0.0, 12.0, -30.0][n])
        np.testing.assert_allclose(
            o, 215.0 * np.array([np.cos(lat) * np.cos(lon),
                                 np.cos(lat) * np.sin(lon), np.sin(lat)]),
            atol=1e-12)


def test_wcs_gnomonic_angles_and_impact_parameter():
    """Gnomonic pixels: the angle between a pixel's ray and the boresight
    satisfies tan^2 = tan^2(theta_u) + tan^2(theta_v), and its impact
    parameter is d sin(theta)."""
    nu, nv = 11, 7
    ptg = synth.pointing_table([33.0], [5.0], 215.0, nu, nv, 40.0,
                               roll_deg=12.0)
    ptg[0, 8] = 1e-3   # crval_u
    ptg[0, 9] = -2e-3  # crval_v
    p = ptg[0]
    _, w = siddon.ray(np.concatenate([p[:8], [0.0, 0.0], p[10:]]), 5, 3)
    for iu, iv in [(0, 0), (10, 6), (3, 5), (7, 1)]:
        o, u = siddon.ray(p, iu, iv)
        tu = math.tan((iu - p[6]) * p[4] + p[8])
        tv = math.tan((iv - p[7]) * p[5] + p[9])
        theta = math.atan(math.hypot(tu, tv))
        assert math.acos(np.clip(np.dot(u, w), -1, 1)) == pytest.approx(
            theta, rel=1e-9)
        assert np.linalg.norm(np.cross(o, u)) == pytest.approx(
            215.0 * math.sin(theta), rel=1e-9)


def test_wcs_orientation_and_roll():
    """At lon = lat = roll = 0 the u axis points to +y and the v axis to +z
    (solar north up); a 90-degree roll turns +u into +v."""
    p = synth.pointing_table([0.0], [0.0], 215.0, 3, 3, 3.2)[0]
    o, u_c = siddon.ray(p, 1, 1)
    _, u_r = siddon.ray(p, 2, 1)  # one pixel along +u
    _, u_t = siddon.ray(p, 1, 2)  # one pixel along +v
    d_r, d_t = u_r - u_c, u_t - u_c
    assert d_r[1] > 0 and abs(d_r[2]) < 1e-15
    assert d_t[2] > 0 and abs(d_t[1]) < 1e-15
    q = synth.pointing_table([0.0], [0.0], 215.0, 3, 3, 3.2, roll_deg=90.0)[0]
    _, ur = siddon.ray(q, 2, 1)
    np.testing.assert_allclose(ur, u_t, atol=1e-14)


def test_wcs_pole_rejected():
    p = synth.pointing_table([0.0], [90.0], 215.0, 3, 3, 3.2)[0]
    with pytest.raises(ValueError):
        siddon.ray(p, 0, 0)


def test_mask_recipe_matches_ray_impact_parameter():
    """The occulter recipe (an image-plane disk) masks exactly the pixels
    whose ray passes within r_occ of Sun centre."""
    ptg = synth.pointing_table([10.0, 200.0], [4.0, -6.0], 215.0, 16, 12, 4.0)
    m = synth.occulter_mask(ptg, 16, 12, r_occ=1.0, r_edge=1.8)
    for n in range(2):
        for iv in range(12):
            for iu in range(16):
                o, u = siddon.ray(ptg[n], iu, iv)
                rho = np.linalg.norm(np.cross(o, u))
                assert bool(m[n, iv, iu]) == (rho < 1.0 or rho > 1.8)


# --------------------------------------------------- operator-level pins

def _small_scene(T=1):
    g = synth.cube_geom(9, 1.5, ny=7, nz=8)
    rng = np.random.default_rng(5)
    ptg = synth.pointing_table(rng.uniform(0, 360, 5), rng.uniform(-20, 20, 5),
                               215.0, 10, 6, 3.4, roll_deg=8.0,
                               gain=rng.uniform(0.5, 2.0, 5),
                               time=rng.uniform(0, max(T - 1, 0), 5))
    mask = (rng.random((5, 6, 10)) < 0.2).astype(np.uint8)
    return g, ptg, mask, rng


@pytest.mark.parametrize("T", [1, 3])
def test_adjoint_identity_fp64(T):
    """<P x, y> = <x, P^T y> to 1e-12 (with mask, gains and, for T = 3,
    time interpolation between frames)."""
    g, ptg, mask, rng = _small_scene(T)
    shape = ((T,) if T > 1 else ()) + (g["nz"], g["ny"], g["nx"])
    x = rng.standard_normal(shape)
    y = rng.standard_normal((5, 6, 10))
    Px = siddon.project(g, x, ptg, 10, 6, mask, n_frames=T)
    Pty = siddon.backproject(g, y, ptg, 10, 6, mask, n_frames=T)
    lhs, rhs = np.sum(Px * y), np.sum(x * Pty)
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert np.all(Px[mask != 0] == 0.0)


def test_dense_matrix_equals_brute_force():
    """Rows of P (projecting unit vectors) equal the brute-force clip of each
    pixel's ray, times the gain."""
    g, ptg, _, _ = _small_scene()
    nvox = g["nx"] * g["ny"] * g["nz"]
    Pm = np.zeros((5 * 6 * 10, nvox))
    eye = np.zeros(nvox)
    for j in range(nvox):
        eye[:] = 0.0
        eye[j] = 1.0
        Pm[:, j] = siddon.project(g, eye.reshape(8, 7, 9), ptg, 10, 6).reshape(-1)
    for r in [0, 17, 123, 299]:
        n, iv, iu = r // 60, (r // 10) % 6, r % 10
        o, u = siddon.ray(ptg[n], iu, iv)
        np.testing.assert_allclose(Pm[r], ptg[n, 10] * checks.brute_force_ray(g, o, u),
                                   atol=1e-12)


def test_gain_scales_projection():
    g, ptg, mask, rng = _small_scene()
    x = rng.random((8, 7, 9))
    y1 = siddon.project(g, x, ptg, 10, 6, mask)
    p2 = ptg.copy()
    p2[:, 10] *= 3.0
    y3 = siddon.project(g, x, p2, 10, 6, mask)
    np.testing.assert_allclose(y3, 3.0 * y1, rtol=1e-14)


def test_time_interpolation_special_cases():
    """Integer time stamps select one frame; tau = T-1 selects the last
    frame; a stamp halfway between frames gives the mean of the two
    projections; a stamp outside [0, T-1] is rejected."""
    g, ptg, _, rng = _small_scene()
    T = 4
    X = rng.random((T, 8, 7, 9))
    per_frame = [siddon.project(g, X[t], ptg, 10, 6) for t in range(T)]
    for tau, want in [(0.0, per_frame[0]), (2.0, per_frame[2]),
                      (3.0, per_frame[3]),
                      (1.5, 0.5 * (per_frame[1] + per_frame[2]))]:
        p = ptg.copy()
        p[:, 11] = tau
        got = siddon.project(g, X, p, 10, 6, n_frames=T)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)
    p = ptg.copy()
    p[0, 11] = 3.5
    with pytest.raises(ValueError):
        siddon.project(g, X, p, 10, 6, n_frames=T)


def test_fd_gradient_of_data_term():
    """Central finite differences of f(x) = 0.5 ||P x - y||^2 (exact for a
    quadratic up to rounding) equal P^T (P x - y)."""
    g, ptg, mask, rng = _small_scene()
    x = rng.random((8, 7, 9))
    y = rng.random((5, 6, 10))
    r = siddon.project(g, x, ptg, 10, 6, mask) - np.where(mask == 0, y, 0.0)
    grad = siddon.backproject(g, r, ptg, 10, 6, mask)

    def f(v):
        rr = siddon.project(g, v, ptg, 10, 6, mask) - np.where(mask == 0, y, 0)
        return 0.5 * np.sum(rr * rr)
    h = 1e-3
    for j in rng.choice(x.size, 12, replace=False):
        e = np.zeros(x.size)
        e[j] = h
        e = e.reshape(x.shape)
        fd = (f(x + e) - f(x - e)) / (2 * h)
        assert fd == pytest.approx(grad.reshape(-1)[j], rel=1e-7, abs=1e-10)


# ---------------------------------------------------------- prior D

def test_DtD_cosine_eigenmodes():
    """Forward differences without wrap make D^T D the path-graph Laplacian
    on each line; its eigenvectors are cos(pi m (i + 1/2) / n) with
    eigenvalues 2 - 2 cos(pi m / n)."""
    nz, ny, nx = 5, 6, 7
    for axis, n in ((2, nx), (1, ny), (0, nz)):
        for m in range(n):
            c = np.cos(np.pi * m * (np.arange(n) + 0.5) / n)
            shape = [1, 1, 1]
            shape[axis] = n
            x = np.broadcast_to(c.reshape(shape), (nz, ny, nx)).copy()
            lam = 2 - 2 * np.cos(np.pi * m / n)
            np.testing.assert_allclose(solver.DtD(x), lam * x, atol=1e-12)


def test_D_adjoint_and_ramp():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 5, 6))
    gs = [rng.standard_normal(d.shape) for d in solver.D(x)]
    lhs = sum(np.sum(a * b) for a, b in zip(solver.D(x), gs))
    assert lhs == pytest.approx(np.sum(x * solver.Dt(*gs)), rel=1e-12)
    # ramp 2 i + 3 j - k: differences are 2, 3, -1 on every line
    k, j, i = np.meshgrid(np.arange(4), np.arange(5), np.arange(6),
                          indexing="ij")
    ramp = 2.0 * i + 3.0 * j - 1.0 * k
    want = 4 * 4 * 5 * 5 + 9 * 4 * 4 * 6 + 1 * 3 * 5 * 6
    assert solver.prior_energy(ramp) == pytest.approx(want, rel=1e-14)


# ---------------------------------------------------------------- CG

def _dense_problem():
    g = synth.cube_geom(5, 1.5, ny=4, nz=4)
    rng = np.random.default_rng(9)
    ptg = synth.pointing_table(rng.uniform(0, 360, 6), rng.uniform(-30, 30, 6),
                               215.0, 8, 8, 3.4)
    mask = (rng.random((6, 8, 8)) < 0.15).astype(np.uint8)
    x_true = rng.random((4, 4, 5))
    y = siddon.project(g, x_true, ptg, 8, 8, mask) + 0.01 * rng.standard_normal(
        (6, 8, 8))
    return solver.Problem(g, ptg, 8, 8, y, mask, lam=0.3)


def _dense_AB(pb):
    """Dense A = M P (brute-force rows, masked pixels zero) and the dense
    forward-difference matrix B of the 5 x 4 x 4 problem."""
    g = pb.geom
    nvox = 80
    A = np.zeros((6 * 64, nvox))
    for r in range(6 * 64):
        n, iv, iu = r // 64, (r // 8) % 8, r % 8
        if pb.mask.reshape(-1)[r]:
            continue
        o, u = siddon.ray(pb.pointing[n], iu, iv)
        A[r] = checks.brute_force_ray(g, o, u)
    # dense forward-difference matrices, built from index arithmetic
    rows = []
    for (dk, dj, di) in ((0, 0, 1), (0, 1, 0), (1, 0, 0)):
        for k in range(4 - dk):
            for j in range(4 - dj):
                for i in range(5 - di):
                    row = np.zeros(nvox)
                    row[((k + dk) * 4 + j + dj) * 5 + i + di] += 1
                    row[(k * 4 + j) * 5 + i] -= 1
                    rows.append(row)
    return A, np.array(rows)


def test_cg_matches_direct_solve():
    """CG on the normal equations reaches the direct solution of
    (A^T A + lambda B^T B) x = A^T y (Eq. criterion) built from dense
    brute-force rows and dense difference matrices."""
    pb = _dense_problem()
    A, B = _dense_AB(pb)
    ym = np.where(pb.mask == 0, pb.y, 0.0).reshape(-1)
    x_direct = np.linalg.solve(A.T @ A + pb.lam * B.T @ B, A.T @ ym)
    x_cg, rep = solver.cg(pb, 400)
    np.testing.assert_allclose(x_cg.reshape(-1), x_direct, rtol=0,
                               atol=1e-9 * np.abs(x_direct).max())
    J = rep["J"]
    assert np.all(np.diff(J) <= 1e-12 * J[0])  # non-increasing
    Jmin = float(np.sum((ym - A @ x_direct) ** 2) + pb.lam * np.sum((B @ x_direct) ** 2))
    assert J[-1] == pytest.approx(Jmin, rel=1e-10)


def test_cg_warm_start_and_J_identity():
    """CG from a warm start continues the same minimisation; and
    J(x) = y^T M y - x^T (r + b) holds for every iterate (the identity the
    device solver reports J through)."""
    pb = _dense_problem()
    x5, rep5 = solver.cg(pb, 5)
    b = pb.rhs()
    r = b - pb.normal(x5)
    ym = pb.masked(pb.y)
    assert pb.J(x5) == pytest.approx(float(np.sum(ym * ym) - np.sum(x5 * (r + b))),
                                     rel=1e-10)
    x_more, rep_more = solver.cg(pb, 30, x0=x5)
    assert rep_more["J"][-1] <= rep5["J"][-1]


def _map_mask_problem(n_excluded, seed=4):
    pb = _dense_problem()
    rng = np.random.default_rng(seed)
    mm = np.zeros(80, np.uint8)
    mm[rng.choice(80, n_excluded, replace=False)] = 1 + rng.integers(0, 255,
                                                                     n_excluded)
    mm = mm.reshape(4, 4, 5)
    return solver.Problem(pb.geom, pb.pointing, 8, 8, pb.y, pb.mask, pb.lam,
                          map_mask=mm), mm


def test_map_mask_solves_the_reduced_system():
    """With a map mask the unknowns are the other voxels: the solution is the
    direct solve of the least-squares problem whose dense matrices have the
    excluded voxels' columns deleted (the excluded voxels stay 0)."""
    pb, mm = _map_mask_problem(23)
    A, B = _dense_AB(pb)
    keep = mm.reshape(-1) == 0
    Ak, Bk = A[:, keep], B[:, keep]
    ym = np.where(pb.mask == 0, pb.y, 0.0).reshape(-1)
    xk = np.linalg.solve(Ak.T @ Ak + pb.lam * Bk.T @ Bk, Ak.T @ ym)
    x_cg, rep = solver.cg(pb, 400, x0=np.ones((4, 4, 5)))
    x_cg = x_cg.reshape(-1)
    assert np.all(x_cg[~keep] == 0.0)
    np.testing.assert_allclose(x_cg[keep], xk, rtol=0,
                               atol=1e-9 * np.abs(xk).max())
    Jmin = float(np.sum((ym - Ak @ xk) ** 2) + pb.lam * np.sum((Bk @ xk) ** 2))
    assert rep["J"][-1] == pytest.approx(Jmin, rel=1e-10)
    # J identity of the device solver holds on the restricted system
    x5, _ = solver.cg(pb, 5)
    b = pb.rhs()
    r = b - pb.normal(x5)
    assert np.all(r.reshape(-1)[~keep] == 0.0)
    yy = pb.masked(pb.y)
    assert pb.J(x5) == pytest.approx(float(np.sum(yy * yy) - np.sum(x5 * (r + b))),
                                     rel=1e-10)


def test_map_mask_projection_special_cases():
    """P with a map mask against brute-force rows times the kept voxels; the
    adjoint identity in FP64; an all-excluded map projects, back-projects and
    reconstructs to 0; an all-kept map changes nothing."""
    g, ptg, mask, rng = _small_scene()
    shape = (g["nz"], g["ny"], g["nx"])
    x = rng.random(shape)
    mm = (rng.random(shape) < 0.3).astype(np.uint8) * 7
    got = siddon.project(g, x, ptg, 10, 6, mask, map_mask=mm)
    keep = (mm == 0).reshape(-1)
    for r in rng.choice(5 * 60, 40, replace=False):
        n, iv, iu = r // 60, (r // 10) % 6, r % 10
        o, u = siddon.ray(ptg[n], iu, iv)
        want = 0.0 if mask[n, iv, iu] else float(
            np.sum(checks.brute_force_ray(g, o, u) * keep * x.reshape(-1)) *
            ptg[n, 10])
        assert got[n, iv, iu] == pytest.approx(want, rel=1e-12, abs=1e-14)
    y = rng.random((5, 6, 10))
    Pty = siddon.backproject(g, y, ptg, 10, 6, mask, map_mask=mm)
    assert np.all(Pty[mm != 0] == 0.0)
    lhs = float(np.sum(np.where(mask == 0, y, 0) * got))
    assert lhs == pytest.approx(float(np.sum(x * Pty)), rel=1e-12)
    full = np.ones(shape, np.uint8)
    assert not np.any(siddon.project(g, x, ptg, 10, 6, mask, map_mask=full))
    assert not np.any(siddon.backproject(g, y, ptg, 10, 6, mask,
                                         map_mask=full))
    zero = np.zeros(shape, np.uint8)
    assert np.array_equal(siddon.project(g, x, ptg, 10, 6, mask, map_mask=zero),
                          siddon.project(g, x, ptg, 10, 6, mask))
    pb, _ = _map_mask_problem(80)
    x_all, rep = solver.cg(pb, 5, x0=np.ones((4, 4, 5)))
    assert not np.any(x_all)
    # the solver's operator reads excluded voxels as 0 (R14) whatever they
    # hold: its P of x equals the masked projection pinned above, and the
    # criterion of x equals that of K x
    pm = solver.Problem(g, ptg, 10, 6, y, mask, lam=0.3, map_mask=mm)
    np.testing.assert_allclose(pm.P(x), got, rtol=1e-13, atol=1e-15)
    assert pm.J(x) == pytest.approx(pm.J(np.where(mm == 0, x, 0.0)),
                                    rel=1e-13)


def test_height_weighted_prior_solves_the_dense_system():
    """Eq. srt_inversion: with B = D R (R diagonal) CG reaches the direct
    solve built from the dense difference matrix times diag(R); with a map
    mask too, the excluded columns are deleted from A and from D R; a
    constant weight c equals the unweighted prior with lambda c^2."""
    pb0 = _dense_problem()
    A, B = _dense_AB(pb0)
    rng = np.random.default_rng(12)
    w = rng.uniform(0.5, 3.0, 80)
    ym = np.where(pb0.mask == 0, pb0.y, 0.0).reshape(-1)
    pb = solver.Problem(pb0.geom, pb0.pointing, 8, 8, pb0.y, pb0.mask,
                        pb0.lam, prior_weight=w.reshape(4, 4, 5))
    BR = B * w[None, :]
    x_direct = np.linalg.solve(A.T @ A + pb.lam * BR.T @ BR, A.T @ ym)
    x_cg, rep = solver.cg(pb, 400)
    np.testing.assert_allclose(x_cg.reshape(-1), x_direct, rtol=0,
                               atol=1e-9 * np.abs(x_direct).max())
    Jmin = float(np.sum((ym - A @ x_direct) ** 2) +
                 pb.lam * np.sum((BR @ x_direct) ** 2))
    assert rep["J"][-1] == pytest.approx(Jmin, rel=1e-10)
    # with a map mask
    _, mm = _map_mask_problem(17)
    keep = mm.reshape(-1) == 0
    pbm = solver.Problem(pb0.geom, pb0.pointing, 8, 8, pb0.y, pb0.mask,
                         pb0.lam, map_mask=mm, prior_weight=w)
    Ak, Bk = A[:, keep], BR[:, keep]
    xk = np.linalg.solve(Ak.T @ Ak + pb.lam * Bk.T @ Bk, Ak.T @ ym)
    x_m, _ = solver.cg(pbm, 400)
    x_m = x_m.reshape(-1)
    assert np.all(x_m[~keep] == 0.0)
    np.testing.assert_allclose(x_m[keep], xk, rtol=0,
                               atol=1e-9 * np.abs(xk).max())
    # constant weight
    pc = solver.Problem(pb0.geom, pb0.pointing, 8, 8, pb0.y, pb0.mask,
                        pb0.lam, prior_weight=np.full(80, 1.7))
    pl = solver.Problem(pb0.geom, pb0.pointing, 8, 8, pb0.y, pb0.mask,
                        pb0.lam * 1.7 ** 2)
    v = rng.random((4, 4, 5))
    np.testing.assert_allclose(pc.normal(v), pl.normal(v), rtol=1e-13)
    assert pc.J(v) == pytest.approx(pl.J(v), rel=1e-13)


def test_crossing_weights():
    """C_j with unit images counts the rays crossing each voxel: it matches
    the brute-force clip (positive lengths), and its total is the number of
    segments; with |y| weights it bounds |P^T y| / (largest length)."""
    g, ptg, mask, rng = _small_scene()
    ones = np.ones((5, 6, 10))
    p1 = ptg.copy()
    p1[:, 10] = 1.0
    Cw = siddon.crossing_weights(g, ones, p1, 10, 6, mask)
    want = np.zeros(g["nx"] * g["ny"] * g["nz"])
    for r in range(300):
        n, iv, iu = r // 60, (r // 10) % 6, r % 10
        if mask.reshape(-1)[r]:
            continue
        o, u = siddon.ray(p1[n], iu, iv)
        want += checks.brute_force_ray(g, o, u) > 0
    np.testing.assert_array_equal(Cw.reshape(-1), want)
    assert Cw.sum() == siddon.count_segments(g, p1, 10, 6, mask)
    y = rng.standard_normal((5, 6, 10))
    Cy = siddon.crossing_weights(g, y, ptg, 10, 6, mask)
    Pty = siddon.backproject(g, y, ptg, 10, 6, mask)
    diag = np.sqrt(sum((g["n" + a] * g["d" + a]) ** 2 for a in "xyz"))
    assert np.all(np.abs(Pty) <= Cy * min(diag, max(g["dx"], g["dy"], g["dz"]) * np.sqrt(3)) + 1e-12)


# ------------------------------------------------------- opaque photosphere

def _obs_geom(n, h, r):
    g = synth.cube_geom(n, h)
    g["r_obs"] = r
    return g


@pytest.mark.parametrize("b", [0.0, 0.31, 0.7, 0.999, 1.2, 1.4])
def test_obstacle_axis_ray_closed_form(b):
    """Ray along -x from (D, b, z) through the cube [-h, h]^3 (z = 0.013
    keeps it off the voxel plane z = 0): its impact parameter is
    p = sqrt(b^2 + z^2); it enters at x = h and, when p < 1, stops on the
    unit sphere at x = sqrt(1 - p^2), so the segment lengths sum to
    h - sqrt(1 - p^2); past the sphere (p > 1) the whole chord 2 h counts."""
    h, D, z = 1.5, 215.0, 0.013
    g = _obs_geom(30, h, 1.0)
    idx, ln, a0, a1 = siddon.segments(g, [D, b, z], [-1.0, 0.0, 0.0])
    p2 = b * b + z * z
    want = h - math.sqrt(1.0 - p2) if p2 < 1.0 else 2 * h
    assert float(np.sum(ln)) == pytest.approx(want, rel=1e-12, abs=1e-12)
    # without the obstacle the same ray crosses the whole cube
    g0 = _obs_geom(30, h, 0.0)
    _, ln0, _, _ = siddon.segments(g0, [D, b, z], [-1.0, 0.0, 0.0])
    assert float(np.sum(ln0)) == pytest.approx(2 * h, rel=1e-12)


def test_obstacle_observer_inside_sphere_sees_nothing():
    g = _obs_geom(10, 1.5, 1.0)
    for o in ([0.2, 0.1, -0.3], [0.0, 0.0, 0.999]):
        idx, ln, _, _ = siddon.segments(g, o, [0.6, 0.0, 0.8])
        assert idx.size == 0


def test_obstacle_brute_force_random_rays():
    """Per-voxel slab clips ended where a scan-and-bisection search finds
    the ray first reaching the sphere, against the oracle's closed-form
    root, on rays aimed near the sphere (some hit it, some miss)."""
    rng = np.random.default_rng(71)
    g = _obs_geom(6, 1.0, 0.55)
    for _ in range(30):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        o = rng.uniform(-0.5, 0.5, 3) - 4.0 * u
        s_end = checks.first_hit(o, u, 0.55, 8.0)
        want = checks.brute_force_ray(g, o, u,
                                      np.inf if s_end is None else s_end)
        np.testing.assert_allclose(_dense(g, o, u), want, rtol=0,
                                   atol=1e-12)


def test_obstacle_fine_sampling_converges():
    rng = np.random.default_rng(72)
    g = _obs_geom(8, 1.0, 0.6)
    x = rng.random((8, 8, 8))
    flat = x.reshape(-1)
    for _ in range(4):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        o = rng.uniform(-0.3, 0.3, 3) - 5.0 * u
        idx, ln, _, _ = siddon.segments(g, o, u)
        exact = float(np.sum(ln * flat[idx]))
        approx = checks.sampled_ray(g, x, o, u, 1e-4, 5.0 + 2 * np.sqrt(3),
                                    r_obs=0.6)
        assert abs(approx - exact) <= (len(idx) + 3) * 1e-4 * x.max()


def test_obstacle_adjoint_identity_and_blocking_fp64():
    """With the photosphere, <P x, y> = <x, P^T y> to FP64 rounding, no
    voxel whose every point lies inside the sphere receives anything, and
    the projection never exceeds the obstacle-free one for a non-negative
    map."""
    rng = np.random.default_rng(73)
    g = _obs_geom(12, 1.5, 1.0)
    ptg = synth.pointing_table([0.0, 70.0, 200.0], [5.0, -10.0, 30.0], 215.0,
                               17, 13, 3.4)
    x = rng.random((12, 12, 12))
    y = rng.random((3, 13, 17))
    Px = siddon.project(g, x, ptg, 17, 13)
    Pty = siddon.backproject(g, y, ptg, 17, 13)
    assert float(np.sum(Px * y)) == pytest.approx(float(np.sum(x * Pty)),
                                                  rel=1e-12)
    c = np.array([(i + 0.5) * g["dx"] + g["x0"] for i in range(12)])
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    far = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2) + np.sqrt(3) * g["dx"] / 2
    assert np.all(Pty[far < 1.0] == 0.0)
    g0 = dict(g, r_obs=0.0)
    assert np.all(Px <= siddon.project(g0, x, ptg, 17, 13) + 1e-12)


# ------------------------------------------------------ Thomson scattering

def _disk_integrals(r, u):
    """Direct quadrature over the limb-darkened solar disk seen from distance
    r (radius 1): an unpolarised ray from direction n, at angle t from the
    direction of Sun centre, scattered at 90 degrees, gives intensity
    1 - (e.n)^2 along each polarisation e; averaged over the azimuth this is
    1 - sin^2(t)/2 for the tangential one and the tangential minus radial
    difference is cos^2(t) - sin^2(t)/2.  The disk's brightness is
    1 - u + u mu with mu the cosine of the emission angle at the surface."""
    from scipy.integrate import quad
    om = math.asin(1.0 / r)

    def bright(t):
        return 1.0 - u + u * math.sqrt(max(1.0 - (r * math.sin(t)) ** 2, 0.0))
    kw = dict(limit=400, epsabs=1e-14, epsrel=1e-12)
    qt = 2 * math.pi * quad(lambda t: bright(t) * (1 - 0.5 * math.sin(t) ** 2)
                            * math.sin(t), 0.0, om, **kw)[0]
    qp = 2 * math.pi * quad(lambda t: bright(t) * (math.cos(t) ** 2 - 0.5 *
                                                   math.sin(t) ** 2)
                            * math.sin(t), 0.0, om, **kw)[0]
    return qt, qp


@pytest.mark.parametrize("r", [1.02, 1.3, 2.0, 5.0])
def test_thomson_coefficients_against_disk_quadrature(r):
    """pi ((1-u) C1 + u C2) and pi ((1-u) C3 + u C4) (Eq. 4C with sin Omega =
    1/r and +1/8 on C4) equal the disk integrals that define them; the
    printed -1/8 on C4 fails them.  Also the surface values and the
    point-source limit (C2/C1 and C4/C3 -> 2/3, the flux ratio of a fully
    limb-darkened disk)."""
    from oracle import thomson
    C1, C2, C3, C4 = [float(v) for v in thomson.coefficients(r)]
    for u in (0.0, 0.4, 1.0):
        qt, qp = _disk_integrals(r, u)
        assert math.pi * ((1 - u) * C1 + u * C2) == pytest.approx(qp, rel=1e-9)
        assert math.pi * ((1 - u) * C3 + u * C4) == pytest.approx(qt, rel=1e-9)
    qt, _ = _disk_integrals(r, 1.0)
    assert math.pi * -C4 != pytest.approx(qt, rel=1e-3)
    c0 = [float(v) for v in thomson.coefficients(1.0)]
    assert c0 == pytest.approx([0.0, 0.25, 4.0 / 3.0, 0.75], abs=1e-15)
    far = [float(v) for v in thomson.coefficients(300.0)]
    assert far[1] / far[0] == pytest.approx(2.0 / 3.0, rel=1e-4)
    assert far[3] / far[2] == pytest.approx(2.0 / 3.0, rel=1e-4)


def test_impact2_matches_pixel_angles():
    """rho^2 of a pixel's ray equals (d sin theta)^2 with theta the angle of
    the pixel from the boresight (boresight on Sun centre, crval 0), for
    rolled views too."""
    ptg = synth.pointing_table([10.0, 200.0], [4.0, -6.0], 215.0, 16, 12, 4.0,
                               roll_deg=17.0)
    r2 = siddon.impact2(ptg, 16, 12)
    for n in range(2):
        d, cu, cv, pu, pv = ptg[n, 0], ptg[n, 4], ptg[n, 5], ptg[n, 6], ptg[n, 7]
        tu = np.tan((np.arange(16) - pu) * cu)
        tv = np.tan((np.arange(12) - pv) * cv)
        t2 = tv[:, None] ** 2 + tu[None, :] ** 2
        np.testing.assert_allclose(r2[n], d * d * t2 / (1 + t2), rtol=1e-10)


def _thomson_golden(golden_dir):
    rows = [ln.split() for ln in open(os.path.join(golden_dir,
                                                   "thomson_voxel_factors.txt"))
            if ln.strip() and not ln.startswith("#")]
    return [tuple(map(float, r)) for r in rows]


def _factors_match_golden(voxel_factors, rows):
    """True when voxel_factors gives the hand-evaluated m and m' at every
    golden voxel centre (one-voxel cubes centred there), and in the same
    [nz][ny][nx] order on a cube whose centres run along each axis."""
    for cx, cy, cz, u, m_want, mp_want in rows:
        g = _geom((1, 1, 1), (cx - 0.05, cy - 0.05, cz - 0.05),
                  (0.1, 0.1, 0.1))
        m, mp = voxel_factors(g, u)
        if not (m.shape == (1, 1, 1) and
                math.isclose(float(m[0, 0, 0]), m_want, rel_tol=1e-13,
                             abs_tol=0.0) and
                math.isclose(float(mp[0, 0, 0]), mp_want, rel_tol=1e-13,
                             abs_tol=0.0)):
            return False
    # centres 2, 3, 4 along one axis, the other two at 0 (u = 0 rows)
    want = {r[0] ** 2 + r[1] ** 2 + r[2] ** 2: (r[4], r[5])
            for r in rows if r[3] == 0.0}
    for axis in range(3):
        n = [1, 1, 1]
        n[axis] = 3
        lo = [-0.5, -0.5, -0.5]
        lo[axis] = 1.5
        m, mp = voxel_factors(_geom(n, lo, (1.0, 1.0, 1.0)), 0.0)
        m, mp = m.reshape(-1), mp.reshape(-1)
        for k, r in enumerate((2.0, 3.0, 4.0)):
            wm, wmp = want[r * r]
            if not (math.isclose(float(m[k]), wm, rel_tol=1e-13) and
                    math.isclose(float(mp[k]), wmp, rel_tol=1e-13)):
                return False
    return True


def test_thomson_voxel_factors_against_hand_values(golden_dir):
    """m and m' (Eq. brightness with Eq. 4C, Section 3.5) equal the values
    reduced by hand at r = sqrt2, 2, 3, 4 for u = 0, 1/2, 1, vanish on and
    inside the photosphere, and come out in [nz][ny][nx] order."""
    from oracle import thomson
    rows = _thomson_golden(golden_dir)
    assert len(rows) == 14
    assert _factors_match_golden(thomson.voxel_factors, rows)


@pytest.mark.parametrize("old,new", [
    ("rr ** 4", "rr ** 2"),                      # r^-2 for r^-4 in m
    ("rr ** 2, 0.0)", "rr ** 4, 0.0)"),          # r^-4 for r^-2 in m'
    ("2.0 * ((1.0 - u) * C3", "((1.0 - u) * C3"),  # factor 2 on m' dropped
    ("u * C2)", "C2)"),                          # Eq. thomson_lo's missing u
    ("u * C4)", "C3)"),                          # C3 for C4
    ("r > 1.0", "r >= 0.0"),                     # scattering inside the Sun
])
def test_thomson_voxel_factors_pin_catches_planted_mistakes(golden_dir, old,
                                                             new):
    """The hand-value pin fails when one of these plausible mistakes is
    planted in a copy of the oracle's voxel_factors (the oracle itself is
    not modified)."""
    import inspect
    import textwrap

    from oracle import thomson
    src = textwrap.dedent(inspect.getsource(thomson.voxel_factors))
    assert src.count(old) == 1, old
    ns = dict(vars(thomson))
    exec(compile(src.replace(old, new), "<planted>", "exec"), ns)
    rows = _thomson_golden(golden_dir)
    assert not _factors_match_golden(ns["voxel_factors"], rows)


@pytest.mark.parametrize("T", [1, 3])
def test_thomson_operators_adjoint_and_rows(T):
    """T_pB and T_B against brute-force rows (exact voxel lengths times the
    voxel-centre factors, rho^2 from the pixel angles), their FP64 adjoint
    identities (pixel mask, map mask, frames), and m = m' = 0 inside the
    photosphere."""
    from oracle import thomson
    g, ptg, mask, rng = _small_scene(T)
    shape = ((T,) if T > 1 else ()) + (g["nz"], g["ny"], g["nx"])
    x = rng.random(shape)
    y = rng.random((5, 6, 10))
    mm = (rng.random((g["nz"], g["ny"], g["nx"])) < 0.2).astype(np.uint8)
    u = 0.6
    m, mp = thomson.voxel_factors(g, u)
    ax = [synth.voxel_centres(g, a) for a in "xyz"]
    rad = np.sqrt(ax[2][:, None, None] ** 2 + ax[1][None, :, None] ** 2 +
                  ax[0][None, None, :] ** 2)
    assert np.all(m[rad <= 1] == 0) and np.all(mp[rad <= 1] == 0)
    assert np.all(m[rad > 1] > 0) and np.all(mp[rad > 1] > 0)
    for kind in (thomson.PB, thomson.B):
        Tx = thomson.project(kind, g, x, ptg, 10, 6, u, mask, T, map_mask=mm)
        Tty = thomson.backproject(kind, g, y, ptg, 10, 6, u, mask, T,
                                  map_mask=mm)
        lhs = float(np.sum(Tx * np.where(mask == 0, y, 0)))
        assert lhs == pytest.approx(float(np.sum(x * Tty)), rel=1e-12)
        if T > 1:
            continue
        keep = (mm == 0).reshape(-1)
        for r in rng.choice(5 * 60, 30, replace=False):
            n, iv, iu = r // 60, (r // 10) % 6, r % 10
            o, dirn = siddon.ray(ptg[n], iu, iv)
            row = checks.brute_force_ray(g, o, dirn) * keep * ptg[n, 10]
            tu = math.tan((iu - ptg[n, 6]) * ptg[n, 4])
            tv = math.tan((iv - ptg[n, 7]) * ptg[n, 5])
            rho2 = ptg[n, 0] ** 2 * (tu * tu + tv * tv) / (1 + tu * tu + tv * tv)
            pm = float(np.sum(row * (m * x).reshape(-1)))
            want = rho2 * pm if kind == thomson.PB else \
                float(np.sum(row * (mp * x).reshape(-1))) - rho2 * pm
            want = 0.0 if mask[n, iv, iu] else want
            assert Tx[n, iv, iu] == pytest.approx(want, rel=1e-10, abs=1e-16)


# ----------------------------------------------- frames and temporal prior

def _temporal_problem(times, lam_t, seed=21):
    g = synth.cube_geom(5, 1.5, ny=4, nz=4)
    rng = np.random.default_rng(seed)
    n = len(times)
    ptg = synth.pointing_table(rng.uniform(0, 360, n), rng.uniform(-30, 30, n),
                               215.0, 8, 8, 3.4, time=np.asarray(times))
    mask = (rng.random((n, 8, 8)) < 0.15).astype(np.uint8)
    y = rng.random((n, 8, 8))
    return g, ptg, mask, y, solver.Problem(g, ptg, 8, 8, y, mask, lam=0.3,
                                           n_frames=2, lam_t=lam_t)


def test_temporal_prior_solves_the_dense_system():
    """Two frames, fractional time stamps, spatial and temporal priors: CG
    reaches the direct solve built from dense rows ((1 - w) and w times the
    brute-force row in the two frames' blocks), block-diagonal spatial
    differences and frame-to-frame differences from index arithmetic."""
    rng = np.random.default_rng(5)
    times = rng.uniform(0, 1, 6)
    g, ptg, mask, y, pb = _temporal_problem(times, lam_t=0.7)
    nv_ = 80
    A = np.zeros((6 * 64, 2 * nv_))
    for r in range(6 * 64):
        n, iv, iu = r // 64, (r // 8) % 8, r % 8
        if mask.reshape(-1)[r]:
            continue
        o, u = siddon.ray(ptg[n], iu, iv)
        row = checks.brute_force_ray(g, o, u) * ptg[n, 10]
        w = times[n]
        A[r, :nv_] = (1 - w) * row
        A[r, nv_:] = w * row
    _, B1 = _dense_AB(_dense_problem())
    B = np.block([[B1, np.zeros_like(B1)], [np.zeros_like(B1), B1]])
    Dt = np.hstack([-np.eye(nv_), np.eye(nv_)])
    ym = np.where(mask == 0, y, 0.0).reshape(-1)
    H = A.T @ A + 0.3 * B.T @ B + 0.7 * Dt.T @ Dt
    x_direct = np.linalg.solve(H, A.T @ ym)
    x_cg, rep = solver.cg(pb, 600)
    np.testing.assert_allclose(x_cg.reshape(-1), x_direct, rtol=0,
                               atol=1e-8 * np.abs(x_direct).max())
    Jmin = float(np.sum((ym - A @ x_direct) ** 2) + 0.3 * np.sum(
        (B @ x_direct) ** 2) + 0.7 * np.sum((Dt @ x_direct) ** 2))
    assert rep["J"][-1] == pytest.approx(Jmin, rel=1e-9)


def test_integer_stamps_without_temporal_prior_decouple():
    """Integer time stamps and lambda_t = 0: the model is block-diagonal, and
    each frame's solution is the static solution of the images taken at its
    time."""
    times = np.array([0, 1, 0, 1, 1, 0], dtype=np.float64)
    g, ptg, mask, y, pb = _temporal_problem(times, lam_t=0.0)
    x, _ = solver.cg(pb, 400)
    for t in (0, 1):
        sel = times == t
        ps = solver.Problem(g, ptg[sel], 8, 8, y[sel], mask[sel], lam=0.3)
        xs, _ = solver.cg(ps, 400)
        np.testing.assert_allclose(x[t], xs, rtol=0,
                                   atol=1e-8 * np.abs(xs).max())
