"""Plane-synchronous walk (TOMO_OPT_PLANE_SYNC = 3: P and P^T) against the
per-ray walk (TOMO_OPT_PLANE_SYNC = 0) and the FP64 oracle.

The plane walk visits every ray's segments in the same order as the per-ray
walk, with the same crossing parameters, so its forward projection must be
bit-identical to the per-ray walk's (zero-length segments at ties add
exact zeros).  Its transpose only reorders float additions: it is held to the
oracle's transpose bound.  The geometries cover every layout and the
fallback: views along x (layout 1: y fastest) and along y (layout 0), rolled
views whose pixel rows run along z (layout 2), views from near the pole
(major axis z), images whose field of view straddles a 45-degree diagonal
(lanes whose major axis differs from the image's take the per-ray walk),
images whose pixels are too dense for the plane walk (all lanes per-ray),
an observer inside the cube, ragged and anisotropic cubes, masks, gains,
time interpolation and bf16 storage.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon
from tests.gpu_util import (assert_close, assert_transpose_close, mask_dev,
                            require_gpu, to_dev, RTOL_F32)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


@pytest.fixture(scope="module")
def ctxs(T):
    plane = T.Context()
    plane.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, 3)
    ray = T.Context()
    ray.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, 0)
    yield plane, ray
    plane.close()
    ray.close()


@pytest.fixture(scope="module")
def auto(T):
    """The default: P^T plane-synchronous, P per image."""
    ctx = T.Context()
    ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, 5)
    yield ctx
    ctx.close()


def _anisotropic():
    return {"nx": 29, "ny": 31, "nz": 33, "x0": -1.4, "y0": -1.55, "z0": -1.3,
            "dx": 2.8 / 29, "dy": 3.1 / 31, "dz": 2.7 / 33}


def _cases():
    """(name, geom, pointing, mask, nu, nv)."""
    rng = np.random.default_rng(21)
    out = []
    g = _anisotropic()
    # axis views (layouts 1 and 0), both directions
    p = synth.pointing_table([0.0, 90.0, 180.0, 270.0], 0.0, 215.0, 37, 53, 3.6)
    out.append(("axis views", g, p, None, 37, 53))
    # rolled by 90 deg: pixel rows run along z (layout 2); random rolls
    p = synth.pointing_table([10.0, 100.0, 200.0, 300.0], [5.0, -5.0, 20.0, -30.0],
                             215.0, 37, 53, 3.6)
    p[:2, 3] = np.pi / 2
    p[2:, 3] = rng.uniform(-np.pi, np.pi, 2)
    out.append(("rolled", g, p, None, 37, 53))
    # near the pole: major axis z
    p = synth.pointing_table([0.0, 45.0, 123.0], [89.0, -88.0, 80.0], 215.0,
                             41, 41, 3.6)
    out.append(("polar", g, p, None, 41, 41))
    # field of view straddling a diagonal (fallback lanes), wide field
    g2 = synth.cube_geom(40, 1.5)
    p = synth.pointing_table([45.0, 135.0, 225.0, 314.8], [0.0, 0.0, 3.0, -3.0],
                             215.0, 64, 48, 8.0)
    out.append(("diagonal", g2, p, None, 64, 48))
    # observer inside the cube, odd cube
    g3 = synth.cube_geom(25, 1.5)
    p = synth.pointing_table([0.0, 90.0, 30.0], [0.0, 0.0, 10.0], 1.2, 31, 31,
                             2.0)
    out.append(("inside", g3, p, None, 31, 31))
    # masks, gains, pointing offsets
    p = synth.pointing_table(rng.uniform(0, 360, 6), rng.uniform(-30, 30, 6),
                             215.0, 37, 53, 3.6, gain=rng.uniform(0.5, 2.0, 6))
    p[:, 8:10] = rng.uniform(-2e-3, 2e-3, (6, 2))
    mask = (rng.random((6, 53, 37)) < 0.1).astype(np.uint8)
    out.append(("masked", g, p, mask, 37, 53))
    c = synth.make_config("single", scale=2)
    out.append(("single/2", c["geom"], c["pointing"], c["mask"], c["nu"], c["nv"]))
    # dense pixels (0.13 voxel apart): the plane hint is not valid and every
    # lane takes the per-ray walk inside the plane kernels
    g4 = synth.cube_geom(33, 1.5)
    p = synth.pointing_table([20.0, 110.0], [3.0, -3.0], 215.0, 250, 40, 3.2)
    out.append(("dense", g4, p, None, 250, 40))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_forward_bit_identical_to_per_ray_walk(T, ctxs, auto, case):
    name, g, ptg, mask, nu, nv = case
    plane, ray = ctxs
    rng = np.random.default_rng(5)
    cube = rng.random((g["nz"], g["ny"], g["nx"])).astype(np.float32)
    md = mask_dev(mask)
    a = T.tomo_project(to_dev(cube), g, ptg, nu, nv, mask=md, ctx=plane)
    b = T.tomo_project(to_dev(cube), g, ptg, nu, nv, mask=md, ctx=ray)
    c = T.tomo_project(to_dev(cube), g, ptg, nu, nv, mask=md, ctx=auto)
    assert torch.equal(a, b), name
    assert torch.equal(c, b), name
    want = siddon.project(g, cube, ptg, nu, nv, mask)
    assert_close(a.cpu().numpy(), want, "P plane %s" % name)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_transpose_against_oracle(T, ctxs, case):
    name, g, ptg, mask, nu, nv = case
    plane, _ = ctxs
    rng = np.random.default_rng(6)
    y = rng.random((ptg.shape[0], nv, nu)).astype(np.float32)
    md = mask_dev(mask)
    got = T.tomo_backproject(to_dev(y), g, ptg, mask=md, ctx=plane)
    want = siddon.backproject(g, y, ptg, nu, nv, mask)
    cw = siddon.crossing_weights(g, y, ptg, nu, nv, mask)
    assert_transpose_close(got.cpu().numpy(), want, cw, g, "P^T plane %s" % name)
    x = rng.random((g["nz"], g["ny"], g["nx"])).astype(np.float32)
    Px = T.tomo_project(to_dev(x), g, ptg, nu, nv, mask=md, ctx=plane)
    lhs = float((Px.double() * to_dev(y).double()).sum())
    rhs = float((to_dev(x).double() * got.double()).sum())
    assert abs(lhs - rhs) <= RTOL_F32 * abs(lhs)


def test_transpose_accumulates(T, ctxs):
    """TOMO_ACCUMULATE adds the transpose (including the parts gathered from
    the layout accumulators) to the cube's content."""
    name, g, ptg, mask, nu, nv = CASES[1]
    plane, _ = ctxs
    rng = np.random.default_rng(7)
    y = to_dev(rng.random((ptg.shape[0], nv, nu)))
    base = to_dev(rng.random((g["nz"], g["ny"], g["nx"])))
    once = T.tomo_backproject(y, g, ptg, ctx=plane)
    acc = base.clone()
    T.tomo_backproject(y, g, ptg, out=acc, accumulate=True, ctx=plane)
    torch.testing.assert_close(acc, base + once, rtol=1e-6, atol=1e-6)
    # a second call must not see leftovers of the first in the accumulators
    again = T.tomo_backproject(y, g, ptg, ctx=plane)
    torch.testing.assert_close(again, once, rtol=1e-6, atol=1e-7 * float(once.abs().max()))


def test_time_interpolation_and_bf16(T, ctxs):
    """Four frames with per-image time stamps: the plane walk equals the
    per-ray walk bit for bit (float32 and bf16 frames), and the transpose
    meets the bound against the oracle."""
    plane, ray = ctxs
    rng = np.random.default_rng(8)
    g = _anisotropic()
    lons = rng.uniform(0, 360, 6)
    ptg = synth.pointing_table(lons, rng.uniform(-20, 20, 6), 215.0, 37, 53,
                               3.6, time=rng.uniform(0, 3, 6))
    ptg[3:, 3] = rng.uniform(-np.pi, np.pi, 3)
    frames = rng.random((4, 33, 31, 29)).astype(np.float32)
    for dt in (torch.float32, torch.bfloat16):
        X = to_dev(frames).to(dt)
        a = T.tomo_project(X, g, ptg, 37, 53, n_frames=4, ctx=plane)
        b = T.tomo_project(X, g, ptg, 37, 53, n_frames=4, ctx=ray)
        assert torch.equal(a, b), dt
        assert torch.equal(T.tomo_project(X, g, ptg, 37, 53, n_frames=4), b), dt
    want = siddon.project(g, frames, ptg, 37, 53, n_frames=4)
    assert_close(T.tomo_project(to_dev(frames), g, ptg, 37, 53, n_frames=4,
                                ctx=plane).cpu().numpy(), want, "P plane time")
    y = rng.random((6, 53, 37)).astype(np.float32)
    got = T.tomo_backproject(to_dev(y), g, ptg, n_frames=4, ctx=plane)
    want_t = siddon.backproject(g, y, ptg, 37, 53, n_frames=4)
    cw = siddon.crossing_weights(g, y, ptg, 37, 53, n_frames=4)
    assert_transpose_close(got.cpu().numpy(), want_t, cw, g, "P^T plane time")


def test_cg256_sampled_bit_identical(T, ctxs):
    """The 256^3 timing workload (240 x 512^2): the plane walk's full
    projection equals the per-ray walk's bit for bit, and its transpose of
    the projection agrees with the per-ray walk's to the float32 summation
    bound on every voxel."""
    plane, ray = ctxs
    c = synth.make_config("cg256")
    md = mask_dev(c["mask"])
    X = to_dev(c["cube"])
    a = T.tomo_project(X, c["geom"], c["pointing"], c["nu"], c["nv"], mask=md,
                       ctx=plane)
    b = T.tomo_project(X, c["geom"], c["pointing"], c["nu"], c["nv"], mask=md,
                       ctx=ray)
    assert torch.equal(a, b)
    ta = T.tomo_backproject(a, c["geom"], c["pointing"], mask=md, ctx=plane)
    tb = T.tomo_backproject(a, c["geom"], c["pointing"], mask=md, ctx=ray)
    # both are float32 sums of the same non-negative terms in different
    # orders: each is within n u of the exact sum, n <= 2 x 240 x 4 terms
    # per voxel at most; 1e-4 relative is far above that and far below any
    # missing or doubled segment
    err = (ta - tb).abs()
    assert float((err - 1e-4 * tb.abs()).max()) <= 1e-6 * float(tb.abs().max())


def test_solve_matches_per_ray_walk(T, ctxs):
    """20 CG iterations on config 'single' at half scale: the plane walk's
    solution and criterion match the per-ray walk's (same FP32 arithmetic
    except for the order of the transpose's atomic additions)."""
    plane, ray = ctxs
    c = synth.make_config("single", scale=2)
    y = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"], c["nv"],
                       c["mask"]).astype(np.float32)
    md = mask_dev(c["mask"])
    xa, ia = T.tomo_solve(to_dev(y), c["geom"], c["pointing"], mask=md,
                          lam=c["lam"], max_iter=20, ctx=plane)
    xb, ib = T.tomo_solve(to_dev(y), c["geom"], c["pointing"], mask=md,
                          lam=c["lam"], max_iter=20, ctx=ray)
    rel = float((xa - xb).norm() / xb.norm())
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(ia["J"], ib["J"], rtol=1e-3)
