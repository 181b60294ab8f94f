"""Opaque photosphere (cube geometry r_obs > 0): lines of sight end where
they first reach the sphere of that radius at the origin (Section 4 ends
the line-of-sight integration at the photosphere).

The GPU path applies it in the FP64 ray setup, so every walk inherits it
through the chord; these cases compare P, P^T and CG with the FP64 oracle
(which implements the sphere separately), the walks with each other, and
the batched path with the single-problem one.  The views include rays that
hit the sphere, rays that graze it and rays that miss it, and an observer
inside the sphere.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon, solver
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


def _scene(seed=0):
    """Anisotropic cube around the Sun with the photosphere, views at
    several longitudes and latitudes, random rolls and a pixel mask."""
    rng = np.random.default_rng(seed)
    g = {"nx": 29, "ny": 31, "nz": 33, "x0": -1.4, "y0": -1.55, "z0": -1.3,
         "dx": 2.8 / 29, "dy": 3.1 / 31, "dz": 2.7 / 33, "r_obs": 1.0}
    ptg = synth.pointing_table([0.0, 90.0, 33.0, 150.0, 260.0],
                               [0.0, 3.0, -8.0, 25.0, 0.5], 215.0, 37, 41, 3.0)
    ptg[2:, 3] = rng.uniform(-np.pi, np.pi, 3)
    mask = (rng.random((5, 41, 37)) < 0.05).astype(np.uint8)
    return g, ptg, mask


def test_projection_and_transpose_against_oracle(T):
    g, ptg, mask = _scene()
    rng = np.random.default_rng(1)
    cube = rng.random((33, 31, 29)).astype(np.float32)
    md = mask_dev(mask)
    want = siddon.project(g, cube, ptg, 37, 41, mask)
    # the sphere really blocks part of the view
    g0 = dict(g, r_obs=0.0)
    assert np.sum(want) < 0.9 * np.sum(siddon.project(g0, cube, ptg, 37, 41,
                                                       mask))
    outs = []
    for mode in (0, 3, 5):
        ctx = T.Context()
        ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, mode)
        got = T.tomo_project(to_dev(cube), g, ptg, 37, 41, mask=md, ctx=ctx)
        assert_close(got.cpu().numpy(), want, "P obstacle mode %d" % mode)
        outs.append(got)
        y = rng.random((5, 41, 37)).astype(np.float32)
        got_t = T.tomo_backproject(to_dev(y), g, ptg, mask=md, ctx=ctx)
        want_t = siddon.backproject(g, y, ptg, 37, 41, mask)
        cw = siddon.crossing_weights(g, y, ptg, 37, 41, mask)
        assert_transpose_close(got_t.cpu().numpy(), want_t, cw, g,
                               "P^T obstacle mode %d" % mode)
        ctx.close()
    # every walk sees the same segments
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_observer_inside_sphere_projects_nothing(T):
    g = synth.cube_geom(17, 1.5)
    g["r_obs"] = 1.0
    ptg = synth.pointing_table([10.0, 200.0], [0.0, 40.0], 0.5, 21, 21, 2.0)
    out = T.tomo_project(torch.ones((17, 17, 17), device="cuda"), g, ptg, 21,
                         21)
    assert float(out.abs().max()) == 0.0
    x = T.tomo_backproject(torch.ones((2, 21, 21), device="cuda"), g, ptg)
    assert float(x.abs().max()) == 0.0


def test_paper_workload_sampled(T):
    """The paper's performance workload (64 x 256^2 around a 128^3 cube,
    no pixel mask) with the photosphere: 1 % of the pixels against the
    oracle, the transpose by a dot test on them."""
    c = synth.make_config("paper128")
    g = dict(c["geom"], r_obs=1.0)
    X = to_dev(c["cube"])
    got = T.tomo_project(X, g, c["pointing"], c["nu"], c["nv"]).cpu().numpy()
    got = got.reshape(-1)
    rng = np.random.default_rng(5)
    ids = np.sort(rng.choice(got.size, got.size // 100, replace=False))
    want = siddon.project(g, c["cube"], c["pointing"], c["nu"], c["nv"],
                          ray_ids=ids)
    assert_close(got[ids], want, "P paper128 obstacle sampled")
    y = np.zeros(got.size, np.float32)
    y[ids] = rng.random(ids.size).astype(np.float32)
    Pty = T.tomo_backproject(to_dev(y.reshape(-1, c["nv"], c["nu"])), g,
                             c["pointing"])
    lhs = float(np.sum(want * y[ids].astype(np.float64)))
    rhs = float(torch.sum(X.double() * Pty.double()))
    assert abs(lhs - rhs) <= RTOL_F32 * abs(lhs)


def test_solve_against_fp64_cg(T):
    """10 CG iterations with the photosphere on the small configuration's
    geometry against FP64 CG (bounds of the solver tests)."""
    c = synth.make_config("small")
    g = dict(c["geom"], r_obs=1.0)
    y = siddon.project(g, c["cube"], c["pointing"], c["nu"],
                       c["nv"]).astype(np.float32)
    pb = solver.Problem(g, c["pointing"], c["nu"], c["nv"], y, None,
                        lam=1e-2)
    x_o, rep_o = solver.cg(pb, 10)
    x_g, info = T.tomo_solve(to_dev(y), g, c["pointing"], lam=1e-2,
                             max_iter=10)
    rel = np.linalg.norm(x_g.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=1e-3)


def test_batched_matches_single(T):
    """The batched forward equals the single-problem forward bit for bit
    with the photosphere, and the batched transpose meets the oracle bound."""
    g, ptg, mask = _scene(2)
    rng = np.random.default_rng(3)
    cube = rng.random((33, 31, 29)).astype(np.float32)
    probs = [{"geom": g, "pointing": ptg, "nu": 37, "nv": 41,
              "cube": to_dev(cube), "mask": mask_dev(mask), "lam": 0.0,
              "images": torch.zeros((5, 41, 37), device="cuda")}]
    T.tomo_project_batched(probs)
    single = T.tomo_project(to_dev(cube), g, ptg, 37, 41, mask=mask_dev(mask))
    assert torch.equal(probs[0]["images"], single)
    y = rng.random((5, 41, 37)).astype(np.float32)
    probs[0]["images"] = to_dev(y)
    T.tomo_backproject_batched(probs)
    want = siddon.backproject(g, y, ptg, 37, 41, mask)
    cw = siddon.crossing_weights(g, y, ptg, 37, 41, mask)
    assert_transpose_close(probs[0]["cube"].cpu().numpy(), want, cw, g,
                           "batched P^T obstacle")
