"""Height-weighted prior (Eq. srt_inversion: B = D R, R diagonal with the
voxels' height) and the multi-spacecraft static workflow (Eq. two_spacecraft,
Eq. lin2space, Eq. srt_multiple_inv: image stacks of several instruments,
each with its own gain, concatenated into one problem).

The weighted stencil runs in the same prior kernels as the unweighted one;
these cases compare it with the FP64 oracle's R D^T D R, the solver with
FP64 CG on the weighted criterion (with and without a map mask), the
batched solver with the single-problem one, and the concatenated stacks of
two spacecraft with the separate ones.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon, solver
from tests.gpu_util import (assert_close, assert_transpose_close, mask_dev,
                            require_gpu, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def test_weighted_prior_matches_oracle(T):
    """lambda R D^T D R x against the oracle, per voxel within the float32
    rounding of the weighted stencil; unit weights give the unweighted
    stencil bit for bit."""
    rng = np.random.default_rng(1)
    g = {"nx": 37, "ny": 21, "nz": 13, "x0": -1.2, "y0": -0.7, "z0": -0.4,
         "dx": 2.4 / 37, "dy": 1.4 / 21, "dz": 0.8 / 13}
    x = rng.standard_normal((13, 21, 37)).astype(np.float32)
    w = synth.height_weights(g, 0.3, 0.02).astype(np.float32)
    lam = 0.37
    want = lam * w * solver.DtD(w.astype(np.float64) * x)
    got = T.tomo_prior_apply(to_dev(x), g, lam,
                             prior_weight=to_dev(w)).cpu().numpy()
    # each of the 12 products and differences rounds once in float32
    bound = 16 * 2.0 ** -24 * lam * w * 12 * float(np.abs(w * x).max())
    err = np.abs(got - want)
    assert np.all(err <= bound), float((err / bound).max())
    acc = T.tomo_prior_apply(to_dev(x), g, lam, out=to_dev(x.copy()),
                             accumulate=True,
                             prior_weight=to_dev(w)).cpu().numpy()
    assert np.all(np.abs(acc - (x + want)) <=
                  bound + 2.0 ** -23 * np.abs(x + want))
    ones = torch.ones((13, 21, 37), device="cuda")
    assert torch.equal(T.tomo_prior_apply(to_dev(x), g, lam, prior_weight=ones),
                       T.tomo_prior_apply(to_dev(x), g, lam))


@pytest.mark.parametrize("with_map_mask", [False, True])
def test_solve_against_fp64_cg(T, with_map_mask):
    """10 CG iterations on ||y - P x||^2 + lambda ||D R x||^2 with R the
    altitude above the photosphere (floored at 0.05) on the small
    configuration, against FP64 CG on the same criterion."""
    c = synth.make_config("small")
    g = c["geom"]
    w = synth.height_weights(g, 1.0, 0.05).astype(np.float32)
    mm = synth.shell_map_mask(g, 1.0) if with_map_mask else None
    y = siddon.project(g, c["cube"], c["pointing"], c["nu"],
                       c["nv"]).astype(np.float32)
    lam = 5e-2
    pb = solver.Problem(g, c["pointing"], c["nu"], c["nv"], y, None, lam=lam,
                        map_mask=mm, prior_weight=w)
    x_o, rep_o = solver.cg(pb, 10)
    x_g, info = T.tomo_solve(to_dev(y), g, c["pointing"], lam=lam,
                             max_iter=10, prior_weight=to_dev(w),
                             map_mask=mask_dev(mm))
    rel = np.linalg.norm(x_g.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=1e-3)
    # the weight changes the solution (it is not ignored)
    pu = solver.Problem(g, c["pointing"], c["nu"], c["nv"], y, None, lam=lam,
                        map_mask=mm)
    x_u, _ = solver.cg(pu, 10)
    assert np.linalg.norm(x_u - x_o) > 0.05 * np.linalg.norm(x_o)


def test_batched_matches_single(T):
    """Batched CG with weighted priors on some problems (and a map mask on
    one) against the single-problem solver."""
    rng = np.random.default_rng(4)
    probs = []
    for k, (n, nimg, npx) in enumerate([(24, 6, 40), (31, 5, 48), (20, 7, 36)]):
        g = synth.cube_geom(n, 1.6)
        ptg = synth.pointing_table(rng.uniform(0, 360, nimg),
                                   rng.uniform(-10, 10, nimg), 215.0, npx,
                                   npx, 3.4)
        cube = rng.random((n, n, n)).astype(np.float32)
        y = siddon.project(g, cube, ptg, npx, npx).astype(np.float32)
        p = {"geom": g, "pointing": ptg, "nu": npx, "nv": npx, "lam": 0.05,
             "images": to_dev(y), "cube": torch.zeros((n, n, n), device="cuda")}
        if k != 1:
            p["prior_weight"] = to_dev(synth.height_weights(g, 1.0, 0.05))
        if k == 2:
            p["map_mask"] = mask_dev(synth.shell_map_mask(g, 0.9))
        probs.append(p)
    infos = T.tomo_solve_batched(probs, 8)
    for p, info in zip(probs, infos):
        x_s, inf_s = T.tomo_solve(p["images"], p["geom"], p["pointing"],
                                  lam=p["lam"], max_iter=8,
                                  prior_weight=p.get("prior_weight"),
                                  map_mask=p.get("map_mask"))
        np.testing.assert_allclose(info["J"], inf_s["J"], rtol=1e-3)
        rel = float(torch.linalg.norm(p["cube"] - x_s) / torch.linalg.norm(x_s))
        assert rel <= 1e-3, rel


def test_two_spacecraft(T):
    """Eq. lin2space: the stack of spacecraft A and B (own distances and
    gains) is one problem.  Its projection is the two projections stacked
    (bit for bit), its transpose meets the oracle bound, and Eq.
    srt_multiple_inv (weighted prior) solved on the stack matches FP64 CG."""
    c = synth.make_config("small")
    g = c["geom"]
    rng = np.random.default_rng(9)
    pa = synth.pointing_table(rng.uniform(0, 360, 6), rng.uniform(-7, 7, 6),
                              215.0, 48, 48, 3.4, gain=1.0)
    pb = synth.pointing_table(rng.uniform(0, 360, 5), rng.uniform(-7, 7, 5),
                              190.0, 48, 48, 3.4, gain=0.6)
    pab = np.concatenate([pa, pb])
    X = to_dev(c["cube"])
    ya = T.tomo_project(X, g, pa, 48, 48)
    yb = T.tomo_project(X, g, pb, 48, 48)
    yab = T.tomo_project(X, g, pab, 48, 48)
    assert torch.equal(yab, torch.cat([ya, yb]))
    want = siddon.project(g, c["cube"], pab, 48, 48)
    assert_close(yab.cpu().numpy(), want, "P_AB")
    v = rng.random((11, 48, 48)).astype(np.float32)
    got_t = T.tomo_backproject(to_dev(v), g, pab).cpu().numpy()
    assert_transpose_close(got_t, siddon.backproject(g, v, pab, 48, 48),
                           siddon.crossing_weights(g, v, pab, 48, 48), g,
                           "P_AB^T")
    w = synth.height_weights(g, 1.0, 0.05).astype(np.float32)
    y = want.astype(np.float32)
    prob = solver.Problem(g, pab, 48, 48, y, None, lam=2e-2, prior_weight=w)
    x_o, rep_o = solver.cg(prob, 10)
    x_g, info = T.tomo_solve(to_dev(y), g, pab, lam=2e-2, max_iter=10,
                             prior_weight=to_dev(w))
    rel = np.linalg.norm(x_g.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=1e-3)
