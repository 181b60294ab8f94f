"""Map mask: voxels excluded from the map (Section 4 names masks of the data
and of the map).  An excluded voxel is not an unknown: P reads it as 0,
P^T gives it nothing, and CG solves the system restricted to the other
voxels.

The GPU path applies the mask element-wise around unchanged walks (a masked
copy of the cube before P, K after P^T, and inside the CG vector kernels);
these cases compare it with the FP64 oracle (which applies the mask in its
own code), with the unmasked path on a host-zeroed cube, and the batched
path with the single-problem one.  Masks: a spherical shell (photosphere
and field edge, the solar-tomography use) and random voxels.
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


def _scene(seed=0, n_frames=1):
    """Anisotropic cube, five views (longitudes, latitudes, rolls, gains and
    time stamps), a pixel mask, a shell map mask with some random voxels
    added."""
    rng = np.random.default_rng(seed)
    g = {"nx": 29, "ny": 31, "nz": 33, "x0": -1.4, "y0": -1.55, "z0": -1.3,
         "dx": 2.8 / 29, "dy": 3.1 / 31, "dz": 2.7 / 33}
    ptg = synth.pointing_table([0.0, 90.0, 33.0, 150.0, 260.0],
                               [0.0, 3.0, -8.0, 25.0, 0.5], 215.0, 37, 41, 3.0,
                               gain=rng.uniform(0.5, 2.0, 5),
                               time=rng.uniform(0, max(n_frames - 1, 0), 5))
    ptg[2:, 3] = rng.uniform(-np.pi, np.pi, 3)
    mask = (rng.random((5, 41, 37)) < 0.05).astype(np.uint8)
    mm = synth.shell_map_mask(g, 0.5, 1.35)
    mm |= (rng.random(mm.shape) < 0.05).astype(np.uint8) * 3
    return g, ptg, mask, mm


@pytest.mark.parametrize("n_frames", [1, 3])
def test_projection_and_transpose_against_oracle(T, n_frames):
    g, ptg, mask, mm = _scene(0, n_frames)
    rng = np.random.default_rng(1)
    shape = ((n_frames,) if n_frames > 1 else ()) + (33, 31, 29)
    cube = rng.random(shape).astype(np.float32)
    md, mmd = mask_dev(mask), mask_dev(mm)
    want = siddon.project(g, cube, ptg, 37, 41, mask, n_frames=n_frames,
                          map_mask=mm)
    y = rng.random((5, 41, 37)).astype(np.float32)
    want_t = siddon.backproject(g, y, ptg, 37, 41, mask, n_frames=n_frames,
                                map_mask=mm)
    cw = siddon.crossing_weights(g, y, ptg, 37, 41, mask, n_frames=n_frames)
    # the same walk on a cube zeroed on the host
    zeroed = to_dev(cube * (mm == 0))
    for mode in (0, 3, 5):
        ctx = T.Context()
        ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, mode)
        X = to_dev(cube)
        got = T.tomo_project(X, g, ptg, 37, 41, mask=md, n_frames=n_frames,
                             map_mask=mmd, ctx=ctx)
        assert_close(got.cpu().numpy(), want, "P map mask mode %d" % mode)
        assert torch.equal(got, T.tomo_project(zeroed, g, ptg, 37, 41, mask=md,
                                               n_frames=n_frames, ctx=ctx))
        assert torch.equal(X, to_dev(cube))  # the caller's cube is untouched
        got_t = T.tomo_backproject(to_dev(y), g, ptg, mask=md,
                                   n_frames=n_frames, map_mask=mmd, ctx=ctx)
        gt = got_t.cpu().numpy()
        assert np.all(gt.reshape(-1, mm.size)[:, mm.reshape(-1) != 0] == 0.0)
        assert_transpose_close(gt, want_t, cw, g, "P^T map mask mode %d" % mode)
        # accumulate: excluded voxels keep their value, the others add K P^T y
        base = rng.random(shape).astype(np.float32)
        acc = to_dev(base)
        T.tomo_backproject(to_dev(y), g, ptg, mask=md, n_frames=n_frames,
                           map_mask=mmd, out=acc, accumulate=True, ctx=ctx)
        out_acc = acc.cpu().numpy().reshape(-1, mm.size)
        out_base = base.reshape(-1, mm.size)
        assert np.array_equal(out_acc[:, mm.reshape(-1) != 0],
                              out_base[:, mm.reshape(-1) != 0])
        # the transpose bound, plus the rounding of the final float addition
        t_max = float(np.sqrt(sum((g["n" + a] * g["d" + a]) ** 2
                                  for a in "xyz")))
        got_a = acc.cpu().numpy().astype(np.float64)
        err = np.abs(got_a - base - want_t)
        bound = (1e-5 * np.abs(want_t) + 8.0 * 2.0 ** -24 * t_max * cw +
                 2.0 ** -23 * (np.abs(base) + np.abs(want_t)))
        assert np.all(err <= bound), float((err / bound).max())
        ctx.close()


def test_bf16_cube(T):
    """The masked copy keeps bf16 storage: P of a bf16 cube with a map mask
    equals P of the host-zeroed bf16 cube bit for bit."""
    g, ptg, mask, mm = _scene(4)
    rng = np.random.default_rng(2)
    cube = rng.random((33, 31, 29)).astype(np.float32)
    Xb = to_dev(cube).to(torch.bfloat16)
    zb = Xb * to_dev(mm == 0).to(torch.bfloat16)
    got = T.tomo_project(Xb, g, ptg, 37, 41, map_mask=mask_dev(mm))
    assert torch.equal(got, T.tomo_project(zb, g, ptg, 37, 41))
    want = siddon.project(g, Xb.float().cpu().numpy(), ptg, 37, 41,
                          map_mask=mm)
    assert_close(got.cpu().numpy(), want, "P bf16 map mask")


def test_all_excluded_and_all_kept(T):
    g, ptg, mask, _ = _scene(5)
    rng = np.random.default_rng(3)
    X = to_dev(rng.random((33, 31, 29)).astype(np.float32))
    y = to_dev(rng.random((5, 41, 37)).astype(np.float32))
    full = torch.ones((33, 31, 29), dtype=torch.uint8, device="cuda")
    none = torch.zeros_like(full)
    assert float(T.tomo_project(X, g, ptg, 37, 41, map_mask=full).abs().max()) == 0
    assert float(T.tomo_backproject(y, g, ptg, map_mask=full).abs().max()) == 0
    x, info = T.tomo_solve(y, g, ptg, lam=0.1, max_iter=3, map_mask=full)
    assert float(x.abs().max()) == 0 and info["iters"] == 0
    assert torch.equal(T.tomo_project(X, g, ptg, 37, 41, map_mask=none),
                       T.tomo_project(X, g, ptg, 37, 41))


def test_solve_against_fp64_cg(T):
    """10 CG iterations on the restricted system (shell map mask on the
    small configuration) against FP64 CG with the same map mask, from zero
    and from a warm start that is nonzero on the excluded voxels."""
    c = synth.make_config("small")
    g = c["geom"]
    mm = synth.shell_map_mask(g, 1.0, 1.6)
    assert 0.2 < mm.mean() < 0.8
    y = siddon.project(g, c["cube"], c["pointing"], c["nu"],
                       c["nv"]).astype(np.float32)
    pb = solver.Problem(g, c["pointing"], c["nu"], c["nv"], y, None, lam=1e-2,
                        map_mask=mm)
    x_o, rep_o = solver.cg(pb, 10)
    x_g, info = T.tomo_solve(to_dev(y), g, c["pointing"], lam=1e-2,
                             max_iter=10, map_mask=mask_dev(mm))
    xg = x_g.cpu().numpy()
    assert np.all(xg[mm != 0] == 0.0)
    rel = np.linalg.norm(xg - x_o) / np.linalg.norm(x_o)
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=1e-3)
    # warm start: x0 is restricted in place first
    x0 = np.random.default_rng(6).random(mm.shape).astype(np.float32)
    x_o2, rep_o2 = solver.cg(pb, 6, x0=x0)
    for bf16 in (False, True):
        x_w, info_w = T.tomo_solve(to_dev(y), g, c["pointing"], lam=1e-2,
                                   max_iter=6, x0=to_dev(x0), bf16=bf16,
                                   map_mask=mask_dev(mm))
        xw = x_w.cpu().numpy()
        assert np.all(xw[mm != 0] == 0.0)
        if not bf16:
            rel = np.linalg.norm(xw - x_o2) / np.linalg.norm(x_o2)
            assert rel <= 1e-3, rel
            np.testing.assert_allclose(info_w["J"], rep_o2["J"], rtol=1e-3)
        else:  # bf16 directions: exact line searches, J decreases
            assert info_w["J"][0] == pytest.approx(rep_o2["J"][0], rel=1e-3)
            assert np.all(np.diff(info_w["J"]) <= 1e-6 * info_w["J"][0])
            assert info_w["J"][-1] < info_w["J"][0]


def _batch(seed, with_mm):
    g, ptg, mask, mm = _scene(seed)
    rng = np.random.default_rng(seed + 10)
    cube = rng.random((33, 31, 29)).astype(np.float32)
    y = rng.random((5, 41, 37)).astype(np.float32)
    p = {"geom": g, "pointing": ptg, "nu": 37, "nv": 41, "cube": to_dev(cube),
         "mask": mask_dev(mask), "lam": 0.05, "images": to_dev(y)}
    if with_mm:
        p["map_mask"] = mask_dev(mm)
    return p, cube, y, mask, mm


def test_batched_matches_single(T):
    """Batched P, P^T (plain and accumulating) and CG with map masks on some
    problems against the single-problem calls."""
    items = [_batch(20, True), _batch(21, False), _batch(22, True)]
    probs = [it[0] for it in items]
    for p, cube, y, mask, mm in items:
        p["images"] = torch.zeros((5, 41, 37), device="cuda")
    T.tomo_project_batched(probs)
    for p, cube, y, mask, mm in items:
        single = T.tomo_project(to_dev(cube), p["geom"], p["pointing"], 37, 41,
                                mask=p["mask"], map_mask=p.get("map_mask"))
        assert torch.equal(p["images"], single)
        assert torch.equal(p["cube"], to_dev(cube))
    for p, cube, y, mask, mm in items:
        p["images"] = to_dev(y)
    base = [p["cube"].clone() for p in probs]
    T.tomo_backproject_batched(probs, accumulate=True)
    acc = [p["cube"].clone() for p in probs]
    T.tomo_backproject_batched(probs)
    for k, (p, cube, y, mask, mm) in enumerate(items):
        use = p.get("map_mask") is not None
        want = siddon.backproject(p["geom"], y, p["pointing"], 37, 41, mask,
                                  map_mask=mm if use else None)
        cw = siddon.crossing_weights(p["geom"], y, p["pointing"], 37, 41, mask)
        got = p["cube"].cpu().numpy()
        assert_transpose_close(got, want, cw, p["geom"], "batched P^T %d" % k)
        if use:
            assert np.all(got[mm != 0] == 0.0)
            assert torch.equal(acc[k][mask_dev(mm) != 0],
                               base[k][mask_dev(mm) != 0])
        torch.testing.assert_close(acc[k] - base[k], p["cube"], rtol=1e-5,
                                   atol=4e-7 * float(base[k].abs().max()))
    for p in probs:
        p["cube"] = torch.zeros_like(p["cube"])
    infos = T.tomo_solve_batched(probs, 8)
    for (p, cube, y, mask, mm), info in zip(items, infos):
        x_s, inf_s = T.tomo_solve(p["images"], p["geom"], p["pointing"],
                                  mask=p["mask"], lam=p["lam"], max_iter=8,
                                  map_mask=p.get("map_mask"))
        np.testing.assert_allclose(info["J"], inf_s["J"], rtol=1e-3)
        rel = float(torch.linalg.norm(p["cube"] - x_s) / torch.linalg.norm(x_s))
        assert rel <= 1e-3, rel
        if p.get("map_mask") is not None:
            assert float(p["cube"][p["map_mask"] != 0].abs().max()) == 0.0
    # warm start from a cube that is nonzero on the excluded voxels
    for p in probs:
        p["cube"].fill_(0.5)
    infos = T.tomo_solve_batched(probs, 3, warm_start=True)
    for p in probs:
        if p.get("map_mask") is not None:
            assert float(p["cube"][p["map_mask"] != 0].abs().max()) == 0.0


def test_autograd(T):
    """The gradient of <w, P K x> is K P^T w."""
    from paper_1103_5904_gb300 import autograd
    g, ptg, mask, mm = _scene(7)
    rng = np.random.default_rng(8)
    X = to_dev(rng.random((33, 31, 29)).astype(np.float32)).requires_grad_(True)
    w = to_dev(rng.random((5, 41, 37)).astype(np.float32))
    y = autograd.project(X, g, ptg, 37, 41, mask=mask_dev(mask),
                         map_mask=mask_dev(mm))
    (y * w).sum().backward()
    want = siddon.backproject(g, w.cpu().numpy(), ptg, 37, 41, mask,
                              map_mask=mm)
    cw = siddon.crossing_weights(g, w.cpu().numpy(), ptg, 37, 41, mask)
    assert_transpose_close(X.grad.cpu().numpy(), want, cw, g, "autograd K P^T")
