"""Batched projector, transpose and CG (one persistent launch / one CUDA
graph for many problems of uneven sizes) against the single-problem path
and the FP64 oracle, plus the tile-shape autotuner."""

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


def _mixed_problems(seed=0, n=6):
    """Uneven cubes (including anisotropic and ragged), image counts and
    sizes, masks and gains; one problem with an empty image stack."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(n):
        side = int(rng.choice([17, 24, 32, 40]))
        g = synth.cube_geom(side, 1.5, ny=side + i, nz=side + 2 * (i % 2))
        n_img = 0 if i == 3 else int(rng.integers(3, 9))
        nu, nv = int(rng.choice([29, 32, 48, 64])), int(rng.choice([24, 33, 64]))
        ptg = synth.pointing_table(rng.uniform(0, 360, n_img),
                                   rng.uniform(-20, 20, n_img), 215.0, nu, nv,
                                   3.4, gain=rng.uniform(0.5, 2.0, n_img))
        cube = rng.random((g["nz"], g["ny"], g["nx"])).astype(np.float32)
        mask = (rng.random((n_img, nv, nu)) < 0.1).astype(np.uint8)
        probs.append({"geom": g, "pointing": ptg, "nu": nu, "nv": nv,
                      "cube_np": cube, "mask_np": mask, "lam": 0.05})
    return probs


def _dev_problems(probs, images=None):
    out = []
    for k, p in enumerate(probs):
        n_img = p["pointing"].shape[0]
        d = dict(p)
        d["cube"] = to_dev(p["cube_np"])
        d["mask"] = mask_dev(p["mask_np"])
        d["images"] = (torch.zeros((n_img, p["nv"], p["nu"]), device="cuda")
                       if images is None else to_dev(images[k]))
        out.append(d)
    return out


def test_project_batched_matches_single_and_oracle(T):
    probs = _mixed_problems()
    dp = _dev_problems(probs)
    T.tomo_project_batched(dp)
    for p, d in zip(probs, dp):
        single = T.tomo_project(d["cube"], p["geom"], p["pointing"], p["nu"],
                                p["nv"], mask=d["mask"])
        # same walk and arithmetic per ray: identical results
        assert torch.equal(d["images"], single)
        want = siddon.project(p["geom"], p["cube_np"], p["pointing"], p["nu"],
                              p["nv"], p["mask_np"])
        assert_close(d["images"].cpu().numpy(), want, "batched P")


def test_backproject_batched_matches_oracle(T):
    probs = _mixed_problems(1)
    rng = np.random.default_rng(5)
    ims = [rng.random((p["pointing"].shape[0], p["nv"], p["nu"])).astype(
        np.float32) for p in probs]
    dp = _dev_problems(probs, ims)
    T.tomo_backproject_batched(dp)
    for p, d, y in zip(probs, dp, ims):
        want = siddon.backproject(p["geom"], y, p["pointing"], p["nu"], p["nv"],
                                  p["mask_np"])
        cw = siddon.crossing_weights(p["geom"], y, p["pointing"], p["nu"],
                                     p["nv"], p["mask_np"])
        assert_transpose_close(d["cube"].cpu().numpy(), want, cw, p["geom"],
                               "batched P^T")
    # accumulate adds a second copy
    before = [d["cube"].clone() for d in dp]
    T.tomo_backproject_batched(dp, accumulate=True)
    for b, d in zip(before, dp):
        torch.testing.assert_close(d["cube"], 2 * b, rtol=1e-5, atol=1e-6)


def test_backproject_batched_walks_every_layout(T):
    """Rolled, polar and axis views (every cube layout of the plane-
    synchronous transpose, and lanes that fall back to the per-ray walk):
    the batched transpose with the plane walk (default) and with the per-ray
    walk both meet the transpose bound against the oracle."""
    rng = np.random.default_rng(9)
    probs = []
    for i, (lons, lats, roll) in enumerate([
            ([0.0, 90.0, 180.0], [0.0, 0.0, 0.0], 0.0),
            ([10.0, 100.0, 230.0], [5.0, -5.0, 10.0], np.pi / 2),
            ([0.0, 45.0, 200.0], [89.0, -88.0, 75.0], 0.3),
            ([45.0, 135.0, 314.8], [0.0, 2.0, -2.0], 0.0)]):
        # odd sides: the exact axis views (lon 0 / 90 / 180, lat 0) must not
        # run inside a voxel plane through the origin, where which voxel gets
        # the segment is decided by 1e-16 perturbations of the input
        side = 25 + 2 * i
        g = synth.cube_geom(side, 1.5, ny=side + 2, nz=side + 4)
        ptg = synth.pointing_table(lons, lats, 215.0, 37, 29, 3.4,
                                   roll_deg=np.degrees(roll))
        probs.append({"geom": g, "pointing": ptg, "nu": 37, "nv": 29,
                      "cube_np": np.zeros((g["nz"], g["ny"], g["nx"]), np.float32),
                      "mask_np": (rng.random((3, 29, 37)) < 0.1).astype(np.uint8),
                      "lam": 0.0})
    ims = [rng.random((3, 29, 37)).astype(np.float32) for _ in probs]
    ray = T.Context()
    ray.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, 0)
    for ctx in (None, ray):
        dp = _dev_problems(probs, ims)
        T.tomo_backproject_batched(dp, ctx=ctx)
        for p, d, y in zip(probs, dp, ims):
            want = siddon.backproject(p["geom"], y, p["pointing"], p["nu"],
                                      p["nv"], p["mask_np"])
            cw = siddon.crossing_weights(p["geom"], y, p["pointing"], p["nu"],
                                         p["nv"], p["mask_np"])
            assert_transpose_close(d["cube"].cpu().numpy(), want, cw,
                                   p["geom"], "batched P^T layouts")
    ray.close()


def _cg_problems(seeds, max_side):
    out = []
    for s in seeds:
        c = synth.configs.batched_problem(s, max_side=max_side)
        y = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"],
                           c["nv"]).astype(np.float32)
        out.append({"geom": c["geom"], "pointing": c["pointing"], "nu": c["nu"],
                    "nv": c["nv"], "cube_np": np.zeros_like(c["cube"]),
                    "mask_np": None, "lam": c["lam"], "y": y,
                    "truth": c["cube"]})
    return out


def test_solve_batched_matches_sequential_and_oracle(T):
    """Eight problems of the batched workload (cube 32-128^3, images capped
    at 64 px): one graph replay of 10 CG iterations equals the one-problem-
    at-a-time solver per problem, and the smaller ones match FP64 CG."""
    probs = _cg_problems(range(100, 108), max_side=64)
    dp = _dev_problems(probs, [p["y"] for p in probs])
    infos = T.tomo_solve_batched(dp, 10)
    for p, d, info in zip(probs, dp, infos):
        x_seq, inf_seq = T.tomo_solve(d["images"], p["geom"], p["pointing"],
                                      lam=p["lam"], max_iter=10)
        # two FP32 runs whose float atomics add in different orders: the
        # same 1e-3 bounds as FP32 CG against FP64 CG (J is reported through
        # y^T M y - x^T (r + b), which loses digits as J falls)
        np.testing.assert_allclose(info["J"], inf_seq["J"], rtol=1e-3)
        rel = float(torch.linalg.norm(d["cube"] - x_seq) /
                    torch.linalg.norm(x_seq))
        assert rel <= 1e-3, rel
    for k in (0, 3):
        p = probs[k]
        pb = solver.Problem(p["geom"], p["pointing"], p["nu"], p["nv"], p["y"],
                            None, lam=p["lam"])
        x_o, rep_o = solver.cg(pb, 10)
        rel = np.linalg.norm(dp[k]["cube"].cpu().numpy() - x_o) / \
            np.linalg.norm(x_o)
        assert rel <= 1e-3, rel
        np.testing.assert_allclose(infos[k]["J"], rep_o["J"], rtol=1e-3)


def test_solve_batched_replay_and_warm_start(T):
    probs = _cg_problems([110, 111, 112], max_side=64)
    dp = _dev_problems(probs, [p["y"] for p in probs])
    a = T.tomo_solve_batched(dp, 6)
    xa = [d["cube"].clone() for d in dp]
    b = T.tomo_solve_batched(dp, 6)  # graph replay, same buffers
    for ia, ib, x, d in zip(a, b, xa, dp):
        np.testing.assert_allclose(ia["J"], ib["J"], rtol=1e-5)
        # float atomics add in a different order on every run
        torch.testing.assert_close(d["cube"], x, rtol=1e-4,
                                   atol=1e-5 * float(x.abs().max()))
    # warm start continues from the current solution
    c = T.tomo_solve_batched(dp, 4, warm_start=True)
    for ib, ic in zip(b, c):
        assert ic["J"][0] == pytest.approx(ib["J"][-1], rel=1e-4)
        assert ic["J"][-1] <= ic["J"][0]


def test_autotune_picks_a_valid_tiling(T):
    c = synth.make_config("small")
    cube = to_dev(c["cube"])
    y = T.tomo_project(cube, c["geom"], c["pointing"], c["nu"], c["nv"])
    ctx = T.Context()
    best = T.tomo_autotune(cube, y, c["geom"], c["pointing"], ctx=ctx)
    assert best["tile_u"] * best["tile_v"] == 256
    assert best["tile_u"] % best["warp_u"] == 0
    assert best["fwd_ms"] > 0 and best["adj_ms"] > 0
    # the tuned shape is used by later calls and gives identical results
    y2 = T.tomo_project(cube, c["geom"], c["pointing"], c["nu"], c["nv"],
                        ctx=ctx)
    assert torch.equal(y, y2)
    ctx.close()


def test_batched_mixes_plane_and_dense_problems(T):
    """One problem with pixels 0.1 voxel apart (it walks per ray, in its own
    schedule) next to two that take the plane walks: the batched forward
    equals the single-problem forward bit for bit, the transpose meets the
    oracle bound, and 4 graph-captured CG iterations match the sequential
    solver."""
    rng = np.random.default_rng(31)
    probs = []
    for side, npx, n_img in [(27, 300, 3), (25, 37, 5), (31, 48, 4)]:
        g = synth.cube_geom(side, 1.5)
        ptg = synth.pointing_table(rng.uniform(0, 360, n_img), 0.0, 215.0,
                                   npx, npx // 2 + 7, 3.2)
        nv = npx // 2 + 7
        probs.append({"geom": g, "pointing": ptg, "nu": npx, "nv": nv,
                      "cube_np": rng.random((side, side, side)).astype(np.float32),
                      "mask_np": None, "lam": 0.05})
    dp = _dev_problems(probs)
    T.tomo_project_batched(dp)
    for p, d in zip(probs, dp):
        single = T.tomo_project(d["cube"], p["geom"], p["pointing"], p["nu"],
                                p["nv"])
        assert torch.equal(d["images"], single)
    ims = [rng.random((p["pointing"].shape[0], p["nv"], p["nu"])).astype(
        np.float32) for p in probs]
    dp = _dev_problems(probs, ims)
    T.tomo_backproject_batched(dp)
    for p, d, y in zip(probs, dp, ims):
        want = siddon.backproject(p["geom"], y, p["pointing"], p["nu"], p["nv"])
        cw = siddon.crossing_weights(p["geom"], y, p["pointing"], p["nu"], p["nv"])
        assert_transpose_close(d["cube"].cpu().numpy(), want, cw, p["geom"],
                               "batched P^T dense mix")
    dp = _dev_problems(probs, ims)
    infos = T.tomo_solve_batched(dp, 4)
    for p, d, info in zip(probs, dp, infos):
        x_seq, inf_seq = T.tomo_solve(d["images"], p["geom"], p["pointing"],
                                      lam=p["lam"], max_iter=4)
        np.testing.assert_allclose(info["J"], inf_seq["J"], rtol=1e-3)
        rel = float(torch.linalg.norm(d["cube"] - x_seq) /
                    torch.linalg.norm(x_seq))
        assert rel <= 1e-3, rel


def test_backproject_batched_layouts_1_and_2_in_one_problem(T):
    """One problem whose images walk in layout 1 (views along x) and in
    layout 2 (rolled views whose pixel rows run along z): both layouts'
    accumulators are added into the same cube in one combine launch."""
    rng = np.random.default_rng(12)
    g = synth.cube_geom(25, 1.5, ny=27, nz=29)
    ptg = synth.pointing_table([0.0, 180.0, 10.0, 190.0], [0.0, 0.0, 5.0, -5.0],
                               215.0, 37, 41, 3.4)
    ptg[2:, 3] = np.pi / 2
    probs = [{"geom": g, "pointing": ptg, "nu": 37, "nv": 41,
              "cube_np": np.zeros((29, 27, 25), np.float32), "mask_np": None,
              "lam": 0.0}]
    y = rng.random((4, 41, 37)).astype(np.float32)
    dp = _dev_problems(probs, [y])
    T.tomo_backproject_batched(dp)
    single = T.tomo_backproject(to_dev(y), g, ptg)
    torch.testing.assert_close(dp[0]["cube"], single, rtol=1e-5,
                               atol=1e-6 * float(single.abs().max()))
    want = siddon.backproject(g, y, ptg, 37, 41)
    cw = siddon.crossing_weights(g, y, ptg, 37, 41)
    assert_transpose_close(dp[0]["cube"].cpu().numpy(), want, cw, g,
                           "batched P^T layouts 1 + 2")


def test_full_batched_workload_against_single_calls_and_oracle(T):
    """The whole 32-problem batched workload (cubes 32-128^3, 16-120 images
    of 64-512^2): the batched forward equals the single-problem forward bit
    for bit on every problem; the batched transpose agrees with the
    single-problem transpose on every voxel of every problem, and with the
    FP64 oracle per voxel on four problems (the largest images among them);
    10 graph-replayed CG iterations match the sequential solver."""
    ctx = T.Context()
    confs = synth.configs.batched()
    probs, ims, singles = [], [], []
    rng = np.random.default_rng(3232)
    for c in confs:
        cube = to_dev(c["cube"])
        n_img = c["pointing"].shape[0]
        probs.append({"geom": c["geom"], "pointing": c["pointing"],
                      "nu": c["nu"], "nv": c["nv"], "cube": cube,
                      "images": torch.zeros((n_img, c["nv"], c["nu"]),
                                            device="cuda"),
                      "lam": c["lam"]})
        ims.append(rng.random((n_img, c["nv"], c["nu"])).astype(np.float32))
    T.tomo_project_batched(probs, ctx=ctx)
    for p in probs:
        single = T.tomo_project(p["cube"], p["geom"], p["pointing"], p["nu"],
                                p["nv"], ctx=ctx)
        assert torch.equal(p["images"], single)
    adj = [dict(p, images=to_dev(y), cube=torch.zeros_like(p["cube"]))
           for p, y in zip(probs, ims)]
    T.tomo_backproject_batched(adj, ctx=ctx)
    for p, d, y in zip(probs, adj, ims):
        single = T.tomo_backproject(d["images"], p["geom"], p["pointing"],
                                    ctx=ctx)
        torch.testing.assert_close(d["cube"], single, rtol=1e-5,
                                   atol=1e-6 * float(single.abs().max()))
    # oracle per voxel: the two problems with the largest images and two
    # with the largest cubes
    by_px = sorted(range(len(confs)), key=lambda i: -confs[i]["nu"])
    by_vox = sorted(range(len(confs)), key=lambda i: -confs[i]["geom"]["nx"])
    pick = []
    for i in by_px[:2] + by_vox:
        if i not in pick:
            pick.append(i)
        if len(pick) == 4:
            break
    for i in pick:
        c, y = confs[i], ims[i]
        want = siddon.backproject(c["geom"], y, c["pointing"], c["nu"], c["nv"])
        cw = siddon.crossing_weights(c["geom"], y, c["pointing"], c["nu"],
                                     c["nv"])
        assert_transpose_close(adj[i]["cube"].cpu().numpy(), want, cw,
                               c["geom"], "batched P^T full workload %d" % i)
    # CG: data = the batched forward of the cube
    cg = [dict(p, cube=torch.zeros_like(p["cube"])) for p in probs]
    infos = T.tomo_solve_batched(cg, 10, ctx=ctx)
    for p, d, info in zip(probs, cg, infos):
        x_seq, inf_seq = T.tomo_solve(p["images"], p["geom"], p["pointing"],
                                      lam=p["lam"], max_iter=10, ctx=ctx)
        np.testing.assert_allclose(info["J"], inf_seq["J"], rtol=1e-3)
        rel = float(torch.linalg.norm(d["cube"] - x_seq) /
                    torch.linalg.norm(x_seq))
        assert rel <= 1e-3, rel
    ctx.close()
