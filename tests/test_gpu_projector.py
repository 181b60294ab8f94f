"""GPU projector P and transpose P^T against the FP64 oracle.

Every case builds its inputs with the seeded ``synth`` generators, runs the
CUDA path through the C ABI (``paper_1103_5904_gb300.tomo``) and the oracle
on the same inputs, and compares element by element (tolerances in
``gpu_util``).  Full-size workloads are compared on seeded pixel subsets the
oracle computes ray by ray.
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


def _ragged_scene(seed=3, T_frames=1):
    """Anisotropic cube with ragged sizes, odd images (so one pixel looks
    exactly along an axis), random observers, roll, pointing offsets, gains,
    masks and time stamps."""
    rng = np.random.default_rng(seed)
    g = {"nx": 29, "ny": 31, "nz": 33, "x0": -1.4, "y0": -1.55, "z0": -1.3,
         "dx": 2.8 / 29, "dy": 3.1 / 31, "dz": 2.7 / 33}
    lons = np.concatenate([[0.0, 90.0], rng.uniform(0, 360, 3)])
    lats = np.concatenate([[0.0, 0.0], rng.uniform(-30, 30, 3)])
    ptg = synth.pointing_table(lons, lats, 215.0, 37, 53, 3.6,
                               gain=rng.uniform(0.5, 2.0, 5),
                               time=rng.uniform(0, max(T_frames - 1, 0), 5))
    ptg[2:, 3] = rng.uniform(-np.pi, np.pi, 3)       # roll
    ptg[2:, 8:10] = rng.uniform(-2e-3, 2e-3, (3, 2))  # crval offsets
    mask = (rng.random((5, 53, 37)) < 0.1).astype(np.uint8)
    shape = ((T_frames,) if T_frames > 1 else ()) + (33, 31, 29)
    cube = rng.random(shape).astype(np.float32)
    return g, ptg, mask, cube


def test_small_config_full_projection(T):
    """Config 'small' (64^3, 8 x 64^2, radial density + 10 % noise): every
    pixel of P within tolerance."""
    c = synth.make_config("small")
    want = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"], c["nv"])
    got = T.tomo_project(to_dev(c["cube"]), c["geom"], c["pointing"],
                         c["nu"], c["nv"]).cpu().numpy()
    assert_close(got, want, "P small")


def test_small_config_full_transpose_and_dot(T):
    c = synth.make_config("small")
    rng = np.random.default_rng(0)
    y = rng.random((8, c["nv"], c["nu"])).astype(np.float32)
    want = siddon.backproject(c["geom"], y, c["pointing"], c["nu"], c["nv"])
    cw = siddon.crossing_weights(c["geom"], y, c["pointing"], c["nu"], c["nv"])
    got = T.tomo_backproject(to_dev(y), c["geom"], c["pointing"]).cpu().numpy()
    assert_transpose_close(got, want, cw, c["geom"], "P^T small")
    # adjoint identity with FP64 dots of FP32 results
    x = c["cube"]
    Px = T.tomo_project(to_dev(x), c["geom"], c["pointing"], c["nu"],
                        c["nv"]).cpu().numpy().astype(np.float64)
    lhs = float(np.sum(Px * y))
    rhs = float(np.sum(x.astype(np.float64) * got))
    assert abs(lhs - rhs) <= RTOL_F32 * abs(lhs)


@pytest.mark.parametrize("seed", [3, 4])
def test_ragged_masked_gains_roll(T, seed):
    g, ptg, mask, cube = _ragged_scene(seed)
    md = mask_dev(mask)
    want = siddon.project(g, cube, ptg, 37, 53, mask)
    got = T.tomo_project(to_dev(cube), g, ptg, 37, 53, mask=md).cpu().numpy()
    assert_close(got, want, "P ragged")
    assert np.all(got[mask != 0] == 0.0)
    y = np.random.default_rng(seed + 10).random((5, 53, 37)).astype(np.float32)
    want_t = siddon.backproject(g, y, ptg, 37, 53, mask)
    cw = siddon.crossing_weights(g, y, ptg, 37, 53, mask)
    got_t = T.tomo_backproject(to_dev(y), g, ptg, mask=md).cpu().numpy()
    assert_transpose_close(got_t, want_t, cw, g, "P^T ragged")


def test_tilings_agree(T):
    """Every supported CTA / warp tiling gives the same projection (the walk
    of one ray does not depend on which thread runs it)."""
    g, ptg, mask, cube = _ragged_scene(5)
    ctx = T.Context()
    ref = None
    for (tu, tv, wu) in [(32, 8, 8), (16, 16, 4), (64, 4, 16), (32, 16, 32),
                         (8, 32, 2), (16, 8, 8)]:
        ctx.set_tiling(tu, tv, wu)
        y = T.tomo_project(to_dev(cube), g, ptg, 37, 53, ctx=ctx).cpu().numpy()
        if ref is None:
            ref = y
        np.testing.assert_array_equal(y, ref)
    ctx.close()


def test_observer_inside_cube_and_axis_rays(T):
    """Observer inside the cube (the half-line starts inside) and rays along
    or nearly along the axes (odd images centred on Sun centre at lon 0, 90).
    The cube has an odd side so the observer sits mid-voxel: with an observer
    on a voxel plane and a ray parallel to it to within FP64 rounding (at
    lon = 90 deg, cos(lon) = 6e-17), which neighbour gets the segment is
    decided by 1e-16 perturbations of the input, i.e. ill-conditioned."""
    g = synth.cube_geom(25, 1.5)
    ptg = synth.pointing_table([0.0, 90.0, 30.0], [0.0, 0.0, 10.0],
                               1.2, 31, 31, 2.0)
    rng = np.random.default_rng(8)
    cube = rng.random((25, 25, 25)).astype(np.float32)
    want = siddon.project(g, cube, ptg, 31, 31)
    got = T.tomo_project(to_dev(cube), g, ptg, 31, 31).cpu().numpy()
    assert_close(got, want, "P inside/axis")


def test_missing_rays_are_zero(T):
    """Pixels whose lines of sight miss the cube project to exactly 0, and
    an image that misses entirely leaves the transpose at 0."""
    g = synth.cube_geom(16, 0.5)
    ptg = synth.pointing_table([10.0], [0.0], 215.0, 40, 40, 8.0)
    ptg_off = ptg.copy()
    ptg_off[0, 8] = 0.2  # boresight 0.2 rad off Sun centre: misses
    cube = np.ones((16, 16, 16), np.float32)
    want = siddon.project(g, cube, ptg, 40, 40)
    got = T.tomo_project(to_dev(cube), g, ptg, 40, 40).cpu().numpy()
    assert_close(got, want, "P partly missing")
    assert np.all(got[want == 0] == 0.0)
    off = T.tomo_project(to_dev(cube), g, ptg_off, 40, 40).cpu().numpy()
    assert np.all(off == 0.0)
    x = T.tomo_backproject(torch.ones((1, 40, 40), device="cuda"), g, ptg_off)
    assert float(x.abs().max()) == 0.0


def test_time_interpolation(T):
    g, ptg, mask, frames = _ragged_scene(6, T_frames=4)
    md = mask_dev(mask)
    want = siddon.project(g, frames, ptg, 37, 53, mask, n_frames=4)
    got = T.tomo_project(to_dev(frames), g, ptg, 37, 53, mask=md,
                         n_frames=4).cpu().numpy()
    assert_close(got, want, "P time")
    y = np.random.default_rng(16).random((5, 53, 37)).astype(np.float32)
    want_t = siddon.backproject(g, y, ptg, 37, 53, mask, n_frames=4)
    cw = siddon.crossing_weights(g, y, ptg, 37, 53, mask, n_frames=4)
    got_t = T.tomo_backproject(to_dev(y), g, ptg, mask=md,
                               n_frames=4).cpu().numpy()
    assert_transpose_close(got_t, want_t, cw, g, "P^T time")


def test_bf16_cube(T):
    """BF16 storage: against the oracle on the rounded cube at the FP32
    tolerance, and against the FP32 cube at 1e-2."""
    c = synth.make_config("small")
    cube_bf = torch.from_numpy(c["cube"]).to(torch.bfloat16)
    rounded = cube_bf.to(torch.float32).numpy()
    got = T.tomo_project(cube_bf.cuda(), c["geom"], c["pointing"], c["nu"],
                         c["nv"]).cpu().numpy()
    want_r = siddon.project(c["geom"], rounded, c["pointing"], c["nu"], c["nv"])
    want_f = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"], c["nv"])
    assert_close(got, want_r, "P bf16 vs rounded cube")
    assert_close(got, want_f, "P bf16 vs f32 cube", rtol=1e-2, atol_frac=1e-4)


def test_segment_count(T):
    c = synth.make_config("single", scale=4)
    want = siddon.count_segments(c["geom"], c["pointing"], c["nu"], c["nv"],
                                 c["mask"])
    got = T.tomo_count_segments(c["geom"], c["pointing"], c["nu"], c["nv"],
                                mask=mask_dev(c["mask"]))
    assert abs(got - want) <= 1e-5 * want


def test_empty_image_stack(T):
    g = synth.cube_geom(8, 1.0)
    ptg = np.zeros((0, 12))
    out = T.tomo_project(torch.ones((8, 8, 8), device="cuda"), g, ptg, 4, 4)
    assert out.shape == (0, 4, 4)
    x = T.tomo_backproject(torch.zeros((0, 4, 4), device="cuda"), g, ptg)
    assert float(x.abs().max()) == 0.0


def test_single_config_full(T):
    """Config 'single' (128^3, 60 x 256^2, streamers, occulter mask): every
    pixel of P, and P^T on non-negative images, against the oracle."""
    c = synth.make_config("single")
    md = mask_dev(c["mask"])
    want = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"],
                          c["nv"], c["mask"])
    got = T.tomo_project(to_dev(c["cube"]), c["geom"], c["pointing"], c["nu"],
                         c["nv"], mask=md).cpu().numpy()
    assert_close(got, want, "P single")
    y = want.astype(np.float32)
    want_t = siddon.backproject(c["geom"], y, c["pointing"], c["nu"], c["nv"],
                                c["mask"])
    cw = siddon.crossing_weights(c["geom"], y, c["pointing"], c["nu"],
                                 c["nv"], c["mask"])
    got_t = T.tomo_backproject(to_dev(y), c["geom"], c["pointing"],
                               mask=md).cpu().numpy()
    assert_transpose_close(got_t, want_t, cw, c["geom"], "P^T single")


def _sampled_parity(T, c, frac, seed, dtype=torch.float32):
    md = mask_dev(c["mask"])
    n_frames = c["n_frames"]
    cube_t = to_dev(c["cube"]).to(dtype)
    got = T.tomo_project(cube_t, c["geom"], c["pointing"], c["nu"], c["nv"],
                         mask=md, n_frames=n_frames).cpu().numpy().reshape(-1)
    n_all = got.size
    rng = np.random.default_rng(seed)
    ids = np.sort(rng.choice(n_all, int(frac * n_all), replace=False))
    cube_o = c["cube"] if dtype == torch.float32 else cube_t.float().cpu().numpy()
    want = siddon.project(c["geom"], cube_o, c["pointing"], c["nu"], c["nv"],
                          c["mask"], n_frames=n_frames, ray_ids=ids)
    assert_close(got[ids], want, "P %s sampled" % c["name"])
    # transpose: dot test with images supported on the sampled pixels
    y = np.zeros(n_all, np.float32)
    y[ids] = rng.random(ids.size).astype(np.float32)
    Pty = T.tomo_backproject(to_dev(y.reshape(-1, c["nv"], c["nu"])),
                             c["geom"], c["pointing"], mask=md,
                             n_frames=n_frames)
    lhs = float(np.sum(want * y[ids].astype(np.float64)))
    rhs = float(torch.sum(cube_t.float().double() * Pty.double()).item())
    assert abs(lhs - rhs) <= RTOL_F32 * abs(lhs), (lhs, rhs)


def test_cg256_sampled(T):
    """The 256^3 CG timing workload (240 x 512^2): 0.1 % of the pixels
    against the oracle, and the transpose by a dot test on those pixels."""
    _sampled_parity(T, synth.make_config("cg256"), 1e-3, 256)


def test_temporal_sampled(T):
    """The time-interpolated workload (8 frames of 256^3, 240 x 512^2),
    float32 and bfloat16 storage, on 0.1 % of the pixels."""
    c = synth.make_config("temporal")
    _sampled_parity(T, c, 1e-3, 4)
    _sampled_parity(T, c, 1e-3, 5, dtype=torch.bfloat16)


@pytest.mark.parametrize("mode", [0, 5])
def test_transpose_kernels_agree_with_oracle(T, mode):
    """Both transpose walks (per ray with lane merging: TOMO_OPT_PLANE_SYNC
    0; plane-synchronous: the default 5) meet the transpose bound against
    the oracle on ragged, masked, gained geometry, an observer inside the
    cube, and the small config, and keep the adjoint identity with the
    forward projection."""
    ctx = T.Context()
    ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, mode)
    cases = []
    g, ptg, mask, cube = _ragged_scene(7)
    cases.append((g, ptg, mask, 37, 53))
    g2 = synth.cube_geom(25, 1.5)
    ptg2 = synth.pointing_table([0.0, 90.0, 30.0], [0.0, 0.0, 10.0], 1.2, 31,
                                31, 2.0)
    cases.append((g2, ptg2, None, 31, 31))
    c = synth.make_config("single", scale=2)
    cases.append((c["geom"], c["pointing"], c["mask"], c["nu"], c["nv"]))
    rng = np.random.default_rng(40 + mode)
    for g, ptg, mask, nu, nv in cases:
        y = rng.random((ptg.shape[0], nv, nu)).astype(np.float32)
        md = mask_dev(mask)
        got = T.tomo_backproject(to_dev(y), g, ptg, mask=md, ctx=ctx)
        want = siddon.backproject(g, y, ptg, nu, nv, mask)
        cw = siddon.crossing_weights(g, y, ptg, nu, nv, mask)
        assert_transpose_close(got.cpu().numpy(), want, cw, g,
                               "P^T mode %d" % mode)
        x = rng.random((g["nz"], g["ny"], g["nx"])).astype(np.float32)
        Px = T.tomo_project(to_dev(x), g, ptg, nu, nv, mask=md, ctx=ctx)
        lhs = float((Px.double() * to_dev(y).double()).sum())
        rhs = float((to_dev(x).double() * got.double()).sum())
        assert abs(lhs - rhs) <= RTOL_F32 * abs(lhs)
    ctx.close()
