"""Two-value plane walks (TOMO_OPT_CHANNELS): time-interpolated P and P^T on
frame pairs stored side by side, and the Thomson B operator in one walk on
(m' x, m x) pairs.

The frame-pair forward forms the same products in the same order as the
separate-frame walks, so its images must be bit-identical to them (and to
the per-ray walk); the single-walk B forward adds the same two sums as the
two-walk form and combines them with the same fused multiply-add, so it is
bit-identical too.  The transposes differ only in the order of float
additions: they are held to the oracle's transpose bound and to the
two-walk / separate-frame results.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon, thomson
from tests.gpu_util import (assert_transpose_close, mask_dev, require_gpu,
                            to_dev)
from tests.test_gpu_plane import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _ctx(T, plane_sync, channels):
    ctx = T.Context()
    ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, plane_sync)
    ctx.set_option(T.tomo.TOMO_OPT_CHANNELS, channels)
    return ctx


def _with_times(ptg, n_frames, seed):
    rng = np.random.default_rng(seed)
    p = np.array(ptg, copy=True)
    p[:, 11] = rng.uniform(0, n_frames - 1, p.shape[0])
    p[0, 11] = n_frames - 1  # the last stamp: k = T - 2, w = 1
    if p.shape[0] > 1:
        p[1, 11] = 0.0
    return np.ascontiguousarray(p)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_frame_pairs(T, case):
    """Four frames: P on frame pairs equals P on separate frames and the
    per-ray P bit for bit (float32 and bf16 frames, plane walk on every
    image and on the images it is chosen for); P^T on frame pairs meets the
    oracle's bound."""
    name, g, ptg, mask, nu, nv = case
    n_frames = 4
    ptg = _with_times(ptg, n_frames, 91)
    rng = np.random.default_rng(92)
    frames = rng.random((n_frames, g["nz"], g["ny"], g["nx"])).astype(np.float32)
    md = mask_dev(mask)
    ray = _ctx(T, 0, 0)
    ctxs = {(ps, ch): _ctx(T, ps, ch) for ps in (3, 5) for ch in (0, 1)}
    for dt in (torch.float32, torch.bfloat16):
        X = to_dev(frames).to(dt)
        want = T.tomo_project(X, g, ptg, nu, nv, mask=md, n_frames=n_frames,
                              ctx=ray)
        for key, ctx in ctxs.items():
            got = T.tomo_project(X, g, ptg, nu, nv, mask=md,
                                 n_frames=n_frames, ctx=ctx)
            assert torch.equal(got, want), (name, dt, key)
    y = rng.random((ptg.shape[0], nv, nu)).astype(np.float32)
    want_t = siddon.backproject(g, y, ptg, nu, nv, mask, n_frames=n_frames)
    cw = siddon.crossing_weights(g, y, ptg, nu, nv, mask, n_frames=n_frames)
    sep = T.tomo_backproject(to_dev(y), g, ptg, mask=md, n_frames=n_frames,
                             ctx=ctxs[(5, 0)])
    got = T.tomo_backproject(to_dev(y), g, ptg, mask=md, n_frames=n_frames,
                             ctx=ctxs[(5, 1)])
    assert_transpose_close(got.cpu().numpy(), want_t, cw, g,
                           "P^T pairs %s" % name)
    torch.testing.assert_close(got, sep, rtol=1e-5,
                               atol=1e-6 * float(sep.abs().max()))
    # accumulate: adds onto what the cube holds
    acc = torch.ones_like(got)
    T.tomo_backproject(to_dev(y), g, ptg, mask=md, n_frames=n_frames,
                       out=acc, accumulate=True, ctx=ctxs[(5, 1)])
    torch.testing.assert_close(acc - 1.0, got, rtol=1e-5,
                               atol=1e-6 * float(got.abs().max()))
    for ctx in list(ctxs.values()) + [ray]:
        ctx.close()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_single_walk_b(T, case):
    """Thomson B: the single walk on (m' x, m x) pairs gives the two-walk
    images bit for bit (per-ray, plane on every image, the default choice;
    float32 and bf16 cubes); its transpose agrees with the two-walk
    transpose, with and without a map mask and when accumulating, and meets
    the oracle's bound."""
    name, g, ptg, mask, nu, nv = case
    g = dict(g)
    g["r_obs"] = 0.0
    u = 0.6
    rng = np.random.default_rng(93)
    x = rng.random((g["nz"], g["ny"], g["nx"])).astype(np.float32)
    y = rng.random((ptg.shape[0], nv, nu)).astype(np.float32)
    md = mask_dev(mask)
    mm = (rng.random((g["nz"], g["ny"], g["nx"])) < 0.1).astype(np.uint8)
    for ps in (0, 3, 5):
        one, two = _ctx(T, ps, 3), _ctx(T, ps, 1)
        for dt in (torch.float32, torch.bfloat16):
            X = to_dev(x).to(dt)
            for map_mask in (None, mask_dev(mm)):
                a = T.tomo_project(X, g, ptg, nu, nv, mask=md, kind="B",
                                   limb_u=u, map_mask=map_mask, ctx=one)
                b = T.tomo_project(X, g, ptg, nu, nv, mask=md, kind="B",
                                   limb_u=u, map_mask=map_mask, ctx=two)
                assert torch.equal(a, b), (name, ps, dt)
        b = T.tomo_backproject(to_dev(y), g, ptg, mask=md, kind="B",
                               limb_u=u, ctx=two)
        scale = float(b.abs().max())
        for map_mask in (None, mask_dev(mm)):
            a = T.tomo_backproject(to_dev(y), g, ptg, mask=md, kind="B",
                                   limb_u=u, map_mask=map_mask, ctx=one)
            w = T.tomo_backproject(to_dev(y), g, ptg, mask=md, kind="B",
                                   limb_u=u, map_mask=map_mask, ctx=two)
            torch.testing.assert_close(a, w, rtol=1e-5, atol=1e-6 * scale)
        # accumulate: adds onto what the cube holds
        acc = torch.ones_like(b)
        T.tomo_backproject(to_dev(y), g, ptg, mask=md, kind="B", limb_u=u,
                           out=acc, accumulate=True, ctx=one)
        torch.testing.assert_close(acc - 1.0, b, rtol=1e-5, atol=1e-6 * scale)
        one.close()
        two.close()
    # against the oracle (the transpose bound of the Thomson tests: the
    # terms of m' P^T y and m P^T rho^2 y each carry the plain bound)
    got = T.tomo_backproject(to_dev(y), g, ptg, mask=md, kind="B",
                             limb_u=u).cpu().numpy()
    want = thomson.backproject(thomson.B, g, y, ptg, nu, nv, u, mask)
    m, mp = thomson.voxel_factors(g, u)
    o = siddon.impact2(ptg, nu, nv)
    t_max = float(np.sqrt(sum((g["n" + a] * g["d" + a]) ** 2 for a in "xyz")))
    absw = (m * siddon.backproject(g, o * y, ptg, nu, nv, mask) +
            mp * siddon.backproject(g, y, ptg, nu, nv, mask))
    cw = (m * siddon.crossing_weights(g, o * y, ptg, nu, nv, mask) +
          mp * siddon.crossing_weights(g, y, ptg, nu, nv, mask))
    err = np.abs(got.astype(np.float64) - want)
    bound = (1e-5 * np.abs(want) + 64 * 2.0 ** -24 * absw +
             8 * 2.0 ** -24 * t_max * cw + 1e-30)
    assert np.all(err <= bound), (name, float((err / bound).max()))


def test_temporal_pairs_full_size_bit_identical(T):
    """The 8-frame 256^3 workload (240 x 512^2): P on frame pairs equals P
    on separate frames bit for bit, float32 and bf16."""
    c = synth.make_config("temporal")
    g, ptg, nu, nv = c["geom"], c["pointing"], c["nu"], c["nv"]
    a_ctx, b_ctx = _ctx(T, 5, 1), _ctx(T, 5, 0)
    for dt in (torch.float32, torch.bfloat16):
        X = to_dev(c["cube"]).to(dt)
        a = T.tomo_project(X, g, ptg, nu, nv, n_frames=8, ctx=a_ctx)
        b = T.tomo_project(X, g, ptg, nu, nv, n_frames=8, ctx=b_ctx)
        assert torch.equal(a, b), dt
        del X, a, b
    a_ctx.close()
    b_ctx.close()
