"""CTA order of the plane walks (TOMO_OPT_GROUP_FWD / TOMO_OPT_GROUP_ADJ).
Images are taken in groups, and inside a group the CTAs of one pixel-row
band of every image run before the next band.  The order changes no segment
(Section 3.3.1: the walk of each ray is the same): P is bit-identical for
every group size, including group sizes that do not divide the image count
(the last group then has padding images) and a group of every image.  P^T
differs only by the order of float additions, and meets the oracle's
transpose bound.  The single-value walks, the frame-pair walks and the
Thomson B pair walks are covered."""

import numpy as np
import pytest
import torch

from oracle import siddon
from tests.gpu_util import (assert_transpose_close, mask_dev, require_gpu,
                            to_dev)
from tests.test_gpu_plane import CASES

pytestmark = pytest.mark.gpu

GROUPS = (1, 2, 3, 1000)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _ctx(T, group):
    ctx = T.Context()
    ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, 3)  # plane P and P^T
    ctx.set_option(T.tomo.TOMO_OPT_GROUP_FWD, group)
    ctx.set_option(T.tomo.TOMO_OPT_GROUP_ADJ, group)
    return ctx


def _times(ptg, n_frames, seed):
    rng = np.random.default_rng(seed)
    p = np.array(ptg, copy=True)
    p[:, 11] = rng.uniform(0, n_frames - 1, p.shape[0])
    return np.ascontiguousarray(p)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_group_order_changes_no_result(T, case):
    name, g, ptg, mask, nu, nv = case
    rng = np.random.default_rng(31)
    x = rng.random((g["nz"], g["ny"], g["nx"])).astype(np.float32)
    y = rng.random((ptg.shape[0], nv, nu)).astype(np.float32)
    md = mask_dev(mask)
    want_t = siddon.backproject(g, y, ptg, nu, nv, mask)
    cw = siddon.crossing_weights(g, y, ptg, nu, nv, mask)
    ref = None
    for grp in GROUPS:
        ctx = _ctx(T, grp)
        P = T.tomo_project(to_dev(x), g, ptg, nu, nv, mask=md, ctx=ctx)
        Pt = T.tomo_backproject(to_dev(y), g, ptg, mask=md, ctx=ctx)
        if ref is None:
            ref = (P, Pt)
        assert torch.equal(P, ref[0]), (name, grp)
        torch.testing.assert_close(Pt, ref[1], rtol=1e-5,
                                   atol=1e-6 * float(ref[1].abs().max()))
        assert_transpose_close(Pt.cpu().numpy(), want_t, cw, g,
                               "P^T group %d %s" % (grp, name))
        ctx.close()


def test_group_order_frame_pairs_and_b(T):
    """Four frames on frame pairs, and the Thomson B operator on (m' x, m x)
    pairs: P bit-identical and P^T within float reordering across group
    sizes."""
    name, g, ptg, mask, nu, nv = CASES[0]
    n_frames = 4
    ptg_t = _times(ptg, n_frames, 41)
    rng = np.random.default_rng(42)
    frames = rng.random((n_frames, g["nz"], g["ny"], g["nx"])).astype(np.float32)
    x = frames[0]
    y = rng.random((ptg.shape[0], nv, nu)).astype(np.float32)
    gb = dict(g, r_obs=0.0)
    ref = None
    for grp in GROUPS:
        ctx = _ctx(T, grp)
        ctx.set_option(T.tomo.TOMO_OPT_CHANNELS, 3)
        out = (T.tomo_project(to_dev(frames), g, ptg_t, nu, nv,
                              n_frames=n_frames, ctx=ctx),
               T.tomo_backproject(to_dev(y), g, ptg_t, n_frames=n_frames,
                                  ctx=ctx),
               T.tomo_project(to_dev(x), gb, ptg, nu, nv, kind="B",
                              limb_u=0.6, ctx=ctx),
               T.tomo_backproject(to_dev(y), gb, ptg, kind="B", limb_u=0.6,
                                  ctx=ctx))
        if ref is None:
            ref = out
        assert torch.equal(out[0], ref[0]), grp
        assert torch.equal(out[2], ref[2]), grp
        for k in (1, 3):
            torch.testing.assert_close(out[k], ref[k], rtol=1e-5,
                                       atol=1e-6 * float(ref[k].abs().max()))
        ctx.close()
