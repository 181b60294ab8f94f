"""The per-ray forward over a device-built image list.

When the host's estimate lets every image of a geometry take the
plane-synchronous forward, the per-ray forward is launched in its listed
form: about one wave of CTAs deals out the tiles of the images whose device
hint rejects the plane forward (the host cannot know them without reading
the hints back).  Rules placed between the host estimate's margin and the
device's own pixel-pitch test make that list hold some or all images.  The
forward stays bit-identical to the per-ray walk of every image (both walk the
same Siddon segments in the same order, Section 3.3.1, Eq. lo) and matches
the FP64 oracle; masked pixels stay 0.  Images of 250 x 246 pixels give
ragged tiles and more tiles than one wave of CTAs, so CTAs take several."""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon
from tests.gpu_util import assert_close, mask_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu

NU, NV = 250, 246
NEVER = 1e30


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _case(d_far):
    """Eight ecliptic views of a 64^3 cube; every second observer at
    distance d_far (its pixels ~d_far/215 times further apart at the cube),
    the others at 215 R_sun.  A seeded mask drops ~10 % of the pixels."""
    g = synth.cube_geom(64, 1.5)
    lons = np.arange(8) * 22.5 + 3.0
    ptg = synth.pointing_table(lons, 0.0, 215.0, NU, NV, 3.2)
    ptg[1::2, 0] = d_far
    rng = np.random.default_rng(7)
    x = rng.random((64, 64, 64)).astype(np.float32)
    mask = (rng.random((8, NV, NU)) < 0.1).astype(np.uint8)
    # pixel pitch in voxels at Sun centre, as the walk rules measure it
    pitch = ptg[:, 0] * np.abs(np.tan(ptg[:, 4])) / g["dx"]
    return g, ptg, x, mask, pitch


@pytest.mark.parametrize("d_far", [245.0, 215.0],
                         ids=["some images listed", "every image listed"])
def test_listed_per_ray_forward(T, d_far):
    g, ptg, x, mask, pitch = _case(d_far)
    near = float(pitch[0])
    # device: plane forward iff pitch >= 1.05 near (the far images only);
    # host estimate: pitch >= 0.9 * 1.05 near holds for every image
    rules = {"min_pitch": 0.01, "fwd_min_pitch": 1.05 * near,
             "fwd_max_ratio": 0.0}
    ctx = T.Context()
    T.tomo_set_plane_rules(rules, g, NU, NV, n_img=ptg.shape[0], ctx=ctx)
    md = mask_dev(mask)
    got = T.tomo_project(to_dev(x), g, ptg, NU, NV, mask=md, ctx=ctx)
    codes = T.tomo_walk_plan(ptg.shape[0], ctx=ctx)
    plane_fwd = (codes & 2) != 0
    assert np.array_equal(plane_fwd, pitch >= 1.05 * near), codes
    if d_far > 215.0:
        assert plane_fwd[1::2].all() and not plane_fwd[0::2].any()
    else:
        assert not plane_fwd.any()
    ctx.close()

    ref_ctx = T.Context()
    T.tomo_set_plane_rules({"min_pitch": NEVER}, ctx=ref_ctx)
    ref = T.tomo_project(to_dev(x), g, ptg, NU, NV, mask=md, ctx=ref_ctx)
    assert np.all((T.tomo_walk_plan(ptg.shape[0], ctx=ref_ctx) & 3) == 0)
    ref_ctx.close()
    assert torch.equal(got, ref)

    y = got.cpu().numpy()
    assert np.all(y[mask != 0] == 0.0)
    want = siddon.project(g, x, ptg, NU, NV, mask)
    assert_close(y, want, "P listed per-ray forward d_far %g" % d_far)
