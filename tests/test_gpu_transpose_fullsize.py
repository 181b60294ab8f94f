"""The transpose P^T at full cube size against the FP64 oracle, voxel by voxel.

The full workloads have too many pixels for the oracle to backproject them
all in a test, so each case keeps every voxel of the full cube (the index
ranges, the layout copies and the accumulators of the full size) and a
seeded subset of the full-size images; every voxel of the result is held to
the transpose bound of ``tests/gpu_util.py`` (Section 3.3.1, Eq. lo read as
P^T: voxel j receives sum_k g_k y_k P_{k,j}).  Images are seeded uniform
values in [0, 1), the non-negative case the bound is derived for.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon
from tests.gpu_util import (assert_transpose_close, mask_dev, require_gpu,
                            to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _subset(c, n_keep, seed):
    rng = np.random.default_rng(seed)
    keep = np.sort(rng.choice(c["pointing"].shape[0], n_keep, replace=False))
    ptg = np.ascontiguousarray(c["pointing"][keep])
    mask = (None if c["mask"] is None
            else np.ascontiguousarray(c["mask"][keep]))
    y = rng.random((n_keep, c["nv"], c["nu"])).astype(np.float32)
    return ptg, mask, y


def _check(T, c, ptg, mask, y, what):
    g, n_frames = c["geom"], c["n_frames"]
    got = T.tomo_backproject(to_dev(y), g, ptg, mask=mask_dev(mask),
                             n_frames=n_frames).cpu().numpy()
    want = siddon.backproject(g, y, ptg, c["nu"], c["nv"], mask,
                              n_frames=n_frames)
    cw = siddon.crossing_weights(g, y, ptg, c["nu"], c["nv"], mask,
                                 n_frames=n_frames)
    assert got.shape == want.shape
    assert float(np.abs(want).max()) > 0.0
    assert_transpose_close(got, want, cw, g, what)


def test_cg256_transpose_every_voxel(T):
    """256^3 cube, 24 of the 240 images of 512^2 (occulter mask)."""
    c = synth.make_config("cg256")
    ptg, mask, y = _subset(c, 24, 2561)
    _check(T, c, ptg, mask, y, "P^T cg256 (24 images)")


def test_temporal_transpose_every_voxel(T):
    """8 frames of 256^3 (each image on its two frames), 16 of the 240
    images of 512^2 with their time stamps."""
    c = synth.make_config("temporal")
    ptg, mask, y = _subset(c, 16, 2562)
    _check(T, c, ptg, mask, y, "P^T temporal (16 images)")


def test_coronagraph_transpose_every_voxel(T):
    """512^3 cube over [-4, 4]^3, 4 of the 360 images of 1024^2 (occulter
    and field-edge mask)."""
    c = synth.make_config("coronagraph")
    ptg, mask, y = _subset(c, 4, 5121)
    _check(T, c, ptg, mask, y, "P^T coronagraph (4 images)")


def test_rolled_and_polar_views_on_256_cube(T):
    """The 256^3 cube seen with image rows along z (roll 90 degrees: the
    z-fastest accumulator), from high latitude (major axis z) and from an
    oblique direction, 512^2 images, every voxel."""
    c = dict(synth.make_config("cg256"))
    lon = np.array([20.0, 110.0, 45.0, 200.0, 300.0])
    lat = np.array([0.0, 3.0, 80.0, -75.0, 30.0])
    roll = np.array([90.0, -90.0, 0.0, 35.0, 10.0])
    ptg = synth.pointing_table(lon, lat, 215.0, 512, 512, 3.2, roll_deg=roll)
    rng = np.random.default_rng(2563)
    y = rng.random((lon.size, 512, 512)).astype(np.float32)
    _check(T, c, ptg, None, y, "P^T rolled/polar 256^3")
