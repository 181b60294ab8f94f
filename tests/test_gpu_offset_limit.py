"""The plane walks address one buffer with 32-bit byte offsets, so they take
cubes of at most 2^32 bytes.  A float32 cube of 1024^3 voxels is exactly that
bound: the plane walks run on it, with offsets up to 2^32 - 4, in all three
layouts.  One voxel plane more and the walk plan must report per-ray walks.
Both cubes are checked against the FP64 oracle: every pixel of P; every
voxel of P^T at the bound, and the transpose identity <P^T y, x> = <y, P x>
above it (Section 3.3.1, Eq. lo and its transpose)."""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon
from tests.gpu_util import (assert_close, assert_transpose_close, require_gpu,
                            to_dev)

pytestmark = pytest.mark.gpu

NU = NV = 96


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _views():
    """Four views through the whole cube, pixels ~11 voxels apart: along x
    (layout 1), along y (layout 0), a rolled view whose rows run along z
    (layout 2), and one from latitude 60 degrees."""
    ptg = synth.pointing_table([30.0, 100.0, 20.0, 200.0],
                               [0.0, 0.0, 0.0, 60.0], 215.0, NU, NV, 3.2)
    ptg[2, 3] = np.pi / 2
    return ptg


def _cube(nz, ny, nx):
    """A structured float32 cube (no two neighbouring voxels equal), built
    one plane at a time."""
    i = np.arange(nx, dtype=np.float32)
    j = np.arange(ny, dtype=np.float32)[:, None]
    base = (np.mod(i, 7.0) * 0.1 + np.mod(j, 5.0) * 0.05 + 0.2).astype(np.float32)
    x = np.empty((nz, ny, nx), dtype=np.float32)
    for k in range(nz):
        x[k] = base + np.float32((k % 13) * 0.01)
    return x


@pytest.mark.parametrize("nz", [1024, 1025], ids=["2^32 bytes", "above"])
def test_cube_at_and_above_the_offset_bound(T, nz):
    g = synth.cube_geom(1024, 1.5, ny=1024, nz=nz)
    ptg = _views()
    x = _cube(nz, 1024, 1024)
    ctx = T.Context()
    y = T.tomo_project(to_dev(x), g, ptg, NU, NV, ctx=ctx)
    codes = T.tomo_walk_plan(ptg.shape[0], ctx=ctx)
    if nz == 1024:
        # plane P and P^T on every view; lateral axes y, x, z, and x or y
        assert np.all((codes & 3) == 3), codes
        assert sorted({int(c >> 5) & 3 for c in codes[:3]}) == [0, 1, 2]
    else:
        assert np.all((codes & 3) == 0), codes
    want = siddon.project(g, x, ptg, NU, NV)
    assert_close(y.cpu().numpy(), want, "P 1024^2 x %d" % nz)
    rng = np.random.default_rng(nz)
    img = rng.random((ptg.shape[0], NV, NU)).astype(np.float32)
    got = T.tomo_backproject(to_dev(img), g, ptg, ctx=ctx).cpu().numpy()
    ctx.close()
    torch.cuda.empty_cache()
    if nz == 1024:
        # every voxel (the plane transposes, up to the largest offset)
        want_t = siddon.backproject(g, img, ptg, NU, NV)
        cw = siddon.crossing_weights(g, img, ptg, NU, NV)
        assert_transpose_close(got, want_t, cw, g, "P^T 1024^2 x 1024")
    else:
        # the per-ray transpose: <P^T y, x> = <y, P x> against the oracle
        lhs = float(np.dot(got.ravel().astype(np.float64),
                           x.ravel().astype(np.float64)))
        rhs = float(np.dot(img.ravel().astype(np.float64), want.ravel()))
        assert lhs == pytest.approx(rhs, rel=1e-5)
