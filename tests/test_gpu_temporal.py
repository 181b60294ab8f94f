"""Several frames in the solver: the smooth temporal model (Section 3.3.3;
block-diagonal for integer time stamps, Eq. srt_t / stsrt) with a temporal
prior lambda_t ||D_t x||^2 between consecutive frames, against FP64 CG on
the same criterion.
"""

import numpy as np
import pytest

import synth
from oracle import siddon, solver
from tests.gpu_util import mask_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _scene(times, seed=3):
    g = synth.cube_geom(24, 1.6, ny=22, nz=20)
    rng = np.random.default_rng(seed)
    n = len(times)
    ptg = synth.pointing_table(rng.uniform(0, 360, n), rng.uniform(-10, 10, n),
                               215.0, 40, 36, 3.4, time=np.asarray(times))
    mask = (rng.random((n, 36, 40)) < 0.05).astype(np.uint8)
    x = rng.random((3, 20, 22, 24))
    y = siddon.project(g, x, ptg, 40, 36, mask, 3).astype(np.float32)
    return g, ptg, mask, y


def test_temporal_prior_against_fp64_cg(T):
    """Three frames, fractional stamps, spatial and temporal priors: 10 CG
    iterations against FP64 CG."""
    times = np.random.default_rng(1).uniform(0, 2, 9)
    g, ptg, mask, y = _scene(times)
    pb = solver.Problem(g, ptg, 40, 36, y, mask, lam=0.05, n_frames=3,
                        lam_t=0.5)
    x_o, rep_o = solver.cg(pb, 10)
    x_g, info = T.tomo_solve(to_dev(y), g, ptg, mask=mask_dev(mask), lam=0.05,
                             lam_t=0.5, n_frames=3, max_iter=10)
    assert tuple(x_g.shape) == (3, 20, 22, 24)
    rel = np.linalg.norm(x_g.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=1e-3)


def test_integer_stamps_block_diagonal(T):
    """Integer stamps and lambda_t = 0 (the block-diagonal model: each frame
    is seen only by its own images): 8 CG iterations against FP64 CG."""
    times = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2], dtype=np.float64)
    g, ptg, mask, y = _scene(times, seed=4)
    pb = solver.Problem(g, ptg, 40, 36, y, mask, lam=0.05, n_frames=3)
    x_o, rep_o = solver.cg(pb, 8)
    x_g, info = T.tomo_solve(to_dev(y), g, ptg, mask=mask_dev(mask), lam=0.05,
                             n_frames=3, max_iter=8)
    rel = np.linalg.norm(x_g.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=1e-3)


def test_map_mask_on_every_frame(T):
    """A map mask restricts every frame: 8 CG iterations with a temporal
    prior against FP64 CG on the restricted system; excluded voxels are 0
    in every frame, also from a warm start that is not 0 there."""
    times = np.random.default_rng(7).uniform(0, 2, 9)
    g, ptg, mask, y = _scene(times, seed=5)
    mm = synth.shell_map_mask(g, 0.6, 1.5)
    pb = solver.Problem(g, ptg, 40, 36, y, mask, lam=0.05, n_frames=3,
                        lam_t=0.3, map_mask=mm)
    x0 = np.random.default_rng(8).random((3, 20, 22, 24)).astype(np.float32)
    x_o, rep_o = solver.cg(pb, 8, x0=x0)
    x_g, info = T.tomo_solve(to_dev(y), g, ptg, mask=mask_dev(mask), lam=0.05,
                             lam_t=0.3, n_frames=3, max_iter=8,
                             map_mask=mask_dev(mm), x0=to_dev(x0))
    xg = x_g.cpu().numpy()
    assert np.all(xg[:, mm != 0] == 0.0)
    rel = np.linalg.norm(xg - x_o) / np.linalg.norm(x_o)
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=1e-3)
