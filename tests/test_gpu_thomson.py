"""Thomson-scattering operators for white-light images (Section 3.5):
T_pB = O P M and T_B = P M' - O P M, with O = diag(rho^2) per pixel and
M, M' the per-voxel factors of Eq. brightness (readings in ``oracle/thomson``:
sin Omega = 1/r, +1/8 on C4, the factor 2 and the u on C2 of Eq.
brightness, no scattering inside the photosphere).

The GPU path runs the plain walks between FP64-computed diagonal factors;
these cases compare T and T^T with the FP64 oracle (its own coefficients
and impact parameters), the map mask and frames with them, and CG on pB
and B data with FP64 CG.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon, solver, thomson
from tests.gpu_util import (assert_close, mask_dev, require_gpu, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _scene(seed=0, n_frames=1):
    """A corona-sized cube (the Sun inside it), five views with rolls,
    gains and time stamps, a pixel mask."""
    rng = np.random.default_rng(seed)
    g = {"nx": 29, "ny": 31, "nz": 27, "x0": -3.0, "y0": -3.1, "z0": -2.8,
         "dx": 6.0 / 29, "dy": 6.2 / 31, "dz": 5.6 / 27}
    ptg = synth.pointing_table([0.0, 90.0, 33.0, 150.0, 260.0],
                               [0.0, 3.0, -8.0, 25.0, 0.5], 215.0, 37, 41, 6.5,
                               gain=rng.uniform(0.5, 2.0, 5),
                               time=rng.uniform(0, max(n_frames - 1, 0), 5))
    ptg[2:, 3] = rng.uniform(-np.pi, np.pi, 3)
    mask = (rng.random((5, 41, 37)) < 0.05).astype(np.uint8)
    return g, ptg, mask, rng


def _transpose_bound(got, want, absw, cw, geom):
    """Float32 bound of the transpose: 1e-5 relative, 64 ulp of the sum of
    absolute terms (``absw``), and, as for the plain transpose, 8 ulp of the
    longest chord per crossing ray (``cw``: the crossing weights of the
    weighted images times the voxel factor), since a segment's length is a
    difference of float crossing parameters and carries an absolute error."""
    t_max = float(np.sqrt(sum((geom["n" + a] * geom["d" + a]) ** 2
                              for a in "xyz")))
    err = np.abs(np.asarray(got, np.float64) - want)
    bound = (1e-5 * np.abs(want) + 64 * 2.0 ** -24 * absw +
             8 * 2.0 ** -24 * t_max * cw + 1e-30)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("kind", ["pB", "B"])
@pytest.mark.parametrize("n_frames", [1, 3])
def test_operators_against_oracle(T, kind, n_frames):
    g, ptg, mask, rng = _scene(1, n_frames)
    u = 0.56
    k = thomson.PB if kind == "pB" else thomson.B
    shape = ((n_frames,) if n_frames > 1 else ()) + (27, 31, 29)
    x = rng.random(shape).astype(np.float32)
    y = rng.random((5, 41, 37)).astype(np.float32)
    mm = (rng.random((27, 31, 29)) < 0.1).astype(np.uint8)
    md = mask_dev(mask)
    for map_mask in (None, mm):
        want = thomson.project(k, g, x, ptg, 37, 41, u, mask, n_frames,
                               map_mask=map_mask)
        for mode in (0, 5):
            ctx = T.Context()
            ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, mode)
            got = T.tomo_project(to_dev(x), g, ptg, 37, 41, mask=md,
                                 n_frames=n_frames, kind=kind, limb_u=u,
                                 map_mask=mask_dev(map_mask), ctx=ctx)
            # pB: products of positive terms; B: a difference of two such
            # sums, bounded by the scale of its parts (1e-5 of the maximum)
            assert_close(got.cpu().numpy(), want, "T %s mode %d" % (kind, mode),
                         rtol=2e-5, atol_frac=1e-7 if kind == "pB" else 1e-5)
            got_t = T.tomo_backproject(to_dev(y), g, ptg, mask=md,
                                       n_frames=n_frames, kind=kind, limb_u=u,
                                       map_mask=mask_dev(map_mask), ctx=ctx)
            want_t = thomson.backproject(k, g, y, ptg, 37, 41, u, mask,
                                         n_frames, map_mask=map_mask)
            m, mp = thomson.voxel_factors(g, u)
            o = siddon.impact2(ptg, 37, 41)
            absw = m * siddon.backproject(g, o * y, ptg, 37, 41, mask, n_frames)
            cw = m * siddon.crossing_weights(g, o * y, ptg, 37, 41, mask,
                                             n_frames)
            if k == thomson.B:
                absw = absw + mp * siddon.backproject(g, y, ptg, 37, 41, mask,
                                                      n_frames)
                cw = cw + mp * siddon.crossing_weights(g, y, ptg, 37, 41, mask,
                                                       n_frames)
            _transpose_bound(got_t.cpu().numpy(), want_t, absw, cw, g)
            ctx.close()


@pytest.mark.parametrize("kind", ["pB", "B"])
def test_solve_against_fp64_cg(T, kind):
    """10 CG iterations on white-light data with a height-weighted prior
    against FP64 CG on the same criterion."""
    g, ptg, mask, rng = _scene(2)
    k = thomson.PB if kind == "pB" else thomson.B
    u = 0.6
    x_true = np.asarray(synth.corona_cube(g), np.float32)
    y = thomson.project(k, g, x_true, ptg, 37, 41, u, mask).astype(np.float32)
    w = synth.height_weights(g, 1.0, 0.05).astype(np.float32)
    lam = 1e-3 * float(np.abs(y).max()) ** 2 / float(np.abs(x_true).max()) ** 2
    pb = solver.Problem(g, ptg, 37, 41, y, mask, lam=lam, prior_weight=w,
                        kind=k, limb_u=u)
    x_o, rep_o = solver.cg(pb, 10)
    x_g, info = T.tomo_solve(to_dev(y), g, ptg, mask=mask_dev(mask), lam=lam,
                             max_iter=10, prior_weight=to_dev(w), kind=kind,
                             limb_u=u)
    rel = np.linalg.norm(x_g.cpu().numpy() - x_o) / np.linalg.norm(x_o)
    assert rel <= 1e-3, rel
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=1e-3)


def test_rejected_kinds(T):
    g, ptg, mask, rng = _scene(3)
    X = torch.ones((27, 31, 29), device="cuda")
    with pytest.raises(ValueError):
        T.tomo_project(X, g, ptg, 37, 41, kind="polarised")
    with pytest.raises(T.TomoError):
        T.tomo_project(X, g, ptg, 37, 41, kind="pB", limb_u=1.5)
    with pytest.raises(T.TomoError):
        T.tomo_project_batched([{"geom": g, "pointing": ptg, "nu": 37,
                                 "nv": 41, "cube": X, "kind": "pB",
                                 "images": torch.zeros((5, 41, 37),
                                                       device="cuda")}])


def test_autograd_pb(T):
    """The gradient of <w, T_pB x> through the autograd Function is
    T_pB^T w."""
    from paper_1103_5904_gb300 import autograd
    g, ptg, mask, rng = _scene(4)
    u = 0.5
    X = to_dev(rng.random((27, 31, 29)).astype(np.float32)).requires_grad_(True)
    w = rng.random((5, 41, 37)).astype(np.float32)
    y = autograd.project(X, g, ptg, 37, 41, mask=mask_dev(mask), kind="pB",
                         limb_u=u)
    assert torch.equal(y.detach(), T.tomo_project(X.detach(), g, ptg, 37, 41,
                                                  mask=mask_dev(mask),
                                                  kind="pB", limb_u=u))
    (y * to_dev(w)).sum().backward()
    want = thomson.backproject(thomson.PB, g, w, ptg, 37, 41, u, mask)
    m, _ = thomson.voxel_factors(g, u)
    o = siddon.impact2(ptg, 37, 41)
    _transpose_bound(X.grad.cpu().numpy(), want,
                     m * siddon.backproject(g, o * w, ptg, 37, 41, mask),
                     m * siddon.crossing_weights(g, o * w, ptg, 37, 41, mask), g)
