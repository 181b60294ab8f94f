"""GPU regulariser D^T D and CG solver against the FP64 oracle.

Tolerances (derived from the arithmetic; see the project design notes):
  prior:  |q - q*| <= 1e-5 |q*| + 1e-6 lambda max|x|
          (six FP32 differences per voxel, each rounded once)
  CG:     ||x - x*|| <= 1e-3 ||x*|| and |J_k - J_k*| <= 1e-3 J_k*
          An FP32-vector CG emulated on the CPU (every vector operation
          rounded to float32 around the FP64 oracle projector) stays within
          2e-5 of FP64 CG after 20 iterations on the 'single' workload; the
          device projector adds ~1e-6 per-pixel rounding on top, and the
          device J = y^T M y - x^T (r + b) loses ~1e-7 y^T M y / J to
          cancellation (about 2.5e-4 once J reaches the noise floor at
          SNR 50).
"""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon, solver
from tests.gpu_util import assert_close, mask_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu

CG_X_RTOL = 1e-3
CG_J_RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _data(c):
    """Noisy data from the oracle projector (FP64), rounded to float32."""
    y = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"], c["nv"],
                       c["mask"])
    if c.get("snr"):
        y = synth.add_noise(y, synth.noise_draw(c["noise_seed"], y.shape),
                            c["mask"], c["snr"])
    return y.astype(np.float32)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b)
                 / np.linalg.norm(b))


def test_prior_matches_oracle(T):
    rng = np.random.default_rng(1)
    g = {"nx": 37, "ny": 21, "nz": 13, "x0": 0, "y0": 0, "z0": 0,
         "dx": 1, "dy": 1, "dz": 1}
    x = rng.standard_normal((13, 21, 37)).astype(np.float32)
    lam = 0.37
    want = lam * solver.DtD(x)
    got = T.tomo_prior_apply(to_dev(x), g, lam).cpu().numpy()
    assert_close(got, want, "lambda D^T D x", atol_frac=1e-6 * np.abs(x).max()
                 * lam / np.abs(want).max())
    acc = T.tomo_prior_apply(to_dev(x), g, lam, out=to_dev(x.copy()),
                             accumulate=True).cpu().numpy()
    assert_close(acc, x + want, "accumulate", atol_frac=1e-6)


def test_cg_small(T):
    """Config 'small' with lambda 1e-2, 20 iterations: iterate and criterion
    per iteration against textbook FP64 CG."""
    c = synth.make_config("small")
    y = _data(c)
    pb = solver.Problem(c["geom"], c["pointing"], c["nu"], c["nv"], y,
                        None, lam=1e-2)
    x_o, rep_o = solver.cg(pb, 20)
    x_g, info = T.tomo_solve(to_dev(y), c["geom"], c["pointing"], lam=1e-2,
                             max_iter=20)
    assert info["iters"] == 20
    assert _rel(x_g.cpu().numpy(), x_o) <= CG_X_RTOL
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=CG_J_RTOL)
    assert np.all(np.diff(info["J"]) <= 1e-6 * info["J"][0])


def test_cg_single_config(T):
    """Config 'single' (128^3, 60 x 256^2, occulter mask, SNR 50, lambda
    1e-2, 20 iterations) against a full 20-iteration FP64 CG."""
    c = synth.make_config("single")
    y = _data(c)
    pb = solver.Problem(c["geom"], c["pointing"], c["nu"], c["nv"], y,
                        c["mask"], lam=c["lam"])
    x_o, rep_o = solver.cg(pb, c["n_iter"], track_J=False)
    x_g, info = T.tomo_solve(to_dev(y), c["geom"], c["pointing"],
                             mask=mask_dev(c["mask"]), lam=c["lam"],
                             max_iter=c["n_iter"])
    assert info["iters"] == c["n_iter"]
    assert _rel(x_g.cpu().numpy(), x_o) <= CG_X_RTOL
    # criterion at the last iterate, evaluated directly by the oracle
    assert info["J"][-1] == pytest.approx(pb.J(x_o), rel=CG_J_RTOL)
    np.testing.assert_allclose(info["rr"][:11], rep_o["rr"][:11], rtol=1e-3)
    assert info["J"][0] == pytest.approx(pb.J(np.zeros(pb.shape)), rel=1e-6)


def test_cg_warm_start_and_tolerance(T):
    c = synth.make_config("small", scale=2)
    y = _data(c)
    pb = solver.Problem(c["geom"], c["pointing"], c["nu"], c["nv"], y, None,
                        lam=1e-2)
    x5, _ = solver.cg(pb, 5)
    x_more, rep_more = solver.cg(pb, 7, x0=x5)
    x_g5, _ = T.tomo_solve(to_dev(y), c["geom"], c["pointing"], lam=1e-2,
                           max_iter=5)
    x_g, info = T.tomo_solve(to_dev(y), c["geom"], c["pointing"], lam=1e-2,
                             max_iter=7, x0=x_g5)
    assert _rel(x_g.cpu().numpy(), x_more) <= CG_X_RTOL
    np.testing.assert_allclose(info["J"], rep_more["J"], rtol=CG_J_RTOL)
    # early stop on the relative residual
    x_t, info_t = T.tomo_solve(to_dev(y), c["geom"], c["pointing"], lam=1e-2,
                               max_iter=50, tol=0.05)
    k = info_t["iters"]
    assert 0 < k < 50
    assert info_t["rr"][k] <= 0.05 ** 2 * info_t["rr"][0]
    assert info_t["rr"][k - 1] > 0.05 ** 2 * info_t["rr"][0]
    assert np.all(np.isnan(info_t["J"][k + 1:]))


def test_cg_all_masked_is_zero(T):
    """Every pixel masked: b = 0, the solver stops at once with x = 0."""
    c = synth.make_config("small", scale=4)
    y = _data(c)
    mask = np.ones((8, c["nv"], c["nu"]), np.uint8)
    x, info = T.tomo_solve(to_dev(y), c["geom"], c["pointing"],
                           mask=mask_dev(mask), lam=1e-2, max_iter=5)
    assert info["iters"] == 0
    assert float(x.abs().max()) == 0.0


def test_cg_bf16_direction_reaches_same_residual(T):
    """BF16 storage of the CG direction (the projector gathers bf16, every
    accumulation is FP32), compared with FP32 storage at equal final
    criterion: the bf16 solve reaches the criterion of 20 FP32 iterations
    within 30 iterations, and its criterion decreases at every iteration
    (each step is an exact line search along the bf16-rounded direction)."""
    c = synth.make_config("single", scale=2)
    y = _data(c)
    md = mask_dev(c["mask"])
    _, i32 = T.tomo_solve(to_dev(y), c["geom"], c["pointing"], mask=md,
                          lam=1e-2, max_iter=60)
    _, i16 = T.tomo_solve(to_dev(y), c["geom"], c["pointing"], mask=md,
                          lam=1e-2, max_iter=60, bf16=True)
    target = i32["J"][20] * (1 + 1e-4)
    k16 = int(np.argmax(i16["J"] <= target))
    assert i16["J"][k16] <= target and k16 <= 30, k16
    assert np.all(np.diff(i16["J"]) <= 1e-6 * i16["J"][0])
    assert i16["J"][-1] < i32["J"][30]


def test_cg_with_per_ray_walks(T):
    """The solver on the per-ray walks (TOMO_OPT_PLANE_SYNC 0) matches FP64
    CG like the default plane-synchronous ones."""
    c = synth.make_config("single", scale=2)
    y = _data(c)
    pb = solver.Problem(c["geom"], c["pointing"], c["nu"], c["nv"], y,
                        c["mask"], lam=c["lam"])
    x_o, rep_o = solver.cg(pb, 10)
    ctx = T.Context()
    ctx.set_option(T.tomo.TOMO_OPT_PLANE_SYNC, 0)
    x_g, info = T.tomo_solve(to_dev(y), c["geom"], c["pointing"],
                             mask=mask_dev(c["mask"]), lam=c["lam"],
                             max_iter=10, ctx=ctx)
    assert _rel(x_g.cpu().numpy(), x_o) <= CG_X_RTOL
    np.testing.assert_allclose(info["J"], rep_o["J"], rtol=CG_J_RTOL)
    ctx.close()
