"""The projector as a torch.autograd.Function (forward = P, backward = the
transpose kernel), on the smoothly time-varying model where every image sees
the linear interpolation of its two neighbouring frames.

Finite differences: for f(x) = 0.5 ||P x - y||^2 the central difference
(f(x + h e_j) - f(x - h e_j)) / 2h equals the gradient exactly up to
rounding (f is quadratic).  The projections of x + h e_j and x - h e_j agree
bit for bit on every pixel whose ray misses voxel j, so only the few
thousand pixels that see voxel j carry FP32 rounding (~1e-7 of their value
against a difference of 2 h times a segment length); summed in FP64 this
bounds the relative FD error near 1e-4, and the tests allow 1e-3.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import siddon
from tests.gpu_util import require_gpu, to_dev, RTOL_F32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _loss(T, X, c, y):
    P = T.autograd.project(X, c["geom"], c["pointing"], c["nu"], c["nv"],
                           n_frames=c["n_frames"])
    r = P.double() - y.double()
    return 0.5 * (r * r).sum()


def _fd_check(T, c, X, y, n_vox, seed, h=1e-3, rtol=1e-3):
    X = X.clone().requires_grad_(True)
    loss = _loss(T, X, c, y)
    loss.backward()
    grad = X.grad.detach().reshape(-1)
    rng = np.random.default_rng(seed)
    flat = X.detach().reshape(-1)
    scale = float(grad.abs().max())
    for j in rng.choice(flat.numel(), n_vox, replace=False):
        xp = flat.clone()
        xm = flat.clone()
        xp[j] += h
        xm[j] -= h
        with torch.no_grad():
            fp = _loss(T, xp.reshape(X.shape), c, y)
            fm = _loss(T, xm.reshape(X.shape), c, y)
        fd = float((fp - fm) / (2 * h))
        g = float(grad[j])
        assert abs(fd - g) <= rtol * abs(g) + 1e-4 * scale, (int(j), fd, g)
    return grad


def test_forward_and_backward_match_kernels_and_oracle(T):
    """Reduced time-varying workload (8 frames of 64^3, 240 images 128^2):
    forward equals tomo_project, the gradient matches the FP64 oracle's
    transpose of the oracle residual, and 64 central differences."""
    c = synth.make_config("temporal", scale=4)
    X = to_dev(c["cube"])
    rng = np.random.default_rng(3)
    y_np = rng.random((240, c["nv"], c["nu"])).astype(np.float32)
    y = to_dev(y_np)
    out = T.autograd.project(X, c["geom"], c["pointing"], c["nu"], c["nv"],
                             n_frames=8)
    ref = T.tomo_project(X, c["geom"], c["pointing"], c["nu"], c["nv"],
                         n_frames=8)
    assert torch.equal(out, ref)
    grad = _fd_check(T, c, X, y, 64, seed=11)
    # FP64 oracle: residual and transpose of the same loss
    r_o = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"], c["nv"],
                         n_frames=8) - y_np
    g_o = siddon.backproject(c["geom"], r_o, c["pointing"], c["nu"], c["nv"],
                             n_frames=8).reshape(-1)
    g = grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
    assert rel <= 1e-5, rel


def test_bf16_frames_give_bf16_gradient(T):
    c = synth.make_config("temporal", scale=8)
    Xb = to_dev(c["cube"]).to(torch.bfloat16).requires_grad_(True)
    y = torch.zeros((240, c["nv"], c["nu"]), device="cuda")
    out = T.autograd.project(Xb, c["geom"], c["pointing"], c["nu"], c["nv"],
                             n_frames=8)
    ref = T.tomo_project(Xb.detach(), c["geom"], c["pointing"], c["nu"],
                         c["nv"], n_frames=8)
    assert torch.equal(out, ref)
    (0.5 * ((out - y) ** 2).sum()).backward()
    assert Xb.grad.dtype == torch.bfloat16
    g32 = T.tomo_backproject(out.detach(), c["geom"], c["pointing"],
                             n_frames=8)
    torch.testing.assert_close(Xb.grad.float(), g32.to(torch.bfloat16).float(),
                               rtol=1e-2, atol=1e-3 * float(g32.abs().max()))


def test_full_size_temporal_gradient(T):
    """The full time-varying workload (8 x 256^3, 240 x 512^2): 64 central
    differences, and the transpose against the FP64 oracle by a dot test on
    a seeded 0.1 % pixel sample."""
    c = synth.make_config("temporal")
    X = to_dev(c["cube"])
    y = torch.zeros((240, c["nv"], c["nu"]), device="cuda")
    _fd_check(T, c, X, y, 64, seed=12)
    rng = np.random.default_rng(13)
    n_all = 240 * c["nv"] * c["nu"]
    ids = np.sort(rng.choice(n_all, n_all // 1000, replace=False))
    w = np.zeros(n_all, np.float32)
    w[ids] = rng.standard_normal(ids.size).astype(np.float32)
    Xg = X.clone().requires_grad_(True)
    P = T.autograd.project(Xg, c["geom"], c["pointing"], c["nu"], c["nv"],
                           n_frames=8)
    (P * to_dev(w.reshape(P.shape))).sum().backward()   # grad = P^T w
    lhs = float((Xg.grad.double() * X.double()).sum())
    Px_o = siddon.project(c["geom"], c["cube"], c["pointing"], c["nu"],
                          c["nv"], n_frames=8, ray_ids=ids)
    rhs = float(np.sum(Px_o * w[ids]))
    assert abs(lhs - rhs) <= RTOL_F32 * np.sum(np.abs(Px_o * w[ids])), (lhs, rhs)
