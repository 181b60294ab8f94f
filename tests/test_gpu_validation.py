"""Host-side argument validation of the C ABI on a real device.

Every invalid call must return its status code before any kernel is
launched, leave the context usable, and set a message.  None of these cases
reaches the GPU with bad data: validation runs first.
"""

import ctypes as C

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu

ARG, UNSUPPORTED = -1, -3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _scene():
    g = synth.cube_geom(16, 1.5)
    ptg = synth.pointing_table([0.0, 60.0], [0.0, 5.0], 215.0, 16, 16, 3.2)
    return g, ptg


def _status(T, fn, *a, **k):
    with pytest.raises(T.TomoError) as e:
        fn(*a, **k)
    return e.value.status


def test_bad_geometry_and_pointing(T):
    g, ptg = _scene()
    cube = torch.ones((16, 16, 16), device="cuda")
    lib = T.load_library()
    ctx = T.default_context()
    out = torch.empty((2, 16, 16), device="cuda")
    cg = T.tomo.cube_geom_struct(dict(g, nx=0))
    ig = T.tomo.ImageGeom(2, 16, 16)
    assert lib.tomo_project(ctx.handle, C.byref(cg), 1,
                            C.c_void_p(cube.data_ptr()), 0, C.byref(ig),
                            T.tomo._ptg_ptr(np.ascontiguousarray(ptg)), None,
                            None, C.c_void_p(out.data_ptr()), None) == ARG
    bad = dict(g, dy=-0.1)
    assert _status(T, T.tomo_project, cube, bad, ptg, 16, 16) == ARG
    p = ptg.copy()
    p[1, 2] = np.pi / 2  # lat = 90 deg
    assert _status(T, T.tomo_project, cube, g, p, 16, 16) == ARG
    p = ptg.copy()
    p[0, 5] = np.nan
    assert _status(T, T.tomo_project, cube, g, p, 16, 16) == ARG
    p = ptg.copy()
    p[0, 4] = 0.25  # 7.5 pixels x 0.25 rad = 1.875 rad: beyond 90 deg
    assert _status(T, T.tomo_project, cube, g, p, 16, 16) == ARG
    p = ptg.copy()
    p[0, 11] = 3.5  # time outside [0, T-1]
    frames = torch.ones((3, 16, 16, 16), device="cuda")
    assert _status(T, T.tomo_project, frames, g, p, 16, 16, n_frames=3) == ARG
    # still usable afterwards
    y = T.tomo_project(cube, g, ptg, 16, 16)
    assert float(y.max()) > 0


def test_bad_pointers_flags_and_options(T):
    g, ptg = _scene()
    lib = T.load_library()
    ctx = T.Context()
    cube = torch.ones((16 * 16 * 16 + 1,), device="cuda")
    out = torch.empty((2, 16, 16), device="cuda")
    cg = T.tomo.cube_geom_struct(g)
    ig = T.tomo.ImageGeom(2, 16, 16)
    pp = T.tomo._ptg_ptr(np.ascontiguousarray(ptg))
    st = lib.tomo_project(ctx.handle, C.byref(cg), 1,
                          C.c_void_p(cube.data_ptr() + 1), 0, C.byref(ig), pp,
                          None, None, C.c_void_p(out.data_ptr()), None)
    assert st == ARG and b"misaligned" in lib.tomo_last_error(ctx.handle)
    st = lib.tomo_project(ctx.handle, C.byref(cg), 1, None, 0, C.byref(ig),
                          pp, None, None, C.c_void_p(out.data_ptr()), None)
    assert st == ARG
    st = lib.tomo_backproject(ctx.handle, C.byref(cg), 1, C.byref(ig), pp,
                              None, None, C.c_void_p(out.data_ptr()),
                              C.c_void_p(cube.data_ptr()), 0x80, None)
    assert st == ARG
    assert lib.tomo_set_option(ctx.handle, 99, 1) == ARG
    ctx.set_tiling(24, 8, 8)  # valid: 3 x 2 warps of 8 x 4 pixels
    ctx.set_option(T.tomo.TOMO_OPT_WARP_U, 16)  # 24 % 16 != 0: rejected at launch
    with pytest.raises(T.TomoError):
        T.tomo_project(cube[:4096].reshape(16, 16, 16), g, ptg, 16, 16, ctx=ctx)
    ctx.set_tiling(32, 8, 8)
    y = T.tomo_project(cube[:4096].reshape(16, 16, 16), g, ptg, 16, 16, ctx=ctx)
    assert float(y.max()) > 0
    ctx.close()


def test_solver_arguments(T):
    g, ptg = _scene()
    y = torch.ones((2, 16, 16), device="cuda")
    for kw in [dict(lam=-1.0), dict(lam=float("nan")), dict(max_iter=-1),
               dict(tol=-0.5)]:
        args = dict(lam=0.1, max_iter=3)
        args.update(kw)
        assert _status(T, T.tomo_solve, y, g, ptg, **args) == ARG


def test_invalid_device(T):
    lib = T.load_library()
    h = C.c_void_p()
    assert lib.tomo_create(C.byref(h), 1 << 20) == ARG


def test_map_mask_arguments(T):
    """A map mask must be a uint8 CUDA tensor of nx * ny * nz elements."""
    g, ptg = _scene()
    cube = torch.ones((16, 16, 16), device="cuda")
    y = torch.ones((2, 16, 16), device="cuda")
    with pytest.raises(ValueError):
        T.tomo_project(cube, g, ptg, 16, 16,
                       map_mask=torch.zeros(100, dtype=torch.uint8,
                                            device="cuda"))
    with pytest.raises(TypeError):
        T.tomo_backproject(y, g, ptg, map_mask=torch.zeros(
            (16, 16, 16), dtype=torch.float32, device="cuda"))
    with pytest.raises(TypeError):
        T.tomo_solve(y, g, ptg, map_mask=torch.zeros((16, 16, 16),
                                                     dtype=torch.uint8))
