"""tomo_project_noalloc: the forward projection for callers that cannot let
the library allocate device memory (programs that reserve and hand out all
of their device memory themselves, or loops in which a cudaMalloc/cudaFree
that waits for queued work would stall other streams).  Its scratch is a
fixed array inside the library, so the checks here are that it returns what
tomo_project returns, bit for bit, call after call on different geometries (the shared
array keeps the previous call's contents), that it leaves the device's free
memory unchanged, and that an oversized request is refused before any
launch.
"""

import ctypes as C

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import mask_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu

UNSUPPORTED = -3


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def T():
    import paper_1103_5904_gb300 as T
    return T


def _noalloc(T, cube_t, geom, ptg, nu, nv, mask_t, n_frames, out):
    lib = T.load_library()
    cg = T.tomo.cube_geom_struct(geom)
    ig = T.tomo.ImageGeom(ptg.shape[0], nu, nv)
    ptg = np.ascontiguousarray(ptg)
    dtype = T.tomo.TOMO_BF16 if cube_t.dtype == torch.bfloat16 else T.tomo.TOMO_F32
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.tomo_project_noalloc(
        C.byref(cg), int(n_frames), C.c_void_p(cube_t.data_ptr()), dtype,
        C.byref(ig), T.tomo._ptg_ptr(ptg),
        None if mask_t is None else C.c_void_p(mask_t.data_ptr()),
        C.c_void_p(out.data_ptr()), stream)


def _cases():
    small = synth.make_config("small")
    rng = np.random.default_rng(21)
    g = {"nx": 29, "ny": 31, "nz": 33, "x0": -1.4, "y0": -1.55, "z0": -1.3,
         "dx": 2.8 / 29, "dy": 3.1 / 31, "dz": 2.7 / 33}
    ptg = synth.pointing_table(rng.uniform(0, 360, 5), rng.uniform(-30, 30, 5),
                               215.0, 37, 53, 3.6,
                               gain=rng.uniform(0.5, 2.0, 5),
                               time=rng.uniform(0, 2, 5))
    frames = rng.random((3, 33, 31, 29)).astype(np.float32)
    mask = (rng.random((5, 53, 37)) < 0.1).astype(np.uint8)
    return [
        (to_dev(small["cube"]), small["geom"], small["pointing"], 64, 64,
         None, 1),
        (to_dev(frames), g, ptg, 37, 53, mask_dev(mask), 3),
        (to_dev(small["cube"]).to(torch.bfloat16), small["geom"],
         small["pointing"], 64, 64, None, 1),
    ]


def test_noalloc_matches_project_on_consecutive_calls(T):
    cases = _cases()
    want = [T.tomo_project(c, g, p, nu, nv, mask=m, n_frames=f)
            for c, g, p, nu, nv, m, f in cases]
    outs = [torch.full_like(w, np.nan) for w in want]
    torch.cuda.synchronize()
    # first call on the device looks up the scratch address
    assert _noalloc(T, *cases[0], outs[0]) == 0
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for k in (1, 2, 0, 1):  # different geometries back to back
        outs[k].fill_(np.nan)
        assert _noalloc(T, *cases[k], outs[k]) == 0
        torch.cuda.synchronize()
        # the same per-ray sums as tomo_project (whose plane walk adds the
        # same segments in the same order): equal bit for bit
        assert torch.equal(outs[k], want[k]), "noalloc case %d" % k
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_rejects_oversized_request(T):
    # 64 images of 256 x 256 need 64 * 65536 * 32 B = 128 MiB of ray records
    g = synth.cube_geom(16, 1.5)
    ptg = synth.pointing_table(np.arange(64) * 5.0, 0.0, 215.0, 256, 256, 3.2)
    cube = torch.ones((16, 16, 16), device="cuda")
    out = torch.full((64, 256, 256), 7.0, device="cuda")
    assert _noalloc(T, cube, g, ptg, 256, 256, None, 1, out) == UNSUPPORTED
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
