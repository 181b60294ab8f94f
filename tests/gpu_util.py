"""Helpers shared by the GPU parity tests.

Tolerances (FP32 path vs the FP64 oracle):
  projection, per pixel:  |y - y*| <= 1e-5 |y*| + 1e-7 max|y*|
  transpose, per voxel:   |x - x*| <= 1e-5 |x*| + 1e-7 max|x*|  (non-negative
                          images, so the sums do not cancel)
  bf16-stored cube:       the same bound against the oracle on the rounded
                          cube; 1e-2 relative against the float32 cube
The relative 1e-5 is the stated accuracy of the FP32 path.  The absolute
floor is one FP32 ulp-scale (1e-7) of the largest value: pixels whose rays
only graze the cube hold values far below the bright ones, and FP32 cannot
resolve them relative to themselves better than the rounding of the entry
point, which is set by the bright pixels' scale of lengths.
"""

import numpy as np
import pytest
import torch

RTOL_F32 = 1e-5
ATOL_FRAC = 1e-7


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1103_5904_gb300 import build
    build.build()


def close_report(got, want, rtol=RTOL_F32, atol_frac=ATOL_FRAC):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = float(np.abs(want).max()) if want.size else 0.0
    err = np.abs(got - want)
    bound = rtol * np.abs(want) + atol_frac * scale
    bad = err > bound
    rel = err / np.maximum(np.abs(want), 1e-300)
    return bad, rel, scale


def assert_close(got, want, what, rtol=RTOL_F32, atol_frac=ATOL_FRAC):
    bad, rel, scale = close_report(got, want, rtol, atol_frac)
    assert not bad.any(), (
        "%s: %d of %d values outside %.1e rel + %.1e x max (max %.3e); worst "
        "rel err %.3e" % (what, int(bad.sum()), bad.size, rtol, atol_frac,
                          scale, float(rel[bad].max())))


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


def mask_dev(mask):
    return None if mask is None else torch.from_numpy(
        np.ascontiguousarray(mask, dtype=np.uint8)).to("cuda")
