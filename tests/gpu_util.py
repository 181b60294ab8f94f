"""Helpers shared by the GPU parity tests.

Tolerances (FP32 path vs the FP64 oracle):
  projection, per pixel:  |y - y*| <= 1e-5 |y*| + 1e-7 max|y*|
  transpose, per voxel:   |x - x*| <= 1e-5 |x*| + 8 u t_max C_j
                                      + 2 u t_max N_j,  u = 2^-24,
                          t_max = the cube's diagonal, C_j = sum of |g y| over
                          the rays crossing voxel j (oracle crossing weights),
                          N_j = sum of C over the 3 x 3 x 3 voxels around j
  bf16-stored cube:       the same bound against the oracle on the rounded
                          cube; 1e-2 relative against the float32 cube
The relative 1e-5 is the stated accuracy of the FP32 path.  Every FP32
segment length is a difference of two crossing parameters measured from the
ray's entry point, so it carries an absolute error of a few ulp(t) <= a few
u t_max whatever its length: along a ray these errors telescope (P), but a
voxel that a ray only clips at a corner receives that absolute error on a
tiny length.  The transpose bound therefore adds 8 u t_max per crossing ray,
weighted by the ray's |g y|.  The projection's absolute floor, 1e-7 of the
largest pixel, covers pixels whose rays only graze the cube: their values
are far below the bright ones, and one crossing's rounding is not small
relative to them.  Where two crossing parameters of a ray lie within an ulp
of each other, the FP32 and FP64 walks can cross the two planes in
different orders; the FP32 walk then charges at most ulp(t_max) <= 2 u t_max
of length to a voxel that shares an edge or corner with the FP64 path and
that the FP64 walk does not cross at all: the N_j term (such a ray crosses
one of the 26 neighbours of j in FP64, so its |g y| is part of N_j).
"""

import numpy as np
import pytest
import torch

RTOL_F32 = 1e-5
ATOL_FRAC = 1e-7

# (what, elements that meet the relative bound only with the absolute term,
# elements compared): printed at the end of the session (tests/conftest.py),
# so that a regression hiding under the absolute term shows as a growing
# share
FLOOR_SHARES = []


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
    floor = (rel > rtol) & ~bad
    FLOOR_SHARES.append((what, int(floor.sum()), int(bad.size)))
    assert not bad.any(), (
        "%s: %d of %d values outside %.1e rel + %.1e x max (max %.3e); worst "
        "rel err %.3e" % (what, int(bad.sum()), bad.size, rtol, atol_frac,
                          scale, float(rel[bad].max())))


def box_sum3(a):
    """Sum of ``a`` over the 3 x 3 x 3 block around every voxel of the last
    three axes (zero outside the array)."""
    s = np.array(a, dtype=np.float64)
    for ax in range(s.ndim - 3, s.ndim):
        t = s.copy()
        lo = [slice(None)] * s.ndim
        hi = [slice(None)] * s.ndim
        lo[ax], hi[ax] = slice(1, None), slice(None, -1)
        t[tuple(lo)] += s[tuple(hi)]
        t[tuple(hi)] += s[tuple(lo)]
        s = t
    return s


def assert_transpose_close(got, want, cw, geom, what, rtol=RTOL_F32):
    """Per-voxel transpose bound (module docstring); ``cw`` are the oracle's
    crossing weights for the same images."""
    t_max = float(np.sqrt(sum((geom["n" + a] * geom["d" + a]) ** 2
                              for a in "xyz")))
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    u = 2.0 ** -24
    bound = (rtol * np.abs(want) + 8.0 * u * t_max * np.asarray(cw)
             + 2.0 * u * t_max * box_sum3(cw))
    err = np.abs(got - want)
    bad = err > bound
    floor = (err > rtol * np.abs(want)) & ~bad
    FLOOR_SHARES.append((what, int(floor.sum()), int(bad.size)))
    assert not bad.any(), (
        "%s: %d of %d voxels outside the bound; worst err/bound %.3f"
        % (what, int(bad.sum()), bad.size, float((err / np.maximum(
            bound, 1e-300)).max())))


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


def mask_dev(mask):
    return None if mask is None else torch.from_numpy(
        np.ascontiguousarray(mask, dtype=np.uint8)).to("cuda")
