"""Corona-shaped density cubes, evaluated at voxel centres.

Recipes (seeded; all in solar radii):

* ``radial_exp``: ``n(r) = exp(-(r - 1) / 0.1)`` for ``r >= 1``, ``0`` inside
  the Sun.  The exponential is continued beyond ``r = 1.5`` (it is below
  6.7e-3 there).
* ``radial_power``: ``n(r) = r**-6 + 0.05 r**-2`` for ``r >= 1``, ``0`` inside.
* streamers / plumes: radial Gaussian cylinders about a unit axis ``a``; a voxel
  at ``p`` with ``p.a > 0`` gets ``amp * n_bg(r) * exp(-d^2 / (2 w^2))`` added,
  with ``d`` its distance to the axis.  Streamer axes are uniform on the sphere;
  plume axes lie within 20 degrees of +z or -z.
* multiplicative uniform noise: ``x * (1 + f * U[-1, 1))``, which keeps the
  solar interior at zero.

Cubes are produced in float64 slab by slab (torch CPU operations, which run
on every host core) and returned rounded to float32, the precision the
projector stores them in.  ``radial_exp``, ``radial_power`` and
``add_structures`` evaluate the same recipes on numpy arrays of points.
"""

import numpy as np
import torch

from .geometry import voxel_centres


def radial_exp(r, scale_height=0.1):
    out = np.zeros_like(r)
    m = r >= 1.0
    out[m] = np.exp(-(r[m] - 1.0) / scale_height)
    return out


def radial_power(r):
    out = np.zeros_like(r)
    m = r >= 1.0
    rm = r[m]
    out[m] = rm ** -6 + 0.05 * rm ** -2
    return out


_BACKGROUNDS = {"exp": radial_exp, "power": radial_power}


def random_axes(rng, n, polar_within_deg=None):
    """``n`` unit vectors: uniform on the sphere, or (``polar_within_deg``)
    uniform on the two polar caps of that half-angle about +z and -z."""
    if n == 0:
        return np.zeros((0, 3))
    if polar_within_deg is None:
        v = rng.standard_normal((n, 3))
        return v / np.linalg.norm(v, axis=1, keepdims=True)
    cmin = np.cos(np.deg2rad(polar_within_deg))
    cz = rng.uniform(cmin, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(phi), sz * np.sin(phi), sign * cz], axis=1)


def add_structures(px, py, pz, bg, axes, width, amp):
    """Sum of radial Gaussian cylinders (see module docstring); returns the
    added density for points ``(px, py, pz)`` with background ``bg``.
    ``amp`` is a scalar or one value per axis."""
    out = np.zeros_like(bg)
    amps = np.broadcast_to(np.asarray(amp, dtype=np.float64), (len(axes),))
    r2 = px * px + py * py + pz * pz
    for a, am in zip(axes, amps):
        proj = px * a[0] + py * a[1] + pz * a[2]
        d2 = np.maximum(r2 - proj * proj, 0.0)
        out += np.where(proj > 0.0,
                        am * bg * np.exp(-d2 / (2.0 * width * width)), 0.0)
    return out


def uniform_noise(x, rng, frac):
    return x * (1.0 + frac * rng.uniform(-1.0, 1.0, size=x.shape))


def _grid(geom, z0, z1):
    """Broadcastable float64 voxel-centre coordinates of slab z0:z1."""
    xs = torch.from_numpy(voxel_centres(geom, "x"))
    ys = torch.from_numpy(voxel_centres(geom, "y"))
    zs = torch.from_numpy(voxel_centres(geom, "z")[z0:z1])
    return xs.view(1, 1, -1), ys.view(1, -1, 1), zs.view(-1, 1, 1)


def _background(name, r):
    one = torch.ones((), dtype=r.dtype)
    if name == "exp":
        val = torch.exp(-(r - 1.0) / 0.1)
    else:
        val = r.pow(-6) + 0.05 * r.pow(-2)
    return torch.where(r >= one, val, torch.zeros((), dtype=r.dtype))


def _profiles(px, py, pz, r2, bg, axes, width):
    """One radial Gaussian cylinder profile (amplitude 1) per axis."""
    out = []
    for a in axes:
        proj = px * float(a[0]) + py * float(a[1]) + pz * float(a[2])
        d2 = torch.clamp(r2 - proj * proj, min=0.0)
        prof = bg * torch.exp(d2 * (-0.5 / (width * width)))
        out.append(torch.where(proj > 0.0, prof, torch.zeros((), dtype=prof.dtype)))
    return out


def corona_frames(geom, axes, width, amps, background="exp", slab=4):
    """Frames ``[T][nz][ny][nx]`` float32 of a background plus cylinders of
    one ``width`` whose amplitudes change from frame to frame: frame t holds
    ``n_bg + sum_s amps[t][s] * profile_s`` (see :func:`add_structures`)."""
    amps = np.asarray(amps, dtype=np.float64)
    nz, ny, nx = geom["nz"], geom["ny"], geom["nx"]
    out = np.empty((amps.shape[0], nz, ny, nx), dtype=np.float32)
    for z0 in range(0, nz, slab):
        px, py, pz = _grid(geom, z0, min(z0 + slab, nz))
        r2 = px * px + py * py + pz * pz
        bg = _background(background, torch.sqrt(r2))
        prof = _profiles(px, py, pz, r2, bg, axes, width)
        for t in range(amps.shape[0]):
            val = bg.clone()
            for s_, p_ in enumerate(prof):
                val += float(amps[t, s_]) * p_
            out[t, z0:z0 + slab] = val.numpy()
    return out


def corona_cube(geom, background="exp", structures=(), noise_frac=0.0,
                noise_rng=None, slab=4):
    """Density cube ``[nz][ny][nx]`` float32.

    ``structures`` is a sequence of ``(axes, width, amp)`` tuples.  The noise
    draws are taken in one call over the whole cube (C order) so that the
    result does not depend on ``slab``.  Evaluated in float64 with torch CPU
    operations (multithreaded), slab by slab.
    """
    nz, ny, nx = geom["nz"], geom["ny"], geom["nx"]
    out = np.empty((nz, ny, nx), dtype=np.float64)
    for z0 in range(0, nz, slab):
        px, py, pz = _grid(geom, z0, min(z0 + slab, nz))
        r2 = px * px + py * py + pz * pz
        bg = _background(background, torch.sqrt(r2))
        val = bg.clone()
        for axes, width, amp in structures:
            amps = np.broadcast_to(np.asarray(amp, dtype=np.float64), (len(axes),))
            for am, prof in zip(amps, _profiles(px, py, pz, r2, bg, axes, width)):
                val += float(am) * prof
        out[z0:z0 + slab] = val.numpy()
    if noise_frac:
        out = uniform_noise(out, noise_rng, noise_frac)
    return out.astype(np.float32)
