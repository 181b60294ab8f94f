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

Cubes are produced in float64 slab by slab and returned rounded to float32,
the precision the projector stores them in.
"""

import numpy as np

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


def corona_frames(geom, axes, width, amps, background="exp", slab=16):
    """Frames ``[T][nz][ny][nx]`` float32 of a background plus cylinders of
    one ``width`` whose amplitudes change from frame to frame: frame t holds
    ``n_bg + sum_s amps[t][s] * profile_s`` (see :func:`add_structures`)."""
    bgf = _BACKGROUNDS[background]
    amps = np.asarray(amps, dtype=np.float64)
    xs = voxel_centres(geom, "x")
    ys = voxel_centres(geom, "y")
    zs = voxel_centres(geom, "z")
    nz, ny, nx = geom["nz"], geom["ny"], geom["nx"]
    out = np.empty((amps.shape[0], nz, ny, nx), dtype=np.float32)
    for z0 in range(0, nz, slab):
        pz, py, px = np.meshgrid(zs[z0:z0 + slab], ys, xs, indexing="ij")
        bg = bgf(np.sqrt(px * px + py * py + pz * pz))
        prof = [add_structures(px, py, pz, bg, [a], width, 1.0) for a in axes]
        for t in range(amps.shape[0]):
            val = bg.copy()
            for s, p in enumerate(prof):
                val += amps[t, s] * p
            out[t, z0:z0 + slab] = val
    return out


def corona_cube(geom, background="exp", structures=(), noise_frac=0.0,
                noise_rng=None, slab=16):
    """Density cube ``[nz][ny][nx]`` float32.

    ``structures`` is a sequence of ``(axes, width, amp)`` tuples.  The noise
    draws are taken in one call over the whole cube (C order) so that the
    result does not depend on ``slab``.
    """
    bgf = _BACKGROUNDS[background]
    xs = voxel_centres(geom, "x")
    ys = voxel_centres(geom, "y")
    zs = voxel_centres(geom, "z")
    nz, ny, nx = geom["nz"], geom["ny"], geom["nx"]
    out = np.empty((nz, ny, nx), dtype=np.float64)
    for z0 in range(0, nz, slab):
        zz = zs[z0:z0 + slab]
        pz, py, px = np.meshgrid(zz, ys, xs, indexing="ij")
        r = np.sqrt(px * px + py * py + pz * pz)
        bg = bgf(r)
        val = bg.copy()
        for axes, width, amp in structures:
            val += add_structures(px, py, pz, bg, axes, width, amp)
        out[z0:z0 + slab] = val
    if noise_frac:
        out = uniform_noise(out, noise_rng, noise_frac)
    return out.astype(np.float32)
