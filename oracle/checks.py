"""Independent FP64 re-derivations of the projector, for pinning the oracle.

Test infrastructure: see ``oracle/__init__.py``.

* :func:`brute_force_ray` — for every voxel box, clip the line against the
  box with the slab method and keep the positive lengths.  Quadratic in the
  cube size: tiny cubes only.  It reaches the definition of the projector
  (length of the line of sight inside each voxel, Eq. lo) without any
  ordering of crossings, so it is independent of the merge enumeration.
* :func:`sampled_ray` — midpoint-rule integration along the ray with step h.
  For a piecewise-constant map its error is at most h * max|x| per voxel
  boundary crossed (each crossing perturbs at most one step), so it
  converges to the exact line integral as h -> 0.
* With an opaque sphere of radius ``r_obs`` at the origin (the photosphere,
  where the paper stops the line-of-sight integration, Section 4): the
  sampled integral keeps the samples before the first one that lies inside
  the sphere, and :func:`first_hit` finds where the ray first reaches the
  sphere by scanning and bisection, which :func:`brute_force_ray` then uses
  as the end of the line.  Neither uses the closed-form root the oracle
  takes.
"""

import numpy as np


def first_hit(o, u, r, s_max, n_scan=200000):
    """Smallest s in [0, s_max] with |o + s u/|u|| <= r, or None: a scan on
    n_scan points followed by bisection to FP64 resolution."""
    o = np.asarray(o, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    u = u / np.linalg.norm(u)
    if np.linalg.norm(o) <= r:
        return 0.0
    s = np.linspace(0.0, s_max, n_scan)
    inside = np.linalg.norm(o[None, :] + s[:, None] * u[None, :], axis=1) <= r
    if not inside.any():
        return None
    k = int(np.argmax(inside))
    a, b = s[k - 1], s[k]
    for _ in range(200):
        m = 0.5 * (a + b)
        if m <= a or m >= b:
            break
        if np.linalg.norm(o + m * u) <= r:
            b = m
        else:
            a = m
    return b


def brute_force_ray(geom, o, u, s_end=np.inf):
    """Dense vector of P_{k,j} (length in each voxel) for one ray,
    ``[nz][ny][nx]`` flattened, over the ray parameters s (distance from o)
    in [0, s_end].  Boxes are closed, so a ray lying exactly in a shared
    face is counted in both voxels: use generic rays."""
    nx, ny, nz = geom["nx"], geom["ny"], geom["nz"]
    lo = np.array([geom["x0"], geom["y0"], geom["z0"]])
    d = np.array([geom["dx"], geom["dy"], geom["dz"]])
    o = np.asarray(o, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    un = np.linalg.norm(u)
    out = np.zeros(nz * ny * nx)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                b0 = lo + np.array([i, j, k]) * d
                b1 = b0 + d
                t_in, t_out = 0.0, np.inf
                miss = False
                for a in range(3):
                    if u[a] == 0.0:
                        if o[a] < b0[a] or o[a] > b1[a]:
                            miss = True
                        continue
                    ta, tb = (b0[a] - o[a]) / u[a], (b1[a] - o[a]) / u[a]
                    t_in = max(t_in, min(ta, tb))
                    t_out = min(t_out, max(ta, tb))
                t_out = min(t_out, s_end / un)
                if miss or t_out <= t_in:
                    continue
                out[(k * ny + j) * nx + i] = (t_out - t_in) * un
    return out


def sampled_ray(geom, cube, o, u, h, s_max, r_obs=0.0):
    """Midpoint-rule line integral of the piecewise-constant map along
    ``o + s u/|u|`` for ``s`` in ``[0, s_max]`` with step ``h``; with
    ``r_obs`` > 0, only the samples before the first one inside the sphere
    of that radius at the origin count."""
    nx, ny, nz = geom["nx"], geom["ny"], geom["nz"]
    lo = np.array([geom["x0"], geom["y0"], geom["z0"]])
    d = np.array([geom["dx"], geom["dy"], geom["dz"]])
    u = np.asarray(u, dtype=np.float64)
    u = u / np.linalg.norm(u)
    n = int(np.ceil(s_max / h))
    s = (np.arange(n) + 0.5) * h
    pts = np.asarray(o, dtype=np.float64)[None, :] + s[:, None] * u[None, :]
    if r_obs > 0.0:
        inside = np.linalg.norm(pts, axis=1) <= r_obs
        if inside.any():
            pts = pts[:int(np.argmax(inside))]
    ijk = np.floor((pts - lo[None, :]) / d[None, :]).astype(np.int64)
    ok = ((ijk[:, 0] >= 0) & (ijk[:, 0] < nx) & (ijk[:, 1] >= 0)
          & (ijk[:, 1] < ny) & (ijk[:, 2] >= 0) & (ijk[:, 2] < nz))
    flat = np.asarray(cube, dtype=np.float64).reshape(-1)
    lin = (ijk[ok, 2] * ny + ijk[ok, 1]) * nx + ijk[ok, 0]
    return float(flat[lin].sum() * h)
