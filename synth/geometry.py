"""Cube and observer descriptions for the synthetic workloads.

The object map is a cube of identical rectangular voxels (Section 3.3.1 of the
paper: a requirement of the Siddon algorithm), described by its voxel counts,
its minimum corner and its voxel size.  Arrays are laid out ``[nz][ny][nx]``
with x fastest.

An observer is described by a WCS-like pointing record (Section 3.2: the
observer position and the pixel mapping come from the standard WCS keywords).
One record is a row of 12 float64 values, in the column order
``POINTING_COLUMNS``.  Angles are in radians, distances in solar radii, the
frame is Sun-centred with z along the rotation axis and x at longitude 0.
"""

import math

import numpy as np

#: Column order of one pointing record (one row per image).
POINTING_COLUMNS = (
    "d_obs",    # observer distance from Sun centre [R_sun]
    "lon",      # observer longitude [rad]
    "lat",      # observer latitude [rad]
    "roll",     # image roll about the boresight [rad]
    "cdelt_u",  # pixel scale along u [rad / pixel]
    "cdelt_v",  # pixel scale along v [rad / pixel]
    "crpix_u",  # reference pixel along u (0-based)
    "crpix_v",  # reference pixel along v (0-based)
    "crval_u",  # angle of the reference pixel from the boresight, u [rad]
    "crval_v",  # same along v [rad]
    "gain",     # per-image gain g (Eq. two_spacecraft / lin2space)
    "time",     # time stamp tau in frame units (smooth temporal model)
)


def cube_geom(n, half_width, ny=None, nz=None):
    """Geometry of a cube of ``n x ny x nz`` voxels spanning
    ``[-half_width, half_width]`` on every axis (solar radii)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    w = 2.0 * float(half_width)
    return {
        "nx": int(n), "ny": int(ny), "nz": int(nz),
        "x0": -float(half_width), "y0": -float(half_width),
        "z0": -float(half_width),
        "dx": w / n, "dy": w / ny, "dz": w / nz,
    }


def voxel_centres(geom, axis):
    """1-D coordinates of the voxel centres along ``axis`` ('x', 'y', 'z')."""
    n = geom["n" + axis]
    return geom[axis + "0"] + (np.arange(n, dtype=np.float64) + 0.5) * geom["d" + axis]


def cdelt_for_fov(fov, d_obs, n_px):
    """Pixel scale [rad/px] such that ``n_px`` pixels span a width ``fov``
    (solar radii) in the plane of the sky through Sun centre, seen from
    distance ``d_obs``."""
    return 2.0 * math.atan(0.5 * fov / d_obs) / n_px


def pointing_table(lon_deg, lat_deg, d_obs, nu, nv, fov, roll_deg=0.0,
                   gain=1.0, time=None):
    """Pointing records for a set of observers looking at Sun centre.

    ``lon_deg`` / ``lat_deg`` give one entry per image.  The reference pixel
    is the image centre, ``(n - 1) / 2``, with ``crval = 0``.
    """
    lon = np.atleast_1d(np.asarray(lon_deg, dtype=np.float64))
    lat = np.broadcast_to(np.asarray(lat_deg, dtype=np.float64), lon.shape)
    n = lon.shape[0]
    t = np.zeros(n) if time is None else np.broadcast_to(
        np.asarray(time, dtype=np.float64), (n,))
    table = np.zeros((n, len(POINTING_COLUMNS)), dtype=np.float64)
    table[:, 0] = d_obs
    table[:, 1] = np.deg2rad(lon)
    table[:, 2] = np.deg2rad(lat)
    table[:, 3] = np.deg2rad(roll_deg)
    table[:, 4] = cdelt_for_fov(fov, d_obs, nu)
    table[:, 5] = cdelt_for_fov(fov, d_obs, nv)
    table[:, 6] = 0.5 * (nu - 1)
    table[:, 7] = 0.5 * (nv - 1)
    table[:, 8] = 0.0
    table[:, 9] = 0.0
    table[:, 10] = gain
    table[:, 11] = t
    return np.ascontiguousarray(table)
