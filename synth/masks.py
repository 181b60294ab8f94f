"""Pixel masks of a coronagraph-like instrument, map masks and the radial
weights of a height-weighted prior.

A coronagraph hides the solar disk behind an occulter and sees out to a field
edge; both are disks in the image plane, centred on the direction of Sun
centre.  A disk of angular radius ``asin(r / d_obs)`` holds exactly the pixels
whose line of sight passes within ``r`` of Sun centre, so the recipe below
is stated in those terms: a pixel is masked (value 1) when the impact
parameter of its line of sight is below ``r_occ`` or above ``r_edge``.

The pixel's angle from the boresight follows the gnomonic (TAN) pixel mapping
of the pointing record: ``tan^2(theta) = tan^2(theta_u) + tan^2(theta_v)``
with ``theta_u = (i_u - crpix_u) cdelt_u + crval_u``.  Masks are uint8
``[n_img][nv][nu]``; nonzero means excluded.
"""

import numpy as np

from .geometry import voxel_centres


def occulter_mask(pointing, nu, nv, r_occ=None, r_edge=None):
    n = pointing.shape[0]
    mask = np.zeros((n, nv, nu), dtype=np.uint8)
    if r_occ is None and r_edge is None:
        return mask
    iu = np.arange(nu, dtype=np.float64)
    iv = np.arange(nv, dtype=np.float64)
    for k in range(n):
        d, _, _, _, cu, cv, pu, pv, vu, vv = pointing[k, :10]
        tu = np.tan((iu - pu) * cu + vu)
        tv = np.tan((iv - pv) * cv + vv)
        t2 = tv[:, None] ** 2 + tu[None, :] ** 2
        # impact parameter rho = d sin(theta), sin^2 = tan^2 / (1 + tan^2)
        rho = d * np.sqrt(t2 / (1.0 + t2))
        m = np.zeros((nv, nu), dtype=bool)
        if r_occ is not None:
            m |= rho < r_occ
        if r_edge is not None:
            m |= rho > r_edge
        mask[k] = m
    return mask


def shell_map_mask(geom, r_in=None, r_out=None):
    """Map mask of a spherical shell: voxels whose centre lies below ``r_in``
    (inside the photosphere) or above ``r_out`` (beyond the field of view)
    are excluded.  uint8 ``[nz][ny][nx]``; nonzero means excluded."""
    x = voxel_centres(geom, "x")
    y = voxel_centres(geom, "y")
    z = voxel_centres(geom, "z")
    r = np.sqrt(z[:, None, None] ** 2 + y[None, :, None] ** 2 +
                x[None, None, :] ** 2)
    m = np.zeros(r.shape, dtype=bool)
    if r_in is not None:
        m |= r < r_in
    if r_out is not None:
        m |= r > r_out
    return m.astype(np.uint8)


def height_weights(geom, r_ref=0.0, floor=0.0):
    """Diagonal of a height-weighted prior: the distance of each voxel centre
    from Sun centre minus ``r_ref`` (``r_ref = 1``: altitude above the
    photosphere), not below ``floor``.  float64 ``[nz][ny][nx]``."""
    x = voxel_centres(geom, "x")
    y = voxel_centres(geom, "y")
    z = voxel_centres(geom, "z")
    r = np.sqrt(z[:, None, None] ** 2 + y[None, :, None] ** 2 +
                x[None, None, :] ** 2)
    return np.maximum(r - r_ref, floor)
