"""FP64 Thomson-scattering operators (white-light pB and B images).

Test infrastructure: see ``oracle/__init__.py``.

Section 3.5 of the paper writes the intensities scattered by coronal
electrons (Eq. thomson_corona) with the van de Hulst coefficients C1..C4 of
the angle Omega (Eq. 4C), splits them into a per-pixel factor o_k = rho_k^2
and per-voxel factors m_j, m'_j (Eq. thomson_lo), and builds the operators
(Eq. brightness, Eq. thomson_direct)

    T_pB = O P M ,            T_B = -O P M + P M' ,

O, M, M' diagonal.  Readings where the paper is garbled, at odds with
itself or silent (each pinned in ``tests/test_oracle_pins.py``):

  * sin(Omega) = 1 / r (r in solar radii): Omega is the half-angle of the
    solar disk seen from the scattering point, the integration limit of the
    coefficients; the caption's wording does not define it.
  * C4 carries +1/8, not -1/8: with -1/8, C4 < 0 for every r > 1 and the
    tangential intensity of a limb-darkened Sun (u = 1) would be negative.
    The coefficients are integrals over the solar disk of positive
    quantities; a direct quadrature of those integrals (the pins) gives pi
    times C1..C4 with +1/8 on C4.
  * m_j = ((1 - u) C1 + u C2) / r^4: Eq. brightness; Eq. thomson_lo drops
    the u on C2.
  * m'_j = 2 ((1 - u) C3 + u C4) / r^2: Eq. brightness has the factor 2
    (B = I_t + I_r = 2 I_t - (I_t - I_r)); Eq. thomson_lo omits it, and
    Eq. thomson_direct then reproduces Eq. brightness only with it.
  * the powers of r (r^-4 in m, r^-2 in m') are the paper's, printed alike
    in Eq. thomson_corona, Eq. thomson_lo and Eq. brightness; the common
    constant pi sigma I0 / 2 is left out (an overall scale, which per-image
    gains can carry).
  * inside the photosphere (r <= 1) there is no scattering: m = m' = 0
    (Omega is undefined there).
"""

import numpy as np

from . import siddon

PB, B = 1, 2


def coefficients(r):
    """C1..C4 of Eq. 4C at distance r > 1 from Sun centre (sin Omega = 1/r),
    C4 with the +1/8 reading.  Returns four arrays."""
    r = np.asarray(r, dtype=np.float64)
    s = 1.0 / r
    c = np.sqrt(1.0 - s * s)
    # (cos^2 / sin) ln((1 + sin) / cos), 0 at sin = 1
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(c > 0.0, c * c / s * np.log((1.0 + s) / c), 0.0)
    C1 = c * s * s
    C2 = -0.125 * (1.0 - 3.0 * s * s - g * (1.0 + 3.0 * s * s))
    C3 = 4.0 / 3.0 - c - c ** 3 / 3.0
    C4 = 0.125 * (5.0 + s * s - g * (5.0 - s * s))
    return C1, C2, C3, C4


def voxel_factors(geom, limb_u):
    """(m, m') at the voxel centres, ``[nz][ny][nx]`` each (Eq. brightness
    readings above); 0 where r <= 1."""
    ax = [geom[a + "0"] + (np.arange(geom["n" + a]) + 0.5) * geom["d" + a]
          for a in "xyz"]
    r = np.sqrt(ax[2][:, None, None] ** 2 + ax[1][None, :, None] ** 2 +
                ax[0][None, None, :] ** 2)
    out = r > 1.0
    rr = np.where(out, r, 2.0)  # placeholder radius inside the Sun
    C1, C2, C3, C4 = coefficients(rr)
    u = float(limb_u)
    m = np.where(out, ((1.0 - u) * C1 + u * C2) / rr ** 4, 0.0)
    mp = np.where(out, 2.0 * ((1.0 - u) * C3 + u * C4) / rr ** 2, 0.0)
    return m, mp


def project(kind, geom, cube, pointing, nu, nv, limb_u, mask=None,
            n_frames=1, map_mask=None):
    """T x for kind PB (O P M x) or B (P M' x - O P M x); images
    ``[n_img][nv][nu]``."""
    m, mp = voxel_factors(geom, limb_u)
    x = np.asarray(cube, dtype=np.float64)
    o = siddon.impact2(pointing, nu, nv)
    pm = siddon.project(geom, x * m, pointing, nu, nv, mask, n_frames,
                        map_mask=map_mask)
    if kind == PB:
        return o * pm
    if kind == B:
        return siddon.project(geom, x * mp, pointing, nu, nv, mask, n_frames,
                              map_mask=map_mask) - o * pm
    raise ValueError("kind must be PB or B")


def backproject(kind, geom, images, pointing, nu, nv, limb_u, mask=None,
                n_frames=1, map_mask=None):
    """T^T y: M P^T O y (PB) or M' P^T y - M P^T O y (B)."""
    m, mp = voxel_factors(geom, limb_u)
    y = np.asarray(images, dtype=np.float64)
    o = siddon.impact2(pointing, nu, nv)
    pto = siddon.backproject(geom, o * y, pointing, nu, nv, mask, n_frames,
                             map_mask=map_mask)
    if kind == PB:
        return m * pto
    if kind == B:
        return mp * siddon.backproject(geom, y, pointing, nu, nv, mask,
                                       n_frames, map_mask=map_mask) - m * pto
    raise ValueError("kind must be PB or B")
