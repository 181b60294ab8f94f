"""FP64 regularised least squares: the finite-difference prior and CG.

Test infrastructure: see ``oracle/__init__.py``.

The criterion is Eq. criterion of the paper (Section 2.2),

    J(x) = ||y - A x||^2 + lambda ||B x||^2 ,
    x_hat = (A^T A + lambda B^T B)^{-1} A^T y ,

with A = M P (the masked projector: the projector skips masked pixels,
Section 4) and B = D, finite differences along each axis of the map (Section
3.3.1).  Reading of D where the paper is silent: forward
differences ``x[i+1] - x[i]`` along x, y and z, without wrap-around (N - 1
differences per line), the same lambda on every axis (as in Table hypers).

Height-weighted prior (Eq. srt_inversion, Section 3.3.1): B = D R with R a
diagonal operator holding the voxels' heights, so that the
smoothing grows with altitude.  The oracle takes the diagonal as given
(``prior_weight``, one value per voxel; which height, e.g. the radius or
the altitude above the photosphere, is the caller's choice); the normal
operator's prior term is lambda R D^T D R.

Several frames (Section 3.3.3 and the block-diagonal smooth temporal model
of Eq. srt_t / stsrt): with ``n_frames`` T > 1 the map is [T][nz][ny][nx],
each image sees its frames through its time stamp (the projector's time
weights; integer stamps make P block-diagonal, one frame per image group),
the spatial prior applies to every frame and a temporal prior
lambda_t ||D_t x||^2, D_t the forward difference x[t+1] - x[t] between
consecutive frames (no wrap), is added.

White-light data (Section 3.5): with ``kind`` PB or B the projector P is
replaced by the Thomson operator T_pB or T_B of ``thomson.py`` (limb
darkening ``limb_u``) in every formula here.

A map mask (nonzero = voxel excluded from the map) restricts the unknowns
to the other voxels; reading: the excluded voxels are zero in the map that P
and D see, so with K = diag(1 - mask) the criterion is
||M (y - P K x)||^2 + lambda ||D K x||^2 over x = K x, whose normal
equations are K (P^T M P + lambda D^T D) K x = K P^T M y.

The solver is the textbook (Hestenes-Stiefel) conjugate-gradient method on
the normal equations, started from x0 (zero unless given), run for a fixed
number of iterations (the paper uses CG throughout, Sections 3.1 and 5.1; it
tried no preconditioner, Section 5.2).
"""

import numpy as np

from . import siddon, thomson


def D(x):
    """Forward differences along x, y, z of a ``[nz][ny][nx]`` map; returns
    the three difference arrays (axis order x, y, z)."""
    x = np.asarray(x, dtype=np.float64)
    return [np.diff(x, axis=2), np.diff(x, axis=1), np.diff(x, axis=0)]


def Dt(dx, dy, dz):
    """Transpose of :func:`D`: sum over axes of the adjoint of one forward
    difference, which maps a difference array g to -g[i] + g[i-1] padded with
    zeros at the ends."""
    def adj(g, axis):
        n = g.shape[axis] + 1
        shape = list(g.shape)
        shape[axis] = n
        out = np.zeros(shape)
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[axis] = slice(0, n - 1)
        sl_hi[axis] = slice(1, n)
        out[tuple(sl_lo)] -= g
        out[tuple(sl_hi)] += g
        return out
    return adj(dx, 2) + adj(dy, 1) + adj(dz, 0)


def DtD(x):
    return Dt(*D(x))


def DtD_frames(x):
    """D^T D applied to every frame of a map (3-D: the map itself)."""
    x = np.asarray(x, dtype=np.float64)
    return DtD(x) if x.ndim == 3 else np.stack([DtD(f) for f in x])


def Dt_time(x):
    """Temporal forward differences x[t+1] - x[t] of a [T][nz][ny][nx] map."""
    return np.diff(np.asarray(x, dtype=np.float64), axis=0)


def DtD_time(x):
    """D_t^T D_t x: the adjoint of one forward difference along t applied to
    D_t x (-g[t] + g[t-1], zero-padded at the ends)."""
    g = Dt_time(x)
    out = np.zeros(np.shape(x))
    out[:-1] -= g
    out[1:] += g
    return out


def prior_energy(x):
    """||D x||^2."""
    return float(sum(np.sum(g * g) for g in D(x)))


class Problem:
    """One static reconstruction: cube geometry, pointing, mask, data, lambda."""

    def __init__(self, geom, pointing, nu, nv, y, mask=None, lam=0.0,
                 map_mask=None, prior_weight=None, kind=0, limb_u=0.0,
                 n_frames=1, lam_t=0.0):
        self.geom, self.pointing = geom, np.asarray(pointing, np.float64)
        self.nu, self.nv = int(nu), int(nv)
        self.mask = mask
        self.y = np.asarray(y, dtype=np.float64)
        self.lam = float(lam)
        self.T, self.lam_t = int(n_frames), float(lam_t)
        space = (geom["nz"], geom["ny"], geom["nx"])
        self.shape = ((self.T,) if self.T > 1 else ()) + space
        self.keep = (None if map_mask is None else
                     (np.asarray(map_mask) == 0).astype(np.float64))
        self.kind, self.limb_u = int(kind), float(limb_u)
        self.w = (None if prior_weight is None else
                  np.asarray(prior_weight, dtype=np.float64).reshape(space))

    def K(self, x):
        """The map mask: excluded voxels set to 0."""
        return x if self.keep is None else x * self.keep

    def R(self, x):
        """The prior's diagonal weight (identity without one)."""
        return x if self.w is None else x * self.w

    def P(self, x):
        if self.kind:
            return thomson.project(self.kind, self.geom, self.K(x),
                                   self.pointing, self.nu, self.nv,
                                   self.limb_u, self.mask, self.T)
        return siddon.project(self.geom, self.K(x), self.pointing, self.nu,
                              self.nv, self.mask, self.T)

    def Pt(self, y):
        if self.kind:
            return self.K(thomson.backproject(self.kind, self.geom, y,
                                              self.pointing, self.nu, self.nv,
                                              self.limb_u, self.mask, self.T))
        return self.K(siddon.backproject(self.geom, y, self.pointing, self.nu,
                                         self.nv, self.mask, self.T))

    def masked(self, y):
        if self.mask is None:
            return y
        return np.where(self.mask == 0, y, 0.0)

    def rhs(self):
        """b = P^T M y."""
        return self.Pt(self.masked(self.y))

    def normal(self, v):
        """K (P^T M P + lambda R D^T D R + lambda_t D_t^T D_t) K v (K, R =
        identity without map mask or prior weight; D^T D per frame)."""
        out = self.Pt(self.P(v)) + self.lam * self.K(
            self.R(DtD_frames(self.R(self.K(v)))))
        if self.T > 1 and self.lam_t != 0.0:
            out = out + self.lam_t * self.K(DtD_time(self.K(v)))
        return out

    def J(self, x):
        """Eq. criterion: ||M (y - P K x)||^2 + lambda ||D R K x||^2
        (+ lambda_t ||D_t K x||^2 with frames)."""
        r = self.masked(self.y - self.P(x))
        kx = self.K(x)
        spatial = (prior_energy(self.R(kx)) if self.T == 1 else
                   sum(prior_energy(self.R(f)) for f in kx))
        j = float(np.sum(r * r)) + self.lam * spatial
        if self.T > 1:
            j += self.lam_t * float(np.sum(Dt_time(kx) ** 2))
        return j


def cg(problem, n_iter, x0=None, track_J=True):
    """Conjugate gradients on the normal equations.

    Returns ``(x, report)`` where ``report`` holds, per iterate k = 0..n_iter,
    ``J`` (Eq. criterion, evaluated directly) and ``rr`` (squared norm of the
    recursively updated residual).
    """
    b = problem.rhs()
    x = (np.zeros(problem.shape) if x0 is None else
         problem.K(np.array(x0, np.float64)))
    r = b - problem.normal(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    Js = [problem.J(x)] if track_J else []
    rrs = [rr]
    for _ in range(n_iter):
        if rr == 0.0:  # exact solution reached: CG stops
            break
        q = problem.normal(p)
        alpha = rr / float(np.sum(p * q))
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(np.sum(r * r))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        rrs.append(rr)
        if track_J:
            Js.append(problem.J(x))
    return x, {"J": np.array(Js), "rr": np.array(rrs)}
