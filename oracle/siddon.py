"""ctypes bindings of the FP64 oracle library (``siddon_oracle.c``).

Test infrastructure: see ``oracle/__init__.py``.  All arrays are float64 and
C-contiguous; cubes are ``[T][nz][ny][nx]`` (or ``[nz][ny][nx]``), images
``[n_img][nv][nu]``, pointing tables ``(n_img, 12)`` in the column order of
the pointing record (d_obs, lon, lat, roll, cdelt_u, cdelt_v, crpix_u,
crpix_v, crval_u, crval_v, gain, time).
"""

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


class _Cube(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("d", C.c_double * 3), ("r_obs", C.c_double)]


def _cube(geom):
    """Cube geometry; an optional ``geom["r_obs"]`` > 0 is the radius of the
    opaque sphere at the origin where lines of sight end."""
    c = _Cube()
    c.n[:] = [geom["nx"], geom["ny"], geom["nz"]]
    c.lo[:] = [geom["x0"], geom["y0"], geom["z0"]]
    c.d[:] = [geom["dx"], geom["dy"], geom["dz"]]
    c.r_obs = float(geom.get("r_obs", 0.0))
    return c


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        lp = C.POINTER(C.c_int64)
        up = C.POINTER(C.c_uint8)
        cp = C.POINTER(_Cube)
        L.orc_ray.argtypes = [dp, C.c_int32, C.c_int32, dp, dp]
        L.orc_ray.restype = C.c_int
        L.orc_clip.argtypes = [cp, dp, dp, dp, dp]
        L.orc_clip.restype = C.c_int
        L.orc_max_segments.argtypes = [cp]
        L.orc_max_segments.restype = C.c_int64
        L.orc_segments.argtypes = [cp, dp, dp, lp, dp, dp, dp]
        L.orc_segments.restype = C.c_int64
        L.orc_project.argtypes = [cp, C.c_int32, dp, C.c_int32, C.c_int32,
                                  C.c_int32, dp, up, C.c_int64, lp, dp]
        L.orc_project.restype = C.c_int
        L.orc_backproject.argtypes = [cp, C.c_int32, C.c_int32, C.c_int32,
                                      C.c_int32, dp, up, dp, C.c_int64, lp,
                                      dp]
        L.orc_backproject.restype = C.c_int
        L.orc_crossing_weights.argtypes = L.orc_backproject.argtypes
        L.orc_crossing_weights.restype = C.c_int
        L.orc_count_segments.argtypes = [cp, C.c_int32, C.c_int32, C.c_int32,
                                         dp, up, C.c_int64, lp]
        L.orc_count_segments.restype = C.c_int64
        L.orc_impact2.argtypes = [C.c_int32, C.c_int32, C.c_int32, dp, dp]
        L.orc_impact2.restype = C.c_int
        L.orc_get_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mask_ptr(mask):
    if mask is None:
        return None, None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    return m, m.ctypes.data_as(C.POINTER(C.c_uint8))


def _rays(ray_ids):
    if ray_ids is None:
        return None, 0, None
    r = np.ascontiguousarray(ray_ids, dtype=np.int64)
    return r, r.shape[0], r.ctypes.data_as(C.POINTER(C.c_int64))


def get_threads():
    return lib().orc_get_threads()


def set_threads(n):
    lib().orc_set_threads(int(n))


def ray(pointing_row, iu, iv):
    """(o, u): observer position and unit direction of pixel (iu, iv)."""
    p = _f64(pointing_row)
    o = np.zeros(3)
    u = np.zeros(3)
    if lib().orc_ray(_dp(p), int(iu), int(iv), _dp(o), _dp(u)) != 0:
        raise ValueError("pointing frame undefined")
    return o, u


def clip(geom, o, u):
    """(hit, amin, amax) of the half-line o + a u against the cube."""
    c = _cube(geom)
    o, u = _f64(o), _f64(u)
    a0 = C.c_double()
    a1 = C.c_double()
    hit = lib().orc_clip(C.byref(c), _dp(o), _dp(u), C.byref(a0), C.byref(a1))
    return bool(hit), a0.value, a1.value


def segments(geom, o, u):
    """(voxel linear indices, lengths, amin, amax) of the ray o + a u."""
    c = _cube(geom)
    cap = lib().orc_max_segments(C.byref(c))
    idx = np.zeros(cap, dtype=np.int64)
    ln = np.zeros(cap)
    o, u = _f64(o), _f64(u)
    a0 = C.c_double()
    a1 = C.c_double()
    n = lib().orc_segments(C.byref(c), _dp(o), _dp(u),
                           idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(ln),
                           C.byref(a0), C.byref(a1))
    return idx[:n].copy(), ln[:n].copy(), a0.value, a1.value


def _keep(map_mask):
    """1 on the voxels that are unknowns, 0 on those a map mask excludes."""
    return (np.asarray(map_mask) == 0).astype(np.float64)


def project(geom, cube, pointing, nu, nv, mask=None, n_frames=1,
            ray_ids=None, map_mask=None):
    """FP64 ``y = P x``; returns ``[n_img][nv][nu]`` or, with ``ray_ids``, the
    values of those rays.  ``map_mask`` ([nz][ny][nx], nonzero = voxel
    excluded from the map, the counterpart of the pixel mask that Section 4
    names for the map): the excluded voxels are read as 0, in every frame."""
    c = _cube(geom)
    cube = _f64(cube)
    if map_mask is not None:
        cube = _f64(cube * _keep(map_mask))
    ptg = _f64(pointing)
    n_img = ptg.shape[0]
    m, mp = _mask_ptr(mask)
    r, nr, rp = _rays(ray_ids)
    out = np.zeros(nr if r is not None else n_img * nv * nu)
    rc = lib().orc_project(C.byref(c), int(n_frames), _dp(cube), n_img,
                           int(nu), int(nv), _dp(ptg), mp, nr, rp, _dp(out))
    if rc != 0:
        raise ValueError("invalid pointing or time stamp")
    return out if r is not None else out.reshape(n_img, nv, nu)


def backproject(geom, images, pointing, nu, nv, mask=None, n_frames=1,
                ray_ids=None, map_mask=None):
    """FP64 ``x = P^T y``; ``images`` is a full ``[n_img][nv][nu]`` stack
    (with ``ray_ids``, only those pixels are used).  With ``map_mask`` the
    excluded voxels receive 0 (the transpose of reading them as 0)."""
    c = _cube(geom)
    ptg = _f64(pointing)
    n_img = ptg.shape[0]
    img = _f64(images).reshape(-1)
    if img.shape[0] != n_img * nv * nu:
        raise ValueError("image stack shape")
    m, mp = _mask_ptr(mask)
    r, nr, rp = _rays(ray_ids)
    T = max(int(n_frames), 1)
    shape = (geom["nz"], geom["ny"], geom["nx"])
    out = np.zeros(((T,) if n_frames > 1 else ()) + shape)
    rc = lib().orc_backproject(C.byref(c), int(n_frames), n_img, int(nu),
                               int(nv), _dp(ptg), mp, _dp(img), nr, rp,
                               _dp(out))
    if rc != 0:
        raise ValueError("invalid pointing or time stamp")
    if map_mask is not None:
        out = out * _keep(map_mask)
    return out


def crossing_weights(geom, images, pointing, nu, nv, mask=None, n_frames=1,
                     ray_ids=None):
    """C_j = sum of |g_k y_k| over the rays k crossing voxel j (positive
    length), time-weighted like the transpose."""
    c = _cube(geom)
    ptg = _f64(pointing)
    n_img = ptg.shape[0]
    img = _f64(images).reshape(-1)
    m, mp = _mask_ptr(mask)
    r, nr, rp = _rays(ray_ids)
    T = max(int(n_frames), 1)
    shape = (geom["nz"], geom["ny"], geom["nx"])
    out = np.zeros(((T,) if n_frames > 1 else ()) + shape)
    rc = lib().orc_crossing_weights(C.byref(c), int(n_frames), n_img, int(nu),
                                    int(nv), _dp(ptg), mp, _dp(img), nr, rp,
                                    _dp(out))
    if rc != 0:
        raise ValueError("invalid pointing or time stamp")
    return out


def count_segments(geom, pointing, nu, nv, mask=None, ray_ids=None):
    """Number of positive-length voxel intersections of the (unmasked) rays."""
    c = _cube(geom)
    ptg = _f64(pointing)
    m, mp = _mask_ptr(mask)
    r, nr, rp = _rays(ray_ids)
    return int(lib().orc_count_segments(C.byref(c), ptg.shape[0], int(nu),
                                        int(nv), _dp(ptg), mp, nr, rp))


def impact2(pointing, nu, nv):
    """rho^2 = |o x u|^2 of every pixel's line of sight, ``[n_img][nv][nu]``
    (the squared distance of Sun centre from the line)."""
    ptg = _f64(pointing)
    out = np.zeros((ptg.shape[0], int(nv), int(nu)))
    if lib().orc_impact2(ptg.shape[0], int(nu), int(nv), _dp(ptg),
                         _dp(out)) != 0:
        raise ValueError("pointing frame undefined")
    return out
