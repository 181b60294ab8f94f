"""Python binding of libtomo (``include/tomo.h``): argument marshalling only.

Every function here has the name of the C entry point it calls.  Tensors are
PyTorch CUDA tensors (device memory and streams only); all computation
happens in the library's CUDA kernels.  There is no CPU fallback: if the
library is missing or cannot be loaded, every call raises.

Geometry arguments:
  ``geom``      dict with nx, ny, nz, x0, y0, z0, dx, dy, dz (the layout of
                ``synth.cube_geom``)
  ``pointing``  float64 array (n_img, 12), one pointing record per row in the
                field order of ``tomo_pointing``
"""

import ctypes as C
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtomo.so")

TOMO_F32, TOMO_BF16 = 0, 1
TOMO_ACCUMULATE, TOMO_SOLVE_X0, TOMO_SOLVE_BF16 = 1, 2, 4
TOMO_OPT_RAY_CACHE, TOMO_OPT_TILE_U, TOMO_OPT_TILE_V, TOMO_OPT_WARP_U = 1, 2, 3, 4
TOMO_OPT_PROFILE = 5
TOMO_OPT_PLANE_SYNC = 7
TOMO_OPT_CHANNELS = 8
TOMO_OPT_GROUP_FWD, TOMO_OPT_GROUP_ADJ = 9, 10
TOMO_BATCH_AUTOTUNE = 8
KERNEL_CLASSES = ("setup", "forward", "adjoint", "prior", "vector", "layout")

STATUS = {0: "TOMO_OK", -1: "TOMO_ERR_ARG", -2: "TOMO_ERR_CUDA",
          -3: "TOMO_ERR_UNSUPPORTED", -4: "TOMO_ERR_OOM",
          -5: "TOMO_ERR_TIMEOUT", -6: "TOMO_ERR_NUMERIC"}


class CubeGeom(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("reserved", C.c_int32), ("x0", C.c_double),
                ("y0", C.c_double), ("z0", C.c_double), ("dx", C.c_double),
                ("dy", C.c_double), ("dz", C.c_double), ("r_obs", C.c_double)]


class ImageGeom(C.Structure):
    _fields_ = [("n_img", C.c_int32), ("nu", C.c_int32), ("nv", C.c_int32),
                ("kind", C.c_int32), ("limb_u", C.c_double)]


# what the images measure (tomo_image_geom.kind): line-of-sight emission,
# polarised brightness pB or total brightness B (Thomson scattering)
KINDS = {"emission": 0, "pB": 1, "B": 2}


def _kind(kind):
    if kind not in KINDS:
        raise ValueError("kind must be one of %s" % sorted(KINDS))
    return KINDS[kind]


class Pointing(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "d_obs", "lon", "lat", "roll", "cdelt_u", "cdelt_v", "crpix_u",
        "crpix_v", "crval_u", "crval_v", "gain", "time")]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * len(KERNEL_CLASSES)),
                ("ms", C.c_double * len(KERNEL_CLASSES))]


class Problem(C.Structure):
    _fields_ = [("cube", CubeGeom), ("img", ImageGeom), ("reserved", C.c_int32),
                ("pointing_host", C.POINTER(Pointing)), ("mask_dev", C.c_void_p),
                ("images_dev", C.c_void_p), ("cube_dev", C.c_void_p),
                ("lam", C.c_double), ("map_mask_dev", C.c_void_p),
                ("prior_weight_dev", C.c_void_p)]


class PlaneRules(C.Structure):
    _fields_ = [("min_pitch", C.c_double), ("fwd_min_pitch", C.c_double),
                ("fwd_max_ratio", C.c_double), ("general_ratio", C.c_double),
                ("fwd_group", C.c_double), ("adj_group", C.c_double)]


class TilingResult(C.Structure):
    _fields_ = [("tile_u", C.c_int32), ("tile_v", C.c_int32),
                ("warp_u", C.c_int32), ("fwd_ms", C.c_float),
                ("adj_ms", C.c_float), ("rules", PlaneRules)]


RULE_FIELDS = ("min_pitch", "fwd_min_pitch", "fwd_max_ratio", "general_ratio",
               "fwd_group", "adj_group")
NEVER = 1e30  # a walk-rule threshold that is never reached


assert C.sizeof(CubeGeom) == 72 and C.sizeof(Pointing) == 96
assert C.sizeof(ImageGeom) == 24
assert C.sizeof(Problem) == 160
assert C.sizeof(PlaneRules) == 48 and C.sizeof(TilingResult) == 72


class TomoError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status,
                                          message))
        self.status = status


_lib = None
_lib_lock = threading.Lock()

# name -> (restype, argtypes); the exported surface of include/tomo.h
_VP, _CP = C.c_void_p, C.c_char_p
_SIGNATURES = {
    "tomo_create": (C.c_int, [C.POINTER(_VP), C.c_int32]),
    "tomo_destroy": (None, [_VP]),
    "tomo_status_string": (_CP, [C.c_int]),
    "tomo_last_error": (_CP, [_VP]),
    "tomo_set_option": (C.c_int, [_VP, C.c_int32, C.c_int64]),
    "tomo_clear_cache": (C.c_int, [_VP]),
    "tomo_profile_read": (C.c_int, [_VP, C.POINTER(Profile), C.c_int32]),
    "tomo_project": (C.c_int, [_VP, C.POINTER(CubeGeom), C.c_int32, _VP,
                               C.c_int, C.POINTER(ImageGeom),
                               C.POINTER(Pointing), _VP, _VP, _VP, _VP]),
    "tomo_backproject": (C.c_int, [_VP, C.POINTER(CubeGeom), C.c_int32,
                                   C.POINTER(ImageGeom), C.POINTER(Pointing),
                                   _VP, _VP, _VP, _VP, C.c_uint32, _VP]),
    "tomo_solve": (C.c_int, [_VP, C.POINTER(CubeGeom), C.c_int32,
                             C.POINTER(ImageGeom),
                             C.POINTER(Pointing), _VP, _VP, _VP, _VP, _VP,
                             C.c_double, C.c_double,
                             C.c_int32, C.c_double, C.c_uint32,
                             C.POINTER(C.c_double), C.POINTER(C.c_int32),
                             _VP]),
    "tomo_prior_apply": (C.c_int, [_VP, C.POINTER(CubeGeom), _VP, _VP, _VP,
                                   C.c_double, C.c_uint32, _VP]),
    "tomo_count_segments": (C.c_int, [_VP, C.POINTER(CubeGeom),
                                      C.POINTER(ImageGeom),
                                      C.POINTER(Pointing), _VP,
                                      C.POINTER(C.c_int64), _VP]),
    "tomo_autotune": (C.c_int, [_VP, C.POINTER(Problem),
                                C.POINTER(TilingResult), _VP]),
    "tomo_set_plane_rules": (C.c_int, [_VP, C.POINTER(CubeGeom),
                                       C.POINTER(ImageGeom),
                                       C.POINTER(PlaneRules)]),
    "tomo_walk_plan": (C.c_int, [_VP, C.c_int32, C.POINTER(C.c_int32)]),
    "tomo_project_batched": (C.c_int, [_VP, C.c_int32, C.POINTER(Problem),
                                       _VP]),
    "tomo_backproject_batched": (C.c_int, [_VP, C.c_int32, C.POINTER(Problem),
                                           C.c_uint32, _VP]),
    "tomo_solve_batched": (C.c_int, [_VP, C.c_int32, C.POINTER(Problem),
                                     C.c_int32, C.c_uint32,
                                     C.POINTER(C.c_double),
                                     C.POINTER(C.c_int32), _VP]),
    "tomo_project_noalloc": (C.c_int, [C.POINTER(CubeGeom), C.c_int32, _VP,
                                       C.c_int, C.POINTER(ImageGeom),
                                       C.POINTER(Pointing), _VP, _VP, _VP]),
}


def exported_symbols():
    return list(_SIGNATURES)


def load_library(path=LIB_PATH):
    """Load libtomo.so (built by ``paper_1103_5904_gb300.build``)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                "libtomo.so not found at %s: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
        lib = C.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# ----------------------------------------------------------------- contexts

class Context:
    """One libtomo context (workspace + ray-record cache) on one device."""

    def __init__(self, device=None):
        lib = load_library()
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = _VP()
        st = lib.tomo_create(C.byref(h), self.device)
        if st != 0:
            raise TomoError(st, lib.tomo_status_string(st).decode())
        self.handle = h

    def check(self, st):
        if st != 0:
            lib = load_library()
            raise TomoError(st, lib.tomo_last_error(self.handle).decode())

    def set_option(self, option, value):
        self.check(load_library().tomo_set_option(self.handle, int(option),
                                                  int(value)))

    def set_tiling(self, tile_u, tile_v, warp_u):
        self.set_option(TOMO_OPT_WARP_U, warp_u)
        self.set_option(TOMO_OPT_TILE_U, tile_u)
        self.set_option(TOMO_OPT_TILE_V, tile_v)

    def clear_cache(self):
        self.check(load_library().tomo_clear_cache(self.handle))

    def profile(self, reset=False):
        """Launch counts and (with TOMO_OPT_PROFILE) summed device ms per
        kernel class: ``{"setup": (launches, ms), ...}``."""
        p = Profile()
        self.check(load_library().tomo_profile_read(self.handle, C.byref(p),
                                                    1 if reset else 0))
        return {k: (int(p.launches[i]), float(p.ms[i]))
                for i, k in enumerate(KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "handle", None):
            load_library().tomo_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = {}


def default_context(device=None):
    if device is None:
        device = torch.cuda.current_device()
    if device not in _default_ctx:
        _default_ctx[device] = Context(device)
    return _default_ctx[device]


# -------------------------------------------------------------- marshalling

def cube_geom_struct(geom):
    """``geom``: nx, ny, nz, x0, y0, z0, dx, dy, dz and optionally r_obs
    (radius of the opaque sphere at the origin; 0 or absent: none)."""
    return CubeGeom(int(geom["nx"]), int(geom["ny"]), int(geom["nz"]), 0,
                    float(geom["x0"]), float(geom["y0"]), float(geom["z0"]),
                    float(geom["dx"]), float(geom["dy"]), float(geom["dz"]),
                    float(geom.get("r_obs", 0.0)))


def pointing_array(pointing):
    a = np.ascontiguousarray(pointing, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 12:
        raise ValueError("pointing must be a (n_img, 12) float64 table")
    return a


def _ptg_ptr(a):
    return a.ctypes.data_as(C.POINTER(Pointing))


def _dev(t, dtype, name):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _check_mask(mask, n_img, nu, nv):
    _dev(mask, torch.uint8, "mask")
    if mask is not None and mask.numel() != n_img * nu * nv:
        raise ValueError("mask must have n_img * nv * nu = %d elements (got %d)"
                         % (n_img * nu * nv, mask.numel()))


def _check_map_mask(map_mask, geom):
    """Map mask: uint8 ``[nz][ny][nx]`` on the device, nonzero = voxel
    excluded from the map (one mask for every frame)."""
    _dev(map_mask, torch.uint8, "map_mask")
    nvox = int(geom["nx"]) * int(geom["ny"]) * int(geom["nz"])
    if map_mask is not None and map_mask.numel() != nvox:
        raise ValueError("map_mask must have nx * ny * nz = %d elements (got %d)"
                         % (nvox, map_mask.numel()))


def _check_weight(w, geom):
    """Prior weight: float32 ``[nz][ny][nx]`` on the device, the diagonal of
    R in the height-weighted prior ``lam ||D R x||^2``."""
    _dev(w, torch.float32, "prior_weight")
    nvox = int(geom["nx"]) * int(geom["ny"]) * int(geom["nz"])
    if w is not None and w.numel() != nvox:
        raise ValueError("prior_weight must have nx * ny * nz = %d elements "
                         "(got %d)" % (nvox, w.numel()))


def _stream_ptr(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return _VP(s.cuda_stream)


def _ptr(t):
    return None if t is None else _VP(t.data_ptr())


def _ctx(ctx):
    return ctx if ctx is not None else default_context()


# ------------------------------------------------------------- entry points

def tomo_project(cube, geom, pointing, nu, nv, mask=None, n_frames=1,
                 out=None, ctx=None, stream=None, map_mask=None,
                 kind="emission", limb_u=0.0):
    """``y = P x``: images ``[n_img][nv][nu]`` float32 from a float32 or
    bfloat16 cube ``[T][nz][ny][nx]``; with ``map_mask`` the excluded voxels
    are read as 0.  ``kind`` "pB" or "B" (white-light images, limb
    darkening ``limb_u``) applies the Thomson operator O P M or
    P M' - O P M instead of P; the transpose and the solver take the same
    keywords."""
    ctx = _ctx(ctx)
    ptg = pointing_array(pointing)
    n_img = ptg.shape[0]
    if cube.dtype == torch.float32:
        dtype = TOMO_F32
    elif cube.dtype == torch.bfloat16:
        dtype = TOMO_BF16
    else:
        raise TypeError("cube must be float32 or bfloat16")
    _dev(cube, cube.dtype, "cube")
    nvox = int(geom["nx"]) * int(geom["ny"]) * int(geom["nz"])
    if cube.numel() != nvox * int(n_frames):
        raise ValueError("cube has %d elements, geometry needs %d"
                         % (cube.numel(), nvox * int(n_frames)))
    if out is None:
        out = torch.empty((n_img, nv, nu), dtype=torch.float32,
                          device=cube.device)
    _dev(out, torch.float32, "out")
    if out.numel() != n_img * nu * nv:
        raise ValueError("out must have n_img * nv * nu elements")
    _check_mask(mask, n_img, nu, nv)
    _check_map_mask(map_mask, geom)
    cg = cube_geom_struct(geom)
    ig = ImageGeom(n_img, int(nu), int(nv), _kind(kind), float(limb_u))
    ctx.check(load_library().tomo_project(
        ctx.handle, C.byref(cg), int(n_frames), _ptr(cube), dtype,
        C.byref(ig), _ptg_ptr(ptg), _ptr(mask), _ptr(map_mask), _ptr(out),
        _stream_ptr(stream, cube.device)))
    return out


def tomo_backproject(images, geom, pointing, mask=None, n_frames=1, out=None,
                     accumulate=False, ctx=None, stream=None, map_mask=None,
                     kind="emission", limb_u=0.0):
    """``x = P^T y``: float32 cube ``[T][nz][ny][nx]`` from float32 images
    ``[n_img][nv][nu]``; with ``map_mask`` the excluded voxels receive 0."""
    ctx = _ctx(ctx)
    ptg = pointing_array(pointing)
    _dev(images, torch.float32, "images")
    n_img, nv, nu = images.shape
    if n_img != ptg.shape[0]:
        raise ValueError("one pointing record per image")
    shape = (int(geom["nz"]), int(geom["ny"]), int(geom["nx"]))
    if n_frames > 1:
        shape = (int(n_frames),) + shape
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=images.device)
        accumulate = False
    _dev(out, torch.float32, "out")
    if out.numel() != int(np.prod(shape)):
        raise ValueError("out has the wrong size")
    _check_mask(mask, n_img, nu, nv)
    _check_map_mask(map_mask, geom)
    cg = cube_geom_struct(geom)
    ig = ImageGeom(n_img, nu, nv, _kind(kind), float(limb_u))
    ctx.check(load_library().tomo_backproject(
        ctx.handle, C.byref(cg), int(n_frames), C.byref(ig), _ptg_ptr(ptg),
        _ptr(mask), _ptr(map_mask), _ptr(images), _ptr(out),
        TOMO_ACCUMULATE if accumulate else 0,
        _stream_ptr(stream, images.device)))
    return out


def tomo_solve(y, geom, pointing, mask=None, lam=0.0, max_iter=10, tol=0.0,
               x0=None, bf16=False, out=None, report=True, ctx=None,
               stream=None, map_mask=None, prior_weight=None,
               kind="emission", limb_u=0.0, n_frames=1, lam_t=0.0):
    """CG on ``(P^T M P + lam R D^T D R) x = P^T M y`` (R = diag of
    ``prior_weight``, else the identity; restricted to the voxels that
    ``map_mask`` keeps).  With ``n_frames`` T > 1 the map is
    ``[T][nz][ny][nx]`` (images reach frames through their time stamps) and
    ``lam_t`` weighs the temporal prior ``||D_t x||^2``.  Returns
    ``(x, info)`` with ``info = {"J": ..., "rr": ..., "iters": ...}`` when
    ``report``."""
    ctx = _ctx(ctx)
    ptg = pointing_array(pointing)
    _dev(y, torch.float32, "y")
    n_img, nv, nu = y.shape
    shape = (int(geom["nz"]), int(geom["ny"]), int(geom["nx"]))
    if int(n_frames) > 1:
        shape = (int(n_frames),) + shape
    flags = 0
    if n_img != ptg.shape[0]:
        raise ValueError("one pointing record per image")
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=y.device)
    _dev(out, torch.float32, "out")
    if out.numel() != int(np.prod(shape)):
        raise ValueError("out has the wrong size")
    if x0 is not None:
        out.copy_(x0.reshape(shape))
        flags |= TOMO_SOLVE_X0
    if bf16:
        flags |= TOMO_SOLVE_BF16
    _check_mask(mask, n_img, nu, nv)
    _check_map_mask(map_mask, geom)
    _check_weight(prior_weight, geom)
    cg = cube_geom_struct(geom)
    ig = ImageGeom(n_img, nu, nv, _kind(kind), float(limb_u))
    rep = np.full(2 * (int(max_iter) + 1), np.nan) if report else None
    iters = C.c_int32(0)
    ctx.check(load_library().tomo_solve(
        ctx.handle, C.byref(cg), int(n_frames), C.byref(ig), _ptg_ptr(ptg),
        _ptr(mask), _ptr(map_mask), _ptr(prior_weight), _ptr(y), _ptr(out),
        float(lam), float(lam_t), int(max_iter), float(tol), flags,
        rep.ctypes.data_as(C.POINTER(C.c_double)) if report else None,
        C.byref(iters) if report else None, _stream_ptr(stream, y.device)))
    info = None
    if report:
        r = rep.reshape(-1, 2)
        info = {"J": r[:, 0].copy(), "rr": r[:, 1].copy(),
                "iters": int(iters.value)}
    return out, info


def tomo_prior_apply(x, geom, lam, out=None, accumulate=False, ctx=None,
                     stream=None, prior_weight=None):
    """``q = lam D^T D x``, or ``lam R D^T D R x`` with ``prior_weight``
    (the diagonal of R), + q with ``accumulate``."""
    ctx = _ctx(ctx)
    _dev(x, torch.float32, "x")
    if out is None:
        out = torch.empty_like(x)
        accumulate = False
    _dev(out, torch.float32, "out")
    nvox = int(geom["nx"]) * int(geom["ny"]) * int(geom["nz"])
    if x.numel() != nvox or out.numel() != nvox:
        raise ValueError("x and out must have nx * ny * nz elements")
    _check_weight(prior_weight, geom)
    cg = cube_geom_struct(geom)
    ctx.check(load_library().tomo_prior_apply(
        ctx.handle, C.byref(cg), _ptr(x), _ptr(prior_weight), _ptr(out),
        float(lam),
        TOMO_ACCUMULATE if accumulate else 0, _stream_ptr(stream, x.device)))
    return out


def tomo_count_segments(geom, pointing, nu, nv, mask=None, ctx=None,
                        stream=None, device=None):
    """Number of positive-length Siddon segments of the unmasked rays."""
    ctx = _ctx(ctx)
    ptg = pointing_array(pointing)
    _check_mask(mask, ptg.shape[0], int(nu), int(nv))
    cg, ig = cube_geom_struct(geom), ImageGeom(ptg.shape[0], int(nu), int(nv))
    n = C.c_int64(0)
    dev = torch.device("cuda", ctx.device)
    ctx.check(load_library().tomo_count_segments(
        ctx.handle, C.byref(cg), C.byref(ig), _ptg_ptr(ptg), _ptr(mask),
        C.byref(n), _stream_ptr(stream, dev)))
    return int(n.value)


# ------------------------------------------------------------------ batches

def _problems(problems, need_cube=True, need_images=True):
    """ctypes array of tomo_problem from dicts with keys geom, pointing, nu,
    nv, cube, images, mask, map_mask, prior_weight, lam (the last four
    optional).  Returns the array and
    the pointing arrays it points into (keep them alive)."""
    arr = (Problem * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        ptg = pointing_array(p["pointing"])
        keep.append(ptg)
        nu, nv = int(p["nu"]), int(p["nv"])
        n_img = ptg.shape[0]
        cube, images, mask = p.get("cube"), p.get("images"), p.get("mask")
        _dev(cube, torch.float32, "cube")
        _dev(images, torch.float32, "images")
        _check_mask(mask, n_img, nu, nv)
        map_mask = p.get("map_mask")
        _check_map_mask(map_mask, p["geom"])
        weight = p.get("prior_weight")
        _check_weight(weight, p["geom"])
        nvox = int(p["geom"]["nx"]) * int(p["geom"]["ny"]) * int(p["geom"]["nz"])
        if need_cube and (cube is None or cube.numel() != nvox):
            raise ValueError("problem %d: cube must have nx*ny*nz elements" % i)
        if need_images and (images is None or images.numel() != n_img * nu * nv):
            raise ValueError("problem %d: images must have n_img*nv*nu elements"
                             % i)
        arr[i].cube = cube_geom_struct(p["geom"])
        arr[i].img = ImageGeom(n_img, nu, nv, _kind(p.get("kind", "emission")),
                               float(p.get("limb_u", 0.0)))
        arr[i].reserved = 0
        arr[i].pointing_host = _ptg_ptr(ptg)
        arr[i].mask_dev = None if mask is None else mask.data_ptr()
        arr[i].images_dev = None if images is None else images.data_ptr()
        arr[i].cube_dev = None if cube is None else cube.data_ptr()
        arr[i].lam = float(p.get("lam", 0.0))
        arr[i].map_mask_dev = None if map_mask is None else map_mask.data_ptr()
        arr[i].prior_weight_dev = None if weight is None else weight.data_ptr()
    return arr, keep


def _batch_device(problems):
    for p in problems:
        for k in ("cube", "images"):
            if p.get(k) is not None:
                return p[k].device
    return torch.device("cuda", torch.cuda.current_device())


def tomo_project_batched(problems, ctx=None, stream=None):
    """``images = P cube`` for every problem (one persistent launch)."""
    ctx = _ctx(ctx)
    arr, keep = _problems(problems)
    ctx.check(load_library().tomo_project_batched(
        ctx.handle, len(problems), arr, _stream_ptr(stream,
                                                    _batch_device(problems))))
    return [p["images"] for p in problems]


def tomo_backproject_batched(problems, accumulate=False, ctx=None,
                             stream=None):
    """``cube = P^T images`` for every problem (one persistent launch)."""
    ctx = _ctx(ctx)
    arr, keep = _problems(problems)
    ctx.check(load_library().tomo_backproject_batched(
        ctx.handle, len(problems), arr, TOMO_ACCUMULATE if accumulate else 0,
        _stream_ptr(stream, _batch_device(problems))))
    return [p["cube"] for p in problems]


def tomo_solve_batched(problems, n_iter, warm_start=False, autotune=False,
                       report=True, ctx=None, stream=None):
    """``n_iter`` CG iterations for every problem (one CUDA graph replay);
    ``problems[i]["images"]`` is the data, ``problems[i]["cube"]`` receives
    the solution.  Returns one info dict per problem when ``report``."""
    ctx = _ctx(ctx)
    arr, keep = _problems(problems)
    n = len(problems)
    flags = (TOMO_SOLVE_X0 if warm_start else 0) | \
        (TOMO_BATCH_AUTOTUNE if autotune else 0)
    rep = np.full(n * 2 * (int(n_iter) + 1), np.nan) if report else None
    iters = (C.c_int32 * max(n, 1))()
    ctx.check(load_library().tomo_solve_batched(
        ctx.handle, n, arr, int(n_iter), flags,
        rep.ctypes.data_as(C.POINTER(C.c_double)) if report else None,
        iters if report else None,
        _stream_ptr(stream, _batch_device(problems))))
    if not report:
        return None
    r = rep.reshape(n, -1, 2)
    return [{"J": r[i, :, 0].copy(), "rr": r[i, :, 1].copy(),
             "iters": int(iters[i])} for i in range(n)]


def tomo_autotune(cube, images, geom, pointing, mask=None, ctx=None,
                  stream=None):
    """Pick the fastest tile shape for this problem size (kept in the
    context); returns it with the measured forward / transpose times."""
    ctx = _ctx(ctx)
    ptg = pointing_array(pointing)
    n_img, nv, nu = images.shape
    arr, keep = _problems([{"geom": geom, "pointing": ptg, "nu": nu, "nv": nv,
                            "cube": cube, "images": images, "mask": mask}])
    best = TilingResult()
    ctx.check(load_library().tomo_autotune(ctx.handle, arr, C.byref(best),
                                           _stream_ptr(stream, cube.device)))
    return {"tile_u": best.tile_u, "tile_v": best.tile_v,
            "warp_u": best.warp_u, "fwd_ms": best.fwd_ms,
            "adj_ms": best.adj_ms,
            "rules": {f: getattr(best.rules, f) for f in RULE_FIELDS}}


def tomo_set_plane_rules(rules=None, geom=None, nu=None, nv=None,
                         n_img=1, ctx=None):
    """Walk rules (dict with the keys of ``RULE_FIELDS``; missing keys take
    the built-in defaults, ``None`` all of them) for the size bucket of
    ``geom`` and ``nu`` x ``nv`` images, or the context's default when
    ``geom`` is None."""
    ctx = _ctx(ctx)
    r = None
    if rules is not None:
        d = {"min_pitch": 0.16, "fwd_min_pitch": 0.75, "fwd_max_ratio": 0.02,
             "general_ratio": 0.035, "fwd_group": 0.0, "adj_group": 0.0}
        unknown = set(rules) - set(RULE_FIELDS)
        if unknown:
            raise ValueError("unknown rule(s) %s" % sorted(unknown))
        d.update(rules)
        r = PlaneRules(*[float(d[f]) for f in RULE_FIELDS])
    cg = ig = None
    if geom is not None:
        cg = C.byref(cube_geom_struct(geom))
        ig = C.byref(ImageGeom(int(n_img), int(nu), int(nv)))
    ctx.check(load_library().tomo_set_plane_rules(
        ctx.handle, cg, ig, None if r is None else C.byref(r)))


def tomo_walk_plan(n_img, ctx=None):
    """Per image of the context's most recent geometry: the walk code of
    ``tomo_walk_plan`` (bit 0 plane-synchronous P^T, bit 1 plane P, bit 2
    every-slab body, bits 3-4 major axis, bits 5-6 lateral axis)."""
    ctx = _ctx(ctx)
    out = np.zeros(int(n_img), dtype=np.int32)
    ctx.check(load_library().tomo_walk_plan(
        ctx.handle, int(n_img), out.ctypes.data_as(C.POINTER(C.c_int32))))
    return out


# short aliases
project = tomo_project
backproject = tomo_backproject
solve = tomo_solve
prior_apply = tomo_prior_apply
count_segments = tomo_count_segments
