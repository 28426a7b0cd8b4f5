"""ctypes front end of the FP64 reference renderer in ``pbr_oracle.c``.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
CPU-baseline leg of the benchmark are the only callers.  Nothing here imports
the CUDA package, and the CUDA package never imports this module.

Every array crossing into C is widened to float64; discrete decisions inside
the library are taken on the fp32-rounded inputs (Sec. 3.2 renders from fp32
point parameters), continuous quantities in double.

Parity status (every function is pinned by ``tests/test_oracle_*.py``):
  sh_basis ............ pinned: Gram matrix by quadrature, addition theorem,
                        printed textbook values, parity under v -> -v
  project ............. pinned: on-axis point lands on the principal point,
                        closed-form pinhole on random points
  bin_tiles ........... pinned: a (tile, 8 x 8 block) is listed exactly when
                        some pixel in it passes the cutoff test (brute force
                        over every pixel of the image, both directions)
  render .............. pinned: isolated splat in closed form, transmittance
                        identity, occlusion, permutation invariance
  backward ............ pinned: central finite differences of ``render``
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Camera(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("R", C.c_double * 9), ("t", C.c_double * 3),
                ("width", C.c_int32), ("height", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("radius_mode", C.c_int32), ("dir_frame", C.c_int32),
                ("cutoff_k", C.c_double), ("alpha_max", C.c_double), ("t_eps", C.c_double),
                ("max_per_pixel", C.c_int32), ("bg", C.c_double * 3), ("z_near", C.c_double),
                ("tile_w", C.c_int32), ("tile_h", C.c_int32), ("screen_fp32", C.c_int32)]


class Rec(C.Structure):
    _fields_ = [("visible", C.c_int32),
                ("z32", C.c_float), ("px32", C.c_float), ("py32", C.c_float), ("s32", C.c_float),
                ("rc32", C.c_float), ("rc2_32", C.c_float),
                ("px_lo", C.c_int32), ("px_hi", C.c_int32), ("py_lo", C.c_int32), ("py_hi", C.c_int32),
                ("tx_lo", C.c_int32), ("tx_hi", C.c_int32), ("ty_lo", C.c_int32), ("ty_hi", C.c_int32),
                ("ntiles", C.c_int64),
                ("X", C.c_double * 3), ("px", C.c_double), ("py", C.c_double), ("s", C.c_double),
                ("dir", C.c_double * 3), ("rgb", C.c_double * 3)]


DEFAULT_OPTS = dict(radius_mode=0, dir_frame=0, cutoff_k=3.0, alpha_max=0.99, t_eps=1e-5,
                    max_per_pixel=0, bg=(0.0, 0.0, 0.0), z_near=0.01, tile_w=16, tile_h=16,
                    screen_fp32=1)


def build(force: bool = False) -> str:
    """Compile ``pbr_oracle.c`` into ``_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.orc_sh_eval.argtypes = [C.c_int, dp, dp, dp]
            L.orc_preprocess.argtypes = [C.c_int64, dp, dp, dp, C.c_int, C.c_int,
                                         C.POINTER(Camera), C.POINTER(Opts), C.POINTER(Rec)]
            L.orc_bin.argtypes = [C.c_int64, C.c_int, C.POINTER(Camera), C.POINTER(Opts),
                                  C.POINTER(Rec), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                  C.c_void_p]
            L.orc_bin.restype = C.c_int64
            L.orc_render.argtypes = [C.c_int64, dp, dp, dp, dp, C.c_int, C.c_int, C.POINTER(Camera),
                                     C.POINTER(Opts), C.c_int64, C.c_void_p, dp, dp, C.c_void_p]
            L.orc_backward.argtypes = [C.c_int64, dp, dp, dp, dp, C.c_int, C.c_int,
                                       C.POINTER(Camera), C.POINTER(Opts), C.c_int64, C.c_void_p,
                                       dp, dp, dp, dp, C.c_void_p]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's later parallel regions (timing only)."""
    lib().orc_set_num_threads(int(n))


# ---------------------------------------------------------------- marshalling
def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_cameras(cams):
    """cams: list of dicts with fx, fy, cx, cy, R (3x3), t (3), width, height."""
    arr = (Camera * max(1, len(cams)))()
    for i, c in enumerate(cams):
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = (float(c["fx"]), float(c["fy"]),
                                                      float(c["cx"]), float(c["cy"]))
        R = np.asarray(c["R"], dtype=np.float64).reshape(9)
        t = np.asarray(c["t"], dtype=np.float64).reshape(3)
        for j in range(9):
            arr[i].R[j] = R[j]
        for j in range(3):
            arr[i].t[j] = t[j]
        arr[i].width, arr[i].height = int(c["width"]), int(c["height"])
    return arr


def make_opts(**kw):
    d = dict(DEFAULT_OPTS)
    d.update(kw)
    o = Opts()
    o.radius_mode, o.dir_frame = int(d["radius_mode"]), int(d["dir_frame"])
    o.cutoff_k, o.alpha_max, o.t_eps = float(d["cutoff_k"]), float(d["alpha_max"]), float(d["t_eps"])
    o.max_per_pixel = int(d["max_per_pixel"])
    for j in range(3):
        o.bg[j] = float(d["bg"][j])
    o.z_near = float(d["z_near"])
    o.tile_w, o.tile_h = int(d["tile_w"]), int(d["tile_h"])
    o.screen_fp32 = int(d["screen_fp32"])
    return o


def sh_basis(deg: int, dirs, grad: bool = False):
    """Real SH basis Y[k] (k = l*l+l+m) at unit directions ``dirs`` [M,3]."""
    dirs = _d(np.atleast_2d(dirs))
    K = (deg + 1) ** 2
    Y = np.zeros((dirs.shape[0], K))
    dY = np.zeros((dirs.shape[0], K, 3))
    L = lib()
    for i in range(dirs.shape[0]):
        y = np.zeros(K)
        dy = np.zeros(K * 3)
        rc = L.orc_sh_eval(deg, _dp(dirs[i]), _dp(y), _dp(dy) if grad else None)
        if rc != 0:
            raise ValueError("orc_sh_eval failed")
        Y[i] = y
        dY[i] = dy.reshape(K, 3)
    return (Y, dY) if grad else Y


def preprocess(pos, sh, radius, deg, cams, **opts):
    """Per (view, point) records as a numpy structured array [V, N]."""
    pos, sh, radius = _d(pos), _d(sh), _d(radius)
    n = pos.shape[0]
    cam_arr = make_cameras(cams)
    o = make_opts(**opts)
    out = (Rec * max(1, len(cams) * n))()
    rc = lib().orc_preprocess(n, _dp(pos), _dp(sh), _dp(radius), deg, len(cams), cam_arr,
                              C.byref(o), out)
    if rc != 0:
        raise ValueError("orc_preprocess failed")
    recs = np.ctypeslib.as_array(out)[: len(cams) * n].copy()
    return recs.reshape(len(cams), n), (cam_arr, o)


def bin_tiles(pos, sh, radius, deg, cams, **opts):
    """Sorted (tile, pv) lists, the pairs' 8 x 8 block masks and per-tile
    [start, end) ranges (Sec. 3.2 cutoff and sort).  A tile lists a
    point-view iff some pixel of the tile passes the cutoff test; bit
    by * (tile_w / 8) + bx of the mask is set iff some pixel of the tile's
    8 x 8 block (bx, by) does.  Returns keys, vals, masks, ranges, recs."""
    recs, (cam_arr, o) = preprocess(pos, sh, radius, deg, cams, **opts)
    n = np.asarray(pos).shape[0]
    flat = np.ascontiguousarray(recs.reshape(-1))
    rp = flat.ctypes.data_as(C.POINTER(Rec))
    L = lib()
    total = L.orc_bin(n, len(cams), cam_arr, C.byref(o), rp, None, None, None, 0, None)
    n_tiles = 0
    for c in cams:
        n_tiles += -(-int(c["width"]) // o.tile_w) * -(-int(c["height"]) // o.tile_h)
    keys = np.zeros(max(total, 1), np.uint32)
    vals = np.zeros(max(total, 1), np.uint32)
    masks = np.zeros(max(total, 1), np.uint8)
    ranges = np.zeros(2 * max(n_tiles, 1), np.uint32)
    got = L.orc_bin(n, len(cams), cam_arr, C.byref(o), rp, keys.ctypes.data, vals.ctypes.data,
                    masks.ctypes.data, total, ranges.ctypes.data)
    if got != total:
        raise RuntimeError("orc_bin failed")
    return (keys[:total], vals[:total], masks[:total], ranges[: 2 * n_tiles].reshape(n_tiles, 2),
            recs)


def _pix(pix):
    if pix is None:
        return None, 0
    p = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 3)
    return p, p.shape[0]


def render(pos, sh, opacity, radius, deg, cams, pix=None, **opts):
    """Image(s) by brute force.  Returns rgb [P,3], T_final [P], count [P]
    where P is every pixel of every view (view-major, row-major) when ``pix``
    is None, else the selected (view, x, y) triples in order."""
    pos, sh, opacity, radius = _d(pos), _d(sh), _d(opacity), _d(radius)
    n = pos.shape[0]
    cam_arr = make_cameras(cams)
    o = make_opts(**opts)
    p, npix = _pix(pix)
    total = npix if p is not None else sum(int(c["width"]) * int(c["height"]) for c in cams)
    rgb = np.zeros((max(total, 1), 3))
    T = np.zeros(max(total, 1))
    cnt = np.zeros(max(total, 1), np.int32)
    rc = lib().orc_render(n, _dp(pos), _dp(sh), _dp(opacity), _dp(radius), deg, len(cams),
                          cam_arr, C.byref(o), npix, p.ctypes.data if p is not None else None,
                          _dp(rgb), _dp(T), cnt.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"orc_render failed ({rc})")
    return rgb[:total], T[:total], cnt[:total]


def backward(pos, sh, opacity, radius, deg, cams, grad_rgb, pix=None, want_g2d=False, **opts):
    """Adjoint of ``render`` for L = sum(grad_rgb * image) over the selected
    pixels.  Returns dpos [N,3], dsh [N,K,3], dopacity [N] (and the
    per-(view,point) screen adjoint [V,N,7] when ``want_g2d``)."""
    pos, sh, opacity, radius = _d(pos), _d(sh), _d(opacity), _d(radius)
    n = pos.shape[0]
    K = (deg + 1) ** 2
    cam_arr = make_cameras(cams)
    o = make_opts(**opts)
    p, npix = _pix(pix)
    g = _d(grad_rgb).reshape(-1, 3)
    dpos = np.zeros((max(n, 1), 3))
    dsh = np.zeros((max(n, 1), K, 3))
    dop = np.zeros(max(n, 1))
    g2d = np.zeros((max(len(cams) * n, 1), 7)) if want_g2d else None
    rc = lib().orc_backward(n, _dp(pos), _dp(sh.reshape(-1)), _dp(opacity), _dp(radius), deg,
                            len(cams), cam_arr, C.byref(o), npix,
                            p.ctypes.data if p is not None else None, _dp(g), _dp(dpos), _dp(dsh),
                            _dp(dop), g2d.ctypes.data if want_g2d else None)
    if rc != 0:
        raise RuntimeError(f"orc_backward failed ({rc})")
    out = (dpos[:n], dsh[:n], dop[:n])
    if want_g2d:
        out = out + (g2d[: len(cams) * n].reshape(len(cams), n, 7),)
    return out
