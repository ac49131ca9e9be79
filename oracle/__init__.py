"""CPU oracle for X-Gaussian's Differentiable Radiative Rasterization (arXiv 2403.04116).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  The product library never does, and this
package never touches the CUDA library.

Two C sources, built here with gcc (OpenMP, ``-ffp-contract=off``):

* ``xg_oracle64.c`` -- the FP64 oracle: per pixel, every Gaussian projected (Eq. 7-9,
  camera of Eq. 12), included ones depth-ordered and blended (Eq. 10); gradients by the
  per-pixel reverse recursion and the analytic chain rule.
* ``xg_replica32.c`` -- the FP32 replica of the index work and per-pixel decisions,
  which the GPU must match bit for bit.
* ``train64.py`` -- FP64 NumPy/SciPy versions of the rest of a training step: the
  activations and RIRF (Eq. 3), the (1 - gamma) L1 + gamma (1 - SSIM) objective (Eq. 11)
  with its gradient, Adam, PSNR.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["xg_oracle64.c", "xg_replica32.c"]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

NEAR_MM = 0.2


class _View(ctypes.Structure):
    _fields_ = [("sod", ctypes.c_double), ("sdd", ctypes.c_double), ("pitch_u", ctypes.c_double),
                ("pitch_v", ctypes.c_double), ("angle", ctypes.c_double), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (skipped when up to date)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        t_lib = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t_lib for s in srcs):
            return _LIB_PATH
    os.makedirs(_BUILD_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           *srcs, "-lm", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            L.xo_render.argtypes = [i64, P, P, P, P, P, ctypes.POINTER(_View), ctypes.c_double, P, i64, P, P, P, P,
                                    ctypes.c_int]
            L.xo_render.restype = ctypes.c_int
            L.xo_render_grad.argtypes = [i64, P, P, P, P, P, ctypes.POINTER(_View), ctypes.c_double, P, i64, P,
                                         P, P, P, P, P, P, P, P, ctypes.c_int]
            L.xo_render_grad.restype = ctypes.c_int
            L.xo_project.argtypes = [i64, P, P, P, P, P, ctypes.POINTER(_View), ctypes.c_double, P]
            L.xo_project.restype = None
            L.xr_project.argtypes = [i64, P, P, P, P, P, ctypes.POINTER(_View), ctypes.c_float, ctypes.c_int,
                                     ctypes.c_int, P, P, P, P]
            L.xr_project.restype = i64
            L.xr_bin.argtypes = [i64, P, P, P, ctypes.c_int, ctypes.c_int, P, P]
            L.xr_bin.restype = i64
            L.xr_render.argtypes = [P, P, P, ctypes.POINTER(_View), ctypes.c_int, ctypes.c_int, P, P, P, P]
            L.xr_render.restype = None
            L.xr_exp_batch.argtypes = [P, P, i64]
            L.xr_log_batch.argtypes = [P, P, i64]
            _lib = L
    return _lib


def _cview(v) -> _View:
    return _View(float(v.sod_mm), float(v.sdd_mm), float(v.pitch_u_mm), float(v.pitch_v_mm), float(v.angle_rad),
                 int(v.width), int(v.height))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _soa(g: dict, dtype) -> tuple:
    keys = ("mean", "scale", "quat", "opacity", "intensity")
    arrs = tuple(np.ascontiguousarray(g[k], dtype=dtype) for k in keys)
    n = arrs[4].shape[0]
    assert arrs[0].shape == (3, n) and arrs[1].shape == (3, n) and arrs[2].shape == (4, n) and arrs[3].shape == (n,)
    return n, arrs


def _pixels(pixels, view):
    if pixels is None:
        return None, 0
    p = np.ascontiguousarray(pixels, dtype=np.int32)
    assert p.ndim == 1 and (p.size == 0 or (p.min() >= 0 and p.max() < view.width * view.height))
    return p, p.size


# ---------------------------------------------------------------------------------------------
# FP64 oracle
# ---------------------------------------------------------------------------------------------

def render64(g: dict, view, near_mm: float = NEAR_MM, pixels=None, threads: int = 0) -> dict:
    """FP64 image of one view (Eq. 10).  Arrays are (H, W); pixels not evaluated are NaN / -1."""
    n, (mean, scale, quat, opac, inten) = _soa(g, np.float64)
    H, W = view.height, view.width
    image = np.full(H * W, np.nan)
    tfin = np.full(H * W, np.nan)
    ncon = np.full(H * W, -1, dtype=np.int32)
    amb = np.zeros(H * W, dtype=np.uint8)
    pix, npix = _pixels(pixels, view)
    cv = _cview(view)
    rc = lib().xo_render(n, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(opac), _ptr(inten), ctypes.byref(cv),
                         near_mm, _ptr(pix) if pix is not None else None, npix, _ptr(image), _ptr(tfin), _ptr(ncon),
                         _ptr(amb), threads)
    if rc:
        raise MemoryError("oracle render ran out of memory")
    return {"image": image.reshape(H, W), "tfinal": tfin.reshape(H, W), "ncontrib": ncon.reshape(H, W),
            "ambiguous": amb.reshape(H, W)}


def grad64(g: dict, view, dL_dimage: np.ndarray, near_mm: float = NEAR_MM, pixels=None, threads: int = 0,
           out: dict | None = None) -> dict:
    """FP64 gradient of sum_p dL_dimage[p] * I(p) for one view, added into ``out`` if given.

    Returns mean (3, n), scale (3, n), quat (4, n), opacity (n,), intensity (n,) and g2d
    (7, n): this view's dL/du_x, dL/du_y, dL/da, dL/db, dL/dc, dL/do, dL/di.  For judging
    floating-point error it also returns mag2d (7, n), the sums of |per-pixel term| behind
    g2d, and ``mag`` (same keys as the gradients, accumulated like them): how much term
    magnitude reaches each parameter gradient through the linear backward map.
    """
    n, (mean, scale, quat, opac, inten) = _soa(g, np.float64)
    if out is None:
        out = {"mean": np.zeros((3, n)), "scale": np.zeros((3, n)), "quat": np.zeros((4, n)),
               "opacity": np.zeros(n), "intensity": np.zeros(n), "mag_all": np.zeros((12, n))}
    g2d = np.zeros((7, n))
    mag2d = np.zeros((7, n))
    dimg = np.ascontiguousarray(dL_dimage, dtype=np.float64).reshape(-1)
    assert dimg.size == view.width * view.height
    pix, npix = _pixels(pixels, view)
    cv = _cview(view)
    rc = lib().xo_render_grad(n, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(opac), _ptr(inten), ctypes.byref(cv),
                              near_mm, _ptr(pix) if pix is not None else None, npix, _ptr(dimg), _ptr(out["mean"]),
                              _ptr(out["scale"]), _ptr(out["quat"]), _ptr(out["opacity"]), _ptr(out["intensity"]),
                              _ptr(g2d), _ptr(mag2d), _ptr(out["mag_all"]), threads)
    if rc:
        raise MemoryError("oracle gradient ran out of memory")
    out["g2d"] = g2d
    out["mag2d"] = mag2d
    m = out["mag_all"]
    out["mag"] = {"mean": m[0:3], "scale": m[3:6], "quat": m[6:10], "opacity": m[10], "intensity": m[11]}
    return out


def project64(g: dict, view, near_mm: float = NEAR_MM) -> np.ndarray:
    """(n, 12): ok, t (3), u (2, detector corner origin), Sigma'' (A, B, C), conic (a, b, c)."""
    n, (mean, scale, quat, opac, inten) = _soa(g, np.float64)
    out = np.zeros((n, 12))
    cv = _cview(view)
    lib().xo_project(n, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(opac), _ptr(inten), ctypes.byref(cv), near_mm,
                     _ptr(out))
    return out


# ---------------------------------------------------------------------------------------------
# FP32 replica of the index work
# ---------------------------------------------------------------------------------------------

def replica_project(g: dict, view, tile=(16, 16), near_mm: float = NEAR_MM) -> dict:
    n, (mean, scale, quat, opac, inten) = _soa(g, np.float32)
    rec = np.zeros((n, 8), np.float32)
    depth = np.zeros(n, np.float32)
    rect = np.zeros((n, 4), np.int32)
    count = np.zeros(n, np.uint32)
    cv = _cview(view)
    nonfinite = lib().xr_project(n, _ptr(mean), _ptr(scale), _ptr(quat), _ptr(opac), _ptr(inten), ctypes.byref(cv),
                                 np.float32(near_mm), tile[0], tile[1], _ptr(rec), _ptr(depth), _ptr(rect),
                                 _ptr(count))
    return {"rec": rec, "depth": depth, "rect": rect, "count": count, "nonfinite": int(nonfinite)}


def tiles_of(view, tile=(16, 16)) -> tuple[int, int]:
    return (view.width + tile[0] - 1) // tile[0], (view.height + tile[1] - 1) // tile[1]


def replica_bin(proj: dict, view, tile=(16, 16)) -> dict:
    tx, ty = tiles_of(view, tile)
    depth, rect, count = proj["depth"], proj["rect"], proj["count"]
    n = depth.shape[0]
    M = int(count.astype(np.int64).sum())
    rng = np.zeros((tx * ty, 2), np.uint32)
    lst = np.zeros(max(M, 1), np.int32)
    m = lib().xr_bin(n, _ptr(depth), _ptr(rect), _ptr(count), tx, ty, _ptr(rng), _ptr(lst))
    if m < 0:
        raise MemoryError("replica binning ran out of memory")
    assert m == M
    return {"range": rng, "list": lst[:M], "M": M}


def replica_render(proj: dict, binned: dict, view, tile=(16, 16)) -> dict:
    H, W = view.height, view.width
    image = np.zeros(H * W, np.float32)
    tfin = np.zeros(H * W, np.float32)
    ncon = np.zeros(H * W, np.uint32)
    last = np.zeros(H * W, np.uint32)
    cv = _cview(view)
    lst = binned["list"] if binned["M"] > 0 else np.zeros(1, np.int32)
    lib().xr_render(_ptr(proj["rec"]), _ptr(binned["range"]), _ptr(lst), ctypes.byref(cv), tile[0], tile[1],
                    _ptr(image), _ptr(tfin), _ptr(ncon), _ptr(last))
    return {"image": image.reshape(H, W), "tfinal": tfin.reshape(H, W), "ncontrib": ncon.reshape(H, W),
            "last": last.reshape(H, W)}


def replica_full(g: dict, view, tile=(16, 16), near_mm: float = NEAR_MM) -> dict:
    """project + bin + render of one view with the FP32 replica."""
    p = replica_project(g, view, tile, near_mm)
    b = replica_bin(p, view, tile)
    r = replica_render(p, b, view, tile)
    return {**p, **b, **r}


def replica_exp(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(x)
    lib().xr_exp_batch(_ptr(x), _ptr(y), x.size)
    return y


def replica_log(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(x)
    lib().xr_log_batch(_ptr(x), _ptr(y), x.size)
    return y
