"""FP64 oracle for the convolution and Jacobi loop nests (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package; the library under
``paper_1302_5586_gb300/`` never does, and this package imports nothing from
it.  The arithmetic lives in ``oracle.c`` (plain C, FP64); this file builds it
with gcc and marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_SRC, when set, names another copy of oracle.c to build (into a _build
# folder beside it) and load instead: the mutation tests plant one mistake in
# such a copy and check that the pin tests catch it.
_SRC = os.path.abspath(os.environ.get("ORACLE_SRC") or os.path.join(_HERE, "oracle.c"))
_BUILD = os.path.join(os.path.dirname(_SRC), "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

DT_F32 = 0
DT_F16 = 1

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so beside it (OpenMP when available).

    FP contraction is switched off so that every multiply and add rounds as
    written, on x86-64 and aarch64 alike.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = ctypes.CDLL(_LIB_PATH)
    i64, i32, vp, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p
    L.oracle_version.restype = i32
    L.oracle_num_threads.restype = i32
    L.oracle_set_num_threads.argtypes = [i32]
    L.oracle_f16_to_f64.argtypes = [ctypes.c_uint16]
    L.oracle_f16_to_f64.restype = ctypes.c_double
    L.oracle_f64_to_f16.argtypes = [ctypes.c_double]
    L.oracle_f64_to_f16.restype = ctypes.c_uint16
    L.oracle_f16_to_f64_array.argtypes = [i64, vp, vp]
    L.oracle_f64_to_f16_array.argtypes = [i64, vp, vp]
    L.oracle_conv2d.argtypes = [i64, i64, i64, vp, i32, i32, i32, vp, dp, dp]
    L.oracle_conv2d.restype = i32
    L.oracle_conv2d_mode.argtypes = [i64, i64, i64, vp, i32, i32, i32, vp, dp, dp, i32]
    L.oracle_conv2d_mode.restype = i32
    L.oracle_conv2d_sep.argtypes = [i64, i64, i64, vp, i32, i32, vp, i32, vp, dp, dp]
    L.oracle_conv2d_sep.restype = i32
    L.oracle_conv2d_points.argtypes = [i64, i64, i64, vp, i32, i32, i32, vp, i64, vp, dp, dp]
    L.oracle_conv2d_points.restype = i32
    L.oracle_conv2d_sep_points.argtypes = [i64, i64, i64, vp, i32, i32, vp, i32, vp, i64, vp, dp, dp]
    L.oracle_conv2d_sep_points.restype = i32
    L.oracle_conv2d_hwc.argtypes = [i64, i64, i64, vp, i32, i32, i32, vp, dp, dp, i32]
    L.oracle_conv2d_hwc.restype = i32
    L.oracle_conv2d_sep_hwc.argtypes = [i64, i64, i64, vp, i32, i32, vp, i32, vp, dp, dp, i32]
    L.oracle_conv2d_sep_hwc.restype = i32
    L.oracle_conv2d_hwc_points.argtypes = [i64, i64, i64, vp, i32, i32, i32, vp, i64, vp, dp, dp]
    L.oracle_conv2d_hwc_points.restype = i32
    L.oracle_residual2d_f64.argtypes = [i64, i64, vp]
    L.oracle_residual2d_f64.restype = ctypes.c_double
    L.oracle_residual2d_f32.argtypes = [i64, i64, vp]
    L.oracle_residual2d_f32.restype = ctypes.c_double
    L.oracle_jacobi2d.argtypes = [i64, i64, vp, i32, i32, vp]
    L.oracle_jacobi2d.restype = i32
    L.oracle_op2_inc.argtypes = [i64, i64, vp, vp, vp]
    L.oracle_op2_inc.restype = i32
    L.oracle_rbsor2d.argtypes = [i64, i64, vp, i32, ctypes.c_double, i32, vp]
    L.oracle_rbsor2d.restype = i32
    _lib = L
    return L


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _image(x: np.ndarray):
    """(array as [c][h][w] contiguous, dtype code)."""
    if x.dtype == np.float16:
        x = np.ascontiguousarray(x).view(np.uint16)
        dt = DT_F16
    elif x.dtype == np.uint16:
        dt = DT_F16
    else:
        x = np.ascontiguousarray(x, dtype=np.float32)
        dt = DT_F32
    x = np.ascontiguousarray(x)
    if x.ndim == 2:
        x = x[None]
    if x.ndim != 3:
        raise ValueError("image must be [h][w] or [c][h][w]")
    return x, dt


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


def f16_to_f64(bits: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(bits).view(np.uint16).ravel()
    out = np.empty(b.size, dtype=np.float64)
    lib().oracle_f16_to_f64_array(b.size, _ptr(b), _ptr(out))
    return out.reshape(np.shape(bits))


def f64_to_f16(x: np.ndarray) -> np.ndarray:
    """binary16 bit patterns (uint16) of round-to-nearest-even(x)."""
    xd = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.empty(xd.size, dtype=np.uint16)
    lib().oracle_f64_to_f16_array(xd.size, _ptr(xd), _ptr(out))
    return out.reshape(np.shape(x))


BORDER = {"clamp": 0, "zero": 1, "reflect": 2, "mirror": 3, "wrap": 4}


def conv2d(img: np.ndarray, k: np.ndarray, want_bound: bool = True, border: str = "clamp"):
    """Correlation of every planar channel with k (FP64) under a border mode
    (clamp-to-edge by default).  Returns (out, bound) shaped like img
    ([h][w] inputs give [1][h][w])."""
    x, dt = _image(img)
    kk = np.ascontiguousarray(k, dtype=np.float32)
    c, h, w = x.shape
    kh, kw = kk.shape
    out = np.empty((c, h, w), dtype=np.float64)
    bound = np.empty((c, h, w), dtype=np.float64) if want_bound else None
    rc = lib().oracle_conv2d_mode(c, h, w, _ptr(x), dt, kh, kw, _ptr(kk), _ptr(out), _ptr(bound),
                                  BORDER[border])
    if rc != 0:
        raise ValueError("oracle_conv2d rejected its arguments")
    return out, bound


def conv2d_sep(img: np.ndarray, gx: np.ndarray, gy: np.ndarray, want_bound: bool = True):
    """Separable filter outer(gy, gx) applied as a direct correlation (FP64)."""
    x, dt = _image(img)
    gx = np.ascontiguousarray(gx, dtype=np.float32).ravel()
    gy = np.ascontiguousarray(gy, dtype=np.float32).ravel()
    c, h, w = x.shape
    out = np.empty((c, h, w), dtype=np.float64)
    bound = np.empty((c, h, w), dtype=np.float64) if want_bound else None
    rc = lib().oracle_conv2d_sep(c, h, w, _ptr(x), dt, gx.size, _ptr(gx), gy.size, _ptr(gy),
                                 _ptr(out), _ptr(bound))
    if rc != 0:
        raise ValueError("oracle_conv2d_sep rejected its arguments")
    return out, bound


def conv2d_points(img: np.ndarray, k: np.ndarray, pts: np.ndarray):
    """The correlation evaluated at sampled (ch, i, j) points: (out, bound)."""
    x, dt = _image(img)
    kk = np.ascontiguousarray(k, dtype=np.float32)
    p = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    c, h, w = x.shape
    kh, kw = kk.shape
    out = np.empty(p.shape[0], dtype=np.float64)
    bound = np.empty(p.shape[0], dtype=np.float64)
    rc = lib().oracle_conv2d_points(c, h, w, _ptr(x), dt, kh, kw, _ptr(kk), p.shape[0], _ptr(p),
                                    _ptr(out), _ptr(bound))
    if rc != 0:
        raise ValueError("oracle_conv2d_points rejected its arguments")
    return out, bound


def conv2d_sep_points(img: np.ndarray, gx: np.ndarray, gy: np.ndarray, pts: np.ndarray):
    """The separable definition evaluated at sampled (ch, i, j) points: (out, bound)."""
    x, dt = _image(img)
    gx = np.ascontiguousarray(gx, dtype=np.float32).ravel()
    gy = np.ascontiguousarray(gy, dtype=np.float32).ravel()
    p = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    c, h, w = x.shape
    out = np.empty(p.shape[0], dtype=np.float64)
    bound = np.empty(p.shape[0], dtype=np.float64)
    rc = lib().oracle_conv2d_sep_points(c, h, w, _ptr(x), dt, gx.size, _ptr(gx), gy.size, _ptr(gy),
                                        p.shape[0], _ptr(p), _ptr(out), _ptr(bound))
    if rc != 0:
        raise ValueError("oracle_conv2d_sep_points rejected its arguments")
    return out, bound


def _image_hwc(x: np.ndarray):
    """(array as [h][w][c] contiguous, dtype code)."""
    if x.dtype == np.float16:
        x = np.ascontiguousarray(x).view(np.uint16)
        dt = DT_F16
    elif x.dtype == np.uint16:
        dt = DT_F16
    else:
        x = np.ascontiguousarray(x, dtype=np.float32)
        dt = DT_F32
    x = np.ascontiguousarray(x)
    if x.ndim != 3:
        raise ValueError("interleaved image must be [h][w][c]")
    return x, dt


def conv2d_hwc(img: np.ndarray, k: np.ndarray, want_bound: bool = True, border: str = "clamp"):
    """Correlation of every channel of an interleaved [h][w][c] image with k
    (FP64) under a border mode.  Returns (out, bound), both [h][w][c]."""
    x, dt = _image_hwc(img)
    kk = np.ascontiguousarray(k, dtype=np.float32)
    h, w, c = x.shape
    kh, kw = kk.shape
    out = np.empty((h, w, c), dtype=np.float64)
    bound = np.empty((h, w, c), dtype=np.float64) if want_bound else None
    rc = lib().oracle_conv2d_hwc(c, h, w, _ptr(x), dt, kh, kw, _ptr(kk), _ptr(out), _ptr(bound), BORDER[border])
    if rc != 0:
        raise ValueError("oracle_conv2d_hwc rejected its arguments")
    return out, bound


def conv2d_sep_hwc(img: np.ndarray, gx: np.ndarray, gy: np.ndarray, want_bound: bool = True,
                   border: str = "clamp"):
    """Separable weights outer(gy, gx) on an interleaved [h][w][c] image (FP64)."""
    x, dt = _image_hwc(img)
    gx = np.ascontiguousarray(gx, dtype=np.float32).ravel()
    gy = np.ascontiguousarray(gy, dtype=np.float32).ravel()
    h, w, c = x.shape
    out = np.empty((h, w, c), dtype=np.float64)
    bound = np.empty((h, w, c), dtype=np.float64) if want_bound else None
    rc = lib().oracle_conv2d_sep_hwc(c, h, w, _ptr(x), dt, gx.size, _ptr(gx), gy.size, _ptr(gy), _ptr(out),
                                     _ptr(bound), BORDER[border])
    if rc != 0:
        raise ValueError("oracle_conv2d_sep_hwc rejected its arguments")
    return out, bound


def conv2d_hwc_points(img: np.ndarray, k: np.ndarray, pts: np.ndarray):
    """The interleaved correlation (clamp-to-edge) at sampled (ch, i, j) points: (out, bound)."""
    x, dt = _image_hwc(img)
    kk = np.ascontiguousarray(k, dtype=np.float32)
    p = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    h, w, c = x.shape
    kh, kw = kk.shape
    out = np.empty(p.shape[0], dtype=np.float64)
    bound = np.empty(p.shape[0], dtype=np.float64)
    rc = lib().oracle_conv2d_hwc_points(c, h, w, _ptr(x), dt, kh, kw, _ptr(kk), p.shape[0], _ptr(p),
                                        _ptr(out), _ptr(bound))
    if rc != 0:
        raise ValueError("oracle_conv2d_hwc_points rejected its arguments")
    return out, bound


def residual2d(u: np.ndarray) -> float:
    """Unscaled L2 norm of 4u - (up + down + left + right) over the interior."""
    if u.dtype == np.float32:
        uu = np.ascontiguousarray(u)
        return lib().oracle_residual2d_f32(uu.shape[0], uu.shape[1], _ptr(uu))
    uu = np.ascontiguousarray(u, dtype=np.float64)
    return lib().oracle_residual2d_f64(uu.shape[0], uu.shape[1], _ptr(uu))


def jacobi2d(u0: np.ndarray, iters: int, check_every: int = 0):
    """iters Jacobi sweeps in FP64 from u0 (widened).  Returns (u, residuals)."""
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    h, w = u.shape
    m = iters // check_every if check_every > 0 else 0
    res = np.zeros(max(m, 1), dtype=np.float64)
    rc = lib().oracle_jacobi2d(h, w, _ptr(u), int(iters), int(check_every), _ptr(res))
    if rc != 0:
        raise ValueError("oracle_jacobi2d rejected its arguments")
    return u, res[:m]


def rbsor2d(u0: np.ndarray, iters: int, omega: float, check_every: int = 0):
    """iters red-black SOR sweeps in FP64 from u0 (widened).  Returns (u, residuals)."""
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    h, w = u.shape
    m = iters // check_every if check_every > 0 else 0
    res = np.zeros(max(m, 1), dtype=np.float64)
    rc = lib().oracle_rbsor2d(h, w, _ptr(u), int(iters), float(omega), int(check_every), _ptr(res))
    if rc != 0:
        raise ValueError("oracle_rbsor2d rejected its arguments")
    return u, res[:m]


def op2_inc(cells: np.ndarray, e2c: np.ndarray, edge: np.ndarray) -> np.ndarray:
    """The sequential edge-to-cell increment (FP64); returns the new cell array."""
    c = np.array(cells, dtype=np.float64, copy=True)
    m = np.ascontiguousarray(e2c, dtype=np.int32).reshape(-1, 2)
    e = np.ascontiguousarray(edge, dtype=np.float64)
    if m.shape[0] != e.size:
        raise ValueError("one pair of cells per edge")
    rc = lib().oracle_op2_inc(c.size, e.size, _ptr(m), _ptr(e), _ptr(c))
    if rc != 0:
        raise ValueError("cell index out of range")
    return c
