"""ctypes binding of libpencilgpu: the C ABI's functions under the same names.

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Array arguments may be torch tensors (device or
host), numpy arrays (host) or raw integer addresses; `stream` may be a
torch.cuda.Stream, a raw cudaStream_t integer, or None for torch's current
stream.  A non-zero status raises PencilError.  If the shared library has not
been built this module raises on first use; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpencilgpu.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pencil.h")

PENCIL_F32 = 0
PENCIL_F16 = 1
PENCIL_CONV_GENERIC = 1
PENCIL_LAYOUT_HWC = 4  # channels interleaved [h][w][c] instead of planar [c][h][w]
PENCIL_CONV_TENSOR = 16  # binary16 images on the tensor cores (within the binary16 tolerance, not the same bits)
PENCIL_BORDER_CLAMP, PENCIL_BORDER_ZERO, PENCIL_BORDER_REFLECT, PENCIL_BORDER_MIRROR, PENCIL_BORDER_WRAP = range(5)
BORDER_MODES = {"clamp": 0, "zero": 1, "reflect": 2, "mirror": 3, "wrap": 4}


def PENCIL_BORDER(m):
    return m << 8
PENCIL_MAX_SPECIALISED_K = 15

PENCIL_OK = 0
PENCIL_ERR_TIMEOUT = -7
STATUS = {
    0: "PENCIL_OK", -1: "PENCIL_ERR_ARG", -2: "PENCIL_ERR_NULL", -3: "PENCIL_ERR_ALIAS",
    -4: "PENCIL_ERR_PTR", -5: "PENCIL_ERR_NOMEM", -6: "PENCIL_ERR_CUDA",
    -7: "PENCIL_ERR_TIMEOUT", -8: "PENCIL_ERR_UNSUPPORTED",
}


class PencilImage(ctypes.Structure):
    """struct pencil_image."""
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("k", ctypes.c_void_p),
                ("h", ctypes.c_int), ("w", ctypes.c_int), ("ks", ctypes.c_int)]


PENCIL_BATCH_VARIANTS = 6


class PencilError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        msg = f"{what}: {self.name}"
        if status == -6:
            msg += f" (cudaError {lib().pencil_last_cuda_error()})"
        super().__init__(msg)


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    i, vp, sz, d = ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p
    sig = {
        "pencil_conv2d": (i, [i, i, vp, i, i, vp, vp]),
        "pencil_conv2d_ex": (i, [i, i, i, vp, i, i, vp, vp, i, i, vp]),
        "pencil_conv2d_sep": (i, [i, i, vp, i, vp, i, vp, vp]),
        "pencil_conv2d_sep_ex": (i, [i, i, i, vp, i, vp, i, vp, vp, i, i, vp]),
        "pencil_jacobi2d": (i, [i, i, vp, i]),
        "pencil_jacobi2d_workspace_size": (sz, [i, i]),
        "pencil_jacobi2d_ex": (i, [i, i, vp, i, i, d, vp, sz, i, vp]),
        "pencil_residual2d": (i, [i, i, vp, d, vp, sz, vp]),
        "pencil_jacobi2d_noalloc": (i, [i, i, vp, i, i, d, i, vp]),
        "pencil_conv2d_chain": (i, [i, i, i, vp, i, i, vp, i, i, vp, vp, i, i, vp]),
        "pencil_conv2d_jacobi": (i, [i, i, i, vp, i, i, vp, i, vp, i, vp]),
        "pencil_op2_plan_create": (i, [i, i, vp, ctypes.POINTER(ctypes.c_void_p)]),
        "pencil_op2_inc": (i, [vp, vp, vp, i, vp]),
        "pencil_op2_plan_destroy": (i, [vp]),
        "pencil_jacobi2d_until": (i, [i, i, vp, i, i, ctypes.c_double, d, ctypes.POINTER(i), vp, sz, i, vp]),
        "pencil_rbsor2d_workspace_size": (sz, [i, i]),
        "pencil_rbsor2d_ex": (i, [i, i, vp, i, ctypes.c_float, i, d, vp, sz, vp]),
        "pencil_rbsor2d_until": (i, [i, i, vp, i, ctypes.c_float, i, ctypes.c_double, d, ctypes.POINTER(i), vp,
                                     sz, vp]),
        "pencil_batch_create": (i, [i, i, ctypes.c_longlong, ctypes.POINTER(ctypes.c_void_p)]),
        "pencil_batch_set_variant": (i, [vp, i, i]),
        "pencil_batch_tiles": (i, [vp, i, vp, ctypes.POINTER(ctypes.c_longlong)]),
        "pencil_batch_run": (i, [vp, i, vp, vp]),
        "pencil_batch_destroy": (i, [vp]),
        "pencil_tune": (i, [vp, i, vp, i, vp, ctypes.POINTER(i)]),
        "pencil_device_info": (i, [ctypes.c_char_p, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "pencil_arena_create": (i, [sz, sz, ctypes.POINTER(ctypes.c_void_p)]),
        "pencil_arena_alloc": (i, [vp, sz, ctypes.POINTER(ctypes.c_size_t)]),
        "pencil_arena_free": (i, [vp, sz]),
        "pencil_arena_free_bytes": (sz, [vp]),
        "pencil_arena_largest_free": (sz, [vp]),
        "pencil_arena_destroy": (None, [vp]),
        "pencil_strerror": (ctypes.c_char_p, [i]),
        "pencil_version": (i, []),
        "pencil_last_cuda_error": (i, []),
        "pencil_device_status": (i, []),
        "pencil_selftest_wait_timeout": (i, [ctypes.c_uint, ctypes.POINTER(i)]),
        "pencil_shutdown": (None, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def declared_symbols() -> list[str]:
    """Names of the functions include/pencil.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pencil_[a-z0-9_]+)\s*\(", text)))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st: int, what: str):
    if st != 0:
        raise PencilError(st, what)


def pencil_conv2d(h, w, in_, kh, kw, k, out):
    _check(lib().pencil_conv2d(h, w, _ptr(in_), kh, kw, _ptr(k), _ptr(out)), "pencil_conv2d")


def pencil_conv2d_ex(c, h, w, in_, kh, kw, k, out, dtype, flags=0, stream=None):
    _check(lib().pencil_conv2d_ex(c, h, w, _ptr(in_), kh, kw, _ptr(k), _ptr(out), dtype, flags,
                                  _stream(stream)), "pencil_conv2d_ex")


def pencil_conv2d_sep(h, w, in_, kx, gx, ky, gy, out):
    _check(lib().pencil_conv2d_sep(h, w, _ptr(in_), kx, _ptr(gx), ky, _ptr(gy), _ptr(out)),
           "pencil_conv2d_sep")


def pencil_conv2d_sep_ex(c, h, w, in_, kx, gx, ky, gy, out, dtype, flags=0, stream=None):
    _check(lib().pencil_conv2d_sep_ex(c, h, w, _ptr(in_), kx, _ptr(gx), ky, _ptr(gy), _ptr(out), dtype,
                                      flags, _stream(stream)), "pencil_conv2d_sep_ex")


def pencil_jacobi2d(h, w, u, iters):
    _check(lib().pencil_jacobi2d(h, w, _ptr(u), iters), "pencil_jacobi2d")


def pencil_jacobi2d_workspace_size(h, w) -> int:
    return int(lib().pencil_jacobi2d_workspace_size(h, w))


def pencil_jacobi2d_ex(h, w, u, iters, check_every, res_out, workspace, ws_bytes, temporal_t=0,
                       stream=None):
    _check(lib().pencil_jacobi2d_ex(h, w, _ptr(u), iters, check_every, _ptr(res_out), _ptr(workspace),
                                    ws_bytes, temporal_t, _stream(stream)), "pencil_jacobi2d_ex")


def pencil_residual2d(h, w, u, res_out, workspace, ws_bytes, stream=None):
    _check(lib().pencil_residual2d(h, w, _ptr(u), _ptr(res_out), _ptr(workspace), ws_bytes,
                                   _stream(stream)), "pencil_residual2d")


def pencil_conv2d_chain(c, h, w, inp, kh1, kw1, k1, kh2, kw2, k2, out, dtype, flags=0, stream=None):
    _check(lib().pencil_conv2d_chain(c, h, w, _ptr(inp), kh1, kw1, _ptr(k1), kh2, kw2, _ptr(k2), _ptr(out),
                                     dtype, flags, _stream(stream)), "pencil_conv2d_chain")


def pencil_conv2d_jacobi(c, h, w, inp, kh, kw, k, sweeps, out, flags=0, stream=None):
    _check(lib().pencil_conv2d_jacobi(c, h, w, _ptr(inp), kh, kw, _ptr(k), sweeps, _ptr(out), flags,
                                      _stream(stream)), "pencil_conv2d_jacobi")


PENCIL_CHAIN_FUSED = 2
PENCIL_MAX_ROWS = 524280
PENCIL_MAX_CHANNELS = 65535
PENCIL_OP2_ORDERED = 0
PENCIL_OP2_ATOMIC = 1


def pencil_op2_plan_create(ncells, nedges, e2c) -> int:
    """e2c: host int32 array of 2*nedges cell indices; returns the plan handle."""
    import numpy as np
    m = np.ascontiguousarray(e2c, dtype=np.int32)
    if m.size != 2 * nedges:
        raise PencilError(-1, f"pencil_op2_plan_create: e2c holds {m.size} indices, expected {2 * nedges}")
    out = ctypes.c_void_p()
    _check(lib().pencil_op2_plan_create(ncells, nedges, m.ctypes.data, ctypes.byref(out)), "pencil_op2_plan_create")
    return out.value


def pencil_op2_inc(plan, edge, cell, mode=PENCIL_OP2_ORDERED, stream=None):
    _check(lib().pencil_op2_inc(plan, _ptr(edge), _ptr(cell), mode, _stream(stream)), "pencil_op2_inc")


def pencil_op2_plan_destroy(plan):
    _check(lib().pencil_op2_plan_destroy(plan), "pencil_op2_plan_destroy")


def pencil_jacobi2d_until(h, w, u, max_iters, check_every, tol, res_out, workspace, ws_bytes, temporal_t=0,
                          stream=None) -> int:
    """Returns the number of sweeps performed."""
    done = ctypes.c_int()
    _check(lib().pencil_jacobi2d_until(h, w, _ptr(u), max_iters, check_every, tol, _ptr(res_out),
                                       ctypes.byref(done), _ptr(workspace), ws_bytes, temporal_t,
                                       _stream(stream)), "pencil_jacobi2d_until")
    return done.value


def pencil_rbsor2d_workspace_size(h, w) -> int:
    return int(lib().pencil_rbsor2d_workspace_size(h, w))


def pencil_rbsor2d_ex(h, w, u, iters, omega, check_every, res_out, workspace, ws_bytes, stream=None):
    _check(lib().pencil_rbsor2d_ex(h, w, _ptr(u), iters, omega, check_every, _ptr(res_out), _ptr(workspace),
                                   ws_bytes, _stream(stream)), "pencil_rbsor2d_ex")


def pencil_rbsor2d_until(h, w, u, max_iters, omega, check_every, tol, res_out, workspace, ws_bytes,
                         stream=None) -> int:
    """Returns the number of sweeps performed."""
    done = ctypes.c_int()
    _check(lib().pencil_rbsor2d_until(h, w, _ptr(u), max_iters, omega, check_every, tol, _ptr(res_out),
                                      ctypes.byref(done), _ptr(workspace), ws_bytes, _stream(stream)),
           "pencil_rbsor2d_until")
    return done.value


def pencil_jacobi2d_noalloc(h, w, u, iters, check_every, res_out, temporal_t=0, stream=None):
    _check(lib().pencil_jacobi2d_noalloc(h, w, _ptr(u), iters, check_every, _ptr(res_out), temporal_t,
                                         _stream(stream)), "pencil_jacobi2d_noalloc")


PENCIL_NOALLOC_SCRATCH_BYTES = 17 << 20


def make_images(items):
    """A ctypes array of pencil_image from (in, out, k, h, w, ks) tuples."""
    arr = (PencilImage * len(items))()
    for j, (i_, o, k, h, w, ks) in enumerate(items):
        arr[j] = PencilImage(_ptr(i_), _ptr(o), _ptr(k), h, w, ks)
    return arr


def pencil_batch_create(dtype, max_images, max_tiles) -> int:
    """Returns the plan handle (an integer address)."""
    out = ctypes.c_void_p()
    _check(lib().pencil_batch_create(dtype, max_images, max_tiles, ctypes.byref(out)), "pencil_batch_create")
    return out.value


def pencil_batch_set_variant(b, ks, variant):
    _check(lib().pencil_batch_set_variant(b, ks, variant), "pencil_batch_set_variant")


def pencil_batch_tiles(b, imgs) -> int:
    t = ctypes.c_longlong()
    _check(lib().pencil_batch_tiles(b, len(imgs), imgs, ctypes.byref(t)), "pencil_batch_tiles")
    return t.value


def pencil_batch_run(b, imgs, stream=None):
    _check(lib().pencil_batch_run(b, len(imgs), imgs, _stream(stream)), "pencil_batch_run")


def pencil_tune(b, imgs, reps=5, stream=None):
    """Measure every tile variant per filter side present in `imgs` (a
    make_images array), keep the fastest on plan b.  Returns {ks: variant}."""
    chosen = (ctypes.c_int * 8)()
    _check(lib().pencil_tune(b, len(imgs), imgs, reps, _stream(stream), chosen), "pencil_tune")
    return {2 * i + 1: chosen[i] for i in range(8) if chosen[i] >= 0}


def pencil_batch_destroy(b):
    _check(lib().pencil_batch_destroy(b), "pencil_batch_destroy")


def pencil_device_info():
    """(device name, SM count, CUDA driver version) of the current device."""
    name = ctypes.create_string_buffer(256)
    sms, drv = ctypes.c_int(), ctypes.c_int()
    _check(lib().pencil_device_info(name, 256, ctypes.byref(sms), ctypes.byref(drv)), "pencil_device_info")
    return name.value.decode(), sms.value, drv.value


def pencil_arena_create(capacity, align=256) -> int:
    out = ctypes.c_void_p()
    _check(lib().pencil_arena_create(capacity, align, ctypes.byref(out)), "pencil_arena_create")
    return out.value


def pencil_arena_alloc(a, nbytes):
    """Offset of a new block, or None when no free block is large enough."""
    off = ctypes.c_size_t()
    st = lib().pencil_arena_alloc(a, nbytes, ctypes.byref(off))
    if st == -5:
        return None
    _check(st, "pencil_arena_alloc")
    return off.value


def pencil_arena_free(a, offset):
    _check(lib().pencil_arena_free(a, offset), "pencil_arena_free")


def pencil_arena_free_bytes(a) -> int:
    return int(lib().pencil_arena_free_bytes(a))


def pencil_arena_largest_free(a) -> int:
    return int(lib().pencil_arena_largest_free(a))


def pencil_arena_destroy(a):
    lib().pencil_arena_destroy(a)


def pencil_strerror(status: int) -> str:
    return lib().pencil_strerror(status).decode()


def pencil_version() -> int:
    return lib().pencil_version()


def pencil_device_status() -> int:
    """PENCIL_OK, or -7 (PENCIL_ERR_TIMEOUT) if a device-side wait ran out
    since the last call (returned, not raised: it is a status report)."""
    st = lib().pencil_device_status()
    if st not in (0, -7):
        _check(st, "pencil_device_status")
    return st


def pencil_selftest_wait_timeout(limit_us: int) -> int:
    """1 if the self-test's never-completing wait completed, 0 if it ran out."""
    done = ctypes.c_int(-1)
    _check(lib().pencil_selftest_wait_timeout(limit_us, ctypes.byref(done)), "pencil_selftest_wait_timeout")
    return done.value


def pencil_last_cuda_error() -> int:
    return lib().pencil_last_cuda_error()


def pencil_shutdown() -> None:
    lib().pencil_shutdown()
