"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds no arithmetic of the convolution, the stencil or the
residual: it only draws random numbers and lays out inputs. Both sides
(the FP64 oracle under ``oracle/`` and the library under
``paper_1302_5586_gb300/``) receive the same arrays from here.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): element ``i`` (0-based) of the
stream started from state ``seed`` is ``mix(seed + (i + 1) * GAMMA)``, so the
stream is counter based and can be generated in any chunking.

Workload recipes (all seeded; sizes follow the workloads the paper's domains
call for, image processing and CFD stencils, Sec. 1 and Sec. 2):
  * images: planar ``[c][h][w]`` FP32, pixels U[0,1) = (z >> 40) * 2^-24;
  * filters: raw weights U[0,1) drawn in FP64 = (z >> 11) * 2^-53, normalised
    to sum 1 in FP64, rounded to FP32;
  * Gaussian taps: exp(-t^2 / (2 sigma^2)) for t = -r..r, normalised in FP64;
  * Jacobi grid: boundary ring u = 0.3 x + 0.7 y + 0.1 with x = j/(w-1),
    y = i/(h-1) evaluated in FP64 and rounded to FP32; interior U[-1,1) in FP32
    (2 * u01 - 1, exact);
  * batches and request streams: sides log-uniform in [lo, hi], odd filter
    sides uniform over {3, 5, ..., 15}, Poisson arrivals.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30 = np.uint64(30)
_S27 = np.uint64(27)
_S31 = np.uint64(31)
_S40 = np.uint64(40)
_S11 = np.uint64(11)

_CHUNK = 1 << 22

# Seeds of the named workloads (one per workload, fixed).
SEEDS = {
    "conv512": 0x5EED0001,
    "conv8192x3": 0x5EED0002,
    "jacobi8192": 0x5EED0003,
    "batch512": 0x5EED0004,
    "serve": 0x5EED0005,
    "op2mesh": 0x5EED0006,
}


def _mix_chunk(seed: int, start: int, n: int) -> np.ndarray:
    z = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    z *= GAMMA
    z += np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    z ^= z >> _S30
    z *= _M1
    z ^= z >> _S27
    z *= _M2
    z ^= z >> _S31
    return z


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Elements offset .. offset+n-1 of the SplitMix64 stream from ``seed``."""
    return _mix_chunk(seed, offset, n)


def _fill_parallel(n: int, fn, dtype) -> np.ndarray:
    out = np.empty(n, dtype=dtype)
    starts = list(range(0, n, _CHUNK))

    def work(s):
        e = min(n, s + _CHUNK)
        out[s:e] = fn(s, e - s)

    if len(starts) <= 1:
        for s in starts:
            work(s)
    else:
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(work, starts))
    return out


def u01_f32(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """U[0,1) in FP32: (z >> 40) * 2^-24, exact."""
    scale = np.float32(2.0 ** -24)

    def fn(s, m):
        return (_mix_chunk(seed, offset + s, m) >> _S40).astype(np.float32) * scale

    return _fill_parallel(n, fn, np.float32)


def u01_f64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """U[0,1) in FP64: (z >> 11) * 2^-53, exact."""
    z = splitmix64(seed, n, offset)
    return (z >> _S11).astype(np.float64) * (2.0 ** -53)


def image_f32(seed: int, c: int, h: int, w: int) -> np.ndarray:
    """Planar [c][h][w] FP32 image, pixels U[0,1)."""
    return u01_f32(seed, c * h * w).reshape(c, h, w)


def to_f16(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to binary16 (numpy's conversion, round to nearest even)."""
    return x.astype(np.float16)


def image_f16(seed: int, c: int, h: int, w: int) -> np.ndarray:
    """The FP32 image of ``image_f32`` rounded to binary16 (what the FP16 path stores)."""
    return to_f16(image_f32(seed, c, h, w))


def filter_f32(seed: int, kh: int, kw: int) -> np.ndarray:
    """kh x kw weights: U[0,1) in FP64, normalised in FP64 to sum 1, rounded to FP32."""
    raw = u01_f64(seed, kh * kw)
    return (raw / raw.sum()).astype(np.float32).reshape(kh, kw)


def gaussian_taps_f32(radius: int, sigma: float) -> np.ndarray:
    """1-D Gaussian taps g_t = exp(-t^2/(2 sigma^2)), t=-radius..radius, normalised in FP64."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-(t * t) / (2.0 * sigma * sigma))
    return (g / g.sum()).astype(np.float32)


def gaussian_2d_f32(radius: int, sigma: float) -> np.ndarray:
    """2-D Gaussian weights g_a * g_b from FP64-normalised taps, rounded to FP32."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-(t * t) / (2.0 * sigma * sigma))
    g = g / g.sum()
    return np.outer(g, g).astype(np.float32)


def jacobi_init_f32(seed: int, h: int, w: int) -> np.ndarray:
    """Jacobi start state: boundary ring 0.3x + 0.7y + 0.1 (FP64 -> FP32), interior U[-1,1)."""
    u = np.empty((h, w), dtype=np.float32)
    if h > 2 and w > 2:
        inner = u01_f32(seed, (h - 2) * (w - 2)).reshape(h - 2, w - 2)
        u[1:-1, 1:-1] = np.float32(2.0) * inner - np.float32(1.0)
    x = np.arange(w, dtype=np.float64) / max(w - 1, 1)
    y = np.arange(h, dtype=np.float64) / max(h - 1, 1)
    ring = lambda yy, xx: (0.3 * xx + 0.7 * yy + 0.1).astype(np.float32)
    u[0, :] = ring(y[0], x)
    u[h - 1, :] = ring(y[h - 1], x)
    u[:, 0] = ring(y, x[0])
    u[:, w - 1] = ring(y, x[w - 1])
    return u


def loguniform_sides(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers floor(lo * (hi/lo)^U), clamped to [lo, hi]."""
    u = u01_f64(seed, n)
    s = np.floor(lo * np.power(hi / lo, u)).astype(np.int64)
    return np.clip(s, lo, hi)


def odd_ksizes(seed: int, n: int, lo: int = 3, hi: int = 15) -> np.ndarray:
    """n odd filter sides, uniform over {lo, lo+2, ..., hi}."""
    m = (hi - lo) // 2 + 1
    z = splitmix64(seed, n)
    return (lo + 2 * (z % np.uint64(m)).astype(np.int64)).astype(np.int64)


def poisson_arrivals(seed: int, rate: float, duration: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate on [0, duration)."""
    n_guess = int(rate * duration * 1.2 + 10 * math.sqrt(rate * duration + 1) + 16)
    u = u01_f64(seed, n_guess)
    gaps = -np.log1p(-u) / rate
    t = np.cumsum(gaps)
    return t[t < duration]


def batch_spec(seed: int, n: int, lo: int, hi: int, klo: int = 3, khi: int = 15):
    """Per-image (h, w, k) for a batch: sides log-uniform, odd square filter sides."""
    h = loguniform_sides(seed ^ 0x1111, n, lo, hi)
    w = loguniform_sides(seed ^ 0x2222, n, lo, hi)
    k = odd_ksizes(seed ^ 0x3333, n, klo, khi)
    return h, w, k


def mesh_edges(seed: int, nx: int, ny: int):
    """Edges of an nx x ny grid of cells (each edge joins two cells that share a
    side), with cells relabelled, edges reordered and each edge's two ends
    swapped at random, so the connectivity looks unstructured.  Returns
    (ncells, e2c int32 [nedges][2])."""
    ncells = nx * ny
    idx = np.arange(ncells, dtype=np.int64).reshape(ny, nx)
    horiz = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1)
    vert = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1)
    e = np.concatenate([horiz, vert])
    z = splitmix64(seed, ncells + 2 * len(e))
    relabel = np.argsort(z[:ncells], kind="stable")
    e = relabel[e]
    e = e[np.argsort(z[ncells:ncells + len(e)], kind="stable")]
    swap = (z[ncells + len(e):] & np.uint64(1)).astype(bool)
    e[swap] = e[swap][:, ::-1]
    return ncells, np.ascontiguousarray(e, dtype=np.int32)
