"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def f16_host(t) -> np.ndarray:
    """A device float16 tensor as a numpy float16 array."""
    return t.cpu().numpy()


def sample_points(seed: int, c: int, h: int, w: int, n: int, borders: bool = True) -> np.ndarray:
    """n random (ch, i, j) points plus, optionally, every pixel of the two outer
    rows and columns of the last channel (where the clamp acts)."""
    r = np.random.default_rng(seed)
    pts = [np.stack([r.integers(0, c, n), r.integers(0, h, n), r.integers(0, w, n)], axis=1)]
    if borders:
        ch = c - 1
        for i in sorted({0, 1, h - 2, h - 1} & set(range(h))):
            pts.append(np.stack([np.full(w, ch), np.full(w, i), np.arange(w)], axis=1))
        for j in sorted({0, 1, w - 2, w - 1} & set(range(w))):
            pts.append(np.stack([np.full(h, ch), np.arange(h), np.full(h, j)], axis=1))
    return np.concatenate(pts).astype(np.int64)


def gather(t, pts: np.ndarray) -> np.ndarray:
    """Values of a [c][h][w] device tensor at the (ch, i, j) points, as float64."""
    p = torch.from_numpy(pts).to(t.device)
    return t[p[:, 0], p[:, 1], p[:, 2]].double().cpu().numpy()
