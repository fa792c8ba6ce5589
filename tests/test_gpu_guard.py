"""Guard bands: every output is written inside its image and nowhere else.

Each output image is a view into a larger buffer whose elements before and
after the view hold a sentinel bit pattern; after the call the sentinels must
be unchanged bit for bit.  The views start at an aligned offset (TMA staging,
aligned stores) or one element off it (rows not 16-byte aligned: cp.async
staging with adaptive copies and per-address stores), and the shapes cover
the small-image tiles, ragged tile counts, and the direct, separable, chain
and batched kernels in FP32 and binary16.
"""
import numpy as np
import pytest

import paper_1302_5586_gb300 as pg
import synth
from gpu_util import to_dev, torch

pytestmark = pytest.mark.gpu

PAD = 256  # elements of sentinel on each side of an output
SENT = {torch.float32: 0x7FC0DEAD, torch.float16: 0x7E55}


def guarded(shape, dtype, misalign):
    """(buffer, view): a view of `shape` inside a sentinel-filled buffer."""
    n = int(np.prod(shape))
    off = PAD + (1 if misalign else 0)
    buf = torch.empty(n + 2 * PAD + 2, dtype=dtype, device="cuda")
    ints = torch.int32 if dtype == torch.float32 else torch.int16
    buf.view(ints).fill_(SENT[dtype])
    return buf, buf[off:off + n].view(shape), off, n


def check(buf, off, n, what):
    ints = torch.int32 if buf.dtype == torch.float32 else torch.int16
    v = buf.view(ints).cpu().numpy()
    want = v[0]
    assert np.all(v[:off] == want) and np.all(v[off + n:] == want), f"{what}: a write outside the output"


SHAPES = [(1, 1, 8), (2, 9, 136), (1, 70, 264), (3, 33, 1032), (1, 300, 400)]


@pytest.mark.parametrize("f16", [False, True])
@pytest.mark.parametrize("misalign", [False, True])
def test_direct_and_separable_write_only_their_output(f16, misalign):
    tdt = torch.float16 if f16 else torch.float32
    dt = pg.PENCIL_F16 if f16 else pg.PENCIL_F32
    for shape in SHAPES:
        c, h, w = shape
        img = synth.image_f32(70 + h, c, h, w)
        d_in = to_dev(synth.to_f16(img) if f16 else img)
        for K in (1, 3, 5, 7, 9, 15):
            k = to_dev(synth.filter_f32(80 + K, K, K))
            for border in (0, 1, 2):
                buf, out, off, n = guarded(shape, tdt, misalign)
                pg.pencil_conv2d_ex(c, h, w, d_in, K, K, k, out, dt, pg.PENCIL_BORDER(border))
                torch.cuda.synchronize()
                check(buf, off, n, f"direct K={K} {shape} border={border}")
        g = to_dev(synth.gaussian_taps_f32(7, 3.0))
        buf, out, off, n = guarded(shape, tdt, misalign)
        pg.pencil_conv2d_sep_ex(c, h, w, d_in, 15, g, 15, g, out, dt)
        torch.cuda.synchronize()
        check(buf, off, n, f"separable {shape}")
        k3 = to_dev(synth.filter_f32(90, 3, 3))
        buf, out, off, n = guarded(shape, tdt, misalign)
        pg.pencil_conv2d_chain(c, h, w, d_in, 3, 3, k3, 3, 3, k3, out, dt)
        torch.cuda.synchronize()
        check(buf, off, n, f"chain {shape}")
    assert pg.pencil_device_status() == pg.PENCIL_OK


@pytest.mark.parametrize("f16", [False, True])
def test_batch_writes_only_its_outputs(f16):
    tdt = torch.float16 if f16 else torch.float32
    dt = pg.PENCIL_F16 if f16 else pg.PENCIL_F32
    items, guards = [], []
    for i, (h, w, ks) in enumerate([(1, 8, 3), (33, 136, 15), (70, 265, 7), (5, 9, 5), (64, 128, 11)]):
        img = synth.image_f32(100 + i, 1, h, w)[0]
        d_in = to_dev(synth.to_f16(img) if f16 else img)
        buf, out, off, n = guarded((h, w), tdt, misalign=i % 2 == 1)
        k = to_dev(synth.filter_f32(110 + i, ks, ks))
        items.append((d_in, out, k, h, w, ks))
        guards.append((buf, off, n))
    plan = pg.pencil_batch_create(dt, 8, 1 << 12)
    try:
        pg.pencil_batch_run(plan, pg.make_images(items))
        torch.cuda.synchronize()
    finally:
        pg.pencil_batch_destroy(plan)
    for i, (buf, off, n) in enumerate(guards):
        check(buf, off, n, f"batch image {i}")
