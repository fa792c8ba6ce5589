"""The batched conv2d kernels: bit-identical to the standalone
kernel on every image, within tolerance of the FP64 oracle, for every tile
variant (and a mix of variants across sides), across batches replayed from
the same captured graph and after a variant change drops the graphs."""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, to_dev, torch
from paper_1302_5586_gb300 import tune

pytestmark = pytest.mark.gpu


def make_batch(seed, n, lo, hi, dtype, ks=None):
    h, w, k = synth.batch_spec(seed, n, lo, hi)
    if ks is not None:
        k = np.full(n, ks)
    items, host = [], []
    for i in range(n):
        img = synth.image_f32(seed * 1000 + i, 1, int(h[i]), int(w[i]))[0]
        if dtype == pg.PENCIL_F16:
            img = synth.to_f16(img)
        filt = synth.filter_f32(seed * 1000 + 500 + i, int(k[i]), int(k[i]))
        d_in, d_k = to_dev(img), to_dev(filt)
        d_out = torch.full_like(d_in, float("nan"))
        items.append((d_in, d_out, d_k, int(h[i]), int(w[i]), int(k[i])))
        host.append((img, filt))
    return items, host


def standalone(it, dtype):
    d_in, _, d_k, h, w, ks = it
    o = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(1, h, w, d_in, ks, ks, d_k, o, dtype)
    return o


@pytest.mark.parametrize("dtype", [pg.PENCIL_F32, pg.PENCIL_F16])
@pytest.mark.parametrize("variant", list(range(pg.PENCIL_BATCH_VARIANTS)) + ["mixed"])
def test_batch_matches_standalone_bitwise_and_oracle(dtype, variant):
    items, host = make_batch(3 + (variant if variant != "mixed" else 7), 48, 1, 300, dtype)
    plan = pg.pencil_batch_create(dtype, 64, 1 << 16)
    try:
        pg.pencil_batch_run(plan, pg.make_images(items))  # captures graphs with variant 0 first
        torch.cuda.synchronize()
        for ks in range(1, 16, 2):
            v = variant if variant != "mixed" else (ks // 2) % pg.PENCIL_BATCH_VARIANTS
            pg.pencil_batch_set_variant(plan, ks, v)
        for it in items:
            it[1].fill_(float("nan"))
        pg.pencil_batch_run(plan, pg.make_images(items))
        torch.cuda.synchronize()
        tol = 1e-6 if dtype == pg.PENCIL_F32 else 2.0 ** -10
        for n, (it, (img, filt)) in enumerate(zip(items, host)):
            ref = standalone(it, dtype)
            assert torch.equal(it[1].view(torch.int16 if dtype else torch.int32),
                               ref.view(torch.int16 if dtype else torch.int32)), n
            if n % 6 == 0:
                o, bound = oracle.conv2d(img, filt)
                err = np.abs(it[1].cpu().numpy().astype(np.float64) - o[0])
                assert np.all(err <= tol * bound[0]), n
    finally:
        pg.pencil_batch_destroy(plan)


def test_one_plan_serves_successive_batches():
    plan = pg.pencil_batch_create(pg.PENCIL_F32, 40, 1 << 15)
    try:
        for seed in (11, 12, 13):
            items, _ = make_batch(seed, 20 + seed, 5, 260, pg.PENCIL_F32)
            pg.pencil_batch_run(plan, pg.make_images(items))
            torch.cuda.synchronize()
            for it in items:
                assert torch.equal(it[1], standalone(it, pg.PENCIL_F32))
    finally:
        pg.pencil_batch_destroy(plan)


@pytest.mark.parametrize("variant", [4, 5])
def test_one_tile_variant_follows_the_tile_count_of_each_batch(variant):
    """Under a one-CTA-per-tile variant the captured graph's grid is reset to
    each run's tile count: batches of one filter side (so one captured graph)
    with more, then fewer, then more tiles all match the standalone kernel
    (outputs start as NaN, so a tile left out shows)."""
    plan = pg.pencil_batch_create(pg.PENCIL_F32, 40, 1 << 15)
    try:
        pg.pencil_batch_set_variant(plan, 5, variant)
        counts = []
        for seed, n, hi in ((31, 30, 300), (32, 3, 40), (33, 36, 260)):
            items, _ = make_batch(seed, n, 5, hi, pg.PENCIL_F32, ks=5)
            imgs = pg.make_images(items)
            counts.append(pg.pencil_batch_tiles(plan, imgs))
            pg.pencil_batch_run(plan, imgs)
            torch.cuda.synchronize()
            for it in items:
                assert torch.equal(it[1], standalone(it, pg.PENCIL_F32))
        assert counts[1] < counts[0] and counts[2] != counts[1]
    finally:
        pg.pencil_batch_destroy(plan)


def test_batch_argument_errors():
    items, _ = make_batch(21, 4, 10, 40, pg.PENCIL_F32)
    plan = pg.pencil_batch_create(pg.PENCIL_F32, 4, 64)
    try:
        bad = list(items)
        bad[1] = bad[1][:5] + (4,)                      # even side
        with pytest.raises(pg.PencilError) as e:
            pg.pencil_batch_run(plan, pg.make_images(bad))
        assert e.value.name == "PENCIL_ERR_ARG"
        bad = list(items)
        bad[2] = (bad[2][0], bad[0][1]) + bad[2][2:]     # two outputs in one buffer
        with pytest.raises(pg.PencilError) as e:
            pg.pencil_batch_run(plan, pg.make_images(bad))
        assert e.value.name == "PENCIL_ERR_ALIAS"
        bad = list(items)
        bad[3] = (bad[3][0], bad[3][0]) + bad[3][2:]     # in place
        with pytest.raises(pg.PencilError) as e:
            pg.pencil_batch_run(plan, pg.make_images(bad))
        assert e.value.name == "PENCIL_ERR_ALIAS"
        more, _ = make_batch(22, 5, 10, 40, pg.PENCIL_F32)
        with pytest.raises(pg.PencilError) as e:
            pg.pencil_batch_run(plan, pg.make_images(more))
        assert e.value.name == "PENCIL_ERR_NOMEM"
        pg.pencil_batch_run(plan, pg.make_images(items))  # the valid batch still runs
        torch.cuda.synchronize()
    finally:
        pg.pencil_batch_destroy(plan)


def test_autotuner_sets_variants_and_caches(tmp_path):
    items, _ = make_batch(31, 24, 100, 600, pg.PENCIL_F32)
    plan = pg.pencil_batch_create(pg.PENCIL_F32, 32, 1 << 16)
    try:
        path = str(tmp_path / "tune.json")
        first = tune.autotune(plan, pg.PENCIL_F32, items, reps=2, path=path)
        assert all(src == "measured" for _, src in first.values())
        again = tune.autotune(plan, pg.PENCIL_F32, items, reps=2, path=path)
        assert {k: v for k, (v, _) in again.items()} == {k: v for k, (v, _) in first.items()}
        assert all(src == "cache" for _, src in again.values())
        pg.pencil_batch_run(plan, pg.make_images(items))
        torch.cuda.synchronize()
        for it in items:
            assert torch.equal(it[1], standalone(it, pg.PENCIL_F32))
    finally:
        pg.pencil_batch_destroy(plan)


@pytest.mark.parametrize("dtype", [pg.PENCIL_F32, pg.PENCIL_F16])
def test_full_size_512_images(dtype):
    """512 images, sides log-uniform in [64, 4096], odd filter sides 3..15: every
    image equals its standalone result bit for bit; 64 sampled pixels per image
    (plus its four corners) against the oracle."""
    seed = synth.SEEDS["batch512"]
    h, w, k = synth.batch_spec(seed, 512, 64, 4096)
    items = []
    rng = np.random.default_rng(5)
    for i in range(512):
        img = synth.image_f32(seed + 17 * i, 1, int(h[i]), int(w[i]))
        if dtype == pg.PENCIL_F16:
            img = synth.to_f16(img)
        filt = synth.filter_f32(seed + 17 * i + 1, int(k[i]), int(k[i]))
        d_in, d_k = to_dev(img), to_dev(filt)
        items.append((d_in, torch.empty_like(d_in), d_k, int(h[i]), int(w[i]), int(k[i]), img, filt))
    plan = pg.pencil_batch_create(dtype, 512, 1 << 22)
    try:
        pg.pencil_batch_run(plan, pg.make_images([it[:6] for it in items]))
        torch.cuda.synchronize()
        tol = 1e-6 if dtype == pg.PENCIL_F32 else 2.0 ** -10
        for d_in, d_out, d_k, hh, ww, ks, img, filt in items:
            ref = torch.empty_like(d_in)
            pg.pencil_conv2d_ex(1, hh, ww, d_in, ks, ks, d_k, ref, dtype)
            assert torch.equal(d_out, ref)
            pts = np.stack([np.zeros(68, np.int64),
                            np.concatenate([rng.integers(0, hh, 64), [0, 0, hh - 1, hh - 1]]),
                            np.concatenate([rng.integers(0, ww, 64), [0, ww - 1, 0, ww - 1]])], axis=1)
            o, bound = oracle.conv2d_points(img, filt, pts)
            got = d_out[0][torch.from_numpy(pts[:, 1]).to(dev()), torch.from_numpy(pts[:, 2]).to(dev())]
            assert np.all(np.abs(got.double().cpu().numpy() - o) <= tol * bound)
    finally:
        pg.pencil_batch_destroy(plan)


def test_native_tune_reports_present_sides_and_keeps_bits():
    """pencil_tune through the C ABI: a variant for every side present (and
    only those), the plan keeps it, and the batch is still the standalone bits."""
    items, _ = make_batch(33, 20, 80, 500, pg.PENCIL_F32)
    plan = pg.pencil_batch_create(pg.PENCIL_F32, 32, 1 << 16)
    try:
        imgs = pg.make_images(items)
        chosen = pg.pencil_tune(plan, imgs, reps=2)
        assert set(chosen) == {it[5] for it in items}
        assert all(0 <= v < pg.PENCIL_BATCH_VARIANTS for v in chosen.values())
        with pytest.raises(pg.PencilError) as e:
            pg.pencil_tune(plan, imgs, reps=0)
        assert e.value.name == "PENCIL_ERR_ARG"
        for it in items:
            it[1].zero_()
        pg.pencil_batch_run(plan, imgs)
        torch.cuda.synchronize()
        for it in items:
            assert torch.equal(it[1], standalone(it, pg.PENCIL_F32))
    finally:
        pg.pencil_batch_destroy(plan)
