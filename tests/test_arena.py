"""The serving arena (host bookkeeping only; no GPU needed): first fit,
alignment, coalescing, exhaustion, and a randomized check against a model."""
import random

import pytest

import paper_1302_5586_gb300 as pg
from paper_1302_5586_gb300 import build as pg_build


@pytest.fixture(scope="module", autouse=True)
def built():
    pg_build.build()


def test_first_fit_alignment_and_exhaustion():
    a = pg.pencil_arena_create(4096, 256)
    try:
        x = pg.pencil_arena_alloc(a, 1)
        y = pg.pencil_arena_alloc(a, 300)
        z = pg.pencil_arena_alloc(a, 256)
        assert (x, y, z) == (0, 256, 768)
        assert pg.pencil_arena_free_bytes(a) == 4096 - 1024
        assert pg.pencil_arena_alloc(a, 4096) is None
        pg.pencil_arena_free(a, y)
        assert pg.pencil_arena_alloc(a, 512) == 256   # reuses the hole
        with pytest.raises(pg.PencilError):
            pg.pencil_arena_free(a, 100)              # not a block start
        with pytest.raises(pg.PencilError):
            pg.pencil_arena_alloc(a, 0)
    finally:
        pg.pencil_arena_destroy(a)


def test_freeing_merges_neighbours():
    a = pg.pencil_arena_create(1 << 20, 256)
    try:
        offs = [pg.pencil_arena_alloc(a, 1000) for _ in range(100)]
        for o in offs[::2]:
            pg.pencil_arena_free(a, o)
        assert pg.pencil_arena_largest_free(a) < 4096 + (1 << 20) - 100 * 1024
        for o in offs[1::2]:
            pg.pencil_arena_free(a, o)
        assert pg.pencil_arena_free_bytes(a) == 1 << 20
        assert pg.pencil_arena_largest_free(a) == 1 << 20
    finally:
        pg.pencil_arena_destroy(a)


def test_random_against_interval_model():
    rnd = random.Random(7)
    cap, align = 1 << 16, 64
    a = pg.pencil_arena_create(cap, align)
    live = {}
    try:
        for _ in range(3000):
            if live and rnd.random() < 0.45:
                off = rnd.choice(list(live))
                pg.pencil_arena_free(a, off)
                del live[off]
            else:
                n = rnd.randint(1, 3000)
                off = pg.pencil_arena_alloc(a, n)
                need = (n + align - 1) // align * align
                if off is None:
                    # first fit failed: no gap of `need` bytes may exist
                    ends = sorted((o, o + s) for o, s in live.items())
                    pos, gaps = 0, []
                    for lo, hi in ends:
                        gaps.append(lo - pos)
                        pos = hi
                    gaps.append(cap - pos)
                    assert max(gaps) < need
                    continue
                assert off % align == 0 and off + need <= cap
                for o, s in live.items():
                    assert off + need <= o or o + s <= off
                live[off] = need
            assert pg.pencil_arena_free_bytes(a) == cap - sum(live.values())
    finally:
        pg.pencil_arena_destroy(a)


def test_arena_argument_errors():
    with pytest.raises(pg.PencilError):
        pg.pencil_arena_create(4096, 3)
    with pytest.raises(pg.PencilError):
        pg.pencil_arena_create(0, 256)
    assert pg.pencil_arena_free_bytes(None) == 0


def test_serving_rejection_rule_matches_the_arena():
    """fits_alone (the serving loop's reject-on-arrival rule) is true exactly
    when an empty arena of that budget takes the request's input and output
    blocks, including budgets that are not a multiple of the alignment and
    sizes just past a block boundary."""
    from paper_1302_5586_gb300.serve import ARENA_ALIGN, fits_alone
    r = random.Random(7)
    cases = [(1, 128, 4, 1024), (1, 129, 4, 1024), (1, 64, 4, 767), (1, 64, 4, 768), (16, 16, 2, 1279)]
    cases += [(r.randint(1, 40), r.randint(1, 40), r.choice((2, 4)), r.randint(256, 20000)) for _ in range(300)]
    for h, w, esz, budget in cases:
        a = pg.pencil_arena_create(budget, ARENA_ALIGN)
        try:
            x = pg.pencil_arena_alloc(a, h * w * esz)
            y = pg.pencil_arena_alloc(a, h * w * esz) if x is not None else None
            assert fits_alone(h, w, esz, budget) == (y is not None), (h, w, esz, budget)
        finally:
            pg.pencil_arena_destroy(a)


def test_trace_recipe():
    """The serving trace: arrivals sorted inside the window, sides and odd
    filter sides inside their ranges, input windows inside the noise pool,
    filter offsets consecutive, and the same seed giving the same trace."""
    from paper_1302_5586_gb300.serve import make_trace
    t = make_trace(5, 400.0, 0.5, lo=64, hi=1024, klo=3, khi=15, pool_elems=1 << 20)
    rq = t.requests
    assert len(rq) > 100
    arr = [q.arrival for q in rq]
    assert arr == sorted(arr) and 0 <= arr[0] and arr[-1] < 0.5
    off = 0
    for q in rq:
        assert 64 <= q.h <= 1024 and 64 <= q.w <= 1024
        assert q.ks % 2 == 1 and 3 <= q.ks <= 15
        assert 0 <= q.src and q.src + q.h * q.w <= t.pool_elems
        assert q.filt == off
        off += q.ks * q.ks
    assert t.filters.size == off and t.filters.dtype.name == "float32"
    u = make_trace(5, 400.0, 0.5, lo=64, hi=1024, klo=3, khi=15, pool_elems=1 << 20)
    assert [(q.arrival, q.h, q.w, q.ks, q.src) for q in u.requests] == [(q.arrival, q.h, q.w, q.ks, q.src) for q in rq]
    empty = make_trace(5, 1e-9, 1e-6)
    assert empty.requests == [] and empty.filters.size == 1
