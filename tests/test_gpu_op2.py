"""Parity of the OP2 edge-to-cell increment (Sec. 3.1) with the FP64 oracle.

The ordered kernel must give the oracle's bits (it adds each cell's
contributions in the sequential loop's order); the atomic kernel adds them in
an order the hardware picks, so it is held to the recursive-summation bound:
both it and the oracle are within gamma_m * sum|terms| of the exact sum, m the
number of additions into the cell, so they differ by at most twice that."""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _inputs(seed, nx, ny):
    ncells, e2c = synth.mesh_edges(seed, nx, ny)
    edge = 2.0 * synth.u01_f64(seed ^ 0x0E, len(e2c)) - 1.0
    cells = synth.u01_f64(seed ^ 0x0C, ncells)
    return ncells, e2c, edge, cells


def _run(e2c, ncells, edge, cells, mode, reps=1):
    plan = pg.pencil_op2_plan_create(ncells, len(e2c), e2c)
    try:
        de = to_dev(edge)
        dc = to_dev(cells)
        for _ in range(reps):
            pg.pencil_op2_inc(plan, de, dc, mode)
        torch.cuda.synchronize()
        return dc.cpu().numpy()
    finally:
        pg.pencil_op2_plan_destroy(plan)


def _atomic_bound(e2c, ncells, edge, cells):
    deg = np.bincount(e2c.ravel(), minlength=ncells)
    mag = np.abs(cells).copy()
    np.add.at(mag, e2c.ravel(), np.repeat(np.abs(edge), 2))
    u = 2.0 ** -53
    gam = deg * u / (1 - deg * u)
    return 2 * gam * mag


@pytest.mark.parametrize("nx,ny", [(1, 2), (7, 5), (33, 17), (129, 95), (300, 211)])
def test_ordered_is_bit_exact(nx, ny):
    dev()
    ncells, e2c, edge, cells = _inputs(nx * 1000 + ny, nx, ny)
    want = oracle.op2_inc(cells, e2c, edge)
    got = _run(e2c, ncells, edge, cells, pg.PENCIL_OP2_ORDERED)
    np.testing.assert_array_equal(got, want)


def test_ordered_repeats_give_the_loop_applied_twice():
    dev()
    ncells, e2c, edge, cells = _inputs(3, 64, 48)
    want = oracle.op2_inc(oracle.op2_inc(cells, e2c, edge), e2c, edge)
    got = _run(e2c, ncells, edge, cells, pg.PENCIL_OP2_ORDERED, reps=2)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("nx,ny", [(7, 5), (129, 95), (512, 384)])
def test_atomic_within_summation_bound(nx, ny):
    dev()
    ncells, e2c, edge, cells = _inputs(nx + 7 * ny, nx, ny)
    want = oracle.op2_inc(cells, e2c, edge)
    got = _run(e2c, ncells, edge, cells, pg.PENCIL_OP2_ATOMIC)
    bound = _atomic_bound(e2c, ncells, edge, cells)
    assert np.all(np.abs(got - want) <= bound)


def test_integer_valued_atomic_is_exact():
    """Small integers add exactly in any order, so the atomic kernel is exact too."""
    dev()
    ncells, e2c = synth.mesh_edges(11, 90, 70)
    edge = np.floor(16 * synth.u01_f64(12, len(e2c))) - 8.0
    cells = np.floor(16 * synth.u01_f64(13, ncells))
    want = oracle.op2_inc(cells, e2c, edge)
    for mode in (pg.PENCIL_OP2_ORDERED, pg.PENCIL_OP2_ATOMIC):
        np.testing.assert_array_equal(_run(e2c, ncells, edge, cells, mode), want)


def test_irregular_degrees_self_loops_and_isolated_cells():
    """A star (one cell with thousands of edges), self-loops (both ends one
    cell: two additions), repeated edges and cells that no edge touches."""
    dev()
    r = np.random.default_rng(5)
    ncells = 5000
    star = np.stack([np.zeros(3000, np.int64), r.integers(1, 2000, 3000)], axis=1)
    loops = np.repeat(r.integers(2000, 2500, 200)[:, None], 2, axis=1)
    rep = np.repeat(np.array([[2600, 2601]]), 50, axis=0)
    e2c = np.concatenate([star, loops, rep])
    e2c = e2c[r.permutation(len(e2c))]
    sw = r.integers(0, 2, len(e2c)).astype(bool)
    e2c[sw] = e2c[sw][:, ::-1]
    e2c = np.ascontiguousarray(e2c, dtype=np.int32)
    edge = r.standard_normal(len(e2c))
    cells = r.standard_normal(ncells)
    want = oracle.op2_inc(cells, e2c, edge)
    np.testing.assert_array_equal(_run(e2c, ncells, edge, cells, pg.PENCIL_OP2_ORDERED), want)
    got = _run(e2c, ncells, edge, cells, pg.PENCIL_OP2_ATOMIC)
    assert np.all(np.abs(got - want) <= _atomic_bound(e2c, ncells, edge, cells))
    np.testing.assert_array_equal(got[2700:], cells[2700:])


def test_ordered_is_bit_exact_on_an_eight_neighbour_mesh():
    """Cells joined to their side and diagonal neighbours (interior cells have
    eight contributions), self-loops on the corners, shuffled: the plan's
    eight-slot table, against the oracle bit for bit."""
    dev()
    nx, ny = 61, 47
    idx = np.arange(nx * ny).reshape(ny, nx)
    pairs = [np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1),
             np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1),
             np.stack([idx[:-1, :-1].ravel(), idx[1:, 1:].ravel()], axis=1),
             np.stack([idx[:-1, 1:].ravel(), idx[1:, :-1].ravel()], axis=1),
             np.repeat(np.array([idx[0, 0], idx[0, -1], idx[-1, 0], idx[-1, -1]])[:, None], 2, axis=1)]
    r = np.random.default_rng(9)
    e2c = np.concatenate(pairs)
    e2c = e2c[r.permutation(len(e2c))]
    sw = r.integers(0, 2, len(e2c)).astype(bool)
    e2c[sw] = e2c[sw][:, ::-1]
    e2c = np.ascontiguousarray(e2c, dtype=np.int32)
    assert np.bincount(e2c.ravel()).max() == 8
    edge = r.standard_normal(len(e2c))
    cells = r.standard_normal(nx * ny)
    want = oracle.op2_inc(cells, e2c, edge)
    np.testing.assert_array_equal(_run(e2c, nx * ny, edge, cells, pg.PENCIL_OP2_ORDERED), want)


def test_no_edges_leaves_cells_unchanged():
    dev()
    cells = synth.u01_f64(2, 37)
    e2c = np.zeros((0, 2), np.int32)
    for mode in (pg.PENCIL_OP2_ORDERED, pg.PENCIL_OP2_ATOMIC):
        plan = pg.pencil_op2_plan_create(37, 0, e2c)
        dc = to_dev(cells)
        de = torch.zeros(1, dtype=torch.float64, device=dev())
        pg.pencil_op2_inc(plan, de, dc, mode)
        torch.cuda.synchronize()
        pg.pencil_op2_plan_destroy(plan)
        np.testing.assert_array_equal(dc.cpu().numpy(), cells)


def test_full_size_mesh_is_bit_exact():
    """The 2048 x 2048-cell mesh (8.4 M edges) of the bench, the whole output."""
    dev()
    ncells, e2c, edge, cells = _inputs(synth.SEEDS["op2mesh"], 2048, 2048)
    want = oracle.op2_inc(cells, e2c, edge)
    got = _run(e2c, ncells, edge, cells, pg.PENCIL_OP2_ORDERED)
    np.testing.assert_array_equal(got, want)
    got = _run(e2c, ncells, edge, cells, pg.PENCIL_OP2_ATOMIC)
    assert np.all(np.abs(got - want) <= _atomic_bound(e2c, ncells, edge, cells))


def test_errors():
    dev()
    e2c = np.array([[0, 1], [1, 2]], np.int32)
    with pytest.raises(pg.PencilError) as ei:
        pg.pencil_op2_plan_create(2, 2, e2c)  # index 2 out of range
    assert ei.value.status == -1
    with pytest.raises(pg.PencilError):
        pg.pencil_op2_plan_create(3, 3, e2c)  # size mismatch, caught in the binding
    plan = pg.pencil_op2_plan_create(3, 2, e2c)
    try:
        buf = torch.zeros(8, dtype=torch.float64, device=dev())
        with pytest.raises(pg.PencilError) as ei:
            pg.pencil_op2_inc(plan, buf[0:2], buf[1:4])
        assert ei.value.status == -3
        with pytest.raises(pg.PencilError) as ei:
            pg.pencil_op2_inc(plan, buf[0:2], buf[4:7], mode=7)
        assert ei.value.status == -1
        host = torch.zeros(3, dtype=torch.float64)
        with pytest.raises(pg.PencilError) as ei:
            pg.pencil_op2_inc(plan, buf[0:2], host)
        assert ei.value.status == -4
    finally:
        pg.pencil_op2_plan_destroy(plan)
