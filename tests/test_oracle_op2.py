"""Pins of the FP64 edge-to-cell increment (the OP2 loop of Sec. 3.1)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_hand_case():
    with open(os.path.join(GOLDEN, "op2_hand.json")) as f:
        cs = json.load(f)["cases"][0]
    out = oracle.op2_inc(np.array(cs["cells"], float), np.array(cs["e2c"]), np.array(cs["edge"], float))
    np.testing.assert_array_equal(out, cs["expected"])


@pytest.mark.parametrize("seed", range(5))
def test_matches_numpy_add_at_in_the_same_order(seed):
    """numpy.add.at accumulates repeated indices in index order: with the
    indices listed edge by edge (second end first) it is the sequential loop,
    bit for bit."""
    ncells, e2c = synth.mesh_edges(seed, 13, 9)
    r = np.random.default_rng(seed)
    edge = r.standard_normal(len(e2c))
    cells = r.standard_normal(ncells)
    out = oracle.op2_inc(cells, e2c, edge)
    ref = cells.copy()
    np.add.at(ref, e2c[:, ::-1].ravel(), np.repeat(edge, 2))
    np.testing.assert_array_equal(out, ref)


def test_integer_data_conserves_the_total_and_counts_degrees():
    ncells, e2c = synth.mesh_edges(3, 17, 11)
    out = oracle.op2_inc(np.zeros(ncells), e2c, np.ones(len(e2c)))
    deg = np.bincount(e2c.ravel(), minlength=ncells)
    np.testing.assert_array_equal(out, deg)
    assert out.sum() == 2 * len(e2c)
    # an nx x ny grid: corner cells have 2 sides, edge cells 3, inner cells 4
    assert sorted(np.unique(deg)) == [2, 3, 4]
    assert np.sum(deg == 2) == 4


def test_rejects_out_of_range_cells():
    with pytest.raises(ValueError):
        oracle.op2_inc(np.zeros(3), np.array([[0, 3]]), np.ones(1))
