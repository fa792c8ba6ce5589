"""Pins of the FP64 Jacobi and residual oracle against closed forms and invariants."""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_hand_cases():
    with open(os.path.join(GOLDEN, "jacobi_hand.json")) as f:
        cases = json.load(f)["cases"]
    for cs in cases:
        g = np.array(cs["grid"], dtype=np.float64)
        assert oracle.residual2d(g) == pytest.approx(cs["residual_before"], rel=1e-15)
        u, _ = oracle.jacobi2d(g, cs["sweeps"])
        np.testing.assert_array_equal(u, np.array(cs["expected"], dtype=np.float64), err_msg=cs["name"])
        assert oracle.residual2d(u) == pytest.approx(cs["residual_after"], rel=1e-15, abs=1e-15)


@pytest.mark.parametrize("n", [17, 65])
def test_linear_field_is_a_fixed_point(n):
    """u = a x + b y + c with dyadic a, b, c and N-1 a power of two: exact fixed point, residual 0."""
    x = np.arange(n) / (n - 1)
    y = np.arange(n) / (n - 1)
    u0 = 0.25 * x[None, :] + 0.5 * y[:, None] + 0.125
    u, res = oracle.jacobi2d(u0, 20, 5)
    np.testing.assert_array_equal(u, u0)
    assert np.all(res == 0.0)


@pytest.mark.parametrize("n,p,q,k", [(17, 1, 1, 7), (33, 2, 3, 25), (20, 5, 1, 3)])
def test_eigenmode_decays_by_lambda_power(n, p, q, k):
    """Zero boundary, u = sin(p pi x) sin(q pi y): k sweeps multiply u by lambda^k with
    lambda = (cos(p pi/(N-1)) + cos(q pi/(N-1))) / 2; the residual is |4 - 4 lambda| lambda^k |u|."""
    x = np.arange(n) / (n - 1)
    phi = np.sin(q * np.pi * x)[:, None] * np.sin(p * np.pi * x)[None, :]
    phi[0, :] = phi[-1, :] = phi[:, 0] = phi[:, -1] = 0.0
    lam = (math.cos(p * math.pi / (n - 1)) + math.cos(q * math.pi / (n - 1))) / 2
    u, res = oracle.jacobi2d(phi, k, 1)
    np.testing.assert_allclose(u, lam ** k * phi, atol=1e-13)
    norm_phi = np.sqrt(np.sum(phi[1:-1, 1:-1] ** 2))
    for m in range(1, k + 1):
        assert res[m - 1] == pytest.approx(abs(4 - 4 * lam) * abs(lam) ** m * norm_phi, rel=1e-11, abs=1e-13)


def test_converges_to_discrete_harmonic_solution():
    """With a linear boundary the limit is the linear field (the discrete harmonic
    function with that boundary); checked against a sparse direct solve as well."""
    h, w = 9, 7
    u0 = synth.jacobi_init_f32(5, h, w).astype(np.float64)
    u, res = oracle.jacobi2d(u0, 3000, 1000)
    x = np.arange(w) / (w - 1)
    y = np.arange(h) / (h - 1)
    # boundary is FP32-rounded 0.3x+0.7y+0.1: solve the Dirichlet problem with those exact values
    n_i, n_j = h - 2, w - 2
    idx = lambda i, j: (i - 1) * n_j + (j - 1)
    A = sp.lil_matrix((n_i * n_j, n_i * n_j))
    b = np.zeros(n_i * n_j)
    for i in range(1, h - 1):
        for j in range(1, w - 1):
            A[idx(i, j), idx(i, j)] = 4.0
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if ii in (0, h - 1) or jj in (0, w - 1):
                    b[idx(i, j)] += u0[ii, jj]
                else:
                    A[idx(i, j), idx(ii, jj)] = -1.0
    sol = spla.spsolve(A.tocsr(), b).reshape(n_i, n_j)
    np.testing.assert_allclose(u[1:-1, 1:-1], sol, atol=1e-12)
    lin = 0.3 * x[None, :] + 0.7 * y[:, None] + 0.1
    np.testing.assert_allclose(u, lin, atol=1e-7)  # boundary carries FP32 rounding only
    assert res[-1] < 1e-10


def test_residual_never_increases():
    u0 = synth.jacobi_init_f32(12, 24, 31).astype(np.float64)
    _, res = oracle.jacobi2d(u0, 200, 1)
    assert np.all(np.diff(res) <= 1e-12 * res[:-1])
    assert res[-1] < res[0]


def test_vertical_mirror_symmetry_is_preserved():
    """Mirroring rows swaps up and down, and (up + down) is commutative: bit-exact."""
    u0 = synth.jacobi_init_f32(3, 16, 13).astype(np.float64)
    u0 = u0 + u0[::-1, :]
    u, _ = oracle.jacobi2d(u0, 30)
    np.testing.assert_array_equal(u, u[::-1, :])
    v0 = synth.jacobi_init_f32(4, 13, 16).astype(np.float64)
    v0 = v0 + v0[:, ::-1]
    v, _ = oracle.jacobi2d(v0, 30)
    np.testing.assert_allclose(v, v[:, ::-1], rtol=1e-14, atol=1e-15)


def test_boundary_ring_is_fixed_and_no_interior_is_noop():
    u0 = synth.jacobi_init_f32(6, 12, 10).astype(np.float64)
    u, _ = oracle.jacobi2d(u0, 17)
    for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
        np.testing.assert_array_equal(u[sl], u0[sl])
    for h, w in ((1, 5), (2, 2), (2, 9), (7, 2)):
        g = np.arange(h * w, dtype=np.float64).reshape(h, w)
        u, res = oracle.jacobi2d(g, 10, 5)
        np.testing.assert_array_equal(u, g)
        assert np.all(res == 0.0)
    g = synth.jacobi_init_f32(1, 6, 6).astype(np.float64)
    u, res = oracle.jacobi2d(g, 0, 10)
    np.testing.assert_array_equal(u, g)
    assert res.size == 0


def test_residual_of_float32_grid_widens_exactly():
    u = synth.jacobi_init_f32(8, 15, 12)
    assert oracle.residual2d(u) == oracle.residual2d(u.astype(np.float64))
    # slicing restatement on a random grid
    d = u.astype(np.float64)
    r = 4 * d[1:-1, 1:-1] - d[:-2, 1:-1] - d[2:, 1:-1] - d[1:-1, :-2] - d[1:-1, 2:]
    assert oracle.residual2d(u) == pytest.approx(math.sqrt(np.sum(r * r)), rel=1e-14)


def test_initial_state_recipe():
    u = synth.jacobi_init_f32(99, 33, 17)
    x = np.arange(17) / 16
    y = np.arange(33) / 32
    lin = (0.3 * x[None, :] + 0.7 * y[:, None] + 0.1).astype(np.float32)
    for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
        np.testing.assert_array_equal(u[sl], lin[sl])
    inner = u[1:-1, 1:-1]
    assert inner.min() >= -1.0 and inner.max() < 1.0


def test_rbsor_golden_hand_case():
    with open(os.path.join(GOLDEN, "rbsor_hand.json")) as f:
        cs = json.load(f)["cases"][0]
    u, _ = oracle.rbsor2d(np.array(cs["grid"], dtype=np.float64), cs["sweeps"], cs["omega"])
    np.testing.assert_array_equal(u, np.array(cs["expected"], dtype=np.float64))


@pytest.mark.parametrize("omega", [0.7, 1.0, 1.5, 1.9])
def test_rbsor_linear_field_is_a_fixed_point(omega):
    n = 33
    x = np.arange(n) / (n - 1)
    u0 = 0.25 * x[None, :] + 0.5 * x[:, None] + 0.125
    u, res = oracle.rbsor2d(u0, 12, omega, 4)
    np.testing.assert_array_equal(u, u0)
    assert np.all(res == 0.0)


@pytest.mark.parametrize("omega", [1.0, 1.6])
def test_rbsor_converges_to_the_direct_solution_faster_than_jacobi(omega):
    h, w = 17, 13
    u0 = synth.jacobi_init_f32(9, h, w).astype(np.float64)
    u, res = oracle.rbsor2d(u0, 400, omega, 400)
    uj, resj = oracle.jacobi2d(u0, 400, 400)
    n_i, n_j = h - 2, w - 2
    idx = lambda i, j: (i - 1) * n_j + (j - 1)
    A = sp.lil_matrix((n_i * n_j, n_i * n_j))
    b = np.zeros(n_i * n_j)
    for i in range(1, h - 1):
        for j in range(1, w - 1):
            A[idx(i, j), idx(i, j)] = 4.0
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if ii in (0, h - 1) or jj in (0, w - 1):
                    b[idx(i, j)] += u0[ii, jj]
                else:
                    A[idx(i, j), idx(ii, jj)] = -1.0
    sol = spla.spsolve(A.tocsr(), b).reshape(n_i, n_j)
    np.testing.assert_allclose(u[1:-1, 1:-1], sol, atol=1e-11)
    assert res[-1] < resj[-1]


def test_rbsor_with_omega_one_matches_a_literal_gauss_seidel_ordering():
    """omega = 1: each colour's points depend only on the other colour, so the
    red-black sweep equals a Gauss-Seidel sweep that visits all even points
    (any order) then all odd points; here the odd points go in reverse order."""
    u0 = synth.jacobi_init_f32(21, 9, 11).astype(np.float64)
    u, _ = oracle.rbsor2d(u0, 3, 1.0)
    v = u0.copy()
    pts = [(i, j) for i in range(1, 8) for j in range(1, 10)]
    for _ in range(3):
        for i, j in [p for p in pts if sum(p) % 2 == 0]:
            v[i, j] = (v[i - 1, j] + v[i + 1, j] + v[i, j - 1] + v[i, j + 1]) / 4.0
        for i, j in reversed([p for p in pts if sum(p) % 2 == 1]):
            v[i, j] = (v[i - 1, j] + v[i + 1, j] + v[i, j - 1] + v[i, j + 1]) / 4.0
    np.testing.assert_allclose(u, v, rtol=1e-15, atol=1e-15)
