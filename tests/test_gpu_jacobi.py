"""GPU parity of the Jacobi sweep and the FP64 residual against the oracle.

Iterate: |gpu - oracle| <= 1e-5 absolute after up to 100 sweeps.
Residual of a GPU iterate u: the GPU forms r in FP32, so its sum of squares
can differ from the exact sum over the same u by at most
  sum_i e_i (2 |r_i| + e_i),  e_i = (2u + u^2)(1 + u) M_i + u |r_i|,
  M_i = |up| + |down| + |left| + |right|, u = 2^-24,
plus 2^-40 of the sum for the compensated per-thread partials and the FP64
accumulation; the test checks exactly that bound.
Residual trajectory against the FP64 oracle's own iterates u_ref: since
|r(u) - r(u')| <= 8 |u - u'| (the residual operator's rows have absolute sum 8),
|res_gpu - res_ref| <= 8 |u_gpu - u_ref|_2 + sqrt(bound above), checked at every
checkpoint with the GPU and oracle iterates of that checkpoint.
"""
import math

import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, to_dev, torch

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def run_jacobi(u0, iters, check_every, temporal_t=0):
    h, w = u0.shape
    d_u = to_dev(u0)
    ws_bytes = pg.pencil_jacobi2d_workspace_size(h, w)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev())
    m = iters // check_every if check_every > 0 else 0
    res = torch.full((max(m, 1),), -1.0, dtype=torch.float64, device=dev())
    pg.pencil_jacobi2d_ex(h, w, d_u, iters, check_every, res if m else None, ws, ws_bytes, temporal_t)
    torch.cuda.synchronize()
    return d_u, res[:m].cpu().numpy()


def residual_gpu(d_u):
    h, w = d_u.shape
    ws_bytes = pg.pencil_jacobi2d_workspace_size(h, w)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev())
    res = torch.zeros(1, dtype=torch.float64, device=dev())
    pg.pencil_residual2d(h, w, d_u, res, ws, ws_bytes)
    torch.cuda.synchronize()
    return float(res.cpu()[0])


def residual_sq_bound(u: np.ndarray):
    """(exact sum of r^2 over u in FP64, bound on |gpu sum - exact sum|).
    The GPU forms r in FP32 (|r_gpu - r| <= e) and rounds r_gpu^2 to FP32
    (relative error <= u, on r_gpu^2 <= (|r| + e)^2), then sums the rounded
    squares to about 2^-44 of the total."""
    d = u.astype(np.float64)
    up, dn, lf, rt = d[:-2, 1:-1], d[2:, 1:-1], d[1:-1, :-2], d[1:-1, 2:]
    r = 4 * d[1:-1, 1:-1] - up - dn - lf - rt
    m = np.abs(up) + np.abs(dn) + np.abs(lf) + np.abs(rt)
    e = (2 * U32 + U32 ** 2) * (1 + U32) * m + U32 * np.abs(r)
    s = float(np.sum(r * r))
    sq = e * (2 * np.abs(r) + e) + U32 * (np.abs(r) + e) ** 2
    return s, float(np.sum(sq)) + 2.0 ** -40 * s + 1e-300


def check_residual(res_gpu, u_gpu_host):
    s, b = residual_sq_bound(u_gpu_host)
    assert abs(res_gpu ** 2 - s) <= b, f"residual^2 {res_gpu**2!r} vs exact {s!r}, bound {b!r}"
    return b


def check_trajectory(u0, iters, check_every, temporal_t=0):
    """Run iters sweeps with residuals every check_every; check the final iterate
    (1e-5 absolute) and every residual against the oracle with the derived bound.
    Returns (final device iterate, residuals)."""
    d_u, res = run_jacobi(u0, iters, check_every, temporal_t)
    u_ref = u0.astype(np.float64)
    done = 0
    for m in range(1, iters // check_every + 1):
        u_ref, _ = oracle.jacobi2d(u_ref, m * check_every - done)
        done = m * check_every
        d_m, res_m = run_jacobi(u0, m * check_every, check_every, temporal_t)
        # the same iterates; with T > 1 the residual of the last checkpoint can come
        # from another kernel (another summation tree) than inside the longer run
        np.testing.assert_allclose(res_m, res[:m], rtol=1e-9, atol=1e-300)
        u_m = d_m.cpu().numpy()
        du = u_m.astype(np.float64) - u_ref
        assert np.max(np.abs(du)) <= 1e-5
        b = check_residual(res[m - 1], u_m)
        res_ref = oracle.residual2d(u_ref)
        slack = 8 * np.sqrt(np.sum(du ** 2)) + np.sqrt(b)
        assert abs(res[m - 1] - res_ref) <= slack, (m, res[m - 1], res_ref, slack)
    u_ref, _ = oracle.jacobi2d(u_ref, iters - done)
    assert np.max(np.abs(d_u.cpu().numpy().astype(np.float64) - u_ref)) <= 1e-5
    return d_u, res


SHAPES = [(37, 53), (64, 128), (131, 260), (3, 3), (5, 4), (200, 17), (96, 2052)]


@pytest.mark.parametrize("shape", SHAPES)
def test_iterate_and_residuals_match_oracle(shape):
    h, w = shape
    u0 = synth.jacobi_init_f32(500 + h, h, w)
    check_trajectory(u0, 30, 10)
    check_trajectory(u0, 23, 7)


@pytest.mark.parametrize("t", [2, 3, 4, 5, 7, 8, 10, 13])
@pytest.mark.parametrize("shape", [(67, 132), (200, 516), (9, 12), (130, 244), (3, 8)])
def test_temporal_tiling_is_bit_identical(t, shape):
    """T sweeps per pass give the same iterate bits as one sweep per pass; the
    residuals (same FP32 r values, another summation tree) agree to 1e-9."""
    h, w = shape
    u0 = synth.jacobi_init_f32(900 + t, h, w)
    for iters, ce in ((23, 4), (20, 10), (7, 1)):
        a, ra = run_jacobi(u0, iters, ce, 1)
        b, rb = run_jacobi(u0, iters, ce, t)
        np.testing.assert_array_equal(a.cpu().numpy().view(np.uint32), b.cpu().numpy().view(np.uint32))
        np.testing.assert_allclose(rb, ra, rtol=1e-9, atol=1e-300)


@pytest.mark.parametrize("t", [1, 5, 10])
def test_tiled_trajectory_matches_oracle(t):
    u0 = synth.jacobi_init_f32(77, 150, 260)
    check_trajectory(u0, 30, 10, t)


def test_boundary_ring_is_untouched_and_ring_only_grids_are_noops():
    u0 = synth.jacobi_init_f32(7, 70, 92)
    u = run_jacobi(u0, 9, 0)[0].cpu().numpy()
    for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
        np.testing.assert_array_equal(u[sl], u0[sl])
    for h, w in ((1, 8), (2, 2), (2, 12), (9, 2), (1, 1)):
        g = synth.u01_f32(3, h * w).reshape(h, w)
        d, res = run_jacobi(g, 10, 5)
        np.testing.assert_array_equal(d.cpu().numpy(), g)
        assert np.all(res == 0.0)
    d, res = run_jacobi(u0, 0, 10)
    np.testing.assert_array_equal(d.cpu().numpy(), u0)
    assert res.size == 0


@pytest.mark.parametrize("n", [17, 65, 1025])
def test_linear_field_is_a_bit_exact_fixed_point(n):
    x = (np.arange(n) / (n - 1)).astype(np.float64)
    u0 = (0.25 * x[None, :] + 0.5 * x[:, None] + 0.125).astype(np.float32)
    d, res = run_jacobi(u0, 20, 10)
    np.testing.assert_array_equal(d.cpu().numpy(), u0)
    assert np.all(res == 0.0)


def test_eigenmode_decay():
    """Zero boundary, u = sin(p pi x) sin(q pi y): k sweeps scale u by lambda^k and the
    residual is |4 - 4 lambda| lambda^k |u|.  The GPU iterate carries FP32 rounding, so the
    residual is compared with slack 8 |u_gpu - lambda^k u0| (the residual operator's norm is
    at most 8) on top of the exact-sum bound."""
    n, p, q = 129, 3, 2
    x = np.arange(n) / (n - 1)
    phi = np.sin(q * np.pi * x)[:, None] * np.sin(p * np.pi * x)[None, :]
    phi[0, :] = phi[-1, :] = phi[:, 0] = phi[:, -1] = 0
    u0 = phi.astype(np.float32)
    u0d = u0.astype(np.float64)
    lam = (math.cos(p * math.pi / (n - 1)) + math.cos(q * math.pi / (n - 1))) / 2
    nrm = np.sqrt(np.sum(u0d[1:-1, 1:-1] ** 2))
    for k in (10, 20, 40):
        d, res = run_jacobi(u0, k, 10)
        u = d.cpu().numpy()
        du = u.astype(np.float64) - lam ** k * u0d
        assert np.max(np.abs(du)) <= 1e-5
        closed = abs(4 - 4 * lam) * lam ** k * nrm
        assert abs(res[-1] - closed) <= 8 * np.sqrt(np.sum(du ** 2)) + 1e-9
        check_residual(res[-1], u)


def test_residuals_never_increase():
    u0 = synth.jacobi_init_f32(17, 150, 190)
    _, res = run_jacobi(u0, 100, 5)
    assert np.all(np.diff(res) <= 1e-6 * res[:-1])


def test_plain_call_host_and_device():
    u0 = synth.jacobi_init_f32(23, 61, 83)
    host = u0.copy()
    pg.pencil_jacobi2d(61, 83, host, 25)
    d = to_dev(u0)
    pg.pencil_jacobi2d(61, 83, d, 25)
    np.testing.assert_array_equal(host, d.cpu().numpy())
    ref, _ = oracle.jacobi2d(u0, 25)
    assert np.max(np.abs(host - ref)) <= 1e-5


def test_odd_sweep_count_ends_in_place():
    u0 = synth.jacobi_init_f32(29, 40, 44)
    d, _ = run_jacobi(u0, 7, 0)
    d6, _ = run_jacobi(u0, 6, 0)
    u7 = d.cpu().numpy()
    # one more plain sweep from the 6-sweep iterate gives the same bits
    d6b, _ = run_jacobi(d6.cpu().numpy(), 1, 0)
    np.testing.assert_array_equal(u7, d6b.cpu().numpy())


def test_residual_entry_point():
    u0 = synth.jacobi_init_f32(31, 77, 130)
    r = residual_gpu(to_dev(u0))
    check_residual(r, u0)
    assert r == pytest.approx(oracle.residual2d(u0), rel=1e-6)


def test_workspace_and_alias_errors():
    u = torch.zeros(64, 64, device=dev())
    ws_bytes = pg.pencil_jacobi2d_workspace_size(64, 64)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev())
    with pytest.raises(pg.PencilError) as e:
        pg.pencil_jacobi2d_ex(64, 64, u, 5, 0, None, ws, ws_bytes - 1)
    assert e.value.name == "PENCIL_ERR_NOMEM"
    with pytest.raises(pg.PencilError) as e:
        pg.pencil_jacobi2d_ex(64, 64, ws, 5, 0, None, ws, ws_bytes)
    assert e.value.name == "PENCIL_ERR_ALIAS"
    with pytest.raises(pg.PencilError) as e:
        pg.pencil_jacobi2d_ex(64, 64, np.zeros((64, 64), np.float32), 5, 0, None, ws, ws_bytes)
    assert e.value.name == "PENCIL_ERR_PTR"


def test_full_size_8192_100_sweeps():
    """The 8192 x 8192, 100-sweep workload in the benchmark's configuration,
    against the FP64 oracle over the whole grid at every checkpoint."""
    n = 8192
    u0 = synth.jacobi_init_f32(synth.SEEDS["jacobi8192"], n, n)
    d_auto, r_auto = check_trajectory(u0, 100, 10)
    d_one, r_one = run_jacobi(u0, 100, 10, 1)
    assert torch.equal(d_auto.view(torch.int32), d_one.view(torch.int32))
    np.testing.assert_allclose(r_auto, r_one, rtol=1e-9)
