"""Red-black SOR and the converge-to-tolerance loop (untilconverged with its
threshold) on the GPU, against the FP64 oracle.

Iterate tolerance for SOR with omega <= 1.5: 1e-5 absolute after 25 sweeps (the
Jacobi bound); for larger omega the FP32 rounding of a sweep is amplified by
the slowly decaying modes, so those runs are checked by properties that hold
exactly (fixed point) or at convergence (the discrete harmonic solution)."""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, to_dev, torch

pytestmark = pytest.mark.gpu


def run_sor(u0, iters, omega, ce):
    h, w = u0.shape
    d = to_dev(u0)
    wsb = pg.pencil_rbsor2d_workspace_size(h, w)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev())
    m = iters // ce if ce else 0
    res = torch.zeros(max(m, 1), dtype=torch.float64, device=dev())
    pg.pencil_rbsor2d_ex(h, w, d, iters, omega, ce, res if m else None, ws, wsb)
    torch.cuda.synchronize()
    return d.cpu().numpy(), res[:m].cpu().numpy()


def run_jacobi(u0, iters, ce, t=0):
    h, w = u0.shape
    d = to_dev(u0)
    wsb = pg.pencil_jacobi2d_workspace_size(h, w)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev())
    m = iters // ce if ce else 0
    res = torch.zeros(max(m, 1), dtype=torch.float64, device=dev())
    pg.pencil_jacobi2d_ex(h, w, d, iters, ce, res if m else None, ws, wsb, t)
    torch.cuda.synchronize()
    return d.cpu().numpy(), res[:m].cpu().numpy()


@pytest.mark.parametrize("omega", [1.0, 1.25, 1.5])
@pytest.mark.parametrize("shape", [(37, 53), (64, 128), (131, 260), (3, 3), (200, 17), (5, 8)])
def test_sor_matches_oracle(omega, shape):
    h, w = shape
    u0 = synth.jacobi_init_f32(60 + h, h, w)
    u, res = run_sor(u0, 25, omega, 5)
    ref, rres = oracle.rbsor2d(u0, 25, omega, 5)
    du = u.astype(np.float64) - ref
    assert np.max(np.abs(du)) <= 1e-5
    # residual of the GPU iterate: exact sum within the FP32-r bound (as for Jacobi)
    from test_gpu_jacobi import check_residual  # noqa: E402
    check_residual(res[-1], u)
    assert abs(res[-1] - rres[-1]) <= 8 * np.sqrt(np.sum(du ** 2)) + 1e-6 * rres[-1] + 1e-12


@pytest.mark.parametrize("omega", [0.5, 1.0, 1.9])
def test_sor_linear_field_is_a_bit_exact_fixed_point(omega):
    n = 129
    x = np.arange(n) / (n - 1)
    u0 = (0.25 * x[None, :] + 0.5 * x[:, None] + 0.125).astype(np.float32)
    u, res = run_sor(u0, 10, omega, 5)
    np.testing.assert_array_equal(u, u0)
    assert np.all(res == 0.0)


def test_sor_converges_to_the_discrete_solution():
    h, w = 33, 29
    u0 = synth.jacobi_init_f32(88, h, w)
    u, res = run_sor(u0, 300, 1.8, 300)
    lim, _ = oracle.rbsor2d(u0, 3000, 1.8)  # converged in FP64
    assert np.max(np.abs(u.astype(np.float64) - lim)) <= 1e-5
    assert res[-1] < 1e-4


def test_jacobi_until_stops_at_the_first_checkpoint_below_tol():
    h, w, ce = 33, 29, 10
    u0 = synth.jacobi_init_f32(91, h, w)
    _, rres = oracle.jacobi2d(u0, 200, ce)
    m = 4  # stop after 40 sweeps: tol between the 3rd and 4th checkpoint residuals
    tol = float(np.sqrt(rres[m - 2] * rres[m - 1]))
    d = to_dev(u0)
    wsb = pg.pencil_jacobi2d_workspace_size(h, w)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev())
    res = torch.full((20,), -1.0, dtype=torch.float64, device=dev())
    done = pg.pencil_jacobi2d_until(h, w, d, 200, ce, tol, res, ws, wsb)
    assert done == m * ce
    ref, _ = run_jacobi(u0, done, 0)
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    r = res.cpu().numpy()
    assert r[m - 1] <= tol < r[m - 2] and np.all(r[m:] == -1.0)
    # tol 0 runs every sweep; a huge tol stops at the first checkpoint
    d2 = to_dev(u0)
    assert pg.pencil_jacobi2d_until(h, w, d2, 50, ce, 0.0, res, ws, wsb) == 50
    d3 = to_dev(u0)
    assert pg.pencil_jacobi2d_until(h, w, d3, 50, ce, 1e30, res, ws, wsb) == ce


def test_sor_until_converges_in_fewer_sweeps_than_jacobi():
    h = w = 65
    u0 = synth.jacobi_init_f32(93, h, w)
    tol, ce, cap = 1e-3, 5, 4000
    wsb = max(pg.pencil_jacobi2d_workspace_size(h, w), pg.pencil_rbsor2d_workspace_size(h, w))
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev())
    res = torch.zeros(cap // ce, dtype=torch.float64, device=dev())
    ds = to_dev(u0)
    n_sor = pg.pencil_rbsor2d_until(h, w, ds, cap, 1.9, ce, tol, res, ws, wsb)
    rs = res.cpu().numpy()
    assert 0 < n_sor < cap and rs[n_sor // ce - 1] <= tol
    if n_sor > ce:
        assert rs[n_sor // ce - 2] > tol
    ref, _ = run_sor(u0, n_sor, 1.9, 0)
    np.testing.assert_array_equal(ds.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    dj = to_dev(u0)
    n_jac = pg.pencil_jacobi2d_until(h, w, dj, cap, ce, tol, res, ws, wsb)
    assert n_sor * 5 < n_jac


def test_iterative_argument_errors():
    u = torch.zeros(16, 16, device=dev())
    wsb = pg.pencil_jacobi2d_workspace_size(16, 16)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev())
    res = torch.zeros(4, dtype=torch.float64, device=dev())
    for args in ((16, 16, u, 10, 0, 1e-3, res, ws, wsb), (16, 16, u, 15, 10, 1e-3, res, ws, wsb),
                 (16, 16, u, 10, 5, -1.0, res, ws, wsb)):
        with pytest.raises(pg.PencilError) as e:
            pg.pencil_jacobi2d_until(*args)
        assert e.value.name == "PENCIL_ERR_ARG"
    for omega in (0.0, 2.0, -1.0):
        with pytest.raises(pg.PencilError) as e:
            pg.pencil_rbsor2d_ex(16, 16, u, 5, omega, 0, None, ws, wsb)
        assert e.value.name == "PENCIL_ERR_ARG"


@pytest.mark.parametrize("omega", [1.0, 1.7])
def test_sor_tiles_equal_the_scalar_kernel_and_any_split(omega):
    """Aligned grids run SOR as register tiles of up to 5 sweeps per pass (halo
    2T); a grid that starts 4 bytes off a 16-byte boundary takes the one-colour
    scalar kernels.  Both apply the same expression in the same colour order,
    so the iterates are the same bits, and so are runs split into several calls."""
    h, w = 300, 264
    u0 = synth.jacobi_init_f32(5, h, w)
    a, _ = run_sor(u0, 23, omega, 0)
    buf = torch.zeros(h * w + 1, dtype=torch.float32, device=dev())
    d = buf[1:].view(h, w)
    d.copy_(torch.from_numpy(u0))
    wsb = pg.pencil_rbsor2d_workspace_size(h, w)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev())
    pg.pencil_rbsor2d_ex(h, w, d, 23, omega, 0, None, ws, wsb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), a.view(np.uint32))
    e = to_dev(u0)
    for n in (1, 7, 15):
        pg.pencil_rbsor2d_ex(h, w, e, n, omega, 0, None, ws, wsb)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(e.cpu().numpy().view(np.uint32), a.view(np.uint32))
