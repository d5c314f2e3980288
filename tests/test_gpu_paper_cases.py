"""The paper's own validation cases through the C ABI.

* Table 1 (Sec. 3.2, eq. manusol): advection-diffusion with the manufactured travelling
  pulses, n = 1000, tol 1e-4, SVD rank m = 2.  The relative error at the final time is the
  serial error the paper prints, 3.05e-4, for every P in 2..32 (tests/golden/
  table1_pebk_serial_error.txt), in FP64 and in the mixed path; at P = 2 the GPU result
  also matches the oracle's on the same inputs (both at tol 1e-11).
* Sec. 4 travelling wave (eq. modifiedSawtooth, Fig. error_differentdx): the smoothed
  sawtooth moving at speed 1/2, forced by f = u_t + u u_x - nu u_xx, solved by the
  averaged-Jacobian waveform relaxation.  After a fixed number of iterations the GPU
  iterate equals the oracle's (both at Krylov tol 1e-12), and at the paper's tol 1e-4 its
  error against the manufactured solution falls by about 4 when dx is halved
  (second-order differences).
* Subintervals of up to 101 samples (Table 1 at P = 2): the source SVD's Jacobi sweep
  over more rows than its CTA has threads.
"""
import os

import numpy as np
import pytest

import oracle.pebk as ob
from gpu_util import ctx, relerr_rows, run_linear
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


@pytest.fixture(scope="module")
def table1():
    return {int(p): e for p, e in np.loadtxt(os.path.join(GOLDEN, "table1_pebk_serial_error.txt"))}


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("P", [2, 4, 8, 16, 32])
def test_table1_final_time_error(c, table1, P, precision):
    pr = wl.travelling_pulses(n=1000, T=1.0, P=P, n_out=201, tol=1e-4)
    Y, rep = run_linear(c, pr, dict(pr.opts, precision=precision), dtype="f32" if precision else "f64")
    assert rep["rc"] == 0, rep["rc"]
    assert all(r == 2 for r in rep["sub_rank"][:P]), rep["sub_rank"][:P]
    ex = pr.meta["exact"](1.0)
    err = np.linalg.norm(Y[-1] - ex) / np.linalg.norm(ex)
    assert abs(err - table1[P]) < 0.03 * table1[P], err
    if P == 2 and not precision:
        # the same inputs against the oracle, both at Krylov tol 1e-11 (at the paper's 1e-4
        # the two sides may stop one step apart)
        tight = dict(pr.opts, tol=1e-11, restart_len=40)
        Yo, _ = ob.solve_linear(pr.op, tight, pr.u0, pr.G)
        Y2, rep2 = run_linear(c, pr, tight)
        assert rep2["rc"] == 0, rep2["rc"]
        assert relerr_rows(Y2, Yo) < 1e-9


def _sawtooth(c, n, iters, tol=1e-4):
    import torch
    pr = wl.burgers_sawtooth(n=n, T=0.5, P=5, s=50, tol=tol, svd_tol=1e-6, wr_tol=1e-14, wr_max_iter=iters,
                             restart_len=40)
    opts = dict(pr.opts, jacobian=1, wr_diverge=0)
    U = torch.zeros((opts["n_out"], n), dtype=torch.float64, device="cuda")
    F = torch.from_numpy(pr.G).cuda()
    rep = c.solve_burgers(pr.op, opts, torch.from_numpy(pr.u0).cuda(), U, forcing=F)
    torch.cuda.synchronize()
    return pr, opts, U.cpu().numpy(), rep


def test_travelling_sawtooth_matches_oracle_iterate(c):
    # Krylov tol 1e-12 on both sides (the paper's 1e-4 leaves each side's stopping step, and
    # so its iterate, free to differ at the 1e-5 level); both cap the source rank at 12
    pr, opts, U, rep = _sawtooth(c, 64, 6, tol=1e-12)
    assert rep["wr_iters"] == 6, rep
    Uo, ro = ob.solve_burgers_jacobian(pr.op, opts, pr.u0, forcing=pr.G)
    assert ro["iters"] == 6
    np.testing.assert_allclose(rep["wr_history"][:6], ro["deltas"], rtol=1e-6)
    assert relerr_rows(U, Uo) < 1e-9


def test_travelling_sawtooth_error_is_second_order_in_dx(c):
    floors = []
    for n in (64, 128, 256):
        pr, _, U, rep = _sawtooth(c, n, 8)
        ex = pr.meta["exact"]
        floors.append(float(np.max(np.linalg.norm(U - ex, axis=1) / np.linalg.norm(ex, axis=1))))
    assert 3.2 < floors[0] / floors[1] < 5.0, floors
    assert 3.2 < floors[1] / floors[2] < 5.0, floors


def _multiscale(n, k0, P=2, s=33, T=0.2):
    """Sec. 4 multiscale example (eq. multiscale_solution) with the forcing built from the
    discrete operators, f = u_t - A u - g(u) at the grid points (the oracle's A and g, on the
    host), so that the semi-discrete solution is the exact one."""
    n_out = P * (s - 1) + 1
    t = wl.out_times(T, n_out)
    x = wl.grid_1d(n)
    op = wl.make_op(n, 1e-2, 0.0)
    A = ob.operator_matrix(op)
    U = np.zeros((n_out, n))
    F = np.zeros((n_out, n))
    for i, tt in enumerate(t):
        u, ut = wl.multiscale_solution(x, tt, k0)
        U[i] = u
        F[i] = ut - A @ u - ob.burgers_source(op, u, 0)
    return op, t, U, F


def _relerr_max(U, Uref):
    """max_i ||U_i - Uref_i|| / max_i ||Uref_i|| (the norm of the WR update; the solution is
    zero at t = 0, so row-wise relative errors are not defined there)."""
    return float(np.max(np.linalg.norm(U - Uref, axis=1)) / np.max(np.linalg.norm(Uref, axis=1)))


@pytest.mark.parametrize("k0", [4, 16])
def test_multiscale_burgers_matches_oracle_and_exact(c, k0):
    """The multiscale case on the GPU (averaged-Jacobian WR, FP64): after 4 iterations the
    iterate equals the oracle's (both at Krylov tol 1e-12 and svd_tol 1e-7, the FP64 path's
    singular-value floor), and after 8 its error against the exact solution is at the
    time-integration floor (< 1e-5, no spatial error), for the wide spectrum (k0 = 16) as
    for the narrow one."""
    import torch
    op, t, Uex, F = _multiscale(128, k0)
    opts = wl.default_opts(T=0.2, P=2, n_out=t.size, tol=1e-12, svd_tol=1e-7, max_rank=12, wr_tol=1e-14,
                           wr_max_iter=4, restart_len=40, jacobian=1, wr_diverge=0)
    Ft = torch.from_numpy(F).cuda()
    u0 = torch.from_numpy(Uex[0].copy()).cuda()
    U = torch.zeros((t.size, 128), dtype=torch.float64, device="cuda")
    rep = c.solve_burgers(op, opts, u0, U, forcing=Ft)
    torch.cuda.synchronize()
    assert rep["wr_iters"] == 4, rep
    Uo, ro = ob.solve_burgers_jacobian(op, opts, Uex[0].copy(), forcing=F)
    np.testing.assert_allclose(rep["wr_history"][:4], ro["deltas"], rtol=1e-6)
    assert _relerr_max(U.cpu().numpy(), Uo) < 1e-9
    opts8 = dict(opts, tol=1e-8, svd_tol=1e-10, wr_max_iter=8)
    rep = c.solve_burgers(op, opts8, u0, U, forcing=Ft)
    torch.cuda.synchronize()
    err = _relerr_max(U.cpu().numpy(), Uex)
    assert err < 1e-5, err
