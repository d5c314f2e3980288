"""Whole-solve parity: the CUDA Paraexp-EBK path (through the C ABI) against the
FP64 CPU oracle on the same seeded inputs.

Tolerances: FP64 path 1e-10 and mixed path 1e-6 in max_i ||Y_i - Y_ref_i||/||Y_ref_i||,
with both sides run at a Krylov tolerance well below the bar."""
import numpy as np
import pytest

import oracle.pebk as ob
from gpu_util import ctx, relerr_rows, run_linear
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


def _oracle(pr, **kw):
    opts = dict(pr.opts)
    opts.update(kw)
    return ob.solve_linear(pr.op, opts, pr.u0, pr.G)[0]


def test_small_case_fp64(c):
    """n = 1024, P = 8 (ragged subintervals of 13/14 samples), 101 output times."""
    pr = wl.adv_diff_1d(n=1024, P=8, n_out=101, tol=1e-12, restart_len=30)
    Yref = _oracle(pr)
    Y, rep = run_linear(c, pr)
    assert rep["rc"] == 0, rep
    assert relerr_rows(Y, Yref) < FP64_TOL
    assert rep["rank_max"] == 2


def test_small_case_mixed(c):
    pr = wl.adv_diff_1d(n=1024, P=8, n_out=101, tol=1e-12, restart_len=30)
    Yref = _oracle(pr)
    opts = dict(pr.opts, precision=1, tol=1e-7)
    Y, rep = run_linear(c, pr, opts, dtype="f32")
    assert relerr_rows(Y, Yref) < MIXED_TOL, rep


@pytest.mark.parametrize("precision,gate", [(0, 1e-12), (1, 1e-6)], ids=["fp64", "mixed"])
def test_krylov_bases_orthonormal(c, precision, gate):
    """max over every block Krylov basis of max|V^T V - I|, measured on the device."""
    pr = wl.adv_diff_1d(n=1024, P=8, n_out=101, tol=1e-12, restart_len=30)
    opts = dict(pr.opts, precision=precision, tol=1e-7 if precision else 1e-12, diagnostics=1)
    Y, rep = run_linear(c, pr, opts, dtype="f32" if precision else "f64")
    assert rep["rc"] == 0, rep
    assert 0.0 <= rep["orth_max"] <= gate, rep["orth_max"]


@pytest.mark.parametrize("P,n_out", [(1, 17), (3, 40), (7, 50), (16, 33)])
def test_partitions_fp64(c, P, n_out):
    pr = wl.adv_diff_1d(n=2000, nu=5e-3, P=P, n_out=n_out, T=0.5, tol=1e-12, restart_len=30)
    Yref = _oracle(pr)
    Y, rep = run_linear(c, pr)
    assert relerr_rows(Y, Yref) < FP64_TOL, rep


def test_zero_source(c):
    pr = wl.adv_diff_1d(n=512, P=4, n_out=21, tol=1e-12, restart_len=30, with_source=False)
    Yref = _oracle(pr)
    Y, rep = run_linear(c, pr)
    assert relerr_rows(Y, Yref) < FP64_TOL, rep
    assert rep["rank_max"] == 1


def test_polynomial_krylov_mildly_stiff(c):
    pr = wl.adv_diff_1d(n=128, nu=1e-3, P=4, n_out=33, T=0.25, tol=1e-12, restart_len=40, krylov=0)
    Yref = _oracle(pr)
    Y, rep = run_linear(c, pr)
    assert relerr_rows(Y, Yref) < FP64_TOL, rep


def test_polynomial_krylov_dirichlet_and_2d(c):
    n = 40
    x = wl.grid_1d(n, bc=wl.BC_DIRICHLET0)
    op = wl.make_op(n, 1e-2, 0.5, bc=wl.BC_DIRICHLET0)
    t = wl.out_times(0.5, 17)
    G = np.cos(3 * t)[:, None] * (x * (1 - x))[None, :]
    pr = wl.Problem("dirichlet", op, wl.default_opts(T=0.5, P=4, n_out=17, tol=1e-13, krylov=0, restart_len=40),
                    np.sin(np.pi * x) * (1 + x), G)
    Y, rep = run_linear(c, pr)
    assert relerr_rows(Y, _oracle(pr)) < FP64_TOL, rep
    nx, ny = 24, 20
    op2 = wl.make_op(nx, 5e-3, 1.0, dim=2, ny=ny, ay=0.5)
    X, Yg = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny)
    u0 = (np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Yg)).ravel()
    t = wl.out_times(0.25, 9)
    G2 = np.cos(2 * np.pi * t)[:, None] * np.sin(2 * np.pi * (X + Yg)).ravel()[None, :]
    pr2 = wl.Problem("2d", op2, wl.default_opts(T=0.25, P=2, n_out=9, tol=1e-13, krylov=0, restart_len=40), u0, G2)
    Y2, rep2 = run_linear(c, pr2)
    assert relerr_rows(Y2, _oracle(pr2)) < FP64_TOL, rep2


def test_host_pointer_entry_matches_device_entry(c):
    pr = wl.adv_diff_1d(n=1024, P=8, n_out=101, tol=1e-10)
    Yd, _ = run_linear(c, pr)
    Yh = np.zeros_like(Yd)
    rep = c.solve_linear_host(pr.op, pr.opts, pr.u0.copy(), pr.G.copy(), Yh)
    assert rep["rc"] == 0
    np.testing.assert_array_equal(Yh, Yd)


def test_invalid_arguments_are_rejected(c):
    import torch
    from paper_1509_04567_gb300 import pexp
    pr = wl.adv_diff_1d(n=64, P=4, n_out=9)
    y0 = torch.zeros(64, dtype=torch.float64, device="cuda")
    Y = torch.zeros((9, 64), dtype=torch.float64, device="cuda")
    for bad in (dict(P=9), dict(n_out=1), dict(tol=0.0), dict(restart_len=100), dict(krylov=5)):
        rep = c.solve_linear(pr.op, dict(pr.opts, **bad), y0, None, Y, check=False)
        assert rep["rc"] == pexp.ERR_INVALID_ARG, bad
    # the shift-and-invert space needs a 1D operator (periodic or bounded)
    op_2d = wl.make_op(8, 1e-2, 0.5, dim=2, ny=8)
    rep = c.solve_linear(op_2d, dict(pr.opts, krylov=1), y0, None, Y, check=False)
    assert rep["rc"] == pexp.ERR_UNSUPPORTED


def test_burgers_waveform_relaxation_fp64(c):
    import torch
    n = 256
    op = wl.make_op(n, 5e-2, 0.0)
    x = wl.grid_1d(n)
    u0 = 0.5 + np.sin(2 * np.pi * x)
    opts = wl.default_opts(T=0.1, P=4, n_out=41, tol=1e-13, svd_tol=1e-13, max_rank=16, wr_tol=1e-10,
                           wr_max_iter=60, restart_len=40)
    Uref, rref = ob.solve_burgers(op, opts, u0)
    U = torch.zeros((41, n), dtype=torch.float64, device="cuda")
    rep = c.solve_burgers(op, opts, torch.from_numpy(u0).cuda(), U)
    assert rep["rc"] == 0, rep
    assert relerr_rows(U.cpu().numpy(), Uref) < 1e-9, (rep, rref["iters"])
