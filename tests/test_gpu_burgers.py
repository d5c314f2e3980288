"""Burgers waveform relaxation (Sec. 2.3-2.4, Fig. 5) through the C ABI against the
FP64 CPU oracle on the same inputs: Picard (eq. ivp3) in FP64 and mixed precision, and
the divergence status on a case where the Picard updates grow.

Gates: FP64 1e-9 (both sides converge the WR to 1e-11 and the Krylov solves to 1e-13);
mixed 1e-6 (the metric's bar for the mixed path)."""
import numpy as np
import pytest

import oracle.pebk as ob
from gpu_util import ctx, relerr_rows
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


def _run(c, op, opts, u0, dtype):
    import torch
    dt = torch.float64 if dtype == "f64" else torch.float32
    U = torch.zeros((opts["n_out"], op["nx"]), dtype=dt, device="cuda")
    rep = c.solve_burgers(op, opts, torch.from_numpy(u0).cuda(), U)
    torch.cuda.synchronize()
    return U.double().cpu().numpy(), rep


def test_picard_fp64_n4096_p8(c):
    """The Burgers viscosity of the 65536-point workload on 4096 points, 8 subintervals."""
    n = 4096
    op = wl.make_op(n, 5e-3, 0.0)
    u0 = 0.5 + np.sin(2 * np.pi * wl.grid_1d(n))
    # svd_tol 1e-7: the FP64 floor of the GPU's Gram-based source SVD (singular values below
    # ~1e-7 sigma_1 are not resolved there), taken by both sides
    opts = wl.default_opts(T=0.04, P=8, n_out=81, tol=1e-13, svd_tol=1e-7, max_rank=16, wr_tol=1e-11,
                           wr_max_iter=40, restart_len=40)
    Uref, rref = ob.solve_burgers(op, opts, u0)
    assert rref["converged"], rref["deltas"]
    U, rep = _run(c, op, opts, u0, "f64")
    assert rep["rc"] == 0, rep
    assert abs(rep["wr_iters"] - rref["iters"]) <= 1, (rep["wr_iters"], rref["iters"])
    assert relerr_rows(U, Uref) < 1e-9
    hist = rep["wr_history"][:rep["wr_iters"]]
    assert hist[-1] <= opts["wr_tol"] and hist[0] > hist[-1]
    assert all(r >= 1 for r in rep["sub_rank"][:8])


def test_picard_mixed_precision(c):
    """Mixed path: FP32 iterates, sources and bases, FP64 small matrices."""
    n = 256
    op = wl.make_op(n, 5e-2, 0.0)
    u0 = 0.5 + np.sin(2 * np.pi * wl.grid_1d(n))
    opts = wl.default_opts(T=0.1, P=4, n_out=41, tol=1e-13, svd_tol=1e-13, max_rank=16, wr_tol=1e-11,
                           wr_max_iter=60, restart_len=40)
    Uref, rref = ob.solve_burgers(op, opts, u0)
    assert rref["converged"]
    mopts = dict(opts, precision=1, tol=1e-8, svd_tol=1e-7, wr_tol=1e-7, wr_max_iter=40, wr_diverge=0)
    U, rep = _run(c, op, mopts, u0, "f32")
    assert rep["rc"] in (0, -6), rep   # the FP32 update may floor near 1e-7
    err = relerr_rows(U, Uref)
    assert err < 1e-6, err
    # the conservative form keeps the mean of u0 (0.5) up to FP32 rounding
    np.testing.assert_allclose(U.mean(axis=1), 0.5, atol=1e-6)


def test_picard_divergence_status(c):
    """T = 0.3, nu = 1e-2: the Picard updates grow; both sides stop after the same number of
    iterations, at the third growth in a row, and return the last iterate."""
    n = 64
    op = wl.make_op(n, 1e-2, 0.0)
    u0 = 0.5 + np.sin(2 * np.pi * wl.grid_1d(n))
    opts = wl.default_opts(T=0.3, P=4, n_out=41, tol=1e-13, svd_tol=1e-13, max_rank=16, wr_tol=1e-10,
                           wr_max_iter=30, restart_len=40, wr_diverge=3)
    Uref, rref = ob.solve_burgers(op, opts, u0)
    assert rref["diverged"] and not rref["converged"], rref["deltas"]
    from paper_1509_04567_gb300 import pexp
    U, rep = _run(c, op, opts, u0, "f64")
    assert rep["rc"] == pexp.ERR_WR_DIVERGED, rep["rc"]
    assert rep["wr_iters"] == rref["iters"], (rep["wr_iters"], rref["iters"])
    np.testing.assert_allclose(rep["wr_history"][:rep["wr_iters"]], rref["deltas"], rtol=1e-6)
    assert relerr_rows(U, Uref) < 1e-6
