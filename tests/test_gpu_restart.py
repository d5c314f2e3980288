"""Restarted block Krylov cycles (Sec. 2.1 "implemented with restarting", Sec. 3 "restarted
every 20 iterations") on the GPU, through the C ABI, against the FP64 CPU oracle and the
circulant closed form on the same seeded inputs.

With max_restarts > 0 a window that has not converged after restart_len block steps of a
cycle starts a new cycle for the error of the cycles so far; the oracle takes the new
cycle's first block from an SVD of the residual factor (I - V V^T) A V, the GPU from the
shift-and-invert Arnoldi relation (or, in the polynomial space, the next block itself).
Tolerances: FP64 1e-10, mixed 1e-6 (max over the output times of the relative 2-norm error).
"""
import numpy as np
import pytest

import closed_forms as cf
import oracle.pebk as ob
from gpu_util import ctx, relerr_rows, run_linear
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


def _exact(pr, nu):
    t, wins = cf.fourier_windows_from_oracle_model(pr.op, pr.opts, pr.u0, pr.G, ob.compress_source,
                                                   ob.spline_segments, ob.partition)
    return cf.exact_piecewise_cubic(cf.circulant_eigs(pr.n, 1.0, nu), pr.u0, t, wins)


def test_restart_polynomial_space_fp64(c):
    """Cycles of 4 block steps in the polynomial space (18 steps without restarts)."""
    pr = wl.adv_diff_1d(n=128, nu=1e-3, P=4, n_out=33, T=0.25, tol=1e-12, restart_len=4, max_restarts=15,
                        krylov=0)
    Y, rep = run_linear(c, pr)
    assert rep["rc"] == 0, rep["rc"]
    assert min(rep["sub_restarts"][:4]) >= 2, rep["sub_restarts"][:4]
    Yo = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)[0]
    assert relerr_rows(Y, Yo) < 1e-10
    assert relerr_rows(Y, _exact(pr, 1e-3)) < 1e-10


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_restart_shift_and_invert_space(c, precision):
    """Cycles of 8 block steps in the shift-and-invert space on a case that needs 24 steps
    without restarts: every subproblem restarts, needs more than 40 block steps in all, and
    converges to the exact solution."""
    pr = wl.adv_diff_1d(n=1024, nu=1e-2, P=4, n_out=41, T=1.0, tol=1e-12, restart_len=8, max_restarts=7)
    Yx = _exact(pr, 1e-2)
    if precision == 0:
        Y, rep = run_linear(c, pr)
        assert rep["rc"] == 0, rep["rc"]
        assert min(rep["sub_restarts"][:4]) >= 2, rep["sub_restarts"][:4]
        assert rep["k_nh_max"] > 40, rep["k_nh_max"]
        Yo = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)[0]
        assert relerr_rows(Y, Yo) < 1e-10
        assert relerr_rows(Y, Yx) < 1e-10
    else:
        opts = dict(pr.opts, precision=1, tol=1e-7, restart_len=4, max_restarts=15, diagnostics=1)
        Y, rep = run_linear(c, pr, opts, dtype="f32")
        assert rep["rc"] == 0, rep["rc"]
        assert min(rep["sub_restarts"][:4]) >= 1, rep["sub_restarts"][:4]
        assert relerr_rows(Y, Yx) < 1e-6
        # every cycle's basis is orthonormal (cycles are not orthogonal to one another)
        assert 0.0 <= rep["orth_max"] <= 1e-6, rep["orth_max"]


def test_dense_projection_driver_mixed_precision(c):
    """max_restarts > 0 runs the dense-projection driver; with a cycle long enough that no
    restart happens, its mixed-precision solve meets the mixed gate like the fused kernels
    (its second Gram-Schmidt pass works on the block normalised by the first Cholesky QR)."""
    pr = wl.adv_diff_1d(n=1024, nu=1e-2, P=4, n_out=41, T=1.0, tol=1e-7, restart_len=32, max_restarts=1,
                        precision=1, diagnostics=1)
    Y, rep = run_linear(c, pr, dtype="f32")
    assert rep["rc"] == 0 and max(rep["sub_restarts"][:4]) == 0
    assert relerr_rows(Y, _exact(pr, 1e-2)) < 1e-6
    assert 0.0 <= rep["orth_max"] <= 1e-6, rep["orth_max"]
