"""Chebyshev sample nodes (Sec. 3: the source is sampled at Chebyshev points of every
subinterval) on the GPU, through the C ABI, against the FP64 CPU oracle on the same
seeded inputs: the source samples come from the Chebyshev points, the spline's knots are
not the output times, and the outputs stay on the uniform grid.

Tolerances as the other parity tests: FP64 path 1e-10, mixed path 1e-6 (max over the output
times of the relative 2-norm error)."""
import numpy as np
import pytest

import oracle.pebk as ob
from gpu_util import ctx, relerr_rows, run_linear
from paper_1509_04567_gb300 import pexp
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


def _case(n_samp, n=1024, P=8, n_out=101, **kw):
    return wl.adv_diff_1d(n=n, P=P, n_out=n_out, tol=1e-12, restart_len=30, nodes=1, n_samp=n_samp, **kw)


@pytest.mark.parametrize("n_samp", [2, 3, 4, 7, 13, 17])
def test_chebyshev_fp64_matches_oracle(c, n_samp):
    """P = 8 over 101 outputs (subintervals of 13 and 14 outputs); 2 and 3 samples give the
    line and the parabola, 4 the single cubic, more the not-a-knot spline."""
    pr = _case(n_samp)
    Yref = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)[0]
    Y, rep = run_linear(c, pr)
    assert rep["rc"] == 0, rep
    assert relerr_rows(Y, Yref) < FP64_TOL


def test_chebyshev_mixed_matches_oracle(c):
    pr = _case(13)
    Yref = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)[0]
    Y, rep = run_linear(c, pr, dict(pr.opts, precision=1, tol=1e-7), dtype="f32")
    assert relerr_rows(Y, Yref) < MIXED_TOL, rep


def test_chebyshev_ragged_partition_and_host_entry(c):
    """P = 7 over 50 outputs (ragged subintervals), 9 samples each; the host-buffer entry
    gives the device entry's result bit for bit."""
    pr = wl.adv_diff_1d(n=2000, nu=5e-3, P=7, n_out=50, T=0.5, tol=1e-12, restart_len=30, nodes=1, n_samp=9)
    assert pr.G.shape == (7 * 8 + 1, 2000)
    Yref = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)[0]
    Y, rep = run_linear(c, pr)
    assert relerr_rows(Y, Yref) < FP64_TOL, rep
    Yh = np.zeros((pr.opts["n_out"], pr.n))
    rh = c.solve_linear_host(pr.op, pr.opts, pr.u0, np.ascontiguousarray(pr.G), Yh)
    assert rh["rc"] == 0
    assert np.array_equal(Yh, Y)


def test_chebyshev_option_checks(c):
    """n_samp outside 2 .. PEXP_MAX_SAMPLES is rejected with nothing written; waveform
    relaxation (samples at the iterate's output times) does not take Chebyshev samples."""
    import torch
    pr = _case(13, n=256)
    dev = torch.device("cuda:0")
    y0 = torch.from_numpy(pr.u0).to(dev)
    Y = torch.full((pr.opts["n_out"], pr.n), 7.0, dtype=torch.float64, device=dev)
    for bad in (1, 113):
        opts = dict(pr.opts, n_samp=bad)
        G = torch.zeros((pexp.source_rows(opts), pr.n), dtype=torch.float64, device=dev)
        rep = c.solve_linear(pr.op, opts, y0, G, Y, check=False)
        assert rep["rc"] == pexp.ERR_INVALID_ARG
    assert bool(torch.all(Y == 7.0))
    bop = wl.make_op(256, 5e-3)
    U = torch.zeros((pr.opts["n_out"], 256), dtype=torch.float64, device=dev)
    rep = c.solve_burgers(bop, dict(pr.opts, P=4, wr_max_iter=2), y0, U, check=False)
    assert rep["rc"] == pexp.ERR_UNSUPPORTED
