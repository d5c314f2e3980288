"""The cooperative launches of the homogeneous chain against the separate launches.

A single-column window on a periodic operator (every link of the homogeneous chain) runs its
three shift-and-invert passes as one grid-synchronised launch, and the four Gram-Schmidt
passes with their two Cholesky QRs as another (the separate launches fold the QRs and the
h1 sums into the passes, 4 launches).  They keep the chunking and the fixed-order
partial sums of the separate kernels, so the outputs must agree bit for bit with the run
that PEXP_DIAG_NOCOOP forces onto the separate launches; the launch count shows that the
cooperative path ran.
"""
import numpy as np
import pytest

from gpu_util import ctx
from paper_1509_04567_gb300 import pexp
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


def _solve(c, pr, opts, prec):
    import torch
    dt = torch.float32 if prec else torch.float64
    Y = torch.zeros((opts["n_out"], pr.n), dtype=dt, device="cuda")
    G = torch.from_numpy(pr.G).to("cuda", dt)
    rep = c.solve_linear(pr.op, opts, torch.from_numpy(pr.u0).cuda(), G, Y)
    torch.cuda.synchronize()
    return Y.cpu(), rep


@pytest.mark.parametrize("prec,n,P,tol", [(1, 1 << 16, 16, 1e-7), (0, 1 << 14, 8, 1e-10), (1, 5000, 7, 1e-7)],
                         ids=["mixed_2p16", "fp64_2p14", "mixed_ragged"])
def test_cooperative_chain_is_bitwise_the_separate_launches(c, prec, n, P, tol):
    import torch
    pr = wl.adv_diff_1d(n=n, nu=1e-3, a=1.0, T=1.0, P=P, n_out=16 * P + 1, tol=tol, svd_tol=1e-10, max_rank=8,
                        restart_len=30)
    opts = dict(pr.opts, precision=prec)
    Y1, r1 = _solve(c, pr, opts, prec)
    Y2, r2 = _solve(c, pr, dict(opts, diagnostics=pexp.DIAG_NOCOOP), prec)
    assert r1["rc"] == 0 and r2["rc"] == 0, (r1["rc"], r2["rc"])
    assert torch.equal(Y1, Y2)
    assert r1["k_hom_sum"] == r2["k_hom_sum"] and r1["k_nh_max"] == r2["k_nh_max"]
    # each chain step: 5 launches instead of 9 (SAI 1 + 3, part B 1 + 4)
    assert r1["launches"] <= r2["launches"] - 3 * r1["k_hom_sum"], (r1["launches"], r2["launches"], r1["k_hom_sum"])
    assert np.isfinite(Y1.double().numpy()).all()


def test_grid_barrier_wait_is_bounded_and_the_context_survives(c):
    """The barrier of the cooperative launches gives up after about 1 s when a CTA never
    arrives (here one CTA of a self-test launch leaves at once): the call returns
    ERR_TIMEOUT, the kernel ends, and the same context then solves as before."""
    import time
    import torch
    assert c.selftest_barrier(-1) == pexp.OK
    t0 = time.time()
    rc = c.selftest_barrier(3)
    dt = time.time() - t0
    assert rc == pexp.ERR_TIMEOUT, rc
    assert dt < 10.0, dt
    assert c.selftest_barrier(-1) == pexp.OK   # the barrier words were reset
    pr = wl.adv_diff_1d(n=1 << 14, nu=1e-3, a=1.0, T=1.0, P=8, n_out=65, tol=1e-7, svd_tol=1e-10, max_rank=8,
                        restart_len=30)
    opts = dict(pr.opts, precision=1)
    Y1, r1 = _solve(c, pr, opts, 1)
    Y2, r2 = _solve(c, pr, dict(opts, diagnostics=pexp.DIAG_NOCOOP), 1)
    assert r1["rc"] == 0 and torch.equal(Y1, Y2)
