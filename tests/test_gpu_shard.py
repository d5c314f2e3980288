"""The subinterval ranges that shard one solve over GPUs (sub_first / sub_last), on one
GPU: the ranges' partial solutions, summed, equal the one-call solve (Sec. 2.2, eq.
superposition), through the device and the host entry points."""
import numpy as np
import pytest

from gpu_util import ctx, relerr_rows, run_linear
from paper_1509_04567_gb300 import shard, workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


@pytest.mark.parametrize("precision,world", [(0, 2), (0, 3), (1, 4)], ids=["fp64-2", "fp64-3", "mixed-4"])
def test_ranges_sum_to_the_full_solve(c, precision, world):
    pr = wl.adv_diff_1d(n=4096, nu=2e-3, P=12, n_out=97, T=0.5, tol=1e-12 if precision == 0 else 1e-7, restart_len=30)
    dtype = "f32" if precision else "f64"
    opts = dict(pr.opts, precision=precision)
    Yfull, _ = run_linear(c, pr, opts, dtype=dtype)
    idx = shard.partition_boundaries(pr.opts["n_out"], pr.opts["P"])
    tot = np.zeros_like(Yfull)
    for r in range(world):
        a, b = shard.rank_range(pr.opts["P"], world, r)
        Yr, rep = run_linear(c, pr, dict(opts, sub_first=a, sub_last=b), dtype=dtype)
        assert rep["rc"] == 0
        if a > 0:
            assert not Yr[:idx[a] + 1].any()      # zero up to T_a (the range from 0 holds u0 at t = 0)
        tot += Yr
    assert relerr_rows(tot, Yfull) < (1e-6 if precision else 1e-10)


def test_range_through_the_host_entry(c):
    pr = wl.adv_diff_1d(n=2048, nu=2e-3, P=8, n_out=65, T=0.5, tol=1e-12, restart_len=30)
    opts = dict(pr.opts, sub_first=3, sub_last=6)
    Yd, _ = run_linear(c, pr, opts)
    Yh = np.full_like(Yd, np.nan)
    rep = c.solve_linear_host(pr.op, opts, pr.u0.copy(), pr.G.copy(), Yh)
    assert rep["rc"] == 0
    np.testing.assert_array_equal(Yh, Yd)


def test_invalid_ranges_are_rejected(c):
    import torch
    from paper_1509_04567_gb300 import pexp
    pr = wl.adv_diff_1d(n=64, P=4, n_out=9)
    y0 = torch.zeros(64, dtype=torch.float64, device="cuda")
    Y = torch.zeros((9, 64), dtype=torch.float64, device="cuda")
    for a, b in ((2, 2), (3, 1), (0, 5), (-1, 2)):
        rep = c.solve_linear(pr.op, dict(pr.opts, sub_first=a, sub_last=b), y0, None, Y, check=False)
        assert rep["rc"] == pexp.ERR_INVALID_ARG, (a, b)
