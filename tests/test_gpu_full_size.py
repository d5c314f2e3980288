"""Whole-solve parity at the full size of the throughput workload: 1D periodic
advection-diffusion, n = 2^20, nu = 1e-3, P = 64 subintervals, 1025 output times.

The oracle's whole solve is too slow at this size, so two references are used.
* The exact semi-discrete solution (every Fourier mode integrated in closed form) of the
  problem with the oracle's own source model (thin SVD + not-a-knot spline per subinterval,
  Sec. 2.1), at sampled output times: interior points of early windows, window ends, and
  the final time, where the homogeneous chain of Sec. 2.2 is longest.  Inside the first
  subinterval only that window's Krylov truncation separates the two, and the FP64 path
  must be within 1e-10 there.  Later, the truncation errors of the windows before add up
  (each window stops once a step changes its answer by less than tol), so the FP64 bound
  at later times is 3 P tol.  The mixed path must meet its 1e-6 gate at every sample.
* The oracle itself on the first subinterval: compression, spline and the nonhomogeneous
  block Krylov solve give u(t_i) = u0 + V Y_i there.  At this stiffness
  (cond(I - gamma A) ~ 7e6) the oracle's own sparse-LU shift-and-invert solves leave it
  up to ~3e-10 from the exact solution, depending on the host's LU and BLAS, so the
  FP64 path must be within 1e-10 plus the oracle's own distance to the exact solution,
  and the mixed path within 1e-6.
The Krylov bases must be orthonormal to 1e-6 (mixed) and 1e-12 (FP64).
"""
import json
import os
import time

import numpy as np
import pytest

import closed_forms as cf
import oracle.pebk as ob
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

N, NU, A, P, NT, T = 1 << 20, 1e-3, 1.0, 64, 1025, 1.0
KEEP = [5, 16, 200, 511, 777, 1008, 1024]
FP64_TOL, MIXED_TOL = 1e-10, 1e-6
ORACLE_TOL = 1e-12
ORTH = {0: 1e-12, 1: 1e-6}


class _SourceRows:
    """g(x, t_i) = sin(4 pi x) cos(2 pi t_i), rows made on request (the whole source
    is 8.6 GB in FP64)."""

    def __init__(self, x, t):
        self.sx, self.t = np.sin(4 * np.pi * x), t

    def __getitem__(self, rows):
        return np.cos(2 * np.pi * self.t[rows])[:, None] * self.sx[None, :]


@pytest.fixture(scope="module")
def exact():
    x = wl.grid_1d(N)
    u0 = np.sin(2 * np.pi * x) + np.exp(-100.0 * (x - 0.5) ** 2)
    opts = wl.default_opts(T=T, P=P, n_out=NT, svd_tol=1e-10, max_rank=8)
    t = wl.out_times(T, NT)
    op = wl.make_op(N, NU, A)
    gen = cf.iter_windows_from_oracle_model(op, opts, u0, _SourceRows(x, t), ob.compress_source,
                                            ob.spline_segments, ob.partition)
    return cf.exact_at_samples(cf.circulant_eigs(N, A, NU), u0, t, gen, KEEP)


@pytest.fixture(scope="module")
def oracle_window1():
    """u0 + V Y_i on the first subinterval from the oracle's own steps (Sec. 2.1)."""
    x = wl.grid_1d(N)
    u0 = np.sin(2 * np.pi * x) + np.exp(-100.0 * (x - 0.5) ** 2)
    op = wl.make_op(N, NU, A)
    opts = wl.default_opts(T=T, P=P, n_out=NT, svd_tol=1e-10, max_rank=8)
    t = wl.out_times(T, NT)
    i0, i1 = ob.partition(NT, P)[:2]
    A_ = ob.operator_matrix(op)
    Ghat = (A_ @ u0)[:, None] + _SourceRows(x, t)[i0:i1 + 1].T
    U, C, _ = ob.compress_source(Ghat, opts["svd_tol"], opts["max_rank"])
    tau = t[i0:i1 + 1] - t[i0]
    kop = ob.KrylovOperator(op, A_, 1, opts["sai_gamma"] * T / P)
    V, Y, info = ob.ebk_nonhomogeneous(kop, U, tau, ob.spline_segments(tau, C), ORACLE_TOL,
                                       float(np.linalg.norm(u0)), 30)
    assert info["converged"], info
    return {k: u0 + V @ Y[k - i0] for k in KEEP if i0 < k <= i1}


@pytest.fixture(scope="module")
def c():
    from gpu_util import ctx
    cc = ctx()
    yield cc
    cc.close()


def _solve(c, precision, tol, restart_len):
    import torch
    dev = torch.device("cuda:0")
    dt = torch.float32 if precision else torch.float64
    x = torch.arange(N, dtype=torch.float64, device=dev) / N
    u0 = torch.sin(2 * np.pi * x) + torch.exp(-100.0 * (x - 0.5) ** 2)
    t = torch.arange(NT, dtype=torch.float64, device=dev) * (T / (NT - 1))
    G = (torch.cos(2 * np.pi * t)[:, None] * torch.sin(4 * np.pi * x)[None, :]).to(dt)
    Y = torch.empty((NT, N), dtype=dt, device=dev)
    opts = wl.default_opts(T=T, P=P, n_out=NT, tol=tol, svd_tol=1e-10, max_rank=8, precision=precision,
                           restart_len=restart_len, diagnostics=1)
    t0 = time.time()
    rep = c.solve_linear(wl.make_op(N, NU, A), opts, u0, G, Y, check=False)
    torch.cuda.synchronize()
    rows = Y[KEEP].double().cpu().numpy()
    del G, Y
    torch.cuda.empty_cache()
    return rows, rep, time.time() - t0


@pytest.mark.parametrize("precision,tol,restart_len", [(0, 1e-11, 30), (1, 1e-7, 20)], ids=["fp64", "mixed"])
def test_full_size_vs_oracle_and_exact(c, exact, oracle_window1, precision, tol, restart_len):
    rows, rep, wall = _solve(c, precision, tol, restart_len)
    got = dict(zip(KEEP, rows))

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    e_ex = {k: rel(got[k], exact[k]) for k in KEEP}
    e_or = {k: rel(got[k], v) for k, v in oracle_window1.items()}
    e_oe = {k: rel(v, exact[k]) for k, v in oracle_window1.items()}
    line = {"precision": ["fp64", "mixed"][precision], "tol": tol, "restart_len": restart_len, "rc": rep["rc"],
            "not_converged": rep["not_converged"], "k_nh_max": rep["k_nh_max"], "k_hom_max": rep["k_hom_max"],
            "wall_s": round(wall, 2), "orth_max": rep["orth_max"], "rank_max": rep["rank_max"],
            "rel_err_exact": {str(k): f"{e:.2e}" for k, e in e_ex.items()},
            "rel_err_oracle_window1": {str(k): f"{e:.2e}" for k, e in e_or.items()},
            "oracle_window1_vs_exact": {str(k): f"{e:.2e}" for k, e in e_oe.items()},
            "max_rel_err_exact": f"{max(e_ex.values()):.3e}",
            "margin_vs_gate": round((MIXED_TOL if precision else 3 * P * tol) / max(e_ex.values()), 3)}
    print(json.dumps(line))
    out = os.environ.get("PEXP_TEST_RECORD")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps(line) + "\n")
    assert rep["rc"] == 0, line
    assert rep["rank_max"] == 2
    assert 0 <= rep["orth_max"] <= ORTH[precision], rep["orth_max"]
    assert e_or, line
    if precision == 0:
        assert max(e_ex[k] for k in oracle_window1) < FP64_TOL, line
        assert max(e_ex.values()) < 3 * P * tol, line
        assert all(e_or[k] < FP64_TOL + e_oe[k] for k in e_or), line
    else:
        assert max(e_ex.values()) < MIXED_TOL, line
        assert max(e_or.values()) < MIXED_TOL, line
