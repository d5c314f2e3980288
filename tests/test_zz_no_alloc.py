"""The allocation-free shift-and-invert entry point (pexp_sai_solve_noalloc).

It shares the kernels of pexp_sai_solve but keeps its scratch in a fixed device
array that every call reuses, so the GPU test makes two different calls in a row
(the second one sees the first one's leftovers) and checks both against
pexp_sai_solve through the C ABI.  Collected last, and passes alone or after the
other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1509_04567_gb300 import workloads as wl

# tolerances of the SAI kernel tests: the FP64 parity gate and the FP32 solve bound
TOL = {"f64": 1e-10, "f32": 2e-6}


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_sai_solve_on_two_calls(dtype):
    import torch
    from gpu_util import ctx
    from paper_1509_04567_gb300 import pexp
    c = ctx()
    dt = torch.float64 if dtype == "f64" else torch.float32
    calls = [  # (n, nvec, nu, a, gamma): ragged chunk counts, different sizes per call
        ((1 << 16) + 77, 3, 1e-3, 1.0, 1.0 / 640),
        (5000, 2, 5e-3, -0.5, 0.03),
    ]
    outs = []
    for n, nvec, nu, a, gamma in calls:
        op = wl.make_op(n, nu, a)
        X = torch.from_numpy(wl.random_block(n, nvec, n % 97).T.copy()).to("cuda:0", dt)
        Y = torch.full_like(X, float("nan"))
        pexp.sai_solve_noalloc(op, gamma, X, Y)
        outs.append((op, gamma, X, Y))
    torch.cuda.synchronize()
    for op, gamma, X, Y in outs:
        Yref = torch.empty_like(X)
        c.sai_solve(op, gamma, X, Yref)
        torch.cuda.synchronize()
        got, ref = Y.double().cpu().numpy(), Yref.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        for r in range(X.shape[0]):
            assert np.linalg.norm(got[r] - ref[r]) <= TOL[dtype] * np.linalg.norm(ref[r]), (op["nx"], r)


def test_noalloc_rejects_requests_beyond_its_scratch():
    """Host-side checks, made before any CUDA call (runs without a GPU)."""
    import __graft_entry__ as g
    g.build()
    from paper_1509_04567_gb300 import pexp
    L = pexp.lib()
    n = 1 << 20  # 512 chunks: 2 + 4*512 doubles per vector, 127 vectors fit in 2 MiB
    op = pexp.make_operator(wl.make_op(n, 1e-3, 1.0))
    fake_x, fake_y = ctypes.c_void_p(1 << 40), ctypes.c_void_p(1 << 41)
    rc = L.pexp_sai_solve_noalloc(ctypes.byref(op), 0.01, fake_x, fake_y, 128, pexp.F64, None)
    assert rc == pexp.ERR_SCRATCH_LIMIT
    assert "scratch" in pexp.status_string(rc)
    rc = L.pexp_sai_solve_noalloc(ctypes.byref(op), -1.0, fake_x, fake_y, 1, pexp.F64, None)
    assert rc == pexp.ERR_INVALID_ARG
    rc = L.pexp_sai_solve_noalloc(ctypes.byref(op), 0.01, fake_x, fake_x, 1, pexp.F64, None)
    assert rc == pexp.ERR_INVALID_ARG
