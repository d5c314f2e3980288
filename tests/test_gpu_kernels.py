"""GPU kernel parity: each kernel-level C-ABI call against the oracle's step or a
library reference of the same operation, element by element."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle.pebk as ob
from gpu_util import ctx
from paper_1509_04567_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    cc = ctx()
    yield cc
    cc.close()


OPS = [
    wl.make_op(1000, 1e-2, 1.0),                         # ragged: not a multiple of any tile
    wl.make_op(4096, 1e-3, -0.7),
    wl.make_op(1 << 20, 1e-3, 1.0),                      # the large advection-diffusion mesh
    wl.make_op(333, 2e-2, 0.5, bc=wl.BC_DIRICHLET0),
    wl.make_op(48, 1e-2, 1.0, dim=2, ny=37, ay=-0.5),    # 2D five-point
    wl.make_op(3, 1e-1, 0.2),                            # smallest mesh
]


@pytest.mark.parametrize("op", OPS, ids=lambda o: f"d{o['dim']}n{o['nx']}x{o['ny']}bc{o['bc']}")
@pytest.mark.parametrize("transpose", [0, 1])
def test_stencil_fp64_matches_oracle_matrix(c, op, transpose):
    import torch
    n = op["nx"] * (op["ny"] if op["dim"] == 2 else 1)
    X = wl.random_block(n, 3, 11).T.copy()   # 3 vectors, row-major (vec, n)
    A = ob.operator_matrix(op)
    ref = (A.T if transpose else A) @ X.T
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    c.apply_operator(op, Xd, Yd, transpose=bool(transpose))
    got = Yd.cpu().numpy().T
    scale = np.abs(A).sum(axis=1).max() * np.abs(X).max()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * scale)


def test_stencil_fp32_smooth_data_relative_accuracy(c):
    """FP32 stencil in difference form: error relative to the (small) result for smooth data."""
    import torch
    op = wl.make_op(1 << 16, 1e-3, 1.0)
    X = wl.smooth_block(1 << 16, 2, 3).T.copy()
    ref = (ob.operator_matrix(op) @ X.T).T
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Yd = torch.empty_like(Xd)
    c.apply_operator(op, Xd, Yd)
    ref32 = (ob.operator_matrix(op) @ X.astype(np.float32).astype(np.float64).T).T
    got = Yd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref32) <= 1e-5 * np.linalg.norm(ref32)


SAI_CASES = [
    (wl.make_op(1000, 1e-2, 1.0), 0.0125),
    (wl.make_op(2049, 1e-3, 1.0), 1.5e-3),
    (wl.make_op(1 << 20, 1e-3, 1.0), 1.0 / 640),       # large mesh, pole of the 64-subinterval case
    (wl.make_op(5000, 1e-4, 2.0), 0.01),               # cell Peclet > 1: negative factor root
    (wl.make_op(100, 1e-1, 0.0), 0.05),                # one chunk, weak damping around the circle
    (wl.make_op(70000, 1e-6, 0.0), 1e-3),              # weak diffusion: slow decay across chunks
]


@pytest.mark.parametrize("op,gamma", SAI_CASES, ids=lambda v: str(v) if not isinstance(v, dict) else f"n{v['nx']}")
def test_sai_solve_fp64_matches_sparse_lu(c, op, gamma):
    import torch
    n = op["nx"]
    X = np.vstack([wl.random_block(n, 1, 5)[:, 0], wl.smooth_block(n, 1, 6)[:, 0]])
    kop = ob.KrylovOperator(op, ob.operator_matrix(op), 1, gamma)
    ref = kop.build(X.T).T
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.empty_like(Xd)
    c.sai_solve(op, gamma, Xd, Yd)
    got = Yd.cpu().numpy()
    # (I - gamma A) has condition ~ 1 + 4 gamma nu/dx^2: forward errors of any
    # backward-stable solver (the sparse LU reference included) scale with it
    M = (ob.operator_matrix(op) * (-gamma))
    M = M + __import__("scipy.sparse", fromlist=["identity"]).identity(n)
    cond = 1.0 + 4.0 * gamma * op["nu"] * n * n
    for r in range(2):
        res = np.linalg.norm(M @ got[r] - X[r])
        assert res <= 1e-15 * cond * (np.linalg.norm(got[r]) + np.linalg.norm(X[r])), (r, res)
        assert np.linalg.norm(got[r] - ref[r]) <= 2e-15 * cond * np.linalg.norm(ref[r]), r


def test_sai_solve_fp32(c):
    import torch
    op = wl.make_op(1 << 20, 1e-3, 1.0)
    gamma = 1.0 / 640
    X = wl.smooth_block(1 << 20, 2, 8).T.copy()
    kop = ob.KrylovOperator(op, ob.operator_matrix(op), 1, gamma)
    ref = kop.build(X.astype(np.float32).astype(np.float64).T).T
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Yd = torch.empty_like(Xd)
    c.sai_solve(op, gamma, Xd, Yd)
    got = Yd.cpu().numpy().astype(np.float64)
    for r in range(2):
        assert np.linalg.norm(got[r] - ref[r]) <= 2e-6 * np.linalg.norm(ref[r])


@pytest.mark.parametrize("N,scale", [(5, 1e-3), (12, 0.2), (20, 0.9), (33, 2.0), (48, 4.0), (64, 60.0), (100, 1e3)])
def test_small_expm_matches_library(c, N, scale):
    import torch
    rng = np.random.default_rng(N)
    M = rng.standard_normal((3, N, N))
    M *= scale / np.abs(M).sum(axis=1).max(axis=1)[:, None, None]
    M[1] -= 0.5 * scale * np.eye(N)
    Md = torch.from_numpy(M).cuda()
    Ed = torch.empty_like(Md)
    c.small_expm(Md, Ed)
    got = Ed.cpu().numpy()
    for b in range(3):
        ref = sla.expm(M[b])
        assert np.linalg.norm(got[b] - ref) <= 1e-12 * max(1.0, np.linalg.norm(ref)) * max(1.0, scale), b


@pytest.mark.parametrize("form", [0, 1])
def test_burgers_source_matches_oracle(c, form):
    import torch
    op = wl.make_op(777, 5e-3, 0.0)
    x = wl.grid_1d(777)
    U = np.vstack([0.5 + np.sin(2 * np.pi * x + s) for s in (0.0, 0.3, 1.1)])
    ref = ob.burgers_source(op, U, form)
    Ud = torch.from_numpy(U).cuda()
    Gd = torch.empty_like(Ud)
    c.burgers_source(op, Ud, Gd, form)
    np.testing.assert_allclose(Gd.cpu().numpy(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
