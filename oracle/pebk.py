"""Oracle: the PEBK method step by step in FP64 on the CPU (test infrastructure only).

Paper: G.L. Kooij, M.A. Botchev, B.J. Geurts, "A block Krylov subspace
implementation of the time-parallel Paraexp method and its extension for
nonlinear partial differential equations", arXiv:1509.04567.

Readings of points the paper leaves open:
  * the projected IVP (the paper used MATLAB ode15s, Sec. 3) is solved exactly
    through the exponential of an augmented block matrix, which is exact for the
    piecewise-cubic source model;
  * "piecewise cubic polynomials" (Sec. 2.1, Sec. 3) = the not-a-knot cubic
    spline through the samples of each subinterval (a line / parabola for 2 / 3
    samples);
  * subinterval boundaries snap to the output grid: T_j = t_floor(j (n_out-1) / P);
  * source samples: by default the output times inside each subinterval; with
    nodes=1 the s = n_samp Chebyshev points of each subinterval (Sec. 3), read as the
    Chebyshev extrema T_{j-1} + dT_j (1 - cos(pi i/(s-1)))/2, i = 0..s-1, so that both
    ends are samples (shared by neighbouring subintervals) and the cubic spline through
    them covers the whole subinterval; the projected solution is then evaluated at the
    output times, from the state at the knot before each one;
  * the Krylov space is either the polynomial block Krylov space of eq.
    blockKrylovSubspace (krylov=0) or its shift-and-invert form (krylov=1,
    Sec. 2.1, the acceleration the paper cites);
    in both cases the projected matrix is the Galerkin matrix V^T A V; the pole is
    gamma = sai_gamma * T / P for every window;
  * a subproblem is converged when the change of the projected solution between
    two successive block steps, max over the window's sample times, is at most
    tol * max(||u0||, max ||v(t_i)||);
  * the homogeneous part of subproblem j on [T_j, T] (Fig. 3) is integrated
    window by window on the same subinterval grid, a new Krylov space per window
    (time stepping of the exponential, the restarting device the paper cites);
  * the Burgers nonlinearity u u_x is discretised in conservative central form
    -(u_{i+1}^2 - u_{i-1}^2)/(4 dx) (burgers_form=0) or advective central form
    -u_i (u_{i+1} - u_{i-1})/(2 dx) (burgers_form=1); waveform relaxation is plain
    Picard iteration (eq. ivp3) stopped on the relative update
    max_i ||u_{k+1}(t_i) - u_k(t_i)|| / max_i ||u_{k+1}(t_i)|| <= wr_tol, or once that
    update has grown in wr_diverge (default 3) successive iterations (divergence; the
    paper states no rule for it).
  * restarting ("restarted every 20 iterations", Sec. 3): with max_restarts = 0 the Krylov
    space grows up to restart_len block steps; with max_restarts > 0 a subproblem that has
    not converged after restart_len block steps of a cycle starts a new cycle that solves
    for the error of the cycles so far.  In a restart cycle the error estimate is the larger
    of the step-to-step change and the size of the cycle's own part of the solution, and it
    is not tested at the cycle's first step: there the new direction alone barely moves the
    solution, and both quantities are far below the error (measured: 4e-7 against 6e-5);
    from the second step of a cycle on the estimate exceeds the error;  That error e obeys e' = A e + r(t) with the
    residual r(t) = (A V_c - V_c H_c) y_c(t) of the cycle's Galerkin solution, whose spatial
    factor (I - V_c V_c^T) A V_c has rank b (the block width): the new cycle's Krylov space
    starts from its range, and its projected problem is coupled to the previous cycle's
    through Q^T A V_c, so that all cycles together form one block lower-triangular projected
    system, solved exactly as one (restart_len (max_restarts + 1) block steps at most);
  * the averaged-Jacobian waveform relaxation (eq. ivp4 with the per-subinterval
    average of eq. piecewiseJac) averages over each subinterval by the trapezoidal
    rule on its samples; the Jacobian is linear in the state for the quadratic
    Burgers term, so this is the Jacobian of the averaged iterate.  Its shifted
    source (eq. sourceParallel) is read as A u0 + g_k - J_k u_hat_k: the printed
    +J_k u0 would move the fixed point.

Parity pins: see tests/test_oracle_pins.py (closed forms, dense brute force,
invariants).  No function here is "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.interpolate as si
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BC_PERIODIC = 0
BC_DIRICHLET0 = 1
KRYLOV_POLY = 0
KRYLOV_SAI = 1
NODES_UNIFORM = 0
NODES_CHEBYSHEV = 1


# --------------------------------------------------------------------------------------
# Spatial discretisation (method of lines, Sec. 2.1 eq. ivp2; Sec. 3.1 eq. ivpAdvDifEq)
# --------------------------------------------------------------------------------------
def _mesh_width(n: int, L: float, bc: int) -> float:
    return L / n if bc == BC_PERIODIC else L / (n + 1)


def _matrix_1d(n: int, a: float, nu: float, L: float, bc: int) -> sp.csr_matrix:
    """Second-order central differences of -a u_x + nu u_xx on n points (Sec. 3.1):
    (A u)_i = nu (u_{i-1} - 2 u_i + u_{i+1}) / dx^2 - a (u_{i+1} - u_{i-1}) / (2 dx),
    indices taken mod n (periodic) or with zero ghost values (homogeneous Dirichlet)."""
    dx = _mesh_width(n, L, bc)
    rows, cols, vals = [], [], []
    for i in range(n):
        for off, c in ((-1, nu / dx ** 2 + a / (2 * dx)), (0, -2.0 * nu / dx ** 2),
                       (1, nu / dx ** 2 - a / (2 * dx))):
            j = i + off
            if bc == BC_PERIODIC:
                j %= n
            elif j < 0 or j >= n:
                continue
            rows.append(i)
            cols.append(j)
            vals.append(c)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def operator_matrix(op: dict) -> sp.csr_matrix:
    """The sparse matrix A of eq. ivp2 for the operator description `op`.

    1D: the three-point matrix above.  2D: the five-point sum A_x (x) I + I (x) A_y
    on an nx-by-ny mesh, unknown (ix, iy) stored at index iy * nx + ix."""
    if op["dim"] == 1:
        return _matrix_1d(op["nx"], op["ax"], op["nu"], op["Lx"], op["bc"])
    Ax = _matrix_1d(op["nx"], op["ax"], op["nu"], op["Lx"], op["bc"])
    Ay = _matrix_1d(op["ny"], op["ay"], op["nu"], op["Ly"], op["bc"])
    return (sp.kron(sp.identity(op["ny"]), Ax) + sp.kron(Ay, sp.identity(op["nx"]))).tocsr()


def apply_A(op: dict, X: np.ndarray, A: sp.csr_matrix | None = None) -> np.ndarray:
    """A X for a vector (n,) or a block (n, b)."""
    if A is None:
        A = operator_matrix(op)
    return A @ X


# --------------------------------------------------------------------------------------
# Time partition (Sec. 2.2) and source model (Sec. 2.1, eq. svd_appr)
# --------------------------------------------------------------------------------------
def partition(n_out: int, P: int) -> list[int]:
    """Grid indices of the subinterval boundaries 0 = T_0 < ... < T_P = T (Sec. 2.2),
    snapped to the output grid: idx_j = floor(j (n_out - 1) / P)."""
    if P < 1 or n_out - 1 < P:
        raise ValueError("need 1 <= P <= n_out - 1")
    idx = [(j * (n_out - 1)) // P for j in range(P + 1)]
    assert all(idx[j + 1] > idx[j] for j in range(P))
    return idx


def sample_partition(opts: dict):
    """Source sample times of the subintervals (Sec. 2.2, Sec. 3).

    Returns (ts, sidx): subinterval j's samples are ts[sidx[j-1] : sidx[j]+1] (both ends
    included, an end shared with the neighbour).  nodes=0 (default): the output times,
    sidx = partition(n_out, P).  nodes=1: s = n_samp Chebyshev extrema per subinterval
    [T_{j-1}, T_j], tau_i = dT_j (1 - cos(pi i / (s-1))) / 2, sidx[j] = j (s-1); "the sample
    points per subinterval are Chebyshev nodes" (Sec. 3).  The boundaries T_j are those of
    partition() in both cases."""
    T, P, n_out = opts["T"], opts["P"], opts["n_out"]
    t = np.arange(n_out) * (T / (n_out - 1))
    idx = partition(n_out, P)
    if opts.get("nodes", NODES_UNIFORM) == NODES_UNIFORM:
        return t, idx
    s = int(opts["n_samp"])
    if s < 2:
        raise ValueError("need n_samp >= 2")
    ts = np.zeros(P * (s - 1) + 1)
    for j in range(1, P + 1):
        a, b = t[idx[j - 1]], t[idx[j]]
        tau = (b - a) * (1.0 - np.cos(np.pi * np.arange(s) / (s - 1))) / 2.0
        ts[(j - 1) * (s - 1):j * (s - 1) + 1] = a + tau
        ts[(j - 1) * (s - 1)] = a
        ts[j * (s - 1)] = b
    return ts, [j * (s - 1) for j in range(P + 1)]


def compress_source(Ghat: np.ndarray, svd_tol: float, max_rank: int):
    """Thin SVD of the source samples and its truncation (Sec. 2.1).

    Ghat: (n, s) sample matrix [g(t_1) ... g(t_s)].  Keeps the m largest singular
    values with sigma_i > svd_tol * sigma_1 (at most max_rank).  Returns U (n, m)
    with orthonormal columns, the coefficient samples C = U^T Ghat (m, s) so that
    g(t_i) ~ U C[:, i], and all singular values."""
    Uf, sig, _ = np.linalg.svd(Ghat, full_matrices=False)
    if sig.size == 0 or sig[0] == 0.0:
        return Uf[:, :0], np.zeros((0, Ghat.shape[1])), sig
    m = int(np.sum(sig > svd_tol * sig[0]))
    m = max(1, min(m, max_rank))
    U = Uf[:, :m].copy()
    return U, U.T @ Ghat, sig


def spline_segments(tau: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Piecewise-cubic coefficient functions p(t) of eq. svd_appr (Sec. 2.1, Sec. 3).

    Not-a-knot cubic spline through (tau_i, C[:, i]) (a straight line for two samples, a
    parabola for three).  Returns coef of shape (s-1, 4, m) with
    p(tau_i + theta) = sum_l coef[i, l] theta^l on [tau_i, tau_{i+1}]."""
    s = tau.size
    m = C.shape[0]
    if m == 0:
        return np.zeros((s - 1, 4, 0))
    spl = si.CubicSpline(tau, C.T, bc_type="not-a-knot")
    coef = np.zeros((s - 1, 4, m))
    # scipy stores c[k, i] as the coefficient of (t - tau_i)^(3-k)
    for l in range(4):
        coef[:, l, :] = spl.c[3 - l]
    return coef


# --------------------------------------------------------------------------------------
# Block Krylov subspace (Sec. 2.1, eq. blockKrylovSubspace)
# --------------------------------------------------------------------------------------
@dataclass
class KrylovOperator:
    """The operator the block Krylov space is built with.

    krylov=0: A itself (polynomial space span{U, AU, A^2 U, ...}).
    krylov=1: the shift-and-invert operator (I - gamma A)^{-1} (Sec. 2.1 cites this
    acceleration), gamma = sai_gamma * window length; solves by sparse LU."""
    op: dict
    A: sp.csr_matrix
    krylov: int = KRYLOV_SAI
    gamma: float = 0.0
    _lu: object = field(default=None, repr=False)

    def __post_init__(self):
        if self.krylov == KRYLOV_SAI:
            n = self.A.shape[0]
            self._lu = spla.splu((sp.identity(n, format="csc") - self.gamma * self.A).tocsc())

    def build(self, X: np.ndarray) -> np.ndarray:
        if self.krylov == KRYLOV_POLY:
            return self.A @ X
        if X.ndim == 1:
            return self._lu.solve(X)
        return np.column_stack([self._lu.solve(np.ascontiguousarray(X[:, c])) for c in range(X.shape[1])])


def block_krylov_step(kop: KrylovOperator, V: np.ndarray, last: np.ndarray, defl_tol: float = 1e-10):
    """One block step: W = Op(last block), orthogonalise W against all basis vectors
    (modified Gram-Schmidt, two full passes), then orthonormalise the block by
    column-pivoted Householder QR.  Columns whose remaining norm is below
    defl_tol * (largest column norm of Op(last)) are dropped (block deflation).
    Returns the new orthonormal block (n, r), r possibly 0."""
    W = kop.build(last)
    if W.ndim == 1:
        W = W[:, None]
    pre = float(np.max(np.linalg.norm(W, axis=0))) if W.size else 0.0
    for _ in range(2):
        for c in range(V.shape[1]):
            v = V[:, c]
            W = W - np.outer(v, v @ W)
    if pre == 0.0:
        return W[:, :0]
    Q, R, _ = sla.qr(W, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    r = int(np.sum(d > defl_tol * pre))
    return Q[:, :r]


# --------------------------------------------------------------------------------------
# Projected problems
# --------------------------------------------------------------------------------------
def _cubic_step(H: np.ndarray, B: np.ndarray, y: np.ndarray, h: float, c: np.ndarray) -> np.ndarray:
    """y(theta = h) for y' = H y + B sum_l c_l theta^l from y(0) = y: the augmented-matrix
    exponential of projected_source_window over one step of length h."""
    K = H.shape[0]
    m = B.shape[1]
    M = np.zeros((K + 4 * m, K + 4 * m))
    M[:K, :K] = h * H
    M[:K, K:K + m] = h * B
    for l in range(3):
        M[K + l * m:K + (l + 1) * m, K + (l + 1) * m:K + (l + 2) * m] = np.eye(m)
    E = sla.expm(M)
    ynew = E[:K, :K] @ y
    for l in range(4):
        ynew = ynew + math.factorial(l) * h ** l * (E[:K, K + l * m:K + (l + 1) * m] @ c[l])
    return ynew


def projected_source_at(H: np.ndarray, B: np.ndarray, knots: np.ndarray, coef: np.ndarray,
                        t_eval: np.ndarray) -> np.ndarray:
    """Exact solution of y' = H y + B p(t), y(knots_0) = 0, at the times t_eval (offsets in
    [knots_0, knots_-1]), for a cubic spline p with arbitrary knots (Chebyshev samples).

    The state is carried from knot to knot (one augmented-matrix exponential per knot
    interval, as in projected_source_window); a time inside a knot interval is reached from
    the state at the knot before it with that interval's cubic.  Returns (len(t_eval), K)."""
    K = H.shape[0]
    s = knots.size
    ys = [np.zeros(K)]
    for r in range(s - 1):
        ys.append(_cubic_step(H, B, ys[r], knots[r + 1] - knots[r], coef[r]))
    Y = np.zeros((t_eval.size, K))
    scale = knots[-1] - knots[0]
    for q, te in enumerate(t_eval):
        # the knot interval [knots_r, knots_{r+1}) holding te; te at a knot takes its state
        r = int(np.searchsorted(knots, te, side="right")) - 1
        r = min(max(r, 0), s - 1)
        if abs(te - knots[r]) <= 1e-14 * scale:
            Y[q] = ys[r]
        else:
            Y[q] = _cubic_step(H, B, ys[r], te - knots[r], coef[min(r, s - 2)])
    return Y


def projected_source_window(H: np.ndarray, B: np.ndarray, tau: np.ndarray, coef: np.ndarray) -> np.ndarray:
    """Exact solution of y' = H y + B p(t), y(tau_0) = 0 at the sample times tau.

    On each sample interval p is the cubic sum_l c_l theta^l; with h = tau_{i+1} - tau_i
    the exponential of the augmented matrix
        M = [[h H, h B, 0, 0, 0], [0, 0, I, 0, 0], [0, 0, 0, I, 0], [0, 0, 0, 0, I], [0]*5]
    holds e^{hH} in its leading block and h phi_{l+1}(hH) B in block column l+1, so
    y(tau_{i+1}) = e^{hH} y(tau_i) + sum_l l! h^l [h phi_{l+1}(hH) B] c_l.
    Returns Y of shape (s, K)."""
    K = H.shape[0]
    m = B.shape[1]
    s = tau.size
    Y = np.zeros((s, K))
    y = np.zeros(K)
    for i in range(s - 1):
        h = tau[i + 1] - tau[i]
        M = np.zeros((K + 4 * m, K + 4 * m))
        M[:K, :K] = h * H
        M[:K, K:K + m] = h * B
        for l in range(3):
            M[K + l * m:K + (l + 1) * m, K + (l + 1) * m:K + (l + 2) * m] = np.eye(m)
        E = sla.expm(M)
        ynew = E[:K, :K] @ y
        for l in range(4):
            ynew = ynew + math.factorial(l) * h ** l * (E[:K, K + l * m:K + (l + 1) * m] @ coef[i, l])
        y = ynew
        Y[i + 1] = y
    return Y


def projected_homogeneous(H: np.ndarray, beta: float, tau: np.ndarray) -> np.ndarray:
    """y(tau) = exp(tau H) beta e_1 at the times tau (tau_0 = 0).  Returns (s, K)."""
    K = H.shape[0]
    e1 = np.zeros(K)
    e1[0] = beta
    return np.array([sla.expm(t * H) @ e1 for t in tau])


# --------------------------------------------------------------------------------------
# EBK on one window (Sec. 2.1) -- nonhomogeneous and homogeneous parts (Fig. 3)
# --------------------------------------------------------------------------------------
def _grow(kop, V, AV, new):
    V = np.hstack([V, new])
    AV = np.hstack([AV, kop.A @ new])
    return V, AV


def restart_block(Vc: np.ndarray, AVc: np.ndarray, width: int, rank_tol: float = 1e-10) -> np.ndarray:
    """First block of the next restart cycle (Sec. 2.1, Sec. 3 "restarted every 20
    iterations"; the residual-correction reading of the module docstring).

    The Galerkin solution V_c y_c(t) of a cycle leaves the residual r(t) = Z y_c(t) with
    Z = A V_c - V_c (V_c^T A V_c) = (I - V_c V_c^T) A V_c, of rank <= the block width in exact
    arithmetic.  Returns an orthonormal basis of its range: the left singular vectors of Z
    whose singular values exceed rank_tol * sigma_1, at most `width` of them."""
    Z = AVc - Vc @ (Vc.T @ AVc)
    Uz, sz, _ = np.linalg.svd(Z, full_matrices=False)
    if sz.size == 0 or sz[0] == 0.0:
        return Vc[:, :0]
    r = min(int(np.sum(sz > rank_tol * sz[0])), width)
    return Uz[:, :r]


def coupled_galerkin(V: np.ndarray, AV: np.ndarray, cyc: list, first: list) -> np.ndarray:
    """Projected matrix of the restarted method: the Galerkin blocks V_c^T A V_c of every
    cycle c on the diagonal, and the coupling Q_{c+1}^T A V_c of cycle c+1's first block
    (the range of cycle c's residual) to cycle c below it; zero elsewhere.
    cyc[i]: cycle of column i; first[i]: column i is in the first block of a cycle > 0."""
    H = V.T @ AV
    c = np.asarray(cyc)
    f = np.asarray(first, dtype=bool)
    keep = (c[:, None] == c[None, :]) | (f[:, None] & (c[:, None] == c[None, :] + 1))
    return np.where(keep, H, 0.0)


class _Cycles:
    """Column bookkeeping of the restart cycles of one Krylov solve."""

    def __init__(self, width: int, restart_len: int | None):
        self.restart_len = restart_len
        self.cyc = [0] * width
        self.first = [False] * width
        self.c = 0          # current cycle
        self.k0 = 0         # its first column
        self.blocks = 1     # its blocks so far

    def restart_due(self) -> bool:
        return self.restart_len is not None and self.blocks >= self.restart_len

    def add(self, width: int, restart: bool):
        if restart:
            self.c += 1
            self.k0 = len(self.cyc)
            self.blocks = 0
        self.cyc += [self.c] * width
        self.first += [restart] * width
        self.blocks += 1

    def H(self, V, AV):
        if self.restart_len is None:
            return V.T @ AV
        return coupled_galerkin(V, AV, self.cyc, self.first)

    def may_stop(self) -> bool:
        """Convergence is not tested at the first step of a restart cycle."""
        return self.c == 0 or self.blocks >= 2

    def correction(self, Y) -> float:
        """max over the times of the size of the current restart cycle's part of the
        projected solution (0 in the first cycle)."""
        if self.c == 0:
            return 0.0
        return float(np.max(np.linalg.norm(Y[:, self.k0:], axis=1)))


def ebk_nonhomogeneous(kop: KrylovOperator, U: np.ndarray, tau: np.ndarray, coef: np.ndarray,
                       tol: float, scale_ref: float, kmax: int, defl_tol: float = 1e-10,
                       t_eval: np.ndarray | None = None, restart_len: int | None = None):
    """EBK for v' = A v + U p(t), v(tau_0) = 0 on one window (Sec. 2.1).

    Grows the block Krylov basis V (V_1 = U) one block step at a time, projects
    (H = V^T A V, B = V^T U), solves the projected problem exactly at the window's
    sample times (or at t_eval, when the samples are not the output times) and stops when
    the change since the previous step is within tolerance.  With restart_len, a cycle of
    restart_len blocks that has not converged is followed by a restart cycle (restart_block,
    coupled_galerkin); the source enters the first cycle only.
    Returns (V, Y) with v(tau_i) ~ V Y[i] (v(t_eval_i) with t_eval), and an info dict."""
    V = U.copy()
    AV = kop.A @ V
    last = U
    prev = None
    cy = _Cycles(U.shape[1], restart_len)
    info = dict(steps=0, converged=False, est=np.inf, dims=[], restarts=0)
    for k in range(1, kmax + 1):
        H = cy.H(V, AV)
        B = V.T @ U
        B[np.asarray(cy.cyc) > 0] = 0.0
        if t_eval is None:
            Y = projected_source_window(H, B, tau, coef)
        else:
            Y = projected_source_at(H, B, tau, coef, t_eval)
        scale = max(scale_ref, float(np.max(np.linalg.norm(Y, axis=1))))
        info["steps"] = k
        info["dims"].append(V.shape[1])
        if prev is not None:
            P_ = np.zeros_like(Y)
            P_[:, :prev.shape[1]] = prev
            est = max(float(np.max(np.linalg.norm(Y - P_, axis=1))), cy.correction(Y))
            info["est"] = est / scale if scale > 0 else 0.0
            if est <= tol * scale and cy.may_stop():
                info["converged"] = True
                return V, Y, info
        prev = Y
        if k == kmax:
            break
        restart = cy.restart_due()
        if restart:
            new = restart_block(V[:, cy.k0:], AV[:, cy.k0:], last.shape[1])
            info["restarts"] += 1
        else:
            new = block_krylov_step(kop, V[:, cy.k0:], last, defl_tol)
        if new.shape[1] == 0:  # invariant subspace: the projection is exact
            info["converged"] = True
            info["est"] = 0.0
            return V, Y, info
        V, AV = _grow(kop, V, AV, new)
        cy.add(new.shape[1], restart)
        last = new
    return V, prev, info


def ebk_homogeneous(kop: KrylovOperator, w: np.ndarray, tau: np.ndarray, tol: float, scale_ref: float,
                    kmax: int, defl_tol: float = 1e-10, restart_len: int | None = None):
    """EBK for v' = A v, v(tau_0) = w on one window: single-vector Krylov space of w,
    projected solution exp(tau H) ||w|| e_1, same stopping rule and restarts as the source
    part."""
    beta = float(np.linalg.norm(w))
    if beta == 0.0:
        return w[:, None] * 0.0, np.zeros((tau.size, 1)), dict(steps=0, converged=True, est=0.0, dims=[],
                                                               restarts=0)
    V = (w / beta)[:, None]
    AV = kop.A @ V
    last = V
    prev = None
    cy = _Cycles(1, restart_len)
    info = dict(steps=0, converged=False, est=np.inf, dims=[], restarts=0)
    for k in range(1, kmax + 1):
        H = cy.H(V, AV)
        Y = projected_homogeneous(H, beta, tau)
        scale = max(scale_ref, float(np.max(np.linalg.norm(Y, axis=1))))
        info["steps"] = k
        info["dims"].append(V.shape[1])
        if prev is not None:
            P_ = np.zeros_like(Y)
            P_[:, :prev.shape[1]] = prev
            est = max(float(np.max(np.linalg.norm(Y - P_, axis=1))), cy.correction(Y))
            info["est"] = est / scale
            if est <= tol * scale and cy.may_stop():
                info["converged"] = True
                return V, Y, info
        prev = Y
        if k == kmax:
            break
        restart = cy.restart_due()
        if restart:
            new = restart_block(V[:, cy.k0:], AV[:, cy.k0:], last.shape[1])
            info["restarts"] += 1
        else:
            new = block_krylov_step(kop, V[:, cy.k0:], last, defl_tol)
        if new.shape[1] == 0:
            info["converged"] = True
            info["est"] = 0.0
            return V, Y, info
        V, AV = _grow(kop, V, AV, new)
        cy.add(new.shape[1], restart)
        last = new
    return V, prev, info


# --------------------------------------------------------------------------------------
# Paraexp time decomposition (Sec. 2.2, Fig. 3)
# --------------------------------------------------------------------------------------
def solve_linear(op: dict, opts: dict, u0: np.ndarray, G: np.ndarray | None,
                 subintervals: list[int] | None = None, return_parts: bool = False):
    """Paraexp-EBK for u' = A u + g(t), u(0) = u0 on [0, T] (Sec. 2.2, Fig. 3).

    Shift u = u0 + u_hat with source g_hat = A u0 + g (eq. linivp_shift); split the
    source over P subintervals (eq. piecewiseSource_linivp); for each subproblem
    (eq. linivpSubproblem) solve the nonhomogeneous part on [T_{j-1}, T_j] and the
    homogeneous part on [T_j, T]; sum the subsolutions (eq. superposition).

    G: (n_out, n) samples g(t_i) or None; with Chebyshev samples (nodes=1) G holds g at the
    sample times of sample_partition, shape (P (n_samp-1) + 1, n).  Returns Y (n_out, n)
    with Y[i] ~ u(t_i) and a report.  `subintervals` restricts the sum to the given j (1-based) -- used
    to time a bounded sample and by superposition tests; u0 is then left out."""
    n = u0.size
    T, P, n_out = opts["T"], opts["P"], opts["n_out"]
    t = np.arange(n_out) * (T / (n_out - 1))
    idx = partition(n_out, P)
    ts, sidx = sample_partition(opts)
    cheb = opts.get("nodes", NODES_UNIFORM) != NODES_UNIFORM
    A = operator_matrix(op)
    Au0 = A @ u0
    kmax = opts["restart_len"] * (opts.get("max_restarts", 0) + 1)
    rlen = opts["restart_len"] if opts.get("max_restarts", 0) > 0 else None
    tol = opts["tol"]
    scale_ref = float(np.linalg.norm(u0))
    js = list(range(1, P + 1)) if subintervals is None else list(subintervals)
    Y = np.zeros((n_out, n)) if subintervals is not None else np.tile(u0, (n_out, 1))
    rep = dict(m=[], sigma_ratio=[], k_nh=[], est_nh=[], conv_nh=[], k_hom=[], conv_hom=[], boundaries=idx,
               restarts_nh=[], restarts_hom=[])
    parts = {}
    # one shift-and-invert pole for all windows: gamma = sai_gamma * T / P
    kop = KrylovOperator(op, A, opts["krylov"], opts.get("sai_gamma", 0.1) * T / P)
    for j in js:
        i0, i1 = idx[j - 1], idx[j]
        s0, s1 = sidx[j - 1], sidx[j]
        tau = ts[s0:s1 + 1] - ts[s0]
        Ghat = np.tile(Au0[:, None], (1, s1 - s0 + 1))
        if G is not None:
            Ghat = Ghat + G[s0:s1 + 1].T
        U, C, sig = compress_source(Ghat, opts["svd_tol"], opts["max_rank"])
        m = U.shape[1]
        rep["m"].append(m)
        rep["sigma_ratio"].append(float(sig[m] / sig[0]) if m < sig.size and sig[0] > 0 else 0.0)
        vj = np.zeros((n_out, n))
        if m == 0:
            rep["k_nh"].append(0); rep["est_nh"].append(0.0); rep["conv_nh"].append(True)
            rep["k_hom"].append([]); rep["conv_hom"].append([])
            rep["restarts_nh"].append(0); rep["restarts_hom"].append([])
            parts[j] = vj
            continue
        coef = spline_segments(tau, C)
        V, Yp, info = ebk_nonhomogeneous(kop, U, tau, coef, tol, scale_ref, kmax,
                                         t_eval=(t[i0:i1 + 1] - t[i0]) if cheb else None, restart_len=rlen)
        rep["k_nh"].append(info["steps"]); rep["est_nh"].append(info["est"]); rep["conv_nh"].append(info["converged"])
        rep["restarts_nh"].append(info["restarts"])
        vj[i0:i1 + 1] = Yp @ V.T
        w = vj[i1].copy()
        khs, chs, rhs = [], [], []
        for mm in range(j + 1, P + 1):
            a0, a1 = idx[mm - 1], idx[mm]
            tau_h = t[a0:a1 + 1] - t[a0]
            Vh, Yh, ih = ebk_homogeneous(kop, w, tau_h, tol, scale_ref, kmax, restart_len=rlen)
            khs.append(ih["steps"]); chs.append(ih["converged"]); rhs.append(ih["restarts"])
            seg = Yh @ Vh.T
            vj[a0 + 1:a1 + 1] = seg[1:]
            w = seg[-1].copy()
        rep["k_hom"].append(khs); rep["conv_hom"].append(chs); rep["restarts_hom"].append(rhs)
        parts[j] = vj
        Y += vj
    if return_parts:
        return Y, rep, parts
    return Y, rep


def solve_linear_piecewise(A_list: list, opts: dict, u0: np.ndarray, G_list: list, op: dict | None = None):
    """Paraexp-EBK with one operator per subinterval (Sec. 2.4, eq. ivpSubproblem, whose
    matrix A + J_k(t) is piecewise constant by eq. piecewiseJac).

    A_list[j-1]: the sparse operator on subinterval j.  G_list[j-1]: the source at the
    s_j samples of subinterval j, shape (s_j, n), both end samples included (a sample
    shared by two subintervals has one value in each).  On subinterval j the shift
    u = u0 + u_hat gives u_hat' = A_j u_hat + (A_j u0 + g_j) (eq. linivp_shift taken piece by
    piece); subproblem j's nonhomogeneous part is solved with A_j and its homogeneous part
    is carried through each later subinterval m with A_m; the parts add up (eq.
    superposition, eq. updateSolution).  Returns (Y, report) with Y (n_out, n)."""
    n = u0.size
    T, P, n_out = opts["T"], opts["P"], opts["n_out"]
    t = np.arange(n_out) * (T / (n_out - 1))
    idx = partition(n_out, P)
    kmax = opts["restart_len"] * (opts.get("max_restarts", 0) + 1)
    rlen = opts["restart_len"] if opts.get("max_restarts", 0) > 0 else None
    tol = opts["tol"]
    scale_ref = float(np.linalg.norm(u0))
    gamma = opts.get("sai_gamma", 0.1) * T / P
    kops = [KrylovOperator(op, sp.csr_matrix(A_list[j]), opts["krylov"], gamma) for j in range(P)]
    Y = np.tile(u0, (n_out, 1))
    rep = dict(m=[], k_nh=[], conv_nh=[], k_hom=[], conv_hom=[], boundaries=idx)
    for j in range(1, P + 1):
        i0, i1 = idx[j - 1], idx[j]
        tau = t[i0:i1 + 1] - t[i0]
        Ghat = (kops[j - 1].A @ u0)[:, None] + np.asarray(G_list[j - 1]).T
        U, C, _ = compress_source(Ghat, opts["svd_tol"], opts["max_rank"])
        rep["m"].append(U.shape[1])
        if U.shape[1] == 0:
            rep["k_nh"].append(0); rep["conv_nh"].append(True); rep["k_hom"].append([]); rep["conv_hom"].append([])
            continue
        V, Yp, info = ebk_nonhomogeneous(kops[j - 1], U, tau, spline_segments(tau, C), tol, scale_ref, kmax,
                                         restart_len=rlen)
        rep["k_nh"].append(info["steps"]); rep["conv_nh"].append(info["converged"])
        Y[i0:i1 + 1] += Yp @ V.T
        w = V @ Yp[-1]
        khs, chs = [], []
        for mm in range(j + 1, P + 1):
            a0, a1 = idx[mm - 1], idx[mm]
            Vh, Yh, ih = ebk_homogeneous(kops[mm - 1], w, t[a0:a1 + 1] - t[a0], tol, scale_ref, kmax,
                                         restart_len=rlen)
            khs.append(ih["steps"]); chs.append(ih["converged"])
            seg = Yh @ Vh.T
            Y[a0 + 1:a1 + 1] += seg[1:]
            w = seg[-1].copy()
        rep["k_hom"].append(khs); rep["conv_hom"].append(chs)
    return Y, rep


# --------------------------------------------------------------------------------------
# Nonlinear problems: waveform relaxation (Sec. 2.3 eqs. source, ivp3; Sec. 2.4; Fig. 5)
# --------------------------------------------------------------------------------------
def burgers_source(op: dict, Usamp: np.ndarray, form: int = 0) -> np.ndarray:
    """g(t, u) = -u u_x on the 1D mesh for each row of Usamp (shape (s, n) or (n,)).

    form 0: conservative central difference -(u_{i+1}^2 - u_{i-1}^2) / (4 dx);
    form 1: advective central difference   -u_i (u_{i+1} - u_{i-1}) / (2 dx).
    Periodic indices mod n; homogeneous Dirichlet uses zero ghost values."""
    n = op["nx"]
    dx = _mesh_width(n, op["Lx"], op["bc"])
    U2 = np.atleast_2d(Usamp)
    out = np.zeros_like(U2)
    for r in range(U2.shape[0]):
        u = U2[r]
        if op["bc"] == BC_PERIODIC:
            um, up = np.roll(u, 1), np.roll(u, -1)
        else:
            um = np.concatenate([[0.0], u[:-1]])
            up = np.concatenate([u[1:], [0.0]])
        if form == 0:
            out[r] = -(up * up - um * um) / (4.0 * dx)
        else:
            out[r] = -u * (up - um) / (2.0 * dx)
    return out if Usamp.ndim == 2 else out[0]


def burgers_jacobian(op: dict, ubar: np.ndarray, form: int = 0) -> sp.csr_matrix:
    """The Jacobian d g / d u of burgers_source at the state ubar (the matrix inside the
    integral of eq. jacobian / eq. piecewiseJac), as a sparse n x n matrix.

    form 0, g_i = -(u_{i+1}^2 - u_{i-1}^2)/(4 dx): dg_i/du_{i+1} = -u_{i+1}/(2 dx),
    dg_i/du_{i-1} = u_{i-1}/(2 dx).  form 1, g_i = -u_i (u_{i+1} - u_{i-1})/(2 dx):
    dg_i/du_i = -(u_{i+1} - u_{i-1})/(2 dx), dg_i/du_{i+1} = -u_i/(2 dx),
    dg_i/du_{i-1} = u_i/(2 dx).  Periodic indices wrap; homogeneous Dirichlet has zero
    ghost values and no entries outside the mesh.  g is quadratic in u, so the Jacobian
    is linear in ubar and its time average is the Jacobian of the time-averaged state."""
    n = op["nx"]
    dx = _mesh_width(n, op["Lx"], op["bc"])
    periodic = op["bc"] == BC_PERIODIC
    i = np.arange(n)
    if periodic:
        im, ip = (i - 1) % n, (i + 1) % n
        has_m = has_p = np.ones(n, bool)
    else:
        im, ip = i - 1, i + 1
        has_m, has_p = i >= 1, i <= n - 2
    ub = np.asarray(ubar, dtype=float)
    u_m = np.where(has_m, ub[np.clip(im, 0, n - 1)], 0.0)
    u_p = np.where(has_p, ub[np.clip(ip, 0, n - 1)], 0.0)
    rows, cols, vals = [], [], []
    if form == 0:
        rows += [i[has_p], i[has_m]]
        cols += [ip[has_p], im[has_m]]
        vals += [-u_p[has_p] / (2 * dx), u_m[has_m] / (2 * dx)]
    else:
        rows += [i, i[has_p], i[has_m]]
        cols += [i, ip[has_p], im[has_m]]
        vals += [-(u_p - u_m) / (2 * dx), -ub[has_p] / (2 * dx), ub[has_m] / (2 * dx)]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def window_average(Uw: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Time average over one subinterval of the sampled iterate Uw (s, n) at the offsets tau
    (tau[0] = 0): the integral of eq. piecewiseJac by the trapezoidal rule on the samples."""
    w = np.zeros(tau.size)
    dt = np.diff(tau)
    w[:-1] += 0.5 * dt
    w[1:] += 0.5 * dt
    return (w @ Uw) / tau[-1]


def _wr_stop(deltas: list, opts: dict):
    """Stopping rule of the waveform relaxation loop on the relative updates so far:
    "converged" once the last one is <= wr_tol; "diverged" once the update has grown in
    wr_diverge successive iterations (default 3; 0 never stops on growth); else None."""
    if deltas[-1] <= opts["wr_tol"]:
        return "converged"
    q = opts.get("wr_diverge", 3)
    if q > 0 and len(deltas) > q and all(deltas[-i] > deltas[-i - 1] for i in range(1, q + 1)):
        return "diverged"
    return None


def solve_burgers_jacobian(op: dict, opts: dict, u0: np.ndarray, forcing: np.ndarray | None = None,
                           init: np.ndarray | None = None, callback=None):
    """Waveform relaxation with the averaged-Jacobian correction (Sec. 2.3 eq. ivp4,
    Sec. 2.4 eqs. piecewiseJac and ivpSubproblem).

    Iterate k: g_k(t_i) = -u_k u_k,x (t_i) + f(t_i) (eq. source); on each subinterval j,
    J_{k,j} = the Jacobian of g at the subinterval's time-averaged iterate (window_average);
    then u_{k+1}' = (A + J_{k,j}) u_{k+1} + g_k - J_{k,j} u_k on subinterval j, u_{k+1}(0) = u0,
    solved by solve_linear_piecewise.  At a fixed point the J terms cancel, so the limit is
    the same as Picard's (solve_burgers); only the convergence speed changes.  The shifted
    source of eq. sourceParallel is read as A u0 + g_k - J_{k,j} u_hat_k (its printed
    +J_k u0 would move the fixed point).  Stops as solve_burgers does.  Returns (U, report)."""
    n_out, P, T = opts["n_out"], opts["P"], opts["T"]
    form = opts.get("burgers_form", 0)
    t = np.arange(n_out) * (T / (n_out - 1))
    idx = partition(n_out, P)
    A = operator_matrix(op)
    Uk = np.tile(u0, (n_out, 1)) if init is None else init.copy()
    rep = dict(iters=0, deltas=[], converged=False, diverged=False)
    for k in range(opts["wr_max_iter"]):
        Gk = burgers_source(op, Uk, form)
        if forcing is not None:
            Gk = Gk + forcing
        A_list, G_list = [], []
        for j in range(1, P + 1):
            i0, i1 = idx[j - 1], idx[j]
            J = burgers_jacobian(op, window_average(Uk[i0:i1 + 1], t[i0:i1 + 1] - t[i0]), form)
            A_list.append((A + J).tocsr())
            G_list.append(Gk[i0:i1 + 1] - (J @ Uk[i0:i1 + 1].T).T)
        Unew, _ = solve_linear_piecewise(A_list, opts, u0, G_list, op)
        delta = float(np.max(np.linalg.norm(Unew - Uk, axis=1)) / np.max(np.linalg.norm(Unew, axis=1)))
        rep["deltas"].append(delta)
        rep["iters"] = k + 1
        Uk = Unew
        if callback is not None:
            callback(k, Uk, delta)
        stop = _wr_stop(rep["deltas"], opts)
        if stop is not None:
            rep[stop] = True
            break
    return Uk, rep


def solve_burgers(op: dict, opts: dict, u0: np.ndarray, forcing: np.ndarray | None = None,
                  init: np.ndarray | None = None, callback=None):
    """Waveform relaxation with Paraexp-EBK (Fig. 5), plain Picard form (eq. ivp3).

    A = nu D2 (the operator `op`, advection velocity zero).  Iterate
    u_{k+1} = PEBK(A, u0, g_k) with g_k(t_i) = -u_k u_k,x (t_i) + f(t_i) (eq. source)
    from u_1(t) = u0 (or `init`), until the relative update is <= wr_tol or
    wr_max_iter iterations have been made.  Returns (U, report) with U (n_out, n)."""
    n_out = opts["n_out"]
    Uk = np.tile(u0, (n_out, 1)) if init is None else init.copy()
    rep = dict(iters=0, deltas=[], converged=False, diverged=False)
    for k in range(opts["wr_max_iter"]):
        Gk = burgers_source(op, Uk, opts.get("burgers_form", 0))
        if forcing is not None:
            Gk = Gk + forcing
        Unew, _ = solve_linear(op, opts, u0, Gk)
        delta = float(np.max(np.linalg.norm(Unew - Uk, axis=1)) / np.max(np.linalg.norm(Unew, axis=1)))
        rep["deltas"].append(delta)
        rep["iters"] = k + 1
        Uk = Unew
        if callback is not None:
            callback(k, Uk, delta)
        stop = _wr_stop(rep["deltas"], opts)
        if stop is not None:
            rep[stop] = True
            break
    return Uk, rep
