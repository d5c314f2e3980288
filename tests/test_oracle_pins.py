"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself: a
closed form, a dense brute-force solution, an invariant, a special case, or a
number the paper prints.  A plausible mistake (a dropped term, a wrong sign or
index, a transposed operand) in any oracle step fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate as sint
import scipy.linalg as sla

import closed_forms as cf
import oracle.pebk as ob
from paper_1509_04567_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- operator (Sec. 3.1)
@pytest.mark.parametrize("n,a,nu", [(16, 1.0, 1e-2), (33, -0.7, 3e-3), (64, 0.0, 1e-1)])
def test_operator_fourier_symbol_periodic(n, a, nu):
    """A e_k = lambda_k e_k for the Fourier modes of the periodic mesh (circulant symbol)."""
    op = wl.make_op(n, nu, a)
    A = ob.operator_matrix(op).toarray()
    lam = cf.circulant_eigs(n, a, nu)
    x = np.arange(n)
    for k in range(n):
        e = np.exp(2j * np.pi * k * x / n)
        np.testing.assert_allclose(A @ e, lam[k] * e, rtol=0, atol=1e-9 * max(1.0, abs(lam).max()))


def test_operator_dirichlet_eigs_and_2d_sum():
    n, nu = 20, 2e-2
    op = wl.make_op(n, nu, 0.0, bc=wl.BC_DIRICHLET0)
    A = ob.operator_matrix(op).toarray()
    dx = 1.0 / (n + 1)
    ref = np.sort(-(4 * nu / dx ** 2) * np.sin(np.arange(1, n + 1) * np.pi / (2 * (n + 1))) ** 2)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), ref, rtol=1e-12)
    # 2D periodic: product Fourier modes have the sum of the 1D symbols
    nx, ny, ax, ay = 8, 6, 1.0, 0.5
    op2 = wl.make_op(nx, nu, ax, dim=2, ny=ny, ay=ay)
    A2 = ob.operator_matrix(op2).toarray()
    lx, ly = cf.circulant_eigs(nx, ax, nu), cf.circulant_eigs(ny, ay, nu)
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny))
    for kx, ky in [(1, 0), (2, 3), (7, 5)]:
        e = (np.exp(2j * np.pi * kx * ix / nx) * np.exp(2j * np.pi * ky * iy / ny)).ravel()
        np.testing.assert_allclose(A2 @ e, (lx[kx] + ly[ky]) * e, atol=1e-9 * abs(lx).max())


# ---------------------------------------------------------------- partition (Sec. 2.2)
def test_partition_golden():
    ref = np.loadtxt(os.path.join(GOLDEN, "partition_n101_P8.txt"), dtype=int)
    assert ob.partition(101, 8) == list(ref)
    assert ob.partition(1025, 64) == list(range(0, 1025, 16))
    with pytest.raises(ValueError):
        ob.partition(5, 8)


# ---------------------------------------------------------------- source model (Sec. 2.1)
def test_compress_source_exact_rank_two():
    """The small advection-diffusion source A u0 + sin(4 pi x) cos(2 pi t) has rank 2."""
    pr = wl.adv_diff_1d(n=1024, P=8, n_out=101)
    A = ob.operator_matrix(pr.op)
    t = wl.out_times(1.0, 101)[:13]
    Ghat = (A @ pr.u0)[:, None] + pr.G[:13].T
    U, C, sig = ob.compress_source(Ghat, 1e-12, 16)
    assert U.shape[1] == 2
    assert sig[2] / sig[0] < 1e-14
    np.testing.assert_allclose(U.T @ U, np.eye(2), atol=1e-14)
    assert np.linalg.norm(Ghat - U @ C) <= 1e-13 * np.linalg.norm(Ghat)
    # singular values agree with the square roots of the Gram eigenvalues (independent route)
    ev = np.sort(np.linalg.eigvalsh(Ghat.T @ Ghat))[::-1]
    np.testing.assert_allclose(sig[:2], np.sqrt(ev[:2]), rtol=1e-12)


def test_compress_source_eckart_young_and_cap():
    """Truncation error equals sqrt(sum of dropped sigma^2) for a matrix of known SVD."""
    rng = np.random.default_rng(3)
    n, s = 300, 9
    Q1, _ = np.linalg.qr(rng.standard_normal((n, s)))
    Q2, _ = np.linalg.qr(rng.standard_normal((s, s)))
    sv = 10.0 ** -np.arange(s, dtype=float)
    Gm = (Q1 * sv) @ Q2.T
    U, C, sig = ob.compress_source(Gm, 2e-4, 16)
    assert U.shape[1] == 4
    np.testing.assert_allclose(sig, sv, rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(Gm - U @ C), np.sqrt(np.sum(sv[4:] ** 2)), rtol=1e-6)
    U2, _, _ = ob.compress_source(Gm, 0.0, 3)
    assert U2.shape[1] == 3
    Uz, Cz, _ = ob.compress_source(np.zeros((n, s)), 1e-12, 16)
    assert Uz.shape[1] == 0 and Cz.shape == (0, s)


def test_theorem1_singular_value_decay():
    """Thm 1: sigma_{j+1} = sqrt(s-j) O(dT^j): halving dT divides sigma_{j+1}/sigma_1 by ~2^j."""
    n, s = 400, 17
    x = np.arange(n) / n
    def sig_of(dT):
        t = np.linspace(0.3, 0.3 + dT, s)
        Gm = (np.sin(2 * np.pi * x[:, None] + 3 * t[None, :]) + np.cos(4 * np.pi * x[:, None] - 5 * t[None, :])
              + np.exp(-t[None, :]) * np.sin(6 * np.pi * x[:, None]))
        return ob.compress_source(Gm, 0.0, s)[2]
    a, b = sig_of(0.05), sig_of(0.025)
    for j in (1, 2, 3):
        ratio = (a[j] / a[0]) / (b[j] / b[0])
        assert 0.6 * 2 ** j < ratio < 1.6 * 2 ** j, (j, ratio)


def test_spline_reproduces_cubics_and_not_a_knot():
    tau = np.linspace(0.0, 0.2, 9) + 0.01 * np.sin(np.arange(9))
    c = np.array([[0.3, -1.0, 2.5, 4.0], [1.0, 0.0, -3.0, 0.5]])
    C = np.array([[np.polyval(cc[::-1], tt) for tt in tau] for cc in c])
    coef = ob.spline_segments(tau, C)
    for i in range(tau.size - 1):
        for r in range(2):
            th = 0.37 * (tau[i + 1] - tau[i])
            ref = np.polyval(c[r][::-1], tau[i] + th)
            assert abs(sum(coef[i, l, r] * th ** l for l in range(4)) - ref) < 1e-12
    # not-a-knot on generic data: third derivative continuous across tau_1 and tau_{s-2}
    D = np.vstack([np.sin(7 * tau), np.exp(tau)])
    cf_ = ob.spline_segments(tau, D)
    np.testing.assert_allclose(cf_[0, 3], cf_[1, 3], rtol=1e-9)
    np.testing.assert_allclose(cf_[-1, 3], cf_[-2, 3], rtol=1e-9)
    # interpolation and C2 continuity
    for i in range(tau.size - 1):
        h = tau[i + 1] - tau[i]
        np.testing.assert_allclose(cf_[i, 0], D[:, i], rtol=1e-14)
        end = sum(cf_[i, l] * h ** l for l in range(4))
        np.testing.assert_allclose(end, D[:, i + 1], rtol=1e-12)
        if i < tau.size - 2:
            d2 = 2 * cf_[i, 2] + 6 * cf_[i, 3] * h
            np.testing.assert_allclose(d2, 2 * cf_[i + 1, 2], rtol=1e-8, atol=1e-10)
    # two samples -> straight line, three -> parabola
    c2 = ob.spline_segments(np.array([0.0, 0.5]), np.array([[1.0, 2.0]]))
    np.testing.assert_allclose(c2[0, :, 0], [1.0, 2.0, 0.0, 0.0], atol=1e-14)
    t3 = np.array([0.0, 0.1, 0.3])
    c3 = ob.spline_segments(t3, np.array([[1.0, 1.0 + 0.1 - 0.01, 1.0 + 0.3 - 0.09]]))
    np.testing.assert_allclose(c3[0, :, 0], [1.0, 1.0, -1.0, 0.0], atol=1e-12)


# ---------------------------------------------------------------- block Krylov (eq. blockKrylovSubspace)
@pytest.mark.parametrize("krylov", [0, 1])
def test_block_krylov_orthonormal_and_spans_power_basis(krylov):
    n, b, steps = 48, 2, 4
    op = wl.make_op(n, 2e-3, 0.8)
    A = ob.operator_matrix(op)
    gamma = 0.01
    kop = ob.KrylovOperator(op, A, krylov, gamma)
    U, _ = np.linalg.qr(wl.smooth_block(n, b, 1, modes=6))
    V, last = U.copy(), U
    for _ in range(steps - 1):
        new = ob.block_krylov_step(kop, V, last)
        V = np.hstack([V, new])
        last = new
    assert V.shape[1] == steps * b
    np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-13)
    Ad = A.toarray()
    Op = Ad if krylov == 0 else np.linalg.inv(np.eye(n) - gamma * Ad)
    blocks, X = [U], U
    for _ in range(steps - 1):
        X = Op @ X
        blocks.append(X / np.linalg.norm(X))
    Pw, _ = np.linalg.qr(np.hstack(blocks))
    cosines = sla.svdvals(Pw.T @ V)
    np.testing.assert_allclose(cosines, 1.0, atol=1e-9)


def test_block_krylov_deflation():
    """An invariant direction in the start block deflates instead of being normalised."""
    n = 64
    op = wl.make_op(n, 1e-2, 1.0)
    A = ob.operator_matrix(op)
    x = np.arange(n) / n
    U, _ = np.linalg.qr(np.column_stack([np.cos(2 * np.pi * x), np.sin(2 * np.pi * x)]))
    kop = ob.KrylovOperator(op, A, 1, 0.01)
    new = ob.block_krylov_step(kop, U, U)
    assert new.shape[1] == 0  # span{cos, sin} is invariant under the circulant A


# ---------------------------------------------------------------- projected problem
def test_projected_source_window_vs_ode_integrator():
    rng = np.random.default_rng(5)
    K, m = 6, 2
    H = rng.standard_normal((K, K)) - 3 * np.eye(K)
    B = rng.standard_normal((K, m))
    tau = np.linspace(0, 0.4, 6)
    C = rng.standard_normal((m, tau.size))
    coef = ob.spline_segments(tau, C)
    Y = ob.projected_source_window(H, B, tau, coef)
    def p(t):
        i = min(int(np.searchsorted(tau, t, side="right")) - 1, tau.size - 2)
        th = t - tau[i]
        return sum(coef[i, l] * th ** l for l in range(4))
    sol = sint.solve_ivp(lambda t, y: H @ y + B @ p(t), (0, 0.4), np.zeros(K), t_eval=tau,
                         method="DOP853", rtol=1e-13, atol=1e-15, max_step=0.005)
    np.testing.assert_allclose(Y, sol.y.T, atol=1e-11)


def test_projected_homogeneous_matches_eigendecomposition():
    rng = np.random.default_rng(6)
    K = 5
    S = rng.standard_normal((K, K))
    d = -np.arange(1, K + 1, dtype=float)
    H = S @ np.diag(d) @ np.linalg.inv(S)
    tau = np.array([0.0, 0.1, 0.7])
    Y = ob.projected_homogeneous(H, 2.0, tau)
    e1 = np.zeros(K); e1[0] = 2.0
    for i, t in enumerate(tau):
        np.testing.assert_allclose(Y[i], S @ (np.exp(d * t) * np.linalg.solve(S, e1)), atol=1e-12)


def test_dense_reference_expm_vs_longdouble_taylor():
    """The dense brute-force reference's expm agrees with a long-double Taylor series."""
    n, m = 12, 2
    A = ob.operator_matrix(wl.make_op(n, 1e-2, 1.0, bc=wl.BC_DIRICHLET0)).toarray()
    h = 0.05
    M = np.zeros((n + 4 * m, n + 4 * m))
    M[:n, :n] = h * A
    M[:n, n:n + m] = h * wl.random_block(n, m, 2)
    for l in range(3):
        M[n + l * m:n + (l + 1) * m, n + (l + 1) * m:n + (l + 2) * m] = np.eye(m)
    np.testing.assert_allclose(sla.expm(M), cf.taylor_expm_longdouble(M).astype(float), atol=1e-13)


# ---------------------------------------------------------------- whole method (Sec. 2.2, Fig. 3)
def test_oracle_matches_circulant_closed_form_small_case():
    """P1: the oracle's PEBK equals the exact semi-discrete solution with the same source model."""
    pr = wl.adv_diff_1d(n=1024, P=8, n_out=101, tol=1e-12, restart_len=30)
    Y, rep = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)
    assert all(rep["conv_nh"]) and all(all(c) for c in rep["conv_hom"])
    t, wins = cf.fourier_windows_from_oracle_model(pr.op, pr.opts, pr.u0, pr.G, ob.compress_source,
                                                   ob.spline_segments, ob.partition)
    Yx = cf.exact_piecewise_cubic(cf.circulant_eigs(pr.n, 1.0, 1e-2), pr.u0, t, wins)
    err = np.max(np.linalg.norm(Y - Yx, axis=1) / np.linalg.norm(Yx, axis=1))
    assert err < 2e-11, err


def test_sampled_closed_form_equals_the_recurrence():
    """The windowed closed sum (used at 2^20 points, where the recurrence is too slow)
    against the per-interval recurrence it sums, at interior points and window ends."""
    pr = wl.adv_diff_1d(n=512, nu=2e-3, P=5, n_out=61, tol=1e-12)
    t, wins = cf.fourier_windows_from_oracle_model(pr.op, pr.opts, pr.u0, pr.G, ob.compress_source,
                                                   ob.spline_segments, ob.partition)
    lam = cf.circulant_eigs(pr.n, 1.0, 2e-3)
    Yx = cf.exact_piecewise_cubic(lam, pr.u0, t, wins)
    keep = [0, 3, 12, 13, 30, 47, 59, 60]
    gen = cf.iter_windows_from_oracle_model(pr.op, pr.opts, pr.u0, pr.G, ob.compress_source,
                                            ob.spline_segments, ob.partition)
    got = cf.exact_at_samples(lam, pr.u0, t, gen, keep)
    assert sorted(got) == keep
    for k in keep:
        assert np.linalg.norm(got[k] - Yx[k]) <= 1e-13 * np.linalg.norm(Yx[k]), k


@pytest.mark.parametrize("krylov", [0, 1])
def test_oracle_matches_dense_bruteforce_dirichlet(krylov):
    """P2: n <= 64, homogeneous Dirichlet, both Krylov operators, vs the full augmented expm."""
    n = 40
    op = wl.make_op(n, 1e-2, 0.5, bc=wl.BC_DIRICHLET0)
    x = wl.grid_1d(n, bc=wl.BC_DIRICHLET0)
    u0 = np.sin(np.pi * x) * (1 + x)
    t = wl.out_times(0.5, 17)
    G = np.cos(3 * t)[:, None] * (x * (1 - x))[None, :] + t[:, None] ** 2 * np.sin(2 * np.pi * x)[None, :]
    opts = wl.default_opts(T=0.5, P=4, n_out=17, tol=1e-13, krylov=krylov, restart_len=40)
    Y, rep = ob.solve_linear(op, opts, u0, G)
    tt, wins = cf.fourier_windows_from_oracle_model(op, opts, u0, G, ob.compress_source,
                                                    ob.spline_segments, ob.partition)
    Yx = cf.dense_exact(ob.operator_matrix(op).toarray(), u0, tt, wins)
    err = np.max(np.linalg.norm(Y - Yx, axis=1) / np.linalg.norm(Yx, axis=1))
    assert err < 1e-10, err


def test_superposition_partition_invariance():
    """P3: with a source exactly cubic in time (so every partition models it exactly) the
    sum of P subsolutions equals the single-interval solve, and parts add up."""
    n = 128
    x = wl.grid_1d(n)
    op = wl.make_op(n, 5e-3, 1.0)
    u0 = np.cos(2 * np.pi * x) + 0.3 * np.sin(6 * np.pi * x)
    t = wl.out_times(0.4, 33)
    G = (1 + t - 2 * t ** 3)[:, None] * np.sin(4 * np.pi * x)[None, :] + (t ** 2)[:, None] * np.cos(8 * np.pi * x)[None, :]
    res = []
    for P in (1, 4):
        opts = wl.default_opts(T=0.4, P=P, n_out=33, tol=1e-13, restart_len=40)
        Y, rep, parts = ob.solve_linear(op, opts, u0, G, return_parts=True)
        np.testing.assert_allclose(sum(parts.values()) + u0, Y, atol=1e-13)
        res.append(Y)
    np.testing.assert_allclose(res[0], res[1], atol=1e-10 * np.abs(res[0]).max())


def test_single_mode_homogeneous_closed_form():
    """P6: g = 0 and u0 a Fourier mode: u(t) = Re(exp(lambda_k t) e^{2 pi i k x})."""
    n, k = 256, 3
    x = wl.grid_1d(n)
    op = wl.make_op(n, 1e-2, 1.0)
    u0 = np.cos(2 * np.pi * k * x)
    opts = wl.default_opts(T=1.0, P=8, n_out=17, tol=1e-13, restart_len=30)
    Y, _ = ob.solve_linear(op, opts, u0, None)
    lam = cf.circulant_eigs(n, 1.0, 1e-2)[k]
    for i, tt in enumerate(wl.out_times(1.0, 17)):
        np.testing.assert_allclose(Y[i], np.real(np.exp(lam * tt) * np.exp(2j * np.pi * k * x)), atol=1e-11)


def test_skew_symmetric_norm_preservation():
    """P6: nu = 0 makes A skew-symmetric, so ||u(t)|| = ||u0|| for g = 0."""
    n = 200
    x = wl.grid_1d(n)
    u0 = np.exp(-50 * (x - 0.5) ** 2)
    opts = wl.default_opts(T=0.5, P=4, n_out=9, tol=1e-12, restart_len=40)
    Y, _ = ob.solve_linear(wl.make_op(n, 0.0, 1.0), opts, u0, None)
    np.testing.assert_allclose(np.linalg.norm(Y, axis=1), np.linalg.norm(u0), rtol=1e-9)


def test_constant_source_phi1_closed_form():
    """P6: u0 = 0 and a constant source c: u(t) = t phi_1(tA) c, per Fourier mode."""
    n = 128
    x = wl.grid_1d(n)
    c = np.exp(np.sin(2 * np.pi * x))
    t = wl.out_times(0.5, 9)
    G = np.tile(c, (9, 1))
    opts = wl.default_opts(T=0.5, P=4, n_out=9, tol=1e-13, restart_len=40)
    Y, _ = ob.solve_linear(wl.make_op(n, 1e-2, 1.0), opts, np.zeros(n), G)
    lam = cf.circulant_eigs(n, 1.0, 1e-2)
    ch = np.fft.fft(c)
    for i, tt in enumerate(t):
        ref = np.real(np.fft.ifft(tt * cf.phi_functions(lam * tt, 1)[1] * ch))
        np.testing.assert_allclose(Y[i], ref, atol=1e-10 * np.abs(ref).max() + 1e-14)


def test_pulse_problem_second_order_in_dx():
    """P8: Sec. 3.1 pulse problem -- error at t = 1 vs the Fourier series is O(dx^2)."""
    errs = []
    for n in (64, 128, 256):
        pr = wl.pulse_ade(n=n, nu=1e-2, a=1.0, T=1.0, P=8, n_out=9, tol=1e-10)
        Y, _ = ob.solve_linear(pr.op, pr.opts, pr.u0, None)
        ex = cf.pulse_series(wl.grid_1d(n), 1.0, 1.0, 1e-2)
        errs.append(np.linalg.norm(Y[-1] - ex) / np.linalg.norm(ex))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


def test_table1_serial_error_golden():
    """P8: the paper's Table 1 PEBK serial error 3.05e-4 (n = 1000, tol 1e-4, m = 2)."""
    ref = np.loadtxt(os.path.join(GOLDEN, "table1_pebk_serial_error.txt"))
    pr = wl.travelling_pulses(n=1000, T=1.0, P=2, n_out=201, tol=1e-4)
    Y, rep = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)
    assert rep["m"] == [2, 2]
    ex = pr.meta["exact"](1.0)
    err = np.linalg.norm(Y[-1] - ex) / np.linalg.norm(ex)
    assert abs(err - ref[0, 1]) < 0.03 * ref[0, 1], err


# ---------------------------------------------------------------- Burgers by waveform relaxation (Sec. 2.3-2.4)
def test_burgers_source_forms():
    n = 64
    op = wl.make_op(n, 1e-2, 0.0)
    x = wl.grid_1d(n)
    u = 0.5 + np.sin(2 * np.pi * x)
    dx = 1.0 / n
    g0 = ob.burgers_source(op, u, 0)
    g1 = ob.burgers_source(op, u, 1)
    i = 10
    assert abs(g0[i] + (u[i + 1] ** 2 - u[i - 1] ** 2) / (4 * dx)) < 1e-12
    assert abs(g1[i] + u[i] * (u[i + 1] - u[i - 1]) / (2 * dx)) < 1e-12
    assert abs(g0.sum()) < 1e-10  # conservative form: discrete mean is conserved
    # both approximate -u u_x to second order
    ex = -u * 2 * np.pi * np.cos(2 * np.pi * x)
    assert np.max(np.abs(g0 - ex)) < 0.05 and np.max(np.abs(g1 - ex)) < 0.05


def test_burgers_wr_converges_to_fine_implicit_reference_and_conserves_mean():
    """P7: the WR fixed point agrees with a tight-tolerance ODE integration of the same
    semi-discrete Burgers system to the level of the cubic source model, and the discrete
    mean is conserved (conservative form)."""
    n = 64
    op = wl.make_op(n, 5e-2, 0.0)
    x = wl.grid_1d(n)
    u0 = 0.5 + np.sin(2 * np.pi * x)
    opts = wl.default_opts(T=0.1, P=4, n_out=41, tol=1e-13, svd_tol=1e-13, max_rank=16,
                           wr_tol=1e-10, wr_max_iter=60, restart_len=40)
    U, rep = ob.solve_burgers(op, opts, u0)
    assert rep["converged"], rep["deltas"][-3:]
    A = ob.operator_matrix(op)
    f = lambda t, u: A @ u + ob.burgers_source(op, u, 0)
    t = wl.out_times(0.1, 41)
    sol = sint.solve_ivp(f, (0, 0.1), u0, t_eval=t, method="Radau", rtol=1e-12, atol=1e-13)
    err = np.max(np.abs(U - sol.y.T))
    assert err < 2e-6, err
    np.testing.assert_allclose(U.mean(axis=1), u0.mean(), atol=1e-10)


# ---------------------------------------------------------------- averaged-Jacobian WR (Sec. 2.3-2.4)
@pytest.mark.parametrize("bc", [wl.BC_PERIODIC, wl.BC_DIRICHLET0])
@pytest.mark.parametrize("form", [0, 1])
def test_burgers_jacobian_matches_central_differences(bc, form):
    """The Jacobian of eq. jacobian against central differences of the source itself
    (exact up to rounding: the discrete nonlinearity is quadratic)."""
    n = 12
    op = wl.make_op(n, 1e-2, 0.0, bc=bc)
    u = np.random.default_rng(7).standard_normal(n)
    J = ob.burgers_jacobian(op, u, form).toarray()
    eps = 1e-3
    for c in range(n):
        e = np.zeros(n)
        e[c] = eps
        col = (ob.burgers_source(op, u + e, form) - ob.burgers_source(op, u - e, form)) / (2 * eps)
        np.testing.assert_allclose(J[:, c], col, rtol=0, atol=1e-9 * np.max(np.abs(J)))


def test_window_average_is_the_trapezoidal_time_mean():
    tau = np.array([0.0, 0.1, 0.3, 0.6])
    Uw = np.stack([np.full(3, 1.0 + 2.0 * s) for s in tau])   # linear in time: trapezoid is exact
    np.testing.assert_allclose(ob.window_average(Uw, tau), 1.0 + 2.0 * 0.3, rtol=1e-15)


def test_piecewise_solver_with_one_operator_is_solve_linear():
    pr = wl.adv_diff_1d(n=256, nu=5e-3, P=5, n_out=41, T=0.5, tol=1e-12, restart_len=30)
    Y, _ = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)
    idx = ob.partition(41, 5)
    A = ob.operator_matrix(pr.op)
    Yp, _ = ob.solve_linear_piecewise([A] * 5, pr.opts, pr.u0, [pr.G[idx[j]:idx[j + 1] + 1] for j in range(5)], pr.op)
    assert np.max(np.linalg.norm(Yp - Y, axis=1) / np.linalg.norm(Y, axis=1)) < 1e-12


@pytest.mark.parametrize("krylov", [0, 1])
def test_piecewise_solver_matches_per_window_circulant_closed_form(krylov):
    """Subintervals with different advection speeds and viscosities (a piecewise-constant
    A + J_k(t), eq. ivpSubproblem) against the exact per-mode solution with each
    subinterval's own eigenvalues and the oracle's source model."""
    n, P, n_out, T = 128, 4, 33, 0.4
    x = wl.grid_1d(n)
    t = wl.out_times(T, n_out)
    u0 = np.sin(2 * np.pi * x) + 0.5 * np.cos(6 * np.pi * x)
    G = np.cos(3 * t)[:, None] * np.sin(4 * np.pi * x)[None, :]
    coeffs = [(1.0, 1e-2), (-0.5, 2e-2), (1.5, 5e-3), (0.25, 1e-2)]   # (a_j, nu_j)
    ops = [wl.make_op(n, nu, a) for a, nu in coeffs]
    A_list = [ob.operator_matrix(o) for o in ops]
    idx = ob.partition(n_out, P)
    G_list = [G[idx[j]:idx[j + 1] + 1] for j in range(P)]
    opts = wl.default_opts(T=T, P=P, n_out=n_out, tol=1e-13, svd_tol=1e-13, max_rank=16, restart_len=40,
                           krylov=krylov)
    Y, rep = ob.solve_linear_piecewise(A_list, opts, u0, G_list, ops[0])
    assert all(rep["conv_nh"]) and all(all(c) for c in rep["conv_hom"])
    wins = []
    for j in range(P):
        i0, i1 = idx[j], idx[j + 1]
        Ghat = (A_list[j] @ u0)[:, None] + G_list[j].T
        U, C, _ = ob.compress_source(Ghat, opts["svd_tol"], opts["max_rank"])
        wins.append((i0, i1, U, ob.spline_segments(t[i0:i1 + 1] - t[i0], C)))
    lams = [cf.circulant_eigs(n, a, nu) for a, nu in coeffs]
    Yx = cf.exact_piecewise_operators(lams, u0, t, wins)
    err = np.max(np.linalg.norm(Y - Yx, axis=1) / np.linalg.norm(Yx, axis=1))
    assert err < 1e-10, err


def _burgers_case(T, nu, max_iter):
    n = 64
    op = wl.make_op(n, nu, 0.0)
    u0 = 0.5 + np.sin(2 * np.pi * wl.grid_1d(n))
    opts = wl.default_opts(T=T, P=4, n_out=41, tol=1e-13, svd_tol=1e-13, max_rank=16, wr_tol=1e-10,
                           wr_max_iter=max_iter, restart_len=40)
    A = ob.operator_matrix(op)
    ref = sint.solve_ivp(lambda tt, u: A @ u + ob.burgers_source(op, u, 0), (0, T), u0,
                         t_eval=wl.out_times(T, 41), method="Radau", rtol=1e-12, atol=1e-13).y.T
    return op, opts, u0, ref


def test_averaged_jacobian_wr_has_picards_limit_in_fewer_iterations():
    """eq. ivp4: the J terms cancel at the fixed point, so the limit is Picard's (eq. ivp3),
    and the averaged Jacobian (eq. piecewiseJac) takes fewer iterations to reach it."""
    op, opts, u0, ref = _burgers_case(0.1, 5e-2, 60)
    Up, rp = ob.solve_burgers(op, opts, u0)
    Uj, rj = ob.solve_burgers_jacobian(op, opts, u0)
    assert rp["converged"] and rj["converged"]
    assert rj["iters"] * 2 <= rp["iters"], (rj["iters"], rp["iters"])
    assert np.max(np.abs(Uj - Up)) < 1e-8
    assert np.max(np.abs(Uj - ref)) < 2e-6
    np.testing.assert_allclose(Uj.mean(axis=1), u0.mean(), atol=1e-10)


def test_averaged_jacobian_wr_converges_where_picard_diverges():
    """Longer interval, smaller viscosity: the Picard updates grow, the averaged-Jacobian
    iteration converges to the semi-discrete solution (to the source model's accuracy)."""
    op, opts, u0, ref = _burgers_case(0.3, 1e-2, 4)
    _, rp = ob.solve_burgers(op, opts, u0)
    assert rp["deltas"][3] > rp["deltas"][0], rp["deltas"]
    opts = dict(opts, wr_max_iter=30)
    Uj, rj = ob.solve_burgers_jacobian(op, opts, u0)
    assert rj["converged"] and rj["iters"] <= 20, rj["deltas"]
    assert np.max(np.abs(Uj - ref)) < 5e-5


def test_smoothed_sawtooth_is_the_sawtooth_series():
    """eq. modifiedSawtooth: with no smoothing, sum_k sin(2 pi k xi)/(pi k) = 1/2 - xi on
    (0, 1) (the sawtooth's Fourier series), so u = xi there; the returned derivatives match
    central differences."""
    xi = np.linspace(0.05, 0.95, 19)
    u, _, _ = wl.smoothed_sawtooth(xi, kmax=20000, eps=1e-9)
    np.testing.assert_allclose(u, xi, atol=2e-4)
    xi = np.linspace(0.0, 1.0, 7)
    h = 1e-5
    u, du, d2u = wl.smoothed_sawtooth(xi)
    up, dup, _ = wl.smoothed_sawtooth(xi + h)
    um, dum, _ = wl.smoothed_sawtooth(xi - h)
    np.testing.assert_allclose(du, (up - um) / (2 * h), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(d2u, (dup - dum) / (2 * h), rtol=1e-6, atol=1e-4)


def test_burgers_travelling_sawtooth_error_is_second_order_in_dx():
    """Sec. 4 travelling wave (Fig. error_differentdx): with the averaged-Jacobian WR the
    error against the manufactured solution settles at a value set by the mesh, and halving
    dx divides it by about 4 (second-order central differences).  Here T = 0.5 with the
    paper's subinterval length 0.1, s = 50 samples, m = 12, tol 1e-4."""
    floors = []
    for n in (64, 128):
        pr = wl.burgers_sawtooth(n=n, T=0.5, P=5, s=50, svd_tol=1e-6, wr_tol=1e-12, wr_max_iter=8, restart_len=40)
        errs = []
        ob.solve_burgers_jacobian(pr.op, pr.opts, pr.u0, forcing=pr.G,
                                  callback=lambda k, Uk, d: errs.append(
                                      np.max(np.linalg.norm(Uk - pr.meta["exact"], axis=1)
                                             / np.linalg.norm(pr.meta["exact"], axis=1))))
        assert errs[-1] < 0.05 * errs[0]
        assert abs(errs[-1] - errs[-2]) < 0.05 * errs[-1]   # settled at the mesh's error
        floors.append(errs[-1])
    assert 3.2 < floors[0] / floors[1] < 5.0, floors


@pytest.mark.parametrize("k0", [4, 16])
def test_burgers_multiscale_with_discrete_forcing_has_no_spatial_error(k0):
    """Sec. 4 multiscale example, with the forcing of the Burgers efficiency runs: it is
    built from the discrete operators (f = u_t - A u - g(u) at the grid points), so the
    semi-discrete solution is the exact one and the WR error is time integration alone.
    Its floor therefore does not change with dx, and widening the spectrum (k0 = 16) does
    not slow the iterations down."""
    floors, reach = [], []
    for n in (64, 128):
        P, s, T = 2, 33, 0.2
        n_out = P * (s - 1) + 1
        t = wl.out_times(T, n_out)
        x = wl.grid_1d(n)
        op = wl.make_op(n, 1e-2, 0.0)
        A = ob.operator_matrix(op)
        U = np.zeros((n_out, n))
        F = np.zeros((n_out, n))
        for i, tt in enumerate(t):
            u, ut = wl.multiscale_solution(x, tt, k0)
            U[i] = u
            F[i] = ut - A @ u - ob.burgers_source(op, u, 0)
        opts = wl.default_opts(T=T, P=P, n_out=n_out, tol=1e-8, svd_tol=1e-10, max_rank=12, wr_tol=1e-12,
                               wr_max_iter=9, restart_len=40)
        errs = []
        ob.solve_burgers_jacobian(op, opts, U[0], forcing=F, callback=lambda k, Uk, d: errs.append(
            np.max(np.linalg.norm(Uk - U, axis=1)) / np.max(np.linalg.norm(U, axis=1))))
        floors.append(errs[-1])
        reach.append(next(k for k, e in enumerate(errs) if e < 2 * errs[-1]) + 1)
    assert max(floors) < 1e-5, floors
    assert 1 / 1.3 < floors[0] / floors[1] < 1.3, floors
    assert max(reach) <= 8, reach


def _sawtooth_discrete_errors(P, T, s, iters, n=64):
    """WR error history on the travelling sawtooth with the discretely manufactured forcing
    (semi-discrete solution exact), max over output times, relative to max ||u||."""
    x = wl.grid_1d(n)
    op = wl.make_op(n, 1e-2, 0.0)
    A = ob.operator_matrix(op)
    n_out = P * (s - 1) + 1
    t = wl.out_times(T, n_out)
    U = np.zeros((n_out, n))
    F = np.zeros((n_out, n))
    for i, tt in enumerate(t):
        u, du, _ = wl.smoothed_sawtooth(x - tt / 2 + 0.5)
        U[i] = u
        F[i] = -0.5 * du - A @ u - ob.burgers_source(op, u, 0)   # u_t = -u'/2 for xi = x - t/2 + 1/2
    opts = wl.default_opts(T=T, P=P, n_out=n_out, tol=1e-8, svd_tol=1e-10, max_rank=12, wr_tol=1e-14,
                           wr_max_iter=iters, restart_len=40)
    errs = []
    ob.solve_burgers_jacobian(op, opts, U[0], forcing=F, callback=lambda k, Uk, d: errs.append(
        np.max(np.linalg.norm(Uk - U, axis=1)) / np.max(np.linalg.norm(U, axis=1))))
    return errs


def test_burgers_iterations_grow_with_the_interval_and_shrink_with_the_subinterval():
    """Sec. 4 (Fig. be1_history): with a fixed subinterval length (T = P dT) the WR error
    after a fixed number of iterations grows with P, because the interval grows; with a
    fixed T (dT = T/P, the samples kept) it falls with P, because the averaged Jacobian is a
    better model on shorter subintervals (Sec. 4, parallel efficiency)."""
    k = 4
    fixed_dt = [_sawtooth_discrete_errors(P, 0.1 * P, 33, k)[-1] for P in (1, 2, 4)]
    fixed_t = [_sawtooth_discrete_errors(P, 0.2, 64 // P + 1, k)[-1] for P in (1, 2, 4)]
    assert fixed_dt[0] < fixed_dt[1] < fixed_dt[2], fixed_dt
    assert fixed_t[0] > fixed_t[1] > fixed_t[2], fixed_t


@pytest.mark.parametrize("krylov", [0, 1])
@pytest.mark.parametrize("bc", [wl.BC_PERIODIC, wl.BC_DIRICHLET0])
def test_oracle_matches_dense_bruteforce_2d(krylov, bc):
    """The 2D five-point operator (the large configuration's operator) in both Krylov
    spaces, nx * ny = 48 <= 64 unknowns, against the exponential of the full augmented
    matrix with the same source model."""
    nx, ny = 8, 6
    op = wl.make_op(nx, 2e-2, 0.7, dim=2, ny=ny, ay=-0.4, bc=bc)
    xs = wl.grid_1d(nx, bc=bc)
    ys = wl.grid_1d(ny, bc=bc)
    X, Yg = np.meshgrid(xs, ys)                   # unknown (ix, iy) at index iy * nx + ix
    u0 = (np.sin(np.pi * X) * np.cos(np.pi * Yg) + 0.3 * X * Yg).ravel()
    t = wl.out_times(0.4, 17)
    G = np.cos(4 * t)[:, None] * (X * (1 - Yg)).ravel()[None, :] + t[:, None] * np.sin(2 * np.pi * Yg).ravel()[None, :]
    opts = wl.default_opts(T=0.4, P=4, n_out=17, tol=1e-13, svd_tol=1e-14, krylov=krylov, restart_len=40)
    Y, rep = ob.solve_linear(op, opts, u0, G)
    assert all(rep["conv_nh"]) and all(all(c) for c in rep["conv_hom"])
    tt, wins = cf.fourier_windows_from_oracle_model(op, opts, u0, G, ob.compress_source,
                                                    ob.spline_segments, ob.partition)
    Yx = cf.dense_exact(ob.operator_matrix(op).toarray(), u0, tt, wins)
    err = np.max(np.linalg.norm(Y - Yx, axis=1) / np.linalg.norm(Yx, axis=1))
    assert err < 1e-10, err


def test_wr_stopping_rule():
    """Waveform relaxation stops on a small update, or on an update that grew wr_diverge
    times in a row (the paper gives no divergence rule); 0 disables the latter."""
    o = dict(wr_tol=1e-6, wr_diverge=3)
    assert ob._wr_stop([1e-2, 1e-7], o) == "converged"
    assert ob._wr_stop([1.0, 2.0, 3.0], o) is None          # two growths
    assert ob._wr_stop([1.0, 2.0, 3.0, 4.0], o) == "diverged"
    assert ob._wr_stop([1.0, 2.0, 1.5, 3.0, 4.0], o) is None  # the run of growths restarted
    assert ob._wr_stop([1.0, 2.0, 3.0, 4.0], dict(o, wr_diverge=0)) is None


def test_picard_divergence_is_detected():
    """The Picard updates grow on this case (the averaged-Jacobian pin below converges on
    it): the oracle stops at the third growth in a row and says so."""
    op, opts, u0, _ = _burgers_case(0.3, 1e-2, 30)
    _, rp = ob.solve_burgers(op, dict(opts, wr_diverge=3), u0)
    d = rp["deltas"]
    assert rp["diverged"] and not rp["converged"] and len(d) < 30, d
    assert d[-1] > d[-2] > d[-3] > d[-4]


# ---------------------------------------------------------------- Chebyshev sample nodes (Sec. 3)
def test_chebyshev_samples_are_the_extrema_of_the_chebyshev_polynomial():
    """The sample times of nodes=1: per subinterval, the ends and the zeros of T'_{s-1} (the
    extrema of the Chebyshev polynomial) mapped onto [T_{j-1}, T_j]; the caller's sampling
    (workloads) and the oracle's agree."""
    from numpy.polynomial import chebyshev as npc
    P, n_out, s = 3, 13, 7
    opts = wl.default_opts(T=0.6, P=P, n_out=n_out, nodes=1, n_samp=s)
    ts, sidx = ob.sample_partition(opts)
    assert sidx == [0, 6, 12, 18] and ts.size == P * (s - 1) + 1
    np.testing.assert_allclose(ts, wl.chebyshev_sample_times(0.6, P, n_out, s), rtol=0, atol=1e-15)
    t = wl.out_times(0.6, n_out)
    ext = np.sort(npc.Chebyshev.basis(s - 1).deriv().roots().real)   # interior extrema in (-1, 1)
    for j, (i0, i1) in enumerate(zip(ob.partition(n_out, P)[:-1], ob.partition(n_out, P)[1:])):
        a, b = t[i0], t[i1]
        w = ts[sidx[j]:sidx[j + 1] + 1]
        assert w[0] == a and w[-1] == b
        # x = -cos(pi i/(s-1)) runs from -1 to 1: t = a + (b - a)(x + 1)/2
        np.testing.assert_allclose(np.sort(2 * (w[1:-1] - a) / (b - a) - 1), ext, atol=1e-13)


def _cubic_in_time_case(s):
    n, nu, a = 256, 1e-2, 1.0
    x = wl.grid_1d(n)
    u0 = np.sin(2 * np.pi * x)
    v = np.sin(4 * np.pi * x)
    fc = np.array([1.0, 2.0, -3.0, 1.5])          # f(t) = sum_l fc_l t^l
    opts = wl.default_opts(T=0.6, P=3, n_out=13, tol=1e-13, restart_len=40, nodes=1, n_samp=s)
    ts, _ = ob.sample_partition(opts)
    f = sum(fc[l] * ts ** l for l in range(4))
    G = f[:, None] * v[None, :]
    return n, nu, a, u0, v, fc, opts, G


@pytest.mark.parametrize("s", [4, 7, 9])
def test_chebyshev_samples_reproduce_a_cubic_source_exactly(s):
    """A source cubic in time is its own spline on any knots, so with Chebyshev samples the
    method is exact up to the Krylov tolerance: per Fourier mode,
    u(t) = e^{lam t} u0 + sum_l l! fc_l t^{l+1} phi_{l+1}(lam t) v (the outputs lie between
    the knots, so this pins the evaluation inside a knot interval)."""
    n, nu, a, u0, v, fc, opts, G = _cubic_in_time_case(s)
    Y, rep = ob.solve_linear(wl.make_op(n, nu, a), opts, u0, G)
    assert all(rep["conv_nh"])
    lam = cf.circulant_eigs(n, a, nu)
    u0h, vh = np.fft.fft(u0), np.fft.fft(v)
    for i, tt in enumerate(wl.out_times(0.6, 13)):
        ph = cf.phi_functions(lam * tt)
        yh = ph[0] * u0h + sum(math.factorial(l) * fc[l] * tt ** (l + 1) * ph[l + 1] * vh for l in range(4))
        ref = np.real(np.fft.ifft(yh))
        assert np.linalg.norm(Y[i] - ref) <= 1e-11 * np.linalg.norm(ref), i


def test_chebyshev_samples_with_the_true_source():
    """g = sin(4 pi x) cos(2 pi t) sampled at Chebyshev points: the solution stays within the
    spline's time error of the exact semi-discrete one (per mode,
    int_0^t e^{lam (t-s)} cos(w s) ds in closed form); samples taken at other times than the
    solver assumes would be O(1e-2) off."""
    n, nu, a, T, P, n_out, s = 512, 1e-2, 1.0, 1.0, 8, 101, 13
    pr = wl.adv_diff_1d(n=n, nu=nu, a=a, T=T, P=P, n_out=n_out, tol=1e-12, restart_len=30, nodes=1, n_samp=s)
    Y, rep = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)
    assert all(rep["conv_nh"])
    x = wl.grid_1d(n)
    lam = cf.circulant_eigs(n, a, nu)
    u0h, gh = np.fft.fft(pr.u0), np.fft.fft(np.sin(4 * np.pi * x))
    w = 2 * np.pi
    err = 0.0
    for i, tt in enumerate(wl.out_times(T, n_out)):
        el = np.exp(lam * tt)
        I = 0.5 * ((np.exp(1j * w * tt) - el) / (1j * w - lam) + (np.exp(-1j * w * tt) - el) / (-1j * w - lam))
        ref = np.real(np.fft.ifft(el * u0h + I * gh))
        err = max(err, np.linalg.norm(Y[i] - ref) / np.linalg.norm(ref))
    assert err < 1e-6, err


# ---------------------------------------------------------------- restarting (Sec. 2.1, Sec. 3)
def _restart_err(krylov, n, nu, P, n_out, T, rl, mr):
    pr = wl.adv_diff_1d(n=n, nu=nu, P=P, n_out=n_out, T=T, tol=1e-12, restart_len=rl, max_restarts=mr,
                        krylov=krylov)
    Y, rep = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)
    t, wins = cf.fourier_windows_from_oracle_model(pr.op, pr.opts, pr.u0, pr.G, ob.compress_source,
                                                   ob.spline_segments, ob.partition)
    Yx = cf.exact_piecewise_cubic(cf.circulant_eigs(n, 1.0, nu), pr.u0, t, wins)
    return float(np.max(np.linalg.norm(Y - Yx, axis=1) / np.linalg.norm(Yx, axis=1))), rep


def test_restarted_polynomial_krylov_matches_the_closed_form():
    """Restart cycles of 4 and 6 block steps in the polynomial space: every subproblem restarts
    and still converges to the exact solution with the same source model, in at most one cycle
    more than without restarts (the cycle's residual lies in the next block)."""
    e0, r0 = _restart_err(0, 128, 1e-3, 4, 33, 0.25, 40, 0)
    for rl, mr in ((4, 20), (6, 10)):
        e, rep = _restart_err(0, 128, 1e-3, 4, 33, 0.25, rl, mr)
        assert all(rep["conv_nh"]) and all(all(c) for c in rep["conv_hom"])
        assert min(rep["restarts_nh"]) >= 2
        assert e < 1e-11, (rl, e)
        assert max(rep["k_nh"]) <= max(r0["k_nh"]) + rl   # at most one cycle more


def test_restarted_shift_and_invert_krylov_matches_the_closed_form():
    """Restart cycles of 8 block steps in the shift-and-invert space, on a case that needs 24
    steps without restarts: the restarted solve converges to the exact solution."""
    e, rep = _restart_err(1, 1024, 1e-2, 4, 41, 1.0, 8, 10)
    assert all(rep["conv_nh"]) and all(all(c) for c in rep["conv_hom"])
    assert min(rep["restarts_nh"]) >= 2 and max(max(r) for r in rep["restarts_hom"] if r) >= 2
    assert e < 1e-10, e


@pytest.mark.parametrize("krylov", [0, 1])
def test_restart_residual_has_the_block_rank(krylov):
    """The residual factor (I - V V^T) A V of a block Krylov basis has rank b: its singular
    values beyond the block width are at round-off level (what restart_block relies on)."""
    n, b = 256, 2
    pr = wl.adv_diff_1d(n=n, nu=1e-2, P=1, n_out=5)
    A = ob.operator_matrix(pr.op)
    kop = ob.KrylovOperator(pr.op, A, krylov, 0.01)
    V, _ = np.linalg.qr(np.column_stack([pr.u0, np.sin(4 * np.pi * wl.grid_1d(n))]))
    last = V
    for _ in range(4):
        new = ob.block_krylov_step(kop, V, last)
        V, last = np.hstack([V, new]), new
    Z = A @ V - V @ (V.T @ (A @ V))
    sv = np.linalg.svd(Z, compute_uv=False)
    assert sv[b] < 1e-8 * sv[0], sv[:b + 2]


def test_restarted_solve_stops_within_its_tolerance():
    """At tol 1e-7 with cycles of 4 and 8 blocks the restarted solve ends within 10 tol of the
    closed form: a restart cycle is not tested for convergence at its first step, where the
    step-to-step change is far below the error."""
    for rl, mr in ((4, 15), (8, 7)):
        pr = wl.adv_diff_1d(n=1024, nu=1e-2, P=4, n_out=41, T=1.0, tol=1e-7, restart_len=rl, max_restarts=mr)
        Y, rep = ob.solve_linear(pr.op, pr.opts, pr.u0, pr.G)
        assert all(rep["conv_nh"]) and min(rep["restarts_nh"]) >= 1
        t, wins = cf.fourier_windows_from_oracle_model(pr.op, pr.opts, pr.u0, pr.G, ob.compress_source,
                                                       ob.spline_segments, ob.partition)
        Yx = cf.exact_piecewise_cubic(cf.circulant_eigs(1024, 1.0, 1e-2), pr.u0, t, wins)
        err = float(np.max(np.linalg.norm(Y - Yx, axis=1) / np.linalg.norm(Yx, axis=1)))
        assert err < 1e-6, (rl, err)


def test_shift_and_invert_arnoldi_relation_gives_the_residual_range():
    """The GPU starts a restart cycle from q = V' - gamma (I - V V^T) A V' (V' the block that
    the cycle's next step would add), by the cycle's Arnoldi relation for (I - gamma A)^{-1};
    the oracle from an SVD of (I - V V^T) A V.  Both are the same subspace."""
    n, b, gamma = 512, 2, 0.02
    pr = wl.adv_diff_1d(n=n, nu=1e-2, P=1, n_out=5)
    A = ob.operator_matrix(pr.op)
    kop = ob.KrylovOperator(pr.op, A, ob.KRYLOV_SAI, gamma)
    x = wl.grid_1d(n)
    V, _ = np.linalg.qr(np.column_stack([pr.u0, np.exp(-50 * (x - 0.3) ** 2)]))
    last = V
    for _ in range(3):
        new = ob.block_krylov_step(kop, V, last)
        assert new.shape[1] == b
        V, last = np.hstack([V, new]), new
    Vn = ob.block_krylov_step(kop, V, last)          # V'
    AVn = A @ Vn
    q = Vn - gamma * (AVn - V @ (V.T @ AVn))
    Q = np.linalg.qr(q)[0]
    R = ob.restart_block(V, A @ V, b)
    assert R.shape[1] == b
    # the two orthonormal bases span the same space: singular values of Q^T R are all 1
    sv = np.linalg.svd(Q.T @ R, compute_uv=False)
    np.testing.assert_allclose(sv, 1.0, atol=1e-9)
