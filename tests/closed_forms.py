"""Closed-form and brute-force references that pin the oracle (test-only).

Nothing here calls into ``oracle/``'s Krylov, projection or time-stepping code.
Each reference follows the mathematics directly:

* ``circulant_eigs``: eigenvalues of the periodic central-difference operator
  (Sec. 3.1) from its symbol, lambda_k = -(4 nu/dx^2) sin^2(pi k/n) - i (a/dx) sin(2 pi k/n).
* ``phi_functions``: scalar phi_l(z) = sum_j z^j/(j+l)! (Taylor for |z| < 2, the
  recurrence phi_{l+1} = (phi_l - 1/l!)/z otherwise).
* ``exact_piecewise_cubic``: the exact solution, mode by mode in Fourier space, of
  u_hat' = A u_hat + U_j p_j(t) with the piecewise-cubic source model, summed over
  subintervals -- the semi-discrete solution the PEBK method approximates.
* ``dense_exact``: the same solution by the exponential of the full (n <= 64)
  augmented matrix, any boundary condition.
* ``pulse_series``: the Fourier-series solution of the pulse problem, eq. pulseADE.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def circulant_eigs(n: int, a: float, nu: float, L: float = 1.0) -> np.ndarray:
    dx = L / n
    k = np.arange(n)
    th = 2 * np.pi * k / n
    return -(4 * nu / dx ** 2) * np.sin(th / 2) ** 2 - 1j * (a / dx) * np.sin(th)


def phi_functions(z: np.ndarray, L: int = 4) -> np.ndarray:
    z = np.asarray(z, dtype=complex)
    out = np.zeros((L + 1,) + z.shape, complex)
    small = np.abs(z) < 2.0
    out[0] = np.exp(z)
    zz = np.where(small, 1.0, z)
    for l in range(1, L + 1):
        out[l] = (out[l - 1] - 1.0 / math.factorial(l - 1)) / zz
    zs = z[small]
    for l in range(1, L + 1):
        acc = np.zeros_like(zs)
        term = np.ones_like(zs) / math.factorial(l)
        for j in range(60):
            acc = acc + term
            term = term * zs / (l + j + 1)
        out[l][small] = acc
    return out


def exact_piecewise_cubic(lam: np.ndarray, u0: np.ndarray, t: np.ndarray, windows) -> np.ndarray:
    """Exact u(t_i) = u0 + u_hat(t_i) for a circulant A (eigenvalues `lam` in FFT order).

    windows: list of (i0, i1, U, coef) per subinterval -- U (n, m) and the cubic
    coefficients coef[i, l] (m,) on each sample interval [t_{i0+i}, t_{i0+i+1}].
    Integrates every Fourier mode exactly with the phi-functions over every sample
    interval: y_{i+1} = e^{lam h} y_i + sum_l l! h^{l+1} phi_{l+1}(lam h) g_l."""
    n = u0.size
    n_out = t.size
    yh = np.zeros(n, complex)
    out = np.zeros((n_out, n))
    out[0] = u0
    seg = {}
    for (i0, i1, U, coef) in windows:
        Uh = np.fft.fft(U, axis=0) if U.shape[1] else np.zeros((n, 0), complex)
        for i in range(i0, i1):
            seg[i] = (Uh, coef[i - i0])
    for i in range(n_out - 1):
        h = t[i + 1] - t[i]
        ph = phi_functions(lam * h)
        yn = ph[0] * yh
        if i in seg:
            Uh, c = seg[i]
            if Uh.shape[1]:
                for l in range(4):
                    yn = yn + math.factorial(l) * h ** (l + 1) * ph[l + 1] * (Uh @ c[l])
        yh = yn
        out[i + 1] = u0 + np.real(np.fft.ifft(yh))
    return out


def exact_at_samples(lam: np.ndarray, u0: np.ndarray, t: np.ndarray, windows, keep) -> dict:
    """exact_piecewise_cubic at the output indices `keep` only, for large n.

    The samples are uniform (spacing h) and `windows` may be a generator consumed in time
    order.  The per-interval recurrence of exact_piecewise_cubic is summed in closed form:
    s intervals after the window start t_{i0},
        y(t_{i0+s}) = e^{lam s h} y(t_{i0})
                      + sum_l l! h^{l+1} phi_{l+1}(lam h) sum_r Uh[:, r] sum_{q<s} e^{lam (s-1-q) h} coef[q, l, r],
    so each window costs a few (n, s) products and only the kept outputs are transformed
    back.  Returns {index: u(t_index)}."""
    keep = sorted(set(int(k) for k in keep))
    h = t[1] - t[0]
    ph = phi_functions(lam * h)
    a = [math.factorial(l) * h ** (l + 1) * ph[l + 1] for l in range(4)]
    yh = np.zeros(u0.size, complex)
    res = {0: u0.copy()} if 0 in keep else {}

    def advance(y, Uh, coef, s):
        out = np.exp(lam * (s * h)) * y
        if Uh is None or s == 0:
            return out
        E = np.empty((s, lam.size), complex)  # E[q] = e^{lam (s-1-q) h}
        E[s - 1] = 1.0
        for q in range(s - 2, -1, -1):
            np.multiply(E[q + 1], ph[0], out=E[q])
        for l in range(4):
            out += a[l] * np.einsum("ir,ir->i", Uh, E.T @ coef[:s, l, :])
        return out

    for (i0, i1, U, coef) in windows:
        Uh = np.fft.fft(U, axis=0) if U.shape[1] else None
        for k in keep:
            if i0 < k < i1:
                res[k] = u0 + np.real(np.fft.ifft(advance(yh, Uh, coef, k - i0)))
        yh = advance(yh, Uh, coef, i1 - i0)
        if i1 in keep:
            res[i1] = u0 + np.real(np.fft.ifft(yh))
    return res


def exact_piecewise_operators(lams: list, u0: np.ndarray, t: np.ndarray, windows) -> np.ndarray:
    """Exact u(t_i) = u0 + u_hat(t_i) when subinterval j has its own circulant operator
    (eigenvalues lams[j-1], FFT order) and source model (U_j, coef_j): u_hat is carried
    across the subinterval ends and advanced in each subinterval, mode by mode, with that
    subinterval's eigenvalues and phi-functions (the recurrence of exact_piecewise_cubic)."""
    n_out = t.size
    yh = np.zeros(u0.size, complex)
    out = np.zeros((n_out, u0.size))
    out[0] = u0
    for lam, (i0, i1, U, coef) in zip(lams, windows):
        Uh = np.fft.fft(U, axis=0) if U.shape[1] else None
        for i in range(i0, i1):
            h = t[i + 1] - t[i]
            ph = phi_functions(lam * h)
            yn = ph[0] * yh
            if Uh is not None:
                for l in range(4):
                    yn = yn + math.factorial(l) * h ** (l + 1) * ph[l + 1] * (Uh @ coef[i - i0][l])
            yh = yn
            out[i + 1] = u0 + np.real(np.fft.ifft(yh))
    return out


def dense_exact(A: np.ndarray, u0: np.ndarray, t: np.ndarray, windows) -> np.ndarray:
    """Same as exact_piecewise_cubic for any dense A (n small): the exponential of the
    augmented matrix [[hA, hU, 0..], [0, 0, I, ..], ...] of size n + 4m on each sample
    interval, cross-checked in tests against a long-double Taylor series."""
    n = u0.size
    out = np.zeros((t.size, n))
    out[0] = u0
    y = np.zeros(n)
    seg = {}
    for (i0, i1, U, coef) in windows:
        for i in range(i0, i1):
            seg[i] = (U, coef[i - i0])
    for i in range(t.size - 1):
        h = t[i + 1] - t[i]
        if i in seg and seg[i][0].shape[1]:
            U, c = seg[i]
            m = U.shape[1]
            M = np.zeros((n + 4 * m, n + 4 * m))
            M[:n, :n] = h * A
            M[:n, n:n + m] = h * U
            for l in range(3):
                M[n + l * m:n + (l + 1) * m, n + (l + 1) * m:n + (l + 2) * m] = np.eye(m)
            E = sla.expm(M)
            yn = E[:n, :n] @ y
            for l in range(4):
                yn = yn + math.factorial(l) * h ** l * (E[:n, n + l * m:n + (l + 1) * m] @ c[l])
            y = yn
        else:
            y = sla.expm(h * A) @ y
        out[i + 1] = u0 + y
    return out


def taylor_expm_longdouble(M: np.ndarray, terms: int = 80) -> np.ndarray:
    """exp(M) by scaling and squaring a long-double Taylor series (brute force)."""
    Ml = M.astype(np.longdouble)
    nrm = float(np.max(np.sum(np.abs(M), axis=0)))
    s = max(0, int(math.ceil(math.log2(nrm))) + 1) if nrm > 0.5 else 0
    Ml = Ml / np.longdouble(2.0) ** s
    E = np.eye(M.shape[0], dtype=np.longdouble)
    term = np.eye(M.shape[0], dtype=np.longdouble)
    for j in range(1, terms):
        term = term @ Ml / np.longdouble(j)
        E = E + term
    for _ in range(s):
        E = E @ E
    return E


def pulse_series(x: np.ndarray, t: float, a: float, nu: float) -> np.ndarray:
    """Exact solution of eq. pulseADE, u0 = sin^20(pi x): by the binomial expansion
    sin^{2N}(th) = 2^{-2N} [C(2N,N) + 2 sum_k (-1)^k C(2N,N-k) cos(2k th)], each cosine
    mode advected with speed a and damped by exp(-(2 k pi)^2 nu t)."""
    N = 10
    u = np.full_like(x, math.comb(2 * N, N) / 4 ** N)
    for k in range(1, N + 1):
        ak = 2 * (-1) ** k * math.comb(2 * N, N - k) / 4 ** N
        u = u + ak * np.cos(2 * k * np.pi * (x - a * t)) * math.exp(-(2 * k * np.pi) ** 2 * nu * t)
    return u


def iter_windows_from_oracle_model(op, opts, u0, G, compress, spline, partition, workers: int = 8):
    """Generator form of fourier_windows_from_oracle_model: windows come in time order,
    built `workers` at a time on threads (the SVDs release the GIL), so at most that many
    windows are held at once."""
    import collections
    from concurrent.futures import ThreadPoolExecutor
    import oracle.pebk as ob
    n_out, P, T = opts["n_out"], opts["P"], opts["T"]
    t = np.arange(n_out) * (T / (n_out - 1))
    idx = partition(n_out, P)
    Au0 = ob.operator_matrix(op) @ u0

    def window(j):
        i0, i1 = idx[j - 1], idx[j]
        Ghat = np.tile(Au0[:, None], (1, i1 - i0 + 1))
        if G is not None:
            Ghat = Ghat + G[i0:i1 + 1].T
        U, C, _ = compress(Ghat, opts["svd_tol"], opts["max_rank"])
        return (i0, i1, U, spline(t[i0:i1 + 1] - t[i0], C))

    with ThreadPoolExecutor(max(1, workers)) as ex:
        pending = collections.deque()
        for j in range(1, P + 1):
            pending.append(ex.submit(window, j))
            if len(pending) >= max(1, workers):
                yield pending.popleft().result()
        while pending:
            yield pending.popleft().result()


def fourier_windows_from_oracle_model(op, opts, u0, G, compress, spline, partition):
    """Per-window source model (U_j, coef_j) built with the oracle's source-compression
    step -- the closed forms then integrate that model exactly."""
    import oracle.pebk as ob
    n_out, P, T = opts["n_out"], opts["P"], opts["T"]
    t = np.arange(n_out) * (T / (n_out - 1))
    idx = partition(n_out, P)
    Au0 = ob.operator_matrix(op) @ u0
    wins = []
    for j in range(1, P + 1):
        i0, i1 = idx[j - 1], idx[j]
        Ghat = np.tile(Au0[:, None], (1, i1 - i0 + 1))
        if G is not None:
            Ghat = Ghat + G[i0:i1 + 1].T
        U, C, _ = compress(Ghat, opts["svd_tol"], opts["max_rank"])
        coef = spline(t[i0:i1 + 1] - t[i0], C)
        wins.append((i0, i1, U, coef))
    return t, wins
