"""Seeded synthetic inputs shaped like the paper's workloads.

This module only generates inputs: grids, initial conditions, source samples
and per-instance parameters.  It holds none of the method's arithmetic (no
difference operator, no shift by the initial condition, no Krylov step), so the
oracle and the CUDA path can both draw their inputs from here while sharing no
computation.

Shapes follow the paper's experiments: 1D periodic advection-diffusion on
[0, 1) with second-order central differences (Sec. 3.1, Sec. 3.2), the viscous
Burgers equation by waveform relaxation (Sec. 4), and output/sample times on a
uniform grid over [0, T].

Array conventions: a state vector is a length-n float array; a time series of
n-vectors (sources G, solutions Y) is an array of shape (n_out, n) in C order,
so that the n values at one output time are contiguous ("time-major").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import Optional

import numpy as np

SEED_BASE = 20150915

BC_PERIODIC = 0
BC_DIRICHLET0 = 1


@dataclass
class Problem:
    """One linear problem u' = A u + g(t), u(0) = u0 on [0, T] (eq. ivp2).

    ``op`` describes A: dim (1 or 2), nx, ny, bc, advection velocities ax, ay,
    diffusivity nu and domain lengths Lx, Ly.  ``opts`` holds the solver
    options (T, P, n_out, tol, ...).  ``u0`` and ``G`` are float64 arrays;
    ``G`` has shape (n_out, n) or is None for a zero source.
    """
    name: str
    op: dict
    opts: dict
    u0: np.ndarray
    G: Optional[np.ndarray]
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.op["nx"] * (self.op["ny"] if self.op["dim"] == 2 else 1))


def default_opts(**kw) -> dict:
    o = dict(T=1.0, P=1, n_out=2, tol=1e-8, svd_tol=1e-12, max_rank=16,
             restart_len=20, max_restarts=0, krylov=1, sai_gamma=0.1,
             precision=0, wr_max_iter=50, wr_tol=1e-6, burgers_form=0, diagnostics=0, jacobian=0,
             wr_diverge=3, sub_first=0, sub_last=0, nodes=0, n_samp=0)
    o.update(kw)
    return o


def make_op(nx, nu, ax=0.0, bc=BC_PERIODIC, dim=1, ny=1, ay=0.0, Lx=1.0, Ly=1.0) -> dict:
    return dict(dim=dim, nx=int(nx), ny=int(ny), bc=int(bc), ax=float(ax), ay=float(ay),
                nu=float(nu), Lx=float(Lx), Ly=float(Ly))


def grid_1d(n: int, L: float = 1.0, bc: int = BC_PERIODIC) -> np.ndarray:
    """Grid points of the 1D mesh: x_i = i*dx on [0, L) for periodic meshes,
    interior points x_i = (i+1)*dx with dx = L/(n+1) for homogeneous Dirichlet."""
    if bc == BC_PERIODIC:
        return np.arange(n, dtype=np.float64) * (L / n)
    return (np.arange(n, dtype=np.float64) + 1.0) * (L / (n + 1))


def out_times(T: float, n_out: int) -> np.ndarray:
    return np.arange(n_out, dtype=np.float64) * (T / (n_out - 1))


def chebyshev_sample_times(T: float, P: int, n_out: int, n_samp: int) -> np.ndarray:
    """Where a caller samples the source for Chebyshev sampling (Sec. 3): n_samp Chebyshev
    extrema in each subinterval [T_{j-1}, T_j], both ends included and shared with the
    neighbour, P (n_samp - 1) + 1 times in all.  The boundaries are output times,
    T_j = t_floor(j (n_out-1)/P); subinterval j's i-th sample is
    T_{j-1} + (T_j - T_{j-1}) (1 - cos(pi i / (n_samp - 1))) / 2."""
    t = out_times(T, n_out)
    bnd = [t[(j * (n_out - 1)) // P] for j in range(P + 1)]
    i = np.arange(n_samp - 1, dtype=np.float64)
    ts = [bnd[j] + (bnd[j + 1] - bnd[j]) * 0.5 * (1.0 - np.cos(np.pi * i / (n_samp - 1))) for j in range(P)]
    return np.concatenate(ts + [np.array([bnd[P]])])


def adv_diff_1d(n=1024, nu=1e-2, a=1.0, T=1.0, P=8, n_out=101, tol=1e-8,
                svd_tol=1e-12, max_rank=16, with_source=True, **kw) -> Problem:
    """1D periodic advection-diffusion, u0 = sin(2 pi x) + exp(-100 (x-0.5)^2),
    g(x,t) = sin(4 pi x) cos(2 pi t).  At n=1024, nu=1e-2, P=8, n_out=101 this is
    the small case; at n=2^20, nu=1e-3, P=64, n_out=1025 the large one.  With
    nodes=1, n_samp=s the source is sampled at s Chebyshev points per subinterval
    (chebyshev_sample_times) instead of at the output times."""
    x = grid_1d(n)
    u0 = np.sin(2 * np.pi * x) + np.exp(-100.0 * (x - 0.5) ** 2)
    t = out_times(T, n_out)
    if kw.get("nodes", 0) == 1:
        t = chebyshev_sample_times(T, P, n_out, kw["n_samp"])
    G = None
    if with_source:
        G = np.cos(2 * np.pi * t)[:, None] * np.sin(4 * np.pi * x)[None, :]
    return Problem(name=f"adv_diff_1d_n{n}", op=make_op(n, nu, a),
                   opts=default_opts(T=T, P=P, n_out=n_out, tol=tol, svd_tol=svd_tol,
                                     max_rank=max_rank, **kw),
                   u0=u0, G=G)


def pulse_ade(n=256, nu=1e-2, a=1.0, T=1.0, P=8, n_out=33, tol=1e-8, **kw) -> Problem:
    """Homogeneous pulse problem of Sec. 3.1 (eq. pulseADE): u0 = sin^20(pi x), no source."""
    x = grid_1d(n)
    u0 = np.sin(np.pi * x) ** 20
    return Problem(name=f"pulse_ade_n{n}", op=make_op(n, nu, a),
                   opts=default_opts(T=T, P=P, n_out=n_out, tol=tol, **kw), u0=u0, G=None)


def travelling_pulses(n=1000, nu=1e-2, a=1.0, T=1.0, P=2, n_out=201, tol=1e-4,
                      max_rank=2, **kw) -> Problem:
    """Manufactured travelling pulses of Sec. 3.2 (eq. manusol), u = 1/2 - 1/2 cos(10 pi (x - t));
    the PDE source is f = u_t + a u_x - nu u_xx evaluated analytically."""
    x = grid_1d(n)
    t = out_times(T, n_out)
    ph = 10 * np.pi * (x[None, :] - t[:, None])
    ut = -5 * np.pi * np.sin(ph)
    ux = 5 * np.pi * np.sin(ph)
    uxx = 50 * np.pi ** 2 * np.cos(ph)
    G = ut + a * ux - nu * uxx
    u0 = 0.5 - 0.5 * np.cos(10 * np.pi * x)
    return Problem(name=f"travelling_pulses_n{n}", op=make_op(n, nu, a),
                   opts=default_opts(T=T, P=P, n_out=n_out, tol=tol, max_rank=max_rank, **kw),
                   u0=u0, G=G, meta=dict(exact=lambda tt: 0.5 - 0.5 * np.cos(10 * np.pi * (x - tt))))


def smoothed_sawtooth(xi: np.ndarray, kmax: int = 100, eps: float = 0.1):
    """The smoothed sawtooth of Sec. 4 (eq. modifiedSawtooth): u(xi) = 1/2 - sum_k
    sin(2 pi k xi) Phi_k / (pi k), Phi_k = (pi k eps/2) / sinh(pi k eps/2), k = 1..kmax.
    Returns (u, u', u'') at the points xi."""
    k = np.arange(1, kmax + 1, dtype=np.float64)[:, None]
    phi = (np.pi * k * eps / 2) / np.sinh(np.pi * k * eps / 2)
    arg = 2 * np.pi * k * np.asarray(xi, dtype=np.float64)[None, :]
    s, c = np.sin(arg), np.cos(arg)
    u = 0.5 - np.sum(s * phi / (np.pi * k), axis=0)
    du = -np.sum(2 * c * phi, axis=0)
    d2u = np.sum(4 * np.pi * k * s * phi, axis=0)
    return u, du, d2u


def burgers_sawtooth(n=400, nu=1e-2, T=1.0, P=10, s=50, tol=1e-4, max_rank=12, kmax=100, eps=0.1,
                     **kw) -> Problem:
    """Burgers travelling wave of Sec. 4: the smoothed sawtooth moving right at speed 1/2,
    u(x, t) = u_saw(x - t/2 + 1/2), kept alive by the forcing f = u_t + u u_x - nu u_xx
    (evaluated analytically, so f = (u - 1/2) u' - nu u'').  s samples per subinterval
    (shared ends): n_out = P (s - 1) + 1.  `meta["exact"]` gives u at the output times."""
    x = grid_1d(n)
    n_out = P * (s - 1) + 1
    t = out_times(T, n_out)
    U = np.zeros((n_out, n))
    F = np.zeros((n_out, n))
    for i, tt in enumerate(t):
        u, du, d2u = smoothed_sawtooth(x - tt / 2 + 0.5, kmax, eps)
        U[i] = u
        F[i] = (u - 0.5) * du - nu * d2u
    return Problem(name=f"burgers_sawtooth_n{n}", op=make_op(n, nu, 0.0),
                   opts=default_opts(T=T, P=P, n_out=n_out, tol=tol, max_rank=max_rank, **kw),
                   u0=U[0].copy(), G=F, meta=dict(exact=U))


def multiscale_solution(x: np.ndarray, t: float, k0: int):
    """The multiscale Burgers solution of Sec. 4 (eq. multiscale_solution),
    u = sin(2 pi x) sin(2 pi t) + sin(2 k0 pi x) sin(2 k0 pi t) / k0, and its time derivative."""
    u = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * t) + np.sin(2 * k0 * np.pi * x) * np.sin(2 * k0 * np.pi * t) / k0
    ut = (2 * np.pi * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * t)
          + 2 * np.pi * np.sin(2 * k0 * np.pi * x) * np.cos(2 * k0 * np.pi * t))
    return u, ut


def burgers_1d(n=65536, nu=5e-3, T=0.5, P=32, n_out=513, tol=1e-8, svd_tol=1e-8,
               max_rank=16, wr_tol=1e-6, wr_max_iter=200, **kw) -> Problem:
    """Viscous Burgers u_t + u u_x = nu u_xx (Sec. 4), periodic, u0 = 0.5 + sin(2 pi x), no forcing."""
    x = grid_1d(n)
    u0 = 0.5 + np.sin(2 * np.pi * x)
    return Problem(name=f"burgers_n{n}", op=make_op(n, nu, 0.0),
                   opts=default_opts(T=T, P=P, n_out=n_out, tol=tol, svd_tol=svd_tol,
                                     max_rank=max_rank, wr_tol=wr_tol, wr_max_iter=wr_max_iter, **kw),
                   u0=u0, G=None)


def batched_params(i: int, n_min_log2=12, n_max_log2=18) -> dict:
    """The seeded draws of instance i of the batched workload: n log-uniform in
    [2^n_min_log2, 2^n_max_log2] rounded to a multiple of 64, nu log-uniform in
    [1e-4, 1e-1], a uniform in [0.5, 2], 16 Fourier amplitudes of u0 (cosine al, sine be,
    each U(-1, 1)), P = 2^U{2..6}, source amplitude gamma ~ U(0, 1)."""
    rng = np.random.default_rng(SEED_BASE + i)
    n = int(round(2.0 ** rng.uniform(n_min_log2, n_max_log2) / 64.0)) * 64
    n = max(n, 64)
    nu = 10.0 ** rng.uniform(-4, -1)
    a = rng.uniform(0.5, 2.0)
    al = rng.uniform(-1, 1, 16)
    be = rng.uniform(-1, 1, 16)
    P = 2 ** int(rng.integers(2, 7))
    gam = rng.uniform(0, 1)
    return dict(n=n, nu=nu, a=a, al=al, be=be, P=P, gam=gam)


def batched_instance(i: int, n_min_log2=12, n_max_log2=18, tol=1e-7, P_max: int | None = None) -> Problem:
    """Instance i of the batched workload (batched_params): u0 = sum_k (al_k cos 2 pi k x +
    be_k sin 2 pi k x) / k over k = 1..16, T = 1, n_out = 16 P + 1,
    g = gamma sin(4 pi x) cos(2 pi t).  P_max caps P (small test sets)."""
    d = batched_params(i, n_min_log2, n_max_log2)
    n, nu, a, al, be, gam = d["n"], d["nu"], d["a"], d["al"], d["be"], d["gam"]
    P = d["P"] if P_max is None else min(d["P"], P_max)
    x = grid_1d(n)
    k = np.arange(1, 17)[:, None]
    u0 = ((al[:, None] * np.cos(2 * np.pi * k * x) + be[:, None] * np.sin(2 * np.pi * k * x)) / k).sum(0)
    n_out = 16 * P + 1
    t = out_times(1.0, n_out)
    G = gam * np.cos(2 * np.pi * t)[:, None] * np.sin(4 * np.pi * x)[None, :]
    return Problem(name=f"batched_{i}", op=make_op(n, nu, a),
                   opts=default_opts(T=1.0, P=P, n_out=n_out, tol=tol, svd_tol=1e-10, max_rank=8),
                   u0=u0, G=G)


def random_block(n: int, b: int, seed: int) -> np.ndarray:
    """Seeded Gaussian n x b block (column-major in the (n, b) numpy sense)."""
    return np.random.default_rng(SEED_BASE + seed).standard_normal((n, b))


def smooth_block(n: int, b: int, seed: int, modes: int = 12) -> np.ndarray:
    """Seeded smooth periodic n x b block: random combinations of the first `modes`
    Fourier modes (the kind of vector the Krylov process works on)."""
    rng = np.random.default_rng(SEED_BASE + 7919 * seed + 1)
    x = grid_1d(n)
    out = np.zeros((n, b))
    for c in range(b):
        for k in range(modes + 1):
            out[:, c] += rng.standard_normal() * np.cos(2 * np.pi * k * x) / (1 + k)
            out[:, c] += rng.standard_normal() * np.sin(2 * np.pi * k * x) / (1 + k)
    return out
