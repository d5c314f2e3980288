"""ctypes binding of the PEBK C ABI (include/pexp.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
The library is loaded from paper_1509_04567_gb300/_lib/libpexp.so; if it is
missing the import raises -- there is no fallback implementation.

Device buffers are passed as torch CUDA tensors (their data_ptr), host buffers
as numpy arrays.  Time series use the time-major layout of the C ABI: a tensor of
shape (n_out, n), C-contiguous.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, fields

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpexp.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_OOM = -2
ERR_CUDA = -3
ERR_BREAKDOWN = -4
ERR_NOT_CONVERGED = -5
ERR_WR_NOT_CONVERGED = -6
ERR_TIMEOUT = -7
ERR_UNSUPPORTED = -8
ERR_SCRATCH_LIMIT = -9
ERR_WR_DIVERGED = -10

BC_PERIODIC = 0
BC_DIRICHLET0 = 1
KRYLOV_POLY = 0
KRYLOV_SAI = 1
DIAG_ORTH = 1
DIAG_KTIME = 2
DIAG_NOCOOP = 4


def DIAG_KTIME_CLASS(cls: int) -> int:
    """diagnostics bit that restricts PEXP_DIAG_KTIME to kernel class `cls` (index into KC_NAMES)."""
    return 1 << (8 + cls)


def DIAG_KTIME_SAMPLE(k: int) -> int:
    """diagnostics bits that make PEXP_DIAG_KTIME time about 1 in 2**k of the chosen launches."""
    return k << 16


KC_NAMES = ["sai", "stencil", "proj", "update", "small", "source", "recon", "other"]
REPORT_SUBS = 128
REPORT_WR = 64
FP64 = 0
MIXED = 1
F64 = 0
F32 = 1
NODES_UNIFORM = 0
NODES_CHEBYSHEV = 1

# Symbols declared in include/pexp.h (checked by the CPU tests).
EXPORTS = ["pexp_create", "pexp_destroy", "pexp_set_stream", "pexp_default_options", "pexp_status_string",
           "pexp_solve_linear", "pexp_solve_linear_host", "pexp_solve_burgers", "pexp_apply_operator",
           "pexp_sai_solve", "pexp_small_expm", "pexp_burgers_source", "pexp_sai_solve_noalloc",
           "pexp_jacobian_sai_solve", "pexp_solve_batched", "pexp_autotune", "pexp_selftest_barrier"]


class Operator(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int64), ("ny", C.c_int64), ("bc", C.c_int),
                ("ax", C.c_double), ("ay", C.c_double), ("nu", C.c_double), ("Lx", C.c_double),
                ("Ly", C.c_double)]


class Options(C.Structure):
    _fields_ = [("T", C.c_double), ("P", C.c_int), ("n_out", C.c_int), ("tol", C.c_double),
                ("svd_tol", C.c_double), ("max_rank", C.c_int), ("restart_len", C.c_int),
                ("max_restarts", C.c_int), ("krylov", C.c_int), ("sai_gamma", C.c_double),
                ("precision", C.c_int), ("wr_max_iter", C.c_int), ("wr_tol", C.c_double),
                ("burgers_form", C.c_int), ("diagnostics", C.c_int), ("jacobian", C.c_int),
                ("wr_diverge", C.c_int), ("sub_first", C.c_int), ("sub_last", C.c_int),
                ("nodes", C.c_int), ("n_samp", C.c_int)]


class Problem(C.Structure):
    _fields_ = [("op", Operator), ("opts", Options), ("y0_dev", C.c_void_p), ("G_dev", C.c_void_p),
                ("g_dtype", C.c_int), ("Y_dev", C.c_void_p), ("y_dtype", C.c_int)]


class Report(C.Structure):
    _fields_ = [("status", C.c_int), ("n_sub", C.c_int), ("rank_max", C.c_int), ("rank_min", C.c_int),
                ("k_nh_max", C.c_int), ("k_hom_max", C.c_int), ("k_hom_sum", C.c_int),
                ("not_converged", C.c_int), ("est_max", C.c_double), ("sigma_ratio_max", C.c_double),
                ("wr_iters", C.c_int), ("wr_delta", C.c_double), ("time_ms", C.c_double),
                ("t_source_ms", C.c_double), ("t_krylov_ms", C.c_double), ("t_hom_ms", C.c_double),
                ("t_recon_ms", C.c_double), ("orth_max", C.c_double), ("k_ms", C.c_double * 8),
                ("k_launches", C.c_int * 8), ("k_bytes", C.c_double * 8), ("bytes_alg", C.c_double),
                ("launches", C.c_int), ("k_bytes_alg", C.c_double * 8), ("sub_rank", C.c_int * REPORT_SUBS),
                ("sub_steps", C.c_int * REPORT_SUBS), ("sub_hom_steps", C.c_int * REPORT_SUBS),
                ("sub_restarts", C.c_int * REPORT_SUBS), ("wr_history", C.c_double * REPORT_WR)]

    def as_dict(self) -> dict:
        d = {}
        for f in self._fields_:
            v = getattr(self, f[0])
            d[f[0]] = list(v) if hasattr(v, "__len__") else v
        return d


_lib = None


def lib() -> C.CDLL:
    """Load libpexp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1509_04567_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.pexp_create.argtypes = [C.POINTER(vp), i, vp]
        L.pexp_destroy.argtypes = [vp]
        L.pexp_set_stream.argtypes = [vp, vp]
        L.pexp_default_options.argtypes = [C.POINTER(Options)]
        L.pexp_default_options.restype = None
        L.pexp_status_string.argtypes = [i]
        L.pexp_status_string.restype = C.c_char_p
        L.pexp_solve_linear.argtypes = [vp, C.POINTER(Operator), C.POINTER(Options), vp, vp, i, vp, i,
                                        C.POINTER(Report)]
        L.pexp_solve_linear_host.argtypes = L.pexp_solve_linear.argtypes
        L.pexp_selftest_barrier.argtypes = [C.c_void_p, C.c_int]
        L.pexp_solve_burgers.argtypes = [vp, C.POINTER(Operator), C.POINTER(Options), vp, vp, vp, vp, i,
                                         C.POINTER(Report)]
        L.pexp_apply_operator.argtypes = [vp, C.POINTER(Operator), vp, vp, i, i, i]
        L.pexp_sai_solve.argtypes = [vp, C.POINTER(Operator), d, vp, vp, i, i]
        L.pexp_small_expm.argtypes = [vp, vp, vp, i, i]
        L.pexp_burgers_source.argtypes = [vp, C.POINTER(Operator), vp, vp, i, i, i]
        L.pexp_sai_solve_noalloc.argtypes = [C.POINTER(Operator), d, vp, vp, i, i, vp]
        L.pexp_jacobian_sai_solve.argtypes = [vp, C.POINTER(Operator), d, vp, vp, vp, i, i]
        L.pexp_solve_batched.argtypes = [vp, i, C.POINTER(Problem), C.POINTER(Report)]
        L.pexp_autotune.argtypes = [vp, i, C.POINTER(Problem), C.c_char_p]
        for name in EXPORTS:
            if name not in ("pexp_default_options", "pexp_status_string"):
                getattr(L, name).restype = i
        _lib = L
    return _lib


class PexpError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lib().pexp_status_string(code).decode()} ({code})")


def status_string(code: int) -> str:
    return lib().pexp_status_string(code).decode()


def _check_vector_pair(X, Y, n: int) -> int:
    """Checks the (nvec, n) or (n,) CUDA tensors X (read) and Y (written) of a call that
    writes nvec * n elements at Y's base pointer; returns nvec."""
    for name, t in (("X", X), ("Y", Y)):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
        if t.dim() not in (1, 2) or t.shape[-1] != n:
            raise ValueError(f"{name} must have shape (nvec, {n}) or ({n},), got {tuple(t.shape)}")
    if X.dtype != Y.dtype or X.shape != Y.shape or X.device != Y.device:
        raise ValueError("X and Y must have the same dtype, shape and device")
    _dtype_code(X)
    return X.shape[0] if X.dim() == 2 else 1


def sai_solve_noalloc(op: dict, gamma: float, X, Y, stream=None) -> None:
    """Y = (I - gamma A)^{-1} X through pexp_sai_solve_noalloc: no context and no
    allocation; enqueued on `stream` (a torch.cuda.Stream; default: the current
    stream of X's device) and asynchronous -- synchronise before reading Y."""
    import torch
    nvec = _check_vector_pair(X, Y, int(op["nx"]) * (int(op.get("ny", 1)) if op["dim"] == 2 else 1))
    st = stream if stream is not None else torch.cuda.current_stream(X.device)
    with torch.cuda.device(X.device):
        rc = lib().pexp_sai_solve_noalloc(C.byref(make_operator(op)), float(gamma), C.c_void_p(X.data_ptr()),
                                          C.c_void_p(Y.data_ptr()), nvec, _dtype_code(X), C.c_void_p(st.cuda_stream))
    if rc != OK:
        raise PexpError(rc, "pexp_sai_solve_noalloc")


def make_operator(op: dict) -> Operator:
    return Operator(int(op["dim"]), int(op["nx"]), int(op.get("ny", 1)), int(op["bc"]), float(op["ax"]),
                    float(op.get("ay", 0.0)), float(op["nu"]), float(op.get("Lx", 1.0)), float(op.get("Ly", 1.0)))


def make_options(opts: dict) -> Options:
    o = Options()
    lib().pexp_default_options(C.byref(o))
    for name, _ in Options._fields_:
        if name in opts:
            setattr(o, name, type(getattr(o, name))(opts[name]))
    return o


def source_rows(opts: dict) -> int:
    """Rows of the source samples G of a linear solve: n_out (samples at the output times), or
    P (n_samp - 1) + 1 with Chebyshev samples (nodes = NODES_CHEBYSHEV)."""
    if int(opts.get("nodes", NODES_UNIFORM)) == NODES_CHEBYSHEV:
        return int(opts["P"]) * (int(opts["n_samp"]) - 1) + 1
    return int(opts["n_out"])


def _check_series_shapes(op: dict, opts: dict, y0, G, Y) -> None:
    """A valid solve reads n values of y0 and source_rows(opts) * n of G and writes n_out * n of
    Y: check that the arrays hold at least that before passing their pointers (invalid options
    are left to the library, which rejects them before touching any buffer)."""
    n = int(op["nx"]) * (int(op.get("ny", 1)) if op["dim"] == 2 else 1)
    if tuple(y0.shape) != (n,):
        raise ValueError(f"y0 must have shape ({n},), got {tuple(y0.shape)}")
    for name, a, rows in (("Y", Y, int(opts["n_out"])), ("G", G, source_rows(opts))):
        if a is None:
            continue
        count = a.numel() if hasattr(a, "numel") else a.size
        if a.shape[-1] != n or count < max(rows, 0) * n:
            raise ValueError(f"{name} must hold ({rows}, {n}) values, got shape {tuple(a.shape)}")


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _np_dtype_code(a) -> int:
    import numpy as np
    if a.dtype == np.float64:
        return F64
    if a.dtype == np.float32:
        return F32
    raise TypeError(f"unsupported dtype {a.dtype}")


class Context:
    """A library context on one CUDA device, bound to a CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        h = C.c_void_p()
        rc = lib().pexp_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PexpError(rc, "pexp_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().pexp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._stream = stream
        rc = lib().pexp_set_stream(self.h, C.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PexpError(rc, "pexp_set_stream")

    # ---------------------------------------------------------------- solvers
    def solve_linear(self, op: dict, opts: dict, y0, G, Y, check: bool = True) -> dict:
        """Paraexp-EBK solve: y0 (n,) FP64, G (source_rows(opts), n) or None, Y (n_out, n) --
        CUDA tensors."""
        import torch
        for t in (y0, Y) + ((G,) if G is not None else ()):
            assert t.is_cuda and t.is_contiguous()
        if y0.dtype != torch.float64:
            raise TypeError("the initial condition must be FP64")
        _check_series_shapes(op, opts, y0, G, Y)
        rep = Report()
        o = make_options(opts)
        rc = lib().pexp_solve_linear(self.h, C.byref(make_operator(op)), C.byref(o), C.c_void_p(y0.data_ptr()),
                                     C.c_void_p(G.data_ptr()) if G is not None else None,
                                     _dtype_code(G) if G is not None else _dtype_code(Y),
                                     C.c_void_p(Y.data_ptr()), _dtype_code(Y), C.byref(rep))
        if check and rc not in (OK, ERR_NOT_CONVERGED):
            raise PexpError(rc, "pexp_solve_linear")
        d = rep.as_dict()
        d["rc"] = rc
        return d

    def solve_linear_host(self, op: dict, opts: dict, y0, G, Y, check: bool = True) -> dict:
        """Same solve with host numpy buffers (copied in and out by the library)."""
        import numpy as np
        for a in (y0, Y) + ((G,) if G is not None else ()):
            assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
        if y0.dtype != np.float64:
            raise TypeError("the initial condition must be FP64")
        _check_series_shapes(op, opts, y0, G, Y)
        rep = Report()
        rc = lib().pexp_solve_linear_host(self.h, C.byref(make_operator(op)), C.byref(make_options(opts)),
                                          C.c_void_p(y0.ctypes.data),
                                          C.c_void_p(G.ctypes.data) if G is not None else None,
                                          _np_dtype_code(G) if G is not None else _np_dtype_code(Y),
                                          C.c_void_p(Y.ctypes.data), _np_dtype_code(Y), C.byref(rep))
        if check and rc not in (OK, ERR_NOT_CONVERGED):
            raise PexpError(rc, "pexp_solve_linear_host")
        d = rep.as_dict()
        d["rc"] = rc
        return d

    def solve_burgers(self, op: dict, opts: dict, u0, U, forcing=None, init=None, check: bool = True) -> dict:
        """Burgers waveform relaxation: u0 (n,) FP64; U, forcing, init (n_out, n) in one dtype."""
        import torch
        if u0.dtype != torch.float64:
            raise TypeError("the initial condition must be FP64")
        rep = Report()
        rc = lib().pexp_solve_burgers(self.h, C.byref(make_operator(op)), C.byref(make_options(opts)),
                                      C.c_void_p(u0.data_ptr()),
                                      C.c_void_p(forcing.data_ptr()) if forcing is not None else None,
                                      C.c_void_p(init.data_ptr()) if init is not None else None,
                                      C.c_void_p(U.data_ptr()), _dtype_code(U), C.byref(rep))
        if check and rc not in (OK, ERR_NOT_CONVERGED, ERR_WR_NOT_CONVERGED, ERR_WR_DIVERGED):
            raise PexpError(rc, "pexp_solve_burgers")
        d = rep.as_dict()
        d["rc"] = rc
        return d

    @staticmethod
    def _problems(items) -> "C.Array":
        """items: (op, opts, y0, G or None, Y) with CUDA tensors, as for solve_linear."""
        import torch
        arr = (Problem * len(items))()
        for k, (op, opts, y0, G, Y) in enumerate(items):
            for t in (y0, Y) + ((G,) if G is not None else ()):
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError("batched problems take contiguous CUDA tensors")
            if y0.dtype != torch.float64:
                raise TypeError("the initial condition must be FP64")
            arr[k].op = make_operator(op)
            arr[k].opts = make_options(opts)
            arr[k].y0_dev = y0.data_ptr()
            arr[k].G_dev = G.data_ptr() if G is not None else None
            arr[k].g_dtype = _dtype_code(G) if G is not None else _dtype_code(Y)
            arr[k].Y_dev = Y.data_ptr()
            arr[k].y_dtype = _dtype_code(Y)
        return arr

    def solve_batched(self, items, check: bool = True) -> list:
        """Solves independent problems concurrently (pexp_solve_batched); returns their reports."""
        arr = self._problems(items)
        reps = (Report * len(items))()
        rc = lib().pexp_solve_batched(self.h, len(items), arr, reps)
        if check and rc not in (OK, ERR_NOT_CONVERGED):
            raise PexpError(rc, "pexp_solve_batched")
        out = []
        for r in reps:
            d = r.as_dict()
            d["rc"] = r.status
            out.append(d)
        return out

    def selftest_barrier(self, absent_cta: int = -1) -> int:
        """pexp_selftest_barrier: a small cooperative launch through the bounded grid barrier;
        with absent_cta >= 0 one CTA never arrives and the wait must expire (ERR_TIMEOUT).
        Returns the status code."""
        return lib().pexp_selftest_barrier(self.h, int(absent_cta))

    def autotune(self, items, path: str | None = None) -> None:
        """Tunes the batched solve on these problems (pexp_autotune); the table goes to `path`."""
        arr = self._problems(items)
        rc = lib().pexp_autotune(self.h, len(items), arr, path.encode() if path else None)
        if rc != OK:
            raise PexpError(rc, "pexp_autotune")

    # ---------------------------------------------------------------- kernel-level calls
    def apply_operator(self, op: dict, X, Y, transpose: bool = False):
        nvec = _check_vector_pair(X, Y, int(op["nx"]) * (int(op.get("ny", 1)) if op["dim"] == 2 else 1))
        rc = lib().pexp_apply_operator(self.h, C.byref(make_operator(op)), C.c_void_p(X.data_ptr()),
                                       C.c_void_p(Y.data_ptr()), nvec, _dtype_code(X), int(transpose))
        if rc != OK:
            raise PexpError(rc, "pexp_apply_operator")

    def sai_solve(self, op: dict, gamma: float, X, Y):
        nvec = _check_vector_pair(X, Y, int(op["nx"]) * (int(op.get("ny", 1)) if op["dim"] == 2 else 1))
        rc = lib().pexp_sai_solve(self.h, C.byref(make_operator(op)), float(gamma), C.c_void_p(X.data_ptr()),
                                  C.c_void_p(Y.data_ptr()), nvec, _dtype_code(X))
        if rc != OK:
            raise PexpError(rc, "pexp_sai_solve")

    def jacobian_sai_solve(self, op: dict, gamma: float, ubar, X, Y):
        """Y = (I - gamma (A + J(ubar)))^{-1} X; ubar: (n,) FP64 CUDA tensor or None (J = 0)."""
        import torch
        nvec = _check_vector_pair(X, Y, int(op["nx"]))
        if ubar is not None and (not ubar.is_cuda or ubar.dtype != torch.float64 or ubar.shape != (int(op["nx"]),)):
            raise ValueError("ubar must be an FP64 CUDA tensor of shape (n,)")
        rc = lib().pexp_jacobian_sai_solve(self.h, C.byref(make_operator(op)), float(gamma),
                                           C.c_void_p(ubar.data_ptr()) if ubar is not None else None,
                                           C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()), nvec, _dtype_code(X))
        if rc != OK:
            raise PexpError(rc, "pexp_jacobian_sai_solve")

    def small_expm(self, M, E):
        import torch
        for t in (M, E):
            if not t.is_cuda or not t.is_contiguous() or t.dtype != torch.float64 or t.dim() != 3:
                raise ValueError("M and E must be contiguous CUDA FP64 tensors of shape (batch, N, N)")
        if M.shape != E.shape or M.shape[1] != M.shape[2]:
            raise ValueError("M and E must have the same shape (batch, N, N)")
        batch, N, _ = M.shape
        rc = lib().pexp_small_expm(self.h, C.c_void_p(M.data_ptr()), C.c_void_p(E.data_ptr()), N, batch)
        if rc != OK:
            raise PexpError(rc, "pexp_small_expm")

    def burgers_source(self, op: dict, U, G, form: int = 0):
        rows = _check_vector_pair(U, G, int(op["nx"]))
        rc = lib().pexp_burgers_source(self.h, C.byref(make_operator(op)), C.c_void_p(U.data_ptr()),
                                       C.c_void_p(G.data_ptr()), rows, _dtype_code(U), form)
        if rc != OK:
            raise PexpError(rc, "pexp_burgers_source")
