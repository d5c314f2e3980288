"""Shared helpers of the GPU tests (CUDA path via the C ABI; references from oracle/)."""
import numpy as np
import pytest


def ctx():
    import __graft_entry__ as g
    g.build()
    from paper_1509_04567_gb300 import pexp
    return pexp.Context(0)


def relerr_rows(Y, Yref):
    """max_i ||Y_i - Yref_i|| / ||Yref_i|| over the output times i."""
    num = np.linalg.norm(Y - Yref, axis=1)
    den = np.linalg.norm(Yref, axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def run_linear(c, pr, opts=None, dtype="f64", G=True):
    import torch
    opts = dict(pr.opts if opts is None else opts)
    dt = torch.float64 if dtype == "f64" else torch.float32
    dev = torch.device("cuda:0")
    y0 = torch.from_numpy(pr.u0).to(dev)
    Gt = torch.from_numpy(pr.G).to(dev, dt) if (G and pr.G is not None) else None
    Y = torch.zeros((opts["n_out"], pr.n), dtype=dt, device=dev)
    rep = c.solve_linear(pr.op, opts, y0, Gt, Y)
    torch.cuda.synchronize()
    return Y.double().cpu().numpy(), rep
