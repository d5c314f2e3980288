"""Writes tests/golden/burgers_c3_n4096.json: the oracle's averaged-Jacobian waveform
relaxation (Sec. 2.3-2.4, eqs. ivp4 and piecewiseJac) on the viscous Burgers workload
(nu = 5e-3, u0 = 0.5 + sin(2 pi x), T = 0.5, P = 32, 513 samples) at n = 4096 points.

Stores the relative update of every iteration and the solution at t = 0.0625, 0.25 and
0.5 on every 8th mesh point.  Calls only oracle/ (and the input formulas); runs for
several minutes.  Run from the repository root:
    python tests/golden/make_burgers_c3_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle.pebk as ob  # noqa: E402
from paper_1509_04567_gb300 import workloads as wl  # noqa: E402

N, NU, T, P, NT = 4096, 5e-3, 0.5, 32, 513
ROWS, STRIDE = (64, 256, 512), 8
# svd_tol 1e-7: the floor of the GPU's Gram-based source SVD in FP64, so that both sides
# truncate the same singular values
OPTS = dict(T=T, P=P, n_out=NT, tol=1e-11, svd_tol=1e-7, max_rank=16, restart_len=40, wr_tol=1e-10,
            wr_max_iter=40, jacobian=1)


def main():
    op = wl.make_op(N, NU, 0.0)
    u0 = 0.5 + np.sin(2 * np.pi * wl.grid_1d(N))
    U, rep = ob.solve_burgers_jacobian(op, wl.default_opts(**OPTS), u0,
                                       callback=lambda k, Uk, d: print(k + 1, f"{d:.3e}", flush=True))
    out = {"source": "oracle.pebk.solve_burgers_jacobian", "n": N, "nu": NU, "opts": OPTS, "rows": list(ROWS),
           "stride": STRIDE, "iters": rep["iters"], "converged": rep["converged"], "deltas": rep["deltas"],
           "samples": {str(i): [float(v) for v in U[i, ::STRIDE]] for i in ROWS},
           "row_norms": {str(i): float(np.linalg.norm(U[i])) for i in ROWS}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "burgers_c3_n4096.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", path, rep["iters"], rep["converged"])


if __name__ == "__main__":
    main()
