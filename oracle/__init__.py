"""Plain FP64 CPU oracle of the Paraexp exponential block Krylov (PEBK) method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA path; both draw their inputs from ``paper_1509_04567_gb300.workloads``,
which holds no arithmetic of the method.

Every function cites the passage of the paper (Kooij, Botchev, Geurts,
arXiv:1509.04567) it follows.  Library primitives (sparse LU, Householder QR,
SVD, cubic spline, dense expm) serve as single steps; nothing is blocked,
fused or reordered beyond what the paper states.
"""
from .pebk import (operator_matrix, apply_A, partition, sample_partition, compress_source, spline_segments,
                   KrylovOperator, block_krylov_step, projected_source_window,
                   projected_homogeneous, ebk_nonhomogeneous, ebk_homogeneous,
                   solve_linear, burgers_source, solve_burgers)

__all__ = ["operator_matrix", "apply_A", "partition", "sample_partition", "compress_source", "spline_segments",
           "KrylovOperator", "block_krylov_step", "projected_source_window",
           "projected_homogeneous", "ebk_nonhomogeneous", "ebk_homogeneous", "solve_linear",
           "burgers_source", "solve_burgers"]
