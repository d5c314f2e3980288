"""GB300-native Paraexp exponential block Krylov (PEBK) hot path.

The solver itself lives in the CUDA/C++ shared library built from ``csrc/``;
``pexp`` is the thin ctypes binding to its C ABI (``include/pexp.h``).
``workloads`` holds the seeded synthetic input generators shared by the tests,
the benchmark and the oracle.
"""
