"""FP64 CPU oracle of MMGKS-OF (arXiv 2501.12497), written from the paper.

TEST INFRASTRUCTURE ONLY. This package is the independent reference that the
CUDA path is checked against. Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import it; the product package never does,
and the two share no code, header, table or constant generator.

Modules:
  ops     -- ctypes/numpy binding of ops.c: H, H^T, Psi, Psi^T, M(s), Mhat,
             Mhat^T, App. C derivative fields, Upsilon, Upsilon^T, L (+) L,
             reverse flow. All FP64.
  solver  -- GKB, the projected problem with DP/GCV, Solve-OF (Alg. 2) and
             MMGKS-OF (Alg. 1), in numpy FP64.

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, library routines (scipy.ndimage, numpy.linalg dense solves),
brute force and invariants; see the module docstrings for the pins.
"""
