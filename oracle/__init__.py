"""FP64 CPU oracle for Katz queries and LRC-Katz (test infrastructure only).

This package is the independent reference that the CUDA path is checked
against.  It is plain NumPy/SciPy in float64, written from the paper's
definitions (Section 3.1, Eqs. 1-3; Lemma 1, Eqs. 4-6; Eqs. 7-14;
Theorem 1; Algorithms 1-2) and shares no code with the CUDA library.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark
may import it.  The product path never calls it.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, the series definition, dense linear algebra on tiny
graphs or invariants (see ``tests/test_oracle_*.py``), except where a
function's docstring says "parity unpinned".
"""
from .katz_oracle import *  # noqa: F401,F403
