"""CPU FP64 oracle for reorthogonalized block classical Gram-Schmidt.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are its only users.  It shares no code with the CUDA path.

Parity status: every function here is pinned by tests/test_oracle_pins.py
against values fixed by the mathematics (closed forms, LAPACK, a 60-digit
reference, special cases, invariants); no function is "parity unpinned".
"""
from .bcgs import (Breakdown, householder_qr, tsqr, chol, solve_right_upper,  # noqa: F401
                   solve_left_upper_t, delayed_projection, gram, project_normalize,
                   bcgsi_plus, bcgsi_plus_p_1s, bcgsi_plus_p_2s, bcgs_pipi_plus, bcgsi_plus_1s,
                   eager_step, factor,
                   VARIANTS, EAGER_FAMILY)
from .metrics import loo, loo_from_gram, residual, kappa  # noqa: F401
