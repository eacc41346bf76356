"""CPU oracle for the Legendre<->Chebyshev connection maps (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never does.
"""
from .oracle import (  # noqa: F401
    build_oracle, lambda_table, entry, entry_geg, geg_tables, apply, dense_matrix, threads, dct, synthesis, analysis,
    L2C, C2L,
)
