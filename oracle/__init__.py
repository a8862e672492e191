"""CPU oracle for the sparse-state gate-application path (test infrastructure).

This package is TEST INFRASTRUCTURE. Only the tests, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it; the
product library never does. It shares no code with the CUDA path.

``liboracle.so`` is built from ``sps_oracle.cpp`` by :func:`build` with plain
g++ and ``-ffp-contract=off``; see that file's header for what each function
computes and which passage of arXiv 2105.01533 it follows.
"""

from .oracle import (  # noqa: F401
    build,
    OracleState,
    dense_run,
    classical_eval,
    sector_run,
    lib_path,
)
