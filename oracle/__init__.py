"""CPU reference ("oracle") for the mixed-precision GMRES-IR method.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the benchmark's
CPU-baseline leg are the only importers.  The oracle shares no code with the
CUDA library (paper_2109_01232_b300) and never imports it; the library never
imports the oracle.  Both consume the seeded inputs from the `gen` package.

Parity pins (tests/test_oracle_*.py, run with -m "not gpu") tie every
function here to something other than itself: dense linear algebra, closed
forms, invariants of the Arnoldi relation and of GMRES optimality, library
conversions for the low-precision rounding, and the paper's printed matrix
sizes and iteration-count structure.
"""
from .gmres import (  # noqa: F401
    OK, NOT_CONVERGED, BREAKDOWN, NONFINITE, INVALID,
    Precision, Cycle, Info, vector_scale,
    spmv, dense, cgs2, givens, back_substitute, gmres_cycle, arnoldi,
    gmres, gmres_ir, gmres_fd,
)
from .lowprec import round_to, unit_roundoff  # noqa: F401
from .poly import (  # noqa: F401
    splitmix64_raw, splitmix64_uniform, harmonic_ritz, leja_order, poly_roots, poly_apply,
)
from . import selector  # noqa: F401
from . import precond  # noqa: F401
