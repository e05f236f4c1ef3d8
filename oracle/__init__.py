"""CPU oracle for the RaNN domain-decomposition solver (float64, numpy).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg may import or run anything in this package; the
product path (paper_2412_19207_gb300) never does, and the two share no code.
Inputs come from rann_inputs (seeded problem data, no method arithmetic).

Modules: hyperdual (exact derivatives), assembly (geometry, windows, the
constraining operator, collocation blocks), linalg (Householder QR, PCG,
GMRES), solver (PCA, Schwarz preconditioners, solves, evaluation).
"""
from . import hyperdual, assembly, linalg, solver  # noqa: F401
