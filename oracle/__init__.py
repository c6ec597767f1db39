"""Plain FP64 CPU oracle for polynomial preconditioned Arnoldi (Embree, Loe & Morgan).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path;
the only common module is the seeded input generator
(``paper_1806_08020_gb300.inputs``), which holds no arithmetic of the method.

Every function cites the passage of the paper it follows.  Pins (tests that tie
the oracle to facts other than itself) live in ``tests/test_oracle_*.py``.
Functions with no such pin say "parity unpinned" in their docstring.
"""
from .ppa import (  # noqa: F401
    Counters,
    Operator,
    Poly,
    add_stability_roots,
    apply_poly,
    balance,
    build_double_poly,
    build_poly,
    build_poly_two,
    cgs2,
    damped_poly,
    eigs,
    harmonic_restart_matrix,
    thick_restart,
    first_cycle_rayleigh,
    gershgorin_shift,
    gmres_arnoldi,
    harmonic_ritz,
    ideal_order,
    modified_leja,
    norm1,
    pof_log10,
    poly_eval,
    to_scipy,
)
