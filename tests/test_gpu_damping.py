"""Damping heuristic (Section 6.3 box) on the GPU against the oracle.

Example 6, diag(1, ..., 10000), Arnoldi(50,20), nev = 15, seeded start
vectors: the device takes the oracle's decisions (damp at d = 50; damp and
halve to d = 40 at d = 80), its polynomial has the oracle's roots, and the
eigensolve with it returns exactly {1, ..., 15} (closed form).
"""
import numpy as np
import pytest

import oracle as O
from paper_1806_08020_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex6():
    Acsr = inputs.diagonal(inputs.example6_diag())
    return Acsr, O.to_scipy(Acsr)


@pytest.mark.parametrize("d,seed", [(50, 2), (50, 7), (80, 2)])
def test_damped_poly_matches_oracle(ex6, d, seed):
    from paper_1806_08020_gb300 import pp
    Acsr, A = ex6
    b = inputs.start_vector(Acsr.n, seed, 0)
    ref = O.damped_poly(A, 0.0, b, d, 50, 20, 15, O.Counters())
    ctx = pp.pp_create(Acsr, target=pp.PP_TARGET_SM)
    poly, info = pp.pp_build_poly_damped(ctx, d, b, 50, 20, 15)
    assert info == {"degree": ref.degree, "damped": ref.damped, "ideal": ref.ideal}
    got = pp.pp_poly_roots(poly)
    assert got.size == ref.poly.roots.size
    for z in ref.poly.roots:
        assert np.min(np.abs(got - z)) <= 1e-8 * abs(z)
    v0 = inputs.start_vector(Acsr.n, seed, 1)
    res = pp.pp_eigs(ctx, poly, 15, 50, 20, 1e-8, v0)
    assert res.status == 0
    assert np.abs(np.sort(res.lam.real)[:15] - np.arange(1.0, 16.0)).max() < 1e-6


def test_damping_arguments_checked(ex6):
    from paper_1806_08020_gb300 import pp
    Acsr, _ = ex6
    ctx = pp.pp_create(Acsr)
    b = inputs.start_vector(Acsr.n, 2, 0)
    for bad in [(0, 50, 20, 15), (50, 50, 15, 15), (50, 19, 20, 15), (50, 128, 20, 15)]:
        with pytest.raises(pp.PPError):
            pp.pp_build_poly_damped(ctx, bad[0], b, bad[1], bad[2], bad[3])


@pytest.mark.parametrize("precision", [0, 1])
def test_two_start_poly_matches_oracle(precision):
    """Polynomial from two starting vectors (Section 5 box) on the GPU: the
    oracle's roots, and on Example 4 with a skewed b1 the eigensolve returns
    exactly {1, ..., 15} (the single skewed vector misses 5..15)."""
    from paper_1806_08020_gb300 import pp
    Acsr = inputs.diagonal(inputs.example4_diag())
    A = O.to_scipy(Acsr)
    n = Acsr.n
    b1 = inputs.start_vector(n, 0, 0)
    b1[-100:] *= 0.01
    b2 = inputs.start_vector(n, 0, 2)
    ref = O.build_poly_two(O.Operator(A, 0.0, O.Counters()), b1, b2, 10, O.Counters())
    ctx = pp.pp_create(Acsr, target=pp.PP_TARGET_SM, precision=precision)
    poly = pp.pp_build_poly_two(ctx, 10, b1, b2)
    got = pp.pp_poly_roots(poly)
    assert got.size == ref.roots.size
    tol = 1e-8 if precision == 0 else 1e-4
    for z in ref.roots:
        assert np.min(np.abs(got - z)) <= tol * abs(z)
    res = pp.pp_eigs(ctx, poly, 15, 50, 20, 1e-8, inputs.start_vector(n, 0, 1))
    assert res.status == 0
    assert np.abs(np.sort(res.lam.real)[:15] - np.arange(1.0, 16.0)).max() < 1e-6
