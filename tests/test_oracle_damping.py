"""Pins for the damping heuristic of the oracle (Section 6.3 box).

* The Rayleigh quotients the paper prints for Example 6 fail the Ideal Order
  Condition; the ideal sequence 1..k passes.
* Example 6 (diag(1..10000), Arnoldi(50,20), nev = 15) on seeded start
  vectors: at d = 50 the first test fails and the damped polynomial (GMRES from
  A b) passes, as the paper reports; at d = 80 damping alone still fails and the
  heuristic halves d to 40 (the paper: at d = 80 "even the damped polynomial
  runs into trouble").
* Closed forms: the damped cycle's Rayleigh quotients are the eigenvalues
  1..15 of the diagonal matrix, and the eigensolve with the damped polynomial
  returns exactly {1, ..., 15}, while the undamped one misses some.
"""
import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from paper_1806_08020_gb300 import inputs


def _golden():
    rows = {r[0]: r[1:] for r in read_golden("example6_ideal_order.txt")}
    return int(rows["nev"][0]), int(rows["k"][0]), np.array([float(x) for x in rows["mu"]])


def test_paper_sequence_fails_ideal_order():
    nev, k, mu = _golden()
    assert not O.ideal_order(mu, nev, k)
    assert O.ideal_order(np.arange(1.0, k + 1), nev, k)


def test_ideal_order_boundaries():
    # equal magnitudes are allowed among the first nev, not across the nev boundary
    assert O.ideal_order(np.array([1, 2, 2, 3, 5]), 3, 5)
    assert not O.ideal_order(np.array([1, 2, 3, 3, 5]), 3, 5)
    assert not O.ideal_order(np.array([2, 1, 3, 4, 5]), 3, 5)
    # magnitudes, not values: a conjugate pair counts by its modulus
    assert O.ideal_order(np.array([1, 2 + 1j, 2 - 1j, 4, 5]), 3, 5)
    assert not O.ideal_order(np.array([1, 1 + 3j, 2, 4, 5]), 3, 5)


@pytest.fixture(scope="module")
def ex6():
    return O.to_scipy(inputs.diagonal(inputs.example6_diag()))


@pytest.mark.parametrize("seed", [2, 5])
def test_example6_d50_damping(ex6, seed):
    b = inputs.start_vector(ex6.shape[0], seed, 0)
    R = O.damped_poly(ex6, 0.0, b, 50, 50, 20, 15, O.Counters())
    assert R.trials == [(50, False, False), (50, True, True)]
    mu = O.first_cycle_rayleigh(ex6, O.ppa.make_operator(O.Operator(ex6, 0.0, O.Counters()), R.poly, O.Counters()),
                                b, 50, 20, O.Counters())
    assert np.abs(mu[:15] - np.arange(1.0, 16.0)).max() < 1e-8


def test_example6_d80_halves_degree(ex6):
    b = inputs.start_vector(ex6.shape[0], 2, 0)
    R = O.damped_poly(ex6, 0.0, b, 80, 50, 20, 15, O.Counters())
    assert R.trials == [(80, False, False), (80, True, False), (40, True, True)]
    assert R.degree == 40 and R.damped and R.ideal


@pytest.mark.slow
def test_example6_eigensolve_with_and_without_damping(ex6):
    n = ex6.shape[0]
    b = inputs.start_vector(n, 2, 0)
    v0 = inputs.start_vector(n, 2, 1)
    op = O.Operator(ex6, 0.0, O.Counters())
    want = np.arange(1.0, 16.0)
    R = O.damped_poly(ex6, 0.0, b, 50, 50, 20, 15, O.Counters())
    E = O.eigs(ex6, O.ppa.make_operator(op, R.poly, O.Counters()), 15, 50, 20, 1e-8, v0, O.Counters(),
               target="SM", max_cycles=20)
    assert E.converged
    assert np.abs(np.sort(E.lam.real) - want).max() < 1e-6
    P0 = O.build_poly(op, b, 50, O.Counters())
    E0 = O.eigs(ex6, O.ppa.make_operator(op, P0, O.Counters()), 15, 50, 20, 1e-8, v0, O.Counters(),
                target="SM", max_cycles=20)
    got = np.sort(E0.lam.real)
    assert np.abs(got - want).max() > 0.5  # some desired eigenvalue is missing (overenthusiastic)
