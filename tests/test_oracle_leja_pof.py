"""Pins of the oracle's modified Leja order, pof and added roots.

* Leja: the defining greedy property checked by brute force with explicit
  products (not logarithms) over every remaining candidate (Section 2 box,
  step 1(c); Bai, Hu & Reichel alg. 3.1), conjugate pairs adjacent.
* pof: the paper's identity |pi'(theta_j)| = pof(j)/|theta_j| (Section 7),
  checked against the derivative of the power-form polynomial.
* Added-root counts at the thresholds printed in Section 7 (double above 1e4,
  triple above 1e18, quadruple above 1e32) and the placement reading.
* Example 7: the largest root near 20000 and MaxPof orders (Section 7).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle.ppa import extra_copies
from paper_1806_08020_gb300 import inputs
from conftest import golden_dict


def _random_roots(rng, nreal, npair):
    re = list(rng.uniform(-3, 5, nreal))
    pr = []
    for _ in range(npair):
        z = complex(rng.uniform(-3, 5), rng.uniform(0.1, 2))
        pr += [z, np.conj(z)]
    r = np.array(re + pr, dtype=complex)
    return r[rng.permutation(r.size)]


@pytest.mark.parametrize("seed", range(12))
def test_leja_greedy_property_brute_force(seed):
    rng = np.random.default_rng(seed)
    roots = _random_roots(rng, int(rng.integers(1, 5)), int(rng.integers(0, 3)))
    out = O.modified_leja(roots)
    # a permutation of the input
    assert sorted(map(lambda z: (z.real, z.imag), out)) == sorted(map(lambda z: (z.real, z.imag), roots))
    # pairs adjacent, Im > 0 first
    i = 0
    units = []
    while i < out.size:
        units.append(out[i])
        if out[i].imag != 0:
            assert out[i].imag > 0 and out[i + 1] == np.conj(out[i])
            i += 2
        else:
            i += 1
    # first unit: largest modulus
    assert abs(units[0]) == max(abs(z) for z in out)
    # each later unit maximises the product of distances to all chosen points
    for k in range(1, len(units)):
        chosen = []
        for z in units[:k]:
            chosen += [z] if z.imag == 0 else [z, np.conj(z)]
        def prod(z):
            return np.prod([abs(z - w) for w in chosen])
        best = max(prod(z) for z in units[k:])
        assert prod(units[k]) >= best * (1 - 1e-12)


def test_leja_tie_break_is_deterministic():
    out = O.modified_leja(np.array([1.0, -1.0, 2.0, -2.0]))
    assert list(out.real) == [2.0, -2.0, 1.0, -1.0]


def test_leja_exhaustive_small_sets_unique_maximiser():
    """For 5 distinct generic reals, greedy Leja equals the brute-force greedy path."""
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1, 4, 5)
    out = O.modified_leja(pts.astype(complex)).real
    for perm in itertools.permutations(range(5)):
        seq = pts[list(perm)]
        ok = abs(seq[0]) == np.max(np.abs(pts))
        for k in range(1, 5):
            prods = [np.prod(np.abs(z - seq[:k])) for z in seq[k:]]
            ok &= np.prod(np.abs(seq[k] - seq[:k])) == max(prods)
        if ok:
            assert np.array_equal(seq, out)


@pytest.mark.parametrize("seed", range(5))
def test_pof_is_scaled_derivative(seed):
    """Section 7: |pi'(theta_j)| = pof(j) / |theta_j|."""
    rng = np.random.default_rng(seed)
    roots = O.modified_leja(_random_roots(rng, 3, 2) + 6.0)
    coef = np.poly(roots) * ((-1) ** roots.size) / np.prod(roots)  # highest degree first
    dcoef = np.polyder(coef)
    lp = O.pof_log10(roots)
    for j, th in enumerate(roots):
        deriv = abs(np.polyval(dcoef, th))
        assert abs(np.log10(deriv * abs(th)) - lp[j]) < 1e-9


def test_extra_copy_thresholds():
    """Section 7: double root above 1e4, triple above 1e18, quadruple above 1e32."""
    assert extra_copies(3.0) == 0
    assert extra_copies(4.0) == 0
    assert extra_copies(4.001) == 1
    assert extra_copies(17.9) == 1
    assert extra_copies(18.2) == 2
    assert extra_copies(32.5) == 3
    assert extra_copies(-5.0) == 0


def test_added_root_placement():
    """First copy at the end, the others spaced evenly from the root to the end."""
    roots = O.modified_leja(np.array([20000.0, 1, 2, 3, 4, 5, 6, 7, 8, 9], dtype=complex))
    assert roots[0] == 20000.0
    lp = O.pof_log10(roots)
    c = extra_copies(lp[0])
    assert c == 3 and all(extra_copies(v) == 0 for v in lp[1:])
    out, added = O.add_stability_roots(roots)
    assert added == 3 and out.size == 13
    pos = [i for i, z in enumerate(out) if z == 20000.0]
    # L = 10 units, root at p = 0, c = 3: copies after positions 3 and 6, then the end
    assert pos == [0, 4, 8, 12]


def test_added_roots_keep_pairs_together():
    z = 30000.0 + 5000.0j
    roots = O.modified_leja(np.array([z, np.conj(z), 1, 2, 3, 4, 5, 6], dtype=complex))
    out, added = O.add_stability_roots(roots)
    assert added % 2 == 0 and added > 0
    for i, v in enumerate(out):
        if v.imag > 0:
            assert out[i + 1] == np.conj(v)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_example7_roots_and_pof(seed):
    """Example 7: theta near 20000 at d = 15; MaxPof ~ 1e17 at d = 25, ~2e28 at d = 40."""
    g = golden_dict("example7.txt")
    A = O.to_scipy(inputs.diagonal(inputs.example7_diag()))
    b = inputs.start_vector(10000, seed, 0)
    P15 = O.build_poly(O.Operator(A, 0.0, O.Counters()), b, 15, O.Counters(), add_roots=False)
    assert abs(P15.roots.real.max() - g["theta_max_d15"]) / 2e4 < 1e-12
    P40 = O.build_poly(O.Operator(A, 0.0, O.Counters()), b, 40, O.Counters(), add_roots=False)
    lp40 = O.pof_log10(P40.roots).max()
    assert abs(lp40 - np.log10(g["maxpof_d40"])) < 1.0
    assert extra_copies(lp40) == 2  # "another extra root is needed" at d = 40
    P25 = O.build_poly(O.Operator(A, 0.0, O.Counters()), b, 25, O.Counters(), add_roots=False)
    lp25 = O.pof_log10(P25.roots).max()
    assert 15.5 < lp25 < 18.0 and extra_copies(lp25) == 1
