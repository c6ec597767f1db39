"""Pins of the oracle's two scalar reductions of A, and planted mistakes that they catch.

* ``norm1`` is the norm of the convergence test (Section 4 asks for a residual
  below 1e-8 ||A|| without naming the norm; the 1-norm is the reading taken).
* ``gershgorin_shift`` is the shift of the "smallest real part" target
  (Section 2, first footnote: run the method on A - sigma I).

The pins are values fixed outside the oracle: a 3 x 3 matrix worked by hand,
and the closed forms of the central-difference convection-diffusion operators
of Example 1 (5-point in 2-D, 7-point in 3-D).  With h = 1/(N+1) the interior
row of the 2-D operator is 4/h^2 on the diagonal, -1/h^2 twice (y), and
-1/h^2 -+ beta/(2h) (x).  When the cell Peclet number beta h / 2 is at most 1
the two x entries have the same sign and their magnitudes add to 2/h^2, so
every interior column sums to 8/h^2 (12/h^2 in 3-D) and every Gershgorin disc
has its left end at 0 or above; above 1 they add to beta/h and the leftmost
disc ends at 2/h^2 - beta/h (2-D interior row).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import oracle.ppa as ppa
from paper_1806_08020_gb300 import inputs

# Hand-worked 3 x 3 example (row and column sums differ, entries of both signs):
#   A = [[ 1, -7,  0],
#        [ 2,  3,  0],
#        [ 0,  1, -4]]
# absolute column sums 3, 11, 4        -> ||A||_1 = 11
# absolute row sums    8, 5, 5         -> ||A||_inf = 8 (a row-sum mistake gives 8)
# signed column sums   3, -3, -4       -> (a missing abs gives 3)
# Gershgorin rows: centre - off-diagonal radius = 1 - 7, 3 - 2, -4 - 1 = -6, 1, -5 -> sigma = -6
# (column radii give 1 - 2, 3 - 8, -4 - 0 -> -5; the diagonal inside the radius gives
#  1 - 8, 3 - 5, -4 - 5 -> -9; signed radii give 1 + 7, 3 - 2, -4 - 1 -> -5)
HAND = np.array([[1.0, -7.0, 0.0], [2.0, 3.0, 0.0], [0.0, 1.0, -4.0]])
HAND_NORM1 = 11.0
HAND_SIGMA = -6.0


def _hand():
    return sp.csr_matrix(HAND)


def test_norm1_hand_example():
    assert O.norm1(_hand()) == HAND_NORM1


def test_gershgorin_hand_example():
    assert O.gershgorin_shift(_hand()) == HAND_SIGMA


def test_gershgorin_positive_discs_give_zero():
    """A matrix whose discs all lie right of 0 is run unshifted (sigma = min(0, ...))."""
    A = sp.csr_matrix(np.array([[5.0, 1.0], [-2.0, 4.0]]))
    assert O.gershgorin_shift(A) == 0.0


@pytest.mark.parametrize("N,beta", [(50, 20.0), (1000, 100.0), (30, 58.0)])
def test_norm1_closed_form_2d(N, beta):
    """||A||_1 = 8/h^2 for the 5-point operator with beta h / 2 <= 1: 20,808 for the
    n = 2,500 workload (N = 50, h = 1/51), 8,016,008 for the n = 10^6 one."""
    h = 1.0 / (N + 1)
    assert beta * h / 2 <= 1
    A = O.to_scipy(inputs.convection_diffusion_2d(N, beta))
    assert O.norm1(A) == pytest.approx(8.0 / h**2, rel=1e-14)
    if N == 50:
        assert O.norm1(A) == pytest.approx(20808.0, rel=1e-14)


def test_norm1_closed_form_3d():
    """||A||_1 = 12/h^2 for the 7-point operator (N = 20, beta = 10, h = 1/21: 5,292)."""
    A = O.to_scipy(inputs.convection_diffusion_3d(20, 10.0))
    assert O.norm1(A) == pytest.approx(12.0 * 21.0**2, rel=1e-14)


@pytest.mark.parametrize("N,beta", [(50, 20.0), (1000, 100.0), (30, 58.0)])
def test_gershgorin_zero_for_cell_peclet_at_most_one(N, beta):
    """Interior discs touch 0 exactly (up to rounding, absorbed by the 1e-12 ||A||_1 rule)."""
    A = O.to_scipy(inputs.convection_diffusion_2d(N, beta))
    assert O.gershgorin_shift(A) == 0.0


def test_gershgorin_closed_form_above_cell_peclet_one():
    """N = 10, beta = 60 (h = 1/11, beta h / 2 = 2.7): sigma = 2/h^2 - beta/h = 242 - 660 = -418."""
    A = O.to_scipy(inputs.convection_diffusion_2d(10, 60.0))
    assert O.gershgorin_shift(A) == pytest.approx(-418.0, rel=1e-13)


def test_gershgorin_closed_form_3d_above_cell_peclet_one():
    """3-D: the interior row has 4 y/z entries of -1/h^2, so sigma = 6/h^2 - 4/h^2 - beta/h.
    N = 8, beta = 40 (h = 1/9, beta h / 2 = 2.2): 162 - 360 = -198."""
    A = O.to_scipy(inputs.convection_diffusion_3d(8, 40.0))
    assert O.gershgorin_shift(A) == pytest.approx(-198.0, rel=1e-13)


# ---- planted mistakes: each must fail at least one pin above ----

def _norm1_row_sums(A):
    return float(np.max(np.asarray(abs(A).sum(axis=1)).ravel()))


def _norm1_no_abs(A):
    return float(np.max(np.asarray(A.sum(axis=0)).ravel()))


def _gersh_column_radius(A):
    d = A.diagonal()
    off = np.asarray(abs(A).sum(axis=0)).ravel() - np.abs(d)
    lo = float(np.min(d - off))
    return 0.0 if lo >= -1e-12 * O.norm1(A) else min(0.0, lo)


def _gersh_diag_in_radius(A):
    d = A.diagonal()
    off = np.asarray(abs(A).sum(axis=1)).ravel()
    lo = float(np.min(d - off))
    return 0.0 if lo >= -1e-12 * O.norm1(A) else min(0.0, lo)


def _gersh_signed_radius(A):
    d = A.diagonal()
    off = np.asarray(A.sum(axis=1)).ravel() - d
    lo = float(np.min(d - off))
    return 0.0 if lo >= -1e-12 * O.norm1(A) else min(0.0, lo)


NORM_PINS = [test_norm1_hand_example, test_norm1_closed_form_3d,
             lambda: test_norm1_closed_form_2d(50, 20.0), lambda: test_norm1_closed_form_2d(30, 58.0)]
GERSH_PINS = [test_gershgorin_hand_example, test_gershgorin_positive_discs_give_zero,
              test_gershgorin_closed_form_above_cell_peclet_one, test_gershgorin_closed_form_3d_above_cell_peclet_one,
              lambda: test_gershgorin_zero_for_cell_peclet_at_most_one(50, 20.0)]


def _failures(pins):
    n = 0
    for t in pins:
        try:
            t()
        except AssertionError:
            n += 1
    return n


def test_unmutated_pins_pass():
    assert _failures(NORM_PINS) == 0 and _failures(GERSH_PINS) == 0


@pytest.mark.parametrize("mutant", [_norm1_row_sums, _norm1_no_abs])
def test_norm1_mutants_caught(mutant, monkeypatch):
    monkeypatch.setattr(ppa, "norm1", mutant)
    monkeypatch.setattr(O, "norm1", mutant)
    assert _failures(NORM_PINS) > 0


@pytest.mark.parametrize("mutant", [_gersh_column_radius, _gersh_diag_in_radius, _gersh_signed_radius])
def test_gershgorin_mutants_caught(mutant, monkeypatch):
    monkeypatch.setattr(ppa, "gershgorin_shift", mutant)
    monkeypatch.setattr(O, "gershgorin_shift", mutant)
    assert _failures(GERSH_PINS) > 0
