"""Pins of the oracle's balancing (a diagonal similarity S = D^-1 A D that makes A
symmetric; not in the paper, an opt-in transformation of the library).

* Closed form: the 5-point convection-diffusion operator with cell Peclet
  number beta h / 2 < 1 has x-neighbour entries -1/h^2 -+ beta/(2h) of one
  sign, so d_{i+1}/d_i = sqrt(a_{i+1,i}/a_{i,i+1}) = rho with
  rho = sqrt((1 + beta h/2)/(1 - beta h/2)) along x and 1 along y:
  log d = (x index) log rho up to a constant.
* S is symmetric and similar to A (same eigenvalues, dense, small n).
* Matrices without such a D are refused: opposite signs (cell Peclet > 1, a
  complex spectrum) and a 3-cycle whose ratios do not multiply to 1.
* Balanced thick-restarted Arnoldi reaches the closed-form eigenvalues to
  1e-8 with every residual on A itself <= 1e-8 ||A||_1, also where A's
  eigenvalue condition numbers (~e^(beta/2)) leave the unbalanced solve on
  pseudo-eigenvalues.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import oracle.ppa as ppa
from oracle.ppa import make_operator
from paper_1806_08020_gb300 import inputs


def _closed_form_2d(N, beta, count):
    h = 1.0 / (N + 1)
    c = np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    lx = (2 - 2 * np.sqrt(1 - (beta * h / 2) ** 2) * c) / h**2
    ly = (2 - 2 * c) / h**2
    return np.sort((lx[:, None] + ly[None, :]).ravel())[:count]


@pytest.mark.parametrize("N,beta", [(10, 15.0), (50, 20.0), (40, 70.0)])
def test_balance_closed_form_scaling(N, beta):
    A = O.to_scipy(inputs.convection_diffusion_2d(N, beta))
    d, S = O.balance(A)
    h = 1.0 / (N + 1)
    rho = np.sqrt((1 + beta * h / 2) / (1 - beta * h / 2))
    ix = np.arange(N * N) % N
    assert np.allclose(np.log(d), (ix - (N - 1)) * np.log(rho), rtol=0, atol=1e-11 * N)
    assert d.max() == 1.0
    assert abs(S - S.T).max() <= 1e-13 * abs(S).max()


def test_balance_similar_and_symmetric_dense():
    A = O.to_scipy(inputs.convection_diffusion_2d(12, 18.0))
    d, S = O.balance(A)
    Sd = S.toarray()
    assert np.allclose(Sd, Sd.T, rtol=0, atol=1e-13 * np.abs(Sd).max())
    # S = D^-1 A D entry by entry
    Ad = A.toarray()
    assert np.allclose(Sd, Ad * d[None, :] / d[:, None], rtol=1e-13, atol=0)
    lam_a = np.sort(np.linalg.eigvals(Ad).real)
    lam_s = np.linalg.eigvalsh(Sd)
    assert np.allclose(lam_a, lam_s, rtol=1e-10)


def test_balance_refuses_opposite_signs():
    A = O.to_scipy(inputs.convection_diffusion_2d(10, 30.0))  # beta h / 2 = 1.36: complex spectrum
    with pytest.raises(ValueError):
        O.balance(A)


def test_balance_refuses_inconsistent_cycle():
    # ratios around 0 -> 1 -> 2 -> 0: sqrt(1/1) sqrt(1/1) sqrt(1/2) != 1
    A = sp.csr_matrix(np.array([[2.0, 1.0, 2.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]))
    with pytest.raises(ValueError):
        O.balance(A)
    # a path (no cycle) is always balanced: d = (1, sqrt(2), sqrt(2)) up to scale
    P = sp.csr_matrix(np.array([[2.0, 1.0, 0.0], [2.0, 2.0, 3.0], [0.0, 3.0, 2.0]]))
    d, S = O.balance(P)
    assert np.allclose(d / d[0], [1.0, np.sqrt(2.0), np.sqrt(2.0)])
    assert np.allclose(S.toarray(), S.toarray().T)


def _balanced_eigs(N, beta, d, nev, m, k, seed=20181806):
    A = O.to_scipy(inputs.convection_diffusion_2d(N, beta))
    dd, S = O.balance(A)
    c = O.Counters()
    op = O.Operator(S, O.gershgorin_shift(S), c)
    n = A.shape[0]
    P = O.build_poly(op, inputs.start_vector(n, seed, 0), d, c)
    R = O.eigs(A, make_operator(op, P, c), nev, m, k, 1e-8, inputs.start_vector(n, seed, 1), c, target="SR",
               scale=dd)
    return A, R


def test_balanced_eigs_plain_small_closed_form():
    """The n = 2,500 workload (N = 50, beta = 20, d = 10, Arnoldi(30, 15), nev = 10) balanced:
    the closed-form eigenvalues to 1e-8 and residuals on A <= 1e-8 ||A||_1."""
    A, R = _balanced_eigs(50, 20.0, 10, 10, 30, 15)
    assert R.converged
    assert np.allclose(np.sort(R.lam.real), _closed_form_2d(50, 20.0, 10), rtol=1e-8, atol=0)
    assert np.max(np.abs(R.lam.imag)) == 0.0
    nA = O.norm1(A)
    for lam, x in zip(R.lam, R.X.T):
        assert abs(np.linalg.norm(x) - 1) < 1e-12
        assert np.linalg.norm(A @ x - lam.real * x) / nA <= 1e-8


def test_balanced_eigs_reach_true_eigenvalues_where_unbalanced_cannot():
    """N = 60, beta = 110 (h = 1/61, beta h / 2 = 0.90): the smallest eigenvalue's
    condition number is ~1e34, so dense FP64 eig and the unbalanced solve land
    on pseudo-eigenvalues; balanced, the closed form to 1e-8."""
    N, beta = 60, 110.0
    A, R = _balanced_eigs(N, beta, 10, 6, 30, 11)
    want = _closed_form_2d(N, beta, 6)
    assert R.converged
    assert np.allclose(np.sort(R.lam.real), want, rtol=1e-8, atol=0)
    # the unbalanced solve of the same operator: residuals meet rtol, values do not
    c = O.Counters()
    op = O.Operator(A, O.gershgorin_shift(A), c)
    P = O.build_poly(op, inputs.start_vector(A.shape[0], 20181806, 0), 10, c)
    U = O.eigs(A, make_operator(op, P, c), 6, 30, 11, 1e-8, inputs.start_vector(A.shape[0], 20181806, 1), c,
               target="SR")
    assert U.converged
    assert np.max(np.abs(np.sort(U.lam.real) - want) / want) > 1e-3


# ---- planted mistakes ----

def _balance_full_log(A, max_log_range=600.0):  # forgets the square root
    A = sp.csr_matrix(A)
    n = A.shape[0]
    logd = np.zeros(n)
    for i in range(n - 1):
        if A[i, i + 1] != 0:
            logd[i + 1] = logd[i] + (np.log(abs(A[i + 1, i])) - np.log(abs(A[i, i + 1])))
        else:
            logd[i + 1] = logd[i]
    d = np.exp(logd - logd.max())
    coo = A.tocoo()
    S = sp.csr_matrix((coo.data * d[coo.col] / d[coo.row], (coo.row, coo.col)), shape=A.shape)
    return d, S


def _balance_inverted(A, max_log_range=600.0):  # d_j/d_i = sqrt(a_ij/a_ji)
    d, S = ppa.balance(A, max_log_range)
    d2 = 1.0 / d
    coo = sp.csr_matrix(A).tocoo()
    S2 = sp.csr_matrix((coo.data * d2[coo.col] / d2[coo.row], (coo.row, coo.col)), shape=A.shape)
    return d2 / d2.max(), S2


@pytest.mark.parametrize("mutant", [_balance_full_log, _balance_inverted])
def test_balance_mutants_caught(mutant, monkeypatch):
    monkeypatch.setattr(O, "balance", mutant)
    failures = 0
    for t in (lambda: test_balance_closed_form_scaling(10, 15.0), test_balance_similar_and_symmetric_dense):
        try:
            t()
        except AssertionError:
            failures += 1
    assert failures == 2
