"""Pins of the oracle's polynomial construction and application.

Each test ties the oracle to a fact fixed by the paper or by the mathematics,
not to a second copy of its own formula:

* GMRES optimality: pi(A)b from the factored roots equals the GMRES residual
  b - A V_d y_d with y_d the least-squares solution (Section 2: the GMRES
  polynomial is the minimum residual polynomial with pi(0) = 1).
* Harmonic Ritz values from a second formulation, the generalized eigenproblem
  (H_{d+1,d}^T H_{d+1,d}, H_d^T) (definition of harmonic Ritz values).
* Full degree d = n: the roots are the eigenvalues of A and pi(A) b = 0.
* Factored apply vs power form (monomial coefficients) and vs the scalar
  polynomial on a diagonal matrix, including conjugate pairs.
* Running sum r = A phi(A) x with pi(z) = 1 - z phi(z) (Section 2 footnote 2).
* Table 1 (Section 3): every row reproduced to the printed 4 digits.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from oracle.ppa import make_operator
from paper_1806_08020_gb300 import inputs
from conftest import read_golden


def _mat(kind):
    if kind == "cd":
        return O.to_scipy(inputs.convection_diffusion_2d(12, 20.0))
    if kind == "cd_complex":  # cell Peclet beta*h/2 > 1: complex spectrum
        return O.to_scipy(inputs.convection_diffusion_2d(10, 60.0))
    if kind == "band":
        return O.to_scipy(inputs.banded_random(200, 3, 5))
    if kind == "ex7":
        return O.to_scipy(inputs.diagonal(inputs.example7_diag()))
    raise KeyError(kind)


@pytest.mark.parametrize("kind", ["cd", "cd_complex", "band", "ex7"])
@pytest.mark.parametrize("d", [1, 4, 10, 16])
def test_factored_poly_is_gmres_residual(kind, d):
    A = _mat(kind)
    n = A.shape[0]
    c = O.Counters()
    sigma = O.gershgorin_shift(A)
    op = O.Operator(A, sigma, c)
    b = inputs.start_vector(n, 11, 0)
    P = O.build_poly(op, b, d, c, add_roots=False)
    assert P.degree == d and not P.breakdown
    # GMRES residual from the least-squares problem min ||beta e1 - H y||
    V, H, _, _ = O.gmres_arnoldi(op, b, d, O.Counters())
    rhs = np.zeros(d + 1)
    rhs[0] = np.linalg.norm(b)
    y = np.linalg.lstsq(H, rhs, rcond=None)[0]
    AV = np.column_stack([op(V[:, j]) for j in range(d)])
    r_gmres = b - AV @ y
    p, _ = O.apply_poly(op, P.roots, b)
    # Section 7: a factor (1 - lambda/theta_j) near cancellation loses about
    # u * pof(j) relative accuracy in that eigencomponent, so the bound scales
    # with the largest pof (Example 7's outlier eigenvalue 20000).
    maxpof = 10.0 ** O.pof_log10(P.roots).max()
    scale = np.linalg.norm(b)
    assert np.linalg.norm(p - r_gmres) <= (1e-10 + 1e-14 * maxpof) * scale


@pytest.mark.parametrize("kind", ["cd", "cd_complex", "band"])
def test_harmonic_ritz_generalized_form(kind):
    A = _mat(kind)
    n = A.shape[0]
    c = O.Counters()
    op = O.Operator(A, O.gershgorin_shift(A), c)
    V, H, d, brk = O.gmres_arnoldi(op, inputs.start_vector(n, 3, 0), 12, c)
    th = O.harmonic_ritz(H)
    gen = sla.eigvals(H.T @ H, H[:d, :d].T)
    key = lambda z: (round(z.real, 6), round(z.imag, 6))  # noqa: E731
    a = np.array(sorted(th, key=key))
    g = np.array(sorted(gen, key=key))
    assert np.max(np.abs(a - g) / np.abs(g)) < 1e-8
    if kind == "cd_complex":
        assert np.any(np.abs(th.imag) > 0)


def test_full_degree_roots_are_eigenvalues():
    rng = np.random.default_rng(0)
    n = 8
    M = rng.standard_normal((n, n)) + 4 * np.eye(n)
    A = O.to_scipy(inputs.CSR(n, np.arange(0, n * n + 1, n, dtype=np.int64),
                              np.tile(np.arange(n, dtype=np.int32), n), M.ravel()))
    c = O.Counters()
    op = O.Operator(A, 0.0, c)
    b = rng.standard_normal(n)
    P = O.build_poly(op, b, n, c, add_roots=False)
    ev = np.linalg.eigvals(M)
    for z in ev:
        assert np.min(np.abs(P.roots - z)) < 1e-8 * np.abs(ev).max()
    p, _ = O.apply_poly(op, P.roots, b)
    assert np.linalg.norm(p) < 1e-9 * np.linalg.norm(b)


@pytest.mark.parametrize("kind", ["cd", "cd_complex", "band"])
def test_factored_matches_power_form_and_running_sum(kind):
    A = _mat(kind)
    n = A.shape[0]
    c = O.Counters()
    sigma = O.gershgorin_shift(A)
    op = O.Operator(A, sigma, c)
    P = O.build_poly(op, inputs.start_vector(n, 1, 0), 8, c, add_roots=False)
    x = inputs.start_vector(n, 2, 0)
    # monomial coefficients of pi(z) = prod(1 - z/theta): lowest degree first
    coef = np.poly(P.roots)[::-1] * ((-1) ** len(P.roots)) / np.prod(P.roots)
    coef = coef.real
    assert abs(coef[0] - 1.0) < 1e-12
    # Horner on A: sum_k coef_k A^k x
    y = coef[-1] * x
    for a in coef[-2::-1]:
        y = op(y) + a * x
    # phi(z) = (1 - pi(z))/z  ->  A phi(A) x = x - pi(A) x by the power form
    p, r = O.apply_poly(op, P.roots, x)
    nx = np.linalg.norm(x)
    assert np.linalg.norm(p - y) <= 1e-9 * nx * max(1.0, np.abs(coef).max())
    phi = -coef[1:]
    z = phi[-1] * x
    for a in phi[-2::-1]:
        z = op(z) + a * x
    Aphi = op(z)
    assert np.linalg.norm(r - Aphi) <= 1e-9 * nx * max(1.0, np.abs(coef).max())
    if kind == "cd_complex":
        assert np.any(np.abs(P.roots.imag) > 0)


def test_apply_on_diagonal_equals_scalar_polynomial():
    """pi(D) x = pi(lambda_i) x_i entrywise, with real roots and conjugate pairs."""
    lam = np.linspace(0.5, 3.0, 40)
    A = O.to_scipy(inputs.diagonal(lam))
    roots = O.modified_leja(np.array([2.5, 1.0 + 0.5j, 1.0 - 0.5j, 0.7, 2.0 + 1.5j, 2.0 - 1.5j]))
    x = inputs.start_vector(40, 4, 0)
    p, r = O.apply_poly(O.Operator(A, 0.0, O.Counters()), roots, x)
    pv = O.poly_eval(roots, lam)
    assert np.max(np.abs(pv.imag)) < 1e-12
    assert np.allclose(p, pv.real * x, rtol=0, atol=1e-13)
    assert np.allclose(r, (1 - pv.real) * x, rtol=0, atol=1e-13)


def test_table1_rows():
    """Table 1 (Section 3): Omega_g, Omega_b and rho for d = standard, 1..8, 16, 24."""
    lam = inputs.figure1_diag()
    A = O.to_scipy(inputs.diagonal(lam))
    nev = 5

    def rho(g, bad):
        lo, hi = bad.min(), bad.max()
        if g.min() <= hi and g.max() >= lo:
            return 1.0
        dist = np.where(g < lo, lo - g, g - hi)
        s = g[np.argmin(dist)]
        K = max(abs(s - lo), abs(s - hi)) / min(abs(s - lo), abs(s - hi))
        return (np.sqrt(K) - 1) / (np.sqrt(K) + 1)

    for row in read_golden("table1.txt"):
        d = int(row[0])
        want = np.array([float(v) for v in row[1:]])
        if d == 0:
            img = lam
        else:
            P = O.build_poly(O.Operator(A, 0.0, O.Counters()), np.ones(lam.size), d,
                             O.Counters(), add_roots=False)
            img = O.poly_eval(P.roots, lam).real
        g, bad = img[:nev], img[nev:]
        got = np.array([g.min(), g.max(), bad.min(), bad.max(), rho(g, bad)])
        assert np.max(np.abs(got - want)) <= 1.5e-4, (d, got, want)


def test_rho_d1_independent_of_start_vector():
    """d = 1: K_m(pi(A), v) = K_m(A, v), so rho equals the standard row (Section 3)."""
    lam = inputs.figure1_diag()
    A = O.to_scipy(inputs.diagonal(lam))
    for s in range(3):
        P = O.build_poly(O.Operator(A, 0.0, O.Counters()), inputs.start_vector(100, s, 0), 1,
                         O.Counters(), add_roots=False)
        img = O.poly_eval(P.roots, lam).real
        g, bad = img[:5], img[5:]
        s_ = g.min()
        K = (s_ - bad.min()) / (s_ - bad.max())
        rho = (np.sqrt(K) - 1) / (np.sqrt(K) + 1)
        assert abs(rho - 0.9416) < 1e-4


def test_double_polynomial_scalar_composition():
    """Section 8: the applied operator equals pi_2(tau(z)) with tau = 1 - pi_1 on eigenvectors."""
    lam = np.concatenate([np.linspace(0.05, 1.0, 30), np.linspace(2.0, 50.0, 170)])
    A = O.to_scipy(inputs.diagonal(lam))
    c = O.Counters()
    op = O.Operator(A, 0.0, c)
    b = inputs.start_vector(lam.size, 9, 0)
    P = O.build_double_poly(op, b, 5, 6, c, add_roots=False)
    x = inputs.start_vector(lam.size, 9, 1)
    y = make_operator(op, P, c)(x)
    tau = 1 - O.poly_eval(P.inner.roots, lam)
    want = O.poly_eval(P.roots, tau) * x
    assert np.max(np.abs(want.imag)) < 1e-10
    assert np.allclose(y, want.real, rtol=0, atol=1e-10 * np.abs(x).max())
