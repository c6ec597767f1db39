"""Pins of the oracle's harmonic restart (the harmonic Arnoldi variant of
Example 2: harmonic Ritz vectors kept at the restart instead of Ritz vectors).

Each pin is a fact independent of the formula the oracle uses:
* the harmonic Ritz values solve the Petrov-Galerkin condition written out as a
  generalised eigenproblem on the explicit vectors (B - tau) V_m and V_m;
* they are tau + 1/mu for the Ritz values mu of (B - tau)^{-1} on the subspace
  (B - tau) V_m (textbook equivalence, with an explicit inverse);
* every harmonic residual is parallel to V_{m+1} c (the oracle's c);
* the restarted basis keeps the Arnoldi relation and orthonormality;
* the restarted eigensolver converges to the eigenvalues of a dense solve.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import oracle.ppa as ppa
from paper_1806_08020_gb300 import inputs


def _arnoldi(B, v, m):
    n = B.shape[0]
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = v / np.linalg.norm(v)
    for j in range(m):
        w = B @ V[:, j]
        for _ in range(2):
            h = V[:, : j + 1].T @ w
            w = w - V[:, : j + 1] @ h
            H[: j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return V, H


def _same_set(a, b, rtol=1e-8):
    """The two multisets of complex numbers agree (optimal matching)."""
    from scipy.optimize import linear_sum_assignment
    a, b = np.asarray(a), np.asarray(b)
    D = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(D)
    return a.size == b.size and np.all(D[r, c] <= rtol * np.maximum(1.0, np.abs(a[r])))


def _case(seed=3, n=60, m=14):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n)) / np.sqrt(n) + np.diag(np.linspace(0.0, 3.0, n))
    V, H = _arnoldi(B, rng.standard_normal(n), m)
    return B, V, H, m


@pytest.mark.parametrize("tau", [0.0, 1.0, 0.37])
def test_harmonic_values_solve_the_galerkin_condition(tau):
    B, V, H, m = _case()
    K, _ = O.harmonic_restart_matrix(H, m, tau)
    theta = np.linalg.eigvals(K)
    W = (B - tau * np.eye(B.shape[0])) @ V[:, :m]
    lam = sla.eigvals(W.T @ W, W.T @ V[:, :m]) + tau
    assert _same_set(theta, lam)


def test_harmonic_values_are_inverse_ritz_values():
    B, V, H, m = _case(seed=7)
    tau = 0.8
    n = B.shape[0]
    K, _ = O.harmonic_restart_matrix(H, m, tau)
    theta = np.linalg.eigvals(K)
    Qw, _ = np.linalg.qr((B - tau * np.eye(n)) @ V[:, :m])
    mu = np.linalg.eigvals(Qw.T @ np.linalg.inv(B - tau * np.eye(n)) @ Qw)
    assert _same_set(theta, tau + 1.0 / mu)


def test_harmonic_residuals_share_one_direction():
    B, V, H, m = _case(seed=11)
    tau = 1.0
    K, c = O.harmonic_restart_matrix(H, m, tau)
    theta, G = np.linalg.eig(K)
    u = V @ c
    u /= np.linalg.norm(u)
    for i in range(m):
        y = V[:, :m] @ G[:, i]
        r = B @ y - theta[i] * y
        assert np.linalg.norm(r - u * np.vdot(u, r)) <= 1e-9 * max(1.0, np.linalg.norm(r))


@pytest.mark.parametrize("harmonic", [False, True])
def test_restart_keeps_the_arnoldi_relation(harmonic):
    B, V, H, m = _case(seed=5)
    tau = 1.0
    if harmonic:
        K, c = O.harmonic_restart_matrix(H, m, tau)
        th, G = np.linalg.eig(K)
    else:
        c = None
        th, G = np.linalg.eig(H[:m, :m])
    order = np.argsort(np.abs(th - tau), kind="stable")
    cols = []
    for i in order[:6]:
        if th[i].imag == 0:
            cols.append(G[:, i].real)
        elif th[i].imag > 0:
            cols += [G[:, i].real, G[:, i].imag]
    if len(cols) > 6:
        cols = cols[:5]  # keep conjugate pairs whole
    Q, _ = np.linalg.qr(np.stack(cols, axis=1))
    kk = Q.shape[1]
    Vk, Hn = O.thick_restart(V, H, m, Q, c)
    assert Vk.shape[1] == kk + 1
    assert np.allclose(Vk.T @ Vk, np.eye(kk + 1), atol=1e-12)
    lhs = B @ Vk[:, :kk]
    rhs = Vk @ Hn[: kk + 1, :kk]
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(B, 2) * np.sqrt(kk)
    if harmonic:  # the kept harmonic Ritz vectors lie in the new basis' first kk columns
        y = V[:, :m] @ G[:, order[0]]
        assert np.linalg.norm(y - Vk[:, :kk] @ (Vk[:, :kk].T @ y)) <= 1e-10 * np.linalg.norm(y)


@pytest.mark.parametrize("case", ["diag_sm", "cd_poly"])
def test_harmonic_eigs_converge_to_dense_eigenvalues(case):
    if case == "diag_sm":
        Acsr = inputs.diagonal(np.arange(1, 401.0))
        A = O.to_scipy(Acsr)
        op = O.Operator(A, 0.0, O.Counters())
        tp, tgt, nev, m, k = 0.0, "SM", 6, 30, 12
        exact = np.arange(1, 7.0)
    else:
        Acsr = inputs.convection_diffusion_2d(20, 10.0)
        A = O.to_scipy(Acsr)
        sig = O.gershgorin_shift(A)
        base = O.Operator(A, sig, O.Counters())
        poly = O.build_poly(base, inputs.start_vector(A.shape[0], 2, 0), 8, O.Counters())
        op = ppa.make_operator(base, poly, O.Counters())
        tp, tgt, nev, m, k = 1.0, "SR", 5, 30, 12
        w = np.linalg.eigvals(A.toarray())
        exact = np.sort(w.real)[:nev]
    sigma = 0.0 if case == "diag_sm" else sig
    v0 = inputs.start_vector(A.shape[0], 2, 1)
    R = O.eigs(A, op, nev, m, k, 1e-9, v0, O.Counters(), target_point=tp, target=tgt, sigma=sigma,
               restart="harmonic")
    assert R.converged
    assert np.all(R.resid <= 1e-9)
    assert np.allclose(np.sort(R.lam.real)[:nev], exact, rtol=1e-7)
    assert np.max(np.abs(R.lam.imag)) < 1e-8 * np.max(np.abs(R.lam))


# --- planted mistakes (on the CPU): each must fail one of the pins above ---

def _k_transposed_solve(H, m, tau):
    Hm = H[:m, :m]
    em = np.eye(m)[:, -1]
    f = np.linalg.solve(Hm - tau * np.eye(m), em)  # M^{-1} e_m instead of M^{-T} e_m
    return Hm + H[m, m - 1] ** 2 * np.outer(f, em)


def _k_h_not_squared(H, m, tau):
    Hm = H[:m, :m]
    em = np.eye(m)[:, -1]
    f = np.linalg.solve((Hm - tau * np.eye(m)).T, em)
    return Hm + H[m, m - 1] * np.outer(f, em)


def _k_shift_dropped(H, m, tau):
    Hm = H[:m, :m]
    em = np.eye(m)[:, -1]
    f = np.linalg.solve(Hm.T, em)  # the target ignored
    return Hm + H[m, m - 1] ** 2 * np.outer(f, em)


@pytest.mark.parametrize("mutant", [_k_transposed_solve, _k_h_not_squared, _k_shift_dropped])
def test_harmonic_matrix_mutants_are_caught(mutant):
    B, V, H, m = _case()
    tau = 0.37
    W = (B - tau * np.eye(B.shape[0])) @ V[:, :m]
    lam = sla.eigvals(W.T @ W, W.T @ V[:, :m]) + tau
    assert not _same_set(np.linalg.eigvals(mutant(H, m, tau)), lam)


def test_restart_without_orthogonalising_c_is_caught():
    B, V, H, m = _case(seed=5)
    K, c = O.harmonic_restart_matrix(H, m, 1.0)
    th, G = np.linalg.eig(K)
    order = np.argsort(np.abs(th - 1.0), kind="stable")
    cols = []
    for i in order[:4]:
        if th[i].imag == 0:
            cols.append(G[:, i].real)
        elif th[i].imag > 0:
            cols += [G[:, i].real, G[:, i].imag]
    Q, _ = np.linalg.qr(np.stack(cols[:4], axis=1))
    kk = Q.shape[1]
    # mutant: P's last column is c / ||c|| without the projection
    P = np.zeros((m + 1, kk + 1))
    P[:m, :kk] = Q
    P[:, kk] = c / np.linalg.norm(c)
    Vk = V @ P
    assert not np.allclose(Vk.T @ Vk, np.eye(kk + 1), atol=1e-12)
