"""Pins of the oracle's restarted Arnoldi(m, k) on pi(A).

* Dense eigendecomposition on small matrices: the nev wanted eigenvalues as a
  set, and residuals ||A x - mu x|| <= rtol ||A||_1 (Section 4).
* Closed-form eigenvalues of the constant-coefficient convection-diffusion
  operator: a tridiagonal Toeplitz matrix tridiag(b, a, c) has eigenvalues
  a + 2 sqrt(bc) cos(j pi/(N+1)); the 2-D operator is a Kronecker sum.
* Shift invariance at d = 1 (Section 3): Ritz values of pi(A) = 1 - A/theta
  are the affine image of plain Arnoldi's Ritz values.
* Example 7 (Section 7): the attainable residual with and without the added
  root, order-of-magnitude pins against the paper's printed values.
* Example 6 (Section 6.2): operation counts against the paper's averages.
"""
import numpy as np
import pytest

import oracle as O
from oracle.ppa import make_operator
from paper_1806_08020_gb300 import inputs
from conftest import golden_dict


def cd2d_closed_form(N, beta):
    h = 1.0 / (N + 1)
    j = np.arange(1, N + 1)
    c = np.cos(j * np.pi / (N + 1))
    x = (2 - 2 * np.sqrt(1 - (beta * h / 2) ** 2 + 0j) * c) / h**2
    y = (2 - 2 * c) / h**2
    return (x[:, None] + y[None, :]).ravel()


def eig_with_condition(M):
    """Eigenvalues and their condition numbers ||x|| ||y|| / |y^H x| (left y, right x)."""
    import scipy.linalg as sla
    w, vl, vr = sla.eig(M, left=True, right=True)
    kap = np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0) / np.abs(np.sum(vl.conj() * vr, axis=0))
    return w, kap


def solve(A_csr, d, nev, m, k, seed, rtol=1e-8, target="SR", maxc=500, add=True):
    A = O.to_scipy(A_csr)
    c = O.Counters()
    sigma = O.gershgorin_shift(A) if target == "SR" else 0.0
    op = O.Operator(A, sigma, c)
    n = A.shape[0]
    b = inputs.start_vector(n, seed, 0)
    v0 = inputs.start_vector(n, seed, 1)
    P = O.build_poly(op, b, d, c, add_roots=add) if d > 0 else None
    R = O.eigs(A, make_operator(op, P, c), nev, m, k, rtol, v0, c,
               target_point=1.0 if d else 0.0, target=target, max_cycles=maxc, sigma=sigma)
    return A, R


def test_closed_form_matches_dense():
    lam = np.sort(cd2d_closed_form(10, 8.0).real)
    A = inputs.convection_diffusion_2d(10, 8.0).to_dense()
    ev = np.sort(np.linalg.eigvals(A).real)
    assert np.max(np.abs(lam - ev) / lam) < 1e-11


def test_plain_small_config_closed_form():
    """n = 2500 CD (beta = 20): 10 smallest eigenvalues vs the closed form at 1e-8."""
    cfg = inputs.plain_small()
    A, R = solve(cfg["A"], cfg["d"], cfg["nev"], cfg["m"], cfg["k"], cfg["seed"])
    assert R.converged
    assert np.all(R.resid <= 1e-8)
    want = np.sort(cd2d_closed_form(50, 20.0).real)[: cfg["nev"]]
    assert np.max(np.abs(np.sort(R.lam.real) - want) / want) < 1e-8
    assert np.max(np.abs(R.lam.imag)) < 1e-8 * want.max()


@pytest.mark.parametrize("case", ["cd_small", "band", "cd_complex", "ex6_small"])
def test_eigs_against_dense(case):
    if case == "cd_small":
        Acsr, d, nev, m, k, tgt = inputs.convection_diffusion_2d(20, 30.0), 8, 6, 24, 11, "SR"
    elif case == "band":
        Acsr, d, nev, m, k, tgt = inputs.banded_random(400, 4, 2), 5, 6, 30, 11, "SR"
    elif case == "cd_complex":
        Acsr, d, nev, m, k, tgt = inputs.convection_diffusion_2d(12, 60.0), 6, 6, 30, 11, "SR"
    else:
        Acsr, d, nev, m, k, tgt = inputs.diagonal(np.arange(1, 801.0)), 10, 8, 30, 13, "SM"
    A, R = solve(Acsr, d, nev, m, k, 21, target=tgt)
    assert R.converged
    assert np.all(R.resid <= 1e-8)
    ev, kap = eig_with_condition(Acsr.to_dense())
    if tgt == "SR":
        sigma = O.gershgorin_shift(A)
        o = np.argsort(np.abs(ev - sigma))
    else:
        o = np.argsort(np.abs(ev))
    ev, kap = ev[o], kap[o]
    nA = O.norm1(A)
    # every returned value is an eigenvalue of A within the first-order bound
    # kappa_j * ||r|| (plus slack), and one of the nev + 2 nearest the target.
    # For the clustered complex spectrum the level curves of pi are not circles
    # about sigma, so the wanted set may reach a few ranks further out.
    slack = 2 * nev if case == "cd_complex" else nev + 2
    for lam, res in zip(R.lam, R.resid):
        dist = np.abs(ev - lam)
        j = int(np.argmin(dist))
        assert dist[j] <= 10 * kap[j] * res * nA + 1e-12 * abs(lam)
        assert j < slack


def test_shift_invariance_degree_one():
    """Section 3: K_m(pi(A), v) = K_m(A, v) for d = 1; Ritz values map by z -> 1 - z/theta."""
    A = O.to_scipy(inputs.convection_diffusion_2d(15, 10.0))
    n = A.shape[0]
    c = O.Counters()
    op = O.Operator(A, 0.0, c)
    P = O.build_poly(op, inputs.start_vector(n, 2, 0), 1, c, add_roots=False)
    th = P.roots[0].real
    v0 = inputs.start_vector(n, 2, 1)
    m = 12
    Rp = O.eigs(A, make_operator(op, P, c), 3, m, 6, 1e-30, v0, c, max_cycles=1)
    Ra = O.eigs(A, op, 3, m, 6, 1e-30, v0, c, target_point=0.0, max_cycles=1)
    # same subspace -> same Rayleigh quotients on A for the wanted vectors
    assert np.allclose(np.sort(Rp.lam.real), np.sort(Ra.lam.real), rtol=1e-9)
    assert np.allclose(np.sort((1 - Ra.ritz / th).real), np.sort(Rp.ritz.real), rtol=1e-9)


@pytest.mark.slow
def test_example7_added_root_restores_accuracy():
    """Section 7 / Example 7: MaxErr ~2e-6 at d = 15 without added roots, ~1e-12 with;
    d = 25: 3.4e1 without, 2.8e-12 with (order-of-magnitude pins)."""
    g = golden_dict("example7.txt")
    Acsr = inputs.diagonal(inputs.example7_diag())

    def maxerr(d, add):
        A, R = solve(Acsr, d, 15, 50, 20, 7, rtol=1e-30, target="SM", maxc=25, add=add)
        return float(np.min(R.history) * O.norm1(A))

    e10 = maxerr(10, False)
    assert g["maxerr_noadd_d10"] / 100 < e10 < g["maxerr_noadd_d10"] * 100
    e15 = maxerr(15, False)
    assert g["maxerr_noadd_d15"] / 100 < e15 < g["maxerr_noadd_d15"] * 100
    e15a = maxerr(15, True)
    assert e15a < 1e-9
    e25 = maxerr(25, False)
    assert e25 > g["maxerr_noadd_d25"] / 100
    e25a = maxerr(25, True)
    assert e25a < g["maxerr_add_d25"] * 100


@pytest.mark.slow
def test_example6_counts():
    """Example 6: regular Arnoldi(50,20) ~1625 mvps; d = 40: vops ~15,390.8 and one or two cycles."""
    g = golden_dict("example6.txt")
    Acsr = inputs.diagonal(inputs.example6_diag())
    mv0, mv40, vo40 = [], [], []
    for s in range(2):
        _, R = solve(Acsr, 0, 15, 50, 20, 100 + s, target="SM")
        assert R.converged and np.allclose(np.sort(R.lam.real), np.arange(1, 16), rtol=1e-8)
        mv0.append(R.counters.mvps)
        _, R = solve(Acsr, 40, 15, 50, 20, 100 + s, target="SM")
        assert R.converged and np.allclose(np.sort(R.lam.real), np.arange(1, 16), rtol=1e-8)
        mv40.append(R.counters.mvps)
        vo40.append(R.counters.vops)
    assert 0.75 * g["mvps_d0"] < np.mean(mv0) < 1.25 * g["mvps_d0"]
    assert abs(np.mean(vo40) / g["vops_d40"] - 1) < 0.10
    # one cycle = 40 (GMRES) + 50*40 mvps; two cycles add 30*40
    assert 2000 <= np.mean(mv40) <= 3300


def test_cgs2_is_the_orthogonal_projection():
    """CGS2 (Section 4: one orthogonalisation and one reorthogonalisation pass)
    against the projection computed another way (least squares): the output is
    w - V c with c = argmin ||w - V c||, and it is orthogonal to V to working
    precision even when w lies almost in span(V); a single pass is not."""
    rng = np.random.default_rng(4)
    n, j = 400, 25
    V, _ = np.linalg.qr(rng.standard_normal((n, j)))
    for eps in (1.0, 1e-10):
        w = V @ rng.standard_normal(j) + eps * rng.standard_normal(n)
        out, h = O.cgs2(V, w.copy(), O.Counters())
        coef = np.linalg.lstsq(V, w, rcond=None)[0]
        assert np.allclose(h, coef, rtol=0, atol=1e-13 * np.linalg.norm(w))
        assert np.linalg.norm(V.T @ out) <= 1e-14 * np.linalg.norm(w) * np.sqrt(j)
        assert np.linalg.norm(out - (w - V @ coef)) <= 1e-13 * np.linalg.norm(w)
    # one pass only (the planted mistake): orthogonality is lost for the nearly dependent w
    one = w - V @ (V.T @ w)
    assert np.linalg.norm(V.T @ one) > 1e3 * np.linalg.norm(V.T @ out)
