"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

Each mutant replaces one oracle step with a subtly wrong version: a dropped
term, a transposed operand, a wrong sign, a wrong selection.  The pin used is
an independent fact (GMRES optimality, the scalar polynomial, the Leja greedy
property, Table 1), so a passing pin suite with a failing mutant here means
the pins are too weak.
"""
import numpy as np
import pytest

import oracle as O
import oracle.ppa as ppa
from paper_1806_08020_gb300 import inputs


def _gmres_identity_error(harmonic=None, apply=None):
    A = O.to_scipy(inputs.convection_diffusion_2d(10, 60.0))  # complex spectrum
    n = A.shape[0]
    op = O.Operator(A, O.gershgorin_shift(A), O.Counters())
    b = inputs.start_vector(n, 11, 0)
    d = 8
    V, H, _, _ = O.gmres_arnoldi(op, b, d, O.Counters())
    th = (harmonic or O.harmonic_ritz)(H)
    roots = O.modified_leja(th)
    rhs = np.zeros(d + 1)
    rhs[0] = np.linalg.norm(b)
    y = np.linalg.lstsq(H, rhs, rcond=None)[0]
    r_gmres = b - np.column_stack([op(V[:, j]) for j in range(d)]) @ y
    p, _ = (apply or O.apply_poly)(op, roots, b)
    return np.linalg.norm(p - r_gmres) / np.linalg.norm(b)


def test_unmutated_passes():
    assert _gmres_identity_error() < 1e-10


def _harm_drop_h2(H, breakdown=False):
    d = H.shape[1]
    return np.linalg.eigvals(H[:d, :d])


def _harm_transposed_f(H, breakdown=False):
    d = H.shape[1]
    Hd = H[:d, :d]
    ed = np.zeros(d)
    ed[-1] = 1
    f = np.linalg.solve(Hd, ed)
    return np.linalg.eigvals(Hd + H[d, d - 1] ** 2 * np.outer(f, ed))


def _harm_h_not_squared(H, breakdown=False):
    d = H.shape[1]
    Hd = H[:d, :d]
    ed = np.zeros(d)
    ed[-1] = 1
    f = np.linalg.solve(Hd.T, ed)
    return np.linalg.eigvals(Hd + H[d, d - 1] * np.outer(f, ed))


def _apply_pair_sign(op, roots, x, c=None):
    p = x.copy()
    i = 0
    while i < roots.size:
        th = roots[i]
        if th.imag == 0:
            p = p - op(p) / th.real
            i += 1
        else:
            m2 = abs(th) ** 2
            t = op(p)
            s = op(t)
            p = p - (2 * th.real / m2) * t - s / m2
            i += 2
    return p, None


def _apply_pair_uses_real_part_only(op, roots, x, c=None):
    p = x.copy()
    for th in roots:
        p = p - op(p) / th.real
    return p, None


@pytest.mark.parametrize("mutant", [_harm_drop_h2, _harm_transposed_f, _harm_h_not_squared])
def test_root_mutants_are_caught(mutant):
    assert _gmres_identity_error(harmonic=mutant) > 1e-6


@pytest.mark.parametrize("mutant", [_apply_pair_sign, _apply_pair_uses_real_part_only])
def test_apply_mutants_are_caught(mutant):
    assert _gmres_identity_error(apply=mutant) > 1e-6


def test_leja_mutant_is_caught():
    """Choosing the minimiser instead of the maximiser breaks the greedy property."""
    def leja_min(roots):
        units = ppa._units(roots)
        chosen = [units.pop(int(np.argmax([abs(z) for z in units])))]
        while units:
            pts = ppa._expand(chosen)
            score = [float(np.sum(np.log(np.abs(z - pts)))) for z in units]
            chosen.append(units.pop(int(np.argmin(score))))
        return ppa._expand(chosen)

    roots = np.array([0.1, 1.0, 2.0, 3.0, 4.0, 5.0], dtype=complex)
    out = leja_min(roots)
    chosen = [out[0]]
    ok = True
    for k in range(1, out.size):
        prods = [np.prod(np.abs(z - np.array(chosen))) for z in out[k:]]
        ok &= np.prod(np.abs(out[k] - np.array(chosen))) >= max(prods) * (1 - 1e-12)
        chosen.append(out[k])
    assert not ok


def test_restart_mutant_is_caught():
    """Dropping the h_{m+1,m} e_m^T Q_k row at restart breaks the Arnoldi relation:
    the n = 2500 config then no longer reaches the closed-form eigenvalues."""
    cfg = inputs.plain_small()
    A = O.to_scipy(cfg["A"])
    c = O.Counters()
    op = O.Operator(A, 0.0, c)
    P = O.build_poly(op, inputs.start_vector(2500, cfg["seed"], 0), cfg["d"], c)
    opp = ppa.make_operator(op, P, c)
    v0 = inputs.start_vector(2500, cfg["seed"], 1)
    got = np.sort(_eigs_without_coupling(A, opp, 10, 30, 15, v0))[:2]
    want = np.array([120.52154374, 149.50971687])  # closed form, 2-D CD N = 50, beta = 20
    assert not np.allclose(got, want, rtol=1e-8)
    # the unmutated oracle reaches them
    R = O.eigs(A, opp, 10, 30, 15, 1e-8, v0, c)
    assert np.allclose(np.sort(R.lam.real)[:2], want, rtol=1e-8)


def _eigs_without_coupling(A, op, nev, m, k, v0, cycles=6):
    n = v0.size
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = v0 / np.linalg.norm(v0)
    j0 = 0
    c = O.Counters()
    for _ in range(cycles):
        for j in range(j0, m):
            w, h = O.cgs2(V[:, : j + 1], op(V[:, j]), c)
            H[: j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            V[:, j + 1] = w / H[j + 1, j]
        nu, S = np.linalg.eig(H[:m, :m])
        order = ppa.ritz_order(nu, 1.0)
        cols = []
        for i in order[:k]:
            if nu[i].imag >= 0:
                cols.append(S[:, i].real)
                if nu[i].imag > 0:
                    cols.append(S[:, i].imag)
        Q, _ = np.linalg.qr(np.stack(cols, axis=1)[:, :k])
        V[:, :k] = V[:, :m] @ Q
        V[:, k] = V[:, m]
        Hn = np.zeros((m + 1, m))
        Hn[:k, :k] = Q.T @ H[:m, :m] @ Q
        H = Hn  # mutant: row k (h_{m+1,m} e_m^T Q_k) left at zero
        j0 = k
    nu, S = np.linalg.eig(H[:m, :m])
    order = ppa.ritz_order(nu, 1.0)[:nev]
    out = []
    for i in order:
        y = V[:, :m] @ S[:, i]
        y /= np.linalg.norm(y)
        out.append(np.vdot(y, A @ y).real)
    return np.array(out)


# ---- damping heuristic (Section 6.3 box) ----

def _ideal_strict_first(mu, nev, k):  # "<" instead of "<=" among the first nev
    a = np.abs(np.asarray(mu)[:k])
    return bool(all(a[i] < a[i + 1] for i in range(nev - 1)) and a[nev - 1] < a[nev:k].min())


def _ideal_no_boundary(mu, nev, k):  # forgets the comparison with the last k - nev
    a = np.abs(np.asarray(mu)[:k])
    return bool(all(a[i] <= a[i + 1] for i in range(nev - 1)))


def _ideal_real_part(mu, nev, k):  # compares real parts instead of magnitudes
    a = np.real(np.asarray(mu)[:k])
    return bool(all(a[i] <= a[i + 1] for i in range(nev - 1)) and a[nev - 1] < a[nev:k].min())


@pytest.mark.parametrize("mutant", [_ideal_strict_first, _ideal_no_boundary, _ideal_real_part])
def test_ideal_order_mutants_caught(mutant, monkeypatch):
    import test_oracle_damping as T
    monkeypatch.setattr(O, "ideal_order", mutant)
    failures = 0
    for t in (T.test_paper_sequence_fails_ideal_order, T.test_ideal_order_boundaries):
        try:
            t()
        except AssertionError:
            failures += 1
    assert failures > 0


def test_damping_without_power_step_caught(monkeypatch):
    """A heuristic that 'damps' by rebuilding from b itself (no A b) never passes at d = 50."""
    import test_oracle_damping as T
    real_build = ppa.build_poly
    calls = []

    def build_no_damp(op, b, d, c, add_roots=True):
        calls.append(d)
        return real_build(op, T_b[0], d, c, add_roots)
    A = O.to_scipy(inputs.diagonal(inputs.example6_diag()))
    T_b = [inputs.start_vector(A.shape[0], 2, 0)]
    monkeypatch.setattr(ppa, "build_poly", build_no_damp)
    with pytest.raises(AssertionError):
        T.test_example6_d50_damping(A, 2)
