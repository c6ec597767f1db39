"""Host FP64 dense steps of the library (no GPU): parity with the oracle and
with LAPACK on small problems, and the C-ABI symbol inventory.

The dense eigensolver is the library's own Francis QR; it is compared with
LAPACK through numpy (eigenvalue sets, eigenvector residuals).  Leja order and
added roots are decisions taken in FP64 on identical inputs, so they must match
the oracle exactly (bit-exact root lists).
"""
import os
import re

import numpy as np
import pytest

import oracle as O
import oracle.ppa as ppa
from paper_1806_08020_gb300 import inputs

pp = pytest.importorskip("paper_1806_08020_gb300.pp")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    text = open(os.path.join(ROOT, "include", "pp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(pp_[a-z0-9_]+)\s*\(", text))
    assert len(names) >= 20
    import ctypes
    lib = ctypes.CDLL(pp.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pp.exported_symbols()) <= names


def _header_struct_fields(text, name):
    """(field, C type) pairs of ``typedef struct { ... } name;`` in the header."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    out = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if decl:
            ctype, field = decl.rsplit(None, 1)
            out.append((field.lstrip("*"), ctype + ("*" if field.startswith("*") else "")))
    return out


@pytest.mark.parametrize("name", ["pp_opts", "pp_stats"])
def test_binding_structs_match_the_header(name):
    """The ctypes structures of the binding have the header's fields, in order,
    with the same widths (a mismatch would shift every later field)."""
    import ctypes
    text = open(os.path.join(ROOT, "include", "pp.h")).read()
    fields = _header_struct_fields(text, name)
    py = getattr(pp, name)._fields_
    assert [f for f, _ in fields] == [f for f, _ in py]
    width = {"int": 4, "int32_t": 4, "int64_t": 8, "double": 8, "void*": ctypes.sizeof(ctypes.c_void_p)}
    for (f, ctype), (_, pytype) in zip(fields, py):
        assert width[ctype] == ctypes.sizeof(pytype), (f, ctype, pytype)


def _match(a, b):
    """max distance from each of a to the nearest of b (relative)."""
    return max(np.min(np.abs(b - z)) / max(1.0, abs(z)) for z in a)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("n", [1, 2, 3, 7, 30, 64])
def test_dense_eig_random(seed, n):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    lam, V = pp.pp_dense_eig(A)
    ref = np.linalg.eigvals(A)
    assert _match(lam, ref) < 1e-10 and _match(ref, lam) < 1e-10
    # conjugate pairs adjacent, im > 0 first, exact conjugates
    i = 0
    while i < n:
        if lam[i].imag != 0:
            assert lam[i].imag > 0 and lam[i + 1] == np.conj(lam[i])
            x = V[:, i] + 1j * V[:, i + 1]
            assert abs(np.linalg.norm(x) - 1) < 1e-12
            assert np.linalg.norm(A @ x - lam[i] * x) < 1e-9 * np.linalg.norm(A)
            i += 2
        else:
            x = V[:, i]
            assert abs(np.linalg.norm(x) - 1) < 1e-12
            assert np.linalg.norm(A @ x - lam[i].real * x) < 1e-9 * np.linalg.norm(A)
            i += 1


def test_dense_eig_structured():
    # Hessenberg from Arnoldi on a CD matrix, a Jordan-like block and a diagonal
    A = O.to_scipy(inputs.convection_diffusion_2d(12, 30.0))
    V, H, d, _ = O.gmres_arnoldi(O.Operator(A, 0.0, O.Counters()), inputs.start_vector(144, 1, 0), 40,
                                 O.Counters())
    Hd = H[:d, :d]
    lam, _ = pp.pp_dense_eig(Hd)
    assert _match(lam, np.linalg.eigvals(Hd)) < 1e-9
    D = np.diag(np.arange(1.0, 11.0))
    lam, V = pp.pp_dense_eig(D)
    assert np.allclose(np.sort(lam.real), np.arange(1.0, 11.0))
    J = np.diag(np.full(6, 2.0)) + np.diag(np.full(5, 1e-3), 1)
    lam, _ = pp.pp_dense_eig(J)
    assert np.allclose(lam, 2.0, atol=1e-2)


@pytest.mark.parametrize("kind", ["cd", "cd_complex", "band", "ex7"])
def test_harmonic_ritz_matches_oracle(kind):
    if kind == "cd":
        A = O.to_scipy(inputs.convection_diffusion_2d(12, 20.0))
    elif kind == "cd_complex":
        A = O.to_scipy(inputs.convection_diffusion_2d(10, 60.0))
    elif kind == "band":
        A = O.to_scipy(inputs.banded_random(300, 4, 3))
    else:
        A = O.to_scipy(inputs.diagonal(inputs.example7_diag()))
    op = O.Operator(A, O.gershgorin_shift(A), O.Counters())
    for d in (1, 5, 12, 25):
        V, H, dd, brk = O.gmres_arnoldi(op, inputs.start_vector(A.shape[0], 4, 0), d, O.Counters())
        assert not brk
        got = pp.pp_harmonic_ritz(H)
        ref = O.harmonic_ritz(H)
        assert _match(got, ref) < 1e-9 and _match(ref, got) < 1e-9


@pytest.mark.parametrize("seed", range(20))
def test_leja_matches_oracle_exactly(seed):
    rng = np.random.default_rng(seed)
    nr, npair = int(rng.integers(0, 12)), int(rng.integers(0, 8))
    if nr + npair == 0:
        nr = 1
    re = list(rng.uniform(-5, 50, nr))
    pr = []
    for _ in range(npair):
        z = complex(rng.uniform(-5, 50), rng.uniform(0.1, 20))
        pr += [z, np.conj(z)]
    r = np.array(re + pr, dtype=complex)
    r = r[rng.permutation(r.size)]
    assert np.array_equal(pp.pp_leja_order(r), O.modified_leja(r))


def test_leja_ties_match_oracle():
    for r in ([1.0, -1.0, 2.0, -2.0], [3.0, 3.0, 1.0], [1 + 1j, 1 - 1j, -1 + 1j, -1 - 1j]):
        r = np.array(r, dtype=complex)
        assert np.array_equal(pp.pp_leja_order(r), O.modified_leja(r))


@pytest.mark.parametrize("d", [8, 15, 25, 40])
def test_added_roots_match_oracle(d):
    A = O.to_scipy(inputs.diagonal(inputs.example7_diag()))
    P = O.build_poly(O.Operator(A, 0.0, O.Counters()), inputs.start_vector(10000, 3, 0), d, O.Counters(),
                     add_roots=False)
    ref, added = O.add_stability_roots(P.roots)
    got = pp.pp_add_stability_roots(P.roots)
    assert np.array_equal(got, ref)
    assert added >= 1


def test_added_roots_pairs_match_oracle():
    z = 30000.0 + 5000.0j
    roots = O.modified_leja(np.array([z, np.conj(z), 1, 2, 3, 4, 5, 6, 20000.0], dtype=complex))
    ref, _ = O.add_stability_roots(roots)
    assert np.array_equal(pp.pp_add_stability_roots(roots), ref)


def test_host_entry_points_reject_bad_input():
    with pytest.raises(pp.PPError):
        pp.pp_leja_order(np.array([1 + 1j, 2 - 1j]))
    with pytest.raises(pp.PPError):
        pp.pp_harmonic_ritz(np.zeros((3, 2)))


def _arnoldi_dense(B, v, m):
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


@pytest.mark.parametrize("harmonic", [False, True])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_restart_basis_matches_oracle(harmonic, seed):
    """The library's host restart step (Ritz or harmonic, Section 4 / Example 2)
    against the oracle's: the same ordered values, the same kept subspace, and
    the Arnoldi relation with the new basis."""
    rng = np.random.default_rng(seed)
    n, m, k, tau = 80, 16, 7, 1.0
    B = rng.standard_normal((n, n)) / np.sqrt(n) + np.diag(np.linspace(0.0, 3.0, n))
    V, H = _arnoldi_dense(B, rng.standard_normal(n), m)
    Q, Hn, kk, vals = pp.pp_restart_basis(H, k, tau, harmonic)
    if harmonic:
        K, cvec = O.harmonic_restart_matrix(H, m, tau)
        nu = np.linalg.eigvals(K)
    else:
        cvec = None
        nu = np.linalg.eigvals(H[:m, :m])
    order = ppa.ritz_order(nu, tau)
    assert np.allclose(vals, nu[order], rtol=1e-10, atol=1e-12)
    assert kk == (k - 1 if nu[order[k - 1]].imag > 0 else k)
    Vk = V @ Q if harmonic else np.column_stack([V[:, :m] @ Q, V[:, m]])
    assert Vk.shape[1] == kk + 1
    assert np.allclose(Vk.T @ Vk, np.eye(kk + 1), atol=1e-12)
    assert np.linalg.norm(B @ Vk[:, :kk] - Vk @ Hn[: kk + 1, :kk]) <= 1e-11 * np.linalg.norm(B, 2)
    # the oracle's restart from its own vectors spans the same space
    w, S = np.linalg.eig(K if harmonic else H[:m, :m])
    o = ppa.ritz_order(w, tau)
    cols = []
    for i in o[:kk]:
        if w[i].imag == 0:
            cols.append(S[:, i].real)
        elif w[i].imag > 0:
            cols += [S[:, i].real, S[:, i].imag]
    Qo, _ = np.linalg.qr(np.stack(cols, axis=1))
    Vo, _ = O.thick_restart(V, H, m, Qo, cvec)
    Pk, Po = Vk[:, :kk], Vo[:, :kk]
    assert np.linalg.norm(Pk @ (Pk.T @ Po) - Po) <= 1e-9
