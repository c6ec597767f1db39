"""Polynomial preconditioned restarted Arnoldi, written out plainly in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain NumPy/SciPy, no
blocking, no fusion, no reordering beyond what the cited passage states.

Citations name the paper's section, equation or algorithm box:

* "Section 2 box, step 1(a)-(c)": construction of the GMRES polynomial
  (one GMRES(d) cycle, harmonic Ritz values, modified Leja order).
* "Eq. (2.1)": the factored form pi(z) = prod_i (1 - z/theta_i).
* "Section 2 footnote 2": pi(z) = 1 - z*phi(z).
* "Section 4 opening paragraph": Arnoldi(m,k), conjugate-pair rule, one pass of
  reorthogonalisation, convergence test on A with Rayleigh quotients.
* "Section 7 box": pof and added roots.
* "Section 8": double polynomial preconditioning.
* "Section 5 box": polynomial determined by two starting vectors.
* "Section 6.3 box": heuristic for damping b and adjusting d.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------------------
# Operation counters (Section 4, Example 1: mvps, vops, dot products)
# ----------------------------------------------------------------------------

@dataclass
class Counters:
    """Matrix-vector products with A, length-n dot products and length-n vector operations.

    Section 4 counts mvps and vops (dot products, daxpys, scalings); Table 3 also
    counts dot products separately.  The paper notes the counts depend on
    implementation details, so they are used only as statistical pins.
    """

    mvps: int = 0
    dots: int = 0
    vops: int = 0


def to_scipy(A) -> sp.csr_matrix:
    """CSR from the shared input generator -> scipy CSR."""
    return sp.csr_matrix((A.vals, A.colind, A.rowptr), shape=(A.n, A.n))


def norm1(A: sp.csr_matrix) -> float:
    """||A||_1, the maximum absolute column sum.

    Section 4 asks for residual <= ||A|| * 1e-8 without naming the norm; the
    1-norm is exact, cheap and deterministic from CSR (reading recorded in the
    design notes).
    """
    return float(np.max(np.asarray(abs(A).sum(axis=0)).ravel()))


def gershgorin_shift(A: sp.csr_matrix) -> float:
    """Shift mu for the 'smallest real part' target (Section 2 footnote 1: use A - mu I).

    mu = min(0, min_i (a_ii - sum_{j != i} |a_ij|)), the leftmost point of the
    Gershgorin discs; a bound above -1e-12*||A||_1 counts as 0 (rounding).
    """
    d = A.diagonal()
    off = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
    lo = float(np.min(d - off))
    if lo >= -1e-12 * norm1(A):
        return 0.0
    return min(0.0, lo)


class Operator:
    """x -> (A - sigma I) x, counting one mvp per call (Section 2 footnote 1)."""

    def __init__(self, A: sp.csr_matrix, sigma: float, counters: Counters):
        self.A = A
        self.sigma = float(sigma)
        self.c = counters

    def __call__(self, x: np.ndarray) -> np.ndarray:
        self.c.mvps += 1
        y = self.A @ x
        if self.sigma != 0.0:
            y = y - self.sigma * x
        return y


# ----------------------------------------------------------------------------
# Gram-Schmidt with one reorthogonalisation pass (Section 4 opening paragraph)
# ----------------------------------------------------------------------------

def cgs2(V: np.ndarray, w: np.ndarray, c: Counters) -> tuple[np.ndarray, np.ndarray]:
    """Classical Gram-Schmidt of w against the orthonormal columns of V, done twice.

    Section 4 runs one reorthogonalisation pass after every orthogonalisation
    step.  Returns (w orthogonalised, h = h1 + h2).
    """
    j = V.shape[1]
    h1 = V.T @ w
    w = w - V @ h1
    h2 = V.T @ w
    w = w - V @ h2
    c.dots += 2 * j
    c.vops += 4 * j
    return w, h1 + h2


def gmres_arnoldi(op: Callable[[np.ndarray], np.ndarray], b: np.ndarray, d: int,
                  c: Counters, breakdown_tol: float = 1e-14):
    """One GMRES(d) cycle's Arnoldi process: A V_d = V_{d+1} H_{d+1,d} (Section 2 box, 1(a)).

    Returns (V, H, steps) where steps <= d is the number of columns actually
    built (a lucky breakdown h_{j+1,j} <= tol*||H||_F ends the process early).
    """
    n = b.size
    V = np.zeros((n, d + 1))
    H = np.zeros((d + 1, d))
    beta = np.linalg.norm(b)
    c.dots += 1
    c.vops += 2
    V[:, 0] = b / beta
    for j in range(d):
        w = op(V[:, j])
        w, h = cgs2(V[:, : j + 1], w, c)
        H[: j + 1, j] = h
        hn = np.linalg.norm(w)
        c.dots += 1
        c.vops += 2
        H[j + 1, j] = hn
        if hn <= breakdown_tol * np.linalg.norm(H[: j + 2, : j + 1]):
            return V[:, : j + 2], H[: j + 2, : j + 1], j + 1, True
        V[:, j + 1] = w / hn
    return V, H, d, False


def harmonic_ritz(H: np.ndarray, breakdown: bool = False) -> np.ndarray:
    """Roots of the GMRES polynomial (Section 2 box, step 1(b)).

    With A V_d = V_{d+1} H_{d+1,d}: the eigenvalues of H_d + h_{d+1,d}^2 f e_d^T,
    f = H_d^{-*} e_d (H is real, so H_d^{-*} = H_d^{-T}).  After a lucky
    breakdown the Krylov space is invariant and the roots are eig(H_d).
    """
    d = H.shape[1]
    Hd = H[:d, :d]
    if breakdown:
        return np.linalg.eigvals(Hd)
    ed = np.zeros(d)
    ed[-1] = 1.0
    f = np.linalg.solve(Hd.T, ed)
    M = Hd + H[d, d - 1] ** 2 * np.outer(f, ed)
    return np.linalg.eigvals(M)


# ----------------------------------------------------------------------------
# Modified Leja ordering (Section 2 box, step 1(c); Bai, Hu & Reichel alg. 3.1)
# ----------------------------------------------------------------------------

def _units(roots: np.ndarray) -> list[complex]:
    """Real roots and the upper member (Im > 0) of each conjugate pair.

    LAPACK returns exact conjugate pairs and exactly-zero imaginary parts for a
    real matrix, so pairs are matched exactly.
    """
    roots = np.asarray(roots, dtype=complex)
    up = [z for z in roots if z.imag > 0]
    lo = [z for z in roots if z.imag < 0]
    re = [z for z in roots if z.imag == 0]
    if sorted((z.real, -z.imag) for z in lo) != sorted((z.real, z.imag) for z in up):
        raise ValueError("roots are not closed under conjugation")
    return re + up


def _expand(units: list[complex]) -> np.ndarray:
    out = []
    for z in units:
        out.append(z)
        if z.imag != 0:
            out.append(np.conj(z))
    return np.asarray(out, dtype=complex)


def modified_leja(roots: np.ndarray) -> np.ndarray:
    """Modified Leja order of a conjugate-closed root set.

    First the root of largest modulus; then, repeatedly, the remaining root z
    that maximises prod_j |z - z_j| over the roots already chosen, evaluated
    as a sum of logarithms (the box's overflow remedy).  When a complex root is
    chosen (its Im > 0 member), its conjugate comes next.  Ties (paper silent):
    the candidate first in the order (-Re, -Im, position in the input).
    """
    units = _units(roots)
    key = sorted(range(len(units)), key=lambda i: (-units[i].real, -units[i].imag, i))
    cand = [units[i] for i in key]
    chosen: list[complex] = []
    # first point: largest modulus
    mags = [abs(z) for z in cand]
    first = int(np.argmax(mags))
    chosen.append(cand.pop(first))
    while cand:
        pts = _expand(chosen)
        score = [float(np.sum(np.log(np.abs(z - pts)))) for z in cand]
        nxt = int(np.argmax(score))
        chosen.append(cand.pop(nxt))
    return _expand(chosen)


# ----------------------------------------------------------------------------
# Stability: pof and added roots (Section 7 box "Adding Roots for Stability")
# ----------------------------------------------------------------------------

def pof_log10(roots: np.ndarray) -> np.ndarray:
    """log10 pof(j) = sum_{i != j} log10 |1 - theta_j/theta_i| (Section 7)."""
    roots = np.asarray(roots, dtype=complex)
    out = np.empty(roots.size)
    for j in range(roots.size):
        others = np.delete(roots, j)
        out[j] = float(np.sum(np.log10(np.abs(1.0 - roots[j] / others))))
    return out


def extra_copies(lp: float) -> int:
    """Number of added copies of a root with log10 pof = lp (Section 7 box, step 3).

    The box asks for the least integer greater than (log10 pof - 4)/14; the prose
    before it says double root above 1e4, triple above 1e18, quadruple above 1e32.
    Reading: ceil((lp - 4)/14) clipped at 0, which matches the prose; the two
    readings differ only when (lp - 4)/14 is an exact integer.
    """
    return max(0, int(np.ceil((lp - 4.0) / 14.0)))


def add_stability_roots(ordered: np.ndarray) -> tuple[np.ndarray, int]:
    """Append copies of roots with large pof (Section 7 box, step 3).

    For each root (a conjugate pair is one unit) with c > 0 copies, in Leja
    order: the first copy goes to the end of the list; copies t = 2..c are
    spaced evenly into the interior between the root's position p and the end,
    at unit positions p + floor((t-1)(L-p)/c), L the current length in units.
    Returns (new root list, number of roots added).
    """
    units = _units_in_order(ordered)
    lp = pof_log10(ordered)
    # pof of a unit = pof of its (first) member; conjugates have equal pof
    unit_lp = []
    pos = 0
    for u in units:
        unit_lp.append(lp[pos])
        pos += 2 if u.imag != 0 else 1
    # list of (value, original-unit-id or None for copies)
    lst: list[tuple[complex, int | None]] = [(u, i) for i, u in enumerate(units)]
    added = 0
    for uid, u in enumerate(units):
        ncop = extra_copies(unit_lp[uid])
        if ncop == 0:
            continue
        p = next(i for i, (_, oid) in enumerate(lst) if oid == uid)
        L = len(lst)
        inserts = [p + ((t - 1) * (L - p)) // ncop for t in range(2, ncop + 1)]
        lst.append((u, None))
        for q in sorted(inserts, reverse=True):
            lst.insert(q + 1, (u, None))
        added += ncop * (2 if u.imag != 0 else 1)
    return _expand([v for v, _ in lst]), added


def _units_in_order(ordered: np.ndarray) -> list[complex]:
    """Units of an already ordered list (pairs adjacent, Im > 0 member first)."""
    ordered = np.asarray(ordered, dtype=complex)
    out = []
    i = 0
    while i < ordered.size:
        z = ordered[i]
        out.append(z)
        if z.imag != 0:
            if i + 1 >= ordered.size or ordered[i + 1] != np.conj(z) or z.imag < 0:
                raise ValueError("conjugate pair not adjacent (Im > 0 first)")
            i += 2
        else:
            i += 1
    return out


# ----------------------------------------------------------------------------
# The polynomial and its application (Eq. (2.1), Section 2 footnote 2)
# ----------------------------------------------------------------------------

@dataclass
class Poly:
    """GMRES polynomial in factored form; ``roots`` in application order."""

    roots: np.ndarray  # complex, pairs adjacent (Im > 0 first)
    degree: int = 0  # GMRES degree actually reached (<= requested d)
    added: int = 0  # roots added for stability
    breakdown: bool = False
    H: np.ndarray | None = None
    inner: "Poly | None" = None  # for a double polynomial: pi_1 (tau = 1 - pi_1)
    info: dict = field(default_factory=dict)


def build_poly(op: Callable[[np.ndarray], np.ndarray], b: np.ndarray, d: int, c: Counters,
               add_roots: bool = True) -> Poly:
    """Section 2 box, steps 1(a)-(c), then the Section 7 box (added roots)."""
    V, H, steps, brk = gmres_arnoldi(op, b, d, c)
    theta = harmonic_ritz(H, breakdown=brk)
    ordered = modified_leja(theta)
    added = 0
    if add_roots:
        ordered, added = add_stability_roots(ordered)
    return Poly(roots=ordered, degree=steps, added=added, breakdown=brk, H=H)


def build_poly_two(op: Callable[[np.ndarray], np.ndarray], b1: np.ndarray, b2: np.ndarray, d: int, c: Counters,
                   add_roots: bool = True) -> Poly:
    """Polynomial determined by two starting vectors (Section 5 box): one GMRES(d)
    cycle on blockdiag(A, A) from [b1; b2] with ||b1|| = ||b2|| = 1/sqrt(2), then
    the roots as in the Section 2 box (and the Section 7 box)."""
    n = b1.size
    bhat = np.concatenate([b1 / (np.sqrt(2.0) * np.linalg.norm(b1)), b2 / (np.sqrt(2.0) * np.linalg.norm(b2))])

    def op2(x: np.ndarray) -> np.ndarray:
        return np.concatenate([op(x[:n]), op(x[n:])])

    return build_poly(op2, bhat, d, c, add_roots=add_roots)


def apply_poly(op: Callable[[np.ndarray], np.ndarray], roots: np.ndarray, x: np.ndarray,
               c: Counters | None = None) -> tuple[np.ndarray, np.ndarray]:
    """pi(A)x = prod_i (I - A/theta_i) x in the listed order (Eq. (2.1)).

    A real root: p <- p - A p/theta.  A conjugate pair (a +- ib), in real
    arithmetic: (I - A/theta)(I - A/conj(theta)) = I - (2a/|theta|^2) A + A^2/|theta|^2.
    Also returns the running sum r = sum_i A p_{i-1}/theta_i, which equals
    A phi(A) x = x - pi(A) x (Section 2 footnote 2) without the cancellation.
    """
    roots = np.asarray(roots, dtype=complex)
    p = np.array(x, dtype=np.float64, copy=True)
    r = np.zeros_like(p)
    i = 0
    while i < roots.size:
        th = roots[i]
        if th.imag == 0:
            t = op(p)
            p = p - t / th.real
            r = r + t / th.real
            i += 1
            nv = 2
        else:
            m2 = th.real**2 + th.imag**2
            t = op(p)
            s = op(t)
            p = p - (2 * th.real / m2) * t + s / m2
            r = r + (2 * th.real / m2) * t - s / m2
            i += 2
            nv = 4
        if c is not None:
            c.vops += nv
    return p, r


def poly_eval(roots: np.ndarray, z: np.ndarray | complex) -> np.ndarray:
    """Scalar pi(z) = prod (1 - z/theta_i) (Eq. (2.1))."""
    z = np.asarray(z, dtype=complex)
    out = np.ones_like(z)
    for th in np.asarray(roots, dtype=complex):
        out = out * (1 - z / th)
    return out


def build_double_poly(op: Callable[[np.ndarray], np.ndarray], b: np.ndarray, d1: int, d2: int,
                      c: Counters, add_roots: bool = True) -> Poly:
    """Double polynomial preconditioning (Section 8).

    pi_1 = GMRES(d1) polynomial of A from b; tau(z) = 1 - pi_1(z), applied as the
    running sum of pi_1's factors; pi_2 = GMRES(d2) polynomial of tau(A), also
    from b (the paper does not name pi_2's start vector; reading: the same b).
    Arnoldi then runs on pi_2(tau(A)).  The Section 7 rule is applied to both
    polynomials' roots (the paper applies it to pi_1 in Example 9 and leaves the
    question open for pi_2).
    """
    p1 = build_poly(op, b, d1, c, add_roots=add_roots)

    def tau(u: np.ndarray) -> np.ndarray:
        return apply_poly(op, p1.roots, u, c)[1]

    p2 = build_poly(tau, b, d2, c, add_roots=add_roots)
    p2.inner = p1
    return p2


def make_operator(op: Callable[[np.ndarray], np.ndarray], poly: Poly | None, c: Counters):
    """x -> pi(A)x, pi_2(tau(A))x for a double polynomial, or A x when poly is None."""
    if poly is None:
        return op
    if poly.inner is None:
        return lambda x: apply_poly(op, poly.roots, x, c)[0]
    inner = poly.inner

    def tau(u):
        return apply_poly(op, inner.roots, u, c)[1]

    return lambda x: apply_poly(tau, poly.roots, x, c)[0]


# ----------------------------------------------------------------------------
# Thick-restarted Arnoldi(m, k) with exact shifts (Section 2 box step 2; Section 4)
# ----------------------------------------------------------------------------

def ritz_order(nu: np.ndarray, target_point: float) -> np.ndarray:
    """Indices of Ritz values by increasing |target_point - nu| (Section 4).

    Ties (paper silent): larger Re first, then Im > 0 first, which keeps each
    conjugate pair adjacent with its Im > 0 member first.
    """
    return np.array(sorted(range(nu.size),
                           key=lambda i: (abs(target_point - nu[i]), -nu[i].real, -nu[i].imag)),
                    dtype=int)


@dataclass
class EigResult:
    lam: np.ndarray  # complex eigenvalue estimates mu_j, sorted by target
    X: np.ndarray  # n x nout real: real vector, or (Re x, Im x) for a pair
    resid: np.ndarray  # ||A x - mu x|| / ||A||_1 per slot
    converged: bool
    cycles: int
    counters: Counters
    ritz: np.ndarray  # Ritz values of the operator for the returned slots
    history: list = field(default_factory=list)  # max relative residual per cycle


def _target_sort(lam: np.ndarray, target: str) -> np.ndarray:
    if target == "SR":
        key = lambda i: (lam[i].real, abs(lam[i].imag), -lam[i].imag)  # noqa: E731
    else:
        key = lambda i: (abs(lam[i]), lam[i].real, -lam[i].imag)  # noqa: E731
    return np.array(sorted(range(lam.size), key=key), dtype=int)


def harmonic_restart_matrix(H: np.ndarray, m: int, tau: float) -> tuple[np.ndarray, np.ndarray]:
    """Harmonic Ritz values of the Arnoldi relation B V_m = V_{m+1} H (H is
    (m+1) x m) with respect to the target tau (Section 4's restart kept
    harmonic Ritz vectors in the harmonic Arnoldi variant of Example 2; Morgan
    and Zeng's harmonic restarted Arnoldi).

    (theta, V_m g) is a harmonic Ritz pair when (B - tau) V_m g - (theta - tau) V_m g
    is orthogonal to (B - tau) V_m.  With M = H_m - tau I, h = h_{m+1,m} and
    f = M^{-T} e_m this is the eigenproblem of K = H_m + h^2 f e_m^T.  Returns
    (K, c) with c = [-h f; 1]: every harmonic residual is a multiple of V_{m+1} c.
    """
    Hm = H[:m, :m]
    h = H[m, m - 1]
    em = np.zeros(m)
    em[-1] = 1.0
    f = np.linalg.solve((Hm - tau * np.eye(m)).T, em)
    K = Hm + h * h * np.outer(f, em)
    return K, np.concatenate([-h * f, [1.0]])


def thick_restart(V: np.ndarray, H: np.ndarray, m: int, Q: np.ndarray,
                  cvec: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """The restarted basis V_{kk+1} and its (m+1) x m Hessenberg array (leading
    (kk+1) x kk block filled) from B V_m = V_{m+1} H and the orthonormal m x kk
    coefficients Q of the kept vectors (Section 4).

    Ritz restart (cvec None): V_kk = V_m Q, v_{kk+1} = v_{m+1},
    H_kk = [Q^T H_m Q ; h_{m+1,m} e_m^T Q].
    Harmonic restart: P = [[Q; 0], p] with p the residual direction cvec
    orthogonalised against [Q; 0] (twice) and normalised; V_{kk+1} = V_{m+1} P,
    H_kk = P^T H Q.  Both keep B V_kk = V_{kk+1} H_kk.
    """
    kk = Q.shape[1]
    Hn = np.zeros((m + 1, m))
    if cvec is None:
        Vk = np.column_stack([V[:, :m] @ Q, V[:, m]])
        Hn[:kk, :kk] = Q.T @ H[:m, :m] @ Q
        Hn[kk, :kk] = H[m, m - 1] * Q[m - 1, :]
        return Vk, Hn
    P = np.zeros((m + 1, kk + 1))
    P[:m, :kk] = Q
    p = np.array(cvec, dtype=float)
    for _ in range(2):
        p = p - P[:, :kk] @ (P[:, :kk].T @ p)
    P[:, kk] = p / np.linalg.norm(p)
    Hn[:kk + 1, :kk] = P.T @ (H @ Q)
    return V[:, :m + 1] @ P, Hn


def eigs(A: sp.csr_matrix, op: Callable[[np.ndarray], np.ndarray], nev: int, m: int, k: int,
         rtol: float, v0: np.ndarray, c: Counters, target_point: float = 1.0,
         target: str = "SM", max_cycles: int = 2000, sigma: float = 0.0,
         log: Callable[[int, float], None] | None = None, restart: str = "ritz",
         scale: np.ndarray | None = None) -> EigResult:
    """Thick-restarted Arnoldi(m, k) on ``op`` (Section 2 box step 2; Section 4).

    * Build V_{m+1}, H_{m+1,m} with CGS2 (one reorthogonalisation pass).
    * Ritz values nu of H_m ordered by |1 - nu| (``target_point`` = 1 for pi(A),
      0 for plain Arnoldi on A, Section 4).
    * Convergence on A: unit Ritz vectors y_j = V_m s_j, Rayleigh quotients
      mu_j = y_j^* A y_j, converged when ||A y_j - mu_j y_j|| <= rtol*||A||_1 for
      the nev wanted (extended by one when the boundary splits a conjugate
      pair).  The paper writes theta_j in the residual; it means mu_j (reading).
    * Restart: keep the k Ritz values nearest the target (k - 1 when the boundary
      would split a conjugate pair, Section 4 footnote), orthonormal basis Q_k of
      the real and imaginary parts of their Ritz vectors (Morgan's thick
      restart), V_k = V_m Q_k, v_{k+1} = v_{m+1},
      H_k = [Q_k^T H_m Q_k ; h_{m+1,m} e_m^T Q_k].
    ``sigma`` is the shift of ``op``'s matrix; Rayleigh quotients use A itself.
    ``log`` (optional) is called as log(cycle, max relative residual) after
    each convergence test; it does not affect the arithmetic.
    ``scale`` (balancing, see ``balance``): ``op`` acts on S = D^-1 A D with
    D = diag(scale); each Ritz vector y of the operator is mapped to x = D y
    before the test on A, which stays on A itself.
    ``restart="harmonic"``: the harmonic Arnoldi variant (Example 2): harmonic
    Ritz values (w.r.t. ``target_point``) and vectors replace the Ritz ones in
    the ordering, the convergence test and the restart, which keeps
    V_{k+1} = V_{m+1} P with P = orth([Q_k; 0], c) and H_k = P^T H Q_k (see
    ``harmonic_restart_matrix``).
    """
    if restart not in ("ritz", "harmonic"):
        raise ValueError("restart must be 'ritz' or 'harmonic'")
    n = v0.size
    nA = norm1(A)
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = v0 / np.linalg.norm(v0)
    c.dots += 1
    c.vops += 2
    j0 = 0
    hist = []
    for cycle in range(1, max_cycles + 1):
        for j in range(j0, m):
            w = op(V[:, j])
            w, h = cgs2(V[:, : j + 1], w, c)
            H[: j + 1, j] = h
            hn = np.linalg.norm(w)
            c.dots += 1
            c.vops += 2
            H[j + 1, j] = hn
            V[:, j + 1] = w / hn
        Hm = H[:m, :m]
        if restart == "harmonic":
            K, cvec = harmonic_restart_matrix(H, m, target_point)
            nu, S = np.linalg.eig(K)
        else:
            nu, S = np.linalg.eig(Hm)
        order = ritz_order(nu, target_point)
        nw = nev + (1 if nu[order[nev - 1]].imag > 0 else 0)
        want = order[:nw]
        lam = np.zeros(nw, dtype=complex)
        res = np.zeros(nw)
        X = np.zeros((n, nw))
        slot = 0
        while slot < nw:
            i = want[slot]
            y = V[:, :m] @ S[:, i]
            if scale is not None:
                y = scale * y
            y = y / np.linalg.norm(y)
            Ay = A @ y
            c.mvps += 1 if nu[i].imag == 0 else 2
            mu = np.vdot(y, Ay)
            r = np.linalg.norm(Ay - mu * y) / nA
            c.vops += 4 * m
            if nu[i].imag == 0:
                lam[slot] = mu.real
                res[slot] = r
                X[:, slot] = y.real
                slot += 1
            else:
                lam[slot], lam[slot + 1] = mu, np.conj(mu)
                res[slot] = res[slot + 1] = r
                X[:, slot], X[:, slot + 1] = y.real, y.imag
                slot += 2
        hist.append(float(res.max()))
        if log is not None:
            log(cycle, float(res.max()))
        if np.all(res <= rtol):
            srt = _target_sort(lam, target)
            return EigResult(lam[srt], X[:, srt], res[srt], True, cycle, c, nu[want][srt], hist)
        kk = k - 1 if nu[order[k - 1]].imag > 0 else k
        cols = []
        for i in order[:kk]:
            if nu[i].imag == 0:
                cols.append(S[:, i].real)
            elif nu[i].imag > 0:
                cols.append(S[:, i].real)
                cols.append(S[:, i].imag)
        Q, _ = np.linalg.qr(np.stack(cols, axis=1))
        Vk, Hn = thick_restart(V, H, m, Q, cvec if restart == "harmonic" else None)
        V[:, :kk + 1] = Vk
        c.vops += (m + 1) * (kk + 1) if restart == "harmonic" else m * kk
        H = Hn
        j0 = kk
    srt = _target_sort(lam, target)
    return EigResult(lam[srt], X[:, srt], res[srt], False, max_cycles, c, nu[want][srt], hist)


# ----------------------------------------------------------------------------
# Balancing: a diagonal similarity (not in the paper; an opt-in transformation)
# ----------------------------------------------------------------------------

def balance(A: sp.csr_matrix, max_log_range: float = 600.0) -> tuple[np.ndarray, sp.csr_matrix]:
    """The diagonal similarity S = D^-1 A D that makes A symmetric, when one exists.

    Not part of the paper's method: a problem transformation for the strongly
    non-normal convection-diffusion operators of Section 4, whose eigenvalue
    condition numbers grow like e^(beta/2).  S symmetric means
    a_ij d_j / d_i = a_ji d_i / d_j for every off-diagonal pair, i.e.
    d_j / d_i = sqrt(a_ji / a_ij): this needs a_ij and a_ji nonzero together and
    of the same sign, and the ratios multiplied around every cycle of the
    graph to give 1.  D is found by walking the graph breadth first from each
    component's first row (log d_root = 0), in log form, then every edge is
    checked.  Returns (d, S) with d = exp(log d - max log d) (largest entry 1);
    ValueError when no such D exists or its range exceeds e^max_log_range.
    """
    A = sp.csr_matrix(A)
    n = A.shape[0]
    At = sp.csr_matrix(A.T)
    logd = np.zeros(n)
    seen = np.zeros(n, dtype=bool)
    for root in range(n):
        if seen[root]:
            continue
        seen[root] = True
        queue = [root]
        head = 0
        while head < len(queue):
            i = queue[head]
            head += 1
            cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
            vals = A.data[A.indptr[i]:A.indptr[i + 1]]
            for j, aij in zip(cols, vals):
                if j == i or aij == 0.0 or seen[j]:
                    continue
                aji = A[j, i]
                if aji == 0.0 or (aji > 0) != (aij > 0):
                    raise ValueError(f"balance: entries ({i},{j}) and ({j},{i}) are not nonzero with one sign")
                logd[j] = logd[i] + 0.5 * (np.log(abs(aji)) - np.log(abs(aij)))
                seen[j] = True
                queue.append(j)
    if logd.max() - logd.min() > max_log_range:
        raise ValueError("balance: the scaling range exceeds e^%g" % max_log_range)
    logd = logd - logd.max()
    d = np.exp(logd)
    coo = A.tocoo()
    S = sp.csr_matrix((coo.data * np.exp(logd[coo.col] - logd[coo.row]), (coo.row, coo.col)), shape=A.shape)
    S.sort_indices()
    asym = abs(S - S.T)
    if asym.nnz and asym.max() > 1e-12 * abs(S).max():
        raise ValueError("balance: no diagonal similarity makes A symmetric (cycle condition fails)")
    return d, S


# ----------------------------------------------------------------------------
# Damped polynomials (Section 6; the heuristic of the Section 6.3 box)
# ----------------------------------------------------------------------------

def ideal_order(mu: np.ndarray, nev: int, k: int) -> bool:
    """Ideal Order Condition (Section 6.3 box, step 4) on Rayleigh quotients mu_1..mu_k
    listed in the Ritz order: |mu_1| <= ... <= |mu_nev| < min_{nev < j <= k} |mu_j|."""
    a = np.abs(np.asarray(mu)[:k])
    nondecreasing = all(a[i] <= a[i + 1] for i in range(nev - 1))
    return bool(nondecreasing and a[nev - 1] < a[nev:k].min())


def first_cycle_rayleigh(A: sp.csr_matrix, op: Callable[[np.ndarray], np.ndarray], b: np.ndarray, m: int,
                         k: int, c: Counters, sigma: float = 0.0) -> np.ndarray:
    """Steps 1-3 of the Section 6.3 box: one Arnoldi(m, k) cycle on op = pi(A) from b
    (CGS2 as in Section 4), Ritz values of H_m ordered by |1 - nu|, and the Rayleigh
    quotients mu_j = y_j^* A y_j of the unit Ritz vectors for the first k of them,
    returned for the shifted operator (mu_j - sigma)."""
    n = b.size
    V = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = b / np.linalg.norm(b)
    for j in range(m):
        w, h = cgs2(V[:, : j + 1], op(V[:, j]), c)
        H[: j + 1, j] = h
        hn = np.linalg.norm(w)
        H[j + 1, j] = hn
        V[:, j + 1] = w / hn
    nu, S = np.linalg.eig(H[:m, :m])
    order = ritz_order(nu, 1.0)
    mu = np.zeros(k, dtype=complex)
    for t, i in enumerate(order[:k]):
        y = V[:, :m] @ S[:, i]
        y = y / np.linalg.norm(y)
        mu[t] = np.vdot(y, A @ y) - sigma
    return mu


@dataclass
class DampResult:
    poly: Poly
    degree: int  # degree finally used (before added roots)
    damped: bool  # the GMRES start vector was replaced by A b
    ideal: bool  # the Ideal Order Condition holds for the returned polynomial
    trials: list  # (degree, damped, condition) per attempt


def damped_poly(A: sp.csr_matrix, sigma: float, b: np.ndarray, d: int, m: int, k: int, nev: int,
                c: Counters, add_roots: bool = True) -> DampResult:
    """Heuristic for damping b and adjusting d (Section 6.3 box).

    1-3. GMRES(d) polynomial from b; one Arnoldi(m, k) cycle on pi(A) from b; Rayleigh
         quotients for A of the k Ritz vectors nearest 1.
    4.   Ideal Order Condition.
    5.   If it fails: a fresh polynomial from A b (one power step damps the components
         of b along the small eigenvalues, Section 6.1); if that fails too, halve d
         (keeping A b) until it holds or d = 1.
    Readings: the Arnoldi cycle always starts from the original b; with a shift
    (smallest-real-part targets on A - sigma I) the polynomial, the damping product and
    the magnitudes all refer to the shifted operator.
    """
    op = Operator(A, sigma, c)
    start, damped, trials = b, False, []
    while True:
        P = build_poly(op, start, d, c, add_roots=add_roots)
        mu = first_cycle_rayleigh(A, make_operator(op, P, c), b, m, k, c, sigma)
        ok = ideal_order(mu, nev, k)
        trials.append((d, damped, ok))
        if ok or (damped and d == 1):
            return DampResult(P, d, damped, ok, trials)
        if not damped:
            start, damped = op(b), True
        else:
            d = max(1, d // 2)
