"""GPU parity of the polynomial build (Section 2 box) and thick-restarted
Arnoldi(m, k) on pi(A) (Section 4) against the oracle, through the C-ABI.

Criteria (derived in the design notes):
* roots: same count, each within 1e-8 relative of an oracle root (GMRES on the
  GPU and on the host differ by rounding only);
* eigenvalues: |lam_gpu - lam_ora| <= 10 kappa_j (res_gpu + res_ora) ||A||_1,
  the first-order perturbation bound, and additionally <= 1e-8 |lam| where that
  bound is below 1e-10 |lam| (well-conditioned eigenvalues);
* residuals: every returned pair has ||A x - lam x|| / ||A||_1 <= rtol, both as
  reported by the library and recomputed here on the CPU from the returned x.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from oracle.ppa import make_operator
from paper_1806_08020_gb300 import inputs

pytestmark = pytest.mark.gpu


def eig_condition(M):
    w, vl, vr = sla.eig(M, left=True, right=True)
    kap = np.linalg.norm(vl, axis=0) * np.linalg.norm(vr, axis=0) / np.abs(np.sum(vl.conj() * vr, axis=0))
    return w, kap


def cpu_residuals(A, lam, X):
    """||A x - lam x|| / ||A||_1 per slot from the returned vectors (pairs: Re, Im columns)."""
    nA = O.norm1(A)
    out = np.zeros(lam.size)
    j = 0
    while j < lam.size:
        if lam[j].imag == 0:
            x = X[:, j]
            out[j] = np.linalg.norm(A @ x - lam[j].real * x) / nA
            j += 1
        else:
            x = X[:, j] + 1j * X[:, j + 1]
            r = np.linalg.norm(A @ x - lam[j] * x) / nA
            out[j] = out[j + 1] = r
            j += 2
    return out


def oracle_solve(Acsr, d, nev, m, k, seed, target="SR", rtol=1e-8, d2=None, restart="ritz"):
    A = O.to_scipy(Acsr)
    c = O.Counters()
    sigma = O.gershgorin_shift(A) if target == "SR" else 0.0
    op = O.Operator(A, sigma, c)
    n = Acsr.n
    b = inputs.start_vector(n, seed, 0)
    v0 = inputs.start_vector(n, seed, 1)
    if d == 0:
        P = None
    elif d2:
        P = O.build_double_poly(op, b, d, d2, c)
    else:
        P = O.build_poly(op, b, d, c)
    R = O.eigs(A, make_operator(op, P, c), nev, m, k, rtol, v0, c, target_point=1.0 if d else 0.0,
               target=target, sigma=sigma, restart=restart)
    return A, P, R


def gpu_solve(Acsr, d, nev, m, k, seed, target="SR", rtol=1e-8, d2=None, **opts):
    from paper_1806_08020_gb300 import pp
    n = Acsr.n
    ctx = pp.pp_create(Acsr, target=pp.PP_TARGET_SR if target == "SR" else pp.PP_TARGET_SM, **opts)
    b = inputs.start_vector(n, seed, 0)
    v0 = inputs.start_vector(n, seed, 1)
    if d == 0:
        poly = None
    elif d2:
        poly = pp.pp_build_poly2(ctx, d, d2, b)
    else:
        poly = pp.pp_build_poly(ctx, d, b)
    res = pp.pp_eigs(ctx, poly, nev, m, k, rtol, v0)
    return ctx, poly, res


def check_eigs(A, R_ora, res, kap_fn=None, rtol=1e-8):
    assert res.status == 0 and R_ora.converged
    assert res.lam.size == R_ora.lam.size
    assert np.all(res.resid <= rtol)
    rc = cpu_residuals(A, res.lam, res.X)
    assert np.all(rc <= rtol * 1.01), rc
    nA = O.norm1(A)
    for j, lam in enumerate(R_ora.lam):
        dist = np.abs(res.lam - lam)
        i = int(np.argmin(dist))
        kap = kap_fn(lam) if kap_fn else 1.0
        bound = 10 * kap * (res.resid[i] + R_ora.resid[j]) * nA
        assert dist[i] <= bound + 1e-12 * abs(lam), (j, lam, res.lam[i], bound)
        if bound < 1e-10 * abs(lam):
            assert dist[i] <= 1e-8 * abs(lam)


def test_build_poly_roots_match_oracle():
    from paper_1806_08020_gb300 import pp
    cfg = inputs.plain_small()
    A = O.to_scipy(cfg["A"])
    b = inputs.start_vector(2500, cfg["seed"], 0)
    ref = O.build_poly(O.Operator(A, 0.0, O.Counters()), b, 10, O.Counters())
    ctx = pp.pp_create(cfg["A"])
    poly = pp.pp_build_poly(ctx, 10, b)
    got = pp.pp_poly_roots(poly)
    assert got.size == ref.roots.size
    for z in ref.roots:
        assert np.min(np.abs(got - z)) <= 1e-8 * abs(z)
    # same decisions: Leja order identical on these well-separated roots
    assert np.allclose(got, ref.roots, rtol=1e-8)
    assert pp.pp_poly_info(poly) == (ref.degree, ref.added)
    c = pp.pp_poly_counts(poly)
    oc = O.Counters()
    O.build_poly(O.Operator(A, 0.0, oc), b, 10, oc)
    assert (c["mvps"], c["dots"], c["vops"]) == (oc.mvps, oc.dots, oc.vops)


def test_build_poly_gmres_optimality():
    """pi from the GPU's roots applied by the oracle equals the GMRES residual (Section 2)."""
    from paper_1806_08020_gb300 import pp
    Acsr = inputs.convection_diffusion_2d(30, 200.0)  # complex spectrum
    A = O.to_scipy(Acsr)
    sigma = O.gershgorin_shift(A)
    op = O.Operator(A, sigma, O.Counters())
    b = inputs.start_vector(Acsr.n, 3, 0)
    ctx = pp.pp_create(Acsr, add_roots=0)
    poly = pp.pp_build_poly(ctx, 12, b)
    roots = pp.pp_poly_roots(poly)
    assert np.any(roots.imag != 0)
    V, H, d, _ = O.gmres_arnoldi(op, b, 12, O.Counters())
    rhs = np.zeros(13)
    rhs[0] = np.linalg.norm(b)
    y = np.linalg.lstsq(H, rhs, rcond=None)[0]
    r = b - np.column_stack([op(V[:, j]) for j in range(12)]) @ y
    p, _ = O.apply_poly(op, roots, b)
    assert np.linalg.norm(p - r) <= 1e-8 * np.linalg.norm(b)


def test_build_poly_breakdown():
    """Diagonal matrix with 4 distinct eigenvalues: GMRES ends at step 4 (invariant subspace)."""
    from paper_1806_08020_gb300 import pp
    lam = np.repeat([1.0, 2.0, 3.0, 5.0], 25)
    ctx = pp.pp_create(inputs.diagonal(lam), target=pp.PP_TARGET_SM)
    poly = pp.pp_build_poly(ctx, 8, np.ones(100))
    assert poly.status == pp.PP_EBREAKDOWN
    assert pp.pp_poly_info(poly)[0] == 4
    assert np.allclose(np.sort(pp.pp_poly_roots(poly).real)[:4], [1, 2, 3, 5])


def test_eigs_plain_small_config():
    """n = 2500 CD (beta = 20), d = 10, Arnoldi(30, 15), nev = 10: oracle, closed form, residuals."""
    cfg = inputs.plain_small()
    A, P, R = oracle_solve(cfg["A"], 10, 10, 30, 15, cfg["seed"])
    _, _, res = gpu_solve(cfg["A"], 10, 10, 30, 15, cfg["seed"])
    M = cfg["A"].to_dense()
    w, kap = eig_condition(M)
    check_eigs(A, R, res, lambda lam: kap[np.argmin(np.abs(w - lam))])
    h = 1 / 51.0
    j = np.arange(1, 51)
    cx = (2 - 2 * np.sqrt(1 - (20 * h / 2) ** 2) * np.cos(j * np.pi / 51)) / h**2
    cy = (2 - 2 * np.cos(j * np.pi / 51)) / h**2
    closed = np.sort((cx[:, None] + cy[None, :]).ravel())[:10]
    assert np.max(np.abs(np.sort(res.lam.real) - closed) / closed) < 1e-8
    assert abs(res.stats["cycles"] - R.cycles) <= 1


@pytest.mark.parametrize("case", ["plain_arnoldi", "complex", "banded", "sm_diag", "ex7_added", "double"])
def test_eigs_variants(case):
    if case == "plain_arnoldi":
        Acsr, d, nev, m, k, tgt, d2 = inputs.convection_diffusion_2d(20, 10.0), 0, 5, 30, 12, "SR", None
    elif case == "complex":
        Acsr, d, nev, m, k, tgt, d2 = inputs.convection_diffusion_2d(12, 60.0), 6, 6, 30, 11, "SR", None
    elif case == "banded":
        Acsr, d, nev, m, k, tgt, d2 = inputs.banded_random(600, 4, 2), 5, 6, 30, 11, "SR", None
    elif case == "sm_diag":
        Acsr, d, nev, m, k, tgt, d2 = inputs.diagonal(np.arange(1, 1001.0)), 10, 8, 30, 13, "SM", None
    elif case == "ex7_added":
        Acsr, d, nev, m, k, tgt, d2 = inputs.diagonal(inputs.example7_diag()), 15, 15, 50, 20, "SM", None
    else:
        Acsr, d, nev, m, k, tgt, d2 = inputs.convection_diffusion_2d(40, 10.0), 4, 6, 30, 11, "SR", 5
    A, P, R = oracle_solve(Acsr, d, nev, m, k, 31, target=tgt, d2=d2)
    _, poly, res = gpu_solve(Acsr, d, nev, m, k, 31, target=tgt, d2=d2)
    if Acsr.n <= 2000:
        w, kap = eig_condition(Acsr.to_dense())
        kf = lambda lam: kap[np.argmin(np.abs(w - lam))]  # noqa: E731
    else:
        kf = None  # normal matrices (diagonal): kappa = 1
    check_eigs(A, R, res, kf)


def test_eigs_argument_errors():
    from paper_1806_08020_gb300 import pp
    ctx = pp.pp_create(inputs.plain_small()["A"])
    with pytest.raises(pp.PPError):
        pp.pp_eigs(ctx, None, 10, 30, 10, 1e-8)  # k <= nev
    with pytest.raises(pp.PPError):
        pp.pp_eigs(ctx, None, 3, 200, 10, 1e-8)  # m > 127
    with pytest.raises(pp.PPError):
        pp.pp_build_poly(ctx, 0, np.ones(2500))
    with pytest.raises(pp.PPError):
        pp.pp_build_poly(ctx, 5, np.zeros(2500))
    bad = inputs.CSR(3, np.array([0, 1, 2, 3]), np.array([0, 5, 2], dtype=np.int32), np.ones(3))
    with pytest.raises(pp.PPError):
        pp.pp_create(bad)
    nan = inputs.CSR(3, np.array([0, 1, 2, 3]), np.array([0, 1, 2], dtype=np.int32), np.array([1.0, np.nan, 1.0]))
    with pytest.raises(pp.PPError):
        pp.pp_create(nan)
    # a non-monotone row pointer whose middle entry points past the arrays: rejected before any entry is read
    back = inputs.CSR(3, np.array([0, 9, 1, 3]), np.array([0, 1, 2], dtype=np.int32), np.ones(3))
    with pytest.raises(pp.PPError):
        pp.pp_create(back)
    # the column-offset width follows the widest |col - row| (16 bits when every one is below 2^15)
    assert pp.pp_format_info(pp.pp_create(inputs.banded_random(40000, 3, 1), format=pp.PP_FMT_SELL))["index_bits"] == 16


def test_eigs_not_converged_status():
    from paper_1806_08020_gb300 import pp
    cfg = inputs.plain_small()
    ctx = pp.pp_create(cfg["A"], max_cycles=1)
    poly = pp.pp_build_poly(ctx, 2, inputs.start_vector(2500, 1, 0))
    res = pp.pp_eigs(ctx, poly, 10, 30, 15, 1e-12, inputs.start_vector(2500, 1, 1))
    assert res.status == pp.PP_ENOTCONV and res.stats["cycles"] == 1
    assert res.lam.size >= 10 and np.all(np.isfinite(res.resid))


def test_build_poly_on_dirty_device_memory():
    """Every device buffer the build reads must be written first: fill and free a
    large block with NaN so that new allocations start out dirty, then build."""
    import torch
    from paper_1806_08020_gb300 import pp
    junk = torch.full((64 << 20,), float("nan"), dtype=torch.float64, device="cuda")
    del junk
    torch.cuda.empty_cache()
    junk2 = torch.full((64 << 20,), 1e300, dtype=torch.float64, device="cuda")
    del junk2
    torch.cuda.empty_cache()
    Acsr = inputs.convection_diffusion_2d(40, 10.0)
    A = O.to_scipy(Acsr)
    b = inputs.start_vector(Acsr.n, 8, 0)
    ref = O.build_poly(O.Operator(A, 0.0, O.Counters()), b, 11, O.Counters())
    for _ in range(3):
        ctx = pp.pp_create(Acsr)
        got = pp.pp_poly_roots(pp.pp_build_poly(ctx, 11, b))
        assert got.size == ref.roots.size
        for z in ref.roots:
            assert np.min(np.abs(got - z)) <= 1e-8 * abs(z)


@pytest.mark.parametrize("precision", [0, 1])
def test_repeated_solves_reuse_workspace(precision):
    """Solves repeated on one context (its workspace reused from the previous
    call, a workspace of another size in between, and after pp_trim) give the
    same bits as the first."""
    from paper_1806_08020_gb300 import pp
    cfg = inputs.plain_small()
    A = cfg["A"]
    ctx = pp.pp_create(A, precision=precision)
    b, v0 = inputs.start_vector(A.n, 5, 0), inputs.start_vector(A.n, 5, 1)

    def solve(m, k):
        poly = pp.pp_build_poly(ctx, 10, b)
        return pp.pp_poly_roots(poly), pp.pp_eigs(ctx, poly, 8, m, k, 1e-8, v0)

    r0, e0 = solve(30, 15)
    runs = [solve(30, 15), solve(40, 20), solve(30, 15)]
    pp.pp_trim(ctx)
    runs.append(solve(30, 15))
    for i, (r, e) in enumerate(runs):
        if i == 1:
            assert e.status == 0
            continue
        assert np.array_equal(r, r0) and np.array_equal(e.lam, e0.lam) and np.array_equal(e.resid, e0.resid), i


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_device_start_vectors(precision):
    """Start vectors passed as device arrays (normalised on the device) give the
    solve of the same vectors passed from the host: the unit start vectors
    differ only by the rounding of ||b|| (summed in another order), so the roots
    and eigenvalues agree to a few units of rounding growth, and the device path
    is deterministic (the same bits on a second call)."""
    import torch
    from paper_1806_08020_gb300 import pp
    cfg = inputs.plain_small()
    A = cfg["A"]
    ctx = pp.pp_create(A, precision=precision)
    b, v0 = inputs.start_vector(A.n, 7, 0), inputs.start_vector(A.n, 7, 1)
    bd, vd = torch.from_numpy(b).cuda(), torch.from_numpy(v0).cuda()
    ph, pd, pd2 = pp.pp_build_poly(ctx, 10, b), pp.pp_build_poly(ctx, 10, bd), pp.pp_build_poly(ctx, 10, bd)
    rh, rd = np.sort_complex(pp.pp_poly_roots(ph)), np.sort_complex(pp.pp_poly_roots(pd))
    assert np.array_equal(rd, np.sort_complex(pp.pp_poly_roots(pd2)))
    if precision == 0:  # FP32 roots move with the O(u32) change of the start vector's rounding
        assert np.max(np.abs(rh - rd) / np.abs(rh)) < 1e-10
    eh = pp.pp_eigs(ctx, ph, 8, 30, 15, 1e-8, v0)
    ed = pp.pp_eigs(ctx, ph, 8, 30, 15, 1e-8, vd)
    assert eh.status == 0 and ed.status == 0
    # both converged to residual 1e-8 ||A||_1 on a mildly non-normal matrix
    lh, ld = np.sort_complex(eh.lam), np.sort_complex(ed.lam)
    assert np.max(np.abs(lh - ld) / np.abs(lh)) <= 1e-6
    with pytest.raises(pp.PPError):
        pp.pp_build_poly(ctx, 10, torch.zeros(A.n, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        pp.pp_build_poly(ctx, 10, bd.float())


@pytest.mark.parametrize("case", ["plain_arnoldi", "complex", "banded", "sm_diag", "double"])
def test_eigs_harmonic_restart_matches_oracle(case):
    """Harmonic restart (PP_RESTART_HARMONIC, Example 2's variant) against the
    oracle's harmonic restart: the same eigenpairs (kappa-gated values, every
    residual <= rtol on A) and the same number of cycles within one."""
    from paper_1806_08020_gb300 import pp
    if case == "plain_arnoldi":
        Acsr, d, nev, m, k, tgt, d2 = inputs.convection_diffusion_2d(20, 10.0), 0, 5, 30, 12, "SR", None
    elif case == "complex":
        Acsr, d, nev, m, k, tgt, d2 = inputs.convection_diffusion_2d(12, 60.0), 6, 6, 30, 11, "SR", None
    elif case == "banded":
        Acsr, d, nev, m, k, tgt, d2 = inputs.banded_random(600, 4, 2), 5, 6, 30, 11, "SR", None
    elif case == "sm_diag":
        Acsr, d, nev, m, k, tgt, d2 = inputs.diagonal(np.arange(1, 1001.0)), 10, 8, 30, 13, "SM", None
    else:
        Acsr, d, nev, m, k, tgt, d2 = inputs.convection_diffusion_2d(40, 10.0), 4, 6, 30, 11, "SR", 5
    A, P, R = oracle_solve(Acsr, d, nev, m, k, 31, target=tgt, d2=d2, restart="harmonic")
    _, poly, res = gpu_solve(Acsr, d, nev, m, k, 31, target=tgt, d2=d2, restart=pp.PP_RESTART_HARMONIC)
    if Acsr.n <= 2000:
        w, kap = eig_condition(Acsr.to_dense())
        kf = lambda lam: kap[np.argmin(np.abs(w - lam))]  # noqa: E731
    else:
        kf = None
    check_eigs(A, R, res, kf)
    assert abs(res.stats["cycles"] - R.cycles) <= 1, (res.stats["cycles"], R.cycles)


def test_harmonic_restart_option_errors():
    from paper_1806_08020_gb300 import pp
    A = inputs.plain_small()["A"]
    with pytest.raises(pp.PPError):
        pp.pp_create(A, restart=7)


def test_harmonic_restart_on_a_fanned_complex_spectrum():
    """Example 2's situation on a stand-in matrix: a degree-10 polynomial cannot
    damp the eigenvalues with large imaginary parts, so the wanted ones are
    interior for pi(A).  Both restarts match their oracle runs (eigenpairs and
    cycles within two), and the harmonic restart needs fewer products with A."""
    from paper_1806_08020_gb300 import pp
    Acsr = inputs.rotation_blocks(1000, 20.0, 3)
    w, kap = eig_condition(Acsr.to_dense())
    kf = lambda lam: kap[np.argmin(np.abs(w - lam))]  # noqa: E731
    mv = {}
    for rs, code in (("ritz", pp.PP_RESTART_RITZ), ("harmonic", pp.PP_RESTART_HARMONIC)):
        A, P, R = oracle_solve(Acsr, 10, 15, 50, 25, 5, target="SM", restart=rs)
        _, poly, res = gpu_solve(Acsr, 10, 15, 50, 25, 5, target="SM", restart=code, max_cycles=300)
        check_eigs(A, R, res, kf)
        assert abs(res.stats["cycles"] - R.cycles) <= 2, (rs, res.stats["cycles"], R.cycles)
        mv[rs] = res.stats["mvps"]
    assert mv["harmonic"] < mv["ritz"], mv
