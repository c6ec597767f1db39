"""Mixed precision: FP32 apply and basis, FP64 Rayleigh-Ritz refinement on A.

* FP32 apply vs the oracle's FP64 apply of the same roots: the forward-error
  bound of the product form with u = 2^-24 (FP32 storage and accumulation).
* FP32 Arnoldi + FP64 refinement vs the FP64 oracle on the same inputs:
  residuals <= 1e-8 ||A||_1 recomputed on the CPU from the returned FP64
  vectors, eigenvalues within the kappa-gated first-order bound.
"""
import numpy as np
import pytest

import oracle as O
from paper_1806_08020_gb300 import inputs
from test_gpu_eigs import cpu_residuals, eig_condition, oracle_solve

pytestmark = pytest.mark.gpu

U32 = 2.0**-24


def _bound32(A, sigma, roots, x):
    Ainf = float(abs(A).sum(axis=1).max()) + abs(sigma)
    op = O.Operator(A, sigma, O.Counters())
    p = x.copy()
    tot = 0.0
    i = 0
    while i < roots.size:
        th = roots[i]
        if th.imag == 0:
            tot += (1 + Ainf / abs(th)) * np.abs(p).max()
            p = p - op(p) / th.real
            i += 1
        else:
            m2 = abs(th) ** 2
            t = op(p)
            tot += (1 + 2 * abs(th.real) * Ainf / m2 + Ainf**2 / m2) * np.abs(p).max() + np.abs(t).max()
            p = p - (2 * th.real / m2) * t + op(t) / m2
            i += 2
    return 16 * U32 * tot


@pytest.mark.parametrize("case", ["cd", "banded"])
def test_fp32_apply_matches_oracle(case):
    from paper_1806_08020_gb300 import pp
    Acsr = inputs.convection_diffusion_2d(40, 20.0) if case == "cd" else inputs.banded_random(5000, 5, 2)
    A = O.to_scipy(Acsr)
    sigma = O.gershgorin_shift(A)
    P = O.build_poly(O.Operator(A, sigma, O.Counters()), inputs.start_vector(Acsr.n, 1, 0), 12, O.Counters())
    ctx = pp.pp_create(Acsr, precision=pp.PP_FP32)
    poly = pp.pp_poly_from_roots(ctx, P.roots)
    x = inputs.start_vector(Acsr.n, 2, 0)
    y = pp.pp_apply_host(poly, x)
    ref, _ = O.apply_poly(O.Operator(A, sigma, O.Counters()), P.roots, x)
    assert np.abs(y - ref).max() <= _bound32(A, sigma, P.roots, x)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("case", ["single", "double", "banded"])
def test_mixed_eigs_match_fp64_oracle(case, precision):
    """FP32 or BF16 basis (FP32 apply), FP64 test, refinement and continuation:
    converged pairs meet the FP64 residual bound and match the oracle's."""
    from paper_1806_08020_gb300 import pp
    if case == "single":
        Acsr, d, d2, nev, m, k = inputs.convection_diffusion_2d(60, 20.0), 10, None, 8, 30, 13
    elif case == "double":
        Acsr, d, d2, nev, m, k = inputs.convection_diffusion_2d(60, 20.0), 4, 5, 8, 30, 13
    else:
        Acsr, d, d2, nev, m, k = inputs.banded_random(2000, 4, 2), 5, None, 6, 30, 11
    A, P, R = oracle_solve(Acsr, d, nev, m, k, 41, d2=d2)
    ctx = pp.pp_create(Acsr, precision=pp.PP_FP32 if precision == "fp32" else pp.PP_FP32_BF16)
    b = inputs.start_vector(Acsr.n, 41, 0)
    v0 = inputs.start_vector(Acsr.n, 41, 1)
    poly = pp.pp_build_poly2(ctx, d, d2, b) if d2 else pp.pp_build_poly(ctx, d, b)
    res = pp.pp_eigs(ctx, poly, nev, m, k, 1e-8, v0)
    assert res.status == 0
    assert np.all(res.resid <= 1e-8)
    rc = cpu_residuals(A, res.lam, res.X)
    assert np.all(rc <= 1.01e-8), rc
    w, kap = eig_condition(Acsr.to_dense())
    nA = O.norm1(A)
    for j, lam in enumerate(R.lam):
        dist = np.abs(res.lam - lam)
        i = int(np.argmin(dist))
        kj = kap[np.argmin(np.abs(w - lam))]
        bound = 10 * kj * (res.resid[i] + R.resid[j]) * nA
        assert dist[i] <= bound + 1e-12 * abs(lam), (j, lam, res.lam[i], bound)


def test_bf16_basis_rejected_by_batched_engines():
    from paper_1806_08020_gb300 import pp
    A = inputs.convection_diffusion_2d(20, 5.0)
    with pytest.raises(pp.PPError):
        pp.pp_batch_create([A], precision=pp.PP_FP32_BF16)
    with pytest.raises(pp.PPError):
        pp.pp_server_create(precision=pp.PP_FP32_BF16)
