"""The library's host analysis of A (pp_csr_info: what pp_create computes before
any device work) against the oracle and against values fixed outside it.

* ||A||_1 is the norm of the convergence test (Section 4: residual below
  1e-8 ||A||); sigma is the shift of the smallest-real-part target (Section 2,
  first footnote).
* Small matrices take one row range; above 2^18 entries the scan runs on host
  threads over 16 row ranges, and with columns scattered over the whole matrix
  it falls back to one pass in row order: each case is covered.
* The scan refuses what pp_create refuses (PP_EINVAL).

No device is needed.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_1806_08020_gb300 import inputs, pp
from test_oracle_norms import HAND, HAND_NORM1, HAND_SIGMA


def _csr(M) -> inputs.CSR:
    M = sp.csr_matrix(M)
    M.sort_indices()
    return inputs.CSR(M.shape[0], M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))


def test_hand_example():
    assert pp.pp_csr_info(_csr(HAND)) == (HAND_NORM1, HAND_SIGMA)


@pytest.mark.parametrize("N,beta", [(50, 20.0), (300, 100.0)])
def test_convection_diffusion_closed_form(N, beta):
    """8/h^2 and sigma = 0 exactly (cell Peclet <= 1); N = 300 has 448,800 entries (threaded scan)."""
    A = inputs.convection_diffusion_2d(N, beta)
    h = 1.0 / (N + 1)
    norm1, sigma = pp.pp_csr_info(A)
    assert norm1 == pytest.approx(8.0 / h**2, rel=1e-14)
    assert sigma == 0.0
    assert norm1 == pytest.approx(O.norm1(O.to_scipy(A)), rel=1e-15)


@pytest.mark.parametrize("n,w", [(500, 5), (20000, 10)])
def test_banded_stream_matrix_matches_oracle(n, w):
    """The request stream's banded matrices: a negative Gershgorin shift; n = 20,000 with
    half-band 10 has 419,890 entries (threaded scan)."""
    A = inputs.banded_random(n, w, 20181806 + n)
    norm1, sigma = pp.pp_csr_info(A)
    S = O.to_scipy(A)
    assert norm1 == pytest.approx(O.norm1(S), rel=1e-14)
    want = O.gershgorin_shift(S)
    assert want < 0
    assert sigma == pytest.approx(want, rel=1e-13)


def test_scattered_columns_match_oracle():
    """Random columns over the whole matrix (every row range spans all columns): the
    one-pass fallback, 300,000 entries."""
    rng = np.random.default_rng(7)
    n = 100_000
    rows = np.repeat(np.arange(n), 3)
    cols = rng.integers(0, n, size=rows.size)
    vals = rng.standard_normal(rows.size)
    S = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    S.sum_duplicates()
    S = S + sp.identity(n, format="csr") * 5.0
    A = _csr(S)
    norm1, sigma = pp.pp_csr_info(A)
    assert norm1 == pytest.approx(O.norm1(S), rel=1e-14)
    assert sigma == pytest.approx(O.gershgorin_shift(S), rel=1e-13)


def test_repeatable():
    A = inputs.convection_diffusion_2d(200, 1000.0)  # cell Peclet 2.5 > 1: sigma < 0
    a = pp.pp_csr_info(A)
    assert a[1] < 0
    for _ in range(3):
        assert pp.pp_csr_info(A) == a


def _refused(A):
    with pytest.raises(pp.PPError) as e:
        pp.pp_csr_info(A)
    assert e.value.status == pp.PP_EINVAL


def test_refusals():
    base = inputs.convection_diffusion_2d(120, 10.0)  # 71,520 entries
    big = inputs.convection_diffusion_2d(300, 10.0)  # threaded scan

    for A in (base, big):
        rp = A.rowptr.copy()
        rp[A.n // 2] = rp[A.n // 2 + 1] + 1  # not monotone
        _refused(inputs.CSR(A.n, rp, A.colind, A.vals))
        for bad in (-1, A.n):
            ci = A.colind.copy()
            ci[len(ci) * 3 // 4] = bad
            _refused(inputs.CSR(A.n, A.rowptr, ci, A.vals))
        for bad in (np.nan, np.inf):
            va = A.vals.copy()
            va[len(va) // 3] = bad
            _refused(inputs.CSR(A.n, A.rowptr, A.colind, va))
        rp = A.rowptr.copy()
        rp[0] = 1
        _refused(inputs.CSR(A.n, rp, A.colind, A.vals))


# ---- the balancing of pp_create (pp_opts.balance) on the host: pp_csr_balance ----

@pytest.mark.parametrize("N,beta", [(10, 15.0), (50, 20.0), (300, 60.0)])
def test_balance_closed_form_and_oracle(N, beta):
    """log d = (x index - (N - 1)) log rho with rho = sqrt((1 + P)/(1 - P)), P = beta h / 2
    (the closed form the oracle is pinned to), and the oracle's d to rounding; N = 300 has
    448,800 entries (the threaded scan in front of it)."""
    A = inputs.convection_diffusion_2d(N, beta)
    d, rng = pp.pp_csr_balance(A)
    h = 1.0 / (N + 1)
    P = beta * h / 2
    lrho = 0.5 * np.log((1 + P) / (1 - P))
    ix = np.arange(N * N) % N
    assert np.allclose(np.log(d), (ix - (N - 1)) * lrho, rtol=0, atol=1e-11 * N)
    assert d.max() == 1.0
    assert rng == pytest.approx((N - 1) * lrho, rel=1e-10)
    if N <= 50:
        dd, _ = O.balance(O.to_scipy(A))
        assert np.allclose(d, dd, rtol=1e-12, atol=0)


def test_balance_path_and_refusals():
    # a path (no cycle) is always balanced: d = (1, sqrt 2, sqrt 2) up to scale (as the oracle's pin)
    P = _csr(np.array([[2.0, 1.0, 0.0], [2.0, 2.0, 3.0], [0.0, 3.0, 2.0]]))
    d, _ = pp.pp_csr_balance(P)
    assert np.allclose(d / d[0], [1.0, np.sqrt(2.0), np.sqrt(2.0)])
    # ratios around 0 -> 1 -> 2 -> 0 that do not multiply to 1; opposite signs (P = beta h / 2 > 1)
    for A in (_csr(np.array([[2.0, 1.0, 2.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]])),
              inputs.convection_diffusion_2d(10, 30.0)):
        with pytest.raises(pp.PPError) as e:
            pp.pp_csr_balance(A)
        assert e.value.status == pp.PP_EINVAL
