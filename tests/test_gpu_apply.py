"""GPU parity of the factored polynomial apply (Eq. (2.1)) and the double
polynomial (Section 8) against the oracle, through the C-ABI.

Both sides apply the same root list to the same seeded vector, so the results
agree up to FP64 rounding order.  Tolerance: the forward error of the product
form is bounded by u times the sum over factors of |1/theta_i| ||A - sigma I||_inf
||p_{i-1}||_inf (each factor's SpMV and axpy), times a small constant for the
per-row accumulation; the bound is computed from the oracle's own intermediates.
"""
import numpy as np
import pytest

import oracle as O
from paper_1806_08020_gb300 import inputs

pytestmark = pytest.mark.gpu

U = np.finfo(np.float64).eps / 2


def _bound(A, sigma, roots, x):
    """u * 64 * sum_i (1 + |c_i| ||A||_inf) ||p_{i-1}||_inf over the factors (pairs: two passes)."""
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
    return 64 * U * tot


CASES = {
    "cd_n2500": lambda: inputs.plain_small()["A"],
    "cd_complex": lambda: inputs.convection_diffusion_2d(30, 200.0),
    "banded": lambda: inputs.banded_random(3001, 7, 1),
    "ex7": lambda: inputs.diagonal(inputs.example7_diag()),
    "ragged_n37": lambda: inputs.banded_random(37, 2, 3),
}


@pytest.mark.parametrize("fmt", ["auto", "csr"])
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("d", [1, 7, 20])
def test_apply_matches_oracle(case, d, fmt):
    from paper_1806_08020_gb300 import pp
    Acsr = CASES[case]()
    A = O.to_scipy(Acsr)
    n = Acsr.n
    sigma = O.gershgorin_shift(A)
    P = O.build_poly(O.Operator(A, sigma, O.Counters()), inputs.start_vector(n, 5, 0), min(d, n - 1),
                     O.Counters())
    ctx = pp.pp_create(Acsr, target=pp.PP_TARGET_SR,
                       format=pp.PP_FMT_CSR if fmt == "csr" else pp.PP_FMT_AUTO)
    assert pp.pp_matrix_info(ctx)[1] == sigma
    poly = pp.pp_poly_from_roots(ctx, P.roots)
    x = inputs.start_vector(n, 6, 0)
    y = pp.pp_apply_host(poly, x)
    ref, _ = O.apply_poly(O.Operator(A, sigma, O.Counters()), P.roots, x)
    err = np.abs(y - ref).max()
    assert err <= _bound(A, sigma, P.roots, x), (err, _bound(A, sigma, P.roots, x))


def test_apply_device_pointers_and_inplace():
    import torch
    from paper_1806_08020_gb300 import pp
    Acsr = inputs.plain_small()["A"]
    A = O.to_scipy(Acsr)
    P = O.build_poly(O.Operator(A, 0.0, O.Counters()), inputs.start_vector(2500, 1, 0), 10, O.Counters())
    ctx = pp.pp_create(Acsr, stream=torch.cuda.current_stream().cuda_stream)
    poly = pp.pp_poly_from_roots(ctx, P.roots)
    x = inputs.start_vector(2500, 2, 0)
    ref, _ = O.apply_poly(O.Operator(A, 0.0, O.Counters()), P.roots, x)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    pp.pp_apply(poly, xd.data_ptr(), yd.data_ptr())
    torch.cuda.synchronize()
    tol = _bound(A, 0.0, P.roots, x)
    assert np.abs(yd.cpu().numpy() - ref).max() <= tol
    assert np.array_equal(xd.cpu().numpy(), x)  # input untouched
    pp.pp_apply(poly, xd.data_ptr(), xd.data_ptr())  # in place
    torch.cuda.synchronize()
    assert np.abs(xd.cpu().numpy() - ref).max() <= tol


def test_apply_pairs_on_diagonal_exact():
    """Conjugate pairs in real arithmetic: pi(D) x = pi(lambda_i) x_i."""
    from paper_1806_08020_gb300 import pp
    lam = np.linspace(0.5, 3.0, 1000)
    roots = O.modified_leja(np.array([2.5, 1.0 + 0.5j, 1.0 - 0.5j, 0.7, 2.0 + 1.5j, 2.0 - 1.5j]))
    ctx = pp.pp_create(inputs.diagonal(lam), target=pp.PP_TARGET_SM)
    poly = pp.pp_poly_from_roots(ctx, roots)
    x = inputs.start_vector(1000, 4, 0)
    y = pp.pp_apply_host(poly, x)
    assert np.allclose(y, O.poly_eval(roots, lam).real * x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("d1,d2", [(3, 4), (5, 6)])
def test_double_poly_apply_matches_oracle(d1, d2):
    """GPU double polynomial: roots as sets vs the oracle's build, and the apply of
    the GPU's own roots vs the oracle's apply of the same roots."""
    from paper_1806_08020_gb300 import pp
    lam = np.concatenate([np.linspace(0.05, 1.0, 300), np.linspace(2.0, 50.0, 1700)])
    Acsr = inputs.diagonal(lam)
    A = O.to_scipy(Acsr)
    b = inputs.start_vector(lam.size, 9, 0)
    ctx = pp.pp_create(Acsr, target=pp.PP_TARGET_SM)
    poly = pp.pp_build_poly2(ctx, d1, d2, b)
    outer, inner = pp.pp_poly_roots(poly), pp.pp_poly_inner_roots(poly)
    ref = O.build_double_poly(O.Operator(A, 0.0, O.Counters()), b, d1, d2, O.Counters())
    for got, want in ((inner, ref.inner.roots), (outer, ref.roots)):
        assert got.size == want.size
        for z in want:
            assert np.min(np.abs(got - z)) <= 1e-8 * abs(z)
    x = inputs.start_vector(lam.size, 9, 1)
    y = pp.pp_apply_host(poly, x)
    tau = 1 - O.poly_eval(inner, lam)
    want = (O.poly_eval(outer, tau) * x).real
    assert np.abs(y - want).max() <= 1e-10 * np.abs(x).max()


@pytest.mark.parametrize("n,j", [(37, 1), (1000, 7), (4099, 33), (100003, 51), (20000, 128)])
def test_orthogonalize_matches_oracle_cgs2(n, j):
    """CGS2 (Section 4) on the device vs the oracle's cgs2 on the same V and w."""
    import torch
    from paper_1806_08020_gb300 import pp
    rng = np.random.default_rng(n + j)
    Q, _ = np.linalg.qr(rng.standard_normal((n, j)))
    w = rng.standard_normal(n) + Q @ rng.standard_normal(j) * 10
    ctx = pp.pp_create(inputs.diagonal(np.ones(n)), stream=torch.cuda.current_stream().cuda_stream)
    ldv = (n + 31) // 32 * 32
    Vd = torch.zeros((j, ldv), dtype=torch.float64, device="cuda")
    Vd[:, :n] = torch.tensor(Q.T)
    wd = torch.tensor(w, device="cuda")
    vd = torch.empty(n, dtype=torch.float64, device="cuda")
    h = pp.pp_orthogonalize(ctx, Vd.data_ptr(), ldv, j, wd.data_ptr(), vd.data_ptr())
    w2, href = O.cgs2(Q, w, O.Counters())
    nw = np.linalg.norm(w)
    # each pass is a sum of n products: error <= n u ||V|| ||w|| per coefficient
    tol = 4 * n * U * nw
    assert np.abs(h[:j] - href).max() <= tol
    assert abs(h[j] - np.linalg.norm(w2)) <= tol
    v = vd.cpu().numpy()
    assert np.abs(v - w2 / np.linalg.norm(w2)).max() <= tol / np.linalg.norm(w2) * 4
    assert np.abs(Q.T @ v).max() <= 1e-12 * np.sqrt(n)


@pytest.mark.parametrize("n,j", [(1000, 7), (100003, 51), (20000, 128)])
def test_orthogonalize_fp32_matches_oracle_cgs2(n, j):
    """CGS2 on an FP32 basis (FP32 first pass, compensated second pass) vs the
    oracle's FP64 cgs2 on the same FP32-rounded V and w.

    h1 + h2 equals V^T w up to V^T of the rounding of w1 = w - V h1 to FP32
    (|.| <= a few u32 ||w||); the compensated second pass adds O(u32^2).
    """
    import torch
    from paper_1806_08020_gb300 import pp
    u32 = 2.0 ** -24
    rng = np.random.default_rng(n + 3 * j)
    Q, _ = np.linalg.qr(rng.standard_normal((n, j)))
    Q = Q.astype(np.float32).astype(np.float64)
    w = (rng.standard_normal(n) + Q @ rng.standard_normal(j) * 10).astype(np.float32).astype(np.float64)
    ctx = pp.pp_create(inputs.diagonal(np.ones(n)), stream=torch.cuda.current_stream().cuda_stream,
                       precision=pp.PP_FP32)
    ldv = (n + 31) // 32 * 32
    Vd = torch.zeros((j, ldv), dtype=torch.float32, device="cuda")
    Vd[:, :n] = torch.tensor(Q.T, dtype=torch.float32)
    wd = torch.tensor(w, dtype=torch.float32, device="cuda")
    vd = torch.empty(n, dtype=torch.float32, device="cuda")
    h = pp.pp_orthogonalize(ctx, Vd.data_ptr(), ldv, j, wd.data_ptr(), vd.data_ptr())
    w2, href = O.cgs2(Q, w, O.Counters())
    nw = np.linalg.norm(w)
    tol = 16 * u32 * nw
    assert np.abs(h[:j] - href).max() <= tol
    assert abs(h[j] - np.linalg.norm(w2)) <= tol
    v = vd.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(v - w2 / np.linalg.norm(w2)) <= 16 * u32 * nw / np.linalg.norm(w2)
    assert np.abs(Q.T @ v).max() <= 16 * u32 * nw / np.linalg.norm(w2)


def _wide_band_matrix():
    """2-D CD (N = 200) plus a few couplings 35,000 rows away: |col - row| >= 2^15,
    so 16-bit column offsets cannot hold it."""
    import scipy.sparse as sp
    base = O.to_scipy(inputs.convection_diffusion_2d(200, 20.0))
    n = base.shape[0]
    rows = np.arange(0, n - 35000, 997)
    far = sp.csr_matrix((np.full(rows.size, 1e-3), (rows, rows + 35000)), shape=(n, n))
    A = (base + far).tocsr()
    A.sort_indices()
    return inputs.CSR(n, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64))


@pytest.mark.parametrize("kind", ["cd", "band", "wide"])
@pytest.mark.parametrize("precision", [0, 1])
def test_sell_formats_bit_identical(kind, precision):
    """Every device format gives the same pi(A) x bit for bit: CSR, SELL with
    chunk height 16 or 32, 16- or 32-bit column indices, any row loop (plain,
    wide, or slice data staged by bulk copies), DIA with one or (FP32) four
    rows per thread, and whatever chunk height,
    block size and row loop the tuner picks.  Each row sums its entries in CSR
    order in every format (SELL padding adds 0 * x = 0 exactly)."""
    from paper_1806_08020_gb300 import pp
    A = {"cd": lambda: inputs.convection_diffusion_2d(150, 50.0),
         "band": lambda: inputs.banded_random(30011, 9, 5),
         "wide": _wide_band_matrix}[kind]()
    ref_ctx = pp.pp_create(A, precision=precision)
    roots = pp.pp_poly_roots(pp.pp_build_poly(ref_ctx, 12, inputs.start_vector(A.n, 3, 0)))
    x = inputs.start_vector(A.n, 3, 1)
    variants = {"csr": dict(format=pp.PP_FMT_CSR), "c16": dict(format=pp.PP_FMT_SELL, sell_c=16, sell_loop=1),
                "c32": dict(format=pp.PP_FMT_SELL, sell_c=32, sell_loop=1),
                "c32_i32": dict(format=pp.PP_FMT_SELL, sell_c=32, sell_index=32, sell_loop=1),
                "c16_wide": dict(format=pp.PP_FMT_SELL, sell_c=16, sell_loop=2),
                "c32_i32_wide": dict(format=pp.PP_FMT_SELL, sell_c=32, sell_index=32, sell_loop=2),
                "c32_staged": dict(format=pp.PP_FMT_SELL, sell_c=32, sell_loop=3),
                "c16_two_rows": dict(format=pp.PP_FMT_SELL, sell_c=16, sell_loop=4),
                "c32_i32_two_rows": dict(format=pp.PP_FMT_SELL, sell_c=32, sell_index=32, sell_loop=4),
                "c32_i32_staged": dict(format=pp.PP_FMT_SELL, sell_c=32, sell_index=32, sell_loop=3),
                "dia": dict(format=pp.PP_FMT_DIA),
                "dia_one_row": dict(format=pp.PP_FMT_DIA, dia_loop=1),
                "dia_four_rows": dict(format=pp.PP_FMT_DIA, dia_loop=2),
                "dia_two_rows": dict(format=pp.PP_FMT_DIA, dia_loop=3),
                "tuned": dict(format=pp.PP_FMT_SELL),
                "auto": dict()}
    out, info = {}, {}
    for name, o in variants.items():
        ctx = pp.pp_create(A, precision=precision, **o)
        info[name] = pp.pp_format_info(ctx)
        out[name] = pp.pp_apply_host(pp.pp_poly_from_roots(ctx, roots), x)
    assert info["csr"]["fmt"] == pp.PP_FMT_CSR
    assert info["c16"]["chunk"] == 16 and info["c32"]["chunk"] == 32
    assert info["c32_i32"]["index_bits"] == 32
    assert info["c32"]["index_bits"] == (32 if kind == "wide" else 16)
    assert info["tuned"]["chunk"] in (16, 32) and info["tuned"]["threads"] in (128, 256, 512)
    assert info["c16_wide"]["row_loop"] == 1 and info["c32"]["row_loop"] == 0
    assert info["c32_staged"]["row_loop"] == 2 and info["c32_i32_staged"]["index_bits"] == 32
    assert info["c16_two_rows"]["row_loop"] == 3
    assert info["dia"]["fmt"] == pp.PP_FMT_DIA and info["dia"]["index_bits"] == 0
    assert info["dia_one_row"]["row_loop"] == 0
    assert info["dia_four_rows"]["row_loop"] == (1 if precision == 1 else 0)  # several rows: FP32 only
    assert info["dia_two_rows"]["row_loop"] == (2 if precision == 1 else 0)
    # the second auto context on this matrix takes the first one's cached choice
    assert info["auto"] == pp.pp_format_info(ref_ctx)
    for name in variants:
        assert np.array_equal(out[name], out["csr"]), name
