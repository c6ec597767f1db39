"""Element-wise parity of the polynomial apply at the benchmark's full sizes.

* n = 10^6 2-D convection-diffusion (N = 1000, beta = 100), FP64, the format
  the tuner picks for it (the kernel the benchmark times): pi(A) x with the
  oracle's GMRES(50) roots (Section 2 box, Eq. (2.1)) against the oracle's
  FP64 apply of the same roots, element by element.
* n = 160^3 3-D convection-diffusion (beta = 50), FP32 values and vectors in
  diagonal storage (the mixed-precision workload's format): the double
  polynomial pi_2(tau(A)) x (Section 8) with the oracle's roots (d1 = 3,
  d2 = 3: nine general passes with the running sum, the pass the mixed
  solve spends its time in) against the oracle's FP64 apply.

Tolerance: the forward-error model of the smaller apply tests, with the unit
roundoff of the arithmetic (2^-53 or 2^-24): 64 u times the sum, over the
factors, of each factor's local rounding (SpMV and axpy, scaled by the
factor's coefficient) evaluated on the oracle's own intermediate vectors.  In
FP32 the rounding of the matrix values and of x to FP32 has the same form
(u |A| |p| per product, u |x| at the input) and is covered by it.
"""
import numpy as np
import pytest

import oracle as O
from paper_1806_08020_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0**-53
U32 = 2.0**-24


def _inf(v):
    return float(np.abs(v).max())


def _factor_bound(apply_op, local_op, roots, x, running_sum=False):
    """Sum of the factors' local rounding terms along the oracle's intermediates.

    apply_op(p) -> the operator applied exactly by the oracle; local_op(p) ->
    the local rounding term of one operator application to p (in units of u).
    With running_sum, also returns r = sum_i op(p_{i-1})/theta_i (tau of the
    double polynomial) and counts its update.
    """
    p = np.array(x, dtype=np.float64, copy=True)
    r = np.zeros_like(p)
    tot = 0.0
    i = 0
    while i < roots.size:
        th = roots[i]
        if th.imag == 0:
            t = apply_op(p)
            d = t / th.real
            tot += local_op(p) / abs(th) + _inf(p) + _inf(d)
            p = p - d
            r = r + d
            tot += _inf(r) if running_sum else 0.0
            i += 1
        else:
            m2 = abs(th) ** 2
            t = apply_op(p)
            s = apply_op(t)
            d = (2 * th.real / m2) * t - s / m2
            tot += (2 * abs(th.real) * local_op(p) + local_op(t)) / m2 + _inf(p) + _inf(t) * 2 * abs(th.real) / m2 \
                + _inf(s) / m2
            p = p - d
            r = r + d
            tot += _inf(r) if running_sum else 0.0
            i += 2
    return p, r, tot


def _spmv_local(A, sigma):
    Ainf = float(abs(A).sum(axis=1).max()) + abs(sigma)
    return lambda p: Ainf * _inf(p)


def test_apply_full_size_plain_large_fp64():
    from paper_1806_08020_gb300 import pp
    cfg = inputs.plain_large()
    A = O.to_scipy(cfg["A"])
    n = A.shape[0]
    sigma = O.gershgorin_shift(A)
    op = O.Operator(A, sigma, O.Counters())
    P = O.build_poly(op, inputs.start_vector(n, cfg["seed"], 0), cfg["d"], O.Counters())
    x = inputs.start_vector(n, cfg["seed"] + 17, 0)
    ref, _, tot = _factor_bound(op, _spmv_local(A, sigma), P.roots, x)
    ctx = pp.pp_create(cfg["A"])  # auto: the tuner's choice, as in the benchmark
    fmt = pp.pp_format_info(ctx)
    poly = pp.pp_poly_from_roots(ctx, P.roots)
    y = pp.pp_apply_host(poly, x)
    err = np.abs(y - ref)
    tol = 64 * U64 * tot
    print(f"n = 1e6 FP64 apply ({fmt}): max err {err.max():.3e}, tolerance {tol:.3e}, ratio {err.max() / tol:.3g}")
    assert np.all(np.isfinite(y))
    assert err.max() <= tol


def test_apply_full_size_precision_3d_fp32_dia():
    from paper_1806_08020_gb300 import pp
    cfg = inputs.precision_3d()
    A = O.to_scipy(cfg["A"])
    n = A.shape[0]
    op = O.Operator(A, O.gershgorin_shift(A), O.Counters())
    assert op.sigma == 0.0
    P = O.build_double_poly(op, inputs.start_vector(n, cfg["seed"], 0), 3, 3, O.Counters())
    inner = P.inner.roots
    local_A = _spmv_local(A, 0.0)

    def tau(u):
        return O.apply_poly(op, inner, u)[1]

    def tau_local(u):
        return _factor_bound(op, local_A, inner, u, running_sum=True)[2]

    x = inputs.start_vector(n, cfg["seed"] + 17, 0)
    ref, _, tot = _factor_bound(tau, tau_local, P.roots, x)
    tot += _inf(x)  # x rounded to FP32 on the way in
    ctx = pp.pp_create(cfg["A"], precision=pp.PP_FP32, format=pp.PP_FMT_DIA)
    assert pp.pp_format_info(ctx)["fmt"] == pp.PP_FMT_DIA
    poly = pp.pp_poly2_from_roots(ctx, inner, P.roots)
    y = pp.pp_apply_host(poly, x)
    err = np.abs(y - ref)
    tol = 64 * U32 * tot
    print(f"n = 160^3 FP32 DIA double-polynomial apply: max err {err.max():.3e}, tolerance {tol:.3e}, "
          f"ratio {err.max() / tol:.3g}")
    assert np.all(np.isfinite(y))
    assert err.max() <= tol
    # the same double polynomial with the oracle's roots in FP64 agrees to FP64 rounding
    ctx64 = pp.pp_create(cfg["A"], format=pp.PP_FMT_DIA)
    y64 = pp.pp_apply_host(pp.pp_poly2_from_roots(ctx64, inner, P.roots), x)
    assert np.abs(y64 - ref).max() <= 64 * U64 * tot
