// Damped GMRES polynomials: the heuristic of the Section 6.3 box on the device.
//
// 1-3. Build pi from b (GMRES(d), Section 2 box); run one Arnoldi(m, k) cycle
//      on pi(A) from b (the same device steps as pp_eigs); order the Ritz
//      values by distance from 1 and form the FP64 Rayleigh quotients for A of
//      the first k Ritz vectors (the convergence test's kernels).
// 4.   Ideal Order Condition |mu_1| <= ... <= |mu_nev| < min_{nev < j <= k} |mu_j|.
// 5.   If it fails, rebuild pi from A b (one power step damps the components of
//      b along the small eigenvalues, Section 6.1); if that fails too, halve d
//      until it holds or d = 1.
// Readings: the Arnoldi cycle always starts from the original b; with a shift
// (A - sigma I for smallest-real-part targets) the damping product and the
// magnitudes refer to the shifted operator.
#include "driver.h"

using namespace ppi;

namespace {

// Steps 1-4 for polynomial p: one cycle from b, Rayleigh quotients, the condition.
pp_status first_cycle_ideal(pp_ctx *c, const pp_poly *p, const double *b, int m, int k, int nev, bool &ideal) {
    const int64_t n = c->n, ldv = c->ldv();
    const ppk::Prec bpr = c->bprec;
    Driver D{c, n, ldv, k + 1};
    void *V = nullptr;
    double *dH = nullptr;
    const int ldh = m + 1;
    CKS(D.alloc(&V, (size_t)ldv * (m + 1) * c->besz));
    CKS(D.alloc((void **)&dH, (size_t)ldh * m * 8));
    CKS(D.alloc_test_buffers(bpr != ppk::F64));
    double nb = 0;
    CKS(load_unit(c, b, bpr, V, &nb, "damping"));
    CK(cudaMemsetAsync(dH, 0, (size_t)ldh * m * 8, c->stream));
    void *W = (p && p->inner) ? c->vec[0] : c->vec[6];
    CKS(arnoldi_extend(c, p, nullptr, bpr, V, ldv, dH, ldh, 0, m, W, nullptr, nullptr));
    std::vector<double> H((size_t)ldh * m);
    CK(cudaMemcpyAsync(H.data(), dH, H.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CKS(check_sweeps(c));
    Cycle cy;
    CKS(wanted_set(H, ldh, m, k, 1.0, cy));  // the k Ritz values nearest 1 (k + 1 slots if a pair splits)
    RitzOut R;
    pp_stats S{};
    CKS(D.ritz_test(V, bpr, m, cy.Sw, cy.sl, 0.0, R, S));
    std::vector<double> a(k);
    for (int s = 0; s < k; ++s) a[s] = std::hypot(R.lre[s] - c->sigma, R.lim[s]);
    bool ok = true;
    for (int s = 0; s + 1 < nev; ++s) ok = ok && a[s] <= a[s + 1];
    double rest = INFINITY;
    for (int s = nev; s < k; ++s) rest = std::min(rest, a[s]);
    ideal = ok && a[nev - 1] < rest;
    return PP_OK;
}

// y = (A - sigma I) b in FP64 on the device (the operator's matrix with its exact
// values: S = D^-1 A D when balanced).
pp_status damp_start(pp_ctx *c, const double *b, std::vector<double> &out) {
    const int64_t n = c->n;
    void *x = nullptr, *y = nullptr;
    CKS(dmalloc(c, &x, (size_t)n * 8));
    pp_status st = dmalloc(c, &y, (size_t)n * 8);
    if (st < 0) {
        dfree(c, x);
        return st;
    }
    ppk::StepArgs a;
    a.x = x;
    a.y = y;
    a.plain = 1;
    a.sigma = c->sigma;
    out.assign(n, 0.0);
    cudaError_t e = cudaMemcpyAsync(x, b, (size_t)n * 8, cudaMemcpyDefault, c->stream);  // b: host or device
    if (e == cudaSuccess) {
        ppk::launch_step(c->S64, a, c->stream);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), y, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->launches += 1;
    dfree(c, x);
    dfree(c, y);
    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "damping: A b: %s", cudaGetErrorString(e));
    return PP_OK;
}

}  // namespace

extern "C" pp_status pp_build_poly_damped(pp_ctx *c, int d, const double *b, int m, int k, int nev, pp_poly **out,
                                          int *degree, int *damped, int *ideal) {
    if (!c || !b || !out || d < 1 || nev < 1 || k <= nev || m < k || m > 127 || m >= c->n)
        return pp_fail(PP_EINVAL, "pp_build_poly_damped: need d >= 1, 1 <= nev < k <= m <= 127, m < n");
    *out = nullptr;
    std::vector<double> start(c->n);  // b, or A b once damped (host copy; b may be on the device)
    CK(cudaMemcpyAsync(start.data(), b, (size_t)c->n * 8, cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    bool dmp = false;
    for (;;) {
        pp_poly *p = nullptr;
        pp_status st = pp_build_poly(c, d, start.data(), &p);
        if (st < 0) return st;
        bool ok = false;
        pp_status s2 = first_cycle_ideal(c, p, b, m, k, nev, ok);
        if (s2 < 0) {
            pp_poly_destroy(p);
            return s2;
        }
        if (ok || (dmp && d == 1)) {
            *out = p;
            if (degree) *degree = d;
            if (damped) *damped = dmp ? 1 : 0;
            if (ideal) *ideal = ok ? 1 : 0;
            return st;  // PP_OK, or PP_EBREAKDOWN from the final build
        }
        pp_poly_destroy(p);
        if (!dmp) {
            CKS(damp_start(c, b, start));
            dmp = true;
        } else {
            d = std::max(1, d / 2);
        }
    }
}
