// Thick-restarted Arnoldi(m, k) on pi(A) (Section 2 box step 2; Section 4),
// with an optional mixed-precision mode.
//
// Each cycle extends the device-resident Arnoldi decomposition to m columns,
// then the host computes the Ritz values of H_m (FP64), orders them by
// distance from 1 and picks the wanted set.  Convergence is always tested in
// FP64 on A itself: Ritz vectors y = V_m s, Rayleigh quotients mu = y*Ay and
// residuals ||Ay - mu y|| <= rtol ||A||_1.  The restart keeps k Ritz vectors
// (k - 1 when a conjugate pair would split) through V_k = V_m Q_k.
//
// Mixed precision (context precision PP_FP32): the Arnoldi cycles run with
// FP32 matrix values, vectors and basis.  Within 50 rtol, or when the FP64
// residuals reach the FP32 floor, the wanted Ritz vectors are refined in FP64
// on A (Driver::refine): pi(A) applied in FP64 by the FP64 context of the twins to
// them (and, from the second round, to the cycle's next Ritz vectors), FP64
// CGS2, A projected onto that space (Rayleigh-Ritz), the refined pairs ranked
// as the Arnoldi ranks its Ritz values.  When that does not reach rtol (the
// FP32 Krylov space does not hold the eigenvectors well enough), the solve
// continues on the twin, started from the sum of the refined Ritz vectors:
// FP64 cycles for an FP32 context; for a BF16 basis (PP_FP32_BF16) FP32-basis
// cycles, which refine and continue in turn.
#include "driver.h"

using namespace ppi;

extern "C" pp_status pp_eigs(pp_ctx *c, const pp_poly *p, int nev, int m, int k, double rtol, const double *v0,
                             double *lam_re, double *lam_im, double *X, double *resid, int *nout, pp_stats *stats) {
    double t_start = now();
    if (!c || nev < 1 || k <= nev || m <= k || m >= c->n || m > 127 || !lam_re || !lam_im || !resid || !nout)
        return pp_fail(PP_EINVAL, "pp_eigs: need 1 <= nev < k < m < n, m <= 127 and output arrays");
    if (!(rtol > 0)) return pp_fail(PP_EINVAL, "pp_eigs: rtol must be positive");
    const int64_t n = c->n, ldv = c->ldv();
    const size_t esz = c->besz;  // basis element bytes
    const ppk::Prec bpr = c->bprec;
    const bool mixed = bpr != ppk::F64;
    const double target = p ? 1.0 : 0.0;
    pp_stats S{};
    const int64_t launches0 = chain_launches(c);
    Driver D{c, n, ldv, nev + 1};
    void *V = nullptr, *V2 = nullptr, *W = (p && p->inner) ? c->vec[0] : c->vec[6];
    double *dH = nullptr;
    const int ldh = m + 1;
    CKS(D.alloc(&V, (size_t)ldv * (m + 1) * esz));
    CKS(D.alloc(&V2, (size_t)ldv * (m + 1) * esz));
    CKS(D.alloc_test_buffers(mixed));
    CKS(D.alloc((void **)&dH, (size_t)ldh * m * 8));
    // start vector (host or device; NULL: all ones)
    double nv = 0;
    if (v0) {
        CKS(load_unit(c, v0, bpr, V, &nv, "pp_eigs"));
    } else {
        std::vector<double> ones(n, 1.0);
        CKS(load_unit(c, ones.data(), bpr, V, &nv, "pp_eigs"));
    }
    CK(cudaMemsetAsync(dH, 0, (size_t)ldh * m * 8, c->stream));
    S.dots += 1;
    S.vops += 2;
    const int64_t opm = op_mvps(p);
    const int64_t opv = op_vops(p);
    Timers tm;
    std::vector<std::pair<int, int>> marks;
    std::vector<double> H((size_t)ldh * m);
    Cycle cy;
    RitzOut R;
    bool converged = false;
    MixedSwitch sw(rtol);
    int j0 = 0;
    for (int64_t cycle = 1; cycle <= c->opts.max_cycles; ++cycle) {
        S.cycles = cycle;
        CKS(arnoldi_extend(c, p, nullptr, bpr, V, ldv, dH, ldh, j0, m, W, &tm, &marks));
        S.mvps += opm * (m - j0);
        for (int j = j0; j < m; ++j) {
            S.dots += 2 * (j + 1) + 1;
            S.vops += 4 * (j + 1) + 2 + opv;
        }
        CK(cudaMemcpyAsync(H.data(), dH, H.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        // the restart clock starts once the cycle's Arnoldi steps have run
        double th0 = now();
        CKS(check_sweeps(c));
        accumulate_times(tm, marks, S.t_apply, S.t_orth);
        CKS(wanted_set(H, ldh, m, nev, target, cy, c->opts.restart == PP_RESTART_HARMONIC));
        CKS(D.ritz_test(V, bpr, m, cy.Sw, cy.sl, rtol, R, S));
        S.nconv = R.nconv;
        trace_cycle("eigs", c, cycle, bpr == ppk::F64 ? 64 : (bpr == ppk::F32 ? 32 : 16), R,
                    R.all ? "converged" : nullptr);
        if (R.all) {
            converged = true;
            S.t_restart += now() - th0;
            break;
        }
        // continue on the twin (one precision up) from `start` (host or device
        // vector, NULL: all ones), the cycle count carried on
        auto continue_on_twin = [&](const double *start) -> pp_status {
            const double t_here = now() - th0;  // this cycle's test and refinement
            pp_ctx *tw = c->twin;
            const int max_c = tw->opts.max_cycles;
            tw->opts.max_cycles = (int)std::max<int64_t>(1, c->opts.max_cycles - cycle);
            pp_stats S2{};
            pp_status st2 = pp_eigs(tw, p, nev, m, k, rtol, start, lam_re, lam_im, X, resid, nout, &S2);
            tw->opts.max_cycles = max_c;
            if (st2 < 0) return st2;
            if (tw->bprec == ppk::F64) S2.fp64_cycles = S2.cycles;  // else as the twin counted them
            S2.cycles += S.cycles;
            S2.mvps += S.mvps;
            S2.dots += S.dots;
            S2.vops += S.vops;
            S2.t_apply += S.t_apply;
            S2.t_orth += S.t_orth;
            S2.t_restart += S.t_restart + t_here;
            S2.kernel_launches = chain_launches(c) - launches0;
            S2.t_total = now() - t_start;
            if (stats) *stats = S2;
            return st2;
        };
        if (bpr == ppk::BF16 && c->twin && cycle < c->opts.max_cycles &&
            *std::max_element(R.res.begin(), R.res.end()) > 10 * rtol) {
            // A BF16 basis stalls near 1e-3 (its unit roundoff), out of the
            // refinement's reach, and a start from its Ritz vectors served the
            // FP32 cycles worse than the original one (measured on the 3-D
            // workload): after one cycle the solve restarts on the FP32 twin from
            // the start vector.
            return continue_on_twin(v0);
        }
        if (mixed && sw.should_refine(R, cycle == c->opts.max_cycles)) {
            CKS(D.refine(p, cy.sl, nev, R, rtol, c->opts.refine_steps, 3, S, &cy, V, bpr, m));
            S.nconv = R.nconv;
            trace_cycle("eigs", c, cycle, 64, R, R.all ? "refined: converged" : "refined");
            converged = R.all;
            if (converged || cycle == c->opts.max_cycles) {
                S.t_restart += now() - th0;
                break;
            }
            if (c->twin) {
                // The Krylov space does not hold the eigenvectors to rtol (the problem
                // is too non-normal for the basis precision): continue on the twin,
                // one precision up, with the same polynomial, started from the sum of
                // the refined Ritz vectors.
                std::vector<double> Yh, w0(n, 0.0);
                CKS(download_vecs(c, D.Y64, ldv, cy.sl.nw, Yh, ppk::F64));
                for (int s = 0; s < cy.sl.nw; ++s)
                    for (int64_t i = 0; i < n; ++i) w0[i] += Yh[(size_t)s * n + i];
                if (!c->h_bal.empty())  // the twin's Krylov space is in S's coordinates (y = D^-1 x)
                    for (int64_t i = 0; i < n; ++i) w0[i] /= c->h_bal[i];
                return continue_on_twin(w0.data());
            }
            sw.reset();  // no twin: keep cycling in this precision (restart below)
        }
        if (cycle == c->opts.max_cycles) {
            S.t_restart += now() - th0;
            break;
        }
        std::vector<double> Q, Hn;
        int kk = restart_basis(cy, H, ldh, k, Q, Hn);
        CK(cudaMemcpyAsync(D.dQ, Q.data(), Q.size() * 8, cudaMemcpyHostToDevice, c->stream));
        if (cy.harmonic) {  // V_{kk+1} = V_{m+1} P
            ppk::launch_rotate(bpr, (int)n, V, ldv, m + 1, D.dQ, kk + 1, V2, ldv, c->stream);
            CKS(check_launch(c));
            S.vops += (int64_t)(m + 1) * (kk + 1);
        } else {  // V_kk = V_m Q, v_{kk+1} = v_{m+1}
            ppk::launch_rotate(bpr, (int)n, V, ldv, m, D.dQ, kk, V2, ldv, c->stream);
            CKS(check_launch(c));
            CK(cudaMemcpyAsync((char *)V2 + (size_t)kk * ldv * esz, (char *)V + (size_t)m * ldv * esz, n * esz,
                               cudaMemcpyDeviceToDevice, c->stream));
            S.vops += (int64_t)m * kk;
        }
        std::swap(V, V2);
        CK(cudaMemcpyAsync(dH, Hn.data(), Hn.size() * 8, cudaMemcpyHostToDevice, c->stream));
        j0 = kk;
        S.t_restart += now() - th0;
    }
    double maxres = 0;
    std::vector<int> srt;
    write_outputs(c->opts.target, n, cy.sl, R, {}, lam_re, lam_im, resid, nullptr, maxres, &srt);
    // eigenvectors scaled and ordered on the device, one copy into X (AY64 is free after the last test)
    if (X) CKS(vectors_out(c, n, cy.sl, R, D.Y64, ldv, srt, D.AY64, X));
    *nout = cy.sl.nw;
    S.converged = converged ? 1 : 0;
    S.max_resid = maxres;
    S.fp64_cycles = mixed ? 0 : S.cycles;
    S.kernel_launches = chain_launches(c) - launches0;
    S.t_total = now() - t_start;
    if (stats) *stats = S;
    if (!converged) return pp_fail(PP_ENOTCONV, "pp_eigs: not converged in %lld cycles", (long long)S.cycles);
    return PP_OK;
}

extern "C" pp_status pp_restart_basis(int m, const double *H, int ldh, int k, double target, int harmonic,
                                      double *Q, double *Hn, int *kk, double *re, double *im) {
    if (!H || !Q || !Hn || !kk || m < 2 || m > 127 || k < 1 || k >= m || ldh < m + 1)
        return pp_fail(PP_EINVAL, "pp_restart_basis: need 1 <= k < m <= 127, ldh >= m + 1");
    std::vector<double> Hv((size_t)ldh * m);
    std::copy(H, H + Hv.size(), Hv.begin());
    Cycle cy;
    CKS(wanted_set(Hv, ldh, m, 1, target, cy, harmonic != 0));
    std::vector<double> Qv, Hnv;
    const int kept = restart_basis(cy, Hv, ldh, k, Qv, Hnv);
    std::copy(Qv.begin(), Qv.end(), Q);
    std::copy(Hnv.begin(), Hnv.end(), Hn);
    *kk = kept;
    for (int i = 0; i < m; ++i) {
        if (re) re[i] = cy.nu[cy.order[i]].real();
        if (im) im[i] = cy.nu[cy.order[i]].imag();
    }
    return PP_OK;
}
