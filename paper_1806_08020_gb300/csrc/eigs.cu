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
// FP32 matrix values, vectors and basis (the CGS2 sums accumulate in FP64).
// When the FP64 residuals reach the FP32 floor the wanted Ritz vectors are
// refined in FP64 on A: a block Krylov space span{Y, AY, ..., A^s Y} is built
// with FP64 SpMVs and FP64 CGS2, A is projected onto it (Rayleigh-Ritz), and
// the Ritz pairs nearest the current estimates replace them.
#include "ctx.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

using namespace ppi;

namespace {

// Wanted slots: a real Ritz pair occupies one slot, a conjugate pair two
// (columns Re, Im of the Im > 0 member's vector).
struct Slots {
    int nw = 0;
    std::vector<int> partner;  // partner column (itself for a real slot)
    std::vector<double> sg;    // +1 Re column of a pair, -1 Im column, 0 real
};

struct RitzOut {
    std::vector<double> lre, lim, res, ynrm;
    int nconv = 0;
    bool all = false;
};

struct Driver {
    pp_ctx *c;
    int64_t n, ldv;
    int wcap;
    std::vector<void *> mine;
    // FP64 test buffers
    double *Y64 = nullptr, *AY64 = nullptr;
    void *Ys = nullptr;  // storage-precision Ritz vectors (mixed mode)
    double *dQ = nullptr, *dq = nullptr, *dmu = nullptr;
    int *dpartner = nullptr;
    // refinement
    double *Z = nullptr, *dG = nullptr;
    static constexpr int kZcap = 128;

    ~Driver() {
        cudaStreamSynchronize(c->stream);
        for (void *q : mine) dfree(c, q);
    }
    pp_status alloc(void **p, size_t bytes) {
        pp_status st = dmalloc(c, p, bytes);
        if (st >= 0) mine.push_back(*p);
        return st;
    }

    // Y64 = B S (B: mcols columns of precision pb), then FP64 Rayleigh quotients
    // and residual norms on A for each slot.
    pp_status ritz_test(const void *B, ppk::Prec pb, int mcols, const std::vector<double> &Sw, const Slots &sl,
                        double rtol, RitzOut &out, pp_stats &S) {
        const int nw = sl.nw;
        CK(cudaMemcpyAsync(dQ, Sw.data(), Sw.size() * 8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(dpartner, sl.partner.data(), nw * 4, cudaMemcpyHostToDevice, c->stream));
        if (pb == ppk::F64) {
            ppk::launch_rotate(ppk::F64, (int)n, B, ldv, mcols, dQ, nw, Y64, ldv, c->stream);
            CKS(check_launch(c));
        } else {
            ppk::launch_rotate(ppk::F32, (int)n, B, ldv, mcols, dQ, nw, Ys, ldv, c->stream);
            CKS(check_launch(c));
            ppk::launch_convert(ppk::F32, ppk::F64, (int)(ldv * nw), Ys, Y64, c->stream);
            CKS(check_launch(c));
        }
        for (int s = 0; s < nw; ++s) {
            ppk::StepArgs a;
            a.x = Y64 + (size_t)s * ldv;
            a.y = AY64 + (size_t)s * ldv;
            a.plain = 1;
            ppk::launch_step(c->A64, a, c->stream);
            CKS(check_launch(c));
        }
        S.mvps += nw;
        S.vops += (int64_t)4 * mcols * nw;
        ppk::ColDotArgs cda;
        cda.n = (int)n;
        cda.nw = nw;
        cda.Y = Y64;
        cda.AY = AY64;
        cda.ld = ldv;
        cda.partner = dpartner;
        cda.q = dq;
        cda.part = c->d_part;
        cda.ticket = c->d_ticket;
        cda.mode = 0;
        ppk::launch_coldots(ppk::F64, cda, c->stream);
        CKS(check_launch(c));
        std::vector<double> q((size_t)4 * nw);
        CK(cudaMemcpyAsync(q.data(), dq, q.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        auto &lre = out.lre, &lim = out.lim;
        lre.assign(nw, 0);
        lim.assign(nw, 0);
        out.ynrm.assign(nw, 0);
        for (int s = 0; s < nw;) {
            if (sl.partner[s] == s) {
                lre[s] = q[4 * s + 1] / q[4 * s];
                out.ynrm[s] = q[4 * s];
                s += 1;
            } else {
                double yy = q[4 * s] + q[4 * (s + 1)];
                lre[s] = lre[s + 1] = (q[4 * s + 1] + q[4 * (s + 1) + 1]) / yy;
                lim[s] = (q[4 * s + 2] - q[4 * (s + 1) + 2]) / yy;
                lim[s + 1] = -lim[s];
                out.ynrm[s] = out.ynrm[s + 1] = yy;
                s += 2;
            }
        }
        // residual columns: Re part AYr - mr Yr + mi Yi, Im part AYi - mr Yi - mi Yr
        std::vector<double> mu((size_t)3 * nw, 0.0);
        for (int s = 0; s < nw; ++s) {
            mu[s] = lre[s];
            mu[nw + s] = (sl.partner[s] == s) ? 0.0 : (sl.sg[s] > 0 ? lim[s] : lim[sl.partner[s]]);
            mu[2 * nw + s] = sl.sg[s];
        }
        CK(cudaMemcpyAsync(dmu, mu.data(), mu.size() * 8, cudaMemcpyHostToDevice, c->stream));
        cda.mode = 1;
        cda.mur = dmu;
        cda.mui = dmu + nw;
        cda.sg = dmu + 2 * nw;
        ppk::launch_coldots(ppk::F64, cda, c->stream);
        CKS(check_launch(c));
        CK(cudaMemcpyAsync(q.data(), dq, q.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        out.res.assign(nw, 0);
        out.all = true;
        out.nconv = 0;
        for (int s = 0; s < nw;) {
            if (sl.partner[s] == s) {
                out.res[s] = std::sqrt(std::max(q[4 * s + 3], 0.0) / out.ynrm[s]) / c->norm1;
                s += 1;
            } else {
                double r2 = (q[4 * s + 3] + q[4 * (s + 1) + 3]) / out.ynrm[s];
                out.res[s] = out.res[s + 1] = std::sqrt(std::max(r2, 0.0)) / c->norm1;
                s += 2;
            }
        }
        for (double r : out.res) {
            bool ok = std::isfinite(r) && r <= rtol;
            out.nconv += ok;
            out.all = out.all && ok;
        }
        return PP_OK;
    }

    // FP64 refinement on A (mixed precision): block Krylov span{Y, AY, ..., A^s Y}
    // with CGS2, Rayleigh-Ritz of A, Ritz pairs matched to the current estimates.
    pp_status refine(const Slots &sl, RitzOut &R, double rtol, int steps, int rounds, pp_stats &S) {
        const int nw = sl.nw;
        steps = std::max(1, std::min(steps, kZcap / nw - 1));
        const int ldg = kZcap + 1;
        double *W = AY64 + (size_t)nw * ldv;  // spare FP64 column (context vectors are FP32 here)
        for (int round = 0; round < rounds; ++round) {
            int nz = 0;
            CK(cudaMemsetAsync(dG, 0, (size_t)ldg * kZcap * 8, c->stream));
            for (int s = 0; s < nw; ++s) {
                CK(cudaMemcpyAsync(W, Y64 + (size_t)s * ldv, n * 8, cudaMemcpyDeviceToDevice, c->stream));
                CKS(cgs2_step(c, ppk::F64, Z, ldv, nz, W, c->d_small + 2048));
                nz++;
            }
            int b0 = 0, b1 = nz;
            for (int st = 0; st < steps; ++st) {
                for (int col = b0; col < b1; ++col) {
                    ppk::StepArgs a;
                    a.x = Z + (size_t)col * ldv;
                    a.y = W;
                    a.plain = 1;
                    ppk::launch_step(c->A64, a, c->stream);
                    CKS(check_launch(c));
                    CKS(cgs2_step(c, ppk::F64, Z, ldv, nz, W, dG + (size_t)col * ldg));
                    S.dots += 2 * nz + 1;
                    S.vops += 4 * nz + 2;
                    nz++;
                }
                S.mvps += b1 - b0;
                b0 = b1;
                b1 = nz;
            }
            // last block: G[:, col] = Z^T A z_col (no new columns)
            for (int col = b0; col < b1; ++col) {
                ppk::StepArgs a;
                a.x = Z + (size_t)col * ldv;
                a.y = W;
                a.plain = 1;
                ppk::launch_step(c->A64, a, c->stream);
                CKS(check_launch(c));
                ppk::CgsArgs ca;
                ca.mode = 0;
                ca.n = (int)n;
                ca.V = Z;
                ca.ldv = ldv;
                ca.j = nz;
                ca.w = W;
                ca.out = dG + (size_t)col * ldg;
                ca.part = c->d_part;
                ca.ticket = c->d_ticket;
                ppk::launch_cgs(ppk::F64, ca, c->stream);
                CKS(check_launch(c));
                S.dots += nz;
                S.vops += nz;
            }
            S.mvps += b1 - b0;
            std::vector<double> Gfull((size_t)ldg * nz), G((size_t)nz * nz);
            CK(cudaMemcpyAsync(Gfull.data(), dG, Gfull.size() * 8, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            for (int j = 0; j < nz; ++j)
                for (int i = 0; i < nz; ++i) G[i + (size_t)j * nz] = Gfull[i + (size_t)j * ldg];
            for (double v : G)
                if (!std::isfinite(v)) return pp_fail(PP_ENUMERIC, "refinement: non-finite projection");
            std::vector<double> wr(nz), wi(nz), Sv((size_t)nz * nz);
            if (!ppd::dense_eig(nz, G.data(), nz, wr.data(), wi.data(), Sv.data(), nz))
                return pp_fail(PP_ENUMERIC, "refinement: Rayleigh-Ritz QR failed");
            // match each wanted unit to the nearest unclaimed Ritz value of the same kind
            std::vector<char> used(nz, 0);
            std::vector<double> Sw((size_t)nz * nw);
            for (int s = 0; s < nw;) {
                bool pair = sl.partner[s] != s;
                cd target(R.lre[s], pair ? std::fabs(R.lim[s]) : 0.0);
                int best = -1;
                double bd = INFINITY;
                for (int pass = 0; pass < 2 && best < 0; ++pass)
                    for (int i = 0; i < nz; ++i) {
                        if (used[i]) continue;
                        bool ipair = wi[i] != 0.0;
                        if (pass == 0 && ipair != pair) continue;
                        if (ipair && wi[i] < 0) continue;
                        double dd = std::abs(cd(wr[i], wi[i]) - target);
                        if (dd < bd) {
                            bd = dd;
                            best = i;
                        }
                    }
                if (best < 0) return pp_fail(PP_ENUMERIC, "refinement: no Ritz value to match");
                used[best] = 1;
                if (wi[best] != 0.0) used[best + 1] = 1;
                if (!pair) {
                    std::copy(&Sv[(size_t)best * nz], &Sv[(size_t)best * nz] + nz, &Sw[(size_t)s * nz]);
                    s += 1;
                } else if (wi[best] != 0.0) {
                    std::copy(&Sv[(size_t)best * nz], &Sv[(size_t)best * nz] + nz, &Sw[(size_t)s * nz]);
                    std::copy(&Sv[(size_t)(best + 1) * nz], &Sv[(size_t)(best + 1) * nz] + nz,
                              &Sw[(size_t)(s + 1) * nz]);
                    s += 2;
                } else {
                    return pp_fail(PP_ENUMERIC, "refinement: a conjugate pair matched a real Ritz value");
                }
            }
            CKS(ritz_test(Z, ppk::F64, nz, Sw, sl, rtol, R, S));
            S.vops += (int64_t)nz * nw;
            if (R.all) return PP_OK;
        }
        return PP_OK;
    }
};

}  // namespace

extern "C" pp_status pp_eigs(pp_ctx *c, const pp_poly *p, int nev, int m, int k, double rtol, const double *v0,
                             double *lam_re, double *lam_im, double *X, double *resid, int *nout, pp_stats *stats) {
    double t_start = now();
    if (!c || nev < 1 || k <= nev || m <= k || m >= c->n || m > 127 || !lam_re || !lam_im || !resid || !nout)
        return pp_fail(PP_EINVAL, "pp_eigs: need 1 <= nev < k < m < n, m <= 127 and output arrays");
    if (!(rtol > 0)) return pp_fail(PP_EINVAL, "pp_eigs: rtol must be positive");
    const int64_t n = c->n, ldv = c->ldv();
    const size_t esz = c->esz;
    const bool mixed = c->A.prec != ppk::F64;
    const double target = p ? 1.0 : 0.0;
    pp_stats S{};
    int64_t launches0 = c->launches;
    Driver D{c, n, ldv, nev + 1};
    void *V = nullptr, *V2 = nullptr, *W = (p && p->inner) ? c->vec[0] : c->vec[6];
    double *dH = nullptr;
    const int ldh = m + 1;
    const int wcap = nev + 1;
    CKS(D.alloc(&V, (size_t)ldv * (m + 1) * esz));
    CKS(D.alloc(&V2, (size_t)ldv * (m + 1) * esz));
    CKS(D.alloc((void **)&D.Y64, (size_t)ldv * (wcap + 1) * 8));
    CKS(D.alloc((void **)&D.AY64, (size_t)ldv * (wcap + 1) * 8));
    if (mixed) {
        CKS(D.alloc(&D.Ys, (size_t)ldv * (wcap + 1) * esz));
        CKS(D.alloc((void **)&D.Z, (size_t)ldv * (Driver::kZcap + 1) * 8));
        CKS(D.alloc((void **)&D.dG, (size_t)(Driver::kZcap + 1) * Driver::kZcap * 8));
    }
    CKS(D.alloc((void **)&dH, (size_t)ldh * m * 8));
    CKS(D.alloc((void **)&D.dQ, (size_t)Driver::kZcap * Driver::kZcap * 8));
    CKS(D.alloc((void **)&D.dq, (size_t)4 * (wcap + 1) * 8));
    CKS(D.alloc((void **)&D.dmu, (size_t)3 * (wcap + 1) * 8));
    CKS(D.alloc((void **)&D.dpartner, (size_t)(wcap + 1) * 4));
    CKS(ensure_part(c, std::max((size_t)ppk::cgs_grid((int)n) * 130, (size_t)(wcap + 1) * 3 * 1024)));
    // start vector
    std::vector<double> v0h(n, 1.0);
    if (v0) std::copy(v0, v0 + n, v0h.begin());
    double nv = 0;
    for (double x : v0h) nv += x * x;
    nv = std::sqrt(nv);
    if (!(nv > 0) || !std::isfinite(nv)) return pp_fail(PP_EINVAL, "pp_eigs: start vector is zero or not finite");
    CKS(upload_vec(c, v0h.data(), 1.0 / nv, V));
    CK(cudaMemsetAsync(dH, 0, (size_t)ldh * m * 8, c->stream));
    S.dots += 1;
    S.vops += 2;
    const int64_t opm = op_mvps(p);
    const int64_t opv = op_vops(p);
    Timers tm;
    std::vector<std::pair<int, int>> marks;
    std::vector<double> H((size_t)ldh * m), Hm((size_t)m * m), wr(m), wi(m), Sv((size_t)m * m);
    std::vector<cd> nu(m);
    Slots sl;
    RitzOut R;
    bool converged = false;
    double best_prev = INFINITY;
    int stall = 0;
    // The FP32 cycles stop at the FP32 floor: residuals below 1e-6 that no
    // longer halve per cycle, or within 10 rtol; then FP64 refinement on A.
    const double tau_floor = std::max(rtol, 1e-6), tau_near = 10 * rtol;
    int j0 = 0;
    for (int64_t cycle = 1; cycle <= c->opts.max_cycles; ++cycle) {
        S.cycles = cycle;
        CKS(arnoldi_extend(c, p, nullptr, V, ldv, dH, ldh, j0, m, W, &tm, &marks));
        S.mvps += opm * (m - j0);
        for (int j = j0; j < m; ++j) {
            S.dots += 2 * (j + 1) + 1;
            S.vops += 4 * (j + 1) + 2 + opv;
        }
        double th0 = now();
        CK(cudaMemcpyAsync(H.data(), dH, H.size() * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        accumulate_times(tm, marks, S.t_apply, S.t_orth);
        for (double v : H)
            if (!std::isfinite(v))
                return pp_fail(PP_ENUMERIC, "pp_eigs: non-finite Hessenberg entry in cycle %lld", (long long)cycle);
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) Hm[i + (size_t)j * m] = H[i + (size_t)j * ldh];
        if (!ppd::dense_eig(m, Hm.data(), m, wr.data(), wi.data(), Sv.data(), m))
            return pp_fail(PP_ENUMERIC, "pp_eigs: Ritz values: QR failed");
        for (int i = 0; i < m; ++i) nu[i] = cd(wr[i], wi[i]);
        std::vector<int> order = ppd::ritz_order(nu, target);
        // wanted set: nev slots, one more when the boundary would split a pair
        sl.nw = nev + (nu[order[nev - 1]].imag() > 0 ? 1 : 0);
        sl.partner.assign(sl.nw, 0);
        sl.sg.assign(sl.nw, 0.0);
        std::vector<double> Sw((size_t)m * sl.nw);
        for (int s = 0; s < sl.nw;) {
            int i = order[s];
            if (wi[i] == 0.0) {
                std::copy(&Sv[(size_t)i * m], &Sv[(size_t)i * m] + m, &Sw[(size_t)s * m]);
                sl.partner[s] = s;
                s += 1;
            } else {
                int base = wi[i] > 0 ? i : i - 1;
                std::copy(&Sv[(size_t)base * m], &Sv[(size_t)base * m] + m, &Sw[(size_t)s * m]);
                std::copy(&Sv[(size_t)(base + 1) * m], &Sv[(size_t)(base + 1) * m] + m, &Sw[(size_t)(s + 1) * m]);
                sl.partner[s] = s + 1;
                sl.partner[s + 1] = s;
                sl.sg[s] = 1.0;
                sl.sg[s + 1] = -1.0;
                s += 2;
            }
        }
        CKS(D.ritz_test(V, c->A.prec, m, Sw, sl, rtol, R, S));
        S.nconv = R.nconv;
        if (R.all) {
            converged = true;
            S.t_restart += now() - th0;
            break;
        }
        if (mixed) {
            double mx = *std::max_element(R.res.begin(), R.res.end());
            stall = (mx < 0.5 * best_prev) ? 0 : stall + 1;
            best_prev = std::min(best_prev, mx);
            if ((mx <= tau_floor && (stall >= 1 || mx <= tau_near)) || stall >= 3 || cycle == c->opts.max_cycles) {
                CKS(D.refine(sl, R, rtol, c->opts.refine_steps, 3, S));
                S.nconv = R.nconv;
                converged = R.all;
                S.t_restart += now() - th0;
                break;
            }
        }
        if (cycle == c->opts.max_cycles) {
            S.t_restart += now() - th0;
            break;
        }
        // thick restart: keep k (k-1 if a pair would split), Q_k = qr([Re, Im] of kept Ritz vectors)
        int kk = (nu[order[k - 1]].imag() > 0) ? k - 1 : k;
        std::vector<double> B((size_t)m * kk);
        int col = 0;
        for (int s = 0; s < kk; ++s) {
            int i = order[s];
            if (wi[i] == 0.0) {
                std::copy(&Sv[(size_t)i * m], &Sv[(size_t)i * m] + m, &B[(size_t)col * m]);
                col++;
            } else if (wi[i] > 0) {
                std::copy(&Sv[(size_t)i * m], &Sv[(size_t)i * m] + m, &B[(size_t)col * m]);
                std::copy(&Sv[(size_t)(i + 1) * m], &Sv[(size_t)(i + 1) * m] + m, &B[(size_t)(col + 1) * m]);
                col += 2;
            }
        }
        std::vector<double> Q((size_t)m * kk);
        ppd::thin_qr(m, kk, B.data(), Q.data());
        CK(cudaMemcpyAsync(D.dQ, Q.data(), Q.size() * 8, cudaMemcpyHostToDevice, c->stream));
        ppk::launch_rotate(c->A.prec, (int)n, V, ldv, m, D.dQ, kk, V2, ldv, c->stream);
        CKS(check_launch(c));
        CK(cudaMemcpyAsync((char *)V2 + (size_t)kk * ldv * esz, (char *)V + (size_t)m * ldv * esz, n * esz,
                           cudaMemcpyDeviceToDevice, c->stream));
        std::swap(V, V2);
        S.vops += (int64_t)m * kk;
        // H_k = [Q^T H_m Q ; h_{m+1,m} e_m^T Q]
        std::vector<double> HQ((size_t)m * kk, 0.0), Hn((size_t)ldh * m, 0.0);
        for (int cc = 0; cc < kk; ++cc)
            for (int r = 0; r < m; ++r) {
                double s = 0;
                for (int t = 0; t < m; ++t) s += Hm[r + (size_t)t * m] * Q[t + (size_t)cc * m];
                HQ[r + (size_t)cc * m] = s;
            }
        for (int cc = 0; cc < kk; ++cc) {
            for (int r = 0; r < kk; ++r) {
                double s = 0;
                for (int t = 0; t < m; ++t) s += Q[t + (size_t)r * m] * HQ[t + (size_t)cc * m];
                Hn[r + (size_t)cc * ldh] = s;
            }
            Hn[kk + (size_t)cc * ldh] = H[m + (size_t)(m - 1) * ldh] * Q[(m - 1) + (size_t)cc * m];
        }
        CK(cudaMemcpyAsync(dH, Hn.data(), Hn.size() * 8, cudaMemcpyHostToDevice, c->stream));
        j0 = kk;
        S.t_restart += now() - th0;
    }
    const int nw = sl.nw;
    // outputs sorted by the target: SR -> (Re, |Im|, Im > 0 first); SM -> (|lam|, Re, Im > 0 first)
    std::vector<int> srt(nw);
    for (int s = 0; s < nw; ++s) srt[s] = s;
    const auto &lre = R.lre, &lim = R.lim;
    bool sr = c->opts.target == PP_TARGET_SR;
    std::stable_sort(srt.begin(), srt.end(), [&](int a, int b) {
        double ka = sr ? lre[a] : std::hypot(lre[a], lim[a]), kb = sr ? lre[b] : std::hypot(lre[b], lim[b]);
        if (ka != kb) return ka < kb;
        if (sr) {
            if (std::fabs(lim[a]) != std::fabs(lim[b])) return std::fabs(lim[a]) < std::fabs(lim[b]);
        } else if (lre[a] != lre[b]) {
            return lre[a] < lre[b];
        }
        return lim[a] > lim[b];
    });
    std::vector<double> Yh;
    if (X) CKS(download_vecs(c, D.Y64, ldv, nw, Yh, ppk::F64));
    double maxres = 0;
    for (int s = 0; s < nw; ++s) {
        int o = srt[s];
        lam_re[s] = lre[o];
        lam_im[s] = lim[o];
        resid[s] = R.res[o];
        maxres = std::max(maxres, R.res[o]);
        if (X) {
            // unit vector: a real slot, or the pair's (Re x, Im x) for the member with
            // Im(lambda) > 0 (x = yr + i yi when the Re column's quotient has Im >= 0,
            // its conjugate otherwise), both scaled by the complex norm
            bool pair = sl.partner[o] != o;
            int cr = pair ? std::min(o, sl.partner[o]) : o, ci = pair ? cr + 1 : o;
            double nrm2 = 0;
            for (int64_t i = 0; i < n; ++i) {
                double a = Yh[(size_t)cr * n + i];
                nrm2 += a * a;
                if (pair) {
                    double b = Yh[(size_t)ci * n + i];
                    nrm2 += b * b;
                }
            }
            double sc = 1.0 / std::sqrt(nrm2);
            if (!pair) {
                for (int64_t i = 0; i < n; ++i) X[(size_t)s * n + i] = Yh[(size_t)o * n + i] * sc;
            } else {
                bool first = lim[o] > 0 || (lim[o] == 0 && o == cr);
                double sgn = (lim[cr] >= 0) ? 1.0 : -1.0;
                const double *src = first ? &Yh[(size_t)cr * n] : &Yh[(size_t)ci * n];
                double f = first ? sc : sgn * sc;
                for (int64_t i = 0; i < n; ++i) X[(size_t)s * n + i] = src[i] * f;
            }
        }
    }
    *nout = nw;
    S.converged = converged ? 1 : 0;
    S.max_resid = maxres;
    S.kernel_launches = c->launches - launches0;
    S.t_total = now() - t_start;
    if (stats) *stats = S;
    if (!converged) return pp_fail(PP_ENOTCONV, "pp_eigs: not converged in %lld cycles", (long long)S.cycles);
    return PP_OK;
}
