// Per-instance Arnoldi driver pieces shared by pp_eigs (one instance) and the
// batched engine: the wanted-set selection and thick restart of Section 4,
// the FP64 Ritz test on A, and the FP64 refinement of the mixed-precision mode.
#pragma once

#include <thread>

#include "ctx.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace ppi {

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

// Ritz values of H_m (host FP64), the wanted set (nev slots, one more when a
// conjugate pair would split) and its Ritz vectors' coefficients (Section 4).
struct Cycle {
    int m = 0;
    std::vector<double> Hm, wr, wi, Sv, Sw;
    std::vector<cd> nu;
    std::vector<int> order;
    Slots sl;
    bool harmonic = false;
    std::vector<double> cvec;  // harmonic: [-h f; 1], the direction of every harmonic residual
};

struct Driver {
    pp_ctx *c;
    int64_t n, ldv;
    int wcap;
    std::vector<void *> mine;
    // FP64 test buffers
    double *Y64 = nullptr, *AY64 = nullptr;
    double *dQ = nullptr, *dq = nullptr, *dmu = nullptr;
    int *dpartner = nullptr;
    // refinement
    double *Z = nullptr, *dG = nullptr, *Yb = nullptr;
    double *Ye = nullptr, *dQe = nullptr;  // extra Ritz vectors of the refinement and their coefficients
    static constexpr int kZcap = 128;

    ~Driver() {
        cudaStreamSynchronize(c->stream);
        for (void *q : mine) ws_put(c, q);
    }
    pp_status alloc(void **p, size_t bytes) {
        pp_status st = ws_get(c, p, bytes);
        if (st >= 0) mine.push_back(*p);
        return st;
    }

    // Buffers of the FP64 Ritz test (and the storage-precision Ritz vectors in
    // mixed mode).  The refinement basis is allocated when first needed, unless
    // the caller supplies a shared one (Z, dG).
    pp_status alloc_test_buffers(bool mixed) {
        CKS(alloc((void **)&Y64, (size_t)ldv * (wcap + 1) * 8));
        CKS(alloc((void **)&AY64, (size_t)ldv * (wcap + 1) * 8));
        CKS(alloc((void **)&dQ, (size_t)kZcap * kZcap * 8));
        CKS(alloc((void **)&dq, (size_t)4 * (wcap + 1) * 8));
        CKS(alloc((void **)&dmu, (size_t)3 * (wcap + 1) * 8));
        CKS(alloc((void **)&dpartner, (size_t)(wcap + 1) * 4));
        CKS(ensure_part(c, std::max(ppk::cgs_part_doubles(ppk::cgs_grid((int)n)), (size_t)(wcap + 1) * 3 * 1024)));
        return PP_OK;
    }

    // Y64 = B S (B: mcols columns of precision pb), then FP64 Rayleigh quotients
    // and residual norms on A for each slot.
    pp_status ritz_test(const void *B, ppk::Prec pb, int mcols, const std::vector<double> &Sw, const Slots &sl,
                        double rtol, RitzOut &out, pp_stats &S) {
        const int nw = sl.nw;
        CK(cudaMemcpyAsync(dQ, Sw.data(), Sw.size() * 8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(dpartner, sl.partner.data(), nw * 4, cudaMemcpyHostToDevice, c->stream));
        // FP64 arithmetic and output whatever the basis precision
        ppk::launch_rotate64(pb, (int)n, B, ldv, mcols, dQ, nw, Y64, ldv, c->stream);
        CKS(check_launch(c));
        if (c->d_bal) {  // balanced: Ritz vectors of S mapped to A's coordinates, x = D y
            ppk::launch_scale_rows((int)n, nw, Y64, ldv, Y64, ldv, c->d_bal, false, c->stream);
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

    // Value of the Arnoldi operator's polynomial at an eigenvalue estimate mu of
    // A: pi(mu - sigma), pi_2(1 - pi_1(mu - sigma)) for a double polynomial, or
    // mu - sigma without one (the operator is then A - sigma I itself).
    cd op_value(const pp_poly *p, cd mu) const {
        const cd z = mu - c->sigma;
        if (!p) return z;
        auto prod = [](const std::vector<cd> &roots, cd x) {
            cd v = 1.0;
            for (const cd &t : roots) v *= 1.0 - x / t;
            return v;
        };
        if (p->inner) return prod(p->roots, 1.0 - prod(p->inner->roots, z));
        return prod(p->roots, z);
    }

    // Extra Ritz vectors carried by the refinement besides the wanted ones: the
    // next ones in the Arnoldi's order.  When the boundary of the wanted set
    // falls inside a cluster that FP32 cannot resolve (eigenvalues closer than
    // u_32 ||A||), only a space holding the whole cluster lets Rayleigh-Ritz
    // separate the wanted members from their neighbours.
    static int refine_extra(int nev, int m, int nw) { return std::max(0, std::min(std::min(nev + 2, m - nw - 1), 32)); }

    // FP64 refinement on A (mixed precision): Rayleigh-Ritz of A itself on a
    // search space built in FP64 from the wanted Ritz vectors Y and, from the
    // second round on (with the polynomial), `extra` further Ritz vectors of the
    // cycle.  With an FP64 copy of the operator the space is span{pi(A) Y}, then
    // span{pi(A) [Y, Y_e]} (pi_1(A) for a double
    // polynomial): the polynomial keeps the wanted part and damps the FP32
    // rounding noise in the unwanted part of the spectrum (one step of subspace
    // iteration).  Without one it is the block Krylov space span{Y, A Y, ...,
    // A^s Y}.  The refined Ritz pairs are ranked as the Arnoldi ranks its Ritz
    // values (distance of the operator's value to its target), the first nev
    // slots replace the wanted ones and the next ones the extras, for up to
    // `rounds` rounds; a round that does not lower the largest residual is
    // undone and ends the refinement (the first one only when no extras
    // follow), so the estimates never get worse.  A
    // failed dense eigensolve or too few candidates also end it.
    // cy, V (mcols columns of precision pb): the cycle the extras come from
    // (may be null: no extras).
    pp_status refine(const pp_poly *p, Slots &sl, int nev, RitzOut &R, double rtol, int steps, int rounds,
                     pp_stats &S, const Cycle *cy = nullptr, const void *V = nullptr, ppk::Prec pb = ppk::F64,
                     int mcols = 0) {
        if (!Z) CKS(alloc((void **)&Z, (size_t)ldv * (kZcap + 1) * 8));
        if (!dG) CKS(alloc((void **)&dG, (size_t)(kZcap + 1) * kZcap * 8));
        if (!Yb) CKS(alloc((void **)&Yb, (size_t)ldv * (wcap + 1) * 8));
        pp_ctx *tw = p ? fp64_context(c->twin) : nullptr;
        // the filter: pi itself, or for a double polynomial its inner factor pi_1
        // (degree d1 instead of d1 d2: it damps the same unwanted part, less
        // sharply, at a d2-th of the FP64 passes)
        const pp_poly *pf = (p && p->inner) ? p->inner : p;
        steps = std::max(1, std::min(steps, kZcap / (nev + 1) - 1));
        const int ldg = kZcap + 1;
        double *W = AY64 + (size_t)(nev + 1) * ldv;  // spare FP64 column (context vectors are FP32 here)
        // extra Ritz vectors of the cycle (with the polynomial and its FP64 copy)
        // extra Ritz vectors of the cycle (with the polynomial and its FP64 copy);
        // the first round goes without them (they double its cost and the wanted
        // vectors alone usually suffice), the following rounds carry them
        int ne = 0;
        const int extra = (tw && cy && V) ? refine_extra(nev, cy->m, sl.nw) : 0;
        auto cycle_extras = [&]() -> pp_status {
            ne = 0;
            if (!Ye) CKS(alloc((void **)&Ye, (size_t)ldv * 32 * 8));
            if (!dQe) CKS(alloc((void **)&dQe, (size_t)kZcap * kZcap * 8));
            std::vector<double> Se;
            const int m = cy->m;
            for (int q = sl.nw; q < m && ne < extra;) {
                const int i = cy->order[q];
                if (cy->wi[i] == 0.0) {
                    Se.insert(Se.end(), &cy->Sv[(size_t)i * m], &cy->Sv[(size_t)i * m] + m);
                    ne += 1;
                    q += 1;
                } else {
                    if (ne + 2 > extra) break;
                    const int base = cy->wi[i] > 0 ? i : i - 1;
                    Se.insert(Se.end(), &cy->Sv[(size_t)base * m], &cy->Sv[(size_t)base * m] + 2 * m);
                    ne += 2;
                    q += 2;
                }
            }
            if (ne) {
                CK(cudaMemcpyAsync(dQe, Se.data(), Se.size() * 8, cudaMemcpyHostToDevice, c->stream));
                ppk::launch_rotate64(pb, (int)n, V, ldv, mcols, dQe, ne, Ye, ldv, c->stream);
                CKS(check_launch(c));
                S.vops += (int64_t)mcols * ne;
            }
            return PP_OK;
        };
        // Y64 holds vectors of A's coordinates (x = D y when balanced): the search
        // space lives in the coordinates of the operator's matrix S (= A unbalanced)
        double *U = AY64;  // spare FP64 column while the space is built
        auto to_operator = [&](const double *y) -> const double * {
            if (!c->d_bal) return y;
            ppk::launch_scale_rows((int)n, 1, y, ldv, U, ldv, c->d_bal, true, c->stream);
            return U;
        };
        auto project = [&](int col, int nz) -> pp_status {  // G[:, col] = Z^T S z_col
            ppk::StepArgs a;
            a.x = Z + (size_t)col * ldv;
            a.y = W;
            a.plain = 1;
            ppk::launch_step(c->S64, a, c->stream);
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
            ca.err = c->err();
            ppk::launch_cgs(ppk::F64, ca, c->stream);
            CKS(check_launch(c));
            S.mvps += 1;
            S.dots += nz;
            S.vops += nz;
            return PP_OK;
        };
        // the best state so far (the input): slots, residuals and Y
        Slots sl_best = sl;
        RitzOut R_best = R;
        double best = R.res.empty() ? INFINITY : *std::max_element(R.res.begin(), R.res.end());
        CK(cudaMemcpyAsync(Yb, Y64, (size_t)ldv * sl.nw * 8, cudaMemcpyDeviceToDevice, c->stream));
        for (int round = 0; round < rounds; ++round) {
            const int nw = sl.nw;  // the wanted slots of this round (the layout may change)
            int nz = 0;
            CK(cudaMemsetAsync(dG, 0, (size_t)ldg * kZcap * 8, c->stream));
            if (tw) {
                for (int s = 0; s < nw + ne; ++s) {
                    const double *y = s < nw ? to_operator(Y64 + (size_t)s * ldv) : Ye + (size_t)(s - nw) * ldv;
                    CKS(check_launch(c));
                    CKS(op_apply(tw, pf, y, W));
                    CKS(cgs2_step(c, ppk::F64, Z, ldv, nz, W, c->d_small + 2048));
                    S.dots += 2 * nz + 1;
                    S.vops += 4 * nz + 2;
                    nz++;
                }
                S.mvps += op_mvps(pf) * (nw + ne);
                for (int col = 0; col < nz; ++col) CKS(project(col, nz));
            } else {
                for (int s = 0; s < nw; ++s) {
                    const double *y = to_operator(Y64 + (size_t)s * ldv);
                    CK(cudaMemcpyAsync(W, y, n * 8, cudaMemcpyDeviceToDevice, c->stream));
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
                        ppk::launch_step(c->S64, a, c->stream);
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
                // the Arnoldi coefficients gave G's first columns; the last block's remain
                for (int col = b0; col < b1; ++col) CKS(project(col, nz));
            }
            std::vector<double> Gfull((size_t)ldg * nz), G((size_t)nz * nz);
            CK(cudaMemcpyAsync(Gfull.data(), dG, Gfull.size() * 8, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            CKS(check_sweeps(c));
            for (int j = 0; j < nz; ++j)
                for (int i = 0; i < nz; ++i) G[i + (size_t)j * nz] = Gfull[i + (size_t)j * ldg];
            for (double v : G)
                if (!std::isfinite(v)) return PP_OK;
            std::vector<double> wr(nz), wi(nz), Sv((size_t)nz * nz);
            if (!ppd::dense_eig(nz, G.data(), nz, wr.data(), wi.data(), Sv.data(), nz)) return PP_OK;
            // the refined Ritz values (a conjugate pair as one unit, its Im > 0
            // member) ranked as the Arnoldi ranks its Ritz values: by the
            // distance of the operator's value at them to its target (FP32 may
            // have shown a pair where FP64 resolves two real values, so the slot
            // layout is rebuilt); the first nev slots are the wanted set, the
            // next ones (up to ne columns) the extras of the next round
            std::vector<int> units;
            std::vector<cd> nuv;
            for (int i = 0; i < nz; ++i) {
                if (wi[i] < 0) continue;
                units.push_back(i);
                nuv.push_back(op_value(p, cd(wr[i], wi[i])));
            }
            const std::vector<int> ord = ppd::ritz_order(nuv, p ? 1.0 : 0.0);
            Slots ns;
            std::vector<int> pick, pick_e;
            int nxe = 0;
            for (int q : ord) {
                const int i = units[q];
                const int w = wi[i] != 0.0 ? 2 : 1;
                if (ns.nw < nev) {
                    pick.push_back(i);
                    ns.nw += w;
                } else if (nxe + w <= ne) {
                    pick_e.push_back(i);
                    nxe += w;
                }
            }
            if (ns.nw < nev) return PP_OK;
            ns.partner.assign(ns.nw, 0);
            ns.sg.assign(ns.nw, 0.0);
            std::vector<double> Sw((size_t)nz * ns.nw), Swe;
            int s = 0;
            for (int i : pick) {
                std::copy(&Sv[(size_t)i * nz], &Sv[(size_t)i * nz] + nz, &Sw[(size_t)s * nz]);
                if (wi[i] == 0.0) {
                    ns.partner[s] = s;
                    s += 1;
                } else {
                    std::copy(&Sv[(size_t)(i + 1) * nz], &Sv[(size_t)(i + 1) * nz] + nz, &Sw[(size_t)(s + 1) * nz]);
                    ns.partner[s] = s + 1;
                    ns.partner[s + 1] = s;
                    ns.sg[s] = 1.0;
                    ns.sg[s + 1] = -1.0;
                    s += 2;
                }
            }
            for (int i : pick_e) Swe.insert(Swe.end(), &Sv[(size_t)i * nz], &Sv[(size_t)i * nz] + (size_t)nz * (wi[i] != 0.0 ? 2 : 1));
            sl = ns;
            CKS(ritz_test(Z, ppk::F64, nz, Sw, sl, rtol, R, S));
            S.vops += (int64_t)nz * nw;
            if (trace_refine())
                std::fprintf(stderr, "[pp] refine %p round %d space %d max_resid %.3e nconv %d\n", (void *)this, round,
                             nz, *std::max_element(R.res.begin(), R.res.end()), R.nconv);
            if (R.all) return PP_OK;
            const double mx = *std::max_element(R.res.begin(), R.res.end());
            if (round == 0 && extra > 0) {
                // the second round adds the cycle's next Ritz vectors to the best wanted ones
                if (mx < best) {
                    best = mx;
                    sl_best = sl;
                    R_best = R;
                    CK(cudaMemcpyAsync(Yb, Y64, (size_t)ldv * sl.nw * 8, cudaMemcpyDeviceToDevice, c->stream));
                } else {
                    sl = sl_best;
                    R = R_best;
                    CK(cudaMemcpyAsync(Y64, Yb, (size_t)ldv * sl.nw * 8, cudaMemcpyDeviceToDevice, c->stream));
                }
                CKS(cycle_extras());
                continue;
            }
            if (!(mx < best)) break;
            best = mx;
            sl_best = sl;
            R_best = R;
            CK(cudaMemcpyAsync(Yb, Y64, (size_t)ldv * sl.nw * 8, cudaMemcpyDeviceToDevice, c->stream));
            // the next round's extras: the following refined Ritz vectors
            ne = nxe;
            if (ne) {
                CK(cudaMemcpyAsync(dQe, Swe.data(), Swe.size() * 8, cudaMemcpyHostToDevice, c->stream));
                ppk::launch_rotate64(ppk::F64, (int)n, Z, ldv, nz, dQe, ne, Ye, ldv, c->stream);
                CKS(check_launch(c));
                S.vops += (int64_t)nz * ne;
            }
        }
        // undo the last round if it did not improve
        const double mx = R.res.empty() ? INFINITY : *std::max_element(R.res.begin(), R.res.end());
        if (!(mx <= best)) {
            sl = sl_best;
            R = R_best;
            CK(cudaMemcpyAsync(Y64, Yb, (size_t)ldv * sl.nw * 8, cudaMemcpyDeviceToDevice, c->stream));
        }
        return PP_OK;
    }
    static bool trace_refine() {
        static const bool on = std::getenv("PP_TRACE") != nullptr;
        return on;
    }
};


// Per-cycle trace on stderr when the environment sets PP_TRACE (diagnostics
// only: the arithmetic is the same either way).
inline bool trace_on() {
    static const bool on = std::getenv("PP_TRACE") != nullptr;
    return on;
}
inline void trace_cycle(const char *who, const void *id, int64_t cycle, int prec_bits, const RitzOut &R,
                        const char *event) {
    if (!trace_on()) return;
    double mx = R.res.empty() ? 0.0 : *std::max_element(R.res.begin(), R.res.end());
    std::fprintf(stderr, "[pp] %s %p cycle %lld fp%d max_resid %.3e nconv %d %s\n", who, id, (long long)cycle,
                 prec_bits, mx, R.nconv, event ? event : "");
}

// When the FP32 cycles of the mixed mode hand over to the FP64 refinement:
// within 50 rtol (the refinement with its extra Ritz vectors gains one to two
// orders of magnitude); at the FP32 floor (below 1e-6 and no longer halving
// per cycle); after two cycles without halving at any level (an operator too
// non-normal for FP32, or an FP32 apply swamped by the growth of the partial
// products of a high-degree polynomial); or at the last cycle.
struct MixedSwitch {
    double rtol, best = INFINITY;
    int stall = 0;
    explicit MixedSwitch(double r) : rtol(r) {}
    bool should_refine(const RitzOut &R, bool last_cycle) {
        double mx = *std::max_element(R.res.begin(), R.res.end());
        stall = (mx < 0.5 * best) ? 0 : stall + 1;
        best = std::min(best, mx);
        if (last_cycle || mx <= 50 * rtol) return true;
        if (mx <= std::max(rtol, 1e-6) && stall >= 1) return true;
        return stall >= 2;
    }
    // after a refinement that missed rtol, keep cycling in FP32 from here
    void reset() {
        stall = 0;
        best = INFINITY;
    }
};


// With harmonic set, the values are the harmonic Ritz values with respect to
// the target t: eigenvalues of K = H_m + h^2 f e_m^T, f = (H_m - t I)^{-T} e_m,
// h = h_{m+1,m} (Example 2's harmonic Arnoldi; the Galerkin condition
// (Op - t) y - (theta - t) y orthogonal to (Op - t) V_m).
inline pp_status wanted_set(const std::vector<double> &H, int ldh, int m, int nev, double target, Cycle &cy,
                            bool harmonic = false) {
    cy.m = m;
    cy.harmonic = harmonic;
    cy.Hm.assign((size_t)m * m, 0.0);
    cy.wr.assign(m, 0.0);
    cy.wi.assign(m, 0.0);
    cy.Sv.assign((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) cy.Hm[i + (size_t)j * m] = H[i + (size_t)j * ldh];
    for (double v : cy.Hm)
        if (!std::isfinite(v)) return pp_fail(PP_ENUMERIC, "non-finite Hessenberg entry");
    std::vector<double> Hc = cy.Hm;
    if (harmonic) {
        const double h = H[m + (size_t)(m - 1) * ldh];
        std::vector<double> Mt((size_t)m * m);
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) Mt[i + (size_t)j * m] = cy.Hm[j + (size_t)i * m] - (i == j ? target : 0.0);
        std::vector<double> f(m, 0.0);
        f[m - 1] = 1.0;
        if (!ppd::lu_solve(m, Mt, f.data()))
            return pp_fail(PP_ENUMERIC, "harmonic Ritz values: H_m - t I is singular");
        for (int i = 0; i < m; ++i) Hc[i + (size_t)(m - 1) * m] += h * h * f[i];
        cy.cvec.assign(m + 1, 1.0);
        for (int i = 0; i < m; ++i) cy.cvec[i] = -h * f[i];
    }
    if (!ppd::dense_eig(m, Hc.data(), m, cy.wr.data(), cy.wi.data(), cy.Sv.data(), m))
        return pp_fail(PP_ENUMERIC, "Ritz values: QR failed");
    cy.nu.resize(m);
    for (int i = 0; i < m; ++i) cy.nu[i] = cd(cy.wr[i], cy.wi[i]);
    cy.order = ppd::ritz_order(cy.nu, target);
    Slots &sl = cy.sl;
    sl.nw = nev + (cy.nu[cy.order[nev - 1]].imag() > 0 ? 1 : 0);
    sl.partner.assign(sl.nw, 0);
    sl.sg.assign(sl.nw, 0.0);
    cy.Sw.assign((size_t)m * sl.nw, 0.0);
    const auto &Sv = cy.Sv;
    for (int s = 0; s < sl.nw;) {
        int i = cy.order[s];
        if (cy.wi[i] == 0.0) {
            std::copy(&Sv[(size_t)i * m], &Sv[(size_t)i * m] + m, &cy.Sw[(size_t)s * m]);
            sl.partner[s] = s;
            s += 1;
        } else {
            int base = cy.wi[i] > 0 ? i : i - 1;
            std::copy(&Sv[(size_t)base * m], &Sv[(size_t)base * m] + m, &cy.Sw[(size_t)s * m]);
            std::copy(&Sv[(size_t)(base + 1) * m], &Sv[(size_t)(base + 1) * m] + m, &cy.Sw[(size_t)(s + 1) * m]);
            sl.partner[s] = s + 1;
            sl.partner[s + 1] = s;
            sl.sg[s] = 1.0;
            sl.sg[s + 1] = -1.0;
            s += 2;
        }
    }
    return PP_OK;
}

// Harmonic restart: from the kept coefficients Q (m x kk, orthonormal), the
// rotation P = [[Q; 0], p] ((m+1) x (kk+1), p = c orthogonalised against
// [Q; 0] twice and normalised) and Hn = P^T Hbar Q ((kk+1) x kk leading block
// of an ldh x m array), Hbar = [H_m; h e_m^T].  Q is replaced by P.
inline int harmonic_basis(const Cycle &cy, const std::vector<double> &H, int ldh, int kk, std::vector<double> &Q,
                          std::vector<double> &Hn) {
    const int m = cy.m, m1 = m + 1;
    std::vector<double> P((size_t)m1 * (kk + 1), 0.0);
    for (int cc = 0; cc < kk; ++cc)
        for (int r = 0; r < m; ++r) P[r + (size_t)cc * m1] = Q[r + (size_t)cc * m];
    std::vector<double> p = cy.cvec;
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<double> proj(kk, 0.0);
        for (int cc = 0; cc < kk; ++cc)
            for (int r = 0; r < m1; ++r) proj[cc] += P[r + (size_t)cc * m1] * p[r];
        for (int cc = 0; cc < kk; ++cc)
            for (int r = 0; r < m1; ++r) p[r] -= P[r + (size_t)cc * m1] * proj[cc];
    }
    double nrm = 0;
    for (double v : p) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (int r = 0; r < m1; ++r) P[r + (size_t)kk * m1] = p[r] / nrm;
    // Hbar Q: (m+1) x kk
    std::vector<double> HQ((size_t)m1 * kk, 0.0);
    for (int cc = 0; cc < kk; ++cc)
        for (int r = 0; r < m1; ++r) {
            double s = 0;
            for (int t = 0; t < m; ++t) s += H[r + (size_t)t * ldh] * Q[t + (size_t)cc * m];
            HQ[r + (size_t)cc * m1] = s;
        }
    Hn.assign((size_t)ldh * m, 0.0);
    for (int cc = 0; cc < kk; ++cc)
        for (int r = 0; r <= kk; ++r) {
            double s = 0;
            for (int t = 0; t < m1; ++t) s += P[t + (size_t)r * m1] * HQ[t + (size_t)cc * m1];
            Hn[r + (size_t)cc * ldh] = s;
        }
    Q.swap(P);
    return kk;
}

// Thick restart (Section 4): keep k Ritz vectors (k - 1 when a pair would
// split), Q = qr([Re, Im] of their coefficients), Hn = [Q^T H_m Q ; h e_m^T Q].
// A harmonic cycle continues in harmonic_basis (Q becomes the (m+1) x (kk+1) P).
inline int restart_basis(const Cycle &cy, const std::vector<double> &H, int ldh, int k, std::vector<double> &Q,
                         std::vector<double> &Hn) {
    const int m = cy.m;
    const auto &Sv = cy.Sv;
    int kk = (cy.nu[cy.order[k - 1]].imag() > 0) ? k - 1 : k;
    std::vector<double> B((size_t)m * kk);
    int col = 0;
    for (int s = 0; s < kk; ++s) {
        int i = cy.order[s];
        if (cy.wi[i] == 0.0) {
            std::copy(&Sv[(size_t)i * m], &Sv[(size_t)i * m] + m, &B[(size_t)col * m]);
            col++;
        } else if (cy.wi[i] > 0) {
            std::copy(&Sv[(size_t)i * m], &Sv[(size_t)i * m] + m, &B[(size_t)col * m]);
            std::copy(&Sv[(size_t)(i + 1) * m], &Sv[(size_t)(i + 1) * m] + m, &B[(size_t)(col + 1) * m]);
            col += 2;
        }
    }
    Q.assign((size_t)m * kk, 0.0);
    ppd::thin_qr(m, kk, B.data(), Q.data());
    if (cy.harmonic) return harmonic_basis(cy, H, ldh, kk, Q, Hn);
    std::vector<double> HQ((size_t)m * kk, 0.0);
    Hn.assign((size_t)ldh * m, 0.0);
    for (int cc = 0; cc < kk; ++cc)
        for (int r = 0; r < m; ++r) {
            double s = 0;
            for (int t = 0; t < m; ++t) s += cy.Hm[r + (size_t)t * m] * Q[t + (size_t)cc * m];
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
    return kk;
}

// Outputs sorted by the target (SR: Re, |Im|, Im > 0 first; SM: |lam|, Re, Im > 0
// first); X gets unit vectors (a pair's Re, Im columns scaled by its complex norm).
inline void write_outputs(int target, int64_t n, const Slots &sl, const RitzOut &R, const std::vector<double> &Yh,
                          double *lam_re, double *lam_im, double *resid, double *X, double &maxres,
                          std::vector<int> *order = nullptr) {
    const int nw = sl.nw;
    std::vector<int> srt(nw);
    for (int s = 0; s < nw; ++s) srt[s] = s;
    const auto &lre = R.lre, &lim = R.lim;
    bool sr = target == PP_TARGET_SR;
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
    if (order) *order = srt;
    maxres = 0;
    for (int s = 0; s < nw; ++s) {
        int o = srt[s];
        lam_re[s] = lre[o];
        lam_im[s] = lim[o];
        resid[s] = R.res[o];
        maxres = std::max(maxres, R.res[o]);
        if (X) {
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
}

// Fault in the pages of a large host buffer with several threads (one write
// per 4 KB page).  A device-to-host copy into pages never touched is slow: the
// copy then takes every page fault itself.
inline void touch_pages(void *p, size_t bytes) {
    char *b = (char *)p;
    const size_t page = 4096;
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt < 1 ? 1 : (nt > 16 ? 16 : nt);
    if (bytes < ((size_t)16 << 20)) nt = 1;
    const size_t chunk = (bytes / nt + page - 1) / page * page;
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
        const size_t lo = t * chunk, hi = std::min(bytes, lo + chunk);
        if (lo >= hi) break;
        th.emplace_back([b, lo, hi, page]() {
            for (size_t off = lo; off < hi; off += page) b[off] = 0;
        });
    }
    for (auto &x : th) x.join();
}

// The eigenvector block of write_outputs formed on the device and copied once
// into the caller's X: slot s (in the sorted order) is the column of Y (FP64,
// leading dimension ld) scaled to unit (complex) norm, the columns of a pair
// being its Re and Im parts (Im sign as in write_outputs).  Xd: FP64 device
// scratch of ld x nw.  The norms are summed on the device.
inline pp_status vectors_out(pp_ctx *c, int64_t n, const Slots &sl, const RitzOut &R, const double *Y, int64_t ld,
                             const std::vector<int> &srt, double *Xd, double *X) {
    const int nw = sl.nw;
    double *nrm = c->d_small + 3200;  // 2 per slot
    CK(cudaMemsetAsync(nrm, 0, (size_t)2 * nw * sizeof(double), c->stream));
    for (int s = 0; s < nw; ++s) {
        const int o = srt[s];
        const bool pair = sl.partner[o] != o;
        const int cr = pair ? std::min(o, sl.partner[o]) : o, ci = pair ? cr + 1 : o;
        ppk::launch_norm2((int)n, Y + (size_t)cr * ld, c->d_part, c->d_ticket, nrm + 2 * s, c->stream);
        CKS(check_launch(c));
        if (pair) {
            ppk::launch_norm2((int)n, Y + (size_t)ci * ld, c->d_part, c->d_ticket, nrm + 2 * s + 1, c->stream);
            CKS(check_launch(c));
        }
        const bool first = !pair || R.lim[o] > 0 || (R.lim[o] == 0 && o == cr);
        const double sgn = (pair && !first && R.lim[cr] < 0) ? -1.0 : 1.0;
        const double *src = (!pair || first) ? Y + (size_t)(pair ? cr : o) * ld : Y + (size_t)ci * ld;
        ppk::launch_slot_scale((int)n, src, nrm + 2 * s, sgn, Xd + (size_t)s * ld, c->stream);
        CKS(check_launch(c));
    }
    touch_pages(X, (size_t)n * nw * sizeof(double));  // while the device scales
    CK(cudaMemcpy2DAsync(X, (size_t)n * 8, Xd, (size_t)ld * 8, (size_t)n * 8, nw, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return PP_OK;
}

}  // namespace ppi
