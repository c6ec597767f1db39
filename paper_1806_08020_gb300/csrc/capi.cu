// C-ABI entry points: contexts, polynomial construction (Section 2 box,
// Section 7 box, Section 8), the factored apply (Eq. (2.1)) and
// thick-restarted Arnoldi(m, k) on pi(A) (Section 2 box step 2, Section 4).
//
// The Arnoldi process runs entirely on the device: each step applies the
// operator with fused root-step kernels, orthogonalises with three CGS2
// passes that write the Hessenberg column on the device, and normalises.
// The host synchronises once per polynomial build and once per cycle, where
// the small dense FP64 steps run (harmonic Ritz roots, Leja order, Ritz
// values, restart basis).
#include "ctx.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <vector>


static thread_local std::string g_last_error;

pp_status pp_fail(pp_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

namespace ppi {

pp_status dmalloc(pp_ctx *c, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pp_fail(PP_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    return PP_OK;
}

void dfree(pp_ctx *c, void *p) {
    if (!p) return;
    cudaFree(p);
    c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), p), c->allocs.end());
}

pp_status ws_get(pp_ctx *c, void **p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    int best = -1;
    for (size_t i = 0; i < c->ws_spare.size(); ++i) {
        const size_t s = c->ws_spare[i].second;
        if (s >= bytes && s - bytes <= bytes / 4 && (best < 0 || s < c->ws_spare[best].second)) best = (int)i;
    }
    if (best >= 0) {
        *p = c->ws_spare[best].first;
        c->ws_live.push_back(c->ws_spare[best]);
        c->ws_spare.erase(c->ws_spare.begin() + best);
        return PP_OK;
    }
    CKS(dmalloc(c, p, bytes));
    c->ws_live.push_back({*p, bytes});
    return PP_OK;
}

void ws_put(pp_ctx *c, void *p) {
    for (size_t i = 0; i < c->ws_live.size(); ++i)
        if (c->ws_live[i].first == p) {
            c->ws_spare.push_back(c->ws_live[i]);
            c->ws_live.erase(c->ws_live.begin() + i);
            return;
        }
    dfree(c, p);
}

void ws_trim(pp_ctx *c) {
    if (c->ws_spare.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto &b : c->ws_spare) dfree(c, b.first);
    c->ws_spare.clear();
}

pp_status check_launch(pp_ctx *c) {
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return PP_OK;
}

// One pass: y/r/oy per StepArgs on matrix A.
pp_status step(pp_ctx *c, const ppk::StepArgs &s) {
    ppk::launch_step(c->A, s, c->stream);
    return check_launch(c);
}

// y = pi(A - sigma I) x with the steps in order; scratch: vec[0], vec[1], vec[2].
pp_status apply_single(pp_ctx *c, const std::vector<StepCoef> &st, const void *x, void *y) {
    const void *cur = x;
    void *P0 = c->vec[0], *P1 = c->vec[1], *T = c->vec[2];
    for (size_t i = 0; i < st.size(); ++i) {
        bool last = (i + 1 == st.size());
        void *dst = (cur == P0) ? P1 : P0;
        if (last && y != cur) dst = y;
        ppk::StepArgs a;
        a.sigma = c->sigma;
        if (!st[i].pair) {
            a.x = cur;
            a.y = dst;
            a.a2 = st[i].c;
        } else {
            ppk::StepArgs t;
            t.sigma = c->sigma;
            t.x = cur;
            t.y = T;
            t.plain = 1;
            CKS(step(c, t));
            a.x = T;
            a.aux = cur;
            a.y = dst;
            a.a1 = st[i].c1;
            a.a2 = -st[i].c2;
        }
        CKS(step(c, a));
        cur = dst;
    }
    if (cur != y) CK(cudaMemcpyAsync(y, cur, c->n * c->esz, cudaMemcpyDeviceToDevice, c->stream));
    return PP_OK;
}

// r = tau(A) u = u - pi_1(A) u as the running sum of pi_1's factors; the optional
// outer epilogue writes oy = obase - (b1 ox + b2 r) in the last pass.
// Scratch: vec[3], vec[4], vec[5].
pp_status apply_tau(pp_ctx *c, const std::vector<StepCoef> &st, const void *u, void *r, bool r_write,
                    const void *obase, const void *ox, void *oy, double b1, double b2) {
    const void *cur = u;
    void *P0 = c->vec[3], *P1 = c->vec[4], *T = c->vec[5];
    for (size_t i = 0; i < st.size(); ++i) {
        bool last = (i + 1 == st.size());
        void *dst = (cur == P0) ? P1 : P0;
        ppk::StepArgs a;
        a.sigma = c->sigma;
        a.r = r;
        a.r_init = (i == 0);
        a.r_write = (!last || r_write) ? 1 : 0;
        a.y = last ? nullptr : dst;
        if (last && oy) {
            a.obase = obase;
            a.ox = ox;
            a.oy = oy;
            a.b1 = b1;
            a.b2 = b2;
        }
        if (!st[i].pair) {
            a.x = cur;
            a.a2 = st[i].c;
        } else {
            ppk::StepArgs t;
            t.sigma = c->sigma;
            t.x = cur;
            t.y = T;
            t.plain = 1;
            CKS(step(c, t));
            a.x = T;
            a.aux = cur;
            a.a1 = st[i].c1;
            a.a2 = -st[i].c2;
        }
        CKS(step(c, a));
        cur = dst;
    }
    return PP_OK;
}

// y = pi_2(tau(A)) x.  Outer scratch: vec[6], vec[7], vec[2] (t) and vec[1] (r).
pp_status apply_double(pp_ctx *c, const pp_poly *p, const void *x, void *y) {
    const auto &outer = p->steps;
    const auto &inner = p->inner->steps;
    const void *cur = x;
    void *O0 = c->vec[6], *O1 = c->vec[7], *OT = c->vec[2], *R = c->vec[1];
    for (size_t i = 0; i < outer.size(); ++i) {
        bool last = (i + 1 == outer.size());
        void *dst = (cur == O0) ? O1 : O0;
        if (last && y != cur) dst = y;
        if (!outer[i].pair) {
            // dst = cur - tau(cur)/eta, fused into the last inner pass
            CKS(apply_tau(c, inner, cur, R, false, cur, nullptr, dst, 0.0, outer[i].c));
        } else {
            // t = tau(cur); dst = cur - c1 t + c2 tau(t)
            CKS(apply_tau(c, inner, cur, OT, true, nullptr, nullptr, nullptr, 0, 0));
            CKS(apply_tau(c, inner, OT, R, false, cur, OT, dst, outer[i].c1, -outer[i].c2));
        }
        cur = dst;
    }
    if (cur != y) CK(cudaMemcpyAsync(y, cur, c->n * c->esz, cudaMemcpyDeviceToDevice, c->stream));
    return PP_OK;
}

// y = Op(x): plain A - sigma I when p == nullptr, pi(A), or pi_2(tau(A)).
pp_status op_apply(pp_ctx *c, const pp_poly *p, const void *x, void *y) {
    if (!p) {
        ppk::StepArgs a;
        a.sigma = c->sigma;
        a.x = x;
        a.y = y;
        a.plain = 1;
        return step(c, a);
    }
    if (p->inner) return apply_double(c, p, x, y);
    return apply_single(c, p->steps, x, y);
}

// tau(A) x into y (operator of the second GMRES in a double polynomial)
pp_status op_tau(pp_ctx *c, const pp_poly *inner, const void *x, void *y) {
    return apply_tau(c, inner->steps, x, y, true, nullptr, nullptr, nullptr, 0, 0);
}

int64_t op_mvps(const pp_poly *p) {
    if (!p) return 1;
    if (p->inner) {
        int64_t in = mvps_of(p->inner->steps);
        return in * mvps_of(p->steps);
    }
    return mvps_of(p->steps);
}

// vector operations per apply, counted as the oracle does: a real factor is
// two length-n updates (polynomial and running sum), a pair four
int64_t vops_of(const std::vector<StepCoef> &s) {
    int64_t v = 0;
    for (auto &x : s) v += x.pair ? 4 : 2;
    return v;
}

int64_t op_vops(const pp_poly *p) {
    if (!p) return 0;
    if (p->inner) return vops_of(p->steps) + (int64_t)mvps_of(p->steps) * vops_of(p->inner->steps);
    return vops_of(p->steps);
}

pp_status ensure_part(pp_ctx *c, size_t doubles) {
    if (doubles <= c->part_cap) return PP_OK;
    if (c->d_part) {
        cudaFree(c->d_part);
        c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), (void *)c->d_part), c->allocs.end());
    }
    c->d_part = nullptr;
    CKS(dmalloc(c, (void **)&c->d_part, doubles * sizeof(double)));
    c->part_cap = doubles;
    return PP_OK;
}

// CGS2 of w against V[:, 0..j) -> V[:, j] normalised, H[0..j, col] on the device.
pp_status cgs2_step(pp_ctx *c, ppk::Prec pr, void *V, int64_t ldv, int j, void *w, double *hcol) {
    return cgs2_step_n(c, pr, c->n, V, ldv, j, w, hcol);
}

pp_status cgs2_step_n(pp_ctx *c, ppk::Prec pr, int64_t n, void *V, int64_t ldv, int j, void *w, double *hcol) {
    double *h1 = c->d_small, *h2 = c->d_small + 256, *scal = c->d_small + 512, *nrm = c->d_small + 513;
    const size_t esz = pr == ppk::F64 ? 8 : (pr == ppk::F32 ? 4 : 2);
    ppk::CgsArgs a;
    a.n = (int)n;
    a.V = V;
    a.ldv = ldv;
    a.j = j;
    a.part = c->d_part;
    a.ticket = c->d_ticket;
    a.err = c->err();
    if (c->stall_sweeps > 0) {
        a.stall = 1;
        c->stall_sweeps--;
    }
    // pass 1: h1 = V^T w
    a.mode = 0;
    a.w = w;
    a.out = h1;
    ppk::launch_cgs(pr, a, c->stream);
    CKS(check_launch(c));
    // pass 2: w1 = w - V h1 (in place); h2 = V^T w1
    a.mode = 1;
    a.h = h1;
    a.wout = w;
    a.out = h2;
    ppk::launch_cgs(pr, a, c->stream);
    CKS(check_launch(c));
    // pass 3: w2 = w1 - V h2 -> V[:, j] (a BF16 basis: into w, then rounded once
    // when scaled into V[:, j]); H column; 1/||w2||
    a.mode = 2;
    a.h = h2;
    a.h1 = h1;
    void *vj = (char *)V + (size_t)j * ldv * esz;
    a.wout = pr == ppk::BF16 ? w : vj;
    a.out = nrm;
    a.hcol = hcol;
    a.scal = scal;
    ppk::launch_cgs(pr, a, c->stream);
    CKS(check_launch(c));
    if (pr == ppk::BF16)
        ppk::launch_scale_bf16((int)n, (const float *)w, scal, vj, c->stream);
    else
        ppk::launch_scale(pr, (int)n, vj, scal, c->stream);
    return check_launch(c);
}

cudaEvent_t Timers::get() {
    if (used == ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ev.push_back(e);
    }
    return ev[used++];
}

Timers::~Timers() {
    for (auto e : ev) cudaEventDestroy(e);
}

// Extend the Arnoldi decomposition from column j0 to m (Section 4): each step
// w = Op(v_j), CGS2, v_{j+1}.  H is (m+1) x m column major on the device.
pp_status arnoldi_extend(pp_ctx *c, const pp_poly *p, const pp_poly *tau_of, ppk::Prec bpr, void *V, int64_t ldv,
                         double *dH, int ldh, int j0, int m, void *W, Timers *tm,
                         std::vector<std::pair<int, int>> *marks) {
    const size_t besz = bpr == ppk::F64 ? 8 : (bpr == ppk::F32 ? 4 : 2);
    for (int j = j0; j < m; ++j) {
        const void *vj = (const char *)V + (size_t)j * ldv * besz;
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        if (tm) {
            e0 = tm->get();
            CK(cudaEventRecord(e0, c->stream));
        }
        if (bpr == ppk::BF16) {  // the operator reads FP32 vectors
            ppk::launch_convert(ppk::BF16, ppk::F32, (int)c->n, vj, c->vec[8], c->stream);
            CKS(check_launch(c));
            vj = c->vec[8];
        }
        if (tau_of)
            CKS(op_tau(c, tau_of, vj, W));
        else
            CKS(op_apply(c, p, vj, W));
        if (tm) {
            e1 = tm->get();
            CK(cudaEventRecord(e1, c->stream));
        }
        CKS(cgs2_step(c, bpr, V, ldv, j + 1, W, dH + (size_t)j * ldh));
        if (tm) {
            e2 = tm->get();
            CK(cudaEventRecord(e2, c->stream));
            marks->push_back({(int)tm->used - 3, (int)tm->used - 1});
        }
    }
    return PP_OK;
}

void accumulate_times(Timers &tm, std::vector<std::pair<int, int>> &marks, double &t_apply, double &t_orth) {
    for (auto &mk : marks) {
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, tm.ev[mk.first], tm.ev[mk.first + 1]);
        cudaEventElapsedTime(&b, tm.ev[mk.first + 1], tm.ev[mk.second]);
        t_apply += a * 1e-3;
        t_orth += b * 1e-3;
    }
    marks.clear();
    tm.used = 0;
}

// Upload a host FP64 vector scaled by s into device storage.
pp_status upload_vec(pp_ctx *c, const double *h, double s, void *d) {
    std::vector<double> tmp(h, h + c->n);
    for (auto &v : tmp) v *= s;
    if (c->A.prec == ppk::F64) {
        CK(cudaMemcpyAsync(d, tmp.data(), c->n * 8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        std::vector<float> f(tmp.begin(), tmp.end());
        CK(cudaMemcpyAsync(d, f.data(), c->n * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return PP_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

pp_status load_unit(pp_ctx *c, const double *x, ppk::Prec pr, void *dst, double *beta, const char *what) {
    const int64_t n = c->n;
    double nb = 0;
    if (!on_device(x)) {
        for (int64_t i = 0; i < n; ++i) nb += x[i] * x[i];
        nb = std::sqrt(nb);
        if (!(nb > 0) || !std::isfinite(nb)) return pp_fail(PP_EINVAL, "%s: start vector is zero or not finite", what);
        if (pr == ppk::BF16) {  // through the FP32 scratch
            CKS(upload_vec(c, x, 1.0 / nb, c->vec[8]));
            ppk::launch_convert(ppk::F32, ppk::BF16, (int)n, c->vec[8], dst, c->stream);
            CKS(check_launch(c));
        } else {
            CKS(upload_vec(c, x, 1.0 / nb, dst));
        }
        *beta = nb;
        return PP_OK;
    }
    double *nrm2 = c->d_small + 3968;
    ppk::launch_norm2((int)n, x, c->d_part, c->d_ticket, nrm2, c->stream);
    CKS(check_launch(c));
    double h = 0;
    CK(cudaMemcpyAsync(&h, nrm2, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    nb = std::sqrt(h);
    if (!(nb > 0) || !std::isfinite(nb)) return pp_fail(PP_EINVAL, "%s: start vector is zero or not finite", what);
    ppk::launch_unit_into(pr, (int)n, x, nrm2, dst, c->stream);
    CKS(check_launch(c));
    *beta = nb;
    return PP_OK;
}

pp_status download_vecs(pp_ctx *c, const void *d, int64_t ld, int cols, std::vector<double> &out, ppk::Prec pr) {
    out.resize((size_t)c->n * cols);
    if (pr == ppk::F64) {
        CK(cudaMemcpy2DAsync(out.data(), c->n * 8, d, ld * 8, c->n * 8, cols, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        std::vector<float> f((size_t)c->n * cols);
        CK(cudaMemcpy2DAsync(f.data(), c->n * 4, d, ld * 4, c->n * 4, cols, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < f.size(); ++i) out[i] = f[i];
    }
    return PP_OK;
}

pp_status check_sweeps(pp_ctx *c) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, c->err(), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!e) return PP_OK;
    CK(cudaMemsetAsync(c->err(), 0, sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->d_ticket, 0, ppk::kTicketWords * sizeof(unsigned), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return pp_fail(PP_ETIMEOUT, "CGS2 sweep: a bounded wait for staged basis tiles expired");
}

// GMRES(d) Arnoldi on Op from b (host), then harmonic Ritz roots, Leja, added roots.
pp_status build_roots(pp_ctx *c, int d, const double *b, const pp_poly *tau_of, pp_poly *out) {
    if (d < 1 || d > 127) return pp_fail(PP_EINVAL, "degree must be in [1, 127] (got %d)", d);
    if (d >= c->n) return pp_fail(PP_EINVAL, "degree %d must be below n = %lld", d, (long long)c->n);
    int64_t ldv = c->ldv();
    void *V = nullptr;
    double *dH = nullptr;
    pp_status st = PP_OK;
    std::vector<void *> mine;
    auto cleanup = [&]() {
        for (void *q : mine) ws_put(c, q);
    };
    if ((st = ws_get(c, &V, (size_t)ldv * (d + 1) * c->esz)) < 0) return st;
    mine.push_back(V);
    if ((st = ws_get(c, (void **)&dH, (size_t)(d + 1) * d * 8)) < 0) {
        cleanup();
        return st;
    }
    mine.push_back(dH);
    double beta = 0;
    std::vector<double> H((size_t)(d + 1) * d, 0.0);
    // CGS2 writes rows 0..j+1 of column j only; the rest of H must read as zero
    if (cudaMemsetAsync(dH, 0, (size_t)(d + 1) * d * 8, c->stream) != cudaSuccess) {
        cleanup();
        return pp_fail(PP_ECUDA, "build: memset failed");
    }
    if ((st = ensure_part(c, ppk::cgs_part_doubles(ppk::cgs_grid((int)c->n)))) < 0 ||
        (st = load_unit(c, b, c->A.prec, V, &beta, "build")) < 0 ||
        (st = arnoldi_extend(c, nullptr, tau_of, c->A.prec, V, ldv, dH, d + 1, 0, d, c->vec[6], nullptr,
                             nullptr)) < 0) {
        cleanup();
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(H.data(), dH, H.size() * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cleanup();
    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "build: %s", cudaGetErrorString(e));
    CKS(check_sweeps(c));
    return roots_from_hessenberg(c, d, H, tau_of ? op_mvps(tau_of) : 1, tau_of ? vops_of(tau_of->steps) : 0, out);
}

// Harmonic Ritz roots of a GMRES(d) Hessenberg matrix (Section 2 box 1(b)), a
// lucky breakdown handled as exact eigenvalues, modified Leja order (1(c)) and
// the Section 7 added roots; the work is counted as the oracle does.
pp_status roots_from_hessenberg(pp_ctx *c, int d, const std::vector<double> &H, int64_t mvps_per_step,
                                int64_t vops_per_step, pp_poly *out) {
    for (double v : H)
        if (!std::isfinite(v)) return pp_fail(PP_ENUMERIC, "build: non-finite Hessenberg entry");
    // lucky breakdown: h_{j+1,j} <= 1e-14 ||H(0:j+2, 0:j+1)||_F
    int steps = d;
    bool brk = false;
    double fro = 0;
    for (int j = 0; j < d; ++j) {
        for (int i = 0; i <= j + 1; ++i) fro += H[i + (size_t)j * (d + 1)] * H[i + (size_t)j * (d + 1)];
        if (H[j + 1 + (size_t)j * (d + 1)] <= 1e-14 * std::sqrt(fro)) {
            steps = j + 1;
            brk = true;
            break;
        }
    }
    std::vector<double> re(steps), im(steps);
    bool ok;
    if (brk) {
        std::vector<double> Hs((size_t)steps * steps);
        for (int j = 0; j < steps; ++j)
            for (int i = 0; i < steps; ++i) Hs[i + (size_t)j * steps] = H[i + (size_t)j * (d + 1)];
        ok = ppd::dense_eig(steps, Hs.data(), steps, re.data(), im.data(), nullptr, 0);
    } else {
        ok = ppd::harmonic_ritz(d, H.data(), d + 1, re.data(), im.data());
    }
    if (!ok) return pp_fail(PP_ENUMERIC, "harmonic Ritz values: singular H_d or QR failure");
    std::vector<cd> th(steps), ord;
    for (int i = 0; i < steps; ++i) th[i] = cd(re[i], im[i]);
    if (!ppd::leja_order(th, ord)) return pp_fail(PP_ENUMERIC, "roots not closed under conjugation");
    int added = 0;
    if (c->opts.add_roots) {
        std::vector<cd> ext;
        if (!ppd::add_stability_roots(ord, ext, added)) return pp_fail(PP_ENUMERIC, "added roots failed");
        ord.swap(ext);
    }
    // work counted as the oracle does: start normalisation, then per step the
    // operator, CGS2 against j+1 vectors and the norm
    out->mvps = 0;
    out->dots = 1;
    out->vops = 2;
    for (int j = 0; j < d; ++j) {
        out->mvps += mvps_per_step;
        out->vops += vops_per_step;
        out->dots += 2 * (j + 1) + 1;
        out->vops += 4 * (j + 1) + 2;
    }
    out->roots = ord;
    out->steps = steps_of(ord);
    out->degree = steps;
    out->added = added;
    out->breakdown = brk;
    return brk ? PP_EBREAKDOWN : PP_OK;
}

}  // namespace ppi

using namespace ppi;

// ===========================================================================
extern "C" {

const char *pp_last_error(void) { return g_last_error.c_str(); }

void pp_opts_default(pp_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = PP_FP64;
    o->format = PP_FMT_AUTO;
    o->target = PP_TARGET_SR;
    o->sigma = NAN;
    o->add_roots = 1;
    o->max_cycles = 2000;
    o->refine_steps = 4;
    o->sell_c = 0;
    o->sell_sigma = 0;
    o->stream = nullptr;
    o->restart = PP_RESTART_RITZ;
}

pp_status pp_trim(pp_ctx *c) {
    if (!c) return pp_fail(PP_EINVAL, "pp_trim: null context");
    for (pp_ctx *t = c; t; t = t->twin) ws_trim(t);
    return PP_OK;
}

void pp_destroy(pp_ctx *c) {
    if (!c) return;
    if (c->twin) pp_destroy(c->twin);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void *p : c->allocs) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

pp_status pp_create(pp_ctx **out, int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals,
                    const pp_opts *opts) {
    return pp_create_internal(out, n, rowptr, colind, vals, opts, 1);
}

}  // extern "C"

// The shift of the smallest-real-part target (Section 2, footnote 1): the
// leftmost Gershgorin point gl when it is negative beyond rounding
// (below -1e-12 ||A||_1), else 0.
static double sr_shift(double gl, double norm1) { return (gl >= -1e-12 * norm1) ? 0.0 : std::min(0.0, gl); }

// 64-bit row pointers to 32-bit on the device (pp_create checks nnz < 2^31).
static __global__ void k_rowptr32(int64_t count, const int64_t *src, int *dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) dst[i] = (int)src[i];
}

static cudaError_t launch_rowptr32(int64_t count, const int64_t *src, int *dst, cudaStream_t st) {
    const int threads = 256;
    k_rowptr32<<<(unsigned)((count + threads - 1) / threads), threads, 0, st>>>(count, src, dst);
    return cudaGetLastError();
}

// Stored entries of SELL-C (C = 1 << cs): each slice padded to its longest row.
static int64_t sell_padded(int64_t n, const int64_t *rowptr, int cs) {
    const int64_t C = (int64_t)1 << cs;
    int64_t tot = 0;
    for (int64_t s0 = 0; s0 < n; s0 += C) {
        int64_t w = 0;
        for (int64_t i = s0; i < std::min(n, s0 + C); ++i) w = std::max(w, rowptr[i + 1] - rowptr[i]);
        tot += w * C;
    }
    return tot;
}

// Most stored entries of SELL-32 in any g consecutive slices (a staged tile).
static int64_t tile_cap(int64_t n, const int64_t *rowptr, int g) {
    int64_t best = 0, cur = 0;
    const int64_t ns = (n + 31) / 32;
    for (int64_t s0 = 0; s0 < ns; ++s0) {
        int64_t w = 0;
        for (int64_t i = s0 * 32; i < std::min(n, s0 * 32 + 32); ++i) w = std::max(w, rowptr[i + 1] - rowptr[i]);
        cur += w * 32;
        if ((s0 + 1) % g == 0 || s0 + 1 == ns) {
            best = std::max(best, cur);
            cur = 0;
        }
    }
    return best;
}

// SELL-C of the device CSR: slice pointers on the host, fill on the device;
// the allocations are returned in mem (the tuner frees the losers).
static pp_status build_sell(pp_ctx *c, ppk::Prec pr, int64_t n, const int64_t *rowptr, int cs, bool off16,
                            const int *d_rowptr, const int *d_col, const double *d_val, ppk::SellView &out,
                            std::vector<void *> &mem) {
    const int64_t C = (int64_t)1 << cs;
    const int nslices = (int)((n + C - 1) / C);
    std::vector<int> sptr(nslices + 1, 0);
    for (int s = 0; s < nslices; ++s) {
        int64_t w = 0;
        for (int64_t i = s * C; i < std::min(n, (s + 1) * C); ++i) w = std::max(w, rowptr[i + 1] - rowptr[i]);
        sptr[s + 1] = sptr[s] + (int)(w * C);
    }
    const int64_t padded = sptr[nslices];
    int *d_sptr = nullptr, *d_scol = nullptr;
    short *d_soff = nullptr;
    void *d_sval = nullptr;
    pp_status st;
    if ((st = dmalloc(c, (void **)&d_sptr, (nslices + 1) * 4)) < 0) return st;
    mem.push_back(d_sptr);
    if (off16) {
        if ((st = dmalloc(c, (void **)&d_soff, padded * 2)) < 0) return st;
        mem.push_back(d_soff);
    } else {
        if ((st = dmalloc(c, (void **)&d_scol, padded * 4)) < 0) return st;
        mem.push_back(d_scol);
    }
    if ((st = dmalloc(c, &d_sval, padded * c->esz)) < 0) return st;
    mem.push_back(d_sval);
    CK(cudaMemcpyAsync(d_sptr, sptr.data(), (nslices + 1) * 4, cudaMemcpyHostToDevice, c->stream));
    ppk::launch_sell_fill(pr, (int)n, nslices, cs, d_rowptr, d_col, d_val, d_sptr, d_scol, d_soff, d_sval, c->stream);
    CK(cudaGetLastError());
    out = {(int)n, nslices, cs, d_sptr, d_scol, d_soff, d_sval};
    return PP_OK;
}

// Tuner cost of a format: a run like an apply's, passes reading the previous
// pass's output (ping-pong over three scratch vectors): eight specialised root
// passes (y = x - A x/theta) then eight running-sum passes (the double
// polynomial's inner pass), the fastest of three runs after one warm-up run,
// CUDA events on the context's stream.  Negative on a launch error.
static double time_product(pp_ctx *c, const ppk::Matrix &M) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1;
    }
    void *buf[3] = {c->vec[0], c->vec[1], c->vec[2]};
    double best = INFINITY;
    for (int run = 0; run < 4 && best >= 0; ++run) {
        cudaEventRecord(e0, c->stream);
        for (int i = 0; i < 16; ++i) {
            ppk::StepArgs a;
            a.x = buf[i % 3];
            a.y = buf[(i + 1) % 3];
            a.a2 = 1e-7;  // keeps the iterates bounded
            if (i >= 8) {
                a.r = c->vec[3];
                a.r_init = i == 8;
            }
            ppk::launch_step(M, a, c->stream);
        }
        cudaEventRecord(e1, c->stream);
        float ms = 0;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            best = -1;
            break;
        }
        if (run >= 1) best = std::min(best, (double)ms * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return best;
}

// Tuner decisions cached per process, keyed by a signature of the matrix (size,
// precision, index width and sampled row pointers and columns): contexts for the
// same matrix skip the timing runs and build only the chosen format.
struct TuneChoice {
    int cs = 5, threads = 256, loop = 0, cap = 0;
    bool dia = false;
    int dia_threads = 256, dia_wide = 0;
};
static std::mutex g_tune_mu;
static std::map<uint64_t, TuneChoice> g_tune_cache;

static uint64_t matrix_signature(int64_t n, const int64_t *rowptr, const int32_t *colind, size_t esz, bool off16) {
    uint64_t h = 1469598103934665603ULL;
    auto mix = [&](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xff;
            h *= 1099511628211ULL;
        }
    };
    mix((uint64_t)n);
    mix((uint64_t)rowptr[n]);
    mix(esz);
    mix(off16 ? 1 : 0);
    const int64_t nnz = rowptr[n];
    for (int t = 0; t < 192; ++t) {
        const int64_t i = t < 64 ? std::min<int64_t>(t, n - 1)
                                 : (t < 128 ? std::max<int64_t>(0, n - 128 + t) : (n - 1) * (t - 128) / 63);
        mix((uint64_t)rowptr[i]);
        if (nnz > 0) mix((uint64_t)(uint32_t)colind[std::min<int64_t>(nnz - 1, (nnz - 1) * t / 191)]);
    }
    return h;
}

pp_status pp_create_internal(pp_ctx **out, int64_t n, const int64_t *rowptr, const int32_t *colind,
                             const double *vals, const pp_opts *opts, int make_twin) {
    if (!out || n <= 0 || !rowptr || !colind || !vals) return pp_fail(PP_EINVAL, "pp_create: bad arguments");
    *out = nullptr;
    int64_t nnz = rowptr[n];
    if (rowptr[0] != 0 || nnz < 0 || nnz >= (int64_t)1 << 31 || n >= (int64_t)1 << 31)
        return pp_fail(PP_EINVAL, "pp_create: rowptr must start at 0 and nnz, n < 2^31");
    // validation, ||A||_1, the Gershgorin bound of the shift and whether 16-bit
    // column offsets fit, in one parallel pass over the entries
    ppd::CsrScan scan;
    {
        std::string why;
        if (!ppd::scan_csr(n, rowptr, colind, vals, scan, why)) return pp_fail(PP_EINVAL, "pp_create: %s", why.c_str());
    }
    double gl = scan.gl;
    const bool fits16 = scan.fits16;
    // balancing (opts.balance): the operator's matrix becomes S = D^-1 A D, the
    // diagonal similarity that makes A symmetric; ||A||_1 and the residual test
    // stay on A, the shift is S's Gershgorin bound
    int balance = opts ? opts->balance : 0;
    if (balance < 0 || balance > 2) return pp_fail(PP_EINVAL, "pp_create: balance must be 0, 1 or 2");
    std::vector<double> logd, svals;
    const double *kvals = vals;  // values of the operator's matrix
    if (balance) {
        std::string why;
        if (!ppd::symmetrizing_scale(n, rowptr, colind, vals, logd, why)) {
            if (balance == 1) return pp_fail(PP_EINVAL, "pp_create: balance: %s", why.c_str());
            balance = 0;  // 2: where a symmetrising D exists, else A as given
        }
    }
    if (balance) {
        svals.resize(nnz);
        gl = INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            double diag = 0, off = 0;
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                svals[k] = vals[k] * std::exp(logd[colind[k]] - logd[i]);
                if (colind[k] == i)
                    diag += svals[k];
                else
                    off += std::fabs(svals[k]);
            }
            gl = std::min(gl, diag - off);
        }
        kvals = svals.data();
    }
    pp_ctx *c = new pp_ctx();
    pp_opts_default(&c->opts);
    if (opts) c->opts = *opts;
    if (c->opts.precision != PP_FP64 && c->opts.precision != PP_FP32 && c->opts.precision != PP_FP32_BF16) {
        delete c;
        return pp_fail(PP_EINVAL, "pp_create: precision %d not supported", c->opts.precision);
    }
    c->n = n;
    c->nnz = nnz;
    // ||A||_1 and the Gershgorin shift on the host (exact, deterministic)
    c->norm1 = scan.norm1;
    if (std::isnan(c->opts.sigma)) {
        if (c->opts.target == PP_TARGET_SR)
            c->sigma = sr_shift(gl, c->norm1);
        else
            c->sigma = 0.0;
    } else {
        c->sigma = c->opts.sigma;
    }
    if (c->opts.stream) {
        c->stream = (cudaStream_t)c->opts.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return pp_fail(PP_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    ppk::Prec pr = c->opts.precision == PP_FP64 ? ppk::F64 : ppk::F32;
    c->esz = pr == ppk::F64 ? 8 : 4;
    c->bprec = c->opts.precision == PP_FP32_BF16 ? ppk::BF16 : pr;
    c->besz = c->bprec == ppk::BF16 ? 2 : c->esz;
    pp_status st = PP_OK;
    auto fail = [&](pp_status s) {
        pp_destroy(c);
        return s;
    };
    // device CSR (int32 row pointers, FP64 values)
    int *d_rowptr = nullptr, *d_col = nullptr;
    double *d_val = nullptr;
    int64_t *d_rp64 = nullptr;  // the row pointers as given, made 32-bit on the device
    if ((st = dmalloc(c, (void **)&d_rowptr, (n + 1) * 4)) < 0 || (st = dmalloc(c, (void **)&d_col, nnz * 4)) < 0 ||
        (st = dmalloc(c, (void **)&d_val, nnz * 8)) < 0 || (st = dmalloc(c, (void **)&d_rp64, (n + 1) * 8)) < 0)
        return fail(st);
    // stream-ordered uploads: the context's stream does not synchronise with the legacy stream
    if (cudaMemcpyAsync(d_rp64, rowptr, (n + 1) * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        launch_rowptr32(n + 1, d_rp64, d_rowptr, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_col, colind, nnz * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_val, kvals, nnz * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return fail(pp_fail(PP_ECUDA, "pp_create: upload failed"));
    double *d_aval = nullptr;  // balanced: A's own values for the residual test
    if (balance) {
        c->h_bal.resize(n);
        for (int64_t i = 0; i < n; ++i) c->h_bal[i] = std::exp(logd[i]);
        if ((st = dmalloc(c, (void **)&d_aval, nnz * 8)) < 0 || (st = dmalloc(c, (void **)&c->d_bal, n * 8)) < 0)
            return fail(st);
        if (cudaMemcpyAsync(d_aval, vals, nnz * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(c->d_bal, c->h_bal.data(), n * 8, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return fail(pp_fail(PP_ECUDA, "pp_create: upload failed"));
    }
    // format: SELL-C unless its padding exceeds 30 % (then CSR); C and the
    // block size of the product kernels from the tuner unless opts fix C
    if (c->opts.sell_c != 0 && c->opts.sell_c != 16 && c->opts.sell_c != 32)
        return fail(pp_fail(PP_EINVAL, "pp_create: sell_c must be 0, 16 or 32"));
    if (c->opts.sell_sigma > 1) return fail(pp_fail(PP_EINVAL, "pp_create: sell_sigma must be 0 or 1"));
    if (c->opts.sell_index != 0 && c->opts.sell_index != 32)
        return fail(pp_fail(PP_EINVAL, "pp_create: sell_index must be 0 or 32"));
    if (c->opts.restart != PP_RESTART_RITZ && c->opts.restart != PP_RESTART_HARMONIC)
        return fail(pp_fail(PP_EINVAL, "pp_create: restart must be PP_RESTART_RITZ or PP_RESTART_HARMONIC"));
    if (c->opts.sell_loop < 0 || c->opts.sell_loop > 4)
        return fail(pp_fail(PP_EINVAL, "pp_create: sell_loop must be 0 to 4"));
    if (c->opts.dia_loop < 0 || c->opts.dia_loop > 3)
        return fail(pp_fail(PP_EINVAL, "pp_create: dia_loop must be 0 to 3"));
    std::vector<int> cands;
    if (c->opts.sell_c) cands.push_back(c->opts.sell_c == 16 ? 4 : 5);
    else cands = {5, 4};
    int64_t best_pad = INT64_MAX;
    {
        std::vector<int> fit;  // candidates whose padded size fits 32-bit slice pointers
        for (int cs : cands) {
            int64_t pd = sell_padded(n, rowptr, cs);
            best_pad = std::min(best_pad, pd);
            if (pd < ((int64_t)1 << 31)) fit.push_back(cs);
        }
        cands = fit;
    }
    int fmt = c->opts.format;
    if (fmt == PP_FMT_AUTO) fmt = (best_pad <= (int64_t)(1.3 * (double)nnz) + 32 * 8) ? PP_FMT_SELL : PP_FMT_CSR;
    if (cands.empty()) fmt = PP_FMT_CSR;
    const bool off16 = c->opts.sell_index == 0 && fits16;
    ppk::Matrix M;
    M.n = (int)n;
    M.prec = pr;
    M.csr = {(int)n, d_rowptr, d_col, d_val};
    if (pr == ppk::F32) {
        void *v32 = nullptr;
        if ((st = dmalloc(c, &v32, nnz * 4)) < 0) return fail(st);
        ppk::launch_csr_convert(pr, nnz, d_val, v32, c->stream);
        M.csr.val = v32;
    }
    // scratch vectors (the tuner times products with them), reduction ticket and
    // the small FP64 area holding the error word of the staged kernels
    for (int i = 0; i < 9; ++i)
        if ((st = dmalloc(c, &c->vec[i], (size_t)c->ldv() * c->esz)) < 0) return fail(st);
    if ((st = dmalloc(c, (void **)&c->d_ticket, ppk::kTicketWords * sizeof(unsigned))) < 0 || (st = dmalloc(c, (void **)&c->d_small, 4096 * 8)) < 0)
        return fail(st);
    // the tuner's vectors: a finite nonzero pattern (0x3f bytes: 0.49 in FP64, 0.75 in FP32)
    if (cudaMemsetAsync(c->vec[0], 0x3f, (size_t)c->ldv() * c->esz, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->vec[3], 0, (size_t)c->ldv() * c->esz, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_ticket, 0, ppk::kTicketWords * sizeof(unsigned), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_small, 0, 4096 * 8, c->stream) != cudaSuccess)
        return fail(pp_fail(PP_ECUDA, "pp_create: memset failed"));
    M.err = c->err();
    c->stored = nnz;
    double sell_t = INFINITY;  // the tuner's time of the chosen SELL format
    std::vector<void *> sell_mem;
    if (fmt == PP_FMT_DIA) fmt = PP_FMT_SELL;  // DIA replaces SELL below when the matrix allows it
    const bool cacheable = c->opts.format == PP_FMT_AUTO && !c->opts.sell_c && !c->opts.sell_loop && !c->opts.dia_loop &&
                           fmt == PP_FMT_SELL;
    const uint64_t sig = cacheable ? matrix_signature(n, rowptr, colind, c->esz, off16) : 0;
    bool cached = false;
    TuneChoice choice;
    if (cacheable) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(sig);
        if (it != g_tune_cache.end()) {
            choice = it->second;
            cached = true;
        }
    }
    if (fmt == PP_FMT_SELL) {
        M.fmt = 2;
        std::vector<int> threads = {256};
        if (!c->opts.sell_c) threads = {128, 256, 512};
        // row loops: 0 unrolled, 1 wide, 2 staged by bulk copies (SELL-32 only), 3 two rows per thread
        std::vector<int> loops = {0, 1, 2, 3};
        if (c->opts.sell_loop) loops = {c->opts.sell_loop - 1};
        if (cached) {  // the decision of an earlier context for this matrix
            cands = {choice.cs};
            threads = {choice.threads};
            loops = {choice.loop};
        }
        const bool tune = cands.size() * threads.size() * loops.size() > 1;
        double best_t = INFINITY;
        int best_threads = 256, best_loop = 0, best_cap = 0;
        ppk::SellView best{};
        std::vector<void *> best_mem;
        for (int cs : cands) {
            ppk::SellView sv{};
            std::vector<void *> mem;
            if ((st = build_sell(c, pr, n, rowptr, cs, off16, d_rowptr, d_col, d_val, sv, mem)) < 0) return fail(st);
            M.sell = sv;
            bool better = false;
            for (int loop : loops)
                for (int t : threads) {
                    int cap = 0;
                    if (loop == 2) {  // staged: SELL-32 and two stages within 200 KB of shared memory
                        if (cs != 5) continue;
                        cap = (int)tile_cap(n, rowptr, t / 32);
                        const size_t esz_i = off16 ? 2 : 4;
                        if (128 + (size_t)cap * (c->esz + esz_i) + 256 > 100 * 1024) continue;
                    }
                    M.threads = t;
                    M.wide = loop == 1 ? 1 : (loop == 3 ? 2 : 0);
                    M.tma = loop == 2;
                    M.tile_cap = cap;
                    double tt = tune ? time_product(c, M) : 0.0;
                    if (tt < 0) return fail(pp_fail(PP_ECUDA, "pp_create: tuner launch failed"));
                    // the plain candidate (SELL-32, unrolled, 256 threads) wins ties within 3 %:
                    // a variant must be clearly faster to be chosen over timing noise
                    if (tune && cs == 5 && loop == 0 && t == 256) tt *= 0.97;
                    if (tt < best_t) {
                        best_t = tt;
                        best_threads = t;
                        best_loop = loop;
                        best_cap = cap;
                        better = true;
                    }
                }
            for (void *q : better ? best_mem : mem) dfree(c, q);
            if (better) {
                best = sv;
                best_mem = mem;
            }
        }
        if (!(best_t < INFINITY) && !tune) return fail(pp_fail(PP_EINVAL, "pp_create: sell_loop 3 needs sell_c 0 or 32"));
        M.sell = best;
        M.threads = best_threads;
        M.wide = best_loop == 1 ? 1 : (best_loop == 3 ? 2 : 0);
        M.tma = best_loop == 2;
        M.tile_cap = best_cap;
        c->stored = sell_padded(n, rowptr, best.cshift);
        sell_t = best_t;
        sell_mem = best_mem;
        choice.cs = best.cshift;
        choice.threads = best_threads;
        choice.loop = best_loop;
        choice.cap = best_cap;
    } else {
        M.fmt = 1;
    }
    // DIA for stencil and banded matrices (no column indices): when asked for,
    // or in auto mode when it times faster than the SELL choice
    std::vector<int> doff;
    const bool auto_tuned = c->opts.format == PP_FMT_AUTO && !c->opts.sell_c && !c->opts.sell_loop && M.fmt == 2;
    // (a cached SELL decision needs no DIA analysis)
    const bool dia_wanted = c->opts.format == PP_FMT_DIA || (auto_tuned && (!cached || choice.dia));
    const bool dia_fits = dia_wanted && ppd::dia_offsets(n, rowptr, colind, ppk::kDiaMax, doff) &&
                          (int64_t)doff.size() * n <= (int64_t)(1.3 * (double)nnz) + 32 * 8;
    if (c->opts.format == PP_FMT_DIA && !dia_fits)
        return fail(pp_fail(PP_EINVAL, "pp_create: DIA needs sorted columns, at most %d diagonals and <= 30 %% padding",
                            ppk::kDiaMax));
    if (dia_fits) {
        const int nd = (int)doff.size();
        const int64_t ld = c->ldv();
        int *d_off = nullptr;
        void *d_dval = nullptr;
        if ((st = dmalloc(c, (void **)&d_off, nd * 4)) < 0 || (st = dmalloc(c, &d_dval, (size_t)nd * ld * c->esz)) < 0)
            return fail(st);
        if (cudaMemcpyAsync(d_off, doff.data(), nd * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return fail(pp_fail(PP_ECUDA, "pp_create: upload failed"));
        ppk::launch_dia_fill(pr, (int)n, d_rowptr, d_col, d_val, d_off, nd, ld, d_dval, c->stream);
        if (cudaGetLastError() != cudaSuccess) return fail(pp_fail(PP_ECUDA, "pp_create: DIA fill failed"));
        ppk::Matrix D = M;
        D.fmt = 3;
        D.wide = 0;
        D.tma = 0;
        D.dia = {(int)n, nd, ld, d_off, d_dval};
        double dia_t = INFINITY;
        int dia_threads = cached ? choice.dia_threads : 256, dia_wide = cached ? choice.dia_wide : 0;
        // row loops (FP32): 0 one row per thread, 1 four rows, 2 two rows; FP64: one row
        std::vector<int> wl = {0};
        if (pr == ppk::F32) wl = {0, 1, 2};
        if (c->opts.dia_loop) wl = {pr == ppk::F32 ? c->opts.dia_loop - 1 : 0};
        if (!cached)
            for (int w : wl)
                for (int t : {128, 256, 512}) {
                    if (w != 0 && t > 256) continue;  // the multi-row kernels take at most 256 threads
                    D.threads = t;
                    D.wide = w;
                    double tt = time_product(c, D);
                    if (tt < 0) return fail(pp_fail(PP_ECUDA, "pp_create: tuner launch failed"));
                    if (tt < dia_t) {
                        dia_t = tt;
                        dia_threads = t;
                        dia_wide = w;
                    }
                }
        choice.dia = cached ? choice.dia : dia_t < sell_t;
        choice.dia_threads = dia_threads;
        choice.dia_wide = dia_wide;
        if (c->opts.format == PP_FMT_DIA || choice.dia) {
            for (void *q : sell_mem) dfree(c, q);
            D.threads = dia_threads;
            D.wide = dia_wide;
            M = D;
            c->stored = (int64_t)nd * n;
        } else {
            dfree(c, d_off);
            dfree(c, d_dval);
        }
    }
    if (cacheable && !cached) {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[sig] = choice;
    }
    c->A = M;
    // FP64 operator for residuals on A (Section 4 tests convergence on A itself)
    c->A64 = M;
    c->A64.prec = ppk::F64;
    c->A64.fmt = 1;
    c->A64.csr = {(int)n, d_rowptr, d_col, d_val};
    if (pr == ppk::F64) c->A64 = M;
    c->S64 = c->A64;
    if (balance) {  // the test on A itself; S64 (the refinement's projections) stays S
        c->A64.prec = ppk::F64;
        c->A64.fmt = 1;
        c->A64.csr = {(int)n, d_rowptr, d_col, d_aval};
    }
    if ((st = ensure_part(c, ppk::cgs_part_doubles(ppk::cgs_grid((int)n)))) < 0) return fail(st);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(pp_fail(PP_ECUDA, "pp_create: setup kernels failed"));
    dfree(c, d_rp64);
    if (c->bprec != ppk::F64 && make_twin) {
        // twin on the same stream, one precision up: the mixed-precision solve
        // continues there when its cycles cannot resolve the eigenvectors
        // (u kappa ~ 1).  FP32 contexts get an FP64 twin; BF16-basis contexts an
        // FP32 one, which has its own FP64 twin (a BF16 basis stalls near 1e-3,
        // an FP32 one near 1e-7, where the FP64 refinement takes over)
        pp_opts o = c->opts;
        o.precision = c->bprec == ppk::BF16 ? PP_FP32 : PP_FP64;
        o.sigma = c->sigma;
        o.stream = c->stream;
        if ((st = pp_create(&c->twin, n, rowptr, colind, vals, &o)) < 0) return fail(st);
    }
    *out = c;
    return PP_OK;
}

extern "C" {

int64_t pp_launch_count(const pp_ctx *c) { return c ? c->launches : 0; }

pp_status pp_orthogonalize(pp_ctx *c, const void *V, int64_t ldv, int j, void *w, void *v, double *h_host) {
    if (!c || !V || !w || !v || !h_host || j < 1 || j > 128 || ldv < c->n)
        return pp_fail(PP_EINVAL, "pp_orthogonalize: bad arguments");
    // the CGS2 passes read V[:, 0..j) and write the result as column j of a
    // basis; here the result goes to v: run the passes with a one-column shim
    double *dh = c->d_small + 1024;  // j+1 doubles of H column
    ppk::Prec pr = c->A.prec;
    double *h1 = c->d_small, *h2 = c->d_small + 256, *scal = c->d_small + 512, *nrm = c->d_small + 513;
    ppk::CgsArgs a;
    a.n = (int)c->n;
    a.V = V;
    a.ldv = ldv;
    a.j = j;
    a.part = c->d_part;
    a.ticket = c->d_ticket;
    a.err = c->err();
    if (c->stall_sweeps > 0) {
        a.stall = 1;
        c->stall_sweeps--;
    }
    a.mode = 0;
    a.w = w;
    a.out = h1;
    ppk::launch_cgs(pr, a, c->stream);
    CKS(check_launch(c));
    a.mode = 1;
    a.h = h1;
    a.wout = w;
    a.out = h2;
    ppk::launch_cgs(pr, a, c->stream);
    CKS(check_launch(c));
    a.mode = 2;
    a.h = h2;
    a.h1 = h1;
    a.wout = v;
    a.out = nrm;
    a.hcol = dh;
    a.scal = scal;
    ppk::launch_cgs(pr, a, c->stream);
    CKS(check_launch(c));
    ppk::launch_scale(pr, (int)c->n, v, scal, c->stream);
    CKS(check_launch(c));
    CK(cudaMemcpyAsync(h_host, dh, (size_t)(j + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return check_sweeps(c);
}

pp_status pp_balance_info(const pp_ctx *c, int *balanced, double *log_range) {
    if (!c) return pp_fail(PP_EINVAL, "pp_balance_info: null context");
    if (balanced) *balanced = c->d_bal ? 1 : 0;
    if (log_range) {
        double lo = 0;
        for (double d : c->h_bal) lo = std::min(lo, std::log(d));
        *log_range = -lo;
    }
    return PP_OK;
}

pp_status pp_csr_balance(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals, double *d,
                         double *log_range) {
    if (n <= 0 || !rowptr || !colind || !vals || !d) return pp_fail(PP_EINVAL, "pp_csr_balance: bad arguments");
    const int64_t nnz = rowptr[n];
    if (rowptr[0] != 0 || nnz < 0 || nnz >= (int64_t)1 << 31 || n >= (int64_t)1 << 31)
        return pp_fail(PP_EINVAL, "pp_csr_balance: rowptr must start at 0 and nnz, n < 2^31");
    ppd::CsrScan scan;  // the same validation as pp_create
    std::string why;
    if (!ppd::scan_csr(n, rowptr, colind, vals, scan, why)) return pp_fail(PP_EINVAL, "pp_csr_balance: %s", why.c_str());
    std::vector<double> logd;
    if (!ppd::symmetrizing_scale(n, rowptr, colind, vals, logd, why))
        return pp_fail(PP_EINVAL, "pp_csr_balance: %s", why.c_str());
    double lo = 0;
    for (int64_t i = 0; i < n; ++i) {
        d[i] = std::exp(logd[i]);
        lo = std::min(lo, logd[i]);
    }
    if (log_range) *log_range = -lo;
    return PP_OK;
}

pp_status pp_csr_info(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals, double *norm1,
                      double *sigma_sr) {
    if (n <= 0 || !rowptr || !colind || !vals) return pp_fail(PP_EINVAL, "pp_csr_info: bad arguments");
    const int64_t nnz = rowptr[n];
    if (rowptr[0] != 0 || nnz < 0 || nnz >= (int64_t)1 << 31 || n >= (int64_t)1 << 31)
        return pp_fail(PP_EINVAL, "pp_csr_info: rowptr must start at 0 and nnz, n < 2^31");
    ppd::CsrScan scan;
    std::string why;
    if (!ppd::scan_csr(n, rowptr, colind, vals, scan, why)) return pp_fail(PP_EINVAL, "pp_csr_info: %s", why.c_str());
    if (norm1) *norm1 = scan.norm1;
    if (sigma_sr) *sigma_sr = sr_shift(scan.gl, scan.norm1);
    return PP_OK;
}

pp_status pp_matrix_info(const pp_ctx *c, double *norm1, double *sigma) {
    if (!c) return pp_fail(PP_EINVAL, "pp_matrix_info: null context");
    if (norm1) *norm1 = c->norm1;
    if (sigma) *sigma = c->sigma;
    return PP_OK;
}

pp_status pp_debug_stall_sweeps(pp_ctx *c, int count) {
    if (!c || count < 0) return pp_fail(PP_EINVAL, "pp_debug_stall_sweeps: bad arguments");
    c->stall_sweeps = count;
    return PP_OK;
}

pp_status pp_format_info(const pp_ctx *c, int *fmt, int *chunk, int *index_bits, int *threads, int *row_loop,
                         int64_t *stored) {
    if (!c) return pp_fail(PP_EINVAL, "pp_format_info: null context");
    const bool sell = c->A.fmt == 2;
    if (fmt) *fmt = sell ? PP_FMT_SELL : (c->A.fmt == 3 ? PP_FMT_DIA : PP_FMT_CSR);
    if (chunk) *chunk = sell ? 1 << c->A.sell.cshift : 0;
    if (index_bits) *index_bits = c->A.fmt == 3 ? 0 : ((sell && c->A.sell.off) ? 16 : 32);
    if (threads) *threads = c->A.fmt != 1 ? c->A.threads : 256;
    if (row_loop) *row_loop = sell ? (c->A.tma ? 2 : (c->A.wide == 2 ? 3 : c->A.wide)) : (c->A.fmt == 3 ? c->A.wide : 0);
    if (stored) *stored = c->stored;
    return PP_OK;
}

pp_status pp_build_poly(pp_ctx *c, int d, const double *b, pp_poly **out) {
    if (!c || !b || !out) return pp_fail(PP_EINVAL, "pp_build_poly: bad arguments");
    pp_poly *p = new pp_poly();
    p->ctx = c;
    pp_status st = build_roots(c, d, b, nullptr, p);
    if (st < 0) {
        delete p;
        return st;
    }
    *out = p;
    return st;
}

// GMRES(d) on blockdiag(A - sigma I, A - sigma I) from [b1; b2] (Section 5 box):
// 2n-vectors; the operator is two products with the context's matrix (the
// halves, through offset pointers), the CGS2 sweeps run over length 2n.
static pp_status build_roots_two(pp_ctx *c, int d, const double *b1, const double *b2, pp_poly *out) {
    if (d < 1 || d > 127) return pp_fail(PP_EINVAL, "degree must be in [1, 127] (got %d)", d);
    const int64_t n = c->n, n2 = 2 * n;
    if (d >= n2) return pp_fail(PP_EINVAL, "degree %d must be below 2n", d);
    std::vector<double> h1, h2;  // host copies of device start vectors
    if (on_device(b1) || on_device(b2)) {
        h1.resize(n);
        h2.resize(n);
        CK(cudaMemcpyAsync(h1.data(), b1, (size_t)n * 8, cudaMemcpyDefault, c->stream));
        CK(cudaMemcpyAsync(h2.data(), b2, (size_t)n * 8, cudaMemcpyDefault, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        b1 = h1.data();
        b2 = h2.data();
    }
    double s1 = 0, s2 = 0;
    for (int64_t i = 0; i < n; ++i) {
        s1 += b1[i] * b1[i];
        s2 += b2[i] * b2[i];
    }
    s1 = std::sqrt(s1);
    s2 = std::sqrt(s2);
    if (!(s1 > 0) || !(s2 > 0) || !std::isfinite(s1) || !std::isfinite(s2))
        return pp_fail(PP_EINVAL, "start vectors must be nonzero and finite");
    // [b1 / (sqrt2 ||b1||); b2 / (sqrt2 ||b2||)] has unit norm
    std::vector<double> bh(n2);
    for (int64_t i = 0; i < n; ++i) {
        bh[i] = b1[i] / (std::sqrt(2.0) * s1);
        bh[n + i] = b2[i] / (std::sqrt(2.0) * s2);
    }
    const int64_t ldv = (n2 + 31) / 32 * 32;
    const size_t esz = c->esz;
    std::vector<void *> mine;
    auto cleanup = [&]() {
        for (void *q : mine) ws_put(c, q);
    };
    void *V = nullptr, *W = nullptr;
    double *dH = nullptr;
    pp_status st;
    if ((st = ws_get(c, &V, (size_t)ldv * (d + 1) * esz)) < 0) return st;
    mine.push_back(V);
    if ((st = ws_get(c, &W, (size_t)ldv * esz)) < 0) {
        cleanup();
        return st;
    }
    mine.push_back(W);
    if ((st = ws_get(c, (void **)&dH, (size_t)(d + 1) * d * 8)) < 0) {
        cleanup();
        return st;
    }
    mine.push_back(dH);
    if ((st = ensure_part(c, ppk::cgs_part_doubles(ppk::cgs_grid((int)n2)))) < 0) {
        cleanup();
        return st;
    }
    cudaError_t e = cudaMemsetAsync(dH, 0, (size_t)(d + 1) * d * 8, c->stream);
    if (e == cudaSuccess) {
        if (c->A.prec == ppk::F64) {
            e = cudaMemcpyAsync(V, bh.data(), (size_t)n2 * 8, cudaMemcpyHostToDevice, c->stream);
        } else {
            std::vector<float> f(bh.begin(), bh.end());
            e = cudaMemcpyAsync(V, f.data(), (size_t)n2 * 4, cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // f goes out of scope
        }
    }
    if (e != cudaSuccess) {
        cleanup();
        return pp_fail(PP_ECUDA, "build: upload: %s", cudaGetErrorString(e));
    }
    for (int j = 0; j < d && st >= 0; ++j) {
        const char *vj = (const char *)V + (size_t)j * ldv * esz;
        for (int h = 0; h < 2 && st >= 0; ++h) {
            ppk::StepArgs a;
            a.sigma = c->sigma;
            a.x = vj + (size_t)h * n * esz;
            a.y = (char *)W + (size_t)h * n * esz;
            a.plain = 1;
            st = step(c, a);
        }
        if (st >= 0) st = cgs2_step_n(c, c->A.prec, n2, V, ldv, j + 1, W, dH + (size_t)j * (d + 1));
    }
    std::vector<double> H((size_t)(d + 1) * d, 0.0);
    if (st >= 0) {
        e = cudaMemcpyAsync(H.data(), dH, H.size() * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = pp_fail(PP_ECUDA, "build: %s", cudaGetErrorString(e));
    }
    cleanup();
    if (st < 0) return st;
    CKS(check_sweeps(c));
    return roots_from_hessenberg(c, d, H, 2, 0, out);
}

pp_status pp_build_poly_two(pp_ctx *c, int d, const double *b1, const double *b2, pp_poly **out) {
    if (!c || !b1 || !b2 || !out) return pp_fail(PP_EINVAL, "pp_build_poly_two: bad arguments");
    pp_poly *p = new pp_poly();
    p->ctx = c;
    pp_status st = build_roots_two(c, d, b1, b2, p);
    if (st < 0) {
        delete p;
        return st;
    }
    *out = p;
    return st;
}

pp_status pp_build_poly2(pp_ctx *c, int d1, int d2, const double *b, pp_poly **out) {
    if (!c || !b || !out) return pp_fail(PP_EINVAL, "pp_build_poly2: bad arguments");
    pp_poly *p1 = new pp_poly();
    p1->ctx = c;
    pp_status s1 = build_roots(c, d1, b, nullptr, p1);
    if (s1 < 0) {
        delete p1;
        return s1;
    }
    pp_poly *p = new pp_poly();
    p->ctx = c;
    p->inner = p1;
    pp_status s2 = build_roots(c, d2, b, p1, p);
    if (s2 < 0) {
        delete p;
        return s2;
    }
    *out = p;
    return (s1 == PP_EBREAKDOWN || s2 == PP_EBREAKDOWN) ? PP_EBREAKDOWN : PP_OK;
}

// A polynomial with the given roots in the given order (validated: finite,
// non-zero, conjugate pairs adjacent with im > 0 first).
static pp_status roots_poly(pp_ctx *c, int count, const double *re, const double *im, const char *who,
                            pp_poly **out) {
    if (!c || count < 1 || !re || !im || !out) return pp_fail(PP_EINVAL, "%s: bad arguments", who);
    std::vector<cd> r(count);
    for (int i = 0; i < count; ++i) {
        r[i] = cd(re[i], im[i]);
        if (!std::isfinite(re[i]) || !std::isfinite(im[i]) || (re[i] == 0 && im[i] == 0))
            return pp_fail(PP_EINVAL, "%s: root %d is zero or not finite", who, i);
    }
    for (int i = 0; i < count;) {
        if (r[i].imag() == 0) {
            ++i;
            continue;
        }
        if (r[i].imag() < 0 || i + 1 >= count || r[i + 1] != std::conj(r[i]))
            return pp_fail(PP_EINVAL, "%s: pair at %d not adjacent (im > 0 first)", who, i);
        i += 2;
    }
    pp_poly *p = new pp_poly();
    p->ctx = c;
    p->roots = r;
    p->steps = steps_of(r);
    p->degree = count;
    *out = p;
    return PP_OK;
}

pp_status pp_poly_from_roots(pp_ctx *c, int count, const double *re, const double *im, pp_poly **out) {
    return roots_poly(c, count, re, im, "pp_poly_from_roots", out);
}

pp_status pp_poly2_from_roots(pp_ctx *c, int count1, const double *re1, const double *im1, int count2,
                              const double *re2, const double *im2, pp_poly **out) {
    if (!out) return pp_fail(PP_EINVAL, "pp_poly2_from_roots: bad arguments");
    pp_poly *inner = nullptr, *p = nullptr;
    CKS(roots_poly(c, count1, re1, im1, "pp_poly2_from_roots (inner)", &inner));
    pp_status st = roots_poly(c, count2, re2, im2, "pp_poly2_from_roots (outer)", &p);
    if (st < 0) {
        delete inner;
        return st;
    }
    p->inner = inner;
    *out = p;
    return PP_OK;
}

static pp_status copy_roots(const std::vector<cd> &r, double *re, double *im, int cap, int *count) {
    if (count) *count = (int)r.size();
    for (int i = 0; i < (int)r.size() && i < cap; ++i) {
        if (re) re[i] = r[i].real();
        if (im) im[i] = r[i].imag();
    }
    return PP_OK;
}

pp_status pp_poly_roots(const pp_poly *p, double *re, double *im, int cap, int *count) {
    if (!p) return pp_fail(PP_EINVAL, "pp_poly_roots: null poly");
    return copy_roots(p->roots, re, im, cap, count);
}

pp_status pp_poly_inner_roots(const pp_poly *p, double *re, double *im, int cap, int *count) {
    if (!p) return pp_fail(PP_EINVAL, "pp_poly_inner_roots: null poly");
    if (!p->inner) {
        if (count) *count = 0;
        return PP_OK;
    }
    return copy_roots(p->inner->roots, re, im, cap, count);
}

pp_status pp_poly_info(const pp_poly *p, int *degree, int *added) {
    if (!p) return pp_fail(PP_EINVAL, "pp_poly_info: null poly");
    if (degree) *degree = p->degree;
    if (added) *added = p->added;
    return PP_OK;
}

pp_status pp_poly_counts(const pp_poly *p, int64_t *mvps, int64_t *dots, int64_t *vops) {
    if (!p) return pp_fail(PP_EINVAL, "pp_poly_counts: null poly");
    int64_t a = p->mvps, b = p->dots, v = p->vops;
    if (p->inner) {
        a += p->inner->mvps;
        b += p->inner->dots;
        v += p->inner->vops;
    }
    if (mvps) *mvps = a;
    if (dots) *dots = b;
    if (vops) *vops = v;
    return PP_OK;
}

void pp_poly_destroy(pp_poly *p) { delete p; }

pp_status pp_apply(const pp_poly *p, const void *x_dev, void *y_dev) {
    if (!p || !x_dev || !y_dev) return pp_fail(PP_EINVAL, "pp_apply: bad arguments");
    return op_apply(p->ctx, p, x_dev, y_dev);
}

pp_status pp_apply_host(const pp_poly *p, const double *x, double *y) {
    if (!p || !x || !y) return pp_fail(PP_EINVAL, "pp_apply_host: bad arguments");
    pp_ctx *c = p->ctx;
    void *dx = nullptr;
    CK(cudaMalloc(&dx, c->ldv() * c->esz));
    pp_status st = upload_vec(c, x, 1.0, dx);
    if (st >= 0) st = op_apply(c, p, dx, dx);
    std::vector<double> out;
    if (st >= 0) st = download_vecs(c, dx, c->ldv(), 1, out, c->A.prec);
    cudaFree(dx);
    if (st < 0) return st;
    std::memcpy(y, out.data(), c->n * 8);
    return PP_OK;
}

}  // extern "C"
