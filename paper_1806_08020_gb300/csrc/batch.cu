// Batched and served polynomial preconditioned Arnoldi: many independent
// eigenproblems of different sizes, degrees and subspace dimensions advance
// together on one GPU.
//
// Every request keeps its own context (matrix, scratch, FP64 residual
// operator), polynomial and basis.  The Arnoldi steps run in lockstep: at
// step jj every request whose window [j0, m) contains jj applies its own
// factored polynomial (Eq. (2.1)) and orthogonalises with CGS2 (Section 4).
// One step is one persistent launch per polynomial pass across all requests
// (each reads its own pass descriptor), three batched CGS2 sweeps and a
// batched normalisation.  Request state lives in device tables; while the set
// of requests does not change, each step is replayed from a CUDA graph
// captured once.  The per-cycle host work (Ritz values, FP64 convergence test
// on A, refinement, thick restart) is the single-instance code of driver.h.
// Mixed precision: each FP32 request runs one FP32 cycle as a warm start; one
// still more than 10 rtol from converging then moves to a second engine of
// FP64 twins, nearer ones are refined in FP64 first.
//
// pp_batch_* solves a fixed set to completion; pp_server_* admits requests as
// device memory and slots free up (continuous batching) and retires each as
// soon as it converges.
#include "driver.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <map>
#include <memory>
#include <mutex>

using namespace ppi;

namespace {

struct Req {
    int64_t id = -1;
    pp_ctx *c = nullptr;     // the context the request currently runs on
    pp_ctx *home = nullptr;  // its own context (c, or c's FP64 twin after a switch)
    bool own_ctx = false;
    bool to64 = false;       // leaves the FP32 engine for the FP64 one
    pp_poly *poly = nullptr;
    std::unique_ptr<Driver> D;
    void *V = nullptr, *V2 = nullptr;
    double *dH = nullptr;
    int d = 0, nev = 0, m = 0, k = 0;
    double rtol = 1e-8;
    int j0 = 0;
    bool done = false, conv = false;
    pp_status status = PP_OK;
    Cycle cy;
    RitzOut R;
    MixedSwitch sw{1e-8};
    pp_stats S{};
    std::vector<ppk::BatchPassEntry> passes;
    int nblk = 0, blk0 = 0;
    int64_t launches0 = 0, cycles32 = 0;
    bool want_x = false;
    std::vector<double> lam_re, lam_im, resid, X;  // results
    int nout = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t bytes = 0;  // device memory estimate (admission)
    // request inputs kept on the host until admission (server)
    int64_t n = 0;
    std::vector<int64_t> rowptr;
    std::vector<int32_t> colind;
    std::vector<double> vals, b, v0;
    std::vector<void *> dev;

    ~Req() { release_device(); }
    void release_device() {
        if (c) cudaStreamSynchronize(c->stream);
        D.reset();
        for (void *p : dev) cudaFree(p);
        dev.clear();
        delete poly;
        poly = nullptr;
        if (own_ctx && home) pp_destroy(home);
        if (own_ctx) c = home = nullptr;
    }
    void dfree(void *p) {
        for (auto it = dev.begin(); it != dev.end(); ++it)
            if (*it == p) {
                cudaFree(p);
                dev.erase(it);
                return;
            }
    }
    int64_t launches_now() const { return home->launches + (home->twin ? home->twin->launches : 0); }
    pp_status dalloc(void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return pp_fail(PP_ENOMEM, "request: cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        }
        dev.push_back(*p);
        return PP_OK;
    }
};

// A context for one instance of the batched engine: diagonal storage when the
// matrix fits it (stencil and banded matrices; opts.format AUTO or DIA), else
// SELL-32.  The batched kernels tune their own block shape, so the per-matrix
// tuner is kept to a minimum (fixed chunk height, row loop and DIA row loop).
static pp_status create_member(pp_ctx **out, int64_t n, const int64_t *rowptr, const int32_t *colind,
                               const double *vals, const pp_opts &base, cudaStream_t stream, int make_twin) {
    pp_opts o = base;
    o.stream = stream;
    if (!o.sell_c) o.sell_c = 32;
    if (!o.sell_loop) o.sell_loop = 1;
    if (!o.dia_loop) o.dia_loop = 1;
    if (base.format == PP_FMT_AUTO || base.format == PP_FMT_DIA) {
        o.format = PP_FMT_DIA;
        pp_status st = pp_create_internal(out, n, rowptr, colind, vals, &o, make_twin);
        if (st != PP_EINVAL || base.format == PP_FMT_DIA) return st;
    }
    o.format = PP_FMT_SELL;
    return pp_create_internal(out, n, rowptr, colind, vals, &o, make_twin);
}

// Device bytes a request holds while admitted (matrix with SELL padding
// headroom, FP64 residual operator, scratch, two basis slabs, Hessenberg,
// FP64 test buffers, reduction scratch).
int64_t request_bytes(int64_t n, int64_t nnz, int m, int nev, int esz) {
    int64_t ldv = (n + 31) / 32 * 32;
    int64_t mat = nnz * (esz + 4) * 13 / 10 + nnz * 12 + 8 * n;
    int64_t vecs = 8 * ldv * esz + 2 * (int64_t)(m + 1) * ldv * esz;
    int64_t test = 2 * (int64_t)(nev + 2) * ldv * 8 + (int64_t)(nev + 2) * ldv * esz;
    int64_t small = (int64_t)(m + 1) * m * 8 + 128 * 128 * 8 + 1300000 * 8;
    int64_t twin = 0;  // FP64 copy of an FP32 request and its basis (if FP32 cannot reach rtol)
    if (esz != 8)
        twin = nnz * 12 * 13 / 10 + nnz * 12 + 8 * n + 8 * ldv * 8 + 1300000 * 8 + 2 * (int64_t)(m + 1) * ldv * (8 - esz) +
               (int64_t)32 * ldv * 8 + 128 * 128 * 8;  // the refinement's extra Ritz vectors
    return mat + vecs + test + small + twin;
}

// Pass schedule of one polynomial (the single-apply schedule with buffer ids:
// 0 input V[:, jj], 1 output W, 2/3 ping-pong, 4 pair temporary).
std::vector<ppk::BatchPassEntry> pass_schedule(const pp_poly *p) {
    std::vector<ppk::BatchPassEntry> out;
    int cur = 0;
    const auto &st = p->steps;
    for (size_t i = 0; i < st.size(); ++i) {
        bool last = i + 1 == st.size();
        int dst = last ? 1 : (cur == 2 ? 3 : 2);
        if (!st[i].pair) {
            out.push_back({1, cur, dst, 0, 0.0, st[i].c, 0.f, (float)st[i].c});
        } else {
            out.push_back({0, cur, 4, 0, 0.0, 0.0, 0.f, 0.f});
            out.push_back({2, 4, dst, cur, st[i].c1, -st[i].c2, (float)st[i].c1, (float)-st[i].c2});
        }
        cur = dst;
    }
    return out;
}

template <typename T>
struct DevArray {
    T *p = nullptr;
    size_t cap = 0;
    ~DevArray() { cudaFree(p); }
    pp_status ensure(size_t count) {
        if (count <= cap) return PP_OK;
        cudaFree(p);
        p = nullptr;
        size_t c2 = std::max(count, cap * 2);
        cudaError_t e = cudaMalloc(&p, sizeof(T) * c2);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cap = 0;
            return pp_fail(PP_ENOMEM, "engine tables: %s", cudaGetErrorString(e));
        }
        cap = c2;
        return PP_OK;
    }
};

class Engine {
  public:
    cudaStream_t st = nullptr;
    int max_cycles = 2000, refine_steps = 4;
    int64_t launches = 0;
    std::vector<Req *> act;  // not owned

    ~Engine() {
        free_graphs();
        cudaFree(Z);
        cudaFree(dG);
    }

    // Build the request's polynomial and Arnoldi state; it joins the set.
    pp_status start(Req *r, const double *b, const double *v0) {
        pp_ctx *c = r->c;
        r->home = c;
        r->launches0 = r->launches_now();
        r->sw = MixedSwitch(r->rtol);
        r->t_start = now();
        CKS(pp_build_poly(c, r->d, b, &r->poly));
        r->passes = pass_schedule(r->poly);
        return begin(r, v0);
    }

    // A request whose FP32 cycle (and refinement, when it was near rtol) did
    // not reach rtol joins the FP64 engine: the FP32 basis is released and
    // FP64 Arnoldi cycles on the FP64 twin start from the sum of its Ritz
    // vectors (the same polynomial; the cycle count continues).
    pp_status start64(Req *r) {
        pp_ctx *c = r->c;
        std::vector<double> Yh, w0(c->n, 0.0);
        CKS(download_vecs(c, r->D->Y64, c->ldv(), r->cy.sl.nw, Yh, ppk::F64));
        for (int q = 0; q < r->cy.sl.nw; ++q)
            for (int64_t x = 0; x < c->n; ++x) w0[x] += Yh[(size_t)q * c->n + x];
        if (!c->h_bal.empty())  // balanced: back to S's coordinates
            for (int64_t x = 0; x < c->n; ++x) w0[x] /= c->h_bal[x];
        r->D.reset();
        r->dfree(r->V);
        r->dfree(r->V2);
        r->dfree(r->dH);
        r->c = c->twin;
        r->to64 = false;
        r->done = false;
        r->conv = false;
        r->status = PP_OK;
        r->cycles32 = r->S.cycles;
        return begin(r, w0.data());
    }

  private:
    // Basis slabs, Hessenberg and test buffers on the request's current
    // context, v_1 = v0 / ||v0|| (all ones when v0 is null); joins the set.
    pp_status begin(Req *r, const double *v0) {
        pp_ctx *c = r->c;
        const int64_t ldv = c->ldv();
        const int ldh = r->m + 1;
        CKS(r->dalloc(&r->V, (size_t)ldv * (r->m + 1) * c->esz));
        CKS(r->dalloc(&r->V2, (size_t)ldv * (r->m + 1) * c->esz));
        CKS(r->dalloc((void **)&r->dH, (size_t)ldh * r->m * 8));
        r->D.reset(new Driver{c, c->n, ldv, r->nev + 1});
        CKS(r->D->alloc_test_buffers(c->A.prec != ppk::F64));
        std::vector<double> v(c->n, 1.0);
        if (v0) std::copy(v0, v0 + c->n, v.begin());
        double nv = 0;
        for (double x : v) nv += x * x;
        nv = std::sqrt(nv);
        if (!(nv > 0)) return pp_fail(PP_EINVAL, "zero start vector");
        CKS(upload_vec(c, v.data(), 1.0 / nv, r->V));
        CK(cudaMemsetAsync(r->dH, 0, (size_t)ldh * r->m * 8, st));
        r->j0 = 0;
        r->S.dots += 1;
        r->S.vops += 2;
        act.push_back(r);
        dirty = true;
        return PP_OK;
    }

  public:

    // Drop finished requests from the set; returns them.
    std::vector<Req *> retire() {
        std::vector<Req *> out, keep;
        for (Req *r : act) (r->done ? out : keep).push_back(r);
        if (!out.empty()) dirty = true;
        act.swap(keep);
        return out;
    }

    // One lockstep cycle: every active request extends its basis from j0 to m,
    // then its host step runs (test, refine or restart).
    pp_status cycle() {
        if (act.empty()) return PP_OK;
        const bool changed = dirty;
        const bool tr = trace_on();
        const double t0 = tr ? now() : 0.0;
        if (dirty) CKS(build_tables());
        const double t1 = tr ? now() : 0.0;
        const int count = (int)act.size();
        int jmin = 1 << 30, jmax = 0;
        std::vector<int> lo(count), hi(count);
        for (int i = 0; i < count; ++i) {
            lo[i] = act[i]->j0;
            hi[i] = act[i]->done ? 0 : act[i]->m;
            if (!act[i]->done) {
                jmin = std::min(jmin, lo[i]);
                jmax = std::max(jmax, hi[i]);
            }
        }
        CK(cudaMemcpyAsync(d_lo.p, lo.data(), 4 * count, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_hi.p, hi.data(), 4 * count, cudaMemcpyHostToDevice, st));
        for (int jj = jmin; jj < jmax; ++jj) {
            if (changed) {
                launch_step(jj);  // the set just changed: plain launches this cycle
            } else {
                if ((int)graphs.size() <= jj) graphs.resize(jj + 1, nullptr);
                if (!graphs[jj]) {
                    cudaGraph_t g = nullptr;
                    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                    launch_step(jj);
                    CK(cudaStreamEndCapture(st, &g));
                    cudaError_t e = cudaGraphInstantiate(&graphs[jj], g, 0);
                    cudaGraphDestroy(g);
                    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "engine: graph: %s", cudaGetErrorString(e));
                }
                CK(cudaGraphLaunch(graphs[jj], st));
            }
            launches += Pmax + 4;
        }
        CK(cudaGetLastError());
        double t2 = 0.0;
        if (tr) {  // (trace only: the wait separates the steps' device time from the host steps)
            CK(cudaStreamSynchronize(st));
            t2 = now();
        }
        for (int i = 0; i < count; ++i) CKS(host_step(i));
        if (tr)
            std::fprintf(stderr, "[pp] engine cycle: %d requests, steps %d..%d, tables %.1f ms, steps %.1f ms, host steps %.1f ms\n",
                         count, jmin, jmax, (t1 - t0) * 1e3, (t2 - t1) * 1e3, (now() - t2) * 1e3);
        return PP_OK;
    }

  private:
    DevArray<ppk::BatchPassInst> d_pinst;
    DevArray<ppk::BatchCgsInst> d_cinst;
    DevArray<ppk::BatchPassEntry> d_tab;
    DevArray<int2> d_items;
    DevArray<ppk::BatchPassEntry> d_tune_tab;
    DevArray<int> d_lo, d_hi;
    int64_t tuned_rows = 0;
    std::vector<ppk::BatchPassInst> pinst;
    std::vector<ppk::BatchCgsInst> cinst;
    std::vector<cudaGraphExec_t> graphs;
    int Pmax = 0, blocks = 0, nitems = 0;
    std::vector<int> item_end;    // work items through instance i (upload_items)
    std::vector<int> pass_items;  // work items of the instances that take pass t (a prefix)
    int groups = 8, grid_per_sm = 8;  // batched-pass block shape (tuned)
    bool dirty = true;
    ppk::Prec pr = ppk::F32;
    double *Z = nullptr, *dG = nullptr;
    int64_t zld = 0;

    void free_graphs() {
        for (auto &g : graphs)
            if (g) cudaGraphExecDestroy(g);
        graphs.clear();
    }

    void launch_step(int jj) {
        const int count = (int)act.size();
        for (int t = 0; t < Pmax; ++t)
            ppk::launch_pass_batch(pr, d_pinst.p, d_tab.p + (size_t)t * count, d_items.p, pass_items[t], d_lo.p,
                                   d_hi.p, jj, groups, grid_per_sm, st);
        for (int mode = 0; mode < 3; ++mode)
            ppk::launch_cgs_batch(pr, d_cinst.p, count, blocks, d_lo.p, d_hi.p, mode, jj, st);
        ppk::launch_scale_batch(pr, d_cinst.p, count, blocks, d_lo.p, d_hi.p, jj, st);
    }

    pp_status build_tables() {
        free_graphs();
        // most passes first: the instances that take pass t are then a prefix of
        // the set, and so are their work items (the pass launches cover only those)
        std::stable_sort(act.begin(), act.end(),
                         [](const Req *a, const Req *b) { return a->passes.size() > b->passes.size(); });
        const int count = (int)act.size();
        pr = act[0]->c->A.prec;
        Pmax = 0;
        for (Req *r : act) Pmax = std::max(Pmax, (int)r->passes.size());
        pinst.assign(count, {});
        cinst.assign(count, {});
        std::vector<ppk::BatchPassEntry> tab((size_t)Pmax * count);
            blocks = 0;
        for (int i = 0; i < count; ++i) {
            Req *r = act[i];
            pp_ctx *c = r->c;
            if (c->A.prec != pr || (c->A.fmt != 2 && c->A.fmt != 3))
                return pp_fail(PP_EINVAL, "engine: mixed precisions or a matrix neither SELL nor DIA");
            const auto &A = c->A.sell;
            pinst[i] = {A, c->sigma, (float)c->sigma, r->V, c->ldv(), c->vec[6], c->vec[0], c->vec[1], c->vec[2],
                        c->A.dia, c->A.fmt == 3 ? 1 : 0};
            r->nblk = ppk::cgs_batch_blocks((int)c->n);
            r->blk0 = blocks;
            blocks += r->nblk;
            cinst[i] = {r->V, c->ldv(), (int)c->n, c->vec[6], r->dH, r->m + 1, c->d_small, c->d_small + 256,
                        c->d_small + 513, c->d_small + 512, c->d_part, c->d_ticket, r->nblk, r->blk0};
            for (int t = 0; t < Pmax; ++t)
                tab[(size_t)t * count + i] =
                    t < (int)r->passes.size() ? r->passes[t] : ppk::BatchPassEntry{-1, 0, 0, 0, 0, 0, 0.f, 0.f};
        }
        CKS(d_pinst.ensure(count));
        CKS(d_cinst.ensure(count));
        CKS(d_tab.ensure(tab.size()));
        CKS(d_lo.ensure(count));
        CKS(d_hi.ensure(count));
        CK(cudaMemcpyAsync(d_pinst.p, pinst.data(), sizeof(pinst[0]) * count, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_cinst.p, cinst.data(), sizeof(cinst[0]) * count, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_tab.p, tab.data(), sizeof(tab[0]) * tab.size(), cudaMemcpyHostToDevice, st));
        int64_t rows = 0;
        for (Req *r : act) rows += r->c->n;
        if (tuned_rows == 0 || rows > 2 * tuned_rows || 2 * rows < tuned_rows) {
            CKS(tune_pass());
            tuned_rows = rows;
        }
        CKS(upload_items(groups));
        pass_items.assign(Pmax, 0);
        for (int t = 0; t < Pmax; ++t) {
            int L = 0;
            while (L < count && (int)act[L]->passes.size() > t) ++L;
            pass_items[t] = L > 0 ? item_end[L - 1] : 0;
        }
        CK(cudaStreamSynchronize(st));
        dirty = false;
        return PP_OK;
    }

    // Work items (instance, first 32-row group), `g` warps per block (a warp takes
    // one 32-row group, two for an FP32 DIA instance).
    pp_status upload_items(int g) {
        std::vector<int2> items;
        item_end.assign(act.size(), 0);
        for (int i = 0; i < (int)act.size(); ++i) {
            const int ngroups = (int)((act[i]->c->n + 31) / 32);
            // an FP32 DIA instance's warps take two 32-row groups each (two rows per lane)
            const int step = act[i]->c->A.fmt == 3 && act[i]->c->A.prec == ppk::F32 ? 2 * g : g;
            for (int g0 = 0; g0 < ngroups; g0 += step) items.push_back(make_int2(i, g0));
            item_end[i] = (int)items.size();
        }
        nitems = (int)items.size();
        CKS(d_items.ensure(items.size()));
        CK(cudaMemcpyAsync(d_items.p, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, st));
        return PP_OK;
    }

    // Batched-pass tuner: the block shape (32-row groups per block: 64 to 512
    // threads) and the grid (blocks per SM) that run one product with A of
    // every instance fastest, timed with CUDA events on the engine's stream
    // (fastest of five launches after two warm-up ones).  The timed pass reads
    // v_1 and writes the operator output, which the first real step overwrites.
    // Re-run when the set's total size changes by more than 2x.  PP_BATCH_SHAPE
    // = "g,b" fixes g warps per block and b blocks per SM instead (for
    // profiling: under a profiler the timings mislead the tuner).
    pp_status tune_pass() {
        if (const char *fix = std::getenv("PP_BATCH_SHAPE")) {
            int g = 0, b = 0;
            if (std::sscanf(fix, "%d,%d", &g, &b) == 2 && (g == 2 || g == 4 || g == 8 || g == 16) && b >= 1 &&
                b <= 32) {
                groups = g;
                grid_per_sm = b;
                return PP_OK;
            }
        }
        const int count = (int)act.size();
        std::vector<ppk::BatchPassEntry> tab(count, ppk::BatchPassEntry{0, 0, 1, 0, 0.0, 0.0, 0.f, 0.f});
        std::vector<int> lo(count, 0), hi(count, 1);
        CKS(d_tune_tab.ensure(count));
        CK(cudaMemcpyAsync(d_tune_tab.p, tab.data(), sizeof(tab[0]) * count, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_lo.p, lo.data(), 4 * count, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_hi.p, hi.data(), 4 * count, cudaMemcpyHostToDevice, st));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        double best = INFINITY;
        for (int g : {2, 4, 8, 16}) {
            pp_status s = upload_items(g);
            if (s < 0) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return s;
            }
            for (int gps : {4, 8, 16, 32}) {
                double t = INFINITY;
                for (int it = 0; it < 7; ++it) {
                    cudaEventRecord(e0, st);
                    ppk::launch_pass_batch(pr, d_pinst.p, d_tune_tab.p, d_items.p, nitems, d_lo.p, d_hi.p, 0, g, gps,
                                           st);
                    cudaEventRecord(e1, st);
                    float ms = 0;
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (it >= 2) t = std::min(t, (double)ms);
                }
                launches += 7;
                if (trace_on())
                    std::fprintf(stderr, "[pp] batch pass tuner: %d instances, %d threads/block, %d blocks/SM: %.1f us\n",
                                 count, 32 * g, gps, t * 1e3);
                if (t < best) {
                    best = t;
                    groups = g;
                    grid_per_sm = gps;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        CK(cudaGetLastError());
        return PP_OK;
    }

    pp_status shared_refinement_basis(Req *r) {
        const int64_t ldv = r->c->ldv();
        if (zld < ldv) {
            cudaFree(Z);
            cudaFree(dG);
            Z = nullptr;
            dG = nullptr;
            CK(cudaMalloc(&Z, (size_t)ldv * (Driver::kZcap + 1) * 8));
            CK(cudaMalloc(&dG, (size_t)(Driver::kZcap + 1) * Driver::kZcap * 8));
            zld = ldv;
        }
        r->D->Z = Z;
        r->D->dG = dG;
        return PP_OK;
    }

    void finish(Req *r) {
        pp_ctx *c = r->c;
        r->done = true;
        r->t_done = now();
        const int cap = r->nev + 1;
        r->lam_re.assign(cap, 0.0);
        r->lam_im.assign(cap, 0.0);
        r->resid.assign(cap, 0.0);
        if (r->status < 0 || r->cy.sl.nw == 0) {
            r->nout = 0;
            return;
        }
        std::vector<double> Yh;
        if (r->want_x) {
            r->X.assign((size_t)c->n * cap, 0.0);
            if (download_vecs(c, r->D->Y64, c->ldv(), r->cy.sl.nw, Yh, ppk::F64) < 0) {
                r->status = PP_ECUDA;
                r->nout = 0;
                return;
            }
        }
        double maxres = 0;
        write_outputs(c->opts.target, c->n, r->cy.sl, r->R, Yh, r->lam_re.data(), r->lam_im.data(), r->resid.data(),
                      r->want_x ? r->X.data() : nullptr, maxres);
        r->nout = r->cy.sl.nw;
        r->S.converged = r->conv ? 1 : 0;
        r->S.max_resid = maxres;
        r->S.kernel_launches = r->launches_now() - r->launches0;
        r->S.t_total = r->t_done - r->t_start;
        r->S.fp64_cycles = c->A.prec == ppk::F64 ? r->S.cycles - r->cycles32 : 0;
    }

    pp_status host_step(int i) {
        Req *r = act[i];
        if (r->done) return PP_OK;
        pp_ctx *c = r->c;
        const int m = r->m, ldh = m + 1;
        r->S.cycles++;
        r->S.mvps += op_mvps(r->poly) * (m - r->j0);
        for (int j = r->j0; j < m; ++j) {
            r->S.dots += 2 * (j + 1) + 1;
            r->S.vops += 4 * (j + 1) + 2 + op_vops(r->poly);
        }
        std::vector<double> H((size_t)ldh * m);
        CK(cudaMemcpyAsync(H.data(), r->dH, H.size() * 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        pp_status s = wanted_set(H, ldh, m, r->nev, 1.0, r->cy);
        if (s >= 0) s = r->D->ritz_test(r->V, c->A.prec, m, r->cy.Sw, r->cy.sl, r->rtol, r->R, r->S);
        if (s < 0) {
            r->status = s;
            finish(r);
            return PP_OK;
        }
        r->S.nconv = r->R.nconv;
        trace_cycle("req", r, r->S.cycles, c->A.prec == ppk::F64 ? 64 : 32, r->R, r->R.all ? "converged" : nullptr);
        if (r->R.all) {
            r->conv = true;
            r->status = PP_OK;
            finish(r);
            return PP_OK;
        }
        const bool last = r->S.cycles >= max_cycles;
        const bool refine_now = c->A.prec != ppk::F64 && r->sw.should_refine(r->R, last);
        if (c->A.prec != ppk::F64 && c->twin && !last) {
            // One FP32 cycle is the warm start: a request not within ten times
            // rtol of converging joins the batched FP64 engine at once, from its
            // FP32 Ritz vectors; within it, the FP64 refinement is tried first.
            // (On the batched workloads the FP32 floor, 1e-7 to 1e-6 relative, is
            // reached in a cycle or two, further FP32 cycles shorten the FP64
            // continuation little, and the refinement runs outside the batched
            // launches: measured on the 64-instance batch, handing over after
            // the first cycle beats waiting for a stalled one by 11 %.)
            const double mx = *std::max_element(r->R.res.begin(), r->R.res.end());
            if (mx > 10 * r->rtol) {
                trace_cycle("req", r, r->S.cycles, 32, r->R, "to fp64");
                r->status = PP_OK;
                r->to64 = true;
                r->done = true;
                return PP_OK;
            }
        }
        if (refine_now) {
            CKS(shared_refinement_basis(r));
            s = r->D->refine(r->poly, r->cy.sl, r->nev, r->R, r->rtol, refine_steps, 3, r->S, &r->cy, r->V, c->A.prec,
                             r->m);
            trace_cycle("req", r, r->S.cycles, 64, r->R, r->R.all ? "refined: converged" : "refined");
            r->conv = s >= 0 && r->R.all;
            r->status = s < 0 ? s : (r->conv ? PP_OK : PP_ENOTCONV);
            if (s >= 0 && !r->conv && c->twin && !last) {
                r->to64 = true;  // continues in the FP64 engine (start64)
                r->done = true;
                return PP_OK;
            }
            if (s < 0 || r->conv || last) {
                finish(r);
                return PP_OK;
            }
            r->status = PP_OK;
            r->sw.reset();  // no FP64 twin: keep cycling in FP32
        }
        if (last) {
            r->status = PP_ENOTCONV;
            finish(r);
            return PP_OK;
        }
        std::vector<double> Q, Hn;
        int kk = restart_basis(r->cy, H, ldh, r->k, Q, Hn);
        const int64_t ldv = c->ldv();
        CK(cudaMemcpyAsync(r->D->dQ, Q.data(), Q.size() * 8, cudaMemcpyHostToDevice, st));
        ppk::launch_rotate(c->A.prec, (int)c->n, r->V, ldv, m, r->D->dQ, kk, r->V2, ldv, st);
        CK(cudaMemcpyAsync((char *)r->V2 + (size_t)kk * ldv * c->esz, (char *)r->V + (size_t)m * ldv * c->esz,
                           c->n * c->esz, cudaMemcpyDeviceToDevice, st));
        std::swap(r->V, r->V2);
        r->S.vops += (int64_t)m * kk;
        CK(cudaMemcpyAsync(r->dH, Hn.data(), Hn.size() * 8, cudaMemcpyHostToDevice, st));
        r->j0 = kk;
        // the tables point at the current basis slab
        pinst[i].V = r->V;
        cinst[i].V = r->V;
        CK(cudaMemcpyAsync(d_pinst.p + i, &pinst[i], sizeof(pinst[i]), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(d_cinst.p + i, &cinst[i], sizeof(cinst[i]), cudaMemcpyHostToDevice, st));
        return PP_OK;
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Batch: a fixed set solved to completion
// ---------------------------------------------------------------------------
struct pp_batch {
    int count = 0;
    pp_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<pp_ctx *> ctx;
    int64_t launches = 0;
    ~pp_batch() {
        if (stream) cudaStreamSynchronize(stream);
        for (pp_ctx *c : ctx) pp_destroy(c);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

// ---------------------------------------------------------------------------
// Server: continuous batching of a request stream
// ---------------------------------------------------------------------------
struct pp_server {
    pp_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t budget = 0, used = 0;
    int max_active = 256;
    int keep_vectors = 0;
    int64_t next_id = 0;
    std::mutex mu;  // guards the queue and the results (submit/result may come from other threads)
    std::deque<std::unique_ptr<Req>> queue;
    std::vector<std::unique_ptr<Req>> running;
    std::map<int64_t, std::unique_ptr<Req>> finished;
    Engine eng, eng64;  // FP32 (or FP64) cycles; FP64 continuations of FP32 requests
    ~pp_server() {
        if (stream) cudaStreamSynchronize(stream);
        running.clear();
        finished.clear();
        queue.clear();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

extern "C" {

pp_status pp_batch_create(pp_batch **out, int count, const int64_t *n, const int64_t *const *rowptr,
                          const int32_t *const *colind, const double *const *vals, const pp_opts *opts) {
    if (!out || count < 1 || !n || !rowptr || !colind || !vals) return pp_fail(PP_EINVAL, "pp_batch_create: bad arguments");
    *out = nullptr;
    auto *b = new pp_batch();
    b->count = count;
    pp_opts_default(&b->opts);
    if (opts) b->opts = *opts;
    if (b->opts.precision == PP_FP32_BF16) {
        delete b;
        return pp_fail(PP_EINVAL, "pp_batch_create: the batched engine runs PP_FP64 or PP_FP32");
    }
    if (b->opts.restart != PP_RESTART_RITZ) {
        delete b;
        return pp_fail(PP_EINVAL, "pp_batch_create: the batched engine restarts with Ritz vectors only");
    }
    if (b->opts.stream) {
        b->stream = (cudaStream_t)b->opts.stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return pp_fail(PP_ECUDA, "pp_batch_create: stream");
        }
        b->own_stream = true;
    }
    b->ctx.assign(count, nullptr);
    for (int i = 0; i < count; ++i) {
        pp_status st = create_member(&b->ctx[i], n[i], rowptr[i], colind[i], vals[i], b->opts, b->stream, 1);
        if (st < 0) {
            delete b;
            return st;
        }
    }
    *out = b;
    return PP_OK;
}

void pp_batch_destroy(pp_batch *b) { delete b; }

int64_t pp_batch_launch_count(const pp_batch *b) { return b ? b->launches : 0; }

pp_status pp_batch_solve(pp_batch *b, const int *d, const double *const *bvec, const double *const *v0, int nev, int m,
                         int k, double rtol, double *const *lam_re, double *const *lam_im, double *const *X,
                         double *const *resid, int *nout, pp_stats *stats) {
    if (!b || !d || !bvec || !lam_re || !lam_im || !resid || !nout || nev < 1 || k <= nev || m <= k || m > 127 ||
        !(rtol > 0))
        return pp_fail(PP_EINVAL, "pp_batch_solve: need 1 <= nev < k < m <= 127, rtol > 0 and outputs");
    for (pp_ctx *c : b->ctx)
        if (m >= c->n) return pp_fail(PP_EINVAL, "pp_batch_solve: m must be below every n");
    Engine eng, eng64;  // FP32 (or FP64) cycles; FP64 continuations of FP32 requests
    for (Engine *e : {&eng, &eng64}) {
        e->st = b->stream;
        e->max_cycles = b->opts.max_cycles;
        e->refine_steps = b->opts.refine_steps;
    }
    std::vector<std::unique_ptr<Req>> reqs;
    int64_t l0 = 0;
    for (pp_ctx *c : b->ctx) l0 += c->launches + (c->twin ? c->twin->launches : 0);
    for (int i = 0; i < b->count; ++i) {
        auto r = std::make_unique<Req>();
        r->c = b->ctx[i];
        r->d = d[i];
        r->nev = nev;
        r->m = m;
        r->k = k;
        r->rtol = rtol;
        r->want_x = X && X[i];
        CKS(eng.start(r.get(), bvec[i], v0 ? v0[i] : nullptr));
        reqs.push_back(std::move(r));
    }
    while (!eng.act.empty() || !eng64.act.empty()) {
        CKS(eng.cycle());
        CKS(eng64.cycle());
        for (Req *r : eng.retire())
            if (r->to64) CKS(eng64.start64(r));
        eng64.retire();
    }
    pp_status worst = PP_OK;
    for (int i = 0; i < b->count; ++i) {
        Req *r = reqs[i].get();
        nout[i] = r->nout;
        std::copy(r->lam_re.begin(), r->lam_re.begin() + r->nout, lam_re[i]);
        std::copy(r->lam_im.begin(), r->lam_im.begin() + r->nout, lam_im[i]);
        std::copy(r->resid.begin(), r->resid.begin() + r->nout, resid[i]);
        if (r->want_x) std::copy(r->X.begin(), r->X.begin() + (size_t)r->c->n * r->nout, X[i]);
        if (stats) stats[i] = r->S;
        if (r->status < 0) worst = r->status;
        if (r->status == PP_ENOTCONV && worst == PP_OK) worst = PP_ENOTCONV;
    }
    int64_t l1 = 0;
    for (pp_ctx *c : b->ctx) l1 += c->launches + (c->twin ? c->twin->launches : 0);
    b->launches += eng.launches + eng64.launches + (l1 - l0);
    if (worst == PP_ENOTCONV) return pp_fail(PP_ENOTCONV, "pp_batch_solve: some instances did not converge");
    return worst;
}

pp_status pp_server_create(pp_server **out, const pp_opts *opts, int64_t mem_budget, int max_active,
                           int keep_vectors) {
    if (!out) return pp_fail(PP_EINVAL, "pp_server_create: null out");
    auto *s = new pp_server();
    pp_opts_default(&s->opts);
    if (opts) s->opts = *opts;
    if (s->opts.precision == PP_FP32_BF16) {
        delete s;
        return pp_fail(PP_EINVAL, "pp_server_create: the served engine runs PP_FP64 or PP_FP32");
    }
    if (s->opts.restart != PP_RESTART_RITZ) {
        delete s;
        return pp_fail(PP_EINVAL, "pp_server_create: the served engine restarts with Ritz vectors only");
    }
    if (s->opts.stream) {
        s->stream = (cudaStream_t)s->opts.stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return pp_fail(PP_ECUDA, "pp_server_create: stream");
        }
        s->own_stream = true;
    }
    if (mem_budget <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        mem_budget = (int64_t)(0.8 * (double)fr);
    }
    s->budget = mem_budget;
    s->max_active = max_active > 0 ? max_active : 256;
    s->keep_vectors = keep_vectors;
    for (Engine *e : {&s->eng, &s->eng64}) {
        e->st = s->stream;
        e->max_cycles = s->opts.max_cycles;
        e->refine_steps = s->opts.refine_steps;
    }
    *out = s;
    return PP_OK;
}

void pp_server_destroy(pp_server *s) { delete s; }

pp_status pp_server_submit(pp_server *s, int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals,
                           int d, int nev, int m, int k, double rtol, const double *b, const double *v0, int64_t *id) {
    if (!s || n <= 0 || !rowptr || !colind || !vals || !b || !id || nev < 1 || k <= nev || m <= k || m > 127 ||
        m >= n || d < 1 || !(rtol > 0))
        return pp_fail(PP_EINVAL, "pp_server_submit: bad arguments");
    auto r = std::make_unique<Req>();
    r->n = n;
    r->rowptr.assign(rowptr, rowptr + n + 1);
    r->colind.assign(colind, colind + rowptr[n]);
    r->vals.assign(vals, vals + rowptr[n]);
    r->b.assign(b, b + n);
    if (v0) r->v0.assign(v0, v0 + n);
    r->d = d;
    r->nev = nev;
    r->m = m;
    r->k = k;
    r->rtol = rtol;
    r->want_x = s->keep_vectors != 0;
    r->t_submit = now();
    r->bytes = request_bytes(n, rowptr[n], m, nev, s->opts.precision == PP_FP64 ? 8 : 4);
    if (r->bytes > s->budget)
        return pp_fail(PP_ENOMEM, "pp_server_submit: request needs %lld bytes, budget %lld", (long long)r->bytes,
                       (long long)s->budget);
    std::lock_guard<std::mutex> g(s->mu);
    r->id = s->next_id++;
    *id = r->id;
    s->queue.push_back(std::move(r));
    return PP_OK;
}

pp_status pp_server_step(pp_server *s, int *active, int *queued) {
    if (!s) return pp_fail(PP_EINVAL, "pp_server_step: null server");
    // admit from the queue head while memory and slots allow (FIFO)
    for (;;) {
        std::unique_ptr<Req> r;
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (s->queue.empty()) break;
            Req *h = s->queue.front().get();
            if ((int)s->running.size() >= s->max_active || s->used + h->bytes > s->budget) break;
            r = std::move(s->queue.front());
            s->queue.pop_front();
        }
        pp_status st = create_member(&r->c, r->n, r->rowptr.data(), r->colind.data(), r->vals.data(), s->opts,
                                     s->stream, s->opts.precision != PP_FP64);
        r->own_ctx = st >= 0;
        if (st >= 0) st = s->eng.start(r.get(), r->b.data(), r->v0.empty() ? nullptr : r->v0.data());
        std::vector<int64_t>().swap(r->rowptr);
        std::vector<int32_t>().swap(r->colind);
        std::vector<double>().swap(r->vals);
        if (st < 0) {
            r->status = st;
            r->done = true;
            r->t_done = now();
            r->release_device();
            std::lock_guard<std::mutex> g(s->mu);
            s->finished[r->id] = std::move(r);
            continue;
        }
        s->used += r->bytes;
        s->running.push_back(std::move(r));
    }
    CKS(s->eng.cycle());
    CKS(s->eng64.cycle());
    std::vector<Req *> out = s->eng64.retire();
    for (Req *r : s->eng.retire()) {
        if (!r->to64) {
            out.push_back(r);
        } else if (s->eng64.start64(r) < 0) {
            r->status = PP_ECUDA;
            out.push_back(r);
        }
    }
    for (Req *r : out) {
        for (auto it = s->running.begin(); it != s->running.end(); ++it)
            if (it->get() == r) {
                std::unique_ptr<Req> own = std::move(*it);
                s->running.erase(it);
                s->used -= own->bytes;
                own->release_device();  // keep only the host results
                std::lock_guard<std::mutex> g(s->mu);
                s->finished[own->id] = std::move(own);
                break;
            }
    }
    std::lock_guard<std::mutex> g(s->mu);
    if (active) *active = (int)s->running.size();
    if (queued) *queued = (int)s->queue.size();
    return PP_OK;
}

pp_status pp_server_result(pp_server *s, int64_t id, double *lam_re, double *lam_im, double *X, double *resid,
                           int *nout, pp_stats *stats, double *latency) {
    if (!s || !lam_re || !lam_im || !resid || !nout) return pp_fail(PP_EINVAL, "pp_server_result: bad arguments");
    std::unique_ptr<Req> r;
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->finished.find(id);
        if (it == s->finished.end()) return PP_EAGAIN;
        r = std::move(it->second);
        s->finished.erase(it);
    }
    *nout = r->nout;
    std::copy(r->lam_re.begin(), r->lam_re.begin() + r->nout, lam_re);
    std::copy(r->lam_im.begin(), r->lam_im.begin() + r->nout, lam_im);
    std::copy(r->resid.begin(), r->resid.begin() + r->nout, resid);
    if (X && r->want_x) std::copy(r->X.begin(), r->X.begin() + (size_t)r->n * r->nout, X);
    if (stats) *stats = r->S;
    if (latency) *latency = r->t_done - r->t_submit;
    return r->status;
}

int64_t pp_server_launch_count(const pp_server *s) { return s ? s->eng.launches + s->eng64.launches : 0; }

int64_t pp_server_request_bytes(const pp_server *s, int64_t n, int64_t nnz, int m, int nev) {
    if (!s) return -1;
    return request_bytes(n, nnz, m, nev, s->opts.precision == PP_FP64 ? 8 : 4);
}

}  // extern "C"
