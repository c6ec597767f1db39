// Private declarations shared by capi.cu (contexts, polynomials, applies)
// and eigs.cu (the Arnoldi driver): the context and polynomial handles and
// the device-side helpers both use.
#pragma once

#include "pp_internal.h"

#include <cuda_runtime.h>

#include <chrono>
#include <complex>
#include <utility>
#include <vector>

using ppd::cd;

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return pp_fail(e_ == cudaErrorMemoryAllocation ? PP_ENOMEM : PP_ECUDA, "%s: %s (%s:%d)", \
                           #call, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
    } while (0)

#define CKS(expr)                          \
    do {                                   \
        pp_status s_ = (expr);             \
        if (s_ < 0) return s_;             \
    } while (0)


namespace ppi {

struct StepCoef {
    int pair;      // 0: real root, 1: conjugate pair
    double c;      // real: 1/theta
    double c1, c2; // pair: 2 Re(theta)/|theta|^2, 1/|theta|^2
};

inline std::vector<StepCoef> steps_of(const std::vector<cd> &roots) {
    std::vector<StepCoef> s;
    for (size_t i = 0; i < roots.size();) {
        cd t = roots[i];
        if (t.imag() == 0.0) {
            s.push_back({0, 1.0 / t.real(), 0, 0});
            i += 1;
        } else {
            double m2 = t.real() * t.real() + t.imag() * t.imag();
            s.push_back({1, 0, 2.0 * t.real() / m2, 1.0 / m2});
            i += 2;
        }
    }
    return s;
}

inline int mvps_of(const std::vector<StepCoef> &s) {
    int m = 0;
    for (auto &x : s) m += x.pair ? 2 : 1;
    return m;
}

inline double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace ppi

struct pp_ctx {
    int64_t n = 0, nnz = 0;
    pp_opts opts{};
    double norm1 = 0, sigma = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    ppk::Matrix A;     // storage precision (shifted operator uses sigma)
    ppk::Matrix A64;   // FP64 copy for residuals on A (same as A in FP64 mode)
    ppk::Matrix S64;   // FP64 copy of the operator's matrix: S = D^-1 A D when balanced, else A64
    // balancing (opts.balance): the diagonal d of D (largest entry 1) on the device
    // and the host; null / empty when A is used as given
    double *d_bal = nullptr;
    std::vector<double> h_bal;
    size_t esz = 8;    // bytes per stored vector element
    ppk::Prec bprec = ppk::F64;  // Arnoldi basis storage (BF16 for PP_FP32_BF16, else as the vectors)
    size_t besz = 8;             // bytes per basis element
    std::vector<void *> allocs;
    // scratch (vec[8]: FP32 copy of a BF16 basis vector)
    void *vec[9] = {};
    double *d_part = nullptr;
    size_t part_cap = 0;
    unsigned *d_ticket = nullptr;
    double *d_small = nullptr;  // h1, h2, scal, misc (4 * 256 doubles)
    int64_t launches = 0;
    // the next precision up for the mixed-precision fallback: the FP64 copy of an
    // FP32 context, the FP32 copy (with its own FP64 twin) of a BF16-basis one
    pp_ctx *twin = nullptr;
    int64_t stored = 0;      // matrix entries held on the device (with SELL padding)
    int stall_sweeps = 0;    // test hook: staged CGS2 sweeps left to run without copies
    // per-call device workspace (bases, test buffers) kept for the next call:
    // blocks in use and their sizes, and blocks free for reuse
    std::vector<std::pair<void *, size_t>> ws_live, ws_spare;
    int64_t ldv() const { return (n + 31) / 32 * 32; }
    // device error word of the TMA-staged sweeps (set when a bounded wait expired)
    int *err() const { return (int *)(d_small + 4000); }
};

struct pp_poly {
    pp_ctx *ctx = nullptr;
    std::vector<cd> roots;
    std::vector<ppi::StepCoef> steps;
    int degree = 0, added = 0;
    bool breakdown = false;
    pp_poly *inner = nullptr;  // pi_1 for a double polynomial (tau = 1 - pi_1)
    int64_t mvps = 0, dots = 0, vops = 0;  // work of the GMRES build(s)
    ~pp_poly() { delete inner; }
};


// pp_create with control over the FP64 twin of an FP32 context (the request
// server creates contexts without it to save memory).
pp_status pp_create_internal(pp_ctx **out, int64_t n, const int64_t *rowptr, const int32_t *colind,
                             const double *vals, const pp_opts *opts, int make_twin);

namespace ppi {

struct Timers {
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    cudaEvent_t get();
    ~Timers();
};

// The FP64 context of c's twin chain (c itself when FP64; null without one).
inline pp_ctx *fp64_context(pp_ctx *c) {
    while (c && c->bprec != ppk::F64) c = c->twin;
    return c;
}
// Kernel launches of c and its twins.
inline int64_t chain_launches(const pp_ctx *c) {
    int64_t l = 0;
    for (; c; c = c->twin) l += c->launches;
    return l;
}
pp_status dmalloc(pp_ctx *c, void **p, size_t bytes);
void dfree(pp_ctx *c, void *p);
// Workspace of one call: a spare block of the context that fits (at most a
// quarter larger), else a new allocation; ws_put hands it back for reuse on
// the context's stream (work queued on it is ordered before any reuse).
pp_status ws_get(pp_ctx *c, void **p, size_t bytes);
void ws_put(pp_ctx *c, void *p);
// Free the spare blocks (pp_trim).
void ws_trim(pp_ctx *c);
pp_status check_launch(pp_ctx *c);
pp_status step(pp_ctx *c, const ppk::StepArgs &s);
pp_status op_apply(pp_ctx *c, const pp_poly *p, const void *x, void *y);
pp_status op_tau(pp_ctx *c, const pp_poly *inner, const void *x, void *y);
int64_t op_mvps(const pp_poly *p);
int64_t op_vops(const pp_poly *p);
int64_t vops_of(const std::vector<StepCoef> &s);
pp_status ensure_part(pp_ctx *c, size_t doubles);
pp_status cgs2_step(pp_ctx *c, ppk::Prec pr, void *V, int64_t ldv, int j, void *w, double *hcol);
// the same over vectors of length n (a block system's basis)
pp_status cgs2_step_n(pp_ctx *c, ppk::Prec pr, int64_t n, void *V, int64_t ldv, int j, void *w, double *hcol);
pp_status roots_from_hessenberg(pp_ctx *c, int d, const std::vector<double> &H, int64_t mvps_per_step,
                                int64_t vops_per_step, pp_poly *out);
// Arnoldi steps j0..m-1 on Op with a basis stored in precision bpr (the
// context's vector precision, or BF16).
pp_status arnoldi_extend(pp_ctx *c, const pp_poly *p, const pp_poly *tau_of, ppk::Prec bpr, void *V, int64_t ldv,
                         double *dH, int ldh, int j0, int m, void *W, Timers *tm,
                         std::vector<std::pair<int, int>> *marks);
void accumulate_times(Timers &tm, std::vector<std::pair<int, int>> &marks, double &t_apply, double &t_orth);
pp_status upload_vec(pp_ctx *c, const double *h, double s, void *d);
// True for device (or managed) memory, false for host memory.
bool on_device(const void *p);
// The unit vector x / ||x|| stored into dst in precision pr (F64 or F32 as the
// context's vectors, or BF16); x: n FP64 values in host or device memory
// (the norm is summed on the host, or on the device in a fixed order).
// beta = ||x||; PP_EINVAL when x is zero or not finite.
pp_status load_unit(pp_ctx *c, const double *x, ppk::Prec pr, void *dst, double *beta, const char *what);
pp_status download_vecs(pp_ctx *c, const void *d, int64_t ld, int cols, std::vector<double> &out, ppk::Prec pr);
// PP_ETIMEOUT (and the error word and reduction ticket cleared) when a
// TMA-staged sweep gave up waiting since the last check; synchronises the stream.
pp_status check_sweeps(pp_ctx *c);

}  // namespace ppi
