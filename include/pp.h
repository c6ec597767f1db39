/*
 * pp.h — C-ABI of the GB300 polynomial preconditioned Arnoldi library.
 *
 * Method: Embree, Loe & Morgan, "Polynomial Preconditioned Arnoldi".
 * The library finds a few eigenvalues of a large sparse real matrix A nearest
 * a target by running thick-restarted Arnoldi(m,k) on pi(A), where pi is the
 * GMRES (minimum residual) polynomial of degree d (Section 2 box), applied in
 * factored form pi(A) = prod_i (I - A/theta_i) with the roots theta_i in
 * modified Leja order (Eq. (2.1)).
 *
 * Conventions for every entry point
 *  - Plain C types only.  "_dev" pointers are CUDA device pointers; every other
 *    pointer is host memory.  Matrices are CSR (row pointers int64, column
 *    indices int32, values double), column indices within a row in any order.
 *  - Ownership: the library copies every input it keeps; caller buffers stay
 *    caller-owned and may be freed after the call returns.  Output arrays are
 *    caller-allocated with the sizes stated.  Handles returned through an out
 *    pointer are owned by the caller and released with the matching destroy.
 *  - Errors: a negative pp_status means nothing valid was written to outputs
 *    (the handle stays usable unless the status is PP_ECUDA); a positive status
 *    is a usable result with a warning.  pp_last_error() returns a message for
 *    the most recent failure on the calling thread.
 *  - Threads: a context and its polynomials are used by one host thread at a
 *    time.  All GPU work of a context runs on its stream, in order.
 *  - Vectors on the device (pp_apply) use the context's storage precision:
 *    double for PP_FP64, float for PP_FP32 and PP_FP32_BF16.
 */
#ifndef PP_H
#define PP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pp_ctx pp_ctx;
typedef struct pp_poly pp_poly;

typedef enum {
    PP_OK = 0,
    PP_ENOTCONV = 1,    /* not converged in max_cycles; best pairs and residuals written */
    PP_EBREAKDOWN = 2,  /* GMRES ended early (invariant subspace); degree reduced, poly usable */
    PP_EAGAIN = 3,      /* a served request has not finished yet */
    PP_EINVAL = -1,     /* bad argument */
    PP_ENOMEM = -2,     /* device or host allocation failed */
    PP_ECUDA = -3,      /* CUDA runtime error; the context must be destroyed */
    PP_ETIMEOUT = -4,   /* a bounded device wait gave up */
    PP_ENUMERIC = -5    /* NaN/Inf or a singular small dense problem */
} pp_status;

/* Storage / arithmetic precision of the hot path.
 *  PP_FP64:      FP64 matrix values, vectors, basis and arithmetic.
 *  PP_FP32:      FP32 values, vectors and Arnoldi basis with FP32 accumulation; the
 *                convergence test, the refinement and (when needed) a continuation run
 *                in FP64 on A (mixed precision).
 *  PP_FP32_BF16: as PP_FP32 but the Arnoldi basis is stored in BF16 (widened to FP32
 *                when read; pp_eigs only, not the batched or served engines). */
enum { PP_FP64 = 0, PP_FP32 = 1, PP_FP32_BF16 = 2 };
/* Sparse format on the device: auto (chosen by the tuner), CSR, SELL-C-sigma, DIA
 * (diagonal storage: stencil and banded matrices with at most 64 distinct diagonals,
 * sorted columns and at most 30 % padding; no column indices are stored). */
enum { PP_FMT_AUTO = 0, PP_FMT_CSR = 1, PP_FMT_SELL = 2, PP_FMT_DIA = 3 };
/* Which eigenvalues: smallest magnitude (Section 2) or smallest real part
 * (run on A - sigma I with sigma the leftmost Gershgorin point, Section 2 footnote 1). */
enum { PP_TARGET_SM = 0, PP_TARGET_SR = 1 };
/* Restart of pp_eigs (Section 4; Example 2).  Harmonic: the values ordered,
 * tested and kept are the harmonic Ritz values of the operator with respect to
 * its target point (1 for pi(A), 0 for plain Arnoldi), i.e. theta with
 * (Op - t) y - (theta - t) y orthogonal to (Op - t) V_m; the restart keeps
 * V_{m+1} P, P = orth([Q_k; 0], c), c = [-h f; 1], f = (H_m - t I)^{-T} e_m,
 * so the residual direction shared by all harmonic pairs stays in the basis. */
enum { PP_RESTART_RITZ = 0, PP_RESTART_HARMONIC = 1 };

typedef struct {
    int precision;      /* PP_FP64 (default), PP_FP32, PP_FP32_BF16 */
    int format;         /* PP_FMT_AUTO (default) */
    int target;         /* PP_TARGET_SR (default) or PP_TARGET_SM */
    double sigma;       /* shift; NaN (default) = automatic from the target */
    int add_roots;      /* 1 (default): Section 7 box, extra copies of roots with large pof */
    int max_cycles;     /* Arnoldi cycles before PP_ENOTCONV; default 2000 */
    int refine_steps;   /* FP64 refinement steps for the mixed-precision path; default 4 */
    int sell_c;         /* SELL chunk height: 16 or 32; 0 (default) = the tuner picks C and the
                           block size of the product kernels by timing them on this matrix */
    int sell_sigma;     /* SELL sorting window: must be 0 or 1 (rows keep their order) */
    int sell_index;     /* SELL column indices: 0 (default) = 16-bit offsets col - row when every
                           |col - row| < 2^15, else 32-bit; 32 = always 32-bit */
    int sell_loop;      /* SELL row loop: 0 (default) = the tuner picks; 1 = unrolled by four;
                           2 = loads of up to eight entries issued together; 3 = slice data staged
                           in shared memory by bulk copies (SELL-32 only); 4 = two rows per thread */
    void *stream;       /* cudaStream_t to run on; NULL = a stream owned by the context */
    int restart;        /* pp_eigs restart: PP_RESTART_RITZ (default) keeps Ritz vectors;
                           PP_RESTART_HARMONIC keeps harmonic Ritz vectors (the harmonic
                           Arnoldi variant of Example 2, for interior targets) */
    int balance;        /* 0 (default): A as given.  1: balancing (not in the paper; an opt-in
                           problem transformation): run the method on S = D^-1 A D, the diagonal
                           similarity that makes A symmetric (d_j/d_i = sqrt(a_ji/a_ij) on every
                           off-diagonal pair; needs a_ij, a_ji nonzero together with one sign and
                           consistent cycles, as for central-difference convection-diffusion
                           with cell Peclet number < 1; else pp_create returns PP_EINVAL; 2: the
                           same where such a D exists, else A as given).  S has
                           the eigenvalues of A with condition numbers 1.  Eigenvectors are
                           returned for A (x = D y, unit norm) and the convergence test stays on
                           A itself; start vectors, pp_apply and pp_orthogonalize act in the
                           coordinates of S, and sigma is S's Gershgorin shift. */
    int dia_loop;       /* DIA row loop: 0 (default) = the tuner picks; 1 = one row per thread;
                           2 = four or 3 = two consecutive rows per thread with 16- or 8-byte
                           loads (FP32 contexts; taken only when the vectors are so aligned,
                           else one row per thread) */
} pp_opts;

/* Counters of Section 4 (mvps, dot products, vector operations) plus timings. */
typedef struct {
    int64_t cycles;       /* Arnoldi cycles run */
    int64_t mvps;         /* products with A (polynomial build, applies, residual checks) */
    int64_t dots;         /* length-n inner products */
    int64_t vops;         /* length-n vector operations (dots, axpys, scalings) */
    int64_t kernel_launches; /* library kernels launched by the call */
    int32_t converged;    /* 1 when every wanted pair met the tolerance */
    int32_t nconv;        /* number of wanted slots that met the tolerance */
    double t_total;       /* seconds, wall clock of the call */
    double t_apply;       /* seconds spent in pi(A) applies (device, event-timed) */
    double t_orth;        /* seconds spent in CGS2 (device, event-timed) */
    double t_restart;     /* seconds in restart + convergence test, host and device */
    double max_resid;     /* largest ||A x - lambda x|| / ||A||_1 among returned slots */
    int64_t fp64_cycles;  /* cycles run in FP64 (all of them for PP_FP64; for PP_FP32 the
                             cycles of the FP64 continuation, 0 when FP32 + refinement sufficed) */
} pp_stats;

/* Fill *o with the defaults listed above. */
void pp_opts_default(pp_opts *o);

/* Message for the last failure on this thread ("" if none).  Static storage. */
const char *pp_last_error(void);

/*
 * pp_create — upload the sparse matrix A (n x n, CSR, host arrays) and prepare
 * the device formats (Section 2: the method needs only products with A).
 * rowptr: n+1 int64; colind: nnz int32 in [0, n); vals: nnz doubles.
 * opts may be NULL (defaults).  On success *out receives a context.
 * In auto mode the tuner's choice (format, chunk, row loop, block size) is kept
 * for the life of the process under a signature of the matrix (n, nnz, element
 * size, index width, sampled row pointers and columns); a later context for a
 * matrix with the same signature reuses it without timing.
 * Errors: PP_EINVAL (n <= 0, bad indices), PP_ENOMEM, PP_ECUDA.
 */
pp_status pp_create(pp_ctx **out, int64_t n, const int64_t *rowptr, const int32_t *colind,
                    const double *vals, const pp_opts *opts);
void pp_destroy(pp_ctx *ctx);

/*
 * pp_trim — free the device workspace a context keeps between calls.
 * pp_build_poly* and pp_eigs hand their per-call buffers (Krylov bases, the
 * FP64 test and refinement buffers) back to the context, which reuses them for
 * later calls of the same sizes instead of allocating again; the memory stays
 * held until pp_trim or pp_destroy.  Synchronises the context's stream.
 * Errors: PP_EINVAL (null context).
 */
pp_status pp_trim(pp_ctx *ctx);

/*
 * pp_debug_stall_sweeps — test support for the failure path of the staged
 * CGS2 sweeps: the next `count` CGS2 steps on this context issue no bulk
 * copies, so every wait for a staged tile runs out its bounded limit; the
 * next host synchronisation of the call returns PP_ETIMEOUT and the context
 * stays usable.  Applies to FP32 contexts whose sweeps are staged (a step
 * that takes the plain sweeps is unaffected).  Not for production use.
 */
pp_status pp_debug_stall_sweeps(pp_ctx *ctx, int count);

/* Number of library kernels launched on this context since pp_create. */
int64_t pp_launch_count(const pp_ctx *ctx);

/* Whether the context runs on the balanced matrix S = D^-1 A D (pp_opts.balance)
 * and the range of its scaling, log(max d / min d).  Outputs may be NULL. */
pp_status pp_balance_info(const pp_ctx *ctx, int *balanced, double *log_range);

/* ||A||_1 (maximum absolute column sum) and the shift sigma used for the target. */
pp_status pp_matrix_info(const pp_ctx *ctx, double *norm1, double *sigma);

/*
 * pp_csr_info — the host analysis pp_create runs on a CSR matrix, without a
 * device: ||A||_1 (maximum absolute column sum; the residual bound of Section
 * 4 is rtol ||A||_1) and the shift of the smallest-real-part target (Section 2,
 * footnote 1: sigma = min(0, min_i (a_ii - sum_{j != i} |a_ij|)), 0 when that
 * bound is above -1e-12 ||A||_1).  Arguments as pp_create (host arrays, read
 * only); either output may be NULL.  PP_EINVAL for the inputs pp_create
 * refuses (row pointers not starting at 0 or not monotone, a column outside
 * [0, n), a value that is not finite, nnz or n >= 2^31).
 */
pp_status pp_csr_info(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals, double *norm1,
                      double *sigma_sr);

/*
 * pp_csr_balance — the balancing pp_create applies with pp_opts.balance, on
 * the host and without a device (not in the paper: an opt-in problem
 * transformation).  d (host, n doubles, caller-owned) receives the diagonal
 * D of the similarity S = D^-1 A D that makes A symmetric (d_j / d_i =
 * sqrt(a_ji / a_ij) on every off-diagonal pair, largest entry 1);
 * *log_range (may be NULL) receives -min_i log d_i.  PP_EINVAL with a reason
 * for the inputs pp_create refuses and when no such D exists (a pair of
 * entries not nonzero together or of opposite signs, ratios that do not
 * multiply to 1 around a cycle, a range beyond e^600); d is then unspecified.
 */
pp_status pp_csr_balance(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals, double *d,
                         double *log_range);

/*
 * pp_format_info — the device format of A chosen at pp_create: fmt
 * (PP_FMT_CSR, PP_FMT_SELL or PP_FMT_DIA), the SELL chunk height (0 otherwise),
 * the column index width in bits (16 or 32; 0 for DIA), the block size of the product kernels, the
 * row loop (SELL: 0 unrolled by four; 1 the loads of up to eight entries
 * issued together; 2 slice data staged by bulk copies; 3 two rows per
 * thread.  DIA: 0 one row per thread; 1 four, 2 two rows per thread), and the
 * stored entries including padding.  Any output pointer may be NULL.
 */
pp_status pp_format_info(const pp_ctx *ctx, int *fmt, int *chunk, int *index_bits, int *threads, int *row_loop,
                         int64_t *stored);

/*
 * pp_build_poly — GMRES polynomial of degree d (Section 2 box, step 1):
 * one GMRES(d) cycle on A - sigma I from b (n doubles, host or device memory:
 * a device vector is normalised on the device, with no copy), harmonic Ritz
 * values as roots (step 1(b)), modified Leja order (step 1(c)), then extra
 * copies of roots with large pof when opts.add_roots (Section 7 box).
 * The Arnoldi process runs on the GPU (SpMV + CGS2); the d x d dense steps run
 * on the host in FP64.  Returns PP_EBREAKDOWN (poly usable, lower degree) when
 * GMRES found an invariant subspace before step d.
 */
pp_status pp_build_poly(pp_ctx *ctx, int d, const double *b, pp_poly **out);

/*
 * pp_build_poly_two — the polynomial determined by two starting vectors
 * (Section 5 box): one GMRES(d) cycle on blockdiag(A, A) (A - sigma I with a
 * shift) from [b1; b2], each half scaled to norm 1/sqrt(2), then roots as in
 * pp_build_poly.  b1, b2: n doubles each, host or device.  Guards against a skewed
 * start vector.  Requires 1 <= d <= 127.  Returns PP_OK or PP_EBREAKDOWN.
 */
pp_status pp_build_poly_two(pp_ctx *ctx, int d, const double *b1, const double *b2, pp_poly **out);

/*
 * pp_build_poly_damped — the heuristic for damping b and adjusting d (Section
 * 6.3 box): build pi from b (as pp_build_poly), run one Arnoldi(m, k) cycle on
 * pi(A) from b, and check the Ideal Order Condition on the Rayleigh quotients
 * for A of the k Ritz vectors nearest 1 (|mu_1| <= ... <= |mu_nev| < the other
 * k - nev).  If it fails, rebuild from A b (damping, Section 6.1); if that
 * fails too, halve d until it holds or d = 1.  With a shift (smallest real
 * part targets) A stands for A - sigma I throughout.  b: n doubles, host or device.
 * Outputs: the polynomial, the degree finally used (before added roots),
 * damped (1 when built from A b) and ideal (1 when the condition holds for
 * it; 0 only when d reached 1 without it).  Requires 1 <= nev < k <= m <= 127,
 * m < n.  Returns PP_OK, or PP_EBREAKDOWN when the final build broke down.
 */
pp_status pp_build_poly_damped(pp_ctx *ctx, int d, const double *b, int m, int k, int nev, pp_poly **out,
                               int *degree, int *damped, int *ideal);

/*
 * pp_build_poly2 — double polynomial (Section 8): pi_1 of degree d1 from b,
 * tau(z) = 1 - pi_1(z) applied as the running sum of pi_1's factors, pi_2 of
 * degree d2 = GMRES polynomial of tau(A) from the same b.  Arnoldi then runs
 * on pi_2(tau(A)), of composite degree d1*d2 (plus added roots).
 */
pp_status pp_build_poly2(pp_ctx *ctx, int d1, int d2, const double *b, pp_poly **out);

/*
 * pp_poly_from_roots — polynomial with the given roots, applied in the given
 * order (no reordering, no added roots).  Conjugate pairs must be adjacent,
 * the member with im > 0 first and exactly conjugate.  count >= 1.
 */
pp_status pp_poly_from_roots(pp_ctx *ctx, int count, const double *re, const double *im,
                             pp_poly **out);

/*
 * pp_poly2_from_roots — double polynomial (Section 8) with given roots:
 * y = pi_2(tau(A)) x with tau(z) = 1 - pi_1(z), pi_1 having roots re1/im1
 * (count1) and pi_2 roots re2/im2 (count2), each applied in the given order
 * (no reordering, no added roots); the same rules as pp_poly_from_roots for
 * each list.  Errors: PP_EINVAL.
 */
pp_status pp_poly2_from_roots(pp_ctx *ctx, int count1, const double *re1, const double *im1, int count2,
                              const double *re2, const double *im2, pp_poly **out);

/*
 * pp_poly_roots — roots in application order (including added roots).
 * re/im: capacity cap each; *count receives the number of roots (if > cap only
 * cap are written).  For a double polynomial these are pi_2's roots;
 * pp_poly_inner_roots gives pi_1's.
 */
pp_status pp_poly_roots(const pp_poly *p, double *re, double *im, int cap, int *count);
pp_status pp_poly_inner_roots(const pp_poly *p, double *re, double *im, int cap, int *count);
/* Degree reached by GMRES (before added roots) and the number of added roots. */
pp_status pp_poly_info(const pp_poly *p, int *degree, int *added);
/* Work of the GMRES build(s) that made p, counted as in Section 4 (both
 * builds for a double polynomial; zero for pp_poly_from_roots). */
pp_status pp_poly_counts(const pp_poly *p, int64_t *mvps, int64_t *dots, int64_t *vops);
void pp_poly_destroy(pp_poly *p);

/*
 * pp_apply — y = pi(A - sigma I) x (Eq. (2.1)); for a double polynomial
 * y = pi_2(tau(A - sigma I)) x (Section 8).  x_dev, y_dev: n elements of the
 * context's storage type on the device; they may be the same buffer.
 * Real roots take one fused SpMV pass each; a conjugate pair takes two passes
 * in real arithmetic.  Asynchronous on the context's stream.
 */
pp_status pp_apply(const pp_poly *p, const void *x_dev, void *y_dev);

/*
 * pp_apply_host — as pp_apply with host x and y (n doubles each): copies in,
 * applies, copies out, synchronises.
 */
pp_status pp_apply_host(const pp_poly *p, const double *x, double *y);

/*
 * pp_eigs — thick-restarted Arnoldi(m, k) on pi(A) (Section 2 box step 2;
 * Section 4): nev eigenvalues of A nearest the target, m the largest subspace
 * dimension, k Ritz vectors kept (k - 1 when a conjugate pair would split),
 * one reorthogonalisation pass per step, convergence tested at the end of each
 * cycle on A itself: ||A y_j - mu_j y_j|| <= rtol * ||A||_1 with mu_j the
 * Rayleigh quotient of the unit Ritz vector y_j.
 * p == NULL runs plain Arnoldi(m, k) on A - sigma I.
 * v0: start vector (n doubles, host or device memory; a device vector is
 * normalised on the device), NULL = e_1 + ... (deterministic ones).
 * Outputs (capacity nev + 1 slots; a conjugate pair takes two slots and the
 * wanted set grows by one when nev would split a pair):
 *   lam_re, lam_im: eigenvalue estimates, sorted by the target;
 *   X: n x (nev+1) column-major (NULL to skip): a real eigenvector, or for a
 *      pair (lam, conj(lam)) the columns (Re x, Im x) of the unit vector x;
 *   resid: ||A x - lam x|| / ||A||_1 per slot;  *nout: slots written.
 * PP_FP32 contexts (mixed precision): the cycles run in FP32 storage; the
 * convergence test is always FP64 on A; within 50 rtol or at the FP32 floor
 * the Ritz vectors are refined in FP64 (Rayleigh-Ritz of A on span{pi(A) Y},
 * pi applied in FP64 by the context's FP64 copy; from the second round the
 * cycle's next Ritz vectors join Y); if that does not reach rtol the solve
 * continues in FP64 from the refined vectors.  PP_FP32_BF16 contexts do the
 * same with a BF16 basis and continue with an FP32 basis (which refines and
 * continues in FP64 in turn).
 * Requires 1 <= nev < k < m, m < n.  Returns PP_ENOTCONV with the best pairs
 * when max_cycles is reached.
 */
pp_status pp_eigs(pp_ctx *ctx, const pp_poly *p, int nev, int m, int k, double rtol,
                  const double *v0, double *lam_re, double *lam_im, double *X, double *resid,
                  int *nout, pp_stats *stats);

/*
 * pp_orthogonalize — one Arnoldi orthogonalisation step (Section 4: classical
 * Gram-Schmidt followed by one reorthogonalisation pass, CGS2): with the j
 * orthonormal columns of V (device, column major, leading dimension ldv >= n,
 * context storage type) and w (device, n), computes h1 = V^T w, w1 = w - V h1,
 * h2 = V^T w1, w2 = w1 - V h2, and writes v = w2 / ||w2|| to v_dev (device, n;
 * may not alias V or w).  w is overwritten by w1.  h_host (host, j + 1
 * doubles) receives h1 + h2 followed by ||w2||.  Synchronises the stream.
 * Requires 1 <= j <= 128.  Arithmetic: FP64 throughout for FP64 contexts; for
 * FP32 contexts, h1 and both updates in FP32, h2 as a compensated FP32 dot
 * product (about twice FP32 precision), norms in FP64.
 */
pp_status pp_orthogonalize(pp_ctx *ctx, const void *V_dev, int64_t ldv, int j, void *w_dev, void *v_dev,
                           double *h_host);

/*
 * pp_orthogonalize_noalloc — the CGS2 step of pp_orthogonalize for callers
 * that cannot allocate device memory.  The paper has no counterpart: this is
 * a deployment variant of the same computation.
 *
 * Who needs it: a caller whose device memory is owned by someone else (a
 * host framework that reserves the whole GPU for its own caching allocator,
 * so a cudaMalloc here would fail or fragment it), a latency-critical loop
 * that cannot pay for cudaMalloc/cudaFree (they may synchronise the device),
 * or a plugin that is not allowed to own device allocations.  Such a caller
 * passes its inputs and outputs and creates no pp_ctx; this call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Computes, in FP64 and on the given stream (NULL = legacy default stream):
 * with the j orthonormal columns of V_dev (n x j, column major, leading
 * dimension ldv >= n) and w_dev (n), h1 = V^T w, w1 = w - V h1 (written back
 * to w_dev), h2 = V^T w1, w2 = w1 - V h2; v_dev (n, not aliasing V or w)
 * receives w2 / ||w2||; h_dev (device, j + 1 doubles) receives h1 + h2 and
 * then ||w2||.  Asynchronous: nothing is copied to the host.
 *
 * Scratch: a file-scope __device__ array of about 656 KB ((608 + 19) x 130 +
 * 552 doubles: partial sums for at most 608 blocks x 130 values and the sums
 * of their groups of 32, the two coefficient vectors, the norm and the
 * reduction ticket), held by every GPU that loads the library until the
 * process exits.  Limits: 1 <= j <= 128 (beyond that PP_EINVAL with a
 * message); n < 2^31.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current and keeps it
 * for the life of the process; make that first call before any stream
 * capture, and do not reset the device (cudaDeviceReset) after it: the kept
 * address would then be stale.  Every call uses the same array and
 * leaves the last call's contents in it (the ticket is cleared at the start
 * of each call); calls that overlap on the GPU, e.g. on two streams, race on
 * it, so issue them on one stream or otherwise serialise them.
 */
pp_status pp_orthogonalize_noalloc(int64_t n, const double *V_dev, int64_t ldv, int j, double *w_dev,
                                   double *v_dev, double *h_dev, void *stream);

/* ----- Batching: many independent instances advanced together ----- */
typedef struct pp_batch pp_batch;

/*
 * pp_batch_create — upload `count` independent sparse matrices (host CSR each,
 * as pp_create) for solving together.  opts applies to all (PP_FP32 for the
 * mixed-precision path); the device format is SELL-32.  Errors: PP_EINVAL for
 * PP_FP32_BF16 or a harmonic restart (the batched engine keeps Ritz vectors).
 */
pp_status pp_batch_create(pp_batch **out, int count, const int64_t *n, const int64_t *const *rowptr,
                          const int32_t *const *colind, const double *const *vals, const pp_opts *opts);

/*
 * pp_batch_solve — for every instance i: the GMRES polynomial of degree d[i]
 * from bvec[i] (Section 2 box), then thick-restarted Arnoldi(m, k) on
 * pi_i(A_i) from v0[i] (NULL or v0[i] NULL: ones) for nev eigenvalues
 * (Section 4), all instances in lockstep: each Arnoldi step is one CUDA graph
 * of one launch per polynomial pass for all active instances plus batched
 * CGS2 sweeps.  Instances stop individually when converged.  Outputs per
 * instance as in pp_eigs: lam_re[i], lam_im[i], resid[i] (capacity nev + 1),
 * X[i] (n[i] x (nev + 1), column major; X or X[i] may be NULL), nout[i],
 * stats[i] (may be NULL).  Returns PP_ENOTCONV if any instance did not
 * converge (its best pairs are written), a negative status on failure.
 */
pp_status pp_batch_solve(pp_batch *b, const int *d, const double *const *bvec, const double *const *v0, int nev,
                         int m, int k, double rtol, double *const *lam_re, double *const *lam_im,
                         double *const *X, double *const *resid, int *nout, pp_stats *stats);
/* Kernels launched by pp_batch_solve calls on this batch so far. */
int64_t pp_batch_launch_count(const pp_batch *b);
void pp_batch_destroy(pp_batch *b);

/* ----- Serving: continuous batching of a request stream ----- */
typedef struct pp_server pp_server;

/*
 * pp_server_create — a request server on the current GPU.  Requests wait in a
 * FIFO queue and are admitted, oldest first, while their estimated device
 * memory fits in mem_budget bytes (0 = 80 % of the free memory) and fewer
 * than max_active (0 = 256) are on the GPU.  Admitted requests share the
 * batched engine of pp_batch_solve: each Arnoldi cycle advances all of them,
 * a request that converges is retired at once (its device memory is freed)
 * and the queue head is admitted in its place, so requests that arrive while
 * others run join them on the device.  opts: precision (PP_FP32 = FP32 apply,
 * FP64 test and refinement), target, max_cycles, refine_steps, stream
 * (PP_FP32_BF16 and a harmonic restart: PP_EINVAL).
 * keep_vectors: return eigenvectors in pp_server_result (host memory n x
 * (nev + 1) per request).
 */
pp_status pp_server_create(pp_server **out, const pp_opts *opts, int64_t mem_budget, int max_active,
                           int keep_vectors);
/*
 * pp_server_submit — queue one eigen-solve (inputs are copied; thread safe):
 * matrix (host CSR, as pp_create), polynomial degree d from b (host, n), and
 * Arnoldi(m, k) for nev eigenvalues from v0 (host or NULL) to rtol.  *id
 * receives the request id.  PP_ENOMEM when the request alone exceeds the
 * memory budget.
 */
pp_status pp_server_submit(pp_server *s, int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals,
                           int d, int nev, int m, int k, double rtol, const double *b, const double *v0, int64_t *id);
/*
 * pp_server_step — admit what fits, run one Arnoldi cycle of every admitted
 * request, retire the finished ones.  *active / *queued (may be NULL) receive
 * the requests on the GPU and waiting.  Call it in a loop (one host thread).
 */
pp_status pp_server_step(pp_server *s, int *active, int *queued);
/*
 * pp_server_result — PP_EAGAIN while request id is queued or running;
 * otherwise its final status with the outputs of pp_eigs (capacity nev + 1;
 * X n x (nev + 1) or NULL) and *latency (seconds from submit to result, may
 * be NULL).  Each result can be fetched once (thread safe).
 */
pp_status pp_server_result(pp_server *s, int64_t id, double *lam_re, double *lam_im, double *X, double *resid,
                           int *nout, pp_stats *stats, double *latency);
/* Kernels launched by the server's batched engine so far (batched passes and sweeps). */
int64_t pp_server_launch_count(const pp_server *s);
/* Device bytes the server reserves for one request of this shape (the
 * admission estimate: matrix with padding headroom, FP64 residual operator,
 * scratch, two basis slabs, test buffers and, for PP_FP32, the FP64 copy used
 * when FP32 cannot reach rtol). */
int64_t pp_server_request_bytes(const pp_server *s, int64_t n, int64_t nnz, int m, int nev);
void pp_server_destroy(pp_server *s);

/* ----- Measurement support (not part of the method) ----- */

/*
 * pp_measure_fp64_rate — FP64 (non-tensor) FMA throughput of the current GPU
 * in flop/s: a kernel of eight independent FMA chains per thread on eight
 * 256-thread blocks per SM, timed with CUDA events on `stream` (NULL = legacy
 * default stream), best of three launches after one warm-up (about 50 ms in
 * all).  The FP64 polynomial passes and CGS2 sweeps are bound by FP64
 * arithmetic on GB300, so their roofline divides by this measured rate.  The
 * paper has no counterpart.  Synchronises the stream.  Errors: PP_EINVAL,
 * PP_ECUDA.
 */
pp_status pp_measure_fp64_rate(void *stream, double *flops_per_s);

/* ----- Host FP64 dense steps (no GPU needed; used by the calls above) ----- */

/*
 * pp_dense_eig — eigenvalues and right eigenvectors of a real n x n matrix
 * (column-major, leading dimension lda), by Householder reduction to
 * Hessenberg form and Francis double-shift QR.  wr/wi: n each; a conjugate
 * pair is adjacent with wi > 0 first and exactly conjugate.  V (n x n, ldv,
 * may be NULL): column j holds the real eigenvector, or for a pair (j, j+1)
 * the real and imaginary parts of the unit eigenvector of wr[j] + i wi[j].
 * Returns PP_ENUMERIC when QR does not converge.
 */
pp_status pp_dense_eig(int n, const double *A, int lda, double *wr, double *wi, double *V, int ldv);

/*
 * pp_harmonic_ritz — roots of the GMRES polynomial from H_{d+1,d}
 * ((d+1) x d, column-major, ldh >= d+1): eigenvalues of H_d + h_{d+1,d}^2 f e_d^T
 * with H_d^T f = e_d (Section 2 box, step 1(b)).  re/im: d each, pairs adjacent.
 */
pp_status pp_harmonic_ritz(int d, const double *H, int ldh, double *re, double *im);

/*
 * pp_leja_order — modified Leja order (Section 2 box, step 1(c); Bai, Hu &
 * Reichel alg. 3.1) with logarithmic products: first the root of largest
 * modulus, then repeatedly the root maximising the product of distances to the
 * roots chosen so far; a complex choice (im > 0 member) is followed by its
 * conjugate.  Ties: first in the order (-re, -im, input position).
 */
pp_status pp_leja_order(int count, const double *re, const double *im, double *out_re,
                        double *out_im);

/*
 * pp_add_stability_roots — Section 7 box: for each root (a conjugate pair is
 * one unit, Leja order) with pof = prod_{i != j} |1 - theta_j/theta_i|, add
 * ceil((log10 pof - 4)/14) copies (none when pof <= 1e4): the first at the end
 * of the list, the others at unit positions p + floor(t (L - p)/c), t = 1..c-1,
 * between the root's position p and the end (L units, c copies).
 * out_re/out_im: capacity cap; *out_count receives the new length.
 */
pp_status pp_add_stability_roots(int count, const double *re, const double *im, int cap,
                                 double *out_re, double *out_im, int *out_count);

/*
 * pp_restart_basis — the host step of one thick restart of pp_eigs (Section 4;
 * Example 2's harmonic variant when harmonic != 0), from the Arnoldi relation
 * Op V_m = V_{m+1} H with H ((m+1) x m, column-major, ldh >= m+1): the values
 * (Ritz values of H_m, or harmonic Ritz values with respect to target) ordered
 * by distance to target, the k nearest kept (k - 1 when a conjugate pair would
 * split), and
 *   Ritz:     Q = (m x kk, ld m) orthonormal basis of their vectors' Re/Im
 *             parts; the new basis is [V_m Q, v_{m+1}];
 *   harmonic: Q = P ((m+1) x (kk+1), ld m+1); the new basis is V_{m+1} P.
 * Hn (ldh x m) receives the new leading (kk+1) x kk block, zero elsewhere.
 * Host arrays; Q needs (m+1) * (m+1) doubles.  Outputs *kk and the values in
 * order (re, im: m each, may be NULL).  Requires 1 <= k < m <= 127.
 * Errors: PP_EINVAL, PP_ENUMERIC (QR failed, H_m - target I singular).
 */
pp_status pp_restart_basis(int m, const double *H, int ldh, int k, double target, int harmonic, double *Q,
                           double *Hn, int *kk, double *re, double *im);

#ifdef __cplusplus
}
#endif

#endif /* PP_H */
