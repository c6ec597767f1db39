// Internal declarations shared by the library's translation units.
#pragma once

#include "pp.h"

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

// Record a failure message for pp_last_error() and return the status.
pp_status pp_fail(pp_status s, const char *fmt, ...);

namespace ppd {
using cd = std::complex<double>;
bool dense_eig(int n, const double *A, int lda, double *wr, double *wi, double *V, int ldv);
bool lu_solve(int n, std::vector<double> M, double *b);
bool harmonic_ritz(int d, const double *H, int ldh, double *re, double *im);
void thin_qr(int m, int k, const double *B, double *Q);
bool leja_order(const std::vector<cd> &roots, std::vector<cd> &out);
double pof_log10(const std::vector<cd> &roots, size_t j);
int extra_copies(double lp);
bool add_stability_roots(const std::vector<cd> &ordered, std::vector<cd> &out, int &added);
std::vector<int> ritz_order(const std::vector<cd> &nu, double target);
// log d of the diagonal similarity D^-1 A D that makes A symmetric (largest
// entry 0); false with a reason when none exists or its range exceeds
// e^max_log_range (balance.cpp).
bool symmetrizing_scale(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals,
                        std::vector<double> &logd, std::string &why, double max_log_range = 600.0);
// Host analysis of a CSR matrix (csr_scan.cpp, parallel over row ranges).
struct CsrScan {
    double norm1 = 0;         // largest column sum of |a_ij|
    double gl = 0;            // min_i (a_ii - sum_{j != i} |a_ij|)
    bool fits16 = true;       // every |j - i| <= 32767
};
// false with a reason for non-monotone row pointers or an entry with a column
// outside [0, n) or a value that is not finite.
bool scan_csr(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals, CsrScan &out,
              std::string &why);
// The distinct diagonals col - row in increasing order; false when the columns
// of some row do not increase strictly or there are more than max_diags.
bool dia_offsets(int64_t n, const int64_t *rowptr, const int32_t *colind, int max_diags, std::vector<int> &off);
}  // namespace ppd

#ifdef __CUDACC__
#include <cuda_runtime.h>
#else
typedef struct CUstream_st *cudaStream_t;
#endif

namespace ppk {

// Storage precisions of device vectors / matrix values (BF16: basis only).
enum Prec { F64 = 0, F32 = 1, BF16 = 2 };

// SELL-C matrix (sigma = 1: rows keep their order) with chunk height
// C = 1 << cshift (16 or 32): slice s holds rows [C s, C s + C); its entries
// occupy [slice_ptr[s], slice_ptr[s+1]) column major within the slice (entry
// k of lane l at slice_ptr[s] + C k + l).  Column indices are 32-bit (col),
// or 16-bit offsets col - row (off) when every |col - row| < 2^15; padding
// repeats the row's last column (its own row when empty) with value 0.
struct SellView {
    int n;
    int nslices;
    int cshift;
    const int *slice_ptr;
    const int *col;
    const short *off;
    const void *val;
};

struct CsrView {
    int n;
    const int *rowptr;
    const int *col;
    const void *val;
};

// Diagonal storage (for stencil and banded matrices): ndiag offsets off[d]
// (increasing) and the values A(row, row + off[d]) (0 where the matrix has no
// entry or row + off[d] lies outside [0, n)) in blocks of 32 rows: the entry
// of diagonal d in row r is at val[(r / 32) * (ndiag * 32) + d * 32 + r % 32],
// so a warp's values for all diagonals are one contiguous run.  ld (n rounded
// up to 32) rows are allocated.  No column indices.
struct DiaView {
    int n;
    int ndiag;
    int64_t ld;
    const int *off;
    const void *val;
};
constexpr int kDiaMax = 64;  // most diagonals the DIA kernels take

// One fused pass of the factored polynomial (Eq. (2.1)):
//   u = (A - sigma I) x
//   plain:  y = u
//   else:   delta = a1 x + a2 u;  y = base - delta (base = aux or x);
//           r = (r_init ? 0 : r) + delta (the running sum of Section 2 footnote 2)
//   outer (double polynomial, Section 8): oy = obase - (b1 ox + b2 r)
struct StepArgs {
    const void *x = nullptr;
    const void *aux = nullptr;
    void *y = nullptr;
    void *r = nullptr;
    int plain = 0;
    int r_init = 0;
    int r_write = 1;
    double a1 = 0, a2 = 0, sigma = 0;
    const void *obase = nullptr;
    const void *ox = nullptr;
    void *oy = nullptr;
    double b1 = 0, b2 = 0;
    // FP32 copies of the coefficients (set by launch_step): FP32 kernels read them
    // instead of converting the doubles per thread (an FP64 instruction each)
    float fa1 = 0, fa2 = 0, fb1 = 0, fb2 = 0, fsigma = 0;
    int has_sigma = 0;
};

struct Matrix {
    int n = 0;
    int fmt = 2;  // 1 CSR, 2 SELL, 3 DIA
    int threads = 256;  // block size of the SELL pass kernels (64..512, chosen by the tuner)
    int wide = 0;       // SELL row loop: 0 unrolled by four, 1 chunks of eight loads, 2 two rows per thread (tuner);
                        // DIA (FP32): 1 four, 2 two consecutive rows per thread with vector loads (tuner)
    int tma = 0;        // SELL-32 slice data staged by bulk copies (tuner); needs tile_cap and err
    int tile_cap = 0;   // most stored entries in threads/32 consecutive slices
    int *err = nullptr; // the context's error word (bounded waits of the staged kernels)
    Prec prec = F64;
    SellView sell{};
    CsrView csr{};
    DiaView dia{};
};

void launch_step(const Matrix &A, const StepArgs &s, cudaStream_t st);

// CGS2 passes over the basis V (column major, leading dimension ldv, j columns).
//  mode 0: out[0..j) = V^T w
//  mode 1: wout = w - V h;  out[0..j) = V^T wout;  out[j] = ||wout||^2
//  mode 2: wout = w - V h;  out[0] = ||wout||^2; then H column: hcol[c] = h1[c] + h[c]
//          (c < j), hcol[j] = ||wout||, scal[0] = 1/||wout||
struct CgsArgs {
    int mode = 0;
    int n = 0;
    const void *V = nullptr;
    int64_t ldv = 0;
    int j = 0;
    const void *w = nullptr;
    void *wout = nullptr;
    const double *h = nullptr;
    const double *h1 = nullptr;
    double *hcol = nullptr;
    double *scal = nullptr;
    double *out = nullptr;
    double *part = nullptr;
    unsigned *ticket = nullptr;
    int *err = nullptr;  // set to 1 by a TMA-staged sweep whose bounded wait expired (null: plain sweeps only)
    int stall = 0;       // test hook: a staged sweep issues no copies, so its waits expire
};
int cgs_grid(int n);
// Grid reductions of the CGS2 sweeps: block partial sums, then the last block
// of each group of 32 consecutive blocks sums its group, then the last group
// sums the group sums.  Tickets: word 0 counts groups, word 1 + g blocks of
// group g (all zero between launches).  Scratch for a grid of `grid` blocks
// and at most 130 outputs: the block partials followed by the group sums.
constexpr int kTicketWords = 64;
inline size_t cgs_part_doubles(int grid) { return ((size_t)grid + (size_t)(grid + 31) / 32) * 130; }
void launch_cgs(Prec p, const CgsArgs &a, cudaStream_t st);
// as launch_cgs with at most grid_cap blocks (the partial sums need grid_cap * (j+1) doubles)
void launch_cgs_grid(Prec p, const CgsArgs &a, int grid_cap, cudaStream_t st);
void launch_scale(Prec p, int n, void *x, const double *scal, cudaStream_t st);
// out[0] = ||x||^2 (FP64 x on the device; part holds one double per block, at
// most 4 blocks per SM; ticket is zero before and after).
void launch_norm2(int n, const double *x, double *part, unsigned *ticket, double *out, cudaStream_t st);
// Y[:, c] = X[:, c] * d (divide: / d) elementwise, c < cols (FP64; X may be Y).
void launch_scale_rows(int n, int cols, const double *X, int64_t ldx, double *Y, int64_t ldy, const double *d,
                       bool divide, cudaStream_t st);
// dst = src * sgn / sqrt(nrm2[0] + nrm2[1]) (FP64 device vectors).
void launch_slot_scale(int n, const double *src, const double *nrm2, double sgn, double *dst, cudaStream_t st);
// dst = x / sqrt(nrm2[0]) stored in precision p.
void launch_unit_into(Prec p, int n, const double *x, const double *nrm2, void *dst, cudaStream_t st);
// out (BF16, n) = w * scal (w FP32): the new column of a BF16 basis
void launch_scale_bf16(int n, const float *w, const double *scal, void *out, cudaStream_t st);

// Batched Arnoldi steps (many instances advance together, one launch per pass).
// Per-instance CGS2 state: the basis V (ldv), the operator output W, the
// Hessenberg matrix H (ldh), reduction scratch, and the instance's block range
// [blk0, blk0 + nblk) in the batched grid.
struct BatchCgsInst {
    const void *V;
    int64_t ldv;
    int n;
    void *W;
    double *H;
    int ldh;
    double *h1, *h2, *nrm, *scal;
    double *part;
    unsigned *ticket;
    int nblk, blk0;
};
// Per-instance data of a batched polynomial pass (work items are groups of
// 32 rows, whatever the instance's chunk height); buffers by id:
// 0 = V[:, jj] (the step's input), 1 = W (output), 2 = P0, 3 = P1, 4 = T (pair temp).
struct BatchPassInst {
    SellView A;
    double sigma;
    float fsigma;  // sigma rounded to FP32 (the FP32 kernel reads it)
    const void *V;
    int64_t ldv;
    void *W, *P0, *P1, *T;
    DiaView D;  // the instance's matrix in diagonal storage when dia != 0 (else A, SELL)
    int dia;
};
// One pass of one instance: kind -1 none, 0 y = u, 1 y = x - a2 u, 2 y = aux - a1 x - a2 u.
struct BatchPassEntry {
    int kind, src, dst, aux;
    double a1, a2;
    float fa1, fa2;  // a1, a2 rounded to FP32
};
int cgs_batch_blocks(int n);
// Instance i takes part in step jj when lo[i] <= jj < hi[i] (device arrays).
void launch_cgs_batch(Prec p, const BatchCgsInst *ci, int count, int nblocks, const int *lo, const int *hi, int mode,
                      int jj, cudaStream_t st);
void launch_scale_batch(Prec p, const BatchCgsInst *ci, int count, int nblocks, const int *lo, const int *hi, int jj,
                        cudaStream_t st);
#ifdef __CUDACC__
// items: (instance, first 32-row group); each block takes `groups` groups
// (32 * groups threads), grid = min(nitems, grid_per_sm * SMs).
void launch_pass_batch(Prec p, const BatchPassInst *pi, const BatchPassEntry *tab, const int2 *items, int nitems,
                       const int *lo, const int *hi, int jj, int groups, int grid_per_sm, cudaStream_t st);
#endif

// Out[:, c] = sum_r V[:, r] Q[r, c] (c < kk), Q column major m x kk on the device,
// in the basis' storage precision and arithmetic.
void launch_rotate(Prec p, int n, const void *V, int64_t ldv, int m, const double *Q, int kk, void *out,
                   int64_t ldo, cudaStream_t st);
// The same product into an FP64 output with FP64 arithmetic (Ritz vectors).
void launch_rotate64(Prec p, int n, const void *V, int64_t ldv, int m, const double *Q, int kk, double *out,
                     int64_t ldo, cudaStream_t st);

// Column dots for the convergence test (Section 4).
//  mode 0: q[4c+0] = Y_c.Y_c, q[4c+1] = Y_c.AY_c, q[4c+2] = Y_c.AY_{pc}
//  mode 1: q[4c+3] = || AY_c - mur_c Y_c + sg_c mui_c Y_{pc} ||^2
struct ColDotArgs {
    int mode = 0;
    int n = 0;
    int nw = 0;
    const void *Y = nullptr;
    const void *AY = nullptr;
    int64_t ld = 0;
    const int *partner = nullptr;
    const double *mur = nullptr;
    const double *mui = nullptr;
    const double *sg = nullptr;
    double *q = nullptr;
    double *part = nullptr;
    unsigned *ticket = nullptr;
};
void launch_coldots(Prec p, const ColDotArgs &a, cudaStream_t st);

// SELL-C fill from a device CSR (slice pointers computed on the host); writes
// scol (32-bit) or soff (16-bit offsets), whichever is non-null.
void launch_sell_fill(Prec p, int n, int nslices, int cshift, const int *rowptr, const int *col, const double *val,
                      const int *slice_ptr, int *scol, short *soff, void *sval, cudaStream_t st);
void launch_csr_convert(Prec p, int64_t nnz, const double *val, void *out, cudaStream_t st);
// DIA fill from a device CSR with sorted columns (off: ndiag device offsets, increasing)
void launch_dia_fill(Prec p, int n, const int *rowptr, const int *col, const double *val, const int *off, int ndiag,
                     int64_t ld, void *dval, cudaStream_t st);
// y = x converted between storage precisions
void launch_convert(Prec from, Prec to, int n, const void *x, void *y, cudaStream_t st);

}  // namespace ppk
