// Kernels of the polynomial apply (sm_103a).
//
//  * k_pass / k_step: one fused pass of the factored GMRES polynomial
//    (Eq. (2.1)) on SELL-C (16- or 32-bit column indices) or CSR: SpMV with
//    A - sigma I plus the root-step axpy and the running sum (Section 2
//    footnote 2) in the same pass; conjugate pairs use two passes in real
//    arithmetic; the double polynomial's outer step (Section 8) is fused into
//    the last inner pass.
//  * k_pass_batch: the same pass for many instances in one launch.
//  * SELL-C construction and precision conversions.
#include "device_common.cuh"
#include "pp_internal.h"

#include <cstdint>

namespace ppk {

namespace {

// ---------------------------------------------------------------------------
// Fused root step
// ---------------------------------------------------------------------------
template <typename T, typename Acc>
__device__ __forceinline__ void step_epilogue(int row, Acc u, const StepArgs &s) {
    const T *x = (const T *)s.x;
    Acc xi = (Acc)x[row];
    if (s.sigma != 0.0) u = u - (Acc)s.sigma * xi;
    if (s.plain) {
        ((T *)s.y)[row] = (T)u;
        return;
    }
    Acc delta = (Acc)s.a1 * xi + (Acc)s.a2 * u;
    if (s.y) {
        Acc base = s.aux ? (Acc)((const T *)s.aux)[row] : xi;
        ((T *)s.y)[row] = (T)(base - delta);
    }
    if (s.r) {
        T *r = (T *)s.r;
        Acc rv = s.r_init ? delta : (Acc)r[row] + delta;
        if (s.r_write) r[row] = (T)rv;
        if (s.oy) {
            Acc od = (Acc)s.b2 * rv;
            if (s.ox) od += (Acc)s.b1 * (Acc)((const T *)s.ox)[row];
            ((T *)s.oy)[row] = (T)((Acc)((const T *)s.obase)[row] - od);
        }
    }
}

// Row sum u = sum_k A(row, col_k) x(col_k) over a SELL-C slice row (the
// slice width is uniform across the slice).  Kept to ~30 registers so that
// 2048 threads stay resident per SM: the gathers are latency-bound and need
// the warps more than a wider unroll.  The sum runs over the row's entries in
// CSR order whatever C, the index width or the block size (padding adds
// 0 * x exactly), so every format gives bit-identical results.
template <typename T, typename V, typename Acc, bool OFF16>
__device__ __forceinline__ Acc sell_row(const SellView &A, const T *__restrict__ x, int row) {
    const int cs = A.cshift;
    const int sl = row >> cs, lane = row & ((1 << cs) - 1);
    const int beg = __ldg(A.slice_ptr + sl);
    const int len = (__ldg(A.slice_ptr + sl + 1) - beg) >> cs;
    const V *val = (const V *)A.val + beg + lane;
    Acc acc = 0;
    if (OFF16) {
        const short *off = A.off + beg + lane;
        const T *xr = x + row;
#pragma unroll 4
        for (int k = 0; k < len; ++k)
            acc = fma((Acc)__ldg(val + (k << cs)), (Acc)__ldg(xr + __ldg(off + (k << cs))), acc);
    } else {
        const int *col = A.col + beg + lane;
#pragma unroll 4
        for (int k = 0; k < len; ++k)
            acc = fma((Acc)__ldg(val + (k << cs)), (Acc)__ldg(x + __ldg(col + (k << cs))), acc);
    }
    return acc;
}

// The same row sum with the loads of up to eight entries issued together:
// indices and values of the chunk first, then its x gathers, then the
// products in entry order (one round of memory latency per eight entries
// instead of one per entry of the loop's remainder).  Needs more registers;
// the tuner decides per matrix.
template <typename T, typename V, typename Acc, bool OFF16>
__device__ __forceinline__ Acc sell_row_wide(const SellView &A, const T *__restrict__ x, int row) {
    const int cs = A.cshift;
    const int sl = row >> cs, lane = row & ((1 << cs) - 1);
    const int beg = __ldg(A.slice_ptr + sl);
    const int len = (__ldg(A.slice_ptr + sl + 1) - beg) >> cs;
    const V *val = (const V *)A.val + beg + lane;
    const short *off = A.off + beg + lane;
    const int *col = A.col + beg + lane;
    Acc acc = 0;
    for (int k0 = 0; k0 < len; k0 += 8) {
        V v[8];
        int c[8];
        T xv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int k = k0 + t;
            if (k < len) {
                v[t] = __ldg(val + (k << cs));
                c[t] = OFF16 ? row + __ldg(off + (k << cs)) : __ldg(col + (k << cs));
            }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (k0 + t < len) xv[t] = __ldg(x + c[t]);
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (k0 + t < len) acc = fma((Acc)v[t], (Acc)xv[t], acc);
    }
    return acc;
}

constexpr int kPassMaxThreads = 512;

// Row sum of the matrix in format FMT: 0 CSR; SELL with 1 32-bit columns,
// 2 16-bit offsets, 3 / 4 the same with the wide row loop.  All sum a row's
// entries in CSR order.
template <typename T, typename V, typename Acc, int FMT>
__device__ __forceinline__ Acc row_sum(const SellView &S, const CsrView &R, const T *__restrict__ x, int row) {
    if constexpr (FMT == 0) {
        const int beg = __ldg(R.rowptr + row), end = __ldg(R.rowptr + row + 1);
        const V *val = (const V *)R.val;
        Acc acc = 0;
        for (int k = beg; k < end; ++k) acc = fma((Acc)__ldg(val + k), (Acc)__ldg(x + __ldg(R.col + k)), acc);
        return acc;
    } else if constexpr (FMT <= 2) {
        return sell_row<T, V, Acc, FMT == 2>(S, x, row);
    } else {
        return sell_row_wide<T, V, Acc, FMT == 4>(S, x, row);
    }
}

// Specialised passes of the factored polynomial (the hot cases):
//   KIND 0 plain:  y = u
//   KIND 1 real:   y = x - a2 u                (a2 = 1/theta)
//   KIND 2 pair 2: y = aux - a1 x - a2 u        (x = t, aux = p, a1 = c1, a2 = -c2)
// with u = A x - sigma x when SIGMA.
template <typename T, typename V, typename Acc, int KIND, bool SIGMA, int FMT>
__global__ void __launch_bounds__(kPassMaxThreads) k_pass(SellView S, CsrView R, StepArgs s) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (FMT == 0 ? R.n : S.n)) return;
    const T *x = (const T *)s.x;
    Acc u = row_sum<T, V, Acc, FMT>(S, R, x, row);
    if (SIGMA) u = fma(-(Acc)s.sigma, (Acc)x[row], u);
    T *y = (T *)s.y;
    if (KIND == 0) {
        y[row] = (T)u;
    } else if (KIND == 1) {
        y[row] = (T)fma(-(Acc)s.a2, u, (Acc)x[row]);
    } else {
        Acc v = fma(-(Acc)s.a1, (Acc)x[row], (Acc)((const T *)s.aux)[row]);
        y[row] = (T)fma(-(Acc)s.a2, u, v);
    }
}

// General pass (running sum, optional output, outer epilogue): see StepArgs.
template <typename T, typename V, typename Acc, int FMT>
__global__ void __launch_bounds__(kPassMaxThreads) k_step(SellView S, CsrView R, StepArgs s) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (FMT == 0 ? R.n : S.n)) return;
    Acc acc = row_sum<T, V, Acc, FMT>(S, R, (const T *)s.x, row);
    step_epilogue<T, Acc>(row, acc, s);
}

// One polynomial pass for every active instance: warp = 32 consecutive rows
// of one instance; a block takes blockDim/32 such groups of one instance
// (a work item) and blocks stride over the work items.
template <typename T>
__global__ void __launch_bounds__(kPassMaxThreads) k_pass_batch(const BatchPassInst *pi, const BatchPassEntry *tab,
                                                                const int2 *items, int nitems, const int *lo,
                                                                const int *hi, int jj) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 itm = items[it];
        const BatchPassEntry e = tab[itm.x];
        if (e.kind < 0 || jj < lo[itm.x] || jj >= hi[itm.x]) continue;
        const BatchPassInst &I = pi[itm.x];
        const int row = (itm.y + warp) * 32 + lane;
        if (row >= I.A.n) continue;
        const T *bufs[5] = {(const T *)I.V + (size_t)jj * I.ldv, (const T *)I.W, (const T *)I.P0, (const T *)I.P1,
                            (const T *)I.T};
        const T *x = bufs[e.src];
        T *y = (T *)bufs[e.dst];
        T u = I.A.off ? sell_row<T, T, T, true>(I.A, x, row) : sell_row<T, T, T, false>(I.A, x, row);
        if (I.sigma != 0.0) u = fma(-(T)I.sigma, x[row], u);
        if (e.kind == 0)
            y[row] = u;
        else if (e.kind == 1)
            y[row] = fma(-(T)e.a2, u, x[row]);
        else
            y[row] = fma(-(T)e.a2, u, fma(-(T)e.a1, x[row], bufs[e.aux][row]));
    }
}

// ---------------------------------------------------------------------------
// SELL-C construction
// ---------------------------------------------------------------------------
template <typename V>
__global__ void k_sell_fill(int n, int nslices, int cshift, const int *rowptr, const int *col, const double *val,
                            const int *slice_ptr, int *scol, short *soff, V *sval) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= (nslices << cshift)) return;
    int sl = row >> cshift, lane = row & ((1 << cshift) - 1);
    int beg = slice_ptr[sl], width = (slice_ptr[sl + 1] - beg) >> cshift;
    int rb = row < n ? rowptr[row] : 0, re = row < n ? rowptr[row + 1] : 0;
    int last = row < n ? (re > rb ? col[re - 1] : row) : 0;
    for (int k = 0; k < width; ++k) {
        int src = rb + k;
        size_t dst = (size_t)beg + ((size_t)k << cshift) + lane;
        int cc = src < re ? col[src] : last;  // padding: repeat a valid column, value 0
        if (scol) scol[dst] = cc;
        if (soff) soff[dst] = row < n ? (short)(cc - row) : (short)0;  // rows past n are never read
        sval[dst] = src < re ? (V)val[src] : (V)0;
    }
}

template <typename V>
__global__ void k_convert_vals(int64_t nnz, const double *val, V *out) {
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * kThreads)
        out[i] = (V)val[i];
}

template <typename A, typename B>
__global__ void k_convert(int n, const A *x, B *y) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) y[i] = (B)x[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename T, int FMT>
static void pass_dispatch(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    const int threads = A.threads;
    const int blocks = (A.n + threads - 1) / threads;
    const bool general = s.r || s.oy || !s.y;
    const bool sig = s.sigma != 0.0;
    if (general || (!s.plain && !s.aux && s.a1 != 0.0)) {  // not one of the specialised forms
        k_step<T, T, T, FMT><<<blocks, threads, 0, st>>>(A.sell, A.csr, s);
        return;
    }
    int kind = s.plain ? 0 : (s.aux ? 2 : 1);
#define PP_PASS(K, S) k_pass<T, T, T, K, S, FMT><<<blocks, threads, 0, st>>>(A.sell, A.csr, s)
    if (kind == 0) {
        if (sig) PP_PASS(0, true); else PP_PASS(0, false);
    } else if (kind == 1) {
        if (sig) PP_PASS(1, true); else PP_PASS(1, false);
    } else {
        if (sig) PP_PASS(2, true); else PP_PASS(2, false);
    }
#undef PP_PASS
}

template <typename T>
static void pass_format(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    if (A.fmt != 2)
        pass_dispatch<T, 0>(A, s, st);
    else if (A.sell.off)
        A.wide ? pass_dispatch<T, 4>(A, s, st) : pass_dispatch<T, 2>(A, s, st);
    else
        A.wide ? pass_dispatch<T, 3>(A, s, st) : pass_dispatch<T, 1>(A, s, st);
}

void launch_step(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    if (A.prec == F64)
        pass_format<double>(A, s, st);
    else
        pass_format<float>(A, s, st);
}

void launch_pass_batch(Prec p, const BatchPassInst *pi, const BatchPassEntry *tab, const int2 *items, int nitems,
                       const int *lo, const int *hi, int jj, int groups, int grid_per_sm, cudaStream_t st) {
    int g = num_sms() * grid_per_sm;
    if (nitems < g) g = nitems;
    if (g < 1) g = 1;
    const int threads = 32 * groups;
    if (p == F64)
        k_pass_batch<double><<<g, threads, 0, st>>>(pi, tab, items, nitems, lo, hi, jj);
    else
        k_pass_batch<float><<<g, threads, 0, st>>>(pi, tab, items, nitems, lo, hi, jj);
}

void launch_sell_fill(Prec p, int n, int nslices, int cshift, const int *rowptr, const int *col, const double *val,
                      const int *slice_ptr, int *scol, short *soff, void *sval, cudaStream_t st) {
    const int rows = nslices << cshift;
    const int blocks = (rows + kThreads - 1) / kThreads;
    if (p == F64)
        k_sell_fill<double><<<blocks, kThreads, 0, st>>>(n, nslices, cshift, rowptr, col, val, slice_ptr, scol, soff,
                                                         (double *)sval);
    else
        k_sell_fill<float><<<blocks, kThreads, 0, st>>>(n, nslices, cshift, rowptr, col, val, slice_ptr, scol, soff,
                                                        (float *)sval);
}

void launch_csr_convert(Prec p, int64_t nnz, const double *val, void *out, cudaStream_t st) {
    int g = num_sms() * 4;
    if (p == F32) k_convert_vals<float><<<g, kThreads, 0, st>>>(nnz, val, (float *)out);
}

void launch_convert(Prec from, Prec to, int n, const void *x, void *y, cudaStream_t st) {
    int g = num_sms() * 4;
    if (from == F64 && to == F32)
        k_convert<double, float><<<g, kThreads, 0, st>>>(n, (const double *)x, (float *)y);
    else if (from == F32 && to == F64)
        k_convert<float, double><<<g, kThreads, 0, st>>>(n, (const float *)x, (double *)y);
    else if (from == F64)
        k_convert<double, double><<<g, kThreads, 0, st>>>(n, (const double *)x, (double *)y);
    else
        k_convert<float, float><<<g, kThreads, 0, st>>>(n, (const float *)x, (float *)y);
}

}  // namespace ppk
