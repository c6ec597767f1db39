// CUDA kernels of the hot path (sm_103a).
//
//  * k_pass / k_step: one fused pass of the factored GMRES polynomial
//    (Eq. (2.1)) on SELL-C (16- or 32-bit column indices) or CSR: SpMV with
//    A - sigma I plus the root-step axpy and the running sum (Section 2
//    footnote 2) in the same pass; conjugate pairs use two passes in real
//    arithmetic; the double polynomial's outer step (Section 8) is fused into
//    the last inner pass.
//  * k_cgs: the three passes of classical Gram-Schmidt with one
//    reorthogonalisation (Section 4), each a single sweep over the basis with
//    a deterministic two-level reduction finished by the last block.
//  * k_rotate: V_m Q_k for the thick restart and Ritz vectors (Section 4).
//  * k_coldots: Rayleigh quotients and residual norms on A (Section 4).
#include "pp_internal.h"

#include <cuda_runtime.h>

namespace ppk {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename T>
__device__ __forceinline__ double ld_acc(const T *p, size_t i) {
    return (double)__ldg(p + i);
}

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

constexpr int kPassMaxThreads = 512;

// Row sum of the matrix in format FMT: 0 CSR, 1 SELL with 32-bit columns,
// 2 SELL with 16-bit offsets.  All three sum a row's entries in CSR order.
template <typename T, typename V, typename Acc, int FMT>
__device__ __forceinline__ Acc row_sum(const SellView &S, const CsrView &R, const T *__restrict__ x, int row) {
    if constexpr (FMT == 0) {
        const int beg = __ldg(R.rowptr + row), end = __ldg(R.rowptr + row + 1);
        const V *val = (const V *)R.val;
        Acc acc = 0;
        for (int k = beg; k < end; ++k) acc = fma((Acc)__ldg(val + k), (Acc)__ldg(x + __ldg(R.col + k)), acc);
        return acc;
    } else {
        return sell_row<T, V, Acc, FMT == 2>(S, x, row);
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

// ---------------------------------------------------------------------------
// Deterministic grid reduction: every block writes `nout` partials to
// part[block * nout + o]; the last block to arrive sums them in block order.
// ---------------------------------------------------------------------------
__device__ bool last_block(unsigned *ticket, unsigned nblocks) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == nblocks - 1);
    __syncthreads();
    return is_last;
}

__device__ bool last_block(unsigned *ticket) { return last_block(ticket, gridDim.x * gridDim.y); }

__device__ void reduce_partials(const double *part, int nblocks, int nout, double *out) {
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int o = warp; o < nout; o += kWarps) {
        double s = 0;
        for (int b = lane; b < nblocks; b += 32) s += __ldcg(part + (size_t)b * nout + o);
#pragma unroll
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) out[o] = s;
    }
}

// ---------------------------------------------------------------------------
// CGS2 passes. A tile is kRows consecutive rows; warp w owns basis columns
// c = w + 8 cc (cc < CPW).  Each lane holds kRows/32 rows of the tile.
// ---------------------------------------------------------------------------
constexpr int kRows = 64;
constexpr int kQ = kRows / 32;

// Per-block partial sums of a sweep, then the last block's reduction and (mode
// 2) the Hessenberg column.  acc[cc] is the block-local projection on column
// warp + kWarps cc; nrm the squared norm of the updated vector's rows.
template <int CPW>
__device__ __forceinline__ void cgs_finish(const CgsArgs &a, int bid, int nblk, const double (&acc)[CPW],
                                           double nrm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int j = a.j;
    __shared__ double nrm_sh[kWarps];
    const int nout = (a.mode == 0) ? j : (a.mode == 1 ? j + 1 : 1);
    double *part = a.part + (size_t)bid * nout;
    if (a.mode != 2) {
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            double s = acc[cc];
#pragma unroll
            for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            int c = warp + kWarps * cc;
            if (lane == 0 && c < j) part[c] = s;
        }
    }
    if (a.mode != 0) {
#pragma unroll
        for (int off = 16; off; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
        if (lane == 0) nrm_sh[warp] = nrm;
        __syncthreads();
        if (tid == 0) {
            double s = 0;
            for (int ww = 0; ww < kWarps; ++ww) s += nrm_sh[ww];
            part[a.mode == 1 ? j : 0] = s;
        }
    }
    if (!last_block(a.ticket, nblk)) return;
    reduce_partials(a.part, nblk, nout, a.out);
    __syncthreads();
    if (tid == 0) *a.ticket = 0;
    if (a.mode == 2) {
        __threadfence_block();
        __syncthreads();
        double nn = sqrt(a.out[0]);
        for (int c = tid; c < j; c += kThreads) a.hcol[c] = a.h1[c] + a.h[c];
        if (tid == 0) {
            a.hcol[j] = nn;
            a.scal[0] = nn > 0 ? 1.0 / nn : 0.0;
        }
    }
}

// The sweep of block `bid` out of `nblk` blocks working on an FP64 basis:
// FP64 throughout.
template <int CPW>
__device__ __forceinline__ void cgs_body_f64(const CgsArgs &a, int bid, int nblk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const double *V = (const double *)a.V;
    const double *w = (const double *)a.w;
    double *wout = (double *)a.wout;
    const int j = a.j, n = a.n;
    __shared__ double red[kWarps][kRows];
    __shared__ double wsh[kRows];
    __shared__ double hs[8 * CPW];
    if (a.mode != 0)
        for (int c = tid; c < j; c += kThreads) hs[c] = a.h[c];
    __syncthreads();
    double acc[CPW];
#pragma unroll
    for (int cc = 0; cc < CPW; ++cc) acc[cc] = 0;
    double nrm = 0;
    const int ntiles = (n + kRows - 1) / kRows;
    for (int tile = bid; tile < ntiles; tile += nblk) {
        const int r0 = tile * kRows;
        double vv[CPW][kQ];
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            int c = warp + kWarps * cc;
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                int row = r0 + lane + 32 * q;
                vv[cc][q] = (c < j && row < n) ? __ldg(V + (size_t)c * a.ldv + row) : 0.0;
            }
        }
        if (a.mode == 0) {
            double wv[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                int row = r0 + lane + 32 * q;
                wv[q] = row < n ? __ldg(w + row) : 0.0;
            }
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc)
                if (warp + kWarps * cc < j)  // warp-uniform: no FMAs on columns past j
#pragma unroll
                    for (int q = 0; q < kQ; ++q) acc[cc] = fma(vv[cc][q], wv[q], acc[cc]);
            continue;
        }
        // w - V h for the tile rows: per-warp partial sums, then across warps
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            double s = 0;
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) {
                int c = warp + kWarps * cc;
                if (c < j) s = fma(vv[cc][q], hs[c], s);
            }
            red[warp][lane + 32 * q] = s;
        }
        __syncthreads();
        if (tid < kRows) {
            int row = r0 + tid;
            double v = 0;
            if (row < n) {
                double s = 0;
#pragma unroll
                for (int ww = 0; ww < kWarps; ++ww) s += red[ww][tid];
                v = __ldg(w + row) - s;
                wout[row] = v;
                nrm = fma(v, v, nrm);
            }
            wsh[tid] = v;
        }
        __syncthreads();
        if (a.mode == 1) {
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc)
                if (warp + kWarps * cc < j)
#pragma unroll
                    for (int q = 0; q < kQ; ++q) acc[cc] = fma(vv[cc][q], wsh[lane + 32 * q], acc[cc]);
        }
    }
    cgs_finish<CPW>(a, bid, nblk, acc, nrm);
}

// One term of the compensated dot product Dot2 (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005)): the
// product's rounding error from an FMA (TwoProduct), the sum's from Knuth's
// TwoSum; the errors accumulate in c, so s + c is the dot product as if
// computed in twice the working precision.  The _rn intrinsics keep the
// compiler from contracting or reassociating the error-free steps.
__device__ __forceinline__ void dot2_term(float x, float y, float &s, float &c) {
    float p = __fmul_rn(x, y);
    float e = fmaf(x, y, -p);
    float t = __fadd_rn(s, p);
    float z = __fsub_rn(t, s);
    float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
}

// The sweep over an FP32 basis.  The first projection h1 = V^T w and both
// updates w - V h run in FP32 (FP32 FMAs are many times faster than FP64 ones
// on this part); the reorthogonalising projection h2 = V^T w1 uses Dot2, so
// the second Gram-Schmidt pass is accurate to about twice FP32 precision.
// Squared norms accumulate in FP64.
template <int CPW>
__device__ __forceinline__ void cgs_body_f32(const CgsArgs &a, int bid, int nblk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const float *V = (const float *)a.V;
    const float *w = (const float *)a.w;
    float *wout = (float *)a.wout;
    const int j = a.j, n = a.n;
    __shared__ float red[kWarps][kRows];
    __shared__ float wsh[kRows];
    __shared__ float hs[8 * CPW];
    if (a.mode != 0)
        for (int c = tid; c < j; c += kThreads) hs[c] = (float)a.h[c];
    __syncthreads();
    float hi[CPW], lo[CPW];
#pragma unroll
    for (int cc = 0; cc < CPW; ++cc) hi[cc] = lo[cc] = 0.f;
    double nrm = 0;
    const int ntiles = (n + kRows - 1) / kRows;
    for (int tile = bid; tile < ntiles; tile += nblk) {
        const int r0 = tile * kRows;
        float vv[CPW][kQ];
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            int c = warp + kWarps * cc;
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                int row = r0 + lane + 32 * q;
                vv[cc][q] = (c < j && row < n) ? __ldg(V + (size_t)c * a.ldv + row) : 0.f;
            }
        }
        if (a.mode == 0) {
            float wv[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                int row = r0 + lane + 32 * q;
                wv[q] = row < n ? __ldg(w + row) : 0.f;
            }
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc)
                if (warp + kWarps * cc < j)
#pragma unroll
                    for (int q = 0; q < kQ; ++q) hi[cc] = fmaf(vv[cc][q], wv[q], hi[cc]);
            continue;
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            float s = 0;
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) {
                int c = warp + kWarps * cc;
                if (c < j) s = fmaf(vv[cc][q], hs[c], s);
            }
            red[warp][lane + 32 * q] = s;
        }
        __syncthreads();
        if (tid < kRows) {
            int row = r0 + tid;
            float v = 0;
            if (row < n) {
                float s = 0;
#pragma unroll
                for (int ww = 0; ww < kWarps; ++ww) s += red[ww][tid];
                v = __ldg(w + row) - s;
                wout[row] = v;
                nrm = fma((double)v, (double)v, nrm);
            }
            wsh[tid] = v;
        }
        __syncthreads();
        if (a.mode == 1) {
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc)
                if (warp + kWarps * cc < j)
#pragma unroll
                    for (int q = 0; q < kQ; ++q) dot2_term(vv[cc][q], wsh[lane + 32 * q], hi[cc], lo[cc]);
        }
    }
    double acc[CPW];
#pragma unroll
    for (int cc = 0; cc < CPW; ++cc) acc[cc] = (double)hi[cc] + (double)lo[cc];
    cgs_finish<CPW>(a, bid, nblk, acc, nrm);
}

template <typename T, int CPW>
__device__ __forceinline__ void cgs_body(const CgsArgs &a, int bid, int nblk) {
    if constexpr (sizeof(T) == 8)
        cgs_body_f64<CPW>(a, bid, nblk);
    else
        cgs_body_f32<CPW>(a, bid, nblk);
}

template <typename T, int CPW>
__global__ void __launch_bounds__(kThreads) k_cgs(CgsArgs a) {
    cgs_body<T, CPW>(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Batched forms: many independent instances in one launch.  Instance state is
// in device tables, so one captured graph serves every cycle; instance i is
// active at Arnoldi step jj when lo[i] <= jj < hi[i] (its restart column and
// its subspace size; hi = 0 once it is done).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_instance(const BatchCgsInst *ci, int count, int b) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ci[mid].blk0 <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename T, int CPW>
__global__ void __launch_bounds__(kThreads) k_cgs_batch(const BatchCgsInst *ci, int count, const int *lo,
                                                        const int *hi, int mode, int jj) {
    const int i = find_instance(ci, count, blockIdx.x);
    if (jj < lo[i] || jj >= hi[i]) return;
    const BatchCgsInst &I = ci[i];
    CgsArgs a;
    a.mode = mode;
    a.n = I.n;
    a.V = I.V;
    a.ldv = I.ldv;
    a.j = jj + 1;
    a.w = I.W;
    a.part = I.part;
    a.ticket = I.ticket;
    if (mode == 0) {
        a.out = I.h1;
    } else if (mode == 1) {
        a.h = I.h1;
        a.wout = I.W;
        a.out = I.h2;
    } else {
        a.h = I.h2;
        a.h1 = I.h1;
        a.wout = (T *)I.V + (size_t)(jj + 1) * I.ldv;
        a.out = I.nrm;
        a.hcol = I.H + (size_t)jj * I.ldh;
        a.scal = I.scal;
    }
    cgs_body<T, CPW>(a, blockIdx.x - I.blk0, I.nblk);
}

template <typename T>
__global__ void k_scale_batch(const BatchCgsInst *ci, int count, const int *lo, const int *hi, int jj) {
    const int i = find_instance(ci, count, blockIdx.x);
    if (jj < lo[i] || jj >= hi[i]) return;
    const BatchCgsInst &I = ci[i];
    T *x = (T *)I.V + (size_t)(jj + 1) * I.ldv;
    const double s = *I.scal;
    for (int r = (blockIdx.x - I.blk0) * kThreads + threadIdx.x; r < I.n; r += I.nblk * kThreads)
        x[r] = (T)((double)x[r] * s);
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

template <typename T>
__global__ void k_scale(int n, T *x, const double *scal) {
    double s = *scal;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = (T)((double)x[i] * s);
}

// ---------------------------------------------------------------------------
// Out = V[:, 0:m] Q  (tile of 32 rows per block iteration; Q and the V tile in
// shared memory; warp w computes output columns w, w+8, ...).  Acc is the
// arithmetic: FP64 for FP64 bases; FP32 for FP32 bases, whose columns are
// rounded to FP32 on store anyway (an FP64 FMA costs many FP32 ones here).
// ---------------------------------------------------------------------------
template <typename T, typename TO, typename Acc>
__global__ void __launch_bounds__(kThreads) k_rotate(int n, const T *V, int64_t ldv, int m, const double *Q,
                                                     int kk, TO *out, int64_t ldo) {
    extern __shared__ double sm_raw[];
    Acc *Qs = (Acc *)sm_raw;          // m * kk
    Acc *Vs = Qs + (size_t)m * kk;    // m * 32
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < m * kk; i += kThreads) Qs[i] = (Acc)Q[i];
    const int ntiles = (n + 31) / 32;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int row = tile * 32 + lane;
        __syncthreads();
        for (int r = warp; r < m; r += kWarps) Vs[r * 32 + lane] = row < n ? (Acc)__ldg(V + (size_t)r * ldv + row) : (Acc)0;
        __syncthreads();
        for (int c = warp; c < kk; c += kWarps) {
            Acc acc = 0;
            const Acc *qc = Qs + (size_t)c * m;
            for (int r = 0; r < m; ++r) acc = fma(Vs[r * 32 + lane], qc[r], acc);
            if (row < n) out[(size_t)c * ldo + row] = (TO)acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Column dots for the convergence test.  grid.y = column, grid.x = row chunks.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_coldots(ColDotArgs a) {
    const int c = blockIdx.y;
    const int p = a.partner[c];
    const T *Y = (const T *)a.Y, *AY = (const T *)a.AY;
    const T *yc = Y + (size_t)c * a.ld, *ayc = AY + (size_t)c * a.ld;
    const T *yp = Y + (size_t)p * a.ld, *ayp = AY + (size_t)p * a.ld;
    double s0 = 0, s1 = 0, s2 = 0;
    double mr = 0, mi = 0;
    if (a.mode == 1) {
        mr = a.mur[c];
        mi = a.sg[c] * a.mui[c];
    }
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < a.n; i += gridDim.x * kThreads) {
        double y = ld_acc(yc, i), ay = ld_acc(ayc, i);
        if (a.mode == 0) {
            s0 = fma(y, y, s0);
            s1 = fma(y, ay, s1);
            s2 = fma(y, ld_acc(ayp, i), s2);
        } else {
            double r = ay - mr * y + mi * ld_acc(yp, i);
            s0 = fma(r, r, s0);
        }
    }
    __shared__ double sh[3][kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if (lane == 0) {
        sh[0][warp] = s0;
        sh[1][warp] = s1;
        sh[2][warp] = s2;
    }
    __syncthreads();
    const int nout = 3;
    double *part = a.part + ((size_t)c * gridDim.x + blockIdx.x) * nout;
    if (threadIdx.x < 3) {
        double s = 0;
        for (int ww = 0; ww < kWarps; ++ww) s += sh[threadIdx.x][ww];
        part[threadIdx.x] = s;
    }
    if (!last_block(a.ticket)) return;
    // reduce: for column cc, entries part[(cc*gx + b)*3 + t]
    const int gx = gridDim.x;
    for (int idx = threadIdx.x >> 5; idx < a.nw * 3; idx += kWarps) {
        int cc = idx / 3, t = idx % 3;
        double s = 0;
        for (int b = lane; b < gx; b += 32) s += __ldcg(a.part + ((size_t)cc * gx + b) * 3 + t);
#pragma unroll
        for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
            if (a.mode == 0)
                a.q[4 * cc + t] = s;
            else if (t == 0)
                a.q[4 * cc + 3] = s;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.ticket = 0;
}

// ---------------------------------------------------------------------------
// SELL-32 construction
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

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 132;
    }
    return sms;
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
        pass_dispatch<T, 2>(A, s, st);
    else
        pass_dispatch<T, 1>(A, s, st);
}

void launch_step(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    if (A.prec == F64)
        pass_format<double>(A, s, st);
    else
        pass_format<float>(A, s, st);
}

int cgs_grid(int n) {
    int tiles = (n + kRows - 1) / kRows;
    int g = num_sms() * 4;
    return tiles < g ? tiles : g;
}

// Blocks of a CGS pass: one wave of resident blocks (at most 4 per SM, which
// bounds the partial-sum buffer), never more than there are tiles.
template <typename T, int CPW>
static int resident_grid(int n, int cap) {
    static int per_sm = 0;  // one per instantiation
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cgs<T, CPW>, kThreads, 0);
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 4) per_sm = 4;
    }
    int tiles = (n + kRows - 1) / kRows;
    int g = per_sm * num_sms();
    if (cap > 0 && g > cap) g = cap;
    return tiles < g ? tiles : g;
}

template <typename T>
static void cgs_dispatch(const CgsArgs &a, int cap, cudaStream_t st) {
    int cpw = (a.j + kWarps - 1) / kWarps;
    if (cpw <= 2)
        k_cgs<T, 2><<<resident_grid<T, 2>(a.n, cap), kThreads, 0, st>>>(a);
    else if (cpw <= 4)
        k_cgs<T, 4><<<resident_grid<T, 4>(a.n, cap), kThreads, 0, st>>>(a);
    else if (cpw <= 8)
        k_cgs<T, 8><<<resident_grid<T, 8>(a.n, cap), kThreads, 0, st>>>(a);
    else
        k_cgs<T, 16><<<resident_grid<T, 16>(a.n, cap), kThreads, 0, st>>>(a);
}

void launch_cgs(Prec p, const CgsArgs &a, cudaStream_t st) {
    if (p == F64)
        cgs_dispatch<double>(a, 0, st);
    else
        cgs_dispatch<float>(a, 0, st);
}

void launch_cgs_batch(Prec p, const BatchCgsInst *ci, int count, int nblocks, const int *lo, const int *hi, int mode,
                      int jj, cudaStream_t st) {
    int cpw = (jj + 1 + kWarps - 1) / kWarps;
#define PP_CB(T, C) k_cgs_batch<T, C><<<nblocks, kThreads, 0, st>>>(ci, count, lo, hi, mode, jj)
    if (p == F64) {
        if (cpw <= 2) PP_CB(double, 2); else if (cpw <= 4) PP_CB(double, 4); else if (cpw <= 8) PP_CB(double, 8); else PP_CB(double, 16);
    } else {
        if (cpw <= 2) PP_CB(float, 2); else if (cpw <= 4) PP_CB(float, 4); else if (cpw <= 8) PP_CB(float, 8); else PP_CB(float, 16);
    }
#undef PP_CB
}

void launch_scale_batch(Prec p, const BatchCgsInst *ci, int count, int nblocks, const int *lo, const int *hi, int jj,
                        cudaStream_t st) {
    if (p == F64)
        k_scale_batch<double><<<nblocks, kThreads, 0, st>>>(ci, count, lo, hi, jj);
    else
        k_scale_batch<float><<<nblocks, kThreads, 0, st>>>(ci, count, lo, hi, jj);
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

int cgs_batch_blocks(int n) {
    // blocks for one instance: tiles of 64 rows, at most one wave share of 3 per SM
    int tiles = (n + kRows - 1) / kRows;
    int cap = num_sms() * 3;
    return tiles < cap ? tiles : cap;
}

void launch_cgs_grid(Prec p, const CgsArgs &a, int grid_cap, cudaStream_t st) {
    if (p == F64)
        cgs_dispatch<double>(a, grid_cap, st);
    else
        cgs_dispatch<float>(a, grid_cap, st);
}

void launch_scale(Prec p, int n, void *x, const double *scal, cudaStream_t st) {
    int g = num_sms() * 4;
    if (p == F64)
        k_scale<double><<<g, kThreads, 0, st>>>(n, (double *)x, scal);
    else
        k_scale<float><<<g, kThreads, 0, st>>>(n, (float *)x, scal);
}

void launch_rotate(Prec p, int n, const void *V, int64_t ldv, int m, const double *Q, int kk, void *out,
                   int64_t ldo, cudaStream_t st) {
    const size_t acc_bytes = p == F64 ? sizeof(double) : sizeof(float);
    size_t smem = ((size_t)m * kk + (size_t)m * 32) * acc_bytes;
    int tiles = (n + 31) / 32;
    int g = num_sms() * 2;
    if (tiles < g) g = tiles;
    if (p == F64) {
        cudaFuncSetAttribute(k_rotate<double, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_rotate<double, double, double><<<g, kThreads, smem, st>>>(n, (const double *)V, ldv, m, Q, kk,
                                                                    (double *)out, ldo);
    } else {
        cudaFuncSetAttribute(k_rotate<float, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_rotate<float, float, float><<<g, kThreads, smem, st>>>(n, (const float *)V, ldv, m, Q, kk, (float *)out,
                                                                 ldo);
    }
}

void launch_rotate64(Prec p, int n, const void *V, int64_t ldv, int m, const double *Q, int kk, double *out,
                     int64_t ldo, cudaStream_t st) {
    size_t smem = ((size_t)m * kk + (size_t)m * 32) * sizeof(double);
    int tiles = (n + 31) / 32;
    int g = num_sms() * 2;
    if (tiles < g) g = tiles;
    if (p == F64) {
        launch_rotate(p, n, V, ldv, m, Q, kk, out, ldo, st);
    } else {
        cudaFuncSetAttribute(k_rotate<float, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_rotate<float, double, double><<<g, kThreads, smem, st>>>(n, (const float *)V, ldv, m, Q, kk, out, ldo);
    }
}

void launch_coldots(Prec p, const ColDotArgs &a, cudaStream_t st) {
    int gx = (a.n + kThreads * 8 - 1) / (kThreads * 8);
    int cap = num_sms() * 2;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    dim3 grid(gx, a.nw);
    if (p == F64)
        k_coldots<double><<<grid, kThreads, 0, st>>>(a);
    else
        k_coldots<float><<<grid, kThreads, 0, st>>>(a);
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
