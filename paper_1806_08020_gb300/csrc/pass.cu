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

// A coefficient in the accumulation type: the FP32 copy for FP32 kernels (set
// on the host), the double itself for FP64 ones.
template <typename Acc>
__device__ __forceinline__ Acc cf(double d, float f) {
    if constexpr (sizeof(Acc) == 4)
        return f;
    else
        return (Acc)d;
}

// ---------------------------------------------------------------------------
// Fused root step
// ---------------------------------------------------------------------------
template <typename T, typename Acc>
__device__ __forceinline__ void step_epilogue(int row, Acc u, const StepArgs &s) {
    const T *x = (const T *)s.x;
    Acc xi = (Acc)x[row];
    if (s.has_sigma) u = u - cf<Acc>(s.sigma, s.fsigma) * xi;
    if (s.plain) {
        ((T *)s.y)[row] = (T)u;
        return;
    }
    Acc delta = cf<Acc>(s.a1, s.fa1) * xi + cf<Acc>(s.a2, s.fa2) * u;
    if (s.y) {
        Acc base = s.aux ? (Acc)((const T *)s.aux)[row] : xi;
        ((T *)s.y)[row] = (T)(base - delta);
    }
    if (s.r) {
        T *r = (T *)s.r;
        Acc rv = s.r_init ? delta : (Acc)r[row] + delta;
        if (s.r_write) r[row] = (T)rv;
        if (s.oy) {
            Acc od = cf<Acc>(s.b2, s.fb2) * rv;
            if (s.ox) od += cf<Acc>(s.b1, s.fb1) * (Acc)((const T *)s.ox)[row];
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

// Two rows per thread (row0 and row0 + blockDim), their entries interleaved
// in one loop: twice the independent loads in flight per thread at the same
// register budget per row.  Each row still sums in CSR order.
template <typename T, typename V, typename Acc, bool OFF16>
__device__ __forceinline__ void sell_row2(const SellView &A, const T *__restrict__ x, int r0, int r1, bool has1,
                                          Acc &u0, Acc &u1) {
    const int cs = A.cshift, mask = (1 << cs) - 1;
    const int b0 = __ldg(A.slice_ptr + (r0 >> cs));
    const int l0 = (__ldg(A.slice_ptr + (r0 >> cs) + 1) - b0) >> cs;
    int b1 = b0, l1 = 0;
    if (has1) {
        b1 = __ldg(A.slice_ptr + (r1 >> cs));
        l1 = (__ldg(A.slice_ptr + (r1 >> cs) + 1) - b1) >> cs;
    }
    const V *v0 = (const V *)A.val + b0 + (r0 & mask), *v1 = (const V *)A.val + b1 + (r1 & mask);
    const short *o0 = A.off + b0 + (r0 & mask), *o1 = A.off + b1 + (r1 & mask);
    const int *c0 = A.col + b0 + (r0 & mask), *c1 = A.col + b1 + (r1 & mask);
    u0 = 0;
    u1 = 0;
    const int L = l0 > l1 ? l0 : l1;
#pragma unroll 4
    for (int k = 0; k < L; ++k) {
        const int e = k << cs;
        if (k < l0) {
            const int c = OFF16 ? r0 + __ldg(o0 + e) : __ldg(c0 + e);
            u0 = fma((Acc)__ldg(v0 + e), (Acc)__ldg(x + c), u0);
        }
        if (k < l1) {
            const int c = OFF16 ? r1 + __ldg(o1 + e) : __ldg(c1 + e);
            u1 = fma((Acc)__ldg(v1 + e), (Acc)__ldg(x + c), u1);
        }
    }
}

constexpr int kPassMaxThreads = 512;

// Row sum of the matrix in format FMT: 0 CSR; SELL with 1 32-bit columns,
// 2 16-bit offsets, 3 / 4 the same with the wide row loop (5 / 6: two rows per
// thread, handled by the kernels).  All sum a row's entries in CSR order.
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
// Row sum over the diagonals (DIA): no index loads; the offsets are in shared
// memory.  Diagonals run in increasing offset, i.e. the row's CSR order; where
// the matrix has no entry the stored value is 0 and adds 0 * x exactly.
template <typename Acc, int K>
__device__ __forceinline__ Acc dia_fmas(const Acc (&a)[8], const Acc (&xv)[8], Acc acc) {
#pragma unroll
    for (int u = 0; u < K; ++u) acc = fma(a[u], xv[u], acc);
    return acc;
}

template <typename T, typename V, typename Acc>
__device__ __forceinline__ Acc dia_row(const DiaView &D, const int *off_s, const T *__restrict__ x, int row) {
    // the row's block of 32 rows holds its ndiag values 32 apart
    const V *val = (const V *)D.val + (size_t)(row >> 5) * ((size_t)D.ndiag * 32) + (row & 31);
    Acc acc = 0;
    // eight diagonals at a time: all their loads issued before the products
    for (int d0 = 0; d0 < D.ndiag; d0 += 8) {
        Acc a[8], xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int d = d0 + u;
            a[u] = 0;
            xv[u] = 0;
            if (d < D.ndiag) {
                const int c = row + off_s[d];
                a[u] = (Acc)__ldg(val + d * 32);
                if (c >= 0 && c < D.n) xv[u] = (Acc)__ldg(x + c);
            }
        }
        // exactly min(8, ndiag - d0) products (a warp-uniform branch): padded
        // slots would still occupy the FP64 pipe, the bound of the FP64 pass
        switch (D.ndiag - d0 < 8 ? D.ndiag - d0 : 8) {
            case 1: acc = dia_fmas<Acc, 1>(a, xv, acc); break;
            case 2: acc = dia_fmas<Acc, 2>(a, xv, acc); break;
            case 3: acc = dia_fmas<Acc, 3>(a, xv, acc); break;
            case 4: acc = dia_fmas<Acc, 4>(a, xv, acc); break;
            case 5: acc = dia_fmas<Acc, 5>(a, xv, acc); break;
            case 6: acc = dia_fmas<Acc, 6>(a, xv, acc); break;
            case 7: acc = dia_fmas<Acc, 7>(a, xv, acc); break;
            default: acc = dia_fmas<Acc, 8>(a, xv, acc); break;
        }
    }
    return acc;
}

template <typename T, typename V, typename Acc, int KIND, bool SIGMA>
__global__ void __launch_bounds__(kPassMaxThreads) k_pass_dia(DiaView D, StepArgs s) {
    grid_trigger();
    grid_wait();
    __shared__ int off_s[kDiaMax];
    for (int d = threadIdx.x; d < D.ndiag; d += blockDim.x) off_s[d] = D.off[d];
    __syncthreads();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= D.n) return;
    const T *x = (const T *)s.x;
    T *y = (T *)s.y;
    Acc u = dia_row<T, V, Acc>(D, off_s, x, row);
    if (SIGMA) u = fma(-cf<Acc>(s.sigma, s.fsigma), (Acc)x[row], u);
    if (KIND == 0) {
        y[row] = (T)u;
    } else if (KIND == 1) {
        y[row] = (T)fma(-cf<Acc>(s.a2, s.fa2), u, (Acc)x[row]);
    } else {
        Acc v = fma(-cf<Acc>(s.a1, s.fa1), (Acc)x[row], (Acc)((const T *)s.aux)[row]);
        y[row] = (T)fma(-cf<Acc>(s.a2, s.fa2), u, v);
    }
}

template <typename T, typename V, typename Acc>
__global__ void __launch_bounds__(kPassMaxThreads) k_step_dia(DiaView D, StepArgs s) {
    grid_trigger();
    grid_wait();
    __shared__ int off_s[kDiaMax];
    for (int d = threadIdx.x; d < D.ndiag; d += blockDim.x) off_s[d] = D.off[d];
    __syncthreads();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= D.n) return;
    step_epilogue<T, Acc>(row, dia_row<T, V, Acc>(D, off_s, (const T *)s.x, row), s);
}

// FP32 DIA with R (2 or 4) consecutive rows per thread (r0 = R q): the values
// of a diagonal for the R rows are one 8- or 16-byte load (the 32-row blocks
// keep them adjacent), x for a diagonal whose offset is a multiple of R is one
// such load too (else R loads), and the epilogue's vectors move in 8- or
// 16-byte loads and stores.  The loads of up to eight diagonals are issued
// before their products.  Products run in increasing diagonal order per row
// with the same operands as dia_row, so the results are bit-identical to the
// one-row kernels.  Needs every vector pointer 4R-byte aligned (checked at
// dispatch).
template <int R>
struct VecR;
template <>
struct VecR<4> {
    __device__ static __forceinline__ void ld(const float *p, float (&o)[4]) {
        const float4 v = __ldg((const float4 *)p);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    }
    __device__ static __forceinline__ void st(float *p, const float (&v)[4]) {
        *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct VecR<2> {
    __device__ static __forceinline__ void ld(const float *p, float (&o)[2]) {
        const float2 v = __ldg((const float2 *)p);
        o[0] = v.x;
        o[1] = v.y;
    }
    __device__ static __forceinline__ void st(float *p, const float (&v)[2]) { *(float2 *)p = make_float2(v[0], v[1]); }
};

template <int R>
__device__ __forceinline__ void dia_rows(const DiaView &D, const int *off_s, const float *__restrict__ x, int r0,
                                         float (&u)[R]) {
    const float *val = (const float *)D.val + (size_t)(r0 >> 5) * ((size_t)D.ndiag * 32) + (r0 & 31);
#pragma unroll
    for (int q = 0; q < R; ++q) u[q] = 0.f;
    for (int d0 = 0; d0 < D.ndiag; d0 += 8) {
        float a[8][R], xv[8][R];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int d = d0 + t;
#pragma unroll
            for (int q = 0; q < R; ++q) a[t][q] = xv[t][q] = 0.f;
            if (d < D.ndiag) {
                VecR<R>::ld(val + d * 32, a[t]);
                const int o = off_s[d], c = r0 + o;
                if (o % R == 0 && c >= 0 && c + R - 1 < D.n) {
                    VecR<R>::ld(x + c, xv[t]);
                } else {
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        if (c + q >= 0 && c + q < D.n) xv[t][q] = __ldg(x + c + q);
                }
            }
        }
        const int cnt = D.ndiag - d0 < 8 ? D.ndiag - d0 : 8;
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (t < cnt)  // warp-uniform
#pragma unroll
                for (int q = 0; q < R; ++q) u[q] = fmaf(a[t][q], xv[t][q], u[q]);
    }
}

// The general pass (step_epilogue) on R rows.
template <int R>
__device__ __forceinline__ void step_epilogue_rows(int r0, float (&u)[R], const StepArgs &s) {
    float xi[R];
    VecR<R>::ld((const float *)s.x + r0, xi);
    if (s.has_sigma) {
#pragma unroll
        for (int q = 0; q < R; ++q) u[q] = u[q] - s.fsigma * xi[q];
    }
    if (s.plain) {
        VecR<R>::st((float *)s.y + r0, u);
        return;
    }
    float delta[R];
#pragma unroll
    for (int q = 0; q < R; ++q) delta[q] = s.fa1 * xi[q] + s.fa2 * u[q];
    if (s.y) {
        float base[R];
        if (s.aux) {
            VecR<R>::ld((const float *)s.aux + r0, base);
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) base[q] = xi[q];
        }
#pragma unroll
        for (int q = 0; q < R; ++q) base[q] = base[q] - delta[q];
        VecR<R>::st((float *)s.y + r0, base);
    }
    if (s.r) {
        float rv[R];
        if (s.r_init) {
#pragma unroll
            for (int q = 0; q < R; ++q) rv[q] = delta[q];
        } else {
            VecR<R>::ld((const float *)s.r + r0, rv);
#pragma unroll
            for (int q = 0; q < R; ++q) rv[q] = rv[q] + delta[q];
        }
        if (s.r_write) VecR<R>::st((float *)s.r + r0, rv);
        if (s.oy) {
            float ob[R], od[R];
            VecR<R>::ld((const float *)s.obase + r0, ob);
#pragma unroll
            for (int q = 0; q < R; ++q) od[q] = s.fb2 * rv[q];
            if (s.ox) {
                float ox[R];
                VecR<R>::ld((const float *)s.ox + r0, ox);
#pragma unroll
                for (int q = 0; q < R; ++q) od[q] += s.fb1 * ox[q];
            }
#pragma unroll
            for (int q = 0; q < R; ++q) ob[q] = ob[q] - od[q];
            VecR<R>::st((float *)s.oy + r0, ob);
        }
    }
}

// KIND as k_pass_dia (0 plain, 1 real root, 2 pair second pass); GENERAL: the
// running-sum pass (step_epilogue).  A last group of rows that runs past n
// takes the one-row code for each of its rows.
template <int R, int KIND, bool SIGMA, bool GENERAL>
__global__ void __launch_bounds__(256) k_dia_rows(DiaView D, StepArgs s) {
    grid_trigger();
    grid_wait();
    __shared__ int off_s[kDiaMax];
    for (int d = threadIdx.x; d < D.ndiag; d += blockDim.x) off_s[d] = D.off[d];
    __syncthreads();
    const int r0 = R * (blockIdx.x * blockDim.x + threadIdx.x);
    if (r0 >= D.n) return;
    const float *x = (const float *)s.x;
    if (r0 + R - 1 >= D.n) {  // ragged tail: one row at a time
        for (int row = r0; row < D.n; ++row) {
            float u = dia_row<float, float, float>(D, off_s, x, row);
            if (GENERAL) {
                step_epilogue<float, float>(row, u, s);
            } else {
                if (SIGMA) u = fmaf(-s.fsigma, x[row], u);
                float *y = (float *)s.y;
                if (KIND == 0)
                    y[row] = u;
                else if (KIND == 1)
                    y[row] = fmaf(-s.fa2, u, x[row]);
                else
                    y[row] = fmaf(-s.fa2, u, fmaf(-s.fa1, x[row], ((const float *)s.aux)[row]));
            }
        }
        return;
    }
    float u[R];
    dia_rows<R>(D, off_s, x, r0, u);
    if (GENERAL) {
        step_epilogue_rows<R>(r0, u, s);
        return;
    }
    float xi[R], out[R];
    VecR<R>::ld(x + r0, xi);
    if (SIGMA) {
#pragma unroll
        for (int q = 0; q < R; ++q) u[q] = fmaf(-s.fsigma, xi[q], u[q]);
    }
    if (KIND == 0) {
        VecR<R>::st((float *)s.y + r0, u);
    } else if (KIND == 1) {
#pragma unroll
        for (int q = 0; q < R; ++q) out[q] = fmaf(-s.fa2, u[q], xi[q]);
        VecR<R>::st((float *)s.y + r0, out);
    } else {
        float ax[R];
        VecR<R>::ld((const float *)s.aux + r0, ax);
#pragma unroll
        for (int q = 0; q < R; ++q) out[q] = fmaf(-s.fa2, u[q], fmaf(-s.fa1, xi[q], ax[q]));
        VecR<R>::st((float *)s.y + r0, out);
    }
}

template <typename T, typename V, typename Acc, int KIND, bool SIGMA, int FMT>
__global__ void __launch_bounds__(kPassMaxThreads) k_pass(SellView S, CsrView R, StepArgs s) {
    grid_trigger();
    grid_wait();
    const T *x = (const T *)s.x;
    T *y = (T *)s.y;
    auto finish = [&](int row, Acc u) {
        if (SIGMA) u = fma(-cf<Acc>(s.sigma, s.fsigma), (Acc)x[row], u);
        if (KIND == 0) {
            y[row] = (T)u;
        } else if (KIND == 1) {
            y[row] = (T)fma(-cf<Acc>(s.a2, s.fa2), u, (Acc)x[row]);
        } else {
            Acc v = fma(-cf<Acc>(s.a1, s.fa1), (Acc)x[row], (Acc)((const T *)s.aux)[row]);
            y[row] = (T)fma(-cf<Acc>(s.a2, s.fa2), u, v);
        }
    };
    if constexpr (FMT >= 5) {  // two rows per thread
        const int r0 = blockIdx.x * 2 * blockDim.x + threadIdx.x, r1 = r0 + blockDim.x;
        if (r0 >= S.n) return;
        Acc u0, u1;
        sell_row2<T, V, Acc, FMT == 6>(S, x, r0, r1, r1 < S.n, u0, u1);
        finish(r0, u0);
        if (r1 < S.n) finish(r1, u1);
    } else {
        const int row = blockIdx.x * blockDim.x + threadIdx.x;
        if (row >= (FMT == 0 ? R.n : S.n)) return;
        finish(row, row_sum<T, V, Acc, FMT>(S, R, x, row));
    }
}

// The fused pass with the slice data staged by the bulk-copy (TMA) engine.
// A tile is G = blockDim/32 consecutive SELL-32 slices (one warp per slice);
// its values and column indices are contiguous, so per tile one thread issues
// two bulk copies into a pipeline stage (with the tile's slice offsets in a
// small header) and arms the stage's mbarrier with their bytes.  Each block
// walks its tiles bid, bid + nblk, ... with up to `stages` tiles in flight;
// only the x gathers and the epilogue's row reads stay direct loads, so a
// row waits for one memory round trip instead of three (slice pointer,
// index, x).  A warp releases a stage through the stage's "empty" mbarrier;
// thread 0 refills it once all warps have.  Every wait is bounded: on expiry
// the thread records it in *err and leaves (the issuing thread first drains
// its copies), and the next host synchronisation reports PP_ETIMEOUT.  The
// row sums run in the entry order of the other formats, so the results are
// bit-identical to theirs.
constexpr int kTmaMaxSlices = kPassMaxThreads / 32;
constexpr int kTmaMaxStages = 4;
constexpr int kTmaHeader = 128;  // bytes: slice offsets of the tile (<= 17 ints)

template <typename T, typename I, int KIND, bool SIGMA>
__global__ void __launch_bounds__(kPassMaxThreads) k_pass_tma(SellView A, StepArgs s, int stages,
                                                              unsigned stage_bytes, unsigned idx_at, int *err) {
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ unsigned long long full[kTmaMaxStages], empty[kTmaMaxStages];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = blockDim.x >> 5;
    const int ntiles = (A.nslices + G - 1) / G;
    const int bid = blockIdx.x, nblk = gridDim.x;
    const int mine = bid < ntiles ? (ntiles - 1 - bid) / nblk + 1 : 0;
    const T *val = (const T *)A.val;
    const I *idx = (const I *)(sizeof(I) == 2 ? (const void *)A.off : (const void *)A.col);
    if (threadIdx.x == 0) {
        for (int q = 0; q < stages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], G);
        }
        mbar_fence_init();
    }
    __syncthreads();
    // thread 0: stage local tile k (its slice offsets, values and indices)
    auto issue = [&](int k) {
        const int st = k % stages;
        unsigned char *stage = tsm + (size_t)st * stage_bytes;
        const int s0 = (bid + k * nblk) * G, s1 = min(s0 + G, A.nslices);
        const int beg = __ldg(A.slice_ptr + s0), end = __ldg(A.slice_ptr + s1);
        int *hdr = (int *)stage;
        for (int q = 0; q <= s1 - s0; ++q) hdr[q] = __ldg(A.slice_ptr + s0 + q) - beg;
        const unsigned ne = (unsigned)(end - beg);
        mbar_arrive_expect(&full[st], ne * (unsigned)(sizeof(T) + sizeof(I)));
        if (ne) {
            bulk_copy_g2s(stage + kTmaHeader, val + beg, ne * (unsigned)sizeof(T), &full[st]);
            bulk_copy_g2s(stage + idx_at, idx + beg, ne * (unsigned)sizeof(I), &full[st]);
        }
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < stages && k < mine; ++k) issue(k);
    const T *x = (const T *)s.x;
    T *y = (T *)s.y;
    for (int k = 0; k < mine; ++k) {
        const int st = k % stages;
        const unsigned par = (unsigned)(k / stages) & 1u;
        if (!mbar_wait_bounded(&full[st], par)) {
            atomicExch(err, 1);
            if (threadIdx.x == 0)  // drain this block's copies still in flight
                for (int kk = k; kk < mine && kk < k + stages; ++kk)
                    mbar_wait_bounded(&full[kk % stages], (unsigned)(kk / stages) & 1u);
            return;
        }
        const unsigned char *stage = tsm + (size_t)st * stage_bytes;
        const int *hdr = (const int *)stage;
        const int s0 = (bid + k * nblk) * G;
        const int sl = s0 + warp;
        const int row = sl * 32 + lane;
        if (sl < A.nslices && row < A.n) {
            const int rb = hdr[warp], len = (hdr[warp + 1] - rb) >> 5;
            const T *vs = (const T *)(stage + kTmaHeader) + rb + lane;
            const I *is = (const I *)(stage + idx_at) + rb + lane;
            T u = 0;
            if (sizeof(I) == 2) {
                const T *xr = x + row;
#pragma unroll 4
                for (int q = 0; q < len; ++q) u = fma(vs[32 * q], __ldg(xr + (int)is[32 * q]), u);
            } else {
#pragma unroll 4
                for (int q = 0; q < len; ++q) u = fma(vs[32 * q], __ldg(x + (int)is[32 * q]), u);
            }
            if (SIGMA) u = fma(-cf<T>(s.sigma, s.fsigma), x[row], u);
            if (KIND == 0) {
                y[row] = u;
            } else if (KIND == 1) {
                y[row] = fma(-cf<T>(s.a2, s.fa2), u, x[row]);
            } else {
                T v = fma(-cf<T>(s.a1, s.fa1), x[row], ((const T *)s.aux)[row]);
                y[row] = fma(-cf<T>(s.a2, s.fa2), u, v);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        if (threadIdx.x == 0 && k + stages < mine) {
            // refill this stage once every warp has released it
            if (!mbar_wait_bounded(&empty[st], par)) {
                atomicExch(err, 1);
                for (int kk = k + 1; kk < mine && kk < k + stages; ++kk)
                    mbar_wait_bounded(&full[kk % stages], (unsigned)(kk / stages) & 1u);
                return;
            }
            issue(k + stages);
        }
    }
}

// General pass (running sum, optional output, outer epilogue): see StepArgs.
template <typename T, typename V, typename Acc, int FMT>
__global__ void __launch_bounds__(kPassMaxThreads) k_step(SellView S, CsrView R, StepArgs s) {
    grid_trigger();
    grid_wait();
    if constexpr (FMT >= 5) {  // two rows per thread
        const int r0 = blockIdx.x * 2 * blockDim.x + threadIdx.x, r1 = r0 + blockDim.x;
        if (r0 >= S.n) return;
        Acc u0, u1;
        sell_row2<T, V, Acc, FMT == 6>(S, (const T *)s.x, r0, r1, r1 < S.n, u0, u1);
        step_epilogue<T, Acc>(r0, u0, s);
        if (r1 < S.n) step_epilogue<T, Acc>(r1, u1, s);
    } else {
        int row = blockIdx.x * blockDim.x + threadIdx.x;
        if (row >= (FMT == 0 ? R.n : S.n)) return;
        Acc acc = row_sum<T, V, Acc, FMT>(S, R, (const T *)s.x, row);
        step_epilogue<T, Acc>(row, acc, s);
    }
}

// Two consecutive DIA rows r0, r0 + 1 (r0 even, both < n) of a batched
// instance in type T: each diagonal's two values and, for an even offset, the
// two x values are one 8- or 16-byte load; the offsets come through the cache.
// Products in increasing diagonal order per row, as dia_row.
template <typename T>
struct Pair2;
template <>
struct Pair2<float> {
    using V = float2;
};
template <>
struct Pair2<double> {
    using V = double2;
};
template <typename T>
__device__ __forceinline__ void ld2(const T *p, T (&o)[2]) {
    const typename Pair2<T>::V v = __ldg((const typename Pair2<T>::V *)p);
    o[0] = v.x;
    o[1] = v.y;
}
template <typename T>
__device__ __forceinline__ void st2(T *p, T a, T b) {
    typename Pair2<T>::V v;
    v.x = a;
    v.y = b;
    *(typename Pair2<T>::V *)p = v;
}

template <typename T>
__device__ __forceinline__ void dia_pair(const DiaView &D, const T *__restrict__ x, int r0, T (&u)[2]) {
    const T *val = (const T *)D.val + (size_t)(r0 >> 5) * ((size_t)D.ndiag * 32) + (r0 & 31);
    u[0] = u[1] = (T)0;
    for (int d0 = 0; d0 < D.ndiag; d0 += 8) {
        T a[8][2], xv[8][2];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int d = d0 + t;
            a[t][0] = a[t][1] = xv[t][0] = xv[t][1] = (T)0;
            if (d < D.ndiag) {
                ld2<T>(val + d * 32, a[t]);
                const int o = __ldg(D.off + d), c = r0 + o;
                if ((o & 1) == 0 && c >= 0 && c + 1 < D.n) {
                    ld2<T>(x + c, xv[t]);
                } else {
                    if (c >= 0 && c < D.n) xv[t][0] = __ldg(x + c);
                    if (c + 1 >= 0 && c + 1 < D.n) xv[t][1] = __ldg(x + c + 1);
                }
            }
        }
        const int cnt = D.ndiag - d0 < 8 ? D.ndiag - d0 : 8;
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (t < cnt) {
                u[0] = fma(a[t][0], xv[t][0], u[0]);
                u[1] = fma(a[t][1], xv[t][1], u[1]);
            }
    }
}

// Two consecutive DIA rows as dia_pair, for an instance with at most eight
// diagonals whose offsets the caller holds in registers: every load of the
// rows is issued at once (no offset load ahead of the x gathers).
template <typename T>
__device__ __forceinline__ void dia_pair8(const T *__restrict__ val, int n, int ndiag, const int (&off)[8],
                                          const T *__restrict__ x, int r0, T (&u)[2]) {
    T a[8][2], xv[8][2];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        a[t][0] = a[t][1] = xv[t][0] = xv[t][1] = (T)0;
        if (t < ndiag) {
            ld2<T>(val + t * 32, a[t]);
            const int c = r0 + off[t];
            if ((off[t] & 1) == 0 && c >= 0 && c + 1 < n) {
                ld2<T>(x + c, xv[t]);
            } else {
                if (c >= 0 && c < n) xv[t][0] = __ldg(x + c);
                if (c + 1 >= 0 && c + 1 < n) xv[t][1] = __ldg(x + c + 1);
            }
        }
    }
    u[0] = u[1] = (T)0;
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (t < ndiag) {
            u[0] = fma(a[t][0], xv[t][0], u[0]);
            u[1] = fma(a[t][1], xv[t][1], u[1]);
        }
}

// The operands of one instance's pass at step jj, resolved once per run of
// work items in that instance and then held in registers.
template <typename T>
struct BatchOperands {
    const T *x, *aux;
    T *y;
    T a1, a2, sg;
    int kind;  // -1: the instance takes no pass at this step
};

template <typename T>
__device__ __forceinline__ T *batch_buf(const BatchPassInst &I, int k, int jj) {
    switch (k) {
        case 0: return (T *)I.V + (size_t)jj * I.ldv;
        case 1: return (T *)I.W;
        case 2: return (T *)I.P0;
        case 3: return (T *)I.P1;
        default: return (T *)I.T;
    }
}

// y from u = (A - sigma I) x at one row (kind 0: u; 1: x - a2 u; 2: aux - a1 x - a2 u).
template <typename T>
__device__ __forceinline__ T batch_out(const BatchOperands<T> &o, T u, T xi, T ai) {
    if (o.sg != (T)0) u = fma(-o.sg, xi, u);
    if (o.kind == 0) return u;
    if (o.kind == 1) return fma(-o.a2, u, xi);
    return fma(-o.a2, u, fma(-o.a1, xi, ai));
}

// One polynomial pass for every active instance in one launch.  A work item
// is g warps' rows of one instance: 32 consecutive rows per warp (SELL, and
// DIA in FP64), or 64 with two consecutive rows per lane (DIA in FP32: the
// lane's two values of a diagonal sit side by side in its 32-row block, one
// 8-byte load).  Blocks take chunks of `chunk` (at
// most kBatchChunk) consecutive work items, strided over the grid.  Consecutive
// items mostly stay in one instance: its operands, and in FP32 for up to eight
// diagonal offsets, are loaded once and kept in registers, and the next
// item's index is read while this one computes.  The launcher shortens the
// chunks when there are few items, so that small sets still fill the GPU.
constexpr int kBatchChunk = 4;

template <typename T>
__global__ void __launch_bounds__(kPassMaxThreads) k_pass_batch(const BatchPassInst *pi, const BatchPassEntry *tab,
                                                                const int2 *items, int nitems, const int *lo,
                                                                const int *hi, int jj, int chunk) {
    grid_trigger();
    grid_wait();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cur = -1, dia = 0, n = 0, ndiag = 0;
    const T *val = nullptr;
    const int *offp = nullptr;
    int off[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) off[t] = 0;
    BatchOperands<T> o{};
    for (int c0 = blockIdx.x * chunk; c0 < nitems; c0 += gridDim.x * chunk) {
        const int c1 = min(nitems, c0 + chunk);
        int2 nxt = items[c0];
        for (int it = c0; it < c1; ++it) {
            const int2 itm = nxt;
            if (it + 1 < c1) nxt = items[it + 1];  // the next index is in flight during this item
            if (itm.x != cur) {
                cur = itm.x;
                const BatchPassInst &I = pi[cur];
                const BatchPassEntry e = tab[cur];
                o.kind = (e.kind < 0 || jj < lo[cur] || jj >= hi[cur]) ? -1 : e.kind;
                o.x = batch_buf<T>(I, e.src, jj);
                o.y = batch_buf<T>(I, e.dst, jj);
                o.aux = batch_buf<T>(I, e.aux, jj);
                o.a1 = cf<T>(e.a1, e.fa1);
                o.a2 = cf<T>(e.a2, e.fa2);
                o.sg = cf<T>(I.sigma, I.fsigma);
                dia = I.dia;
                n = dia ? I.D.n : I.A.n;
                ndiag = dia ? I.D.ndiag : 0;
                val = (const T *)I.D.val;
                offp = I.D.off;
                if (sizeof(T) == 4 && dia && ndiag <= 8) {
#pragma unroll
                    for (int t = 0; t < 8; ++t) off[t] = t < ndiag ? __ldg(offp + t) : 0;
                }
            }
            if (o.kind >= 0) {
                if (dia && sizeof(T) == 4) {
                    const int r0 = (itm.y + 2 * warp) * 32 + 2 * lane;
                    if (r0 + 1 < n) {
                        T u[2], xi[2], ax[2] = {(T)0, (T)0};
                        if (ndiag <= 8) {
                            dia_pair8<T>(val + (size_t)(r0 >> 5) * ((size_t)ndiag * 32) + (r0 & 31), n, ndiag, off, o.x,
                                         r0, u);
                        } else {
                            dia_pair<T>(DiaView{n, ndiag, 0, offp, val}, o.x, r0, u);
                        }
                        ld2<T>(o.x + r0, xi);
                        if (o.kind == 2) ld2<T>(o.aux + r0, ax);
                        st2<T>(o.y + r0, batch_out<T>(o, u[0], xi[0], ax[0]), batch_out<T>(o, u[1], xi[1], ax[1]));
                    } else if (r0 < n) {  // the last row of an odd n
                        const DiaView D{n, ndiag, 0, offp, val};
                        const T u = dia_row<T, T, T>(D, offp, o.x, r0);
                        o.y[r0] = batch_out<T>(o, u, o.x[r0], o.kind == 2 ? o.aux[r0] : (T)0);
                    }
                } else {  // one row per lane: SELL, and DIA in FP64 (bound by FP64 arithmetic, not loads)
                    const int row = (itm.y + warp) * 32 + lane;
                    if (row < n) {
                        T u;
                        if (dia) {
                            u = dia_row<T, T, T>(DiaView{n, ndiag, 0, offp, val}, offp, o.x, row);
                        } else {
                            const SellView &A = pi[cur].A;
                            u = A.off ? sell_row<T, T, T, true>(A, o.x, row) : sell_row<T, T, T, false>(A, o.x, row);
                        }
                        o.y[row] = batch_out<T>(o, u, o.x[row], o.kind == 2 ? o.aux[row] : (T)0);
                    }
                }
            }
        }
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
__global__ void k_dia_fill(int n, const int *rowptr, const int *col, const double *val, const int *off, int ndiag,
                           int64_t ld, V *dval) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    int k = rowptr[row];
    const int end = rowptr[row + 1];
    for (int d = 0; d < ndiag; ++d) {  // columns sorted: walk the row and the offsets together
        const int c = row + off[d];
        double v = 0.0;
        while (k < end && col[k] < c) ++k;
        if (k < end && col[k] == c) v = val[k];
        dval[(size_t)(row >> 5) * ((size_t)ndiag * 32) + (size_t)d * 32 + (row & 31)] = (V)v;
    }
}

template <typename V>
__global__ void k_convert_vals(int64_t nnz, const double *val, V *out) {
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * kThreads)
        out[i] = (V)val[i];
}

__global__ void k_bf16_to_f32(int n, const __nv_bfloat16 *x, float *y) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) y[i] = ld_f32(x + i);
}

__global__ void k_f32_to_bf16(int n, const float *x, __nv_bfloat16 *y) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) y[i] = __float2bfloat16_rn(x[i]);
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
    const int rows_per_block = FMT >= 5 ? 2 * threads : threads;
    const int blocks = (A.n + rows_per_block - 1) / rows_per_block;
    const bool general = s.r || s.oy || !s.y;
    const bool sig = s.sigma != 0.0;
    if (general || (!s.plain && !s.aux && s.a1 != 0.0)) {  // not one of the specialised forms
        launch_dependent(k_step<T, T, T, FMT>, blocks, threads, 0, st, A.sell, A.csr, s);
        return;
    }
    int kind = s.plain ? 0 : (s.aux ? 2 : 1);
#define PP_PASS(K, S) launch_dependent(k_pass<T, T, T, K, S, FMT>, blocks, threads, 0, st, A.sell, A.csr, s)
    if (kind == 0) {
        if (sig) PP_PASS(0, true); else PP_PASS(0, false);
    } else if (kind == 1) {
        if (sig) PP_PASS(1, true); else PP_PASS(1, false);
    } else {
        if (sig) PP_PASS(2, true); else PP_PASS(2, false);
    }
#undef PP_PASS
}

template <typename T, typename I, int KIND, bool SIGMA>
static void tma_pass_launch(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    static int attr = 0;  // one per instantiation
    if (!attr) {
        cudaFuncSetAttribute(k_pass_tma<T, I, KIND, SIGMA>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = 1;
    }
    const unsigned vbytes = (unsigned)(((size_t)A.tile_cap * sizeof(T) + 127) / 128 * 128);
    const unsigned ibytes = (unsigned)(((size_t)A.tile_cap * sizeof(I) + 127) / 128 * 128);
    const unsigned idx_at = kTmaHeader + vbytes, stage = idx_at + ibytes;
    int stages = (int)((64u * 1024u) / stage);
    stages = stages < 2 ? 2 : (stages > kTmaMaxStages ? kTmaMaxStages : stages);
    const size_t smem = (size_t)stages * stage;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass_tma<T, I, KIND, SIGMA>, A.threads, smem);
    if (per_sm < 1) per_sm = 1;
    const int G = A.threads / 32;
    const int ntiles = (A.sell.nslices + G - 1) / G;
    int grid = per_sm * num_sms();
    if (grid > ntiles) grid = ntiles;
    k_pass_tma<T, I, KIND, SIGMA><<<grid, A.threads, smem, st>>>(A.sell, s, stages, stage, idx_at, A.err);
}

template <typename T, typename I>
static bool tma_pass_dispatch(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    const bool general = s.r || s.oy || !s.y;
    if (general || (!s.plain && !s.aux && s.a1 != 0.0)) return false;
    const bool sig = s.sigma != 0.0;
    const int kind = s.plain ? 0 : (s.aux ? 2 : 1);
#define PP_TPASS(K, S) tma_pass_launch<T, I, K, S>(A, s, st)
    if (kind == 0) {
        if (sig) PP_TPASS(0, true); else PP_TPASS(0, false);
    } else if (kind == 1) {
        if (sig) PP_TPASS(1, true); else PP_TPASS(1, false);
    } else {
        if (sig) PP_TPASS(2, true); else PP_TPASS(2, false);
    }
#undef PP_TPASS
    return true;
}

// The R-rows-per-thread FP32 DIA kernels (R = 4 for row loop 1, R = 2 for row
// loop 2) when the tuner chose them and every vector the pass touches is
// 4R-byte aligned; false otherwise.
template <int R>
static bool dia_rows_launch(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    for (const void *p : {s.x, s.aux, (const void *)s.y, (const void *)s.r, s.obase, s.ox, (const void *)s.oy})
        if (p && ((uintptr_t)p & (uintptr_t)(4 * R - 1)) != 0) return false;
    const int threads = A.threads > 256 ? 256 : A.threads;
    const int groups = (A.n + R - 1) / R;
    const int blocks = (groups + threads - 1) / threads;
    const bool general = s.r || s.oy || !s.y;
    const bool sig = s.sigma != 0.0;
    if (general || (!s.plain && !s.aux && s.a1 != 0.0)) {
        launch_dependent(k_dia_rows<R, 0, false, true>, blocks, threads, 0, st, A.dia, s);
        return true;
    }
    const int kind = s.plain ? 0 : (s.aux ? 2 : 1);
#define PP_DR(K, S) launch_dependent(k_dia_rows<R, K, S, false>, blocks, threads, 0, st, A.dia, s)
    if (kind == 0) {
        if (sig) PP_DR(0, true); else PP_DR(0, false);
    } else if (kind == 1) {
        if (sig) PP_DR(1, true); else PP_DR(1, false);
    } else {
        if (sig) PP_DR(2, true); else PP_DR(2, false);
    }
#undef PP_DR
    return true;
}

static bool dia_rows_dispatch(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    if (A.prec != F32) return false;
    if (A.wide == 1) return dia_rows_launch<4>(A, s, st);
    if (A.wide == 2) return dia_rows_launch<2>(A, s, st);
    return false;
}

template <typename T>
static void dia_dispatch(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    if (dia_rows_dispatch(A, s, st)) return;
    const int threads = A.threads;
    const int blocks = (A.n + threads - 1) / threads;
    const bool general = s.r || s.oy || !s.y;
    const bool sig = s.sigma != 0.0;
    if (general || (!s.plain && !s.aux && s.a1 != 0.0)) {
        launch_dependent(k_step_dia<T, T, T>, blocks, threads, 0, st, A.dia, s);
        return;
    }
    const int kind = s.plain ? 0 : (s.aux ? 2 : 1);
#define PP_DPASS(K, S) launch_dependent(k_pass_dia<T, T, T, K, S>, blocks, threads, 0, st, A.dia, s)
    if (kind == 0) {
        if (sig) PP_DPASS(0, true); else PP_DPASS(0, false);
    } else if (kind == 1) {
        if (sig) PP_DPASS(1, true); else PP_DPASS(1, false);
    } else {
        if (sig) PP_DPASS(2, true); else PP_DPASS(2, false);
    }
#undef PP_DPASS
}

template <typename T>
static void pass_format(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    if (A.fmt == 3) {
        dia_dispatch<T>(A, s, st);
        return;
    }
    if (A.fmt == 2 && A.tma && A.err) {
        const bool done = A.sell.off ? tma_pass_dispatch<T, short>(A, s, st) : tma_pass_dispatch<T, int>(A, s, st);
        if (done) return;
    }
    if (A.fmt != 2)
        pass_dispatch<T, 0>(A, s, st);
    else if (A.sell.off)
        A.wide == 2 ? pass_dispatch<T, 6>(A, s, st)
                    : (A.wide ? pass_dispatch<T, 4>(A, s, st) : pass_dispatch<T, 2>(A, s, st));
    else
        A.wide == 2 ? pass_dispatch<T, 5>(A, s, st)
                    : (A.wide ? pass_dispatch<T, 3>(A, s, st) : pass_dispatch<T, 1>(A, s, st));
}

void launch_step(const Matrix &A, const StepArgs &s, cudaStream_t st) {
    StepArgs t = s;
    t.fa1 = (float)s.a1;
    t.fa2 = (float)s.a2;
    t.fb1 = (float)s.b1;
    t.fb2 = (float)s.b2;
    t.fsigma = (float)s.sigma;
    t.has_sigma = s.sigma != 0.0;
    if (A.prec == F64)
        pass_format<double>(A, t, st);
    else
        pass_format<float>(A, t, st);
}

void launch_pass_batch(Prec p, const BatchPassInst *pi, const BatchPassEntry *tab, const int2 *items, int nitems,
                       const int *lo, const int *hi, int jj, int groups, int grid_per_sm, cudaStream_t st) {
    int g = num_sms() * grid_per_sm;
    // chunks of up to kBatchChunk items, shorter where that leaves fewer than
    // four blocks per SM
    int chunk = nitems / (num_sms() * 4);
    chunk = chunk < 1 ? 1 : (chunk > kBatchChunk ? kBatchChunk : chunk);
    const int chunks = (nitems + chunk - 1) / chunk;
    if (chunks < g) g = chunks;
    if (g < 1) g = 1;
    const int threads = 32 * groups;
    if (p == F64)
        launch_dependent(k_pass_batch<double>, g, threads, 0, st, pi, tab, items, nitems, lo, hi, jj, chunk);
    else
        launch_dependent(k_pass_batch<float>, g, threads, 0, st, pi, tab, items, nitems, lo, hi, jj, chunk);
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

void launch_dia_fill(Prec p, int n, const int *rowptr, const int *col, const double *val, const int *off, int ndiag,
                     int64_t ld, void *dval, cudaStream_t st) {
    const int blocks = (n + kThreads - 1) / kThreads;
    if (p == F64)
        k_dia_fill<double><<<blocks, kThreads, 0, st>>>(n, rowptr, col, val, off, ndiag, ld, (double *)dval);
    else
        k_dia_fill<float><<<blocks, kThreads, 0, st>>>(n, rowptr, col, val, off, ndiag, ld, (float *)dval);
}

void launch_csr_convert(Prec p, int64_t nnz, const double *val, void *out, cudaStream_t st) {
    int g = num_sms() * 4;
    if (p == F32) k_convert_vals<float><<<g, kThreads, 0, st>>>(nnz, val, (float *)out);
}

void launch_convert(Prec from, Prec to, int n, const void *x, void *y, cudaStream_t st) {
    int g = num_sms() * 4;
    if (from == BF16 && to == F32)
        k_bf16_to_f32<<<g, kThreads, 0, st>>>(n, (const __nv_bfloat16 *)x, (float *)y);
    else if (from == F32 && to == BF16)
        k_f32_to_bf16<<<g, kThreads, 0, st>>>(n, (const float *)x, (__nv_bfloat16 *)y);
    else if (from == F64 && to == F32)
        k_convert<double, float><<<g, kThreads, 0, st>>>(n, (const double *)x, (float *)y);
    else if (from == F32 && to == F64)
        k_convert<float, double><<<g, kThreads, 0, st>>>(n, (const float *)x, (double *)y);
    else if (from == F64)
        k_convert<double, double><<<g, kThreads, 0, st>>>(n, (const double *)x, (double *)y);
    else
        k_convert<float, float><<<g, kThreads, 0, st>>>(n, (const float *)x, (float *)y);
}

}  // namespace ppk
