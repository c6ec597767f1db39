// Kernels of the orthogonalisation and the restart (sm_103a).
//
//  * k_cgs: the three passes of classical Gram-Schmidt with one
//    reorthogonalisation (Section 4), each a single sweep over the basis with
//    a deterministic two-level reduction finished by the last block;
//    k_cgs_tma stages the basis tiles in shared memory with the bulk-copy
//    engine; k_cgs_batch serves many instances in one launch.
//  * k_rotate: V_m Q_k for the thick restart and Ritz vectors (Section 4).
//  * k_coldots: Rayleigh quotients and residual norms on A (Section 4).
#include "device_common.cuh"
#include "pp_internal.h"

#include <cstdint>
#include <cstdlib>
#include <type_traits>

namespace ppk {

namespace {

template <typename T>
__device__ __forceinline__ double ld_acc(const T *p, size_t i) {
    return (double)__ldg(p + i);
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
    // Run by every thread of the last block while the other SMs wait, so the
    // loads are spread over the whole block and issued eight at a time: thread
    // t sums output t % nout over the blocks t / nout, t / nout + S, ... (S =
    // threads / nout slices), then thread o adds its output's S slice sums in
    // slice order.  The order is fixed, so every run gives the same bits.
    __shared__ double slice_sum[kThreads];
    const int nt = blockDim.x, t = threadIdx.x;
    if (nout > nt || nt > kThreads) {  // not taken by the sweeps here (nout <= j + 1 <= threads)
        for (int o = t; o < nout; o += nt) {
            double s = 0;
            for (int b = 0; b < nblocks; ++b) s += __ldcg(part + (size_t)b * nout + o);
            out[o] = s;
        }
        return;
    }
    const int S = nt / nout;
    double acc = 0;
    if (t < S * nout) {
        const int o = t % nout;
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0, a6 = 0, a7 = 0;
        int b = t / nout;
        for (; b + 7 * S < nblocks; b += 8 * S) {
            const double *p = part + (size_t)b * nout + o;
            const size_t st = (size_t)S * nout;
            a0 += __ldcg(p);
            a1 += __ldcg(p + st);
            a2 += __ldcg(p + 2 * st);
            a3 += __ldcg(p + 3 * st);
            a4 += __ldcg(p + 4 * st);
            a5 += __ldcg(p + 5 * st);
            a6 += __ldcg(p + 6 * st);
            a7 += __ldcg(p + 7 * st);
        }
        for (; b < nblocks; b += S) a0 += __ldcg(part + (size_t)b * nout + o);
        acc = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    }
    slice_sum[t] = acc;
    __syncthreads();
    if (t < nout) {
        double s = 0;
        for (int k = 0; k < S; ++k) s += slice_sum[k * nout + t];
        out[t] = s;
    }
}

// ---------------------------------------------------------------------------
// CGS2 passes. A tile is kRows consecutive rows; warp w owns basis columns
// c = w + 8 cc (cc < CPW).  Each lane holds kRows/32 rows of the tile.
// ---------------------------------------------------------------------------
constexpr int kRows = 64;
constexpr int kQ = kRows / 32;

// The grid reduction of a sweep once every block has written its `nout`
// partials part[bid * nout + o]: the last block of each group of 32 sums the
// group's partials (block order), the last group sums the group sums (group
// order) into a.out, and in mode 2 writes the Hessenberg column.
template <int NW>
__device__ __forceinline__ void cgs_reduce_tail(const CgsArgs &a, int bid, int nblk, int nout) {
    const int tid = threadIdx.x;
    const int j = a.j;
    const int ng = (nblk + 31) / 32, g = bid / 32;
    const int gsize = nblk - 32 * g < 32 ? nblk - 32 * g : 32;
    double *gpart = a.part + (size_t)nblk * nout;
    if (!last_block(a.ticket + 1 + g, gsize)) return;
    reduce_partials(a.part + (size_t)g * 32 * nout, gsize, nout, gpart + (size_t)g * nout);
    __syncthreads();
    if (tid == 0) a.ticket[1 + g] = 0;
    if (!last_block(a.ticket, ng)) return;
    reduce_partials(gpart, ng, nout, a.out);
    __syncthreads();
    if (tid == 0) *a.ticket = 0;
    if (a.mode == 2) {
        __threadfence_block();
        __syncthreads();
        double nn = sqrt(a.out[0]);
        for (int c = tid; c < j; c += NW * 32) a.hcol[c] = a.h1[c] + a.h[c];
        if (tid == 0) {
            a.hcol[j] = nn;
            a.scal[0] = nn > 0 ? 1.0 / nn : 0.0;
        }
    }
}

// Per-block partial sums of an FP64 sweep, then the grid reduction.  acc[cc]
// is the block-local projection on column warp + NW cc (NW warps per block);
// nrm the squared norm of the updated vector's rows.
template <int CPW, int NW = kWarps>
__device__ __forceinline__ void cgs_finish(const CgsArgs &a, int bid, int nblk, const double (&acc)[CPW],
                                           double nrm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int j = a.j;
    __shared__ double nrm_sh[NW];
    const int nout = (a.mode == 0) ? j : (a.mode == 1 ? j + 1 : 1);
    double *part = a.part + (size_t)bid * nout;
    if (a.mode != 2) {
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            double s = acc[cc];
#pragma unroll
            for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            int c = warp + NW * cc;
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
            for (int ww = 0; ww < NW; ++ww) s += nrm_sh[ww];
            part[a.mode == 1 ? j : 0] = s;
        }
    }
    cgs_reduce_tail<NW>(a, bid, nblk, nout);
}

// (h, l) += (bh, bl) for compensated FP32 sums: Knuth's TwoSum of the leading
// parts, the error added to the trailing parts.
__device__ __forceinline__ void pair_add(float &h, float &l, float bh, float bl) {
    const float t = __fadd_rn(h, bh);
    const float z = __fsub_rn(t, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(t, z)), __fsub_rn(bh, z));
    h = t;
    l = __fadd_rn(__fadd_rn(l, bl), e);
}

// The same for an FP32 sweep whose projections are compensated pairs (hi +
// lo): their warp sums stay compensated FP32 pairs (on this part an FP64
// instruction costs as much as a few dozen FP32 ones), lane 0 hands hi + lo
// to the FP64 partials; the squared norm nrm is FP64.
template <int CPW>
__device__ __forceinline__ void cgs_finish_f32(const CgsArgs &a, int bid, int nblk, float (&hi)[CPW],
                                               float (&lo)[CPW], double nrm) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int j = a.j;
    __shared__ double nrm_sh[kWarps];
    const int nout = (a.mode == 0) ? j : (a.mode == 1 ? j + 1 : 1);
    double *part = a.part + (size_t)bid * nout;
    if (a.mode != 2) {
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            float h = hi[cc], l = lo[cc];
#pragma unroll
            for (int off = 16; off; off >>= 1)
                pair_add(h, l, __shfl_xor_sync(0xffffffffu, h, off), __shfl_xor_sync(0xffffffffu, l, off));
            int c = warp + kWarps * cc;
            if (lane == 0 && c < j) part[c] = (double)h + (double)l;
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
    cgs_reduce_tail<kWarps>(a, bid, nblk, nout);
}

// The sweep of block `bid` out of `nblk` blocks working on an FP64 basis:
// FP64 throughout.  NW warps per block: warp w owns columns w + NW cc.  Four
// warps (the default for bases of up to 52 columns) keep the column slots
// within 3 of j and the cross-warp row sums at four terms; the FP64 pipe is
// the bound, and both cost FP64 instructions.
template <int CPW, int NW>
__device__ __forceinline__ void cgs_body_f64(const CgsArgs &a, int bid, int nblk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const double *V = (const double *)a.V;
    const double *w = (const double *)a.w;
    double *wout = (double *)a.wout;
    const int j = a.j, n = a.n;
    __shared__ double red[NW][kRows];
    __shared__ double wsh[kRows];
    __shared__ double hs[NW * CPW];
    if (a.mode != 0)
        for (int c = tid; c < j; c += NW * 32) hs[c] = a.h[c];
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
            int c = warp + NW * cc;
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
                if (warp + NW * cc < j)  // warp-uniform: no FMAs on columns past j
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
                int c = warp + NW * cc;
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
                for (int ww = 0; ww < NW; ++ww) s += red[ww][tid];
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
                if (warp + NW * cc < j)
#pragma unroll
                    for (int q = 0; q < kQ; ++q) acc[cc] = fma(vv[cc][q], wsh[lane + 32 * q], acc[cc]);
        }
    }
    cgs_finish<CPW, NW>(a, bid, nblk, acc, nrm);
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

// The sweep over an FP32 or BF16 basis (BF16 elements widened to FP32 on
// load; w is FP32).  The first projection h1 = V^T w and both updates w - V h
// run in FP32 (FP32 FMAs are many times faster than FP64 ones on this part);
// the reorthogonalising projection h2 = V^T w1 uses Dot2, so the second
// Gram-Schmidt pass is accurate to about twice FP32 precision; their warp
// sums are compensated FP32 pairs.  Squared norms accumulate in FP64.
template <typename TV, int CPW>
__device__ __forceinline__ void cgs_body_f32(const CgsArgs &a, int bid, int nblk) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const TV *V = (const TV *)a.V;
    const float *w = (const float *)a.w;
    float *wout = (float *)a.wout;  // FP32 always (a BF16 basis column is written by the scaling kernel)
    const int j = a.j, n = a.n;
    // 128-row tiles: four rows per lane and column, so each warp has twice the
    // loads of the FP64 sweep in flight (the FP32 sweeps are bound by memory
    // latency, not arithmetic)
    constexpr int RT = 2 * kRows, QT = RT / 32;
    __shared__ float red[kWarps][RT];
    __shared__ float wsh[RT];
    __shared__ float hs[8 * CPW];
    if (a.mode != 0)
        for (int c = tid; c < j; c += kThreads) hs[c] = (float)a.h[c];
    __syncthreads();
    float hi[CPW], lo[CPW];
#pragma unroll
    for (int cc = 0; cc < CPW; ++cc) hi[cc] = lo[cc] = 0.f;
    // the squared norm in FP64: the entries of pi(A) v_j can exceed sqrt of the
    // FP32 range (high-degree polynomials), where an FP32 square overflows
    double nrm = 0;
    const int ntiles = (n + RT - 1) / RT;
    for (int tile = bid; tile < ntiles; tile += nblk) {
        const int r0 = tile * RT;
        float vv[CPW][QT];
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
            int c = warp + kWarps * cc;
#pragma unroll
            for (int q = 0; q < QT; ++q) {
                int row = r0 + lane + 32 * q;
                vv[cc][q] = (c < j && row < n) ? ld_f32(V + (size_t)c * a.ldv + row) : 0.f;
            }
        }
        if (a.mode == 0) {
            float wv[QT];
#pragma unroll
            for (int q = 0; q < QT; ++q) {
                int row = r0 + lane + 32 * q;
                wv[q] = row < n ? __ldg(w + row) : 0.f;
            }
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc)
                if (warp + kWarps * cc < j)
#pragma unroll
                    for (int q = 0; q < QT; ++q) hi[cc] = fmaf(vv[cc][q], wv[q], hi[cc]);
            continue;
        }
#pragma unroll
        for (int q = 0; q < QT; ++q) {
            float s = 0;
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) {
                int c = warp + kWarps * cc;
                if (c < j) s = fmaf(vv[cc][q], hs[c], s);
            }
            red[warp][lane + 32 * q] = s;
        }
        __syncthreads();
        if (tid < RT) {
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
                    for (int q = 0; q < QT; ++q) dot2_term(vv[cc][q], wsh[lane + 32 * q], hi[cc], lo[cc]);
        }
    }
    cgs_finish_f32<CPW>(a, bid, nblk, hi, lo, nrm);
}

template <typename T, int CPW, int NW>
__device__ __forceinline__ void cgs_body(const CgsArgs &a, int bid, int nblk) {
    if constexpr (sizeof(T) == 8) {
        cgs_body_f64<CPW, NW>(a, bid, nblk);
    } else {
        static_assert(NW == kWarps, "FP32 and BF16 sweeps run eight warps per block");
        cgs_body_f32<T, CPW>(a, bid, nblk);
    }
}

template <typename T, int CPW, int NW>
__global__ void __launch_bounds__(NW * 32) k_cgs(CgsArgs a) {
    grid_trigger();
    grid_wait();
    cgs_body<T, CPW, NW>(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// CGS2 sweeps with the basis staged in shared memory by the bulk-copy (TMA)
// engine (FP32 bases).  A tile is RT = 256 consecutive rows (128 when the
// basis is too wide for two 256-row stages); block bid owns the full tiles
// bid, bid + nblk, ...  Warp 0 stages a tile with j + 1 bulk copies (the
// tile's segment of each basis column and of w) into a pipeline stage whose
// "full" mbarrier is armed with their bytes; warps release a stage through its
// "empty" mbarrier and warp 0 refills it, so up to `stages` tiles are in
// flight while the block computes on the oldest.  Work per tile:
//  mode 0   column-owned projections (warp w: columns w, w + 8, ...);
//  mode 1   row-owned update w1 = w - V h1 (one thread per row over all j
//           columns), one block barrier, then column-owned Dot2 projections
//           of w1 (double-buffered row vector, so one barrier per tile);
//  mode 2   row-owned update only.
// One vote per tile (a block barrier) makes a bounded wait that expired end
// the sweep in every thread together; the issuing warp then drains its copies
// (bounded), the block contributes zero partials so the grid reduction
// completes, and the host reports PP_ETIMEOUT.  A ragged last tile is read
// with plain loads.  The row sums run over the columns in a different order
// than the plain sweeps, so the two agree to rounding.
// ---------------------------------------------------------------------------
constexpr int kMaxStages = 8;
constexpr int kTmaRows = 256;

template <typename T, int CPW, int RT>
__global__ void __launch_bounds__(kThreads) k_cgs_tma(CgsArgs a, int stages, int *err) {
    using Acc = float;  // FP32 bases only
    extern __shared__ __align__(128) unsigned char tma_smem[];
    __shared__ unsigned long long full[kMaxStages], empty[kMaxStages];
    __shared__ Acc wsh[2][RT];
    __shared__ Acc hs[8 * CPW];
    __shared__ int stop;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int j = a.j, n = a.n, bid = blockIdx.x, nblk = gridDim.x;
    const size_t stage_elems = (size_t)(j + 1) * RT;  // basis columns, then w
    T *const stage0 = (T *)tma_smem;
    const int nfull = n / RT;
    const int mine = bid < nfull ? (nfull - 1 - bid) / nblk + 1 : 0;
    if (a.mode != 0)
        for (int c = tid; c < j; c += kThreads) hs[c] = (Acc)a.h[c];
    if (tid == 0) {
        for (int q = 0; q < stages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kWarps);
        }
        mbar_fence_init();
        stop = 0;
    }
    __syncthreads();
    const bool feed = !a.stall;  // the failure-path test withholds the copies
    int issued = 0;              // tiles issued (warp 0)
    auto issue = [&](int k) {   // warp 0
        const int q = k % stages;
        const size_t r0 = (size_t)(bid + (size_t)k * nblk) * RT;
        T *dst = stage0 + (size_t)q * stage_elems;
        if (lane == 0) mbar_arrive_expect(&full[q], (unsigned)(stage_elems * sizeof(T)));
        __syncwarp();
        for (int c = lane; c <= j; c += 32) {
            const T *src = c < j ? (const T *)a.V + (size_t)c * a.ldv + r0 : (const T *)a.w + r0;
            bulk_copy_g2s(dst + (size_t)c * RT, src, (unsigned)(RT * sizeof(T)), &full[q]);
        }
        issued = k + 1;
    };
    float hi[CPW], lo[CPW];
#pragma unroll
    for (int cc = 0; cc < CPW; ++cc) hi[cc] = lo[cc] = 0.f;
    double nrm = 0;
    // One tile of `rows` rows starting at r0: V(c, i), W(i) give its basis and w entries.
    auto tile = [&](int r0, int rows, int buf, auto V, auto W) {
        if (a.mode == 0) {
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) {
                const int c = warp + kWarps * cc;
                if (c < j)
                    for (int i = lane; i < rows; i += 32) hi[cc] = fmaf(V(c, i), W(i), hi[cc]);
            }
            return;
        }
        for (int i = tid; i < rows; i += kThreads) {  // row-owned update
            // eight interleaved partial sums (columns c mod 8), combined pairwise: the
            // rounding error of a sum over ~j/8 + 3 terms, as in the plain sweeps
            Acc p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int c = 0; c < j; ++c) p[c & 7] = fmaf(V(c, i), hs[c], p[c & 7]);
            const Acc s = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
            const Acc v = W(i) - s;
            ((float *)a.wout)[r0 + i] = v;
            nrm = fma((double)v, (double)v, nrm);
            wsh[buf][i] = v;
        }
        if (a.mode == 1) {
            __syncthreads();
#pragma unroll
            for (int cc = 0; cc < CPW; ++cc) {
                const int c = warp + kWarps * cc;
                if (c < j)
                    for (int i = lane; i < rows; i += 32) dot2_term(V(c, i), wsh[buf][i], hi[cc], lo[cc]);
            }
        }
    };
    if (warp == 0 && feed)
        for (int k = 0; k < stages && k < mine; ++k) issue(k);
    bool bad = false;
    int k = 0;
    for (; k < mine; ++k) {
        const int q = k % stages;
        const unsigned par = (unsigned)(k / stages) & 1u;
        const bool ok = mbar_wait_bounded(&full[q], par);
        if (__syncthreads_or(!ok || stop)) {
            bad = true;
            break;
        }
        const T *Vs = stage0 + (size_t)q * stage_elems;
        const T *Ws = Vs + (size_t)j * RT;
        // shared-memory stage: plain loads (the __ldg path is for global memory only)
        tile((bid + k * nblk) * RT, RT, k & 1, [&](int c, int i) { return (Acc)Vs[(size_t)c * RT + i]; },
             [&](int i) { return (Acc)Ws[i]; });
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[q]);
        if (warp == 0 && feed && k + stages < mine) {
            bool ok2 = true;
            if (lane == 0) ok2 = mbar_wait_bounded(&empty[q], par);  // every warp released the stage
            ok2 = __shfl_sync(0xffffffffu, ok2 ? 1 : 0, 0) != 0;
            if (ok2)
                issue(k + stages);
            else if (lane == 0)
                stop = 1;
        }
    }
    if (bad) {
        if (tid == 0) atomicExch(err, 1);
        if (warp == 0 && lane == 0)  // drain this block's copies still in flight (bounded)
            for (int kk = k; kk < issued; ++kk) mbar_wait_bounded(&full[kk % stages], (unsigned)(kk / stages) & 1u);
        __syncthreads();
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) hi[cc] = lo[cc] = 0.f;
        nrm = 0;
    } else if (n % RT != 0 && (nfull % nblk) == bid) {
        // ragged last tile: plain loads
        __syncthreads();  // wsh of the last full tile may still be read (mode 1)
        const int r0 = nfull * RT, rows = n - r0;
        const T *V = (const T *)a.V;
        const T *w = (const T *)a.w;
        tile(r0, rows, mine & 1, [&](int c, int i) { return ld_f32(V + (size_t)c * a.ldv + r0 + i); },
             [&](int i) { return ld_f32(w + r0 + i); });
    }
    double accd[CPW];
#pragma unroll
    for (int cc = 0; cc < CPW; ++cc) accd[cc] = (double)hi[cc] + (double)lo[cc];
    cgs_finish<CPW>(a, bid, nblk, accd, nrm);
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

template <typename T, int CPW, int NW>
__global__ void __launch_bounds__(NW * 32) k_cgs_batch(const BatchCgsInst *ci, int count, const int *lo,
                                                       const int *hi, int mode, int jj) {
    grid_trigger();
    grid_wait();
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
    cgs_body<T, CPW, NW>(a, blockIdx.x - I.blk0, I.nblk);
}

template <typename T>
__global__ void k_scale_batch(const BatchCgsInst *ci, int count, const int *lo, const int *hi, int jj) {
    grid_trigger();
    grid_wait();
    const int i = find_instance(ci, count, blockIdx.x);
    if (jj < lo[i] || jj >= hi[i]) return;
    const BatchCgsInst &I = ci[i];
    T *x = (T *)I.V + (size_t)(jj + 1) * I.ldv;
    const double s = *I.scal;
    for (int r = (blockIdx.x - I.blk0) * kThreads + threadIdx.x; r < I.n; r += I.nblk * kThreads)
        x[r] = (T)((double)x[r] * s);
}

template <typename T>
__global__ void k_scale(int n, T *x, const double *scal) {
    grid_trigger();
    grid_wait();
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
template <typename Acc, typename T>
__device__ __forceinline__ Acc load_acc(const T *p) {
    return (Acc)__ldg(p);
}
template <>
__device__ __forceinline__ float load_acc<float, __nv_bfloat16>(const __nv_bfloat16 *p) {
    return ld_f32(p);
}
template <>
__device__ __forceinline__ double load_acc<double, __nv_bfloat16>(const __nv_bfloat16 *p) {
    return (double)ld_f32(p);
}
template <typename TO, typename Acc>
__device__ __forceinline__ TO store_as(Acc v) {
    return (TO)v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 store_as<__nv_bfloat16, float>(float v) {
    return __float2bfloat16_rn(v);
}

// ||x||^2 of an FP64 vector into out[0]: per-block partials, summed in block
// order by the last block (the same bits on every run).
__global__ void __launch_bounds__(kThreads) k_norm2(int n, const double *x, double *part, unsigned *ticket,
                                                    double *out) {
    __shared__ double wsum[kWarps];
    double s = 0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) s = fma(x[i], x[i], s);
#pragma unroll
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0;
        for (int w = 0; w < kWarps; ++w) b += wsum[w];
        part[blockIdx.x] = b;
    }
    if (!last_block(ticket)) return;
    reduce_partials(part, gridDim.x, 1, out);
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0;
}

// dst = x / sqrt(nrm2[0]) in the basis precision; the FP64 product is rounded
// to FP32 first for FP32 and BF16 (as a host vector uploaded to FP32 storage).
template <typename T>
__global__ void k_unit_into(int n, const double *x, const double *nrm2, T *dst) {
    const double sc = 1.0 / sqrt(*nrm2);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = x[i] * sc;
        if constexpr (std::is_same<T, double>::value)
            dst[i] = v;
        else if constexpr (std::is_same<T, float>::value)
            dst[i] = (float)v;
        else
            dst[i] = __float2bfloat16_rn((float)v);
    }
}

// Y[:, c] = X[:, c] * d (or / d), c < cols: the diagonal similarity of balancing
// applied to (or removed from) a block of FP64 vectors, elementwise.
__global__ void k_scale_rows(int n, int cols, const double *X, int64_t ldx, double *Y, int64_t ldy, const double *d,
                             int divide) {
    const int64_t total = (int64_t)n * cols;
    for (int64_t t = blockIdx.x * (int64_t)kThreads + threadIdx.x; t < total; t += (int64_t)gridDim.x * kThreads) {
        const int64_t c = t / n, r = t - c * n;
        const double x = X[c * ldx + r], dr = __ldg(d + r);
        Y[c * ldy + r] = divide ? x / dr : x * dr;
    }
}

// dst = src * sgn / sqrt(nrm2[0] + nrm2[1]) (an output eigenvector scaled to
// unit real or complex norm).
__global__ void k_slot_scale(int n, const double *src, const double *nrm2, double sgn, double *dst) {
    const double sc = sgn / sqrt(nrm2[0] + nrm2[1]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i] * sc;
}

// A BF16 basis column: out = bf16(w * scal) (w is the FP32 orthogonalised vector).
__global__ void k_scale_bf16(int n, const float *w, const double *scal, __nv_bfloat16 *out) {
    const float sc = (float)*scal;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(w[i] * sc);
}

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
        for (int r = warp; r < m; r += kWarps) Vs[r * 32 + lane] = row < n ? load_acc<Acc>(V + (size_t)r * ldv + row) : (Acc)0;
        __syncthreads();
        for (int c = warp; c < kk; c += kWarps) {
            Acc acc = 0;
            const Acc *qc = Qs + (size_t)c * m;
            for (int r = 0; r < m; ++r) acc = fma(Vs[r * 32 + lane], qc[r], acc);
            if (row < n) out[(size_t)c * ldo + row] = store_as<TO>(acc);
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

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// The most blocks any CGS2 sweep launches (sizes the partial-sum buffers; at
// most 32 (kTicketWords - 1) blocks, so every group has a ticket word).
int cgs_grid(int n) {
    int tiles = (n + kRows - 1) / kRows;
    int g = num_sms() * 8;
    if (g > 32 * (kTicketWords - 1)) g = 32 * (kTicketWords - 1);
    return tiles < g ? tiles : g;
}

// Blocks of a CGS pass: one wave of resident blocks (at most 8 per SM, which
// bounds the partial-sum buffer at cgs_grid), never more than there are tiles.
template <typename T, int CPW, int NW>
static int resident_grid(int n, int cap) {
    static int per_sm = 0;  // one per instantiation
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cgs<T, CPW, NW>, NW * 32, 0);
        const int most = 8;
        if (per_sm < 1) per_sm = 1;
        if (per_sm > most) per_sm = most;
    }
    int g = per_sm * num_sms();
    if (cap > 0 && g > cap) g = cap;
    const int most_blocks = cgs_grid(n);  // also caps at the tile count
    return g < most_blocks ? g : most_blocks;
}

// TMA-staged sweeps are opt-in (PP_TMA_CGS in the environment): on the bases
// measured here (j <= 51, n up to 4e6) they ran no faster than the plain
// sweeps, and their different summation order moved the mixed-precision
// solves onto slower paths.  They need FP32 bases, 16-byte aligned column
// starts and w, a context's error word, and one full tile.  FP64 bases always
// take the plain sweeps (bound by FP64 arithmetic, which staging cannot relieve).
static bool tma_usable(const CgsArgs &a, size_t esz) {
    static const bool on = std::getenv("PP_TMA_CGS") != nullptr;
    return (on || a.stall) && esz == 4 && a.err && a.n >= kTmaRows && ((uintptr_t)a.V % 16) == 0 && ((uintptr_t)a.w % 16) == 0 &&
           (a.ldv * (int64_t)esz) % 16 == 0 && a.j >= 1 && a.j <= 128;
}

template <typename T, int CPW, int RT>
static void cgs_tma_launch_rt(const CgsArgs &a, int cap, cudaStream_t st) {
    static bool attr = false;  // one per instantiation
    if (!attr) {
        cudaFuncSetAttribute(k_cgs_tma<T, CPW, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr = true;
    }
    // up to four stages in 96 KB; as many blocks per SM as fit (measured faster than
    // one block per SM with a deeper pipeline: eight warps cannot keep the stages busy)
    const size_t stage = (size_t)(a.j + 1) * RT * sizeof(T);
    int stages = (int)(96 * 1024 / stage);
    stages = stages < 2 ? 2 : (stages > 4 ? 4 : stages);
    const size_t smem = stage * stages;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cgs_tma<T, CPW, RT>, kThreads, smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 4) per_sm = 4;
    const int tiles = (a.n + RT - 1) / RT;
    int g = per_sm * num_sms();
    if (cap > 0 && g > cap) g = cap;
    if (g > tiles) g = tiles;
    k_cgs_tma<T, CPW, RT><<<g, kThreads, smem, st>>>(a, stages, a.err);
}

// 256-row tiles while two stages fit in 200 KB, else 128-row tiles.
template <typename T, int CPW>
static void cgs_tma_launch(const CgsArgs &a, int cap, cudaStream_t st) {
    if ((size_t)(a.j + 1) * kTmaRows * sizeof(T) * 2 <= 200 * 1024)
        cgs_tma_launch_rt<T, CPW, kTmaRows>(a, cap, st);
    else
        cgs_tma_launch_rt<T, CPW, kTmaRows / 2>(a, cap, st);
}

// Calls f(std::integral_constant<int, C>) with C the smallest instantiated
// columns-per-warp count >= cpw.  Every count up to 8 (bases of up to 64
// columns) has its own instantiation: a warp's column slots past j are skipped
// by a warp-uniform test that the compiler may turn into predicated FMAs, which
// still occupy the FP64 pipe, so the slots are kept within 7 of j.
template <typename F>
static void with_cpw(int cpw, F &&f) {
    switch (cpw) {
        case 0:
        case 1: f(std::integral_constant<int, 1>{}); break;
        case 2: f(std::integral_constant<int, 2>{}); break;
        case 3: f(std::integral_constant<int, 3>{}); break;
        case 4: f(std::integral_constant<int, 4>{}); break;
        case 5: f(std::integral_constant<int, 5>{}); break;
        case 6: f(std::integral_constant<int, 6>{}); break;
        case 7: f(std::integral_constant<int, 7>{}); break;
        case 8: f(std::integral_constant<int, 8>{}); break;
        case 9:
        case 10:
        case 11:
        case 12: f(std::integral_constant<int, 12>{}); break;
        default: f(std::integral_constant<int, 16>{}); break;
    }
}

// f(std::integral_constant<int, C>) with C = max(cpw, 1) for cpw <= CMAX.
template <int CMAX, typename F>
static void with_cpw_exact(int cpw, F &&f) {
    if constexpr (CMAX > 1) {
        if (cpw < CMAX) {
            with_cpw_exact<CMAX - 1>(cpw, f);
            return;
        }
    }
    f(std::integral_constant<int, CMAX>{});
}

// FP64 bases of up to kCgs4Cols columns take the four-warp sweeps.
constexpr int kCgs4Cols = 52;

template <typename T>
static void cgs_dispatch(const CgsArgs &a, int cap, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (tma_usable(a, sizeof(T))) {
        int cpw = (a.j + kWarps - 1) / kWarps;
        if (cpw <= 2)
            cgs_tma_launch<T, 2>(a, cap, st);
        else if (cpw <= 4)
            cgs_tma_launch<T, 4>(a, cap, st);
        else if (cpw <= 8)
            cgs_tma_launch<T, 8>(a, cap, st);
        else
            cgs_tma_launch<T, 16>(a, cap, st);
        return;
        }
    }
    if constexpr (sizeof(T) == 8) {
        if (a.j <= kCgs4Cols) {
            with_cpw_exact<kCgs4Cols / 4>((a.j + 3) / 4, [&](auto C) {
                launch_dependent(k_cgs<T, C.value, 4>, resident_grid<T, C.value, 4>(a.n, cap), 128, 0, st, a);
            });
            return;
        }
    }
    with_cpw((a.j + kWarps - 1) / kWarps, [&](auto C) {
        launch_dependent(k_cgs<T, C.value, kWarps>, resident_grid<T, C.value, kWarps>(a.n, cap), kThreads, 0, st, a);
    });
}

void launch_cgs(Prec p, const CgsArgs &a, cudaStream_t st) {
    if (p == F64)
        cgs_dispatch<double>(a, 0, st);
    else if (p == F32)
        cgs_dispatch<float>(a, 0, st);
    else
        cgs_dispatch<__nv_bfloat16>(a, 0, st);
}

void launch_scale_bf16(int n, const float *w, const double *scal, void *out, cudaStream_t st) {
    k_scale_bf16<<<num_sms() * 4, kThreads, 0, st>>>(n, w, scal, (__nv_bfloat16 *)out);
}

void launch_cgs_batch(Prec p, const BatchCgsInst *ci, int count, int nblocks, const int *lo, const int *hi, int mode,
                      int jj, cudaStream_t st) {
    if (p == F64 && jj + 1 <= kCgs4Cols) {
        with_cpw_exact<kCgs4Cols / 4>((jj + 1 + 3) / 4, [&](auto C) {
            launch_dependent(k_cgs_batch<double, C.value, 4>, nblocks, 128, 0, st, ci, count, lo, hi, mode, jj);
        });
        return;
    }
    with_cpw((jj + 1 + kWarps - 1) / kWarps, [&](auto C) {
        if (p == F64)
            launch_dependent(k_cgs_batch<double, C.value, kWarps>, nblocks, kThreads, 0, st, ci, count, lo, hi, mode, jj);
        else
            launch_dependent(k_cgs_batch<float, C.value, kWarps>, nblocks, kThreads, 0, st, ci, count, lo, hi, mode, jj);
    });
}

void launch_scale_batch(Prec p, const BatchCgsInst *ci, int count, int nblocks, const int *lo, const int *hi, int jj,
                        cudaStream_t st) {
    if (p == F64)
        launch_dependent(k_scale_batch<double>, nblocks, kThreads, 0, st, ci, count, lo, hi, jj);
    else
        launch_dependent(k_scale_batch<float>, nblocks, kThreads, 0, st, ci, count, lo, hi, jj);
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
    else if (p == F32)
        cgs_dispatch<float>(a, grid_cap, st);
    else
        cgs_dispatch<__nv_bfloat16>(a, grid_cap, st);
}

void launch_norm2(int n, const double *x, double *part, unsigned *ticket, double *out, cudaStream_t st) {
    int g = (n + kThreads - 1) / kThreads;
    if (g > num_sms() * 4) g = num_sms() * 4;
    if (g < 1) g = 1;
    k_norm2<<<g, kThreads, 0, st>>>(n, x, part, ticket, out);
}

void launch_scale_rows(int n, int cols, const double *X, int64_t ldx, double *Y, int64_t ldy, const double *d,
                       bool divide, cudaStream_t st) {
    k_scale_rows<<<num_sms() * 4, kThreads, 0, st>>>(n, cols, X, ldx, Y, ldy, d, divide ? 1 : 0);
}

void launch_slot_scale(int n, const double *src, const double *nrm2, double sgn, double *dst, cudaStream_t st) {
    k_slot_scale<<<num_sms() * 4, kThreads, 0, st>>>(n, src, nrm2, sgn, dst);
}

void launch_unit_into(Prec p, int n, const double *x, const double *nrm2, void *dst, cudaStream_t st) {
    const int g = num_sms() * 4;
    if (p == F64)
        k_unit_into<double><<<g, kThreads, 0, st>>>(n, x, nrm2, (double *)dst);
    else if (p == F32)
        k_unit_into<float><<<g, kThreads, 0, st>>>(n, x, nrm2, (float *)dst);
    else
        k_unit_into<__nv_bfloat16><<<g, kThreads, 0, st>>>(n, x, nrm2, (__nv_bfloat16 *)dst);
}

void launch_scale(Prec p, int n, void *x, const double *scal, cudaStream_t st) {
    int g = num_sms() * 4;
    if (p == F64)
        launch_dependent(k_scale<double>, g, kThreads, 0, st, n, (double *)x, scal);
    else
        launch_dependent(k_scale<float>, g, kThreads, 0, st, n, (float *)x, scal);
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
    } else if (p == F32) {
        cudaFuncSetAttribute(k_rotate<float, float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_rotate<float, float, float><<<g, kThreads, smem, st>>>(n, (const float *)V, ldv, m, Q, kk, (float *)out,
                                                                 ldo);
    } else {
        using B = __nv_bfloat16;
        cudaFuncSetAttribute(k_rotate<B, B, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_rotate<B, B, float><<<g, kThreads, smem, st>>>(n, (const B *)V, ldv, m, Q, kk, (B *)out, ldo);
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
    } else if (p == F32) {
        cudaFuncSetAttribute(k_rotate<float, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_rotate<float, double, double><<<g, kThreads, smem, st>>>(n, (const float *)V, ldv, m, Q, kk, out, ldo);
    } else {
        using B = __nv_bfloat16;
        cudaFuncSetAttribute(k_rotate<B, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_rotate<B, double, double><<<g, kThreads, smem, st>>>(n, (const B *)V, ldv, m, Q, kk, out, ldo);
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

}  // namespace ppk
