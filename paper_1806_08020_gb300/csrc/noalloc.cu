// pp_orthogonalize_noalloc: the CGS2 step of pp_orthogonalize for callers
// that cannot allocate device memory.  Its scratch (per-block partial sums,
// the two coefficient vectors, the norm and the completion ticket of the
// grid reductions) lives in one file-scope __device__ array of fixed size
// instead of memory owned by a pp_ctx.
#include "pp_internal.h"

#include <cuda_runtime.h>

#include <mutex>

namespace {

constexpr int kMaxCols = 128;    // largest j accepted
constexpr int kMaxBlocks = 608;  // grid cap of the three passes (4 blocks x 152 SMs)
// block partials and the sums of groups of 32 blocks (two-level grid reduction)
constexpr size_t kPartDoubles = ((size_t)kMaxBlocks + (kMaxBlocks + 31) / 32) * (kMaxCols + 2);
constexpr size_t kH1 = kPartDoubles, kH2 = kH1 + 256, kScal = kH2 + 256, kNrm = kScal + 1, kTicket = kScal + 8;
constexpr size_t kScratchDoubles = kTicket + ppk::kTicketWords / 2;
// (608 + 19) x 130 + 552 doubles: about 656 KB, held by every GPU that loads the library until exit.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device
// and kept for the life of the process (a cudaDeviceReset after the first call
// would leave it stale; the header says so).
pp_status scratch_on_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "pp_orthogonalize_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return pp_fail(PP_EINVAL, "pp_orthogonalize_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess)
            return pp_fail(PP_ECUDA, "pp_orthogonalize_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_addr[dev] = (double *)p;
    }
    *out = g_addr[dev];
    return PP_OK;
}

}  // namespace

extern "C" pp_status pp_orthogonalize_noalloc(int64_t n, const double *V_dev, int64_t ldv, int j, double *w_dev,
                                              double *v_dev, double *h_dev, void *stream) {
    if (n < 1 || n >= ((int64_t)1 << 31) || ldv < n || !V_dev || !w_dev || !v_dev || !h_dev)
        return pp_fail(PP_EINVAL, "pp_orthogonalize_noalloc: bad arguments");
    if (j < 1 || j > kMaxCols)
        return pp_fail(PP_EINVAL, "pp_orthogonalize_noalloc: j = %d outside [1, %d] (the static scratch holds "
                                  "partial sums for at most %d basis columns)", j, kMaxCols, kMaxCols);
    double *base = nullptr;
    pp_status st = scratch_on_current_device(&base);
    if (st < 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *ticket = (unsigned *)(base + kTicket);
    // the reduction ticket must start at zero; an earlier call leaves it at zero
    // unless it was interrupted, so clear it every time
    cudaError_t e = cudaMemsetAsync(ticket, 0, ppk::kTicketWords * sizeof(unsigned), s);
    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "pp_orthogonalize_noalloc: %s", cudaGetErrorString(e));
    int grid = ppk::cgs_grid((int)n);
    if (grid > kMaxBlocks) grid = kMaxBlocks;
    ppk::CgsArgs a;
    a.n = (int)n;
    a.V = V_dev;
    a.ldv = ldv;
    a.j = j;
    a.part = base;
    a.ticket = ticket;
    a.mode = 0;  // h1 = V^T w
    a.w = w_dev;
    a.out = base + kH1;
    ppk::launch_cgs_grid(ppk::F64, a, grid, s);
    a.mode = 1;  // w1 = w - V h1 (in place), h2 = V^T w1
    a.h = base + kH1;
    a.wout = w_dev;
    a.out = base + kH2;
    ppk::launch_cgs_grid(ppk::F64, a, grid, s);
    a.mode = 2;  // v = w1 - V h2, h = h1 + h2, h[j] = ||v||, scal = 1/||v||
    a.h = base + kH2;
    a.h1 = base + kH1;
    a.wout = v_dev;
    a.out = base + kNrm;
    a.hcol = h_dev;
    a.scal = base + kScal;
    ppk::launch_cgs_grid(ppk::F64, a, grid, s);
    ppk::launch_scale(ppk::F64, (int)n, v_dev, base + kScal, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pp_fail(PP_ECUDA, "pp_orthogonalize_noalloc: launch: %s", cudaGetErrorString(e));
    return PP_OK;
}
