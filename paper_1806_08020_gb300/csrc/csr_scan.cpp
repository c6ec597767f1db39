// Host analysis of a CSR matrix for pp_create, in parallel over row ranges:
// validation, ||A||_1 (the largest column sum of |a_ij|), the Gershgorin
// bound min_i (a_ii - sum_{j != i} |a_ij|) of the shift, whether 16-bit
// column offsets fit, and the diagonals of a DIA layout.  Not part of the
// method; the work a single core would spend on a 10^6-row matrix (~25 ms)
// sits inside every end-to-end solve.
//
// The rows are split into a fixed number of ranges of about equal entry
// counts (independent of the machine's cores), so the column sums, summed
// within a range in row order and then over the ranges in order, are the
// same on every machine.
#include "pp_internal.h"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <thread>

namespace ppd {

namespace {

constexpr int kParts = 16;

// fn(p) for p = 0..parts-1 on up to `parts` threads (the caller's included).
template <typename F>
void for_parts(int parts, F &&fn) {
    if (parts == 1) {
        fn(0);
        return;
    }
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int T = (int)std::min<unsigned>(hw, (unsigned)parts);
    std::atomic<int> next{0};
    auto worker = [&] {
        for (int p = next++; p < parts; p = next++) fn(p);
    };
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t) th.emplace_back(worker);
    worker();
    for (auto &x : th) x.join();
}

// A barrier for the threads of one team (spinning with yields: the phases it
// separates last a millisecond or less).
class SpinBarrier {
  public:
    explicit SpinBarrier(int n) : n_(n) {}
    void wait() {
        if (n_ == 1) return;
        const int g = gen_.load(std::memory_order_acquire);
        if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
            count_.store(0, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_release);
        } else {
            while (gen_.load(std::memory_order_acquire) == g) std::this_thread::yield();
        }
    }

  private:
    const int n_;
    std::atomic<int> count_{0};
    std::atomic<int> gen_{0};
};

// fn(t, T, barrier) on T = min(cores, parts) threads (the caller's included).
template <typename F>
void run_team(int parts, F &&fn) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int T = (int)std::min<unsigned>(hw, (unsigned)std::max(1, parts));
    SpinBarrier bar(T);
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t) th.emplace_back([&, t] { fn(t, T, bar); });
    fn(0, T, bar);
    for (auto &x : th) x.join();
}

// How many row ranges: kParts, or one for small matrices (threads would cost
// more than they save).
int row_split(int64_t n, const int64_t *rowptr) {
    return rowptr[n] < ((int64_t)1 << 18) ? 1 : (int)std::min<int64_t>(kParts, n);
}

// Row boundaries of `parts` ranges with about nnz / parts entries each.
std::vector<int64_t> row_parts(int64_t n, const int64_t *rowptr, int parts) {
    std::vector<int64_t> b(parts + 1, n);
    b[0] = 0;
    const int64_t nnz = rowptr[n];
    for (int p = 1; p < parts; ++p) {
        const int64_t target = nnz / parts * p + std::min<int64_t>(p, nnz % parts);
        b[p] = std::lower_bound(rowptr, rowptr + n, target) - rowptr;
        b[p] = std::max(b[p], b[p - 1]);
    }
    return b;
}

}  // namespace

bool scan_csr(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals, CsrScan &out,
              std::string &why) {
    char buf[160];
    const int parts = row_split(n, rowptr);
    struct Part {
        int64_t bad = INT64_MAX;  // first invalid entry
        double gl = INFINITY;
        bool fits16 = true;
        int32_t cmin = INT32_MAX, cmax = -1;
        std::vector<double> cs;  // column sums over [cmin, cmax]
    };
    std::vector<Part> P(parts);
    std::vector<int64_t> first(parts, INT64_MAX);  // first non-monotone row per range
    std::vector<int64_t> rb;
    std::vector<double> bmax(parts, 0.0);
    int stop = 0;  // 1: row pointers, 2: an entry, 3: scattered columns (set by thread 0)
    // One team of threads through all phases, a barrier between them (starting
    // threads for each phase cost more than the work); thread t takes ranges
    // t, t + T, ...
    run_team(parts, [&](int t, int T, SpinBarrier &bar) {
        // row pointers first: monotone and ending at nnz, every row stays inside the arrays
        const int64_t ev = (n + parts - 1) / parts;
        for (int p = t; p < parts; p += T)
            for (int64_t i = p * ev, e = std::min(n, (p + 1) * ev); i < e; ++i)
                if (rowptr[i + 1] < rowptr[i]) {
                    first[p] = i;
                    break;
                }
        bar.wait();
        if (t == 0) {
            for (int64_t i : first)
                if (i != INT64_MAX) stop = 1;
            if (!stop) rb = row_parts(n, rowptr, parts);
        }
        bar.wait();
        if (stop) return;
        // pass 1: validation, Gershgorin bound, offsets, column span (each range's
        // results in locals, stored once: the Part records share cache lines)
        for (int p = t; p < parts; p += T) {
            double gl = INFINITY;
            bool fits16 = true, bad = false;
            int32_t cmin = INT32_MAX, cmax = -1;
            for (int64_t i = rb[p]; i < rb[p + 1] && !bad; ++i) {
                double diag = 0, off = 0;
                for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                    const int64_t col = colind[k];
                    const double v = vals[k];
                    if (col < 0 || col >= n || !std::isfinite(v)) {
                        P[p].bad = k;
                        bad = true;
                        break;
                    }
                    if (col == i)
                        diag += v;
                    else
                        off += std::fabs(v);
                    fits16 = fits16 && std::llabs((long long)(col - i)) <= 32767;
                    cmin = std::min(cmin, (int32_t)col);
                    cmax = std::max(cmax, (int32_t)col);
                }
                gl = std::min(gl, diag - off);
            }
            P[p].gl = gl;
            P[p].fits16 = fits16;
            P[p].cmin = cmin;
            P[p].cmax = cmax;
        }
        bar.wait();
        if (t == 0) {
            int64_t span = 0;
            for (const Part &q : P) {
                if (q.bad != INT64_MAX) stop = 2;
                if (q.cmax >= q.cmin) span += (int64_t)q.cmax - q.cmin + 1;
            }
            // banded and stencil matrices: about n + parts x band column sums in all
            if (!stop && span > 4 * n + 64) stop = 3;
        }
        bar.wait();
        if (stop) return;
        // pass 2: column sums per range over its span, then over the ranges in
        // order, and their largest value per block of columns
        for (int p = t; p < parts; p += T) {
            Part &q = P[p];
            if (q.cmax < q.cmin) continue;
            std::vector<double> cs((size_t)(q.cmax - q.cmin + 1), 0.0);
            double *a = cs.data() - q.cmin;
            for (int64_t k = rowptr[rb[p]]; k < rowptr[rb[p + 1]]; ++k) a[colind[k]] += std::fabs(vals[k]);
            q.cs.swap(cs);
        }
        bar.wait();
        const int64_t cb = (n + parts - 1) / parts;
        for (int b = t; b < parts; b += T) {
            const int64_t c0 = b * cb, c1 = std::min(n, c0 + cb);
            std::vector<double> sum((size_t)std::max<int64_t>(0, c1 - c0), 0.0);
            for (const Part &q : P) {  // the ranges in order
                const int64_t lo = std::max<int64_t>(c0, q.cmin), hi = std::min<int64_t>(c1, (int64_t)q.cmax + 1);
                for (int64_t c = lo; c < hi; ++c) sum[c - c0] += q.cs[c - q.cmin];
            }
            double mx = 0.0;
            for (double v : sum) mx = std::max(mx, v);
            bmax[b] = mx;
        }
    });
    if (stop == 1) {
        for (int64_t i : first)
            if (i != INT64_MAX) {
                std::snprintf(buf, sizeof buf, "rowptr not monotone at %lld", (long long)i);
                break;
            }
        why = buf;
        return false;
    }
    if (stop == 2) {
        int64_t bad = INT64_MAX;
        for (const Part &q : P) bad = std::min(bad, q.bad);
        std::snprintf(buf, sizeof buf, "bad entry %lld", (long long)bad);
        why = buf;
        return false;
    }
    out.gl = INFINITY;
    out.fits16 = true;
    for (const Part &q : P) {
        out.gl = std::min(out.gl, q.gl);
        out.fits16 = out.fits16 && q.fits16;
    }
    out.norm1 = 0.0;
    if (stop == 3) {  // scattered columns: one pass in row order
        std::vector<double> colsum(n, 0.0);
        for (int64_t k = 0; k < rowptr[n]; ++k) colsum[colind[k]] += std::fabs(vals[k]);
        out.norm1 = *std::max_element(colsum.begin(), colsum.end());
    } else {
        for (double v : bmax) out.norm1 = std::max(out.norm1, v);
    }
    return true;
}

bool dia_offsets(int64_t n, const int64_t *rowptr, const int32_t *colind, int max_diags, std::vector<int> &off) {
    const int parts = row_split(n, rowptr);
    const std::vector<int64_t> rb = row_parts(n, rowptr, parts);
    std::vector<std::vector<int>> seen(parts);
    std::vector<char> ok(parts, 1);
    for_parts(parts, [&](int p) {
        std::vector<int> &s = seen[p];
        std::vector<int> prev;  // the previous row's offsets: stencil rows repeat them
        for (int64_t i = rb[p]; i < rb[p + 1]; ++i) {
            const int64_t k0 = rowptr[i], len = rowptr[i + 1] - k0;
            bool same = (int64_t)prev.size() == len;
            for (int64_t t = 0; t < len; ++t) {
                const int64_t k = k0 + t;
                if (t > 0 && colind[k] <= colind[k - 1]) {
                    ok[p] = 0;
                    return;
                }
                same = same && prev[t] == (int)(colind[k] - i);
            }
            if (same) continue;
            prev.resize(len);
            for (int64_t t = 0; t < len; ++t) {
                prev[t] = (int)(colind[k0 + t] - i);
                auto it = std::lower_bound(s.begin(), s.end(), prev[t]);
                if (it == s.end() || *it != prev[t]) s.insert(it, prev[t]);
            }
            if ((int)s.size() > max_diags) {
                ok[p] = 0;
                return;
            }
        }
    });
    std::vector<int> all;
    for (int p = 0; p < parts; ++p) {
        if (!ok[p]) return false;
        all.insert(all.end(), seen[p].begin(), seen[p].end());
    }
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    if ((int)all.size() > max_diags) return false;
    off = all;
    return true;
}

}  // namespace ppd
