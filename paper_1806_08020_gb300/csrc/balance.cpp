// Balancing (pp_opts.balance): the diagonal similarity S = D^-1 A D that makes
// A symmetric, when one exists.  Not part of the paper's method: a problem
// transformation for strongly non-normal operators such as the central-
// difference convection-diffusion operators of Section 4, whose eigenvalue
// condition numbers grow like e^(beta/2) while those of S are 1.
//
// S symmetric means a_ij d_j / d_i = a_ji d_i / d_j for every off-diagonal
// pair, i.e. d_j / d_i = sqrt(a_ji / a_ij): a_ij and a_ji must be nonzero
// together and of one sign, and the ratios multiplied around every cycle of
// the graph must give 1.  log d is found by a breadth-first walk from the
// first row of each connected component (log d = 0 there); every pair is then
// checked.
#include "pp_internal.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

namespace ppd {

namespace {

// Rows of A (or of its transpose) with sorted columns and duplicates summed.
struct SortedRows {
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
};

SortedRows sorted_rows(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals, bool transpose) {
    SortedRows r;
    std::vector<std::pair<int32_t, double>> ent;
    if (!transpose) {
        r.ptr.assign(n + 1, 0);
        for (int64_t i = 0; i < n; ++i) {
            ent.clear();
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) ent.emplace_back(colind[k], vals[k]);
            std::sort(ent.begin(), ent.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
            for (size_t q = 0; q < ent.size(); ++q) {
                if (!r.col.empty() && (int64_t)r.col.size() > r.ptr[i] && r.col.back() == ent[q].first)
                    r.val.back() += ent[q].second;
                else {
                    r.col.push_back(ent[q].first);
                    r.val.push_back(ent[q].second);
                }
            }
            r.ptr[i + 1] = (int64_t)r.col.size();
        }
        return r;
    }
    // transpose by counting, then the same sort and merge per row
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t k = 0; k < rowptr[n]; ++k) cnt[colind[k] + 1]++;
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> tcol(rowptr[n]);
    std::vector<double> tval(rowptr[n]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int64_t dst = fill[colind[k]]++;
            tcol[dst] = (int32_t)i;
            tval[dst] = vals[k];
        }
    return sorted_rows(n, cnt.data(), tcol.data(), tval.data(), false);
}

}  // namespace

bool symmetrizing_scale(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals,
                        std::vector<double> &logd, std::string &why, double max_log_range) {
    const SortedRows R = sorted_rows(n, rowptr, colind, vals, false);
    const SortedRows T = sorted_rows(n, rowptr, colind, vals, true);  // row i of T: column i of A
    logd.assign(n, 0.0);
    std::vector<char> seen(n, 0);
    std::vector<int64_t> queue;
    queue.reserve(n);
    char buf[160];
    // a_ij (row i of R) against a_ji (row i of T) for every j != i, zeros treated as absent
    auto walk_pairs = [&](int64_t i, auto &&visit) -> bool {
        int64_t p = R.ptr[i], q = T.ptr[i];
        const int64_t pe = R.ptr[i + 1], qe = T.ptr[i + 1];
        while (p < pe || q < qe) {
            int32_t jr = p < pe ? R.col[p] : INT32_MAX, jt = q < qe ? T.col[q] : INT32_MAX;
            const int32_t j = std::min(jr, jt);
            const double aij = (jr == j) ? R.val[p] : 0.0, aji = (jt == j) ? T.val[q] : 0.0;
            if (jr == j) ++p;
            if (jt == j) ++q;
            if (j == i || (aij == 0.0 && aji == 0.0)) continue;
            if (aij == 0.0 || aji == 0.0 || (aij > 0) != (aji > 0)) {
                std::snprintf(buf, sizeof buf, "entries (%lld,%d) and (%d,%lld) are not nonzero with one sign",
                              (long long)i, j, j, (long long)i);
                why = buf;
                return false;
            }
            if (!visit(j, aij, aji)) return false;
        }
        return true;
    };
    for (int64_t root = 0; root < n; ++root) {
        if (seen[root]) continue;
        seen[root] = 1;
        queue.clear();
        queue.push_back(root);
        for (size_t h = 0; h < queue.size(); ++h) {
            const int64_t i = queue[h];
            const bool ok = walk_pairs(i, [&](int32_t j, double aij, double aji) {
                if (!seen[j]) {
                    logd[j] = logd[i] + 0.5 * (std::log(std::fabs(aji)) - std::log(std::fabs(aij)));
                    seen[j] = 1;
                    queue.push_back(j);
                }
                return true;
            });
            if (!ok) return false;
        }
    }
    const double lo = *std::min_element(logd.begin(), logd.end()), hi = *std::max_element(logd.begin(), logd.end());
    if (hi - lo > max_log_range) {
        std::snprintf(buf, sizeof buf, "the scaling spans e^%.0f, beyond e^%.0f", hi - lo, max_log_range);
        why = buf;
        return false;
    }
    for (double &l : logd) l -= hi;
    // every pair symmetric in S: a_ij e^(l_j - l_i) = a_ji e^(l_i - l_j)
    double smax = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = R.ptr[i]; p < R.ptr[i + 1]; ++p)
            smax = std::max(smax, std::fabs(R.val[p] * std::exp(logd[R.col[p]] - logd[i])));
    for (int64_t i = 0; i < n; ++i) {
        const bool ok = walk_pairs(i, [&](int32_t j, double aij, double aji) {
            const double sij = aij * std::exp(logd[j] - logd[i]), sji = aji * std::exp(logd[i] - logd[j]);
            if (std::fabs(sij - sji) > 1e-12 * smax) {
                std::snprintf(buf, sizeof buf, "no diagonal similarity makes A symmetric (cycle through row %lld)",
                              (long long)i);
                why = buf;
                return false;
            }
            return true;
        });
        if (!ok) return false;
    }
    return true;
}

}  // namespace ppd
