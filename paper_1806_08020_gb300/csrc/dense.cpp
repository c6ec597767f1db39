// Host FP64 small dense linear algebra for the polynomial preconditioned
// Arnoldi method: the d x d and m x m steps of the Section 2 box and the
// thick restart of Section 4 run here, once per polynomial build or cycle.
//
//  * real nonsymmetric eigenproblem: Householder reduction to upper
//    Hessenberg form, Francis implicit double-shift QR to real Schur form
//    (2 x 2 diagonal blocks for conjugate pairs), eigenvectors by back
//    substitution on the quasi-triangular factor;
//  * LU with partial pivoting (harmonic Ritz values, Section 2 box 1(b));
//  * Householder QR with explicit thin Q (thick-restart basis, Section 4);
//  * modified Leja order (Section 2 box 1(c)) and pof / added roots (Section 7).
#include "pp_internal.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

namespace ppd {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------
// Householder reduction to upper Hessenberg form: A = Z H Z^T.
// a: n x n column-major (ld n), overwritten by H; z: n x n, receives Z.
// ---------------------------------------------------------------------------
static void hessenberg(int n, double *a, double *z) {
    auto A = [&](int i, int j) -> double & { return a[i + (size_t)j * n]; };
    auto Z = [&](int i, int j) -> double & { return z[i + (size_t)j * n]; };
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) Z(i, j) = (i == j) ? 1.0 : 0.0;
    std::vector<double> v(n);
    for (int k = 0; k + 2 < n; ++k) {
        // reflector that zeroes A(k+2:n, k)
        double scale = 0;
        for (int i = k + 1; i < n; ++i) scale = std::max(scale, std::fabs(A(i, k)));
        if (scale == 0) continue;
        double ss = 0;
        for (int i = k + 1; i < n; ++i) {
            v[i] = A(i, k) / scale;
            ss += v[i] * v[i];
        }
        double alpha = std::sqrt(ss);
        if (v[k + 1] > 0) alpha = -alpha;  // x - alpha e1 without cancellation
        v[k + 1] -= alpha;
        double vv = 0;
        for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
        if (vv == 0) continue;
        double tau = 2.0 / vv;
        // H <- P H  (rows k+1..n-1, all columns from k)
        for (int j = k; j < n; ++j) {
            double s = 0;
            for (int i = k + 1; i < n; ++i) s += v[i] * A(i, j);
            s *= tau;
            for (int i = k + 1; i < n; ++i) A(i, j) -= s * v[i];
        }
        // H <- H P  (all rows, columns k+1..n-1)
        for (int i = 0; i < n; ++i) {
            double s = 0;
            for (int j = k + 1; j < n; ++j) s += A(i, j) * v[j];
            s *= tau;
            for (int j = k + 1; j < n; ++j) A(i, j) -= s * v[j];
        }
        // Z <- Z P
        for (int i = 0; i < n; ++i) {
            double s = 0;
            for (int j = k + 1; j < n; ++j) s += Z(i, j) * v[j];
            s *= tau;
            for (int j = k + 1; j < n; ++j) Z(i, j) -= s * v[j];
        }
        A(k + 1, k) = alpha * scale;
        for (int i = k + 2; i < n; ++i) A(i, k) = 0.0;
    }
}

// Apply the 3-element reflector (I - tau v v^T), v = (1, v1, v2), to rows
// r..r+2 (columns c0..c1) from the left, or to columns r..r+2 (rows c0..c1)
// from the right.
static inline void refl3_left(int n, double *h, int r, int c0, int c1, double tau, double v1,
                              double v2) {
    for (int j = c0; j <= c1; ++j) {
        double *col = h + (size_t)j * n;
        double s = tau * (col[r] + v1 * col[r + 1] + v2 * col[r + 2]);
        col[r] -= s;
        col[r + 1] -= s * v1;
        col[r + 2] -= s * v2;
    }
}
static inline void refl3_right(int n, double *h, int c, int r0, int r1, double tau, double v1,
                               double v2) {
    double *c0 = h + (size_t)c * n, *c1 = c0 + n, *c2 = c1 + n;
    for (int i = r0; i <= r1; ++i) {
        double s = tau * (c0[i] + v1 * c1[i] + v2 * c2[i]);
        c0[i] -= s;
        c1[i] -= s * v1;
        c2[i] -= s * v2;
    }
}
static inline void refl2_left(int n, double *h, int r, int c0, int c1, double tau, double v1) {
    for (int j = c0; j <= c1; ++j) {
        double *col = h + (size_t)j * n;
        double s = tau * (col[r] + v1 * col[r + 1]);
        col[r] -= s;
        col[r + 1] -= s * v1;
    }
}
static inline void refl2_right(int n, double *h, int c, int r0, int r1, double tau, double v1) {
    double *c0 = h + (size_t)c * n, *c1 = c0 + n;
    for (int i = r0; i <= r1; ++i) {
        double s = tau * (c0[i] + v1 * c1[i]);
        c0[i] -= s;
        c1[i] -= s * v1;
    }
}

// Reflector P = I - tau v v^T, v = (1, v1[, v2]) with P x = beta e1.
static inline bool make_reflector(double x, double y, double z, double &tau, double &v1,
                                  double &v2, double &beta) {
    double nrm = std::sqrt(x * x + y * y + z * z);
    if (nrm == 0.0) {
        tau = 0;
        v1 = v2 = 0;
        beta = 0;
        return false;
    }
    beta = (x > 0) ? -nrm : nrm;
    double d = x - beta;
    tau = -d / beta;  // (beta - x)/beta
    v1 = y / d;
    v2 = z / d;
    return true;
}

// Rotation [c -s; s c] applied as G^T (rows p, p+1) and G (cols p, p+1).
static void rot_rows(int n, double *h, int p, int c0, int c1, double c, double s) {
    for (int j = c0; j <= c1; ++j) {
        double *col = h + (size_t)j * n;
        double a = col[p], b = col[p + 1];
        col[p] = c * a + s * b;
        col[p + 1] = -s * a + c * b;
    }
}
static void rot_cols(int n, double *h, int p, int r0, int r1, double c, double s) {
    double *x = h + (size_t)p * n, *y = x + n;
    for (int i = r0; i <= r1; ++i) {
        double a = x[i], b = y[i];
        x[i] = c * a + s * b;
        y[i] = -s * a + c * b;
    }
}

// Split a 2 x 2 diagonal block at (p, p+1): if its eigenvalues are real,
// rotate it to upper triangular form; otherwise leave it and report the pair.
static void split_2x2(int n, double *h, double *z, int p, double *wr, double *wi) {
    auto H = [&](int i, int j) -> double & { return h[i + (size_t)j * n]; };
    double a = H(p, p), b = H(p, p + 1), c = H(p + 1, p), d = H(p + 1, p + 1);
    double half = 0.5 * (a - d);
    double disc = std::fma(half, half, b * c);
    if (disc >= 0) {
        double r = std::sqrt(disc);
        double mean = 0.5 * (a + d);
        // l1 - d = half +- r without cancellation when the sign follows half
        double l1 = (half >= 0) ? mean + r : mean - r;
        // eigenvector for l1: (l1 - d, c) or (b, l1 - a), the larger
        double x0 = l1 - d, x1 = c;
        double y0 = b, y1 = l1 - a;
        if (std::hypot(y0, y1) > std::hypot(x0, x1)) {
            x0 = y0;
            x1 = y1;
        }
        double nr = std::hypot(x0, x1);
        double cs = 1, sn = 0;
        if (nr > 0) {
            cs = x0 / nr;
            sn = x1 / nr;
        }
        // G = [cs -sn; sn cs]; G^T B G has zero (2,1) entry
        rot_rows(n, h, p, p, n - 1, cs, sn);
        rot_cols(n, h, p, 0, p + 1, cs, sn);
        rot_cols(n, z, p, 0, n - 1, cs, sn);
        H(p + 1, p) = 0.0;
        wr[p] = H(p, p);
        wr[p + 1] = H(p + 1, p + 1);
        wi[p] = wi[p + 1] = 0.0;
    } else {
        double mean = 0.5 * (a + d);
        double im = std::sqrt(-disc);
        wr[p] = wr[p + 1] = mean;
        wi[p] = im;
        wi[p + 1] = -im;
    }
}

// Francis implicit double-shift QR on upper Hessenberg h (n x n), accumulating
// the transformations into z.  On success h is quasi-upper-triangular.
static bool francis_qr(int n, double *h, double *z, double *wr, double *wi) {
    auto H = [&](int i, int j) -> double & { return h[i + (size_t)j * n]; };
    double anorm = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= std::min(j + 1, n - 1); ++i) anorm = std::max(anorm, std::fabs(H(i, j)));
    const double eps = DBL_EPSILON;
    int hi = n - 1;
    int its = 0, total = 0;
    while (hi >= 0) {
        int l = hi;
        while (l > 0) {
            double s = std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l));
            if (s == 0) s = anorm;
            if (std::fabs(H(l, l - 1)) <= eps * s) {
                H(l, l - 1) = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {
            wr[hi] = H(hi, hi);
            wi[hi] = 0;
            --hi;
            its = 0;
            continue;
        }
        if (l == hi - 1) {
            split_2x2(n, h, z, hi - 1, wr, wi);
            hi -= 2;
            its = 0;
            continue;
        }
        if (++total > 60 * n) return false;
        ++its;
        double s, t;
        if (its % 11 == 10) {  // exceptional shift to break cycles
            double e = std::fabs(H(hi, hi - 1)) + std::fabs(H(hi - 1, hi - 2));
            s = 1.5 * e + H(hi, hi);
            t = e * e;
        } else {
            s = H(hi - 1, hi - 1) + H(hi, hi);
            t = H(hi - 1, hi - 1) * H(hi, hi) - H(hi - 1, hi) * H(hi, hi - 1);
        }
        // first column of (H - s1 I)(H - s2 I) with s1 + s2 = s, s1 s2 = t
        double x = H(l, l) * H(l, l) + H(l, l + 1) * H(l + 1, l) - s * H(l, l) + t;
        double y = H(l + 1, l) * (H(l, l) + H(l + 1, l + 1) - s);
        double w = H(l + 1, l) * H(l + 2, l + 1);
        for (int k = l; k <= hi - 2; ++k) {
            double tau, v1, v2, beta;
            bool ok = make_reflector(x, y, w, tau, v1, v2, beta);
            if (ok) {
                int c0 = (k > l) ? k - 1 : l;
                refl3_left(n, h, k, c0, n - 1, tau, v1, v2);
                refl3_right(n, h, k, 0, std::min(k + 3, hi), tau, v1, v2);
                refl3_right(n, z, k, 0, n - 1, tau, v1, v2);
                if (k > l) {
                    H(k, k - 1) = beta;
                    H(k + 1, k - 1) = 0.0;
                    H(k + 2, k - 1) = 0.0;
                }
            }
            x = H(k + 1, k);
            y = H(k + 2, k);
            w = (k < hi - 2) ? H(k + 3, k) : 0.0;
        }
        // final 2-element reflector on rows hi-1, hi
        {
            double tau, v1, v2, beta;
            if (make_reflector(x, y, 0.0, tau, v1, v2, beta)) {
                int k = hi - 1;
                refl2_left(n, h, k, k - 1, n - 1, tau, v1);
                refl2_right(n, h, k, 0, hi, tau, v1);
                refl2_right(n, z, k, 0, n - 1, tau, v1);
                H(k, k - 1) = beta;
                H(k + 1, k - 1) = 0.0;
            }
        }
    }
    return true;
}

// Eigenvectors of the quasi-triangular T (real Schur form), back-transformed by Z.
static void schur_vectors(int n, const double *t, const double *z, const double *wr,
                          const double *wi, double *V, int ldv) {
    auto T = [&](int i, int j) { return t[i + (size_t)j * n]; };
    double tnorm = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= std::min(j + 1, n - 1); ++i) tnorm = std::max(tnorm, std::fabs(T(i, j)));
    const double small = std::max(tnorm, 1e-300) * DBL_EPSILON;
    std::vector<cd> x(n);
    int k = 0;
    while (k < n) {
        bool pair = (wi[k] != 0.0);
        cd lam(wr[k], wi[k]);
        std::fill(x.begin(), x.end(), cd(0));
        int top;  // first row of the eigenvalue's own block
        if (!pair) {
            x[k] = 1.0;
            top = k;
        } else {
            // eigenvector of the 2 x 2 block for lam = wr + i wi (wi > 0)
            double a = T(k, k), b = T(k, k + 1), c = T(k + 1, k), d = T(k + 1, k + 1);
            cd u0(b), u1 = lam - a;
            cd w0 = lam - d, w1(c);
            if (std::abs(w0) + std::abs(w1) > std::abs(u0) + std::abs(u1)) {
                u0 = w0;
                u1 = w1;
            }
            x[k] = u0;
            x[k + 1] = u1;
            top = k;
        }
        // back substitution for rows above the block
        int i = top - 1;
        while (i >= 0) {
            bool blk = (i > 0 && T(i, i - 1) != 0.0);
            int last = pair ? k + 1 : k;
            if (!blk) {
                cd r(0);
                for (int j = i + 1; j <= last; ++j) r += T(i, j) * x[j];
                cd den = T(i, i) - lam;
                if (std::abs(den) < small) den = small;
                x[i] = -r / den;
                --i;
            } else {
                // 2 x 2 system on rows i-1, i
                cd r0(0), r1(0);
                for (int j = i + 1; j <= last; ++j) {
                    r0 += T(i - 1, j) * x[j];
                    r1 += T(i, j) * x[j];
                }
                cd a11 = T(i - 1, i - 1) - lam, a12 = T(i - 1, i);
                cd a21 = T(i, i - 1), a22 = T(i, i) - lam;
                cd det = a11 * a22 - a12 * a21;
                if (std::abs(det) < small * small) det = small * small;
                x[i - 1] = (-r0 * a22 + a12 * r1) / det;
                x[i] = (-a11 * r1 + a21 * r0) / det;
                i -= 2;
            }
            // rescale to avoid overflow in long back substitutions
            double mx = 0;
            for (int j = std::max(i + 1, 0); j <= last; ++j) mx = std::max(mx, std::abs(x[j]));
            if (mx > 1e100)
                for (int j = 0; j <= last; ++j) x[j] /= mx;
        }
        // v = Z x, normalise to unit 2-norm
        int last = pair ? k + 1 : k;
        std::vector<cd> v(n, cd(0));
        for (int j = 0; j <= last; ++j) {
            if (x[j] == cd(0)) continue;
            const double *zc = z + (size_t)j * n;
            for (int r = 0; r < n; ++r) v[r] += zc[r] * x[j];
        }
        double nrm = 0;
        for (int r = 0; r < n; ++r) nrm += std::norm(v[r]);
        nrm = std::sqrt(nrm);
        if (nrm == 0) nrm = 1;
        if (!pair) {
            for (int r = 0; r < n; ++r) V[r + (size_t)k * ldv] = v[r].real() / nrm;
            k += 1;
        } else {
            for (int r = 0; r < n; ++r) {
                V[r + (size_t)k * ldv] = v[r].real() / nrm;
                V[r + (size_t)(k + 1) * ldv] = v[r].imag() / nrm;
            }
            k += 2;
        }
    }
}

bool dense_eig(int n, const double *A, int lda, double *wr, double *wi, double *V, int ldv) {
    if (n <= 0) return true;
    std::vector<double> h((size_t)n * n), z((size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) h[i + (size_t)j * n] = A[i + (size_t)j * lda];
    hessenberg(n, h.data(), z.data());
    if (!francis_qr(n, h.data(), z.data(), wr, wi)) return false;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(wr[i]) || !std::isfinite(wi[i])) return false;
    if (V) schur_vectors(n, h.data(), z.data(), wr, wi, V, ldv);
    return true;
}

// ---------------------------------------------------------------------------
// LU with partial pivoting: solve M x = b in place (M n x n column-major).
// ---------------------------------------------------------------------------
bool lu_solve(int n, std::vector<double> M, double *b) {
    auto A = [&](int i, int j) -> double & { return M[i + (size_t)j * n]; };
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(A(i, k)) > std::fabs(A(p, k))) p = i;
        if (A(p, k) == 0.0) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(A(k, j), A(p, j));
            std::swap(b[k], b[p]);
        }
        for (int i = k + 1; i < n; ++i) {
            double f = A(i, k) / A(k, k);
            A(i, k) = f;
            for (int j = k + 1; j < n; ++j) A(i, j) -= f * A(k, j);
            b[i] -= f * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A(i, j) * b[j];
        b[i] = s / A(i, i);
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(b[i])) return false;
    return true;
}

bool harmonic_ritz(int d, const double *H, int ldh, double *re, double *im) {
    // H_d^T f = e_d
    std::vector<double> Mt((size_t)d * d);
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) Mt[i + (size_t)j * d] = H[j + (size_t)i * ldh];
    std::vector<double> f(d, 0.0);
    f[d - 1] = 1.0;
    if (!lu_solve(d, Mt, f.data())) return false;
    double h = H[d + (size_t)(d - 1) * ldh];
    std::vector<double> M((size_t)d * d);
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) M[i + (size_t)j * d] = H[i + (size_t)j * ldh];
    for (int i = 0; i < d; ++i) M[i + (size_t)(d - 1) * d] += h * h * f[i];
    return dense_eig(d, M.data(), d, re, im, nullptr, 0);
}

// ---------------------------------------------------------------------------
// Householder QR, explicit thin Q (m x k, column-major, ld m) of B (m x k).
// ---------------------------------------------------------------------------
void thin_qr(int m, int k, const double *B, double *Q) {
    std::vector<double> a(B, B + (size_t)m * k);
    std::vector<std::vector<double>> vs;
    std::vector<double> taus;
    for (int j = 0; j < k; ++j) {
        std::vector<double> v(m, 0.0);
        double ss = 0;
        for (int i = j; i < m; ++i) ss += a[i + (size_t)j * m] * a[i + (size_t)j * m];
        double nrm = std::sqrt(ss);
        double x0 = a[j + (size_t)j * m];
        double alpha = (x0 > 0) ? -nrm : nrm;
        double tau = 0;
        if (nrm > 0) {
            for (int i = j; i < m; ++i) v[i] = a[i + (size_t)j * m];
            v[j] -= alpha;
            double vv = 0;
            for (int i = j; i < m; ++i) vv += v[i] * v[i];
            tau = (vv > 0) ? 2.0 / vv : 0.0;
            for (int c = j; c < k; ++c) {
                double s = 0;
                for (int i = j; i < m; ++i) s += v[i] * a[i + (size_t)c * m];
                s *= tau;
                for (int i = j; i < m; ++i) a[i + (size_t)c * m] -= s * v[i];
            }
        }
        vs.push_back(std::move(v));
        taus.push_back(tau);
    }
    for (int c = 0; c < k; ++c)
        for (int i = 0; i < m; ++i) Q[i + (size_t)c * m] = (i == c) ? 1.0 : 0.0;
    for (int j = k - 1; j >= 0; --j) {
        const auto &v = vs[j];
        double tau = taus[j];
        if (tau == 0) continue;
        for (int c = 0; c < k; ++c) {
            double s = 0;
            for (int i = j; i < m; ++i) s += v[i] * Q[i + (size_t)c * m];
            s *= tau;
            for (int i = j; i < m; ++i) Q[i + (size_t)c * m] -= s * v[i];
        }
    }
}

// ---------------------------------------------------------------------------
// Modified Leja order and added roots
// ---------------------------------------------------------------------------
static bool units_of(const std::vector<cd> &roots, std::vector<cd> &units) {
    std::vector<cd> up, lo;
    units.clear();
    for (const cd &z : roots) {
        if (z.imag() == 0.0)
            units.push_back(z);
        else if (z.imag() > 0)
            up.push_back(z);
        else
            lo.push_back(z);
    }
    if (up.size() != lo.size()) return false;
    std::vector<std::pair<double, double>> a, b;
    for (auto &z : up) a.push_back({z.real(), z.imag()});
    for (auto &z : lo) b.push_back({z.real(), -z.imag()});
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) return false;
    for (auto &z : up) units.push_back(z);
    return true;
}

static void expand(const std::vector<cd> &units, std::vector<cd> &out) {
    out.clear();
    for (const cd &z : units) {
        out.push_back(z);
        if (z.imag() != 0.0) out.push_back(std::conj(z));
    }
}

bool leja_order(const std::vector<cd> &roots, std::vector<cd> &out) {
    std::vector<cd> units;
    if (!units_of(roots, units)) return false;
    // canonical candidate order: (-re, -im, position)
    std::vector<int> idx(units.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int p, int q) {
        if (units[p].real() != units[q].real()) return units[p].real() > units[q].real();
        if (units[p].imag() != units[q].imag()) return units[p].imag() > units[q].imag();
        return p < q;
    });
    std::vector<cd> cand;
    for (int i : idx) cand.push_back(units[i]);
    std::vector<cd> chosen, pts;
    // first: largest modulus (first in canonical order on ties)
    size_t best = 0;
    for (size_t i = 1; i < cand.size(); ++i)
        if (std::abs(cand[i]) > std::abs(cand[best])) best = i;
    chosen.push_back(cand[best]);
    cand.erase(cand.begin() + best);
    while (!cand.empty()) {
        expand(chosen, pts);
        size_t bi = 0;
        double bs = -INFINITY;
        for (size_t i = 0; i < cand.size(); ++i) {
            double s = 0;
            for (const cd &p : pts) s += std::log(std::hypot(cand[i].real() - p.real(), cand[i].imag() - p.imag()));
            if (i == 0 || s > bs) {  // strict: the first maximiser wins ties
                bs = s;
                bi = i;
            }
        }
        chosen.push_back(cand[bi]);
        cand.erase(cand.begin() + bi);
    }
    expand(chosen, out);
    return true;
}

double pof_log10(const std::vector<cd> &roots, size_t j) {
    double s = 0;
    for (size_t i = 0; i < roots.size(); ++i) {
        if (i == j) continue;
        s += std::log10(std::abs(1.0 - roots[j] / roots[i]));
    }
    return s;
}

int extra_copies(double lp) {
    double x = std::ceil((lp - 4.0) / 14.0);
    return x > 0 ? (int)x : 0;
}

bool add_stability_roots(const std::vector<cd> &ordered, std::vector<cd> &out, int &added) {
    // units in the given order (pairs adjacent, im > 0 first)
    std::vector<cd> units;
    std::vector<size_t> first;  // index of each unit's first member in `ordered`
    for (size_t i = 0; i < ordered.size();) {
        cd z = ordered[i];
        units.push_back(z);
        first.push_back(i);
        if (z.imag() != 0.0) {
            if (z.imag() < 0 || i + 1 >= ordered.size() || ordered[i + 1] != std::conj(z)) return false;
            i += 2;
        } else {
            i += 1;
        }
    }
    struct Item {
        cd v;
        int id;  // original unit id, -1 for a copy
    };
    std::vector<Item> lst;
    for (size_t u = 0; u < units.size(); ++u) lst.push_back({units[u], (int)u});
    added = 0;
    for (size_t u = 0; u < units.size(); ++u) {
        int c = extra_copies(pof_log10(ordered, first[u]));
        if (c == 0) continue;
        int p = 0;
        while (lst[p].id != (int)u) ++p;
        int L = (int)lst.size();
        std::vector<int> ins;
        for (int t = 1; t < c; ++t) ins.push_back(p + (int)(((long long)t * (L - p)) / c));
        lst.push_back({units[u], -1});
        std::sort(ins.begin(), ins.end(), std::greater<int>());
        for (int q : ins) lst.insert(lst.begin() + q + 1, Item{units[u], -1});
        added += c * (units[u].imag() != 0.0 ? 2 : 1);
    }
    std::vector<cd> uv;
    for (auto &it : lst) uv.push_back(it.v);
    expand(uv, out);
    return true;
}

// Order of Ritz values by increasing |target - nu|; ties: larger re first, then im > 0 first.
std::vector<int> ritz_order(const std::vector<cd> &nu, double target) {
    std::vector<int> idx(nu.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::vector<double> dist(nu.size());
    for (size_t i = 0; i < nu.size(); ++i)
        dist[i] = std::hypot(target - nu[i].real(), -nu[i].imag());
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        if (dist[a] != dist[b]) return dist[a] < dist[b];
        if (nu[a].real() != nu[b].real()) return nu[a].real() > nu[b].real();
        return nu[a].imag() > nu[b].imag();
    });
    return idx;
}

}  // namespace ppd

// ---------------------------------------------------------------------------
// C-ABI wrappers (host only)
// ---------------------------------------------------------------------------
extern "C" {

pp_status pp_dense_eig(int n, const double *A, int lda, double *wr, double *wi, double *V, int ldv) {
    if (n < 0 || !A || !wr || !wi || lda < n || (V && ldv < n)) return pp_fail(PP_EINVAL, "pp_dense_eig: bad arguments");
    if (!ppd::dense_eig(n, A, lda, wr, wi, V, ldv)) return pp_fail(PP_ENUMERIC, "pp_dense_eig: QR did not converge");
    return PP_OK;
}

pp_status pp_harmonic_ritz(int d, const double *H, int ldh, double *re, double *im) {
    if (d <= 0 || !H || ldh < d + 1 || !re || !im) return pp_fail(PP_EINVAL, "pp_harmonic_ritz: bad arguments");
    if (!ppd::harmonic_ritz(d, H, ldh, re, im)) return pp_fail(PP_ENUMERIC, "pp_harmonic_ritz: singular H_d or QR failure");
    return PP_OK;
}

pp_status pp_leja_order(int count, const double *re, const double *im, double *out_re, double *out_im) {
    if (count <= 0 || !re || !im || !out_re || !out_im) return pp_fail(PP_EINVAL, "pp_leja_order: bad arguments");
    std::vector<ppd::cd> r(count), o;
    for (int i = 0; i < count; ++i) r[i] = ppd::cd(re[i], im[i]);
    if (!ppd::leja_order(r, o)) return pp_fail(PP_EINVAL, "pp_leja_order: roots not closed under conjugation");
    for (int i = 0; i < count; ++i) {
        out_re[i] = o[i].real();
        out_im[i] = o[i].imag();
    }
    return PP_OK;
}

pp_status pp_add_stability_roots(int count, const double *re, const double *im, int cap, double *out_re,
                                 double *out_im, int *out_count) {
    if (count <= 0 || !re || !im || !out_re || !out_im || !out_count) return pp_fail(PP_EINVAL, "pp_add_stability_roots: bad arguments");
    std::vector<ppd::cd> r(count), o;
    for (int i = 0; i < count; ++i) r[i] = ppd::cd(re[i], im[i]);
    int added = 0;
    if (!ppd::add_stability_roots(r, o, added)) return pp_fail(PP_EINVAL, "pp_add_stability_roots: conjugate pair not adjacent");
    *out_count = (int)o.size();
    for (int i = 0; i < (int)o.size() && i < cap; ++i) {
        out_re[i] = o[i].real();
        out_im[i] = o[i].imag();
    }
    return PP_OK;
}

}  // extern "C"
