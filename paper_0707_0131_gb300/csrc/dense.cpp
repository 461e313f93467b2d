// Host FP64 small-matrix linear algebra (see dense.h).  Algorithms follow the
// textbook statements: Householder tridiagonal reduction, Sturm-sequence
// bisection, inverse iteration with a partially pivoted tridiagonal LU, Cholesky,
// and modified Gram-Schmidt.
#include "dense.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace eig {
namespace dense {

static const double EPS = std::numeric_limits<double>::epsilon();

void herm_tridiag(int n, cd *A, double *d, double *e, cd *Q) {
    for (int i = 0; i < n * n; i++) Q[i] = 0.0;
    for (int i = 0; i < n; i++) Q[i * n + i] = 1.0;
    std::vector<cd> v(n), p(n);
    for (int k = 0; k + 2 < n; k++) {
        const int m = n - k - 1;  // length of the sub-column
        double xn = 0.0;
        for (int i = 0; i < m; i++) xn += std::norm(A[(k + 1 + i) * n + k]);
        xn = std::sqrt(xn);
        if (xn == 0.0) continue;
        const cd x0 = A[(k + 1) * n + k];
        const cd phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cd(1.0);
        const cd alpha = -phase * xn;
        for (int i = 0; i < m; i++) v[i] = A[(k + 1 + i) * n + k];
        v[0] -= alpha;
        double vn2 = 0.0;
        for (int i = 0; i < m; i++) vn2 += std::norm(v[i]);
        if (vn2 == 0.0) continue;
        const double tau = 2.0 / vn2;
        // p = tau * A_sub v
        for (int i = 0; i < m; i++) {
            cd s = 0.0;
            const cd *row = A + (k + 1 + i) * n + (k + 1);
            for (int j = 0; j < m; j++) s += row[j] * v[j];
            p[i] = tau * s;
        }
        cd vp = 0.0;
        for (int i = 0; i < m; i++) vp += std::conj(v[i]) * p[i];
        const double K = 0.5 * tau * vp.real();
        for (int i = 0; i < m; i++) p[i] -= K * v[i];  // w
        for (int i = 0; i < m; i++) {
            cd *row = A + (k + 1 + i) * n + (k + 1);
            for (int j = 0; j < m; j++) row[j] -= v[i] * std::conj(p[j]) + p[i] * std::conj(v[j]);
        }
        A[(k + 1) * n + k] = alpha;
        A[k * n + (k + 1)] = std::conj(alpha);
        for (int i = 1; i < m; i++) {
            A[(k + 1 + i) * n + k] = 0.0;
            A[k * n + (k + 1 + i)] = 0.0;
        }
        // Q <- Q (I - tau v v^H) on columns k+1..n-1
        for (int r = 0; r < n; r++) {
            cd *qr = Q + r * n + (k + 1);
            cd s = 0.0;
            for (int j = 0; j < m; j++) s += qr[j] * v[j];
            s *= tau;
            for (int j = 0; j < m; j++) qr[j] -= s * std::conj(v[j]);
        }
    }
    // diagonal, then absorb the phases of the off-diagonal into Q
    std::vector<cd> phi(n);
    phi[0] = 1.0;
    for (int i = 0; i < n; i++) d[i] = A[i * n + i].real();
    for (int i = 0; i + 1 < n; i++) {
        const cd c = A[(i + 1) * n + i];
        const double a = std::abs(c);
        e[i] = a;
        phi[i + 1] = a > 0.0 ? phi[i] * (c / a) : phi[i];
    }
    for (int r = 0; r < n; r++)
        for (int j = 0; j < n; j++) Q[r * n + j] *= phi[j];
}

// number of eigenvalues of (d, e) smaller than x
static int sturm_count(int n, const double *d, const double *e2, double x, double pivmin) {
    int cnt = 0;
    double q = d[0] - x;
    if (std::fabs(q) < pivmin) q = -pivmin;
    if (q < 0) cnt++;
    for (int i = 1; i < n; i++) {
        q = d[i] - x - e2[i - 1] / q;
        if (std::fabs(q) < pivmin) q = -pivmin;
        if (q < 0) cnt++;
    }
    return cnt;
}

// Solves (T - lambda I) y = y in place with a partially pivoted LU of the tridiagonal.
// Pivots smaller than pivmin (eps * ||T||) are replaced by +-pivmin: the shift is an
// eigenvalue to rounding, so exact singularity is expected and harmless.
static void tridiag_shift_solve(int n, const double *d, const double *e, double lambda, double pivmin,
                                std::vector<double> &y) {
    std::vector<double> a(n), b(n > 1 ? n - 1 : 1), c(n > 1 ? n - 1 : 1), u2(n > 2 ? n - 2 : 1);
    std::vector<int> swp(n > 1 ? n - 1 : 1);
    for (int i = 0; i < n; i++) a[i] = d[i] - lambda;
    for (int i = 0; i + 1 < n; i++) b[i] = c[i] = e[i];
    for (int i = 0; i + 1 < n; i++) {
        if (std::fabs(a[i]) >= std::fabs(c[i])) {
            if (std::fabs(a[i]) < pivmin) a[i] = a[i] < 0 ? -pivmin : pivmin;
            const double mult = c[i] / a[i];
            c[i] = mult;
            a[i + 1] -= mult * b[i];
            if (i + 2 < n) u2[i] = 0.0;
            swp[i] = 0;
        } else {
            const double mult = a[i] / c[i];
            a[i] = c[i];
            const double tmp = a[i + 1];
            a[i + 1] = b[i] - mult * tmp;
            if (i + 2 < n) {
                u2[i] = b[i + 1];
                b[i + 1] = -mult * b[i + 1];
            }
            b[i] = tmp;
            c[i] = mult;
            swp[i] = 1;
        }
    }
    if (a[n - 1] == 0.0) a[n - 1] = pivmin;
    for (int i = 0; i < n; i++)
        if (std::fabs(a[i]) < pivmin) a[i] = a[i] < 0 ? -pivmin : pivmin;
    // forward: L
    for (int i = 0; i + 1 < n; i++) {
        if (!swp[i]) {
            y[i + 1] -= c[i] * y[i];
        } else {
            const double t = y[i];
            y[i] = y[i + 1];
            y[i + 1] = t - c[i] * y[i];
        }
    }
    // backward: U (diagonal a, super b, second super u2)
    y[n - 1] /= a[n - 1];
    if (n > 1) y[n - 2] = (y[n - 2] - b[n - 2] * y[n - 1]) / a[n - 2];
    for (int i = n - 3; i >= 0; i--) y[i] = (y[i] - b[i] * y[i + 1] - u2[i] * y[i + 2]) / a[i];
}

void tridiag_eig(int n, const double *d, const double *e, int lo, int hi, double *w, double *Z) {
    if (hi <= lo) return;
    if (n == 1) {
        w[0] = d[0];
        Z[0] = 1.0;
        return;
    }
    std::vector<double> e2(n - 1);
    double gl = d[0], gu = d[0];
    for (int i = 0; i < n; i++) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        gl = std::min(gl, d[i] - r);
        gu = std::max(gu, d[i] + r);
    }
    double emax = 0.0;
    for (int i = 0; i + 1 < n; i++) {
        e2[i] = e[i] * e[i];
        emax = std::max(emax, e2[i]);
    }
    const double tnorm = std::max(std::fabs(gl), std::fabs(gu));
    const double pivmin = std::max(std::numeric_limits<double>::min(), tnorm * 1e-300 + std::numeric_limits<double>::min() * emax);
    gl -= 2.0 * EPS * tnorm * n + pivmin;
    gu += 2.0 * EPS * tnorm * n + pivmin;
    // eigenvalues by bisection
    for (int idx = lo; idx < hi; idx++) {
        double a = gl, b = gu;
        for (int it = 0; it < 200; it++) {
            const double mid = 0.5 * (a + b);
            if (b - a <= 2.0 * EPS * std::max(std::fabs(a), std::fabs(b)) + 4.0 * pivmin) break;
            if (mid <= a || mid >= b) break;
            if (sturm_count(n, d, e2.data(), mid, pivmin) > idx)
                b = mid;
            else
                a = mid;
        }
        w[idx - lo] = 0.5 * (a + b);
    }
    // eigenvectors by inverse iteration; re-orthogonalise within clusters
    const double ortol = 1e-3 * tnorm;
    const double sep = 10.0 * EPS * tnorm;
    std::vector<double> y(n);
    int cluster_start = 0;
    double lam_prev = 0.0;
    for (int q = 0; q < hi - lo; q++) {
        double lam = w[q];
        if (q > 0) {
            if (lam - w[q - 1] > ortol) cluster_start = q;
            if (lam - lam_prev < sep) lam = lam_prev + sep;  // separate equal shifts
        }
        lam_prev = lam;
        for (int i = 0; i < n; i++) y[i] = 1.0 + 0.5 * std::sin(0.7 * (i + 1) + 1.3 * (q + 1));
        for (int it = 0; it < 4; it++) {
            // scale to avoid overflow
            double mx = 0.0;
            for (int i = 0; i < n; i++) mx = std::max(mx, std::fabs(y[i]));
            if (mx > 0) for (int i = 0; i < n; i++) y[i] /= mx;
            tridiag_shift_solve(n, d, e, lam, std::max(pivmin, EPS * tnorm), y);
            for (int p = cluster_start; p < q; p++) {
                const double *zp = Z + (size_t)p * n;
                double dot = 0.0;
                for (int i = 0; i < n; i++) dot += zp[i] * y[i];
                for (int i = 0; i < n; i++) y[i] -= dot * zp[i];
            }
            double nr = 0.0;
            for (int i = 0; i < n; i++) nr += y[i] * y[i];
            nr = std::sqrt(nr);
            if (nr == 0.0 || !std::isfinite(nr)) {
                for (int i = 0; i < n; i++) y[i] = (i == q % n) ? 1.0 : 0.0;
                nr = 1.0;
            }
            for (int i = 0; i < n; i++) y[i] /= nr;
        }
        // one more orthogonalisation pass for tight clusters
        for (int p = cluster_start; p < q; p++) {
            const double *zp = Z + (size_t)p * n;
            double dot = 0.0;
            for (int i = 0; i < n; i++) dot += zp[i] * y[i];
            for (int i = 0; i < n; i++) y[i] -= dot * zp[i];
        }
        double nr = 0.0;
        for (int i = 0; i < n; i++) nr += y[i] * y[i];
        nr = std::sqrt(nr);
        for (int i = 0; i < n; i++) Z[(size_t)q * n + i] = y[i] / nr;
    }
}

void herm_eig_lowest(int n, const cd *A, int k, double *w, cd *Y) {
    std::vector<cd> B(A, A + (size_t)n * n), Q((size_t)n * n);
    std::vector<double> d(n), e(n > 1 ? n - 1 : 1), Z((size_t)n * k);
    herm_tridiag(n, B.data(), d.data(), e.data(), Q.data());
    tridiag_eig(n, d.data(), e.data(), 0, k, w, Z.data());
    for (int c = 0; c < k; c++)
        for (int r = 0; r < n; r++) {
            cd s = 0.0;
            for (int j = 0; j < n; j++) s += Q[(size_t)r * n + j] * Z[(size_t)c * n + j];
            Y[(size_t)c * n + r] = s;
        }
}

void window_lowest(int m, const cd *T, int kh, int n, int k, double *w, cd *Y) {
    if (kh > 0 && n < kh + 1) {  // the leading block lies inside the diagonal head
        std::vector<cd> B((size_t)n * n);
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) B[(size_t)i * n + j] = T[(size_t)i * m + j];
        herm_eig_lowest(n, B.data(), k, w, Y);
        return;
    }
    // head block in the order [kh, 0, 1, ..., kh-1], reduced with index 0 fixed
    const int nb = kh + 1;
    std::vector<cd> Bp((size_t)nb * nb), Qb((size_t)nb * nb);
    auto orig = [kh](int q) { return q == 0 ? kh : q - 1; };
    for (int q = 0; q < nb; q++)
        for (int p = 0; p < nb; p++) Bp[(size_t)q * nb + p] = T[(size_t)orig(q) * m + orig(p)];
    std::vector<double> db(nb), eb(nb > 1 ? nb - 1 : 1);
    if (nb > 1) {
        herm_tridiag(nb, Bp.data(), db.data(), eb.data(), Qb.data());
    } else {
        db[0] = Bp[0].real();
        Qb[0] = 1.0;
    }
    // chain: positions 0..kh hold Tb indices kh..0, positions > kh the tail of T
    std::vector<double> dc(n), ec(n > 1 ? n - 1 : 1);
    std::vector<cd> phi(n);
    for (int q = 0; q < nb; q++) dc[kh - q] = db[q];
    for (int q = 0; q < kh; q++) ec[kh - q - 1] = eb[q];
    for (int p = 0; p <= kh && p < n; p++) phi[p] = 1.0;
    for (int p = kh + 1; p < n; p++) {
        dc[p] = T[(size_t)p * m + p].real();
        const cd c = T[(size_t)p * m + p - 1];
        const double a = std::abs(c);
        ec[p - 1] = a;
        phi[p] = a > 0.0 ? phi[p - 1] * (c / a) : phi[p - 1];
    }
    std::vector<double> Z((size_t)n * k);
    tridiag_eig(n, dc.data(), ec.data(), 0, k, w, Z.data());
    std::vector<cd> zc(n), u(nb);
    for (int c = 0; c < k; c++) {
        for (int p = 0; p < n; p++) zc[p] = phi[p] * Z[(size_t)c * n + p];
        cd *y = Y + (size_t)c * n;
        for (int p = kh + 1; p < n; p++) y[p] = zc[p];
        for (int q = 0; q < nb; q++) {
            cd s = 0.0;
            for (int j = 0; j < nb; j++) s += Qb[(size_t)q * nb + j] * zc[kh - j];
            u[q] = s;
        }
        for (int q = 0; q < nb; q++) y[orig(q)] = u[q];
    }
}

int orth_columns(int n, int c, cd *X, double drop_tol, int *keep) {
    int r = 0;
    for (int j = 0; j < c; j++) {
        cd *x = X + (size_t)j * n;
        double n0 = 0.0;
        for (int i = 0; i < n; i++) n0 += std::norm(x[i]);
        n0 = std::sqrt(n0);
        for (int pass = 0; pass < 2; pass++) {
            for (int q = 0; q < r; q++) {
                const cd *u = X + (size_t)q * n;
                cd s = 0.0;
                for (int i = 0; i < n; i++) s += std::conj(u[i]) * x[i];
                for (int i = 0; i < n; i++) x[i] -= s * u[i];
            }
        }
        double nr = 0.0;
        for (int i = 0; i < n; i++) nr += std::norm(x[i]);
        nr = std::sqrt(nr);
        if (n0 == 0.0 || nr <= drop_tol * n0) continue;
        cd *dst = X + (size_t)r * n;
        for (int i = 0; i < n; i++) dst[i] = x[i] / nr;
        if (keep) keep[r] = j;
        r++;
    }
    return r;
}

int restart_coefficients(int m, const cd *T, int kh, int nev, double drop_tol, cd *QZ, double *M) {
    std::vector<cd> X((size_t)m * 2 * nev, cd(0.0));
    std::vector<double> w(nev);
    window_lowest(m, T, kh, m, nev, w.data(), X.data());
    std::vector<cd> Yb((size_t)(m - 1) * nev);
    window_lowest(m, T, kh, m - 1, nev, w.data(), Yb.data());
    for (int c = 0; c < nev; c++)
        for (int i = 0; i < m - 1; i++) X[(size_t)(nev + c) * m + i] = Yb[(size_t)c * (m - 1) + i];
    const int r = orth_columns(m, 2 * nev, X.data(), drop_tol, nullptr);
    // H = Q^H T Q
    std::vector<cd> TQ((size_t)m * r), H((size_t)r * r);
    for (int c = 0; c < r; c++)
        for (int i = 0; i < m; i++) {
            cd s = 0.0;
            for (int j = 0; j < m; j++) s += T[(size_t)i * m + j] * X[(size_t)c * m + j];
            TQ[(size_t)c * m + i] = s;
        }
    for (int a = 0; a < r; a++)
        for (int b = 0; b < r; b++) {
            cd s = 0.0;
            for (int i = 0; i < m; i++) s += std::conj(X[(size_t)a * m + i]) * TQ[(size_t)b * m + i];
            H[(size_t)a * r + b] = s;
        }
    for (int a = 0; a < r; a++) {
        H[(size_t)a * r + a] = H[(size_t)a * r + a].real();
        for (int b = a + 1; b < r; b++) {
            const cd avg = 0.5 * (H[(size_t)a * r + b] + std::conj(H[(size_t)b * r + a]));
            H[(size_t)a * r + b] = avg;
            H[(size_t)b * r + a] = std::conj(avg);
        }
    }
    std::vector<cd> Zc((size_t)r * r);
    herm_eig_lowest(r, H.data(), r, M, Zc.data());
    for (int c = 0; c < r; c++)
        for (int i = 0; i < m; i++) {
            cd s = 0.0;
            for (int j = 0; j < r; j++) s += X[(size_t)j * m + i] * Zc[(size_t)c * r + j];
            QZ[(size_t)c * m + i] = s;
        }
    return r;
}

bool cholesky(int n, cd *L) {
    for (int j = 0; j < n; j++) {
        double s = L[(size_t)j * n + j].real();
        for (int k = 0; k < j; k++) s -= std::norm(L[(size_t)j * n + k]);
        if (!(s > 0.0) || !std::isfinite(s)) return false;
        const double ljj = std::sqrt(s);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; i++) {
            cd t = L[(size_t)i * n + j];
            for (int k = 0; k < j; k++) t -= L[(size_t)i * n + k] * std::conj(L[(size_t)j * n + k]);
            L[(size_t)i * n + j] = t / ljj;
        }
        for (int i = 0; i < j; i++) L[(size_t)i * n + j] = 0.0;
    }
    return true;
}

void chol_solve(int n, const cd *L, cd *B, int nrhs) {
    for (int c = 0; c < nrhs; c++) {
        cd *b = B + (size_t)c * n;
        for (int i = 0; i < n; i++) {
            cd s = b[i];
            for (int k = 0; k < i; k++) s -= L[(size_t)i * n + k] * b[k];
            b[i] = s / L[(size_t)i * n + i].real();
        }
        for (int i = n - 1; i >= 0; i--) {
            cd s = b[i];
            for (int k = i + 1; k < n; k++) s -= std::conj(L[(size_t)k * n + i]) * b[k];
            b[i] = s / L[(size_t)i * n + i].real();
        }
    }
}

// Gaussian elimination with partial pivoting (row interchanges): A (n x n row-major)
// is overwritten by its LU factors, B (column-major n x nrhs) by the solution.
bool lu_solve(int n, cd *A, cd *B, int nrhs) {
    std::vector<int> piv(n);
    for (int j = 0; j < n; j++) {
        int pr = j;
        double best = std::abs(A[(size_t)j * n + j]);
        for (int i = j + 1; i < n; i++)
            if (std::abs(A[(size_t)i * n + j]) > best) {
                best = std::abs(A[(size_t)i * n + j]);
                pr = i;
            }
        if (!(best > 0.0) || !std::isfinite(best)) return false;
        piv[j] = pr;
        if (pr != j)
            for (int k = 0; k < n; k++) std::swap(A[(size_t)j * n + k], A[(size_t)pr * n + k]);
        const cd d = A[(size_t)j * n + j];
        for (int i = j + 1; i < n; i++) {
            const cd f = A[(size_t)i * n + j] / d;
            A[(size_t)i * n + j] = f;
            for (int k = j + 1; k < n; k++) A[(size_t)i * n + k] -= f * A[(size_t)j * n + k];
        }
    }
    for (int c = 0; c < nrhs; c++) {
        cd *b = B + (size_t)c * n;
        for (int j = 0; j < n; j++)
            if (piv[j] != j) std::swap(b[j], b[piv[j]]);
        for (int i = 0; i < n; i++)
            for (int k = 0; k < i; k++) b[i] -= A[(size_t)i * n + k] * b[k];
        for (int i = n - 1; i >= 0; i--) {
            for (int k = i + 1; k < n; k++) b[i] -= A[(size_t)i * n + k] * b[k];
            b[i] /= A[(size_t)i * n + i];
        }
    }
    return true;
}

}  // namespace dense
}  // namespace eig
