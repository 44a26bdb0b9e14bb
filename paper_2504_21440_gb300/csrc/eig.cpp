// Dense complex eigendecomposition A = V diag(lambda) V^-1, on the host, in
// FP64.  It is the one-time set-up of the stationary-state preconditioner
// (steady.cu): the Sylvester operator X -> A X + X A^H of the no-jump part of
// the Liouvillian is inverted through the eigenvectors of A = -i H_eff.
//
// Steps (textbook algorithms, Golub & Van Loan, Matrix Computations, Ch. 7):
//   1. Householder reduction to upper Hessenberg form, A = Q0 Hs Q0^H;
//   2. the shifted QR algorithm on Hs (Wilkinson shifts, Givens rotations,
//      deflation of negligible subdiagonal entries, exceptional shifts after
//      10 and 20 iterations without deflation) to the complex Schur form
//      A = Q T Q^H, T upper triangular;
//   3. eigenvectors of T by back substitution, V = Q Y, columns normalised;
//   4. V^-1 by LU factorisation with partial pivoting.
// Matrices are column-major: a[i + n * j].
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace qtl {

using cd = std::complex<double>;

static inline cd& at(std::vector<cd>& m, int n, int i, int j) { return m[(size_t)i + (size_t)n * j]; }

static void hessenberg(int n, std::vector<cd>& H, std::vector<cd>& Q) {
    std::vector<cd> v(n);
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;  // rows k+1 .. n-1
        double xn2 = 0.0;
        for (int i = 0; i < m; ++i) xn2 += std::norm(at(H, n, k + 1 + i, k));
        const double xn = std::sqrt(xn2);
        if (xn == 0.0) continue;
        const cd x0 = at(H, n, k + 1, k);
        const cd ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cd(1.0, 0.0);
        for (int i = 0; i < m; ++i) v[i] = at(H, n, k + 1 + i, k);
        v[0] += ph * xn;
        double vn2 = 0.0;
        for (int i = 0; i < m; ++i) vn2 += std::norm(v[i]);
        if (vn2 == 0.0) continue;
        const double beta = 2.0 / vn2;
        // H <- P H, P = I - beta v v^H on rows k+1..n-1
        for (int j = k; j < n; ++j) {
            cd s = 0.0;
            for (int i = 0; i < m; ++i) s += std::conj(v[i]) * at(H, n, k + 1 + i, j);
            s *= beta;
            for (int i = 0; i < m; ++i) at(H, n, k + 1 + i, j) -= v[i] * s;
        }
        // H <- H P and Q <- Q P on columns k+1..n-1
        for (int i = 0; i < n; ++i) {
            cd s = 0.0, t = 0.0;
            for (int l = 0; l < m; ++l) {
                s += at(H, n, i, k + 1 + l) * v[l];
                t += at(Q, n, i, k + 1 + l) * v[l];
            }
            s *= beta;
            t *= beta;
            for (int l = 0; l < m; ++l) {
                at(H, n, i, k + 1 + l) -= s * std::conj(v[l]);
                at(Q, n, i, k + 1 + l) -= t * std::conj(v[l]);
            }
        }
        for (int i = k + 2; i < n; ++i) at(H, n, i, k) = 0.0;
    }
}

// Givens rotation G = [[c, s], [-conj(s), c]] with G [x; y] = [r; 0].
static void givens(cd x, cd y, double& c, cd& s) {
    const double ax = std::abs(x), ay = std::abs(y);
    if (ay == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    if (ax == 0.0) {
        c = 0.0;
        s = std::conj(y) / ay;
        return;
    }
    const double r = std::hypot(ax, ay);
    c = ax / r;
    s = (x / ax) * std::conj(y) / r;
}

// Complex Schur form of the Hessenberg matrix H (in place), Q accumulated.
static bool schur(int n, std::vector<cd>& H, std::vector<cd>& Q) {
    const double eps = 2.220446049250313e-16;
    double hnorm = 0.0;
    for (const cd& z : H) hnorm = std::max(hnorm, std::abs(z));
    if (hnorm == 0.0) return true;
    std::vector<double> cs(n);
    std::vector<cd> ss(n);
    int hi = n - 1, iter = 0, total = 0;
    while (hi > 0) {
        int l = hi;
        for (; l > 0; --l) {
            double s = std::abs(at(H, n, l, l)) + std::abs(at(H, n, l - 1, l - 1));
            if (s == 0.0) s = hnorm;
            if (std::abs(at(H, n, l, l - 1)) <= eps * s) {
                at(H, n, l, l - 1) = 0.0;
                break;
            }
        }
        if (l == hi) {
            --hi;
            iter = 0;
            continue;
        }
        if (++total > 100 * n) return false;
        ++iter;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer its last diagonal entry
        const cd a = at(H, n, hi - 1, hi - 1), b = at(H, n, hi - 1, hi), c = at(H, n, hi, hi - 1),
                 d = at(H, n, hi, hi);
        const cd half = 0.5 * (a + d), disc = std::sqrt(half * half - (a * d - b * c));
        const cd m1 = half + disc, m2 = half - disc;
        cd mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        if (iter == 10 || iter == 20)
            mu = d + cd(std::abs(at(H, n, hi, hi - 1)) + (hi >= 2 ? std::abs(at(H, n, hi - 1, hi - 2)) : 0.0), 0.0);
        // one explicit shifted QR step on the active block l..hi: H - mu I = G^H R,
        // then H <- R G^H + mu I; rows beyond the block keep the Schur form exact
        for (int i = l; i <= hi; ++i) at(H, n, i, i) -= mu;
        for (int k = l; k < hi; ++k) {
            givens(at(H, n, k, k), at(H, n, k + 1, k), cs[k], ss[k]);
            const double cc = cs[k];
            const cd sk = ss[k];
            for (int j = k; j < n; ++j) {
                const cd x = at(H, n, k, j), y = at(H, n, k + 1, j);
                at(H, n, k, j) = cc * x + sk * y;
                at(H, n, k + 1, j) = -std::conj(sk) * x + cc * y;
            }
            at(H, n, k + 1, k) = 0.0;
        }
        for (int k = l; k < hi; ++k) {
            const double cc = cs[k];
            const cd sk = ss[k];
            const int imax = std::min(k + 2, hi);
            for (int i = 0; i <= imax; ++i) {
                const cd x = at(H, n, i, k), y = at(H, n, i, k + 1);
                at(H, n, i, k) = cc * x + std::conj(sk) * y;
                at(H, n, i, k + 1) = -sk * x + cc * y;
            }
            for (int i = 0; i < n; ++i) {
                const cd x = at(Q, n, i, k), y = at(Q, n, i, k + 1);
                at(Q, n, i, k) = cc * x + std::conj(sk) * y;
                at(Q, n, i, k + 1) = -sk * x + cc * y;
            }
        }
        for (int i = l; i <= hi; ++i) at(H, n, i, i) += mu;
    }
    return true;
}

// In-place inverse by LU with partial pivoting; false if singular.
static bool invert(int n, std::vector<cd> M, std::vector<cd>& inv) {
    std::vector<int> piv(n);
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::abs(at(M, n, k, k));
        for (int i = k + 1; i < n; ++i)
            if (std::abs(at(M, n, i, k)) > best) {
                best = std::abs(at(M, n, i, k));
                p = i;
            }
        if (best == 0.0) return false;
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) std::swap(at(M, n, k, j), at(M, n, p, j));
        const cd inv_d = 1.0 / at(M, n, k, k);
        for (int i = k + 1; i < n; ++i) {
            const cd f = at(M, n, i, k) * inv_d;
            at(M, n, i, k) = f;
            if (f == cd(0.0))
                continue;
            for (int j = k + 1; j < n; ++j) at(M, n, i, j) -= f * at(M, n, k, j);
        }
    }
    inv.assign((size_t)n * n, 0.0);
    std::vector<cd> col(n);
    for (int c = 0; c < n; ++c) {
        std::fill(col.begin(), col.end(), cd(0.0));
        col[c] = 1.0;
        for (int k = 0; k < n; ++k)
            if (piv[k] != k) std::swap(col[k], col[piv[k]]);
        for (int i = 1; i < n; ++i)
            for (int k = 0; k < i; ++k) col[i] -= at(M, n, i, k) * col[k];
        for (int i = n - 1; i >= 0; --i) {
            for (int k = i + 1; k < n; ++k) col[i] -= at(M, n, i, k) * col[k];
            col[i] /= at(M, n, i, i);
        }
        for (int i = 0; i < n; ++i) at(inv, n, i, c) = col[i];
    }
    return true;
}

bool eig_dense(int n, const std::vector<cd>& A, std::vector<cd>& lam, std::vector<cd>& V,
               std::vector<cd>& Vinv, double* cond) {
    std::vector<cd> T(A), Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) at(Q, n, i, i) = 1.0;
    hessenberg(n, T, Q);
    if (!schur(n, T, Q)) return false;
    lam.resize(n);
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) {
        lam[i] = at(T, n, i, i);
        for (int j = i; j < n; ++j) tnorm = std::max(tnorm, std::abs(at(T, n, i, j)));
    }
    const double small = std::max(tnorm, 1e-300) * 1e-14;
    // eigenvectors of T: (T - lam_k I) y = 0 with y_k = 1, y_j = 0 for j > k
    std::vector<cd> Y((size_t)n * n, 0.0);
    std::vector<cd> y(n);
    for (int k = 0; k < n; ++k) {
        std::fill(y.begin(), y.end(), cd(0.0));
        y[k] = 1.0;
        for (int j = k - 1; j >= 0; --j) {
            cd s = 0.0;
            for (int l = j + 1; l <= k; ++l) s += at(T, n, j, l) * y[l];
            cd den = at(T, n, j, j) - lam[k];
            if (std::abs(den) < small) den = small;
            y[j] = -s / den;
            // keep the vector representable
            const double big = std::abs(y[j]);
            if (big > 1e100)
                for (int l = j; l <= k; ++l) y[l] /= big;
        }
        for (int j = 0; j <= k; ++j) at(Y, n, j, k) = y[j];
    }
    // V = Q Y, unit columns
    V.assign((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        double nr = 0.0;
        for (int i = 0; i < n; ++i) {
            cd s = 0.0;
            for (int j = 0; j <= k; ++j) s += at(Q, n, i, j) * at(Y, n, j, k);
            at(V, n, i, k) = s;
            nr += std::norm(s);
        }
        nr = std::sqrt(nr);
        if (nr > 0.0)
            for (int i = 0; i < n; ++i) at(V, n, i, k) /= nr;
    }
    if (!invert(n, V, Vinv)) return false;
    if (cond) {
        double a = 0.0, b = 0.0;
        for (const cd& z : V) a += std::norm(z);
        for (const cd& z : Vinv) b += std::norm(z);
        *cond = std::sqrt(a) * std::sqrt(b) / n;   // Frobenius-norm estimate (1 for unitary V)
    }
    return true;
}

}  // namespace qtl
