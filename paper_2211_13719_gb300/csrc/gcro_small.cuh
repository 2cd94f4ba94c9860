// Small dense complex linear algebra of GCRO-DR (one RHS per call, FP64),
// written for one GPU thread per RHS and compilable for the host as well:
// Householder least squares, modified Gram-Schmidt QR, upper triangular
// inverse, Hessenberg reduction, the complex QR algorithm with Wilkinson
// shifts to Schur form, and eigenvectors of the Schur form.  Matrices are
// row-major local arrays with leading dimension LD; sizes are at most GCRO_MM.
//
// The two drivers compute, for one RHS, everything a GCRO-DR cycle needs from
// its small matrices (the method of Parks, de Sturler et al.; the steps are
// listed at gcro_seed and gcro_cycle below).
#pragma once

#include <math.h>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#endif

namespace mrhs {
namespace gcro {

constexpr int GCRO_MM = 16;       // largest restart length m
constexpr int LD = GCRO_MM + 1;   // leading dimension of the local matrices

struct zc {
    double re, im;
};
__host__ __device__ inline zc zmk(double r, double i) { return zc{r, i}; }
__host__ __device__ inline zc zadd(zc a, zc b) { return zc{a.re + b.re, a.im + b.im}; }
__host__ __device__ inline zc zsub(zc a, zc b) { return zc{a.re - b.re, a.im - b.im}; }
__host__ __device__ inline zc zmul(zc a, zc b) { return zc{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ inline zc zconj(zc a) { return zc{a.re, -a.im}; }
__host__ __device__ inline zc zscale(zc a, double s) { return zc{a.re * s, a.im * s}; }
__host__ __device__ inline double zabs2(zc a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ inline double zabs(zc a) { return hypot(a.re, a.im); }
__host__ __device__ inline zc zdiv(zc a, zc b) {
    // Smith's division
    if (fabs(b.re) >= fabs(b.im)) {
        const double r = b.im / b.re, d = b.re + b.im * r;
        return zc{(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    }
    const double r = b.re / b.im, d = b.im + b.re * r;
    return zc{(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
__host__ __device__ inline zc zsqrt(zc a) {
    const double r = zabs(a);
    if (r == 0.0) return zc{0.0, 0.0};
    double x = sqrt(0.5 * (r + fabs(a.re)));
    double y = a.im / (2.0 * x);
    if (a.re < 0.0) {
        const double t = x;
        x = fabs(y);
        y = a.im < 0.0 ? -t : t;
    }
    return zc{x, y};
}

// Givens rotation G = [[c, s], [-conj(s), c]] with G [x; y] = [r; 0], c real
__host__ __device__ inline void givens(zc x, zc y, double &c, zc &s) {
    const double ax = zabs(x), ay = zabs(y);
    if (ay == 0.0) {
        c = 1.0;
        s = zc{0.0, 0.0};
    } else if (ax == 0.0) {
        c = 0.0;
        s = zscale(zconj(y), 1.0 / ay);
    } else {
        const double t = hypot(ax, ay);
        c = ax / t;
        s = zmul(zscale(x, 1.0 / ax), zscale(zconj(y), 1.0 / t));
    }
}

// y minimising |b - A y| for A (rows x cols, rows >= cols, full column rank),
// by Householder QR; A and b are overwritten.
__host__ __device__ inline void lstsq(zc *A, zc *b, int rows, int cols, zc *y) {
    for (int k = 0; k < cols; ++k) {
        double nrm2 = 0.0;
        for (int i = k; i < rows; ++i) nrm2 += zabs2(A[i * LD + k]);
        const double nrm = sqrt(nrm2);
        if (nrm == 0.0) continue;
        const zc a0 = A[k * LD + k];
        const double a0abs = zabs(a0);
        const zc ph = a0abs > 0.0 ? zscale(a0, 1.0 / a0abs) : zc{1.0, 0.0};
        // v = x + ph |x| e_1, H = I - 2 v v^H / (v^H v)
        zc v[LD];
        for (int i = 0; i < rows - k; ++i) v[i] = A[(k + i) * LD + k];
        v[0] = zadd(v[0], zscale(ph, nrm));
        double vv = 0.0;
        for (int i = 0; i < rows - k; ++i) vv += zabs2(v[i]);
        for (int j = k; j < cols; ++j) {
            zc d = {0.0, 0.0};
            for (int i = 0; i < rows - k; ++i) d = zadd(d, zmul(zconj(v[i]), A[(k + i) * LD + j]));
            d = zscale(d, 2.0 / vv);
            for (int i = 0; i < rows - k; ++i) A[(k + i) * LD + j] = zsub(A[(k + i) * LD + j], zmul(v[i], d));
        }
        zc d = {0.0, 0.0};
        for (int i = 0; i < rows - k; ++i) d = zadd(d, zmul(zconj(v[i]), b[k + i]));
        d = zscale(d, 2.0 / vv);
        for (int i = 0; i < rows - k; ++i) b[k + i] = zsub(b[k + i], zmul(v[i], d));
    }
    for (int i = cols - 1; i >= 0; --i) {
        zc s = b[i];
        for (int j = i + 1; j < cols; ++j) s = zsub(s, zmul(A[i * LD + j], y[j]));
        const zc d = A[i * LD + i];
        y[i] = zabs2(d) > 0.0 ? zdiv(s, d) : zc{0.0, 0.0};
    }
}

// thin QR of A (rows x cols) by modified Gram-Schmidt: Q (rows x cols), R (cols x cols)
__host__ __device__ inline void qr_mgs(const zc *A, int rows, int cols, zc *Q, zc *R) {
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) Q[i * LD + j] = A[i * LD + j];
    for (int i = 0; i < cols; ++i)
        for (int j = 0; j < cols; ++j) R[i * LD + j] = zc{0.0, 0.0};
    for (int j = 0; j < cols; ++j) {
        for (int p = 0; p < j; ++p) {
            zc d = {0.0, 0.0};
            for (int i = 0; i < rows; ++i) d = zadd(d, zmul(zconj(Q[i * LD + p]), Q[i * LD + j]));
            R[p * LD + j] = d;
            for (int i = 0; i < rows; ++i) Q[i * LD + j] = zsub(Q[i * LD + j], zmul(Q[i * LD + p], d));
        }
        double n2 = 0.0;
        for (int i = 0; i < rows; ++i) n2 += zabs2(Q[i * LD + j]);
        const double nr = sqrt(n2);
        R[j * LD + j] = zc{nr, 0.0};
        const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
        for (int i = 0; i < rows; ++i) Q[i * LD + j] = zscale(Q[i * LD + j], inv);
    }
}

// X = A R^{-1} for R upper triangular (cols x cols), A (rows x cols)
__host__ __device__ inline void right_solve_upper(const zc *A, const zc *R, int rows, int cols, zc *X) {
    for (int i = 0; i < rows; ++i)
        for (int j = 0; j < cols; ++j) {
            zc s = A[i * LD + j];
            for (int p = 0; p < j; ++p) s = zsub(s, zmul(X[i * LD + p], R[p * LD + j]));
            const zc d = R[j * LD + j];
            X[i * LD + j] = zabs2(d) > 0.0 ? zdiv(s, d) : zc{0.0, 0.0};
        }
}

// A = Q H Q^H with H upper Hessenberg (in A) and Q unitary (n x n), Householder reflections
__host__ __device__ inline void hessenberg(zc *A, zc *Q, int n) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Q[i * LD + j] = zc{i == j ? 1.0 : 0.0, 0.0};
    for (int k = 0; k + 2 < n; ++k) {
        double nrm2 = 0.0;
        for (int i = k + 1; i < n; ++i) nrm2 += zabs2(A[i * LD + k]);
        if (nrm2 == 0.0) continue;
        const double nrm = sqrt(nrm2);
        const zc a0 = A[(k + 1) * LD + k];
        const double a0abs = zabs(a0);
        const zc ph = a0abs > 0.0 ? zscale(a0, 1.0 / a0abs) : zc{1.0, 0.0};
        zc v[LD];
        const int len = n - k - 1;
        for (int i = 0; i < len; ++i) v[i] = A[(k + 1 + i) * LD + k];
        v[0] = zadd(v[0], zscale(ph, nrm));
        double vv = 0.0;
        for (int i = 0; i < len; ++i) vv += zabs2(v[i]);
        const double f = 2.0 / vv;
        // A <- H A (rows k+1..n-1)
        for (int j = 0; j < n; ++j) {
            zc d = {0.0, 0.0};
            for (int i = 0; i < len; ++i) d = zadd(d, zmul(zconj(v[i]), A[(k + 1 + i) * LD + j]));
            d = zscale(d, f);
            for (int i = 0; i < len; ++i) A[(k + 1 + i) * LD + j] = zsub(A[(k + 1 + i) * LD + j], zmul(v[i], d));
        }
        // A <- A H, Q <- Q H (columns k+1..n-1)
        for (int i = 0; i < n; ++i) {
            zc d = {0.0, 0.0}, e = {0.0, 0.0};
            for (int p = 0; p < len; ++p) {
                d = zadd(d, zmul(A[i * LD + k + 1 + p], v[p]));
                e = zadd(e, zmul(Q[i * LD + k + 1 + p], v[p]));
            }
            d = zscale(d, f);
            e = zscale(e, f);
            for (int p = 0; p < len; ++p) {
                A[i * LD + k + 1 + p] = zsub(A[i * LD + k + 1 + p], zmul(d, zconj(v[p])));
                Q[i * LD + k + 1 + p] = zsub(Q[i * LD + k + 1 + p], zmul(e, zconj(v[p])));
            }
        }
        for (int i = k + 2; i < n; ++i) A[i * LD + k] = zc{0.0, 0.0};
    }
}

// Schur form of an upper Hessenberg H (n x n): H <- T = Z^H H Z upper
// triangular, Z <- Z Zq (pass the Hessenberg reduction's Q).  Single-shift
// complex QR sweeps with Wilkinson shifts (an exceptional shift every 10
// sweeps without deflation).  Returns false if 30 n sweeps did not converge.
__host__ __device__ inline bool schur(zc *H, zc *Z, int n) {
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0, total = 0;
    while (hi > 0) {
        int l = hi;
        while (l > 0) {
            const double s = zabs(H[(l - 1) * LD + l - 1]) + zabs(H[l * LD + l]);
            if (zabs(H[l * LD + l - 1]) <= eps * (s > 0.0 ? s : 1.0)) break;
            --l;
        }
        if (l == hi) {
            if (hi > 0) H[hi * LD + hi - 1] = zc{0.0, 0.0};
            --hi;
            iter = 0;
            continue;
        }
        if (l > 0) H[l * LD + l - 1] = zc{0.0, 0.0};
        if (++total > 30 * n) return false;
        ++iter;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer to its last entry
        zc mu;
        if (iter % 10 == 0) {
            const double ex = fabs(H[hi * LD + hi - 1].re) + (hi >= 2 ? fabs(H[(hi - 1) * LD + hi - 2].re) : 0.0);
            mu = zadd(H[hi * LD + hi], zc{ex, 0.0});
        } else {
            const zc a = H[(hi - 1) * LD + hi - 1], b = H[(hi - 1) * LD + hi], c = H[hi * LD + hi - 1],
                     d = H[hi * LD + hi];
            const zc half = zscale(zsub(a, d), 0.5);
            const zc disc = zsqrt(zadd(zmul(half, half), zmul(b, c)));
            const zc m = zscale(zadd(a, d), 0.5);
            const zc e1 = zadd(m, disc), e2 = zsub(m, disc);
            mu = zabs2(zsub(e1, d)) <= zabs2(zsub(e2, d)) ? e1 : e2;
        }
        // implicit QR sweep on the active block l..hi
        zc x = zsub(H[l * LD + l], mu), y = H[(l + 1) * LD + l];
        for (int k = l; k < hi; ++k) {
            double c;
            zc s;
            givens(x, y, c, s);
            // rows k, k+1: G = [[c, s], [-conj(s), c]]
            for (int j = (k > l ? k - 1 : l); j < n; ++j) {
                const zc a = H[k * LD + j], b = H[(k + 1) * LD + j];
                H[k * LD + j] = zadd(zscale(a, c), zmul(s, b));
                H[(k + 1) * LD + j] = zadd(zscale(b, c), zmul(zscale(zconj(s), -1.0), a));
            }
            // columns k, k+1 of H (rows 0..min(k+2, hi)) and of Z: times G^H
            const int rmax = k + 2 < hi ? k + 2 : hi;
            for (int i = 0; i <= rmax; ++i) {
                const zc a = H[i * LD + k], b = H[i * LD + k + 1];
                H[i * LD + k] = zadd(zscale(a, c), zmul(b, zconj(s)));
                H[i * LD + k + 1] = zsub(zscale(b, c), zmul(a, s));
            }
            for (int i = 0; i < n; ++i) {
                const zc a = Z[i * LD + k], b = Z[i * LD + k + 1];
                Z[i * LD + k] = zadd(zscale(a, c), zmul(b, zconj(s)));
                Z[i * LD + k + 1] = zsub(zscale(b, c), zmul(a, s));
            }
            if (k + 1 < hi) {
                x = H[(k + 1) * LD + k];
                y = H[(k + 2) * LD + k];
            }
        }
    }
    for (int i = 1; i < n; ++i)
        for (int j = 0; j < i; ++j) H[i * LD + j] = zc{0.0, 0.0};
    return true;
}

// eigenvector x = Z y of the eigenvalue T[s][s] of the Schur form (T upper triangular)
__host__ __device__ inline void schur_eigvec(const zc *T, const zc *Z, int n, int s, zc *x) {
    zc y[LD];
    const zc lam = T[s * LD + s];
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) tnorm = fmax(tnorm, zabs(T[i * LD + j]));
    const double small = 2.220446049250313e-16 * (tnorm > 0.0 ? tnorm : 1.0);
    for (int i = 0; i < n; ++i) y[i] = zc{0.0, 0.0};
    y[s] = zc{1.0, 0.0};
    for (int j = s - 1; j >= 0; --j) {
        zc acc = {0.0, 0.0};
        for (int l = j + 1; l <= s; ++l) acc = zadd(acc, zmul(T[j * LD + l], y[l]));
        zc d = zsub(T[j * LD + j], lam);
        if (zabs(d) < small) d = zc{small, 0.0};
        y[j] = zdiv(zscale(acc, -1.0), d);
    }
    for (int i = 0; i < n; ++i) {
        zc acc = {0.0, 0.0};
        for (int l = 0; l <= s; ++l) acc = zadd(acc, zmul(Z[i * LD + l], y[l]));
        x[i] = acc;
    }
}

// eigen-decomposition of a general M (n x n, overwritten): eigenvalues lam[n],
// eigenvectors as the columns of X; Z: LD x LD scratch; false if the QR
// algorithm did not converge
__host__ __device__ inline bool eig(zc *M, int n, zc *lam, zc *X, zc *Z) {
    hessenberg(M, Z, n);
    if (!schur(M, Z, n)) return false;
    for (int s = 0; s < n; ++s) lam[s] = M[s * LD + s];
    zc x[LD];
    for (int s = 0; s < n; ++s) {
        schur_eigvec(M, Z, n, s, x);
        for (int i = 0; i < n; ++i) X[i * LD + s] = x[i];
    }
    return true;
}

// indices of the k eigenvalues of largest modulus (ties: lower index first)
__host__ __device__ inline void largest(const zc *lam, int n, int k, int *sel) {
    bool used[LD];
    for (int i = 0; i < n; ++i) used[i] = false;
    for (int q = 0; q < k; ++q) {
        int best = -1;
        double bv = -1.0;
        for (int i = 0; i < n; ++i)
            if (!used[i] && zabs(lam[i]) > bv) {
                bv = zabs(lam[i]);
                best = i;
            }
        used[best] = true;
        sel[q] = best;
    }
}

// indices of the k eigenvalues of smallest modulus (ties: lower index first)
__host__ __device__ inline void smallest(const zc *lam, int n, int k, int *sel) {
    bool used[LD];
    for (int i = 0; i < n; ++i) used[i] = false;
    for (int q = 0; q < k; ++q) {
        int best = -1;
        double bv = 0.0;
        for (int i = 0; i < n; ++i) {
            const double a = zabs(lam[i]);
            if (!used[i] && (best < 0 || a < bv)) {
                bv = a;
                best = i;
            }
        }
        used[best] = true;
        sel[q] = best;
    }
}

// ------------------------------------------------------------ drivers
// A GMRES(m) cycle that seeds a recycle space of k vectors.  In: the Arnoldi
// Hessenberg H ((m+1) x m) of the cycle and beta = |r|.  Out:
//   y (m): the GMRES correction x += V_m y;
//   with k > 0, the k harmonic Ritz vectors of smallest modulus: the
//   eigenvectors P of F = H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^T, the thin QR
//   H P = Q R, and the coefficients of C = V_{m+1} Q (qc, (m+1) x k) and of
//   U = V_m P R^{-1} (pu, m x k).
// Returns false if an eigen-decomposition failed.
// workspace of the drivers: GCRO_WS matrices of LD x LD complex numbers
constexpr int GCRO_WS = 14;

__host__ __device__ inline bool gcro_seed(const zc *H, double beta, int m, int k, zc *y, zc *qc, zc *pu, zc *ws) {
    zc *A = ws, *Hh = ws + LD * LD, *F = ws + 2 * LD * LD, *X = ws + 3 * LD * LD, *P = ws + 4 * LD * LD,
       *HP = ws + 5 * LD * LD, *Q = ws + 6 * LD * LD, *R = ws + 7 * LD * LD, *Z = ws + 8 * LD * LD;
    zc b[LD];
    for (int i = 0; i <= m; ++i) {
        for (int j = 0; j < m; ++j) A[i * LD + j] = H[i * LD + j];
        b[i] = zc{i == 0 ? beta : 0.0, 0.0};
    }
    lstsq(A, b, m + 1, m, y);
    if (k == 0) return true;
    // w = H_m^{-H} e_m: solve H_m^H w = e_m (H_m^H lower Hessenberg), by least squares on the square system
    zc e[LD], w[LD];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Hh[i * LD + j] = zconj(H[j * LD + i]);
    for (int i = 0; i < m; ++i) e[i] = zc{i == m - 1 ? 1.0 : 0.0, 0.0};
    lstsq(Hh, e, m, m, w);
    const double h2 = zabs2(H[m * LD + m - 1]);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) F[i * LD + j] = H[i * LD + j];
    for (int i = 0; i < m; ++i) F[i * LD + m - 1] = zadd(F[i * LD + m - 1], zscale(w[i], h2));
    zc lam[LD];
    if (!eig(F, m, lam, X, Z)) return false;
    int sel[LD];
    smallest(lam, m, k, sel);
    for (int i = 0; i < m; ++i)
        for (int q = 0; q < k; ++q) P[i * LD + q] = X[i * LD + sel[q]];
    for (int i = 0; i <= m; ++i)
        for (int q = 0; q < k; ++q) {
            zc s = {0.0, 0.0};
            for (int j = 0; j < m; ++j) s = zadd(s, zmul(H[i * LD + j], P[j * LD + q]));
            HP[i * LD + q] = s;
        }
    qr_mgs(HP, m + 1, k, Q, R);
    for (int i = 0; i <= m; ++i)
        for (int q = 0; q < k; ++q) qc[i * LD + q] = Q[i * LD + q];
    right_solve_upper(P, R, m, k, pu);
    return true;
}

// A cycle with a recycle space (U, C: k vectors, C = A U orthonormal) and
// p = m - k Arnoldi steps of (I - C C^H) A.  In:
//   H ((p+1) x p) and B = C^H A V_p (k x p) of the Arnoldi process,
//   un2 (k): |u_i|^2,  wr ((m+1)): W^H r with W = [C, V_{p+1}],
//   wu ((m+1) x k): W^H U.
// With D = diag(1/|u_i|), G = [[D, B], [0, H]] ((m+1) x m) and
// V^ = [U D, V_p] (W^H V^ = [W^H U D | [0; I]], the V_p columns orthonormal
// and orthogonal to C):
//   y = argmin |W^H r - G y|                      (x += V^ y),
//   P: the k eigenvectors of smallest |theta| of G^H G z = theta G^H W^H V^ z,
//      computed as the k of largest |mu| of mu z = R_G^{-1} Q_G^H W^H V^ z
//      (G = Q_G R_G, mu = 1 / theta),
//   G P = Q R,  C_new = W Q (qc),  U_new = V^ P R^{-1} (pu, rows of U scaled by D).
// Out: y (m, its first k entries already scaled by D for the U part), qc
// ((m+1) x k), pu (m x k, first k rows scaled by D).
__host__ __device__ inline bool gcro_cycle(const zc *H, const zc *B, const double *un2, const zc *wr,
                                           const zc *wu, int m, int k, zc *y, zc *qc, zc *pu, zc *ws) {
    const int p = m - k;
    zc *G = ws, *A = ws + LD * LD, *WV = ws + 2 * LD * LD, *QG = ws + 3 * LD * LD, *RG = ws + 4 * LD * LD,
       *Mt = ws + 5 * LD * LD, *M = ws + 6 * LD * LD, *X = ws + 7 * LD * LD, *P = ws + 8 * LD * LD,
       *GP = ws + 9 * LD * LD, *Q = ws + 10 * LD * LD, *R = ws + 11 * LD * LD, *PR = ws + 12 * LD * LD,
       *Z = ws + 13 * LD * LD;
    double dn[LD];
    for (int i = 0; i < k; ++i) dn[i] = un2[i] > 0.0 ? 1.0 / sqrt(un2[i]) : 0.0;
    for (int i = 0; i <= m; ++i)
        for (int j = 0; j < m; ++j) G[i * LD + j] = zc{0.0, 0.0};
    for (int i = 0; i < k; ++i) {
        G[i * LD + i] = zc{dn[i], 0.0};
        for (int j = 0; j < p; ++j) G[i * LD + k + j] = B[i * LD + j];
    }
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j < p; ++j) G[(k + i) * LD + k + j] = H[i * LD + j];
    // least squares
    zc b[LD];
    for (int i = 0; i <= m; ++i) {
        for (int j = 0; j < m; ++j) A[i * LD + j] = G[i * LD + j];
        b[i] = wr[i];
    }
    zc yy[LD];
    lstsq(A, b, m + 1, m, yy);
    for (int i = 0; i < m; ++i) y[i] = i < k ? zscale(yy[i], dn[i]) : yy[i];
    // W^H V^ ((m+1) x m)
    for (int i = 0; i <= m; ++i) {
        for (int j = 0; j < k; ++j) WV[i * LD + j] = zscale(wu[i * LD + j], dn[j]);
        for (int j = 0; j < p; ++j) WV[i * LD + k + j] = zc{(i == k + j) ? 1.0 : 0.0, 0.0};
    }
    // G = Q_G R_G; M = R_G^{-1} Q_G^H W^H V^
    qr_mgs(G, m + 1, m, QG, RG);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            zc s = {0.0, 0.0};
            for (int l = 0; l <= m; ++l) s = zadd(s, zmul(zconj(QG[l * LD + i]), WV[l * LD + j]));
            Mt[i * LD + j] = s;
        }
    // back substitution R_G M = Mt, column by column
    for (int j = 0; j < m; ++j)
        for (int i = m - 1; i >= 0; --i) {
            zc s = Mt[i * LD + j];
            for (int l = i + 1; l < m; ++l) s = zsub(s, zmul(RG[i * LD + l], M[l * LD + j]));
            const zc d = RG[i * LD + i];
            M[i * LD + j] = zabs2(d) > 0.0 ? zdiv(s, d) : zc{0.0, 0.0};
        }
    zc lam[LD];
    if (!eig(M, m, lam, X, Z)) return false;
    int sel[LD];
    largest(lam, m, k, sel);
    for (int i = 0; i < m; ++i)
        for (int q = 0; q < k; ++q) P[i * LD + q] = X[i * LD + sel[q]];
    for (int i = 0; i <= m; ++i)
        for (int q = 0; q < k; ++q) {
            zc s = {0.0, 0.0};
            for (int j = 0; j < m; ++j) s = zadd(s, zmul(G[i * LD + j], P[j * LD + q]));
            GP[i * LD + q] = s;
        }
    qr_mgs(GP, m + 1, k, Q, R);
    for (int i = 0; i <= m; ++i)
        for (int q = 0; q < k; ++q) qc[i * LD + q] = Q[i * LD + q];
    right_solve_upper(P, R, m, k, PR);
    for (int i = 0; i < m; ++i)
        for (int q = 0; q < k; ++q) pu[i * LD + q] = i < k ? zscale(PR[i * LD + q], dn[i]) : PR[i * LD + q];
    return true;
}

}  // namespace gcro
}  // namespace mrhs
