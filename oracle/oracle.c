/*
 * Plain FP64 CPU oracle for the slice-solve hot path.  TEST INFRASTRUCTURE ONLY:
 * only the tests, the package smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA path.
 *
 * Every routine is the textbook definition written out as plain loops (OpenMP only
 * splits independent loop iterations; there is no blocking, fusion or reordering):
 *
 *  or_gen_eig       eigenpairs of the symmetric-definite pencil A x = lambda B x
 *                   (problem statement, Eq. 1): Cholesky B = L L^T, C = L^-1 A L^-T,
 *                   Householder tridiagonalisation, implicit-shift QL, back-transform
 *                   X = L^-T Y, so that X^T B X = I.
 *  or_ldlt_bk       dense Bunch-Kaufman LDL^T of a symmetric matrix with 1x1 / 2x2
 *                   pivots; returns the Sylvester inertia of D (Section 2.2, inertia
 *                   count of the shifted matrix A - sigma B).
 *  or_band_ldlt     unpivoted LDL^T of a banded symmetric matrix in natural order;
 *                   inertia by Sylvester's law when every pivot is well away from 0.
 *  or_csr_mm        Y = M X for a CSR matrix and a row-major block X (residuals).
 *  or_tridiag_eig   eigenpairs of a symmetric tridiagonal matrix (Lanczos DOS, Eq. 5).
 *  or_gen_eig_lowest the lowest m eigenpairs of the pencil by the same reduction, with
 *                   the eigenvectors of the tridiagonal matrix from inverse iteration
 *                   (Gaussian elimination with partial pivoting on T - theta I) and the
 *                   Householder back-transform; the caller takes the Rayleigh quotient
 *                   x^T A x / x^T B x of each x on the original pencil, which removes the
 *                   first-order error that forming L^-1 A L^-T leaves in theta when B is
 *                   ill-conditioned.
 *
 * Return codes: 0 ok, 1 not SPD (Cholesky hit a non-positive pivot), 2 QL did not
 * converge, 3 a band pivot fell below the reliability threshold, 4 bad size.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, n) ((size_t)(i) * (size_t)(n) + (size_t)(j))

/* ---- Cholesky of a dense SPD matrix (row-major, lower factor written to L) ---- */
static int cholesky_lower(int64_t n, const double *B, double *L) {
    memset(L, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        double s = B[IDX(j, j, n)];
        const double *lj = L + IDX(j, 0, n);
        for (int64_t k = 0; k < j; ++k) s -= lj[k] * lj[k];
        if (!(s > 0.0)) return 1;
        double djj = sqrt(s);
        L[IDX(j, j, n)] = djj;
#pragma omp parallel for schedule(static)
        for (int64_t i = j + 1; i < n; ++i) {
            const double *li = L + IDX(i, 0, n);
            double t = B[IDX(i, j, n)];
            for (int64_t k = 0; k < j; ++k) t -= li[k] * lj[k];
            L[IDX(i, j, n)] = t / djj;
        }
    }
    return 0;
}

/* ---- W = L^-1 M by forward substitution, all columns of M at once (row-major) ---- */
static void forward_subst(int64_t n, int64_t m, const double *L, const double *M, double *W) {
    const int64_t cb = 64;
#pragma omp parallel for schedule(dynamic)
    for (int64_t c0 = 0; c0 < m; c0 += cb) {
        int64_t c1 = c0 + cb < m ? c0 + cb : m;
        for (int64_t i = 0; i < n; ++i) {
            double *wi = W + IDX(i, 0, m);
            for (int64_t c = c0; c < c1; ++c) wi[c] = M[IDX(i, c, m)];
            for (int64_t k = 0; k < i; ++k) {
                double lik = L[IDX(i, k, n)];
                if (lik == 0.0) continue;
                const double *wk = W + IDX(k, 0, m);
                for (int64_t c = c0; c < c1; ++c) wi[c] -= lik * wk[c];
            }
            double inv = 1.0 / L[IDX(i, i, n)];
            for (int64_t c = c0; c < c1; ++c) wi[c] *= inv;
        }
    }
}

/* ---- X = L^-T Y by backward substitution, all columns at once (row-major n x m) ---- */
static void backward_subst_t(int64_t n, int64_t m, const double *L, const double *Y, double *X) {
    const int64_t cb = 64;
#pragma omp parallel for schedule(dynamic)
    for (int64_t c0 = 0; c0 < m; c0 += cb) {
        int64_t c1 = c0 + cb < m ? c0 + cb : m;
        for (int64_t i = n - 1; i >= 0; --i) {
            double *xi = X + IDX(i, 0, m);
            for (int64_t c = c0; c < c1; ++c) xi[c] = Y[IDX(i, c, m)];
            for (int64_t k = i + 1; k < n; ++k) {
                double lki = L[IDX(k, i, n)];
                if (lki == 0.0) continue;
                const double *xk = X + IDX(k, 0, m);
                for (int64_t c = c0; c < c1; ++c) xi[c] -= lki * xk[c];
            }
            double inv = 1.0 / L[IDX(i, i, n)];
            for (int64_t c = c0; c < c1; ++c) xi[c] *= inv;
        }
    }
}

/* ---- Householder reduction of a full symmetric C to tridiagonal (d, e) ----
 * Step k annihilates C[k+2:, k] with H_k = I - 2 v v^T acting on indices k+1..n-1.
 * The reflectors are kept in V (row k holds v_k, zero-padded) when V != NULL. */
static void householder_tridiag(int64_t n, double *C, double *d, double *e, double *V) {
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    if (V) memset(V, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int64_t k = 0; k + 2 < n; ++k) {
        /* x = C[k+1:, k] read from row k (C is kept fully symmetric) */
        const double *ck = C + IDX(k, 0, n);
        double xnorm2 = 0.0;
        for (int64_t i = k + 1; i < n; ++i) xnorm2 += ck[i] * ck[i];
        double x0 = ck[k + 1];
        double tail2 = xnorm2 - x0 * x0;
        d[k] = ck[k];
        if (tail2 == 0.0) {           /* already tridiagonal in this column */
            e[k] = x0;
            continue;
        }
        double alpha = (x0 >= 0.0) ? -sqrt(xnorm2) : sqrt(xnorm2);
        for (int64_t i = 0; i <= k; ++i) v[i] = 0.0;
        for (int64_t i = k + 1; i < n; ++i) v[i] = ck[i];
        v[k + 1] -= alpha;
        double vn = sqrt(tail2 + v[k + 1] * v[k + 1]);
        for (int64_t i = k + 1; i < n; ++i) v[i] /= vn;
        if (V) memcpy(V + IDX(k, 0, n), v, sizeof(double) * (size_t)n);
        /* p = C22 v, K = v^T p, w = p - K v, C22 -= 2 (v w^T + w v^T) */
#pragma omp parallel for schedule(static)
        for (int64_t i = k + 1; i < n; ++i) {
            const double *ci = C + IDX(i, 0, n);
            double s = 0.0;
            for (int64_t j = k + 1; j < n; ++j) s += ci[j] * v[j];
            p[i] = s;
        }
        double K = 0.0;
        for (int64_t i = k + 1; i < n; ++i) K += v[i] * p[i];
        for (int64_t i = k + 1; i < n; ++i) p[i] -= K * v[i];   /* p now holds w */
#pragma omp parallel for schedule(static)
        for (int64_t i = k + 1; i < n; ++i) {
            double *ci = C + IDX(i, 0, n);
            double vi = v[i], wi = p[i];
            for (int64_t j = k + 1; j < n; ++j) ci[j] -= 2.0 * (vi * p[j] + wi * v[j]);
        }
        e[k] = alpha;
        C[IDX(k, k + 1, n)] = alpha;
        C[IDX(k + 1, k, n)] = alpha;
        for (int64_t i = k + 2; i < n; ++i) { C[IDX(k, i, n)] = 0.0; C[IDX(i, k, n)] = 0.0; }
    }
    if (n >= 2) { d[n - 2] = C[IDX(n - 2, n - 2, n)]; e[n - 2] = C[IDX(n - 2, n - 1, n)]; }
    if (n >= 1) { d[n - 1] = C[IDX(n - 1, n - 1, n)]; e[n - 1] = 0.0; }
    free(p);
    free(v);
}

/* ---- implicit-shift QL on the tridiagonal (d, e[i] couples i and i+1) ----
 * When Zt != NULL the rotations are applied to its rows (row i of Zt = column i of Z). */
static int tridiag_ql(int64_t n, double *d, double *e, double *Zt) {
    const double eps = 2.220446049250313e-16;
    for (int64_t l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int64_t m = l;
            for (; m < n - 1; ++m) {
                double dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) <= eps * dd) break;
            }
            if (m == l) break;
            if (++iter > 200) return 2;
            /* Wilkinson-type shift from the leading 2x2 block at l */
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? fabs(r) : -fabs(r)));
            double s = 1.0, c = 1.0, p = 0.0;
            int64_t i;
            int deflated = 0;
            for (i = m - 1; i >= l; --i) {
                double f = s * e[i];
                double b = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {            /* split: restart from this block */
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    deflated = 1;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                if (Zt) {
                    double *zi = Zt + IDX(i, 0, n), *zj = Zt + IDX(i + 1, 0, n);
                    for (int64_t k = 0; k < n; ++k) {
                        double zf = zj[k];
                        zj[k] = s * zi[k] + c * zf;
                        zi[k] = c * zi[k] - s * zf;
                    }
                }
            }
            if (deflated) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    return 0;
}

/* ---- sort eigenvalues ascending, permuting the rows of Zt alongside ---- */
static void sort_eig(int64_t n, double *d, double *Zt, double *tmp) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i;
        for (int64_t j = i + 1; j < n; ++j) if (d[j] < d[k]) k = j;
        if (k != i) {
            double t = d[i]; d[i] = d[k]; d[k] = t;
            if (Zt) {
                memcpy(tmp, Zt + IDX(i, 0, n), sizeof(double) * (size_t)n);
                memcpy(Zt + IDX(i, 0, n), Zt + IDX(k, 0, n), sizeof(double) * (size_t)n);
                memcpy(Zt + IDX(k, 0, n), tmp, sizeof(double) * (size_t)n);
            }
        }
    }
}

/* Eigenpairs of A x = lambda B x (dense, row-major, symmetric A, SPD B).
 * lam[n] ascending; X (n x n row-major, X[i][j] = component i of vector j) when X != NULL. */
int or_gen_eig(int64_t n, const double *A, const double *B, double *lam, double *X) {
    size_t nn = (size_t)n * (size_t)n;
    double *L = (double *)malloc(sizeof(double) * nn);
    double *W = (double *)malloc(sizeof(double) * nn);
    double *C = (double *)malloc(sizeof(double) * nn);
    double *e = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    int rc = cholesky_lower(n, B, L);
    if (rc) goto done;
    /* C = L^-1 A L^-T = L^-1 (L^-1 A)^T, symmetrised */
    forward_subst(n, n, L, A, W);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) C[IDX(i, j, n)] = W[IDX(j, i, n)];
    forward_subst(n, n, L, C, W);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) C[IDX(i, j, n)] = 0.5 * (W[IDX(i, j, n)] + W[IDX(j, i, n)]);
    if (!X) {
        householder_tridiag(n, C, lam, e, NULL);
        rc = tridiag_ql(n, lam, e, NULL);
        if (!rc) sort_eig(n, lam, NULL, NULL);
        goto done;
    }
    {
        double *V = W; /* reflectors */
        householder_tridiag(n, C, lam, e, V);
        /* Zt = (H_0 H_1 ... H_{n-3})^T, built as Q = H_0 (H_1 (...)) then transposed:
         * rows of Q^T are columns of Q.  Q is formed in C (free now). */
        memset(C, 0, sizeof(double) * nn);
        for (int64_t i = 0; i < n; ++i) C[IDX(i, i, n)] = 1.0;
        for (int64_t k = n - 3; k >= 0; --k) {
            const double *v = V + IDX(k, 0, n);
            /* Q[k+1:, k+1:] <- Q - 2 v (v^T Q) */
            double *vq = (double *)calloc((size_t)n, sizeof(double));
            for (int64_t i = k + 1; i < n; ++i) {
                if (v[i] == 0.0) continue;
                const double *qi = C + IDX(i, 0, n);
                for (int64_t j = k + 1; j < n; ++j) vq[j] += v[i] * qi[j];
            }
#pragma omp parallel for schedule(static)
            for (int64_t i = k + 1; i < n; ++i) {
                double *qi = C + IDX(i, 0, n);
                double vi2 = 2.0 * v[i];
                for (int64_t j = k + 1; j < n; ++j) qi[j] -= vi2 * vq[j];
            }
            free(vq);
        }
        /* Zt = Q^T */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) W[IDX(i, j, n)] = C[IDX(j, i, n)];
        rc = tridiag_ql(n, lam, e, W);
        if (rc) goto done;
        sort_eig(n, lam, W, e);
        /* Y (row-major, column j = eigenvector j of C) = Zt^T, then X = L^-T Y */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) C[IDX(i, j, n)] = W[IDX(j, i, n)];
        backward_subst_t(n, n, L, C, X);
    }
done:
    free(L); free(W); free(C); free(e);
    return rc;
}

/* ---- one eigenvector of the tridiagonal T (diagonal d, off-diagonal e[i] coupling i and
 * i+1) for an eigenvalue estimate theta: inverse iteration y <- (T - theta I)^-1 y with
 * Gaussian elimination with partial pivoting (the row-interchange LU of a tridiagonal
 * matrix: U has a diagonal and two super-diagonals).  Each iterate is orthogonalised
 * against the vectors in prev[0..nprev) (eigenvectors already found for estimates in the
 * same cluster), then normalised.  A zero pivot is replaced by eps * ||T||_1. */
static void tridiag_inverse_iteration(int64_t n, const double *d, const double *e, double theta,
                                      double tnorm, int iters, const double *const *prev, int nprev,
                                      double *y, double *u0, double *u1, double *u2, double *mult,
                                      unsigned char *piv) {
    const double tiny = 2.220446049250313e-16 * (tnorm > 0.0 ? tnorm : 1.0);
    /* factor T - theta I */
    for (int64_t i = 0; i < n; ++i) { u0[i] = d[i] - theta; u1[i] = (i + 1 < n) ? e[i] : 0.0; u2[i] = 0.0; }
    for (int64_t i = 0; i + 1 < n; ++i) {
        const double sub = e[i];                 /* M[i+1][i] */
        if (fabs(sub) > fabs(u0[i])) {           /* swap rows i and i+1 */
            const double m = u0[i] / sub;
            const double r1 = u1[i], r2 = u2[i];     /* old row i at columns i+1, i+2 */
            const double a1 = u0[i + 1], b1 = u1[i + 1];  /* old row i+1 at columns i+1, i+2 */
            u0[i] = sub; u1[i] = a1; u2[i] = b1;
            u0[i + 1] = r1 - m * a1;
            u1[i + 1] = r2 - m * b1;
            mult[i] = m;
            piv[i] = 1;
        } else {
            if (u0[i] == 0.0) u0[i] = tiny;
            const double m = sub / u0[i];
            u0[i + 1] -= m * u1[i];
            u1[i + 1] -= m * u2[i];
            mult[i] = m;
            piv[i] = 0;
        }
    }
    if (u0[n - 1] == 0.0) u0[n - 1] = tiny;
    /* start vector: all ones */
    for (int64_t i = 0; i < n; ++i) y[i] = 1.0;
    for (int it = 0; it < iters; ++it) {
        /* forward: apply the row operations to y */
        for (int64_t i = 0; i + 1 < n; ++i) {
            if (piv[i]) { double t = y[i]; y[i] = y[i + 1]; y[i + 1] = t - mult[i] * y[i]; }
            else y[i + 1] -= mult[i] * y[i];
        }
        /* back substitution with U */
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = y[i];
            if (i + 1 < n) s -= u1[i] * y[i + 1];
            if (i + 2 < n) s -= u2[i] * y[i + 2];
            y[i] = s / u0[i];
        }
        for (int q = 0; q < nprev; ++q) {
            double dot = 0.0;
            for (int64_t i = 0; i < n; ++i) dot += prev[q][i] * y[i];
            for (int64_t i = 0; i < n; ++i) y[i] -= dot * prev[q][i];
        }
        double nrm = 0.0;
        for (int64_t i = 0; i < n; ++i) nrm += y[i] * y[i];
        nrm = sqrt(nrm);
        for (int64_t i = 0; i < n; ++i) y[i] /= nrm;
    }
}

/* The lowest m eigenpairs of A x = lambda B x (dense row-major, symmetric A, SPD B):
 * Cholesky B = L L^T, C = L^-1 A L^-T, Householder tridiagonalisation C = Q T Q^T,
 * eigenvalues of T by implicit QL (ascending), the eigenvector of T for each of the m
 * lowest by inverse iteration (three steps; estimates closer than 1e-3 max(1, |theta|)
 * to the previous one form a cluster whose vectors are orthogonalised), then z = Q y
 * (the reflectors applied in reverse order) and x = L^-T z, so x^T B x = 1.
 * lam[m] (eigenvalues of T, ascending), X (n x m row-major, column j = vector j). */
int or_gen_eig_lowest(int64_t n, const double *A, const double *B, int64_t m, double *lam, double *X) {
    if (m < 1 || m > n) return 4;
    size_t nn = (size_t)n * (size_t)n;
    double *L = (double *)malloc(sizeof(double) * nn);
    double *W = (double *)malloc(sizeof(double) * nn);
    double *C = (double *)malloc(sizeof(double) * nn);
    double *d = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *e = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *th = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *ee = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *Y = NULL;
    int rc = cholesky_lower(n, B, L);
    if (rc) goto done;
    forward_subst(n, n, L, A, W);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) C[IDX(i, j, n)] = W[IDX(j, i, n)];
    forward_subst(n, n, L, C, W);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) C[IDX(i, j, n)] = 0.5 * (W[IDX(i, j, n)] + W[IDX(j, i, n)]);
    householder_tridiag(n, C, d, e, W);           /* W now holds the reflectors */
    memcpy(th, d, sizeof(double) * (size_t)n);
    memcpy(ee, e, sizeof(double) * (size_t)n);
    rc = tridiag_ql(n, th, ee, NULL);
    if (rc) goto done;
    sort_eig(n, th, NULL, NULL);
    {
        double tnorm = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
            if (r > tnorm) tnorm = r;
        }
        /* eigenvectors of T: vector j stored contiguously in C (free now), row j */
        double *u0 = (double *)malloc(sizeof(double) * (size_t)n);
        double *u1 = (double *)malloc(sizeof(double) * (size_t)n);
        double *u2 = (double *)malloc(sizeof(double) * (size_t)n);
        double *mu = (double *)malloc(sizeof(double) * (size_t)n);
        unsigned char *pv = (unsigned char *)malloc((size_t)n);
        const double **prev = (const double **)malloc(sizeof(double *) * (size_t)m);
        int64_t c0 = 0;                          /* first index of the current cluster */
        for (int64_t j = 0; j < m; ++j) {
            if (j > 0 && !(th[j] - th[j - 1] <= 1e-3 * (fabs(th[j]) > 1.0 ? fabs(th[j]) : 1.0))) c0 = j;
            int np = 0;
            for (int64_t q = c0; q < j; ++q) prev[np++] = C + IDX(q, 0, n);
            tridiag_inverse_iteration(n, d, e, th[j], tnorm, 3, prev, np, C + IDX(j, 0, n), u0, u1, u2, mu, pv);
            lam[j] = th[j];
        }
        free(u0); free(u1); free(u2); free(mu); free(pv); free(prev);
        /* Y (n x m row-major) = the vectors of T as columns, then Y <- Q Y with
         * Q = H_0 H_1 ... H_{n-3}: H_{n-3} first */
        Y = (double *)malloc(sizeof(double) * (size_t)n * (size_t)m);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < m; ++j) Y[IDX(i, j, m)] = C[IDX(j, i, n)];
        const int64_t cb = 64;
#pragma omp parallel for schedule(dynamic)
        for (int64_t q0 = 0; q0 < m; q0 += cb) {
            const int64_t q1 = q0 + cb < m ? q0 + cb : m;
            double s[64];
            for (int64_t k = n - 3; k >= 0; --k) {
                const double *v = W + IDX(k, 0, n);
                for (int64_t q = q0; q < q1; ++q) s[q - q0] = 0.0;
                for (int64_t r = k + 1; r < n; ++r) {
                    const double vr = v[r];
                    if (vr == 0.0) continue;
                    const double *yr = Y + IDX(r, 0, m);
                    for (int64_t q = q0; q < q1; ++q) s[q - q0] += vr * yr[q];
                }
                for (int64_t r = k + 1; r < n; ++r) {
                    const double vr2 = 2.0 * v[r];
                    if (vr2 == 0.0) continue;
                    double *yr = Y + IDX(r, 0, m);
                    for (int64_t q = q0; q < q1; ++q) yr[q] -= vr2 * s[q - q0];
                }
            }
        }
        backward_subst_t(n, m, L, Y, X);
    }
done:
    free(L); free(W); free(C); free(d); free(e); free(th); free(ee); free(Y);
    return rc;
}

/* Eigenpairs of a symmetric tridiagonal matrix: diagonal d[m], off-diagonal off[m-1].
 * theta[m] ascending; Z (m x m row-major, column j = eigenvector j) when Z != NULL. */
int or_tridiag_eig(int64_t m, const double *d, const double *off, double *theta, double *Z) {
    double *e = (double *)calloc((size_t)m + 1, sizeof(double));
    double *Zt = Z ? (double *)calloc((size_t)m * (size_t)m, sizeof(double)) : NULL;
    double *tmp = (double *)malloc(sizeof(double) * ((size_t)m + 1));
    for (int64_t i = 0; i < m; ++i) theta[i] = d[i];
    for (int64_t i = 0; i + 1 < m; ++i) e[i] = off[i];
    if (Zt) for (int64_t i = 0; i < m; ++i) Zt[IDX(i, i, m)] = 1.0;
    int rc = tridiag_ql(m, theta, e, Zt);
    if (!rc) {
        sort_eig(m, theta, Zt, tmp);
        if (Z) for (int64_t i = 0; i < m; ++i)
            for (int64_t j = 0; j < m; ++j) Z[IDX(i, j, m)] = Zt[IDX(j, i, m)];
    }
    free(e); free(Zt); free(tmp);
    return rc;
}

/* Dense Bunch-Kaufman LDL^T (partial pivoting, alpha = (1 + sqrt 17)/8) of a symmetric
 * row-major M (overwritten).  Inertia of D is written to inertia[3] = {neg, zero, pos}.
 * Optional outputs: piv_kind[n] (1 = 1x1 pivot, 2 = first row of a 2x2 block, 0 = second
 * row), dvals[2n] (the diagonal then sub-diagonal of the block diagonal D). */
int or_ldlt_bk(int64_t n, double *M, int64_t *inertia, int32_t *piv_kind, double *dvals) {
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;
    int64_t neg = 0, zero = 0, pos = 0;
    if (dvals) memset(dvals, 0, sizeof(double) * 2 * (size_t)n);
#define SWAP_SYM(a, b)                                                                  \
    do {                                                                                \
        if ((a) != (b)) {                                                               \
            for (int64_t t = 0; t < n; ++t) {                                           \
                double x = M[IDX(a, t, n)]; M[IDX(a, t, n)] = M[IDX(b, t, n)]; M[IDX(b, t, n)] = x; \
            }                                                                           \
            for (int64_t t = 0; t < n; ++t) {                                           \
                double x = M[IDX(t, a, n)]; M[IDX(t, a, n)] = M[IDX(t, b, n)]; M[IDX(t, b, n)] = x; \
            }                                                                           \
        }                                                                               \
    } while (0)
    int64_t k = 0;
    while (k < n) {
        double akk = fabs(M[IDX(k, k, n)]);
        int64_t r = k;
        double lam = 0.0;
        for (int64_t i = k + 1; i < n; ++i) {
            double v = fabs(M[IDX(i, k, n)]);
            if (v > lam) { lam = v; r = i; }
        }
        int size = 1;
        if (akk == 0.0 && lam == 0.0) {
            zero++;
            if (piv_kind) piv_kind[k] = 1;
            k += 1;
            continue;
        }
        if (akk < alpha * lam) {
            double sig = 0.0;
            for (int64_t j = k; j < n; ++j) {
                if (j == r) continue;
                double v = fabs(M[IDX(r, j, n)]);
                if (v > sig) sig = v;
            }
            if (akk * sig >= alpha * lam * lam) {
                size = 1;                       /* keep k */
            } else if (fabs(M[IDX(r, r, n)]) >= alpha * sig) {
                size = 1;
                SWAP_SYM(k, r);
            } else {
                size = 2;
                SWAP_SYM(k + 1, r);
            }
        }
        if (size == 1) {
            double d = M[IDX(k, k, n)];
            if (d < 0) neg++; else if (d > 0) pos++; else zero++;
            if (piv_kind) piv_kind[k] = 1;
            if (dvals) dvals[k] = d;
#pragma omp parallel for schedule(static)
            for (int64_t i = k + 1; i < n; ++i) {
                double li = M[IDX(i, k, n)] / d;
                for (int64_t j = k + 1; j <= i; ++j) M[IDX(i, j, n)] -= li * M[IDX(j, k, n)];
            }
            for (int64_t i = k + 1; i < n; ++i) {
                M[IDX(i, k, n)] /= d;
                for (int64_t j = k + 1; j < i; ++j) M[IDX(j, i, n)] = M[IDX(i, j, n)];
            }
            k += 1;
        } else {
            double a = M[IDX(k, k, n)], b = M[IDX(k + 1, k, n)], c = M[IDX(k + 1, k + 1, n)];
            double det = a * c - b * b;
            if (det < 0) { neg++; pos++; }
            else if (det > 0) { if (a + c > 0) pos += 2; else neg += 2; }
            else { zero++; if (a + c > 0) pos++; else if (a + c < 0) neg++; else zero++; }
            if (piv_kind) { piv_kind[k] = 2; piv_kind[k + 1] = 0; }
            if (dvals) { dvals[k] = a; dvals[k + 1] = c; dvals[n + k] = b; }
            /* E^-1 = [c -b; -b a] / det ; trailing -= C E^-1 C^T */
#pragma omp parallel for schedule(static)
            for (int64_t i = k + 2; i < n; ++i) {
                double ci0 = M[IDX(i, k, n)], ci1 = M[IDX(i, k + 1, n)];
                double li0 = (c * ci0 - b * ci1) / det;
                double li1 = (-b * ci0 + a * ci1) / det;
                for (int64_t j = k + 2; j <= i; ++j)
                    M[IDX(i, j, n)] -= li0 * M[IDX(j, k, n)] + li1 * M[IDX(j, k + 1, n)];
            }
            for (int64_t i = k + 2; i < n; ++i) {
                double ci0 = M[IDX(i, k, n)], ci1 = M[IDX(i, k + 1, n)];
                M[IDX(i, k, n)] = (c * ci0 - b * ci1) / det;
                M[IDX(i, k + 1, n)] = (-b * ci0 + a * ci1) / det;
                for (int64_t j = k + 2; j < i; ++j) M[IDX(j, i, n)] = M[IDX(i, j, n)];
            }
            k += 2;
        }
    }
#undef SWAP_SYM
    inertia[0] = neg; inertia[1] = zero; inertia[2] = pos;
    return 0;
}

/* Unpivoted LDL^T of a banded symmetric matrix (lower band, bandwidth bw) held as
 * band[j*(bw+1) + t] = M[j+t][j], t = 0..bw.  The band is overwritten.  inertia[3] =
 * {neg, zero, pos}; min_ratio = min_j |d_j| / max|M_jj| is returned so a caller can
 * tell when a pivot is too small for the sign count to be trusted (returns 3 if a
 * pivot is exactly zero). */
int or_band_ldlt(int64_t n, int64_t bw, double *band, int64_t *inertia, double *min_ratio) {
    int64_t neg = 0, zero = 0, pos = 0;
    const int64_t ld = bw + 1;
    double dmax = 0.0;
    for (int64_t j = 0; j < n; ++j) { double v = fabs(band[j * ld]); if (v > dmax) dmax = v; }
    double rmin = INFINITY;
    int rc = 0;
    for (int64_t j = 0; j < n; ++j) {
        double *cj = band + j * ld;
        double d = cj[0];
        if (d < 0) neg++; else if (d > 0) pos++; else { zero++; rc = 3; continue; }
        double ratio = fabs(d) / dmax;
        if (ratio < rmin) rmin = ratio;
        int64_t tmax = (n - 1 - j) < bw ? (n - 1 - j) : bw;
        /* M[j+i][j+t] -= (M[j+i][j] / d) * M[j+t][j], 1 <= t <= i <= tmax */
#pragma omp parallel for schedule(static) if (tmax > 256)
        for (int64_t t = 1; t <= tmax; ++t) {
            double *ct = band + (j + t) * ld;      /* column j+t: ct[i-t] = M[j+i][j+t] */
            double mt = cj[t];
            if (mt == 0.0) continue;
            double f = mt / d;
            for (int64_t i = t; i <= tmax; ++i) ct[i - t] -= cj[i] * f;
        }
        for (int64_t t = 1; t <= tmax; ++t) cj[t] /= d;
    }
    inertia[0] = neg; inertia[1] = zero; inertia[2] = pos;
    if (min_ratio) *min_ratio = rmin;
    return rc;
}

/* Y = M X for CSR M (n rows) and row-major X (ncols_m x k); Y is n x k row-major. */
void or_csr_mm(int64_t n, const int64_t *rowptr, const int32_t *colind, const double *vals,
               int64_t k, const double *X, double *Y) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double *yi = Y + IDX(i, 0, k);
        for (int64_t c = 0; c < k; ++c) yi[c] = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            double v = vals[p];
            const double *xj = X + IDX(colind[p], 0, k);
            for (int64_t c = 0; c < k; ++c) yi[c] += v * xj[c];
        }
    }
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
