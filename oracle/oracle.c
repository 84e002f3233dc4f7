/*
 * Oracle implementation -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain loops in IEEE FP64, compiled with -ffp-contract=off so that every
 * multiply and add rounds separately.  The only parallelism is an OpenMP loop
 * over the independent columns of Z in the back-transformation (columns do not
 * interact under left multiplication, so the arithmetic of each column is the
 * same as in a serial run).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define A_(i, j) A[(size_t)(j) * (size_t)lda + (size_t)(i)]

/* ------------------------------------------------------------------------ */
/* Reflector storage layout of the bulge chase (shared contract with the
 * library; this is the oracle's own plain restatement of it).               */

static int nk_of(int n, int b, int s) { return (n - s + b - 1) / b; }

long long or_hh_count(int n, int b)
{
    if (n < 1 || b < 1) return -1;
    long long c = 0;
    for (int s = 1; s <= n - 1; s++) c += nk_of(n, b, s);
    return c;
}

long long or_hh_index(int n, int b, int s, int k)
{
    if (n < 1 || b < 1 || s < 1 || s > n - 1 || k < 0 || k >= nk_of(n, b, s)) return -1;
    long long idx = 0;
    for (int sp = 1; sp < s; sp++) idx += nk_of(n, b, sp);
    return idx + k;
}

/* ------------------------------------------------------------------------ */
/* Elementary reflectors (Sec. 2: Q_i = I - beta_i v_i v_i^H, here written with
 * LAPACK's names tau for beta_i and v[0] = 1).                              */

int or_larfg_d(int m, double *alpha, double *x, double *tau)
{
    if (m < 0) return -1;
    double ss = 0.0;
    for (int i = 0; i < m; i++) ss += x[i] * x[i];
    if (ss == 0.0) {              /* nothing to annihilate: H = I */
        *tau = 0.0;
        return 0;
    }
    double a = *alpha;
    double nrm = sqrt(a * a + ss);
    double beta = (a >= 0.0) ? -nrm : nrm; /* beta = -sign(alpha) ||[alpha; x]||, sign(0)=+1 */
    *tau = (beta - a) / beta;
    double scal = 1.0 / (a - beta);
    for (int i = 0; i < m; i++) x[i] *= scal;
    *alpha = beta;
    return 0;
}

int or_larfg_z(int m, double complex *alpha, double complex *x, double complex *tau)
{
    if (m < 0) return -1;
    double ss = 0.0;
    for (int i = 0; i < m; i++) ss += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
    double ar = creal(*alpha), ai = cimag(*alpha);
    if (ss == 0.0 && ai == 0.0) { /* already real and nothing below: H = I */
        *tau = 0.0;
        return 0;
    }
    double nrm = sqrt(ar * ar + ai * ai + ss);
    double beta = (ar >= 0.0) ? -nrm : nrm; /* real beta */
    *tau = ((beta - ar) - I * ai) / beta;
    double complex scal = 1.0 / (*alpha - beta);
    for (int i = 0; i < m; i++) x[i] *= scal;
    *alpha = beta;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Two-sided application of one reflector to a dense symmetric/Hermitian
 * matrix: A <- H^H A H, H = I - tau v v^H acting on rows/cols r..r+len-1.   */

static void two_sided_d(int n, double *A, int lda, int r, int len, const double *v, double tau)
{
    if (tau == 0.0) return;
    /* left: rows r.., every column j: A[R,j] -= tau v (v^T A[R,j]) */
    for (int j = 0; j < n; j++) {
        double w = 0.0;
        for (int i = 0; i < len; i++) w += v[i] * A_(r + i, j);
        for (int i = 0; i < len; i++) A_(r + i, j) -= tau * v[i] * w;
    }
    /* right: cols r.., every row i: A[i,R] -= tau (A[i,R] v) v^T */
    for (int i = 0; i < n; i++) {
        double w = 0.0;
        for (int j = 0; j < len; j++) w += A_(i, r + j) * v[j];
        for (int j = 0; j < len; j++) A_(i, r + j) -= tau * w * v[j];
    }
}

static void two_sided_z(int n, double complex *A, int lda, int r, int len,
                        const double complex *v, double complex tau)
{
    if (tau == 0.0) return;
    /* left with H^H = I - conj(tau) v v^H */
    for (int j = 0; j < n; j++) {
        double complex w = 0.0;
        for (int i = 0; i < len; i++) w += conj(v[i]) * A_(r + i, j);
        for (int i = 0; i < len; i++) A_(r + i, j) -= conj(tau) * v[i] * w;
    }
    /* right with H = I - tau v v^H */
    for (int i = 0; i < n; i++) {
        double complex w = 0.0;
        for (int j = 0; j < len; j++) w += A_(i, r + j) * v[j];
        for (int j = 0; j < len; j++) A_(i, r + j) -= tau * w * conj(v[j]);
    }
}

/* ------------------------------------------------------------------------ */
/* Band -> tridiagonal bulge chase (the second step of the two-stage
 * reduction, Sec. 2).  Sweep s removes column s below the sub-diagonal; its
 * k-th reflector starts at row s+1+k*b and annihilates, below that row, the
 * column it was generated from: column s for k = 0, otherwise the first
 * column (s+1+(k-1)*b) of the bulge that the previous reflector created.
 * Working on the dense matrix keeps every step a plain two-sided update.    */

int or_bulge_chase_d(int n, int b, double *A, int lda, double *d, double *e,
                     double *hh_v, double *hh_tau)
{
    if (n < 1) return -1;
    if (b < 1) return -2;
    if (lda < n) return -4;
    double *v = (double *)malloc(sizeof(double) * (size_t)b);
    long long idx = 0;
    for (int s = 1; s <= n - 1; s++) {
        for (int k = 0; k < nk_of(n, b, s); k++, idx++) {
            int r = s + 1 + k * b;            /* 1-based first row */
            int len = n - r + 1 < b ? n - r + 1 : b;
            int c = (k == 0) ? s : s + 1 + (k - 1) * b; /* 1-based source column */
            int r0 = r - 1, c0 = c - 1;       /* 0-based */
            double alpha = A_(r0, c0), tau;
            v[0] = 1.0;
            for (int i = 1; i < len; i++) v[i] = A_(r0 + i, c0);
            or_larfg_d(len - 1, &alpha, v + 1, &tau);
            for (int i = 0; i < b; i++) hh_v[idx * b + i] = (i < len) ? v[i] : 0.0;
            hh_tau[idx] = tau;
            two_sided_d(n, A, lda, r0, len, v, tau);
            if (tau != 0.0) { /* the annihilated entries are exact by construction */
                A_(r0, c0) = alpha;
                A_(c0, r0) = alpha;
                for (int i = 1; i < len; i++) { A_(r0 + i, c0) = 0.0; A_(c0, r0 + i) = 0.0; }
            }
        }
    }
    free(v);
    for (int i = 0; i < n; i++) d[i] = A_(i, i);
    for (int i = 0; i < n - 1; i++) e[i] = A_(i + 1, i);
    return 0;
}

int or_bulge_chase_z(int n, int b, double complex *A, int lda, double *d, double *e,
                     double complex *hh_v, double complex *hh_tau)
{
    if (n < 1) return -1;
    if (b < 1) return -2;
    if (lda < n) return -4;
    double complex *v = (double complex *)malloc(sizeof(double complex) * (size_t)b);
    long long idx = 0;
    for (int s = 1; s <= n - 1; s++) {
        for (int k = 0; k < nk_of(n, b, s); k++, idx++) {
            int r = s + 1 + k * b;
            int len = n - r + 1 < b ? n - r + 1 : b;
            int c = (k == 0) ? s : s + 1 + (k - 1) * b;
            int r0 = r - 1, c0 = c - 1;
            double complex alpha = A_(r0, c0), tau;
            v[0] = 1.0;
            for (int i = 1; i < len; i++) v[i] = A_(r0 + i, c0);
            or_larfg_z(len - 1, &alpha, v + 1, &tau);
            for (int i = 0; i < b; i++) hh_v[idx * b + i] = (i < len) ? v[i] : 0.0;
            hh_tau[idx] = tau;
            two_sided_z(n, A, lda, r0, len, v, tau);
            if (tau != 0.0) {
                A_(r0, c0) = alpha;        /* alpha = beta is real */
                A_(c0, r0) = conj(alpha);
                for (int i = 1; i < len; i++) { A_(r0 + i, c0) = 0.0; A_(c0, r0 + i) = 0.0; }
            }
        }
    }
    free(v);
    for (int i = 0; i < n; i++) d[i] = creal(A_(i, i));
    for (int i = 0; i < n - 1; i++) e[i] = creal(A_(i + 1, i));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The hot path (Sec. 2, two-stage paragraph: every eigenvector of T is
 * transformed by the bulge-chasing reflectors; Sec. 3.1: the non-BLAS part of
 * the back transformation).  Definition: Z <- Q2 Z, applying the reflectors
 * one at a time starting from the last one generated.                        */

int or_trans_ev_d(int n, int b, int nev, const double *hh_v, const double *hh_tau,
                  double *Z, int ldz)
{
    if (n < 1) return -1;
    if (b < 1) return -2;
    if (nev < 0) return -3;
    if (ldz < n) return -7;
    long long total = or_hh_count(n, b);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nev; j++) {
        double *z = Z + (size_t)j * (size_t)ldz;
        long long idx = total;
        for (int s = n - 1; s >= 1; s--) {
            for (int k = nk_of(n, b, s) - 1; k >= 0; k--) {
                idx--; /* idx == or_hh_index(n, b, s, k) */
                int r0 = s + k * b; /* 0-based first row */
                int len = n - r0 < b ? n - r0 : b;
                const double *v = hh_v + idx * b;
                double tau = hh_tau[idx];
                double w = 0.0;
                for (int i = 0; i < len; i++) w += v[i] * z[r0 + i];
                for (int i = 0; i < len; i++) z[r0 + i] -= tau * w * v[i];
            }
        }
    }
    return 0;
}

int or_trans_ev_z(int n, int b, int nev, const double complex *hh_v,
                  const double complex *hh_tau, double complex *Z, int ldz)
{
    if (n < 1) return -1;
    if (b < 1) return -2;
    if (nev < 0) return -3;
    if (ldz < n) return -7;
    long long total = or_hh_count(n, b);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nev; j++) {
        double complex *z = Z + (size_t)j * (size_t)ldz;
        long long idx = total;
        for (int s = n - 1; s >= 1; s--) {
            for (int k = nk_of(n, b, s) - 1; k >= 0; k--) {
                idx--;
                int r0 = s + k * b;
                int len = n - r0 < b ? n - r0 : b;
                const double complex *v = hh_v + idx * b;
                double complex tau = hh_tau[idx];
                double complex w = 0.0;
                for (int i = 0; i < len; i++) w += conj(v[i]) * z[r0 + i];
                for (int i = 0; i < len; i++) z[r0 + i] -= tau * w * v[i];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tridiagonal eigensolver (Sec. 2, Eq. 5) by implicit QL iteration with a
 * Wilkinson shift.  One step on the unreduced block [l, m]: the shift mu is
 * the eigenvalue of the top 2x2 block nearest d[l]; a plane rotation in
 * (m-1, m) is chosen so that its last column is parallel to the last column
 * of T - mu I, and the bulge it creates is chased to the top by rotations in
 * (i, i+1), i = m-2..l, each zeroing T[i+2][i].  Rotations act on rows as
 * [r_i; r_i+1] <- [[c, -s], [s, c]] [r_i; r_i+1] and on columns (and Z) by the
 * transpose.                                                                  */

static void rot_block(double *a, double *f, double *cc, double c, double s)
{
    double A = *a, F = *f, C = *cc;
    *a = c * c * A - 2.0 * c * s * F + s * s * C;
    *cc = s * s * A + 2.0 * c * s * F + c * c * C;
    *f = c * s * A + (c * c - s * s) * F - c * s * C;
}

int or_tridiag_ql(int n, double *d, double *e, double *Z, int ldz)
{
    if (n < 1) return -1;
    if (ldz < n) return -5;
    const double eps = 0x1p-53;
    int l = 0, iter = 0;
    while (l < n - 1) {
        int m = l;
        while (m < n - 1) {
            if (fabs(e[m]) <= eps * (fabs(d[m]) + fabs(d[m + 1]))) { e[m] = 0.0; break; }
            m++;
        }
        if (m == l) { l++; iter = 0; continue; }
        if (++iter > 60) return 1 + l;
        /* Wilkinson shift from the top 2x2 block */
        double a = d[l], bb = e[l], c2 = d[l + 1];
        double delta = 0.5 * (c2 - a);
        double root = sqrt(delta * delta + bb * bb);
        double mu = a - bb * bb / (delta + (delta >= 0.0 ? root : -root));
        double bulge = 0.0;
        for (int i = m - 1; i >= l; i--) {
            double x, y;
            if (i == m - 1) { x = d[m] - mu; y = e[m - 1]; }
            else            { x = e[i + 1]; y = bulge; }
            double r = sqrt(x * x + y * y);
            double c, s;
            if (r == 0.0) { c = 1.0; s = 0.0; } else { c = x / r; s = y / r; }
            if (i < m - 1) e[i + 1] = r;          /* T[i+2][i+1] <- s p + c g */
            rot_block(&d[i], &e[i], &d[i + 1], c, s);
            if (i > l) {                           /* column i-1 entries */
                double h = e[i - 1];
                e[i - 1] = c * h;
                bulge = s * h;                     /* new T[i+1][i-1] */
            }
            double *zi = Z + (size_t)i * ldz, *zj = Z + (size_t)(i + 1) * ldz;
            for (int q = 0; q < n; q++) {
                double p = zi[q], t = zj[q];
                zi[q] = c * p - s * t;
                zj[q] = s * p + c * t;
            }
        }
    }
    /* ascending order (selection sort, swapping eigenvector columns) */
    for (int i = 0; i < n - 1; i++) {
        int mn = i;
        for (int j = i + 1; j < n; j++) if (d[j] < d[mn]) mn = j;
        if (mn != i) {
            double t = d[i]; d[i] = d[mn]; d[mn] = t;
            double *zi = Z + (size_t)i * ldz, *zj = Z + (size_t)mn * ldz;
            for (int q = 0; q < n; q++) { t = zi[q]; zi[q] = zj[q]; zj[q] = t; }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cyclic Jacobi (used as brute force for n <= 64).  Each rotation in plane
 * (p, q) is the symmetric Schur decomposition of the 2x2 block
 * [[A_pp, A_pq], [A_pq, A_qq]]: theta = (A_qq - A_pp) / (2 A_pq),
 * t = sign(theta) / (|theta| + sqrt(1 + theta^2)), c = 1/sqrt(1+t^2), s = t c,
 * J = [[c, s], [-s, c]] in (p, q), A <- J^T A J, V <- V J.                    */

int or_jacobi_d(int n, double *A, int lda, double *w, double *V, int ldv)
{
    if (n < 1 || n > 64) return -1;
    if (lda < n) return -3;
    if (ldv < n) return -6;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) V[(size_t)j * ldv + i] = (i == j) ? 1.0 : 0.0;
    int sweep;
    for (sweep = 0; sweep < 100; sweep++) {
        int rotated = 0;
        for (int p = 0; p < n - 1; p++) {
            for (int q = p + 1; q < n; q++) {
                double apq = A_(p, q);
                /* skip entries already negligible next to their diagonal */
                if (apq == 0.0 || fabs(apq) <= 0x1p-53 * sqrt(fabs(A_(p, p)) * fabs(A_(q, q))))
                    continue;
                rotated = 1;
                double theta = (A_(q, q) - A_(p, p)) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; k++) { /* columns p, q: A <- A J */
                    double akp = A_(k, p), akq = A_(k, q);
                    A_(k, p) = c * akp - s * akq;
                    A_(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) { /* rows p, q: A <- J^T A */
                    double apk = A_(p, k), aqk = A_(q, k);
                    A_(p, k) = c * apk - s * aqk;
                    A_(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = V[(size_t)p * ldv + k], vkq = V[(size_t)q * ldv + k];
                    V[(size_t)p * ldv + k] = c * vkp - s * vkq;
                    V[(size_t)q * ldv + k] = s * vkp + c * vkq;
                }
            }
        }
        if (!rotated) break;
    }
    if (sweep == 100) return 1;
    for (int i = 0; i < n; i++) w[i] = A_(i, i);
    for (int i = 0; i < n - 1; i++) { /* ascending order */
        int mn = i;
        for (int j = i + 1; j < n; j++) if (w[j] < w[mn]) mn = j;
        if (mn != i) {
            double t = w[i]; w[i] = w[mn]; w[mn] = t;
            for (int k = 0; k < n; k++) {
                t = V[(size_t)i * ldv + k];
                V[(size_t)i * ldv + k] = V[(size_t)mn * ldv + k];
                V[(size_t)mn * ldv + k] = t;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One-stage Householder tridiagonalisation (Sec. 2, Eq. 4) and its
 * back-transformation (Eq. 6).  Used to build and check end-to-end cases. */

int or_sytrd_d(int n, double *A, int lda, double *d, double *e, double *v, int ldv,
               double *tau)
{
    if (n < 1) return -1;
    if (lda < n) return -3;
    if (ldv < n) return -7;
    for (int j = 0; j < n - 1; j++) {
        double *vj = v + (size_t)j * ldv;
        for (int i = 0; i < n; i++) vj[i] = 0.0;
        tau[j] = 0.0;
    }
    for (int i = 0; i + 1 < n; i++) {
        int r0 = i + 1, len = n - r0;
        double *vi = v + (size_t)i * ldv;
        double alpha = A_(r0, i), t;
        vi[r0] = 1.0;
        for (int q = 1; q < len; q++) vi[r0 + q] = A_(r0 + q, i);
        or_larfg_d(len - 1, &alpha, vi + r0 + 1, &t);
        tau[i] = t;
        two_sided_d(n, A, lda, r0, len, vi + r0, t);
        if (t != 0.0) {
            A_(r0, i) = alpha; A_(i, r0) = alpha;
            for (int q = 1; q < len; q++) { A_(r0 + q, i) = 0.0; A_(i, r0 + q) = 0.0; }
        }
    }
    for (int i = 0; i < n; i++) d[i] = A_(i, i);
    for (int i = 0; i < n - 1; i++) e[i] = A_(i + 1, i);
    return 0;
}

int or_sytrd_apply_d(int n, int nev, const double *v, int ldv, const double *tau,
                     double *Z, int ldz)
{
    if (n < 1) return -1;
    if (nev < 0) return -2;
    if (ldv < n) return -4;
    if (ldz < n) return -7;
    for (int j = 0; j < nev; j++) {
        double *z = Z + (size_t)j * ldz;
        for (int i = n - 2; i >= 0; i--) {
            const double *vi = v + (size_t)i * ldv;
            double w = 0.0;
            for (int q = i + 1; q < n; q++) w += vi[q] * z[q];
            for (int q = i + 1; q < n; q++) z[q] -= tau[i] * w * vi[q];
        }
    }
    return 0;
}
