/*
 * Oracle for the two-stage symmetric/Hermitian eigensolver's back-transformation
 * from tridiagonal to band form (trans_ev_tridi_to_band) and its companion steps.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct CPU
 * implementation in IEEE FP64 (built with -ffp-contract=off).  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * The product path (the CUDA library) never calls, links or includes it, and
 * it shares no code with that path.
 *
 * Paper: Kus et al., "Optimizations of the Eigensolvers in the ELPA Library",
 * Sec. 2 (Eqs. 4-6 and the two-stage paragraph) and Sec. 3.1 (the non-BLAS
 * back-transformation kernel).
 *
 * Conventions (all column-major, 1-based sweep index s, 0-based block index k):
 *   - Sweep s = 1..n-1 of the band->tridiagonal bulge chase emits
 *     nk(s) = ceil((n-s)/b) reflectors H(s,k), k = 0..nk(s)-1.
 *   - H(s,k) = I - tau * v * v^H acts on rows s+1+k*b .. min(s+(k+1)*b, n)
 *     (1-based), i.e. len(s,k) = min(b, n-s-k*b) rows; v[0] = 1.
 *   - Storage: reflector index idx(s,k) = sum_{s'<s} nk(s') + k;
 *     hh_v[idx*b + i] holds v[i] for i < len (v[0] stored as 1.0) and 0 for
 *     len <= i < b; hh_tau[idx] holds tau.
 *   - Q2 = H(1,0) H(1,1) ... H(1,nk(1)-1) H(2,0) ... H(n-1,0) (generation
 *     order) and T = Q2^H B Q2; the back-transformation is Z <- Q2 Z.
 *
 * Every function returns 0 on success and a negative value for an invalid
 * argument (-i: argument i) or a positive value when an iteration fails to
 * converge.
 */
#ifndef ELPA_ORACLE_H
#define ELPA_ORACLE_H

#include <complex.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of reflectors a bulge chase of an n x n band matrix with b
 * super-diagonals emits, and the storage index of H(s,k). */
long long or_hh_count(int n, int b);
long long or_hh_index(int n, int b, int s, int k);

/* Elementary reflector in LAPACK form.  On entry *alpha and x[0..m-1] hold the
 * vector [alpha; x]; on exit *alpha = beta, x holds v[1..m] (v[0] = 1) and
 * *tau is set so that H^H [alpha; x] = [beta; 0] with H = I - tau v v^H. */
int or_larfg_d(int m, double *alpha, double *x, double *tau);
int or_larfg_z(int m, double complex *alpha, double complex *x, double complex *tau);

/* Band -> tridiagonal bulge chase on a dense symmetric (Hermitian) matrix A
 * whose entries beyond b off-diagonals are zero.  A is overwritten by T;
 * d (n) and e (n-1) receive T's diagonal and sub-diagonal (real); the
 * reflectors are written in the storage layout above. */
int or_bulge_chase_d(int n, int b, double *A, int lda, double *d, double *e,
                     double *hh_v, double *hh_tau);
int or_bulge_chase_z(int n, int b, double complex *A, int lda, double *d, double *e,
                     double complex *hh_v, double complex *hh_tau);

/* The hot path's definition: Z <- Q2 Z on nev columns (Z is n x nev, ldz). */
int or_trans_ev_d(int n, int b, int nev, const double *hh_v, const double *hh_tau,
                  double *Z, int ldz);
int or_trans_ev_z(int n, int b, int nev, const double complex *hh_v,
                  const double complex *hh_tau, double complex *Z, int ldz);

/* Implicit QL with Wilkinson shift on the symmetric tridiagonal (d, e).
 * Z (n x n, ldz) is post-multiplied by the accumulated rotations (pass the
 * identity to get T's eigenvectors).  On exit d holds the eigenvalues in
 * ascending order with Z's columns permuted to match. */
int or_tridiag_ql(int n, double *d, double *e, double *Z, int ldz);

/* Cyclic Jacobi on a dense symmetric A (n <= 64): eigenvalues w ascending,
 * eigenvectors in V.  A is destroyed. */
int or_jacobi_d(int n, double *A, int lda, double *w, double *V, int ldv);

/* One-stage Householder tridiagonalisation (Sec. 2, Eq. 4): A <- Q^T A Q with
 * Q = Q_1 Q_2 ... Q_{n-2}; reflector i (0-based) acts on rows i+1..n-1 and is
 * stored in v (n x (n-1), column i, v[i+1] = 1) and tau[i].  Then
 * or_sytrd_apply_d computes Z <- Q Z (Eq. 6). */
int or_sytrd_d(int n, double *A, int lda, double *d, double *e, double *v, int ldv,
               double *tau);
int or_sytrd_apply_d(int n, int nev, const double *v, int ldv, const double *tau,
                     double *Z, int ldz);

#ifdef __cplusplus
}
#endif
#endif
