// FP64 matrix products on the FP64 FMA pipe (DFMA), used by the solver's
// GEMM-shaped stages: full->band trailing updates (SYMM, SYR2K), the block
// reflector products, band->full back-transformation and the Newton-Schulz
// step.  All matrices are column-major.  On GB300 the FP64 tensor path
// (DMMA, which cuBLAS's DGEMM uses) peaks near 1.10 TFLOP/s while DFMA
// reaches the FP64 pipe's 1.26 TFLOP/s, so these tiled DFMA kernels are the
// faster FP64 GEMMs on this part.
//
// `work` (doubles) holds split-K partial products; a call splits the
// reduction only while splits * m * n fits in work_elems (pass 0 to never
// split).  Errors are the CUDA launch status.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace gb {

// C (m x n) = alpha op(A) op(B) + beta C; op = 'N' or 'T'; op(A) is m x k.
cudaError_t dfma_gemm(char transa, char transb, int m, int n, int k, double alpha, const double *A, long long lda,
                      const double *B, long long ldb, double beta, double *C, long long ldc, double *work,
                      size_t work_elems, cudaStream_t st);

// side 'L': C (m x n) = alpha S B + beta C, S (m x m) symmetric, lower
// triangle stored; side 'R': C (m x n) = alpha B S + beta C, S (n x n).
cudaError_t dfma_symm(char side, int m, int n, double alpha, const double *S, long long lds, const double *B,
                      long long ldb, double beta, double *C, long long ldc, double *work, size_t work_elems,
                      cudaStream_t st);

// Lower triangle of C (n x n) = alpha (A B^T + B A^T) + beta C; A, B n x k.
cudaError_t dfma_syr2k_lower(int n, int k, double alpha, const double *A, long long lda, const double *B,
                             long long ldb, double beta, double *C, long long ldc, cudaStream_t st);

// Lower triangle of C (n x n) = alpha A^T A + beta C; A is k x n.
cudaError_t dfma_syrk_lower_t(int n, int k, double alpha, const double *A, long long lda, double beta, double *C,
                              long long ldc, cudaStream_t st);

// Complex128 (interleaved re, im): C (m x n) = alpha op(A) op(B) + beta C,
// op(A) = 'N', 'C' (conjugate transpose) or 'H' (A Hermitian, m x m, lower
// triangle stored), op(B) = 'N' or 'C'; lower_only: only the lower triangle
// of C is written, its diagonal made real.  `work` (doubles) holds split-K
// partial products as for dfma_gemm (2 doubles per entry).
cudaError_t dfma_zgemm(char opa, char opb, int m, int n, int k, double2 alpha, const double *A, long long lda,
                       const double *B, long long ldb, double2 beta, double *C, long long ldc, int lower_only,
                       double *work, size_t work_elems, cudaStream_t st);

}  // namespace gb
