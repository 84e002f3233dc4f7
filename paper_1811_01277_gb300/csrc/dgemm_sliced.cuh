// FP64 matrix products on the bf16 tensor cores by exact digit slicing (the
// error-free splitting idea of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59 (2012), in its fixed-point form).
//
// Every row of op(A) and every column of op(B) is scaled by a power of two
// so that its largest entry is below one, and each entry's magnitude is cut
// into kSlices digits of kDigitBits bits (|digit| <= 127, all digits carry
// the entry's sign).  Digit t is stored as the bf16 value d * 2^(-7t), which
// bf16 holds exactly.  The product of digit planes i (of A) and j (of B) is
// an exact multiple of 2^(-7(i+j)) and lands in "level" i+j.  Pairs with
// i+j <= 8 are formed; the rest lie 2^-62 below the scaled row/column
// maxima, and digits are cut from the magnitude rounded to nearest, so the
// errors stay unbiased and grow like sqrt(k) even in sums of one sign.  Every level has its own FP32 tensor-core
// accumulator; over kFlushK consecutive k its sum is an integer multiple of
// 2^(-7 level) below 2^24 units (kSlices * 127^2 * kFlushK < 2^24), so it is
// exact, and it is folded into two 64-bit integers per output every kFlushK.
// The result is rounded to FP64 once, at the end.  (A shared FP32
// accumulator for the low levels is not enough: its truncating additions
// reach 2^-46 of the result on sums of one sign.)
//
// Accuracy is that of an FP64 product measured against the scaled maxima:
// |C - AB| <~ 2^-53 k max_j|a_ij| max_i|b_ij| per entry.  Inputs must be
// finite; subnormal inputs are read as zero.
//
// FP32 products (digits = kSplitPlanes): every entry is rounded to FP32 and
// split exactly into three bf16 parts h0 + h1 + h2 with their own
// exponents (no row scaling); the pairs i + j <= 2 (six products per k16
// step) accumulate in one FP32 tensor-core accumulator, folded into FP64
// every kFlushK.  The error is that of an FP32 product: about 2^-24 of
// sum_k |a_ik b_kj| from the rounding to FP32 and the dropped pairs, plus
// the FP32 accumulation over kFlushK terms.  This is the low-precision half
// of the mixed-precision solve.
//
// A sliced operand is an R x K "slice-row" matrix; its rows are the rows of
// op(A) (for the left operand) or the columns of op(B) (for the right).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace gb {

constexpr int kSlices = 8;
constexpr int kLevels = 9;  // digit pairs i + j <= 8 are formed
constexpr int kDigitBits = 7;
constexpr int kFlushK = 128;
constexpr int kSplitPlanes = 3;  // `digits` value of the FP32 split

// How a slice-row matrix reads a column-major FP64 source `src` (leading
// dimension ld): element (r, k) is
//   kViewRow: src[r + k ld]     (slice rows are the source's rows)
//   kViewCol: src[k + r ld]     (slice rows are the source's columns)
//   kViewSym: the symmetric matrix whose lower triangle src holds.
// Complex sources (interleaved re, im; ld in complex elements).  A complex
// product C = op(A) B is the real product of the expanded op(A), whose
// entry a = x + iy becomes the 2 x 2 block [x -y; y x], with B and C read
// as real matrices of twice the rows (their interleaved storage as is):
//   kViewZExpandN:   expanded A (2 rows x 2 columns per complex entry)
//   kViewZExpandC:   expanded A^H
//   kViewZHermExpand: expanded Hermitian matrix whose lower triangle src
//                    holds (the diagonal's imaginary part read as zero)
//   kViewZRowConj:   row r of the real form of B^H for a complex B with
//                    rows r: element (r, 2k + c) = c ? -Im B(r, k) : Re B(r, k)
enum SliceView {
    kViewRow = 0,
    kViewCol = 1,
    kViewSym = 2,
    kViewZExpandN = 3,
    kViewZExpandC = 4,
    kViewZHermExpand = 5,
    kViewZRowConj = 6
};

struct SlicedOp {
    const uint16_t *planes;  // digits planes of Rp x Kp bf16, row-major (k fastest)
    const int *e;            // Rp row exponents: the row's entries are below 2^e
    int R, K, Rp, Kp;        // Rp: R rounded up to 64; Kp: K rounded up to 32
    int digits;              // kSlices digit planes, or kSplitPlanes (the FP32 split)
};

// Bytes a sliced R x K operand occupies (planes, exponents and a reduction
// scratch), 256-byte multiple.
size_t sliced_bytes(int R, int K);

// Slices an R x K view of src into buf (sliced_bytes(R, K) bytes, 256-byte
// aligned); fills *out.  Two launches and a memset on st.  `digits`:
// kSlices (the FP64-accurate digits) or kSplitPlanes (the FP32 split; both
// operands of a product must then be split).
cudaError_t slice_matrix(SliceView view, int R, int K, const double *src, long long ld, void *buf, SlicedOp *out,
                         cudaStream_t st, int digits = kSlices);

// Which part of C a product writes.
enum SlicedFill {
    kFillAll = 0,
    kFillLower = 1,       // entries r >= c
    kFillZLower = 2,      // C is the real form of a complex matrix (rows 2r, 2r+1 = re, im of
                          // complex row r): complex entries r >= c, diagonal imaginary parts zeroed
};

// C (m x n, column-major) = alpha A B^T + beta C where A, B are sliced
// (A.R >= m, B.R >= n, A.K == B.K): row r of A times row c of B; `fill`
// selects the entries written.  Both operands split: the FP32 product.  `work` (doubles) holds split-K partials; the
// reduction splits while splits * m * n <= work_elems.
cudaError_t sliced_gemm(const SlicedOp &A, const SlicedOp &B, int m, int n, double alpha, double beta, double *C,
                        long long ldc, int fill, double *work, size_t work_elems, cudaStream_t st);

// Whole products (slice both operands into ws, multiply), with the DFMA
// forms' conventions (dgemm_dfma.cuh); ws must hold the matching *_ws_bytes.
// `digits` as for slice_matrix (kSlices: FP64 accuracy).
size_t sliced_gemm_ws_bytes(int m, int n, int k);
size_t sliced_symm_ws_bytes(char side, int m, int n);
size_t sliced_syr2k_ws_bytes(int n, int k);
size_t sliced_syrk_ws_bytes(int n, int k);
cudaError_t sliced_dgemm(char transa, char transb, int m, int n, int k, double alpha, const double *A, long long lda,
                         const double *B, long long ldb, double beta, double *C, long long ldc, void *ws,
                         cudaStream_t st, int digits = kSlices);
cudaError_t sliced_dsymm(char side, int m, int n, double alpha, const double *S, long long lds, const double *B,
                         long long ldb, double beta, double *C, long long ldc, void *ws, cudaStream_t st,
                         int digits = kSlices);
cudaError_t sliced_dsyr2k_lower(int n, int k, double alpha, const double *A, long long lda, const double *B,
                                long long ldb, double beta, double *C, long long ldc, void *ws, cudaStream_t st,
                                int digits = kSlices);
cudaError_t sliced_dsyrk_lower_t(int n, int k, double alpha, const double *A, long long lda, double beta, double *C,
                                 long long ldc, void *ws, cudaStream_t st, int digits = kSlices);

// Complex (interleaved) products with real alpha, beta; lda etc. in complex
// elements.  C (m x n) = alpha op(A) B + beta C, op = 'N' or 'C'.
size_t sliced_zgemm_ws_bytes(int m, int n, int k);
cudaError_t sliced_zgemm(char transa, int m, int n, int k, double alpha, const double *A, long long lda,
                         const double *B, long long ldb, double beta, double *C, long long ldc, void *ws,
                         cudaStream_t st);
// C (m x n) = alpha S B + beta C, S Hermitian (lower triangle stored).
size_t sliced_zhemm_ws_bytes(int m, int n);
cudaError_t sliced_zhemm_left(int m, int n, double alpha, const double *S, long long lds, const double *B,
                              long long ldb, double beta, double *C, long long ldc, void *ws, cudaStream_t st);
// Lower triangle of C (n x n) = alpha (X Y^H + Y X^H) + beta C, X, Y n x k;
// the diagonal's imaginary parts are set to zero.
size_t sliced_zher2k_ws_bytes(int n, int k);
cudaError_t sliced_zher2k_lower(int n, int k, double alpha, const double *X, long long ldx, const double *Y,
                                long long ldy, double beta, double *C, long long ldc, void *ws, cudaStream_t st);

}  // namespace gb
