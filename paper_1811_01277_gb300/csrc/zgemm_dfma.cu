// Complex128 matrix products on the FP64 FMA pipe, for the complex solver's
// panel products (b x b results over long reductions, tall m x b results
// over short ones) and for its large products where the sliced tensor-core
// form does not pay (small n, or GB_SOLVE_DFMA_PRODUCTS):
//     C (m x n) = alpha op(A) op(B) + beta C,
// op(A) in {N, C (conjugate transpose), H (A Hermitian, lower triangle
// stored)}, op(B) in {N, C}; the result either full or only its lower
// triangle (with the diagonal's imaginary part set to zero: the Hermitian
// rank-2k update).  Column-major, interleaved (re, im).
//
// One 256-thread block per 32 x 32 tile of C, 2 x 2 complex accumulators per
// thread (rows ty + 16 i, columns tx + 16 j: the shared-memory reads are
// broadcasts along ty and consecutive along tx), K in steps of 16 staged in
// shared memory.  When the output has too few tiles to fill the GPU the
// reduction is split: partial tiles go to `work` and one pass adds them in
// a fixed order, so results do not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dgemm_dfma.cuh"

namespace gb {

namespace {

constexpr int kZT = 32;   // tile of C
constexpr int kZK = 16;   // K step

__device__ __forceinline__ double2 zfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// op(A)(r, kk)
__device__ __forceinline__ double2 load_a(char opa, const double2 *A, long long lda, int r, int kk)
{
    if (opa == 'N') return A[r + (long long)kk * lda];
    if (opa == 'C') return zconj(A[kk + (long long)r * lda]);
    // Hermitian, lower triangle stored
    return r >= kk ? A[r + (long long)kk * lda] : zconj(A[kk + (long long)r * lda]);
}

__device__ __forceinline__ double2 load_b(char opb, const double2 *B, long long ldb, int kk, int c)
{
    return opb == 'N' ? B[kk + (long long)c * ldb] : zconj(B[c + (long long)kk * ldb]);
}

// out != nullptr: partial tile (split s of `splits`) to out[s][m][n];
// else C = alpha acc + beta C (lower: only r >= c, real diagonal)
__global__ void __launch_bounds__(256) zgemm_tile(char opa, char opb, int m, int n, int k, int kchunk, double2 alpha,
                                                  const double2 *__restrict__ A, long long lda,
                                                  const double2 *__restrict__ B, long long ldb, double2 beta,
                                                  double2 *__restrict__ C, long long ldc, int lower,
                                                  double2 *__restrict__ out)
{
    __shared__ double2 As[kZK][kZT + 1];
    __shared__ double2 Bs[kZK][kZT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * kZT, n0 = blockIdx.x * kZT;
    if (lower && n0 > m0 + kZT - 1) return;   // tile wholly above the diagonal
    const int k0 = blockIdx.z * kchunk, k1 = min(k, k0 + kchunk);
    double2 acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) acc[i][j] = make_double2(0.0, 0.0);
    for (int kt = k0; kt < k1; kt += kZK) {
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
            const int e = threadIdx.x + 256 * rr;
            // A: consecutive threads along the rows for N, along k otherwise
            const int ar = opa == 'N' ? e % kZT : e / kZK, ak = opa == 'N' ? e / kZT : e % kZK;
            const int r = m0 + ar, kk = kt + ak;
            As[ak][ar] = (r < m && kk < k1) ? load_a(opa, A, lda, r, kk) : make_double2(0.0, 0.0);
            // B: consecutive threads along k for N, along the columns for C
            const int bc = opb == 'N' ? e / kZK : e % kZT, bk = opb == 'N' ? e % kZK : e / kZT;
            const int c = n0 + bc, kb = kt + bk;
            Bs[bk][bc] = (c < n && kb < k1) ? load_b(opb, B, ldb, kb, c) : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kZK; kk++) {
            const double2 a0 = As[kk][ty], a1 = As[kk][ty + 16];
            const double2 b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = zfma(a0, b0, acc[0][0]);
            acc[0][1] = zfma(a0, b1, acc[0][1]);
            acc[1][0] = zfma(a1, b0, acc[1][0]);
            acc[1][1] = zfma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int r = m0 + ty + 16 * i, c = n0 + tx + 16 * j;
            if (r >= m || c >= n) continue;
            if (out) {
                out[((size_t)blockIdx.z * m + r) * n + c] = acc[i][j];
            } else {
                if (lower && r < c) continue;
                double2 *cp = C + r + (long long)c * ldc;
                double2 v = zmul(alpha, acc[i][j]);
                if (beta.x != 0.0 || beta.y != 0.0) {
                    const double2 old = *cp;
                    v.x += beta.x * old.x - beta.y * old.y;
                    v.y += beta.x * old.y + beta.y * old.x;
                }
                if (lower && r == c) v.y = 0.0;
                *cp = v;
            }
        }
}

__global__ void zgemm_reduce(int m, int n, int splits, double2 alpha, const double2 *__restrict__ part, double2 beta,
                             double2 *__restrict__ C, long long ldc, int lower)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m * n) return;
    const int r = (int)(idx / n), c = (int)(idx % n);
    if (lower && r < c) return;
    double2 s = make_double2(0.0, 0.0);
    for (int z = 0; z < splits; z++) {
        const double2 p = part[((size_t)z * m + r) * n + c];
        s.x += p.x;
        s.y += p.y;
    }
    double2 *cp = C + r + (long long)c * ldc;
    double2 v = zmul(alpha, s);
    if (beta.x != 0.0 || beta.y != 0.0) {
        const double2 old = *cp;
        v.x += beta.x * old.x - beta.y * old.y;
        v.y += beta.x * old.y + beta.y * old.x;
    }
    if (lower && r == c) v.y = 0.0;
    *cp = v;
}

}  // namespace

cudaError_t dfma_zgemm(char opa, char opb, int m, int n, int k, double2 alpha, const double *A, long long lda,
                       const double *B, long long ldb, double2 beta, double *C, long long ldc, int lower_only,
                       double *work, size_t work_elems, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((n + kZT - 1) / kZT, (m + kZT - 1) / kZT, 1);
    const long long tiles = (long long)grid.x * grid.y;
    // split the reduction while the tiles alone cannot fill two blocks per SM
    int splits = 1;
    if (k > 0) {
        const long long want = (2 * 152 + tiles - 1) / tiles;
        const long long by_k = k / 256 > 0 ? k / 256 : 1;
        const long long by_ws = work ? (long long)(work_elems / 2 / ((size_t)m * n)) : 1;
        long long s = want < by_k ? want : by_k;
        s = s < by_ws ? s : by_ws;
        splits = s > 1 ? (int)s : 1;
    }
    const int kchunk = k > 0 ? ((k + splits - 1) / splits + kZK - 1) / kZK * kZK : kZK;
    if (splits == 1) {
        zgemm_tile<<<grid, 256, 0, st>>>(opa, opb, m, n, k, kchunk, alpha, (const double2 *)A, lda, (const double2 *)B,
                                         ldb, beta, (double2 *)C, ldc, lower_only, nullptr);
        return cudaGetLastError();
    }
    // the partial tiles cover the whole output (lower-only tiles are skipped
    // and never read: the reduction skips those entries too)
    grid.z = splits;
    zgemm_tile<<<grid, 256, 0, st>>>(opa, opb, m, n, k, kchunk, alpha, (const double2 *)A, lda, (const double2 *)B, ldb,
                                     beta, (double2 *)C, ldc, lower_only, (double2 *)work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long total = (long long)m * n;
    zgemm_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(m, n, splits, alpha, (const double2 *)work, beta,
                                                                  (double2 *)C, ldc, lower_only);
    return cudaGetLastError();
}

}  // namespace gb
