// One step of Ogita and Aishima's iterative refinement of a full symmetric
// eigendecomposition (the FP64 refinement the mixed-precision configuration
// pairs with a low-precision solve): for A (n x n, symmetric) and approximate
// eigenvectors X (n x n),
//     R = I - X^T X,  S = X^T A X,  lambda_i = s_ii / (1 - r_ii),
//     delta = 2 (||S - diag(lambda)|| + ||A|| ||R||),
//     E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)  if |lambda_i - lambda_j| > delta,
//            r_ij / 2                                          otherwise,
//     X <- X + X E.
// The error of X falls quadratically while eigenvalues are separated by more
// than delta; inside a cluster the step refines the cluster's invariant
// subspace.  The three n^3 products (X^T X, A X, X^T (A X)) and X E run
// sliced on the bf16 tensor cores (FP64-accurate products); ||A||_2 is taken
// as max |lambda_i| and the other spectral norms are bounded by Frobenius
// norms.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dgemm_sliced.cuh"
#include "elpa_gb300.h"

namespace gb {

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kNormBlocks = 152 * 4;

struct RefWs {
    double *G, *W, *S, *E, *lam, *norms, *part;
    void *sl;
    size_t total;
};

RefWs ref_carve(int n, char *base)
{
    RefWs w{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    const size_t nn = (size_t)n * n * 8;
    w.G = (double *)take(nn);
    w.W = (double *)take(nn);
    w.S = (double *)take(nn);
    w.E = (double *)take(nn);
    w.lam = (double *)take((size_t)n * 8);
    w.norms = (double *)take(64);
    w.part = (double *)take((size_t)3 * kNormBlocks * 8);
    size_t s = sliced_gemm_ws_bytes(n, n, n);
    s = s > sliced_symm_ws_bytes('L', n, n) ? s : sliced_symm_ws_bytes('L', n, n);
    s = s > sliced_syrk_ws_bytes(n, n) ? s : sliced_syrk_ws_bytes(n, n);
    w.sl = take(s);
    w.total = off;
    return w;
}

// lambda_i = s_ii / g_ii (g = X^T X, so 1 - r_ii = g_ii)
__global__ void ref_lambda(int n, const double *__restrict__ S, const double *__restrict__ G, double *__restrict__ lam)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) lam[i] = S[i + (size_t)i * n] / G[i + (size_t)i * n];
}

// Per block: partial sums over the lower triangle (off-diagonal entries
// counted twice) of (s_ij - lambda_i delta_ij)^2 and of r_ij^2, and the
// largest |lambda_i|, into part[3 b ..]; ref_norms_final adds the blocks'
// partials in a fixed order into norms[0..2].
__global__ void __launch_bounds__(256) ref_norms(int n, const double *__restrict__ S, const double *__restrict__ G,
                                                 const double *__restrict__ lam, double *__restrict__ part)
{
    __shared__ double red[3][8];
    double s2 = 0.0, r2 = 0.0, lm = 0.0;
    const long long total = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(idx / n), i = (int)(idx - (long long)j * n);
        if (i < j) continue;
        const double w = i == j ? 1.0 : 2.0;
        const double sv = S[i + (size_t)j * n] - (i == j ? lam[i] : 0.0);
        const double rv = (i == j ? 1.0 : 0.0) - G[i + (size_t)j * n];
        s2 += w * sv * sv;
        r2 += w * rv * rv;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        lm = fmax(lm, fabs(lam[i]));
    for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        r2 += __shfl_down_sync(0xffffffffu, r2, o);
        lm = fmax(lm, __shfl_down_sync(0xffffffffu, lm, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = s2;
        red[1][w] = r2;
        red[2][w] = lm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
            a += red[0][k];
            b += red[1][k];
            c = fmax(c, red[2][k]);
        }
        part[3 * blockIdx.x] = a;
        part[3 * blockIdx.x + 1] = b;
        part[3 * blockIdx.x + 2] = c;
    }
}

__global__ void ref_norms_final(int blocks, const double *__restrict__ part, double *__restrict__ norms)
{
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int k = 0; k < blocks; k++) {
        a += part[3 * k];
        b += part[3 * k + 1];
        c = fmax(c, part[3 * k + 2]);
    }
    norms[0] = a;
    norms[1] = b;
    norms[2] = c;
}

// E from S (full, symmetric up to rounding: the lower triangle is used for
// both halves), R = I - G (lower triangle of G), lambda and delta
__global__ void ref_correction(int n, const double *__restrict__ S, const double *__restrict__ G,
                               const double *__restrict__ lam, const double *__restrict__ norms,
                               double *__restrict__ E)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int j = (int)(idx / n), i = (int)(idx - (long long)j * n);
    const int lo = i > j ? i : j, hi = i > j ? j : i;  // (lo, hi) in the lower triangle
    const double s = S[lo + (size_t)hi * n];
    const double r = (i == j ? 1.0 : 0.0) - G[lo + (size_t)hi * n];
    const double delta = 2.0 * (sqrt(norms[0]) + norms[2] * sqrt(norms[1]));
    const double li = lam[i], lj = lam[j];
    double e;
    if (i != j && fabs(li - lj) > delta) e = (s + lj * r) / (lj - li);
    else e = 0.5 * r;
    E[i + (size_t)j * n] = e;
}

__global__ void ref_update(long long n, double *__restrict__ X, long long ldx, const double *__restrict__ W,
                           double *__restrict__ lam_out, const double *__restrict__ lam)
{
    const long long total = n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long j = idx / n, i = idx - j * n;
        X[i + j * ldx] += W[idx];
        if (i == 0) lam_out[j] = lam[j];
    }
}

}  // namespace

}  // namespace gb

extern "C" {

size_t gb_refine_syev_workspace_bytes(int n) { return n >= 1 ? gb::ref_carve(n, nullptr).total : 0; }

int gb_refine_syev_d(int n, const double *A, int lda, double *lam, double *X, int ldx, void *workspace,
                     size_t ws_bytes, void *stream)
{
    if (n < 1) return -1;
    if (!A || ((uintptr_t)A % 8) != 0) return -2;
    if (lda < n) return -3;
    if (!lam || ((uintptr_t)lam % 8) != 0) return -4;
    if (!X || ((uintptr_t)X % 8) != 0) return -5;
    if (ldx < n) return -6;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -7;
    if (ws_bytes < gb_refine_syev_workspace_bytes(n)) return -8;
    const cudaStream_t st = (cudaStream_t)stream;
    gb::RefWs w = gb::ref_carve(n, (char *)workspace);
    cudaError_t e;
#define GB_RF(x)                                  \
    do {                                          \
        if ((e = (x)) != cudaSuccess) return GB_ERR_CUDA; \
    } while (0)
    GB_RF(gb::sliced_dsyrk_lower_t(n, n, 1.0, X, ldx, 0.0, w.G, n, w.sl, st));                  // G = X^T X
    GB_RF(gb::sliced_dsymm('L', n, n, 1.0, A, lda, X, ldx, 0.0, w.W, n, w.sl, st));            // W = A X
    GB_RF(gb::sliced_dgemm('T', 'N', n, n, n, 1.0, X, ldx, w.W, n, 0.0, w.S, n, w.sl, st));    // S = X^T W
    gb::ref_lambda<<<(n + 255) / 256, 256, 0, st>>>(n, w.S, w.G, w.lam);
    GB_RF(cudaGetLastError());
    gb::ref_norms<<<gb::kNormBlocks, 256, 0, st>>>(n, w.S, w.G, w.lam, w.part);
    GB_RF(cudaGetLastError());
    gb::ref_norms_final<<<1, 32, 0, st>>>(gb::kNormBlocks, w.part, w.norms);
    GB_RF(cudaGetLastError());
    const long long total = (long long)n * n;
    gb::ref_correction<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, w.S, w.G, w.lam, w.norms, w.E);
    GB_RF(cudaGetLastError());
    GB_RF(gb::sliced_dgemm('N', 'N', n, n, n, 1.0, X, ldx, w.E, n, 0.0, w.W, n, w.sl, st));    // W = X E
    gb::ref_update<<<152 * 8, 256, 0, st>>>(n, X, ldx, w.W, lam, w.lam);
    GB_RF(cudaGetLastError());
#undef GB_RF
    return GB_OK;
}

}  // extern "C"
