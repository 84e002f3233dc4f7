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
// than delta.  Close eigenvalues are handled by Rayleigh-Ritz on clusters:
// neighbouring columns (in the order of lambda) are linked when their gap is
// within delta or their first-order correction would exceed kTheta, runs of
// linked columns form clusters (cut at kClusterMax), and each cluster's
// block X_J is replaced by X_J G_JJ^(-1/2) Y_J, with Y_J the eigenvectors of
// G_JJ^(-1/2) S_JJ G_JJ^(-1/2) (cyclic Jacobi); S and G are transformed to
// the new basis (block-diagonal), the formula above runs on the transformed
// entries between different clusters, and inside a cluster E = R / 2.
// Without this the first-order formula mixes the vectors of a cluster whose
// width is below the eigenvectors' current error, and the iteration
// oscillates.  The products run sliced on the bf16 tensor cores at FP64
// accuracy: X is sliced once (by columns) for G = X^T X, W = A X and
// S = X^T W; G and S are formed on their lower triangles only (both are
// symmetric and only the lower triangles are read), so a step costs 6 n^3
// flops.  ||A||_2 is taken as max |lambda_i| and the other spectral norms
// are bounded by Frobenius norms.
//
// The mixed-precision solve (gb_solve_mixed_d) runs the two-stage solver for
// all eigenpairs with FP32 products in full -> band and band -> full
// (the tridiagonal step, the bulge chase and the back-transformation stay
// FP64), then refinement steps in FP64, and returns the lowest nev pairs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "dgemm_sliced.cuh"
#include "elpa_gb300.h"
#include "trans_ev_kernels.cuh"

namespace gb {

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kNormBlocks = 152 * 4;

constexpr size_t kPartialElems = (size_t)4 << 20;  // split-K partials of the products (32 MB)
constexpr int kClusterMax = 64;   // longest cluster solved as one Ritz block
constexpr double kTheta = 1e-3;   // a first-order correction above this links the pair
constexpr int kJacobiSweeps = 30; // bound on the Jacobi sweeps of a Ritz block

// G = X^T X, S = X^T W (then X E), W = A X (then E); two slice buffers;
// lamr: the Rayleigh quotients in the rotated basis; cbeg/clen: each
// column's cluster (start, length); clist/ccount: starts of the clusters of
// two or more columns; Vst: row j holds column j - cbeg[j] of its cluster's
// rotation
struct RefWs {
    double *G, *S, *W, *lam, *lamr, *norms, *part, *pw, *Vst;
    int *cbeg, *clen, *clist, *ccount;
    unsigned char *link;
    void *slX, *slY;
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
    w.S = (double *)take(nn);
    w.W = (double *)take(nn);
    w.lam = (double *)take((size_t)n * 8);
    w.lamr = (double *)take((size_t)n * 8);
    w.Vst = (double *)take((size_t)n * kClusterMax * 8);
    w.cbeg = (int *)take((size_t)n * 4);
    w.clen = (int *)take((size_t)n * 4);
    w.clist = (int *)take((size_t)n * 4);
    w.ccount = (int *)take(4);
    w.link = (unsigned char *)take((size_t)n);
    w.norms = (double *)take(64);
    w.part = (double *)take((size_t)3 * kNormBlocks * 8);
    w.pw = (double *)take(kPartialElems * 8);
    w.slX = take(sliced_bytes(n, n));
    w.slY = take(sliced_bytes(n, n));
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

__device__ __forceinline__ double ref_delta(const double *__restrict__ norms)
{
    return 2.0 * (sqrt(norms[0]) + norms[2] * sqrt(norms[1]));
}

// link[i] = 1 when columns i and i + 1 join one cluster: their gap is within
// delta, or the first-order correction (s + lambda r) / gap of the pair
// exceeds kTheta in either direction
__global__ void ref_links(int n, const double *__restrict__ S, const double *__restrict__ G,
                          const double *__restrict__ lam, const double *__restrict__ norms,
                          unsigned char *__restrict__ link)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const double delta = ref_delta(norms);
    const double gap = fabs(lam[i + 1] - lam[i]);
    const double s = S[(i + 1) + (size_t)i * n], r = -G[(i + 1) + (size_t)i * n];
    const double num = fmax(fabs(s + lam[i + 1] * r), fabs(s + lam[i] * r));
    link[i] = (gap <= delta || num > kTheta * gap) ? 1 : 0;
}

// One thread: runs of linked columns, cut into pieces of at most kClusterMax
__global__ void ref_clusters(int n, const unsigned char *__restrict__ link, int *__restrict__ cbeg,
                             int *__restrict__ clen, int *__restrict__ clist, int *__restrict__ ccount)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int count = 0, b = 0;
    for (int i = 0; i < n; i++) {
        if (i == n - 1 || !link[i] || i + 1 - b >= kClusterMax) {
            const int len = i + 1 - b;
            for (int j = b; j <= i; j++) {
                cbeg[j] = b;
                clen[j] = len;
            }
            if (len > 1) clist[count++] = b;
            b = i + 1;
        }
    }
    *ccount = count;
}

// entry (r, c) of a symmetric n x n matrix whose lower triangle M holds
__device__ __forceinline__ double sym_at(const double *__restrict__ M, int n, int r, int c)
{
    return r >= c ? M[r + (size_t)c * n] : M[c + (size_t)r * n];
}

// Cyclic Jacobi (Golub and Van Loan, symmetric Schur decomposition by plane
// rotations) on the k x k symmetric block B (leading dimension kClusterMax)
// in shared memory: B <- Q^T B Q diagonal, Q accumulated from the identity.
// All threads of the block take part; thread 0 picks each rotation.
__device__ void ritz_jacobi(int k, double *B, double *Q, double *rot)
{
    constexpr int L = kClusterMax;
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int r = t % k, c = t / k;
        Q[r + c * L] = r == c ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < kJacobiSweeps; sweep++) {
        if (threadIdx.x == 0) {
            double off = 0.0, dg = 0.0;
            for (int c = 0; c < k; c++) {
                dg += B[c + c * L] * B[c + c * L];
                for (int r = c + 1; r < k; r++) off += B[r + c * L] * B[r + c * L];
            }
            rot[2] = (off <= 1e-33 * dg || off == 0.0) ? 1.0 : 0.0;
        }
        __syncthreads();
        if (rot[2] != 0.0) break;
        for (int p = 0; p < k - 1; p++)
            for (int q = p + 1; q < k; q++) {
                if (threadIdx.x == 0) {
                    const double bpq = B[p + q * L], bpp = B[p + p * L], bqq = B[q + q * L];
                    double c = 1.0, sn = 0.0;
                    if (fabs(bpq) > 1e-300 && fabs(bpq) > 1e-18 * sqrt(fabs(bpp * bqq))) {
                        const double th = (bqq - bpp) / (2.0 * bpq);
                        const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + hypot(th, 1.0));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        sn = tt * c;
                    }
                    rot[0] = c;
                    rot[1] = sn;
                }
                __syncthreads();
                const double c = rot[0], sn = rot[1];
                if (sn != 0.0) {
                    // columns p, q of B and Q: M <- M J
                    for (int r = threadIdx.x; r < k; r += blockDim.x) {
                        const double bp = B[r + p * L], bq = B[r + q * L];
                        B[r + p * L] = c * bp - sn * bq;
                        B[r + q * L] = sn * bp + c * bq;
                        const double qp = Q[r + p * L], qq = Q[r + q * L];
                        Q[r + p * L] = c * qp - sn * qq;
                        Q[r + q * L] = sn * qp + c * qq;
                    }
                    __syncthreads();
                    // rows p, q of B: B <- J^T B
                    for (int r = threadIdx.x; r < k; r += blockDim.x) {
                        const double bp = B[p + r * L], bq = B[q + r * L];
                        B[p + r * L] = c * bp - sn * bq;
                        B[q + r * L] = sn * bp + c * bq;
                    }
                }
                __syncthreads();
            }
    }
}

// Per cluster (blocks stride over the cluster list): M = G_JJ^(-1/2) from
// the Jacobi decomposition of G_JJ, H = M S_JJ M, Y = eigenvectors of H in
// ascending order of the Ritz values; Vst rows of the cluster = columns of
// M Y.
__global__ void __launch_bounds__(128) ref_ritz(int n, const double *__restrict__ S, const double *__restrict__ G,
                                                const int *__restrict__ clist, const int *__restrict__ ccount,
                                                const int *__restrict__ clen, double *__restrict__ Vst)
{
    constexpr int L = kClusterMax;
    extern __shared__ double sm[];
    double *Gc = sm, *Sc = Gc + L * L, *Q = Sc + L * L, *T = Q + L * L, *rot = T + L * L;
    int *perm = (int *)(rot + 4);
    const int count = *ccount;
    for (int ci = blockIdx.x; ci < count; ci += gridDim.x) {
        const int b0 = clist[ci], k = clen[b0];
        __syncthreads();
        for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
            const int r = t % k, c = t / k;
            Gc[r + c * L] = sym_at(G, n, b0 + r, b0 + c);
            Sc[r + c * L] = sym_at(S, n, b0 + r, b0 + c);
        }
        __syncthreads();
        ritz_jacobi(k, Gc, Q, rot);  // G_JJ = Q diag(Gc) Q^T
        for (int t = threadIdx.x; t < k * k; t += blockDim.x) {  // T = Q diag(g)^(-1/2) Q^T
            const int r = t % k, c = t / k;
            double acc = 0.0;
            for (int a = 0; a < k; a++) acc += Q[r + a * L] * Q[c + a * L] / sqrt(Gc[a + a * L]);
            T[r + c * L] = acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < k * k; t += blockDim.x) {  // Q = S_JJ T
            const int r = t % k, c = t / k;
            double acc = 0.0;
            for (int a = 0; a < k; a++) acc += Sc[r + a * L] * T[a + c * L];
            Q[r + c * L] = acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < k * k; t += blockDim.x) {  // Gc = T Q = T S_JJ T (T symmetric)
            const int r = t % k, c = t / k;
            double acc = 0.0;
            for (int a = 0; a < k; a++) acc += T[a + r * L] * Q[a + c * L];
            Gc[r + c * L] = acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < k * k; t += blockDim.x) {  // symmetrise H
            const int r = t % k, c = t / k;
            if (r > c) {
                const double h = 0.5 * (Gc[r + c * L] + Gc[c + r * L]);
                Gc[r + c * L] = h;
                Gc[c + r * L] = h;
            }
        }
        __syncthreads();
        ritz_jacobi(k, Gc, Q, rot);  // H = Q diag Q^T
        if (threadIdx.x == 0) {      // ascending Ritz values
            for (int a = 0; a < k; a++) perm[a] = a;
            for (int a = 1; a < k; a++) {
                const int v = perm[a];
                int b = a - 1;
                while (b >= 0 && Gc[perm[b] + perm[b] * L] > Gc[v + v * L]) {
                    perm[b + 1] = perm[b];
                    b--;
                }
                perm[b + 1] = v;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < k * k; t += blockDim.x) {  // V = T Y (column jj of V -> row b0 + jj of Vst)
            const int a = t % k, jj = t / k;
            const int pc = perm[jj];
            double acc = 0.0;
            for (int c = 0; c < k; c++) acc += T[a + c * L] * Q[c + pc * L];
            Vst[(size_t)(b0 + jj) * L + a] = acc;
        }
    }
}

// Copies the lower triangle of the n x n matrix M onto its upper triangle
// (32 x 32 tiles through shared memory, both sides coalesced).
__global__ void __launch_bounds__(256) ref_symmetrize(int n, double *__restrict__ M)
{
    __shared__ double t[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;  // lower tile (bi, bj), bi >= bj
    if (bi < bj) return;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int q = ty; q < 32; q += 8) {
        const int r = bi * 32 + tx, c = bj * 32 + q;
        if (r < n && c < n) t[q][tx] = M[r + (size_t)c * n];
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {  // M[c, r] = M[r, c] for r > c
        const int c = bj * 32 + tx, r = bi * 32 + q;
        if (r < n && c < n && r > c) M[c + (size_t)r * n] = t[tx][q];
    }
}

// M[J, c] <- V_J^T M[J, c] for every cluster J and column c, in place: a
// warp per (cluster, column), the column's k entries contiguous.
__global__ void __launch_bounds__(256) ref_rotate_rows(int n, double *__restrict__ M, const int *__restrict__ clist,
                                                       const int *__restrict__ ccount, const int *__restrict__ clen,
                                                       const double *__restrict__ Vst)
{
    constexpr int L = kClusterMax;
    extern __shared__ double sm[];
    double *vs = sm, *buf = sm + L * L;  // buf: L doubles per warp
    const int count = *ccount;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *old = buf + warp * L;
    for (int ci = blockIdx.y; ci < count; ci += gridDim.y) {
        const int b0 = clist[ci], k = clen[b0];
        __syncthreads();
        for (int t = threadIdx.x; t < k * L; t += blockDim.x) vs[t] = Vst[(size_t)b0 * L + t];
        __syncthreads();
        for (int c = blockIdx.x * 8 + warp; c < n; c += gridDim.x * 8) {
            double *col = M + (size_t)c * n + b0;
            for (int a = lane; a < k; a += 32) old[a] = col[a];
            __syncwarp();
            for (int jj = lane; jj < k; jj += 32) {
                double acc = 0.0;
                for (int a = 0; a < k; a++) acc += vs[jj * L + a] * old[a];
                col[jj] = acc;
            }
            __syncwarp();
        }
    }
}

// lamr[j] = s'_jj / g'_jj in the rotated basis
__global__ void ref_lamr(int n, const double *__restrict__ S, const double *__restrict__ G, double *__restrict__ lamr)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) lamr[j] = S[j + (size_t)j * n] / G[j + (size_t)j * n];
}

// E from the rotated S' = V^T S V and G' = V^T G V (full matrices; the
// lower triangle is read for both halves), r' = delta_ij - g'; inside one
// cluster, on the diagonal and for pairs within delta E = r' / 2, else
// E = (s' + lambda_j r') / (lambda_j - lambda_i).
__global__ void ref_correction(int n, const double *__restrict__ S, const double *__restrict__ G,
                               const double *__restrict__ lamr, const double *__restrict__ norms,
                               const int *__restrict__ cbeg, const int *__restrict__ clen, double *__restrict__ E)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int j = (int)(idx / n), i = (int)(idx - (long long)j * n);
    const double s = sym_at(S, n, i, j);
    const double r = (i == j ? 1.0 : 0.0) - sym_at(G, n, i, j);
    const bool same = clen[i] > 1 && cbeg[i] == cbeg[j];
    const double li = lamr[i], lj = lamr[j];
    double e;
    if (i != j && !same && fabs(li - lj) > ref_delta(norms)) e = (s + lj * r) / (lj - li);
    else e = 0.5 * r;
    E[i + (size_t)j * n] = e;
}

// X_J <- X_J V_J for every cluster (columns J of X), in place (each thread
// a row; blocks along y stride over the cluster list)
__global__ void __launch_bounds__(128) ref_rotate_x(int n, double *__restrict__ X, long long ldx,
                                                    const int *__restrict__ clist, const int *__restrict__ ccount,
                                                    const int *__restrict__ clen, const double *__restrict__ Vst)
{
    constexpr int L = kClusterMax;
    extern __shared__ double vs[];
    const int count = *ccount;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    for (int ci = blockIdx.y; ci < count; ci += gridDim.y) {
        const int b0 = clist[ci], k = clen[b0];
        __syncthreads();
        for (int t = threadIdx.x; t < k * L; t += blockDim.x) vs[t] = Vst[(size_t)b0 * L + t];
        __syncthreads();
        if (r < n) {
            double xo[L];
            for (int a = 0; a < k; a++) xo[a] = X[r + (long long)(b0 + a) * ldx];
            for (int jj = 0; jj < k; jj++) {
                double acc = 0.0;
                for (int a = 0; a < k; a++) acc += xo[a] * vs[jj * L + a];
                X[r + (long long)(b0 + jj) * ldx] = acc;
            }
        }
    }
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
    gb::SlicedOp xc, ay, wc, xr, ec;
#define GB_RF(x)                                   \
    do {                                           \
        if ((x) != cudaSuccess) return GB_ERR_CUDA; \
    } while (0)
    using gb::kFillAll;
    using gb::kFillLower;
    GB_RF(gb::slice_matrix(gb::kViewCol, n, n, X, ldx, w.slX, &xc, st));                         // columns of X
    GB_RF(gb::sliced_gemm(xc, xc, n, n, 1.0, 0.0, w.G, n, kFillLower, w.pw, gb::kPartialElems, st));  // G = X^T X
    GB_RF(gb::slice_matrix(gb::kViewSym, n, n, A, lda, w.slY, &ay, st));
    GB_RF(gb::sliced_gemm(ay, xc, n, n, 1.0, 0.0, w.W, n, kFillAll, w.pw, gb::kPartialElems, st));    // W = A X
    GB_RF(gb::slice_matrix(gb::kViewCol, n, n, w.W, n, w.slY, &wc, st));
    GB_RF(gb::sliced_gemm(xc, wc, n, n, 1.0, 0.0, w.S, n, kFillLower, w.pw, gb::kPartialElems, st));  // S = X^T W
    gb::ref_lambda<<<(n + 255) / 256, 256, 0, st>>>(n, w.S, w.G, w.lam);
    GB_RF(cudaGetLastError());
    gb::ref_norms<<<gb::kNormBlocks, 256, 0, st>>>(n, w.S, w.G, w.lam, w.part);
    GB_RF(cudaGetLastError());
    gb::ref_norms_final<<<1, 32, 0, st>>>(gb::kNormBlocks, w.part, w.norms);
    GB_RF(cudaGetLastError());
    const long long total = (long long)n * n;
    // clusters, their Ritz rotations, E in the rotated basis, X <- X V
    const unsigned g1 = (unsigned)((n + 255) / 256);
    if (n > 1) gb::ref_links<<<g1, 256, 0, st>>>(n, w.S, w.G, w.lam, w.norms, w.link);
    GB_RF(cudaGetLastError());
    gb::ref_clusters<<<1, 1, 0, st>>>(n, w.link, w.cbeg, w.clen, w.clist, w.ccount);
    GB_RF(cudaGetLastError());
    constexpr int L = gb::kClusterMax;
    const size_t ritz_smem = (size_t)4 * L * L * 8 + 4 * 8 + L * 4;
    GB_RF(cudaFuncSetAttribute(gb::ref_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ritz_smem));
    gb::ref_ritz<<<std::max(1, std::min(n / 2, 152 * 4)), 128, ritz_smem, st>>>(n, w.S, w.G, w.clist, w.ccount,
                                                                                w.clen, w.Vst);
    GB_RF(cudaGetLastError());
    // S' = V^T S V and G' = V^T G V in place: full matrices, then the
    // columns and the rows of every cluster rotated
    const unsigned tiles = (unsigned)((n + 31) / 32);
    const size_t rot_smem = (size_t)L * L * 8;
    const size_t rows_smem = (size_t)L * L * 8 + (size_t)8 * L * 8;
    GB_RF(cudaFuncSetAttribute(gb::ref_rotate_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rot_smem));
    GB_RF(cudaFuncSetAttribute(gb::ref_rotate_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem));
    const dim3 gcols((unsigned)((n + 127) / 128), 32), grows((unsigned)std::min((n + 7) / 8, 152 * 2), 32);
    for (double *M : {w.S, w.G}) {
        gb::ref_symmetrize<<<dim3(tiles, tiles), 256, 0, st>>>(n, M);
        GB_RF(cudaGetLastError());
        gb::ref_rotate_x<<<gcols, 128, rot_smem, st>>>(n, M, n, w.clist, w.ccount, w.clen, w.Vst);
        GB_RF(cudaGetLastError());
        gb::ref_rotate_rows<<<grows, 256, rows_smem, st>>>(n, M, w.clist, w.ccount, w.clen, w.Vst);
        GB_RF(cudaGetLastError());
    }
    gb::ref_lamr<<<g1, 256, 0, st>>>(n, w.S, w.G, w.lamr);
    GB_RF(cudaGetLastError());
    double *E = w.W;  // W is no longer needed
    gb::ref_correction<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, w.S, w.G, w.lamr, w.norms, w.cbeg,
                                                                        w.clen, E);
    GB_RF(cudaGetLastError());
    gb::ref_rotate_x<<<gcols, 128, rot_smem, st>>>(n, X, ldx, w.clist, w.ccount, w.clen, w.Vst);
    GB_RF(cudaGetLastError());
    GB_RF(gb::slice_matrix(gb::kViewRow, n, n, X, ldx, w.slX, &xr, st));                          // rows of X V
    GB_RF(gb::slice_matrix(gb::kViewCol, n, n, E, n, w.slY, &ec, st));
    double *XE = w.S;  // S is no longer needed
    GB_RF(gb::sliced_gemm(xr, ec, n, n, 1.0, 0.0, XE, n, kFillAll, w.pw, gb::kPartialElems, st));     // X E
    gb::ref_update<<<152 * 8, 256, 0, st>>>(n, X, ldx, XE, lam, w.lamr);
    GB_RF(cudaGetLastError());
#undef GB_RF
    return GB_OK;
}

}  // extern "C"

// ---- mixed-precision solve ----

namespace gb {

namespace {

// status slots (2 x 256 bytes) | X (n x n) | lambda (n) | one region that
// the low-precision solve and then the refinement steps use
struct MixedWs {
    char *status;
    double *X, *lam;
    char *region;
    size_t region_bytes, total;
};

MixedWs mixed_carve(int n, int nbw, char *base)
{
    MixedWs w{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    w.status = take(512);
    w.X = (double *)take((size_t)n * n * 8);
    w.lam = (double *)take((size_t)n * 8);
    w.region_bytes = std::max(gb_solve_workspace_bytes(n, n, nbw), gb_refine_syev_workspace_bytes(n));
    w.region = take(w.region_bytes);
    w.total = off;
    return w;
}

}  // namespace

}  // namespace gb

extern "C" {

size_t gb_solve_mixed_workspace_bytes(int n, int nev, int nbw)
{
    if (gb_solve_workspace_bytes(n, nev, nbw) == 0) return 0;
    return gb::mixed_carve(n, nbw, nullptr).total;
}

int gb_solve_mixed_d(int n, int nev, int nbw, const double *A, int lda, double *ev, double *Z, int ldz,
                     int refine_steps, void *workspace, size_t ws_bytes, void *stream)
{
    if (n < 2) return -1;
    if (nev < 1 || nev > n) return -2;
    if (nbw < 1 || nbw > 64 || nbw >= n) return -3;
    if (!A || ((uintptr_t)A % 8) != 0) return -4;
    if (lda < n) return -5;
    if (!ev || ((uintptr_t)ev % 8) != 0) return -6;
    if (!Z || ((uintptr_t)Z % 8) != 0) return -7;
    if (ldz < n) return -8;
    if (refine_steps < 0 || refine_steps > GB_SOLVE_MIXED_MAX_STEPS) return -9;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -10;
    if (ws_bytes < gb_solve_mixed_workspace_bytes(n, nev, nbw)) return -11;
    const cudaStream_t st = (cudaStream_t)stream;
    gb::MixedWs w = gb::mixed_carve(n, nbw, (char *)workspace);
    // all eigenpairs with FP32 products in full -> band and band -> full
    int rc = gb_solve_d(n, n, nbw, A, lda, w.lam, w.X, n, w.region, w.region_bytes, stream, GB_SOLVE_FP32_PRODUCTS);
    if (rc != GB_OK) return rc;
    if (gb::solve_status_copy(w.region, n, n, nbw, w.status, st) != cudaSuccess) return GB_ERR_CUDA;
    for (int k = 0; k < refine_steps; k++) {
        rc = gb_refine_syev_d(n, A, lda, w.lam, w.X, n, w.region, w.region_bytes, stream);
        if (rc != GB_OK) return rc;
    }
    if (cudaMemcpy2DAsync(Z, (size_t)ldz * 8, w.X, (size_t)n * 8, (size_t)n * 8, nev, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(ev, w.lam, (size_t)nev * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return GB_ERR_CUDA;
    return GB_OK;
}

int gb_solve_mixed_query(const void *workspace, int n, int nev, int nbw, void *stream)
{
    (void)nev;
    if (!workspace) return -1;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GB_ERR_CUDA;
    const gb::MixedWs w = gb::mixed_carve(n, nbw, (char *)workspace);
    for (int i = 0; i < 2; i++) {
        int head[3] = {0, 0, 0};  // ticket, abort, error
        if (cudaMemcpy(head, w.status + 256 * i, sizeof(head), cudaMemcpyDeviceToHost) != cudaSuccess)
            return GB_ERR_CUDA;
        if (head[2]) return head[2];
    }
    return GB_OK;
}

}  // extern "C"
