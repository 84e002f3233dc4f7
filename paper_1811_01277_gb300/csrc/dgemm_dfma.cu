// Tiled FP64 products on the DFMA pipe (see dgemm_dfma.cuh).
//
// One CTA of 256 threads computes a 64 x 64 tile of C; thread (tx, ty) owns
// rows tx + 16i and columns ty + 16j (i, j < 4), so the shared-memory reads of
// a k step are broadcasts without bank conflicts.  The reduction runs in
// steps of 8: the next step's operand tiles are loaded from global memory
// into registers while the current step's 128 DFMAs per thread run from
// shared memory (double-buffered).  An FP64 FMA occupies a scheduler's
// narrow FP64 pipe for many cycles, so a 4 x 4 register tile leaves the
// issue slots free for the loads and address arithmetic.
//
// Operand modes: N (as stored), T (transposed) and SYM (symmetric, lower
// triangle stored).  Each mode has its own thread-to-element mapping so that
// consecutive threads read consecutive addresses; a symmetric tile that
// crosses the diagonal is read element by element.
#include <cuda_runtime.h>

#include <stdint.h>

#include "dgemm_dfma.cuh"
#include "elpa_gb300.h"

namespace gb {

namespace {

constexpr int BM = 64, BN = 64, BK = 8, NT = 256;
constexpr int MODE_N = 0, MODE_T = 1, MODE_SYM = 2;

struct Gemm {
    int m, n;                 // C is m x n
    int k, k2;                // reduction lengths of product 1 and (optional) product 2
    const double *A, *B;      // product 1: op(A) (m x k) op(B) (k x n)
    const double *A2, *B2;    // product 2, same modes, k2 long (k2 = 0: none)
    long long lda, ldb, lda2, ldb2;
    double *C;
    long long ldc;
    double alpha, beta;
    double *partial;          // split-K partials [splits][n][m] (splits > 1)
    int kchunk;               // reduction length per split, multiple of BK
    int lower;                // 1: tiles with row tile >= column tile only, elements r >= c
    int tiles_m;
};

// op(A)(r, q) of a BM x BK tile at (r0, q0); 2 elements per thread.
template <int MODE>
__device__ __forceinline__ void load_a(const double *__restrict__ A, long long lda, int m, int kend, int r0, int q0,
                                       double (&v)[2], int (&sr)[2], int (&sq)[2])
{
    const bool below = r0 >= q0 + BK - 1;       // every r >= q in the tile
    const bool above = r0 + BM - 1 < q0;        // every r < q in the tile
    const bool tmap = (MODE == MODE_T) || (MODE == MODE_SYM && above);
#pragma unroll
    for (int t = 0; t < 2; t++) {
        const int e = threadIdx.x + NT * t;
        int r, q;
        if (tmap) {
            q = e % BK;
            r = e / BK;
        } else {
            r = e % BM;
            q = e / BM;
        }
        sr[t] = r;
        sq[t] = q;
        const int gr = r0 + r, gq = q0 + q;
        double x = 0.0;
        if (gr < m && gq < kend) {
            if (MODE == MODE_N) x = A[(long long)gq * lda + gr];
            else if (MODE == MODE_T) x = A[(long long)gr * lda + gq];
            else if (below || (!above && gr >= gq)) x = A[(long long)gq * lda + gr];
            else x = A[(long long)gr * lda + gq];
        }
        v[t] = x;
    }
}

// op(B)(q, c) of a BK x BN tile at (q0, c0); 2 elements per thread.
template <int MODE>
__device__ __forceinline__ void load_b(const double *__restrict__ B, long long ldb, int n, int kend, int q0, int c0,
                                       double (&v)[2], int (&sq)[2], int (&sc)[2])
{
    const bool below = q0 >= c0 + BN - 1;       // every q >= c
    const bool above = q0 + BK - 1 < c0;        // every q < c
    const bool cmap = (MODE == MODE_T) || (MODE == MODE_SYM && above);
#pragma unroll
    for (int t = 0; t < 2; t++) {
        const int e = threadIdx.x + NT * t;
        int q, c;
        if (cmap) {
            c = e % BN;
            q = e / BN;
        } else {
            q = e % BK;
            c = e / BK;
        }
        sq[t] = q;
        sc[t] = c;
        const int gq = q0 + q, gc = c0 + c;
        double x = 0.0;
        if (gq < kend && gc < n) {
            if (MODE == MODE_N) x = B[(long long)gc * ldb + gq];
            else if (MODE == MODE_T) x = B[(long long)gq * ldb + gc];
            else if (below || (!above && gq >= gc)) x = B[(long long)gc * ldb + gq];
            else x = B[(long long)gq * ldb + gc];
        }
        v[t] = x;
    }
}

template <int MA, int MB>
__global__ void __launch_bounds__(NT) dfma_gemm_kernel(Gemm g)
{
    __shared__ double As[2][BK][BM + 1];
    __shared__ double Bs[2][BK][BN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int ti, tj;
    if (g.lower) {  // blockIdx.x enumerates the lower tiles row by row
        const long long L = blockIdx.x;
        int i = (int)((sqrt(8.0 * (double)L + 1.0) - 1.0) * 0.5);
        while ((long long)(i + 1) * (i + 2) / 2 <= L) i++;
        while ((long long)i * (i + 1) / 2 > L) i--;
        ti = i;
        tj = (int)(L - (long long)i * (i + 1) / 2);
    } else {
        ti = blockIdx.x;
        tj = blockIdx.y;
    }
    const int r0 = ti * BM, c0 = tj * BN;
    const int split = blockIdx.z;

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    const int npairs = g.k2 > 0 ? 2 : 1;
    for (int p = 0; p < npairs; p++) {
        const double *A = p ? g.A2 : g.A;
        const double *B = p ? g.B2 : g.B;
        const long long lda = p ? g.lda2 : g.lda, ldb = p ? g.ldb2 : g.ldb;
        const int K = p ? g.k2 : g.k;
        const int kb = p ? 0 : split * g.kchunk;
        const int ke = p ? K : min(K, kb + g.kchunk);
        if (kb >= ke) continue;
        double va[2], vb[2];
        int ar[2], aq[2], bq[2], bc[2];
        load_a<MA>(A, lda, g.m, ke, r0, kb, va, ar, aq);
        load_b<MB>(B, ldb, g.n, ke, kb, c0, vb, bq, bc);
        __syncthreads();  // the previous pair's last reads of the buffers are done
#pragma unroll
        for (int t = 0; t < 2; t++) {
            As[0][aq[t]][ar[t]] = va[t];
            Bs[0][bq[t]][bc[t]] = vb[t];
        }
        __syncthreads();
        int buf = 0;
        for (int q0 = kb; q0 < ke; q0 += BK) {
            const bool more = q0 + BK < ke;
            if (more) {
                load_a<MA>(A, lda, g.m, ke, r0, q0 + BK, va, ar, aq);
                load_b<MB>(B, ldb, g.n, ke, q0 + BK, c0, vb, bq, bc);
            }
#pragma unroll
            for (int q = 0; q < BK; q++) {
                double a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; i++) a[i] = As[buf][q][tx + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; j++) b[j] = Bs[buf][q][ty + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            if (more) {
#pragma unroll
                for (int t = 0; t < 2; t++) {
                    As[buf ^ 1][aq[t]][ar[t]] = va[t];
                    Bs[buf ^ 1][bq[t]][bc[t]] = vb[t];
                }
            }
            __syncthreads();
            buf ^= 1;
        }
    }

    const bool diag = g.lower && ti == tj;
    if (g.partial) {  // split-K: raw partial product
        double *P = g.partial + (long long)split * g.m * g.n;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int r = r0 + tx + 16 * i, c = c0 + ty + 16 * j;
                if (r < g.m && c < g.n) P[(long long)c * g.m + r] = acc[i][j];
            }
        return;
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int r = r0 + tx + 16 * i, c = c0 + ty + 16 * j;
            if (r < g.m && c < g.n && (!diag || r >= c)) {
                double *cp = g.C + (long long)c * g.ldc + r;
                *cp = (g.beta == 0.0) ? g.alpha * acc[i][j] : fma(g.alpha, acc[i][j], g.beta * *cp);
            }
        }
}

// C = alpha sum_s P[s] + beta C, the splits added in a fixed order.
__global__ void __launch_bounds__(256) splitk_reduce(int m, int n, int splits, const double *__restrict__ P,
                                                     double alpha, double beta, double *__restrict__ C,
                                                     long long ldc)
{
    const long long total = (long long)m * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int z = 0; z < splits; z++) s += P[(long long)z * total + e];
        const long long c = e / m, r = e - c * m;
        double *cp = C + c * ldc + r;
        *cp = (beta == 0.0) ? alpha * s : fma(alpha, s, beta * *cp);
    }
}

int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 148;
    return sms;
}

// Split the reduction until about four CTAs per SM are busy, keeping at
// least 8 steps of BK per split and the partials within the workspace.
int choose_splits(long long tiles, int k, int m, int n, size_t work_elems)
{
    const long long target = 4LL * sm_count();
    int s = 1;
    while (tiles * s < target && (long long)k >= 2LL * s * 8 * BK && s < 512 &&
           (size_t)(2 * s) * (size_t)m * (size_t)n <= work_elems)
        s *= 2;
    return s;
}

template <int MA, int MB>
cudaError_t launch(Gemm g, int splits, cudaStream_t st)
{
    if (g.m <= 0 || g.n <= 0) return cudaSuccess;
    const int tm = (g.m + BM - 1) / BM, tn = (g.n + BN - 1) / BN;
    g.tiles_m = tm;
    if ((g.k <= 0 && g.k2 <= 0) || g.k2 > 0 || g.lower) splits = 1;  // split-K: one product, full tiles
    g.kchunk = ((g.k + splits - 1) / splits + BK - 1) / BK * BK;
    if (g.kchunk <= 0) g.kchunk = BK;
    g.partial = splits > 1 ? g.partial : nullptr;
    dim3 grid;
    if (g.lower) grid = dim3((unsigned)((long long)tm * (tm + 1) / 2), 1, (unsigned)splits);
    else grid = dim3((unsigned)tm, (unsigned)tn, (unsigned)splits);
    dfma_gemm_kernel<MA, MB><<<grid, NT, 0, st>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    splitk_reduce<<<1024, 256, 0, st>>>(g.m, g.n, splits, g.partial, g.alpha, g.beta, g.C, g.ldc);
    return cudaGetLastError();
}

Gemm base(int m, int n, int k, double alpha, const double *A, long long lda, const double *B, long long ldb,
          double beta, double *C, long long ldc, double *work)
{
    Gemm g{};
    g.m = m;
    g.n = n;
    g.k = k;
    g.k2 = 0;
    g.A = A;
    g.B = B;
    g.lda = lda;
    g.ldb = ldb;
    g.C = C;
    g.ldc = ldc;
    g.alpha = alpha;
    g.beta = beta;
    g.partial = work;
    g.lower = 0;
    return g;
}

}  // namespace

cudaError_t dfma_gemm(char transa, char transb, int m, int n, int k, double alpha, const double *A, long long lda,
                      const double *B, long long ldb, double beta, double *C, long long ldc, double *work,
                      size_t work_elems, cudaStream_t st)
{
    Gemm g = base(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, work);
    const long long tiles = (long long)((m + BM - 1) / BM) * ((n + BN - 1) / BN);
    const int s = work ? choose_splits(tiles, k, m, n, work_elems) : 1;
    const bool ta = transa == 'T' || transa == 't', tb = transb == 'T' || transb == 't';
    if (!ta && !tb) return launch<MODE_N, MODE_N>(g, s, st);
    if (ta && !tb) return launch<MODE_T, MODE_N>(g, s, st);
    if (!ta && tb) return launch<MODE_N, MODE_T>(g, s, st);
    return launch<MODE_T, MODE_T>(g, s, st);
}

cudaError_t dfma_symm(char side, int m, int n, double alpha, const double *S, long long lds, const double *B,
                      long long ldb, double beta, double *C, long long ldc, double *work, size_t work_elems,
                      cudaStream_t st)
{
    const long long tiles = (long long)((m + BM - 1) / BM) * ((n + BN - 1) / BN);
    if (side == 'L' || side == 'l') {
        Gemm g = base(m, n, m, alpha, S, lds, B, ldb, beta, C, ldc, work);
        const int s = work ? choose_splits(tiles, m, m, n, work_elems) : 1;
        return launch<MODE_SYM, MODE_N>(g, s, st);
    }
    Gemm g = base(m, n, n, alpha, B, ldb, S, lds, beta, C, ldc, work);
    const int s = work ? choose_splits(tiles, n, m, n, work_elems) : 1;
    return launch<MODE_N, MODE_SYM>(g, s, st);
}

cudaError_t dfma_syr2k_lower(int n, int k, double alpha, const double *A, long long lda, const double *B,
                             long long ldb, double beta, double *C, long long ldc, cudaStream_t st)
{
    // A B^T + B A^T as two products with op(A) = N, op(B) = T
    Gemm g = base(n, n, k, alpha, A, lda, B, ldb, beta, C, ldc, nullptr);
    g.A2 = B;
    g.lda2 = ldb;
    g.B2 = A;
    g.ldb2 = lda;
    g.k2 = k;
    g.lower = 1;
    return launch<MODE_N, MODE_T>(g, 1, st);
}

cudaError_t dfma_syrk_lower_t(int n, int k, double alpha, const double *A, long long lda, double beta, double *C,
                              long long ldc, cudaStream_t st)
{
    Gemm g = base(n, n, k, alpha, A, lda, A, lda, beta, C, ldc, nullptr);
    g.lower = 1;
    return launch<MODE_T, MODE_N>(g, 1, st);
}

}  // namespace gb

extern "C" {

size_t gb_dgemm_workspace_bytes(int m, int n)
{
    if (m < 0 || n < 0) return 0;
    return (size_t)512 * (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1) * 8;
}

static bool bad_ptr(const void *p) { return !p || ((uintptr_t)p % 8) != 0; }

int gb_dgemm(char transa, char transb, int m, int n, int k, double alpha, const double *A, int lda,
             const double *B, int ldb, double beta, double *C, int ldc, void *workspace, size_t ws_bytes,
             void *stream)
{
    const bool ta = transa == 'T' || transa == 't', tb = transb == 'T' || transb == 't';
    if (!ta && transa != 'N' && transa != 'n') return -1;
    if (!tb && transb != 'N' && transb != 'n') return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    if (m == 0 || n == 0) return GB_OK;
    if (k > 0 && bad_ptr(A)) return -7;
    if (lda < (ta ? (k > 1 ? k : 1) : m)) return -8;
    if (k > 0 && bad_ptr(B)) return -9;
    if (ldb < (tb ? n : (k > 1 ? k : 1))) return -10;
    if (bad_ptr(C)) return -12;
    if (ldc < m) return -13;
    if (ws_bytes > 0 && bad_ptr(workspace)) return -14;
    cudaError_t e = gb::dfma_gemm(ta ? 'T' : 'N', tb ? 'T' : 'N', m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                  ws_bytes ? (double *)workspace : nullptr, ws_bytes / 8, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int gb_dsymm(char side, int m, int n, double alpha, const double *S, int lds, const double *B, int ldb,
             double beta, double *C, int ldc, void *workspace, size_t ws_bytes, void *stream)
{
    const bool left = side == 'L' || side == 'l';
    if (!left && side != 'R' && side != 'r') return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (m == 0 || n == 0) return GB_OK;
    if (bad_ptr(S)) return -5;
    if (lds < (left ? m : n)) return -6;
    if (bad_ptr(B)) return -7;
    if (ldb < m) return -8;
    if (bad_ptr(C)) return -10;
    if (ldc < m) return -11;
    if (ws_bytes > 0 && bad_ptr(workspace)) return -12;
    cudaError_t e = gb::dfma_symm(left ? 'L' : 'R', m, n, alpha, S, lds, B, ldb, beta, C, ldc,
                                  ws_bytes ? (double *)workspace : nullptr, ws_bytes / 8, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int gb_dsyr2k(int n, int k, double alpha, const double *A, int lda, const double *B, int ldb, double beta,
              double *C, int ldc, void *stream)
{
    if (n < 0) return -1;
    if (k < 0) return -2;
    if (n == 0) return GB_OK;
    if (k > 0 && bad_ptr(A)) return -4;
    if (lda < n) return -5;
    if (k > 0 && bad_ptr(B)) return -6;
    if (ldb < n) return -7;
    if (bad_ptr(C)) return -9;
    if (ldc < n) return -10;
    cudaError_t e = gb::dfma_syr2k_lower(n, k, alpha, A, lda, B, ldb, beta, C, ldc, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int gb_dsyrk(int n, int k, double alpha, const double *A, int lda, double beta, double *C, int ldc, void *stream)
{
    if (n < 0) return -1;
    if (k < 0) return -2;
    if (n == 0) return GB_OK;
    if (k > 0 && bad_ptr(A)) return -4;
    if (lda < (k > 1 ? k : 1)) return -5;
    if (bad_ptr(C)) return -7;
    if (ldc < n) return -8;
    cudaError_t e = gb::dfma_syrk_lower_t(n, k, alpha, A, lda, beta, C, ldc, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

}  // extern "C"
