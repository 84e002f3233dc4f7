// Device kernels of the full -> band reduction (the first step of the
// two-stage reduction, Sec. 2) and of the band -> full back-transformation:
// Householder QR of a tall panel, the block-reflector T matrix, and the
// small conversions around the GEMMs (which run in cuBLAS, see solve.cu).
//
// Panel QR (m x nb, column-major, leading dimension lda): for each column i
// the reflector that annihilates rows i+1..m-1 is built and applied to the
// columns to its right, in two launches over row chunks of kChunk rows:
//   refl_dots:  every block sums the partial squared norms of column i (left
//               by the previous launch), forms alpha, beta, tau, scales its
//               rows of v = x / (alpha - beta) in place and writes partial
//               dot products v^T A[:, j] for j > i;
//   update:     every block sums those partials, applies
//               A[:, j] -= tau v (v^T A[:, j]) to its rows and leaves the
//               partial squared norm of column i+1 for the next step.
// Each block reduces the (few) partials itself, so no atomics are needed.
// On exit the panel holds R on and above the diagonal and v below it
// (LAPACK layout, v_0 = 1 implicit); tau holds the nb scalars.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

namespace gb {

namespace cg = cooperative_groups;

namespace {

constexpr int kChunk = 128;   // rows per block
constexpr int kPanelMax = 64; // nb <= 64

__device__ double block_reduce_sum(double x, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = x;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
    return t;
}

// partial squared norm of column 0 below its first row, per chunk
__device__ __forceinline__ void first_norm_phase(int m, const double *__restrict__ P, double *__restrict__ part)
{
    __shared__ double red[kChunk / 32];
    const int r = blockIdx.x * kChunk + threadIdx.x;
    const double x = (r >= 1 && r < m) ? P[r] : 0.0;
    const double s = block_reduce_sum(x * x, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kChunk) panel_first_norm(int m, const double *__restrict__ P, long long lda,
                                                           double *__restrict__ part)
{
    first_norm_phase(m, P, part);
}

__device__ __forceinline__ void refl_dots_phase(int m, int nb, int i, double *__restrict__ P, long long lda,
                                                const double *__restrict__ part_norm, int nchunks,
                                                double *__restrict__ part_dot, double *__restrict__ tau)
{
    __shared__ double red[kChunk / 32];
    __shared__ double s_tau, s_scal;
    double ss = 0.0;
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) ss += part_norm[c];
    ss = block_reduce_sum(ss, red);
    double *col = P + (long long)i * lda;
    if (threadIdx.x == 0) {
        const double alpha = col[i];
        double t = 0.0, scal = 0.0;
        if (ss != 0.0) {
            const double nrm = sqrt(alpha * alpha + ss);
            const double beta = (alpha >= 0.0) ? -nrm : nrm;
            t = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
        }
        s_tau = t;
        s_scal = scal;
        if (blockIdx.x == 0) tau[i] = t;
    }
    __syncthreads();
    const double t = s_tau;
    const int r = blockIdx.x * kChunk + threadIdx.x;
    // v for this row (v_i = 1 implicit, rows above i are not part of v)
    double v = 0.0;
    if (r == i) v = 1.0;
    else if (r > i && r < m) {
        v = (t != 0.0) ? col[r] * s_scal : 0.0;
    }
    // partial v^T A[:, j] for every j > i in one pass: warp sums, then one
    // shared-memory sum over the block's warps
    __shared__ double wsum[kChunk / 32][kPanelMax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = i + 1; j < nb; j++) {
        double a = (r >= i && r < m) ? P[(long long)j * lda + r] : 0.0;
        double x = v * a;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) wsum[warp][j] = x;
    }
    __syncthreads();
    for (int j = i + 1 + threadIdx.x; j < nb; j += blockDim.x) {
        double t2 = 0.0;
        for (int w2 = 0; w2 < kChunk / 32; w2++) t2 += wsum[w2][j];
        part_dot[(long long)blockIdx.x * kPanelMax + j] = t2;
    }
    __syncthreads();
    // store v below the diagonal (needs every block to have read col[i] first:
    // alpha is read by thread 0 of each block before any block writes row r > i,
    // and only rows > i are written, so alpha = col[i] is never overwritten here)
    if (r > i && r < m && t != 0.0) col[r] = v;
}

__global__ void __launch_bounds__(kChunk) panel_refl_dots(int m, int nb, int i, double *__restrict__ P, long long lda,
                                                          const double *__restrict__ part_norm, int nchunks,
                                                          double *__restrict__ part_dot, double *__restrict__ tau)
{
    refl_dots_phase(m, nb, i, P, lda, part_norm, nchunks, part_dot, tau);
}

__device__ __forceinline__ void update_phase(int m, int nb, int i, double *__restrict__ P, long long lda,
                                             const double *__restrict__ part_dot, int nchunks,
                                             const double *__restrict__ tau, double *__restrict__ part_norm,
                                             const double *__restrict__ part_norm_prev)
{
    __shared__ double red[kChunk / 32];
    __shared__ double w[kPanelMax];
    __shared__ double s_beta;
    const double t = tau[i];
    for (int j = i + 1 + threadIdx.x; j < nb; j += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunks; c++) s += part_dot[(long long)c * kPanelMax + j];
        w[j] = t * s;
    }
    if (threadIdx.x == 0) {
        // beta = -sign(alpha) * sqrt(alpha^2 + ss) (same arithmetic as refl_dots)
        double ss = 0.0;
        for (int c = 0; c < nchunks; c++) ss += part_norm_prev[c];
        const double alpha = P[(long long)i * lda + i];
        double beta = alpha;
        if (ss != 0.0) {
            const double nrm = sqrt(alpha * alpha + ss);
            beta = (alpha >= 0.0) ? -nrm : nrm;
        }
        s_beta = beta;
    }
    __syncthreads();
    const int r = blockIdx.x * kChunk + threadIdx.x;
    double *col = P + (long long)i * lda;
    double v = 0.0;
    if (r == i) v = 1.0;
    else if (r > i && r < m) v = (t != 0.0) ? col[r] : 0.0;
    double next = 0.0;
    for (int j = i + 1; j < nb; j++) {
        if (r >= i && r < m && t != 0.0) {
            double *a = P + (long long)j * lda + r;
            *a = fma(-w[j], v, *a);
        }
        if (j == i + 1 && r > i + 1 && r < m) {
            const double a = P[(long long)j * lda + r];
            next = a * a;
        }
    }
    if (i + 1 < nb) {
        const double s = block_reduce_sum(next, red);
        if (threadIdx.x == 0) part_norm[blockIdx.x] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) col[i] = s_beta;  // R's diagonal entry
}

__global__ void __launch_bounds__(kChunk) panel_update(int m, int nb, int i, double *__restrict__ P, long long lda,
                                                       const double *__restrict__ part_dot, int nchunks,
                                                       const double *__restrict__ tau, double *__restrict__ part_norm,
                                                       const double *__restrict__ part_norm_prev)
{
    update_phase(m, nb, i, P, lda, part_dot, nchunks, tau, part_norm, part_norm_prev);
}

// The whole panel in one cooperative launch: the same phases, separated by
// grid-wide barriers instead of kernel boundaries (2 nb + 1 launches become
// one).  Launched only when every block of the grid can be resident.
__global__ void __launch_bounds__(kChunk) panel_qr_fused(int m, int nb, double *__restrict__ P, long long lda,
                                                         double *__restrict__ tau, double *__restrict__ norm_a,
                                                         double *__restrict__ norm_b, double *__restrict__ dots,
                                                         int nchunks)
{
    cg::grid_group grid = cg::this_grid();
    first_norm_phase(m, P, norm_a);
    grid.sync();
    for (int i = 0; i < nb && i < m; i++) {
        double *cur = (i % 2 == 0) ? norm_a : norm_b;
        double *nxt = (i % 2 == 0) ? norm_b : norm_a;
        refl_dots_phase(m, nb, i, P, lda, cur, nchunks, dots, tau);
        grid.sync();
        update_phase(m, nb, i, P, lda, dots, nchunks, tau, nxt, cur);
        grid.sync();
    }
}

// Y (m x nb, explicit unit lower trapezoidal) from the QR'd panel.
__global__ void __launch_bounds__(256) panel_explicit_y(int m, int nb, const double *__restrict__ P, long long lda,
                                                        double *__restrict__ Y, long long ldy)
{
    const long long total = (long long)m * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / m), r = (int)(e - (long long)j * m);
        Y[(long long)j * ldy + r] = (r < j) ? 0.0 : (r == j ? 1.0 : P[(long long)j * lda + r]);
    }
}

// T (nb x nb upper triangular) of the block reflector I - Y T Y^T from
// G = Y^T Y and tau: T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j].
__global__ void __launch_bounds__(kPanelMax) panel_build_t(int nb, const double *__restrict__ G, long long ldg,
                                                           const double *__restrict__ tau, double *__restrict__ T,
                                                           long long ldt)
{
    __shared__ double Ts[kPanelMax][kPanelMax + 1];
    __shared__ double g[kPanelMax];
    const int r = threadIdx.x;
    for (int j = 0; j < nb; j++) {
        if (r < nb) Ts[r][j] = 0.0;
    }
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        if (r < j) g[r] = G[(long long)j * ldg + r];
        __syncthreads();
        if (r < j) {
            double s = 0.0;
            for (int q = r; q < j; q++) s = fma(Ts[r][q], g[q], s);
            Ts[r][j] = -tau[j] * s;
        }
        if (r == j) Ts[j][j] = tau[j];
        __syncthreads();
    }
    if (r < nb)
        for (int j = 0; j < nb; j++) T[(long long)j * ldt + r] = Ts[r][j];
}

// W = X - 0.5 * Y * M is done by cuBLAS; H = 1.5 I - 0.5 G for Newton-Schulz.
__global__ void __launch_bounds__(256) ns_matrix(int k, double *__restrict__ G, long long ldg)
{
    const long long total = (long long)k * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / k, r = e - j * k;
        double *g = G + j * ldg + r;
        *g = (r == j ? 1.5 : 0.0) - 0.5 * (*g);
    }
}

// Lower band storage (b+1) x n of the reduced matrix; entries of the
// full matrix A (lda) with 0 <= i - j <= b.
__global__ void __launch_bounds__(256) extract_band(int n, int b, const double *__restrict__ A, long long lda,
                                                    double *__restrict__ AB, long long ldab)
{
    const long long total = (long long)n * (b + 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / (b + 1), dd = e - j * (b + 1);
        AB[j * ldab + dd] = (j + dd < n) ? A[j * lda + j + dd] : 0.0;
    }
}

// Mirror the lower triangle of rows/cols [j0, n) into the upper one.
__global__ void __launch_bounds__(256) symmetrize_lower(int n, int j0, double *__restrict__ A, long long lda)
{
    const long long m = n - j0;
    const long long total = m * m;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / m, r = e - j * m;
        if (r > j) A[(j0 + r) * lda + (j0 + j)] = A[(j0 + j) * lda + (j0 + r)];
    }
}

}  // namespace

int panel_chunks(int m) { return (m + kChunk - 1) / kChunk; }

// Householder QR of the m x nb panel P (lda); part holds 2*nchunks + nchunks*64 doubles.
cudaError_t panel_qr(int m, int nb, double *P, long long lda, double *tau, double *part, cudaStream_t st)
{
    const int nch = panel_chunks(m);
    double *norm_a = part, *norm_b = part + nch, *dots = part + 2 * nch;
    // columns past the last reflector (m < nb) keep tau = 0
    cudaError_t e = cudaMemsetAsync(tau, 0, sizeof(double) * nb, st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_qr_fused, kChunk, 0)) != cudaSuccess)
        return e;
    // a quarter of the co-resident capacity at most, so that concurrent
    // solves on other streams keep room beside it; never while the stream is
    // being captured into a graph, whose kernel nodes carry no co-residency
    // guarantee for the grid-wide barriers
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return e;
    if (coop && cap == cudaStreamCaptureStatusNone && (long long)nch * 4 <= (long long)per_sm * sms) {
        void *args[] = {&m, &nb, &P, &lda, &tau, &norm_a, &norm_b, &dots, (void *)&nch};
        return cudaLaunchCooperativeKernel((const void *)panel_qr_fused, dim3(nch), dim3(kChunk), args, 0, st);
    }
    panel_first_norm<<<nch, kChunk, 0, st>>>(m, P, lda, norm_a);
    for (int i = 0; i < nb && i < m; i++) {
        double *cur = (i % 2 == 0) ? norm_a : norm_b;
        double *nxt = (i % 2 == 0) ? norm_b : norm_a;
        panel_refl_dots<<<nch, kChunk, 0, st>>>(m, nb, i, P, lda, cur, nch, dots, tau);
        panel_update<<<nch, kChunk, 0, st>>>(m, nb, i, P, lda, dots, nch, tau, nxt, cur);
    }
    return cudaGetLastError();
}

cudaError_t panel_y_and_t_prep(int m, int nb, const double *P, long long lda, double *Y, long long ldy,
                               cudaStream_t st)
{
    panel_explicit_y<<<256, 256, 0, st>>>(m, nb, P, lda, Y, ldy);
    return cudaGetLastError();
}

cudaError_t panel_t(int nb, const double *G, long long ldg, const double *tau, double *T, long long ldt,
                    cudaStream_t st)
{
    panel_build_t<<<1, kPanelMax, 0, st>>>(nb, G, ldg, tau, T, ldt);
    return cudaGetLastError();
}

cudaError_t newton_schulz_matrix(int k, double *G, long long ldg, cudaStream_t st)
{
    ns_matrix<<<1024, 256, 0, st>>>(k, G, ldg);
    return cudaGetLastError();
}

cudaError_t band_from_full(int n, int b, const double *A, long long lda, double *AB, long long ldab, cudaStream_t st)
{
    extract_band<<<1024, 256, 0, st>>>(n, b, A, lda, AB, ldab);
    return cudaGetLastError();
}

cudaError_t mirror_lower(int n, int j0, double *A, long long lda, cudaStream_t st)
{
    symmetrize_lower<<<1024, 256, 0, st>>>(n, j0, A, lda);
    return cudaGetLastError();
}

}  // namespace gb
