// Complex Hermitian counterparts of the full -> band panel kernels
// (full_to_band.cu): Householder QR of a complex panel with H^H applied
// from the left (beta real, tau complex), the block reflector T from Y^H Y,
// lower-band extraction, and the real -> complex promotion of the
// tridiagonal eigenvectors.  Complex values are interleaved (re, im) doubles.
#include <cuda_runtime.h>

namespace gb {

namespace {

constexpr int kChunk = 128;
constexpr int kPanelMax = 64;

struct Zd {
    double re, im;
};

__device__ __forceinline__ Zd zm(Zd a, Zd b) { return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)}; }

__device__ double bsum(double x, double *red)
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

__global__ void __launch_bounds__(kChunk) zpanel_first_norm(int m, const Zd *__restrict__ P, double *__restrict__ part)
{
    __shared__ double red[kChunk / 32];
    const int r = blockIdx.x * kChunk + threadIdx.x;
    const Zd x = (r >= 1 && r < m) ? P[r] : Zd{0.0, 0.0};
    const double s = bsum(x.re * x.re + x.im * x.im, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// alpha, beta, tau, 1/(alpha-beta) from the column's head and the squared norm below it
__device__ void zreflector(Zd alpha, double ss, Zd *tau, Zd *scal, double *beta)
{
    *tau = {0.0, 0.0};
    *scal = {0.0, 0.0};
    *beta = alpha.re;
    if (ss == 0.0 && alpha.im == 0.0) return;
    const double nrm = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + ss);
    const double b = (alpha.re >= 0.0) ? -nrm : nrm;
    *beta = b;
    *tau = {(b - alpha.re) / b, -alpha.im / b};
    const Zd den{alpha.re - b, alpha.im};
    const double dd = den.re * den.re + den.im * den.im;
    *scal = {den.re / dd, -den.im / dd};
}

__global__ void __launch_bounds__(kChunk) zpanel_refl_dots(int m, int nb, int i, Zd *__restrict__ P, long long lda,
                                                           const double *__restrict__ part_norm, int nchunks,
                                                           Zd *__restrict__ part_dot, Zd *__restrict__ tau)
{
    __shared__ double red[kChunk / 32];
    __shared__ Zd s_tau, s_scal;
    __shared__ Zd wsum[kChunk / 32][kPanelMax];
    double ss = 0.0;
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) ss += part_norm[c];
    ss = bsum(ss, red);
    Zd *col = P + (long long)i * lda;
    if (threadIdx.x == 0) {
        Zd t, sc;
        double beta;
        zreflector(col[i], ss, &t, &sc, &beta);
        s_tau = t;
        s_scal = sc;
        if (blockIdx.x == 0) tau[i] = t;
    }
    __syncthreads();
    const Zd t = s_tau;
    const bool act = !(t.re == 0.0 && t.im == 0.0);
    const int r = blockIdx.x * kChunk + threadIdx.x;
    Zd v{0.0, 0.0};
    if (r == i) v = {1.0, 0.0};
    else if (r > i && r < m && act) v = zm(col[r], s_scal);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = i + 1; j < nb; j++) {
        const Zd a = (r >= i && r < m) ? P[(long long)j * lda + r] : Zd{0.0, 0.0};
        // conj(v) * a
        double xr = v.re * a.re + v.im * a.im, xi = v.re * a.im - v.im * a.re;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            xr += __shfl_xor_sync(0xffffffffu, xr, o);
            xi += __shfl_xor_sync(0xffffffffu, xi, o);
        }
        if (lane == 0) wsum[warp][j] = Zd{xr, xi};
    }
    __syncthreads();
    for (int j = i + 1 + threadIdx.x; j < nb; j += blockDim.x) {
        Zd s2{0.0, 0.0};
        for (int w2 = 0; w2 < kChunk / 32; w2++) {
            s2.re += wsum[w2][j].re;
            s2.im += wsum[w2][j].im;
        }
        part_dot[(long long)blockIdx.x * kPanelMax + j] = s2;
    }
    __syncthreads();
    if (r > i && r < m && act) col[r] = v;
}

__global__ void __launch_bounds__(kChunk) zpanel_update(int m, int nb, int i, Zd *__restrict__ P, long long lda,
                                                        const Zd *__restrict__ part_dot, int nchunks,
                                                        const Zd *__restrict__ tau, double *__restrict__ part_norm,
                                                        const double *__restrict__ part_norm_prev)
{
    __shared__ double red[kChunk / 32];
    __shared__ Zd w[kPanelMax];
    __shared__ double s_beta;
    const Zd t = tau[i];
    const Zd ct{t.re, -t.im};  // H^H = I - conj(tau) v v^H from the left
    for (int j = i + 1 + threadIdx.x; j < nb; j += blockDim.x) {
        Zd s{0.0, 0.0};
        for (int c = 0; c < nchunks; c++) {
            s.re += part_dot[(long long)c * kPanelMax + j].re;
            s.im += part_dot[(long long)c * kPanelMax + j].im;
        }
        w[j] = zm(ct, s);
    }
    if (threadIdx.x == 0) {
        double ss = 0.0;
        for (int c = 0; c < nchunks; c++) ss += part_norm_prev[c];
        Zd tt, sc;
        double beta;
        zreflector(P[(long long)i * lda + i], ss, &tt, &sc, &beta);
        s_beta = beta;
    }
    __syncthreads();
    const bool act = !(t.re == 0.0 && t.im == 0.0);
    const int r = blockIdx.x * kChunk + threadIdx.x;
    Zd *col = P + (long long)i * lda;
    Zd v{0.0, 0.0};
    if (r == i) v = {1.0, 0.0};
    else if (r > i && r < m && act) v = col[r];
    double next = 0.0;
    for (int j = i + 1; j < nb; j++) {
        if (r >= i && r < m && act) {
            Zd *a = P + (long long)j * lda + r;
            const Zd vw = zm(v, w[j]);
            a->re -= vw.re;
            a->im -= vw.im;
        }
        if (j == i + 1 && r > i + 1 && r < m) {
            const Zd a = P[(long long)j * lda + r];
            next = a.re * a.re + a.im * a.im;
        }
    }
    if (i + 1 < nb) {
        const double s = bsum(next, red);
        if (threadIdx.x == 0) part_norm[blockIdx.x] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && act) col[i] = Zd{s_beta, 0.0};
}

__global__ void __launch_bounds__(256) zpanel_explicit_y(int m, int nb, const Zd *__restrict__ P, long long lda,
                                                         Zd *__restrict__ Y, long long ldy)
{
    const long long total = (long long)m * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / m), r = (int)(e - (long long)j * m);
        Y[(long long)j * ldy + r] = (r < j) ? Zd{0.0, 0.0} : (r == j ? Zd{1.0, 0.0} : P[(long long)j * lda + r]);
    }
}

// T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j], G = Y^H Y
__global__ void __launch_bounds__(kPanelMax) zpanel_build_t(int nb, const Zd *__restrict__ G, long long ldg,
                                                            const Zd *__restrict__ tau, Zd *__restrict__ T,
                                                            long long ldt)
{
    __shared__ Zd Ts[kPanelMax][kPanelMax + 1];
    __shared__ Zd g[kPanelMax];
    const int r = threadIdx.x;
    for (int j = 0; j < nb; j++)
        if (r < nb) Ts[r][j] = Zd{0.0, 0.0};
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        if (r < j) g[r] = G[(long long)j * ldg + r];
        __syncthreads();
        if (r < j) {
            Zd s{0.0, 0.0};
            for (int q = r; q < j; q++) {
                const Zd p = zm(Ts[r][q], g[q]);
                s.re += p.re;
                s.im += p.im;
            }
            const Zd ts = zm(tau[j], s);
            Ts[r][j] = Zd{-ts.re, -ts.im};
        }
        if (r == j) Ts[j][j] = tau[j];
        __syncthreads();
    }
    if (r < nb)
        for (int j = 0; j < nb; j++) T[(long long)j * ldt + r] = Ts[r][j];
}

__global__ void __launch_bounds__(256) zextract_band(int n, int b, const Zd *__restrict__ A, long long lda,
                                                     Zd *__restrict__ AB, long long ldab)
{
    const long long total = (long long)n * (b + 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / (b + 1), dd = e - j * (b + 1);
        AB[j * ldab + dd] = (j + dd < n) ? A[j * lda + j + dd] : Zd{0.0, 0.0};
    }
}

__global__ void __launch_bounds__(256) real_to_complex(long long rows, long long cols, const double *__restrict__ X,
                                                       long long ldx, Zd *__restrict__ Z, long long ldz)
{
    const long long total = rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / rows, r = e - j * rows;
        Z[j * ldz + r] = Zd{X[j * ldx + r], 0.0};
    }
}

}  // namespace

int panel_chunks(int m);

cudaError_t zpanel_qr(int m, int nb, double *P, long long lda, double *tau, double *part, cudaStream_t st)
{
    const int nch = panel_chunks(m);
    double *norm_a = part, *norm_b = part + nch;
    Zd *dots = (Zd *)(part + 2 * nch);  // nch * 64 complex
    cudaError_t e = cudaMemsetAsync(tau, 0, sizeof(double) * 2 * nb, st);
    if (e != cudaSuccess) return e;
    zpanel_first_norm<<<nch, kChunk, 0, st>>>(m, (const Zd *)P, norm_a);
    for (int i = 0; i < nb && i < m; i++) {
        double *cur = (i % 2 == 0) ? norm_a : norm_b;
        double *nxt = (i % 2 == 0) ? norm_b : norm_a;
        zpanel_refl_dots<<<nch, kChunk, 0, st>>>(m, nb, i, (Zd *)P, lda, cur, nch, dots, (Zd *)tau);
        zpanel_update<<<nch, kChunk, 0, st>>>(m, nb, i, (Zd *)P, lda, dots, nch, (const Zd *)tau, nxt, cur);
    }
    return cudaGetLastError();
}

cudaError_t zpanel_y(int m, int nb, const double *P, long long lda, double *Y, long long ldy, cudaStream_t st)
{
    zpanel_explicit_y<<<256, 256, 0, st>>>(m, nb, (const Zd *)P, lda, (Zd *)Y, ldy);
    return cudaGetLastError();
}

cudaError_t zpanel_t(int nb, const double *G, long long ldg, const double *tau, double *T, long long ldt, cudaStream_t st)
{
    zpanel_build_t<<<1, kPanelMax, 0, st>>>(nb, (const Zd *)G, ldg, (const Zd *)tau, (Zd *)T, ldt);
    return cudaGetLastError();
}

cudaError_t zband_from_full(int n, int b, const double *A, long long lda, double *AB, long long ldab, cudaStream_t st)
{
    zextract_band<<<1024, 256, 0, st>>>(n, b, (const Zd *)A, lda, (Zd *)AB, ldab);
    return cudaGetLastError();
}

cudaError_t promote_real(long long rows, long long cols, const double *X, long long ldx, double *Z, long long ldz,
                         cudaStream_t st)
{
    real_to_complex<<<1024, 256, 0, st>>>(rows, cols, X, ldx, (Zd *)Z, ldz);
    return cudaGetLastError();
}

}  // namespace gb
