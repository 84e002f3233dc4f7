// Eigenpairs of the real symmetric tridiagonal T = tridiag(e, d, e) (Sec. 2,
// Eq. 5) for the nev smallest eigenvalues, on the device.
//
// 1. Bisection on the Sturm count: the number of negative pivots of the
//    LDL^T factorisation of T - xI is the number of eigenvalues below x.  One
//    thread per eigenvalue, starting from the Gershgorin interval, halving
//    until the interval stops shrinking in FP64.
// 2. Inverse iteration, one thread per cluster: T - lambda I is factored by
//    Gaussian elimination with partial pivoting (a tridiagonal LU with one
//    extra super-diagonal from the interchanges); three solves from a
//    deterministic pseudo-random start, each followed by Gram-Schmidt
//    against the cluster's earlier vectors and normalisation.  Eigenvalues
//    closer than the cluster gap are treated together, so nearly equal
//    eigenvalues get orthogonal vectors.
// The caller finishes with one Newton-Schulz step Z <- Z (3I - Z^T Z)/2
// (two GEMMs), which makes all columns orthonormal to rounding level; it
// mixes columns i, j only by their O(u ||T|| / |lambda_i - lambda_j|)
// overlap, so residuals stay O(u ||T||).
//
// Work arrays are interleaved by eigenvalue index ([i * nev + k]) so that the
// threads of a warp access consecutive addresses.
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb {

namespace {

__device__ __forceinline__ double dabs(double x) { return x < 0 ? -x : x; }

// Gershgorin interval and the norm bound ||T||_inf (single block).
__global__ void __launch_bounds__(256) tridiag_bounds(int n, const double *__restrict__ d,
                                                      const double *__restrict__ e, double *out)
{
    __shared__ double slo[256], shi[256], snr[256];
    double lo = 1e308, hi = -1e308, nr = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double r = (i > 0 ? dabs(e[i - 1]) : 0.0) + (i < n - 1 ? dabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        nr = fmax(nr, dabs(d[i]) + r);
    }
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    snr[threadIdx.x] = nr;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            slo[threadIdx.x] = fmin(slo[threadIdx.x], slo[threadIdx.x + o]);
            shi[threadIdx.x] = fmax(shi[threadIdx.x], shi[threadIdx.x + o]);
            snr[threadIdx.x] = fmax(snr[threadIdx.x], snr[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double nrm = snr[0] > 0 ? snr[0] : 1.0;
        out[0] = slo[0] - 2.0 * 0x1p-52 * nrm;
        out[1] = shi[0] + 2.0 * 0x1p-52 * nrm;
        out[2] = nrm;
    }
}

__global__ void __launch_bounds__(256) square_offdiag(int n, const double *__restrict__ e, double *__restrict__ e2,
                                                      double *pivmin_out)
{
    // e2[i] = e[i]^2 ; pivmin = (smallest normal) * max(1, max e^2)
    __shared__ double sm[256];
    double mx = 1.0;
    for (int i = threadIdx.x; i < n - 1; i += blockDim.x) {
        double v = e[i] * e[i];
        e2[i] = v;
        mx = fmax(mx, v);
    }
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *pivmin_out = 0x1p-1022 * sm[0];
}

// Number of eigenvalues of T below x.
__device__ int sturm_count(int n, const double *__restrict__ d, const double *__restrict__ e2, double x,
                           double pivmin)
{
    int cnt = 0;
    double q = d[0] - x;
    if (dabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
#pragma unroll 4
    for (int i = 1; i < n; i++) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (dabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
    }
    return cnt;
}

__global__ void __launch_bounds__(32) tridiag_bisect(int n, int nev, const double *__restrict__ d,
                                                      const double *__restrict__ e2, const double *bounds,
                                                      const double *pivmin_p, double *__restrict__ lam)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nev) return;
    const double pivmin = *pivmin_p;
    double lo = bounds[0], hi = bounds[1];
    for (int it = 0; it < 200; it++) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;  // interval cannot shrink further
        if (sturm_count(n, d, e2, mid, pivmin) <= k) lo = mid;
        else hi = mid;
    }
    lam[k] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double start_value(int k, int i)
{
    uint32_t x = (uint32_t)k * 0x9E3779B1u ^ (uint32_t)i * 0x85EBCA77u ^ 0x1811u;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    x *= 0x297A2D39u;
    x ^= x >> 15;
    return (double)(x >> 8) * 0x1p-24 - 0.5;  // uniform in [-0.5, 0.5)
}

// One thread per cluster leader k (lam[k] - lam[k-1] > gap, or k = 0): the
// cluster's eigenvectors, written to Z (n x nev, column-major, ldz).
__global__ void __launch_bounds__(32) tridiag_invit(int n, int nev, const double *__restrict__ d,
                                                    const double *__restrict__ e, const double *__restrict__ lam,
                                                    const double *bounds, double gap_rel, double *__restrict__ A,
                                                    double *__restrict__ Bs, double *__restrict__ C,
                                                    double *__restrict__ D2, unsigned char *__restrict__ piv,
                                                    double *__restrict__ X, double *__restrict__ Z, long long ldz)
{
    const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (k0 >= nev) return;
    const double tnorm = bounds[2];
    const double gap = gap_rel * tnorm;
    if (k0 > 0 && lam[k0] - lam[k0 - 1] <= gap) return;  // not a cluster leader
    const long long S = nev;                                // interleave stride
    const double tiny = 0x1p-52 * tnorm;                    // pivot perturbation
    int k = k0;
    do {
        const double lk = lam[k];
        // ---- LU with partial pivoting of T - lk I (A: diag of U, Bs: first
        // super-diagonal, D2: second super-diagonal, C: multipliers).  The
        // row below the pivot is untouched before its step, so the running
        // diagonal and super-diagonal entries are carried in registers.
        {
            double a_cur = d[0] - lk;
            double b_cur = (n > 1) ? e[0] : 0.0;
#pragma unroll 8
            for (int i = 0; i < n - 1; i++) {
                const double c = e[i];
                const double a1 = d[i + 1] - lk;
                const double b1 = (i < n - 2) ? e[i + 1] : 0.0;
                double a = a_cur;
                if (dabs(a) >= dabs(c)) {
                    if (a == 0.0) a = tiny;
                    const double m = c / a;
                    A[i * S + k0] = a;
                    Bs[i * S + k0] = b_cur;
                    D2[i * S + k0] = 0.0;
                    C[i * S + k0] = m;
                    piv[i * S + k0] = 0;
                    a_cur = a1 - m * b_cur;
                    b_cur = b1;
                } else {
                    const double m = a / c;
                    A[i * S + k0] = c;
                    Bs[i * S + k0] = a1;
                    D2[i * S + k0] = b1;
                    C[i * S + k0] = m;
                    piv[i * S + k0] = 1;
                    a_cur = b_cur - m * a1;
                    b_cur = -m * b1;
                }
            }
            A[(n - 1) * S + k0] = (a_cur == 0.0) ? tiny : a_cur;
            Bs[(n - 1) * S + k0] = 0.0;
            D2[(n - 1) * S + k0] = 0.0;
        }
        for (int i = 0; i < n; i++) X[i * S + k0] = start_value(k, i);
        for (int iter = 0; iter < 3; iter++) {
            // forward: row interchanges and L^-1, the running entry in a register
            {
                double x_cur = X[k0];
#pragma unroll 8
                for (int i = 0; i < n - 1; i++) {
                    double x_next = X[(i + 1) * S + k0];
                    if (piv[i * S + k0]) { const double t = x_cur; x_cur = x_next; x_next = t; }
                    X[i * S + k0] = x_cur;
                    x_cur = x_next - C[i * S + k0] * x_cur;
                }
                X[(n - 1) * S + k0] = x_cur;
            }
            // backward: U^-1 (tiny pivots perturbed), the two later entries in registers
            {
                double x1 = 0.0, x2 = 0.0;
#pragma unroll 8
                for (int i = n - 1; i >= 0; i--) {
                    double sv = X[i * S + k0] - Bs[i * S + k0] * x1 - D2[i * S + k0] * x2;
                    double a = A[i * S + k0];
                    if (dabs(a) < tiny) a = (a < 0 ? -tiny : tiny);
                    const double xi = sv / a;
                    X[i * S + k0] = xi;
                    x2 = x1;
                    x1 = xi;
                }
            }
            // Gram-Schmidt against the cluster's earlier vectors (already in Z)
            for (int j = k0; j < k; j++) {
                const double *zj = Z + (long long)j * ldz;
                double dot = 0.0;
                for (int i = 0; i < n; i++) dot = fma(zj[i], X[i * S + k0], dot);
                for (int i = 0; i < n; i++) X[i * S + k0] = fma(-dot, zj[i], X[i * S + k0]);
            }
            // normalise (scale by the largest entry first to avoid overflow)
            double mx = 0.0;
            for (int i = 0; i < n; i++) mx = fmax(mx, dabs(X[i * S + k0]));
            const double sc = mx > 0 ? 1.0 / mx : 1.0;
            double nrm2 = 0.0;
            for (int i = 0; i < n; i++) {
                const double t = X[i * S + k0] * sc;
                nrm2 = fma(t, t, nrm2);
            }
            const double inv = sc / sqrt(nrm2);
            for (int i = 0; i < n; i++) X[i * S + k0] *= inv;
        }
        // deterministic sign: the entry of largest magnitude is positive
        double big = 0.0;
        for (int i = 0; i < n; i++) {
            const double t = X[i * S + k0];
            if (dabs(t) > dabs(big)) big = t;
        }
        const double sgn = big < 0 ? -1.0 : 1.0;
        double *zk = Z + (long long)k * ldz;
        for (int i = 0; i < n; i++) zk[i] = sgn * X[i * S + k0];
        k++;
    } while (k < nev && lam[k] - lam[k - 1] <= gap);
}

}  // namespace

size_t tridiag_eig_workspace_bytes(int n, int nev)
{
    size_t per = (size_t)n * (size_t)nev;
    size_t bytes = 256 + 2 * 256 + (size_t)n * 8 + 5 * per * 8 + per;  // bounds, e2, arrays, piv
    return (bytes + 255) & ~(size_t)255;
}

// lam (nev) and Z (n x nev, ldz) of the tridiagonal (d, e); before the final
// orthogonalisation step, which the caller applies.  Two phases so that the
// caller can time them separately.
static void carve_eig(int n, int nev, void *ws, double **bounds, double **pivmin, double **e2, double **A,
                      double **Bs, double **C, double **D2, double **X, unsigned char **piv)
{
    char *p = (char *)ws;
    size_t per = (size_t)n * (size_t)nev;
    *bounds = (double *)p;            // lo, hi, ||T||
    *pivmin = (double *)(p + 256);
    *e2 = (double *)(p + 512);
    *A = *e2 + n;
    *Bs = *A + per;
    *C = *Bs + per;
    *D2 = *C + per;
    *X = *D2 + per;
    *piv = (unsigned char *)(*X + per);
}

cudaError_t tridiag_bisect_d(int n, int nev, const double *d, const double *e, double *lam, void *ws, cudaStream_t st)
{
    double *bounds, *pivmin, *e2, *A, *Bs, *C, *D2, *X;
    unsigned char *piv;
    carve_eig(n, nev, ws, &bounds, &pivmin, &e2, &A, &Bs, &C, &D2, &X, &piv);
    tridiag_bounds<<<1, 256, 0, st>>>(n, d, e, bounds);
    square_offdiag<<<1, 256, 0, st>>>(n, e, e2, pivmin);
    // one warp per block: the per-eigenvalue chains are latency-bound, so
    // they are spread over as many SMs as possible
    tridiag_bisect<<<(nev + 31) / 32, 32, 0, st>>>(n, nev, d, e2, bounds, pivmin, lam);
    return cudaGetLastError();
}

cudaError_t tridiag_invit_d(int n, int nev, const double *d, const double *e, const double *lam, double *Z,
                            long long ldz, void *ws, cudaStream_t st)
{
    double *bounds, *pivmin, *e2, *A, *Bs, *C, *D2, *X;
    unsigned char *piv;
    carve_eig(n, nev, ws, &bounds, &pivmin, &e2, &A, &Bs, &C, &D2, &X, &piv);
    tridiag_invit<<<(nev + 31) / 32, 32, 0, st>>>(n, nev, d, e, lam, bounds, 1e-7, A, Bs, C, D2, piv, X, Z, ldz);
    return cudaGetLastError();
}

cudaError_t tridiag_eig_d(int n, int nev, const double *d, const double *e, double *lam, double *Z, long long ldz,
                          void *ws, cudaStream_t st)
{
    cudaError_t err = tridiag_bisect_d(n, nev, d, e, lam, ws, st);
    if (err != cudaSuccess) return err;
    return tridiag_invit_d(n, nev, d, e, lam, Z, ldz, ws, st);
}

}  // namespace gb
