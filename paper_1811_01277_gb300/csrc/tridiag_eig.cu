// Eigenpairs of the real symmetric tridiagonal T = tridiag(e, d, e) (Sec. 2,
// Eq. 5) for the nev smallest eigenvalues, on the device.
//
// 1. Multisection on the Sturm count: the number of negative pivots of the
//    LDL^T factorisation of T - xI is the number of eigenvalues below x.
//    Four lanes per eigenvalue evaluate the count at four interior points of
//    the current interval (which shrinks five-fold per round), starting from
//    the Gershgorin interval, until it stops shrinking in FP64.
// 2. Inverse iteration, one thread per eigenvalue: T - lambda I is factored
//    by Gaussian elimination with partial pivoting (a tridiagonal LU with one
//    extra super-diagonal from the interchanges); three solves from a
//    deterministic pseudo-random start, each followed by normalisation.
// 3. One block per cluster of eigenvalues closer than the cluster gap:
//    modified Gram-Schmidt (twice) of the cluster's vectors, so nearly equal
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

#include "tridiag_eig.cuh"

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

// |x| as an ordered integer key: for finite a, b, |a| < |b| iff
// abs_key(a) < abs_key(b).  Comparisons and sign tests on the bit pattern run
// on the integer pipes, not on the (narrow) FP64 pipe.
__device__ __forceinline__ unsigned long long abs_key(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__device__ __forceinline__ int sign_bit(double x) { return (int)((unsigned)__double2hiint(x) >> 31); }

// 1/q by Newton-Raphson refinement r <- r + r(1 - q r) (each step squares the
// relative error) of the hardware's approximate FP64 reciprocal
// (rcp.approx.ftz.f64): two steps give the reciprocal to about one ulp with
// four FMAs.  Outside 2^-1000 <= |q| < 2^1000, where the approximation
// flushes to zero or overflows, the IEEE division is used.
__device__ __forceinline__ double recip(double q)
{
    const unsigned ex = ((unsigned)__double2hiint(q) >> 20) & 0x7FFu;
    if (ex - 23u < 2000u) {
        double r;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(q));
        double t = fma(-q, r, 1.0);
        r = fma(r, t, r);
        t = fma(-q, r, 1.0);
        return fma(r, t, r);
    }
    return 1.0 / q;
}

// Number of eigenvalues of T below x: negative pivots of the LDL^T
// factorisation of T - xI (Sylvester's law of inertia), pivots smaller than
// pivmin in magnitude replaced by -pivmin.
__device__ __forceinline__ int sturm_count(int n, const double *__restrict__ d, const double *__restrict__ e2,
                                           double x, double pivmin, unsigned long long pivkey)
{
    double q = d[0] - x;
    if (abs_key(q) < pivkey) q = -pivmin;
    int cnt = sign_bit(q);
#pragma unroll 4
    for (int i = 1; i < n; i++) {
        q = fma(-e2[i - 1], recip(q), d[i] - x);
        if (abs_key(q) < pivkey) q = -pivmin;
        cnt += sign_bit(q);
    }
    return cnt;
}

// Multisection: kMultisect lanes per eigenvalue k (0-based, ascending).  In
// each round the lanes evaluate the Sturm count at the kMultisect points that
// split [lo, hi] into kMultisect + 1 equal parts, exchange the counts, and the
// group keeps the part in which the count passes k.  Rounds stop when the
// interval is within max(u ||T||, 2 (kMultisect + 1) u |x|) or cannot shrink.
constexpr int kMultisect = 4;

__global__ void __launch_bounds__(128) tridiag_bisect(int n, int nev, const double *__restrict__ d,
                                                       const double *__restrict__ e2, const double *bounds,
                                                       const double *pivmin_p, double *__restrict__ lam)
{
    constexpr int P = kMultisect;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = gt / P;
    const int j = gt % P;
    const int lane0 = (threadIdx.x & 31) & ~(P - 1);  // first lane of this group in the warp
    const double pivmin = *pivmin_p;
    const unsigned long long pivkey = abs_key(pivmin);
    const double abstol = 0x1p-53 * bounds[2];
    double lo = bounds[0], hi = bounds[1];
    bool done = k >= nev;
    for (int round = 0; round < 400; round++) {
        const double w = hi - lo;
        if (!done) {
            const double tol = fmax(abstol, (2.0 * (P + 1) * 0x1p-53) * fmax(fabs(lo), fabs(hi)));
            done = !(w > tol);
        }
        if (__all_sync(0xffffffffu, done)) break;
        const double h = w * (1.0 / (P + 1));
        const int c = done ? 0 : sturm_count(n, d, e2, fma((double)(j + 1), h, lo), pivmin, pivkey);
        int first = P;  // first point whose count exceeds k
#pragma unroll
        for (int m = P - 1; m >= 0; m--) {
            const int cm = __shfl_sync(0xffffffffu, c, lane0 + m);
            if (cm > k) first = m;
        }
        if (!done) {
            const double nlo = (first == 0) ? lo : fma((double)first, h, lo);
            const double nhi = (first == P) ? hi : fma((double)(first + 1), h, lo);
            if (nlo <= lo && nhi >= hi) done = true;  // no progress in FP64
            lo = nlo;
            hi = nhi;
        }
    }
    if (j == 0 && k < nev) lam[k] = 0.5 * (lo + hi);
}

// Deterministic pseudo-random start vector entry in [-0.5, 0.5): 52 hashed
// bits placed in the mantissa of a number in [1, 2), then shifted.
__device__ __forceinline__ double start_value(int k, int i)
{
    uint32_t x = (uint32_t)k * 0x9E3779B1u ^ (uint32_t)i * 0x85EBCA77u ^ 0x1811u;
    x ^= x >> 15;
    x *= 0x2C1B3C6Du;
    x ^= x >> 12;
    x *= 0x297A2D39u;
    x ^= x >> 15;
    const uint32_t y = x * 0x9E3779B1u ^ (x >> 16);
    return __hiloint2double(0x3FF00000 | (int)(x >> 12), (int)(y ^ (x << 20))) - 1.5;
}

// One thread per eigenvalue k: its inverse-iteration vector, normalised
// (largest entry positive), written to column k of Z (n x nev, column-major,
// ldz).  Eigenvalues closer than the cluster gap are orthogonalised
// afterwards by cluster_orthonormalise.
//
// Per eigenvalue: one pass factors P(T - lk I) = LU with partial pivoting
// (U0 = 1/pivot, U1 = first super-diagonal of U, Cm = multiplier, piv =
// interchange; the second super-diagonal is e[i+1] where piv[i] = 1, else 0)
// and applies L^-1 P to the start vector on the fly (Y); then three rounds of
// back substitution U^-1 (Y -> X, tracking max |x|) and -- for the next
// round -- L^-1 P applied to X (X -> Y, X first rescaled by 1/max|x| only
// when max|x| leaves [2^-200, 2^200]).  Each vector uses its own eigenvalue
// as the shift, so components along other eigenvectors shrink by
// (|lk - lambda_k| / |lk - lambda_i|)^3 in three rounds: vectors of close
// but distinct eigenvalues separate by themselves, and those of eigenvalues
// equal to working accuracy are independent combinations (different start
// vectors) of the same invariant subspace, which the cluster step makes
// orthonormal.
//
// Every pass is a chain over rows, so memory latency, not arithmetic, bounds
// it: rows are processed in blocks of kRows, all loads of a block are issued
// before its chain steps (and an L2 prefetch runs kPrefetch rows ahead), so a
// block pays one memory latency.  Pivoting decisions and magnitude tracking
// use integer compares of the bit patterns, and each pivot costs one
// reciprocal.  Work arrays are interleaved by thread ([i * S + k]) so that a
// warp's accesses to one row are contiguous.
__device__ __forceinline__ double select(bool c, double a, double b) { return c ? a : b; }

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

constexpr int kRows = 8;        // rows per staged block
constexpr int kRowsLU = 8;      // rows per staged block of the factorisation pass
constexpr int kPrefetch = 64;   // L2 prefetch distance, rows
constexpr double kClusterGap = 1e-7;  // relative to ||T||

__device__ __forceinline__ double rcp_pivot(double p, unsigned long long tiny_key, double inv_tiny)
{
    return (abs_key(p) < tiny_key) ? (sign_bit(p) ? -inv_tiny : inv_tiny) : recip(p);
}

__global__ void __launch_bounds__(32) tridiag_invit(int n, int nev, const double *__restrict__ d,
                                                    const double *__restrict__ e, const double *__restrict__ lam,
                                                    const double *__restrict__ bounds,
                                                    double *__restrict__ U0, double *__restrict__ U1,
                                                    double *__restrict__ Cm, unsigned char *__restrict__ piv,
                                                    double *__restrict__ Y, double *__restrict__ X,
                                                    double *__restrict__ Z, long long ldz)
{
    constexpr int R = kRows;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nev) return;
    const double tnorm = bounds[2];
    const long long S = nev;                                // interleave stride
    const double tiny = 0x1p-52 * tnorm;                    // smallest pivot magnitude used
    const unsigned long long tiny_key = abs_key(tiny);
    const double inv_tiny = 1.0 / tiny;
    U0 += k;
    U1 += k;
    Cm += k;
    piv += k;
    Y += k;
    X += k;
    {
        const double lk = lam[k];
        // ---- factor and apply L^-1 P to the start vector (step i eliminates
        // row i+1 with rows i, i+1 pivoted)
        {
            double a_cur = d[0] - lk;
            double b_cur = (n > 1) ? e[0] : 0.0;
            double y_cur = start_value(k, 0);
            constexpr int RL = kRowsLU;
            for (int i0 = 0; i0 < n - 1; i0 += RL) {
                double cv[RL], av[RL], bv[RL];
#pragma unroll
                for (int r = 0; r < RL; r++) {
                    const int i = i0 + r;
                    cv[r] = (i < n - 1) ? e[i] : 0.0;
                    av[r] = (i < n - 1) ? d[i + 1] : 0.0;
                    bv[r] = (i < n - 2) ? e[i + 1] : 0.0;
                }
#pragma unroll
                for (int r = 0; r < RL; r++) {
                    const int i = i0 + r;
                    if (i < n - 1) {
                        const double c = cv[r], a1 = av[r] - lk, b1 = bv[r];
                        const double y_next = start_value(k, i + 1);
                        const unsigned long long ka = abs_key(a_cur), kc = abs_key(c);
                        const bool sw = kc > ka;  // interchange rows i and i+1
                        const double p = sw ? c : (ka == 0 ? tiny : a_cur);
                        const double rp = recip(p);
                        const double m = (sw ? a_cur : c) * rp;
                        U0[i * S] = (abs_key(p) < tiny_key) ? (sign_bit(p) ? -inv_tiny : inv_tiny) : rp;
                        U1[i * S] = select(sw, a1, b_cur);
                        Cm[i * S] = m;
                        piv[i * S] = sw;
                        Y[i * S] = select(sw, y_next, y_cur);
                        y_cur = fma(-m, select(sw, y_next, y_cur), select(sw, y_cur, y_next));
                        a_cur = fma(-m, select(sw, a1, b_cur), select(sw, b_cur, a1));
                        b_cur = b1 * select(sw, -m, 1.0);
                    }
                }
            }
            U0[(n - 1) * S] = rcp_pivot((abs_key(a_cur) == 0) ? tiny : a_cur, tiny_key, inv_tiny);
            U1[(n - 1) * S] = 0.0;
            piv[(n - 1) * S] = 0;
            Y[(n - 1) * S] = y_cur;
        }
        unsigned long long mx_key = 0;
        for (int iter = 0; iter < 3; iter++) {
            if (iter > 0) {
                // L^-1 P X -> Y (X rescaled first if its magnitude drifted far)
                if (mx_key < abs_key(0x1p-200) || mx_key > abs_key(0x1p200)) {
                    const double sc = (mx_key == 0) ? 1.0 : recip(__longlong_as_double((long long)mx_key));
                    for (int i = 0; i < n; i++) X[i * S] *= sc;
                }
                double y_cur = X[0];
                for (int i0 = 0; i0 < n - 1; i0 += R) {
                    double xv[R], mv[R];
                    bool pv[R];
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int i = i0 + r;
                        if (i < n - 1) {
                            xv[r] = X[(i + 1) * S];
                            mv[r] = Cm[i * S];
                            pv[r] = piv[i * S];
                        }
                    }
                    {
                        const long long ip = (long long)min(i0 + kPrefetch, n - 1) * S;
#pragma unroll
                        for (int r = 0; r < R; r += 4) {
                            const long long q = ip + (long long)min(r, n - 1 - min(i0 + kPrefetch, n - 1)) * S;
                            prefetch_l2(X + q);
                            prefetch_l2(Cm + q);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int i = i0 + r;
                        if (i < n - 1) {
                            const bool sw = pv[r];
                            const double y_next = xv[r];
                            Y[i * S] = select(sw, y_next, y_cur);
                            y_cur = fma(-mv[r], select(sw, y_next, y_cur), select(sw, y_cur, y_next));
                        }
                    }
                }
                Y[(n - 1) * S] = y_cur;
            }
            // U^-1 Y -> X, with max |x|
            {
                double x1 = 0.0, x2 = 0.0;
                mx_key = 0;
                for (int i0 = n - 1; i0 >= 0; i0 -= R) {
                    double yv[R], u1v[R], u0v[R], d2v[R];
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int i = i0 - r;
                        if (i >= 0) {
                            yv[r] = Y[i * S];
                            u1v[r] = U1[i * S];
                            u0v[r] = U0[i * S];
                            d2v[r] = (i < n - 2 && piv[i * S]) ? e[i + 1] : 0.0;
                        }
                    }
                    {
                        const int ib = max(i0 - kPrefetch, 0);
#pragma unroll
                        for (int r = 0; r < R; r += 4) {
                            const long long q = (long long)max(ib - r, 0) * S;
                            prefetch_l2(Y + q);
                            prefetch_l2(U1 + q);
                            prefetch_l2(U0 + q);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < R; r++) {
                        const int i = i0 - r;
                        if (i >= 0) {
                            const double t = fma(-d2v[r], x2, yv[r]);
                            const double xi = fma(-u1v[r], x1, t) * u0v[r];
                            X[i * S] = xi;
                            x2 = x1;
                            x1 = xi;
                            const unsigned long long kx = abs_key(xi);
                            mx_key = kx > mx_key ? kx : mx_key;
                        }
                    }
                }
            }
        }
        // ---- normalise (sum of squares of X / max|x|); the entry of largest
        // magnitude (the first, scanning upwards from row 0) is made positive
        const double sc = (mx_key == 0) ? 1.0 : recip(__longlong_as_double((long long)mx_key));
        double ssq[4] = {0.0, 0.0, 0.0, 0.0}, big = 0.0;
        for (int i0 = 0; i0 < n; i0 += R) {
            double xv[R];
#pragma unroll
            for (int r = 0; r < R; r++) xv[r] = (i0 + r < n) ? X[(i0 + r) * S] : 0.0;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const double t = xv[r] * sc;
                ssq[r & 3] = fma(t, t, ssq[r & 3]);
                if (abs_key(xv[r]) == mx_key && big == 0.0) big = xv[r];
            }
        }
        const double nrm = sqrt((ssq[0] + ssq[1]) + (ssq[2] + ssq[3])) *
                           __longlong_as_double((long long)(mx_key == 0 ? abs_key(1.0) : mx_key));
        const double f = nrm > 0.0 ? (sign_bit(big) ? -1.0 : 1.0) / nrm : 0.0;
        double *zk = Z + (long long)k * ldz;
        for (int i0 = 0; i0 < n; i0 += R) {
            double xv[R];
#pragma unroll
            for (int r = 0; r < R; r++) xv[r] = (i0 + r < n) ? X[(i0 + r) * S] : 0.0;
#pragma unroll
            for (int r = 0; r < R; r++)
                if (i0 + r < n) zk[i0 + r] = xv[r] * f;
        }
    }
}

// Sum over a block of 256 threads (all threads get the result).
__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();  // red is free (previous use finished)
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

__device__ __forceinline__ unsigned long long block_max_key(unsigned long long v, unsigned long long *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    unsigned long long t = (l < (int)(blockDim.x >> 5)) ? red[l] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, t, o);
        t = u > t ? u : t;
    }
    return t;
}

// One block per cluster of eigenvalues closer than the gap (consecutive
// differences <= gap, two or more members): modified Gram-Schmidt of the
// members' columns of Z in order, each member orthogonalised twice against
// the earlier ones, then normalised with its largest entry positive.  Rows
// are spread over the block, so each dot product is one block reduction.
__global__ void __launch_bounds__(256) cluster_orthonormalise(int n, int nev, const double *__restrict__ lam,
                                                              const double *__restrict__ bounds, double gap_rel,
                                                              double *__restrict__ Z, long long ldz)
{
    __shared__ double red[32];
    __shared__ unsigned long long redk[32];
    const int k0 = blockIdx.x;
    const double gap = gap_rel * bounds[2];
    if (k0 > 0 && lam[k0] - lam[k0 - 1] <= gap) return;   // not the first member
    if (k0 + 1 >= nev || lam[k0 + 1] - lam[k0] > gap) return;  // a single eigenvalue
    int k1 = k0 + 1;
    while (k1 + 1 < nev && lam[k1 + 1] - lam[k1] <= gap) k1++;
    for (int k = k0 + 1; k <= k1; k++) {
        double *zk = Z + (long long)k * ldz;
        for (int pass = 0; pass < 2; pass++) {
            for (int j = k0; j < k; j++) {
                const double *zj = Z + (long long)j * ldz;
                double s = 0.0;
                for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(zj[i], zk[i], s);
                const double dot = block_sum(s, red);
                for (int i = threadIdx.x; i < n; i += blockDim.x) zk[i] = fma(-dot, zj[i], zk[i]);
            }
        }
        unsigned long long mk = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long t = abs_key(zk[i]);
            mk = t > mk ? t : mk;
        }
        mk = block_max_key(mk, redk);
        const double sc = (mk == 0) ? 1.0 : recip(__longlong_as_double((long long)mk));
        double s2 = 0.0;
        int first = n;  // first row holding the largest magnitude
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double t = zk[i] * sc;
            s2 = fma(t, t, s2);
            if (abs_key(zk[i]) == mk && i < first) first = i;
        }
        const double nrm = sqrt(block_sum(s2, red)) * __longlong_as_double((long long)(mk == 0 ? abs_key(1.0) : mk));
        // smallest such row over the block
        __syncthreads();
        if (threadIdx.x < 32) redk[threadIdx.x] = ~0ull;
        __syncthreads();
        atomicMin(&redk[0], (unsigned long long)first);
        __syncthreads();
        const int f0 = (int)redk[0];
        const double big = (f0 < n) ? zk[f0] : 1.0;
        const double f = nrm > 0.0 ? (sign_bit(big) ? -1.0 : 1.0) / nrm : 0.0;
        __syncthreads();  // every thread has read zk[f0]
        for (int i = threadIdx.x; i < n; i += blockDim.x) zk[i] *= f;
        __syncthreads();  // column k final before the next member reads it
    }
}

}  // namespace

size_t tridiag_eig_workspace_bytes(int n, int nev)
{
    size_t per = (size_t)n * (size_t)nev;
    size_t bytes = 256 + 2 * 256 + (size_t)n * 8 + 5 * per * 8 + per;  // bounds, e2, arrays, piv
    return (bytes + 255) & ~(size_t)255;
}

namespace {

struct EigWork {
    double *bounds;  // lo, hi, ||T||
    double *pivmin;
    double *e2;
    double *U0, *U1, *Cm, *Y, *X;  // n x nev each, interleaved
    unsigned char *piv;
};

EigWork carve_eig(int n, int nev, void *ws)
{
    EigWork w;
    char *p = (char *)ws;
    size_t per = (size_t)n * (size_t)nev;
    w.bounds = (double *)p;
    w.pivmin = (double *)(p + 256);
    w.e2 = (double *)(p + 512);
    w.U0 = w.e2 + n;
    w.U1 = w.U0 + per;
    w.Cm = w.U1 + per;
    w.Y = w.Cm + per;
    w.X = w.Y + per;
    w.piv = (unsigned char *)(w.X + per);
    return w;
}

int clamp_threads(int threads) { return threads < 1 ? 1 : threads > 32 ? 32 : threads; }

}  // namespace

// lam (nev) and Z (n x nev, ldz) of the tridiagonal (d, e); before the final
// orthogonalisation step, which the caller applies.  Two phases so that the
// caller can time them separately.  `threads` = threads per block (1..32):
// the per-eigenvalue chains are latency-bound, so they are spread over as
// many SMs and schedulers as possible.
cudaError_t tridiag_bisect_d(int n, int nev, const double *d, const double *e, double *lam, void *ws, cudaStream_t st)
{
    EigWork w = carve_eig(n, nev, ws);
    tridiag_bounds<<<1, 256, 0, st>>>(n, d, e, w.bounds);
    square_offdiag<<<1, 256, 0, st>>>(n, e, w.e2, w.pivmin);
    const long long lanes = (long long)nev * kMultisect;
    tridiag_bisect<<<(unsigned)((lanes + 127) / 128), 128, 0, st>>>(n, nev, d, w.e2, w.bounds, w.pivmin, lam);
    return cudaGetLastError();
}

cudaError_t tridiag_invit_d(int n, int nev, const double *d, const double *e, const double *lam, double *Z,
                            long long ldz, void *ws, cudaStream_t st, int threads)
{
    EigWork w = carve_eig(n, nev, ws);
    threads = clamp_threads(threads);
    tridiag_invit<<<(nev + threads - 1) / threads, threads, 0, st>>>(n, nev, d, e, lam, w.bounds, w.U0, w.U1, w.Cm,
                                                                      w.piv, w.Y, w.X, Z, ldz);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    cluster_orthonormalise<<<nev, 256, 0, st>>>(n, nev, lam, w.bounds, kClusterGap, Z, ldz);
    return cudaGetLastError();
}

cudaError_t tridiag_eig_d(int n, int nev, const double *d, const double *e, double *lam, double *Z, long long ldz,
                          void *ws, cudaStream_t st)
{
    cudaError_t err = tridiag_bisect_d(n, nev, d, e, lam, ws, st);
    if (err != cudaSuccess) return err;
    return tridiag_invit_d(n, nev, d, e, lam, Z, ldz, ws, st, kTridiagThreads);
}

}  // namespace gb
