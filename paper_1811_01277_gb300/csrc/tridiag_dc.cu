// Divide and conquer for all eigenpairs of a real symmetric tridiagonal
// matrix T (the tridiagonal step of the two-stage solver, Sec. 2, when every
// eigenvector is wanted): Cuppen's splitting with the deflation of small
// couplings and close poles, the secular equation solved per root, the
// Gu-Eisenstat recomputation of the rank-one vector (orthogonal eigenvectors
// without extra precision), and the merged eigenvectors as products on the
// tensor cores.
//
// Tree: T is cut into 2^D leaves of one or two rows by repeated halving
// (left half floor(s/2)); every node of depth t < D is a merge.  Leaves this
// small have closed-form eigenpairs, so all the work is in the merges, whose
// steps run in parallel over roots and columns (a serial eigensolver per
// leaf is a chain of scalar FP64 operations, and each costs a warp
// instruction's full issue time on this part's narrow FP64 pipe).  At the cut
// between rows k and k+1 with coupling beta = e[k],
//     T = diag(T1', T2') + rho u u^T,  rho = |beta|,  u = e_k + sign(beta) e_{k+1},
// with T1', T2' the halves whose touching diagonal entries are reduced by rho.
// The merges run bottom-up, all merges of one depth in the same launches.
//
// One merge (size s = n1 + n2, children's eigenpairs (D1, Q1), (D2, Q2)):
//   * z = [last row of Q1, sign(beta) first row of Q2] / sqrt 2, rho' = 2 rho;
//     D sorted by a stable merge of the two ascending lists (permutation P);
//   * deflation (one thread, in ascending order): a component with
//     rho' |z_j| <= tol drops out; two neighbours whose poles are so close
//     that the rotation zeroing one z-component leaves an off-diagonal
//     |t c s| <= tol are rotated (G) and one of them drops out;
//     tol = 8 eps max(max |d|, max |z|);
//   * the K remaining roots of 1 + rho' sum z_j^2 / (d_j - lambda) = 0, one
//     per warp: lambda_k = d_o + tau with the origin d_o the nearer pole
//     (k or k+1), iterated by the two-pole rational model of Bunch, Nielsen
//     and Sorensen, safeguarded by bisection of the bracket;
//   * zhat_j^2 = prod_k (lambda_k - d_j) / (rho' prod_{k != j} (d_k - d_j)),
//     sign of z_j (Gu and Eisenstat), from the stored (o, tau) so that every
//     difference lambda_k - d_j = (d_o - d_j) + tau is accurate;
//   * eigenvector k of the deflated problem: zhat_j / (d_j - lambda_k),
//     normalised; a dropped component is its own unit vector;
//   * U = P G [eigenvectors] with the columns in ascending eigenvalue order,
//     so the merged eigenvectors are diag(Q1, Q2) U: two products,
//     Q1 U[:n1, :] and Q2 U[n1:, :] (sliced on the tensor cores when large,
//     a batched DFMA kernel when small).
// Every loop is bounded; T is scaled by its largest entry first.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "dgemm_sliced.cuh"
#include "elpa_gb300.h"

namespace gb {

namespace {

constexpr int kDcLeaf = 2;
constexpr int kDcSetupThreads = 256;
constexpr int kSecularIters = 100;
constexpr int kSmemColumnMax = 24576;   // build_u keeps a column in shared memory up to this size
constexpr int kSetupSmemRows = 12288;   // setup stages a merge's sorted d and z in shared memory up to this size
constexpr double kEps = 1.1102230246251565e-16;  // 2^-53
constexpr double kSlicedMinFlops = 5e7;  // per product; the merges' products are square-ish

__host__ __device__ inline int dc_depth(int n)
{
    int D = 0;
    while ((n + (1 << D) - 1) / (1 << D) > kDcLeaf) D++;
    return D;
}

// offset and size of node m of depth t (left halves floor(s/2))
__host__ __device__ inline void dc_node(int n, int t, int m, int *off, int *sz)
{
    int o = 0, s = n;
    for (int b = t - 1; b >= 0; b--) {
        const int left = s / 2;
        if ((m >> b) & 1) {
            o += left;
            s -= left;
        } else {
            s = left;
        }
    }
    *off = o;
    *sz = s;
}

// node of depth t containing row g
__device__ inline int dc_node_of(int n, int t, int g, int *off, int *sz)
{
    int o = 0, s = n, m = 0;
    for (int b = 0; b < t; b++) {
        const int left = s / 2;
        m <<= 1;
        if (g >= o + left) {
            o += left;
            s -= left;
            m |= 1;
        } else {
            s = left;
        }
    }
    *off = o;
    *sz = s;
    return m;
}

// per-position arrays of the merges of one depth (each merge uses the slice
// [off, off + s) of every array) and one counter triple per merge at [off]
struct DcArrays {
    double *ds, *zs, *dK, *zK, *tau, *lamK, *zhat, *defl_d, *rot_c, *rot_s, *rho;
    int *perm, *ndidx, *ndpos, *org, *defl_idx, *rot_p, *rot_j, *colsrc, *cnt;  // cnt[3 off]: K, deflated, rotations
};

__device__ inline double block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (l == 0) red[0] = v;
    }
    __syncthreads();
    return red[0];
}

__device__ inline double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) red[0] = v;
    }
    __syncthreads();
    return red[0];
}

// The scale of T: its largest entry (1 for a zero matrix).  One block.
__global__ void __launch_bounds__(1024) dc_scale(int n, const double *__restrict__ d, const double *__restrict__ e,
                                                 double *__restrict__ scale)
{
    __shared__ double red[32];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(d[i]));
    for (int i = threadIdx.x; i < n - 1; i += blockDim.x) m = fmax(m, fabs(e[i]));
    m = block_max(m, red);
    if (threadIdx.x == 0) *scale = m > 0.0 && isfinite(m) ? m : 1.0;
}

// One leaf (one or two rows) per thread: its rows of the scaled T with the
// diagonal reduced by |e| at the cuts on either side (every leaf boundary is
// a cut), and the closed-form eigenpairs, in ascending order, into lam[off..]
// and the diagonal block of Q.  A 2 x 2
// block [a b; b c] is diagonalised by the rotation with t = tan(theta),
// |theta| <= pi/4: eigenvalues a - t b and c + t b, eigenvectors
// (cs, -sn) and (sn, cs).
__global__ void dc_leaf(int n, int D, const double *__restrict__ d, const double *__restrict__ e,
                        const double *__restrict__ scale, double *__restrict__ lam, double *__restrict__ Q)
{
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= (1 << D)) return;
    int off, m;
    dc_node(n, D, leaf, &off, &m);
    const size_t ld = (size_t)n;
    const double sc = *scale;
    const double cut_lo = off > 0 ? fabs(e[off - 1] / sc) : 0.0;
    const double cut_hi = off + m < n ? fabs(e[off + m - 1] / sc) : 0.0;
    if (m == 1) {
        lam[off] = d[off] / sc - cut_lo - cut_hi;
        Q[off + off * ld] = 1.0;
        return;
    }
    const double a = d[off] / sc - cut_lo, b = e[off] / sc, c = d[off + 1] / sc - cut_hi;
    double l0 = a, l1 = c, cs = 1.0, sn = 0.0;
    if (b != 0.0) {
        const double zeta = (c - a) / (2.0 * b);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        cs = 1.0 / sqrt(1.0 + t * t);
        sn = t * cs;
        l0 = a - t * b;
        l1 = c + t * b;
    }
    // columns: (cs, -sn) for l0, (sn, cs) for l1; ascending
    const bool sw = l1 < l0;
    lam[off] = sw ? l1 : l0;
    lam[off + 1] = sw ? l0 : l1;
    double *q0 = Q + off + off * ld, *q1 = Q + off + (off + 1) * ld;
    q0[0] = sw ? sn : cs;
    q0[1] = sw ? cs : -sn;
    q1[0] = sw ? cs : sn;
    q1[1] = sw ? -sn : cs;
}

// Per merge (one block): z, the sorted order, deflation, and the lists the
// later kernels read.
__global__ void __launch_bounds__(kDcSetupThreads) dc_setup(int n, int t, const double *__restrict__ Q,
                                                            const double *__restrict__ lam,
                                                            const double *__restrict__ e,
                                                            const double *__restrict__ scale, DcArrays a,
                                                            int smem_rows)
{
    __shared__ double red[32];
    extern __shared__ double stage[];  // sorted d and z for the serial scan (smem_rows entries each)
    int off, s;
    dc_node(n, t, blockIdx.x, &off, &s);
    const int n1 = s / 2, k = off + n1 - 1;
    const double beta = e[k] / *scale;
    const double rho = fabs(beta), sg = beta >= 0.0 ? 1.0 : -1.0;
    const double r2 = 0.7071067811865476;
    // stable merge of the ascending halves: rank of each entry
    double dmax = 0.0, zmax = 0.0;
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const double v = lam[off + j];
        int lo, hi, rank;
        if (j < n1) {  // entries of the right half below v
            lo = 0;
            hi = s - n1;
            while (lo < hi) {
                const int md = (lo + hi) >> 1;
                if (lam[off + n1 + md] < v) lo = md + 1;
                else hi = md;
            }
            rank = j + lo;
        } else {  // entries of the left half at or below v
            lo = 0;
            hi = n1;
            while (lo < hi) {
                const int md = (lo + hi) >> 1;
                if (lam[off + md] <= v) lo = md + 1;
                else hi = md;
            }
            rank = (j - n1) + lo;
        }
        const double z = j < n1 ? Q[(size_t)(off + n1 - 1) + (size_t)(off + j) * n] * r2
                                : sg * Q[(size_t)(off + n1) + (size_t)(off + j) * n] * r2;
        a.perm[off + rank] = j;
        if (s <= smem_rows) {
            stage[rank] = v;
            stage[smem_rows + rank] = z;
        } else {
            a.ds[off + rank] = v;
            a.zs[off + rank] = z;
        }
        dmax = fmax(dmax, fabs(v));
        zmax = fmax(zmax, fabs(z));
    }
    dmax = block_max(dmax, red);
    zmax = block_max(zmax, red);
    if (threadIdx.x != 0) return;
    const double rho2 = 2.0 * rho;
    const double tol = 8.0 * kEps * fmax(dmax, zmax);
    double *ds = s <= smem_rows ? stage : a.ds + off, *zs = s <= smem_rows ? stage + smem_rows : a.zs + off;
    int K = 0, nd = 0, nr = 0, pend = -1;
    for (int j = 0; j < s; j++) {
        a.ndpos[off + j] = -1;
        if (rho2 * fabs(zs[j]) <= tol) {
            a.defl_idx[off + nd] = j;
            a.defl_d[off + nd] = ds[j];
            nd++;
            continue;
        }
        if (pend < 0) {
            pend = j;
            continue;
        }
        const double sv = zs[pend], cv = zs[j];
        const double tt = ds[j] - ds[pend];
        // |t c s| <= tol with c s = -z_p z_j / (z_p^2 + z_j^2): tested
        // without the square root first (most pairs fail it)
        if (fabs(tt) * fabs(sv) * fabs(cv) <= tol * (sv * sv + cv * cv)) {
            const double tau = hypot(cv, sv);
            const double c = cv / tau, sn = -sv / tau;
            zs[j] = tau;
            zs[pend] = 0.0;
            const double dp = ds[pend] * c * c + ds[j] * sn * sn;
            const double dj = ds[pend] * sn * sn + ds[j] * c * c;
            a.rot_p[off + nr] = pend;
            a.rot_j[off + nr] = j;
            a.rot_c[off + nr] = c;
            a.rot_s[off + nr] = sn;
            nr++;
            ds[j] = dj;
            ds[pend] = dp;
            a.defl_idx[off + nd] = pend;
            a.defl_d[off + nd] = dp;
            nd++;
            pend = j;
            continue;
        }
        a.ndidx[off + K] = pend;
        a.ndpos[off + pend] = K;
        a.dK[off + K] = ds[pend];
        a.zK[off + K] = zs[pend];
        K++;
        pend = j;
    }
    if (pend >= 0) {
        a.ndidx[off + K] = pend;
        a.ndpos[off + pend] = K;
        a.dK[off + K] = ds[pend];
        a.zK[off + K] = zs[pend];
        K++;
    }
    // the dropped values are nearly ascending already: insertion sort
    for (int i = 1; i < nd; i++) {
        const double v = a.defl_d[off + i];
        const int id = a.defl_idx[off + i];
        int j = i - 1;
        while (j >= 0 && a.defl_d[off + j] > v) {
            a.defl_d[off + j + 1] = a.defl_d[off + j];
            a.defl_idx[off + j + 1] = a.defl_idx[off + j];
            j--;
        }
        a.defl_d[off + j + 1] = v;
        a.defl_idx[off + j + 1] = id;
    }
    a.cnt[3 * off] = K;
    a.cnt[3 * off + 1] = nd;
    a.cnt[3 * off + 2] = nr;
    a.rho[off] = rho2;
}

// Warp reductions to lane 0, then broadcast: every lane gets the same bits,
// so the lanes' iterates (and their branches) never diverge.
__device__ inline double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

__device__ inline double warp_prod(double v)
{
    for (int o = 16; o > 0; o >>= 1) v *= __shfl_down_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// One root per warp (the lanes split the sums; every lane holds the same
// iterate): origin index (into dK) and tau, lambda = dK[o] + tau.
__global__ void __launch_bounds__(256) dc_secular(int n, int t, DcArrays a)
{
    const int g = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (g >= n) return;
    int off, s;
    dc_node_of(n, t, g, &off, &s);
    const int K = a.cnt[3 * off], k = g - off;
    if (k >= K) return;
    const double *dK = a.dK + off, *zK = a.zK + off;
    const double rho = a.rho[off];
    if (K == 1) {
        if (lane == 0) {
            a.org[g] = 0;
            a.tau[g] = rho * zK[0] * zK[0];
            a.lamK[g] = dK[0] + rho * zK[0] * zK[0];
        }
        return;
    }
    int o;
    double lo, hi;
    if (k < K - 1) {
        const double gap = dK[k + 1] - dK[k], mid = 0.5 * gap;
        double fm = 0.0;
        for (int j = lane; j < K; j += 32) fm += rho * zK[j] * zK[j] / ((dK[j] - dK[k]) - mid);
        fm = 1.0 + warp_sum(fm);
        if (fm >= 0.0) {
            o = k;
            lo = 0.0;
            hi = mid;
        } else {
            o = k + 1;
            lo = -(gap - mid);
            hi = 0.0;
        }
    } else {
        o = K - 1;
        double z2 = 0.0;
        for (int j = lane; j < K; j += 32) z2 += zK[j] * zK[j];
        lo = 0.0;
        hi = rho * warp_sum(z2);
    }
    const double dO = dK[o];
    double tau = 0.5 * (lo + hi);
    for (int it = 0; it < kSecularIters; it++) {
        double psi = 0.0, dpsi = 0.0, phi = 0.0, dphi = 0.0;
        for (int j = lane; j < K; j += 32) {
            const double del = (dK[j] - dO) - tau, w = rho * zK[j] * zK[j] / del;
            if (j <= k) {
                psi += w;
                dpsi += w / del;
            } else {
                phi += w;
                dphi += w / del;
            }
        }
        psi = warp_sum(psi);
        dpsi = warp_sum(dpsi);
        phi = warp_sum(phi);
        dphi = warp_sum(dphi);
        const double f = 1.0 + psi + phi;
        if (f > 0.0) hi = tau;
        else if (f < 0.0) lo = tau;
        else break;
        if (fabs(f) <= 8.0 * kEps * (1.0 + fabs(psi) + fabs(phi))) break;
        // two-pole model of psi (pole k) and phi (pole k+1), matched in value
        // and slope at tau; its root in the interval is the next iterate
        const double a_ = (dK[k] - dO) - tau;
        const double q1 = dpsi * a_ * a_, p1 = psi - dpsi * a_;
        double eta = 0.0;
        bool have = false;
        if (k < K - 1) {
            const double b_ = (dK[k + 1] - dO) - tau;
            const double q2 = dphi * b_ * b_, p2 = phi - dphi * b_;
            const double c = 1.0 + p1 + p2;
            const double A = c, B = c * (a_ + b_) + q1 + q2, C = c * a_ * b_ + q1 * b_ + q2 * a_;
            const double disc = sqrt(fmax(0.0, B * B - 4.0 * A * C));
            const double den = B >= 0.0 ? B + disc : B - disc;
            if (den != 0.0) {
                const double r1 = 2.0 * C / den;
                if (r1 > a_ && r1 < b_) {
                    eta = r1;
                    have = true;
                }
            }
            if (!have && A != 0.0) {
                const double r2 = den / (2.0 * A);
                if (r2 > a_ && r2 < b_) {
                    eta = r2;
                    have = true;
                }
            }
        } else {
            const double c = 1.0 + p1;
            if (c > 0.0) {
                eta = a_ + q1 / c;
                have = true;
            }
        }
        double tn = tau + eta;
        if (!have || !(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        const bool done = fabs(tn - tau) <= 2.0 * kEps * fabs(tn) || hi - lo <= 2.0 * kEps * fmax(fabs(lo), fabs(hi));
        tau = tn;
        if (done) break;
    }
    if (lane == 0) {
        a.org[g] = o;
        a.tau[g] = tau;
        a.lamK[g] = dO + tau;
    }
}

// zhat_j (Gu-Eisenstat), one per warp: paired factors, each in (0, 1) but
// the last, so no partial product over- or underflows
__global__ void __launch_bounds__(256) dc_zhat(int n, int t, DcArrays a)
{
    const int g = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (g >= n) return;
    int off, s;
    dc_node_of(n, t, g, &off, &s);
    const int K = a.cnt[3 * off], j = g - off;
    if (j >= K) return;
    const double *dK = a.dK + off;
    if (K == 1) {
        if (lane == 0) a.zhat[g] = a.zK[off];
        return;
    }
    const double rho = a.rho[off], dj = dK[j];
    double prod = 1.0;
    for (int k = lane; k < K; k += 32) {
        const double lk_dj = (dK[a.org[off + k]] - dj) + a.tau[off + k];
        if (k < j) prod *= lk_dj / (dK[k] - dj);
        else if (k < K - 1) prod *= lk_dj / (dK[k + 1] - dj);
        else prod *= lk_dj / rho;
    }
    prod = warp_prod(prod);
    if (lane == 0) a.zhat[g] = copysign(sqrt(fmax(prod, 0.0)), a.zK[off + j]);
}

// Final ascending order of a merge's eigenvalues (roots and dropped values,
// both ascending): column source and value per output position.
__global__ void dc_order(int n, int t, DcArrays a, double *__restrict__ lam_out)
{
    int off, s;
    dc_node(n, t, blockIdx.x, &off, &s);
    const int K = a.cnt[3 * off], nd = a.cnt[3 * off + 1];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const double v = a.lamK[off + k];
        int lo = 0, hi = nd;
        while (lo < hi) {
            const int md = (lo + hi) >> 1;
            if (a.defl_d[off + md] < v) lo = md + 1;
            else hi = md;
        }
        lam_out[off + k + lo] = v;
        a.colsrc[off + k + lo] = k;
    }
    for (int p = threadIdx.x; p < nd; p += blockDim.x) {
        const double v = a.defl_d[off + p];
        int lo = 0, hi = K;
        while (lo < hi) {
            const int md = (lo + hi) >> 1;
            if (a.lamK[off + md] <= v) lo = md + 1;
            else hi = md;
        }
        lam_out[off + p + lo] = v;
        a.colsrc[off + p + lo] = -1 - p;
    }
}

// One output column per block: the column of U = P G [eigenvectors] for
// output position c of its merge.  U of a merge is s x s (ld s) at U + off*n.
__global__ void __launch_bounds__(128) dc_build_u(int n, int t, DcArrays a, double *__restrict__ U,
                                                  double *__restrict__ Vg, int smem_cols)
{
    extern __shared__ double vs[];
    __shared__ double red[32];
    const int g = blockIdx.x;
    int off, s;
    dc_node_of(n, t, g, &off, &s);
    const int c = g - off;
    double *v = smem_cols ? vs : Vg + (size_t)off * n + (size_t)c * s;
    const int src = a.colsrc[g];
    const int K = a.cnt[3 * off];
    for (int i = threadIdx.x; i < s; i += blockDim.x) v[i] = 0.0;
    __syncthreads();
    if (src >= 0) {
        const double dO = a.dK[off + a.org[off + src]], tau = a.tau[off + src];
        double ss = 0.0;
        for (int q = threadIdx.x; q < K; q += blockDim.x) {
            const double w = a.zhat[off + q] / ((a.dK[off + q] - dO) - tau);
            v[a.ndidx[off + q]] = w;
            ss += w * w;
        }
        ss = block_sum(ss, red);
        const double inv = 1.0 / sqrt(ss);
        for (int q = threadIdx.x; q < K; q += blockDim.x) v[a.ndidx[off + q]] *= inv;
    } else if (threadIdx.x == 0) {
        v[a.defl_idx[off + (-1 - src)]] = 1.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // Q_sorted G_1 ... G_r: the last rotation acts first on U
        const int nr = a.cnt[3 * off + 2];
        for (int r = nr - 1; r >= 0; r--) {
            const int p = a.rot_p[off + r], j = a.rot_j[off + r];
            const double cc = a.rot_c[off + r], sn = a.rot_s[off + r];
            const double x = v[p], y = v[j];
            v[p] = cc * x - sn * y;
            v[j] = sn * x + cc * y;
        }
    }
    __syncthreads();
    double *Uc = U + (size_t)off * n + (size_t)c * s;
    for (int i = threadIdx.x; i < s; i += blockDim.x) Uc[a.perm[off + i]] = v[i];
}

// The two block products of every merge of a depth, for small merges:
// Qn[off + r, off + c] = sum over the half of r: Q[off + r, off + kk] U[kk, c].
// Grid: (column tiles, row tiles, merges), 32 x 32 tiles, 256 threads.
__global__ void __launch_bounds__(256) dc_block_gemm(int n, int t, const double *__restrict__ Q,
                                                     const double *__restrict__ U, double *__restrict__ Qn)
{
    __shared__ double As[32][33], Bs[32][33];
    int off, s;
    dc_node(n, t, blockIdx.z, &off, &s);
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    if (r0 >= s || c0 >= s) return;
    const int n1 = s / 2;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 4
    const double *Um = U + (size_t)off * n;
    // a tile of rows lies in one half unless it straddles n1: each row takes
    // its own half's range of k
    const int klo = r0 >= n1 ? n1 : 0, khi = r0 + 31 < n1 ? n1 : s;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k0 = klo; k0 < khi; k0 += 32) {
        for (int i = ty; i < 32; i += 8) {  // consecutive threads read consecutive rows
            const int r = r0 + tx, kk = k0 + i;
            const bool ok = r < s && kk < khi && (r < n1 ? kk < n1 : kk >= n1);
            As[tx][i] = ok ? Q[(size_t)(off + r) + (size_t)(off + kk) * n] : 0.0;
            const int kr = k0 + tx, cc = c0 + i;
            Bs[tx][i] = (kr < khi && cc < s) ? Um[kr + (size_t)cc * s] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; kk++) {
            const double b = Bs[kk][tx];
#pragma unroll
            for (int q = 0; q < 4; q++) acc[q] = fma(As[ty + 8 * q][kk], b, acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int r = r0 + ty + 8 * q, cc = c0 + tx;
        if (r < s && cc < s) Qn[(size_t)(off + r) + (size_t)(off + cc) * n] = acc[q];
    }
}

__global__ void dc_output(int n, int nev, const double *__restrict__ Q, const double *__restrict__ lam,
                          const double *__restrict__ scale, double *__restrict__ lam_out, double *__restrict__ Z,
                          long long ldz)
{
    const long long total = (long long)n * nev;
    const double sc = *scale;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = i / n, r = i - c * n;
        Z[r + c * ldz] = Q[r + c * (long long)n];
        if (r == 0) lam_out[c] = lam[c] * sc;
    }
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct DcWs {
    double *Qa, *Qb, *U, *V, *lamA, *lamB, *scale;
    DcArrays arr;
    void *sl;
    size_t total;
};

bool dc_sliced(int m, int nn, int k) { return 2.0 * m * nn * k >= kSlicedMinFlops; }

size_t dc_sliced_bytes(int n)
{
    const int n2 = n - n / 2;
    return dc_sliced(n2, n, n2) ? sliced_gemm_ws_bytes(n2, n, n2) : 0;
}

DcWs dc_carve(int n, char *base)
{
    DcWs w{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    const size_t nn = (size_t)n * n * 8;
    w.Qa = (double *)take(nn);
    w.Qb = (double *)take(nn);
    w.U = (double *)take(nn);
    w.V = n > kSmemColumnMax ? (double *)take(nn) : nullptr;
    w.lamA = (double *)take((size_t)n * 8);
    w.lamB = (double *)take((size_t)n * 8);
    w.scale = (double *)take(8);
    DcArrays &a = w.arr;
    double **dp[] = {&a.ds, &a.zs, &a.dK, &a.zK, &a.tau, &a.lamK, &a.zhat, &a.defl_d, &a.rot_c, &a.rot_s, &a.rho};
    for (double **p : dp) *p = (double *)take((size_t)n * 8);
    int **ip[] = {&a.perm, &a.ndidx, &a.ndpos, &a.org, &a.defl_idx, &a.rot_p, &a.rot_j, &a.colsrc};
    for (int **p : ip) *p = (int *)take((size_t)n * 4);
    a.cnt = (int *)take((size_t)n * 12);
    const size_t sb = dc_sliced_bytes(n);
    w.sl = sb ? take(sb) : nullptr;
    w.total = off;
    return w;
}

}  // namespace

size_t tridiag_dc_workspace_bytes(int n) { return n >= 1 ? dc_carve(n, nullptr).total : 0; }

// lam[0..nev) ascending and Z[:, 0..nev) (ldz) the matching eigenvectors of
// the tridiagonal (d, e); asynchronous on st.
cudaError_t tridiag_dc_d(int n, int nev, const double *d, const double *e, double *lam, double *Z, long long ldz,
                         void *ws, cudaStream_t st)
{
    if (n < 1 || nev < 1) return cudaSuccess;
    DcWs w = dc_carve(n, (char *)ws);
    cudaError_t err;
    dc_scale<<<1, 1024, 0, st>>>(n, d, e, w.scale);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    const int D = dc_depth(n);
    dc_leaf<<<((1 << D) + 127) / 128, 128, 0, st>>>(n, D, d, e, w.scale, w.lamA, w.Qa);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    double *Q = w.Qa, *Qn = w.Qb, *lam_c = w.lamA, *lam_n = w.lamB;
    for (int t = D - 1; t >= 0; t--) {
        const int M = 1 << t;
        int smax = 0;
        for (int m = 0; m < M; m++) {
            int off, s;
            dc_node(n, t, m, &off, &s);
            smax = std::max(smax, s);
        }
        const int srows = smax <= kSetupSmemRows ? smax : 0;
        const size_t ssmem = (size_t)srows * 16;
        if (ssmem > 48 * 1024 &&
            (err = cudaFuncSetAttribute(dc_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem)) !=
                cudaSuccess)
            return err;
        dc_setup<<<M, kDcSetupThreads, ssmem, st>>>(n, t, Q, lam_c, e, w.scale, w.arr, srows);
        const unsigned grid = (unsigned)((n + 7) / 8);  // a warp per position, 8 per block
        dc_secular<<<grid, 256, 0, st>>>(n, t, w.arr);
        dc_zhat<<<grid, 256, 0, st>>>(n, t, w.arr);
        dc_order<<<M, 256, 0, st>>>(n, t, w.arr, lam_n);
        const int smem_cols = smax <= kSmemColumnMax ? 1 : 0;
        const size_t smem = smem_cols ? (size_t)smax * 8 : 0;
        if (smem > 48 * 1024 &&
            (err = cudaFuncSetAttribute(dc_build_u, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
            return err;
        dc_build_u<<<n, 128, smem, st>>>(n, t, w.arr, w.U, w.V, smem_cols);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if (!w.sl || !dc_sliced(smax / 2, smax, smax / 2)) {
            const int tiles = (smax + 31) / 32;
            dc_block_gemm<<<dim3(tiles, tiles, M), 256, 0, st>>>(n, t, Q, w.U, Qn);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
        } else {
            for (int m = 0; m < M; m++) {
                int off, s;
                dc_node(n, t, m, &off, &s);
                const int n1 = s / 2, n2 = s - n1;
                const double *Um = w.U + (size_t)off * n;
                const size_t ld = (size_t)n;
                if ((err = sliced_dgemm('N', 'N', n1, s, n1, 1.0, Q + off + off * ld, n, Um, s, 0.0, Qn + off + off * ld,
                                        n, w.sl, st)) != cudaSuccess)
                    return err;
                if ((err = sliced_dgemm('N', 'N', n2, s, n2, 1.0, Q + (off + n1) + (off + n1) * ld, n, Um + n1, s, 0.0,
                                        Qn + (off + n1) + off * ld, n, w.sl, st)) != cudaSuccess)
                    return err;
            }
        }
        std::swap(Q, Qn);
        std::swap(lam_c, lam_n);
    }
    const long long total = (long long)n * nev;
    const unsigned og = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 16);
    dc_output<<<og, 256, 0, st>>>(n, nev, Q, lam_c, w.scale, lam, Z, ldz);
    return cudaGetLastError();
}

}  // namespace gb

extern "C" {

size_t gb_tridiag_dc_workspace_bytes(int n) { return gb::tridiag_dc_workspace_bytes(n); }

int gb_tridiag_dc_d(int n, const double *d, const double *e, double *lam, double *Q, int ldq, void *workspace,
                    size_t ws_bytes, void *stream)
{
    if (n < 1) return -1;
    if (!d || ((uintptr_t)d % 8) != 0) return -2;
    if (n > 1 && (!e || ((uintptr_t)e % 8) != 0)) return -3;
    if (!lam || ((uintptr_t)lam % 8) != 0) return -4;
    if (!Q || ((uintptr_t)Q % 8) != 0) return -5;
    if (ldq < n) return -6;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -7;
    if (ws_bytes < gb::tridiag_dc_workspace_bytes(n)) return -8;
    const cudaError_t err = gb::tridiag_dc_d(n, n, d, e, lam, Q, ldq, workspace, (cudaStream_t)stream);
    return err == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

}  // extern "C"
