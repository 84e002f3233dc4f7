// Band -> tridiagonal reduction by bulge chasing on the device (the second
// step of the two-stage reduction, Sec. 2), emitting the reflectors in the
// layout trans_ev_tridi_to_band consumes.
//
// Task (s,k) generates H(s,k) from the column it annihilates (column s for
// k = 0, the first column s+1+(k-1)b of the previous bulge otherwise; rows
// r = s+k*b .. r+len-1, 0-based) and applies it from both sides to the
// entries it touches, all in the lower triangle:
//   left block   rows R x columns c+1..r-1   (the rest of the bulge),
//   diagonal     rows R x columns R          (symmetric two-sided update),
//   below block  rows r+len..r+len+b-1 x R   (this creates the next bulge).
// The working matrix is kept in lower band storage of width 2b (entries up
// to 2b-1 below the diagonal, where the bulges live), in a workspace.
//
// A persistent grid (at most one block per SM) takes sweeps by ticket in
// increasing s; the tasks of a sweep run in order in the block that took it, each with
// one round of loads into registers, the reductions, and one round of
// stores.  Task (s,k) overlaps tasks of sweep
// s-1 up to k+2, so it waits until sweep s-1 has finished min(k+3, nk(s-1))
// tasks (progress flags, acquire/release, bounded waits as in the pipeline
// back-transformation).
#include <cuda_runtime.h>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "trans_ev_kernels.cuh"

#include <vector>

namespace gb {

namespace {

constexpr int kChaseThreads = 256;
constexpr int kLag = 3;

__device__ __forceinline__ int ld_acq(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_rel(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct ChaseState {
    int ticket;
    int abort;
    int error;
};

// One problem of a batched chase: its working band and reflector arrays and
// its progress flags.
struct ChaseProblem {
    int n, b;
    double *W;
    long long ldw;
    double *hh_v, *hh_tau;
    int *progress;
};

// Lower band storage of width 2b: A(i,j), i >= j, at W[(i-j) + j*ldw].
struct Band {
    double *W;
    long long ldw;
    __device__ __forceinline__ double *at(int i, int j) const
    {
        return (i >= j) ? W + (i - j) + (long long)j * ldw : W + (j - i) + (long long)i * ldw;
    }
    __device__ __forceinline__ double get(int i, int j) const { return __ldcg(at(i, j)); }
};

// Sum over the 4 lanes of a quad (lanes 4m..4m+3).
__device__ __forceinline__ double quad_sum(double x)
{
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    return x;
}

__device__ double block_sum(double x, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = x;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kChaseThreads / 32; w++) t += red[w];
    return t;
}

__global__ void __launch_bounds__(256) band_init(int n, int b, const double *__restrict__ AB, long long ldab,
                                                 double *__restrict__ W, long long ldw)
{
    const long long total = (long long)n * ldw;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long j = e / ldw, d = e - j * ldw;
        W[e] = (d <= b && j + d < n) ? AB[d + j * ldab] : 0.0;
    }
}

__global__ void __launch_bounds__(256) band_extract(int n, const double *__restrict__ W, long long ldw,
                                                    double *__restrict__ dd, double *__restrict__ ee)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        dd[j] = W[(long long)j * ldw];
        if (j < n - 1) ee[j] = W[1 + (long long)j * ldw];
    }
}

// Shared scratch of one chase block.
struct ChaseSmem {
    double v[64];
    double q[64];
    double red[kChaseThreads / 32];
    double s_tau, s_scal;
    int s_sweep, s_abort;
};

// All tasks of sweep s of one problem, in order (the whole block); returns
// true when the call has to stop (abort raised or a wait timed out).
__device__ bool chase_sweep_d(int n, int b, const Band &A, double *__restrict__ hh_v, double *__restrict__ hh_tau,
                              ChaseState *state, int *progress, long long timeout_ns, int s, ChaseSmem &sm)
{
    double *v = sm.v, *q = sm.q, *red = sm.red;
    double &s_tau = sm.s_tau, &s_scal = sm.s_scal;
    int &s_abort = sm.s_abort;
    const int tid = threadIdx.x;
    const int quad = tid >> 2, part = tid & 3;  // 64 quads of 4 lanes; lane 'part' owns rows/cols part+4t
    const int nk = sweep_count(n, b, s);
    const int nk_prev = (s > 1) ? sweep_count(n, b, s - 1) : 0;
    const long long first = sweep_first(n, b, s);

    for (int k = 0; k < nk; k++) {
        // ---- wait for sweep s-1 to be kLag tasks ahead (bounded)
        if (tid == 0) {
            int abort = 0;
            if (s > 1) {
                const int need = min(k + kLag, nk_prev);
                const unsigned long long t0 = now_ns();
                while (ld_acq(progress + (s - 2)) < need) {
                    if (*(volatile int *)&state->abort) { abort = 1; break; }
                    if ((long long)(now_ns() - t0) > timeout_ns) {
                        atomicExch(&state->error, GB_ERR_TIMEOUT);
                        atomicExch(&state->abort, 1);
                        abort = 1;
                        break;
                    }
                    __nanosleep(32);
                }
            } else if (*(volatile int *)&state->abort) {
                abort = 1;
            }
            s_abort = abort;
        }
        __syncthreads();
        if (s_abort) return true;

        const int r = s + k * b;   // 0-based first row of H(s,k)
        const int len = min(b, n - r);
        const int c = (k == 0) ? s - 1 : s + (k - 1) * b;
        const int rb = r + len;
        const int nleft = r - c - 1, nbelow = min(b, n - rb);
        const long long idx = first + k;

        // ---- one round of loads: the source column and the three blocks
        const double xi = (tid >= 1 && tid < len) ? A.get(r + tid, c) : 0.0;
        double L[16], Bl[16], D[16];
#pragma unroll
        for (int t = 0; t < 16; t++) {
            const int i = part + 4 * t;
            L[t] = (quad < nleft && i < len) ? A.get(r + i, c + 1 + quad) : 0.0;
            Bl[t] = (quad < nbelow && i < len) ? A.get(rb + quad, r + i) : 0.0;
            D[t] = (quad < len && i < len) ? A.get(r + quad, r + i) : 0.0;
        }

        // ---- reflector from column c (LAPACK form, v_0 = 1)
        const double ss = block_sum(xi * xi, red);
        if (tid == 0) {
            const double alpha = A.get(r, c);
            double tau = 0.0, scal = 0.0, beta = alpha;
            if (ss != 0.0) {
                const double nrm = sqrt(alpha * alpha + ss);
                beta = (alpha >= 0.0) ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
            s_tau = tau;
            s_scal = scal;
            hh_tau[idx] = tau;
            if (tau != 0.0) *A.at(r, c) = beta;
        }
        __syncthreads();
        const double tau = s_tau;
        const double vt = (tid == 0) ? 1.0 : ((tid < len && tau != 0.0) ? xi * s_scal : 0.0);
        if (tid < 64) v[tid] = vt;
        if (tid < b) hh_v[idx * b + tid] = vt;
        if (tau != 0.0 && tid >= 1 && tid < len) *A.at(r + tid, c) = 0.0;
        __syncthreads();

        if (tau != 0.0) {
            // ---- the three reductions (every lane runs the quad shuffles)
            double al = 0.0, ab = 0.0, ad = 0.0;
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const double vi = v[part + 4 * t];  // v is zero past len
                al = fma(vi, L[t], al);
                ab = fma(Bl[t], vi, ab);
                ad = fma(D[t], vi, ad);
            }
            const double tw = tau * quad_sum(al);   // left: tau v^T A[R, j]
            const double ty = tau * quad_sum(ab);   // below: tau A[i, R] v
            const double pi = tau * quad_sum(ad);   // diagonal: p_i = tau (A v)_i
            // K = tau/2 v^T p, q = p - K v
            const double K = 0.5 * tau * block_sum((part == 0 && quad < len) ? v[quad] * pi : 0.0, red);
            if (part == 0 && quad < len) q[quad] = pi - K * v[quad];
            __syncthreads();
            const double vq = v[quad], qq = (quad < len) ? q[quad] : 0.0;
            // ---- updates from registers, one store each
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const int i = part + 4 * t;
                if (i < len) {
                    const double vi = v[i];
                    if (quad < nleft) *A.at(r + i, c + 1 + quad) = fma(-tw, vi, L[t]);
                    if (quad < nbelow) *A.at(rb + quad, r + i) = fma(-ty, vi, Bl[t]);
                    if (quad < len && i <= quad) *A.at(r + quad, r + i) = D[t] - vq * q[i] - qq * vi;
                }
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_rel(progress + (s - 1), k + 1);
    }
    return false;
}

__global__ void __launch_bounds__(kChaseThreads)
chase_d(int n, int b, Band A, double *__restrict__ hh_v, double *__restrict__ hh_tau, ChaseState *state,
        int *progress, long long timeout_ns)
{
    __shared__ ChaseSmem sm;
    for (;;) {  // persistent: sweeps by ticket, in increasing s
        __syncthreads();
        if (threadIdx.x == 0) sm.s_sweep = 1 + atomicAdd(&state->ticket, 1);
        __syncthreads();
        const int s = sm.s_sweep;
        if (s > n - 1) return;
        if (chase_sweep_d(n, b, A, hh_v, hh_tau, state, progress, timeout_ns, s, sm)) return;
    }
}

// The chases of many independent problems in one persistent launch: ticket
// t is sweep 1 + t / count of problem t % count (skipped past that problem's
// last sweep), so every problem's sweeps are taken in increasing order and a
// task waits only on a sweep with a smaller ticket, which a running block
// holds: no deadlock at any residency.  One state word (ticket, abort,
// error) for the launch; progress flags per problem.
__global__ void __launch_bounds__(kChaseThreads)
chase_batched_d(int count, int smax, const ChaseProblem *__restrict__ probs, ChaseState *state, long long timeout_ns)
{
    __shared__ ChaseSmem sm;
    const long long total = (long long)count * smax;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sm.s_sweep = atomicAdd(&state->ticket, 1);
        __syncthreads();
        const long long t = sm.s_sweep;
        if (t >= total) return;
        const ChaseProblem pr = probs[t % count];
        const int s = 1 + (int)(t / count);
        if (s > pr.n - 1) continue;
        if (chase_sweep_d(pr.n, pr.b, Band{pr.W, pr.ldw}, pr.hh_v, pr.hh_tau, state, pr.progress, timeout_ns, s, sm))
            return;
    }
}

// ---------------------------------------------------------------- complex
// Hermitian band (lower storage, complex entries): the same task structure
// with H = I - tau v v^H applied as H^H from the left and H from the right;
// the sub-diagonal comes out real because every kept entry is a real beta.
struct Zc {
    double re, im;
};
__device__ __forceinline__ Zc zmul(Zc a, Zc b) { return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)}; }
__device__ __forceinline__ Zc zconj(Zc a) { return {a.re, -a.im}; }
// acc += conj(a) * b
__device__ __forceinline__ void zdotc(Zc &acc, Zc a, Zc b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}
// acc += a * b
__device__ __forceinline__ void zfma(Zc &acc, Zc a, Zc b)
{
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}

struct BandZ {
    Zc *W;
    long long ldw;
    __device__ __forceinline__ Zc *at_lower(int i, int j) const { return W + (i - j) + (long long)j * ldw; }
    __device__ __forceinline__ Zc get(int i, int j) const
    {
        if (i >= j) {
            const double2 t = __ldcg(reinterpret_cast<const double2 *>(at_lower(i, j)));
            return {t.x, t.y};
        }
        const double2 t = __ldcg(reinterpret_cast<const double2 *>(at_lower(j, i)));
        return {t.x, -t.y};
    }
    __device__ __forceinline__ void set_lower(int i, int j, Zc v) const { *at_lower(i, j) = v; }
};

__device__ __forceinline__ Zc quad_sum_z(Zc x)
{
    x.re = quad_sum(x.re);
    x.im = quad_sum(x.im);
    return x;
}

struct ChaseSmemZ {
    Zc v[64];
    Zc q[64];
    double red[kChaseThreads / 32];
    Zc s_tau, s_scal;
    int s_sweep, s_abort;
};

// All tasks of sweep s of one Hermitian problem (the whole block); returns
// true when the call has to stop.
__device__ bool chase_sweep_z(int n, int b, const BandZ &A, Zc *__restrict__ hh_v, Zc *__restrict__ hh_tau,
                              ChaseState *state, int *progress, long long timeout_ns, int s, ChaseSmemZ &sm)
{
    Zc *v = sm.v, *q = sm.q;
    double *red = sm.red;
    Zc &s_tau = sm.s_tau, &s_scal = sm.s_scal;
    int &s_abort = sm.s_abort;
    const int tid = threadIdx.x;
    const int quad = tid >> 2, part = tid & 3;
    const int nk = sweep_count(n, b, s);
    const int nk_prev = (s > 1) ? sweep_count(n, b, s - 1) : 0;
    const long long first = sweep_first(n, b, s);

    for (int k = 0; k < nk; k++) {
        if (tid == 0) {
            int abort = 0;
            if (s > 1) {
                const int need = min(k + kLag, nk_prev);
                const unsigned long long t0 = now_ns();
                while (ld_acq(progress + (s - 2)) < need) {
                    if (*(volatile int *)&state->abort) { abort = 1; break; }
                    if ((long long)(now_ns() - t0) > timeout_ns) {
                        atomicExch(&state->error, GB_ERR_TIMEOUT);
                        atomicExch(&state->abort, 1);
                        abort = 1;
                        break;
                    }
                    __nanosleep(32);
                }
            } else if (*(volatile int *)&state->abort) {
                abort = 1;
            }
            s_abort = abort;
        }
        __syncthreads();
        if (s_abort) return true;

        const int r = s + k * b;
        const int len = min(b, n - r);
        const int c = (k == 0) ? s - 1 : s + (k - 1) * b;
        const int rb = r + len;
        const int nleft = r - c - 1, nbelow = min(b, n - rb);
        const long long idx = first + k;

        // ---- reflector (complex, beta real)
        const Zc xi = (tid >= 1 && tid < len) ? A.get(r + tid, c) : Zc{0.0, 0.0};
        const double ss = block_sum(xi.re * xi.re + xi.im * xi.im, red);
        if (tid == 0) {
            const Zc alpha = A.get(r, c);
            Zc tau{0.0, 0.0}, scal{0.0, 0.0};
            if (!(ss == 0.0 && alpha.im == 0.0)) {
                const double nrm = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + ss);
                const double beta = (alpha.re >= 0.0) ? -nrm : nrm;
                tau = {(beta - alpha.re) / beta, -alpha.im / beta};
                const Zc den{alpha.re - beta, alpha.im};           // 1 / (alpha - beta)
                const double dd = den.re * den.re + den.im * den.im;
                scal = {den.re / dd, -den.im / dd};
                A.set_lower(r, c, Zc{beta, 0.0});
            }
            s_tau = tau;
            s_scal = scal;
            hh_tau[idx] = tau;
        }
        __syncthreads();
        const Zc tau = s_tau;
        const bool active = !(tau.re == 0.0 && tau.im == 0.0);
        Zc vt{0.0, 0.0};
        if (tid == 0) vt = {1.0, 0.0};
        else if (tid < len && active) vt = zmul(xi, s_scal);
        if (tid < 64) v[tid] = vt;
        if (tid < b) hh_v[idx * b + tid] = vt;
        if (active && tid >= 1 && tid < len) A.set_lower(r + tid, c, Zc{0.0, 0.0});
        __syncthreads();

        if (active) {
            const Zc ctau = zconj(tau);
            // ---- left block: A[R,j] -= conj(tau) v (v^H A[R,j])
            {
                const bool act = quad < nleft;
                const int j = c + 1 + quad;
                Zc Lr[16];
                Zc acc{0.0, 0.0};
#pragma unroll
                for (int t = 0; t < 16; t++) {
                    const int i = part + 4 * t;
                    Lr[t] = (act && i < len) ? A.get(r + i, j) : Zc{0.0, 0.0};
                    zdotc(acc, v[i], Lr[t]);
                }
                const Zc w = zmul(ctau, quad_sum_z(acc));
#pragma unroll
                for (int t = 0; t < 16; t++) {
                    const int i = part + 4 * t;
                    if (act && i < len) {
                        Zc a = Lr[t];
                        const Zc vw = zmul(v[i], w);
                        a.re -= vw.re;
                        a.im -= vw.im;
                        A.set_lower(r + i, j, a);
                    }
                }
            }
            // ---- below block: A[i,R] -= tau (A[i,R] v) v^H
            {
                const bool act = quad < nbelow;
                const int i = rb + quad;
                Zc Br[16];
                Zc acc{0.0, 0.0};
#pragma unroll
                for (int t = 0; t < 16; t++) {
                    const int j = part + 4 * t;
                    Br[t] = (act && j < len) ? A.get(i, r + j) : Zc{0.0, 0.0};
                    zfma(acc, Br[t], v[j]);
                }
                const Zc y = zmul(tau, quad_sum_z(acc));
#pragma unroll
                for (int t = 0; t < 16; t++) {
                    const int j = part + 4 * t;
                    if (act && j < len) {
                        Zc a = Br[t];
                        const Zc yv = zmul(y, zconj(v[j]));
                        a.re -= yv.re;
                        a.im -= yv.im;
                        A.set_lower(i, r + j, a);
                    }
                }
            }
            // ---- diagonal block: p = tau A v, K = conj(tau)/2 v^H p, q = p - K v,
            //      A -= q v^H + v q^H on the lower triangle
            Zc Dr[16];
            Zc pa{0.0, 0.0};
            const bool actd = quad < len;
#pragma unroll
            for (int t = 0; t < 16; t++) {
                const int j = part + 4 * t;
                Dr[t] = (actd && j < len) ? A.get(r + quad, r + j) : Zc{0.0, 0.0};
                zfma(pa, Dr[t], v[j]);
            }
            const Zc pi = zmul(tau, quad_sum_z(pa));
            Zc vp{0.0, 0.0};
            if (part == 0 && actd) zdotc(vp, v[quad], pi);
            const double kre = block_sum(vp.re, red), kim = block_sum(vp.im, red);
            const Zc K = zmul(Zc{0.5 * ctau.re, 0.5 * ctau.im}, Zc{kre, kim});
            if (part == 0 && actd) {
                const Zc kv = zmul(K, v[quad]);
                q[quad] = Zc{pi.re - kv.re, pi.im - kv.im};
            }
            __syncthreads();
            if (actd) {
                const Zc vq = v[quad], qq = q[quad];
#pragma unroll
                for (int t = 0; t < 16; t++) {
                    const int j = part + 4 * t;
                    if (j < len && j <= quad) {
                        const Zc t1 = zmul(qq, zconj(v[j])), t2 = zmul(vq, zconj(q[j]));
                        A.set_lower(r + quad, r + j, Zc{Dr[t].re - t1.re - t2.re, Dr[t].im - t1.im - t2.im});
                    }
                }
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_rel(progress + (s - 1), k + 1);
    }
    return false;
}

__global__ void __launch_bounds__(kChaseThreads)
chase_z(int n, int b, BandZ A, Zc *__restrict__ hh_v, Zc *__restrict__ hh_tau, ChaseState *state, int *progress,
        long long timeout_ns)
{
    __shared__ ChaseSmemZ sm;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sm.s_sweep = 1 + atomicAdd(&state->ticket, 1);
        __syncthreads();
        const int s = sm.s_sweep;
        if (s > n - 1) return;
        if (chase_sweep_z(n, b, A, hh_v, hh_tau, state, progress, timeout_ns, s, sm)) return;
    }
}

// The Hermitian chases of many problems in one launch (the ticket order of
// chase_batched_d); the table's W, hh_v, hh_tau point at complex data.
__global__ void __launch_bounds__(kChaseThreads)
chase_batched_z(int count, int smax, const ChaseProblem *__restrict__ probs, ChaseState *state, long long timeout_ns)
{
    __shared__ ChaseSmemZ sm;
    const long long total = (long long)count * smax;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sm.s_sweep = atomicAdd(&state->ticket, 1);
        __syncthreads();
        const long long t = sm.s_sweep;
        if (t >= total) return;
        const ChaseProblem pr = probs[t % count];
        const int s = 1 + (int)(t / count);
        if (s > pr.n - 1) continue;
        if (chase_sweep_z(pr.n, pr.b, BandZ{(Zc *)pr.W, pr.ldw}, (Zc *)pr.hh_v, (Zc *)pr.hh_tau, state, pr.progress,
                          timeout_ns, s, sm))
            return;
    }
}

__global__ void __launch_bounds__(256) band_init_z(int n, int b, const Zc *__restrict__ AB, long long ldab,
                                                   Zc *__restrict__ W, long long ldw)
{
    const long long total = (long long)n * ldw;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long j = e / ldw, d = e - j * ldw;
        W[e] = (d <= b && j + d < n) ? AB[d + j * ldab] : Zc{0.0, 0.0};
    }
}

__global__ void __launch_bounds__(256) band_extract_z(int n, const Zc *__restrict__ W, long long ldw,
                                                      double *__restrict__ dd, double *__restrict__ ee)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        dd[j] = W[(long long)j * ldw].re;
        if (j < n - 1) ee[j] = W[1 + (long long)j * ldw].re;
    }
}

}  // namespace

// Workspace: [256-byte head {ticket, abort, error}][progress: n ints] then,
// 256-byte aligned, the 2b x n working band.
static size_t flags_bytes(int n) { return (256 + (size_t)n * sizeof(int) + 255) & ~(size_t)255; }

size_t band_to_tridi_workspace_bytes(int n, int b)
{
    size_t band = 2 * (size_t)b * (size_t)n * sizeof(double);
    return flags_bytes(n) + ((band + 255) & ~(size_t)255);
}

size_t band_to_tridi_workspace_bytes_z(int n, int b)
{
    size_t band = 2 * (size_t)b * (size_t)n * 2 * sizeof(double);
    return flags_bytes(n) + ((band + 255) & ~(size_t)255);
}

// Persistent blocks for the chase: at most one per SM, and no more than the
// sweeps that can be in flight at once (sweep s trails sweep s-1 by kLag
// tasks, so about nk(1)/kLag sweeps are active); further blocks would only
// poll, holding SM slots that concurrent work on other streams could use.
static int chase_grid(int n, int b, int sms)
{
    const int nk1 = (n - 1 + b - 1) / b;
    const int active = (nk1 + kLag - 1) / kLag + 2;
    return max(1, min(min(n - 1, sms), active));
}

cudaError_t band_to_tridi_prepare_z(int n, int b, const double *AB, int ldab, void *ws, cudaStream_t st)
{
    const long long ldw = 2LL * b;
    char *flags = (char *)ws;
    Zc *W = (Zc *)(flags + flags_bytes(n));
    cudaError_t err = cudaMemsetAsync(flags, 0, flags_bytes(n), st);
    if (err != cudaSuccess) return err;
    band_init_z<<<1024, 256, 0, st>>>(n, b, (const Zc *)AB, ldab, W, ldw);
    return cudaGetLastError();
}

cudaError_t band_to_tridi_finish_z(int n, int b, const void *ws, double *d, double *e, cudaStream_t st)
{
    const long long ldw = 2LL * b;
    const Zc *W = (const Zc *)((const char *)ws + flags_bytes(n));
    band_extract_z<<<64, 256, 0, st>>>(n, W, ldw, d, e);
    return cudaGetLastError();
}

cudaError_t band_to_tridi_z(int n, int b, const double *AB, int ldab, double *d, double *e, double *hh_v,
                            double *hh_tau, void *ws, long long timeout_ns, cudaStream_t st)
{
    const long long ldw = 2LL * b;
    char *flags = (char *)ws;
    Zc *W = (Zc *)(flags + flags_bytes(n));
    cudaError_t err = band_to_tridi_prepare_z(n, b, AB, ldab, ws, st);
    if (err != cudaSuccess) return err;
    if (n > 1) {
        int dev = 0, sms = 0;
        if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
        const int grid = chase_grid(n, b, sms);
        chase_z<<<(unsigned)grid, kChaseThreads, 0, st>>>(n, b, BandZ{W, ldw}, (Zc *)hh_v, (Zc *)hh_tau,
                                                         (ChaseState *)flags, (int *)(flags + 256), timeout_ns);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return band_to_tridi_finish_z(n, b, ws, d, e, st);
}

cudaError_t band_to_tridi_prepare_d(int n, int b, const double *AB, int ldab, void *ws, cudaStream_t st)
{
    const long long ldw = 2LL * b;
    char *flags = (char *)ws;
    double *W = (double *)(flags + flags_bytes(n));
    cudaError_t err = cudaMemsetAsync(flags, 0, flags_bytes(n), st);
    if (err != cudaSuccess) return err;
    band_init<<<1024, 256, 0, st>>>(n, b, AB, ldab, W, ldw);
    return cudaGetLastError();
}

cudaError_t band_to_tridi_finish_d(int n, int b, const void *ws, double *d, double *e, cudaStream_t st)
{
    const long long ldw = 2LL * b;
    const double *W = (const double *)((const char *)ws + flags_bytes(n));
    band_extract<<<64, 256, 0, st>>>(n, W, ldw, d, e);
    return cudaGetLastError();
}

cudaError_t band_to_tridi_d(int n, int b, const double *AB, int ldab, double *d, double *e, double *hh_v,
                            double *hh_tau, void *ws, size_t ws_bytes, long long timeout_ns, cudaStream_t st)
{
    (void)ws_bytes;
    const long long ldw = 2LL * b;
    char *flags = (char *)ws;
    double *W = (double *)(flags + flags_bytes(n));
    cudaError_t err = band_to_tridi_prepare_d(n, b, AB, ldab, ws, st);
    if (err != cudaSuccess) return err;
    if (n > 1) {
        int dev = 0, sms = 0;
        if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
        const int grid = chase_grid(n, b, sms);
        chase_d<<<(unsigned)grid, kChaseThreads, 0, st>>>(n, b, Band{W, ldw}, hh_v, hh_tau, (ChaseState *)flags,
                                                         (int *)(flags + 256), timeout_ns);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    return band_to_tridi_finish_d(n, b, ws, d, e, st);
}

size_t chase_batched_table_bytes(int count) { return 256 + (((size_t)count * sizeof(ChaseProblem) + 255) & ~(size_t)255); }

// The chases of `count` problems in one persistent launch, in two calls on
// one stream: band_to_tridi_chase_batched_upload_d writes the launch's state
// word (ticket, abort, error; read it with gb_trans_ev_query) and the problem
// table into `table` (device, chase_batched_table_bytes(count)), from the
// host (a copy from pageable memory waits for the stream's earlier work, so
// issue it before that work); band_to_tridi_chase_batched_d launches once
// band_to_tridi_prepare_d has run on every problem's workspace ws[i].
cudaError_t band_to_tridi_chase_batched_upload_d(int count, const int *n, const int *b, void *const *ws,
                                                 double *const *hh_v, double *const *hh_tau, void *table,
                                                 cudaStream_t st)
{
    if (count < 1) return cudaSuccess;
    std::vector<ChaseProblem> host((size_t)count);
    for (int i = 0; i < count; i++) {
        char *flags = (char *)ws[i];
        host[i] = ChaseProblem{n[i], b[i], (double *)(flags + flags_bytes(n[i])), 2LL * b[i], hh_v[i], hh_tau[i],
                               (int *)(flags + 256)};
    }
    cudaError_t err = cudaMemsetAsync(table, 0, 256, st);
    if (err != cudaSuccess) return err;
    // from pageable memory: staged before the call returns, so `host` may go
    return cudaMemcpyAsync((char *)table + 256, host.data(), host.size() * sizeof(ChaseProblem),
                           cudaMemcpyHostToDevice, st);
}

cudaError_t band_to_tridi_chase_batched_d(int count, const int *n, const int *b, void *table, long long timeout_ns,
                                          cudaStream_t st)
{
    return band_to_tridi_chase_batched(count, n, b, table, timeout_ns, st, 0);
}

cudaError_t band_to_tridi_chase_batched(int count, const int *n, const int *b, void *table, long long timeout_ns,
                                        cudaStream_t st, int is_complex)
{
    int smax = 0;
    for (int i = 0; i < count; i++) smax = max(smax, n[i] - 1);
    if (count < 1 || smax < 1) return cudaSuccess;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t err;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, is_complex ? (const void *)chase_batched_z
                                                                                 : (const void *)chase_batched_d,
                                                             kChaseThreads, 0)) != cudaSuccess)
        return err;
    // no more blocks than the problems' sweeps that can be in flight at once
    // (as for one problem): extra blocks would only poll, holding SM slots
    // that work on other streams could use
    long long active = 0;
    for (int i = 0; i < count; i++) active += chase_grid(n[i], b[i], sms);
    const long long tickets = (long long)count * smax;
    const long long grid = min(min((long long)sms * max(per_sm, 1), tickets), max(active, 1LL));
    const ChaseProblem *tab = (const ChaseProblem *)((char *)table + 256);
    if (is_complex)
        chase_batched_z<<<(unsigned)grid, kChaseThreads, 0, st>>>(count, smax, tab, (ChaseState *)table, timeout_ns);
    else
        chase_batched_d<<<(unsigned)grid, kChaseThreads, 0, st>>>(count, smax, tab, (ChaseState *)table, timeout_ns);
    return cudaGetLastError();
}

}  // namespace gb
