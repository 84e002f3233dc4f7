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
// One block per sweep, sweeps taken by ticket in increasing s; the tasks of
// a sweep run in order in that block.  Task (s,k) overlaps tasks of sweep
// s-1 up to k+2, so it waits until sweep s-1 has finished min(k+3, nk(s-1))
// tasks (progress flags, acquire/release, bounded waits as in the pipeline
// back-transformation).
#include <cuda_runtime.h>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "trans_ev_kernels.cuh"

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

__global__ void __launch_bounds__(kChaseThreads)
chase_d(int n, int b, Band A, double *__restrict__ hh_v, double *__restrict__ hh_tau, ChaseState *state,
        int *progress, long long timeout_ns)
{
    __shared__ double v[64];
    __shared__ double p[64];
    __shared__ double red[kChaseThreads / 32];
    __shared__ double s_tau, s_K;
    __shared__ int s_sweep, s_abort;
    const int tid = threadIdx.x;

    if (tid == 0) s_sweep = 1 + atomicAdd(&state->ticket, 1);
    __syncthreads();
    const int s = s_sweep;
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
                    __nanosleep(64);
                }
            }
            s_abort = abort;
        }
        __syncthreads();
        if (s_abort) return;

        const int r = s + k * b;             // 0-based first row of H(s,k)
        const int len = min(b, n - r);
        const int c = (k == 0) ? s - 1 : s + (k - 1) * b;
        const long long idx = first + k;

        // ---- reflector from column c, rows r..r+len-1 (LAPACK form, v_0 = 1)
        double xi = (tid >= 1 && tid < len) ? A.get(r + tid, c) : 0.0;
        const double ss = block_sum(xi * xi, red);
        if (tid == 0) {
            const double alpha = A.get(r, c);
            double tau = 0.0, scal = 0.0;
            if (ss != 0.0) {
                const double nrm = sqrt(alpha * alpha + ss);
                const double beta = (alpha >= 0.0) ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
                *A.at(r, c) = beta;
            }
            s_tau = tau;
            s_K = scal;
            hh_tau[idx] = tau;
        }
        __syncthreads();
        const double tau = s_tau;
        if (tid < b) {
            double vi = 0.0;
            if (tid == 0) vi = 1.0;
            else if (tid < len) vi = (tau != 0.0) ? xi * s_K : 0.0;
            if (tid < len) v[tid] = vi;
            hh_v[idx * b + tid] = vi;
            if (tau != 0.0 && tid >= 1 && tid < len) *A.at(r + tid, c) = 0.0;
        }
        __syncthreads();

        if (tau != 0.0) {
            const int quad = tid >> 2, part = tid & 3;  // 64 quads of 4 lanes
            // Every lane runs the quad reductions (full-mask shuffles); only the
            // memory accesses are guarded by the activity tests.
            // ---- left block: columns c+1..r-1, w_j = v^T A[R,j], A[R,j] -= tau v w_j
            {
                const bool act = quad < r - c - 1;
                const int j = c + 1 + quad;
                double acc = 0.0;
                if (act)
                    for (int i = part; i < len; i += 4) acc = fma(v[i], A.get(r + i, j), acc);
                const double tw = tau * quad_sum(acc);
                if (act)
                    for (int i = part; i < len; i += 4) {
                        double *a = A.at(r + i, j);
                        *a = fma(-tw, v[i], __ldcg(a));
                    }
            }
            // ---- below block: rows r+len..min(r+len+b,n)-1, y_i = A[i,R] v, A[i,R] -= tau y_i v^T
            {
                const int rb = r + len;
                const bool act = quad < min(b, n - rb);
                const int i = rb + quad;
                double acc = 0.0;
                if (act)
                    for (int j = part; j < len; j += 4) acc = fma(A.get(i, r + j), v[j], acc);
                const double ty = tau * quad_sum(acc);
                if (act)
                    for (int j = part; j < len; j += 4) {
                        double *a = A.at(i, r + j);
                        *a = fma(-ty, v[j], __ldcg(a));
                    }
            }
            // ---- diagonal block: p = tau A v (symmetric, read before any write)
            {
                const bool act = quad < len;
                double acc = 0.0;
                if (act)
                    for (int j = part; j < len; j += 4) acc = fma(A.get(r + quad, r + j), v[j], acc);
                acc = quad_sum(acc);
                if (act && part == 0) p[quad] = tau * acc;
            }
            __syncthreads();
            double kv = (tid < len) ? v[tid] * p[tid] : 0.0;
            const double K = 0.5 * tau * block_sum(kv, red);
            // q = p - K v, A[R,R] -= v q^T + q v^T on the lower triangle
            const int ntri = len * (len + 1) / 2;
            for (int e = tid; e < ntri; e += kChaseThreads) {
                // e -> (i, j), j <= i, row-major over the lower triangle
                int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);  // FP32: keep the FP64 pipe free
                while ((i + 1) * (i + 2) / 2 <= e) i++;
                while (i * (i + 1) / 2 > e) i--;
                const int j = e - i * (i + 1) / 2;
                const double qi = p[i] - K * v[i], qj = p[j] - K * v[j];
                double *a = A.at(r + i, r + j);
                *a = __ldcg(a) - v[i] * qj - qi * v[j];
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) st_rel(progress + (s - 1), k + 1);
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

cudaError_t band_to_tridi_d(int n, int b, const double *AB, int ldab, double *d, double *e, double *hh_v,
                            double *hh_tau, void *ws, size_t ws_bytes, long long timeout_ns, cudaStream_t st)
{
    (void)ws_bytes;
    const long long ldw = 2LL * b;
    char *flags = (char *)ws;
    double *W = (double *)(flags + flags_bytes(n));
    cudaError_t err = cudaMemsetAsync(flags, 0, flags_bytes(n), st);
    if (err != cudaSuccess) return err;
    band_init<<<1024, 256, 0, st>>>(n, b, AB, ldab, W, ldw);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (n > 1) {
        chase_d<<<(unsigned)(n - 1), kChaseThreads, 0, st>>>(n, b, Band{W, ldw}, hh_v, hh_tau,
                                                            (ChaseState *)flags, (int *)(flags + 256), timeout_ns);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    band_extract<<<64, 256, 0, st>>>(n, W, ldw, d, e);
    return cudaGetLastError();
}

}  // namespace gb
