// trans_ev_tridi_to_band, shared-memory window: complex Hermitian case (any
// nbw) and real case with nbw above the register kernels' limit.
//
// Same tile schedule as the register wavefront (one launch per anti-diagonal
// of the tile graph, tiles of nb sweeps at one block index), but the window
// of b+nb-1 rows x THREADS columns lives in shared memory: a complex window
// of 64+nb rows would need over 256 registers per thread.  Each thread still
// owns one column, so the FP64 work is the algorithmic count: for complex
// data 4 DFMA per element for w = v^H z and 4 for z -= (tau w) v.
#include <cuda_runtime.h>

#include "layout.cuh"
#include "trans_ev_kernels.cuh"

namespace gb {

struct Cplx {
    double re, im;
};

template <typename T>
struct Ops;

template <>
struct Ops<double> {
    __device__ static double zero() { return 0.0; }
    __device__ static double one() { return 1.0; }
    __device__ static bool is_zero(double t) { return t == 0.0; }
    // acc += conj(v) * z
    __device__ static void dot(double &acc, double v, double z) { acc = fma(v, z, acc); }
    // z -= t * v
    __device__ static void axpy(double &z, double t, double v) { z = fma(-t, v, z); }
    __device__ static double mul(double a, double b) { return a * b; }
    __device__ static void sub(double &z, double t) { z -= t; }
};

template <>
struct Ops<Cplx> {
    __device__ static Cplx zero() { return {0.0, 0.0}; }
    __device__ static Cplx one() { return {1.0, 0.0}; }
    __device__ static bool is_zero(Cplx t) { return t.re == 0.0 && t.im == 0.0; }
    __device__ static void dot(Cplx &acc, Cplx v, Cplx z)
    {
        // conj(v) z = (vr zr + vi zi) + i (vr zi - vi zr)
        acc.re = fma(v.re, z.re, acc.re);
        acc.re = fma(v.im, z.im, acc.re);
        acc.im = fma(v.re, z.im, acc.im);
        acc.im = fma(-v.im, z.re, acc.im);
    }
    __device__ static void axpy(Cplx &z, Cplx t, Cplx v)
    {
        // t v = (tr vr - ti vi) + i (tr vi + ti vr)
        z.re = fma(-t.re, v.re, z.re);
        z.re = fma(t.im, v.im, z.re);
        z.im = fma(-t.re, v.im, z.im);
        z.im = fma(-t.im, v.re, z.im);
    }
    __device__ static Cplx mul(Cplx a, Cplx b)
    {
        return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
    }
    __device__ static void sub(Cplx &z, Cplx t)
    {
        z.re -= t.re;
        z.im -= t.im;
    }
};

template <typename T, int NB, int THREADS>
__global__ void __launch_bounds__(THREADS)
wavefront_smem(int n, int b, int nev, const T *__restrict__ hh_v, const T *__restrict__ hh_tau,
               T *__restrict__ Z, long long ldz, int t, int G, int jmin)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = b + NB - 1;
    T *vs = reinterpret_cast<T *>(smem_raw);  // [NB][b]
    T *ts = vs + NB * b;                       // [NB]
    T *zs = ts + NB;                           // [L][THREADS]

    const int j = jmin + (int)blockIdx.x;
    const int g = G - 1 - j;
    const int k = t - j;
    const int s0 = 1 + g * NB;

    for (int e = threadIdx.x; e < NB * b; e += THREADS) {
        int q = e / b, i = e - q * b;
        int s = s0 + q;
        T val = Ops<T>::zero();
        if (s <= n - 1 && s + k * b < n) {
            int len = min(b, n - s - k * b);
            if (i == 0) val = Ops<T>::one();
            else if (i < len) val = hh_v[(sweep_first(n, b, s) + k) * (long long)b + i];
        }
        vs[e] = val;
    }
    if (threadIdx.x < NB) {
        int s = s0 + threadIdx.x;
        ts[threadIdx.x] = (s <= n - 1 && s + k * b < n) ? hh_tau[sweep_first(n, b, s) + k] : Ops<T>::zero();
    }
    const int col = blockIdx.y * THREADS + threadIdx.x;
    const bool active = col < nev;
    const T *zc_in = Z + (long long)(active ? col : 0) * ldz;
    const long long row0 = (long long)s0 + (long long)k * b;
    for (int i = 0; i < L; i++) {
        long long r = row0 + i;
        zs[i * THREADS + threadIdx.x] = (active && r < n) ? zc_in[r] : Ops<T>::zero();
    }
    __syncthreads();

    T *zcol = zs + threadIdx.x;
    for (int q = NB - 1; q >= 0; q--) {
        const T tau = ts[q];
        if (Ops<T>::is_zero(tau)) continue;
        const T *v = vs + q * b;
        T *zq = zcol + q * THREADS;
        T acc = zq[0];
        for (int i = 1; i < b; i++) Ops<T>::dot(acc, v[i], zq[i * THREADS]);
        const T tw = Ops<T>::mul(tau, acc);
        Ops<T>::sub(zq[0], tw);
        for (int i = 1; i < b; i++) Ops<T>::axpy(zq[i * THREADS], tw, v[i]);
    }

    if (active) {
        T *zc = Z + (long long)col * ldz;
        for (int i = 0; i < L; i++) {
            long long r = row0 + i;
            if (r < n) zc[r] = zs[i * THREADS + threadIdx.x];
        }
    }
}

template <typename T, int NB, int THREADS>
static cudaError_t run_smem(int n, int b, int nev, const T *hh_v, const T *hh_tau, T *Z, long long ldz,
                            cudaStream_t st)
{
    const int G = group_count(n, NB);
    if (G <= 0 || nev <= 0) return cudaSuccess;
    const size_t smem = sizeof(T) * ((size_t)NB * b + NB + (size_t)(b + NB - 1) * THREADS);
    cudaError_t e = cudaFuncSetAttribute(wavefront_smem<T, NB, THREADS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int T_ = 0;
    for (int j = 0; j < G; j++) T_ = max(T_, j + group_tiles(n, b, NB, G - 1 - j));
    const unsigned cols = (unsigned)((nev + THREADS - 1) / THREADS);
    int jmin = 0;
    if (cudaError_t em = mark_kernel_begin(st)) return em;
    for (int t = 0; t < T_; t++) {
        while (jmin < G && jmin + group_tiles(n, b, NB, G - 1 - jmin) <= t) jmin++;
        int jmax = min(t, G - 1);
        if (jmin > jmax) continue;
        dim3 grid((unsigned)(jmax - jmin + 1), cols);
        wavefront_smem<T, NB, THREADS><<<grid, THREADS, smem, st>>>(n, b, nev, hh_v, hh_tau, Z, ldz, t, G, jmin);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return mark_kernel_end(st);
}

template <typename T>
static cudaError_t dispatch_smem(int n, int b, int nev, const T *hh_v, const T *hh_tau, T *Z, long long ldz,
                                 int nb, int threads, cudaStream_t st)
{
#define GB_SM(NBB, TT) return run_smem<T, NBB, TT>(n, b, nev, hh_v, hh_tau, Z, ldz, st)
#define GB_SM_T(NBB)                         \
    do {                                     \
        if (threads <= 32) GB_SM(NBB, 32);   \
        GB_SM(NBB, 64);                      \
    } while (0)
    if (nb <= 4) GB_SM_T(4);
    if (nb <= 8) GB_SM_T(8);
    GB_SM_T(16);
#undef GB_SM_T
#undef GB_SM
}

cudaError_t wavefront_smem_z(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                             long long ldz, int nb, int threads, cudaStream_t st)
{
    return dispatch_smem<Cplx>(n, b, nev, reinterpret_cast<const Cplx *>(hh_v),
                               reinterpret_cast<const Cplx *>(hh_tau), reinterpret_cast<Cplx *>(Z), ldz, nb,
                               threads, st);
}

cudaError_t wavefront_smem_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                             long long ldz, int nb, int threads, cudaStream_t st)
{
    return dispatch_smem<double>(n, b, nev, hh_v, hh_tau, Z, ldz, nb, threads, st);
}

size_t wavefront_smem_bytes(int b, int nb, int threads, int is_complex)
{
    int NB = nb <= 4 ? 4 : nb <= 8 ? 8 : 16;
    int TT = threads <= 32 ? 32 : 64;
    return (is_complex ? 16 : 8) * ((size_t)NB * b + NB + (size_t)(b + NB - 1) * TT);
}

}  // namespace gb
