// trans_ev_tridi_to_band, wavefront variant: one launch per anti-diagonal of
// the tile dependency graph.
//
// The reflectors are regrouped into tiles (g, k): the H(s,k) of nb
// consecutive sweeps s0..s0+nb-1 at one block index k.  Within a tile the
// sweeps are applied in descending order (the last-generated first); H(s,k)
// overlaps a reflector of a later sweep s' > s only when k' = k or k' = k-1
// (rows of one sweep are disjoint), so tile (g,k) must follow (g,k-1),
// (g+1,k) and (g+1,k-1), and all tiles on the anti-diagonal
// t = k + (G-1-g) touch disjoint rows and run concurrently.
//
// GB300's FP64 throughput is about 2 DFMA per clock per SM (measured:
// 1.19 TFLOP/s for DFMA, 1.05 TFLOP/s for the f64 mma.sync shapes), so the
// kernel issues exactly the algorithmic FP64 work: per column and reflector
// len-1 DFMA for w = v^T z (v_0 = 1), one DMUL for tau*w and len DFMA/DADD for
// z -= (tau w) v.  Each thread owns one column of Z; the tile's window of
// b+nb-1 rows lives in registers (indices are compile-time after unrolling)
// and the nb reflectors of the tile are staged in shared memory, read as
// warp-wide broadcasts.
#include <cuda_runtime.h>

#include "layout.cuh"
#include "trans_ev_kernels.cuh"

namespace gb {

template <int B, int NB, int THREADS>
__global__ void __launch_bounds__(THREADS)
wavefront_tile_d(int n, int b, int nev, const double *__restrict__ hh_v,
                 const double *__restrict__ hh_tau, double *__restrict__ Z, long long ldz,
                 int t, int G, int jmin)
{
    constexpr int L = B + NB - 1;
    __shared__ __align__(16) double vs[NB][B];
    __shared__ double ts[NB];

    const int j = jmin + (int)blockIdx.x;  // j = G-1-g
    const int g = G - 1 - j;
    const int k = t - j;
    const int s0 = 1 + g * NB;

    // Stage the tile's reflectors: rows q = s - s0; v_0 = 1; zero past len.
    for (int e = threadIdx.x; e < NB * B; e += THREADS) {
        int q = e / B, i = e - q * B;
        int s = s0 + q;
        double val = 0.0;
        if (s <= n - 1 && s + k * b < n) {
            int len = min(b, n - s - k * b);
            if (i == 0) val = 1.0;
            else if (i < len) val = hh_v[(sweep_first(n, b, s) + k) * (long long)b + i];
        }
        vs[q][i] = val;
    }
    if (threadIdx.x < NB) {
        int s = s0 + threadIdx.x;
        ts[threadIdx.x] = (s <= n - 1 && s + k * b < n) ? hh_tau[sweep_first(n, b, s) + k] : 0.0;
    }
    __syncthreads();

    const int col = blockIdx.y * THREADS + threadIdx.x;
    if (col >= nev) return;
    double *zc = Z + (long long)col * ldz;
    const long long row0 = (long long)s0 + (long long)k * b;  // 0-based top row of the window
    const int wrows = b + NB - 1;                             // rows this tile owns

    double w[L];
#pragma unroll
    for (int i = 0; i < L; i++) {
        long long r = row0 + i;
        w[i] = (i < wrows && r < n) ? zc[r] : 0.0;
    }
    apply_tile_regs<B, NB>(w, vs, ts);
#pragma unroll
    for (int i = 0; i < L; i++) {
        long long r = row0 + i;
        if (i < wrows && r < n) zc[r] = w[i];
    }
}

// Host side: launches for one call.  Returns a cudaError_t.
template <int B, int NB, int THREADS>
static cudaError_t run_wavefront_d(int n, int b, int nev, const double *hh_v, const double *hh_tau,
                                   double *Z, long long ldz, cudaStream_t st)
{
    const int G = group_count(n, NB);
    if (G <= 0 || nev <= 0) return cudaSuccess;
    // K(j) = tiles of group G-1-j, nondecreasing in j; j + K(j) strictly increasing.
    int T = 0;
    for (int j = 0; j < G; j++) T = max(T, j + group_tiles(n, b, NB, G - 1 - j));
    const unsigned cols = (unsigned)((nev + THREADS - 1) / THREADS);
    int jmin = 0;
    if (cudaError_t em = mark_kernel_begin(st)) return em;
    for (int t = 0; t < T; t++) {
        while (jmin < G && jmin + group_tiles(n, b, NB, G - 1 - jmin) <= t) jmin++;
        int jmax = min(t, G - 1);
        if (jmin > jmax) continue;
        dim3 grid((unsigned)(jmax - jmin + 1), cols);
        wavefront_tile_d<B, NB, THREADS><<<grid, THREADS, 0, st>>>(n, b, nev, hh_v, hh_tau, Z, ldz,
                                                                   t, G, jmin);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return mark_kernel_end(st);
}

template <int NB>
static long long wavefront_launches(int n, int b)
{
    const int G = group_count(n, NB);
    if (G <= 0) return 0;
    int T = 0;
    for (int j = 0; j < G; j++) T = max(T, j + group_tiles(n, b, NB, G - 1 - j));
    long long cnt = 0;
    int jmin = 0;
    for (int t = 0; t < T; t++) {
        while (jmin < G && jmin + group_tiles(n, b, NB, G - 1 - jmin) <= t) jmin++;
        if (jmin <= min(t, G - 1)) cnt++;
    }
    return cnt;
}

cudaError_t wavefront_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                        long long ldz, int nb, int threads, cudaStream_t st)
{
#define GB_WF(BB, NBB, TT) return run_wavefront_d<BB, NBB, TT>(n, b, nev, hh_v, hh_tau, Z, ldz, st)
#define GB_WF_T(BB, NBB)          \
    do {                          \
        if (threads == 32) GB_WF(BB, NBB, 32);  \
        if (threads == 64) GB_WF(BB, NBB, 64);  \
        GB_WF(BB, NBB, 128);      \
    } while (0)
#define GB_WF_NB(BB)              \
    do {                          \
        if (nb <= 4) GB_WF_T(BB, 4);   \
        if (nb <= 8) GB_WF_T(BB, 8);   \
        GB_WF_T(BB, 16);          \
    } while (0)
    if (b <= 8) GB_WF_NB(8);
    if (b <= 16) GB_WF_NB(16);
    if (b <= 32) GB_WF_NB(32);
    GB_WF_NB(64);
#undef GB_WF_NB
#undef GB_WF_T
#undef GB_WF
}

long long wavefront_launch_count(int n, int b, int nb)
{
    if (nb <= 4) return wavefront_launches<4>(n, b);
    if (nb <= 8) return wavefront_launches<8>(n, b);
    return wavefront_launches<16>(n, b);
}

}  // namespace gb
