// trans_ev_tridi_to_band, pipeline variant: one persistent-style launch.
//
// Work item (g, c) = all tiles k = 0..K_g-1 of sweep group g for column
// block c.  A block takes a ticket from a global counter; tickets run over
// batches of CB column blocks, and within a batch in the order g = G-1 down
// to 0 (the highest sweeps are applied first), so every item waits only on
// an item with a smaller ticket, which is already running or done: the
// launch cannot deadlock, whatever the residency.  Batching keeps the
// resident blocks on few columns, so consecutive groups of one column block
// run about one tile apart and the rows group g+1 writes are still in L2
// when group g reads them (without batching the resident groups spread over
// the whole matrix and every row round-trips through DRAM).
//
// The window of b+nb-1 rows slides down one column block: after tile k the
// top b rows are final for this group and are stored, the bottom nb-1 rows
// are carried in registers into tile k+1, and b new rows are loaded.  Those
// rows come from group g+1, which publishes progress[g+1][c] = k+1 after it
// has stored the rows final after its tile k (and the whole window after its
// last tile); tile k of group g needs progress[g+1][c] >= min(k+1, K_{g+1}).
// Rows that group g overwrites have already been read by group g+1, which
// is at least one tile ahead.
//
// Lead limit: once group g-1 of the same column block has started, group g
// runs tile k only after g-1 has completed k - lead tiles.  Without it the
// groups of a batch drift many tiles apart, the live rows of a batch span
// the whole column height, and rows round-trip through DRAM between
// consecutive groups.  Progress words start at -1 ("not started"); an item
// publishes 0 when it starts.  No deadlock for lead >= 1: the lowest started
// group of a column block has no started successor, so it is never held by
// the limit, and if it waits for its predecessor then that one is not held
// by the limit either (it is less than one tile ahead), and so on up to the
// highest unfinished group, whose predecessor has finished.
//
// Waits are bounded: thread 0 polls with an acquire load and a short sleep;
// after spin_polls polls or timeout_ns nanoseconds it records
// GB_ERR_TIMEOUT, raises an abort flag that every other waiter also checks,
// and the block returns.  The host reads the status with gb_trans_ev_query.
#include <cuda_runtime.h>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "trans_ev_kernels.cuh"

namespace gb {

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Default column blocks per ticket batch, and no lead limit: on GB300 at
// n = 16384 every limit that cut the DRAM traffic (2 tiles: 175 -> 50 GB per
// launch) also stalled the chains (1.97 -> 4.4 s), because a group that
// starts at tile 0 holds back the groups started before it.
constexpr int kColumnBatch = 16;
constexpr int kLeadTiles = 1 << 30;

struct PipeState {  // head of the workspace (zeroed before every launch)
    int ticket;
    int abort;
    int error;
};

template <int B, int NB, int THREADS>
__global__ void __launch_bounds__(THREADS)
pipeline_d(int n, int nev, const double *__restrict__ hh_v, const double *__restrict__ hh_tau,
           double *__restrict__ Z, long long ldz, int G, int C, int CB, int lead, PipeState *state,
           int *progress, long long spin_polls, long long timeout_ns, int hold_group)
{
    constexpr int L = B + NB - 1;
    constexpr int b = B;
    __shared__ __align__(16) double vs[NB][B];
    __shared__ double ts[NB];
    __shared__ int s_item, s_abort;

    if (threadIdx.x == 0) s_item = atomicAdd(&state->ticket, 1);
    __syncthreads();
    const int item = s_item;
    const int batch = item / (G * CB);                // all earlier batches are full
    const int rem = item - batch * G * CB;
    const int cb = min(CB, C - batch * CB);           // column blocks in this batch
    const int g = G - 1 - rem / cb;
    const int c = batch * CB + rem % cb;
    const int s0 = 1 + g * NB;
    const int K = group_tiles(n, b, NB, g);
    const int Knext = (g + 1 < G) ? group_tiles(n, b, NB, g + 1) : 0;
    const int col = c * THREADS + threadIdx.x;
    const bool active = col < nev;
    double *zc = Z + (long long)(active ? col : 0) * ldz;

    double w[L];
#pragma unroll
    for (int i = 0; i < L; i++) w[i] = 0.0;
    if (threadIdx.x == 0 && g + 1 != hold_group) st_release_gpu(progress + (long long)g * C + c, 0);

    for (int k = 0; k < K; k++) {
        // ---- wait for group g+1 to have finalised the rows this tile reads,
        // and for group g-1 (once started) to be at most `lead` tiles behind
        if (threadIdx.x == 0) {
            int abort = 0;
            const int need = (g + 1 < G) ? min(k + 1, Knext) : 0;
            const int *flag = progress + (long long)(g + 1) * C + c;
            const int behind = k - lead;  // tiles g-1 must have completed
            const int *succ = progress + (long long)(g - 1) * C + c;
            unsigned long long t0 = 0;
            long long polls = 0;
            for (;;) {
                bool ok = need == 0 || ld_acquire_gpu(flag) >= need;
                if (ok && g > 0 && behind > 0) {
                    const int p = *(volatile const int *)succ;
                    ok = p < 0 || p >= behind;
                }
                if (ok) break;
                if (*(volatile int *)&state->abort) { abort = 1; break; }
                if (polls == 0) t0 = global_ns();
                if (++polls >= spin_polls || (long long)(global_ns() - t0) > timeout_ns) {
                    atomicExch(&state->error, GB_ERR_TIMEOUT);
                    atomicExch(&state->abort, 1);
                    abort = 1;
                    break;
                }
                __nanosleep(128);
            }
            if (!abort && *(volatile int *)&state->abort) abort = 1;
            s_abort = abort;
        }
        // ---- stage the tile's reflectors (v_0 = 1, zero past len)
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
        if (s_abort) return;

        // ---- bring the window to tile k: carry nb-1 rows, load the rest
        const long long row0 = (long long)s0 + (long long)k * b;
        if (k > 0) {
#pragma unroll
            for (int i = 0; i < NB - 1; i++) w[i] = w[i + B];
        }
#pragma unroll
        for (int i = 0; i < L; i++) {
            if (k == 0 || i >= NB - 1) {
                long long r = row0 + i;
                w[i] = (active && r < n) ? __ldcg(zc + r) : 0.0;
            }
        }

        apply_tile_regs<B, NB>(w, vs, ts);

        // ---- store the rows that are final for this group
        const bool last = (k == K - 1);
#pragma unroll
        for (int i = 0; i < L; i++) {
            long long r = row0 + i;
            if (active && r < n && (i < B || last)) zc[r] = w[i];
        }
        __threadfence();
        __syncthreads();  // all rows stored (and vs/ts free for the next tile)
        if (threadIdx.x == 0 && g + 1 != hold_group)
            st_release_gpu(progress + (long long)g * C + c, k + 1);
    }
}

template <int B, int NB, int THREADS>
static cudaError_t run_pipeline_d(int n, int nev, const double *hh_v, const double *hh_tau, double *Z,
                                  long long ldz, int column_batch, int lead_tiles, void *ws, size_t ws_bytes,
                                  long long spin_polls, long long timeout_ns, int hold_group, cudaStream_t st)
{
    const int G = group_count(n, NB);
    const int C = (nev + THREADS - 1) / THREADS;
    if (G <= 0 || nev <= 0) return cudaSuccess;
    // head zeroed, progress words set to -1 ("not started")
    cudaError_t e = cudaMemsetAsync(ws, 0, 256, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync((char *)ws + 256, 0xff, ws_bytes - 256, st)) != cudaSuccess) return e;
    PipeState *state = (PipeState *)ws;
    int *progress = (int *)((char *)ws + 256);
    const int lead = lead_tiles > 0 ? lead_tiles : kLeadTiles;
    const int want = column_batch > 0 ? column_batch : kColumnBatch;
    const int CB = C < want ? C : want;
    if ((e = mark_kernel_begin(st)) != cudaSuccess) return e;
    pipeline_d<B, NB, THREADS><<<(unsigned)G * (unsigned)C, THREADS, 0, st>>>(
        n, nev, hh_v, hh_tau, Z, ldz, G, C, CB, lead, state, progress, spin_polls, timeout_ns, hold_group);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = mark_kernel_end(st)) != cudaSuccess) return e;
    return cudaSuccess;
}

size_t pipeline_workspace_bytes(int n, int nev, int nb, int threads)
{
    int NB = nb <= 8 ? 8 : 16;
    long long G = group_count(n, NB);
    long long C = (nev + threads - 1) / threads;
    size_t bytes = 256 + (size_t)(G * C) * sizeof(int);
    return (bytes + 255) & ~(size_t)255;
}

bool pipeline_supported(int b) { return b == 8 || b == 16 || b == 32 || b == 64; }

cudaError_t pipeline_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                       long long ldz, int nb, int threads, int column_batch, int lead_tiles, void *ws,
                       size_t ws_bytes, long long spin_polls, long long timeout_ns, int hold_group, cudaStream_t st)
{
#define GB_PL(BB, NBB, TT)                                                                                \
    return run_pipeline_d<BB, NBB, TT>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, lead_tiles, ws, ws_bytes, \
                                       spin_polls, timeout_ns, hold_group, st)
#define GB_PL_T(BB, NBB)                        \
    do {                                        \
        if (threads <= 64) GB_PL(BB, NBB, 64);  \
        GB_PL(BB, NBB, 128);                    \
    } while (0)
#define GB_PL_NB(BB)                  \
    do {                              \
        if (nb <= 8) GB_PL_T(BB, 8);  \
        GB_PL_T(BB, 16);              \
    } while (0)
    if (b == 8) GB_PL_NB(8);
    if (b == 16) GB_PL_NB(16);
    if (b == 32) GB_PL_NB(32);
    if (b == 64) GB_PL_NB(64);
    return cudaErrorInvalidValue;
#undef GB_PL_NB
#undef GB_PL_T
#undef GB_PL
}

}  // namespace gb
