// trans_ev_tridi_to_band on the tcgen05 tensor cores (the default for real
// data with nbw in {16, 32, 64}).
//
// Schedule (as in the other pipelines): work item (g, c) = all tiles of
// sweep group g (NB = 16 sweeps) for column block c (128 columns); items
// take tickets in batches of column blocks, groups descending, so every
// dependency wait targets an item that is already running; tile k of group
// g waits until group g+1 has published min(k+1, K_{g+1}) tiles.  All waits
// are bounded.
//
// Tile algebra (Sec. 3.1's blocked Householder aggregation): the tile's 16
// reflectors, applied last sweep first, multiply to I - V T V^T, with V the
// (b+15) x 16 parallelogram of reflectors and T upper triangular; with
// U = V T (V's columns scaled to unit length, U's by the inverse factors),
//     Z_win <- Z_win - U (V^T Z_win).
// Both products run on the tensor cores, transposed so that the 128
// eigenvector columns are the MMA's M dimension:
//     W^T  (128 x 16)  = Z_win^T (128 x LP) . V   (LP x 16)
//     dZ^T (128 x LP)  = W^T     (128 x 16) . U^T (16 x LP)
//
// Exact FP64-accurate arithmetic from FP16 digits:
//  * Z is per-column 64-bit fixed point for the whole call (tc_fixed.cuh),
//    |Zi| < 2^61.  V and U rows are fixed point against per-row powers of
//    two, |Vi|, |Ui| <= 2^62.
//  * Every 64-bit value x is cut into eight balanced base-256 digits
//    d_s in [-128, 127] (s = 0 most significant): with y = x +
//    0x8080808080808080 (mod 2^64), d_s = byte_{7-s}(y) - 128, and
//    x = sum_s d_s 256^(7-s).  Each digit is exact in FP16.
//  * Digit products of level l = s + t <= 8 (43 pairs) accumulate in FP32 in
//    TMEM, one accumulator per level.  A level sums at most 8 pairs x K
//    products of magnitude <= 2^14; for K = 80 that is < 2^23.4, so every
//    level sum is an exact integer.  The dropped levels (>= 9) are below
//    2^-69 of the products' scale.
//  * Levels are folded into 64-bit integers (one rounding per entry) and the
//    update Zi -= dZi is an integer subtraction.
//
// Data movement per tile (b = 64, LP = 80):
//  * the tile record (V and U^T digit planes in the MMA's canonical
//    K-major layout, row exponents; 41 KB, built once per tile by
//    tc5_tile_prep) arrives by cp.async.bulk on an mbarrier, one tile ahead;
//  * the window (LP rows x 128 columns, int64) lives in shared memory;
//    the 64 new rows come from global memory through L2, 15 rows carry over;
//  * Z's digit planes are cut by the threads straight into TMEM (tcgen05.st)
//    and are the A operand of the first product (A from TMEM); W's digit
//    planes are the A operand of the second.
// TMEM (512 columns): Z digits [0, 64 KSTEPS), W levels [64 KSTEPS, +144);
// then W digits [0, 64) and the dZ levels of a row chunk [64, 64 + 9 N).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "mma_bf16.cuh"
#include "tc_fixed.cuh"
#include "tcgen05.cuh"
#include "trans_ev_kernels.cuh"

namespace gb {

namespace {

constexpr int kNB5 = 16;          // sweeps per tile
constexpr int kCols5 = 128;       // eigenvector columns per work item (the MMA's M)
constexpr int kThreads5 = 512;    // 16 warps: four per TMEM lane quarter (and per SM sub-partition)
constexpr int kPlanes = 8;        // balanced base-256 digits of a 64-bit value
constexpr int kLevels5 = 9;       // digit-pair levels 0..8
constexpr int kColumnBatch5 = 4;  // 128-column blocks per ticket batch
constexpr int kTmemCols = 512;
constexpr unsigned long long kDigitBias = 0x8080808080808080ull;
constexpr long long kMbarTimeoutNs = 2000000000ll;  // an MMA batch or a record copy takes microseconds

template <int B>
struct Geo {
    static constexpr int L = B + kNB5 - 1;             // window rows
    static constexpr int LP = (L + 15) / 16 * 16;      // padded to the MMA's K step
    static constexpr int KSTEPS = LP / 16;
    static constexpr int PLANE = 32 * LP;              // bytes of one V (16 x LP) or U^T (LP x 16) digit plane
    // tile record (global and shared): V planes, U^T planes, eV[16], eU[LP]
    static constexpr int R_V = 0;
    static constexpr int R_U = kPlanes * PLANE;
    static constexpr int R_EV = 2 * kPlanes * PLANE;
    static constexpr int R_EU = R_EV + 16 * 4;
    static constexpr int REC = (R_EU + LP * 4 + 127) / 128 * 128;
    // window: [128 columns][ZROW] int64, ZROW = 2 mod 4 so that a warp's
    // 16-byte accesses to one row pair of 32 columns are conflict-free
    static constexpr int ZROW = LP + 2;
    // dZ row chunks of up to 32 rows (an MMA's N = 32 rows x up to 8 U
    // planes <= 256); the U^T record is laid out chunk by chunk, the planes
    // of a chunk contiguous along N
    static constexpr int NCH = 32;
    static constexpr int CHUNKS = (LP + NCH - 1) / NCH;
    // TMEM columns
    static constexpr int T_ZD = 0;
    static constexpr int T_WACC = 64 * KSTEPS;
    static constexpr int T_WD = 0;
    static constexpr int T_DZ = 64;
    // shared memory
    static constexpr int S_REC = 0;                          // two record buffers
    static constexpr int S_Z = 2 * REC;
    static constexpr int S_BAR = S_Z + kCols5 * ZROW * 8;    // 3 mbarriers + TMEM base
    static constexpr int SMEM = S_BAR + 64;
    static_assert(T_WACC + 16 * kLevels5 <= kTmemCols, "Z digits and W levels fit in TMEM");
    static_assert(T_DZ + kLevels5 * NCH <= kTmemCols, "dZ levels fit");
    static_assert(8 * LP * 128 * 128 < (1 << 24), "W level sums stay exact in FP32");
    static_assert(LP % 16 == 0 && (NCH / 4) % 4 == 0, "row chunks (the last one 16 or 32 rows)");
    static_assert((LP / 8) * 8 == LP, "cut units of 8 rows");
    static_assert(REC % 128 == 0 && SMEM <= 227 * 1024, "shared memory");
};

// ---- digits ----------------------------------------------------------------

// FP16 pair (low half from a, high half from b) of the balanced digits held
// in byte `bi` of a and of b (biased bytes: digit = byte - 128).  0x6400|m is
// the FP16 value 1024 + m for 0 <= m < 1024, so subtracting 1152 is exact.
__device__ __forceinline__ uint32_t digit_pair(uint32_t a, uint32_t b, int bi)
{
    const uint32_t sel = (uint32_t)bi | ((uint32_t)bi << 4) | ((uint32_t)(4 + bi) << 8) | ((uint32_t)(4 + bi) << 12);
    const uint32_t r = (__byte_perm(a, b, sel) & 0x00ff00ffu) | 0x64006400u;
    const __half2 h = __hsub2(*(const __half2 *)&r, __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));
    return *(const uint32_t *)&h;
}

// the eight digit planes of the pair (x0, x1): out[s] holds plane s
__device__ __forceinline__ void cut_pair(long long x0, long long x1, uint32_t (&out)[kPlanes])
{
    const unsigned long long y0 = (unsigned long long)x0 + kDigitBias;
    const unsigned long long y1 = (unsigned long long)x1 + kDigitBias;
    const uint32_t a_hi = (uint32_t)(y0 >> 32), a_lo = (uint32_t)y0;
    const uint32_t b_hi = (uint32_t)(y1 >> 32), b_lo = (uint32_t)y1;
#pragma unroll
    for (int s = 0; s < 4; s++) out[s] = digit_pair(a_hi, b_hi, 3 - s);
#pragma unroll
    for (int s = 4; s < 8; s++) out[s] = digit_pair(a_lo, b_lo, 7 - s);
}

// sum_l L_l 2^(50 - 8 l + e) from nine exact level sums, rounded once:
// hi = sum_{l<4} L_l 2^(8(3-l)), lo = sum_{l>=4} L_l 2^(8(8-l)).
// (mod 2^64 arithmetic; the result fits since it is a fixed-point entry)
__device__ __forceinline__ long long fold9(const int (&Lv)[kLevels5], int e)
{
    const long long hi = ((long long)Lv[0] << 24) + ((long long)Lv[1] << 16) + ((long long)Lv[2] << 8) + Lv[3];
    const long long lo = ((long long)Lv[4] << 32) + ((long long)Lv[5] << 24) + ((long long)Lv[6] << 16) +
                         ((long long)Lv[7] << 8) + Lv[8];
    return (long long)((unsigned long long)shift_ll(hi, 26 + e) + (unsigned long long)shift_ll(lo, e - 14));
}

// An FP32 level sum x (an integer, |x| < 2^22) plus 1.5 2^23 has the bit
// pattern 0x4B400000 + x.  Two such patterns combine into the int32
// L_a 2^8 + L_b with one multiply-add and one subtraction of the combined
// offset (257 * 0x4B400000 mod 2^32), exact whenever |L_a 2^8 + L_b| < 2^31.
constexpr uint32_t kMagicBits = 0x4B400000u;
constexpr uint32_t kPairBias = 0x4B400000u * 257u;

__device__ __forceinline__ uint32_t magic_bits(uint32_t f)
{
    return __float_as_uint(__fadd_rn(__uint_as_float(f), 12582912.0f));
}

__device__ __forceinline__ int pair_from_bits(uint32_t a, uint32_t b) { return (int)(a * 256u + b - kPairBias); }

// fold9 for level sums below 2^22 given as magic bit patterns (the dZ
// product: K = 16, at most 8 pairs of magnitude <= 2^14 per level)
__device__ __forceinline__ long long fold9_bits(const uint32_t (&b)[kLevels5], int e)
{
    const int p0 = pair_from_bits(b[0], b[1]), p1 = pair_from_bits(b[2], b[3]);
    const int p2 = pair_from_bits(b[4], b[5]), p3 = pair_from_bits(b[6], b[7]);
    const int l8 = (int)(b[8] - kMagicBits);
    const long long hi = (long long)p0 * 65536 + p1;
    const long long lo = ((long long)p2 * 65536 + p3) * 256 + l8;
    return (long long)((unsigned long long)shift_ll(hi, 26 + e) + (unsigned long long)shift_ll(lo, e - 14));
}

// round(x 2^(62 - e)) for |x| < 2^e: the row's fixed point (|result| <= 2^62)
__device__ __forceinline__ long long fixed_row(double x, int e) { return __double2ll_rn(scale_by_pow2(x, 62 - e)); }

// ---- per-tile records ------------------------------------------------------

template <int B>
__global__ void __launch_bounds__(128) tc5_tile_prep(int n, const double *__restrict__ hh_v,
                                                     const double *__restrict__ hh_tau,
                                                     const long long *__restrict__ off,
                                                     unsigned char *__restrict__ rec)
{
    using Gm = Geo<B>;
    constexpr int L = Gm::L, LP = Gm::LP;
    const int k = blockIdx.x, g = blockIdx.y;
    const int b = B;
    if (k >= group_tiles(n, b, kNB5, g)) return;
    __shared__ double V[LP][kNB5 + 1];
    __shared__ double U[LP][kNB5 + 1];
    __shared__ double T[kNB5][kNB5 + 1];
    __shared__ double Gr[kNB5][kNB5 + 1];
    __shared__ double tau[kNB5];
    __shared__ double nv[kNB5];
    __shared__ int seV[kNB5], seU[LP];
    const int s0 = 1 + g * kNB5;
    // reflector q of the tile occupies window rows q .. q+len-1 of column q
    for (int e = threadIdx.x; e < LP * kNB5; e += blockDim.x) {
        const int j = e / kNB5, q = e % kNB5;
        const int s = s0 + q;
        double val = 0.0;
        if (s <= n - 1 && s + k * b < n && j - q >= 0 && j - q < b && j < L) {
            const long long idx = sweep_first(n, b, s) + k;
            const int len = min(b, n - s - k * b);
            const double t = hh_tau[idx];
            const int i = j - q;
            if (t != 0.0 && i < len) val = (i == 0) ? 1.0 : hh_v[idx * b + i];
        }
        V[j][q] = val;
    }
    if (threadIdx.x < kNB5) {
        const int s = s0 + threadIdx.x;
        tau[threadIdx.x] = (s <= n - 1 && s + k * b < n) ? hh_tau[sweep_first(n, b, s) + k] : 0.0;
    }
    __syncthreads();
    // Gram matrix (upper triangle), T by the forward recurrence
    // T(q,q) = tau_q, T(0:q,q) = -tau_q T(0:q,0:q) V(:,0:q)^T v_q
    for (int e = threadIdx.x; e < kNB5 * kNB5; e += blockDim.x) {
        const int p = e / kNB5, q = e % kNB5;
        double a = 0.0;
        if (p < q)
            for (int j = q; j < min(p + b, LP); j++) a = fma(V[j][p], V[j][q], a);
        Gr[p][q] = a;
    }
    __syncthreads();
    for (int q = 0; q < kNB5; q++) {
        if (threadIdx.x < kNB5) {
            const int i = threadIdx.x;
            double t = 0.0;
            if (i < q) {
                for (int p = i; p < q; p++) t = fma(T[i][p], Gr[p][q], t);
                t = -tau[q] * t;
            } else if (i == q) {
                t = tau[q];
            }
            T[i][q] = t;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < LP * kNB5; e += blockDim.x) {
        const int j = e / kNB5, q = e % kNB5;
        double a = 0.0;
        for (int p = 0; p <= q; p++) a = fma(V[j][p], T[p][q], a);
        U[j][q] = a;
    }
    // unit columns of V (U rescaled to keep U V^T): |v_q^T z| <= ||z||, so W
    // stays inside the column's fixed-point range whatever tau is
    if (threadIdx.x < kNB5) {
        double a = 0.0;
        for (int j = 0; j < LP; j++) a = fma(V[j][threadIdx.x], V[j][threadIdx.x], a);
        nv[threadIdx.x] = sqrt(a);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LP * kNB5; e += blockDim.x) {
        const int j = e / kNB5, q = e % kNB5;
        if (nv[q] > 0.0) {
            V[j][q] = V[j][q] / nv[q];
            U[j][q] = U[j][q] * nv[q];
        }
    }
    __syncthreads();
    unsigned char *r = rec + ((size_t)off[g] + k) * Gm::REC;
    if (threadIdx.x < kNB5) {
        unsigned long long m = 0;
        for (int j = 0; j < LP; j++) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(V[j][threadIdx.x]) & ~(1ull << 63);
            m = u > m ? u : m;
        }
        seV[threadIdx.x] = exponent_above(m);
        ((int *)(r + Gm::R_EV))[threadIdx.x] = seV[threadIdx.x];
    }
    for (int j = threadIdx.x; j < LP; j += blockDim.x) {
        unsigned long long m = 0;
        for (int q = 0; q < kNB5; q++) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(U[j][q]) & ~(1ull << 63);
            m = u > m ? u : m;
        }
        seU[j] = exponent_above(m);
        ((int *)(r + Gm::R_EU))[j] = seU[j];
    }
    __syncthreads();
    // digit planes in the canonical K-major layout of the B operands:
    // V (N = q, K = j), plane t: byte t 32 LP + (q/8) 16 LP + (j/8) 128 +
    // (q%8) 16 + (j%8) 2, so the planes follow each other along N at the same
    // 8-row stride (an MMA's B may span planes t0, t0+1, ...);
    // U^T (N = j, K = q), by chunks of 32 rows: chunk c = j/32 at c 8192,
    // within it plane t at t (rows of the chunk / 8) 256, then (j%32/8) 256 +
    // (q/8) 128 + (j%8) 16 + (q%8) 2 (again the planes contiguous along N)
    for (int e = threadIdx.x; e < kNB5 * LP; e += blockDim.x) {
        const int q = e / LP, j = e % LP;
        const unsigned long long y = (unsigned long long)fixed_row(V[j][q], seV[q]) + kDigitBias;
        const int o = (q >> 3) * 16 * LP + (j >> 3) * 128 + (q & 7) * 16 + (j & 7) * 2;
#pragma unroll
        for (int t = 0; t < kPlanes; t++)
            *(__half *)(r + Gm::R_V + t * Gm::PLANE + o) =
                __float2half_rn((float)((int)((y >> (56 - 8 * t)) & 0xff) - 128));
    }
    for (int e = threadIdx.x; e < LP * kNB5; e += blockDim.x) {
        const int j = e / kNB5, q = e % kNB5;
        const unsigned long long y = (unsigned long long)fixed_row(U[j][q], seU[j]) + kDigitBias;
        const int ch = j / Gm::NCH, rows = min(Gm::NCH, LP - ch * Gm::NCH);
        const int o = ch * Gm::NCH * 256 + ((j % Gm::NCH) >> 3) * 256 + (q >> 3) * 128 + (j & 7) * 16 + (q & 7) * 2;
#pragma unroll
        for (int t = 0; t < kPlanes; t++)
            *(__half *)(r + Gm::R_U + t * (rows / 8) * 256 + o) =
                __float2half_rn((float)((int)((y >> (56 - 8 * t)) & 0xff) - 128));
    }
}

// ---- the main kernel ------------------------------------------------------

struct Tc5Shared {
    int item;
    int abort;
};

template <int B>
__global__ void __launch_bounds__(kThreads5, 1)
pipeline_tc5(int n, int nev, long long *__restrict__ Zi, long long ldz, const unsigned char *__restrict__ rec,
             const long long *__restrict__ off, int G, int C, int CB, TcState *state, int *progress,
             long long spin_polls, long long timeout_ns, int hold_group)
{
    using Gm = Geo<B>;
    constexpr int L = Gm::L, LP = Gm::LP, ZROW = Gm::ZROW, KSTEPS = Gm::KSTEPS;
    extern __shared__ __align__(1024) unsigned char smem[];
    long long *Zs = (long long *)(smem + Gm::S_Z);
    const uint32_t bar_rec0 = tc5::smem_addr(smem + Gm::S_BAR);
    const uint32_t bar_mma = bar_rec0 + 16;
    uint32_t *tmem_slot = (uint32_t *)(smem + Gm::S_BAR + 32);
    __shared__ Tc5Shared sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, wq = warp >> 2;            // lane quarter, and which of its four warps
    const int col = quarter * 32 + lane;                    // this thread's column of the item (its TMEM lane)
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int b = B;

    if (tid == 0) {
        sh.item = atomicAdd(&state->ticket, 1);
        sh.abort = 0;
        tc5::mbar_init(bar_rec0, 1);
        tc5::mbar_init(bar_rec0 + 8, 1);
        tc5::mbar_init(bar_mma, 1);
        tc5::mbar_init_fence();
    }
    if (warp == 0) tc5::tmem_alloc(tc5::smem_addr(tmem_slot), kTmemCols);
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tmem = *(volatile uint32_t *)tmem_slot;

    const int item = sh.item;
    const int batch = item / (G * CB);
    const int rem = item - batch * G * CB;
    const int cb = min(CB, C - batch * CB);
    const int g = G - 1 - rem / cb;
    const int c = batch * CB + rem % cb;
    const int s0 = 1 + g * kNB5;
    const int K = group_tiles(n, b, kNB5, g);
    const int Knext = (g + 1 < G) ? group_tiles(n, b, kNB5, g + 1) : 0;
    const int col0 = c * kCols5;
    const unsigned char *rec_g = rec + (size_t)off[g] * Gm::REC;

    int issued = 0;        // records requested so far (thread 0)
    uint32_t mma_phase = 0;
    bool mma_pending = false;

    if (tid == 0) {
        if (g + 1 != hold_group) st_release(progress + (long long)g * C + c, 0);
        tc5::fence_proxy_async_smem();
        tc5::bulk_load(tc5::smem_addr(smem + Gm::S_REC), rec_g, Gm::REC, bar_rec0);
        issued = 1;
    }
    // window padding rows stay zero for the whole item
    for (int e = tid; e < kCols5 * (LP - L); e += kThreads5) Zs[(e / (LP - L)) * ZROW + L + e % (LP - L)] = 0;

    for (int k = 0; k < K; k++) {
        const int buf = k & 1;
        const unsigned char *srec = smem + Gm::S_REC + buf * Gm::REC;
        const int *eV = (const int *)(srec + Gm::R_EV);
        const int *eU = (const int *)(srec + Gm::R_EU);
        // ---- dependency wait; then request the next tile's record
        if (tid == 0) {
            int abort = 0;
            const int need = (g + 1 < G) ? min(k + 1, Knext) : 0;
            const int *flag = progress + (long long)(g + 1) * C + c;
            unsigned long long t0 = 0;
            long long polls = 0;
            while (need > 0 && ld_acquire(flag) < need) {
                if (*(volatile int *)&state->abort) { abort = 1; break; }
                if (polls == 0) t0 = now_ns();
                if (++polls >= spin_polls || (long long)(now_ns() - t0) > timeout_ns) {
                    tc_set_error(state, GB_ERR_TIMEOUT);
                    atomicExch(&state->abort, 1);
                    abort = 1;
                    break;
                }
                __nanosleep(128);
            }
            if (!abort && *(volatile int *)&state->abort) abort = 1;
            if (abort) sh.abort = 1;
            if (!abort && k + 1 < K) {
                tc5::fence_proxy_async_smem();
                tc5::bulk_load(tc5::smem_addr(smem + Gm::S_REC + (buf ^ 1) * Gm::REC), rec_g + (size_t)(k + 1) * Gm::REC,
                               Gm::REC, bar_rec0 + 8 * (buf ^ 1));
                issued = k + 2;
            }
        }
        __syncthreads();
        if (sh.abort) break;
        // ---- window: new rows from global memory (through L2: rows written
        // by other SMs), the 15 rows shared with the previous tile carried
        const long long row0 = (long long)s0 + (long long)k * b;
        const int jlo = (k == 0) ? 0 : kNB5 - 1;
        {
            constexpr int H = (L + 31) / 32;           // passes of 32 rows per column
            constexpr int CW = kCols5 / (kThreads5 / 32);  // columns per warp
            long long v[CW][H];
#pragma unroll
            for (int i = 0; i < CW; i++) {
                const int cc = warp * CW + i;
                const long long *zc = Zi + (long long)(col0 + cc < nev ? col0 + cc : 0) * ldz;
#pragma unroll
                for (int h = 0; h < H; h++) {
                    const int j = jlo + lane + 32 * h;
                    v[i][h] = (col0 + cc < nev && j < L && row0 + j < n) ? __ldcg(zc + row0 + j) : 0ll;
                }
            }
            if (k > 0) {
                for (int e = tid; e < kCols5 * (kNB5 - 1); e += kThreads5) {
                    const int cc = e / (kNB5 - 1), j = e % (kNB5 - 1);
                    Zs[cc * ZROW + j] = Zs[cc * ZROW + j + b];
                }
                __syncthreads();  // carried rows read before the new rows overwrite them
            }
#pragma unroll
            for (int i = 0; i < CW; i++) {
                const int cc = warp * CW + i;
#pragma unroll
                for (int h = 0; h < H; h++) {
                    const int j = jlo + lane + 32 * h;
                    if (j < L) Zs[cc * ZROW + j] = v[i][h];
                }
            }
        }
        __syncthreads();
        // ---- Z^T digit planes into TMEM: K step kk, plane s at columns
        // kk*64 + s*8 .. +7 (pairs of rows); units of 8 rows (half a K
        // step) go round-robin to the four warps of the lane quarter
        {
            const long long *zc = Zs + col * ZROW;
            for (int u = wq; u < LP / 8; u += 4) {
                uint32_t w[kPlanes][4];
#pragma unroll
                for (int p = 0; p < 4; p++) {
                    const longlong2 z2 = *(const longlong2 *)(zc + u * 8 + 2 * p);
                    uint32_t d[kPlanes];
                    cut_pair(z2.x, z2.y, d);
#pragma unroll
                    for (int s = 0; s < kPlanes; s++) w[s][p] = d[s];
                }
#pragma unroll
                for (int s = 0; s < kPlanes; s++)
                    tc5::st_x4(tmem + lane_off + Gm::T_ZD + (u >> 1) * 64 + s * 8 + (u & 1) * 4, w[s]);
            }
            tc5::wait_st();
        }
        // every thread sees the record land (its row exponents are read below)
        if (!tc5::mbar_wait(bar_rec0 + 8 * buf, (uint32_t)((k >> 1) & 1), kMbarTimeoutNs)) {
            tc_set_error(state, GB_ERR_TIMEOUT);
            atomicExch(&state->abort, 1);
            sh.abort = 1;
        }
        tc5::fence_before_sync();
        __syncthreads();
        if (sh.abort) break;
        // ---- W^T = Z^T V: 43 digit pairs x KSTEPS MMAs (M 128, N 16, K 16)
        if (tid == 0) {
            tc5::fence_after_sync();
            // one MMA per Z digit plane s and K step: B spans V planes
            // 0 .. 8-s along N, so plane t lands in level s+t (D columns
            // T_WACC + 16 (s+t)); in the first K step level 8 is first
            // written by its own MMA (s = 1, t = 7), every other level by s = 0
            const uint32_t sbase = tc5::smem_addr(srec);
            const uint64_t vdesc = tc5::smem_desc(sbase + Gm::R_V, 128, 16 * LP);
#pragma unroll
            for (int kk = 0; kk < KSTEPS; kk++)
#pragma unroll
                for (int s = 0; s < kPlanes; s++) {
                    const uint32_t a_t = tmem + Gm::T_ZD + kk * 64 + s * 8;
                    const uint64_t b0 = vdesc + (uint64_t)((kk * 256) >> 4);
                    const int nt = s == 0 ? kPlanes : kLevels5 - s;          // planes t = 0 .. nt-1
                    if (kk == 0 && s == 1) {
                        tc5::mma_tmem_a(tmem + Gm::T_WACC + 16 * 8, a_t, b0 + (uint64_t)((7 * Gm::PLANE) >> 4),
                                        tc5::idesc_f16_f32(128, 16), 0u);
                        tc5::mma_tmem_a(tmem + Gm::T_WACC + 16, a_t, b0, tc5::idesc_f16_f32(128, 16 * 7), 1u);
                    } else {
                        tc5::mma_tmem_a(tmem + Gm::T_WACC + 16 * s, a_t, b0, tc5::idesc_f16_f32(128, 16 * nt),
                                        (kk > 0 || s > 0) ? 1u : 0u);
                    }
                }
            tc5::commit(bar_mma);
            // publish the previous tile while the products run: its stores
            // happened before the barriers since, and the fence and release
            // here make them visible at GPU scope before the flag
            if (k > 0 && g + 1 != hold_group) {
                __threadfence();
                st_release(progress + (long long)g * C + c, k);
            }
        }
        mma_pending = true;
        if (!tc5::mbar_wait(bar_mma, mma_phase & 1, kMbarTimeoutNs)) {
            tc_set_error(state, GB_ERR_TIMEOUT);
            atomicExch(&state->abort, 1);
            sh.abort = 1;
        } else {
            mma_pending = false;
        }
        mma_phase++;
        tc5::fence_after_sync();
        // ---- fold W's levels (reflectors 4*wq .. +3 of this column), cut
        // W into digit planes (TMEM columns s*8 + 2*wq .. +1)
        {
            uint32_t a[kLevels5][4];
#pragma unroll
            for (int l = 0; l < kLevels5; l++) tc5::ld_x4(tmem + lane_off + Gm::T_WACC + 16 * l + 4 * wq, a[l]);
            tc5::wait_ld();
            uint32_t wd[kPlanes][2];
#pragma unroll
            for (int p = 0; p < 2; p++) {
                long long wi[2];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const int i = 2 * p + u;
                    int Lv[kLevels5];
#pragma unroll
                    for (int l = 0; l < kLevels5; l++) Lv[l] = __float2int_rn(__uint_as_float(a[l][i]));
                    wi[u] = fold9(Lv, eV[4 * wq + i]);
                }
                uint32_t d[kPlanes];
                cut_pair(wi[0], wi[1], d);
#pragma unroll
                for (int s = 0; s < kPlanes; s++) wd[s][p] = d[s];
            }
            // (the W digits go to the Z-digit columns, dead since the W
            // products completed; the W levels stay untouched until the dZ
            // products, issued after the barrier below)
#pragma unroll
            for (int s = 0; s < kPlanes; s++) tc5::st_x2(tmem + lane_off + Gm::T_WD + s * 8 + 2 * wq, wd[s]);
            tc5::wait_st();
        }
        tc5::fence_before_sync();
        __syncthreads();
        if (sh.abort) break;
        // ---- dZ^T = W^T U^T by row chunks (M 128, N = chunk, K 16), fold
        // into the window: Zs -= dZ
#pragma unroll
        for (int ch = 0; ch < Gm::CHUNKS; ch++) {
            const int j0 = ch * Gm::NCH;
            const int N = (LP - j0) < Gm::NCH ? (LP - j0) : Gm::NCH;
            if (ch) {
                tc5::fence_before_sync();
                __syncthreads();  // the previous chunk's levels are read before they are overwritten
                if (sh.abort) break;
            }
            if (tid == 0) {
                tc5::fence_after_sync();
                // per W digit plane s one MMA whose B spans the chunk's U
                // planes 0 .. 8-s along N (level l = s+t at D columns
                // T_DZ + l N); level 8 first written alone (s = 1, t = 7)
                const uint32_t sbase = tc5::smem_addr(srec);
                const uint64_t udesc = tc5::smem_desc(sbase + Gm::R_U + j0 * 256, 128, 256);
                const uint32_t pstride = (uint32_t)(N / 8) * 256;   // bytes between the chunk's planes
#pragma unroll
                for (int s = 0; s < kPlanes; s++) {
                    const uint32_t a_t = tmem + Gm::T_WD + s * 8;
                    const int nt = s == 0 ? kPlanes : kLevels5 - s;
                    if (s == 1) {
                        tc5::mma_tmem_a(tmem + Gm::T_DZ + 8 * N, a_t, udesc + (uint64_t)((7 * pstride) >> 4),
                                        tc5::idesc_f16_f32(128, N), 0u);
                        tc5::mma_tmem_a(tmem + Gm::T_DZ + N, a_t, udesc, tc5::idesc_f16_f32(128, 7 * N), 1u);
                    } else {
                        tc5::mma_tmem_a(tmem + Gm::T_DZ + s * N, a_t, udesc, tc5::idesc_f16_f32(128, nt * N),
                                        s > 0 ? 1u : 0u);
                    }
                }
                tc5::commit(bar_mma);
            }
            mma_pending = true;
            if (!tc5::mbar_wait(bar_mma, mma_phase & 1, kMbarTimeoutNs)) {
                tc_set_error(state, GB_ERR_TIMEOUT);
                atomicExch(&state->abort, 1);
                sh.abort = 1;
            } else {
                mma_pending = false;
            }
            mma_phase++;
            tc5::fence_after_sync();
            // this thread: rows j0 + wq*N/4 .. +N/4 of its column (8 or 4),
            // all levels fetched in one round of TMEM loads
            long long *zc = Zs + col * ZROW;
            const int jb = wq * (N / 4);
            uint32_t a8[kLevels5][8];
            if (N == 32) {
#pragma unroll
                for (int l = 0; l < kLevels5; l++) tc5::ld_x8(tmem + lane_off + Gm::T_DZ + l * N + jb, a8[l]);
            } else {
#pragma unroll
                for (int l = 0; l < kLevels5; l++) {
                    uint32_t a4[4];
                    tc5::ld_x4(tmem + lane_off + Gm::T_DZ + l * N + jb, a4);
#pragma unroll
                    for (int i = 0; i < 4; i++) a8[l][i] = a4[i];
                }
            }
            tc5::wait_ld();
#pragma unroll
            for (int blk = 0; blk < 2; blk++) {
                if (blk * 4 >= N / 4) break;
                const int jj = jb + blk * 4;
                uint32_t a[kLevels5][4];
#pragma unroll
                for (int l = 0; l < kLevels5; l++)
#pragma unroll
                    for (int i = 0; i < 4; i++) a[l][i] = a8[l][blk * 4 + i];
#pragma unroll
                for (int p = 0; p < 2; p++) {
                    const int j = j0 + jj + 2 * p;
                    if (j >= L) continue;
                    long long dz[2];
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        uint32_t bits[kLevels5];
#pragma unroll
                        for (int l = 0; l < kLevels5; l++) bits[l] = magic_bits(a[l][2 * p + u]);
                        dz[u] = fold9_bits(bits, eU[j + u]);
                    }
                    longlong2 *zp = (longlong2 *)(zc + j);
                    longlong2 z2 = *zp;
                    z2.x -= dz[0];
                    if (j + 1 < L) z2.y -= dz[1];
                    *zp = z2;
                }
            }
        }
        tc5::fence_before_sync();   // this tile's TMEM reads precede the next tile's TMEM writes
        __syncthreads();
        tc5::fence_after_sync();
        if (sh.abort) break;
        // ---- store the rows final for this group (all rows after the last tile)
        {
            const int jhi = (k == K - 1) ? L : b;
            for (int cc = warp; cc < kCols5; cc += kThreads5 / 32) {
                if (col0 + cc >= nev) continue;
                long long *zg = Zi + (long long)(col0 + cc) * ldz;
                for (int j = lane; j < jhi; j += 32) {
                    const long long r = row0 + j;
                    if (r < n) {
                        const long long v = Zs[cc * ZROW + j];
                        if (tc_out_of_range(v)) tc_set_error(state, GB_ERR_RANGE);
                        zg[r] = v;
                    }
                }
            }
        }
        // every thread's stores happen before thread 0's fence and release
        // (barrier, then a cumulative release at GPU scope); the release of
        // tile k is issued during tile k+1 (after its products are issued),
        // that of the item's last tile right here
        __syncthreads();
        if (tid == 0 && k == K - 1 && g + 1 != hold_group) {
            __threadfence();
            st_release(progress + (long long)g * C + c, k + 1);
        }
    }
    // ---- leave: no copy or MMA of this CTA may still be in flight when its
    // TMEM is released (bounded waits; a timeout was already recorded)
    if (tid == 0) {
        for (int r = issued - 2; r < issued; r++)
            if (r >= 0) tc5::mbar_wait(bar_rec0 + 8 * (r & 1), (uint32_t)((r >> 1) & 1), kMbarTimeoutNs);
    }
    if (mma_pending) tc5::mbar_wait(bar_mma, (mma_phase - 1) & 1, kMbarTimeoutNs);
    tc5::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc5::fence_after_sync();
        tc5::tmem_dealloc(tmem, kTmemCols);
    }
}

template <int B>
size_t tc5_bytes(int n, int nev)
{
    using Gm = Geo<B>;
    const long long G = group_count(n, kNB5);
    const long long C = (nev + kCols5 - 1) / kCols5;
    long long tiles = 0;
    for (long long g = 0; g < G; g++) tiles += group_tiles(n, B, kNB5, (int)g);
    size_t o = 256 + (size_t)(G * C) * 4;                   // head + progress
    o = (o + 255) & ~(size_t)255;
    o += ((size_t)nev * 4 + 255) & ~(size_t)255;            // column scales
    o += ((size_t)(G + 1) * 8 + 255) & ~(size_t)255;        // tile offsets
    o += (size_t)tiles * Gm::REC;                           // tile records
    return o;
}

template <int B>
cudaError_t run_tc5(int n, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                    int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                    int hold_group, cudaStream_t st)
{
    using Gm = Geo<B>;
    const int G = group_count(n, kNB5);
    const int C = (nev + kCols5 - 1) / kCols5;
    if (G <= 0 || nev <= 0) return cudaSuccess;
    if (ws_bytes < tc5_bytes<B>(n, nev)) return cudaErrorInvalidValue;
    char *base = (char *)ws;
    TcState *state = (TcState *)base;
    int *progress = (int *)(base + 256);
    size_t o = (256 + (size_t)G * C * 4 + 255) & ~(size_t)255;
    int *E = (int *)(base + o);
    o += ((size_t)nev * 4 + 255) & ~(size_t)255;
    long long *toff = (long long *)(base + o);
    o += ((size_t)(G + 1) * 8 + 255) & ~(size_t)255;
    unsigned char *rec = (unsigned char *)(base + o);

    cudaError_t e = cudaMemsetAsync(ws, 0, 256, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(progress, 0xff, (size_t)G * C * 4, st)) != cudaSuccess) return e;
    const dim3 conv_grid((n + 255) / 256 < 64 ? (n + 255) / 256 : 64, nev < 65535 ? nev : 65535);
    tc_col_scale<<<(nev + 7) / 8, 256, 0, st>>>(n, nev, Z, ldz, E, state);
    tc_convert<<<conv_grid, 256, 0, st>>>(n, nev, Z, ldz, E, 1);
    tc_tile_offsets<<<1, 1, 0, st>>>(n, B, kNB5, G, toff);
    tc5_tile_prep<B><<<dim3(group_tiles(n, B, kNB5, 0), G), 128, 0, st>>>(n, hh_v, hh_tau, toff, rec);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pipeline_tc5<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM)) !=
        cudaSuccess)
        return e;
    const int want = column_batch > 0 ? column_batch : kColumnBatch5;
    const int CB = C < want ? C : want;
    pipeline_tc5<B><<<(unsigned)G * (unsigned)C, kThreads5, Gm::SMEM, st>>>(
        n, nev, (long long *)Z, ldz, rec, toff, G, C, CB, state, progress, spin_polls, timeout_ns, hold_group);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    tc_convert<<<conv_grid, 256, 0, st>>>(n, nev, Z, ldz, E, 0);
    return cudaGetLastError();
}

}  // namespace

bool pipeline_tc5_supported(int b) { return b == 16 || b == 32 || b == 64; }

size_t pipeline_tc5_workspace_bytes(int n, int b, int nev)
{
    if (n < 2 || nev < 1) return 256;
    if (b == 16) return tc5_bytes<16>(n, nev);
    if (b == 32) return tc5_bytes<32>(n, nev);
    return tc5_bytes<64>(n, nev);
}

cudaError_t pipeline_tc5_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                           int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                           int hold_group, cudaStream_t st)
{
    if (b == 16)
        return run_tc5<16>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                           hold_group, st);
    if (b == 32)
        return run_tc5<32>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                           hold_group, st);
    if (b == 64)
        return run_tc5<64>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                           hold_group, st);
    return cudaErrorInvalidValue;
}

}  // namespace gb
