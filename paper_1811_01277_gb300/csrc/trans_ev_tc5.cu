// trans_ev_tridi_to_band on the tcgen05 tensor cores (the default for real
// data with nbw in {16, 32, 64}).
//
// Schedule (as in the other pipelines): work item (g, c) = all tiles of
// sweep group g (NB sweeps: 32 for nbw = 64, else 16) for column block c
// (128 columns); items take tickets in batches of column blocks, groups
// descending, so every dependency wait targets an item that is already
// running; tile k of group g waits until group g+1 has published
// min(k+1, K_{g+1}) tiles.  All waits are bounded.
//
// Tile algebra (Sec. 3.1's blocked Householder aggregation): the tile's NB
// reflectors, applied last sweep first, multiply to I - V T V^T, with V the
// (b+NB-1) x NB parallelogram of reflectors and T upper triangular; with
// U = V T (V's columns scaled to unit length, U's by the inverse factors),
//     Z_win <- Z_win - U (V^T Z_win).
// Both products run on the tensor cores, transposed so that the 128
// eigenvector columns are the MMA's M dimension:
//     W^T  (128 x NB)  = Z_win^T (128 x LP) . V   (LP x NB)
//     dZ^T (128 x LP)  = W^T     (128 x NB) . U^T (NB x LP)
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
//    products of magnitude <= 2^14: for the first product K = LP <= 96,
//    below 2^24 (exact); for the second K = NB <= 32, and because the top
//    digits are bounded by 32 (W) and 64 (U), below 2^22 (exact, and
//    convertible by one floating-point addition).  The dropped levels
//    (>= 9) are below 2^-69 of the products' scale.
//  * One MMA per digit plane s of the A operand: its B operand spans the
//    other operand's planes t = 0 .. 8-s along N (the planes follow each
//    other in shared memory at the same 8-row stride), so plane t's product
//    lands in the accumulator of level s+t.  9 MMAs per K step instead of 43.
//  * Levels are folded into 64-bit integers (one rounding per entry) and the
//    update Zi -= dZi is an integer subtraction.
//
// Data movement per tile (b = 64, NB = 32, LP = 96):
//  * the tile record is a V part (V digit planes in the MMA's canonical
//    K-major layout, 48 KB) and a U part (U^T digit planes by 32-row
//    chunks, the row exponents of V and U; 48.5 KB), built once per tile by
//    tc5_tile_prep; each part arrives by cp.async.bulk on its own mbarrier,
//    requested as soon as the previous tile no longer needs the buffer;
//  * the window (LP rows x 128 columns, int64) lives in shared memory; the
//    64 new rows come from global memory through L2, NB-1 rows carry over;
//  * Z's digit planes are cut by the threads straight into TMEM (tcgen05.st)
//    and are the A operand of the first product, W's digit planes the A
//    operand of the second.
// TMEM (512 columns): Z digits of up to ZR K steps [0, 64 ZR) (two rounds
// when all K steps do not fit), W levels [64 ZR, + 9 NB); then W digits
// [0, 64 NB/16) and the dZ levels of a 32-row chunk [64 NB/16, + 9 32).
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

constexpr int kCols5 = 128;       // eigenvector columns per work item (the MMA's M)
constexpr int kThreads5 = 512;    // 16 warps: four per TMEM lane quarter (and per SM sub-partition)
constexpr int kPlanes = 8;        // balanced base-256 digits of a 64-bit value
constexpr int kLevels5 = 9;       // digit-pair levels 0..8
constexpr int kColumnBatch5 = 8;  // 128-column blocks per ticket batch (2 and 4 re-read the records more, 16 gains nothing)
constexpr int kTmemCols = 512;
constexpr unsigned long long kDigitBias = 0x8080808080808080ull;
constexpr long long kMbarTimeoutNs = 2000000000ll;  // an MMA batch or a record copy takes microseconds

// RF = 1: real data.  RF = 2: complex data in its real form (interleaved
// re/im storage of Z read as a real column of 2n rows; every complex entry
// of V and U expanded to a 2 x 2 real block), so the tile is a real tile of
// 2 NB reflector columns over a window of 2 (b + NB - 1) rows.
template <int B, int RF>
struct Geo {
    static constexpr int NB = RF == 2 ? 8 : (B == 64 ? 32 : 16);  // sweeps per tile
    static constexpr int NBC = RF * NB;                 // reflector columns of the real form (W's N)
    static constexpr int ADV = RF * B;                  // window rows advanced per tile
    static constexpr int LC = B + NB - 1;               // window rows of the data (complex rows for RF = 2)
    static constexpr int L = RF * LC;                   // window rows of the real form
    static constexpr int CARRY = L - ADV;               // rows carried from tile to tile
    static constexpr int LP = (L + 15) / 16 * 16;       // padded to the MMA's K step
    static constexpr int KSTEPS = LP / 16;              // K steps of the first product
    static constexpr int KD = NBC / 16;                 // K steps of the second
    // tile record: V part [8 planes][NBC rows q][LP] and U part [chunks of
    // 32 rows][8 planes][rows][NBC] + eV[NBC] + eU[LP], canonical K-major
    static constexpr int VPLANE = NBC * LP * 2;
    static constexpr int VBYTES = kPlanes * VPLANE;
    static constexpr int UBYTES = kPlanes * LP * NBC * 2;
    static constexpr int U_EV = UBYTES;
    static constexpr int U_EU = UBYTES + NBC * 4;
    static constexpr int UPART = (UBYTES + (NBC + LP) * 4 + 127) / 128 * 128;
    static constexpr int REC = VBYTES + UPART;
    static constexpr int SBO_V = 16 * LP;               // bytes between 8-row groups of V (N = q)
    static constexpr int SBO_U = 16 * NBC;              // bytes between 8-row groups of U^T (N = j)
    // window: [128 columns][ZROW] int64, ZROW = 2 mod 4 so that a warp's
    // 16-byte accesses to one row pair of 32 columns are conflict-free
    static constexpr int ZROW = LP + 2;
    // dZ row chunks of up to 32 rows (N = 32 rows x up to 8 U planes <= 256)
    static constexpr int NCH = 32;
    static constexpr int CHUNKS = (LP + NCH - 1) / NCH;
    // TMEM columns
    static constexpr int WLEV = kLevels5 * NBC;                     // W level accumulators
    static constexpr int ZR = (kTmemCols - WLEV) / 64 < KSTEPS ? (kTmemCols - WLEV) / 64 : KSTEPS;
    static constexpr int ROUNDS = (KSTEPS + ZR - 1) / ZR;
    static constexpr int T_ZD = 0;
    static constexpr int T_WACC = 64 * ZR;
    static constexpr int T_WD = 0;
    static constexpr int T_DZ = 64 * KD;
    // shared memory
    static constexpr int S_V = 0;
    static constexpr int S_U = VBYTES;
    static constexpr int S_Z = REC;
    static constexpr int S_BAR = S_Z + kCols5 * ZROW * 8;    // 3 mbarriers + TMEM base
    // at least 116 KB, so that shared memory alone keeps the kernel at one
    // CTA per SM: every CTA allocates all 512 TMEM columns
    static constexpr int SMEM = (S_BAR + 64) > 116 * 1024 ? (S_BAR + 64) : 116 * 1024;
    static_assert(ZR >= 1 && T_WACC + WLEV <= kTmemCols, "Z digits and W levels fit in TMEM");
    static_assert(T_DZ + kLevels5 * NCH <= kTmemCols, "W digits and dZ levels fit in TMEM");
    // level bounds per K with the top digits bounded by 32 (Z, W) and 64
    // (V, U): at most 7 x 2^14 + 32 128 + 128 64 (level 7) or 7 x 2^14 (level 8)
    static_assert(LP * (7 * 128 * 128) < (1 << 24), "W level sums stay exact in FP32");
    static_assert(NBC * (7 * 128 * 128) < (1 << 22), "dZ level sums stay below 2^22");
    static_assert(LP * (32 * 128 + 128 * 128 + 128 * 64) < (1 << 22), "W levels 0..2 stay below 2^22");
    static_assert(LP % 16 == 0 && NBC % 16 == 0 && NB <= B && CARRY <= ADV, "tile shape");
    static_assert(VBYTES % 128 == 0 && REC % 128 == 0 && S_Z % 16 == 0, "record alignment");
    static_assert(SMEM <= 227 * 1024, "shared memory");
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

// fold9 for level sums below 2^22 given as magic bit patterns (the dZ product)
__device__ __forceinline__ long long fold9_bits(const uint32_t (&b)[kLevels5], int e)
{
    const int p0 = pair_from_bits(b[0], b[1]), p1 = pair_from_bits(b[2], b[3]);
    const int p2 = pair_from_bits(b[4], b[5]), p3 = pair_from_bits(b[6], b[7]);
    const int l8 = (int)(b[8] - kMagicBits);
    const long long hi = (long long)p0 * 65536 + p1;
    const long long lo = ((long long)p2 * 65536 + p3) * 256 + l8;
    return (long long)((unsigned long long)shift_ll(hi, 26 + e) + (unsigned long long)shift_ll(lo, e - 14));
}

// round(x 2^(62 - e)) for |x| < 2^e, to nearest with ties to even: the row's
// fixed point (|result| <= 2^62), from the bit pattern with integer
// operations only (x = M 2^p, M the 53-bit significand; subnormals too)
__device__ __forceinline__ long long fixed_row(double x, int e)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((u >> 52) & 0x7ff);
    const unsigned long long M = (u & 0xfffffffffffffull) | (ex ? (1ull << 52) : 0ull);
    const int sh = (ex ? ex : 1) - 1075 + 62 - e;     // x 2^(62-e) = M 2^sh, sh <= 10
    unsigned long long r;
    if (sh >= 0) {
        r = M << sh;
    } else if (sh > -64) {
        const int k = -sh;
        r = M >> k;
        const unsigned long long rem = M & ((1ull << k) - 1), half = 1ull << (k - 1);
        if (rem > half || (rem == half && (r & 1))) r++;
    } else {
        r = 0;
    }
    return (u >> 63) ? -(long long)r : (long long)r;
}

// ---- per-tile records ------------------------------------------------------

template <int B>
constexpr size_t prep_smem_bytes()
{
    using Gm = Geo<B, 1>;
    return (size_t)(2 * Gm::LP * (Gm::NB + 1) + 2 * Gm::NB * (Gm::NB + 1) + 2 * Gm::NB) * 8 +
           (size_t)(Gm::NB + Gm::LP) * 4;
}

template <int B>
constexpr size_t prep_smem_bytes_z()
{
    using Gm = Geo<B, 2>;
    return (size_t)(2 * Gm::LC * (Gm::NB + 1) + 2 * Gm::NB * (Gm::NB + 1) + Gm::NB) * 16 + (size_t)Gm::NB * 8 +
           (size_t)(Gm::NB + Gm::LC) * 4;
}

template <int B>
__global__ void __launch_bounds__(256) tc5_tile_prep(int n, const double *__restrict__ hh_v,
                                                     const double *__restrict__ hh_tau,
                                                     const long long *__restrict__ off,
                                                     unsigned char *__restrict__ rec)
{
    using Gm = Geo<B, 1>;
    constexpr int L = Gm::L, LP = Gm::LP, NB = Gm::NB, NB1 = NB + 1;
    const int k = blockIdx.x, g = blockIdx.y;
    const int b = B;
    if (k >= group_tiles(n, b, NB, g)) return;
    extern __shared__ double psm[];
    double *V = psm;                      // [LP][NB1]
    double *U = V + LP * NB1;             // [LP][NB1]
    double *T = U + LP * NB1;             // [NB][NB1]
    double *Gr = T + NB * NB1;            // [NB][NB1]
    double *tau = Gr + NB * NB1;          // [NB]
    double *nv = tau + NB;                // [NB]
    int *seV = (int *)(nv + NB);          // [NB]
    int *seU = seV + NB;                  // [LP]
    const int s0 = 1 + g * NB;
    // reflector q of the tile occupies window rows q .. q+len-1 of column q
    for (int e = threadIdx.x; e < LP * NB; e += blockDim.x) {
        const int j = e / NB, q = e % NB;
        const int s = s0 + q;
        double val = 0.0;
        if (s <= n - 1 && s + k * b < n && j - q >= 0 && j - q < b && j < L) {
            const long long idx = sweep_first(n, b, s) + k;
            const int len = min(b, n - s - k * b);
            const double t = hh_tau[idx];
            const int i = j - q;
            if (t != 0.0 && i < len) val = (i == 0) ? 1.0 : hh_v[idx * b + i];
        }
        V[j * NB1 + q] = val;
    }
    if (threadIdx.x < NB) {
        const int s = s0 + threadIdx.x;
        tau[threadIdx.x] = (s <= n - 1 && s + k * b < n) ? hh_tau[sweep_first(n, b, s) + k] : 0.0;
    }
    __syncthreads();
    // Gram matrix (upper triangle), T by the forward recurrence
    // T(q,q) = tau_q, T(0:q,q) = -tau_q T(0:q,0:q) V(:,0:q)^T v_q
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int p = e / NB, q = e % NB;
        double a = 0.0;
        if (p < q)
            for (int j = q; j < min(p + b, LP); j++) a = fma(V[j * NB1 + p], V[j * NB1 + q], a);
        Gr[p * NB1 + q] = a;
    }
    __syncthreads();
    for (int q = 0; q < NB; q++) {
        if (threadIdx.x < NB) {
            const int i = threadIdx.x;
            double t = 0.0;
            if (i < q) {
                for (int p = i; p < q; p++) t = fma(T[i * NB1 + p], Gr[p * NB1 + q], t);
                t = -tau[q] * t;
            } else if (i == q) {
                t = tau[q];
            }
            T[i * NB1 + q] = t;
        }
        __syncthreads();
    }
    // U = V T; V(j, p) vanishes outside p <= j < p + b
    for (int e = threadIdx.x; e < LP * NB; e += blockDim.x) {
        const int j = e / NB, q = e % NB;
        double a = 0.0;
        for (int p = max(0, j - b + 1); p <= min(q, j); p++) a = fma(V[j * NB1 + p], T[p * NB1 + q], a);
        U[j * NB1 + q] = a;
    }
    // unit columns of V (U rescaled to keep U V^T): |v_q^T z| <= ||z||, so W
    // stays inside the column's fixed-point range whatever tau is
    if (threadIdx.x < NB) {
        const int q = threadIdx.x;
        double a = 0.0;
        for (int j = q; j < min(q + b, LP); j++) a = fma(V[j * NB1 + q], V[j * NB1 + q], a);
        nv[q] = sqrt(a);
        Gr[q] = a > 0.0 ? 1.0 / nv[q] : 0.0;  // the Gram matrix is no longer needed
    }
    __syncthreads();
    // one division per column, not per entry (the FP64 pipe bounds this kernel)
    for (int e = threadIdx.x; e < LP * NB; e += blockDim.x) {
        const int j = e / NB, q = e % NB;
        if (nv[q] > 0.0) {
            V[j * NB1 + q] = V[j * NB1 + q] * Gr[q];
            U[j * NB1 + q] = U[j * NB1 + q] * nv[q];
        }
    }
    __syncthreads();
    unsigned char *r = rec + ((size_t)off[g] + k) * Gm::REC;
    unsigned char *ru = r + Gm::VBYTES;
    if (threadIdx.x < NB) {
        unsigned long long m = 0;
        for (int j = 0; j < LP; j++) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(V[j * NB1 + threadIdx.x]) & ~(1ull << 63);
            m = u > m ? u : m;
        }
        seV[threadIdx.x] = exponent_above(m);
        ((int *)(ru + Gm::U_EV))[threadIdx.x] = seV[threadIdx.x];
    }
    for (int j = threadIdx.x; j < LP; j += blockDim.x) {
        unsigned long long m = 0;
        for (int q = 0; q < NB; q++) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(U[j * NB1 + q]) & ~(1ull << 63);
            m = u > m ? u : m;
        }
        seU[j] = exponent_above(m);
        ((int *)(ru + Gm::U_EU))[j] = seU[j];
    }
    __syncthreads();
    // digit planes in the canonical K-major layout of the B operands:
    // V (N = q, K = j), plane t: byte t VPLANE + (q/8) SBO_V + (j/8) 128 +
    // (q%8) 16 + (j%8) 2, so the planes follow each other along N at the same
    // 8-row stride (an MMA's B may span planes t0, t0+1, ...);
    // U^T (N = j, K = q), by chunks of 32 rows: chunk c = j/32 at c 32 SBO_U,
    // within it plane t at t (rows of the chunk / 8) SBO_U, then
    // (j%32/8) SBO_U + (q/8) 128 + (j%8) 16 + (q%8) 2 (again the planes of a
    // chunk contiguous along N)
    for (int e = threadIdx.x; e < NB * LP; e += blockDim.x) {
        const int q = e / LP, j = e % LP;
        const unsigned long long y = (unsigned long long)fixed_row(V[j * NB1 + q], seV[q]) + kDigitBias;
        const int o = (q >> 3) * Gm::SBO_V + (j >> 3) * 128 + (q & 7) * 16 + (j & 7) * 2;
#pragma unroll
        for (int t = 0; t < kPlanes; t++)
            *(__half *)(r + t * Gm::VPLANE + o) = __float2half_rn((float)((int)((y >> (56 - 8 * t)) & 0xff) - 128));
    }
    for (int e = threadIdx.x; e < LP * NB; e += blockDim.x) {
        const int j = e / NB, q = e % NB;
        const unsigned long long y = (unsigned long long)fixed_row(U[j * NB1 + q], seU[j]) + kDigitBias;
        const int ch = j / Gm::NCH, rows = min(Gm::NCH, LP - ch * Gm::NCH);
        const int o = ch * Gm::NCH * Gm::SBO_U + ((j % Gm::NCH) >> 3) * Gm::SBO_U + (q >> 3) * 128 + (j & 7) * 16 +
                      (q & 7) * 2;
#pragma unroll
        for (int t = 0; t < kPlanes; t++)
            *(__half *)(ru + t * (rows / 8) * Gm::SBO_U + o) =
                __float2half_rn((float)((int)((y >> (56 - 8 * t)) & 0xff) - 128));
    }
}

// Complex tile record: the complex V, T, U of the tile (the same forward
// recurrence with V^H), then their real forms: V's entry v at (row j,
// column q) becomes the 2 x 2 block [[re v, -im v], [im v, re v]] of
// V' (rows 2j+p, columns 2q+p'), so that (z^T V')_(2q+p') are the real and
// imaginary parts of (z^T conj(V))_q; U's entry u becomes, in the B operand
// of the second product (rows 2q+p', columns 2j+p), [[re u, im u],
// [-im u, re u]], so that (w'^T B)_(2j+p) are the parts of (w^T U^T)_j.
// Row exponents are shared by the two real rows of a complex row.
__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// conj(a) b + c
__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}

template <int B>
__global__ void __launch_bounds__(256) tc5_tile_prep_z(int n, const double2 *__restrict__ hh_v,
                                                       const double2 *__restrict__ hh_tau,
                                                       const long long *__restrict__ off,
                                                       unsigned char *__restrict__ rec)
{
    using Gm = Geo<B, 2>;
    constexpr int LC = Gm::LC, LP = Gm::LP, NB = Gm::NB, NB1 = NB + 1, NBC = Gm::NBC;
    const int k = blockIdx.x, g = blockIdx.y;
    const int b = B;
    if (k >= group_tiles(n, b, NB, g)) return;
    extern __shared__ double2 zsm[];
    double2 *V = zsm;                     // [LC][NB1]
    double2 *U = V + LC * NB1;            // [LC][NB1]
    double2 *T = U + LC * NB1;            // [NB][NB1]
    double2 *Gr = T + NB * NB1;           // [NB][NB1]
    double2 *tau = Gr + NB * NB1;         // [NB]
    double *nv = (double *)(tau + NB);    // [NB]
    int *seV = (int *)(nv + NB);          // [NB]
    int *seU = seV + NB;                  // [LC]
    const int s0 = 1 + g * NB;
    const double2 zero = make_double2(0.0, 0.0);
    for (int e = threadIdx.x; e < LC * NB; e += blockDim.x) {
        const int j = e / NB, q = e % NB;
        const int s = s0 + q;
        double2 val = zero;
        if (s <= n - 1 && s + k * b < n && j - q >= 0 && j - q < b) {
            const long long idx = sweep_first(n, b, s) + k;
            const int len = min(b, n - s - k * b);
            const double2 t = hh_tau[idx];
            const int i = j - q;
            if ((t.x != 0.0 || t.y != 0.0) && i < len) val = (i == 0) ? make_double2(1.0, 0.0) : hh_v[idx * b + i];
        }
        V[j * NB1 + q] = val;
    }
    if (threadIdx.x < NB) {
        const int s = s0 + threadIdx.x;
        tau[threadIdx.x] = (s <= n - 1 && s + k * b < n) ? hh_tau[sweep_first(n, b, s) + k] : zero;
    }
    __syncthreads();
    // Gram matrix v_p^H v_q (p < q), T by T(q,q) = tau_q,
    // T(0:q,q) = -tau_q T(0:q,0:q) V(:,0:q)^H v_q
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int p = e / NB, q = e % NB;
        double2 a = zero;
        if (p < q)
            for (int j = q; j < min(p + b, LC); j++) a = cfma_conj(V[j * NB1 + p], V[j * NB1 + q], a);
        Gr[p * NB1 + q] = a;
    }
    __syncthreads();
    for (int q = 0; q < NB; q++) {
        if (threadIdx.x < NB) {
            const int i = threadIdx.x;
            double2 t = zero;
            if (i < q) {
                for (int p = i; p < q; p++) t = cfma(T[i * NB1 + p], Gr[p * NB1 + q], t);
                t = cmul(make_double2(-tau[q].x, -tau[q].y), t);
            } else if (i == q) {
                t = tau[q];
            }
            T[i * NB1 + q] = t;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < LC * NB; e += blockDim.x) {
        const int j = e / NB, q = e % NB;
        double2 a = zero;
        for (int p = max(0, j - b + 1); p <= min(q, j); p++) a = cfma(V[j * NB1 + p], T[p * NB1 + q], a);
        U[j * NB1 + q] = a;
    }
    if (threadIdx.x < NB) {
        const int q = threadIdx.x;
        double a = 0.0;
        for (int j = q; j < min(q + b, LC); j++) {
            const double2 v = V[j * NB1 + q];
            a = fma(v.x, v.x, fma(v.y, v.y, a));
        }
        nv[q] = sqrt(a);
        ((double *)Gr)[q] = a > 0.0 ? 1.0 / nv[q] : 0.0;  // the Gram matrix is no longer needed
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LC * NB; e += blockDim.x) {
        const int j = e / NB, q = e % NB;
        if (nv[q] > 0.0) {
            const double2 v = V[j * NB1 + q], u = U[j * NB1 + q];
            const double rn = ((const double *)Gr)[q];
            V[j * NB1 + q] = make_double2(v.x * rn, v.y * rn);
            U[j * NB1 + q] = make_double2(u.x * nv[q], u.y * nv[q]);
        }
    }
    __syncthreads();
    unsigned char *r = rec + ((size_t)off[g] + k) * Gm::REC;
    unsigned char *ru = r + Gm::VBYTES;
    auto absbits = [](double x) { return (unsigned long long)__double_as_longlong(x) & ~(1ull << 63); };
    if (threadIdx.x < NB) {
        unsigned long long m = 0;
        for (int j = 0; j < LC; j++) {
            const double2 v = V[j * NB1 + threadIdx.x];
            m = max(m, max(absbits(v.x), absbits(v.y)));
        }
        seV[threadIdx.x] = exponent_above(m);
        ((int *)(ru + Gm::U_EV))[2 * threadIdx.x] = seV[threadIdx.x];
        ((int *)(ru + Gm::U_EV))[2 * threadIdx.x + 1] = seV[threadIdx.x];
    }
    for (int j = threadIdx.x; j < LP / 2; j += blockDim.x) {
        unsigned long long m = 0;
        if (j < LC)
            for (int q = 0; q < NB; q++) {
                const double2 u = U[j * NB1 + q];
                m = max(m, max(absbits(u.x), absbits(u.y)));
            }
        const int ev = exponent_above(m);
        if (j < LC) seU[j] = ev;
        ((int *)(ru + Gm::U_EU))[2 * j] = ev;
        ((int *)(ru + Gm::U_EU))[2 * j + 1] = ev;
    }
    __syncthreads();
    // V' (N = q' = 2q+p', K = j' = 2j+p) and the second product's B
    // (N = j', K = q'), in the layouts of the real record
    for (int e = threadIdx.x; e < NBC * LP; e += blockDim.x) {
        const int qq = e / LP, jj = e % LP;
        const int q = qq >> 1, pq = qq & 1, j = jj >> 1, pj = jj & 1;
        double x = 0.0;
        if (j < LC) {
            const double2 v = V[j * NB1 + q];
            x = (pj == pq) ? v.x : (pj ? v.y : -v.y);
        }
        const unsigned long long y = (unsigned long long)fixed_row(x, seV[q]) + kDigitBias;
        const int o = (qq >> 3) * Gm::SBO_V + (jj >> 3) * 128 + (qq & 7) * 16 + (jj & 7) * 2;
#pragma unroll
        for (int t = 0; t < kPlanes; t++)
            *(__half *)(r + t * Gm::VPLANE + o) = __float2half_rn((float)((int)((y >> (56 - 8 * t)) & 0xff) - 128));
    }
    for (int e = threadIdx.x; e < LP * NBC; e += blockDim.x) {
        const int jj = e / NBC, qq = e % NBC;
        const int q = qq >> 1, pq = qq & 1, j = jj >> 1, pj = jj & 1;
        double x = 0.0;
        int ev = 0;
        if (j < LC) {
            const double2 u = U[j * NB1 + q];
            x = (pj == pq) ? u.x : (pq ? -u.y : u.y);
            ev = seU[j];
        }
        const unsigned long long y = (unsigned long long)fixed_row(x, ev) + kDigitBias;
        const int ch = jj / Gm::NCH, rows = min(Gm::NCH, LP - ch * Gm::NCH);
        const int o = ch * Gm::NCH * Gm::SBO_U + ((jj % Gm::NCH) >> 3) * Gm::SBO_U + (qq >> 3) * 128 + (jj & 7) * 16 +
                      (qq & 7) * 2;
#pragma unroll
        for (int t = 0; t < kPlanes; t++)
            *(__half *)(ru + t * (rows / 8) * Gm::SBO_U + o) =
                __float2half_rn((float)((int)((y >> (56 - 8 * t)) & 0xff) - 128));
    }
}

// ---- the main kernel ------------------------------------------------------

struct Tc5Shared {
    int item;
    int abort;
    int u_issued;   // U parts requested so far (written by the thread that requests them)
};

// every thread: wait for an mbarrier phase; on giving up record the timeout
__device__ __forceinline__ bool tc5_wait(uint32_t bar, uint32_t parity, TcState *state, Tc5Shared &sh)
{
    if (tc5::mbar_wait(bar, parity, kMbarTimeoutNs)) return true;
    tc_set_error(state, GB_ERR_TIMEOUT);
    atomicExch(&state->abort, 1);
    sh.abort = 1;
    return false;
}

// n: the data's order (complex rows for RF = 2); Zi, ldz: the real form
// (ldz in 64-bit words, RF times the data's leading dimension)
template <int B, int RF>
__global__ void __launch_bounds__(kThreads5, 1)
pipeline_tc5(int n, int nev, long long *__restrict__ Zi, long long ldz, const unsigned char *__restrict__ rec,
             const long long *__restrict__ off, int G, int C, int CB, TcState *state, int *progress,
             long long spin_polls, long long timeout_ns, int hold_group)
{
    using Gm = Geo<B, RF>;
    constexpr int L = Gm::L, LP = Gm::LP, ZROW = Gm::ZROW, KSTEPS = Gm::KSTEPS, NB = Gm::NB, NBC = Gm::NBC;
    constexpr int ZR = Gm::ZR, KD = Gm::KD, ADV = Gm::ADV, CARRY = Gm::CARRY;
    const long long nrows = (long long)RF * n;             // rows of the real form
    extern __shared__ __align__(1024) unsigned char smem[];
    long long *Zs = (long long *)(smem + Gm::S_Z);
    const uint32_t bar_v = tc5::smem_addr(smem + Gm::S_BAR);
    const uint32_t bar_u = bar_v + 8;
    const uint32_t bar_mma = bar_v + 16;
    uint32_t *tmem_slot = (uint32_t *)(smem + Gm::S_BAR + 32);
    const int *eV = (const int *)(smem + Gm::S_U + Gm::U_EV);
    const int *eU = (const int *)(smem + Gm::S_U + Gm::U_EU);
    __shared__ Tc5Shared sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, wq = warp >> 2;            // lane quarter, and which of its four warps
    const int col = quarter * 32 + lane;                    // this thread's column of the item (its TMEM lane)
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int b = B;

    if (tid == 0) {
        sh.item = atomicAdd(&state->ticket, 1);
        sh.abort = 0;
        sh.u_issued = 1;
        tc5::mbar_init(bar_v, 1);
        tc5::mbar_init(bar_u, 1);
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
    const int s0 = 1 + g * NB;
    const int K = group_tiles(n, b, NB, g);
    const int Knext = (g + 1 < G) ? group_tiles(n, b, NB, g + 1) : 0;
    const int col0 = c * kCols5;
    const unsigned char *rec_g = rec + (size_t)off[g] * Gm::REC;

    uint32_t mma_phase = 0;
    bool mma_pending = false;
    int v_issued = 0;   // V parts requested so far (thread 0)

    if (tid == 0) {
        if (g + 1 != hold_group) st_release(progress + (long long)g * C + c, 0);
        tc5::bulk_load(tc5::smem_addr(smem + Gm::S_V), rec_g, Gm::VBYTES, bar_v);
        tc5::bulk_load(tc5::smem_addr(smem + Gm::S_U), rec_g + Gm::VBYTES, Gm::UPART, bar_u);
        v_issued = 1;
    }
    // window padding rows stay zero for the whole item
    for (int e = tid; e < kCols5 * (LP - L); e += kThreads5) Zs[(e / (LP - L)) * ZROW + L + e % (LP - L)] = 0;

    for (int k = 0; k < K; k++) {
        // ---- dependency wait
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
        }
        __syncthreads();
        if (sh.abort) break;
        // ---- window: new rows from global memory (through L2: rows written
        // by other SMs), the NB-1 rows shared with the previous tile carried
        const long long row0 = (long long)RF * ((long long)s0 + (long long)k * b);
        const int jlo = (k == 0) ? 0 : CARRY;
        {
            constexpr int H = (L + 31) / 32;               // passes of 32 rows per column
            constexpr int CW = kCols5 / (kThreads5 / 32);  // columns per warp
            long long v[CW][H];
#pragma unroll
            for (int i = 0; i < CW; i++) {
                const int cc = warp * CW + i;
                const long long *zc = Zi + (long long)(col0 + cc < nev ? col0 + cc : 0) * ldz;
#pragma unroll
                for (int h = 0; h < H; h++) {
                    const int j = jlo + lane + 32 * h;
                    v[i][h] = (col0 + cc < nev && j < L && row0 + j < nrows) ? __ldcg(zc + row0 + j) : 0ll;
                }
            }
            if (k > 0) {
                for (int e = tid; e < kCols5 * CARRY; e += kThreads5) {
                    const int cc = e / CARRY, j = e % CARRY;
                    Zs[cc * ZROW + j] = Zs[cc * ZROW + j + ADV];
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
        // ---- W^T = Z^T V, in rounds of ZR K steps (Z digit planes cut into
        // TMEM, K step kk of the round at columns (kk - r ZR) 64 + s 8 + pair;
        // units of 8 rows go round-robin to the four warps of a lane quarter)
        const long long *zc = Zs + col * ZROW;
#pragma unroll 1
        for (int r = 0; r < Gm::ROUNDS; r++) {
            const int kk0 = r * ZR, kk1 = (kk0 + ZR < KSTEPS) ? kk0 + ZR : KSTEPS;
            if (r > 0) {   // the previous round's MMAs read the Z-digit columns
                mma_pending = true;
                if (tc5_wait(bar_mma, mma_phase & 1, state, sh)) mma_pending = false;
                mma_phase++;
                tc5::fence_after_sync();
            }
            for (int u = 2 * kk0 + wq; u < 2 * kk1; u += 4) {
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
                    tc5::st_x4(tmem + lane_off + Gm::T_ZD + ((u >> 1) - kk0) * 64 + s * 8 + (u & 1) * 4, w[s]);
            }
            tc5::wait_st();
            if (r == 0) tc5_wait(bar_v, (uint32_t)(k & 1), state, sh);   // this tile's V planes
            tc5::fence_before_sync();
            __syncthreads();
            if (sh.abort) break;
            if (tid == 0) {
                // one MMA per Z digit plane s and K step: B spans V planes
                // 0 .. 8-s along N, so plane t lands in level s+t (D columns
                // T_WACC + NB (s+t)); in the first K step level 8 is first
                // written by its own MMA (s = 1, t = 7), every other level by s = 0
                tc5::fence_after_sync();
                const uint64_t vdesc = tc5::smem_desc(tc5::smem_addr(smem + Gm::S_V), 128, Gm::SBO_V);
                for (int kk = kk0; kk < kk1; kk++)
#pragma unroll
                    for (int s = 0; s < kPlanes; s++) {
                        const uint32_t a_t = tmem + Gm::T_ZD + (kk - kk0) * 64 + s * 8;
                        const uint64_t b0 = vdesc + (uint64_t)((kk * 256) >> 4);
                        const int nt = s == 0 ? kPlanes : kLevels5 - s;          // planes t = 0 .. nt-1
                        if (kk == 0 && s == 1) {
                            tc5::mma_tmem_a(tmem + Gm::T_WACC + NBC * 8, a_t, b0 + (uint64_t)((7 * Gm::VPLANE) >> 4),
                                            tc5::idesc_f16_f32(128, NBC), 0u);
                            tc5::mma_tmem_a(tmem + Gm::T_WACC + NBC, a_t, b0, tc5::idesc_f16_f32(128, NBC * 7), 1u);
                        } else {
                            tc5::mma_tmem_a(tmem + Gm::T_WACC + NBC * s, a_t, b0, tc5::idesc_f16_f32(128, NBC * nt),
                                            (kk > 0 || s > 0) ? 1u : 0u);
                        }
                    }
                tc5::commit(bar_mma);
                // publish the previous tile while the products run: its stores
                // happened before the barriers since, and the fence and release
                // here make them visible at GPU scope before the flag
                if (r == 0 && k > 0 && g + 1 != hold_group) {
                    __threadfence();
                    st_release(progress + (long long)g * C + c, k);
                }
            }
        }
        if (sh.abort) break;
        mma_pending = true;
        if (tc5_wait(bar_mma, mma_phase & 1, state, sh)) mma_pending = false;
        mma_phase++;
        tc5::fence_after_sync();
        // the V buffer is free: request the next tile's V planes
        if (tid == 0 && k + 1 < K) {
            tc5::bulk_load(tc5::smem_addr(smem + Gm::S_V), rec_g + (size_t)(k + 1) * Gm::REC, Gm::VBYTES, bar_v);
            v_issued = k + 2;
        }
        // ---- fold W's levels (reflectors q0 .. q0+NB/4-1 of this column), cut
        // W into digit planes (TMEM: K step q/16, columns s*8 + (q%16)/2)
        tc5_wait(bar_u, (uint32_t)(k & 1), state, sh);   // this tile's U part (row exponents)
        {
            constexpr int QW = NBC / 4;
            const int q0 = wq * QW;
            uint32_t a[kLevels5][QW];
#pragma unroll
            for (int l = 0; l < kLevels5; l++) {
                if constexpr (QW == 8) {
                    tc5::ld_x8(tmem + lane_off + Gm::T_WACC + NBC * l + q0, a[l]);
                } else {
                    tc5::ld_x4(tmem + lane_off + Gm::T_WACC + NBC * l + q0, a[l]);
                }
            }
            tc5::wait_ld();
            uint32_t wd[kPlanes][QW / 2];
#pragma unroll
            for (int p = 0; p < QW / 2; p++) {
                long long wi[2];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const int i = 2 * p + u;
                    int Lv[kLevels5];
                    // levels 0..2 stay below 2^22 (at most 3 pairs, the top
                    // digits bounded by 32 and 64): one addition converts them
#pragma unroll
                    for (int l = 0; l < 3; l++) Lv[l] = (int)(magic_bits(a[l][i]) - kMagicBits);
#pragma unroll
                    for (int l = 3; l < kLevels5; l++) Lv[l] = __float2int_rn(__uint_as_float(a[l][i]));
                    wi[u] = fold9(Lv, eV[q0 + i]);
                }
                uint32_t d[kPlanes];
                cut_pair(wi[0], wi[1], d);
#pragma unroll
                for (int s = 0; s < kPlanes; s++) wd[s][p] = d[s];
            }
            // (the W digits go to the Z-digit columns, dead since the W
            // products completed; the W levels stay untouched until the dZ
            // products, issued after the barrier below)
            const uint32_t wcol = Gm::T_WD + (q0 >> 4) * 64 + (q0 & 15) / 2;
#pragma unroll
            for (int s = 0; s < kPlanes; s++) {
                if constexpr (QW == 8) {
                    tc5::st_x4(tmem + lane_off + wcol + s * 8, wd[s]);
                } else {
                    tc5::st_x2(tmem + lane_off + wcol + s * 8, wd[s]);
                }
            }
            tc5::wait_st();
        }
        tc5::fence_before_sync();
        __syncthreads();
        if (sh.abort) break;
        // ---- dZ^T = W^T U^T by row chunks (M 128, N = rows x planes, K NB),
        // folded into the window: Zs -= dZ
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
                // per W digit plane s and K step one MMA whose B spans the
                // chunk's U planes 0 .. 8-s along N (level l = s+t at D
                // columns T_DZ + l N); level 8 first written alone (s = 1, t = 7)
                tc5::fence_after_sync();
                const uint64_t udesc =
                    tc5::smem_desc(tc5::smem_addr(smem + Gm::S_U) + (uint32_t)j0 * Gm::SBO_U, 128, Gm::SBO_U);
                const uint32_t pstride = (uint32_t)(N / 8) * Gm::SBO_U;   // bytes between the chunk's planes
#pragma unroll
                for (int kd = 0; kd < KD; kd++)
#pragma unroll
                    for (int s = 0; s < kPlanes; s++) {
                        const uint32_t a_t = tmem + Gm::T_WD + kd * 64 + s * 8;
                        const uint64_t b0 = udesc + (uint64_t)((kd * 256) >> 4);
                        const int nt = s == 0 ? kPlanes : kLevels5 - s;
                        if (kd == 0 && s == 1) {
                            tc5::mma_tmem_a(tmem + Gm::T_DZ + 8 * N, a_t, b0 + (uint64_t)((7 * pstride) >> 4),
                                            tc5::idesc_f16_f32(128, N), 0u);
                            tc5::mma_tmem_a(tmem + Gm::T_DZ + N, a_t, b0, tc5::idesc_f16_f32(128, 7 * N), 1u);
                        } else {
                            tc5::mma_tmem_a(tmem + Gm::T_DZ + s * N, a_t, b0, tc5::idesc_f16_f32(128, nt * N),
                                            (kd > 0 || s > 0) ? 1u : 0u);
                        }
                    }
                tc5::commit(bar_mma);
            }
            mma_pending = true;
            if (tc5_wait(bar_mma, mma_phase & 1, state, sh)) mma_pending = false;
            mma_phase++;
            tc5::fence_after_sync();
            // this thread: rows j0 + wq*N/4 .. +N/4 of its column (8 or 4),
            // all levels fetched in one round of TMEM loads
            long long *zw = Zs + col * ZROW;
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
            for (int p = 0; p < 4; p++) {
                if (2 * p >= N / 4) break;
                const int j = j0 + jb + 2 * p;
                if (j >= L) continue;
                long long dz[2];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    uint32_t bits[kLevels5];
#pragma unroll
                    for (int l = 0; l < kLevels5; l++) bits[l] = magic_bits(a8[l][2 * p + u]);
                    dz[u] = fold9_bits(bits, eU[j + u]);
                }
                longlong2 *zp = (longlong2 *)(zw + j);
                longlong2 z2 = *zp;
                z2.x -= dz[0];
                if (j + 1 < L) z2.y -= dz[1];
                *zp = z2;
            }
        }
        tc5::fence_before_sync();   // this tile's TMEM reads precede the next tile's TMEM writes
        __syncthreads();
        tc5::fence_after_sync();
        if (sh.abort) break;
        // the U part is consumed (planes by the MMAs, exponents by the folds
        // above): request the next tile's (a thread other than the one that
        // polls the dependency flags and issues the MMAs)
        if (tid == 32 && k + 1 < K) {
            tc5::fence_proxy_async_smem();
            tc5::bulk_load(tc5::smem_addr(smem + Gm::S_U), rec_g + (size_t)(k + 1) * Gm::REC + Gm::VBYTES, Gm::UPART,
                           bar_u);
            sh.u_issued = k + 2;
        }
        // ---- store the rows final for this group (all rows after the last
        // tile): all of a warp's shared-memory reads first, then the stores
        {
            constexpr int CW = kCols5 / (kThreads5 / 32);
            constexpr int H = (L + 31) / 32;
            const int jhi = (k == K - 1) ? L : ADV;
            long long v[CW][H];
#pragma unroll
            for (int i = 0; i < CW; i++)
#pragma unroll
                for (int h = 0; h < H; h++) {
                    const int j = lane + 32 * h;
                    v[i][h] = (j < jhi) ? Zs[(warp * CW + i) * ZROW + j] : 0ll;
                }
            bool bad = false;
#pragma unroll
            for (int i = 0; i < CW; i++) {
                const int cc = warp * CW + i;
                if (col0 + cc >= nev) continue;
                long long *zg = Zi + (long long)(col0 + cc) * ldz;
#pragma unroll
                for (int h = 0; h < H; h++) {
                    const int j = lane + 32 * h;
                    if (j < jhi && row0 + j < nrows) {
                        bad |= tc_out_of_range(v[i][h]);
                        zg[row0 + j] = v[i][h];
                    }
                }
            }
            if (bad) tc_set_error(state, GB_ERR_RANGE);
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
    __syncthreads();
    if (tid == 0) {
        if (v_issued > 0) tc5::mbar_wait(bar_v, (uint32_t)((v_issued - 1) & 1), kMbarTimeoutNs);
        if (sh.u_issued > 0) tc5::mbar_wait(bar_u, (uint32_t)((sh.u_issued - 1) & 1), kMbarTimeoutNs);
    }
    if (mma_pending) tc5::mbar_wait(bar_mma, (mma_phase - 1) & 1, kMbarTimeoutNs);
    tc5::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc5::fence_after_sync();
        tc5::tmem_dealloc(tmem, kTmemCols);
    }
}

template <int B, int RF>
size_t tc5_bytes(int n, int nev)
{
    using Gm = Geo<B, RF>;
    const long long G = group_count(n, Gm::NB);
    const long long C = (nev + kCols5 - 1) / kCols5;
    long long tiles = 0;
    for (long long g = 0; g < G; g++) tiles += group_tiles(n, B, Gm::NB, (int)g);
    size_t o = 256 + (size_t)(G * C) * 4;                   // head + progress
    o = (o + 255) & ~(size_t)255;
    o += ((size_t)nev * 4 + 255) & ~(size_t)255;            // column scales
    o += ((size_t)(G + 1) * 8 + 255) & ~(size_t)255;        // tile offsets
    o += (size_t)tiles * Gm::REC;                           // tile records
    return o;
}

// Z, ldz: the data (complex entries interleaved for RF = 2, ldz in entries)
template <int B, int RF>
cudaError_t run_tc5(int n, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                    int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                    int hold_group, cudaStream_t st)
{
    using Gm = Geo<B, RF>;
    const int G = group_count(n, Gm::NB);
    const int C = (nev + kCols5 - 1) / kCols5;
    if (G <= 0 || nev <= 0) return cudaSuccess;
    if (ws_bytes < tc5_bytes<B, RF>(n, nev)) return cudaErrorInvalidValue;
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
    // the per-column fixed point works on the real form: 2n rows of a complex column
    const int nr = RF * n;
    const long long ldr = RF * ldz;
    const dim3 conv_grid((nr + 255) / 256 < 64 ? (nr + 255) / 256 : 64, nev < 65535 ? nev : 65535);
    tc_col_scale<<<(nev + 7) / 8, 256, 0, st>>>(nr, nev, Z, ldr, E, state);
    tc_convert<<<conv_grid, 256, 0, st>>>(nr, nev, Z, ldr, E, 1);
    tc_tile_offsets<<<1, 1, 0, st>>>(n, B, Gm::NB, G, toff);
    const dim3 prep_grid(group_tiles(n, B, Gm::NB, 0), G);
    if constexpr (RF == 1) {
        constexpr size_t prep_smem = prep_smem_bytes<B>();
        if ((e = cudaFuncSetAttribute(tc5_tile_prep<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)prep_smem)) !=
            cudaSuccess)
            return e;
        tc5_tile_prep<B><<<prep_grid, 256, prep_smem, st>>>(n, hh_v, hh_tau, toff, rec);
    } else {
        constexpr size_t prep_smem = prep_smem_bytes_z<B>();
        if ((e = cudaFuncSetAttribute(tc5_tile_prep_z<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)prep_smem)) != cudaSuccess)
            return e;
        tc5_tile_prep_z<B><<<prep_grid, 256, prep_smem, st>>>(n, (const double2 *)hh_v, (const double2 *)hh_tau, toff,
                                                              rec);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pipeline_tc5<B, RF>, cudaFuncAttributeMaxDynamicSharedMemorySize, Gm::SMEM)) !=
        cudaSuccess)
        return e;
    const int want = column_batch > 0 ? column_batch : kColumnBatch5;
    const int CB = C < want ? C : want;
    if ((e = mark_kernel_begin(st)) != cudaSuccess) return e;
    pipeline_tc5<B, RF><<<(unsigned)G * (unsigned)C, kThreads5, Gm::SMEM, st>>>(
        n, nev, (long long *)Z, ldr, rec, toff, G, C, CB, state, progress, spin_polls, timeout_ns, hold_group);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = mark_kernel_end(st)) != cudaSuccess) return e;
    tc_convert<<<conv_grid, 256, 0, st>>>(nr, nev, Z, ldr, E, 0);
    return cudaGetLastError();
}

}  // namespace

bool pipeline_tc5_supported(int b) { return b == 16 || b == 32 || b == 64; }

int pipeline_tc5_sweeps_per_tile(int b, int is_complex)
{
    if (is_complex) return Geo<64, 2>::NB;
    return b == 64 ? Geo<64, 1>::NB : Geo<16, 1>::NB;
}

size_t pipeline_tc5_workspace_bytes(int n, int b, int nev, int is_complex)
{
    if (n < 2 || nev < 1) return 256;
    if (is_complex) {
        if (b == 16) return tc5_bytes<16, 2>(n, nev);
        if (b == 32) return tc5_bytes<32, 2>(n, nev);
        return tc5_bytes<64, 2>(n, nev);
    }
    if (b == 16) return tc5_bytes<16, 1>(n, nev);
    if (b == 32) return tc5_bytes<32, 1>(n, nev);
    return tc5_bytes<64, 1>(n, nev);
}

cudaError_t pipeline_tc5_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                           int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                           int hold_group, cudaStream_t st)
{
    if (b == 16)
        return run_tc5<16, 1>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                              hold_group, st);
    if (b == 32)
        return run_tc5<32, 1>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                              hold_group, st);
    if (b == 64)
        return run_tc5<64, 1>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                              hold_group, st);
    return cudaErrorInvalidValue;
}

cudaError_t pipeline_tc5_z(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                           int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                           int hold_group, cudaStream_t st)
{
    if (b == 16)
        return run_tc5<16, 2>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                              hold_group, st);
    if (b == 32)
        return run_tc5<32, 2>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                              hold_group, st);
    if (b == 64)
        return run_tc5<64, 2>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                              hold_group, st);
    return cudaErrorInvalidValue;
}

}  // namespace gb
