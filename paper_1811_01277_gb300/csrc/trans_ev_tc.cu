// trans_ev_tridi_to_band on the bf16 tensor cores (tensor-core pipeline).
//
// Same schedule as the pipeline variant (trans_ev_pipeline.cu): work item
// (g, c) = all tiles of sweep group g (NB = 16 sweeps) for column block c
// (64 columns); tickets in batches of column blocks, descending g; tile k of
// group g waits for group g+1 to have published k+1 tiles; bounded waits.
//
// Each tile is applied in compact WY form (the blocked form of Sec. 3.1's
// Householder aggregation): the tile's reflectors, applied last sweep first,
// multiply to H_0 H_1 ... H_{NB-1} = I - V T V^T with V the (b+NB-1) x NB
// parallelogram of reflectors and T upper triangular (forward recurrence
// T(q,q) = tau_q, T(0:q,q) = -tau_q T(0:q,0:q) V(:,0:q)^T v_q).  With
// U = V T precomputed per tile, and V's columns scaled to unit length (U's
// by the inverse factors),
//     Z_win <- Z_win - U (V^T Z_win).
// Both products run on mma.sync bf16 by exact digit slicing (see
// dgemm_sliced.cuh): V^T and U are cut into nine 7-bit digits per entry
// against per-row powers of two, once per tile, by tc_tile_prep.
//
// Z itself is held as 64-bit fixed point per column for the whole call:
// z = Zi 2^(E_c - 62) with ||z_c||_2 < 2^(E_c - 1) (and a margin of at least
// 2^-30 of that bound, see tc_col_scale), so |Zi| < 2^61 and every update
// |dZi| <= 2 ||z|| 2^(62 - E_c) < 2^62.  Householder reflectors
// are orthogonal, so every entry of every intermediate column stays below
// its initial 2-norm: one scale per column serves the whole sweep, digits
// come straight from the integer's bits, each level's tensor-core sum is
// exact (below 2^24 units) and is folded into 64-bit integers, and the
// update Zi -= dZi is an integer subtraction.  No FP64 instruction touches
// the tile updates; Z is converted in place before and after.
#include <cuda_runtime.h>
#include <stdint.h>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "mma_bf16.cuh"
#include "tc_fixed.cuh"
#include "trans_ev_kernels.cuh"

namespace gb {

namespace {

constexpr int kNB = 16;      // sweeps per tile
constexpr int kCols = 64;    // eigenvector columns per work item
constexpr int kThreads = 256;
constexpr int kDigits = 9;   // 63 bits: the fixed-point Z and W are cut exactly
constexpr int kLevels = 10;  // digit pairs i + j <= 9
// column blocks per ticket batch: at n = 16384 on GB300, 8 blocks cost 0.8%
// against 16 and move 102 GB of DRAM traffic per call instead of 340 GB
// (the rows passed from group to group stay in L2)
constexpr int kColumnBatchTc = 8;
constexpr int kFlushBound = kDigits * 127 * 127;  // per k value of one level (at most 9 pairs)

// window rows of a tile, padded to a multiple of 16 (the mma k step)
template <int B>
struct Win {
    static constexpr int L = B + kNB - 1;
    static constexpr int LP = (L + 15) / 16 * 16;
    // window column stride (int64): 4 mod 16, so that the 64-bit updates of
    // a warp (rows g, columns 2t) take the minimum two wavefronts, and even
    // for the 16-byte fragment loads
    static constexpr int ZROW = (LP + 4) / 16 * 16 + 4 + ((LP + 4) % 16 > 4 ? 16 : 0);
    // tile record in global memory, 256-byte multiple: V^T planes [9][16][LP],
    // U planes [9][LP][16] (bf16), exponents eV[16], eU[LP]
    static constexpr size_t VT_BYTES = (size_t)kDigits * kNB * LP * 2;
    static constexpr size_t U_BYTES = (size_t)kDigits * LP * kNB * 2;
    static constexpr size_t E_BYTES = (size_t)(kNB + LP) * 4;
    static constexpr size_t REC = (VT_BYTES + U_BYTES + E_BYTES + 255) / 256 * 256;
    // shared memory of the main kernel: the record (same layout, 16-byte
    // chunks XOR-swizzled), W planes [9][64][16], window [64][ZROW] int64
    static constexpr size_t S_WP = (size_t)kDigits * kCols * kNB * 2;
    static constexpr size_t S_Z = (size_t)kCols * ZROW * 8;
    static constexpr size_t S_EC = (size_t)kCols * 4;
    static constexpr size_t SMEM = REC + S_WP + S_Z + S_EC;
    static_assert(kFlushBound * LP < (1 << 24), "level sums of one tile product must stay exact in FP32");
    static_assert((LP / 8) % 2 == 0, "V^T rows hold an even number of 16-byte chunks");
};

// ---- per-tile V^T and U digit planes ---------------------------------------

template <int B>
__global__ void __launch_bounds__(128) tc_tile_prep(int n, const double *__restrict__ hh_v,
                                                    const double *__restrict__ hh_tau,
                                                    const long long *__restrict__ off,
                                                    unsigned char *__restrict__ rec)
{
    using W = Win<B>;
    constexpr int L = W::L, LP = W::LP;
    const int k = blockIdx.x, g = blockIdx.y;
    const int b = B;
    if (k >= group_tiles(n, b, kNB, g)) return;
    __shared__ double V[LP][kNB + 1];
    __shared__ double U[LP][kNB + 1];
    __shared__ double T[kNB][kNB + 1];
    __shared__ double Gm[kNB][kNB + 1];
    __shared__ double tau[kNB];
    const int s0 = 1 + g * kNB;
    // reflectors of the tile: column q of V is v_q placed at window rows q..q+len-1
    for (int e = threadIdx.x; e < LP * kNB; e += blockDim.x) {
        const int j = e / kNB, q = e % kNB;
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
    if (threadIdx.x < kNB) {
        const int s = s0 + threadIdx.x;
        tau[threadIdx.x] = (s <= n - 1 && s + k * b < n) ? hh_tau[sweep_first(n, b, s) + k] : 0.0;
    }
    __syncthreads();
    // Gram matrix of the reflectors (upper triangle)
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
        const int p = e / kNB, q = e % kNB;
        double a = 0.0;
        if (p < q)
            for (int j = q; j < min(p + b, LP); j++) a = fma(V[j][p], V[j][q], a);
        Gm[p][q] = a;
    }
    __syncthreads();
    // T by the forward recurrence, column by column (rows in parallel)
    for (int q = 0; q < kNB; q++) {
        if (threadIdx.x < kNB) {
            const int i = threadIdx.x;
            double t = 0.0;
            if (i < q) {
                for (int p = i; p < q; p++) t = fma(T[i][p], Gm[p][q], t);
                t = -tau[q] * t;
            } else if (i == q) {
                t = tau[q];
            }
            T[i][q] = t;
        }
        __syncthreads();
    }
    // U = V T
    for (int e = threadIdx.x; e < LP * kNB; e += blockDim.x) {
        const int j = e / kNB, q = e % kNB;
        double a = 0.0;
        for (int p = 0; p <= q; p++) a = fma(V[j][p], T[p][q], a);
        U[j][q] = a;
    }
    // ||v_q||_2, to rescale V D^-1 and U D (U V^T is unchanged): with unit
    // columns |v_q^T z| <= ||z||, so W = V^T Z stays within the column's
    // fixed-point range whatever the reflectors' tau
    __shared__ double nv[kNB];
    if (threadIdx.x < kNB) {
        double a = 0.0;
        for (int j = 0; j < LP; j++) a = fma(V[j][threadIdx.x], V[j][threadIdx.x], a);
        nv[threadIdx.x] = sqrt(a);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LP * kNB; e += blockDim.x) {
        const int j = e / kNB, q = e % kNB;
        if (nv[q] > 0.0) {
            V[j][q] = V[j][q] / nv[q];
            U[j][q] = U[j][q] * nv[q];
        }
    }
    __syncthreads();
    unsigned char *r = rec + ((size_t)off[g] + k) * W::REC;
    uint16_t *vt = (uint16_t *)r;
    uint16_t *up = (uint16_t *)(r + W::VT_BYTES);
    int *eV = (int *)(r + W::VT_BYTES + W::U_BYTES);
    int *eU = eV + kNB;
    // row exponents: rows of V^T (reflectors) and rows of U (window rows)
    __shared__ int seV[kNB], seU[LP];
    if (threadIdx.x < kNB) {
        unsigned long long m = 0;
        for (int j = 0; j < LP; j++) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(V[j][threadIdx.x]) & ~(1ull << 63);
            m = u > m ? u : m;
        }
        seV[threadIdx.x] = exponent_above(m);
        eV[threadIdx.x] = seV[threadIdx.x];
    }
    for (int j = threadIdx.x; j < LP; j += blockDim.x) {
        unsigned long long m = 0;
        for (int q = 0; q < kNB; q++) {
            const unsigned long long u = (unsigned long long)__double_as_longlong(U[j][q]) & ~(1ull << 63);
            m = u > m ? u : m;
        }
        seU[j] = exponent_above(m);
        eU[j] = seU[j];
    }
    __syncthreads();
    // digit planes: vt[s][q][j] (rows q, k = j), up[s][j][q] (rows j, k = q)
    for (int e = threadIdx.x; e < kNB * LP; e += blockDim.x) {
        const int q = e / LP, j = e % LP;
        const double x = V[j][q];
        const unsigned long long Y = fixed63(x, seV[q]);
        const bool neg = x < 0.0;
#pragma unroll
        for (int s = 0; s < kDigits; s++)
            vt[((size_t)s * kNB + q) * LP + j] = bf16_digit((int)((Y >> (56 - 7 * s)) & 127u), s, neg);
    }
    for (int e = threadIdx.x; e < LP * kNB; e += blockDim.x) {
        const int j = e / kNB, q = e % kNB;
        const double x = U[j][q];
        const unsigned long long Y = fixed63(x, seU[j]);
        const bool neg = x < 0.0;
#pragma unroll
        for (int s = 0; s < kDigits; s++)
            up[((size_t)s * LP + j) * kNB + q] = bf16_digit((int)((Y >> (56 - 7 * s)) & 127u), s, neg);
    }
}

// ---- the main kernel ------------------------------------------------------

// Exact bf16 of a digit: with eb = the exponent bits of 2^(23 - 7s),
// float(eb | d) - float(eb) = d 2^(-7s) exactly (Sterbenz), and its upper 16
// bits are the bf16 (d has at most 7 significant bits).
template <int S>
__device__ __forceinline__ float digit_f(unsigned d)
{
    constexpr unsigned eb = (unsigned)(150 - 7 * S) << 23;
    return __uint_as_float(eb | d) - __uint_as_float(eb);
}

// the two bf16 halves of a and b packed into one register (a low, b high),
// with the sign words sa, sb (0 or 0x80000000) applied
__device__ __forceinline__ unsigned pack_bf16(float a, float b, unsigned sa, unsigned sb)
{
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632) ^ ((sa >> 16) | sb);
}

// The 63-bit magnitude of a fixed-point value |x| < 2^61 (bits 60..0, two
// zero bits appended: exact) and its sign word
__device__ __forceinline__ unsigned long long mag63(long long x, unsigned &sign)
{
    sign = x < 0 ? 0x80000000u : 0u;
    const unsigned long long mag = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
    return mag << 2;
}

// digit s (0 = most significant) of a 63-bit magnitude
__device__ __forceinline__ unsigned digit_of(unsigned long long Y, int s)
{
    return (unsigned)(Y >> (56 - 7 * s)) & 127u;
}


// Folds level accumulators (level l in units of 2^(-7l)) into
// hi = sum_{l<4} L_l 2^(7(3-l)) and lo = sum_{l>=4} L_l 2^(7(9-l)), so the sum
// in level-0 units is hi 2^-21 + lo 2^-63.  Large: level sums up to 2^24
// (F2I); otherwise below 2^22 (exact by adding 1.5 2^23 in FP32).
template <bool Large>
__device__ __forceinline__ void fold_levels(const float (&acc)[kLevels][4], long long (&hi)[4], long long (&lo)[4])
{
#pragma unroll
    for (int q = 0; q < 4; q++) {
        hi[q] = 0;
        lo[q] = 0;
    }
#pragma unroll
    for (int l = 0; l < kLevels; l++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float unit = __uint_as_float((unsigned)(127 + 7 * l) << 23);  // 2^(7l)
            int iv;
            if (Large) iv = __float2int_rn(acc[l][q] * unit);
            else iv = (int)(__float_as_uint(fmaf(acc[l][q], unit, 12582912.0f)) - 0x4B400000u);
            // one 32 x 32 + 64 multiply-add per level
            if (l < 4) hi[q] += (long long)iv * (long long)(1 << (7 * (3 - l)));
            else lo[q] += (long long)iv * (1ll << (7 * (9 - l)));
        }
}

// swizzled 16-byte chunk of row r: rows r and r + 4 use different banks
__device__ __forceinline__ int swz(int chunk, int r) { return chunk ^ ((r >> 2) & 1); }

template <int B>
__global__ void __launch_bounds__(kThreads, 2)
pipeline_tc(int n, int nev, long long *__restrict__ Zi, long long ldz, const int *__restrict__ Ecol,
            const unsigned char *__restrict__ rec, const long long *__restrict__ off, int G, int C, int CB,
            TcState *state, int *progress, long long spin_polls, long long timeout_ns, int hold_group)
{
    using W = Win<B>;
    constexpr int L = W::L, LP = W::LP, ZROW = W::ZROW;
    extern __shared__ __align__(16) unsigned char smem[];
    uint16_t *VtP = (uint16_t *)smem;                                  // [9][16][LP]
    uint16_t *UP = (uint16_t *)(smem + W::VT_BYTES);                   // [9][LP][16]
    const int *eV = (const int *)(smem + W::VT_BYTES + W::U_BYTES);   // [16]
    const int *eU = eV + kNB;                                          // [LP]
    uint16_t *WP = (uint16_t *)(smem + W::REC);                        // [9][64][16]
    long long *Zs = (long long *)(smem + W::REC + W::S_WP);            // [64][ZROW]
    int *Es = (int *)(smem + W::REC + W::S_WP + W::S_Z);               // [64]
    __shared__ int s_item, s_abort;

    const int b = B;
    if (threadIdx.x == 0) s_item = atomicAdd(&state->ticket, 1);
    __syncthreads();
    const int item = s_item;
    const int batch = item / (G * CB);
    const int rem = item - batch * G * CB;
    const int cb = min(CB, C - batch * CB);
    const int g = G - 1 - rem / cb;
    const int c = batch * CB + rem % cb;
    const int s0 = 1 + g * kNB;
    const int K = group_tiles(n, b, kNB, g);
    const int Knext = (g + 1 < G) ? group_tiles(n, b, kNB, g + 1) : 0;
    const int col0 = c * kCols;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gq = lane >> 2, tig = lane & 3;
    const int wcol = warp * 8;  // the warp's eight columns of the item

    for (int i = threadIdx.x; i < kCols; i += kThreads) Es[i] = (col0 + i < nev) ? Ecol[col0 + i] : 0;
    if (threadIdx.x == 0 && g + 1 != hold_group) st_release(progress + (long long)g * C + c, 0);

    for (int k = 0; k < K; k++) {
        // ---- dependency wait (group g+1 has finalised the rows this tile reads)
        if (threadIdx.x == 0) {
            int abort = 0;
            const int need = (g + 1 < G) ? min(k + 1, Knext) : 0;
            const int *flag = progress + (long long)(g + 1) * C + c;
            unsigned long long t0 = 0;
            long long polls = 0;
            while (need > 0 && ld_acquire(flag) < need) {
                if (*(volatile int *)&state->abort) { abort = 1; break; }
                if (polls == 0) t0 = now_ns();
                if (++polls >= spin_polls || (long long)(now_ns() - t0) > timeout_ns) {
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
        // ---- stage the tile record (independent of Z); chunks swizzled per row
        {
            const unsigned char *r = rec + ((size_t)off[g] + k) * W::REC;
            constexpr int VT_CH = kDigits * kNB * (LP / 8);
            constexpr int U_CH = kDigits * LP * 2;
            constexpr int E_CH = (int)((W::E_BYTES + 15) / 16);
            for (int ch = threadIdx.x; ch < VT_CH + U_CH + E_CH; ch += kThreads) {
                if (ch < VT_CH) {
                    const int row = ch / (LP / 8), part = ch % (LP / 8);  // row = s * 16 + q
                    cp_async16(VtP + (size_t)row * LP + swz(part, row & 15) * 8, r + ((size_t)row * LP + part * 8) * 2);
                } else if (ch < VT_CH + U_CH) {
                    const int c2 = ch - VT_CH;
                    const int row = c2 >> 1, part = c2 & 1;  // row = s * LP + j
                    cp_async16(UP + (size_t)row * kNB + swz(part, row % LP) * 8,
                               r + W::VT_BYTES + ((size_t)row * kNB + part * 8) * 2);
                } else {
                    const int c3 = ch - VT_CH - U_CH;
                    cp_async16(smem + W::VT_BYTES + W::U_BYTES + c3 * 16, r + W::VT_BYTES + W::U_BYTES + c3 * 16);
                }
            }
            cp_async_commit();
        }
        __syncthreads();
        if (s_abort) {
            cp_async_wait_all();
            return;
        }
        // ---- window: load the new rows (all of a warp's loads in flight at
        // once), carry NB-1 rows meanwhile, then store (rows past n are zero)
        const long long row0 = (long long)s0 + (long long)k * b;
        {
            constexpr int H = (LP + 31) / 32;        // row strides of 32 per column
            constexpr int CW = kCols / (kThreads / 32);  // columns per warp
            const int jlo = (k == 0) ? 0 : kNB - 1;
            long long v[CW][H];
#pragma unroll
            for (int i = 0; i < CW; i++) {
                const int col = col0 + warp + i * (kThreads / 32);
                const long long *zc = Zi + (long long)(col < nev ? col : 0) * ldz;
#pragma unroll
                for (int h = 0; h < H; h++) {
                    const int j = jlo + lane + 32 * h;
                    v[i][h] = (col < nev && j < L && row0 + j < n) ? __ldcg(zc + row0 + j) : 0ll;
                }
            }
            if (k > 0) {
                for (int e = threadIdx.x; e < kCols * (kNB - 1); e += kThreads) {
                    const int cc = e / (kNB - 1), j = e % (kNB - 1);
                    Zs[cc * ZROW + j] = Zs[cc * ZROW + j + b];
                }
                __syncthreads();  // carried rows read before the new rows overwrite them
            }
#pragma unroll
            for (int i = 0; i < CW; i++) {
                const int cc = warp + i * (kThreads / 32);
#pragma unroll
                for (int h = 0; h < H; h++) {
                    const int j = jlo + lane + 32 * h;
                    if (j < LP) Zs[cc * ZROW + j] = v[i][h];
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
        // ---- W = V^T Z_win (16 x 64, k = LP): warp w owns columns 8w..8w+7.
        // The B fragments (rows 2t, 2t+1, 2t+8, 2t+9 of column g) are cut
        // into digits in registers straight from the fixed-point window.
        {
            float acc[kLevels][4];
#pragma unroll
            for (int l = 0; l < kLevels; l++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[l][q] = 0.f;
            const int a_row = (lane & 7) + ((lane >> 3) & 1) * 8;
            const long long *zcol = Zs + (wcol + gq) * ZROW + 2 * tig;
#pragma unroll 1
            for (int ks = 0; ks < LP / 16; ks++) {
                unsigned bf0[kDigits], bf1[kDigits];
                {
                    const longlong2 p0 = *(const longlong2 *)(zcol + ks * 16);
                    const longlong2 p1 = *(const longlong2 *)(zcol + ks * 16 + 8);
                    unsigned sg0, sg1, sg2, sg3;
                    const unsigned long long y0 = mag63(p0.x, sg0), y1 = mag63(p0.y, sg1);
                    const unsigned long long y2 = mag63(p1.x, sg2), y3 = mag63(p1.y, sg3);
#define GB_TC_DIGITS(S)                                                                                 \
    bf0[S] = pack_bf16(digit_f<S>(digit_of(y0, S)), digit_f<S>(digit_of(y1, S)), sg0, sg1);              \
    bf1[S] = pack_bf16(digit_f<S>(digit_of(y2, S)), digit_f<S>(digit_of(y3, S)), sg2, sg3);
                    GB_TC_DIGITS(0) GB_TC_DIGITS(1) GB_TC_DIGITS(2) GB_TC_DIGITS(3)
                    GB_TC_DIGITS(4) GB_TC_DIGITS(5) GB_TC_DIGITS(6) GB_TC_DIGITS(7) GB_TC_DIGITS(8)
#undef GB_TC_DIGITS
                }
                unsigned af[kDigits][4];
#pragma unroll
                for (int s = 0; s < kDigits; s++)
                    ldsm_x4(af[s][0], af[s][1], af[s][2], af[s][3],
                            VtP + ((size_t)s * kNB + a_row) * LP + swz(ks * 2 + (lane >> 4), a_row) * 8);
#pragma unroll
                for (int jd = 0; jd < kDigits; jd++)
#pragma unroll
                    for (int i = 0; i < kDigits; i++)
                        if (i + jd < kLevels) mma_bf16(acc[i + jd], af[i], bf0[jd], bf1[jd]);
            }
            long long hi[4], lo[4];
            fold_levels<true>(acc, hi, lo);
            // W in the column's fixed point (Wi = W 2^(62 - E_c) = S 2^(eV + 47):
            // the digits of Z stand for 2^(E_c - 1) sum d_s 2^(-7(s+1)); |Wi| < 2^61
            // since |v_q^T z| <= ||z||), cut into digits: WP[s][c][q], chunk of
            // q swizzled by c
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int qr = gq + (q >> 1) * 8;          // reflector (row of W)
                const int cc = wcol + tig * 2 + (q & 1);
                const int ev = eV[qr];
                const long long wi = shift_ll(hi[q], ev + 26) + shift_ll(lo[q], ev - 16);
                unsigned sg;
                const unsigned long long y = mag63(wi, sg);
                uint16_t *wp = WP + (size_t)cc * kNB + swz(qr >> 3, cc) * 8 + (qr & 7);
                const unsigned sh = sg >> 16;
#define GB_TC_WDIGIT(S) wp[(size_t)(S) * kCols * kNB] = (uint16_t)((__float_as_uint(digit_f<S>(digit_of(y, S))) >> 16) | sh);
                GB_TC_WDIGIT(0) GB_TC_WDIGIT(1) GB_TC_WDIGIT(2) GB_TC_WDIGIT(3)
                GB_TC_WDIGIT(4) GB_TC_WDIGIT(5) GB_TC_WDIGIT(6) GB_TC_WDIGIT(7) GB_TC_WDIGIT(8)
#undef GB_TC_WDIGIT
            }
        }
        __syncthreads();
        // ---- dZ = U W (LP x 64, k = 16), Zs -= dZ: warp w owns columns 8w..8w+7
        {
            unsigned bw[kDigits][2];
            const int b_row = wcol + (lane & 7);
#pragma unroll
            for (int jd = 0; jd < kDigits; jd++)
                ldsm_x2(bw[jd][0], bw[jd][1], WP + ((size_t)jd * kCols + b_row) * kNB + swz((lane >> 3) & 1, b_row) * 8);
            const int a_row = (lane & 7) + ((lane >> 3) & 1) * 8;
#pragma unroll 1
            for (int mt = 0; mt < LP / 16; mt++) {
                float acc[kLevels][4];
#pragma unroll
                for (int l = 0; l < kLevels; l++)
#pragma unroll
                    for (int q = 0; q < 4; q++) acc[l][q] = 0.f;
                const int j_a = mt * 16 + a_row;
                unsigned au[kDigits][4];
#pragma unroll
                for (int s = 0; s < kDigits; s++)
                    ldsm_x4(au[s][0], au[s][1], au[s][2], au[s][3],
                            UP + ((size_t)s * LP + j_a) * kNB + swz(lane >> 4, j_a) * 8);
#pragma unroll
                for (int jd = 0; jd < kDigits; jd++)
#pragma unroll
                    for (int i = 0; i < kDigits; i++)
                        if (i + jd < kLevels) mma_bf16(acc[i + jd], au[i], bw[jd][0], bw[jd][1]);
                long long hi[4], lo[4];
                fold_levels<false>(acc, hi, lo);
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int j = mt * 16 + gq + (q >> 1) * 8;  // window row
                    const int cc = wcol + tig * 2 + (q & 1);
                    if (j < L) {
                        const int eu = eU[j];
                        Zs[cc * ZROW + j] -= shift_ll(hi[q], eu + 26) + shift_ll(lo[q], eu - 16);
                    }
                }
            }
        }
        __syncthreads();
        // ---- store the rows final for this group (all rows after the last tile)
        {
            const int jhi = (k == K - 1) ? L : b;
            for (int cc = warp; cc < kCols; cc += kThreads / 32) {
                const int col = col0 + cc;
                if (col >= nev) continue;
                long long *zc = Zi + (long long)col * ldz;
                for (int j = lane; j < jhi; j += 32) {
                    const long long r = row0 + j;
                    if (r < n) {
                        const long long v = Zs[cc * ZROW + j];
                        if (tc_out_of_range(v)) tc_set_error(state, GB_ERR_RANGE);
                        zc[r] = v;
                    }
                }
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0 && g + 1 != hold_group) st_release(progress + (long long)g * C + c, k + 1);
    }
}

template <int B>
size_t tc_bytes(int n, int nev)
{
    using W = Win<B>;
    const long long G = group_count(n, kNB);
    const long long C = (nev + kCols - 1) / kCols;
    long long tiles = 0;
    for (long long g = 0; g < G; g++) tiles += group_tiles(n, B, kNB, (int)g);
    size_t off = 256 + (size_t)(G * C) * 4;                 // head + progress
    off = (off + 255) & ~(size_t)255;
    off += ((size_t)nev * 4 + 255) & ~(size_t)255;          // column scales
    off += ((size_t)(G + 1) * 8 + 255) & ~(size_t)255;      // tile offsets
    off += (size_t)tiles * W::REC;                          // tile records
    return off;
}

template <int B>
cudaError_t run_tc(int n, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                   int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                   int hold_group, cudaStream_t st)
{
    using W = Win<B>;
    const int G = group_count(n, kNB);
    const int C = (nev + kCols - 1) / kCols;
    if (G <= 0 || nev <= 0) return cudaSuccess;
    if (ws_bytes < tc_bytes<B>(n, nev)) return cudaErrorInvalidValue;
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
    tc_tile_offsets<<<1, 1, 0, st>>>(n, B, kNB, G, toff);
    tc_tile_prep<B><<<dim3(group_tiles(n, B, kNB, 0), G), 128, 0, st>>>(n, hh_v, hh_tau, toff, rec);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pipeline_tc<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W::SMEM)) !=
        cudaSuccess)
        return e;
    const int want = column_batch > 0 ? column_batch : kColumnBatchTc;
    const int CB = C < want ? C : want;
    if ((e = mark_kernel_begin(st)) != cudaSuccess) return e;
    pipeline_tc<B><<<(unsigned)G * (unsigned)C, kThreads, W::SMEM, st>>>(
        n, nev, (long long *)Z, ldz, E, rec, toff, G, C, CB, state, progress, spin_polls, timeout_ns, hold_group);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = mark_kernel_end(st)) != cudaSuccess) return e;
    tc_convert<<<conv_grid, 256, 0, st>>>(n, nev, Z, ldz, E, 0);
    return cudaGetLastError();
}

}  // namespace

bool pipeline_tc_supported(int b) { return b == 16 || b == 32 || b == 64; }

size_t pipeline_tc_workspace_bytes(int n, int b, int nev)
{
    if (n < 2 || nev < 1) return 256;
    if (b == 16) return tc_bytes<16>(n, nev);
    if (b == 32) return tc_bytes<32>(n, nev);
    return tc_bytes<64>(n, nev);
}

cudaError_t pipeline_tc_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                          int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                          int hold_group, cudaStream_t st)
{
    if (b == 16)
        return run_tc<16>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                          hold_group, st);
    if (b == 32)
        return run_tc<32>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                          hold_group, st);
    if (b == 64)
        return run_tc<64>(n, nev, hh_v, hh_tau, Z, ldz, column_batch, ws, ws_bytes, spin_polls, timeout_ns,
                          hold_group, st);
    return cudaErrorInvalidValue;
}

}  // namespace gb
