// FP64 products on the bf16 tensor cores by exact digit slicing; the scheme
// and its accuracy are described in dgemm_sliced.cuh.
//
// Slicing: two passes over 32 x 32 tiles of the slice-row view, staged in
// shared memory so that global reads follow the source's contiguous index;
// pass 1 takes each row's largest magnitude (atomicMax on the bit pattern),
// pass 2 cuts every entry into digits with integer arithmetic on its bit
// pattern (no FP64 instructions) and writes the bf16 planes, k fastest.
//
// Product: one 256-thread block per 64 x 32 tile of C, warps 4 (rows) x 2
// (columns), each warp 16 x 16 = two m16n8 accumulator tiles per level.
// K advances 32 at a time through a two-stage cp.async pipeline holding the
// D digit planes of the A and B tiles that the product forms (rows padded to
// 80 bytes so that the ldmatrix row addresses of a phase fall in distinct
// banks).  Per k16 step the warp loads the D A-plane fragments once and, per
// B plane j, issues mma.sync m16n8k16 bf16 for every A plane i whose level
// i + j is formed, into the accumulator of that level.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "dgemm_sliced.cuh"
#include "mma_bf16.cuh"

namespace gb {

namespace {

constexpr int kBM = 64, kBN = 32, kBK = 32;
constexpr int kRowPad = 40;  // bf16 per staged row (32 used)
constexpr int kThreads = 256;
constexpr int kStages = 2;
// bf16 per pipeline stage and dynamic shared memory of a D-digit product
template <int D>
__host__ __device__ constexpr size_t stage_elems() { return (size_t)D * (kBM + kBN) * kRowPad; }
template <int D>
__host__ __device__ constexpr size_t product_smem() { return kStages * stage_elems<D>() * sizeof(uint16_t); }

static_assert(kSlices * kDigitBits <= 56, "digits come from the 56-bit fixed-point magnitude");
static_assert(kSlices == 8 && kLevels == 9, "the level folding below assumes at most eight digits, levels 0..8");
static_assert(kSlices * 127 * 127 * kFlushK < (1 << 24), "every level must stay below 2^24 units per flush");
constexpr int kMaxSplitK = 65536;  // keeps lo below 2^61: 512 flushes of at most 2^52

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct SliceLayout {
    size_t planes, e, rmax, total;
};

// (the layout always has room for kSlices planes, so one buffer serves every
// digit count)
SliceLayout slice_layout(int R, int K)
{
    const size_t Rp = (size_t)round_up(R > 0 ? R : 1, kBM), Kp = (size_t)round_up(K > 0 ? K : 1, kBK);
    SliceLayout L;
    L.planes = 0;
    L.e = a256(L.planes + (size_t)kSlices * Rp * Kp * sizeof(uint16_t));
    L.rmax = a256(L.e + Rp * sizeof(int));
    L.total = a256(L.rmax + Rp * sizeof(unsigned long long));
    return L;
}

// entry (a, b) of the 2 x 2 real block [x -y; y x] of x + iy
__device__ __forceinline__ double zblock(double x, double y, int a, int b) { return a == b ? x : (a ? y : -y); }

// element (r, k) of the view (r < R, k < K)
__device__ __forceinline__ double view_at(int view, const double *__restrict__ src, long long ld, int r, int k)
{
    switch (view) {
    case kViewRow: return src[r + (long long)k * ld];
    case kViewCol: return src[k + (long long)r * ld];
    case kViewSym: return r >= k ? src[r + (long long)k * ld] : src[k + (long long)r * ld];
    case kViewZExpandN: {
        const double *p = src + 2 * ((r >> 1) + (long long)(k >> 1) * ld);
        return zblock(p[0], p[1], r & 1, k & 1);
    }
    case kViewZExpandC: {  // A^H(i, j) = conj(A(j, i))
        const double *p = src + 2 * ((k >> 1) + (long long)(r >> 1) * ld);
        return zblock(p[0], -p[1], r & 1, k & 1);
    }
    case kViewZHermExpand: {
        const int i = r >> 1, j = k >> 1;
        if (i > j) {
            const double *p = src + 2 * (i + (long long)j * ld);
            return zblock(p[0], p[1], r & 1, k & 1);
        }
        const double *p = src + 2 * (j + (long long)i * ld);
        return zblock(p[0], i == j ? 0.0 : -p[1], r & 1, k & 1);
    }
    default: {  // kViewZRowConj
        const double *p = src + 2 * (r + (long long)(k >> 1) * ld);
        return (k & 1) ? -p[1] : p[0];
    }
    }
}

// Loads the 32 x 32 tile at (r0, k0) into t[r][k] (zero outside R x K), with
// the thread index running along the source's contiguous index.
__device__ __forceinline__ void load_tile(int view, const double *__restrict__ src, long long ld, int R, int K,
                                          int r0, int k0, double (*t)[33])
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    // which index is contiguous in memory for this tile
    bool along_r;
    if (view == kViewRow || view == kViewZExpandN || view == kViewZRowConj) along_r = true;
    else if (view == kViewCol || view == kViewZExpandC) along_r = false;
    else along_r = (r0 >= k0 + 31) || !(r0 + 31 < k0);  // lower or diagonal tiles: read src[r + k ld]
    for (int i = ty; i < 32; i += 8) {
        const int a = along_r ? i : tx, bb = along_r ? tx : i;  // a: k offset, bb: r offset
        const int r = r0 + bb, k = k0 + a;
        double v = 0.0;
        if (r < R && k < K) v = view_at(view, src, ld, r, k);
        t[bb][a] = v;
    }
}

__global__ void __launch_bounds__(256) slice_rowmax(int view, const double *__restrict__ src, long long ld, int R,
                                                     int K, unsigned long long *__restrict__ rmax)
{
    __shared__ double t[32][33];
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    load_tile(view, src, ld, R, K, r0, k0, t);
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        unsigned long long m = (unsigned long long)__double_as_longlong(t[i][threadIdx.x]) & 0x7fffffffffffffffull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
            m = u > m ? u : m;
        }
        if (threadIdx.x == 0 && r0 + i < R && m) atomicMax(rmax + r0 + i, m);
    }
}


// Writes the eight digit planes, or the three planes of the FP32 split.
__global__ void __launch_bounds__(256) slice_digits(int view, const double *__restrict__ src, long long ld, int R,
                                                     int K, int Rp, int Kp, const unsigned long long *__restrict__ rmax,
                                                     uint16_t *__restrict__ planes, int *__restrict__ e_out,
                                                     int digits)
{
    __shared__ double t[32][33];
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    load_tile(view, src, ld, R, K, r0, k0, t);
    __syncthreads();
    const size_t plane = (size_t)Rp * Kp;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, k = k0 + threadIdx.x;
        if (r >= Rp || k >= Kp) continue;
        const double x = t[i][threadIdx.x];
        if (digits == kSplitPlanes) {  // FP32 value split into three bf16 parts (exact)
            if (blockIdx.x == 0 && threadIdx.x == 0) e_out[r] = 0;
            const float f = __double2float_rn(x);
            const __nv_bfloat16 h0 = __float2bfloat16_rn(f);
            const float r1 = f - __bfloat162float(h0);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
            const __nv_bfloat16 h2 = __float2bfloat16_rn(r1 - __bfloat162float(h1));
            const size_t at = (size_t)r * Kp + k;
            planes[at] = __bfloat16_as_ushort(h0);
            planes[plane + at] = __bfloat16_as_ushort(h1);
            planes[2 * plane + at] = __bfloat16_as_ushort(h2);
            continue;
        }
        const int er = r < R ? exponent_above(rmax[r]) : 0;
        if (blockIdx.x == 0 && threadIdx.x == 0) e_out[r] = er;
        const unsigned long long Y = fixed56(x, er);
        const bool neg = x < 0.0;
#pragma unroll
        for (int s = 0; s < kSlices; s++) {
            if (s >= digits) break;
            const uint16_t h = bf16_digit((int)((Y >> (kDigitBits * (kSlices - 1 - s))) & 127u), s, neg);
            planes[s * plane + (size_t)r * Kp + k] = h;
        }
    }
}

// Stage loader: the leading D digit planes of the A rows [m0, m0+kBM) and B
// rows [n0, n0+kBN) for k in [kt, kt+32).
template <int D>
__device__ __forceinline__ void load_stage(uint16_t *stage, const uint16_t *__restrict__ Ap, size_t a_plane,
                                           int a_kp, const uint16_t *__restrict__ Bp, size_t b_plane, int b_kp,
                                           int m0, int n0, int kt)
{
    // D planes x rows x 4 chunks of 16 bytes (32 bf16 of k)
    constexpr int kChunksA = D * kBM * 4, kChunksB = D * kBN * 4;
    constexpr int kTotal = kChunksA + kChunksB;
#pragma unroll
    for (int it = 0; it < (kTotal + kThreads - 1) / kThreads; it++) {
        const int c = threadIdx.x + it * kThreads;
        if (kTotal % kThreads != 0 && c >= kTotal) break;
        const bool isA = c < kChunksA;
        const int rem = isA ? c : c - kChunksA;
        const int rows = isA ? kBM : kBN;
        const int s = rem / (rows * 4), row = (rem / 4) % rows, part = rem % 4;
        const uint16_t *g = isA ? Ap + s * a_plane + (size_t)(m0 + row) * a_kp + kt + part * 8
                                : Bp + s * b_plane + (size_t)(n0 + row) * b_kp + kt + part * 8;
        uint16_t *d = isA ? stage + ((size_t)s * kBM + row) * kRowPad + part * 8
                          : stage + (size_t)D * kBM * kRowPad + ((size_t)s * kBN + row) * kRowPad + part * 8;
        cp_async16(d, g);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Levels a product forms: i + j <= 8 for the eight digits; the FP32 split
// (D = kSplitPlanes) sums its pairs i + j <= 2 in one FP32 accumulator.
template <int D>
__host__ __device__ constexpr int product_levels() { return D == kSlices ? kLevels : 1; }

// One kBM x kBN tile of C (or of split z's partial product).  Warps 4 x 2,
// each 16 x 16 (two m16n8 tiles); level l = i + j < product_levels<D>() of
// the digit pairs has its own FP32 accumulator, exact over kFlushK values of
// k, folded into two 64-bit integers: hi = sum_{l<4} L_l 2^(7(3-l)),
// lo = sum_{l>=4} L_l 2^(7(8-l)), with L_l the level's sum in units of
// 2^(-7l).
template <int D>
__global__ void __launch_bounds__(kThreads, D == kSlices ? 1 : 2)
sliced_product(const uint16_t *__restrict__ Ap, const int *__restrict__ ea, int a_rp, int a_kp,
               const uint16_t *__restrict__ Bp, const int *__restrict__ eb, int b_rp, int b_kp, int m, int n,
               int ksplit, int K, double alpha, double beta, double *__restrict__ C, long long ldc, int fill,
               double *__restrict__ part)
{
    constexpr int kLev = product_levels<D>();
    constexpr bool kSplit = D == kSplitPlanes;
    constexpr size_t kStageElems = stage_elems<D>();
    extern __shared__ __align__(16) uint16_t smem[];
    const int tm = blockIdx.y, tn = blockIdx.x;
    const int m0 = tm * kBM, n0 = tn * kBN;
    if (fill == kFillLower && m0 + kBM - 1 < n0) return;          // tile wholly above the diagonal
    if (fill == kFillZLower && ((m0 + kBM - 1) >> 1) < n0) return;
    const int kbeg = blockIdx.z * ksplit, kend = min(K, kbeg + ksplit);
    const size_t a_plane = (size_t)a_rp * a_kp, b_plane = (size_t)b_rp * b_kp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 3, wn = warp >> 2;

    float acc[kLev][2][4];
    long long hi[2][4], lo[2][4];
    double dacc[2][4];  // FP32 split: the FP32 sums folded every kFlushK
#pragma unroll
    for (int l = 0; l < kLev; l++)
#pragma unroll
        for (int t = 0; t < 2; t++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[l][t][q] = 0.f;
#pragma unroll
    for (int t = 0; t < 2; t++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            hi[t][q] = lo[t][q] = 0;
            dacc[t][q] = 0.0;
        }

    // ldmatrix lane offsets within a stage's operand block
    const int a_row = wm * 16 + (lane & 7) + ((lane >> 3) & 1) * 8, a_k = (lane >> 4) * 8;
    const int b_row = wn * 16 + (lane & 7) + (lane >> 4) * 8, b_k = ((lane >> 3) & 1) * 8;

    int stage = 0;
    if (kbeg < kend) load_stage<D>(smem, Ap, a_plane, a_kp, Bp, b_plane, b_kp, m0, n0, kbeg);
    int steps = 0;
    for (int kt = kbeg; kt < kend; kt += kBK, steps++) {
        const bool more = kt + kBK < kend;
        if (more)
            load_stage<D>(smem + (size_t)(stage ^ 1) * kStageElems, Ap, a_plane, a_kp, Bp, b_plane, b_kp, m0, n0,
                          kt + kBK);
        if (more) asm volatile("cp.async.wait_group 1;" ::: "memory");
        else asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const uint16_t *As = smem + (size_t)stage * kStageElems;
        const uint16_t *Bs = As + (size_t)D * kBM * kRowPad;
#pragma unroll
        for (int ks = 0; ks < kBK / 16; ks++) {
            unsigned af[D][4];
#pragma unroll
            for (int s = 0; s < D; s++)
                ldsm_x4(af[s][0], af[s][1], af[s][2], af[s][3],
                        As + ((size_t)s * kBM + a_row) * kRowPad + ks * 16 + a_k);
#pragma unroll
            for (int j = 0; j < D; j++) {
                unsigned bf[2][2];
                ldsm_x4(bf[0][0], bf[0][1], bf[1][0], bf[1][1],
                        Bs + ((size_t)j * kBN + b_row) * kRowPad + ks * 16 + b_k);
#pragma unroll
                for (int i = 0; i < D; i++)
                    if (kSplit ? i + j <= 2 : i + j < kLev)
#pragma unroll
                        for (int t = 0; t < 2; t++) mma_bf16(acc[kSplit ? 0 : i + j][t], af[i], bf[t][0], bf[t][1]);
            }
        }
        __syncthreads();  // this stage's buffer is refilled two steps later
        stage ^= 1;
        // fold the levels into the integer accumulators every kFlushK
        if ((steps + 1) % (kFlushK / kBK) == 0 || !more) {
#pragma unroll
            for (int l = 0; l < kLev; l++)
#pragma unroll
                for (int t = 0; t < 2; t++)
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        if (kSplit) {
                            dacc[t][q] += (double)acc[l][t][q];
                            acc[l][t][q] = 0.f;
                            continue;
                        }
                        // level l holds an integer multiple of 2^(-7l) below 2^24 units
                        const float unit = __int_as_float((127 + kDigitBits * l) << 23);  // 2^(7l)
                        const long long iv = __float2int_rn(acc[l][t][q] * unit);
                        if (l < 4) hi[t][q] += iv << (kDigitBits * (3 - l));
                        else lo[t][q] += iv << (kDigitBits * (kLevels - 1 - l));
                        acc[l][t][q] = 0.f;
                    }
        }
    }

    // epilogue: value = (hi 2^-21 + lo 2^-56) 2^(ea + eb - 14)
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int t = 0; t < 2; t++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = m0 + wm * 16 + g + (q >> 1) * 8;
            const int c = n0 + wn * 16 + t * 8 + tig * 2 + (q & 1);
            if (r >= m || c >= n || (fill == kFillLower && r < c) || (fill == kFillZLower && (r >> 1) < c))
                continue;
            double v;
            if (kSplit) {
                v = dacc[t][q];
            } else {
                v = (double)hi[t][q] * 0x1p-21 + (double)lo[t][q] * 0x1p-56;
                v = scale_by_pow2(v, ea[r] + eb[c] - 2 * kDigitBits);
            }
            if (fill == kFillZLower && (r >> 1) == c && (r & 1)) {  // Hermitian diagonal: real
                if (part) part[(size_t)blockIdx.z * m * n + (size_t)c * m + r] = 0.0;
                else C[r + (long long)c * ldc] = 0.0;
                continue;
            }
            if (part) {
                part[(size_t)blockIdx.z * m * n + (size_t)c * m + r] = v;
            } else {
                double *cp = C + r + (long long)c * ldc;
                *cp = beta == 0.0 ? alpha * v : fma(alpha, v, beta * *cp);
            }
        }
}

__global__ void __launch_bounds__(256) sliced_reduce(int m, int n, int splits, const double *__restrict__ part,
                                                      double alpha, double beta, double *__restrict__ C,
                                                      long long ldc, int fill)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m * n) return;
    const int r = (int)(idx % m), c = (int)(idx / m);
    if ((fill == kFillLower && r < c) || (fill == kFillZLower && (r >> 1) < c)) return;
    if (fill == kFillZLower && (r >> 1) == c && (r & 1)) {
        C[r + (long long)c * ldc] = 0.0;
        return;
    }
    double s = 0.0;
    for (int z = 0; z < splits; z++) s += part[(size_t)z * m * n + idx];
    double *cp = C + r + (long long)c * ldc;
    *cp = beta == 0.0 ? alpha * s : fma(alpha, s, beta * *cp);
}

}  // namespace

size_t sliced_bytes(int R, int K) { return slice_layout(R, K).total; }

cudaError_t slice_matrix(SliceView view, int R, int K, const double *src, long long ld, void *buf, SlicedOp *out,
                         cudaStream_t st, int digits)
{
    if (digits != kSplitPlanes && digits != kSlices) return cudaErrorInvalidValue;
    const SliceLayout L = slice_layout(R, K);
    const int Rp = round_up(R > 0 ? R : 1, kBM), Kp = round_up(K > 0 ? K : 1, kBK);
    char *base = (char *)buf;
    uint16_t *planes = (uint16_t *)(base + L.planes);
    int *e = (int *)(base + L.e);
    unsigned long long *rmax = (unsigned long long *)(base + L.rmax);
    out->planes = planes;
    out->e = e;
    out->R = R;
    out->K = K;
    out->Rp = Rp;
    out->Kp = Kp;
    out->digits = digits;
    cudaError_t err = cudaMemsetAsync(rmax, 0, (size_t)Rp * sizeof(unsigned long long), st);
    if (err != cudaSuccess) return err;
    const dim3 block(32, 8);
    if (R > 0 && K > 0 && digits != kSplitPlanes) {  // the split needs no row maxima
        const dim3 grid((K + 31) / 32, (R + 31) / 32);
        slice_rowmax<<<grid, block, 0, st>>>((int)view, src, ld, R, K, rmax);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    // digits over the padded extent (zeros outside R x K)
    const dim3 grid2(Kp / 32, Rp / 32);
    slice_digits<<<grid2, block, 0, st>>>((int)view, src, ld, R, K, Rp, Kp, rmax, planes, e, digits);
    return cudaGetLastError();
}

namespace {

template <int D>
cudaError_t launch_product(dim3 grid, cudaStream_t st, const SlicedOp &A, const SlicedOp &B, int m, int n, int ksplit,
                           int Kp, double alpha, double beta, double *C, long long ldc, int fill, double *part)
{
    // opt in to the large dynamic shared memory (cheap; per device, so every call)
    cudaError_t e = cudaFuncSetAttribute(sliced_product<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)product_smem<D>());
    if (e != cudaSuccess) return e;
    sliced_product<D><<<grid, kThreads, product_smem<D>(), st>>>(A.planes, A.e, A.Rp, A.Kp, B.planes, B.e, B.Rp,
                                                                B.Kp, m, n, ksplit, Kp, alpha, beta, C, ldc, fill,
                                                                part);
    return cudaGetLastError();
}

}  // namespace

cudaError_t sliced_gemm(const SlicedOp &A, const SlicedOp &B, int m, int n, double alpha, double beta, double *C,
                        long long ldc, int fill, double *work, size_t work_elems, cudaStream_t st)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (A.K != B.K || A.Kp != B.Kp || m > A.R || n > B.R) return cudaErrorInvalidValue;
    const int D = std::min(A.digits, B.digits);
    const int tiles_m = (m + kBM - 1) / kBM, tiles_n = (n + kBN - 1) / kBN;
    long long tiles = (long long)tiles_m * tiles_n;
    if (fill != kFillAll) {  // tiles not wholly above the diagonal
        tiles = 0;
        for (int tm = 0; tm < tiles_m; tm++) {
            const int top = fill == kFillZLower ? (tm * kBM + kBM - 1) >> 1 : tm * kBM + kBM - 1;
            tiles += std::min(tiles_n, top / kBN + 1);
        }
    }
    const int Kp = A.Kp;
    // split the reduction when the tiles alone cannot fill the device
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int splits = 1;
    if (tiles < 2LL * sms && work) {
        splits = (int)((2LL * sms + tiles - 1) / tiles);
        const int max_by_k = Kp / (4 * kFlushK);  // keep at least 4 flush chunks per split
        if (splits > max_by_k) splits = max_by_k > 1 ? max_by_k : 1;
        while (splits > 1 && (size_t)splits * m * n > work_elems) splits--;
    }
    if (splits < (Kp + kMaxSplitK - 1) / kMaxSplitK) {  // very long sums: split so every part stays exact
        splits = (Kp + kMaxSplitK - 1) / kMaxSplitK;
        if (!work || (size_t)splits * m * n > work_elems) return cudaErrorInvalidValue;
    }
    int ksplit = Kp;
    if (splits > 1) {
        ksplit = round_up((Kp + splits - 1) / splits, kFlushK);
        splits = (Kp + ksplit - 1) / ksplit;
    }
    const dim3 grid(tiles_n, tiles_m, splits);
    double *part = splits > 1 ? work : nullptr;
    cudaError_t e;
    if ((A.digits == kSplitPlanes) != (B.digits == kSplitPlanes)) return cudaErrorInvalidValue;
    if (D == kSplitPlanes) e = launch_product<kSplitPlanes>(grid, st, A, B, m, n, ksplit, Kp, alpha, beta, C, ldc, fill, part);
    else if (D == kSlices) e = launch_product<kSlices>(grid, st, A, B, m, n, ksplit, Kp, alpha, beta, C, ldc, fill, part);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess || splits == 1) return e;
    const long long total = (long long)m * n;
    sliced_reduce<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(m, n, splits, work, alpha, beta, C, ldc, fill);
    return cudaGetLastError();
}

}  // namespace gb

// ---- whole products: slice both operands into the workspace, multiply ----

namespace gb {

namespace {

constexpr size_t kPartialElems = (size_t)4 << 20;  // split-K partials (32 MB)

struct SlicedWs {
    char *a, *b, *cat1, *cat2;
    double *part;
    size_t total;
};

// Workspace of a product whose slice-row operands are Ra x K and Rb x K; cat
// holds two Rc x Kc FP64 concatenation buffers (SYR2K), or nothing.
SlicedWs sliced_ws(int Ra, int Rb, int K, int Rc, int Kc, void *base)
{
    SlicedWs w{};
    size_t off = 0;
    char *p = (char *)base;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += a256(bytes);
        return q;
    };
    w.a = take(sliced_bytes(Ra, K));
    w.b = Rb > 0 ? take(sliced_bytes(Rb, K)) : nullptr;
    w.cat1 = Rc > 0 ? take((size_t)Rc * Kc * 8) : nullptr;
    w.cat2 = Rc > 0 ? take((size_t)Rc * Kc * 8) : nullptr;
    w.part = (double *)take(kPartialElems * 8);
    w.total = off;
    return w;
}

}  // namespace

size_t sliced_gemm_ws_bytes(int m, int n, int k) { return sliced_ws(m, n, k, 0, 0, nullptr).total; }
size_t sliced_symm_ws_bytes(char side, int m, int n)
{
    return side == 'L' ? sliced_ws(m, n, m, 0, 0, nullptr).total : sliced_ws(m, n, n, 0, 0, nullptr).total;
}
size_t sliced_syr2k_ws_bytes(int n, int k) { return sliced_ws(n, n, 2 * k, n, 2 * k, nullptr).total; }
size_t sliced_syrk_ws_bytes(int n, int k) { return sliced_ws(n, 0, k, 0, 0, nullptr).total; }

cudaError_t sliced_dgemm(char transa, char transb, int m, int n, int k, double alpha, const double *A, long long lda,
                         const double *B, long long ldb, double beta, double *C, long long ldc, void *ws,
                         cudaStream_t st, int digits)
{
    SlicedWs w = sliced_ws(m, n, k, 0, 0, ws);
    SlicedOp a, b;
    cudaError_t e = slice_matrix(transa == 'N' ? kViewRow : kViewCol, m, k, A, lda, w.a, &a, st, digits);
    if (e != cudaSuccess) return e;
    if ((e = slice_matrix(transb == 'N' ? kViewCol : kViewRow, n, k, B, ldb, w.b, &b, st, digits)) != cudaSuccess)
        return e;
    return sliced_gemm(a, b, m, n, alpha, beta, C, ldc, kFillAll, w.part, kPartialElems, st);
}

cudaError_t sliced_dsymm(char side, int m, int n, double alpha, const double *S, long long lds, const double *B,
                         long long ldb, double beta, double *C, long long ldc, void *ws, cudaStream_t st, int digits)
{
    const int K = side == 'L' ? m : n;
    SlicedWs w = sliced_ws(m, n, K, 0, 0, ws);
    SlicedOp a, b;
    cudaError_t e;
    if (side == 'L') {  // C = S B: rows of S, columns of B
        if ((e = slice_matrix(kViewSym, m, m, S, lds, w.a, &a, st, digits)) != cudaSuccess) return e;
        if ((e = slice_matrix(kViewCol, n, m, B, ldb, w.b, &b, st, digits)) != cudaSuccess) return e;
    } else {            // C = B S: rows of B, columns (= rows) of S
        if ((e = slice_matrix(kViewRow, m, n, B, ldb, w.a, &a, st, digits)) != cudaSuccess) return e;
        if ((e = slice_matrix(kViewSym, n, n, S, lds, w.b, &b, st, digits)) != cudaSuccess) return e;
    }
    return sliced_gemm(a, b, m, n, alpha, beta, C, ldc, kFillAll, w.part, kPartialElems, st);
}

cudaError_t sliced_dsyr2k_lower(int n, int k, double alpha, const double *A, long long lda, const double *B,
                                long long ldb, double beta, double *C, long long ldc, void *ws, cudaStream_t st,
                                int digits)
{
    // A B^T + B A^T = [A B] [B A]^T
    SlicedWs w = sliced_ws(n, n, 2 * k, n, 2 * k, ws);
    double *AB = (double *)w.cat1, *BA = (double *)w.cat2;
    const size_t row = (size_t)n * 8;
    cudaError_t e;
    if (k > 0) {
        if ((e = cudaMemcpy2DAsync(AB, row, A, lda * 8, row, k, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(AB + (size_t)n * k, row, B, ldb * 8, row, k, cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess ||
            (e = cudaMemcpy2DAsync(BA, row, B, ldb * 8, row, k, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(BA + (size_t)n * k, row, A, lda * 8, row, k, cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess)
            return e;
    }
    SlicedOp a, b;
    if ((e = slice_matrix(kViewRow, n, 2 * k, AB, n, w.a, &a, st, digits)) != cudaSuccess) return e;
    if ((e = slice_matrix(kViewRow, n, 2 * k, BA, n, w.b, &b, st, digits)) != cudaSuccess) return e;
    return sliced_gemm(a, b, n, n, alpha, beta, C, ldc, kFillLower, w.part, kPartialElems, st);
}

cudaError_t sliced_dsyrk_lower_t(int n, int k, double alpha, const double *A, long long lda, double beta, double *C,
                                 long long ldc, void *ws, cudaStream_t st, int digits)
{
    // A^T A: both operands are the columns of A
    SlicedWs w = sliced_ws(n, 0, k, 0, 0, ws);
    SlicedOp a;
    cudaError_t e = slice_matrix(kViewCol, n, k, A, lda, w.a, &a, st, digits);
    if (e != cudaSuccess) return e;
    return sliced_gemm(a, a, n, n, alpha, beta, C, ldc, kFillLower, w.part, kPartialElems, st);
}

// ---- complex products (interleaved storage; real alpha, beta) ----

size_t sliced_zgemm_ws_bytes(int m, int n, int k) { return sliced_ws(2 * m, n, 2 * k, 0, 0, nullptr).total; }
size_t sliced_zhemm_ws_bytes(int m, int n) { return sliced_ws(2 * m, n, 2 * m, 0, 0, nullptr).total; }
size_t sliced_zher2k_ws_bytes(int n, int k)
{
    // two n x 2k complex concatenations = n x 4k doubles each
    return sliced_ws(2 * n, n, 4 * k, n, 4 * k, nullptr).total;
}

cudaError_t sliced_zgemm(char transa, int m, int n, int k, double alpha, const double *A, long long lda,
                         const double *B, long long ldb, double beta, double *C, long long ldc, void *ws,
                         cudaStream_t st)
{
    SlicedWs w = sliced_ws(2 * m, n, 2 * k, 0, 0, ws);
    SlicedOp a, b;
    cudaError_t e = slice_matrix(transa == 'N' ? kViewZExpandN : kViewZExpandC, 2 * m, 2 * k, A, lda, w.a, &a, st);
    if (e != cudaSuccess) return e;
    if ((e = slice_matrix(kViewCol, n, 2 * k, B, 2 * ldb, w.b, &b, st)) != cudaSuccess) return e;
    return sliced_gemm(a, b, 2 * m, n, alpha, beta, C, 2 * ldc, kFillAll, w.part, kPartialElems, st);
}

cudaError_t sliced_zhemm_left(int m, int n, double alpha, const double *S, long long lds, const double *B,
                              long long ldb, double beta, double *C, long long ldc, void *ws, cudaStream_t st)
{
    SlicedWs w = sliced_ws(2 * m, n, 2 * m, 0, 0, ws);
    SlicedOp a, b;
    cudaError_t e = slice_matrix(kViewZHermExpand, 2 * m, 2 * m, S, lds, w.a, &a, st);
    if (e != cudaSuccess) return e;
    if ((e = slice_matrix(kViewCol, n, 2 * m, B, 2 * ldb, w.b, &b, st)) != cudaSuccess) return e;
    return sliced_gemm(a, b, 2 * m, n, alpha, beta, C, 2 * ldc, kFillAll, w.part, kPartialElems, st);
}

cudaError_t sliced_zher2k_lower(int n, int k, double alpha, const double *X, long long ldx, const double *Y,
                                long long ldy, double beta, double *C, long long ldc, void *ws, cudaStream_t st)
{
    // X Y^H + Y X^H = [X Y] [Y X]^H
    SlicedWs w = sliced_ws(2 * n, n, 4 * k, n, 4 * k, ws);
    double *XY = (double *)w.cat1, *YX = (double *)w.cat2;
    const size_t row = (size_t)n * 16;
    cudaError_t e;
    if (k > 0) {
        if ((e = cudaMemcpy2DAsync(XY, row, X, ldx * 16, row, k, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(XY + (size_t)2 * n * k, row, Y, ldy * 16, row, k, cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess ||
            (e = cudaMemcpy2DAsync(YX, row, Y, ldy * 16, row, k, cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(YX + (size_t)2 * n * k, row, X, ldx * 16, row, k, cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess)
            return e;
    }
    SlicedOp a, b;
    if ((e = slice_matrix(kViewZExpandN, 2 * n, 4 * k, XY, n, w.a, &a, st)) != cudaSuccess) return e;
    if ((e = slice_matrix(kViewZRowConj, n, 4 * k, YX, n, w.b, &b, st)) != cudaSuccess) return e;
    return sliced_gemm(a, b, 2 * n, n, alpha, beta, C, 2 * ldc, kFillZLower, w.part, kPartialElems, st);
}

}  // namespace gb

#include "elpa_gb300.h"

extern "C" {

static bool sl_bad_ptr(const void *p) { return !p || ((uintptr_t)p % 8) != 0; }
static bool sl_bad_ws(const void *p) { return !p || ((uintptr_t)p % 256) != 0; }

size_t gb_dgemm_sliced_workspace_bytes(int m, int n, int k)
{
    if (m < 0 || n < 0 || k < 0) return 0;
    return gb::sliced_gemm_ws_bytes(m, n, k);
}

static int dgemm_sliced_digits(char transa, char transb, int m, int n, int k, double alpha, const double *A,
                               int lda, const double *B, int ldb, double beta, double *C, int ldc, void *workspace,
                               size_t ws_bytes, void *stream, int digits)
{
    const bool ta = transa == 'T' || transa == 't', tb = transb == 'T' || transb == 't';
    if (!ta && transa != 'N' && transa != 'n') return -1;
    if (!tb && transb != 'N' && transb != 'n') return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    if (m == 0 || n == 0) return GB_OK;
    if (k > 0 && sl_bad_ptr(A)) return -7;
    if (lda < (ta ? (k > 1 ? k : 1) : m)) return -8;
    if (k > 0 && sl_bad_ptr(B)) return -9;
    if (ldb < (tb ? n : (k > 1 ? k : 1))) return -10;
    if (sl_bad_ptr(C)) return -12;
    if (ldc < m) return -13;
    if (sl_bad_ws(workspace)) return -14;
    if (ws_bytes < gb::sliced_gemm_ws_bytes(m, n, k)) return -15;
    cudaError_t e = gb::sliced_dgemm(ta ? 'T' : 'N', tb ? 'T' : 'N', m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                     workspace, (cudaStream_t)stream, digits);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int gb_dgemm_sliced(char transa, char transb, int m, int n, int k, double alpha, const double *A, int lda,
                    const double *B, int ldb, double beta, double *C, int ldc, void *workspace, size_t ws_bytes,
                    void *stream)
{
    return dgemm_sliced_digits(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace, ws_bytes,
                               stream, gb::kSlices);
}

int gb_dgemm_fp32split(char transa, char transb, int m, int n, int k, double alpha, const double *A, int lda,
                       const double *B, int ldb, double beta, double *C, int ldc, void *workspace, size_t ws_bytes,
                       void *stream)
{
    return dgemm_sliced_digits(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace, ws_bytes,
                               stream, gb::kSplitPlanes);
}

size_t gb_dsymm_sliced_workspace_bytes(char side, int m, int n)
{
    const bool left = side == 'L' || side == 'l';
    if ((!left && side != 'R' && side != 'r') || m < 0 || n < 0) return 0;
    return gb::sliced_symm_ws_bytes(left ? 'L' : 'R', m, n);
}

int gb_dsymm_sliced(char side, int m, int n, double alpha, const double *S, int lds, const double *B, int ldb,
                    double beta, double *C, int ldc, void *workspace, size_t ws_bytes, void *stream)
{
    const bool left = side == 'L' || side == 'l';
    if (!left && side != 'R' && side != 'r') return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (m == 0 || n == 0) return GB_OK;
    if (sl_bad_ptr(S)) return -5;
    if (lds < (left ? m : n)) return -6;
    if (sl_bad_ptr(B)) return -7;
    if (ldb < m) return -8;
    if (sl_bad_ptr(C)) return -10;
    if (ldc < m) return -11;
    if (sl_bad_ws(workspace)) return -12;
    if (ws_bytes < gb::sliced_symm_ws_bytes(left ? 'L' : 'R', m, n)) return -13;
    cudaError_t e = gb::sliced_dsymm(left ? 'L' : 'R', m, n, alpha, S, lds, B, ldb, beta, C, ldc, workspace,
                                     (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

size_t gb_dsyr2k_sliced_workspace_bytes(int n, int k)
{
    if (n < 0 || k < 0) return 0;
    return gb::sliced_syr2k_ws_bytes(n, k);
}

int gb_dsyr2k_sliced(int n, int k, double alpha, const double *A, int lda, const double *B, int ldb, double beta,
                     double *C, int ldc, void *workspace, size_t ws_bytes, void *stream)
{
    if (n < 0) return -1;
    if (k < 0) return -2;
    if (n == 0) return GB_OK;
    if (k > 0 && sl_bad_ptr(A)) return -4;
    if (lda < n) return -5;
    if (k > 0 && sl_bad_ptr(B)) return -6;
    if (ldb < n) return -7;
    if (sl_bad_ptr(C)) return -9;
    if (ldc < n) return -10;
    if (sl_bad_ws(workspace)) return -11;
    if (ws_bytes < gb::sliced_syr2k_ws_bytes(n, k)) return -12;
    cudaError_t e = gb::sliced_dsyr2k_lower(n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace,
                                            (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

size_t gb_dsyrk_sliced_workspace_bytes(int n, int k)
{
    if (n < 0 || k < 0) return 0;
    return gb::sliced_syrk_ws_bytes(n, k);
}

int gb_dsyrk_sliced(int n, int k, double alpha, const double *A, int lda, double beta, double *C, int ldc,
                    void *workspace, size_t ws_bytes, void *stream)
{
    if (n < 0) return -1;
    if (k < 0) return -2;
    if (n == 0) return GB_OK;
    if (k > 0 && sl_bad_ptr(A)) return -4;
    if (lda < (k > 1 ? k : 1)) return -5;
    if (sl_bad_ptr(C)) return -7;
    if (ldc < n) return -8;
    if (sl_bad_ws(workspace)) return -9;
    if (ws_bytes < gb::sliced_syrk_ws_bytes(n, k)) return -10;
    cudaError_t e = gb::sliced_dsyrk_lower_t(n, k, alpha, A, lda, beta, C, ldc, workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

size_t gb_zgemm_sliced_workspace_bytes(int m, int n, int k)
{
    if (m < 0 || n < 0 || k < 0) return 0;
    return gb::sliced_zgemm_ws_bytes(m, n, k);
}

static bool sl_bad_z(const void *p) { return !p || ((uintptr_t)p % 16) != 0; }

int gb_zgemm_sliced(char transa, int m, int n, int k, double alpha, const double *A, int lda, const double *B,
                    int ldb, double beta, double *C, int ldc, void *workspace, size_t ws_bytes, void *stream)
{
    const bool ta = transa == 'C' || transa == 'c';
    if (!ta && transa != 'N' && transa != 'n') return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (k < 0) return -4;
    if (m == 0 || n == 0) return GB_OK;
    if (k > 0 && sl_bad_z(A)) return -6;
    if (lda < (ta ? (k > 1 ? k : 1) : m)) return -7;
    if (k > 0 && sl_bad_z(B)) return -8;
    if (ldb < (k > 1 ? k : 1)) return -9;
    if (sl_bad_z(C)) return -11;
    if (ldc < m) return -12;
    if (sl_bad_ws(workspace)) return -13;
    if (ws_bytes < gb::sliced_zgemm_ws_bytes(m, n, k)) return -14;
    cudaError_t e = gb::sliced_zgemm(ta ? 'C' : 'N', m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace,
                                     (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

size_t gb_zhemm_sliced_workspace_bytes(int m, int n)
{
    if (m < 0 || n < 0) return 0;
    return gb::sliced_zhemm_ws_bytes(m, n);
}

int gb_zhemm_sliced(int m, int n, double alpha, const double *S, int lds, const double *B, int ldb, double beta,
                    double *C, int ldc, void *workspace, size_t ws_bytes, void *stream)
{
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (m == 0 || n == 0) return GB_OK;
    if (sl_bad_z(S)) return -4;
    if (lds < m) return -5;
    if (sl_bad_z(B)) return -6;
    if (ldb < m) return -7;
    if (sl_bad_z(C)) return -9;
    if (ldc < m) return -10;
    if (sl_bad_ws(workspace)) return -11;
    if (ws_bytes < gb::sliced_zhemm_ws_bytes(m, n)) return -12;
    cudaError_t e = gb::sliced_zhemm_left(m, n, alpha, S, lds, B, ldb, beta, C, ldc, workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

size_t gb_zher2k_sliced_workspace_bytes(int n, int k)
{
    if (n < 0 || k < 0) return 0;
    return gb::sliced_zher2k_ws_bytes(n, k);
}

int gb_zher2k_sliced(int n, int k, double alpha, const double *X, int ldx, const double *Y, int ldy, double beta,
                     double *C, int ldc, void *workspace, size_t ws_bytes, void *stream)
{
    if (n < 0) return -1;
    if (k < 0) return -2;
    if (n == 0) return GB_OK;
    if (k > 0 && sl_bad_z(X)) return -4;
    if (ldx < n) return -5;
    if (k > 0 && sl_bad_z(Y)) return -6;
    if (ldy < n) return -7;
    if (sl_bad_z(C)) return -9;
    if (ldc < n) return -10;
    if (sl_bad_ws(workspace)) return -11;
    if (ws_bytes < gb::sliced_zher2k_ws_bytes(n, k)) return -12;
    cudaError_t e = gb::sliced_zher2k_lower(n, k, alpha, X, ldx, Y, ldy, beta, C, ldc, workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

}  // extern "C"
