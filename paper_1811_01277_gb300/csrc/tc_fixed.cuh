// Per-column 64-bit fixed point of Z for the tensor-core back-transformation
// kernels (trans_ev_tc.cu on mma.sync, trans_ev_tc5.cu on tcgen05), and the
// small device helpers their schedules share.
//
// Every column c of Z is held for the whole call as z = Zi 2^(E_c - 62) with
// ||z_c||_2 < 2^(E_c - 1), so |Zi| < 2^61.  Householder reflectors are
// orthogonal, so no entry of an intermediate column exceeds the column's
// initial 2-norm: one scale per column serves the whole call, and the tile
// updates are integer additions.
//
// Inputs the fixed point cannot carry are reported, not converted:
//  * a column holding NaN or Inf is flagged (E_c = kTcNonFinite), runs as a
//    zero column and comes back as all NaN; the call's status word records
//    GB_ERR_NONFINITE;
//  * a column whose maximum is subnormal is scaled like any other (the
//    exponent of a subnormal is read from its leading mantissa bit);
//  * a stored fixed-point entry at or above 2^61 in magnitude (possible only
//    when the reflectors are not orthogonal, e.g. a tau of the wrong
//    convention) records GB_ERR_RANGE.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "mma_bf16.cuh"

namespace gb {
namespace {

constexpr int kTcNonFinite = 0x7fffffff;             // E_c of a column holding NaN or Inf
constexpr long long kTcFixedLimit = 1ll << 61;        // |Zi| stays below this for orthogonal reflectors

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct TcState {  // head of the workspace (zeroed before every launch)
    int ticket;
    int abort;
    int error;
};

// record a device-side status; the first one recorded wins
__device__ __forceinline__ void tc_set_error(TcState *st, int code) { atomicCAS(&st->error, 0, code); }

// x * 2^sh for a 64-bit integer, rounded to nearest when sh < 0 (so that
// the rescaling adds no bias)
__device__ __forceinline__ long long shift_ll(long long x, int sh)
{
    if (sh >= 0) return (long long)((unsigned long long)x << sh);
    if (sh <= -63) return 0;
    return (x + (1ll << (-sh - 1))) >> -sh;
}

// true if a stored fixed-point entry has left the range orthogonal
// reflectors keep it in
__device__ __forceinline__ bool tc_out_of_range(long long v) { return v >= kTcFixedLimit || v <= -kTcFixedLimit; }

// E_c with ||z_c||_2 < 2^(E_c - 1), one warp per column.  The sum of squares
// is taken on the column scaled by 2^-em (max|z| < 2^em, an exact scaling),
// so it neither overflows nor underflows: ||z||^2 < 2^(e2 + 2 em) gives
// E_c = ceil(e2 / 2) + em + 1 (0 for a zero column).  For even e2 the bound
// is tight, and where ||z|| sits within 2^-30 of it, E_c takes one more bit.
// Rounding (of s, and of the fixed-point updates) can then never carry an
// entry past 2^61, even if the whole norm gathers in it.  A column holding
// NaN or Inf gets E_c = kTcNonFinite and sets GB_ERR_NONFINITE.
__global__ void __launch_bounds__(256) tc_col_scale(int n, int nev, const double *__restrict__ Z, long long ldz,
                                                    int *__restrict__ E, TcState *state)
{
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= nev) return;
    const double *z = Z + (long long)c * ldz;
    unsigned long long m = 0;
    for (int r = lane; r < n; r += 32) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(z[r]) & ~(1ull << 63);
        m = u > m ? u : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
        m = u > m ? u : m;
    }
    if (m >= 0x7ff0000000000000ull) {  // Inf or NaN somewhere in the column
        if (lane == 0) {
            E[c] = kTcNonFinite;
            tc_set_error(state, GB_ERR_NONFINITE);
        }
        return;
    }
    if (m == 0) {
        if (lane == 0) E[c] = 0;
        return;
    }
    const int em = exponent_above(m);
    double s = 0.0;
    for (int r = lane; r < n; r += 32) {
        const double x = scale_by_pow2(z[r], -em);
        s = fma(x, x, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int e2 = exponent_above((unsigned long long)__double_as_longlong(s));
        int ec = ((e2 + 1) >> 1) + em + 1;
        if (!(e2 & 1) && s > scale_by_pow2(1.0 - 0x1p-29, e2)) ec += 1;  // 1/4 <= s < n: -1 <= e2 <= 32
        E[c] = ec;
    }
}

// In place: z -> round(z 2^(62 - E_c)) as int64 (to_fixed) or back
// (from_fixed).  Flagged columns become zero on the way in and NaN on the
// way out.
__global__ void __launch_bounds__(256) tc_convert(int n, int nev, double *__restrict__ Z, long long ldz,
                                                  const int *__restrict__ E, int to_fixed)
{
    for (int c = blockIdx.y; c < nev; c += gridDim.y) {
        const int e = E[c];
        double *z = Z + (long long)c * ldz;
        long long *zi = (long long *)z;
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
            if (e == kTcNonFinite) {
                if (to_fixed) zi[r] = 0;
                else z[r] = __longlong_as_double(0x7ff8000000000000ll);
            } else if (to_fixed) {
                zi[r] = __double2ll_rn(scale_by_pow2(z[r], 62 - e));
            } else {
                z[r] = scale_by_pow2(__ll2double_rn(zi[r]), e - 62);
            }
        }
    }
}

// first tile of every sweep group of nb sweeps, and the total (off[G])
__global__ void tc_tile_offsets(int n, int b, int nb, int G, long long *__restrict__ off)
{
    long long acc = 0;
    for (int g = 0; g < G; g++) {
        off[g] = acc;
        acc += group_tiles(n, b, nb, g);
    }
    off[G] = acc;
}

}  // namespace
}  // namespace gb
