// Warp-level bf16 tensor-core building blocks shared by the digit-sliced
// FP64 kernels (dgemm_sliced.cu, trans_ev_tc.cu): cp.async staging,
// ldmatrix fragment loads, mma.sync m16n8k16 with FP32 accumulation, and the
// bf16 encoding of a signed 7-bit digit scaled by 2^(-7 s).
//
// Fragment layouts (PTX ISA, mma.m16n8k16 with .bf16): lane = 4 g + t.
//   A (16 x 16, row-major): a0 (g, 2t..2t+1), a1 (g+8, 2t..), a2 (g, 2t+8..),
//     a3 (g+8, 2t+8..); ldmatrix.x4 of the four 8 x 8 quadrants in that order.
//   B (16 x 8, stored n-major: row n holds k): b0 (k 2t..2t+1, n g),
//     b1 (k 2t+8.., n g); ldmatrix.x2 of the two 8 x 8 halves along k.
//   C (16 x 8, FP32): c0 c1 (g, 2t..2t+1), c2 c3 (g+8, 2t..2t+1).
#pragma once
#include <stdint.h>

namespace gb {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x2(unsigned &r0, unsigned &r1, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// bf16 bit pattern of (neg ? -1 : 1) * d * 2^(-7 s), 0 <= d <= 127: exact,
// since d has at most 7 significant bits (d = 1.f x 2^p).
__device__ __forceinline__ uint16_t bf16_digit(int d, int s, bool neg)
{
    if (!d) return 0;
    const int p = 31 - __clz(d);
    const unsigned frac = ((unsigned)d << (7 - p)) & 0x7fu;
    const unsigned expo = (unsigned)(127 + p - 7 * s);
    return (uint16_t)((neg ? 0x8000u : 0u) | (expo << 7) | frac);
}

// Row exponent e with max|row| < 2^e from the bit pattern of the row's
// largest magnitude (0 for an all-zero row).  A subnormal maximum m 2^-1074
// with m < 2^L gives e = L - 1074.
__device__ __forceinline__ int exponent_above(unsigned long long maxbits)
{
    const int ex = (int)(maxbits >> 52) & 0x7ff;
    if (ex) return ex - 1022;
    if (!maxbits) return 0;
    return (64 - __clzll((long long)maxbits)) - 1074;
}

// Y = round(|x| 2^(56 - e)) for |x| < 2^e, at most 2^56 - 1: the 56-bit
// fixed-point magnitude whose 7-bit groups are the digits (subnormals read
// as zero).  Rounding to nearest keeps the representation error unbiased, so
// that it grows like sqrt(k) and not like k in sums of one sign.
__device__ __forceinline__ unsigned long long fixed56(double x, int e)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((u >> 52) & 0x7ff);
    if (ex == 0) return 0ull;
    const unsigned long long M = (u & 0xfffffffffffffull) | (1ull << 52);
    const int sh = ex - 1075 - e + 56;
    unsigned long long Y;
    if (sh >= 0) Y = M << sh;
    else if (sh > -54) Y = (M + (1ull << (-sh - 1))) >> -sh;
    else Y = 0ull;
    return Y < (1ull << 56) ? Y : (1ull << 56) - 1;
}

// Y = round(|x| 2^(63 - e)) for |x| < 2^e, at most 2^63 - 1: nine 7-bit
// digits (exact for entries within 10 binades of the row's largest)
__device__ __forceinline__ unsigned long long fixed63(double x, int e)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((u >> 52) & 0x7ff);
    if (ex == 0) return 0ull;
    const unsigned long long M = (u & 0xfffffffffffffull) | (1ull << 52);
    const int sh = ex - 1075 - e + 63;
    unsigned long long Y;
    if (sh >= 0) Y = M << sh;
    else if (sh > -54) Y = (M + (1ull << (-sh - 1))) >> -sh;
    else Y = 0ull;
    return Y < (1ull << 63) ? Y : (1ull << 63) - 1;
}

// v * 2^e for -1022 <= e <= 1023, and for wider e as two factors
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }
__device__ __forceinline__ double scale_by_pow2(double v, int e)
{
    const int e1 = e / 2, e2 = e - e1;
    return v * pow2(e1) * pow2(e2);
}

}  // namespace gb
