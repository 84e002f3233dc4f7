// Reflector layout of the band -> tridiagonal bulge chase, as the kernels see
// it (the contract is spelled out in include/elpa_gb300.h).
//
// Sweep s (1-based, 1..n-1) has nk(s) = ceil((n-s)/b) reflectors; H(s,k) acts
// on 0-based rows s+k*b .. s+k*b+len-1 with len = min(b, n-s-k*b).  The index
// of the first reflector of sweep s is
//     sum_{s'=1}^{s-1} ceil((n-s')/b) = F(n-1) - F(n-s),
//     F(m) = sum_{j=1}^{m} ceil(j/b) = b*q*(q+1)/2 + r*(q+1),  m = q*b + r,
// which lets every kernel locate H(s,k) without a table.
#pragma once
#include <cstdint>

namespace gb {

__host__ __device__ __forceinline__ long long ceil_sum(long long m, long long b)
{
    if (m <= 0) return 0;
    long long q = m / b, r = m % b;
    return b * q * (q + 1) / 2 + r * (q + 1);
}

__host__ __device__ __forceinline__ long long sweep_first(int n, int b, int s)
{
    return ceil_sum(n - 1, b) - ceil_sum(n - s, b);
}

__host__ __device__ __forceinline__ int sweep_count(int n, int b, int s)
{
    return (n - s + b - 1) / b;
}

__host__ __device__ __forceinline__ long long hh_total(int n, int b)
{
    return ceil_sum(n - 1, b);
}

// Tiles: group g holds sweeps s0 = 1 + g*nb .. min(s0+nb-1, n-1); tile (g,k)
// holds H(s,k) for the group's sweeps.  It touches the b+nb-1 rows starting at
// 0-based row s0 + k*b.  Group g has nk(s0) tiles.
__host__ __device__ __forceinline__ int group_count(int n, int nb)
{
    return (n - 1 + nb - 1) / nb;
}

__host__ __device__ __forceinline__ int group_tiles(int n, int b, int nb, int g)
{
    return sweep_count(n, b, 1 + g * nb);
}

}  // namespace gb
