// Device eigenpairs of a real symmetric tridiagonal matrix (bisection and
// inverse iteration), used by the solver entry points.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace gb {

// Threads per block of the inverse-iteration kernel.
constexpr int kTridiagThreads = 32;

size_t tridiag_eig_workspace_bytes(int n, int nev);
cudaError_t tridiag_bisect_d(int n, int nev, const double *d, const double *e, double *lam, void *ws, cudaStream_t st);
cudaError_t tridiag_invit_d(int n, int nev, const double *d, const double *e, const double *lam, double *Z,
                            long long ldz, void *ws, cudaStream_t st, int threads = kTridiagThreads);
cudaError_t tridiag_eig_d(int n, int nev, const double *d, const double *e, double *lam, double *Z, long long ldz,
                          void *ws, cudaStream_t st);

}  // namespace gb
