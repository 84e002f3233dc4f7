// gb_trans_ev_tridi_to_band_d_noalloc: the pipeline back-transformation for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool
// or an arena that owns all device memory, allocation-free real-time or
// interrupt-style service loops, and hosts that forbid allocation after
// start-up.  They still own their inputs and outputs (reflectors and Z) and
// pass them in; only the pipeline kernel's small scratch area (ticket,
// abort/error words and one progress flag per work item) has to come from
// somewhere else.  Here it is a file-scope __device__ array, created when
// the library's module is loaded on a device and held until the process
// exits.
//
// In host code the array's name is only a host-side stand-in, so every call
// looks up the device address with cudaGetSymbolAddress, with the call's
// device current (the lookup allocates nothing).  Looking it up each time,
// rather than caching it per device, keeps the address right after a
// cudaDeviceReset or any other re-creation of the device's primary context,
// which loads the module again and may place the array elsewhere.  The first
// call on a device loads the module there, so it should come before any
// stream capture.  Every call reuses the same array: the pipeline launcher
// clears it (cudaMemsetAsync, no allocation) before each launch, and calls
// whose device work overlaps on the GPU race on it.  The device-side status
// word is copied (cudaMemcpyAsync, no allocation) to the caller's optional
// status int after the kernel, in stream order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "trans_ev_kernels.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GB_NOALLOC_SCRATCH_BYTES];

constexpr long long kNoallocSpinPolls = 1LL << 40;
constexpr long long kNoallocTimeoutNs = 10LL * 1000 * 1000 * 1000;
constexpr int kNoallocNb = 16;       // same tiling as the library default
constexpr int kNoallocThreads = 64;

// Device address of the scratch array on the current device, looked up on
// every call (no cache that could outlive the context).
cudaError_t scratch_address(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" int gb_trans_ev_tridi_to_band_d_noalloc(int n, int nbw, int nev, const double *hh_v,
                                                   const double *hh_tau, double *Z, int ldz, int *status,
                                                   void *stream)
{
    if (n < 1) return -1;
    if (!gb::pipeline_supported(nbw)) return -2;
    if (nev < 0) return -3;
    if (n > 1 && (!hh_v || ((uintptr_t)hh_v % sizeof(double)) != 0)) return -4;
    if (n > 1 && (!hh_tau || ((uintptr_t)hh_tau % sizeof(double)) != 0)) return -5;
    if (nev > 0 && (!Z || ((uintptr_t)Z % sizeof(double)) != 0)) return -6;
    if (ldz < n) return -7;
    if (status && ((uintptr_t)status % sizeof(int)) != 0) return -8;
    const bool noop = (n == 1 || nev == 0);
    const size_t need = noop ? 0 : gb::pipeline_workspace_bytes(n, nev, kNoallocNb, kNoallocThreads);
    if (need > (size_t)GB_NOALLOC_SCRATCH_BYTES) return GB_ERR_WORKSPACE;
    if (noop && !status) return GB_OK;
    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return GB_ERR_CUDA;
    if (noop) {  // nothing to launch: report a zero status through the scratch error word
        char *err = (char *)scratch + 2 * sizeof(int);
        cudaStream_t st = (cudaStream_t)stream;
        if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
            cudaMemcpyAsync(status, err, sizeof(int), cudaMemcpyDefault, st) != cudaSuccess)
            return GB_ERR_CUDA;
        return GB_OK;
    }
    cudaError_t e = gb::pipeline_d(n, nbw, nev, hh_v, hh_tau, Z, ldz, kNoallocNb, kNoallocThreads, 0, 0, scratch, need,
                                   kNoallocSpinPolls, kNoallocTimeoutNs, 0, (cudaStream_t)stream);
    if (e != cudaSuccess) return GB_ERR_CUDA;
    if (status) {
        // the scratch head holds {ticket, abort, error}; copy the error word
        e = cudaMemcpyAsync(status, (const char *)scratch + 2 * sizeof(int), sizeof(int), cudaMemcpyDefault,
                            (cudaStream_t)stream);
        if (e != cudaSuccess) return GB_ERR_CUDA;
    }
    return GB_OK;
}
