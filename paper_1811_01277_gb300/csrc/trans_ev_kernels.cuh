// Device building blocks and host launch entry points shared by the
// trans_ev_tridi_to_band variants.
#pragma once
#include <cuda_runtime.h>

namespace gb {

// Apply one tile: the nb reflectors staged in vs/ts, sweep offset q = nb-1
// down to 0 (descending sweep = reverse generation order), to the window w
// of one column.  Reflector q covers window rows q .. q+B-1; vs[q][0] is the
// implicit 1 and vs[q][i] = 0 past the reflector's length, so truncated
// reflectors need no special case.  Per reflector: B-1 DFMA for the dot
// product (the v_0 term is the initial value), one DMUL for tau*w, one DADD
// and B-1 DFMA for the update: 2*B FP64 operations, the algorithmic count.
template <int B, int NB>
__device__ __forceinline__ void apply_tile_regs(double (&w)[B + NB - 1], const double (*vs)[B],
                                                const double *ts)
{
#pragma unroll
    for (int q = NB - 1; q >= 0; q--) {
        const double tau = ts[q];
        if (tau != 0.0) {
            double acc = w[q];
#pragma unroll
            for (int i = 1; i < B; i++) acc = fma(vs[q][i], w[q + i], acc);
            const double tw = tau * acc;
            w[q] -= tw;
            // Re-read v from shared memory instead of keeping B values live
            // across both loops (the window already holds B+NB-1 registers).
            const volatile double *vq = vs[q];
#pragma unroll
            for (int i = 1; i < B; i++) w[q + i] = fma(-tw, vq[i], w[q + i]);
        }
    }
}

cudaError_t wavefront_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                        long long ldz, int nb, int threads, cudaStream_t st);
long long wavefront_launch_count(int n, int b, int nb);

cudaError_t wavefront_smem_z(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                             long long ldz, int nb, int threads, cudaStream_t st);
cudaError_t wavefront_smem_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                             long long ldz, int nb, int threads, cudaStream_t st);
size_t wavefront_smem_bytes(int b, int nb, int threads, int is_complex);

size_t band_to_tridi_workspace_bytes(int n, int b);
cudaError_t band_to_tridi_d(int n, int b, const double *AB, int ldab, double *d, double *e, double *hh_v,
                            double *hh_tau, void *ws, size_t ws_bytes, long long timeout_ns, cudaStream_t st);

size_t pipeline_workspace_bytes(int n, int nev, int nb, int threads);
bool pipeline_supported(int b);
cudaError_t pipeline_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                       long long ldz, int nb, int threads, void *ws, size_t ws_bytes, long long spin_polls,
                       long long timeout_ns, int hold_group, cudaStream_t st);

}  // namespace gb
