// Device building blocks and host launch entry points shared by the
// trans_ev_tridi_to_band variants.
#pragma once
#include <cuda_runtime.h>

#include "tile_apply.cuh"

namespace gb {

// Events a caller asked for (gb_trans_ev_opts.kernel_begin_event/_end_event),
// recorded on the call's stream right before and after the launch(es) of the
// call's dominant kernel.  The entry points set them for the duration of one
// call on the issuing thread; null = not asked for.
struct KernelMarks {
    cudaEvent_t begin = nullptr, end = nullptr;
};
extern thread_local KernelMarks g_kernel_marks;
inline cudaError_t mark_kernel_begin(cudaStream_t st)
{
    return g_kernel_marks.begin ? cudaEventRecord(g_kernel_marks.begin, st) : cudaSuccess;
}
inline cudaError_t mark_kernel_end(cudaStream_t st)
{
    return g_kernel_marks.end ? cudaEventRecord(g_kernel_marks.end, st) : cudaSuccess;
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

// the chase in three steps, and the chases of many problems in one launch
cudaError_t band_to_tridi_prepare_d(int n, int b, const double *AB, int ldab, void *ws, cudaStream_t st);
cudaError_t band_to_tridi_finish_d(int n, int b, const void *ws, double *d, double *e, cudaStream_t st);
size_t chase_batched_table_bytes(int count);
cudaError_t band_to_tridi_chase_batched_upload_d(int count, const int *n, const int *b, void *const *ws,
                                                 double *const *hh_v, double *const *hh_tau, void *table,
                                                 cudaStream_t st);
cudaError_t band_to_tridi_chase_batched_d(int count, const int *n, const int *b, void *table, long long timeout_ns,
                                          cudaStream_t st);
cudaError_t band_to_tridi_chase_batched(int count, const int *n, const int *b, void *table, long long timeout_ns,
                                        cudaStream_t st, int is_complex);
cudaError_t band_to_tridi_prepare_z(int n, int b, const double *AB, int ldab, void *ws, cudaStream_t st);
cudaError_t band_to_tridi_finish_z(int n, int b, const void *ws, double *d, double *e, cudaStream_t st);

size_t band_to_tridi_workspace_bytes_z(int n, int b);
cudaError_t band_to_tridi_z(int n, int b, const double *AB, int ldab, double *d, double *e, double *hh_v,
                            double *hh_tau, void *ws, long long timeout_ns, cudaStream_t st);

size_t pipeline_workspace_bytes(int n, int nev, int nb, int threads);
bool pipeline_supported(int b);
// column_batch: column blocks per ticket batch; lead_tiles: how far a sweep
// group may run ahead of the next (0 = defaults)
cudaError_t pipeline_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z,
                       long long ldz, int nb, int threads, int column_batch, int lead_tiles, void *ws,
                       size_t ws_bytes, long long spin_polls, long long timeout_ns, int hold_group, cudaStream_t st);

// Tensor-core pipeline (real case, nbw in {16, 32, 64}): same schedule,
// tiles applied in compact WY form on mma.sync bf16 by exact digit slicing,
// Z in per-column 64-bit fixed point for the call (converted in place).
bool pipeline_tc_supported(int b);
size_t pipeline_tc_workspace_bytes(int n, int b, int nev);
cudaError_t pipeline_tc_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                          int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                          int hold_group, cudaStream_t st);

// tcgen05 pipeline (nbw in {16, 32, 64}; real data, and complex data in its
// real 2 x 2-block form): compact WY tiles with 128-column items, FP16 digit
// planes and FP32 level sums in tensor memory.
bool pipeline_tc5_supported(int b);
int pipeline_tc5_sweeps_per_tile(int b, int is_complex);
size_t pipeline_tc5_workspace_bytes(int n, int b, int nev, int is_complex);
cudaError_t pipeline_tc5_d(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                           int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                           int hold_group, cudaStream_t st);
// complex128 data: hh_v, hh_tau and Z interleaved (re, im), ldz in complex entries
cudaError_t pipeline_tc5_z(int n, int b, int nev, const double *hh_v, const double *hh_tau, double *Z, long long ldz,
                           int column_batch, void *ws, size_t ws_bytes, long long spin_polls, long long timeout_ns,
                           int hold_group, cudaStream_t st);

// Copies the device-side status words of the last real solve that used
// `ws` (its bulge chase's and its back-transformation's) into dst (two
// 256-byte slots), in stream order, so that the workspace can be reused
// before gb_solve_query-style reads of dst.
cudaError_t solve_status_copy(const void *ws, int n, int nev, int nbw, void *dst, cudaStream_t st);

}  // namespace gb
