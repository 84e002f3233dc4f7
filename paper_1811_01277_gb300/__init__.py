"""GB300 (sm_103a) back-transformation of eigenvectors from tridiagonal to
band form -- the hot path of the two-stage ELPA eigensolver (Kus et al.,
"Optimizations of the Eigensolvers in the ELPA Library", Sec. 2 and 3.1).

The computation runs in ``libelpa_gb300.so`` (CUDA C++, C ABI declared in
``include/elpa_gb300.h``).  This package is its thin ctypes binding plus the
seeded input generators; PyTorch only provides device memory and streams.
"""
from ._lib import (  # noqa: F401
    EXPORTS, GB_ERR_CUDA, GB_ERR_TIMEOUT, GB_ERR_UNSUPPORTED, GB_ERR_WORKSPACE, GB_ERR_NONFINITE, GB_ERR_RANGE, GB_OK,
    GB_NOALLOC_SCRATCH_BYTES, GB_SOLVE_FP64_EMULATED_GEMM, GB_VARIANT_AUTO, GB_VARIANT_PIPELINE, GB_VARIANT_PIPELINE_TC,
    GB_VARIANT_PIPELINE_TC5, GB_VARIANT_WAVEFRONT, GbError, LIB_PATH, gb_trans_ev_variant,
    gb_band_to_tridi_d, gb_band_to_tridi_workspace_bytes, gb_band_to_tridi_workspace_bytes_z, gb_band_to_tridi_z, gb_hh_count, gb_hh_index, gb_max_nbw, gb_status_string, gb_trans_ev_host_buffer_bytes,
    gb_trans_ev_launch_count, gb_trans_ev_opts, gb_trans_ev_query, gb_trans_ev_tridi_to_band_d,
    gb_trans_ev_tridi_to_band_d_host, gb_trans_ev_tridi_to_band_d_noalloc, gb_trans_ev_tridi_to_band_z, gb_trans_ev_workspace_bytes,
    GB_AUTOTUNE_FAST, GB_AUTOTUNE_MEDIUM, elpa_b200_solve, gb_autotune_best, gb_autotune_create,
    gb_autotune_destroy, gb_autotune_load, gb_autotune_progress, gb_autotune_report, gb_autotune_save,
    gb_autotune_step, gb_solve_batched_d, gb_solve_batched_workspace_bytes, gb_solve_d,
    gb_solve_default_nbw, gb_solve_stage_ms, gb_solve_release, gb_solve_workspace_bytes_z, gb_solve_z, gb_solve_query_z, GB_SOLVE_RECORD_STAGES, SOLVE_STAGES, gb_solve_query, gb_solve_workspace_bytes, load,
    gb_dgemm, gb_dgemm_workspace_bytes, gb_dsymm, gb_dsyr2k, gb_dsyrk,
    GB_SOLVE_DFMA_PRODUCTS, gb_dgemm_sliced, gb_dgemm_sliced_workspace_bytes, gb_dsymm_sliced,
    gb_dsymm_sliced_workspace_bytes, gb_dsyr2k_sliced, gb_dsyr2k_sliced_workspace_bytes, gb_dsyrk_sliced,
    gb_dsyrk_sliced_workspace_bytes, gb_zgemm_sliced, gb_zgemm_sliced_workspace_bytes, gb_zhemm_sliced,
    gb_zhemm_sliced_workspace_bytes, gb_zher2k_sliced, gb_zher2k_sliced_workspace_bytes,
    gb_solve_batched_workspace_bytes_nbw, gb_solve_batched_nbw_d, gb_solve_batched_graph_create,
    gb_solve_batched_graph_launch, gb_solve_batched_graph_nodes, gb_solve_batched_graph_destroy,
    gb_solve_tuner_create, gb_solve_tuner_destroy, gb_solve_tuner_step, gb_solve_tuner_report, gb_solve_tuner_nbw,
    gb_solve_tuner_save, gb_solve_tuner_load, gb_tridiag_dc_workspace_bytes, gb_tridiag_dc_d, GB_SOLVE_TRIDIAG_BISECT,
    gb_refine_syev_workspace_bytes, gb_refine_syev_d, gb_solve_batched_staged_workspace_bytes,
    gb_solve_batched_staged_d, gb_solve_batched_staged_query, gb_solve_stage_table_bytes, gb_solve_stage_front,
    gb_solve_stage_chase_batched, gb_solve_stage_back, GB_SOLVE_FP32_PRODUCTS, GB_SOLVE_MIXED_MAX_STEPS,
    gb_solve_mixed_workspace_bytes, gb_solve_mixed_d, gb_solve_mixed_query, gb_dgemm_fp32split,
)


def trans_ev_tridi_to_band(n, nbw, hh_v, hh_tau, Z, stream=None, opts=None):
    """Z <- Q2 Z in place for device tensors (float64 or complex128).

    Allocates the workspace the call needs with torch and forwards to the
    C entry point; ``Z`` is column-major (a transposed row-major tensor, i.e.
    ``Z.T`` contiguous) with leading dimension ``Z.stride(1)``."""
    import torch
    cplx = Z.is_complex()
    nev = Z.shape[1]
    ldz = Z.stride(1) if nev > 1 else max(n, 1)
    if Z.stride(0) != 1:
        raise ValueError("Z must be column-major (stride(0) == 1)")
    ws_bytes = gb_trans_ev_workspace_bytes(n, nbw, nev, cplx, opts)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=Z.device) if ws_bytes else None
    f = gb_trans_ev_tridi_to_band_z if cplx else gb_trans_ev_tridi_to_band_d
    f(n, nbw, nev, hh_v, hh_tau, Z, ldz, ws, ws_bytes,
      stream if stream is not None else torch.cuda.current_stream(Z.device), opts)
    return Z
