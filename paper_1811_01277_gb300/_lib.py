"""ctypes binding of libelpa_gb300.so (argument marshalling only).

Every function here has the name of the C entry point it forwards to (see
``include/elpa_gb300.h``).  Pointer arguments accept a ``torch.Tensor``
(its ``data_ptr()``), a numpy array (host pointer), an ``int`` or ``None``.
No step of the computation runs in Python: if the library is missing the
calls raise instead of falling back to anything else.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libelpa_gb300.so")

GB_OK = 0
GB_ERR_CUDA = 1
GB_ERR_TIMEOUT = 2
GB_ERR_WORKSPACE = 3
GB_ERR_UNSUPPORTED = 4
GB_ERR_NONFINITE = 5
GB_ERR_RANGE = 6
GB_VARIANT_AUTO = 0
GB_VARIANT_WAVEFRONT = 1
GB_VARIANT_PIPELINE = 2
GB_VARIANT_PIPELINE_TC = 3
GB_VARIANT_PIPELINE_TC5 = 4

EXPORTS = (
    "gb_hh_count", "gb_hh_index", "gb_max_nbw", "gb_trans_ev_workspace_bytes",
    "gb_trans_ev_tridi_to_band_d", "gb_trans_ev_tridi_to_band_z",
    "gb_trans_ev_host_buffer_bytes", "gb_trans_ev_tridi_to_band_d_host",
    "gb_trans_ev_launch_count", "gb_trans_ev_variant", "gb_status_string", "gb_trans_ev_query",
    "gb_trans_ev_tridi_to_band_d_noalloc", "gb_band_to_tridi_workspace_bytes", "gb_band_to_tridi_d",
    "gb_solve_workspace_bytes", "gb_solve_d", "gb_solve_query", "elpa_b200_solve",
    "gb_autotune_create", "gb_autotune_destroy", "gb_autotune_step", "gb_autotune_report",
    "gb_autotune_best", "gb_autotune_progress", "gb_autotune_save", "gb_autotune_load",
    "gb_solve_default_nbw", "gb_solve_batched_workspace_bytes", "gb_solve_batched_d", "gb_solve_stage_ms",
    "gb_solve_release", "gb_solve_batched_workspace_bytes_nbw", "gb_solve_batched_nbw_d",
    "gb_solve_batched_graph_create", "gb_solve_batched_graph_launch", "gb_solve_batched_graph_nodes",
    "gb_solve_batched_graph_destroy", "gb_solve_tuner_create", "gb_solve_tuner_destroy", "gb_solve_tuner_step",
    "gb_solve_tuner_report", "gb_solve_tuner_nbw", "gb_solve_tuner_save", "gb_solve_tuner_load",
    "gb_tridiag_dc_workspace_bytes", "gb_tridiag_dc_d", "gb_refine_syev_workspace_bytes", "gb_refine_syev_d",
    "gb_solve_mixed_workspace_bytes", "gb_solve_mixed_d", "gb_solve_mixed_query",
    "gb_solve_batched_staged_workspace_bytes", "gb_solve_batched_staged_d", "gb_solve_batched_staged_query",
    "gb_solve_stage_table_bytes", "gb_solve_stage_front", "gb_solve_stage_chase_batched", "gb_solve_stage_back",
    "gb_band_to_tridi_workspace_bytes_z", "gb_band_to_tridi_z",
    "gb_solve_workspace_bytes_z", "gb_solve_z", "gb_solve_query_z",
    "gb_dgemm_workspace_bytes", "gb_dgemm", "gb_dsymm", "gb_dsyr2k", "gb_dsyrk",
    "gb_dgemm_sliced_workspace_bytes", "gb_dgemm_sliced", "gb_dgemm_fp32split", "gb_dsymm_sliced_workspace_bytes",
    "gb_dsymm_sliced",
    "gb_dsyr2k_sliced_workspace_bytes", "gb_dsyr2k_sliced", "gb_dsyrk_sliced_workspace_bytes", "gb_dsyrk_sliced",
    "gb_zgemm_sliced_workspace_bytes", "gb_zgemm_sliced", "gb_zhemm_sliced_workspace_bytes", "gb_zhemm_sliced",
    "gb_zher2k_sliced_workspace_bytes", "gb_zher2k_sliced",
)
GB_SOLVE_RECORD_STAGES = 2
GB_SOLVE_DFMA_PRODUCTS = 4
GB_SOLVE_TRIDIAG_BISECT = 8
GB_SOLVE_FP32_PRODUCTS = 16
GB_SOLVE_MIXED_MAX_STEPS = 8
# stage 2 is the whole tridiagonal step when it runs as divide and conquer
# (stages 3 and 4 are then empty)
SOLVE_STAGES = ("full_to_band", "band_to_tridi", "tridiag_bisection_or_dc", "inverse_iteration", "orthogonalise",
                "trans_ev_tridi_to_band", "band_to_full")
GB_AUTOTUNE_FAST = 1
GB_AUTOTUNE_MEDIUM = 2
GB_SOLVE_FP64_EMULATED_GEMM = 1
GB_NOALLOC_SCRATCH_BYTES = 1 << 20


class gb_trans_ev_opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("sweeps_per_tile", ctypes.c_int),
                ("cols_per_block", ctypes.c_int), ("spin_limit", ctypes.c_int),
                ("test_hold_group", ctypes.c_int), ("column_batch", ctypes.c_int),
                ("lead_tiles", ctypes.c_int), ("kernel_begin_event", ctypes.c_void_p),
                ("kernel_end_event", ctypes.c_void_p)]


class GbError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what} returned {status}: {gb_status_string(status)}")


_lib = None


def load(path=None):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library not found at {path}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    i, ll, sz, p = ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t, ctypes.c_void_p
    po = ctypes.POINTER(gb_trans_ev_opts)
    L.gb_hh_count.argtypes = [i, i]; L.gb_hh_count.restype = ll
    L.gb_hh_index.argtypes = [i, i, i, i]; L.gb_hh_index.restype = ll
    L.gb_max_nbw.argtypes = []; L.gb_max_nbw.restype = i
    L.gb_trans_ev_workspace_bytes.argtypes = [i, i, i, i, po]; L.gb_trans_ev_workspace_bytes.restype = sz
    for nm in ("gb_trans_ev_tridi_to_band_d", "gb_trans_ev_tridi_to_band_z"):
        getattr(L, nm).argtypes = [i, i, i, p, p, p, i, p, sz, p, po]
        getattr(L, nm).restype = i
    L.gb_trans_ev_host_buffer_bytes.argtypes = [i, i, i, i, i, po]
    L.gb_trans_ev_host_buffer_bytes.restype = sz
    L.gb_trans_ev_tridi_to_band_d_host.argtypes = [i, i, i, p, p, p, i, p, sz, p, po]
    L.gb_trans_ev_tridi_to_band_d_host.restype = i
    L.gb_trans_ev_launch_count.argtypes = [i, i, i, i, po]; L.gb_trans_ev_launch_count.restype = ll
    L.gb_trans_ev_variant.argtypes = [i, i, i, i, po]; L.gb_trans_ev_variant.restype = i
    L.gb_status_string.argtypes = [i]; L.gb_status_string.restype = ctypes.c_char_p
    L.gb_trans_ev_query.argtypes = [p, sz, p]; L.gb_trans_ev_query.restype = i
    L.gb_trans_ev_tridi_to_band_d_noalloc.argtypes = [i, i, i, p, p, p, i, p, p]
    L.gb_trans_ev_tridi_to_band_d_noalloc.restype = i
    L.gb_band_to_tridi_workspace_bytes.argtypes = [i, i]; L.gb_band_to_tridi_workspace_bytes.restype = sz
    L.gb_band_to_tridi_d.argtypes = [i, i, p, i, p, p, p, p, p, sz, p]; L.gb_band_to_tridi_d.restype = i
    L.gb_solve_workspace_bytes.argtypes = [i, i, i]; L.gb_solve_workspace_bytes.restype = sz
    L.gb_solve_d.argtypes = [i, i, i, p, i, p, p, i, p, sz, p, i]; L.gb_solve_d.restype = i
    L.gb_solve_query.argtypes = [p, i, i, i, p]; L.gb_solve_query.restype = i
    L.elpa_b200_solve.argtypes = [i, i, p, i, p, p, i]; L.elpa_b200_solve.restype = i
    L.gb_autotune_create.argtypes = [i, i, i, i]; L.gb_autotune_create.restype = p
    L.gb_autotune_destroy.argtypes = [p]; L.gb_autotune_destroy.restype = None
    L.gb_autotune_step.argtypes = [p, po]; L.gb_autotune_step.restype = i
    L.gb_autotune_report.argtypes = [p, ctypes.c_double]; L.gb_autotune_report.restype = i
    L.gb_autotune_best.argtypes = [p, po, ctypes.POINTER(ctypes.c_double)]; L.gb_autotune_best.restype = i
    L.gb_autotune_progress.argtypes = [p, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.gb_autotune_progress.restype = i
    L.gb_autotune_save.argtypes = [p, ctypes.c_char_p]; L.gb_autotune_save.restype = i
    L.gb_autotune_load.argtypes = [ctypes.c_char_p]; L.gb_autotune_load.restype = p
    L.gb_solve_default_nbw.argtypes = [i]; L.gb_solve_default_nbw.restype = i
    L.gb_solve_stage_ms.argtypes = [p, ctypes.POINTER(ctypes.c_float)]; L.gb_solve_stage_ms.restype = i
    L.gb_solve_release.argtypes = [p, i]; L.gb_solve_release.restype = i
    L.gb_band_to_tridi_workspace_bytes_z.argtypes = [i, i]; L.gb_band_to_tridi_workspace_bytes_z.restype = sz
    L.gb_band_to_tridi_z.argtypes = [i, i, p, i, p, p, p, p, p, sz, p]; L.gb_band_to_tridi_z.restype = i
    L.gb_solve_workspace_bytes_z.argtypes = [i, i, i]; L.gb_solve_workspace_bytes_z.restype = sz
    L.gb_solve_z.argtypes = [i, i, i, p, i, p, p, i, p, sz, p, i]; L.gb_solve_z.restype = i
    L.gb_solve_query_z.argtypes = [p, i, i, i, p]; L.gb_solve_query_z.restype = i
    pi_ = ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.gb_solve_batched_workspace_bytes.argtypes = [i, pi_, pi_, i]
    L.gb_solve_batched_workspace_bytes.restype = sz
    L.gb_solve_batched_d.argtypes = [i, pi_, pi_, pp, pi_, pp, pp, pi_, p, sz, i, pp, pp, pp]
    L.gb_solve_batched_d.restype = i
    L.gb_solve_batched_workspace_bytes_nbw.argtypes = [i, pi_, pi_, pi_, i]
    L.gb_solve_batched_workspace_bytes_nbw.restype = sz
    L.gb_solve_batched_nbw_d.argtypes = [i, pi_, pi_, pi_, pp, pi_, pp, pp, pi_, p, sz, i, pp, pp, pp]
    L.gb_solve_batched_nbw_d.restype = i
    L.gb_solve_batched_staged_workspace_bytes.argtypes = [i, pi_, pi_, pi_, i]
    L.gb_solve_batched_staged_workspace_bytes.restype = sz
    L.gb_solve_batched_staged_d.argtypes = [i, pi_, pi_, pi_, pp, pi_, pp, pp, pi_, p, sz, i, pp, pp, pp]
    L.gb_solve_batched_staged_d.restype = i
    L.gb_solve_batched_staged_query.argtypes = [p, i, pi_, pi_, pi_, i, pp]
    L.gb_solve_batched_staged_query.restype = i
    L.gb_solve_stage_table_bytes.argtypes = [i]; L.gb_solve_stage_table_bytes.restype = sz
    L.gb_solve_stage_front.argtypes = [i, i, i, i, p, i, p, sz, p]; L.gb_solve_stage_front.restype = i
    L.gb_solve_stage_chase_batched.argtypes = [i, i, pi_, pi_, pi_, pp, p, sz, p]
    L.gb_solve_stage_chase_batched.restype = i
    L.gb_solve_stage_back.argtypes = [i, i, i, i, p, p, i, p, sz, p, i]; L.gb_solve_stage_back.restype = i
    L.gb_solve_batched_graph_create.argtypes = [i, pi_, pi_, pi_, pp, pi_, pp, pp, pi_, p, sz, i, pp, pp, pp]
    L.gb_solve_batched_graph_create.restype = i
    L.gb_solve_batched_graph_launch.argtypes = [p, p]; L.gb_solve_batched_graph_launch.restype = i
    L.gb_solve_batched_graph_nodes.argtypes = [p]; L.gb_solve_batched_graph_nodes.restype = ctypes.c_longlong
    L.gb_solve_batched_graph_destroy.argtypes = [p]; L.gb_solve_batched_graph_destroy.restype = i
    L.gb_solve_tuner_create.argtypes = [i, i, i]; L.gb_solve_tuner_create.restype = p
    L.gb_solve_tuner_destroy.argtypes = [p]; L.gb_solve_tuner_destroy.restype = None
    L.gb_solve_tuner_step.argtypes = [p, pi_, pi_]; L.gb_solve_tuner_step.restype = i
    L.gb_solve_tuner_report.argtypes = [p, ctypes.c_double]; L.gb_solve_tuner_report.restype = i
    L.gb_solve_tuner_nbw.argtypes = [p, i]; L.gb_solve_tuner_nbw.restype = i
    L.gb_solve_tuner_save.argtypes = [p, ctypes.c_char_p]; L.gb_solve_tuner_save.restype = i
    L.gb_solve_tuner_load.argtypes = [ctypes.c_char_p]; L.gb_solve_tuner_load.restype = p
    L.gb_tridiag_dc_workspace_bytes.argtypes = [i]; L.gb_tridiag_dc_workspace_bytes.restype = sz
    L.gb_tridiag_dc_d.argtypes = [i, p, p, p, p, i, p, sz, p]; L.gb_tridiag_dc_d.restype = i
    L.gb_refine_syev_workspace_bytes.argtypes = [i]; L.gb_refine_syev_workspace_bytes.restype = sz
    L.gb_refine_syev_d.argtypes = [i, p, i, p, p, i, p, sz, p]; L.gb_refine_syev_d.restype = i
    L.gb_solve_mixed_workspace_bytes.argtypes = [i, i, i]; L.gb_solve_mixed_workspace_bytes.restype = sz
    L.gb_solve_mixed_d.argtypes = [i, i, i, p, i, p, p, i, i, p, sz, p]; L.gb_solve_mixed_d.restype = i
    L.gb_solve_mixed_query.argtypes = [p, i, i, i, p]; L.gb_solve_mixed_query.restype = i
    ch, dd = ctypes.c_char, ctypes.c_double
    L.gb_dgemm_workspace_bytes.argtypes = [i, i]; L.gb_dgemm_workspace_bytes.restype = sz
    L.gb_dgemm.argtypes = [ch, ch, i, i, i, dd, p, i, p, i, dd, p, i, p, sz, p]; L.gb_dgemm.restype = i
    L.gb_dsymm.argtypes = [ch, i, i, dd, p, i, p, i, dd, p, i, p, sz, p]; L.gb_dsymm.restype = i
    L.gb_dsyr2k.argtypes = [i, i, dd, p, i, p, i, dd, p, i, p]; L.gb_dsyr2k.restype = i
    L.gb_dsyrk.argtypes = [i, i, dd, p, i, dd, p, i, p]; L.gb_dsyrk.restype = i
    L.gb_dgemm_sliced_workspace_bytes.argtypes = [i, i, i]; L.gb_dgemm_sliced_workspace_bytes.restype = sz
    L.gb_dgemm_sliced.argtypes = [ch, ch, i, i, i, dd, p, i, p, i, dd, p, i, p, sz, p]
    L.gb_dgemm_sliced.restype = i
    L.gb_dgemm_fp32split.argtypes = [ch, ch, i, i, i, dd, p, i, p, i, dd, p, i, p, sz, p]
    L.gb_dgemm_fp32split.restype = i
    L.gb_dsymm_sliced_workspace_bytes.argtypes = [ch, i, i]; L.gb_dsymm_sliced_workspace_bytes.restype = sz
    L.gb_dsymm_sliced.argtypes = [ch, i, i, dd, p, i, p, i, dd, p, i, p, sz, p]; L.gb_dsymm_sliced.restype = i
    L.gb_dsyr2k_sliced_workspace_bytes.argtypes = [i, i]; L.gb_dsyr2k_sliced_workspace_bytes.restype = sz
    L.gb_dsyr2k_sliced.argtypes = [i, i, dd, p, i, p, i, dd, p, i, p, sz, p]; L.gb_dsyr2k_sliced.restype = i
    L.gb_dsyrk_sliced_workspace_bytes.argtypes = [i, i]; L.gb_dsyrk_sliced_workspace_bytes.restype = sz
    L.gb_dsyrk_sliced.argtypes = [i, i, dd, p, i, dd, p, i, p, sz, p]; L.gb_dsyrk_sliced.restype = i
    L.gb_zgemm_sliced_workspace_bytes.argtypes = [i, i, i]; L.gb_zgemm_sliced_workspace_bytes.restype = sz
    L.gb_zgemm_sliced.argtypes = [ch, i, i, i, dd, p, i, p, i, dd, p, i, p, sz, p]; L.gb_zgemm_sliced.restype = i
    L.gb_zhemm_sliced_workspace_bytes.argtypes = [i, i]; L.gb_zhemm_sliced_workspace_bytes.restype = sz
    L.gb_zhemm_sliced.argtypes = [i, i, dd, p, i, p, i, dd, p, i, p, sz, p]; L.gb_zhemm_sliced.restype = i
    L.gb_zher2k_sliced_workspace_bytes.argtypes = [i, i]; L.gb_zher2k_sliced_workspace_bytes.restype = sz
    L.gb_zher2k_sliced.argtypes = [i, i, dd, p, i, p, i, dd, p, i, p, sz, p]; L.gb_zher2k_sliced.restype = i
    _lib = L
    return L


def _p(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")



def _dp(x):
    """Pointer of an argument the library dereferences on the device: a CUDA
    tensor, a raw integer address or None.  Host tensors and arrays are
    refused here, before a kernel could read them."""
    if hasattr(x, "is_cuda") and not x.is_cuda:
        raise TypeError("expected a CUDA tensor (device memory), got a host tensor")
    if hasattr(x, "ctypes") and not hasattr(x, "data_ptr"):
        raise TypeError("expected device memory, got a host array")
    return _p(x)


def _opts(o):
    if o is None:
        return None
    if isinstance(o, gb_trans_ev_opts):
        return ctypes.byref(o)
    return ctypes.byref(gb_trans_ev_opts(**o))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def gb_hh_count(n, nbw):
    return load().gb_hh_count(n, nbw)


def gb_hh_index(n, nbw, s, k):
    return load().gb_hh_index(n, nbw, s, k)


def gb_max_nbw():
    return load().gb_max_nbw()


def gb_trans_ev_workspace_bytes(n, nbw, nev, is_complex=0, opts=None):
    return load().gb_trans_ev_workspace_bytes(n, nbw, nev, int(is_complex), _opts(opts))


def gb_trans_ev_tridi_to_band_d(n, nbw, nev, hh_v, hh_tau, Z, ldz, workspace=None, ws_bytes=0,
                                stream=None, opts=None, check=True):
    rc = load().gb_trans_ev_tridi_to_band_d(n, nbw, nev, _dp(hh_v), _dp(hh_tau), _dp(Z), ldz,
                                            _dp(workspace), ws_bytes, _stream(stream), _opts(opts))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_trans_ev_tridi_to_band_d")
    return rc


def gb_trans_ev_tridi_to_band_z(n, nbw, nev, hh_v, hh_tau, Z, ldz, workspace=None, ws_bytes=0,
                                stream=None, opts=None, check=True):
    rc = load().gb_trans_ev_tridi_to_band_z(n, nbw, nev, _dp(hh_v), _dp(hh_tau), _dp(Z), ldz,
                                            _dp(workspace), ws_bytes, _stream(stream), _opts(opts))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_trans_ev_tridi_to_band_z")
    return rc


def gb_trans_ev_host_buffer_bytes(n, nbw, nev, ldz, is_complex=0, opts=None):
    return load().gb_trans_ev_host_buffer_bytes(n, nbw, nev, ldz, int(is_complex), _opts(opts))


def gb_trans_ev_tridi_to_band_d_host(n, nbw, nev, hh_v, hh_tau, Z, ldz, dev_buf, dev_bytes,
                                     stream=None, opts=None, check=True):
    rc = load().gb_trans_ev_tridi_to_band_d_host(n, nbw, nev, _p(hh_v), _p(hh_tau), _p(Z), ldz,
                                                 _dp(dev_buf), dev_bytes, _stream(stream), _opts(opts))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_trans_ev_tridi_to_band_d_host")
    return rc


def gb_trans_ev_launch_count(n, nbw, nev, is_complex=0, opts=None):
    return load().gb_trans_ev_launch_count(n, nbw, nev, int(is_complex), _opts(opts))


def gb_trans_ev_variant(n, nbw, nev, is_complex=0, opts=None):
    return load().gb_trans_ev_variant(n, nbw, nev, int(is_complex), _opts(opts))


def gb_trans_ev_query(workspace=None, ws_bytes=0, stream=None):
    return load().gb_trans_ev_query(_dp(workspace), ws_bytes, _stream(stream))


def gb_trans_ev_tridi_to_band_d_noalloc(n, nbw, nev, hh_v, hh_tau, Z, ldz, status=None, stream=None,
                                        check=True):
    """No-allocation form for callers that cannot allocate device memory
    (scratch in a fixed device array of GB_NOALLOC_SCRATCH_BYTES)."""
    rc = load().gb_trans_ev_tridi_to_band_d_noalloc(n, nbw, nev, _dp(hh_v), _dp(hh_tau), _dp(Z), ldz,
                                                    _p(status), _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_trans_ev_tridi_to_band_d_noalloc")
    return rc


def gb_band_to_tridi_workspace_bytes(n, nbw):
    return load().gb_band_to_tridi_workspace_bytes(n, nbw)


def gb_band_to_tridi_d(n, nbw, AB, ldab, d, e, hh_v, hh_tau, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_band_to_tridi_d(n, nbw, _dp(AB), ldab, _dp(d), _dp(e), _dp(hh_v), _dp(hh_tau), _dp(workspace),
                                   ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_band_to_tridi_d")
    return rc


def gb_solve_workspace_bytes(n, nev, nbw):
    return load().gb_solve_workspace_bytes(n, nev, nbw)


def gb_solve_d(n, nev, nbw, A, lda, ev, Z, ldz, workspace, ws_bytes, stream=None, flags=0, check=True):
    rc = load().gb_solve_d(n, nev, nbw, _dp(A), lda, _dp(ev), _dp(Z), ldz, _dp(workspace), ws_bytes,
                           _stream(stream), flags)
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_d")
    return rc


def gb_solve_query(workspace, n, nev, nbw, stream=None):
    return load().gb_solve_query(_dp(workspace), n, nev, nbw, _stream(stream))


def elpa_b200_solve(n, nev, A, lda, ev, Z, ldz, check=True):
    rc = load().elpa_b200_solve(n, nev, _dp(A), lda, _dp(ev), _dp(Z), ldz)
    if check and rc != GB_OK:
        raise GbError(rc, "elpa_b200_solve")
    return rc


def gb_autotune_create(level, n, nbw, nev):
    return load().gb_autotune_create(level, n, nbw, nev)


def gb_autotune_destroy(t):
    load().gb_autotune_destroy(t)


def gb_autotune_step(t):
    """Returns the next setting to try (a gb_trans_ev_opts) or None when done."""
    o = gb_trans_ev_opts()
    rc = load().gb_autotune_step(t, ctypes.byref(o))
    if rc < 0:
        raise GbError(rc, "gb_autotune_step")
    return o if rc == 1 else None


def gb_autotune_report(t, seconds):
    return load().gb_autotune_report(t, seconds)


def gb_autotune_best(t):
    o = gb_trans_ev_opts()
    s = ctypes.c_double()
    rc = load().gb_autotune_best(t, ctypes.byref(o), ctypes.byref(s))
    return (o, s.value) if rc == GB_OK else (None, None)


def gb_autotune_progress(t):
    a, b = ctypes.c_int(), ctypes.c_int()
    load().gb_autotune_progress(t, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def gb_autotune_save(t, path):
    return load().gb_autotune_save(t, os.fsencode(path))


def gb_autotune_load(path):
    return load().gb_autotune_load(os.fsencode(path))


def gb_band_to_tridi_workspace_bytes_z(n, nbw):
    return load().gb_band_to_tridi_workspace_bytes_z(n, nbw)


def gb_band_to_tridi_z(n, nbw, AB, ldab, d, e, hh_v, hh_tau, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_band_to_tridi_z(n, nbw, _dp(AB), ldab, _dp(d), _dp(e), _dp(hh_v), _dp(hh_tau), _dp(workspace),
                                   ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_band_to_tridi_z")
    return rc


def gb_solve_workspace_bytes_z(n, nev, nbw):
    return load().gb_solve_workspace_bytes_z(n, nev, nbw)


def gb_solve_z(n, nev, nbw, A, lda, ev, Z, ldz, workspace, ws_bytes, stream=None, flags=0, check=True):
    rc = load().gb_solve_z(n, nev, nbw, _dp(A), lda, _dp(ev), _dp(Z), ldz, _dp(workspace), ws_bytes,
                           _stream(stream), flags)
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_z")
    return rc


def gb_solve_query_z(workspace, n, nev, nbw, stream=None):
    return load().gb_solve_query_z(_dp(workspace), n, nev, nbw, _stream(stream))


def gb_solve_stage_ms(stream=None):
    ms = (ctypes.c_float * 7)()
    rc = load().gb_solve_stage_ms(_stream(stream), ms)
    if rc != GB_OK:
        raise GbError(rc, "gb_solve_stage_ms")
    return dict(zip(SOLVE_STAGES, [float(x) for x in ms]))


def gb_solve_release(stream=None, all_streams=False, check=True):
    rc = load().gb_solve_release(_stream(stream), int(bool(all_streams)))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_release")
    return rc


def gb_solve_default_nbw(n):
    return load().gb_solve_default_nbw(n)


def _iarr(xs):
    return (ctypes.c_int * len(xs))(*[int(x) for x in xs])


def _parr(xs):
    return (ctypes.c_void_p * len(xs))(*[_dp(x) if x is not None else None for x in xs])


def gb_solve_batched_workspace_bytes(n, nev, nslots):
    return load().gb_solve_batched_workspace_bytes(len(n), _iarr(n), _iarr(nev), nslots)


def _handle(x):
    """Raw handle of a torch.cuda.Stream / torch.cuda.Event (or an int)."""
    if hasattr(x, "cuda_stream"):
        return x.cuda_stream
    if hasattr(x, "cuda_event"):
        if not x.cuda_event:      # torch creates the CUDA event on its first record
            x.record()
        return x.cuda_event
    return int(x)


def _harr(xs):
    return (ctypes.c_void_p * len(xs))(*[_handle(x) for x in xs]) if xs else None


def gb_solve_batched_d(n, nev, A, lda, ev, Z, ldz, workspace, ws_bytes, streams, ev_start=None, ev_end=None,
                       check=True):
    """Lists of per-problem sizes and device buffers; streams / events are
    torch.cuda.Stream / torch.cuda.Event objects or raw handles."""
    rc = load().gb_solve_batched_d(len(n), _iarr(n), _iarr(nev), _parr(A), _iarr(lda), _parr(ev), _parr(Z),
                                   _iarr(ldz), _dp(workspace), ws_bytes, len(streams), _harr(streams),
                                   _harr(ev_start), _harr(ev_end))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_batched_d")
    return rc


def gb_solve_batched_workspace_bytes_nbw(n, nev, nbw, nslots):
    return load().gb_solve_batched_workspace_bytes_nbw(len(n), _iarr(n), _iarr(nev),
                                                       _iarr(nbw) if nbw is not None else None, nslots)


def gb_solve_batched_nbw_d(n, nev, nbw, A, lda, ev, Z, ldz, workspace, ws_bytes, streams, ev_start=None,
                           ev_end=None, check=True):
    rc = load().gb_solve_batched_nbw_d(len(n), _iarr(n), _iarr(nev), _iarr(nbw) if nbw is not None else None,
                                       _parr(A), _iarr(lda), _parr(ev), _parr(Z), _iarr(ldz), _dp(workspace),
                                       ws_bytes, len(streams), _harr(streams), _harr(ev_start), _harr(ev_end))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_batched_nbw_d")
    return rc


def gb_solve_batched_staged_workspace_bytes(n, nev, nbw, nslots):
    return load().gb_solve_batched_staged_workspace_bytes(len(n), _iarr(n), _iarr(nev),
                                                          _iarr(nbw) if nbw is not None else None, nslots)


def gb_solve_batched_staged_d(n, nev, nbw, A, lda, ev, Z, ldz, workspace, ws_bytes, streams, ev_start=None,
                              ev_end=None, check=True):
    rc = load().gb_solve_batched_staged_d(len(n), _iarr(n), _iarr(nev), _iarr(nbw) if nbw is not None else None,
                                          _parr(A), _iarr(lda), _parr(ev), _parr(Z), _iarr(ldz), _dp(workspace),
                                          ws_bytes, len(streams), _harr(streams), _harr(ev_start), _harr(ev_end))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_batched_staged_d")
    return rc


def gb_solve_batched_staged_query(workspace, n, nev, nbw, streams):
    return load().gb_solve_batched_staged_query(_dp(workspace), len(n), _iarr(n), _iarr(nev),
                                                _iarr(nbw) if nbw is not None else None, len(streams), _harr(streams))


def gb_solve_stage_table_bytes(count):
    return load().gb_solve_stage_table_bytes(count)


def gb_solve_stage_front(is_complex, n, nev, nbw, A, lda, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_solve_stage_front(int(is_complex), n, nev, nbw, _dp(A), lda, _dp(workspace), ws_bytes,
                                     _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_stage_front")
    return rc


def gb_solve_stage_chase_batched(is_complex, n, nev, nbw, workspaces, table, table_bytes, stream=None, check=True):
    ws = (ctypes.c_void_p * len(workspaces))(*[_dp(w) for w in workspaces])
    rc = load().gb_solve_stage_chase_batched(int(is_complex), len(n), _iarr(n), _iarr(nev), _iarr(nbw), ws,
                                             _dp(table), table_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_stage_chase_batched")
    return rc


def gb_solve_stage_back(is_complex, n, nev, nbw, ev, Z, ldz, workspace, ws_bytes, stream=None, flags=0, check=True):
    rc = load().gb_solve_stage_back(int(is_complex), n, nev, nbw, _dp(ev), _dp(Z), ldz, _dp(workspace), ws_bytes,
                                    _stream(stream), flags)
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_stage_back")
    return rc


def gb_solve_batched_graph_create(n, nev, nbw, A, lda, ev, Z, ldz, workspace, ws_bytes, nbranches,
                                  ev_start=None, ev_end=None):
    """Returns the graph handle (an int); raises GbError on failure."""
    g = ctypes.c_void_p()
    rc = load().gb_solve_batched_graph_create(len(n), _iarr(n), _iarr(nev), _iarr(nbw) if nbw is not None else None,
                                              _parr(A), _iarr(lda), _parr(ev), _parr(Z), _iarr(ldz),
                                              _dp(workspace), ws_bytes, nbranches, _harr(ev_start), _harr(ev_end),
                                              ctypes.byref(g))
    if rc != GB_OK:
        raise GbError(rc, "gb_solve_batched_graph_create")
    return g.value


def gb_solve_batched_graph_launch(graph, stream=None, check=True):
    rc = load().gb_solve_batched_graph_launch(graph, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_batched_graph_launch")
    return rc


def gb_solve_batched_graph_nodes(graph):
    return load().gb_solve_batched_graph_nodes(graph)


def gb_solve_batched_graph_destroy(graph):
    return load().gb_solve_batched_graph_destroy(graph)


def gb_solve_tuner_create(n_lo, n_hi, classes):
    return load().gb_solve_tuner_create(n_lo, n_hi, classes)


def gb_solve_tuner_destroy(t):
    load().gb_solve_tuner_destroy(t)


def gb_solve_tuner_step(t):
    """The next trial (n, nbw), or None when every trial is handed out."""
    n, b = ctypes.c_int(), ctypes.c_int()
    rc = load().gb_solve_tuner_step(t, ctypes.byref(n), ctypes.byref(b))
    if rc == 0:
        return None
    if rc != 1:
        raise GbError(rc, "gb_solve_tuner_step")
    return n.value, b.value


def gb_solve_tuner_report(t, seconds):
    return load().gb_solve_tuner_report(t, seconds)


def gb_solve_tuner_nbw(t, n):
    return load().gb_solve_tuner_nbw(t, n)


def gb_solve_tuner_save(t, path):
    return load().gb_solve_tuner_save(t, str(path).encode())


def gb_solve_tuner_load(path):
    return load().gb_solve_tuner_load(str(path).encode())


def gb_refine_syev_workspace_bytes(n):
    return load().gb_refine_syev_workspace_bytes(n)


def gb_refine_syev_d(n, A, lda, lam, X, ldx, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_refine_syev_d(n, _dp(A), lda, _dp(lam), _dp(X), ldx, _dp(workspace), ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_refine_syev_d")
    return rc


def gb_solve_mixed_workspace_bytes(n, nev, nbw):
    return load().gb_solve_mixed_workspace_bytes(n, nev, nbw)


def gb_solve_mixed_d(n, nev, nbw, A, lda, ev, Z, ldz, refine_steps, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_solve_mixed_d(n, nev, nbw, _dp(A), lda, _dp(ev), _dp(Z), ldz, refine_steps, _dp(workspace),
                                 ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_solve_mixed_d")
    return rc


def gb_solve_mixed_query(workspace, n, nev, nbw, stream=None):
    return load().gb_solve_mixed_query(_dp(workspace), n, nev, nbw, _stream(stream))


def gb_tridiag_dc_workspace_bytes(n):
    return load().gb_tridiag_dc_workspace_bytes(n)


def gb_tridiag_dc_d(n, d, e, lam, Q, ldq, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_tridiag_dc_d(n, _dp(d), _dp(e), _dp(lam), _dp(Q), ldq, _dp(workspace), ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_tridiag_dc_d")
    return rc


def gb_dgemm_workspace_bytes(m, n):
    return load().gb_dgemm_workspace_bytes(m, n)


def _c(ch):
    return ch.encode() if isinstance(ch, str) else ch


def gb_dgemm(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace=None, ws_bytes=0,
             stream=None, check=True):
    rc = load().gb_dgemm(_c(transa), _c(transb), m, n, k, alpha, _dp(A), lda, _dp(B), ldb, beta, _dp(C), ldc,
                         _dp(workspace), ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dgemm")
    return rc


def gb_dsymm(side, m, n, alpha, S, lds, B, ldb, beta, C, ldc, workspace=None, ws_bytes=0, stream=None,
             check=True):
    rc = load().gb_dsymm(_c(side), m, n, alpha, _dp(S), lds, _dp(B), ldb, beta, _dp(C), ldc, _dp(workspace),
                         ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dsymm")
    return rc


def gb_dsyr2k(n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None, check=True):
    rc = load().gb_dsyr2k(n, k, alpha, _dp(A), lda, _dp(B), ldb, beta, _dp(C), ldc, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dsyr2k")
    return rc


def gb_dsyrk(n, k, alpha, A, lda, beta, C, ldc, stream=None, check=True):
    rc = load().gb_dsyrk(n, k, alpha, _dp(A), lda, beta, _dp(C), ldc, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dsyrk")
    return rc


def gb_dgemm_sliced_workspace_bytes(m, n, k):
    return load().gb_dgemm_sliced_workspace_bytes(m, n, k)


def gb_dgemm_sliced(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace, ws_bytes,
                    stream=None, check=True):
    rc = load().gb_dgemm_sliced(_c(transa), _c(transb), m, n, k, alpha, _dp(A), lda, _dp(B), ldb, beta, _dp(C), ldc,
                                _dp(workspace), ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dgemm_sliced")
    return rc


def gb_dgemm_fp32split(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace, ws_bytes,
                       stream=None, check=True):
    rc = load().gb_dgemm_fp32split(_c(transa), _c(transb), m, n, k, alpha, _dp(A), lda, _dp(B), ldb, beta, _dp(C),
                                   ldc, _dp(workspace), ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dgemm_fp32split")
    return rc


def gb_dsymm_sliced_workspace_bytes(side, m, n):
    return load().gb_dsymm_sliced_workspace_bytes(_c(side), m, n)


def gb_dsymm_sliced(side, m, n, alpha, S, lds, B, ldb, beta, C, ldc, workspace, ws_bytes, stream=None,
                    check=True):
    rc = load().gb_dsymm_sliced(_c(side), m, n, alpha, _dp(S), lds, _dp(B), ldb, beta, _dp(C), ldc, _dp(workspace),
                                ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dsymm_sliced")
    return rc


def gb_dsyr2k_sliced_workspace_bytes(n, k):
    return load().gb_dsyr2k_sliced_workspace_bytes(n, k)


def gb_dsyr2k_sliced(n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_dsyr2k_sliced(n, k, alpha, _dp(A), lda, _dp(B), ldb, beta, _dp(C), ldc, _dp(workspace), ws_bytes,
                                 _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dsyr2k_sliced")
    return rc


def gb_dsyrk_sliced_workspace_bytes(n, k):
    return load().gb_dsyrk_sliced_workspace_bytes(n, k)


def gb_dsyrk_sliced(n, k, alpha, A, lda, beta, C, ldc, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_dsyrk_sliced(n, k, alpha, _dp(A), lda, beta, _dp(C), ldc, _dp(workspace), ws_bytes,
                                _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_dsyrk_sliced")
    return rc


def gb_zgemm_sliced_workspace_bytes(m, n, k):
    return load().gb_zgemm_sliced_workspace_bytes(m, n, k)


def gb_zgemm_sliced(transa, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, workspace, ws_bytes, stream=None,
                    check=True):
    rc = load().gb_zgemm_sliced(_c(transa), m, n, k, alpha, _dp(A), lda, _dp(B), ldb, beta, _dp(C), ldc,
                                _dp(workspace), ws_bytes, _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_zgemm_sliced")
    return rc


def gb_zhemm_sliced_workspace_bytes(m, n):
    return load().gb_zhemm_sliced_workspace_bytes(m, n)


def gb_zhemm_sliced(m, n, alpha, S, lds, B, ldb, beta, C, ldc, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_zhemm_sliced(m, n, alpha, _dp(S), lds, _dp(B), ldb, beta, _dp(C), ldc, _dp(workspace), ws_bytes,
                                _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_zhemm_sliced")
    return rc


def gb_zher2k_sliced_workspace_bytes(n, k):
    return load().gb_zher2k_sliced_workspace_bytes(n, k)


def gb_zher2k_sliced(n, k, alpha, X, ldx, Y, ldy, beta, C, ldc, workspace, ws_bytes, stream=None, check=True):
    rc = load().gb_zher2k_sliced(n, k, alpha, _dp(X), ldx, _dp(Y), ldy, beta, _dp(C), ldc, _dp(workspace), ws_bytes,
                                 _stream(stream))
    if check and rc != GB_OK:
        raise GbError(rc, "gb_zher2k_sliced")
    return rc


def gb_status_string(status):
    try:
        return load().gb_status_string(status).decode()
    except RuntimeError:
        return f"status {status}"
