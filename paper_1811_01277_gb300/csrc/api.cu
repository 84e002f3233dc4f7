// C ABI of the library (declarations and the operation's definition are in
// include/elpa_gb300.h).  This file validates arguments, picks the kernel
// variant and launches it; it never allocates device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "trans_ev_kernels.cuh"

namespace {

constexpr int kMaxNbw = 256;       // shared-memory window kernels
constexpr int kMaxRegNbw = 64;     // register-window kernels (real case)
constexpr size_t kMaxSmem = 227 * 1024;

struct Opts {
    int variant, nb, threads, hold, column_batch, lead_tiles;
    long long spin;
};

constexpr int kTcMinN = 512;  // below it the tensor-core pipeline's per-call preparation dominates
constexpr long long kDefaultSpinPolls = 1LL << 40;  // effectively bounded by the timeout
constexpr long long kTimeoutNs = 10LL * 1000 * 1000 * 1000;

// Returns 0 or -11 (opts is the 11th argument of the device entry points).
// AUTO picks PIPELINE_TC5 (tcgen05) for real or complex data with nbw in
// {16,32,64} and n >= 512, PIPELINE for the other real cases with nbw in
// {8,16,32,64} (nb = 16, 64 columns per block) and WAVEFRONT otherwise;
// PIPELINE requested for other cases runs as WAVEFRONT, either tensor-core
// variant requested for unsupported real cases runs as PIPELINE, and for
// complex data PIPELINE_TC (real only) and an unsupported PIPELINE_TC5 run as
// WAVEFRONT.
int resolve(const gb_trans_ev_opts *o, int n, int nbw, int is_complex, Opts *r)
{
    int variant = GB_VARIANT_AUTO, nb = 0, threads = 0;
    r->spin = kDefaultSpinPolls;
    r->hold = 0;
    r->column_batch = 0;
    r->lead_tiles = 0;
    if (o) {
        if (o->variant < 0 || o->variant > GB_VARIANT_PIPELINE_TC5) return -11;
        if (o->sweeps_per_tile < 0 || o->sweeps_per_tile > 32) return -11;
        if (o->cols_per_block != 0 && o->cols_per_block != 32 && o->cols_per_block != 64 &&
            o->cols_per_block != 128)
            return -11;
        if (o->spin_limit < 0 || o->test_hold_group < 0) return -11;
        if (o->column_batch < 0 || o->column_batch > 1024) return -11;
        r->column_batch = o->column_batch;
        if (o->lead_tiles < 0 || o->lead_tiles > 65536) return -11;
        r->lead_tiles = o->lead_tiles;
        variant = o->variant;
        nb = o->sweeps_per_tile;
        threads = o->cols_per_block;
        if (o->spin_limit) r->spin = o->spin_limit;
        r->hold = o->test_hold_group;
    }
    const bool pipe_ok = !is_complex && gb::pipeline_supported(nbw);
    if (variant == GB_VARIANT_PIPELINE_TC && (is_complex || !gb::pipeline_tc_supported(nbw)))
        variant = GB_VARIANT_PIPELINE;
    if (variant == GB_VARIANT_PIPELINE_TC5 && !gb::pipeline_tc5_supported(nbw))
        variant = GB_VARIANT_PIPELINE;
    if (variant == GB_VARIANT_AUTO) {
        if (gb::pipeline_tc5_supported(nbw) && n >= kTcMinN) variant = GB_VARIANT_PIPELINE_TC5;
        else variant = pipe_ok ? GB_VARIANT_PIPELINE : GB_VARIANT_WAVEFRONT;
    }
    if (variant == GB_VARIANT_PIPELINE && !pipe_ok) variant = GB_VARIANT_WAVEFRONT;
    r->variant = variant;
    const bool smem = is_complex || nbw > kMaxRegNbw;
    r->nb = nb ? nb : (smem ? 8 : 16);
    r->threads = threads ? threads : (variant == GB_VARIANT_PIPELINE || smem ? 64 : 128);
    // the shared-memory kernels take 32 or 64 columns per block and shrink
    // them or the tile depth until the window fits
    if (smem) {
        if (r->threads > 64) r->threads = 64;
        while (gb::wavefront_smem_bytes(nbw, r->nb, r->threads, is_complex) > kMaxSmem) {
            if (r->threads > 32) r->threads = 32;
            else if (r->nb > 4) r->nb = r->nb > 8 ? 8 : 4;
            else return -2;
        }
    }
    return 0;
}

int check_common(int n, int nbw, int nev, const void *hh_v, const void *hh_tau, const void *Z,
                 int ldz, size_t elem)
{
    if (n < 1) return -1;
    if (nbw < 1 || nbw > kMaxNbw) return -2;
    if (nev < 0) return -3;
    bool has_hh = n > 1;
    if (has_hh && (!hh_v || ((uintptr_t)hh_v % elem) != 0)) return -4;
    if (has_hh && (!hh_tau || ((uintptr_t)hh_tau % elem) != 0)) return -5;
    if (nev > 0 && (!Z || ((uintptr_t)Z % elem) != 0)) return -6;
    if (ldz < n) return -7;
    return 0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

namespace gb {
thread_local KernelMarks g_kernel_marks;
}

namespace {

// Sets the caller's kernel events (if any) for one call on this thread.
struct MarksGuard {
    explicit MarksGuard(const gb_trans_ev_opts *o)
    {
        gb::g_kernel_marks.begin = o ? (cudaEvent_t)o->kernel_begin_event : nullptr;
        gb::g_kernel_marks.end = o ? (cudaEvent_t)o->kernel_end_event : nullptr;
    }
    ~MarksGuard() { gb::g_kernel_marks = gb::KernelMarks(); }
};

}  // namespace

extern "C" {

long long gb_hh_count(int n, int nbw)
{
    if (n < 1 || nbw < 1) return -1;
    return gb::hh_total(n, nbw);
}

long long gb_hh_index(int n, int nbw, int s, int k)
{
    if (n < 1 || nbw < 1 || s < 1 || s > n - 1 || k < 0 || k >= gb::sweep_count(n, nbw, s)) return -1;
    return gb::sweep_first(n, nbw, s) + k;
}

int gb_max_nbw(void) { return kMaxNbw; }

size_t gb_trans_ev_workspace_bytes(int n, int nbw, int nev, int is_complex, const gb_trans_ev_opts *opts)
{
    Opts o;
    if (n < 1 || nbw < 1 || nev < 0 || resolve(opts, n, nbw, is_complex, &o) != 0) return 0;
    if (o.variant == GB_VARIANT_PIPELINE_TC && n > 1 && nev > 0) return gb::pipeline_tc_workspace_bytes(n, nbw, nev);
    if (o.variant == GB_VARIANT_PIPELINE_TC5 && n > 1 && nev > 0)
        return gb::pipeline_tc5_workspace_bytes(n, nbw, nev, is_complex);
    if (o.variant == GB_VARIANT_PIPELINE && !is_complex && n > 1 && nev > 0)
        return gb::pipeline_workspace_bytes(n, nev, o.nb, o.threads);
    return 0;  // the wavefront variant needs no workspace
}

int gb_trans_ev_tridi_to_band_d(int n, int nbw, int nev, const double *hh_v, const double *hh_tau,
                                double *Z, int ldz, void *workspace, size_t ws_bytes, void *stream,
                                const gb_trans_ev_opts *opts)
{
    int rc = check_common(n, nbw, nev, hh_v, hh_tau, Z, ldz, sizeof(double));
    if (rc) return rc;
    Opts o;
    if ((rc = resolve(opts, n, nbw, 0, &o)) != 0) return rc;
    size_t need = gb_trans_ev_workspace_bytes(n, nbw, nev, 0, opts);
    if (need > 0 && (!workspace || ((uintptr_t)workspace % 256) != 0)) return -8;
    if (ws_bytes < need) return -9;
    if (n == 1 || nev == 0) return GB_OK;
    MarksGuard marks(opts);
    cudaError_t e;
    if (o.variant == GB_VARIANT_PIPELINE_TC5)
        e = gb::pipeline_tc5_d(n, nbw, nev, hh_v, hh_tau, Z, ldz, o.column_batch, workspace, need, o.spin, kTimeoutNs,
                               o.hold, (cudaStream_t)stream);
    else if (o.variant == GB_VARIANT_PIPELINE_TC)
        e = gb::pipeline_tc_d(n, nbw, nev, hh_v, hh_tau, Z, ldz, o.column_batch, workspace, need, o.spin, kTimeoutNs,
                              o.hold, (cudaStream_t)stream);
    else if (o.variant == GB_VARIANT_PIPELINE)
        e = gb::pipeline_d(n, nbw, nev, hh_v, hh_tau, Z, ldz, o.nb, o.threads, o.column_batch, o.lead_tiles, workspace, need,
                           o.spin, kTimeoutNs, o.hold, (cudaStream_t)stream);
    else if (nbw > kMaxRegNbw)
        e = gb::wavefront_smem_d(n, nbw, nev, hh_v, hh_tau, Z, ldz, o.nb, o.threads, (cudaStream_t)stream);
    else
        e = gb::wavefront_d(n, nbw, nev, hh_v, hh_tau, Z, ldz, o.nb, o.threads, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int gb_trans_ev_tridi_to_band_z(int n, int nbw, int nev, const double *hh_v, const double *hh_tau,
                                double *Z, int ldz, void *workspace, size_t ws_bytes, void *stream,
                                const gb_trans_ev_opts *opts)
{
    int rc = check_common(n, nbw, nev, hh_v, hh_tau, Z, ldz, 2 * sizeof(double));
    if (rc) return rc;
    Opts o;
    if ((rc = resolve(opts, n, nbw, 1, &o)) != 0) return rc;
    const size_t need = gb_trans_ev_workspace_bytes(n, nbw, nev, 1, opts);
    if (need > 0 && (!workspace || ((uintptr_t)workspace % 256) != 0)) return -8;
    if (ws_bytes < need) return -9;
    if (n == 1 || nev == 0) return GB_OK;
    MarksGuard marks(opts);
    cudaError_t e;
    if (o.variant == GB_VARIANT_PIPELINE_TC5)
        e = gb::pipeline_tc5_z(n, nbw, nev, hh_v, hh_tau, Z, ldz, o.column_batch, workspace, need, o.spin, kTimeoutNs,
                               o.hold, (cudaStream_t)stream);
    else  // the shared-memory wavefront kernel, which needs no workspace
        e = gb::wavefront_smem_z(n, nbw, nev, hh_v, hh_tau, Z, ldz, o.nb, o.threads, (cudaStream_t)stream);
    return e == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

size_t gb_trans_ev_host_buffer_bytes(int n, int nbw, int nev, int ldz, int is_complex,
                                     const gb_trans_ev_opts *opts)
{
    if (n < 1 || nbw < 1 || nev < 0 || ldz < n) return 0;
    size_t el = is_complex ? 16 : 8;
    size_t cnt = (size_t)gb::hh_total(n, nbw);
    return align256(cnt * (size_t)nbw * el) + align256(cnt * el) + align256((size_t)ldz * nev * el) +
           align256(gb_trans_ev_workspace_bytes(n, nbw, nev, is_complex, opts));
}

int gb_trans_ev_tridi_to_band_d_host(int n, int nbw, int nev, const double *hh_v, const double *hh_tau,
                                     double *Z, int ldz, void *dev_buf, size_t dev_bytes, void *stream,
                                     const gb_trans_ev_opts *opts)
{
    int rc = check_common(n, nbw, nev, hh_v, hh_tau, Z, ldz, sizeof(double));
    if (rc) return rc;
    Opts o;
    if ((rc = resolve(opts, n, nbw, 0, &o)) != 0) return rc;
    size_t need = gb_trans_ev_host_buffer_bytes(n, nbw, nev, ldz, 0, opts);
    if (!dev_buf || ((uintptr_t)dev_buf % 256) != 0) return -8;
    if (dev_bytes < need) return -9;
    if (n == 1 || nev == 0) return GB_OK;
    cudaStream_t st = (cudaStream_t)stream;
    size_t cnt = (size_t)gb::hh_total(n, nbw);
    char *p = (char *)dev_buf;
    double *d_v = (double *)p;   p += align256(cnt * nbw * sizeof(double));
    double *d_t = (double *)p;   p += align256(cnt * sizeof(double));
    double *d_z = (double *)p;   p += align256((size_t)ldz * nev * sizeof(double));
    void *d_ws = p;
    size_t zbytes = ((size_t)ldz * (nev - 1) + n) * sizeof(double);
    if (cudaMemcpyAsync(d_v, hh_v, cnt * nbw * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_t, hh_tau, cnt * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_z, Z, zbytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GB_ERR_CUDA;
    rc = gb_trans_ev_tridi_to_band_d(n, nbw, nev, d_v, d_t, d_z, ldz, d_ws,
                                     gb_trans_ev_workspace_bytes(n, nbw, nev, 0, opts), stream, opts);
    if (rc != GB_OK) return rc;
    if (cudaMemcpyAsync(Z, d_z, zbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return GB_ERR_CUDA;
    return gb_trans_ev_query(d_ws, gb_trans_ev_workspace_bytes(n, nbw, nev, 0, opts), stream);
}

int gb_trans_ev_query(const void *workspace, size_t ws_bytes, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GB_ERR_CUDA;
    if (!workspace || ws_bytes < 256) return GB_OK;
    int head[3] = {0, 0, 0};  // ticket, abort, error
    if (cudaMemcpy(head, workspace, sizeof(head), cudaMemcpyDeviceToHost) != cudaSuccess) return GB_ERR_CUDA;
    return head[2] ? head[2] : GB_OK;
}

int gb_trans_ev_variant(int n, int nbw, int nev, int is_complex, const gb_trans_ev_opts *opts)
{
    Opts o;
    if (n < 1 || nbw < 1 || nbw > kMaxNbw || nev < 0 || resolve(opts, n, nbw, is_complex, &o) != 0) return -1;
    return o.variant;
}

long long gb_trans_ev_launch_count(int n, int nbw, int nev, int is_complex, const gb_trans_ev_opts *opts)
{
    Opts o;
    if (n < 1 || nbw < 1 || nbw > kMaxNbw || nev < 0 || resolve(opts, n, nbw, is_complex, &o) != 0) return -1;
    if (n == 1 || nev == 0) return 0;
    if (o.variant == GB_VARIANT_PIPELINE) return 1;
    if (o.variant == GB_VARIANT_PIPELINE_TC || o.variant == GB_VARIANT_PIPELINE_TC5)
        return 6;  // scales, to fixed, offsets, tile prep, pipeline, back
    return gb::wavefront_launch_count(n, nbw, o.nb);
}

size_t gb_band_to_tridi_workspace_bytes(int n, int nbw)
{
    if (n < 1 || nbw < 1 || nbw > kMaxRegNbw) return 0;
    return gb::band_to_tridi_workspace_bytes(n, nbw);
}

int gb_band_to_tridi_d(int n, int nbw, const double *AB, int ldab, double *d, double *e, double *hh_v,
                       double *hh_tau, void *workspace, size_t ws_bytes, void *stream)
{
    if (n < 1) return -1;
    if (nbw < 1 || nbw > kMaxRegNbw) return -2;
    if (!AB || ((uintptr_t)AB % sizeof(double)) != 0) return -3;
    if (ldab < nbw + 1) return -4;
    if (!d || ((uintptr_t)d % sizeof(double)) != 0) return -5;
    if (n > 1 && (!e || ((uintptr_t)e % sizeof(double)) != 0)) return -6;
    if (n > 1 && (!hh_v || ((uintptr_t)hh_v % sizeof(double)) != 0)) return -7;
    if (n > 1 && (!hh_tau || ((uintptr_t)hh_tau % sizeof(double)) != 0)) return -8;
    const size_t need = gb::band_to_tridi_workspace_bytes(n, nbw);
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -9;
    if (ws_bytes < need) return -10;
    cudaError_t err = gb::band_to_tridi_d(n, nbw, AB, ldab, d, e, hh_v, hh_tau, workspace, need, kTimeoutNs,
                                          (cudaStream_t)stream);
    return err == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

size_t gb_band_to_tridi_workspace_bytes_z(int n, int nbw)
{
    if (n < 1 || nbw < 1 || nbw > kMaxRegNbw) return 0;
    return gb::band_to_tridi_workspace_bytes_z(n, nbw);
}

int gb_band_to_tridi_z(int n, int nbw, const double *AB, int ldab, double *d, double *e, double *hh_v,
                       double *hh_tau, void *workspace, size_t ws_bytes, void *stream)
{
    if (n < 1) return -1;
    if (nbw < 1 || nbw > kMaxRegNbw) return -2;
    if (!AB || ((uintptr_t)AB % 16) != 0) return -3;
    if (ldab < nbw + 1) return -4;
    if (!d || ((uintptr_t)d % sizeof(double)) != 0) return -5;
    if (n > 1 && (!e || ((uintptr_t)e % sizeof(double)) != 0)) return -6;
    if (n > 1 && (!hh_v || ((uintptr_t)hh_v % 16) != 0)) return -7;
    if (n > 1 && (!hh_tau || ((uintptr_t)hh_tau % 16) != 0)) return -8;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -9;
    if (ws_bytes < gb::band_to_tridi_workspace_bytes_z(n, nbw)) return -10;
    cudaError_t err = gb::band_to_tridi_z(n, nbw, AB, ldab, d, e, hh_v, hh_tau, workspace, kTimeoutNs,
                                          (cudaStream_t)stream);
    return err == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

const char *gb_status_string(int status)
{
    switch (status) {
    case GB_OK: return "success";
    case GB_ERR_CUDA: return "a CUDA runtime call failed";
    case GB_ERR_TIMEOUT: return "a device-side dependency wait exceeded its bound";
    case GB_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case GB_ERR_UNSUPPORTED: return "arguments valid but not supported by this build";
    case GB_ERR_NONFINITE: return "Z held NaN or Inf; those columns were returned as NaN";
    case GB_ERR_RANGE: return "a column left its fixed-point range (reflectors not orthogonal); Z unspecified";
    default: break;
    }
    if (status < 0) return "invalid argument (status -i names argument i)";
    return "unknown status";
}

}  // extern "C"
