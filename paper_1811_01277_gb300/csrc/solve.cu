// Two-stage symmetric eigensolver on one GPU (Sec. 2): full -> band ->
// tridiagonal -> eigenpairs of T -> back-transformation to band
// (trans_ev_tridi_to_band) -> back-transformation to full.
//
//   full -> band   panel p (columns j..j+b-1): Householder QR of A[j+b:, j:j+b]
//                  (panel kernels), block reflector Q_p = I - Y T Y^T, and the
//                  two-sided trailing update A2 <- Q_p^T A2 Q_p on the lower
//                  triangle: X = A2 (Y T) (SYMM), M = T^T (Y^T X),
//                  W = X - Y M / 2, A2 -= W Y^T + Y W^T (SYR2K)
//   band -> tri    gb::band_to_tridi_d (bulge chasing)
//   tridiagonal    gb::tridiag_eig_d (bisection + inverse iteration) and one
//                  Newton-Schulz step Z <- Z (3I - Z^T Z)/2
//   tri -> band    the pipeline trans_ev_tridi_to_band kernel
//   band -> full   Z <- Q_0 Q_1 ... Q_{P-1} Z, last panel first:
//                  Z_p -= Y (T (Y^T Z_p))
// The real solve's large products (SYMM, SYR2K, the band->full GEMMs, the
// Newton-Schulz SYRK and SYMM) run on the bf16 tensor cores by exact digit
// slicing (dgemm_sliced.cuh), the small ones in the DFMA kernels
// (dgemm_dfma.cuh, and the complex DFMA kernel for the complex solve).
// With GB_SOLVE_FP32_PRODUCTS the sliced products of full -> band and
// band -> full are FP32 products (operands rounded to FP32, split into three
// bf16 parts, six tensor-core products per step, FP32 accumulation).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <thread>
#include <utility>
#include <vector>

#include "elpa_gb300.h"
#include "layout.cuh"
#include "trans_ev_kernels.cuh"
#include "dgemm_dfma.cuh"
#include "dgemm_sliced.cuh"
#include "tridiag_eig.cuh"

namespace gb {

size_t tridiag_dc_workspace_bytes(int n);
cudaError_t tridiag_dc_d(int n, int nev, const double *d, const double *e, double *lam, double *Z, long long ldz,
                         void *ws, cudaStream_t st);

int panel_chunks(int m);
cudaError_t panel_qr(int m, int nb, double *P, long long lda, double *tau, double *part, cudaStream_t st);
cudaError_t panel_y_and_t_prep(int m, int nb, const double *P, long long lda, double *Y, long long ldy,
                               cudaStream_t st);
cudaError_t panel_t(int nb, const double *G, long long ldg, const double *tau, double *T, long long ldt,
                    cudaStream_t st);
cudaError_t newton_schulz_matrix(int k, double *G, long long ldg, cudaStream_t st);
cudaError_t band_from_full(int n, int b, const double *A, long long lda, double *AB, long long ldab, cudaStream_t st);

cudaError_t zpanel_qr(int m, int nb, double *P, long long lda, double *tau, double *part, cudaStream_t st);
cudaError_t zpanel_y(int m, int nb, const double *P, long long lda, double *Y, long long ldy, cudaStream_t st);
cudaError_t zpanel_t(int nb, const double *G, long long ldg, const double *tau, double *T, long long ldt,
                     cudaStream_t st);
cudaError_t zband_from_full(int n, int b, const double *A, long long lda, double *AB, long long ldab,
                            cudaStream_t st);
cudaError_t promote_real(long long rows, long long cols, const double *X, long long ldx, double *Z, long long ldz,
                         cudaStream_t st);

}  // namespace gb

namespace {

// Per-(device, stream) resources of the solvers are created on first use and
// kept until gb_solve_release or process exit; one mutex guards the caches.
std::mutex g_cache_mutex;

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Look-ahead helper per (device, caller stream): a high-priority stream on
// which the next panel is factored while the caller's stream runs the
// current trailing update, and the events that order the two.  Created on
// first use, kept until the process exits.
struct Lookahead {
    cudaStream_t side;
    cudaEvent_t start, ready, factored;
};
std::map<std::pair<int, cudaStream_t>, Lookahead> g_lookahead;
constexpr int kLookaheadMinN = 4096;

const Lookahead *lookahead(cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    auto key = std::make_pair(dev, st);
    auto it = g_lookahead.find(key);
    if (it != g_lookahead.end()) return &it->second;
    Lookahead la{};
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return nullptr;
    if (cudaStreamCreateWithPriority(&la.side, cudaStreamNonBlocking, hi) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&la.start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&la.ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&la.factored, cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    return &(g_lookahead[key] = la);
}



// Stage boundaries recorded when GB_SOLVE_RECORD_STAGES is set: events
// cached per (device, stream), created on first use.
constexpr int kStages = 7;  // full->band, band->tri, bisection, inverse iteration, orthogonalise, tri->band, band->full
std::map<std::pair<int, cudaStream_t>, cudaEvent_t *> g_stage_events;

cudaEvent_t *stage_events(cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    auto key = std::make_pair(dev, st);
    auto it = g_stage_events.find(key);
    if (it != g_stage_events.end()) return it->second;
    cudaEvent_t *ev = new cudaEvent_t[kStages + 1];
    for (int i = 0; i <= kStages; i++)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) return nullptr;
    g_stage_events[key] = ev;
    return ev;
}

// Workspace carve-up (all pieces 256-byte aligned).
struct SolveWs {
    double *Aw, *tauP, *Tall, *Y, *Y2, *YT, *X, *Pm, *M, *G, *part, *AB, *d, *e, *hv, *ht, *Ztri, *Gns, *S, *S2, *gw,
        *gw2;
    void *chase, *eig, *tev, *sl, *dc;
    size_t chase_bytes, tev_bytes, gw_elems, gw2_elems, sl_bytes, total, ptotal;
};

// More than half of the eigenvectors: divide and conquer (all of them, by
// products on the tensor cores) instead of bisection + inverse iteration
// (O(n nev) per pass, plus the orthogonalisation step).
bool use_dc(int n, int nev) { return 2LL * nev > n; }

// Products of at least this many flops go to the sliced tensor-core kernels
// (below it the extra launches of slicing cost more than they save).
constexpr double kSlicedMinFlops = 2.5e8;

bool sliced_pays(double m, double n, double k) { return 2.0 * m * n * k >= kSlicedMinFlops; }

// Workspace of the largest sliced product of a solve (0 if none is large).
size_t sliced_region_bytes(int n, int nev, int b)
{
    if (!sliced_pays(n, b, n)) return 0;
    size_t s = std::max(gb::sliced_symm_ws_bytes('L', n, b), gb::sliced_syr2k_ws_bytes(n, b));
    s = std::max(s, gb::sliced_gemm_ws_bytes(b, nev, n));
    s = std::max(s, gb::sliced_gemm_ws_bytes(n, nev, b));
    s = std::max(s, gb::sliced_syrk_ws_bytes(nev, n));
    s = std::max(s, gb::sliced_symm_ws_bytes('R', n, nev));
    return s;
}

// Split-K partials of the DFMA products (the kernels split only as far as
// this holds).
size_t gemm_work_elems(int n, int b) { return std::max((size_t)8 * n * b, (size_t)1 << 22); }

// With split set, the pieces a problem keeps from its first stage to its
// last (the panels' reflectors and T factors, the bulge chase's band and
// reflectors) go to pbase, the rest (scratch of one stage at a time) to
// base; without it everything is in base.
SolveWs carve(int n, int nev, int b, char *base, char *pbase = nullptr, bool split = false)
{
    SolveWs w{};
    size_t off = 0, poff = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    auto ptake = [&](size_t bytes) {
        if (!split) return take(bytes);
        char *p = pbase ? pbase + poff : nullptr;
        poff += a256(bytes);
        return p;
    };
    const size_t P = (size_t)(n + b - 1) / b;
    const size_t cnt = (size_t)gb::hh_total(n, b);
    const size_t nch = (size_t)gb::panel_chunks(n);
    w.Aw = (double *)ptake((size_t)n * n * 8);
    w.tauP = (double *)ptake(P * b * 8);
    w.Tall = (double *)ptake(P * b * b * 8);
    w.Y = (double *)take((size_t)n * b * 8);
    w.Y2 = (double *)take((size_t)n * b * 8);
    w.YT = (double *)take((size_t)n * b * 8);
    w.X = (double *)take((size_t)n * b * 8);
    w.Pm = (double *)take((size_t)b * b * 8);
    w.M = (double *)take((size_t)b * b * 8);
    w.G = (double *)take((size_t)b * b * 8);
    w.part = (double *)take((2 * nch + 64 * nch) * 8);
    w.AB = (double *)take((size_t)(b + 1) * n * 8);
    w.d = (double *)take((size_t)n * 8);
    w.e = (double *)take((size_t)n * 8);
    w.hv = (double *)ptake((cnt ? cnt : 1) * b * 8);
    w.ht = (double *)ptake((cnt ? cnt : 1) * 8);
    w.Ztri = (double *)take((size_t)n * nev * 8);
    w.Gns = (double *)take((size_t)nev * nev * 8);
    w.S = (double *)take((size_t)b * nev * 8);
    w.S2 = (double *)take((size_t)b * nev * 8);
    w.gw_elems = gemm_work_elems(n, b);
    w.gw = (double *)take(w.gw_elems * 8);
    w.gw2_elems = (size_t)512 * b * b;  // split-K partials of the panel's Y^T Y on the helper stream
    w.gw2 = (double *)take(w.gw2_elems * 8);
    w.chase_bytes = gb::band_to_tridi_workspace_bytes(n, b);
    w.chase = ptake(w.chase_bytes);
    w.eig = take(gb::tridiag_eig_workspace_bytes(n, nev));
    w.tev_bytes = gb_trans_ev_workspace_bytes(n, b, nev, 0, nullptr);
    w.tev = take(w.tev_bytes ? w.tev_bytes : 256);
    w.sl_bytes = sliced_region_bytes(n, nev, b);
    w.sl = w.sl_bytes ? take(w.sl_bytes) : nullptr;
    w.dc = use_dc(n, nev) ? take(gb::tridiag_dc_workspace_bytes(n)) : nullptr;
    w.total = off;
    w.ptotal = poff;
    return w;
}

// Complex workspace: complex pieces hold 2 doubles per entry.
struct SolveWsZ {
    double *Aw, *tauP, *Tall, *Y, *YT, *X, *Pm, *M, *G, *part, *AB, *d, *e, *hv, *ht, *Zre, *Gns, *Zns, *S, *S2, *gw;
    void *chase, *eig, *sl, *tev, *dc;
    size_t chase_bytes, gw_elems, sl_bytes, tev_bytes, total;
};

// complex products: 8 real flops per complex multiply-add
bool zsliced_pays(double m, double n, double k) { return 8.0 * m * n * k >= kSlicedMinFlops; }

size_t zsliced_region_bytes(int n, int nev, int b)
{
    if (!zsliced_pays(n, b, n)) return 0;
    size_t s = std::max(gb::sliced_zhemm_ws_bytes(n, b), gb::sliced_zher2k_ws_bytes(n, b));
    s = std::max(s, gb::sliced_zgemm_ws_bytes(b, nev, n));
    s = std::max(s, gb::sliced_zgemm_ws_bytes(n, nev, b));
    s = std::max(s, gb::sliced_syrk_ws_bytes(nev, n));            // the real Newton-Schulz step
    s = std::max(s, gb::sliced_symm_ws_bytes('R', n, nev));
    return s;
}

SolveWsZ carve_z(int n, int nev, int b, char *base)
{
    SolveWsZ w{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += a256(bytes);
        return p;
    };
    const size_t P = (size_t)(n + b - 1) / b;
    const size_t cnt = (size_t)gb::hh_total(n, b);
    const size_t nch = (size_t)gb::panel_chunks(n);
    w.Aw = (double *)take((size_t)n * n * 16);
    w.tauP = (double *)take(P * b * 16);
    w.Tall = (double *)take(P * b * b * 16);
    w.Y = (double *)take((size_t)n * b * 16);
    w.YT = (double *)take((size_t)n * b * 16);
    w.X = (double *)take((size_t)n * b * 16);
    w.Pm = (double *)take((size_t)b * b * 16);
    w.M = (double *)take((size_t)b * b * 16);
    w.G = (double *)take((size_t)b * b * 16);
    w.part = (double *)take((2 * nch + 128 * nch) * 8);
    w.AB = (double *)take((size_t)(b + 1) * n * 16);
    w.d = (double *)take((size_t)n * 8);
    w.e = (double *)take((size_t)n * 8);
    w.hv = (double *)take((cnt ? cnt : 1) * b * 16);
    w.ht = (double *)take((cnt ? cnt : 1) * 16);
    w.Zre = (double *)take((size_t)n * nev * 8);
    w.Gns = (double *)take((size_t)nev * nev * 8);
    w.Zns = (double *)take((size_t)n * nev * 8);
    w.S = (double *)take((size_t)b * nev * 16);
    w.S2 = (double *)take((size_t)b * nev * 16);
    w.gw_elems = gemm_work_elems(n, b);
    w.gw = (double *)take(w.gw_elems * 8);
    w.chase_bytes = gb::band_to_tridi_workspace_bytes_z(n, b);
    w.chase = take(w.chase_bytes);
    w.eig = take(gb::tridiag_eig_workspace_bytes(n, nev));
    w.sl_bytes = zsliced_region_bytes(n, nev, b);
    w.sl = w.sl_bytes ? take(w.sl_bytes) : nullptr;
    w.tev_bytes = gb_trans_ev_workspace_bytes(n, b, nev, 1, nullptr);
    w.tev = take(w.tev_bytes ? w.tev_bytes : 256);
    w.dc = use_dc(n, nev) ? take(gb::tridiag_dc_workspace_bytes(n)) : nullptr;
    w.total = off;
    return w;
}

#define GB_CU(x)                                     \
    do {                                             \
        if ((x) != cudaSuccess) return GB_ERR_CUDA;  \
    } while (0)

}  // namespace

extern "C" {

size_t gb_solve_workspace_bytes(int n, int nev, int nbw)
{
    if (n < 2 || nev < 1 || nev > n || nbw < 1 || nbw > 64 || nbw >= n) return 0;
    return carve(n, nev, nbw, nullptr).total;
}

}  // extern "C"

namespace {

// Parts of the real solve, so that the batched form can run one stage for
// every problem at once: the front (copy, full -> band, the band's
// storage), the chase, and the back (tridiagonal eigenpairs, the
// back-transformations).
constexpr int kPartFront = 1, kPartChase = 2, kPartBack = 4;

int solve_d_parts(int n, int nev, int nbw, const double *A, int lda, double *ev, double *Z, int ldz, void *workspace,
                  size_t ws_bytes, void *stream, int flags, int parts, const SolveWs *pre = nullptr)
{
    if (n < 2) return -1;
    if (nev < 1 || nev > n) return -2;
    if (nbw < 1 || nbw > 64 || nbw >= n) return -3;
    if (!A || ((uintptr_t)A % 8) != 0) return -4;
    if (lda < n) return -5;
    if (!ev || ((uintptr_t)ev % 8) != 0) return -6;
    if (!Z || ((uintptr_t)Z % 8) != 0) return -7;
    if (ldz < n) return -8;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -9;
    const int b = nbw;
    SolveWs w = pre ? *pre : carve(n, nev, b, (char *)workspace);
    if (!pre && ws_bytes < w.total) return -10;
    if (flags & ~(GB_SOLVE_FP64_EMULATED_GEMM | GB_SOLVE_RECORD_STAGES | GB_SOLVE_DFMA_PRODUCTS |
                  GB_SOLVE_TRIDIAG_BISECT | GB_SOLVE_FP32_PRODUCTS))
        return -12;
    // large products on the tensor cores unless the caller asks for DFMA
    const bool slice_ok = w.sl && !(flags & GB_SOLVE_DFMA_PRODUCTS);
    auto use_sliced = [&](double m_, double n_, double k_) { return slice_ok && sliced_pays(m_, n_, k_); };
    // the sliced products of full -> band and band -> full: FP32 products
    // (the FP32 split) for the low-precision half of the mixed-precision solve
    const int pd = (flags & GB_SOLVE_FP32_PRODUCTS) ? gb::kSplitPlanes : gb::kSlices;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t *sev = nullptr;
    if (flags & GB_SOLVE_RECORD_STAGES) {
        sev = stage_events(st);
        if (!sev) return GB_ERR_CUDA;
    }
#define GB_STAGE(i)                                                        \
    do {                                                                   \
        if (sev && cudaEventRecord(sev[i], st) != cudaSuccess) return GB_ERR_CUDA; \
    } while (0)
    const long long ldw = n;
    const int P = b < n ? (n - 1) / b : 0;  // panels of full -> band
    if (parts & kPartFront) {

    // ---- full -> band, with look-ahead: panel p+1 is factored on the helper
    // stream as soon as its columns have received panel p's update, while
    // the caller's stream applies the rest of that update (the rank-2b update
    // of the trailing lower triangle, the bulk of the flops)
    GB_STAGE(0);
    GB_CU(cudaMemcpy2DAsync(w.Aw, (size_t)n * 8, A, (size_t)lda * 8, (size_t)n * 8, n, cudaMemcpyDeviceToDevice, st));
    // small problems factor their panels in line: the helper stream would
    // gain little there and would double the streams concurrent solves use
    // (streams beyond the device's hardware queues share them)
    const bool ahead = n >= kLookaheadMinN;
    const Lookahead *la = ahead ? lookahead(st) : nullptr;
    if (ahead && !la) return GB_ERR_CUDA;
    const cudaStream_t fst = ahead ? la->side : st;  // stream that factors panels
    double *Ybuf[2] = {w.Y, w.Y2};
    auto factor = [&](int p) -> cudaError_t {  // on the panel stream
        const int j = p * b, m = n - j - b;
        double *panel = w.Aw + (long long)j * ldw + (j + b);
        double *Yp = Ybuf[p & 1];
        cudaError_t e;
        if ((e = gb::panel_qr(m, b, panel, ldw, w.tauP + (long long)p * b, w.part, fst)) != cudaSuccess) return e;
        if ((e = gb::panel_y_and_t_prep(m, b, panel, ldw, Yp, m, fst)) != cudaSuccess) return e;
        if ((e = gb::dfma_gemm('T', 'N', b, b, m, 1.0, Yp, m, Yp, m, 0.0, w.G, b, w.gw2, w.gw2_elems, fst)) !=
            cudaSuccess)
            return e;
        if ((e = gb::panel_t(b, w.G, b, w.tauP + (long long)p * b, w.Tall + (long long)p * b * b, b, fst)) !=
            cudaSuccess)
            return e;
        return ahead ? cudaEventRecord(la->factored, fst) : cudaSuccess;
    };
    int pp = 0;
    if (b < n) {
        if (ahead) {
            GB_CU(cudaEventRecord(la->start, st));
            GB_CU(cudaStreamWaitEvent(la->side, la->start, 0));
        }
        GB_CU(factor(0));
    }
    for (int j = 0; j + b < n; j += b, pp++) {
        const int m = n - j - b;
        double *A2 = w.Aw + (long long)(j + b) * ldw + (j + b);
        const double *T = w.Tall + (long long)pp * b * b;
        const double *Yp = Ybuf[pp & 1];
        if (ahead) GB_CU(cudaStreamWaitEvent(st, la->factored, 0));
        GB_CU(gb::dfma_gemm('N', 'N', m, b, b, 1.0, Yp, m, T, b, 0.0, w.YT, m, w.gw, w.gw_elems, st));
        // only the lower triangle of A2 is kept: X = A2 (Y T) (symmetric
        // product), W = X - Y M / 2, then A2 -= W Y^T + Y W^T on the lower triangle
        if (use_sliced(m, b, m))
            GB_CU(gb::sliced_dsymm('L', m, b, 1.0, A2, ldw, w.YT, m, 0.0, w.X, m, w.sl, st, pd));
        else
            GB_CU(gb::dfma_symm('L', m, b, 1.0, A2, ldw, w.YT, m, 0.0, w.X, m, w.gw, w.gw_elems, st));
        GB_CU(gb::dfma_gemm('T', 'N', b, b, m, 1.0, Yp, m, w.X, m, 0.0, w.Pm, b, w.gw, w.gw_elems, st));
        GB_CU(gb::dfma_gemm('T', 'N', b, b, b, 1.0, T, b, w.Pm, b, 0.0, w.M, b, w.gw, w.gw_elems, st));
        GB_CU(gb::dfma_gemm('N', 'N', m, b, b, -0.5, Yp, m, w.M, b, 1.0, w.X, m, w.gw, w.gw_elems, st));
        if (m > b) {
            // the next panel's columns first (all m rows; the upper triangle
            // of their diagonal block is updated too and never read), then
            // the next panel is factored on the helper stream while the rest
            // of the trailing update runs here
            GB_CU(gb::dfma_gemm('N', 'T', m, b, b, -1.0, w.X, m, Yp, m, 1.0, A2, ldw, w.gw, w.gw_elems, st));
            GB_CU(gb::dfma_gemm('N', 'T', m, b, b, -1.0, Yp, m, w.X, m, 1.0, A2, ldw, w.gw, w.gw_elems, st));
            if (ahead) {
                GB_CU(cudaEventRecord(la->ready, st));
                GB_CU(cudaStreamWaitEvent(la->side, la->ready, 0));
            }
            GB_CU(factor(pp + 1));
            if (use_sliced(m - b, m - b, b))
                GB_CU(gb::sliced_dsyr2k_lower(m - b, b, -1.0, w.X + b, m, Yp + b, m, 1.0, A2 + (long long)b * ldw + b,
                                              ldw, w.sl, st, pd));
            else
                GB_CU(gb::dfma_syr2k_lower(m - b, b, -1.0, w.X + b, m, Yp + b, m, 1.0, A2 + (long long)b * ldw + b,
                                           ldw, st));
        } else {
            if (use_sliced(m, m, b))
                GB_CU(gb::sliced_dsyr2k_lower(m, b, -1.0, w.X, m, Yp, m, 1.0, A2, ldw, w.sl, st, pd));
            else
                GB_CU(gb::dfma_syr2k_lower(m, b, -1.0, w.X, m, Yp, m, 1.0, A2, ldw, st));
        }
    }
    GB_CU(gb::band_from_full(n, b, w.Aw, ldw, w.AB, b + 1, st));
    }

    // ---- band -> tridiagonal
    if (parts & kPartChase) {
        GB_STAGE(1);
        GB_CU(gb::band_to_tridi_d(n, b, w.AB, b + 1, w.d, w.e, w.hv, w.ht, w.chase, w.chase_bytes,
                                  10LL * 1000 * 1000 * 1000, st));
    }
    if (!(parts & kPartBack)) return GB_OK;

    // ---- eigenpairs of T: divide and conquer straight into Z, or bisection,
    // inverse iteration and one Newton-Schulz orthogonalisation step
    GB_STAGE(2);
    if (w.dc && !(flags & GB_SOLVE_TRIDIAG_BISECT)) {
        GB_CU(gb::tridiag_dc_d(n, nev, w.d, w.e, ev, Z, ldz, w.dc, st));
        GB_STAGE(3);
        GB_STAGE(4);
    } else {
        GB_CU(gb::tridiag_bisect_d(n, nev, w.d, w.e, ev, w.eig, st));
        GB_STAGE(3);
        GB_CU(gb::tridiag_invit_d(n, nev, w.d, w.e, ev, w.Ztri, n, w.eig, st));
        GB_STAGE(4);
        // G = Z^T Z (lower triangle), M = (3I - G)/2, Z <- Z M
        if (use_sliced(nev, nev, n))
            GB_CU(gb::sliced_dsyrk_lower_t(nev, n, 1.0, w.Ztri, n, 0.0, w.Gns, nev, w.sl, st));
        else
            GB_CU(gb::dfma_syrk_lower_t(nev, n, 1.0, w.Ztri, n, 0.0, w.Gns, nev, st));
        GB_CU(gb::newton_schulz_matrix(nev, w.Gns, nev, st));
        if (use_sliced(n, nev, nev))
            GB_CU(gb::sliced_dsymm('R', n, nev, 1.0, w.Gns, nev, w.Ztri, n, 0.0, Z, ldz, w.sl, st));
        else
            GB_CU(gb::dfma_symm('R', n, nev, 1.0, w.Gns, nev, w.Ztri, n, 0.0, Z, ldz, w.gw, w.gw_elems, st));
    }

    // ---- tridiagonal -> band (the hot path)
    GB_STAGE(5);
    int rc = gb_trans_ev_tridi_to_band_d(n, b, nev, w.hv, w.ht, Z, ldz, w.tev, w.tev_bytes, stream, nullptr);
    if (rc != GB_OK) return rc;

    // ---- band -> full, last panel first
    GB_STAGE(6);
    for (int p = P - 1; p >= 0; p--) {
        const int j = p * b, m = n - j - b;
        const double *panel = w.Aw + (long long)j * ldw + (j + b);
        const double *T = w.Tall + (long long)p * b * b;
        double *Zr = Z + (j + b);
        GB_CU(gb::panel_y_and_t_prep(m, b, panel, ldw, w.Y, m, st));
        if (use_sliced(b, nev, m))
            GB_CU(gb::sliced_dgemm('T', 'N', b, nev, m, 1.0, w.Y, m, Zr, ldz, 0.0, w.S, b, w.sl, st, pd));
        else
            GB_CU(gb::dfma_gemm('T', 'N', b, nev, m, 1.0, w.Y, m, Zr, ldz, 0.0, w.S, b, w.gw, w.gw_elems, st));
        GB_CU(gb::dfma_gemm('N', 'N', b, nev, b, 1.0, T, b, w.S, b, 0.0, w.S2, b, w.gw, w.gw_elems, st));
        if (use_sliced(m, nev, b))
            GB_CU(gb::sliced_dgemm('N', 'N', m, nev, b, -1.0, w.Y, m, w.S2, b, 1.0, Zr, ldz, w.sl, st, pd));
        else
            GB_CU(gb::dfma_gemm('N', 'N', m, nev, b, -1.0, w.Y, m, w.S2, b, 1.0, Zr, ldz, w.gw, w.gw_elems, st));
    }
    GB_STAGE(7);
#undef GB_STAGE
    GB_CU(cudaGetLastError());
    return GB_OK;
}

}  // namespace

extern "C" {

int gb_solve_d(int n, int nev, int nbw, const double *A, int lda, double *ev, double *Z, int ldz, void *workspace,
               size_t ws_bytes, void *stream, int flags)
{
    return solve_d_parts(n, nev, nbw, A, lda, ev, Z, ldz, workspace, ws_bytes, stream, flags,
                         kPartFront | kPartChase | kPartBack);
}

size_t gb_solve_workspace_bytes_z(int n, int nev, int nbw)
{
    if (n < 2 || nev < 1 || nev > n || nbw < 1 || nbw > 64 || nbw >= n) return 0;
    return carve_z(n, nev, nbw, nullptr).total;
}

}  // extern "C"

namespace {

int solve_z_parts(int n, int nev, int nbw, const double *A, int lda, double *ev, double *Z, int ldz, void *workspace,
                  size_t ws_bytes, void *stream, int flags, int parts)
{
    if (n < 2) return -1;
    if (nev < 1 || nev > n) return -2;
    if (nbw < 1 || nbw > 64 || nbw >= n) return -3;
    if (!A || ((uintptr_t)A % 16) != 0) return -4;
    if (lda < n) return -5;
    if (!ev || ((uintptr_t)ev % 8) != 0) return -6;
    if (!Z || ((uintptr_t)Z % 16) != 0) return -7;
    if (ldz < n) return -8;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -9;
    const int b = nbw;
    SolveWsZ w = carve_z(n, nev, b, (char *)workspace);
    if (ws_bytes < w.total) return -10;
    if (flags & ~(GB_SOLVE_FP64_EMULATED_GEMM | GB_SOLVE_RECORD_STAGES | GB_SOLVE_DFMA_PRODUCTS |
                  GB_SOLVE_TRIDIAG_BISECT))
        return -12;
    // large products sliced on the tensor cores unless the caller asks for
    // the FP64 path; every other product (the b x b panel products, the
    // small-k updates, and the large ones on the FP64 path) in this
    // library's complex DFMA kernel
    const bool zslice_ok = w.sl && !(flags & GB_SOLVE_DFMA_PRODUCTS);
    auto use_zsliced = [&](double m_, double n_, double k_) { return zslice_ok && zsliced_pays(m_, n_, k_); };
    cudaStream_t st = (cudaStream_t)stream;
    const double2 one{1.0, 0.0}, zero{0.0, 0.0}, mone{-1.0, 0.0}, mhalf{-0.5, 0.0};
    const long long ldw = n;
    typedef double2 C;
    auto zg = [&](char oa, char ob, int m_, int n_, int k_, double2 al, const C *A_, long long la, const C *B_,
                  long long lb, double2 be, C *C_, long long lc, int lower) {
        return gb::dfma_zgemm(oa, ob, m_, n_, k_, al, (const double *)A_, la, (const double *)B_, lb, be,
                              (double *)C_, lc, lower, w.gw, w.gw_elems, st);
    };
    C *Aw = (C *)w.Aw, *Y = (C *)w.Y, *YT = (C *)w.YT, *X = (C *)w.X, *Pm = (C *)w.Pm, *M = (C *)w.M,
      *G = (C *)w.G, *S = (C *)w.S, *S2 = (C *)w.S2, *Zc = (C *)Z;

    const int P = b < n ? (n - 1) / b : 0;  // panels of full -> band
    if (parts & kPartFront) {
    // ---- full -> band: A2 <- Q^H A2 Q, Q = I - Y T Y^H
    GB_CU(cudaMemcpy2DAsync(Aw, (size_t)n * 16, A, (size_t)lda * 16, (size_t)n * 16, n, cudaMemcpyDeviceToDevice, st));
    int pp = 0;
    for (int j = 0; j + b < n; j += b, pp++) {
        const int m = n - j - b;
        C *panel = Aw + (long long)j * ldw + (j + b);
        C *A2 = Aw + (long long)(j + b) * ldw + (j + b);
        double *tau = w.tauP + (long long)pp * b * 2;
        C *T = (C *)(w.Tall + (long long)pp * b * b * 2);
        GB_CU(gb::zpanel_qr(m, b, (double *)panel, ldw, tau, w.part, st));
        GB_CU(gb::zpanel_y(m, b, (const double *)panel, ldw, (double *)Y, m, st));
        GB_CU(zg('C', 'N', b, b, m, one, Y, m, Y, m, zero, G, b, 0));
        GB_CU(gb::zpanel_t(b, (const double *)G, b, tau, (double *)T, b, st));
        GB_CU(zg('N', 'N', m, b, b, one, Y, m, T, b, zero, YT, m, 0));
        if (use_zsliced(m, b, m))
            GB_CU(gb::sliced_zhemm_left(m, b, 1.0, (const double *)A2, ldw, (const double *)YT, m, 0.0, (double *)X, m,
                                        w.sl, st));
        else
            GB_CU(zg('H', 'N', m, b, m, one, A2, ldw, YT, m, zero, X, m, 0));
        GB_CU(zg('C', 'N', b, b, m, one, Y, m, X, m, zero, Pm, b, 0));
        GB_CU(zg('C', 'N', b, b, b, one, T, b, Pm, b, zero, M, b, 0));
        GB_CU(zg('N', 'N', m, b, b, mhalf, Y, m, M, b, one, X, m, 0));
        // lower triangle of A2 -= X Y^H + Y X^H (Hermitian rank-2b update)
        if (use_zsliced(m, m, b)) {
            GB_CU(gb::sliced_zher2k_lower(m, b, -1.0, (const double *)X, m, (const double *)Y, m, 1.0, (double *)A2,
                                          ldw, w.sl, st));
        } else {
            GB_CU(zg('N', 'C', m, m, b, mone, X, m, Y, m, one, A2, ldw, 1));
            GB_CU(zg('N', 'C', m, m, b, mone, Y, m, X, m, one, A2, ldw, 1));
        }
    }
    GB_CU(gb::zband_from_full(n, b, (const double *)Aw, ldw, w.AB, b + 1, st));
    }

    // ---- band -> tridiagonal (complex reflectors, real T)
    if (parts & kPartChase)
        GB_CU(gb::band_to_tridi_z(n, b, w.AB, b + 1, w.d, w.e, w.hv, w.ht, w.chase, 10LL * 1000 * 1000 * 1000, st));
    if (!(parts & kPartBack)) return GB_OK;

    // ---- real tridiagonal eigenpairs (divide and conquer, or bisection,
    // inverse iteration and Newton-Schulz), promoted to complex Z
    if (w.dc && !(flags & GB_SOLVE_TRIDIAG_BISECT)) {
        GB_CU(gb::tridiag_dc_d(n, nev, w.d, w.e, ev, w.Zns, n, w.dc, st));
    } else {
        GB_CU(gb::tridiag_eig_d(n, nev, w.d, w.e, ev, w.Zre, n, w.eig, st));
        if (zslice_ok && sliced_pays(nev, nev, n))
            GB_CU(gb::sliced_dsyrk_lower_t(nev, n, 1.0, w.Zre, n, 0.0, w.Gns, nev, w.sl, st));
        else
            GB_CU(gb::dfma_syrk_lower_t(nev, n, 1.0, w.Zre, n, 0.0, w.Gns, nev, st));
        GB_CU(gb::newton_schulz_matrix(nev, w.Gns, nev, st));
        if (zslice_ok && sliced_pays(n, nev, nev))
            GB_CU(gb::sliced_dsymm('R', n, nev, 1.0, w.Gns, nev, w.Zre, n, 0.0, w.Zns, n, w.sl, st));
        else
            GB_CU(gb::dfma_symm('R', n, nev, 1.0, w.Gns, nev, w.Zre, n, 0.0, w.Zns, n, w.gw, w.gw_elems, st));
    }
    GB_CU(gb::promote_real(n, nev, w.Zns, n, Z, ldz, st));

    // ---- tridiagonal -> band (complex back-transformation)
    int rc = gb_trans_ev_tridi_to_band_z(n, b, nev, w.hv, w.ht, Z, ldz, w.tev, w.tev_bytes, stream, nullptr);
    if (rc != GB_OK) return rc;

    // ---- band -> full: Z_p -= Y (T (Y^H Z_p)), last panel first
    for (int p = P - 1; p >= 0; p--) {
        const int j = p * b, m = n - j - b;
        const C *panel = Aw + (long long)j * ldw + (j + b);
        const C *T = (const C *)(w.Tall + (long long)p * b * b * 2);
        C *Zr = Zc + (j + b);
        GB_CU(gb::zpanel_y(m, b, (const double *)panel, ldw, (double *)Y, m, st));
        if (use_zsliced(b, nev, m))
            GB_CU(gb::sliced_zgemm('C', b, nev, m, 1.0, (const double *)Y, m, (const double *)Zr, ldz, 0.0,
                                   (double *)S, b, w.sl, st));
        else
            GB_CU(zg('C', 'N', b, nev, m, one, Y, m, Zr, ldz, zero, S, b, 0));
        GB_CU(zg('N', 'N', b, nev, b, one, T, b, S, b, zero, S2, b, 0));
        if (use_zsliced(m, nev, b))
            GB_CU(gb::sliced_zgemm('N', m, nev, b, -1.0, (const double *)Y, m, (const double *)S2, b, 1.0,
                                   (double *)Zr, ldz, w.sl, st));
        else
            GB_CU(zg('N', 'N', m, nev, b, mone, Y, m, S2, b, one, Zr, ldz, 0));
    }
    GB_CU(cudaGetLastError());
    return GB_OK;
}

}  // namespace

extern "C" {

int gb_solve_z(int n, int nev, int nbw, const double *A, int lda, double *ev, double *Z, int ldz, void *workspace,
               size_t ws_bytes, void *stream, int flags)
{
    return solve_z_parts(n, nev, nbw, A, lda, ev, Z, ldz, workspace, ws_bytes, stream, flags,
                         kPartFront | kPartChase | kPartBack);
}

// ---- the solve in three calls, so that a server can run one stage for
// several requests at once (the bulge chases in one launch)

size_t gb_solve_stage_table_bytes(int count) { return count >= 1 ? gb::chase_batched_table_bytes(count) : 0; }

int gb_solve_stage_front(int is_complex, int n, int nev, int nbw, const double *A, int lda, void *workspace,
                         size_t ws_bytes, void *stream)
{
    const cudaStream_t st = (cudaStream_t)stream;
    // ev and Z are not touched by the front; any aligned non-null pointer passes the checks
    double *dummy = (double *)workspace;
    int rc;
    if (is_complex) {
        rc = solve_z_parts(n, nev, nbw, A, lda, dummy, dummy, n, workspace, ws_bytes, stream, 0, kPartFront);
        if (rc != GB_OK) return rc;
        const SolveWsZ w = carve_z(n, nev, nbw, (char *)workspace);
        return gb::band_to_tridi_prepare_z(n, nbw, w.AB, nbw + 1, w.chase, st) == cudaSuccess ? GB_OK : GB_ERR_CUDA;
    }
    rc = solve_d_parts(n, nev, nbw, A, lda, dummy, dummy, n, workspace, ws_bytes, stream, 0, kPartFront);
    if (rc != GB_OK) return rc;
    const SolveWs w = carve(n, nev, nbw, (char *)workspace);
    return gb::band_to_tridi_prepare_d(n, nbw, w.AB, nbw + 1, w.chase, st) == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

int gb_solve_stage_chase_batched(int is_complex, int count, const int *n, const int *nev, const int *nbw,
                                 void *const *workspaces, void *table, size_t table_bytes, void *stream)
{
    if (count < 1) return -2;
    if (!n || !nev || !nbw) return -3;
    if (!workspaces) return -6;
    if (!table || ((uintptr_t)table % 256) != 0) return -7;
    if (table_bytes < gb_solve_stage_table_bytes(count)) return -8;
    std::vector<void *> cws((size_t)count);
    std::vector<double *> hv((size_t)count), ht((size_t)count);
    for (int i = 0; i < count; i++) {
        if (!workspaces[i]) return -6;
        if (is_complex) {
            const SolveWsZ w = carve_z(n[i], nev[i], nbw[i], (char *)workspaces[i]);
            cws[i] = w.chase;
            hv[i] = w.hv;
            ht[i] = w.ht;
        } else {
            const SolveWs w = carve(n[i], nev[i], nbw[i], (char *)workspaces[i]);
            cws[i] = w.chase;
            hv[i] = w.hv;
            ht[i] = w.ht;
        }
    }
    const cudaStream_t st = (cudaStream_t)stream;
    if (gb::band_to_tridi_chase_batched_upload_d(count, n, nbw, cws.data(), hv.data(), ht.data(), table, st) !=
        cudaSuccess)
        return GB_ERR_CUDA;
    return gb::band_to_tridi_chase_batched(count, n, nbw, table, 10LL * 1000 * 1000 * 1000, st, is_complex) == cudaSuccess
               ? GB_OK
               : GB_ERR_CUDA;
}

int gb_solve_stage_back(int is_complex, int n, int nev, int nbw, double *ev, double *Z, int ldz, void *workspace,
                        size_t ws_bytes, void *stream, int flags)
{
    const cudaStream_t st = (cudaStream_t)stream;
    if (n < 2 || nbw < 1 || nbw > 64 || nbw >= n || nev < 1 || nev > n) return -2;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -7;
    if (is_complex) {
        const SolveWsZ w = carve_z(n, nev, nbw, (char *)workspace);
        if (ws_bytes < w.total) return -8;
        if (gb::band_to_tridi_finish_z(n, nbw, w.chase, w.d, w.e, st) != cudaSuccess) return GB_ERR_CUDA;
        return solve_z_parts(n, nev, nbw, (const double *)workspace, n, ev, Z, ldz, workspace, ws_bytes, stream,
                             flags, kPartBack);
    }
    const SolveWs w = carve(n, nev, nbw, (char *)workspace);
    if (ws_bytes < w.total) return -8;
    if (gb::band_to_tridi_finish_d(n, nbw, w.chase, w.d, w.e, st) != cudaSuccess) return GB_ERR_CUDA;
    return solve_d_parts(n, nev, nbw, (const double *)workspace, n, ev, Z, ldz, workspace, ws_bytes, stream, flags,
                         kPartBack);
}

int gb_solve_query_z(const void *workspace, int n, int nev, int nbw, void *stream)
{
    if (!workspace) return -1;
    SolveWsZ w = carve_z(n, nev, nbw, (char *)workspace);
    int rc = gb_trans_ev_query(w.chase, w.chase_bytes, stream);
    if (rc != GB_OK) return rc;
    return gb_trans_ev_query(w.tev, w.tev_bytes, stream);
}

int gb_solve_release(void *stream, int all_streams)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    const cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    auto match = [&](const std::pair<int, cudaStream_t> &k) {
        return all_streams || (k.first == dev && k.second == st);
    };
    int rc = GB_OK;
    auto on_device = [&](int d) {  // resources are destroyed with their own device current
        if (cudaSetDevice(d) != cudaSuccess) rc = GB_ERR_CUDA;
    };
    for (auto it = g_lookahead.begin(); it != g_lookahead.end();) {
        if (!match(it->first)) {
            ++it;
            continue;
        }
        on_device(it->first.first);
        const Lookahead &la = it->second;
        if (cudaStreamSynchronize(la.side) != cudaSuccess) rc = GB_ERR_CUDA;
        cudaEventDestroy(la.start);
        cudaEventDestroy(la.ready);
        cudaEventDestroy(la.factored);
        if (cudaStreamDestroy(la.side) != cudaSuccess) rc = GB_ERR_CUDA;
        it = g_lookahead.erase(it);
    }
    for (auto it = g_stage_events.begin(); it != g_stage_events.end();) {
        if (!match(it->first)) {
            ++it;
            continue;
        }
        on_device(it->first.first);
        for (int i = 0; i <= kStages; i++) cudaEventDestroy(it->second[i]);
        delete[] it->second;
        it = g_stage_events.erase(it);
    }
    if (cudaSetDevice(dev) != cudaSuccess) rc = GB_ERR_CUDA;
    return rc;
}

int gb_solve_stage_ms(void *stream, float *ms)
{
    if (!ms) return -2;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t *sev = stage_events(st);
    if (!sev) return GB_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GB_ERR_CUDA;
    for (int i = 0; i < kStages; i++)
        if (cudaEventElapsedTime(&ms[i], sev[i], sev[i + 1]) != cudaSuccess) return GB_ERR_CUDA;
    return GB_OK;
}

}  // extern "C"

namespace gb {

cudaError_t solve_status_copy(const void *ws, int n, int nev, int nbw, void *dst, cudaStream_t st)
{
    SolveWs w = carve(n, nev, nbw, (char *)ws);
    const void *src[2] = {w.chase, w.tev};
    const size_t bytes[2] = {w.chase_bytes, w.tev_bytes};
    for (int i = 0; i < 2; i++) {
        char *d = (char *)dst + 256 * i;
        const cudaError_t e = bytes[i] >= 256 ? cudaMemcpyAsync(d, src[i], 16, cudaMemcpyDeviceToDevice, st)
                                              : cudaMemsetAsync(d, 0, 16, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gb

extern "C" {

int gb_solve_query(const void *workspace, int n, int nev, int nbw, void *stream)
{
    if (!workspace) return -1;
    SolveWs w = carve(n, nev, nbw, (char *)workspace);
    int rc = gb_trans_ev_query(w.chase, w.chase_bytes, stream);
    if (rc != GB_OK) return rc;
    return gb_trans_ev_query(w.tev, w.tev_bytes, stream);
}

int gb_solve_default_nbw(int n)
{
    if (n < 2) return -1;
    const int b = n >= 1024 ? 64 : 32;
    return b < n ? b : n - 1;
}

size_t gb_solve_batched_workspace_bytes_nbw(int count, const int *n, const int *nev, const int *nbw, int nslots)
{
    if (count < 1 || !n || !nev || nslots < 1) return 0;
    size_t slot = 0;
    for (int i = 0; i < count; i++) {
        const size_t b = gb_solve_workspace_bytes(n[i], nev[i], nbw ? nbw[i] : gb_solve_default_nbw(n[i]));
        if (b == 0) return 0;
        if (b > slot) slot = b;
    }
    return a256(slot) * (size_t)nslots;
}

size_t gb_solve_batched_workspace_bytes(int count, const int *n, const int *nev, int nslots)
{
    return gb_solve_batched_workspace_bytes_nbw(count, n, nev, nullptr, nslots);
}

int gb_solve_batched_nbw_d(int count, const int *n, const int *nev, const int *nbw, const double *const *A,
                           const int *lda, double *const *ev, double *const *Z, const int *ldz, void *workspace,
                           size_t ws_bytes, int nslots, void *const *streams, void *const *ev_start,
                           void *const *ev_end)
{
    if (count < 1) return -1;
    if (!n || !nev || !A || !lda || !ev || !Z || !ldz) return -2;
    if (nslots < 1 || !streams) return -12;
    const size_t need = gb_solve_batched_workspace_bytes_nbw(count, n, nev, nbw, nslots);
    if (need == 0) return -2;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -10;
    if (ws_bytes < need) return -11;
    const size_t slot = need / (size_t)nslots;
    // One host thread per slot issues that slot's problems in order: a solve
    // is thousands of launches, and a single issuing thread would block on
    // one stream's full launch queue while the other streams run dry.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    const int nthreads = nslots < count ? nslots : count;
    std::vector<int> rcs(nthreads, GB_OK);
    auto issue = [&](int s) {
        if (cudaSetDevice(dev) != cudaSuccess) {
            rcs[s] = GB_ERR_CUDA;
            return;
        }
        cudaStream_t st = (cudaStream_t)streams[s];
        for (int i = s; i < count; i += nslots) {
            if (ev_start && cudaEventRecord((cudaEvent_t)ev_start[i], st) != cudaSuccess) {
                rcs[s] = GB_ERR_CUDA;
                return;
            }
            const int b = nbw ? nbw[i] : gb_solve_default_nbw(n[i]);
            const int rc = gb_solve_d(n[i], nev[i], b, A[i], lda[i], ev[i], Z[i], ldz[i], (char *)workspace + s * slot,
                                      slot, (void *)st, 0);
            if (rc != GB_OK) {
                rcs[s] = rc;
                return;
            }
            if (ev_end && cudaEventRecord((cudaEvent_t)ev_end[i], st) != cudaSuccess) {
                rcs[s] = GB_ERR_CUDA;
                return;
            }
        }
    };
    std::vector<std::thread> pool;
    for (int s = 1; s < nthreads; s++) pool.emplace_back(issue, s);
    issue(0);
    for (auto &t : pool) t.join();
    for (int rc : rcs)
        if (rc != GB_OK) return rc;
    return GB_OK;
}

int gb_solve_batched_d(int count, const int *n, const int *nev, const double *const *A, const int *lda,
                       double *const *ev, double *const *Z, const int *ldz, void *workspace, size_t ws_bytes,
                       int nslots, void *const *streams, void *const *ev_start, void *const *ev_end)
{
    const int rc = gb_solve_batched_nbw_d(count, n, nev, nullptr, A, lda, ev, Z, ldz, workspace, ws_bytes, nslots,
                                          streams, ev_start, ev_end);
    // the argument numbers of this signature (no nbw array)
    return rc < -2 ? rc + 1 : rc;
}

}  // extern "C"

// The batched form as one CUDA graph: every solve of the batch issued once,
// by stream capture, into nbranches parallel branches.
struct gb_solve_graph {
    int device = 0;
    cudaStream_t origin = nullptr;
    std::vector<cudaStream_t> branch;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    long long nodes = 0;
};

namespace {

void destroy_graph_object(gb_solve_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    for (cudaStream_t s : g->branch) gb_solve_release((void *)s, 0);
    for (cudaStream_t s : g->branch)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : g->join)
        if (e) cudaEventDestroy(e);
    if (g->fork) cudaEventDestroy(g->fork);
    if (g->origin) cudaStreamDestroy(g->origin);
    delete g;
}

}  // namespace

extern "C" {

int gb_solve_batched_graph_create(int count, const int *n, const int *nev, const int *nbw, const double *const *A,
                                  const int *lda, double *const *ev, double *const *Z, const int *ldz,
                                  void *workspace, size_t ws_bytes, int nbranches, void *const *ev_start,
                                  void *const *ev_end, gb_solve_graph **graph)
{
    if (!graph) return -15;
    *graph = nullptr;
    if (count < 1) return -1;
    if (!n || !nev || !A || !lda || !ev || !Z || !ldz) return -2;
    if (nbranches < 1) return -12;
    const size_t need = gb_solve_batched_workspace_bytes_nbw(count, n, nev, nbw, nbranches);
    if (need == 0) return -2;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -10;
    if (ws_bytes < need) return -11;
    const size_t slot = need / (size_t)nbranches;
    const int nb = nbranches < count ? nbranches : count;
    gb_solve_graph *g = new gb_solve_graph;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return GB_ERR_CUDA;
    }
    int rc = GB_OK;
    g->branch.assign(nb, nullptr);
    g->join.assign(nb, nullptr);
    bool ok = cudaStreamCreateWithFlags(&g->origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int s = 0; ok && s < nb; s++)
        ok = cudaStreamCreateWithFlags(&g->branch[s], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&g->join[s], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        destroy_graph_object(g);
        return GB_ERR_CUDA;
    }
    // relaxed mode: the solves make non-stream calls (function attributes,
    // occupancy queries) that the stricter capture modes would refuse
    if (cudaStreamBeginCapture(g->origin, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        destroy_graph_object(g);
        return GB_ERR_CUDA;
    }
    ok = cudaEventRecord(g->fork, g->origin) == cudaSuccess;
    for (int s = 0; ok && s < nb; s++) ok = cudaStreamWaitEvent(g->branch[s], g->fork, 0) == cudaSuccess;
    if (!ok) rc = GB_ERR_CUDA;
    for (int i = 0; rc == GB_OK && i < count; i++) {
        const int s = i % nb;
        const cudaStream_t st = g->branch[s];
        // external event-record nodes: the caller's events are recorded
        // when the graph runs (a plain record inside a capture would only
        // order the graph's own nodes)
        if (ev_start && cudaEventRecordWithFlags((cudaEvent_t)ev_start[i], st, cudaEventRecordExternal) != cudaSuccess) {
            rc = GB_ERR_CUDA;
            break;
        }
        const int b = nbw ? nbw[i] : gb_solve_default_nbw(n[i]);
        rc = gb_solve_d(n[i], nev[i], b, A[i], lda[i], ev[i], Z[i], ldz[i], (char *)workspace + s * slot, slot,
                        (void *)st, 0);
        if (rc == GB_OK && ev_end &&
            cudaEventRecordWithFlags((cudaEvent_t)ev_end[i], st, cudaEventRecordExternal) != cudaSuccess)
            rc = GB_ERR_CUDA;
    }
    for (int s = 0; s < nb; s++) {  // join every branch, also after a failure, so the capture can end
        if (cudaEventRecord(g->join[s], g->branch[s]) != cudaSuccess ||
            cudaStreamWaitEvent(g->origin, g->join[s], 0) != cudaSuccess)
            rc = rc == GB_OK ? GB_ERR_CUDA : rc;
    }
    cudaGraph_t cg = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(g->origin, &cg);
    if (rc == GB_OK && (ee != cudaSuccess || !cg)) rc = GB_ERR_CUDA;
    size_t nodes = 0;
    if (rc == GB_OK && cudaGraphGetNodes(cg, nullptr, &nodes) != cudaSuccess) rc = GB_ERR_CUDA;
    if (rc == GB_OK && cudaGraphInstantiate(&g->exec, cg, 0) != cudaSuccess) rc = GB_ERR_CUDA;
    if (cg) cudaGraphDestroy(cg);
    cudaGetLastError();  // a failed capture leaves its error behind; it is reported through rc
    if (rc != GB_OK) {
        destroy_graph_object(g);
        return rc;
    }
    g->nodes = (long long)nodes;
    *graph = g;
    return GB_OK;
}

int gb_solve_batched_graph_launch(gb_solve_graph *graph, void *stream)
{
    if (!graph || !graph->exec) return -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    if (dev != graph->device) return GB_ERR_UNSUPPORTED;
    return cudaGraphLaunch(graph->exec, (cudaStream_t)stream) == cudaSuccess ? GB_OK : GB_ERR_CUDA;
}

long long gb_solve_batched_graph_nodes(const gb_solve_graph *graph) { return graph ? graph->nodes : -1; }

int gb_solve_batched_graph_destroy(gb_solve_graph *graph)
{
    if (!graph) return -1;
    destroy_graph_object(graph);
    return GB_OK;
}

// ---- the batch stage by stage: every problem's front on the streams, all
// bulge chases in one persistent launch, every problem's back on the streams

namespace {

struct StagedLayout {
    size_t table, scratch_slot, total;
    std::vector<size_t> persist_off;  // per problem, from the workspace base
};

bool staged_layout(int count, const int *n, const int *nev, const int *nbw, int nslots, StagedLayout *L)
{
    if (count < 1 || !n || !nev || nslots < 1) return false;
    L->table = a256(gb::chase_batched_table_bytes(count));
    L->persist_off.assign((size_t)count, 0);
    size_t off = L->table, slot = 0;
    for (int i = 0; i < count; i++) {
        const int b = nbw ? nbw[i] : gb_solve_default_nbw(n[i]);
        if (gb_solve_workspace_bytes(n[i], nev[i], b) == 0) return false;
        const SolveWs w = carve(n[i], nev[i], b, nullptr, nullptr, true);
        L->persist_off[i] = off;
        off += a256(w.ptotal);
        slot = std::max(slot, a256(w.total));
    }
    L->scratch_slot = slot;
    L->total = off + slot * (size_t)nslots;
    return true;
}

}  // namespace

size_t gb_solve_batched_staged_workspace_bytes(int count, const int *n, const int *nev, const int *nbw, int nslots)
{
    StagedLayout L;
    return staged_layout(count, n, nev, nbw, nslots, &L) ? L.total : 0;
}

int gb_solve_batched_staged_d(int count, const int *n, const int *nev, const int *nbw, const double *const *A,
                              const int *lda, double *const *ev, double *const *Z, const int *ldz, void *workspace,
                              size_t ws_bytes, int nslots, void *const *streams, void *const *ev_start,
                              void *const *ev_end)
{
    if (count < 1) return -1;
    if (!n || !nev || !A || !lda || !ev || !Z || !ldz) return -2;
    if (nslots < 1 || !streams) return -12;
    StagedLayout L;
    if (!staged_layout(count, n, nev, nbw, nslots, &L)) return -2;
    if (!workspace || ((uintptr_t)workspace % 256) != 0) return -10;
    if (ws_bytes < L.total) return -11;
    char *base = (char *)workspace;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GB_ERR_CUDA;
    const int nthreads = nslots < count ? nslots : count;
    std::vector<SolveWs> ws((size_t)count);
    std::vector<int> bw((size_t)count);
    for (int i = 0; i < count; i++) {
        bw[i] = nbw ? nbw[i] : gb_solve_default_nbw(n[i]);
        const int s = i % nslots;
        char *scr = base + (L.total - L.scratch_slot * (size_t)nslots) + L.scratch_slot * (size_t)s;
        ws[i] = carve(n[i], nev[i], bw[i], scr, base + L.persist_off[i], true);
    }
    {  // the chase's problem table goes up first: its copy from the host waits for the stream
        std::vector<void *> cws((size_t)count);
        std::vector<double *> hv((size_t)count), ht((size_t)count);
        for (int i = 0; i < count; i++) {
            cws[i] = ws[i].chase;
            hv[i] = ws[i].hv;
            ht[i] = ws[i].ht;
        }
        if (gb::band_to_tridi_chase_batched_upload_d(count, n, bw.data(), cws.data(), hv.data(), ht.data(), base,
                                                     (cudaStream_t)streams[0]) != cudaSuccess)
            return GB_ERR_CUDA;
    }
    std::vector<int> rcs(nthreads, GB_OK);
    auto phase = [&](int s, int which) {
        if (cudaSetDevice(dev) != cudaSuccess) {
            rcs[s] = GB_ERR_CUDA;
            return;
        }
        cudaStream_t st = (cudaStream_t)streams[s];
        for (int i = s; i < count && rcs[s] == GB_OK; i += nslots) {
            const SolveWs &w = ws[i];
            int rc = GB_OK;
            if (which == 0) {
                if (ev_start && cudaEventRecord((cudaEvent_t)ev_start[i], st) != cudaSuccess) rc = GB_ERR_CUDA;
                if (rc == GB_OK)
                    rc = solve_d_parts(n[i], nev[i], bw[i], A[i], lda[i], ev[i], Z[i], ldz[i], base, 0, (void *)st, 0,
                                       kPartFront, &w);
                if (rc == GB_OK && gb::band_to_tridi_prepare_d(n[i], bw[i], w.AB, bw[i] + 1, w.chase, st) != cudaSuccess)
                    rc = GB_ERR_CUDA;
            } else {
                if (gb::band_to_tridi_finish_d(n[i], bw[i], w.chase, w.d, w.e, st) != cudaSuccess) rc = GB_ERR_CUDA;
                if (rc == GB_OK)
                    rc = solve_d_parts(n[i], nev[i], bw[i], A[i], lda[i], ev[i], Z[i], ldz[i], base, 0, (void *)st, 0,
                                       kPartBack, &w);
                if (rc == GB_OK && ev_end && cudaEventRecord((cudaEvent_t)ev_end[i], st) != cudaSuccess)
                    rc = GB_ERR_CUDA;
            }
            rcs[s] = rc;
        }
    };
    auto run_phase = [&](int which) {
        std::vector<std::thread> pool;
        for (int s = 1; s < nthreads; s++) pool.emplace_back(phase, s, which);
        phase(0, which);
        for (auto &t : pool) t.join();
        for (int rc : rcs)
            if (rc != GB_OK) return rc;
        return (int)GB_OK;
    };
    int rc = run_phase(0);
    if (rc != GB_OK) return rc;
    // every front done -> one chase launch on the first stream -> every back
    std::vector<cudaEvent_t> evs((size_t)nthreads + 1, nullptr);
    for (auto &e : evs)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = GB_ERR_CUDA;
    const cudaStream_t st0 = (cudaStream_t)streams[0];
    for (int s = 1; rc == GB_OK && s < nthreads; s++)
        if (cudaEventRecord(evs[s], (cudaStream_t)streams[s]) != cudaSuccess ||
            cudaStreamWaitEvent(st0, evs[s], 0) != cudaSuccess)
            rc = GB_ERR_CUDA;
    if (rc == GB_OK && gb::band_to_tridi_chase_batched_d(count, n, bw.data(), base, 10LL * 1000 * 1000 * 1000, st0) != cudaSuccess)
        rc = GB_ERR_CUDA;
    if (rc == GB_OK && cudaEventRecord(evs[0], st0) != cudaSuccess) rc = GB_ERR_CUDA;
    for (int s = 1; rc == GB_OK && s < nthreads; s++)
        if (cudaStreamWaitEvent((cudaStream_t)streams[s], evs[0], 0) != cudaSuccess) rc = GB_ERR_CUDA;
    for (auto &e : evs)
        if (e) cudaEventDestroy(e);  // released once the work recorded on them completes
    if (rc != GB_OK) return rc;
    return run_phase(1);
}

int gb_solve_batched_staged_query(const void *workspace, int count, const int *n, const int *nev, const int *nbw,
                                  int nslots, void *const *streams)
{
    StagedLayout L;
    if (!workspace || !streams || !staged_layout(count, n, nev, nbw, nslots, &L)) return -1;
    for (int s = 0; s < nslots; s++)
        if (cudaStreamSynchronize((cudaStream_t)streams[s]) != cudaSuccess) return GB_ERR_CUDA;
    void *stream = streams[0];
    int rc = gb_trans_ev_query(workspace, 256, stream);  // the batched chase's state word
    if (rc != GB_OK) return rc;
    const char *base = (const char *)workspace;
    for (int i = 0; i < count; i++) {
        const int b = nbw ? nbw[i] : gb_solve_default_nbw(n[i]);
        const int s = i % nslots;
        char *scr = (char *)base + (L.total - L.scratch_slot * (size_t)nslots) + L.scratch_slot * (size_t)s;
        const SolveWs w = carve(n[i], nev[i], b, scr, (char *)base + L.persist_off[i], true);
        // each slot's last problem left its back-transformation's status in the slot
        if (i + nslots >= count && (rc = gb_trans_ev_query(w.tev, w.tev_bytes, stream)) != GB_OK) return rc;
    }
    return GB_OK;
}

int elpa_b200_solve(int n, int nev, const double *A, int lda, double *ev, double *Z, int ldz)
{
    const int nbw = n > 64 ? 64 : (n > 1 ? n - 1 : 1);
    size_t bytes = gb_solve_workspace_bytes(n, nev, nbw);
    if (bytes == 0) return n < 2 ? -1 : -2;
    void *ws = nullptr;
    if (cudaMalloc(&ws, bytes) != cudaSuccess) return GB_ERR_WORKSPACE;
    int rc = gb_solve_d(n, nev, nbw, A, lda, ev, Z, ldz, ws, bytes, nullptr, 0);
    if (rc == GB_OK) rc = gb_solve_query(ws, n, nev, nbw, nullptr);
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(ws);
    if (rc == GB_OK && e != cudaSuccess) rc = GB_ERR_CUDA;
    return rc;
}

}  // extern "C"
