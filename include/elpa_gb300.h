/*
 * elpa_gb300 -- C ABI of the GB300 (sm_103a) back-transformation of
 * eigenvectors from tridiagonal to band form (trans_ev_tridi_to_band).
 *
 * Operation (Kus et al., "Optimizations of the Eigensolvers in the ELPA
 * Library", Sec. 2, two-stage paragraph and Eq. 6; Sec. 3.1, the
 * non-BLAS kernel of the two-stage back transformation):
 *
 *     Z <- Q2 Z,   Q2 = H(1,0) H(1,1) ... H(1,nk(1)-1) H(2,0) ... H(n-1,0),
 *
 * where H(s,k) = I - tau(s,k) v(s,k) v(s,k)^H are the Householder reflectors
 * that the band -> tridiagonal bulge chase emits (T = Q2^H B Q2), and Z holds
 * nev eigenvectors of T.  The result holds the corresponding eigenvectors of
 * the band matrix B.  Columns of Z are independent.
 *
 * Reflector storage layout (n = matrix order, b = nbw = band width, i.e. the
 * number of super-diagonals of B; 1-based sweep s, 0-based block k):
 *   - sweep s = 1..n-1 has nk(s) = ceil((n-s)/b) reflectors, k = 0..nk(s)-1;
 *   - H(s,k) acts on rows s+1+k*b .. min(s+(k+1)*b, n) (1-based), so its
 *     length is len(s,k) = min(b, n-s-k*b) >= 1;
 *   - idx(s,k) = sum_{s'<s} nk(s') + k  (see gb_hh_index);
 *   - hh_v[idx*b + i], i = 0..b-1, holds v_i for 0 < i < len; v_0 = 1 is
 *     implicit and hh_v[idx*b] is not read; entries len <= i < b are not read;
 *   - hh_tau[idx] holds tau.
 *   Complex data (the _z entry points) is interleaved (re, im) doubles, i.e.
 *   C99 double complex / std::complex<double> / numpy complex128.
 *
 * All matrices are column-major.  Z is n x nev with leading dimension ldz.
 *
 * Ownership: the caller owns every buffer.  Z is updated in place.  The
 * device entry points allocate nothing; the calls are asynchronous on the
 * given CUDA stream (NULL = legacy default stream).  Input buffers must stay
 * valid and unmodified until the stream reaches the end of the call.  While
 * a call of the tensor-core variant runs, Z holds an intermediate
 * per-column 64-bit fixed-point form of its values (converted in place
 * before and after), so Z must not be read on another stream meanwhile.
 *
 * Errors: every entry point returns 0 on success; -i when argument i
 * (1-based) is invalid (nothing is launched); a positive GB_ERR_* code when a
 * CUDA call fails or a device-side wait gives up.  No entry point aborts or
 * throws.
 */
#ifndef ELPA_GB300_H
#define ELPA_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GB_OK 0
#define GB_ERR_CUDA 1        /* a CUDA runtime call failed (launch, copy, ...) */
#define GB_ERR_TIMEOUT 2     /* a device-side dependency wait exceeded its bound */
#define GB_ERR_WORKSPACE 3   /* workspace pointer NULL/misaligned or too small */
#define GB_ERR_UNSUPPORTED 4 /* valid arguments outside what this build supports */
#define GB_ERR_NONFINITE 5   /* Z held NaN or Inf (tensor-core variants): those columns come back
                                as all NaN, the other columns are exact results */
#define GB_ERR_RANGE 6       /* a column left its fixed-point range (tensor-core variants): the
                                reflectors were not orthogonal / unitary; Z is unspecified but finite */

/* Kernel variants for gb_trans_ev_opts.variant. */
#define GB_VARIANT_AUTO 0      /* library picks: PIPELINE_TC5 for real data with nbw in
                                  {16,32,64} and n >= 512, else PIPELINE for real
                                  data with nbw in {8,16,32,64}, else WAVEFRONT */
#define GB_VARIANT_WAVEFRONT 1 /* one launch per anti-diagonal of the tile DAG */
#define GB_VARIANT_PIPELINE 2  /* one persistent launch, tiles ordered by flags */
#define GB_VARIANT_PIPELINE_TC 3 /* the pipeline's schedule with every tile applied in
                                    compact WY form on the bf16 tensor cores (exact
                                    digit slicing, Z in per-column 64-bit fixed point
                                    during the call) issued as warp-level mma.sync;
                                    real data, nbw in {16,32,64}, otherwise runs as
                                    PIPELINE */
#define GB_VARIANT_PIPELINE_TC5 4 /* the same compact WY tiles on the tcgen05 tensor
                                     cores: 128 eigenvector columns per work item as
                                     the MMA's M, FP16 digit planes of Z and W in
                                     tensor memory, FP32 level accumulators in tensor
                                     memory, tile records by bulk copy; real data,
                                     nbw in {16,32,64}, otherwise runs as PIPELINE */

/* Tuning knobs (the paper's MEDIUM autotuning level tunes the blocking of the
 * back transformation, Sec. 4.3 and Sec. 5.3).  Zero fields mean "default". */
typedef struct gb_trans_ev_opts {
    int variant;         /* GB_VARIANT_*; PIPELINE needs nbw in {8,16,32,64} and
                            otherwise runs as WAVEFRONT */
    int sweeps_per_tile; /* nb: consecutive sweeps per tile, 1..32 (rounded up to
                            4, 8 or 16 for WAVEFRONT and 8 or 16 for PIPELINE) */
    int cols_per_block;  /* eigenvector columns per thread block: 32, 64 or 128
                            (PIPELINE: 64 or 128) */
    int spin_limit;      /* PIPELINE only: polls before a dependency wait gives up
                            (0 = default; every wait also gives up after 10 s) */
    int test_hold_group; /* fault-injection hook for tests: when g+1 > 0, sweep
                            group g never publishes its progress so that the
                            next group's wait must give up; 0 = off */
    int column_batch;    /* PIPELINE, PIPELINE_TC and PIPELINE_TC5: column blocks
                            per ticket batch, 1..1024 (0 = default: 16, 8 for
                            PIPELINE_TC (64-column blocks), 8 for PIPELINE_TC5
                            (128-column blocks)).  Items of one batch run
                            group after group; smaller batches keep fewer
                            eigenvector rows live in L2, larger ones read the
                            reflectors fewer times. */
    int lead_tiles;      /* PIPELINE only: how many tiles a sweep group may run
                            ahead of the next group of the same columns, 1..65536
                            (0 = default: no limit).  Small leads keep the rows
                            passed from group to group in L2 but hold groups
                            back. */
    void *kernel_begin_event; /* optional cudaEvent_t (NULL = none), recorded on the
                            call's stream right before the call's dominant kernel
                            is launched: the pipeline kernel, or the first of the
                            wavefront's launches.  Lets a caller time that kernel
                            alone with cudaEventElapsedTime.  An invalid event
                            makes the call return GB_ERR_CUDA. */
    void *kernel_end_event; /* optional cudaEvent_t recorded right after that
                            kernel (the wavefront's last launch) */
} gb_trans_ev_opts;

/* Number of reflectors of the layout above (-1 if n < 1 or nbw < 1). */
long long gb_hh_count(int n, int nbw);

/* Storage index idx(s,k) (-1 if (s,k) is not a reflector of the layout). */
long long gb_hh_index(int n, int nbw, int s, int k);

/* Largest band width the kernels of this build accept. */
int gb_max_nbw(void);

/* Bytes of device workspace a call needs (0 is possible); the workspace must
 * be 256-byte aligned.  Returns 0 for invalid arguments as well. */
size_t gb_trans_ev_workspace_bytes(int n, int nbw, int nev, int is_complex,
                                   const gb_trans_ev_opts *opts);

/* Z <- Q2 Z, real symmetric case (FP64).  All pointers are device pointers.
 * Arguments: 1 n >= 1; 2 nbw in 1..gb_max_nbw(); 3 nev >= 0; 4 hh_v
 * (gb_hh_count * nbw doubles); 5 hh_tau (gb_hh_count doubles); 6 Z (8-byte
 * aligned); 7 ldz >= n; 8 workspace; 9 ws_bytes >=
 * gb_trans_ev_workspace_bytes(...); 10 stream (cudaStream_t); 11 opts (may be
 * NULL for defaults). */
int gb_trans_ev_tridi_to_band_d(int n, int nbw, int nev, const double *hh_v,
                                const double *hh_tau, double *Z, int ldz,
                                void *workspace, size_t ws_bytes, void *stream,
                                const gb_trans_ev_opts *opts);

/* Complex Hermitian case: same arguments, complex128 data interleaved as
 * doubles (hh_v: 2 * count * nbw doubles, hh_tau: 2 * count, Z: 2 * ldz * nev). */
int gb_trans_ev_tridi_to_band_z(int n, int nbw, int nev, const double *hh_v,
                                const double *hh_tau, double *Z, int ldz,
                                void *workspace, size_t ws_bytes, void *stream,
                                const gb_trans_ev_opts *opts);

/* Host-buffer form of the real case: hh_v, hh_tau and Z are HOST pointers
 * (pinned memory gives the fastest copies).  dev_buf is a caller-owned device
 * buffer of at least gb_trans_ev_host_buffer_bytes(...) bytes (256-byte
 * aligned) that receives the copies and the workspace.  The call copies the
 * inputs to the device, runs the back-transformation, copies Z back and
 * synchronises the stream before it returns. */
size_t gb_trans_ev_host_buffer_bytes(int n, int nbw, int nev, int ldz, int is_complex,
                                     const gb_trans_ev_opts *opts);
int gb_trans_ev_tridi_to_band_d_host(int n, int nbw, int nev, const double *hh_v,
                                     const double *hh_tau, double *Z, int ldz,
                                     void *dev_buf, size_t dev_bytes, void *stream,
                                     const gb_trans_ev_opts *opts);

/* Completion status of the device work of earlier calls that used this
 * workspace: synchronises the stream, then returns GB_OK, GB_ERR_TIMEOUT (a
 * PIPELINE dependency wait gave up; Z is then unspecified), GB_ERR_NONFINITE
 * (tensor-core variants: Z held NaN or Inf; those columns are returned as
 * all NaN, the others are exact), GB_ERR_RANGE (tensor-core variants: a
 * column left its fixed-point range because the reflectors were not
 * orthogonal; Z is unspecified but finite) or GB_ERR_CUDA.
 * workspace may be NULL (WAVEFRONT calls need none): then only the stream is
 * synchronised. */
int gb_trans_ev_query(const void *workspace, size_t ws_bytes, void *stream);

/* Number of kernel launches one call with these arguments issues. */
long long gb_trans_ev_launch_count(int n, int nbw, int nev, int is_complex,
                                   const gb_trans_ev_opts *opts);

/* The kernel variant (GB_VARIANT_WAVEFRONT, _PIPELINE, _PIPELINE_TC or
 * _PIPELINE_TC5) a call with these arguments runs, after AUTO and the
 * fallbacks are resolved; -1 for invalid arguments.  Host only. */
int gb_trans_ev_variant(int n, int nbw, int nev, int is_complex, const gb_trans_ev_opts *opts);

/* No-allocation form of the real case, for callers that cannot call
 * cudaMalloc (code running inside a memory pool or arena that owns all
 * device memory, allocation-free service loops, hosts that forbid allocation
 * after start-up).  The paper has no counterpart; it exists for such callers.
 *
 * Same operation and arguments 1-7 as gb_trans_ev_tridi_to_band_d, always
 * with the pipeline kernel (nb = 16, 64 columns per block); nbw must be 8,
 * 16, 32 or 64 (else -2).  Its scratch area (pipeline ticket, status words
 * and progress flags) is a fixed array of GB_NOALLOC_SCRATCH_BYTES in device
 * memory that every GPU loading the library holds until the process exits;
 * a problem needing more (gb_trans_ev_workspace_bytes with variant PIPELINE,
 * sweeps_per_tile 16, cols_per_block 64) is rejected with GB_ERR_WORKSPACE
 * before anything is launched (n = 16384, nev = 4096 needs 256.25 KiB).
 * Every call looks the array's address up on the current device (this
 * allocates nothing, and stays right if the context is re-created); the
 * first call on a device loads the array there, so make it before any
 * stream capture.  All calls share the array and it
 * keeps the last call's contents; each call clears what must start at zero,
 * and calls whose device work overlaps on the GPU race on it.
 * status (argument 8) may be NULL, or a device or pinned-host int that
 * receives, in stream order after the kernel, 0 or GB_ERR_TIMEOUT (a
 * dependency wait gave up; Z is then unspecified).  stream (argument 9): the
 * call is asynchronous on it.  Allocates nothing. */
#define GB_NOALLOC_SCRATCH_BYTES (1 << 20)
int gb_trans_ev_tridi_to_band_d_noalloc(int n, int nbw, int nev, const double *hh_v,
                                        const double *hh_tau, double *Z, int ldz,
                                        int *status, void *stream);

/* Band -> tridiagonal reduction by bulge chasing (the second step of the
 * two-stage reduction, Sec. 2), producing the reflectors that
 * gb_trans_ev_tridi_to_band_d consumes.  B is real symmetric with nbw
 * super-diagonals, given in LAPACK lower band storage: AB[(i-j) + j*ldab] =
 * B(i,j) for 0 <= i-j <= nbw (device pointer, not modified).  Outputs
 * (device pointers, caller-owned): d (n) and e (n-1), the diagonal and
 * sub-diagonal of T = Q2^T B Q2; hh_v (gb_hh_count * nbw) and hh_tau
 * (gb_hh_count) in the layout above (hh_v[idx*nbw] = 1, zero padding past
 * len).  Arguments: 1 n >= 1; 2 nbw in 1..64; 3 AB; 4 ldab >= nbw+1; 5 d;
 * 6 e; 7 hh_v; 8 hh_tau; 9 workspace (256-byte aligned); 10 ws_bytes >=
 * gb_band_to_tridi_workspace_bytes(n, nbw); 11 stream.  Asynchronous;
 * device-side status (a dependency wait that gave up after 10 s) through
 * gb_trans_ev_query(workspace, ws_bytes, stream). */
size_t gb_band_to_tridi_workspace_bytes(int n, int nbw);
int gb_band_to_tridi_d(int n, int nbw, const double *AB, int ldab, double *d, double *e,
                       double *hh_v, double *hh_tau, void *workspace, size_t ws_bytes,
                       void *stream);

/* Complex Hermitian form of gb_band_to_tridi_d: AB holds complex128 entries
 * (interleaved re, im) of the lower band, hh_v / hh_tau complex128 in the
 * same layout; d and e are real (every kept sub-diagonal entry is made real
 * by the reflector generation, length-1 reflectors included).  Arguments and
 * status as for gb_band_to_tridi_d, with ldab counted in complex elements. */
size_t gb_band_to_tridi_workspace_bytes_z(int n, int nbw);
int gb_band_to_tridi_z(int n, int nbw, const double *AB, int ldab, double *d, double *e,
                       double *hh_v, double *hh_tau, void *workspace, size_t ws_bytes,
                       void *stream);

/* Two-stage symmetric eigensolver (Sec. 2): A = Z diag(ev) Z^T for the nev
 * smallest eigenvalues of the real symmetric n x n matrix A.
 *   full -> band (Householder panels; trailing updates as symmetric
 *   products on the lower triangle),
 *   band -> tridiagonal (gb_band_to_tridi_d's bulge chase),
 *   eigenpairs of the tridiagonal: divide and conquer (gb_tridiag_dc_d)
 *   when more than half of the eigenvectors are wanted (2 nev > n), else
 *   multisection, inverse iteration and one Newton-Schulz orthogonalisation
 *   step,
 *   tridiagonal -> band (gb_trans_ev_tridi_to_band_d, pipeline kernel),
 *   band -> full (block reflectors as matrix products).
 * Every matrix product runs in this library's own kernels (no vendor BLAS).
 * Arguments (device pointers): 1 n >= 2; 2 nev in 1..n; 3 nbw in 1..min(64,
 * n-1), the intermediate band width; 4 A (column-major, lda; read only, both
 * triangles used); 5 lda >= n; 6 ev (nev, ascending); 7 Z (n x nev,
 * column-major); 8 ldz >= n; 9 workspace (256-byte aligned); 10 ws_bytes >=
 * gb_solve_workspace_bytes(n, nev, nbw); 11 stream; 12 flags: 0 or an OR
 * of GB_SOLVE_RECORD_STAGES, GB_SOLVE_DFMA_PRODUCTS, GB_SOLVE_TRIDIAG_BISECT
 * (bisection and inverse iteration even when 2 nev > n),
 * GB_SOLVE_FP32_PRODUCTS (the sliced products of full->band and band->full
 * become FP32 products: operands rounded to FP32 and split exactly into
 * three bf16 parts, six bf16 tensor-core products per step accumulated in
 * FP32; the low-precision half of gb_solve_mixed_d) and GB_SOLVE_FP64_EMULATED_GEMM (accepted and ignored:
 * no product of either solver goes through a vendor BLAS).  By
 * default the large products (the full->band SYMM and SYR2K, the band->full
 * GEMMs, the Newton-Schulz SYRK and SYMM) run on the bf16 tensor cores by
 * exact digit slicing (gb_dgemm_sliced below); GB_SOLVE_DFMA_PRODUCTS runs
 * them on the FP64 FMA pipe instead.  Asynchronous; device-side status of
 * the dependency waits through gb_solve_query. */
#define GB_SOLVE_FP64_EMULATED_GEMM 1
#define GB_SOLVE_RECORD_STAGES 2 /* record CUDA events at the stage boundaries */
#define GB_SOLVE_DFMA_PRODUCTS 4 /* products on the FP64 FMA pipe, not sliced */
#define GB_SOLVE_TRIDIAG_BISECT 8 /* tridiagonal step by bisection + inverse iteration */
#define GB_SOLVE_FP32_PRODUCTS 16 /* FP32 products in full->band and band->full */
size_t gb_solve_workspace_bytes(int n, int nev, int nbw);
int gb_solve_d(int n, int nev, int nbw, const double *A, int lda, double *ev, double *Z, int ldz,
               void *workspace, size_t ws_bytes, void *stream, int flags);
/* Synchronises the stream and returns GB_OK or the first device-side error
 * (GB_ERR_TIMEOUT) of the last gb_solve_d that used this workspace. */
int gb_solve_query(const void *workspace, int n, int nev, int nbw, void *stream);
/* Complex Hermitian two-stage solve: A (complex128, interleaved, lda) =
 * Z diag(ev) Z^H with real ev (nev, ascending) and complex Z (n x nev, ldz);
 * same arguments, workspace rule (gb_solve_workspace_bytes_z) and flags as
 * gb_solve_d (GB_SOLVE_RECORD_STAGES is ignored; GB_SOLVE_FP32_PRODUCTS is
 * refused with -12: the mixed-precision solve is real only).  The large complex
 * products run sliced on the bf16 tensor cores (GB_SOLVE_DFMA_PRODUCTS:
 * on the FP64 FMA pipe), the b x b panel products in this library's complex
 * DFMA kernel, and the back-transformation on the tcgen05 tensor cores
 * (nbw in {16, 32, 64}, n >= 512).  Device-side status of the waits of the
 * bulge chase and of the back-transformation through gb_solve_query_z. */
size_t gb_solve_workspace_bytes_z(int n, int nev, int nbw);
int gb_solve_z(int n, int nev, int nbw, const double *A, int lda, double *ev, double *Z, int ldz,
               void *workspace, size_t ws_bytes, void *stream, int flags);
int gb_solve_query_z(const void *workspace, int n, int nev, int nbw, void *stream);

/* Milliseconds of the seven stages (full->band, band->tridiagonal,
 * bisection, inverse iteration, orthogonalisation, tridiagonal->band,
 * band->full) of the last gb_solve_d on this stream that had
 * GB_SOLVE_RECORD_STAGES set; ms has 7 entries.  Synchronises the stream. */
int gb_solve_stage_ms(void *stream, float *ms);
/* The solvers cache per (device, stream) a look-ahead helper stream with
 * its events (n >= 4096) and the stage events; they are created on first
 * use and otherwise kept until the process exits.  gb_solve_release frees those of `stream` on the current
 * device, or of every stream on every device if all_streams is nonzero.
 * Call it only when no solve is in flight on the streams concerned (it
 * waits for the helper streams).  A later solve on such a stream creates
 * them again.  Returns GB_OK, or GB_ERR_CUDA if a CUDA call failed (the
 * cache entries are dropped either way). */
int gb_solve_release(void *stream, int all_streams);
/* Convenience form with host-side defaults: nbw = min(64, n-1), legacy
 * default stream, and a workspace it allocates with cudaMalloc and frees
 * before returning (synchronous).  All pointers are device pointers. */
int elpa_b200_solve(int n, int nev, const double *A, int lda, double *ev, double *Z, int ldz);

/* Batched form: count independent problems (A[i] n[i] x n[i], lda[i]; ev[i],
 * Z[i] n[i] x nev[i], ldz[i]; all device pointers), each with band width
 * gb_solve_default_nbw(n[i]).  Problem i runs on streams[i % nslots] in
 * workspace slot i % nslots, so up to nslots solves overlap on the GPU; the
 * host only enqueues (asynchronous), one host thread per slot, and returns
 * when every problem is enqueued.  If ev_start / ev_end are non-NULL,
 * events ev_start[i] / ev_end[i] (cudaEvent_t, created by the caller) are
 * recorded around problem i on its stream.  Arguments: 1 count >= 1; 2-8 the
 * per-problem arrays; 9 workspace (256-byte aligned); 10 ws_bytes >=
 * gb_solve_batched_workspace_bytes(count, n, nev, nslots); 11 nslots >= 1;
 * 12 streams (nslots cudaStream_t); 13-14 event arrays or NULL. */
int gb_solve_default_nbw(int n);
size_t gb_solve_batched_workspace_bytes(int count, const int *n, const int *nev, int nslots);

/* All eigenpairs of the real symmetric tridiagonal matrix with diagonal d[0..n)
 * and off-diagonal e[0..n-1) by divide and conquer (Cuppen's method with
 * deflation; the secular equation solved per root with the two-pole model of
 * Bunch, Nielsen and Sorensen; the rank-one vector recomputed from the roots
 * as Gu and Eisenstat do, so the eigenvectors are orthogonal to working
 * accuracy; the merged eigenvectors as products, sliced onto the tensor
 * cores when large).  This is the tridiagonal step of the two-stage solver
 * (Sec. 2) when all eigenvectors are wanted.
 * Arguments (device pointers): 1 n >= 1; 2 d (n); 3 e (n-1; may be NULL for
 * n = 1); 4 lam (n, out, ascending); 5 Q (n x n, column-major, ldq; out:
 * column j is the eigenvector of lam[j]); 6 ldq >= n; 7 workspace (256-byte
 * aligned); 8 ws_bytes >= gb_tridiag_dc_workspace_bytes(n) (about 3 n^2
 * doubles).  Asynchronous on `stream`; d and e are not modified. */
/* One step of Ogita and Aishima's iterative refinement of a full symmetric
 * eigendecomposition (the FP64 refinement that the mixed-precision
 * configuration pairs with a low-precision solve): with R = I - X^T X,
 * S = X^T A X, lambda_i = s_ii / (1 - r_ii), delta = 2 (||S - diag(lambda)||
 * + ||A|| ||R||), E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) where
 * |lambda_i - lambda_j| > delta and r_ij / 2 elsewhere, X <- X + X E.  The
 * error of X falls quadratically for eigenvalues separated by more than
 * delta.  Clusters (runs of neighbouring columns whose gap is within delta
 * or whose first-order correction exceeds 1e-3; at most 64 columns) first
 * get a Rayleigh-Ritz rotation X_J <- X_J G_JJ^(-1/2) Y_J (Y_J the
 * eigenvectors of G_JJ^(-1/2) S_JJ G_JJ^(-1/2)), and E is taken in the
 * rotated basis (r / 2 inside a cluster).  The products are sliced on the
 * bf16 tensor cores (FP64-accurate; 6 n^3 flops a step: X^T X and
 * X^T (A X) on their lower triangles); ||A||_2 is taken as max |lambda_i|,
 * the other norms bounded by Frobenius norms.
 * Arguments (device pointers): 1 n >= 1; 2 A (n x n symmetric, lower
 * triangle read, lda); 3 lda >= n; 4 lam (n, out: the Rayleigh quotients of
 * the input X after the clusters' rotation, i.e. Ritz values inside
 * clusters); 5 X (n x n, ldx; in: approximate eigenvectors in the columns,
 * ordered by eigenvalue, out: refined); 6 ldx >= n; 7 workspace (256-byte
 * aligned); 8 ws_bytes >= gb_refine_syev_workspace_bytes(n) (3 n^2 doubles
 * plus two n x n operands' digit planes, 16 n^2 bytes each, plus 512 n
 * bytes of cluster rotations).  Asynchronous on `stream`. */
size_t gb_refine_syev_workspace_bytes(int n);
int gb_refine_syev_d(int n, const double *A, int lda, double *lam, double *X, int ldx, void *workspace,
                     size_t ws_bytes, void *stream);

/* Mixed-precision two-stage solve (the FP32 tensor-core reduction and
 * back-transformation with FP64 Ogita-Aishima refinement): all n eigenpairs
 * by gb_solve_d with GB_SOLVE_FP32_PRODUCTS (the tridiagonal step, the bulge
 * chase and trans_ev_tridi_to_band stay FP64), then refine_steps steps of
 * gb_refine_syev_d in FP64 on the whole decomposition, then the lowest nev
 * pairs copied out.  ev are the Rayleigh quotients of the eigenvectors
 * before the last step (ascending up to rounding within clusters; the low-
 * precision solve's eigenvalues if refine_steps = 0).  The refinement
 * converges where the low-precision eigenvectors' errors are small against
 * the eigenvalue gaps; inside clusters narrower than its threshold it
 * refines the cluster's subspace only.
 * Arguments 1-8 as for gb_solve_d; 9 refine_steps in 0..GB_SOLVE_MIXED_MAX_STEPS;
 * 10 workspace (256-byte aligned); 11 ws_bytes >=
 * gb_solve_mixed_workspace_bytes(n, nev, nbw) (n x n eigenvectors plus the
 * larger of the all-pairs solve's and the refinement's workspaces).
 * Asynchronous on `stream`; device-side status through gb_solve_mixed_query
 * (synchronises the stream). */
#define GB_SOLVE_MIXED_MAX_STEPS 8
size_t gb_solve_mixed_workspace_bytes(int n, int nev, int nbw);
int gb_solve_mixed_d(int n, int nev, int nbw, const double *A, int lda, double *ev, double *Z, int ldz,
                     int refine_steps, void *workspace, size_t ws_bytes, void *stream);
int gb_solve_mixed_query(const void *workspace, int n, int nev, int nbw, void *stream);

size_t gb_tridiag_dc_workspace_bytes(int n);
int gb_tridiag_dc_d(int n, const double *d, const double *e, double *lam, double *Q, int ldq,
                    void *workspace, size_t ws_bytes, void *stream);
int gb_solve_batched_d(int count, const int *n, const int *nev, const double *const *A, const int *lda,
                       double *const *ev, double *const *Z, const int *ldz, void *workspace,
                       size_t ws_bytes, int nslots, void *const *streams, void *const *ev_start,
                       void *const *ev_end);

/* The same with a band width per problem: nbw[i] in 1..min(64, n[i]-1), or
 * nbw == NULL for gb_solve_default_nbw(n[i]) (e.g. the choices of a
 * gb_solve_tuner).  Arguments as above with nbw inserted as the 4th, so the
 * later ones are numbered one higher (workspace -10, ws_bytes -11, nslots
 * -12). */
size_t gb_solve_batched_workspace_bytes_nbw(int count, const int *n, const int *nev, const int *nbw,
                                            int nslots);
int gb_solve_batched_nbw_d(int count, const int *n, const int *nev, const int *nbw,
                           const double *const *A, const int *lda, double *const *ev,
                           double *const *Z, const int *ldz, void *workspace, size_t ws_bytes,
                           int nslots, void *const *streams, void *const *ev_start,
                           void *const *ev_end);

/* The two-stage solve (real, is_complex = 0, or complex Hermitian, 1) in
 * three calls, so that a server can run one stage for several requests at
 * once -- the bulge chases of all the requests it holds in one launch:
 *  * gb_solve_stage_front: copy, full -> band and the chase's working band,
 *    in the request's workspace (gb_solve_workspace_bytes[_z](n, nev, nbw));
 *  * gb_solve_stage_chase_batched: the bulge chases of `count` requests whose
 *    fronts have run, in ONE persistent launch on `stream` (tickets
 *    (request, sweep) in sweep-major order, deadlock-free at any residency);
 *    `table` is gb_solve_stage_table_bytes(count) device bytes, 256-byte
 *    aligned, reused only after the launch is done; its first 256 bytes hold
 *    the launch's status (gb_trans_ev_query(table, 256, stream)).  The table
 *    goes up by a copy from pageable host memory, which waits for the work
 *    already on `stream`;
 *  * gb_solve_stage_back: the tridiagonal eigenpairs and both
 *    back-transformations into ev and Z (flags as gb_solve_d).
 * The caller orders the calls of one request (events across streams).  The
 * three calls give bit-identical results to gb_solve_d / gb_solve_z.
 * Argument errors return -i as in the single-call forms. */
size_t gb_solve_stage_table_bytes(int count);
int gb_solve_stage_front(int is_complex, int n, int nev, int nbw, const double *A, int lda,
                         void *workspace, size_t ws_bytes, void *stream);
int gb_solve_stage_chase_batched(int is_complex, int count, const int *n, const int *nev,
                                 const int *nbw, void *const *workspaces, void *table,
                                 size_t table_bytes, void *stream);
int gb_solve_stage_back(int is_complex, int n, int nev, int nbw, double *ev, double *Z, int ldz,
                        void *workspace, size_t ws_bytes, void *stream, int flags);

/* The batch stage by stage: every problem's first stage (copy, full ->
 * band) on the streams as in gb_solve_batched_nbw_d, then the bulge chases
 * of ALL problems in one persistent launch (tickets (problem, sweep) in
 * sweep-major order, so the chains of all problems advance together and no
 * wait can deadlock), then every problem's remaining stages on the streams.
 * The chase is a latency-bound chain per problem; one launch over the whole
 * batch keeps the SMs busy with many chains at once.  Per-solve latency
 * grows (every problem waits for the last front), throughput rises.  Each
 * problem keeps its reflectors, T factors and chase band in the workspace
 * for the whole call; the scratch of the other stages is per slot.
 * Arguments as gb_solve_batched_nbw_d (nbw may be NULL), with ws_bytes >=
 * gb_solve_batched_staged_workspace_bytes(count, n, nev, nbw, nslots).
 * gb_solve_batched_staged_query synchronises every stream of the batch and
 * returns the device-side status of the batched chase and of each slot's
 * last back-transformation (earlier problems' statuses in a slot are
 * overwritten by its later problems). */
size_t gb_solve_batched_staged_workspace_bytes(int count, const int *n, const int *nev, const int *nbw,
                                               int nslots);
int gb_solve_batched_staged_d(int count, const int *n, const int *nev, const int *nbw,
                              const double *const *A, const int *lda, double *const *ev,
                              double *const *Z, const int *ldz, void *workspace, size_t ws_bytes,
                              int nslots, void *const *streams, void *const *ev_start,
                              void *const *ev_end);
int gb_solve_batched_staged_query(const void *workspace, int count, const int *n, const int *nev,
                                  const int *nbw, int nslots, void *const *streams);

/* The batched form as ONE CUDA graph.  The paper's SCF loop solves the same
 * set of problems again and again with new matrix entries (Sec. 5.1), so the
 * batch is issued once and replayed:
 *  * gb_solve_batched_graph_create records every solve of the batch (band
 *    width nbw[i], or the default when nbw is NULL) by stream capture into a
 *    graph of nbranches parallel branches -- problem i on branch
 *    i % nbranches, in workspace slot i % nbranches, after the branch's
 *    previous problem -- and instantiates it.  Nothing runs during creation.
 *    Events ev_start[i] / ev_end[i] (or NULL arrays), created by the caller,
 *    become event-record nodes around problem i.  Panel factorisations inside
 *    the graph take their non-cooperative form (a graph's kernel nodes carry
 *    no co-residency guarantee).  The graph owns its branch streams; the
 *    caller's buffers must stay allocated while it exists.
 *  * gb_solve_batched_graph_launch runs the whole batch as one graph launch
 *    on `stream` (asynchronous; on the device the graph was made on).  Each
 *    launch reads A[i] and writes ev[i] and Z[i] at the pointers given at
 *    creation, so the caller refreshes the matrices in place between
 *    launches.  Launches on one stream run one after another.
 *  * gb_solve_batched_graph_nodes: the graph's node count (-1 for NULL).
 *  * gb_solve_batched_graph_destroy: call it when no launch of the graph is
 *    still running.
 * Arguments of create: 1 count >= 1; 2-3 n, nev; 4 nbw or NULL; 5-9 A, lda,
 * ev, Z, ldz; 10 workspace (256-byte aligned); 11 ws_bytes >=
 * gb_solve_batched_workspace_bytes_nbw(count, n, nev, nbw, nbranches);
 * 12 nbranches >= 1; 13-14 event arrays or NULL; 15 graph (out).  Returns
 * GB_OK, -i, or GB_ERR_CUDA if the capture or instantiation failed (nothing
 * is left behind). */
typedef struct gb_solve_graph gb_solve_graph;
int gb_solve_batched_graph_create(int count, const int *n, const int *nev, const int *nbw,
                                  const double *const *A, const int *lda, double *const *ev,
                                  double *const *Z, const int *ldz, void *workspace,
                                  size_t ws_bytes, int nbranches, void *const *ev_start,
                                  void *const *ev_end, gb_solve_graph **graph);
int gb_solve_batched_graph_launch(gb_solve_graph *graph, void *stream);
long long gb_solve_batched_graph_nodes(const gb_solve_graph *graph);
int gb_solve_batched_graph_destroy(gb_solve_graph *graph);

/* Band-width tuning for the two-stage solve by problem size (the paper's
 * autotuning, Sec. 4.3 and 5.3, applied to the solver's blocking: the band
 * width is the panel width of full->band, the bulge chase's band and the
 * back-transformation's tile height).  Orders in [n_lo, n_hi] fall into
 * `classes` size classes of equal width in log(n).  For each class the tuner
 * hands out trials (n, nbw): n the class's geometric middle, nbw each of 16,
 * 32 and 64 below n.  The caller runs one solve per trial and reports its
 * seconds.  gb_solve_tuner_nbw(t, n) then gives the fastest measured band
 * width of n's class, capped below n (gb_solve_default_nbw(n) for a class
 * with no measurement or an n outside [n_lo, n_hi]).
 * gb_solve_tuner_step returns 1 with a trial, 0 when all are handed out, -1
 * while the previous trial is unreported.  save/load write and read the
 * state as text (a trial handed out but not reported is handed out again).
 * create returns NULL unless 2 <= n_lo <= n_hi and 1 <= classes <= 64.
 * Host-side only. */
typedef struct gb_solve_tuner gb_solve_tuner;
gb_solve_tuner *gb_solve_tuner_create(int n_lo, int n_hi, int classes);
void gb_solve_tuner_destroy(gb_solve_tuner *t);
int gb_solve_tuner_step(gb_solve_tuner *t, int *n, int *nbw);
int gb_solve_tuner_report(gb_solve_tuner *t, double seconds);
int gb_solve_tuner_nbw(const gb_solve_tuner *t, int n);
int gb_solve_tuner_save(const gb_solve_tuner *t, const char *path);
gb_solve_tuner *gb_solve_tuner_load(const char *path);

/* Autotuning of the back-transformation (modelled on the paper's autotuning,
 * Sec. 4.3 and 5.3): a tuning object walks a fixed list of settings; the
 * caller runs one back-transformation (or one solve) with each setting it
 * is handed and reports the elapsed seconds; the fastest is kept.  The walk
 * can be saved to a text file and resumed, so it can be spread over the
 * iterations of a self-consistency loop.  Host-side only.
 *   GB_AUTOTUNE_FAST   : kernel variant (wavefront, pipeline)
 *   GB_AUTOTUNE_MEDIUM : variant and blocking (sweeps per tile, columns per block)
 * gb_autotune_create returns NULL for invalid arguments.  gb_autotune_step
 * returns 1 and fills *next with the setting to try, 0 when every setting has
 * been handed out, -1 while the previous one is still unreported.
 * gb_autotune_report records the seconds of the last setting handed out.
 * gb_autotune_best returns GB_OK with the fastest measured setting (and its
 * seconds if non-NULL) or GB_ERR_UNSUPPORTED if none has been measured.
 * gb_autotune_save/_load write and read the state (a setting handed out but
 * not reported is handed out again after loading). */
#define GB_AUTOTUNE_FAST 1
#define GB_AUTOTUNE_MEDIUM 2
typedef struct gb_autotune gb_autotune;
gb_autotune *gb_autotune_create(int level, int n, int nbw, int nev);
void gb_autotune_destroy(gb_autotune *t);
int gb_autotune_step(gb_autotune *t, gb_trans_ev_opts *next);
int gb_autotune_report(gb_autotune *t, double seconds);
int gb_autotune_best(const gb_autotune *t, gb_trans_ev_opts *best, double *seconds);
int gb_autotune_progress(const gb_autotune *t, int *tried, int *total);
int gb_autotune_save(const gb_autotune *t, const char *path);
gb_autotune *gb_autotune_load(const char *path);

/* FP64 matrix products (column-major, device pointers, asynchronous on
 * `stream`).  The paper's solver hands these steps to BLAS (Sec. 3.2: the
 * GPU version calls cuBLAS for the matrix products of the reduction and the
 * back-transformations); here they run in this library's DFMA-tiled kernels,
 * which the solver uses internally.  `workspace` (8-byte aligned, or NULL
 * with ws_bytes 0) holds split-K partial products: a call splits the
 * reduction only as far as ws_bytes allows (gb_dgemm_workspace_bytes(m, n)
 * is always enough).  Returns GB_OK, -i for invalid argument i (nothing
 * launched), or GB_ERR_CUDA.
 *   gb_dgemm : C (m x n) = alpha op(A) op(B) + beta C, trans = 'N' or 'T',
 *              op(A) m x k, op(B) k x n; lda >= rows of A as stored, etc.
 *   gb_dsymm : side 'L': C (m x n) = alpha S B + beta C, S (m x m);
 *              side 'R': C = alpha B S + beta C, S (n x n); S symmetric,
 *              only its lower triangle is read.
 *   gb_dsyr2k: lower triangle of C (n x n) = alpha (A B^T + B A^T) + beta C,
 *              A, B n x k; the strict upper triangle of C is not touched.
 *   gb_dsyrk : lower triangle of C (n x n) = alpha A^T A + beta C, A k x n.
 * beta = 0 does not read C. */
size_t gb_dgemm_workspace_bytes(int m, int n);
int gb_dgemm(char transa, char transb, int m, int n, int k, double alpha, const double *A, int lda,
             const double *B, int ldb, double beta, double *C, int ldc, void *workspace, size_t ws_bytes,
             void *stream);
int gb_dsymm(char side, int m, int n, double alpha, const double *S, int lds, const double *B, int ldb,
             double beta, double *C, int ldc, void *workspace, size_t ws_bytes, void *stream);
int gb_dsyr2k(int n, int k, double alpha, const double *A, int lda, const double *B, int ldb, double beta,
              double *C, int ldc, void *stream);
int gb_dsyrk(int n, int k, double alpha, const double *A, int lda, double beta, double *C, int ldc,
             void *stream);

/* The same products computed on the bf16 tensor cores: every row of op(A)
 * and every column of op(B) is scaled by a power of two and cut exactly into
 * eight 7-bit digits (error-free splitting, Ozaki, Ogita, Oishi and Rump,
 * Numer. Algorithms 59, 2012); digit-plane products are formed with
 * mma.sync bf16, accumulated exactly (one FP32 accumulator per digit level,
 * exact over 128 values of k, folded into 64-bit integers), and the result
 * is rounded to FP64 once.  Accuracy is that of an FP64 product measured
 * against the scaled maxima: |C - alpha op(A) op(B)| <~ 2^-53 k |alpha|
 * max_j |op(A)_ij| max_i |op(B)_ij| per entry.  Inputs must be finite;
 * subnormal inputs are read as zero.  The paper's products are BLAS calls
 * (Sec. 3.2); this is how they run fastest on a part whose FP64 pipe is
 * narrow.  `workspace` (256-byte aligned) must hold the *_workspace_bytes
 * figure: the digit planes of both operands and split-K partials.  Same
 * argument numbering as the DFMA forms, then workspace, ws_bytes, stream;
 * -i for invalid argument i, GB_ERR_CUDA for a launch error. */
size_t gb_dgemm_sliced_workspace_bytes(int m, int n, int k);
int gb_dgemm_sliced(char transa, char transb, int m, int n, int k, double alpha, const double *A, int lda,
                    const double *B, int ldb, double beta, double *C, int ldc, void *workspace,
                    size_t ws_bytes, void *stream);
/* The FP32 product of the mixed-precision solve, with gb_dgemm_sliced's
 * arguments, statuses and workspace (gb_dgemm_sliced_workspace_bytes): each
 * entry of op(A) and op(B) is rounded to FP32 and split exactly into three
 * bf16 parts with their own exponents; the six part products of weight at
 * least 2^-16 per k16 step run on mma.sync bf16 into one FP32 accumulator,
 * folded into FP64 every 128 values of k.  Error: about (3 + 128) 2^-24
 * |alpha| sum_k |op(A)_ik| |op(B)_kj| per entry at most (the FP32 rounding
 * of the inputs, the dropped parts, the FP32 sums over 128 terms); typical
 * errors are near 2^-24 of that sum. */
int gb_dgemm_fp32split(char transa, char transb, int m, int n, int k, double alpha, const double *A, int lda,
                       const double *B, int ldb, double beta, double *C, int ldc, void *workspace,
                       size_t ws_bytes, void *stream);
size_t gb_dsymm_sliced_workspace_bytes(char side, int m, int n);
int gb_dsymm_sliced(char side, int m, int n, double alpha, const double *S, int lds, const double *B, int ldb,
                    double beta, double *C, int ldc, void *workspace, size_t ws_bytes, void *stream);
size_t gb_dsyr2k_sliced_workspace_bytes(int n, int k);
int gb_dsyr2k_sliced(int n, int k, double alpha, const double *A, int lda, const double *B, int ldb,
                     double beta, double *C, int ldc, void *workspace, size_t ws_bytes, void *stream);
size_t gb_dsyrk_sliced_workspace_bytes(int n, int k);
int gb_dsyrk_sliced(int n, int k, double alpha, const double *A, int lda, double beta, double *C, int ldc,
                    void *workspace, size_t ws_bytes, void *stream);

/* Complex (complex128, interleaved re/im; leading dimensions in complex
 * elements) forms of the sliced products, real alpha and beta.  The complex
 * product is computed as the real product of the expanded left operand,
 * whose entries x + iy become 2 x 2 blocks [x -y; y x], with the right
 * operand and C in their interleaved storage; same accuracy statement as the
 * real forms.
 *   gb_zgemm_sliced : C (m x n) = alpha op(A) B + beta C, transa = 'N' or
 *                     'C' (conjugate transpose), op(A) m x k, B k x n.
 *   gb_zhemm_sliced : C (m x n) = alpha S B + beta C, S (m x m) Hermitian,
 *                     only its lower triangle is read (the diagonal's
 *                     imaginary parts are read as zero).
 *   gb_zher2k_sliced: lower triangle of C (n x n) = alpha (X Y^H + Y X^H)
 *                     + beta C, X, Y n x k; the diagonal's imaginary parts
 *                     are set to zero; the strict upper triangle is not
 *                     touched.
 * Pointers 16-byte aligned, workspace 256-byte aligned and at least the
 * *_workspace_bytes figure; -i for invalid argument i, GB_ERR_CUDA for a
 * launch error. */
size_t gb_zgemm_sliced_workspace_bytes(int m, int n, int k);
int gb_zgemm_sliced(char transa, int m, int n, int k, double alpha, const double *A, int lda, const double *B,
                    int ldb, double beta, double *C, int ldc, void *workspace, size_t ws_bytes, void *stream);
size_t gb_zhemm_sliced_workspace_bytes(int m, int n);
int gb_zhemm_sliced(int m, int n, double alpha, const double *S, int lds, const double *B, int ldb, double beta,
                    double *C, int ldc, void *workspace, size_t ws_bytes, void *stream);
size_t gb_zher2k_sliced_workspace_bytes(int n, int k);
int gb_zher2k_sliced(int n, int k, double alpha, const double *X, int ldx, const double *Y, int ldy, double beta,
                     double *C, int ldc, void *workspace, size_t ws_bytes, void *stream);

/* Human-readable text for a status code (never NULL). */
const char *gb_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
