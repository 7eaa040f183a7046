/*
 * bsvd.h -- batched one-sided Jacobi SVD on NVIDIA GB300 (sm_103a).
 *
 * Computes, for every matrix A_i (m_i x n_i) of a batch, the reduced SVD
 *     A_i = U_i Sigma_i V_i^H,
 * U_i: m_i x k_i and V_i: n_i x k_i with orthonormal columns, Sigma_i: k_i
 * non-negative reals in descending order, k_i = min(m_i, n_i) (Sec. 1,
 * Eq. svd, of Abdelfattah and Fasi, "An Efficient Batch Solver for the
 * Singular Value Decomposition on GPUs").  The method is the blocked
 * one-sided (Hestenes) Jacobi algorithm of Sec. 3 (Eq. block-gram, right-sv)
 * run as in Sec. 4 (steps S1-S5) with the optimisations of Sec. 5-7: one
 * inner Jacobi sweep per Gram block (Design-2), fused vector update
 * (Design-3, Alg. 4) and per-matrix masking (Design-4).
 *
 * Conventions (all entry points):
 *  - Storage is column-major with a leading dimension, LAPACK style.  Types:
 *    s = float, d = double, c = complex float, z = complex double, complex
 *    data interleaved (re, im).  Sigma is always real (float for s/c, double
 *    for d/z).
 *  - Every device pointer must be to memory of the current CUDA device; the
 *    call is asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) and returns after argument checks and kernel enqueue.
 *  - A is read only.  The caller owns every buffer, including the workspace;
 *    the library allocates no device memory.  The on-chip (FUSED) path needs
 *    no workspace for the strided form; the multi-kernel paths need
 *    bsvd_gesvj_workspace() bytes (W, V, Gram and rotation blocks per matrix).
 *  - Status codes are synchronous (argument and launch errors).  On
 *    BSVD_ERR_INVALID, bsvd_last_arg() gives the 1-based position of the
 *    offending argument.  Per-matrix results go to d_info on the device:
 *        0   converged (a full sweep in which no pair rotated);
 *        k>0 not converged after k = max_sweeps sweeps (outputs still written);
 *        -1  A_i holds a NaN or infinity (outputs set to NaN).
 *  - m < n is solved on A^H (Sec. 6.2: A^H = V Sigma U^H).
 *  - The sign (real) or phase (complex) of each singular-vector pair is
 *    unspecified; within exactly repeated singular values any orthonormal
 *    basis may be returned.
 */
#ifndef BSVD_H
#define BSVD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSVD_VERSION 1

typedef struct bsvd_handle_s* bsvd_handle;

typedef enum {
    BSVD_OK = 0,
    BSVD_ERR_INVALID = -1,          /* bad argument; see bsvd_last_arg()        */
    BSVD_ERR_WORKSPACE = -2,        /* work_bytes smaller than the query result */
    BSVD_ERR_CUDA = -3,             /* a CUDA call failed; see bsvd_last_cuda() */
    BSVD_ERR_TIMEOUT = -4,          /* a bounded device wait expired            */
    BSVD_ERR_NOT_IMPLEMENTED = -5,  /* shape/type/option combination not built  */
    BSVD_ERR_NOMEM = -6,            /* host allocation failed                   */
    BSVD_ERR_CANCELLED = -7         /* a server request cancelled before it ran */
} bsvd_status;

typedef enum { BSVD_JOB_NONE = 0, BSVD_JOB_SOME = 1 } bsvd_job;   /* economy-size vectors */

typedef enum {
    BSVD_PATH_AUTO = 0,     /* FUSED when the matrix fits on chip, else BLOCKED          */
    BSVD_PATH_FUSED = 1,    /* one kernel per matrix, A and V resident in shared memory  */
    BSVD_PATH_PLAIN = 2,    /* the paper's baseline (Sec. 4): one launch per stage and
                               round, inner eigensolver run to convergence (default 30
                               inner sweeps), two-stage vector update, no masks, batch-
                               level convergence checked on the host once per sweep (the
                               call then synchronises `stream`); FP64 comparison path   */
    BSVD_PATH_BLOCKED = 3,  /* the multi-kernel path with Designs 2-4 (one inner sweep,
                               fused update, masks); any matrix size; asynchronous      */
    BSVD_PATH_PERSISTENT = 4 /* pointer-array form: all shapes in a few persistent
                               launches, one per segment (block width x where W and V
                               live); each matrix takes the block width of its shape
                               (opts->nb, else the bucket's autotuned choice, else the
                               AUTO rule) and keeps W and V in shared memory when they
                               fit in half an SM (at least two CTAs per SM), else in a per-CTA
                               global workspace slot; CTAs take matrices from their
                               segment's queue, largest first, each solved whole.  The
                               segments run on streams the handle owns, forked from and
                               joined back to `stream` (the strided form treats it as
                               AUTO)                                                     */
} bsvd_path;

typedef enum {
    BSVD_PREC_NATIVE = 0,   /* every step in the working precision                          */
    BSVD_PREC_MIXED = 1     /* FP64 output from mostly FP32 work: FP32 sweeps on an FP32 copy
                               until the FP32 test passes, V restored to an orthonormal FP64
                               matrix, A V formed in FP64, then FP64 polish sweeps until the
                               FP64 test passes (d_sweeps reports the polish sweeps)         */
} bsvd_prec;

/* Solver options.  Zero-initialise, then set what you need; 0 = default. */
typedef struct {
    int nb;            /* block width (Sec. 4); 0 = chosen from n and the type            */
    int max_sweeps;    /* outer sweep limit; 0 = 40                                        */
    double tol;        /* pair rotates iff |g_ij| >= tol sqrt(g_ii g_jj) (Alg. 1, Alg. 2);
                          0 = 30 u, u the unit roundoff of the type (Sec. 5.4, k = 30)      */
    int inner_sweeps;  /* inner eigensolver sweeps per Gram block; 0 = 1 (Design-2, Sec. 5) */
    int path;          /* bsvd_path                                                         */
    int flags;         /* bit 0: skip the final orthogonality correction of V;
                          bit 1: two-stage vector update (Design-3 off; multi-kernel path);
                          bit 2: no masks (Design-4 off; multi-kernel path, host-checked
                          batch convergence).  Bits 1-2 with AUTO select the multi-kernel
                          path.
                          bit 3: no CUDA graph (the masked multi-kernel path otherwise
                          runs its sweeps as one graph whose conditional WHILE node
                          repeats one recorded sweep until no matrix is active or
                          max_sweeps sweeps have run, decided on the device; without
                          graphs it launches max_sweeps sweeps);
                          bit 4: without the device-side loop (graphs off, or a driver
                          without conditional graph nodes) the masked multi-kernel path
                          reads the batch's convergence on the host every 4 sweeps and
                          launches no more sweeps once every matrix has converged (the
                          call then synchronises `stream`; results are unchanged);
                          bit 5: QR pre-processing (Sec. "Pre-processing the SVD using a
                          QR Factorization"; strided form, native precision): A = Q [R; 0]
                          by Householder QR (of A^H when m < n), the SVD of the
                          min(m, n)-square R by the path `path` selects, U = Q [U_R; 0].
                          Workspace: bsvd_gesvj_workspace with the same options;
                          bit 6: with BSVD_PATH_PERSISTENT on a complex64 pointer-array
                          batch, the matrices with min(m, n) >= 112 run as one
                          variable-shape batch on the masked multi-kernel path (same
                          per-matrix arithmetic as that path on each shape alone), on a
                          stream the handle owns that is forked from and joined back to
                          `stream`, beside the persistent launch for the rest; other
                          types ignore it.  With bit 4 the call returns once those
                          matrices have converged.  Workspace: bsvd_gesvj_workspace with
                          the same options;
                          bit 7: real FP32 with nb = 8 or 16 (and complex64 on the
                          multi-kernel path) forms the Gram blocks and the rotation
                          updates on the FMA pipes instead of the tensor cores
                          (split-TF32 mma, FP32 accuracy);
                          bit 8: single-precision data (and the FP32 sweeps of MIXED)
                          take the pair test and the rotation (Eq. sin-cos) in FP64,
                          rounded once to FP32;
                          bit 9: BSVD_PATH_PERSISTENT keeps every matrix in a global
                          workspace slot (no shared-memory segments);
                          bit 10: with bit 6, real FP32 batches split the same way,
                          from min(m, n) >= 144;
                          bit 11: the masked multi-kernel path replays a one-sweep
                          graph from the host (bit 4 applies) instead of the
                          device-side conditional loop;
                          bit 12: single precision (FP32, complex64) with nb = 8 or
                          16 on the multi-kernel path runs each round as three
                          kernels (Gram, eigensolver, update, G and J through global
                          memory) instead of one pair-step kernel (same results)      */
    int prec;          /* bsvd_prec; MIXED only for d/z.  Pointer-array batches run MIXED per
                          shape group (also with BSVD_PATH_PERSISTENT), reading A and
                          writing S, U, V through the pointer arrays                     */
    int reserved[5];
} bsvd_opts;

/* Handle: caches device properties and per-device kernel set-up; owns no
 * device memory.  Not thread-safe: use one handle per host thread. */
bsvd_status bsvd_create(bsvd_handle* handle);
bsvd_status bsvd_destroy(bsvd_handle handle);
const char* bsvd_status_string(bsvd_status status);
int bsvd_last_arg(bsvd_handle handle);          /* 1-based argument index of the last INVALID */
int bsvd_last_cuda(bsvd_handle handle);         /* cudaError_t of the last ERR_CUDA            */
int bsvd_version(void);

/*
 * Workspace query for one call.  dtype is 's', 'd', 'c' or 'z'.  For the
 * strided form pass m_arr = &m, n_arr = &n and uniform = 1; for the
 * pointer-array form pass the host arrays m[batch], n[batch] and uniform = 0.
 * *bytes receives the size of d_work the call needs (possibly 0).  The query
 * uses the current device's shared-memory limit to decide which shapes run
 * on chip; with no CUDA device it assumes the GB300's 227 KB.
 */
bsvd_status bsvd_gesvj_workspace(bsvd_handle handle, char dtype, int batch, const int* m_arr,
                                 const int* n_arr, int uniform, bsvd_job jobu, bsvd_job jobv,
                                 const bsvd_opts* opts, size_t* bytes);

/*
 * How a BSVD_PATH_PERSISTENT pointer-array call with these arguments would
 * run each matrix (host only; nothing is launched).  The per-(shape, type)
 * decision layer of Sec. 4.2 ("Computation of the Gram Matrices") made
 * explicit for batches of mixed shapes.  Arguments:
 *   1 handle  2 dtype ('s','d','c','z')  3 batch >= 0  4 m[batch]  5 n[batch]
 *   6 jobu  7 jobv  8 opts  9 nb_out[batch]  10 where_out[batch]  11 launches
 * nb_out[i] receives matrix i's block width; where_out[i] 1 for W and V in
 * shared memory, 0 for a global workspace slot, 2 for the variable-shape
 * multi-kernel batch (flags bit 6), -1 for an empty matrix; *launches (may
 * be NULL) the number of persistent launches.  All arrays are host memory,
 * owned by the caller.  Returns BSVD_ERR_INVALID (bsvd_last_arg) for a bad
 * argument and BSVD_ERR_NOT_IMPLEMENTED for an unsupported block width.
 */
bsvd_status bsvd_persistent_plan(bsvd_handle handle, char dtype, int batch, const int* m_arr, const int* n_arr,
                                 bsvd_job jobu, bsvd_job jobv, const bsvd_opts* opts, int* nb_out,
                                 int* where_out, int* launches);

/*
 * Strided batch: every matrix has the same m and n; matrix i of X starts at
 * dX + i * strideX (in elements).  Arguments (1-based positions for
 * bsvd_last_arg):
 *   1 handle   2 jobu   3 jobv   4 batch >= 0   5 m >= 0   6 n >= 0
 *   7 dA (device, read only)   8 lda >= max(1, m)   9 strideA >= lda * n
 *  10 dS (device, k reals per matrix)   11 strideS >= k
 *  12 dU (device; ignored when jobu = NONE)   13 ldu >= max(1, m)   14 strideU >= ldu * k
 *  15 dV (device; ignored when jobv = NONE)   16 ldv >= max(1, n)   17 strideV >= ldv * k
 *  18 d_info (device, batch ints)   19 d_sweeps (device, batch ints, or NULL)
 *  20 d_work (device, 16-byte aligned)   21 work_bytes   22 opts (NULL = defaults)
 *  23 stream
 */
#define BSVD_STRIDED_ARGS(T, R)                                                             \
    bsvd_handle handle, bsvd_job jobu, bsvd_job jobv, int batch, int m, int n,               \
    const T* dA, int lda, long long strideA, R* dS, long long strideS,                       \
    T* dU, int ldu, long long strideU, T* dV, int ldv, long long strideV,                    \
    int* d_info, int* d_sweeps, void* d_work, size_t work_bytes, const bsvd_opts* opts,      \
    void* stream

bsvd_status bsvd_sgesvj_strided(BSVD_STRIDED_ARGS(float, float));
bsvd_status bsvd_dgesvj_strided(BSVD_STRIDED_ARGS(double, double));
bsvd_status bsvd_cgesvj_strided(BSVD_STRIDED_ARGS(void, float));    /* T = complex float  */
bsvd_status bsvd_zgesvj_strided(BSVD_STRIDED_ARGS(void, double));   /* T = complex double */

/*
 * Strided batch with HOST buffers (the paper has no counterpart; for callers
 * whose matrices live in host memory).  Same arguments as the strided call,
 * with A, S, U, V, info and sweeps in host memory -- page-locked
 * (cudaHostAlloc / cudaHostRegister) for the copies to overlap, pageable
 * works but each copy then waits -- and d_work a device workspace of
 * bsvd_gesvj_host_workspace() bytes (256-byte aligned).  The batch is cut
 * into up to four chunks of at least 4 x SMs matrices: chunk c+1 is copied in
 * and chunk c-1's results copied out while chunk c is solved, on two
 * handle-owned copy streams, and alternate chunks are solved on `stream` and
 * a second handle-owned stream so one chunk's last wave overlaps the next
 * chunk's first.  Returns after enqueueing; the host outputs are complete
 * once `stream` reaches the end of the call.  Do not touch the host buffers
 * before then.  Argument positions as for the strided call (host pointers in
 * place of device ones); opts as for the strided call.
 */
#define BSVD_STRIDED_HOST_ARGS(T, R)                                                        \
    bsvd_handle handle, bsvd_job jobu, bsvd_job jobv, int batch, int m, int n,               \
    const T* hA, int lda, long long strideA, R* hS, long long strideS,                       \
    T* hU, int ldu, long long strideU, T* hV, int ldv, long long strideV,                    \
    int* h_info, int* h_sweeps, void* d_work, size_t work_bytes, const bsvd_opts* opts,      \
    void* stream

bsvd_status bsvd_gesvj_host_workspace(bsvd_handle handle, char dtype, int batch, int m, int n,
                                      bsvd_job jobu, bsvd_job jobv, const bsvd_opts* opts, size_t* bytes);
bsvd_status bsvd_sgesvj_strided_host(BSVD_STRIDED_HOST_ARGS(float, float));
bsvd_status bsvd_dgesvj_strided_host(BSVD_STRIDED_HOST_ARGS(double, double));
bsvd_status bsvd_cgesvj_strided_host(BSVD_STRIDED_HOST_ARGS(void, float));
bsvd_status bsvd_zgesvj_strided_host(BSVD_STRIDED_HOST_ARGS(void, double));

/*
 * Autotuner (the paper's "decision layer" of Sec. 4.2 picks a GEMM kernel from
 * an offline table; here the whole configuration is timed online).  Times the
 * candidates -- block width nb in {4, 8, 16, 32} x {on-chip fused path,
 * multi-kernel path}, which also fixes the threads per matrix -- on the first
 * min(batch, 512) matrices of the caller's strided batch (read only), keeps
 * the fastest one whose every matrix converged, records it in the handle for
 * the bucket (type, m and n rounded up to powers of two, jobu, jobv), and
 * writes it to *best (base options with path and nb set).  Later AUTO calls
 * without an explicit nb in that bucket follow it.  times_ms (8 floats, or
 * NULL) receives each candidate's time, -1 when not run.  Synchronises
 * `stream`.  Workspace: bsvd_autotune_workspace bytes.  Arguments:
 *   1 handle 2 dtype 3 jobu 4 jobv 5 batch 6 m 7 n 8 dA 9 lda 10 strideA
 *  11 d_work 12 work_bytes 13 base (NULL = defaults) 14 best 15 times_ms 16 stream
 */
bsvd_status bsvd_autotune_workspace(bsvd_handle handle, char dtype, int batch, int m, int n,
                                    bsvd_job jobu, bsvd_job jobv, const bsvd_opts* base, size_t* bytes);
bsvd_status bsvd_autotune(bsvd_handle handle, char dtype, bsvd_job jobu, bsvd_job jobv, int batch, int m,
                          int n, const void* dA, int lda, long long strideA, void* d_work,
                          size_t work_bytes, const bsvd_opts* base, bsvd_opts* best, float* times_ms,
                          void* stream);

/*
 * Autotuner for pointer-array batches of mixed shapes (the decision layer of
 * Sec. 4.2, per size bucket).  The batch's matrices are grouped into buckets
 * (type, m and n rounded up to powers of two, jobu, jobv); for each bucket
 * persistent launches (BSVD_PATH_PERSISTENT) of a sample -- its first
 * min(count, sample) matrices, fewer (at least 2) for shapes whose M N^2
 * exceeds 64 times that of a 64 x 64 matrix -- are timed with block width
 * nb = 4 (N <= 32), 8 and 16 (N >= 16), N rounded up to a power of two
 * (the width also fixes the threads per matrix: 64, 128, 256 per CTA; on
 * chip or in global slots follows from the fit at each width).  The fastest width
 * whose every matrix converged is recorded in the handle for the bucket;
 * later persistent calls (and AUTO strided calls) of that bucket use it.  The
 * caller's matrices are read only; the sample's results go to d_work.
 * Synchronises `stream`.  Workspace: bsvd_autotune_batched_workspace bytes.
 * Arguments:
 *   1 handle 2 dtype 3 jobu 4 jobv 5 batch 6 m[] 7 n[] (host) 8 dA[] (device
 *   array of device pointers) 9 lda[] (host) 10 d_work 11 work_bytes 12 base
 *   (NULL = defaults) 13 sample >= 1 14 max_out >= 0 15 bucket_mn[2 max_out]
 *   16 nb_out[max_out] 17 times_ms[3 max_out] 18 buckets 19 stream
 * For the first max_out buckets (in ascending key order), bucket_mn receives
 * the bucket's rounded (M, N), nb_out the chosen width (0: no candidate
 * converged), times_ms the three candidates' times (-1: not run); each may
 * be NULL.  *buckets (may be NULL) receives the number of buckets.
 */
bsvd_status bsvd_autotune_batched_workspace(bsvd_handle handle, char dtype, int batch, const int* m, const int* n,
                                            bsvd_job jobu, bsvd_job jobv, const bsvd_opts* base, int sample,
                                            size_t* bytes);
bsvd_status bsvd_autotune_batched(bsvd_handle handle, char dtype, bsvd_job jobu, bsvd_job jobv, int batch,
                                  const int* m, const int* n, const void* const* dA, const int* lda, void* d_work,
                                  size_t work_bytes, const bsvd_opts* base, int sample, int max_out,
                                  int* bucket_mn, int* nb_out, float* times_ms, int* buckets, void* stream);

/*
 * Strided FP64 batch that allocates nothing (the paper has no counterpart).
 * For callers that cannot allocate device memory: code inside a framework
 * that owns the device-memory budget, code on a latency path where
 * cudaMalloc's implicit device synchronisation is not acceptable, or callers
 * with no allocator to size and pass a workspace.  Same arguments as
 * bsvd_dgesvj_strided minus d_work / work_bytes; the multi-kernel path runs
 * (PLAIN if opts->path asks for it, BLOCKED otherwise) with its workspace in a
 * static 32 MiB device array that every GPU loading the library holds until
 * exit.  A batch whose workspace exceeds 32 MiB (more than 203 matrices of
 * 128 x 64) returns BSVD_ERR_WORKSPACE and launches nothing.  Every call
 * looks up the array's device address with the calling thread's device
 * current (so a cudaDeviceReset leaves no stale address behind); the first
 * call on a device may load the module, so make it before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU
 * race: serialise them.
 */
bsvd_status bsvd_dgesvj_strided_noalloc(bsvd_handle handle, bsvd_job jobu, bsvd_job jobv, int batch,
                                        int m, int n, const double* dA, int lda, long long strideA,
                                        double* dS, long long strideS, double* dU, int ldu,
                                        long long strideU, double* dV, int ldv, long long strideV,
                                        int* d_info, int* d_sweeps, const bsvd_opts* opts,
                                        void* stream);

/*
 * Pointer-array batch (per-matrix shapes).  dA, dS, dU, dV are DEVICE arrays
 * of `batch` device pointers (as in batched BLAS); m, n, lda, ldu, ldv are
 * HOST arrays of `batch` ints.  Matrices are grouped by shape on the host and
 * each group runs as one launch.  Arguments:
 *   1 handle 2 jobu 3 jobv 4 batch 5 m[] 6 n[] 7 dA[] 8 lda[] 9 dS[]
 *  10 dU[] 11 ldu[] 12 dV[] 13 ldv[] 14 d_info 15 d_sweeps 16 d_work
 *  17 work_bytes 18 opts 19 stream
 */
#define BSVD_BATCHED_ARGS(T, R)                                                             \
    bsvd_handle handle, bsvd_job jobu, bsvd_job jobv, int batch, const int* m, const int* n, \
    const T* const* dA, const int* lda, R* const* dS, T* const* dU, const int* ldu,          \
    T* const* dV, const int* ldv, int* d_info, int* d_sweeps, void* d_work,                  \
    size_t work_bytes, const bsvd_opts* opts, void* stream

bsvd_status bsvd_sgesvj_batched(BSVD_BATCHED_ARGS(float, float));
bsvd_status bsvd_dgesvj_batched(BSVD_BATCHED_ARGS(double, double));
bsvd_status bsvd_cgesvj_batched(BSVD_BATCHED_ARGS(void, float));
bsvd_status bsvd_zgesvj_batched(BSVD_BATCHED_ARGS(void, double));

/*
 * Serving loop: a stream of single-matrix requests, solved with continuous
 * batching.  The paper solves whole batches given at once and has no
 * serving layer; this one is built on the persistent launch above (Sec. 7's
 * per-matrix masking carried to its end: a matrix that converges leaves its
 * CTA, which takes the next matrix of the batch).
 *
 * A worker thread owned by the server takes queued requests in arrival
 * order, groups them into batches of one key (type, jobs, block width 4/8/16
 * from min(m, n) as the AUTO choice; above big_k columns also the shape),
 * and launches each batch on a stream of its own, up to max_inflight batches
 * at once: requests that arrive while batches run start as soon as a stream
 * and device memory are free, and new batches take over SMs as the CTAs of
 * earlier ones run out of matrices.  Requests with min(m, n) <= big_k run in
 * the persistent kernel (one CTA per matrix, its A, V and sweep state
 * resident until it converges), and each one completes the moment its CTA
 * raises its flag in host-mapped memory, without waiting for the rest of its
 * batch.  Larger requests run on the multi-kernel path (many CTAs per
 * matrix) and complete with their batch.  A request's arithmetic does not
 * depend on what it is batched with, so its result is the same, bit for
 * bit, alone or in any mix.
 *
 * Memory: every device byte the server uses comes from the caller's arena
 * (d_arena, arena_bytes; 256-byte aligned, owned by the caller, not freed):
 * per batch its workspace (freed when the batch ends) and its requests'
 * outputs S, U, V (freed when the last of them is released).  A batch is
 * admitted only if both fit; otherwise the queue waits (first come, first
 * served) until memory is released.  A request that could not fit even in
 * an empty arena completes at once with status BSVD_ERR_WORKSPACE.
 * Unreleased results hold their memory: release them.
 *
 * Inputs are read in place by the kernels: A must be device memory or
 * page-locked host memory (cudaHostAlloc / cudaHostRegister), checked at
 * submit (pageable memory returns BSVD_ERR_INVALID), and must stay valid and
 * unchanged until the request completes.
 *
 * Times are seconds of the steady clock bsvd_server_clock() reads; a
 * request's latency is t_done - t_submit, t_done the moment the worker saw
 * its completion.
 */
typedef struct bsvd_server_s* bsvd_server;

typedef struct {
    int max_inflight;   /* batches on the GPU at once, each on its own stream; 0 = 32, at most 64;
                           multi-kernel batches hold at most max_inflight - max(2, max_inflight/4) */
    int max_batch;      /* requests per persistent batch; 0 = 4096                               */
    int big_k;          /* min(m, n) above which the multi-kernel path serves; 0 = 256          */
    int max_big_batch;  /* requests per multi-kernel batch; 0 = 8                                */
    int fp64_prec;      /* bsvd_prec of FP64 / complex128 requests on the multi-kernel path
                           (min(m, n) > big_k): BSVD_PREC_NATIVE (0, default) or
                           BSVD_PREC_MIXED (FP32 sweeps + FP64 polish, FP64 accuracy)      */
    int big_flags;      /* further bsvd_opts.flags bits for multi-kernel batches (which always
                           run with bits 4 and 11: a host-replayed one-sweep graph)        */
    int big_k_fp64;     /* big_k for FP64 / complex128 requests; 0 = big_k.  A persistent
                           batch solves each matrix on one SM: a smaller limit spreads
                           the medium FP64 requests over the GPU                           */
    int reserved[1];    /* zero                                                                  */
} bsvd_server_opts;

double bsvd_server_clock(void);

/* Creates a server on the current device (opts NULL = defaults).
 * BSVD_ERR_INVALID: null out, arena NULL, misaligned or under 1 MiB, bad opts. */
bsvd_status bsvd_server_create(void* d_arena, size_t arena_bytes, const bsvd_server_opts* opts,
                               bsvd_server* out);

/* Queues the SVD of one m x n matrix (column-major, leading dimension lda) of
 * type dtype ('s', 'd', 'c', 'z'); jobu / jobv as for the batch calls.  Returns
 * a request id (> 0) in *id.  Thread-safe. */
bsvd_status bsvd_server_submit(bsvd_server server, char dtype, int m, int n, const void* A, int lda,
                               bsvd_job jobu, bsvd_job jobv, long long* id);

/* Submits `count` requests, request i at t0 + t_offset[i] (t0 = the clock at
 * the call, t_offset ascending, seconds), each with that scheduled time as
 * its t_submit: a load generator that replays an arrival trace at the
 * server, returning once the last request is queued.  ids (count) receives
 * the ids, *t0 the start time.  Stops at the first request submit rejects
 * and returns its status (ids of the ones before are valid). */
bsvd_status bsvd_server_replay(bsvd_server server, int count, const double* t_offset, const char* dtype,
                               const int* m, const int* n, const void* const* A, const int* lda,
                               bsvd_job jobu, bsvd_job jobv, long long* ids, double* t0);

/* 1: done (results ready), 0: queued or running, BSVD_ERR_WORKSPACE: the
 * request can never fit the arena, BSVD_ERR_CUDA: its batch failed to launch
 * or run, BSVD_ERR_CANCELLED: cancelled, BSVD_ERR_INVALID: unknown or
 * released id. */
int bsvd_server_test(bsvd_server server, long long id);

/* Blocks until the request completes or timeout_s passes (< 0: no limit;
 * BSVD_ERR_TIMEOUT then).  info: as d_info of the batch calls (for a request
 * whose batch failed to launch with BSVD_ERR_CUDA, the cudaError_t); sweeps; t_done.
 * Any output pointer may be NULL.  Returns the request's status (see test). */
bsvd_status bsvd_server_wait(bsvd_server server, long long id, double timeout_s, int* info, int* sweeps,
                             double* t_done);

/* Device pointers to a done request's S (k reals), U (m x k, ld *ldu) and
 * V (n x k, ld *ldv) in the arena, valid until it is released (NULL when
 * not computed). */
bsvd_status bsvd_server_result(bsvd_server server, long long id, void** dS, void** dU, int* ldu,
                               void** dV, int* ldv);

/* Copies a done request's S, U (ldu >= m), V (ldv >= n) into caller memory
 * (host or device; NULL skips), synchronously.  Do not release the request
 * while a fetch of it runs. */
bsvd_status bsvd_server_fetch(bsvd_server server, long long id, void* S, void* U, int ldu, void* V,
                              int ldv);

/* Frees a completed request's outputs and forgets it.  BSVD_ERR_INVALID if
 * it is unknown or not complete. */
bsvd_status bsvd_server_release(bsvd_server server, long long id);

/* Completion queue: writes up to max requests completed since the last
 * collect (in completion order) and returns how many; with release != 0 they
 * are released as they are collected.  status: 0 or the failure status;
 * info, sweeps as for wait; any array may be NULL. */
int bsvd_server_collect(bsvd_server server, int max, int release, long long* ids, int* status, int* info,
                        int* sweeps, double* t_submit, double* t_done);

/* Cancels every queued request and stops the running persistent batches
 * from starting more matrices (those already started finish; multi-kernel
 * batches run to their end).  Each request that does not run completes with
 * status BSVD_ERR_CANCELLED.  Returns at once. */
bsvd_status bsvd_server_cancel(bsvd_server server);

/* paused != 0: admit no new batch (queued requests wait, running batches
 * go on); 0: resume.  For draining a server or forming one batch on purpose. */
bsvd_status bsvd_server_pause(bsvd_server server, int paused);

/* counters[10]: submitted, completed, failed, queued, running requests,
 * running batches, arena bytes in use, peak arena bytes in use, cancelled,
 * batches launched. */
bsvd_status bsvd_server_stats(bsvd_server server, long long* counters);

/* Cancels as bsvd_server_cancel does, waits for the running batches to end,
 * frees everything the server owns (not the arena).  Not concurrent with
 * other calls on the server. */
bsvd_status bsvd_server_destroy(bsvd_server server);

#ifdef __cplusplus
}
#endif

#endif /* BSVD_H */
