/*
 * edm.h -- C ABI of libedm: all-to-all convergent cross mapping (CCM) on one
 * NVIDIA GB300 (sm_103a), after kEDM (Takahashi, Widanage, Pao; PEARC'21).
 *
 * Method (kEDM section 2.1, steps 1-4):
 *   1. embed a library series X with lag tau in E dimensions:
 *        x(t) = (X(t), X(t-tau), ..., X(t-(E-1)tau));
 *   2. find the k = E+1 nearest neighbours t_1..t_k of every library point
 *      (Euclidean distance, the point itself excluded);
 *   3. predict a target Y as  Yhat(t+Tp) = sum_r w_r Y(t_r+Tp) / sum_r w_r,
 *      w_r = exp(-d(t,t_r) / d(t,t_1));
 *   4. score the prediction with Pearson's rho against Y(t+Tp).
 * The neighbour table of a library is built once and reused for every target
 * (closing paragraph of section 2.1).
 *
 * Conventions shared by every call:
 *   - Series are float32, row-major [N][L]; a series is a row.
 *   - The points of a library are the times P = {t : (E-1)tau <= t <= L-1-Tp};
 *     n = L-(E-1)tau-Tp of them.  The library set is the prediction set
 *     (leave-one-out).  Row i of any per-point output is time t = (E-1)tau+i.
 *   - Neighbours are ranked by the squared distance accumulated in lag order
 *     with fused multiply-adds; exact ties go to the lower time index.  The
 *     neighbour sets equal those of an FP64 evaluation of that definition.
 *   - If the nearest distance is 0 then w_r = 1 for d_r = 0, else 0.
 *   - A zero-variance prediction or observation gives rho = NaN.
 *
 * Memory and streams: every array argument is a DEVICE pointer owned by the
 * caller (unless stated otherwise); libedm never frees it.  A context owns
 * its own workspace (neighbour tables, transposed targets), grown on demand
 * with cudaMalloc and freed by edm_destroy.  All work is enqueued on the
 * context's stream and is asynchronous to the host.
 *
 * Errors: arguments are checked before anything is enqueued; a bad argument
 * returns EDM_ERR_INVALID_ARG and enqueues nothing.  Launch failures return
 * EDM_ERR_CUDA.  Conditions found on the device (an out-of-range E in a
 * device array, a bounded wait that gave up) are recorded in the context and
 * reported by edm_ctx_sync.  No call throws; no call aborts the process.
 */
#ifndef EDM_H
#define EDM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum edm_status {
    EDM_OK = 0,
    EDM_ERR_INVALID_ARG = 1, /* an argument is out of range or NULL        */
    EDM_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed       */
    EDM_ERR_OOM = 3,         /* workspace allocation failed                */
    EDM_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up         */
    EDM_ERR_INTERNAL = 5     /* an internal consistency check failed       */
} edm_status;

/* Storage of the target series inside the CCM calls.  Library distances,
 * weights and the Pearson moments are FP32 in every mode; the 16-bit modes
 * halve the bytes of every gathered target value.  Each target is centred on
 * its FP64 mean before it is stored.
 *   EDM_BF16_TARGETS: 8 significant bits.  Measured |rho - rho_FP64| stays
 *     below 1e-3 for library lengths of 300 points or more; at 100 points it
 *     reaches about 1.5e-3 on a few pairs in a thousand.
 *   EDM_FP16_TARGETS: 11 significant bits.  Each centred target is first
 *     multiplied by a power of two that puts its largest magnitude in
 *     [2^13, 2^14), so no value overflows; rho does not depend on the scale.
 *     About 8 times more accurate than BF16 for the same bytes. */
typedef enum edm_precision {
    EDM_FP32 = 0,          /* targets stored as float32                   */
    EDM_BF16_TARGETS = 1,  /* targets stored as bfloat16 (half the bytes) */
    EDM_FP16_TARGETS = 2   /* targets stored as scaled float16 (half the bytes) */
} edm_precision;

enum {
    EDM_E_MAX = 20, /* largest embedding dimension accepted             */
    EDM_K_MAX = 24, /* largest neighbour count accepted by edm_knn      */
    EDM_L_MAX = 65535 /* longest series (neighbour indices are 16-bit)  */
};

typedef struct edm_ctx edm_ctx;

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  Returns EDM_ERR_CUDA when no such device exists. */
edm_status edm_create(edm_ctx **out, int device, void *cuda_stream);

/* Synchronise the context's stream and free its workspace and itself. */
edm_status edm_destroy(edm_ctx *ctx);

/* Enqueue subsequent calls on `cuda_stream` (a cudaStream_t). */
edm_status edm_set_stream(edm_ctx *ctx, void *cuda_stream);

/* Block until the context's stream is idle; return (and clear) the first
 * device-side error recorded since the previous edm_ctx_sync. */
edm_status edm_ctx_sync(edm_ctx *ctx);

/* Static English text for a status code. */
const char *edm_status_string(edm_status s);

/* Detail of the last host-side error of this context (static buffer owned by
 * the context; empty when none). */
const char *edm_last_error(edm_ctx *ctx);

/* Number of kernels libedm has launched through this context. */
uint64_t edm_kernel_launches(edm_ctx *ctx);

/* Diagnostics of the exact kNN (no counterpart in the paper).  With the
 * option "diagnostics" set to 1, every kernel that selects neighbours counts
 * the query rows (one per row and E) whose FP32 ranking left a candidate
 * inside the band around the k-th distance, so that the row was resolved in
 * FP64 (band_rows), and among them the rows with so many tied candidates
 * that a full FP64 scan was needed (brute_rows).  This call synchronises the
 * context's stream, returns both counts accumulated since the previous call
 * and resets them. */
edm_status edm_fallback_counts(edm_ctx *ctx, uint64_t *band_rows, uint64_t *brute_rows);

/* Measurement aids (no counterpart in the paper).
 * edm_profile_enable(ctx, 1) clears the record and times every kernel this
 * context launches from then on with CUDA events on its stream; 0 stops.
 * edm_profile_read synchronises the stream and returns, for the kernels
 * whose name equals `kernel` (e.g. "lookup_kernel"), the summed device time
 * in milliseconds and the number of launches. */
edm_status edm_profile_enable(edm_ctx *ctx, int on);
edm_status edm_profile_read(edm_ctx *ctx, const char *kernel, double *total_ms,
                            int *launches);

/* Shared-memory gather bandwidth of this GPU in bytes/s, the roofline of the
 * lookup kernel: every SM runs warps that read whole 128-byte rows of a
 * shared-memory tile at data-dependent row indexes (the lookup's access
 * pattern, one conflict-free wavefront per read) for about `ms` ms. */
edm_status edm_probe_smem_bandwidth(edm_ctx *ctx, double ms, double *bytes_per_s);

/* L2 gather bandwidth of this GPU in bytes/s, the roofline of the lookup
 * when a target tile does not fit shared memory (series longer than about
 * 3,300 points) and its gathers go to L2: warps read whole 128-byte rows of
 * a 48 MB global buffer (resident in L2) at scattered row indexes for about
 * `ms` ms.  Allocates and frees its buffer. */
edm_status edm_probe_l2_bandwidth(edm_ctx *ctx, double ms, double *bytes_per_s);

/* Failure-detection check (no counterpart in the paper).  Every wait inside
 * a libedm kernel is bounded: after its limit it records EDM_ERR_TIMEOUT in
 * the context, sets an abort word of its thread block so that the block's
 * later waits return at once, and the kernel runs to its end, so a lost
 * arrival never hangs the GPU.  This call enqueues one thread that waits
 * twice, with that same bounded wait, on a barrier nothing completes: the
 * first wait gives up after `ms` milliseconds (1..10000), the second returns
 * at once.  The next edm_ctx_sync then returns EDM_ERR_TIMEOUT (and clears
 * it); the context stays usable. */
edm_status edm_check_wait_timeout(edm_ctx *ctx, int ms);

/* Section 2.1 step 1: time-delay embedding of one series.
 * x [L] float32; out [L-(E-1)tau][E] float32, row i = time (E-1)tau+i,
 * column l = x[t - l*tau].  1 <= E <= EDM_E_MAX, tau >= 1, (E-1)tau < L. */
edm_status edm_embed(edm_ctx *ctx, const float *x, int L, int E, int tau,
                     float *out);

/* Section 2.1 step 2 (and Algorithms 1-2): exhaustive all-kNN of N series.
 * X [N][L] float32.  For each series and each point t in P, the k nearest
 * points of P\{t}, ascending by (squared distance, time index).
 * idx  [N][n][k] int32: the neighbour's time index u (not shifted by Tp);
 * dist [N][n][k] float32: the Euclidean distance, i.e. the FP64 square root
 * of the FP64 squared distance, rounded to float32.  dist may be NULL.
 * 1 <= E <= EDM_E_MAX, tau >= 1, Tp >= 0, 1 <= k <= EDM_K_MAX, k <= n-1,
 * 2 <= L <= EDM_L_MAX, N >= 1. */
edm_status edm_knn(edm_ctx *ctx, const float *X, int N, int L, int E, int tau,
                   int Tp, int k, int32_t *idx, float *dist);

/* edm_knn computed the way of the paper's Algorithms 1 and 2, as a measured
 * baseline for the fused kernels (no new capability): for each series, one
 * kernel writes the full n x n matrix of FP32 squared distances to device
 * memory (a context workspace of 4 n^2 bytes), then a second kernel selects
 * every row's k nearest from it, with the same exact FP64 ordering step.
 * Arguments and results as for edm_knn; the results are identical. */
edm_status edm_knn_materialized(edm_ctx *ctx, const float *X, int N, int L, int E, int tau,
                                int Tp, int k, int32_t *idx, float *dist);

/* Optimal embedding dimension per series (named in section 3.3; the method
 * is leave-one-out simplex projection of the series onto itself at horizon
 * Tp_sel, E = 1..E_max).  X [N][L] float32.
 * E_opt [N] int32: argmax_E rho_E (NaN ranks below every number, ties go
 * to the smaller E; 1 when every rho_E is NaN).
 * rho_E [N][E_max] float32 or NULL: the skill of every E (NaN when E leaves
 * fewer than E+2 points).  1 <= E_max <= EDM_E_MAX, tau >= 1, Tp_sel >= 0. */
edm_status edm_simplex_optimal_E(edm_ctx *ctx, const float *X, int N, int L,
                                 int E_max, int tau, int Tp_sel,
                                 int32_t *E_opt, float *rho_E);

/* edm_simplex_optimal_E for callers that must not allocate device memory.
 * The paper has no counterpart; this is a deployment variant.  It is meant
 * for code that may not call cudaMalloc once it is running: a latency-bound
 * streaming pipeline (cudaMalloc can synchronise the whole device and takes
 * unbounded time), a plug-in inside a host application or framework whose
 * own allocator owns the GPU's memory, or a service that reserves all device
 * memory at start-up.  It takes no context and allocates nothing: the
 * caller passes inputs and outputs (device pointers, as for
 * edm_simplex_optimal_E) and a stream (cudaStream_t; NULL = legacy default).
 * Its only scratch memory, the partial Pearson moments, is a fixed array of
 * 2^19 doubles (4 MiB) compiled into the library, which every GPU that loads
 * the library keeps until the process exits.  Capacity: N * E_max must not
 * exceed 104,857 (for example N <= 5,242 series at E_max = 20); larger
 * requests return EDM_ERR_INVALID_ARG before anything is enqueued.
 * The first call on a device looks up the array's device address (with that
 * device current), so make that first call before any stream capture.
 * Every call shares the one array: the sweep kernel rewrites every entry the
 * finishing kernel reads, so nothing stale is used, but two calls whose work
 * overlaps on the GPU (different streams, or different host threads) race
 * and both results are then undefined.  Serialise them.
 * It runs the same sweep and finishing kernels, with the same split of query
 * rows into blocks, as edm_simplex_optimal_E, so the results are the same.
 * Only if that split's partial moments did not fit the array (possible on a
 * GPU with many more SMs) would it use one block per series; the FP64
 * summation order then changes, rho_E can differ in the last bits and E*
 * only at a near-tie.  Errors are returned only as status codes (there is no
 * context to hold a message): EDM_ERR_CUDA for a launch failure, and also
 * when a CUDA error was already pending before the call (it is left pending
 * for its owner). */
edm_status edm_simplex_optimal_E_noalloc(const float *X, int N, int L, int E_max,
                                         int tau, int Tp_sel, int32_t *E_opt,
                                         float *rho_E, void *cuda_stream);

/* Section 2.1 steps 1-4 for every (library, target) pair (pairwise CCM,
 * section 3.3 "Lookup").  X_lib [N_lib][L], Y_tgt [N_tgt][L] float32 (they
 * may be the same array).  E_lib [N_lib] int32 on the device: the embedding
 * dimension of each library (1..EDM_E_MAX; a value out of range, or one that
 * leaves fewer than E+2 points, gives a row of NaN and EDM_ERR_INVALID_ARG
 * from the next edm_ctx_sync).
 * rho [N_lib][N_tgt] float32 row-major: rho[i][j] = Pearson skill of library
 * i's manifold predicting target j; high means "target j CCM-causes library
 * i".  prec selects the storage of the targets. */
edm_status edm_ccm_all(edm_ctx *ctx, const float *X_lib, int N_lib,
                       const float *Y_tgt, int N_tgt, int L,
                       const int32_t *E_lib, int tau, int Tp,
                       edm_precision prec, float *rho);

/* Row block of one all-to-all CCM problem (section 2.1: libraries are
 * independent, so the rows of rho can be computed in blocks, e.g. one block
 * per GPU with the series replicated on every GPU).  X [N][L] float32 holds
 * the series, which serve both as libraries and as targets; E_lib [N] int32
 * (device) the E of every series; only the library rows lib_begin ..
 * lib_end-1 are computed: rho [lib_end-lib_begin][N] float32, row r = library
 * lib_begin + r.  0 <= lib_begin <= lib_end <= N; an empty block does
 * nothing.  Otherwise as edm_ccm_all. */
edm_status edm_ccm_rows(edm_ctx *ctx, const float *X, int N, int L, int lib_begin, int lib_end,
                        const int32_t *E_lib, int tau, int Tp, edm_precision prec, float *rho);

/* edm_ccm_all that also delivers rho to host memory (no counterpart in the
 * paper).  rho [N_lib][N_tgt] (device) as in edm_ccm_all; rho_host: a
 * page-locked host buffer of the same shape (cudaMallocHost or
 * cudaHostRegister; other memory returns EDM_ERR_INVALID_ARG).  Library rows
 * are computed in about 16 blocks; each finished block is copied to rho_host
 * on a second stream while the next block computes, so only the last
 * block's copy is not hidden.  Everything, copies included, is complete
 * when work queued afterwards on the context's stream runs (edm_ctx_sync
 * waits for it). */
edm_status edm_ccm_all_host(edm_ctx *ctx, const float *X_lib, int N_lib,
                            const float *Y_tgt, int N_tgt, int L,
                            const int32_t *E_lib, int tau, int Tp,
                            edm_precision prec, float *rho, float *rho_host);

/* Stream-ordered upload of N series of L float32 values (no counterpart in
 * the paper): X_host, page-locked host memory (cudaMallocHost or
 * cudaHostRegister; other memory returns EDM_ERR_INVALID_ARG), is copied to
 * the device array X [N][L] on the context's stream, so that a whole CCM
 * step -- upload, optimal E, tables, lookup, download through
 * edm_ccm_all_host -- is one ordered sequence of library calls.  The copy is
 * complete when work queued after it on the context's stream runs. */
edm_status edm_upload_series(edm_ctx *ctx, const float *X_host, int N, int L, float *X);

/* Pairwise CCM with the embedding dimension chosen per TARGET (section 3.3:
 * targets are grouped by their optimal E, and for each group every library
 * is embedded at that E and gets one neighbour table).  Arguments as for
 * edm_ccm_all, except E_tgt [N_tgt] int32 (device): the E of each target;
 * rho[i][j] is then the skill of library i embedded at E_tgt[j] predicting
 * target j.  The call reads E_tgt back to the host (it synchronises the
 * context's stream once) and runs one CCM pass per distinct E.  An E_tgt
 * value outside 1..EDM_E_MAX, or one leaving fewer than E+2 points, returns
 * EDM_ERR_INVALID_ARG before any work is enqueued. */
edm_status edm_ccm_all_target_E(edm_ctx *ctx, const float *X_lib, int N_lib,
                                const float *Y_tgt, int N_tgt, int L,
                                const int32_t *E_tgt, int tau, int Tp,
                                edm_precision prec, float *rho);

/* Section 2.1 step 3 / Algorithm 3 with its output written: simplex
 * predictions (forecasts at horizon Tp) of target series from library
 * manifolds.  X_lib [N_lib][L], Y_tgt [N_tgt][L] float32; E_lib [N_lib] int32
 * (device); tgt_of_lib [N_lib] int32 (device): the target row each library
 * predicts, or NULL for target i = library i (then N_tgt >= N_lib).
 * pred [N_lib][L] float32: pred[i][t+Tp] = sum_r w_r Y_j[u_r+Tp] for every
 * library point t of library i (j its target, u_r its neighbours, w_r the
 * normalised simplex weights); every other entry is NaN.  With Y = X and
 * tgt_of_lib = NULL this is the leave-one-out simplex forecast of each
 * series.  An E or a target index out of range gives a NaN row and
 * EDM_ERR_INVALID_ARG from the next edm_ctx_sync. */
edm_status edm_predict(edm_ctx *ctx, const float *X_lib, int N_lib, const float *Y_tgt,
                       int N_tgt, int L, const int32_t *E_lib, const int32_t *tgt_of_lib,
                       int tau, int Tp, float *pred);

/* Convergence with library length (the "convergent" of CCM, section 2.1):
 * all-to-all CCM restricted to the window X[i][offset .. offset+L_win) of
 * every series, which serves both as library and as target.  X [N][ld]
 * float32 (row stride ld >= offset + L_win); E_lib [N] int32 (device);
 * rho [N][N] float32 as in edm_ccm_all.  Calling it for growing L_win shows
 * whether the cross-map skill converges. */
edm_status edm_ccm_window(edm_ctx *ctx, const float *X, int N, int ld, int offset,
                          int L_win, const int32_t *E_lib, int tau, int Tp,
                          edm_precision prec, float *rho);

/* Convergence over several library windows of the same length (random or
 * chosen windows, e.g. to average the skill at each library length):
 * edm_ccm_window for every window w = 0..n_windows-1 starting at offsets[w]
 * (a HOST array, read before the call returns; 0 <= offsets[w] and
 * offsets[w] + L_win <= ld).  rho [n_windows][N][N] float32 (device):
 * block w is the rho matrix of window w. */
edm_status edm_ccm_windows(edm_ctx *ctx, const float *X, int N, int ld, const int *offsets,
                           int n_windows, int L_win, const int32_t *E_lib, int tau, int Tp,
                           edm_precision prec, float *rho);

/* One all-to-all CCM problem inside a batch: the series X [N][L] are both
 * the libraries and the targets; only the library rows lib_begin..lib_end-1
 * are computed (so a problem can be split or resumed by row block).
 * E_lib [N] int32 (device); rho [lib_end-lib_begin][N] float32 (device). */
typedef struct edm_instance {
    const float *X;
    int N;
    int L;
    const int32_t *E_lib;
    int tau;
    int Tp;
    float *rho;
    int lib_begin;
    int lib_end;
} edm_instance;

/* Run n_inst independent CCM problems of uneven N and L.  `inst` is a HOST
 * array of n_inst descriptors (read before the call returns); the pointers
 * inside are device pointers.  Same per-instance rules as edm_ccm_all.
 * Execution (no counterpart in the paper): the instances are spread over
 * several internal streams, largest first, each stream with its own
 * workspace; by default the whole batch is captured once into a CUDA graph
 * and the graph is replayed when the same batch (same descriptors) comes
 * again.  Before the first capture the autotuner times the lookup's number
 * of libraries per CTA for every new size bucket of the batch.  The work is
 * ordered after what was queued on the context's stream before the call and
 * before what is queued after it. */
edm_status edm_ccm_batched(edm_ctx *ctx, const edm_instance *inst, int n_inst,
                           edm_precision prec);

/* Optimal E (as edm_simplex_optimal_E) of every series of every instance.
 * Only X, N, L and tau of each descriptor are used; E_out is a HOST array of
 * n_inst DEVICE pointers, E_out[i] [N_i] int32.
 * Execution (no counterpart in the paper): by default every instance's work
 * items -- (series, block of query times) -- go into one device work queue
 * per kind of sweep (the register-resident sweep of each candidate count,
 * and the chunked sweep of series longer than 2,048 points); each kind with
 * work gets one persistent launch whose thread blocks take items from the
 * queue until it is empty, largest problems first, and one kernel then
 * finishes every series.  The query times per work item are autotuned per
 * kind (128, 256 or 512, timed on the first batch that needs the kind).  The
 * sequence is captured once into a CUDA graph and replayed for the same
 * batch.  Option "batch_queue" 0 (or an instance longer than 24,576 points)
 * runs the instances as separate launches over concurrent streams instead,
 * like edm_ccm_batched. */
edm_status edm_simplex_optimal_E_batched(edm_ctx *ctx, const edm_instance *inst,
                                         int n_inst, int E_max, int Tp_sel,
                                         int32_t *const *E_out);

/* Execution options (no counterpart in the paper):
 *   "batch_streams"        1..32  concurrent streams of batched calls (8)
 *   "batch_graph"          0/1    capture batched calls into a CUDA graph (1)
 *   "autotune"             0/1    tune the lookup's libraries per CTA (1)
 *   "lookup_libs_per_cta"  0..4096 fixed libraries per CTA, 0 = tuned (0)
 *   "table_budget_mb"      >= 16  workspace for neighbour tables (2048)
 *   "autotune_reset"       1      forget the tuned values
 *   "diagnostics"          0/1    count FP64 band and brute-force rows (0)
 *   "batch_queue"          0/1    batched optimal E through work queues (1)
 * Returns EDM_ERR_INVALID_ARG for an unknown name or value. */
edm_status edm_set_option(edm_ctx *ctx, const char *name, long long value);

#ifdef __cplusplus
}
#endif

#endif /* EDM_H */
