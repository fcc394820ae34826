// edm_internal.cuh -- shared host/device definitions of libedm (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <vector>

#include "../../include/edm.h"

struct edm_prof_rec {
    const char *kernel;
    cudaEvent_t start, stop;
};

struct edm_ctx {
    int device;
    cudaStream_t stream;
    int num_sms;
    int max_smem_optin;        // bytes of dynamic shared memory a CTA may opt into
    void *ws;                  // workspace (neighbour tables, transposed targets, partials)
    size_t ws_bytes;
    int *d_flags;              // device-side error flags (EDMF_*)
    unsigned long long *d_stats;  // [2]: rows resolved in the FP64 band, by FP64 brute force
    bool diag = false;         // count those rows (edm_set_option "diagnostics")
    uint64_t launches;         // kernels launched through this context
    size_t table_budget;       // bytes of workspace a chunk of neighbour tables may use
    char last_error[256];
    bool prof_on;              // time every launch with CUDA events
    cudaEvent_t prof_pending;  // start event of the launch in progress
    std::vector<edm_prof_rec> prof;
    std::vector<cudaEvent_t> prof_pool;

    // options (edm_set_option)
    int batch_streams = 8;     // concurrent streams of a batched call
    bool batch_graph = true;   // capture a batched call into a CUDA graph
    bool autotune = true;      // tune the lookup's libraries per CTA
    int lookup_lb = 0;         // fixed libraries per CTA (0: tuned or heuristic)

    // autotuner: bucket key -> libraries per CTA (owned by the main context)
    std::map<uint64_t, int> *tune = nullptr;

    // batched execution: sub-contexts (own stream and workspace), the stream a
    // graph is captured on and launched from, and the cached graph
    bool is_sub = false;
    std::vector<edm_ctx *> subs;
    cudaStream_t origin = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
    std::vector<cudaEvent_t> ev_join;
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_key = 0;
    uint64_t graph_kernels = 0;  // kernels one replay of graph_exec launches
    bool batch_queue = true;     // batched optimal E through the work queues
    cudaGraphExec_t qgraph_exec = nullptr;  // the cached graph of the queues
    uint64_t qgraph_key = 0;
    uint64_t qgraph_kernels = 0;

    // copies of finished rho blocks to host memory (edm_ccm_all_host)
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> copy_ev;
};

// device-side error flags, OR-ed into ctx->d_flags
enum { EDMF_TIMEOUT = 1, EDMF_BADARG = 2, EDMF_INTERNAL = 4 };

namespace edm {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARP = 32;

// ---------------------------------------------------------------- host side

edm_status set_error(edm_ctx *ctx, edm_status s, const char *fmt, ...);
edm_status cuda_check(edm_ctx *ctx, cudaError_t e, const char *what);
// Make sure the workspace holds at least `bytes`; returns its base.
edm_status ws_reserve(edm_ctx *ctx, size_t bytes);
// Call right before a kernel launch (records the start event when profiling).
void before_launch(edm_ctx *ctx);
// Record a kernel launch and check for a launch error.
edm_status after_launch(edm_ctx *ctx, const char *kernel);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
// The fallback counters a kernel adds to, or NULL when diagnostics are off.
inline unsigned long long *diag_stats(edm_ctx *ctx) { return ctx->diag ? ctx->d_stats : nullptr; }

// Layout of a CCM neighbour table (k = E+1 neighbours, n rows).  Rows are
// stored in pairs (2p, 2p+1).  A row's logical words are its first k-1
// normalised weights (float32; the k-th is 1 minus their sum) followed by
// its k neighbour rows (time index + Tp) packed two per 32-bit word (low half
// first).  In a pair block, logical word j of row 2p sits at word 2j and that
// of row 2p+1 at word 2j+1, so one 16-byte read gives both rows' values as
// register pairs.  Blocks are padded to 16 bytes.  When n is odd the last
// block's second row is a dummy: weights 0 and every neighbour row equal to
// L, the all-zero time row that every target tile carries after its L rows.
__host__ __device__ constexpr int table_row_words(int k) { return (k - 1) + (k + 1) / 2; }
__host__ __device__ constexpr int table_pair_bytes(int k) {
    return ((8 * table_row_words(k) + 15) / 16) * 16;
}

// Libraries of one chunk run in groups of G that share E (hence k, the
// number of table rows and the first query time), so that the lookup reads
// each observation row once per group instead of once per library.  A
// group's tables are interleaved: pair block p of member m sits at byte
// off + (p * G + m) * table_pair_bytes(E+1).  Libraries whose E is invalid
// form groups with E = 0 (no tables; their rho rows are NaN).
// A library can be cross-mapped when 1 <= E <= EDM_E_MAX and its n =
// L-(E-1)tau-Tp points leave at least E+2 of them (k = E+1 neighbours plus
// the point itself).
__host__ __device__ inline bool ccm_E_valid(int E, int L, int tau, int Tp) {
    return E >= 1 && E <= EDM_E_MAX && L - (E - 1) * tau - Tp >= E + 2;
}

constexpr int LK_GROUP_FP32 = 4;
constexpr int LK_GROUP_16 = 2;   // 16-bit targets: two per lane, so fewer libraries
inline int lookup_group(edm_precision prec) {
    return prec != EDM_FP32 ? LK_GROUP_16 : LK_GROUP_FP32;
}
inline bool precision_ok(edm_precision prec) {
    return prec == EDM_FP32 || prec == EDM_BF16_TARGETS || prec == EDM_FP16_TARGETS;
}
struct CcmGroups {
    int32_t *E;      // [ngroups_max] E of the members (0: invalid E)
    int32_t *n;      // [ngroups_max] members, 1..G
    int32_t *lib;    // [ngroups_max * G] library index; slots n..G-1 of a
                     // group repeat its first member; -1 past the last group
    long long *off;  // [ngroups_max] byte offset of the group's tables
    int32_t *count;  // number of groups (device scalar)
    int G;
    int ngroups_max;
};
inline int groups_max(int nlib, int G) { return (nlib + G - 1) / G + EDM_E_MAX + 1; }
// Bytes of the group arrays of a chunk of nlib libraries (see carve_groups).
size_t groups_bytes(int nlib, int G);
// Lay the group arrays out in `mem` (groups_bytes(nlib, G) bytes).
CcmGroups carve_groups(uint8_t *mem, int nlib, int G);
// Group the libraries lib0 .. lib0+nlib-1 by E (one CTA; order within an E
// is not specified and does not change any result).  E of library i is
// E_lib[i], or E_uniform for every library when E_uniform > 0.
edm_status launch_group_libs(edm_ctx *ctx, const int32_t *E_lib, int E_uniform, int lib0,
                             int nlib, int L, int tau, int Tp, const CcmGroups &g);

// Launchers (one translation unit each).
edm_status launch_embed(edm_ctx *ctx, const float *x, int L, int E, int tau, float *out);
edm_status launch_knn(edm_ctx *ctx, const float *X, int N, int L, int E, int tau, int Tp,
                      int k, int32_t *idx, float *dist);
edm_status launch_knn_materialized(edm_ctx *ctx, const float *X, int N, int L, int E, int tau,
                                   int Tp, int k, int32_t *idx, float *dist);
// X: library series with row stride ld (>= L) floats; the libraries are
// those of the groups g (indexes into X), tables laid out as described at
// CcmGroups.
edm_status launch_ccm_tables(edm_ctx *ctx, const float *X, long long ld, int nlib, int L,
                             int tau, int Tp, const CcmGroups &g, uint8_t *tables);
edm_status launch_simplex(edm_ctx *ctx, const float *X, int N, int L, int E_max, int tau,
                          int Tp_sel, int32_t *E_opt, float *rho_E);
// Optimal E of every series of every instance through one persistent
// work-queue launch per kind of sweep (autotuned rows per work item when
// `tune`), captured into a cached graph when `capture`.  Instances longer
// than 24,576 points are not supported here (see sweep_queue_ok).
edm_status launch_simplex_queue(edm_ctx *ctx, const edm_instance *inst, int n, int E_max,
                                int Tp_sel, int32_t *const *E_out, bool tune, bool capture);
inline bool sweep_queue_ok(int L) { return L <= 24576; }
// Transposed, centred target tiles plus, per E = 1..EDM_E_MAX, the FP64 sums
// of the stored values and of their squares over the observation window of
// E (times (E-1)tau+Tp .. L-1): ysum / yysum [EDM_E_MAX][N_tgt].  mean_ws
// holds 2 * N_tgt doubles (each target's mean, then its FP16 scale).
// Y: target series with row stride ld (>= L) floats; target r of the store is
// series rows[r] (series r when rows is NULL).  rw: 32-bit words per tile
// row (lookup_row_words).
edm_status launch_target_store(edm_ctx *ctx, const float *Y, long long ld, const int32_t *rows,
                               int N_tgt, int L, int tau, int Tp, edm_precision prec, int rw,
                               uint8_t *Yt, double *mean_ws, double *ysum, double *yysum);
// Words per target-tile row for series of length L: 32 (128-byte rows) when
// such a tile fits a CTA's shared memory or nothing smaller does, 16 when
// only the half-width tile fits.
int lookup_row_words(edm_ctx *ctx, int L, edm_precision prec);
// rho points at the row of library lib0; row of library i = rho + (i - lib0) * rho_ld;
// stored target r goes to column rho_col[r] (column r when rho_col is NULL).
edm_status launch_lookup(edm_ctx *ctx, const uint8_t *Yt, int N_tgt, int L,
                         const uint8_t *tables, const CcmGroups &g, int lib0, int nlib, int tau,
                         int Tp, edm_precision prec, int rw, const double *ysum,
                         const double *yysum, float *rho, long long rho_ld,
                         const int32_t *rho_col);
// Predictions of libraries lib0.. (groups g, tables built by launch_ccm_tables)
// for their targets Y[tgt_of[lib]] (Y[lib] when tgt_of is NULL).
edm_status launch_predict(edm_ctx *ctx, const float *Y, long long ld_tgt, int N_tgt,
                          const int32_t *tgt_of, int L, int tau, int Tp, const CcmGroups &g,
                          const uint8_t *tables, int lib0, float *pred, long long ld_pred);
edm_status launch_smem_probe(edm_ctx *ctx, double ms, double *bytes_per_s);
edm_status launch_l2_probe(edm_ctx *ctx, double ms, double *bytes_per_s);
edm_status launch_wait_check(edm_ctx *ctx, int ms);
size_t simplex_workspace_bytes(edm_ctx *ctx, int N, int L, int E_max);
// Autotuner bucket of a lookup launch.
uint64_t lookup_bucket(int L, int N_tgt, int nlib, edm_precision prec);
int lookup_default_lb(edm_ctx *ctx, int nlib, int n_tiles);
size_t ccm_slot_bytes(int L, int tau, int Tp);
size_t target_store_bytes(int N_tgt, int L, edm_precision prec, int rw);

// --------------------------------------------------------------- device side

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ void set_flag(int *flags, int f) {
    if (flags) atomicOr(flags, f);
}

// Ascending bitonic sort of one 64-bit key per lane; returns the key at
// position r (broadcast to every lane).
__device__ __forceinline__ uint64_t warp_sorted_at(uint64_t key, int r) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint64_t other = __shfl_xor_sync(FULL, key, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            uint64_t lo = key < other ? key : other;
            uint64_t hi = key < other ? other : key;
            key = (lower == up) ? lo : hi;
        }
    }
    return __shfl_sync(FULL, key, r);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Pearson's rho from the five raw moments of n pairs (a, b), in FP64.
// A variance that is not positive gives NaN.
__device__ __forceinline__ double pearson_from_moments(double n, double sa, double sb,
                                                       double saa, double sbb, double sab) {
    double va = saa - sa * sa / n;
    double vb = sbb - sb * sb / n;
    double cv = sab - sa * sb / n;
    if (!(va > 0.0) || !(vb > 0.0)) return __longlong_as_double(0x7ff8000000000000LL);
    return cv / sqrt(va * vb);
}

// ------------------------------------------------ mbarrier + bulk copy (PTX)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_try_wait, but the thread may be suspended in hardware for up to
// `hint_ns` nanoseconds while the phase is incomplete (it resumes as soon as
// the phase completes), instead of spinning on the barrier.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity,
                                                    uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity to complete, for at most
// limit_ns nanoseconds (two seconds by default).  On timeout the context's
// error flag is raised, the CTA's abort word (when given) is set and false
// is returned; the caller carries on without the data it waited for, so that
// every thread still reaches every later barrier and the kernel always ends.
// Once the abort word is set, every later wait of the CTA that passes it
// returns false at once instead of spinning for its own limit, so a CTA
// whose pipeline broke ends within about one limit.
// While waiting the thread sleeps in try_wait (up to 20 us a try, woken
// when the phase completes) rather than spinning, so a waiting warp leaves
// the issue slots to the warps that work; the timer is read once every 8
// tries.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *flags,
                                                  volatile int *abort,
                                                  uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort && *abort) return false;
    const uint64_t t0 = global_timer_ns();
    for (unsigned tries = 1;; ++tries) {
        if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (abort && *abort) return false;
        if ((tries & 7u) == 0 && global_timer_ns() - t0 > limit_ns) {
            set_flag(flags, EDMF_TIMEOUT);
            if (abort) *abort = 1;
            return false;
        }
    }
}

// 1-D bulk copy global -> this CTA's shared memory, completing on `bar`.
// dst and src must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace edm
