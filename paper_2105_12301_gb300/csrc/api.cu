// api.cu -- the C ABI of libedm (include/edm.h): argument checks, the
// context and its workspace, and the order in which the kernels run.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "edm_internal.cuh"

namespace edm {

edm_status set_error(edm_ctx *ctx, edm_status s, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->last_error, sizeof(ctx->last_error), fmt, ap);
        va_end(ap);
    }
    return s;
}

edm_status cuda_check(edm_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return EDM_OK;
    return set_error(ctx, e == cudaErrorMemoryAllocation ? EDM_ERR_OOM : EDM_ERR_CUDA, "%s: %s",
                     what, cudaGetErrorString(e));
}

static cudaEvent_t prof_event(edm_ctx *ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

static void prof_clear(edm_ctx *ctx) {
    for (auto &r : ctx->prof) {
        ctx->prof_pool.push_back(r.start);
        ctx->prof_pool.push_back(r.stop);
    }
    ctx->prof.clear();
}

void before_launch(edm_ctx *ctx) {
    if (!ctx->prof_on) return;
    ctx->prof_pending = prof_event(ctx);
    if (ctx->prof_pending) cudaEventRecord(ctx->prof_pending, ctx->stream);
}

edm_status after_launch(edm_ctx *ctx, const char *kernel) {
    ctx->launches++;
    edm_status st = cuda_check(ctx, cudaGetLastError(), kernel);
    if (ctx->prof_on && ctx->prof_pending) {
        cudaEvent_t stop = prof_event(ctx);
        if (stop) {
            cudaEventRecord(stop, ctx->stream);
            ctx->prof.push_back({kernel, ctx->prof_pending, stop});
        } else {
            ctx->prof_pool.push_back(ctx->prof_pending);
        }
        ctx->prof_pending = nullptr;
    }
    return st;
}

edm_status ws_reserve(edm_ctx *ctx, size_t bytes) {
    bytes = align_up(std::max<size_t>(bytes, 256), 1 << 20);
    if (bytes <= ctx->ws_bytes) return EDM_OK;
    // the old workspace may still be read by queued kernels
    edm_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "workspace sync");
    if (st != EDM_OK) return st;
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    st = cuda_check(ctx, cudaMalloc(&ctx->ws, bytes), "workspace allocation");
    if (st != EDM_OK) return st;
    ctx->ws_bytes = bytes;
    return EDM_OK;
}

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static bool series_len_ok(int L) { return L >= 2 && L <= EDM_L_MAX; }

// All-to-all CCM of N_lib libraries against N_tgt targets of length L whose
// rows are ld_lib / ld_tgt floats apart.  Libraries are processed in chunks
// whose neighbour tables fit the table budget; each chunk is grouped by E
// (launch_group_libs), its tables are built in the grouped layout, then the
// lookup runs over every (group, target tile).
static int ccm_chunk(edm_ctx *ctx, int N_lib, size_t slot) {
    const size_t per = std::max<size_t>(1, ctx->table_budget / slot);
    return static_cast<int>(std::max<size_t>(1, std::min<size_t>(N_lib, per)));
}

static size_t ccm_workspace_bytes(edm_ctx *ctx, int N_lib, int N_tgt, int L, int tau, int Tp,
                                  edm_precision prec) {
    const size_t yt_bytes = target_store_bytes(N_tgt, L, prec, lookup_row_words(ctx, L, prec));
    const size_t mean_bytes = align_up(2 * sizeof(double) * N_tgt, 256);
    const size_t sums_bytes = align_up(sizeof(double) * N_tgt * EDM_E_MAX, 256);
    const size_t slot = ccm_slot_bytes(L, tau, Tp);
    if (slot == 0) return yt_bytes + mean_bytes + 2 * sums_bytes;
    const int G = lookup_group(prec);
    const int chunk = ccm_chunk(ctx, N_lib, slot);
    return yt_bytes + mean_bytes + 2 * sums_bytes + groups_bytes(chunk, G) +
           static_cast<size_t>(groups_max(chunk, G)) * G * slot;
}

// E_lib: E per library, unless E_uniform > 0 (every library at that E).
// The N_tgt stored targets are Y rows tgt_rows[r] (rows 0.. when NULL); rho
// rows are rho_ld apart and stored target r goes to column rho_cols[r]
// (column r when NULL).
// rho_host (optional, page-locked, rows rho_ld apart like rho): each block of
// finished rows is copied there on the context's copy stream while the next
// block computes; blocks are then at most max_block libraries.
static edm_status ccm_one(edm_ctx *ctx, const float *X_lib, long long ld_lib, int N_lib,
                          const float *Y_tgt, long long ld_tgt, int N_tgt, int L,
                          const int32_t *E_lib, int E_uniform, int tau, int Tp, edm_precision prec,
                          float *rho, long long rho_ld, const int32_t *tgt_rows,
                          const int32_t *rho_cols, float *rho_host = nullptr,
                          int max_block = 0) {
    const int rw = lookup_row_words(ctx, L, prec);
    const size_t yt_bytes = target_store_bytes(N_tgt, L, prec, rw);
    const size_t mean_bytes = align_up(2 * sizeof(double) * N_tgt, 256);
    const size_t sums_bytes = align_up(sizeof(double) * N_tgt * EDM_E_MAX, 256);
    const size_t slot = ccm_slot_bytes(L, tau, Tp);
    if (slot == 0) return set_error(ctx, EDM_ERR_INVALID_ARG, "series too short");
    const int G = lookup_group(prec);
    const int chunk = ccm_chunk(ctx, N_lib, slot);
    edm_status st = ws_reserve(ctx, ccm_workspace_bytes(ctx, N_lib, N_tgt, L, tau, Tp, prec));
    if (st != EDM_OK) return st;
    uint8_t *base = static_cast<uint8_t *>(ctx->ws);
    uint8_t *Yt = base;
    double *mean = reinterpret_cast<double *>(base + yt_bytes);
    double *ysum = reinterpret_cast<double *>(base + yt_bytes + mean_bytes);
    double *yysum = reinterpret_cast<double *>(base + yt_bytes + mean_bytes + sums_bytes);
    uint8_t *gmem = base + yt_bytes + mean_bytes + 2 * sums_bytes;
    uint8_t *tables = gmem + groups_bytes(chunk, G);
    st = launch_target_store(ctx, Y_tgt, ld_tgt, tgt_rows, N_tgt, L, tau, Tp, prec, rw, Yt, mean,
                             ysum, yysum);
    if (st != EDM_OK) return st;
    const int block = max_block > 0 ? std::min(chunk, max_block) : chunk;
    int nblk = 0;
    for (int c0 = 0; c0 < N_lib; c0 += block) {
        const int nlib = std::min(block, N_lib - c0);
        const CcmGroups grp = carve_groups(gmem, nlib, G);
        st = launch_group_libs(ctx, E_lib, E_uniform, c0, nlib, L, tau, Tp, grp);
        if (st != EDM_OK) return st;
        st = launch_ccm_tables(ctx, X_lib, ld_lib, nlib, L, tau, Tp, grp, tables);
        if (st != EDM_OK) return st;
        st = launch_lookup(ctx, Yt, N_tgt, L, tables, grp, c0, nlib, tau, Tp, prec, rw, ysum,
                           yysum, rho + static_cast<size_t>(c0) * rho_ld, rho_ld, rho_cols);
        if (st != EDM_OK) return st;
        if (rho_host) {
            // copy this block's rows while the next block computes
            if (static_cast<int>(ctx->copy_ev.size()) <= nblk) {
                cudaEvent_t e = nullptr;
                st = cuda_check(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming),
                                "copy event");
                if (st != EDM_OK) return st;
                ctx->copy_ev.push_back(e);
            }
            cudaEvent_t ev = ctx->copy_ev[nblk++];
            const size_t off = static_cast<size_t>(c0) * rho_ld;
            st = cuda_check(ctx, cudaEventRecord(ev, ctx->stream), "copy order");
            if (st == EDM_OK)
                st = cuda_check(ctx, cudaStreamWaitEvent(ctx->copy_stream, ev, 0), "copy order");
            if (st == EDM_OK)
                st = cuda_check(ctx, cudaMemcpyAsync(rho_host + off, rho + off,
                                                     sizeof(float) * nlib * rho_ld,
                                                     cudaMemcpyDeviceToHost, ctx->copy_stream),
                                "rho copy");
            if (st != EDM_OK) return st;
        }
    }
    if (rho_host && nblk > 0) {
        // the context's stream (and a sync on it) waits for the copies
        cudaEvent_t done = ctx->copy_ev[0];
        st = cuda_check(ctx, cudaEventRecord(done, ctx->copy_stream), "copy done");
        if (st == EDM_OK) st = cuda_check(ctx, cudaStreamWaitEvent(ctx->stream, done, 0), "copy done");
        if (st != EDM_OK) return st;
    }
    return EDM_OK;
}


// ------------------------------------------------------------ batched calls

static edm_ctx *make_sub(edm_ctx *main) {
    edm_ctx *sub = new (std::nothrow) edm_ctx();
    if (!sub) return nullptr;
    sub->device = main->device;
    sub->num_sms = main->num_sms;
    sub->max_smem_optin = main->max_smem_optin;
    sub->d_flags = main->d_flags;
    sub->d_stats = main->d_stats;
    sub->diag = main->diag;
    sub->table_budget = main->table_budget;
    sub->tune = main->tune;
    sub->is_sub = true;
    if (cudaStreamCreateWithFlags(&sub->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete sub;
        return nullptr;
    }
    return sub;
}

static void free_sub(edm_ctx *sub) {
    cudaStreamSynchronize(sub->stream);
    if (sub->ws) cudaFree(sub->ws);
    prof_clear(sub);
    for (cudaEvent_t e : sub->prof_pool) cudaEventDestroy(e);
    cudaStreamDestroy(sub->stream);
    delete sub;
}

static edm_status ensure_batch_state(edm_ctx *ctx, int S) {
    if (!ctx->origin && cudaStreamCreateWithFlags(&ctx->origin, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(ctx, EDM_ERR_CUDA, "batch stream creation failed");
    if (!ctx->ev_fork && cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return set_error(ctx, EDM_ERR_CUDA, "batch event creation failed");
    if (!ctx->ev_done && cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming) != cudaSuccess)
        return set_error(ctx, EDM_ERR_CUDA, "batch event creation failed");
    while (static_cast<int>(ctx->subs.size()) < S) {
        edm_ctx *sub = make_sub(ctx);
        if (!sub) return set_error(ctx, EDM_ERR_CUDA, "batch stream creation failed");
        ctx->subs.push_back(sub);
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return set_error(ctx, EDM_ERR_CUDA, "batch event creation failed");
        ctx->ev_join.push_back(e);
    }
    return EDM_OK;
}

static uint64_t fnv1a(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

// Time the kernels named `kernel` launched by fn(sub) on a sub-context (ms).
template <class Fn>
static double time_kernel_ms(edm_ctx *sub, const char *kernel, Fn fn, edm_status &st) {
    cudaStreamSynchronize(sub->stream);
    prof_clear(sub);
    sub->prof_on = true;
    st = fn();
    sub->prof_on = false;
    cudaStreamSynchronize(sub->stream);
    double tot = 0.0;
    for (auto &r : sub->prof) {
        if (strcmp(r.kernel, kernel) != 0) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.start, r.stop);
        tot += ms;
    }
    prof_clear(sub);
    return tot;
}

// Run fn(sub, i) for every instance i on S concurrent sub-streams, the
// largest work first to the least-loaded stream; when enabled, the whole
// fork/join is captured once into a CUDA graph (cached under `key`) and
// replayed.  Work queued on ctx->stream before the call runs first; work
// queued after it waits for the batch.
template <class Fn>
static edm_status run_batched(edm_ctx *ctx, int n, const std::vector<double> &work,
                              const std::vector<size_t> &ws_need, uint64_t key, Fn fn) {
    const int S = std::max(1, std::min({ctx->batch_streams, n, 32}));
    edm_status st = ensure_batch_state(ctx, S);
    if (st != EDM_OK) return st;
    std::vector<int> order(n), assign(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<double> load(S, 0.0);
    std::vector<size_t> need(S, 0);
    for (int i : order) {
        const int s = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
        assign[i] = s;
        load[s] += work[i];
        need[s] = std::max(need[s], ws_need[i]);
    }
    for (int s = 0; s < S; ++s) {
        edm_ctx *sub = ctx->subs[s];
        sub->table_budget = ctx->table_budget;
        sub->autotune = ctx->autotune;
        sub->lookup_lb = ctx->lookup_lb;
        st = ws_reserve(sub, need[s]);
        if (st != EDM_OK) return set_error(ctx, st, "%s", sub->last_error);
    }
    auto enqueue = [&](cudaStream_t from) -> edm_status {
        edm_status e = cuda_check(ctx, cudaEventRecord(ctx->ev_fork, from), "batch fork");
        for (int s = 0; s < S && e == EDM_OK; ++s)
            e = cuda_check(ctx, cudaStreamWaitEvent(ctx->subs[s]->stream, ctx->ev_fork, 0),
                           "batch fork wait");
        if (e != EDM_OK) return e;
        for (int i : order) {
            e = fn(ctx->subs[assign[i]], i);
            if (e != EDM_OK) return set_error(ctx, e, "instance %d: %s", i, ctx->subs[assign[i]]->last_error);
        }
        for (int s = 0; s < S && e == EDM_OK; ++s) {
            e = cuda_check(ctx, cudaEventRecord(ctx->ev_join[s], ctx->subs[s]->stream), "batch join");
            if (e == EDM_OK)
                e = cuda_check(ctx, cudaStreamWaitEvent(from, ctx->ev_join[s], 0), "batch join wait");
        }
        return e;
    };
    uint64_t before = 0;
    for (int s = 0; s < S; ++s) before += ctx->subs[s]->launches;
    if (!ctx->batch_graph) {
        st = enqueue(ctx->stream);
        for (int s = 0; s < S; ++s) ctx->launches += ctx->subs[s]->launches;
        ctx->launches -= before;
        return st;
    }
    key = fnv1a(key, &S, sizeof(S));
    if (!ctx->graph_exec || ctx->graph_key != key) {
        if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
        if (cudaStreamBeginCapture(ctx->origin, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return set_error(ctx, EDM_ERR_CUDA, "graph capture could not begin");
        st = enqueue(ctx->origin);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(ctx->origin, &graph);
        if (st != EDM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ce != cudaSuccess || !graph) return cuda_check(ctx, ce, "graph capture");
        const cudaError_t ie = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_check(ctx, ie, "graph instantiation");
        ctx->graph_key = key;
        uint64_t after = 0;
        for (int s = 0; s < S; ++s) after += ctx->subs[s]->launches;
        ctx->graph_kernels = after - before;
    }
    // order the replay after the caller's stream, and the caller's stream after it
    if (cudaEventRecord(ctx->ev_fork, ctx->stream) != cudaSuccess ||
        cudaStreamWaitEvent(ctx->origin, ctx->ev_fork, 0) != cudaSuccess)
        return set_error(ctx, EDM_ERR_CUDA, "batch ordering failed");
    st = cuda_check(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->origin), "graph launch");
    if (st != EDM_OK) return st;
    cudaEventRecord(ctx->ev_done, ctx->origin);
    cudaStreamWaitEvent(ctx->stream, ctx->ev_done, 0);
    ctx->launches += ctx->graph_kernels;
    return EDM_OK;
}

// Autotuner: for every lookup bucket of the batch not tuned yet, time the
// lookup of its first instance with each candidate number of libraries per
// CTA and keep the fastest (before capture: timing needs synchronisation).
template <class Fn>
static edm_status autotune_lookup(edm_ctx *ctx, int n, const std::vector<uint64_t> &bucket, Fn fn) {
    if (!ctx->autotune || ctx->lookup_lb > 0) return EDM_OK;
    edm_ctx *sub = ctx->subs[0];
    for (int i = 0; i < n; ++i) {
        if (ctx->tune->count(bucket[i])) continue;
        int best = 0;
        double best_ms = 0.0;
        for (int cand = 1; cand <= 128; cand *= 2) {
            sub->lookup_lb = cand;
            edm_status st = EDM_OK;
            const double ms = time_kernel_ms(sub, "lookup_kernel", [&] { return fn(sub, i); }, st);
            if (st != EDM_OK) {
                sub->lookup_lb = 0;
                return st;
            }
            if (best == 0 || ms < best_ms) {
                best = cand;
                best_ms = ms;
            }
        }
        sub->lookup_lb = 0;
        (*ctx->tune)[bucket[i]] = best;
        ctx->graph_key = 0;  // a captured graph may hold the old choice
    }
    return EDM_OK;
}

}  // namespace edm

using namespace edm;

extern "C" {

const char *edm_status_string(edm_status s) {
    switch (s) {
    case EDM_OK: return "ok";
    case EDM_ERR_INVALID_ARG: return "invalid argument";
    case EDM_ERR_CUDA: return "CUDA error";
    case EDM_ERR_OOM: return "out of device memory";
    case EDM_ERR_TIMEOUT: return "device-side wait timed out";
    case EDM_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

edm_status edm_create(edm_ctx **out, int device, void *cuda_stream) {
    if (!out) return EDM_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return EDM_ERR_CUDA;
    }
    DeviceGuard g(device);
    if (!g.ok) return EDM_ERR_CUDA;
    edm_ctx *ctx = new (std::nothrow) edm_ctx();
    if (!ctx) return EDM_ERR_OOM;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    ctx->table_budget = static_cast<size_t>(2) << 30;
    ctx->tune = new (std::nothrow) std::map<uint64_t, int>();
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                               device) != cudaSuccess ||
        cudaMalloc(&ctx->d_flags, 32) != cudaSuccess ||   // flags word, then the two counters
        cudaMemset(ctx->d_flags, 0, 32) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_flags) cudaFree(ctx->d_flags);
        delete ctx;
        return EDM_ERR_CUDA;
    }
    ctx->d_stats = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(ctx->d_flags) + 16);
    *out = ctx;
    return EDM_OK;
}

edm_status edm_destroy(edm_ctx *ctx) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (edm_ctx *sub : ctx->subs) free_sub(sub);
    for (cudaEvent_t e : ctx->ev_join) cudaEventDestroy(e);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_done) cudaEventDestroy(ctx->ev_done);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->qgraph_exec) cudaGraphExecDestroy(ctx->qgraph_exec);
    if (ctx->origin) cudaStreamDestroy(ctx->origin);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (cudaEvent_t e : ctx->copy_ev) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    prof_clear(ctx);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    delete ctx->tune;
    delete ctx;
    return EDM_OK;
}

edm_status edm_set_stream(edm_ctx *ctx, void *cuda_stream) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return EDM_OK;
}

edm_status edm_ctx_sync(edm_ctx *ctx) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    edm_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "stream sync");
    if (st != EDM_OK) return st;
    int flags = 0;
    st = cuda_check(ctx, cudaMemcpyAsync(&flags, ctx->d_flags, sizeof(int),
                                         cudaMemcpyDeviceToHost, ctx->stream), "flag read");
    if (st == EDM_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "flag sync");
    if (st != EDM_OK) return st;
    if (flags) {
        cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream);
        cudaStreamSynchronize(ctx->stream);
    }
    if (flags & EDMF_TIMEOUT)
        return set_error(ctx, EDM_ERR_TIMEOUT, "a device-side wait gave up");
    if (flags & EDMF_BADARG)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "an E value on the device is out of range");
    if (flags & EDMF_INTERNAL) return set_error(ctx, EDM_ERR_INTERNAL, "device check failed");
    return EDM_OK;
}

const char *edm_last_error(edm_ctx *ctx) { return ctx ? ctx->last_error : ""; }

edm_status edm_fallback_counts(edm_ctx *ctx, uint64_t *band_rows, uint64_t *brute_rows) {
    if (!ctx || !band_rows || !brute_rows) return EDM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    unsigned long long c[2] = {0, 0};
    edm_status st = cuda_check(ctx, cudaMemcpyAsync(c, ctx->d_stats, sizeof(c),
                                                    cudaMemcpyDeviceToHost, ctx->stream),
                               "counter read");
    if (st == EDM_OK)
        st = cuda_check(ctx, cudaMemsetAsync(ctx->d_stats, 0, sizeof(c), ctx->stream), "counter reset");
    if (st == EDM_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "counter sync");
    if (st != EDM_OK) return st;
    *band_rows = c[0];
    *brute_rows = c[1];
    return EDM_OK;
}

edm_status edm_profile_enable(edm_ctx *ctx, int on) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (on) {
        edm_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "profile sync");
        if (st != EDM_OK) return st;
        prof_clear(ctx);
    }
    ctx->prof_on = on != 0;
    return EDM_OK;
}

edm_status edm_profile_read(edm_ctx *ctx, const char *kernel, double *total_ms, int *launches) {
    if (!ctx || !kernel || !total_ms || !launches) return EDM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    edm_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "profile sync");
    if (st != EDM_OK) return st;
    double tot = 0.0;
    int cnt = 0;
    for (auto &r : ctx->prof) {
        if (strcmp(r.kernel, kernel) != 0) continue;
        float ms = 0.f;
        st = cuda_check(ctx, cudaEventElapsedTime(&ms, r.start, r.stop), "profile read");
        if (st != EDM_OK) return st;
        tot += ms;
        ++cnt;
    }
    *total_ms = tot;
    *launches = cnt;
    return EDM_OK;
}

edm_status edm_probe_smem_bandwidth(edm_ctx *ctx, double ms, double *bytes_per_s) {
    if (!ctx || !bytes_per_s || !(ms > 0.0)) return EDM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return launch_smem_probe(ctx, ms, bytes_per_s);
}

edm_status edm_probe_l2_bandwidth(edm_ctx *ctx, double ms, double *bytes_per_s) {
    if (!ctx || !bytes_per_s || !(ms > 0.0)) return EDM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    return launch_l2_probe(ctx, ms, bytes_per_s);
}

uint64_t edm_kernel_launches(edm_ctx *ctx) { return ctx ? ctx->launches : 0; }

edm_status edm_check_wait_timeout(edm_ctx *ctx, int ms) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (ms < 1 || ms > 10000)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_check_wait_timeout: ms out of range");
    DeviceGuard g(ctx->device);
    return launch_wait_check(ctx, ms);
}

edm_status edm_embed(edm_ctx *ctx, const float *x, int L, int E, int tau, float *out) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!x || !out || !series_len_ok(L) || E < 1 || E > EDM_E_MAX || tau < 1 ||
        (E - 1) * tau >= L)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_embed: bad arguments");
    DeviceGuard g(ctx->device);
    return launch_embed(ctx, x, L, E, tau, out);
}

edm_status edm_knn(edm_ctx *ctx, const float *X, int N, int L, int E, int tau, int Tp, int k,
                   int32_t *idx, float *dist) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X || !idx || N < 1 || !series_len_ok(L) || E < 1 || E > EDM_E_MAX || tau < 1 ||
        Tp < 0 || k < 1 || k > EDM_K_MAX)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_knn: bad arguments");
    const long long n = static_cast<long long>(L) - static_cast<long long>(E - 1) * tau - Tp;
    if (n < 2 || k > n - 1)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_knn: k=%d needs more than %lld points", k,
                         n);
    DeviceGuard g(ctx->device);
    return launch_knn(ctx, X, N, L, E, tau, Tp, k, idx, dist);
}

edm_status edm_knn_materialized(edm_ctx *ctx, const float *X, int N, int L, int E, int tau,
                                int Tp, int k, int32_t *idx, float *dist) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X || !idx || N < 1 || !series_len_ok(L) || E < 1 || E > EDM_E_MAX || tau < 1 ||
        Tp < 0 || k < 1 || k > EDM_K_MAX)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_knn_materialized: bad arguments");
    const long long n = static_cast<long long>(L) - static_cast<long long>(E - 1) * tau - Tp;
    if (n < 2 || k > n - 1)
        return set_error(ctx, EDM_ERR_INVALID_ARG,
                         "edm_knn_materialized: k=%d needs more than %lld points", k, n);
    DeviceGuard g(ctx->device);
    return launch_knn_materialized(ctx, X, N, L, E, tau, Tp, k, idx, dist);
}

edm_status edm_simplex_optimal_E(edm_ctx *ctx, const float *X, int N, int L, int E_max, int tau,
                                 int Tp_sel, int32_t *E_opt, float *rho_E) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X || !E_opt || N < 1 || !series_len_ok(L) || E_max < 1 || E_max > EDM_E_MAX ||
        tau < 1 || Tp_sel < 0 || L - Tp_sel < 3)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_simplex_optimal_E: bad arguments");
    DeviceGuard g(ctx->device);
    return launch_simplex(ctx, X, N, L, E_max, tau, Tp_sel, E_opt, rho_E);
}

edm_status edm_ccm_all(edm_ctx *ctx, const float *X_lib, int N_lib, const float *Y_tgt, int N_tgt,
                       int L, const int32_t *E_lib, int tau, int Tp, edm_precision prec,
                       float *rho) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X_lib || !Y_tgt || !E_lib || !rho || N_lib < 1 || N_tgt < 1 || !series_len_ok(L) ||
        tau < 1 || Tp < 0 || L - Tp < 3 || !precision_ok(prec))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_all: bad arguments");
    DeviceGuard g(ctx->device);
    return ccm_one(ctx, X_lib, L, N_lib, Y_tgt, L, N_tgt, L, E_lib, 0, tau, Tp, prec, rho, N_tgt,
                   nullptr, nullptr);
}

edm_status edm_ccm_rows(edm_ctx *ctx, const float *X, int N, int L, int lib_begin, int lib_end,
                        const int32_t *E_lib, int tau, int Tp, edm_precision prec, float *rho) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X || !E_lib || !rho || N < 1 || lib_begin < 0 || lib_end > N || lib_begin > lib_end ||
        !series_len_ok(L) || tau < 1 || Tp < 0 || L - Tp < 3 || !precision_ok(prec))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_rows: bad arguments");
    if (lib_begin == lib_end) return EDM_OK;
    DeviceGuard g(ctx->device);
    return ccm_one(ctx, X + static_cast<size_t>(lib_begin) * L, L, lib_end - lib_begin, X, L, N, L,
                   E_lib + lib_begin, 0, tau, Tp, prec, rho, N, nullptr, nullptr);
}

edm_status edm_ccm_all_host(edm_ctx *ctx, const float *X_lib, int N_lib, const float *Y_tgt,
                            int N_tgt, int L, const int32_t *E_lib, int tau, int Tp,
                            edm_precision prec, float *rho, float *rho_host) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X_lib || !Y_tgt || !E_lib || !rho || !rho_host || N_lib < 1 || N_tgt < 1 ||
        !series_len_ok(L) || tau < 1 || Tp < 0 || L - Tp < 3 ||
        !precision_ok(prec))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_all_host: bad arguments");
    DeviceGuard g(ctx->device);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, rho_host) != cudaSuccess ||
        attr.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return set_error(ctx, EDM_ERR_INVALID_ARG,
                         "edm_ccm_all_host: rho_host must be page-locked host memory");
    }
    if (!ctx->copy_stream &&
        cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(ctx, EDM_ERR_CUDA, "copy stream creation failed");
    // about 16 blocks, so that only the last block's copy is left exposed
    const int block = std::max(64, (N_lib + 15) / 16);
    return ccm_one(ctx, X_lib, L, N_lib, Y_tgt, L, N_tgt, L, E_lib, 0, tau, Tp, prec, rho, N_tgt,
                   nullptr, nullptr, rho_host, block);
}

edm_status edm_upload_series(edm_ctx *ctx, const float *X_host, int N, int L, float *X) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X_host || !X || N < 1 || L < 1)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_upload_series: bad arguments");
    DeviceGuard g(ctx->device);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, X_host) != cudaSuccess ||
        attr.type != cudaMemoryTypeHost) {
        cudaGetLastError();
        return set_error(ctx, EDM_ERR_INVALID_ARG,
                         "edm_upload_series: X_host must be page-locked host memory");
    }
    return cuda_check(ctx, cudaMemcpyAsync(X, X_host, sizeof(float) * static_cast<size_t>(N) * L,
                                           cudaMemcpyHostToDevice, ctx->stream),
                      "series upload");
}

edm_status edm_ccm_all_target_E(edm_ctx *ctx, const float *X_lib, int N_lib, const float *Y_tgt,
                                int N_tgt, int L, const int32_t *E_tgt, int tau, int Tp,
                                edm_precision prec, float *rho) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X_lib || !Y_tgt || !E_tgt || !rho || N_lib < 1 || N_tgt < 1 || !series_len_ok(L) ||
        tau < 1 || Tp < 0 || L - Tp < 3 || !precision_ok(prec))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_all_target_E: bad arguments");
    DeviceGuard g(ctx->device);
    // the targets' E values decide which tables exist: read them (one sync)
    std::vector<int32_t> E(N_tgt);
    edm_status st = cuda_check(ctx, cudaMemcpyAsync(E.data(), E_tgt, sizeof(int32_t) * N_tgt,
                                                    cudaMemcpyDeviceToHost, ctx->stream),
                               "E_tgt read");
    if (st == EDM_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "E_tgt read");
    if (st != EDM_OK) return st;
    std::vector<int32_t> order;  // target indexes grouped by E, ascending E
    std::vector<int> begin(EDM_E_MAX + 2, 0);
    for (int e = 1; e <= EDM_E_MAX; ++e) {
        begin[e] = static_cast<int>(order.size());
        for (int j = 0; j < N_tgt; ++j)
            if (E[j] == e) order.push_back(j);
    }
    begin[EDM_E_MAX + 1] = static_cast<int>(order.size());
    if (static_cast<int>(order.size()) != N_tgt)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_all_target_E: E_tgt out of 1..%d",
                         EDM_E_MAX);
    for (int e = 1; e <= EDM_E_MAX; ++e)
        if (begin[e + 1] > begin[e] && !ccm_E_valid(e, L, tau, Tp))
            return set_error(ctx, EDM_ERR_INVALID_ARG,
                             "edm_ccm_all_target_E: E=%d leaves too few points", e);
    // workspace: the largest CCM pass, then the target index list after it
    const size_t ccm_bytes = align_up(ccm_workspace_bytes(ctx, N_lib, N_tgt, L, tau, Tp, prec), 256);
    st = ws_reserve(ctx, ccm_bytes + sizeof(int32_t) * N_tgt);
    if (st != EDM_OK) return st;
    int32_t *d_order = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(ctx->ws) + ccm_bytes);
    st = cuda_check(ctx, cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * N_tgt,
                                         cudaMemcpyHostToDevice, ctx->stream), "target order");
    // the host vector must outlive the copy
    if (st == EDM_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "target order");
    if (st != EDM_OK) return st;
    for (int e = 1; e <= EDM_E_MAX; ++e) {
        const int n = begin[e + 1] - begin[e];
        if (n == 0) continue;
        const int32_t *rows = d_order + begin[e];
        st = ccm_one(ctx, X_lib, L, N_lib, Y_tgt, L, n, L, nullptr, e, tau, Tp, prec, rho, N_tgt,
                     rows, rows);
        if (st != EDM_OK) return st;
    }
    return EDM_OK;
}

edm_status edm_ccm_window(edm_ctx *ctx, const float *X, int N, int ld, int offset, int L_win,
                          const int32_t *E_lib, int tau, int Tp, edm_precision prec, float *rho) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X || !E_lib || !rho || N < 1 || offset < 0 || !series_len_ok(L_win) ||
        static_cast<long long>(offset) + L_win > ld || tau < 1 || Tp < 0 || L_win - Tp < 3 ||
        !precision_ok(prec))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_window: bad arguments");
    DeviceGuard g(ctx->device);
    const float *base = X + offset;
    return ccm_one(ctx, base, ld, N, base, ld, N, L_win, E_lib, 0, tau, Tp, prec, rho, N,
                   nullptr, nullptr);
}

edm_status edm_predict(edm_ctx *ctx, const float *X_lib, int N_lib, const float *Y_tgt, int N_tgt,
                       int L, const int32_t *E_lib, const int32_t *tgt_of_lib, int tau, int Tp,
                       float *pred) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X_lib || !Y_tgt || !E_lib || !pred || N_lib < 1 || N_tgt < 1 || !series_len_ok(L) ||
        tau < 1 || Tp < 0 || L - Tp < 3 || (!tgt_of_lib && N_tgt < N_lib))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_predict: bad arguments");
    DeviceGuard g(ctx->device);
    const size_t slot = ccm_slot_bytes(L, tau, Tp);
    if (slot == 0) return set_error(ctx, EDM_ERR_INVALID_ARG, "series too short");
    const int G = LK_GROUP_FP32;
    const int chunk = ccm_chunk(ctx, N_lib, slot);
    edm_status st = ws_reserve(ctx, groups_bytes(chunk, G) +
                                        static_cast<size_t>(groups_max(chunk, G)) * G * slot);
    if (st != EDM_OK) return st;
    uint8_t *gmem = static_cast<uint8_t *>(ctx->ws);
    uint8_t *tables = gmem + groups_bytes(chunk, G);
    for (int c0 = 0; c0 < N_lib; c0 += chunk) {
        const int nlib = std::min(chunk, N_lib - c0);
        const CcmGroups grp = carve_groups(gmem, nlib, G);
        st = launch_group_libs(ctx, E_lib, 0, c0, nlib, L, tau, Tp, grp);
        if (st != EDM_OK) return st;
        st = launch_ccm_tables(ctx, X_lib, L, nlib, L, tau, Tp, grp, tables);
        if (st != EDM_OK) return st;
        st = launch_predict(ctx, Y_tgt, L, N_tgt, tgt_of_lib, L, tau, Tp, grp, tables, c0,
                            pred + static_cast<size_t>(c0) * L, L);
        if (st != EDM_OK) return st;
    }
    return EDM_OK;
}

edm_status edm_ccm_windows(edm_ctx *ctx, const float *X, int N, int ld, const int *offsets,
                           int n_windows, int L_win, const int32_t *E_lib, int tau, int Tp,
                           edm_precision prec, float *rho) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X || !offsets || !E_lib || !rho || N < 1 || n_windows < 1 || !series_len_ok(L_win) ||
        tau < 1 || Tp < 0 || L_win - Tp < 3 || !precision_ok(prec))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_windows: bad arguments");
    for (int w = 0; w < n_windows; ++w)
        if (offsets[w] < 0 || static_cast<long long>(offsets[w]) + L_win > ld)
            return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_windows: window %d out of range", w);
    DeviceGuard g(ctx->device);
    for (int w = 0; w < n_windows; ++w) {
        const float *base = X + offsets[w];
        edm_status st = ccm_one(ctx, base, ld, N, base, ld, N, L_win, E_lib, 0, tau, Tp, prec,
                                rho + static_cast<size_t>(w) * N * N, N, nullptr, nullptr);
        if (st != EDM_OK) return st;
    }
    return EDM_OK;
}

static bool instance_ok(const edm_instance &p) {
    return p.X && p.E_lib && p.N >= 1 && series_len_ok(p.L) && p.tau >= 1 && p.Tp >= 0 &&
           p.L - p.Tp >= 3 && p.lib_begin >= 0 && p.lib_end <= p.N && p.lib_begin <= p.lib_end;
}

edm_status edm_ccm_batched(edm_ctx *ctx, const edm_instance *inst, int n_inst,
                           edm_precision prec) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!inst || n_inst < 0 || !precision_ok(prec))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_batched: bad arguments");
    for (int i = 0; i < n_inst; ++i)
        if (!instance_ok(inst[i]) || !inst[i].rho)
            return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_batched: instance %d is invalid",
                             i);
    DeviceGuard g(ctx->device);
    std::vector<int> live;
    for (int i = 0; i < n_inst; ++i)
        if (inst[i].lib_end > inst[i].lib_begin) live.push_back(i);
    const int n = static_cast<int>(live.size());
    if (n == 0) return EDM_OK;
    std::vector<double> work(n);
    std::vector<size_t> need(n);
    std::vector<uint64_t> bucket(n);
    uint64_t key = 1469598103934665603ull;
    key = fnv1a(key, "ccm", 3);
    key = fnv1a(key, &prec, sizeof(prec));
    for (int j = 0; j < n; ++j) {
        const edm_instance &p = inst[live[j]];
        const int nl = p.lib_end - p.lib_begin;
        work[j] = static_cast<double>(nl) * p.N * p.L;
        need[j] = ccm_workspace_bytes(ctx, nl, p.N, p.L, p.tau, p.Tp, prec);
        bucket[j] = lookup_bucket(p.L, p.N, nl, prec);
        key = fnv1a(key, &p, sizeof(p));
    }
    auto fn = [&](edm_ctx *sub, int j) {
        const edm_instance &p = inst[live[j]];
        return ccm_one(sub, p.X + static_cast<size_t>(p.lib_begin) * p.L, p.L,
                       p.lib_end - p.lib_begin, p.X, p.L, p.N, p.L, p.E_lib + p.lib_begin, 0,
                       p.tau, p.Tp, prec, p.rho, p.N, nullptr, nullptr);
    };
    edm_status st = ensure_batch_state(ctx, std::max(1, std::min({ctx->batch_streams, n, 32})));
    if (st != EDM_OK) return st;
    st = ws_reserve(ctx->subs[0], *std::max_element(need.begin(), need.end()));
    if (st != EDM_OK) return st;
    st = autotune_lookup(ctx, n, bucket, fn);
    if (st != EDM_OK) return st;
    for (auto &kv : *ctx->tune) key = fnv1a(key, &kv, sizeof(kv));
    key = fnv1a(key, &ctx->lookup_lb, sizeof(ctx->lookup_lb));
    key = fnv1a(key, &ctx->autotune, sizeof(ctx->autotune));
    return run_batched(ctx, n, work, need, key, fn);
}

edm_status edm_simplex_optimal_E_batched(edm_ctx *ctx, const edm_instance *inst, int n_inst,
                                         int E_max, int Tp_sel, int32_t *const *E_out) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!inst || !E_out || n_inst < 0 || E_max < 1 || E_max > EDM_E_MAX || Tp_sel < 0)
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_simplex_optimal_E_batched: bad arguments");
    for (int i = 0; i < n_inst; ++i) {
        const edm_instance &p = inst[i];
        if (!p.X || !E_out[i] || p.N < 1 || !series_len_ok(p.L) || p.tau < 1 || p.L - Tp_sel < 3)
            return set_error(ctx, EDM_ERR_INVALID_ARG,
                             "edm_simplex_optimal_E_batched: instance %d is invalid", i);
    }
    if (n_inst == 0) return EDM_OK;
    DeviceGuard g(ctx->device);
    bool queue_ok = ctx->batch_queue;
    for (int i = 0; i < n_inst && queue_ok; ++i) queue_ok = sweep_queue_ok(inst[i].L);
    if (queue_ok) {
        return launch_simplex_queue(ctx, inst, n_inst, E_max, Tp_sel, E_out, true,
                                    ctx->batch_graph);
    }
    std::vector<double> work(n_inst);
    std::vector<size_t> need(n_inst);
    uint64_t key = 1469598103934665603ull;
    key = fnv1a(key, "simplex", 7);
    key = fnv1a(key, &E_max, sizeof(E_max));
    key = fnv1a(key, &Tp_sel, sizeof(Tp_sel));
    for (int i = 0; i < n_inst; ++i) {
        const edm_instance &p = inst[i];
        work[i] = static_cast<double>(p.N) * p.L * p.L;
        need[i] = simplex_workspace_bytes(ctx, p.N, p.L, E_max);
        key = fnv1a(key, &p, sizeof(p));
        key = fnv1a(key, &E_out[i], sizeof(E_out[i]));
    }
    auto fn = [&](edm_ctx *sub, int i) {
        const edm_instance &p = inst[i];
        return launch_simplex(sub, p.X, p.N, p.L, E_max, p.tau, Tp_sel, E_out[i], nullptr);
    };
    return run_batched(ctx, n_inst, work, need, key, fn);
}

edm_status edm_set_option(edm_ctx *ctx, const char *name, long long value) {
    if (!ctx || !name) return EDM_ERR_INVALID_ARG;
    if (!strcmp(name, "batch_streams") && value >= 1 && value <= 32) {
        ctx->batch_streams = static_cast<int>(value);
    } else if (!strcmp(name, "batch_graph") && (value == 0 || value == 1)) {
        ctx->batch_graph = value != 0;
    } else if (!strcmp(name, "autotune") && (value == 0 || value == 1)) {
        ctx->autotune = value != 0;
    } else if (!strcmp(name, "lookup_libs_per_cta") && value >= 0 && value <= 4096) {
        ctx->lookup_lb = static_cast<int>(value);
    } else if (!strcmp(name, "table_budget_mb") && value >= 16) {
        ctx->table_budget = static_cast<size_t>(value) << 20;
    } else if (!strcmp(name, "autotune_reset") && value == 1) {
        ctx->tune->clear();
    } else if (!strcmp(name, "diagnostics") && (value == 0 || value == 1)) {
        ctx->diag = value != 0;
    } else if (!strcmp(name, "batch_queue") && (value == 0 || value == 1)) {
        ctx->batch_queue = value != 0;
    } else {
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_set_option: bad option %s=%lld", name,
                         value);
    }
    ctx->graph_key = 0;  // options change what a captured graph would hold
    ctx->qgraph_key = 0;
    return EDM_OK;
}

}  // extern "C"
