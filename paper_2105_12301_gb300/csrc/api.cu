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
// rows are ld_lib / ld_tgt floats apart.
static edm_status ccm_one(edm_ctx *ctx, const float *X_lib, long long ld_lib, int N_lib,
                          const float *Y_tgt, long long ld_tgt, int N_tgt, int L,
                          const int32_t *E_lib, int tau, int Tp, edm_precision prec, float *rho) {
    const size_t yt_bytes = target_store_bytes(N_tgt, L, prec);
    const size_t mean_bytes = align_up(sizeof(double) * N_tgt, 256);
    const size_t sums_bytes = align_up(sizeof(double) * N_tgt * EDM_E_MAX, 256);
    const size_t slot = ccm_slot_bytes(L, tau, Tp);
    if (slot == 0) return set_error(ctx, EDM_ERR_INVALID_ARG, "series too short");
    const int chunk = static_cast<int>(
        std::max<size_t>(1, std::min<size_t>(N_lib, ctx->table_budget / slot)));
    edm_status st = ws_reserve(ctx, yt_bytes + mean_bytes + 2 * sums_bytes + chunk * slot);
    if (st != EDM_OK) return st;
    uint8_t *base = static_cast<uint8_t *>(ctx->ws);
    uint8_t *Yt = base;
    double *mean = reinterpret_cast<double *>(base + yt_bytes);
    double *ysum = reinterpret_cast<double *>(base + yt_bytes + mean_bytes);
    double *yysum = reinterpret_cast<double *>(base + yt_bytes + mean_bytes + sums_bytes);
    uint8_t *tables = base + yt_bytes + mean_bytes + 2 * sums_bytes;
    st = launch_target_store(ctx, Y_tgt, ld_tgt, N_tgt, L, tau, Tp, prec, Yt, mean, ysum, yysum);
    if (st != EDM_OK) return st;
    for (int c0 = 0; c0 < N_lib; c0 += chunk) {
        const int nlib = std::min(chunk, N_lib - c0);
        st = launch_ccm_tables(ctx, X_lib, ld_lib, c0, nlib, L, E_lib, tau, Tp, tables, slot);
        if (st != EDM_OK) return st;
        st = launch_lookup(ctx, Yt, N_tgt, L, tables, slot, E_lib, c0, nlib, tau, Tp, prec, ysum,
                           yysum, rho + static_cast<size_t>(c0) * N_tgt, N_tgt);
        if (st != EDM_OK) return st;
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
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                               device) != cudaSuccess ||
        cudaMalloc(&ctx->d_flags, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_flags, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_flags) cudaFree(ctx->d_flags);
        delete ctx;
        return EDM_ERR_CUDA;
    }
    *out = ctx;
    return EDM_OK;
}

edm_status edm_destroy(edm_ctx *ctx) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    prof_clear(ctx);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
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

uint64_t edm_kernel_launches(edm_ctx *ctx) { return ctx ? ctx->launches : 0; }

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
        tau < 1 || Tp < 0 || L - Tp < 3 || (prec != EDM_FP32 && prec != EDM_BF16_TARGETS))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_all: bad arguments");
    DeviceGuard g(ctx->device);
    return ccm_one(ctx, X_lib, L, N_lib, Y_tgt, L, N_tgt, L, E_lib, tau, Tp, prec, rho);
}

edm_status edm_ccm_window(edm_ctx *ctx, const float *X, int N, int ld, int offset, int L_win,
                          const int32_t *E_lib, int tau, int Tp, edm_precision prec, float *rho) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!X || !E_lib || !rho || N < 1 || offset < 0 || !series_len_ok(L_win) ||
        static_cast<long long>(offset) + L_win > ld || tau < 1 || Tp < 0 || L_win - Tp < 3 ||
        (prec != EDM_FP32 && prec != EDM_BF16_TARGETS))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_window: bad arguments");
    DeviceGuard g(ctx->device);
    const float *base = X + offset;
    return ccm_one(ctx, base, ld, N, base, ld, N, L_win, E_lib, tau, Tp, prec, rho);
}

edm_status edm_ccm_batched(edm_ctx *ctx, const edm_instance *inst, int n_inst,
                           edm_precision prec) {
    if (!ctx) return EDM_ERR_INVALID_ARG;
    if (!inst || n_inst < 0 || (prec != EDM_FP32 && prec != EDM_BF16_TARGETS))
        return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_batched: bad arguments");
    for (int i = 0; i < n_inst; ++i) {
        const edm_instance &p = inst[i];
        if (!p.X || !p.E_lib || !p.rho || p.N < 1 || !series_len_ok(p.L) || p.tau < 1 ||
            p.Tp < 0 || p.L - p.Tp < 3 || p.lib_begin < 0 || p.lib_end > p.N ||
            p.lib_begin > p.lib_end)
            return set_error(ctx, EDM_ERR_INVALID_ARG, "edm_ccm_batched: instance %d is invalid",
                             i);
    }
    DeviceGuard g(ctx->device);
    for (int i = 0; i < n_inst; ++i) {
        const edm_instance &p = inst[i];
        if (p.lib_end == p.lib_begin) continue;
        edm_status st = ccm_one(ctx, p.X + static_cast<size_t>(p.lib_begin) * p.L, p.L,
                                p.lib_end - p.lib_begin, p.X, p.L, p.N, p.L,
                                p.E_lib + p.lib_begin, p.tau, p.Tp, prec, p.rho);
        if (st != EDM_OK) return st;
    }
    return EDM_OK;
}

}  // extern "C"
