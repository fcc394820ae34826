// probe.cu -- measured shared-memory gather bandwidth (the lookup roofline).
//
// Each warp reads whole 128-byte rows of a 32 KB shared-memory tile (lane l
// reads word l of the row), visiting rows in a scattered order fixed at
// compile time, and folds the values into four independent FP32 sums.  Every
// read is one conflict-free wavefront and needs one add, so the loop is
// limited by the shared-memory pipe, as the lookup's gathers are.
#include "edm_internal.cuh"

namespace edm {

constexpr int PR_ROWS = 256;       // 32 KB tile
constexpr int PR_WARPS = 16;
constexpr int PR_UNROLL = 64;

__global__ void __launch_bounds__(PR_WARPS * 32) smem_probe_kernel(int iters, float *sink) {
    __shared__ __align__(128) float tile[PR_ROWS * 32];
    for (int i = threadIdx.x; i < PR_ROWS * 32; i += blockDim.x) tile[i] = static_cast<float>(i & 7);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float *tl = tile + lane;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int base = (threadIdx.x >> 5) * 37;
    for (int it = 0; it < iters; ++it) {
        // base row <= 127 and offset <= 127: every row read is < PR_ROWS
        const float *p = tl + ((base & (PR_ROWS / 2 - 1)) << 5);
        // scattered compile-time row offsets (149 j) mod 128
#pragma unroll
        for (int j = 0; j < PR_UNROLL; j += 4) {
            a0 += p[((149 * (j + 0)) & (PR_ROWS / 2 - 1)) << 5];
            a1 += p[((149 * (j + 1)) & (PR_ROWS / 2 - 1)) << 5];
            a2 += p[((149 * (j + 2)) & (PR_ROWS / 2 - 1)) << 5];
            a3 += p[((149 * (j + 3)) & (PR_ROWS / 2 - 1)) << 5];
        }
        base += 97;
        base &= (PR_ROWS / 2 - 1);
    }
    const float s = a0 + a1 + a2 + a3;
    if (s == -1.f) sink[blockIdx.x] = s;  // never true; keeps the loads alive
}

edm_status launch_smem_probe(edm_ctx *ctx, double ms, double *bytes_per_s) {
    float *sink = nullptr;
    edm_status st = cuda_check(ctx, cudaMalloc(&sink, sizeof(float) * 4 * ctx->num_sms), "probe");
    if (st != EDM_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = 4 * ctx->num_sms;  // 4 CTAs x 16 warps per SM
    int iters = 64;
    double got = 0.0;
    for (int attempt = 0; attempt < 6; ++attempt) {
        cudaEventRecord(e0, ctx->stream);
        before_launch(ctx);
        smem_probe_kernel<<<blocks, PR_WARPS * 32, 0, ctx->stream>>>(iters, sink);
        st = after_launch(ctx, "smem_probe_kernel");
        if (st != EDM_OK) break;
        cudaEventRecord(e1, ctx->stream);
        st = cuda_check(ctx, cudaEventSynchronize(e1), "probe sync");
        if (st != EDM_OK) break;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        const double bytes = static_cast<double>(blocks) * PR_WARPS * iters * PR_UNROLL * 128.0;
        got = bytes / (t * 1e-3);
        if (t >= 0.5 * ms) break;
        iters = static_cast<int>(std::min<double>(1 << 24, iters * std::max(2.0, ms / std::max(t, 0.01f))));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    *bytes_per_s = got;
    return st;
}

// L2 gather bandwidth: the access pattern of the lookup when the target tile
// stays in global memory (series longer than a shared-memory tile allows):
// every warp reads whole 128-byte rows (lane l reads word l) of a global
// buffer at scattered row indexes, through the read-only path.  The buffer
// (PL2_ROWS rows, 48 MB) fits the L2 cache but not L1, so after the first
// pass every read is an L2 hit.
constexpr int PL2_ROWS = 3 << 17;   // 393,216 rows of 128 B = 48 MB
constexpr int PL2_UNROLL = 16;

__global__ void __launch_bounds__(PR_WARPS * 32) l2_probe_kernel(const float *__restrict__ buf,
                                                                 int iters, float *sink) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // a per-warp linear congruential walk over the rows (row < PL2_ROWS)
    uint32_t r = 2654435761u * static_cast<uint32_t>(gw + 1);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < PL2_UNROLL; j += 4) {
            r = r * 1664525u + 1013904223u;
            a0 += __ldg(buf + static_cast<size_t>((r >> 8) % PL2_ROWS) * 32 + lane);
            r = r * 1664525u + 1013904223u;
            a1 += __ldg(buf + static_cast<size_t>((r >> 8) % PL2_ROWS) * 32 + lane);
            r = r * 1664525u + 1013904223u;
            a2 += __ldg(buf + static_cast<size_t>((r >> 8) % PL2_ROWS) * 32 + lane);
            r = r * 1664525u + 1013904223u;
            a3 += __ldg(buf + static_cast<size_t>((r >> 8) % PL2_ROWS) * 32 + lane);
        }
    }
    const float s = a0 + a1 + a2 + a3;
    if (s == -1.f) sink[blockIdx.x] = s;  // never true; keeps the loads alive
}

edm_status launch_l2_probe(edm_ctx *ctx, double ms, double *bytes_per_s) {
    float *buf = nullptr, *sink = nullptr;
    const size_t bytes = static_cast<size_t>(PL2_ROWS) * 128;
    edm_status st = cuda_check(ctx, cudaMalloc(&buf, bytes), "l2 probe");
    if (st != EDM_OK) return st;
    st = cuda_check(ctx, cudaMalloc(&sink, sizeof(float) * 8 * ctx->num_sms), "l2 probe");
    if (st != EDM_OK) {
        cudaFree(buf);
        return st;
    }
    cudaMemsetAsync(buf, 0, bytes, ctx->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = 4 * ctx->num_sms;  // 64 warps per SM
    int iters = 16;
    double got = 0.0;
    before_launch(ctx);
    l2_probe_kernel<<<blocks, PR_WARPS * 32, 0, ctx->stream>>>(buf, iters, sink);  // warm L2
    st = after_launch(ctx, "l2_probe_kernel");
    for (int attempt = 0; st == EDM_OK && attempt < 6; ++attempt) {
        cudaEventRecord(e0, ctx->stream);
        before_launch(ctx);
        l2_probe_kernel<<<blocks, PR_WARPS * 32, 0, ctx->stream>>>(buf, iters, sink);
        st = after_launch(ctx, "l2_probe_kernel");
        if (st != EDM_OK) break;
        cudaEventRecord(e1, ctx->stream);
        st = cuda_check(ctx, cudaEventSynchronize(e1), "l2 probe sync");
        if (st != EDM_OK) break;
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        got = static_cast<double>(blocks) * PR_WARPS * iters * PL2_UNROLL * 128.0 / (t * 1e-3);
        if (t >= 0.5 * ms) break;
        iters = static_cast<int>(std::min<double>(1 << 22, iters * std::max(2.0, ms / std::max(t, 0.01f))));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(buf);
    *bytes_per_s = got;
    return st;
}

// One thread waits, with the bounded wait every pipelined kernel of the
// library uses, on an mbarrier that expects one arrival which never comes.
// The wait gives up after `ms` milliseconds, raises the timeout flag and sets
// the CTA's abort word; a second wait on the same barrier then returns at
// once, so the kernel ends after about one limit, not two.
__global__ void wait_check_kernel(uint64_t limit_ns, int *flags) {
    __shared__ uint64_t bar;
    __shared__ int abort_word;
    abort_word = 0;
    mbar_init(&bar, 1);
    fence_barrier_init();
    mbar_wait_bounded(&bar, 0, flags, &abort_word, limit_ns);
    mbar_wait_bounded(&bar, 0, flags, &abort_word, limit_ns);
}

edm_status launch_wait_check(edm_ctx *ctx, int ms) {
    before_launch(ctx);
    wait_check_kernel<<<1, 1, 0, ctx->stream>>>(static_cast<uint64_t>(ms) * 1000000ull,
                                                ctx->d_flags);
    return after_launch(ctx, "wait_check_kernel");
}

}  // namespace edm
