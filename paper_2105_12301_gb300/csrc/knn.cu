// knn.cu -- time-delay embedding and exhaustive all-kNN (kEDM section 2.1
// steps 1-3, Algorithms 1 and 2).
//
// One CTA holds one series in shared memory (the paper's "team scratch"
// caching of x) and a block of its query rows; one warp per query row runs
// knn_row (knn_core.cuh).  Embedding is fused: lagged values are read from
// the staged series, the embedded points are never written.
#include "knn_core.cuh"

namespace edm {

constexpr int KNN_WARPS = 8;
constexpr int SERIES_SMEM_MAX = 96 * 1024;  // stage the series when it fits

// Series longer than 2,048 points: candidates in chunks of 32 slots per lane
// (1,024 candidates) held in registers, selected against a running list.
constexpr int TL_CH = 32;

struct TableLongScratch {
    WarpScratch ws;
    uint64_t list[32];  // the R smallest FP32 keys seen so far, ascending
};

// ------------------------------------------------------------------ embed

__global__ void embed_kernel(const float *__restrict__ x, int L, int E, int tau,
                             float *__restrict__ out) {
    const int n = L - (E - 1) * tau;
    const long long total = static_cast<long long>(n) * E;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int row = static_cast<int>(i / E), l = static_cast<int>(i % E);
        out[i] = x[(E - 1) * tau + row - l * tau];
    }
}

edm_status launch_embed(edm_ctx *ctx, const float *x, int L, int E, int tau, float *out) {
    const long long total = static_cast<long long>(L - (E - 1) * tau) * E;
    const int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 4LL * ctx->num_sms));
    before_launch(ctx);
    embed_kernel<<<blocks, 256, 0, ctx->stream>>>(x, L, E, tau, out);
    return after_launch(ctx, "embed_kernel");
}

// ------------------------------------------------------- series staging

// Copy the series into shared memory when it fits (SMEM), else read it from
// global memory through L1.  Returns the pointer the rows read from.
template <bool SMEM>
__device__ __forceinline__ const float *stage_series(const float *xg, int L, float *xs_s) {
    if constexpr (!SMEM) {
        return xg;
    } else {
        for (int i = threadIdx.x; i < L; i += blockDim.x) xs_s[i] = xg[i];
        __syncthreads();
        return xs_s;
    }
}

static size_t knn_smem_bytes(bool smem_series, int L) {
    return KNN_WARPS * sizeof(WarpScratch) + (smem_series ? align_up(sizeof(float) * L, 16) : 0);
}

// Rows per CTA: enough CTAs to fill the GPU several times over.
static int rows_per_cta(edm_ctx *ctx, int N, int n) {
    const long long want_ctas = 8LL * ctx->num_sms;
    long long blocks_per_series = (want_ctas + N - 1) / N;
    int rb = static_cast<int>((n + blocks_per_series - 1) / blocks_per_series);
    rb = std::max(rb, 4 * KNN_WARPS);
    return std::min(rb, n);
}

// ---------------------------------------------------------------- edm_knn

template <int E, bool SMEM>
__global__ void __launch_bounds__(KNN_WARPS * 32)
    knn_out_kernel(const float *__restrict__ X, int L, int tau, int Tp, int K, int RB,
                   int32_t *__restrict__ idx, float *__restrict__ dist,
                   unsigned long long *stats) {
    extern __shared__ __align__(16) uint8_t smem[];
    WarpScratch *wsa = reinterpret_cast<WarpScratch *>(smem);
    float *xs_s = reinterpret_cast<float *>(smem + KNN_WARPS * sizeof(WarpScratch));
    const int series = blockIdx.x;
    const float *xs = stage_series<SMEM>(X + static_cast<size_t>(series) * L, L, xs_s);
    const int lo = (E - 1) * tau, hi = L - 1 - Tp, n = hi - lo + 1;
    const int r0 = blockIdx.y * RB, r1 = min(n, r0 + RB);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    WarpScratch *ws = wsa + warp;
    FallbackCount fc;
    for (int i = r0 + warp; i < r1; i += KNN_WARPS) {
        int u = 0;
        float d = 0.f;
        fc.add(knn_row<E, KNN_ORDERED>(xs, lo + i, lo, hi, tau, K, ws, &u, &d));
        const size_t o = (static_cast<size_t>(series) * n + i) * K;
        if (lane < K) {
            idx[o + lane] = u;
            if (dist) dist[o + lane] = d;
        }
    }
    fc.flush(stats);
}

// edm_knn for series longer than 2,048 points: chunked candidates held in
// registers against a running list (knn_row_chunked, exact FP64 order).
template <bool SMEM>
__global__ void __launch_bounds__(KNN_WARPS * 32)
    knn_out_long_kernel(const float *__restrict__ X, int L, int E, int tau, int Tp, int K, int RB,
                        int32_t *__restrict__ idx, float *__restrict__ dist,
                        unsigned long long *stats);

template <int E>
static edm_status launch_knn_E(edm_ctx *ctx, const float *X, int N, int L, int tau, int Tp, int K,
                               int32_t *idx, float *dist) {
    const int n = L - (E - 1) * tau - Tp;
    const int RB = rows_per_cta(ctx, N, n);
    dim3 grid(N, (n + RB - 1) / RB);
    const bool smem_series = sizeof(float) * static_cast<size_t>(L) <= SERIES_SMEM_MAX;
    const size_t smem = knn_smem_bytes(smem_series, L);
    if (smem_series) {
        auto kern = knn_out_kernel<E, true>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        before_launch(ctx);
        kern<<<grid, KNN_WARPS * 32, smem, ctx->stream>>>(X, L, tau, Tp, K, RB, idx, dist,
                                                          diag_stats(ctx));
    } else {
        auto kern = knn_out_kernel<E, false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        before_launch(ctx);
        kern<<<grid, KNN_WARPS * 32, smem, ctx->stream>>>(X, L, tau, Tp, K, RB, idx, dist,
                                                          diag_stats(ctx));
    }
    return after_launch(ctx, "knn_out_kernel");
}

edm_status launch_knn(edm_ctx *ctx, const float *X, int N, int L, int E, int tau, int Tp, int k,
                      int32_t *idx, float *dist) {
    if (L > 2048 && E >= 1 && E <= EDM_E_MAX) {
        const int n = L - (E - 1) * tau - Tp;
        const int RB = rows_per_cta(ctx, N, n);
        dim3 grid(N, (n + RB - 1) / RB);
        const bool smem_series = sizeof(float) * static_cast<size_t>(L) <= SERIES_SMEM_MAX;
        const size_t smem = KNN_WARPS * sizeof(TableLongScratch) +
                            (smem_series ? align_up(sizeof(float) * L, 16) : 0);
        auto kern = smem_series ? knn_out_long_kernel<true> : knn_out_long_kernel<false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        before_launch(ctx);
        kern<<<grid, KNN_WARPS * 32, smem, ctx->stream>>>(X, L, E, tau, Tp, k, RB, idx, dist,
                                                          diag_stats(ctx));
        return after_launch(ctx, "knn_out_kernel");
    }
    switch (E) {
#define EDM_CASE(e) \
    case e: return launch_knn_E<e>(ctx, X, N, L, tau, Tp, k, idx, dist);
        EDM_CASE(1) EDM_CASE(2) EDM_CASE(3) EDM_CASE(4) EDM_CASE(5) EDM_CASE(6) EDM_CASE(7)
        EDM_CASE(8) EDM_CASE(9) EDM_CASE(10) EDM_CASE(11) EDM_CASE(12) EDM_CASE(13)
        EDM_CASE(14) EDM_CASE(15) EDM_CASE(16) EDM_CASE(17) EDM_CASE(18) EDM_CASE(19)
        EDM_CASE(20)
#undef EDM_CASE
    default: return set_error(ctx, EDM_ERR_INVALID_ARG, "E=%d out of range", E);
    }
}

// ----------------------------------------------------- CCM neighbour tables

// Write row i of a library's table (pair-interleaved layout, see
// table_pair_bytes).  Lane r < K holds neighbour r (time index u) and its
// normalised weight w.  The warp that writes the last row of an odd table
// also writes the dummy row that completes its pair.
__device__ __forceinline__ void write_table_row(uint8_t *slot, size_t pair_stride, int i, int n,
                                                int K, int L, int Tp, int u, float w) {
    const int lane = lane_id();
    const int words = table_row_words(K);
    const int h = lane - (K - 1);
    const int ua = __shfl_sync(FULL, u, min(max(2 * h, 0), 31));
    const int ub = __shfl_sync(FULL, u, min(max(2 * h + 1, 0), 31));
    uint32_t word = 0;
    if (lane < K - 1) {
        word = __float_as_uint(w);
    } else if (h >= 0 && 2 * h < K) {
        word = static_cast<uint32_t>(ua + Tp) & 0xffffu;
        if (2 * h + 1 < K) word |= (static_cast<uint32_t>(ub + Tp) & 0xffffu) << 16;
    }
    uint32_t *block = reinterpret_cast<uint32_t *>(slot + static_cast<size_t>(i >> 1) * pair_stride);
    if (lane < words) block[2 * lane + (i & 1)] = word;
    if ((n & 1) && i == n - 1 && lane < words)
        block[2 * lane + 1] = lane < K - 1 ? 0u : (static_cast<uint32_t>(L) | (static_cast<uint32_t>(L) << 16));
}

// The library of group slot s (blockIdx.x), its E, where its table starts and
// the distance between its consecutive pair blocks.  False for an empty slot
// or a library whose E is invalid (its group has E = 0; the lookup writes its
// NaN row and raises the flag).
struct TableSlot {
    int lib, E;
    uint8_t *base;
    size_t pair_stride;
};

__device__ __forceinline__ bool table_slot(const CcmGroups &g, uint8_t *tables, TableSlot &ts) {
    const int s = blockIdx.x;
    ts.lib = g.lib[s];
    if (ts.lib < 0) return false;
    const int grp = s / g.G, m = s % g.G;
    ts.E = g.E[grp];
    if (ts.E == 0) return false;
    const size_t pb = table_pair_bytes(ts.E + 1);
    ts.base = tables + g.off[grp] + m * pb;
    ts.pair_stride = pb * g.G;
    return true;
}

// Resident CTAs per SM that the register budget of the table builder is set
// for: the distances take CH registers a thread, and with these bounds no
// slot count spills.
constexpr int table_min_blocks(int CH) { return CH >= 16 && CH <= 24 ? 3 : CH <= 48 ? 2 : 1; }

// Register-resident variant for series of up to 32*CH points: the FP32
// distances from x(t) to every candidate are accumulated lag by lag in
// registers (lag order 0..E-1, the same operations as dist32) and the
// neighbours are selected from registers (select_set_regs), one pass over
// the candidates.  HEAD1: every lag offset (E-1)tau is below 32, so only
// candidate slot 0 can reach before the start of the series.
template <int CH, bool HEAD1>
__global__ void __launch_bounds__(KNN_WARPS * 32, table_min_blocks(CH))
    ccm_table_regs_kernel(const float *__restrict__ X, long long ld, int L, int tau, int Tp,
                          int RB, const CcmGroups g, uint8_t *__restrict__ tables,
                          unsigned long long *stats) {
    extern __shared__ __align__(16) uint8_t smem[];
    WarpScratch *wsa = reinterpret_cast<WarpScratch *>(smem);
    float *xs = reinterpret_cast<float *>(smem + KNN_WARPS * sizeof(WarpScratch));
    TableSlot ts;
    if (!table_slot(g, tables, ts)) return;
    const int E = ts.E;
    const int K = E + 1;
    const int lo = (E - 1) * tau, hi = L - 1 - Tp, n = hi - lo + 1;
    const int r0 = blockIdx.y * RB, r1 = min(n, r0 + RB);
    if (r0 >= r1) return;
    const float *xg = X + static_cast<size_t>(ts.lib) * ld;
    for (int i = threadIdx.x; i < 32 * CH; i += blockDim.x) xs[i] = i < L ? xg[i] : 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = lane_id();
    WarpScratch *ws = wsa + warp;
    const unsigned keep = bitonic_keep_min_bits();
    FallbackCount fc;
    for (int i = r0 + warp; i < r1; i += KNN_WARPS) {
        const int t = lo + i;
        float s[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int u = lane + 32 * j;
            s[j] = (u >= lo && u <= hi && u != t) ? 0.f : EDM_INF;
        }
        for (int l = 0; l < E; ++l) {
            const int off = l * tau;
            const float q = xs[t - off];
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int u = lane + 32 * j;
                const float x = (!HEAD1 || j == 0) ? xs[max(u - off, 0)] : xs[u - off];
                const float d = __fsub_rn(q, x);
                s[j] = __fmaf_rn(d, d, s[j]);
            }
        }
        int u = 0;
        float d = 0.f;
        fc.add(select_set_regs<CH>(s, xs, t, lo, hi, E, tau, K, ws, u, d, keep));
        const float w = simplex_weight(d, K);
        write_table_row(ts.base, ts.pair_stride, i, n, K, L, Tp, u, w);
    }
    fc.flush(stats);
}

// ------------------------------------------- tables of long series (> 2,048)

// The K nearest neighbours of the query time t among the times lo..hi, from
// chunks of 1,024 candidates whose FP32 squared distances are accumulated in
// registers (lag order 0..E-1, one fma per lag, the same operations as
// dist32).  Each chunk is selected against a running list of the R smallest
// keys, as in the long optimal-E sweep; then the FP64 step of knn_row:
//   KNN_SET (R = K+1): the exact FP64 neighbour set, FP32 order and
//     distances unless the band had to be resolved;
//   KNN_ORDERED (R = K+KNN_MARGIN): the exact FP64 order (s64, u), d the
//     FP64 square root rounded to float.
// On return lane r < K holds the r-th neighbour and its distance.
//
// drow (optional): the row's FP32 squared distances already materialised in
// memory, drow[u - lo] for u in lo..hi (the value at t itself is ignored);
// they are read instead of computed and must equal the values computed here
// (same operations, same order), which the FP64 band step relies on.
template <int MODE>
__device__ int knn_row_chunked(const float *xs, int L, int t, int lo, int hi, int E, int tau,
                               int K, TableLongScratch *sc, int &u_out, float &d_out,
                               const float *drow = nullptr) {
    const int lane = lane_id();
    WarpScratch *ws = &sc->ws;
    uint64_t *list = sc->list;
    const int nc = hi - lo;
    const int R = MODE == KNN_ORDERED ? min(K + KNN_MARGIN, nc) : min(K + 1, nc);
    int have = 0;
    bool deg = false;
    for (int c0 = 0; c0 <= hi; c0 += 32 * TL_CH) {
        float s[TL_CH];
        if (drow) {
#pragma unroll
            for (int j = 0; j < TL_CH; ++j) {
                const int u = c0 + lane + 32 * j;
                s[j] = (u >= lo && u <= hi && u != t) ? __ldg(drow + (u - lo)) : EDM_INF;
            }
        } else if (c0 >= lo && c0 + 32 * TL_CH - 1 <= hi) {
            // every candidate is a point of P: no clamp, only t itself is out
            const float *xl = xs + (c0 + lane);
#pragma unroll
            for (int j = 0; j < TL_CH; ++j) s[j] = (c0 + lane + 32 * j == t) ? EDM_INF : 0.f;
            for (int l = 0; l < E; ++l) {
                const float q = xs[t - l * tau];
                const float *xo = xl - l * tau;
#pragma unroll
                for (int j = 0; j < TL_CH; ++j) {
                    const float d = __fsub_rn(q, xo[32 * j]);
                    s[j] = __fmaf_rn(d, d, s[j]);
                }
            }
        } else {
            // non-candidates start at +inf and stay there (fma(d, d, inf) = inf)
#pragma unroll
            for (int j = 0; j < TL_CH; ++j) {
                const int u = c0 + lane + 32 * j;
                s[j] = (u >= lo && u <= hi && u != t) ? 0.f : EDM_INF;
            }
            for (int l = 0; l < E; ++l) {
                const float q = xs[t - l * tau];
#pragma unroll
                for (int j = 0; j < TL_CH; ++j) {
                    const int u = c0 + lane + 32 * j;
                    const float d = __fsub_rn(q, xs[min(max(u - l * tau, 0), L - 1)]);
                    s[j] = __fmaf_rn(d, d, s[j]);
                }
            }
        }
        if (deg) continue;
        float gm[TL_CH / 4];
        group_minima<TL_CH>(s, gm);
        float bound = have == R ? key_s(list[R - 1]) : EDM_INF;
        if (have < R) {
            float lmin = EDM_INF;
#pragma unroll
            for (int g = 0; g < TL_CH / 4; ++g) lmin = fminf(lmin, gm[g]);
            bound = fminf(bound, warp_sorted_at_f(lmin, min(R, 32) - 1));
        }
        int c = bound == EDM_INF ? compact_le<TL_CH>(s, bound, ws, c0)
                                 : compact_le_groups<TL_CH>(s, gm, bound, ws, c0);
        if (c > KNN_CAP - 32) {
            auto in_list = [&](float b) {
                const bool p = lane < have && key_s(list[lane]) <= b;
                return __popc(__ballot_sync(FULL, p));
            };
            const float b = shrink_bound<TL_CH>(s, bound, c, R, KNN_CAP - 32, in_list);
            if (b >= 0.f) c = compact_le_groups<TL_CH>(s, gm, b, ws, c0);
        }
        if (c > KNN_CAP - 32) {
            deg = true;  // more values tie than the buffer holds: FP64 below
            continue;
        }
        if (c == 0) continue;
        for (int e = lane; e < have; e += 32) ws->key[c + e] = list[e];
        __syncwarp();
        const int tot = c + have;
        rank_keys(ws, tot, min(R, tot));
        have = min(R, tot);
        for (int e = lane; e < have; e += 32) list[e] = ws->sel[e];
        __syncwarp();
    }
    int flags = 0;
    if (!deg) {
        const float edge = band_edge(key_s(list[K - 1]), E);
        if (MODE == KNN_SET && (R <= K || key_s(list[K]) > edge)) {
            if (lane < K) {
                u_out = key_u(list[lane]);
                d_out = sqrtf(key_s(list[lane]));
            }
            __syncwarp();
            return 0;
        }
        if (MODE == KNN_ORDERED && (R == nc || key_s(list[R - 1]) > edge)) {
            // the R collected keys cover the band: rank them in FP64
            double s64 = __longlong_as_double(0x7ff0000000000000LL);
            int u = 0x7fffffff;
            if (lane < R) {
                u = key_u(list[lane]);
                s64 = dist64(xs, t, u, E, tau);
            }
            int rank = 0;
            for (int j = 0; j < R; ++j) {
                const double sj = __shfl_sync(FULL, s64, j);
                const int uj = __shfl_sync(FULL, u, j);
                rank += less64(sj, uj, s64, u);
            }
            if (lane < R && rank < K) {
                ws->sel_s64[rank] = s64;
                ws->sel_u[rank] = u;
            }
            __syncwarp();
            if (lane < K) {
                u_out = ws->sel_u[lane];
                d_out = __double2float_rn(__dsqrt_rn(ws->sel_s64[lane]));
            }
            __syncwarp();
            return 0;
        }
        // resolve the band in FP64: every candidate with s32 <= edge
        if (lane == 0) ws->count = 0;
        __syncwarp();
        for (int u = lo + lane; u <= hi; u += 32) {
            if (u == t) continue;
            float v = 0.f;
            for (int l = 0; l < E; ++l) {
                const float d = __fsub_rn(xs[t - l * tau], xs[u - l * tau]);
                v = __fmaf_rn(d, d, v);
            }
            if (v <= edge) {
                const int pos = atomicAdd(&ws->count, 1);
                if (pos < KNN_CAP) ws->key[pos] = mk_key(v, u);
            }
        }
        __syncwarp();
        const int c = ws->count;
        __syncwarp();
        flags = KNN_USED_BAND;
        if (c <= KNN_CAP) {
            rank_band_fp64(xs, t, E, tau, ws, c, K);
        } else {
            brute_fp64(xs, t, lo, hi, E, tau, ws, K);
            flags |= KNN_USED_BRUTE;
        }
    } else {
        brute_fp64(xs, t, lo, hi, E, tau, ws, K);
        flags = KNN_USED_BAND | KNN_USED_BRUTE;
    }
    if (lane < K) {
        u_out = ws->sel_u[lane];
        d_out = __double2float_rn(__dsqrt_rn(ws->sel_s64[lane]));
    }
    __syncwarp();
    return flags;
}

template <bool SMEM>
__global__ void __launch_bounds__(KNN_WARPS * 32)
    ccm_table_long_kernel(const float *__restrict__ X, long long ld, int L, int tau, int Tp,
                          int RB, const CcmGroups g, uint8_t *__restrict__ tables,
                          unsigned long long *stats) {
    extern __shared__ __align__(16) uint8_t smem[];
    TableLongScratch *sca = reinterpret_cast<TableLongScratch *>(smem);
    float *xs_s = reinterpret_cast<float *>(smem + KNN_WARPS * sizeof(TableLongScratch));
    TableSlot ts;
    if (!table_slot(g, tables, ts)) return;
    const int E = ts.E;
    const int lo = (E - 1) * tau, hi = L - 1 - Tp, n = hi - lo + 1;
    const int r0 = blockIdx.y * RB, r1 = min(n, r0 + RB);
    if (r0 >= r1) return;
    const float *xs = stage_series<SMEM>(X + static_cast<size_t>(ts.lib) * ld, L, xs_s);
    const int warp = threadIdx.x >> 5;
    TableLongScratch *sc = sca + warp;
    FallbackCount fc;
    for (int i = r0 + warp; i < r1; i += KNN_WARPS) {
        int u = 0;
        float d = 0.f;
        fc.add(knn_row_chunked<KNN_SET>(xs, L, lo + i, lo, hi, E, tau, E + 1, sc, u, d));
        const float w = simplex_weight(d, E + 1);
        write_table_row(ts.base, ts.pair_stride, i, n, E + 1, L, Tp, u, w);
    }
    fc.flush(stats);
}

template <bool SMEM>
__global__ void __launch_bounds__(KNN_WARPS * 32)
    knn_out_long_kernel(const float *__restrict__ X, int L, int E, int tau, int Tp, int K, int RB,
                        int32_t *__restrict__ idx, float *__restrict__ dist,
                        unsigned long long *stats) {
    extern __shared__ __align__(16) uint8_t smem[];
    TableLongScratch *sca = reinterpret_cast<TableLongScratch *>(smem);
    float *xs_s = reinterpret_cast<float *>(smem + KNN_WARPS * sizeof(TableLongScratch));
    const int series = blockIdx.x;
    const float *xs = stage_series<SMEM>(X + static_cast<size_t>(series) * L, L, xs_s);
    const int lo = (E - 1) * tau, hi = L - 1 - Tp, n = hi - lo + 1;
    const int r0 = blockIdx.y * RB, r1 = min(n, r0 + RB);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    TableLongScratch *sc = sca + warp;
    FallbackCount fc;
    for (int i = r0 + warp; i < r1; i += KNN_WARPS) {
        int u = 0;
        float d = 0.f;
        fc.add(knn_row_chunked<KNN_ORDERED>(xs, L, lo + i, lo, hi, E, tau, K, sc, u, d));
        const size_t o = (static_cast<size_t>(series) * n + i) * K;
        if (lane < K) {
            idx[o + lane] = u;
            if (dist) dist[o + lane] = d;
        }
    }
    fc.flush(stats);
}

// ---------------------------------------- materialised distances (baseline)
//
// The paper's two-kernel kNN (Algorithm 1 writes the n x n distance matrix
// to memory, Algorithm 2 selects each row's k nearest from it), kept as a
// measured baseline for the fused kernels above.  dmat_kernel writes the FP32
// squared distances D[i][j] = s(lo+i, lo+j) of one series with the
// operations of dist32 in the same order; knn_from_dmat_kernel runs one warp
// per row through knn_row_chunked reading D instead of computing it, with the
// same FP64 band step, so the output equals edm_knn's.
constexpr int DM_TILE = 64;  // rows and columns of a dmat_kernel tile

__global__ void __launch_bounds__(256)
    dmat_kernel(const float *__restrict__ x, int lo, int n, int E, int tau,
                float *__restrict__ D) {
    // rows i0..i0+63 and columns j0..j0+63 need x[lo + i - l tau] for l < E
    extern __shared__ __align__(16) float seg[];  // [2][64 + (E-1) tau]
    const int span = DM_TILE + (E - 1) * tau;
    float *ra = seg, *ca = seg + span;
    const int i0 = blockIdx.y * DM_TILE, j0 = blockIdx.x * DM_TILE;
    // ra[k] = x[lo + i0 - (E-1) tau + k], likewise for the columns
    for (int k = threadIdx.x; k < span; k += blockDim.x) {
        const int ti = lo + i0 - (E - 1) * tau + k, tj = lo + j0 - (E - 1) * tau + k;
        ra[k] = (ti >= 0 && ti < lo + n) ? x[ti] : 0.f;
        ca[k] = (tj >= 0 && tj < lo + n) ? x[tj] : 0.f;
    }
    __syncthreads();
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 columns x 4 row groups
    const int off = (E - 1) * tau;
    float acc[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc[r] = 0.f;
    for (int l = 0; l < E; ++l) {
        const float b = ca[off + tx - l * tau];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const float d = __fsub_rn(ra[off + ty + 4 * r - l * tau], b);
            acc[r] = __fmaf_rn(d, d, acc[r]);
        }
    }
    const int j = j0 + tx;
    if (j >= n) return;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int i = i0 + ty + 4 * r;
        if (i < n) D[static_cast<size_t>(i) * n + j] = acc[r];
    }
}

template <bool SMEM>
__global__ void __launch_bounds__(KNN_WARPS * 32)
    knn_from_dmat_kernel(const float *__restrict__ x, const float *__restrict__ D, int L, int E,
                         int tau, int Tp, int K, int RB, int32_t *__restrict__ idx,
                         float *__restrict__ dist) {
    extern __shared__ __align__(16) uint8_t smem[];
    TableLongScratch *sca = reinterpret_cast<TableLongScratch *>(smem);
    float *xs_s = reinterpret_cast<float *>(smem + KNN_WARPS * sizeof(TableLongScratch));
    const float *xs = stage_series<SMEM>(x, L, xs_s);
    const int lo = (E - 1) * tau, hi = L - 1 - Tp, n = hi - lo + 1;
    const int r0 = blockIdx.x * RB, r1 = min(n, r0 + RB);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    TableLongScratch *sc = sca + warp;
    for (int i = r0 + warp; i < r1; i += KNN_WARPS) {
        int u = 0;
        float d = 0.f;
        knn_row_chunked<KNN_ORDERED>(xs, L, lo + i, lo, hi, E, tau, K, sc, u, d,
                                     D + static_cast<size_t>(i) * n);
        if (lane < K) {
            idx[static_cast<size_t>(i) * K + lane] = u;
            if (dist) dist[static_cast<size_t>(i) * K + lane] = d;
        }
    }
}

edm_status launch_knn_materialized(edm_ctx *ctx, const float *X, int N, int L, int E, int tau,
                                   int Tp, int k, int32_t *idx, float *dist) {
    const int lo = (E - 1) * tau, n = L - lo - Tp;
    edm_status st = ws_reserve(ctx, sizeof(float) * static_cast<size_t>(n) * n);
    if (st != EDM_OK) return st;
    float *D = static_cast<float *>(ctx->ws);
    const int tiles = (n + DM_TILE - 1) / DM_TILE;
    const size_t seg = 2 * sizeof(float) * (DM_TILE + (E - 1) * tau);
    const int RB = rows_per_cta(ctx, 1, n);
    const bool smem_series = sizeof(float) * static_cast<size_t>(L) <= SERIES_SMEM_MAX;
    const size_t smem = KNN_WARPS * sizeof(TableLongScratch) +
                        (smem_series ? align_up(sizeof(float) * L, 16) : 0);
    auto sel = smem_series ? knn_from_dmat_kernel<true> : knn_from_dmat_kernel<false>;
    cudaFuncSetAttribute(sel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(dmat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)seg);
    // one series at a time: its matrix is the workspace
    for (int sidx = 0; sidx < N; ++sidx) {
        const float *x = X + static_cast<size_t>(sidx) * L;
        before_launch(ctx);
        dmat_kernel<<<dim3(tiles, tiles), 256, seg, ctx->stream>>>(x, lo, n, E, tau, D);
        st = after_launch(ctx, "dmat_kernel");
        if (st != EDM_OK) return st;
        before_launch(ctx);
        sel<<<(n + RB - 1) / RB, KNN_WARPS * 32, smem, ctx->stream>>>(
            x, D, L, E, tau, Tp, k, RB, idx + static_cast<size_t>(sidx) * n * k,
            dist ? dist + static_cast<size_t>(sidx) * n * k : nullptr);
        st = after_launch(ctx, "knn_from_dmat_kernel");
        if (st != EDM_OK) return st;
    }
    return EDM_OK;
}

size_t ccm_slot_bytes(int L, int tau, int Tp) {
    size_t best = 0;
    for (int E = 1; E <= EDM_E_MAX; ++E) {
        const int n = L - (E - 1) * tau - Tp;
        if (n < 1) break;
        best = std::max(best, static_cast<size_t>((n + 1) / 2) * table_pair_bytes(E + 1));
    }
    return align_up(best, 256);
}

edm_status launch_ccm_tables(edm_ctx *ctx, const float *X, long long ld, int nlib, int L,
                             int tau, int Tp, const CcmGroups &g, uint8_t *tables) {
    const int n_max = L - Tp;  // rows at E = 1, the most of any E
    const int RB = rows_per_cta(ctx, nlib, n_max);
    dim3 grid(g.ngroups_max * g.G, (n_max + RB - 1) / RB);
    const int ch = (L + 31) / 32;
    if (ch <= 64) {
        const int CHs[] = {8, 16, 24, 32, 48, 64};
        int CH = 64;
        for (int c : CHs)
            if (c >= ch) { CH = c; break; }
        const bool head1 = (EDM_E_MAX - 1) * tau < 32;
        void (*kern)(const float *, long long, int, int, int, int, const CcmGroups, uint8_t *,
                     unsigned long long *) = nullptr;
        switch (CH) {
        case 8: kern = head1 ? ccm_table_regs_kernel<8, true> : ccm_table_regs_kernel<8, false>; break;
        case 16: kern = head1 ? ccm_table_regs_kernel<16, true> : ccm_table_regs_kernel<16, false>; break;
        case 24: kern = head1 ? ccm_table_regs_kernel<24, true> : ccm_table_regs_kernel<24, false>; break;
        case 32: kern = head1 ? ccm_table_regs_kernel<32, true> : ccm_table_regs_kernel<32, false>; break;
        case 48: kern = head1 ? ccm_table_regs_kernel<48, true> : ccm_table_regs_kernel<48, false>; break;
        default: kern = head1 ? ccm_table_regs_kernel<64, true> : ccm_table_regs_kernel<64, false>; break;
        }
        const size_t smem = KNN_WARPS * sizeof(WarpScratch) + sizeof(float) * 32 * CH;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        before_launch(ctx);
        kern<<<grid, KNN_WARPS * 32, smem, ctx->stream>>>(X, ld, L, tau, Tp, RB, g, tables,
                                                          diag_stats(ctx));
        return after_launch(ctx, "ccm_table_kernel");
    }
    // longer series: chunks of 1,024 candidates against a running list
    const bool smem_series = sizeof(float) * static_cast<size_t>(L) <= SERIES_SMEM_MAX;
    const size_t smem = KNN_WARPS * sizeof(TableLongScratch) +
                        (smem_series ? align_up(sizeof(float) * L, 16) : 0);
    auto kern = smem_series ? ccm_table_long_kernel<true> : ccm_table_long_kernel<false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    before_launch(ctx);
    kern<<<grid, KNN_WARPS * 32, smem, ctx->stream>>>(X, ld, L, tau, Tp, RB, g, tables,
                                                      diag_stats(ctx));
    return after_launch(ctx, "ccm_table_kernel");
}

// ------------------------------------------------------ grouping by E

size_t groups_bytes(int nlib, int G) {
    const size_t ng = static_cast<size_t>(groups_max(nlib, G));
    return 3 * align_up(4 * ng, 256) + align_up(8 * ng, 256) + align_up(4 * ng * G, 256) + 256;
}

CcmGroups carve_groups(uint8_t *mem, int nlib, int G) {
    const size_t ng = static_cast<size_t>(groups_max(nlib, G));
    CcmGroups g;
    g.G = G;
    g.ngroups_max = static_cast<int>(ng);
    g.off = reinterpret_cast<long long *>(mem);
    mem += align_up(8 * ng, 256);
    g.E = reinterpret_cast<int32_t *>(mem);
    mem += align_up(4 * ng, 256);
    g.n = reinterpret_cast<int32_t *>(mem);
    mem += align_up(4 * ng, 256);
    g.lib = reinterpret_cast<int32_t *>(mem);
    mem += align_up(4 * ng * G, 256);
    g.count = reinterpret_cast<int32_t *>(mem);
    return g;
}

constexpr int GROUP_THREADS = 1024;

// One CTA: histogram of E (bucket 0 for an invalid E), then groups of G per
// bucket in bucket order with the byte offsets of their tables, then every
// library placed in a slot of its bucket's groups.
__global__ void __launch_bounds__(GROUP_THREADS)
    group_libs_kernel(const int32_t *__restrict__ E_lib, int E_uniform, int lib0, int nlib, int L,
                      int tau, int Tp, const CcmGroups g) {
    __shared__ int cnt[EDM_E_MAX + 1], fill[EDM_E_MAX + 1], gbase[EDM_E_MAX + 2];
    __shared__ long long obase[EDM_E_MAX + 1], gbytes[EDM_E_MAX + 1];
    const int tid = threadIdx.x, G = g.G;
    if (tid <= EDM_E_MAX) {
        cnt[tid] = 0;
        fill[tid] = 0;
    }
    for (int s = tid; s < g.ngroups_max * G; s += GROUP_THREADS) g.lib[s] = -1;
    __syncthreads();
    for (int i = tid; i < nlib; i += GROUP_THREADS) {
        const int E = E_uniform > 0 ? E_uniform : E_lib[lib0 + i];
        atomicAdd(&cnt[ccm_E_valid(E, L, tau, Tp) ? E : 0], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int ng = 0;
        long long off = 0;
        for (int b = 0; b <= EDM_E_MAX; ++b) {
            const int groups = (cnt[b] + G - 1) / G;
            const long long npairs = b ? (L - (b - 1) * tau - Tp + 1) / 2 : 0;
            gbase[b] = ng;
            obase[b] = off;
            gbytes[b] = npairs * G * table_pair_bytes(b + 1);
            ng += groups;
            off += groups * gbytes[b];
        }
        gbase[EDM_E_MAX + 1] = ng;
        *g.count = ng;
    }
    __syncthreads();
    const int ng = gbase[EDM_E_MAX + 1];
    for (int gi = tid; gi < ng; gi += GROUP_THREADS) {
        int b = 0;
        while (gbase[b + 1] <= gi) ++b;  // gbase is nondecreasing; gi < gbase[E_MAX+1]
        const int j = gi - gbase[b];
        g.E[gi] = b;
        g.n[gi] = min(G, cnt[b] - j * G);
        g.off[gi] = obase[b] + j * gbytes[b];
    }
    for (int i = tid; i < nlib; i += GROUP_THREADS) {
        const int E = E_uniform > 0 ? E_uniform : E_lib[lib0 + i];
        const int b = ccm_E_valid(E, L, tau, Tp) ? E : 0;
        const int pos = atomicAdd(&fill[b], 1);
        g.lib[(gbase[b] + pos / G) * G + pos % G] = lib0 + i;
    }
    __syncthreads();
    // the empty slots of a partial group repeat its first member: their
    // tables are built and gathered like the others (the lookup then needs no
    // per-member test) and their results are never written
    for (int gi = tid; gi < ng; gi += GROUP_THREADS) {
        int b = 0;
        while (gbase[b + 1] <= gi) ++b;
        const int nm = min(G, cnt[b] - (gi - gbase[b]) * G);
        for (int m = nm; m < G; ++m) g.lib[gi * G + m] = g.lib[gi * G];
    }
}

edm_status launch_group_libs(edm_ctx *ctx, const int32_t *E_lib, int E_uniform, int lib0,
                             int nlib, int L, int tau, int Tp, const CcmGroups &g) {
    before_launch(ctx);
    group_libs_kernel<<<1, GROUP_THREADS, 0, ctx->stream>>>(E_lib, E_uniform, lib0, nlib, L, tau,
                                                            Tp, g);
    return after_launch(ctx, "group_libs_kernel");
}

}  // namespace edm
