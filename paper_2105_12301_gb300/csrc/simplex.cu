// simplex.cu -- optimal embedding dimension by simplex projection.
//
// kEDM section 3.3 groups targets by their "optimal embedding dimension"
// without saying how it is found; the method used here is leave-one-out
// simplex projection of each series onto itself (section 2.1 steps 1-4 with
// Y = X and horizon Tp_sel), E = 1..E_max, E* = argmax rho_E.
//
// One CTA owns one series (staged in shared memory) and a block of query
// times; one warp per query time keeps the FP32 squared distances to every
// candidate, adds one lag per E, and selects the exact FP64 neighbour set of
// every E from them, then forms the weighted prediction.  Prediction and
// observation are centred on the series mean before their moments are
// accumulated (FP32 per warp, FP64 across warps and CTAs); rho is finished in
// FP64 by a second kernel.
#include <mutex>

#include "knn_core.cuh"

namespace edm {

constexpr int SX_WARPS = 8;
constexpr int SX_SERIES_SMEM_MAX = 96 * 1024;

// ---------------------------------------------------------------------------
// Incremental sweep over E (series of up to 32*CH points).  The selection from
// registers (select_set_regs) is shared with the neighbour-table builder.
//
// A warp owns one query time t and keeps the FP32 squared distance from x(t)
// to every candidate u = lane + 32 j in registers (slot j), so that
// neighbouring times -- often neighbours of t together on a smooth series --
// sit in different lanes and the lane minima below make a tight bound.
// Going from E-1 to E adds one lag: s = fma(d, d, s) with d = X[t-(E-1)tau]
// - X[u-(E-1)tau], which is exactly the operation sequence of the direct sum
// over l = 0..E-1, so the values are bit-identical to those of knn_row.
// Candidates below the first point of P_E, past its last point, or equal to
// t hold +inf.  Each E then selects from the registers: lane minimum, the
// (K+1)-th smallest of the 32 minima as a bound, compaction of every value at
// or below it through 4-slot cells, exact ranking of the few collected keys,
// and the FP64 band check of knn_row's KNN_SET mode.  The neighbour set of
// every E is written to the warp's list; after the last E, lane E-1 forms the
// simplex prediction of E from it (section 2.1 step 4) and accumulates its
// moments, so the per-E work holds no warp-wide reduction.

constexpr int SX_NB = 232;  // per-warp neighbour lists: sum over E = 1..20 of (E+1) = 230
static_assert(EDM_E_MAX <= 20, "the neighbour lists hold E = 1..20");

// First entry of the list of E (K = E+1 entries each).
__device__ __forceinline__ int nb_off(int E) { return (E - 1) * (E + 2) / 2; }

// Simplex prediction of x(t+Tp) from the K neighbours of one E held in a
// list (distance d_r, time u_r as float bits; entry 0 the nearest):
// sum_r w_r y_r / sum_r w_r with w_r = exp(-d_r/d_1) (or the d_1 = 0 limit)
// and y_r = x[u_r+Tp] - mu (section 2.1 steps 3-4), accumulated with the
// observation into the moments m (sums of a, b, a^2, b^2, ab).
__device__ __forceinline__ void predict_into_moments(const float2 *nb, int K, const float *xs,
                                                     int t, int Tp, float mu, float (&m)[5]) {
    const float d1 = nb[0].x;
    float w_sum = 0.f, wy_sum = 0.f;
    for (int r = 0; r < K; ++r) {
        const float2 e = nb[r];
        float w;
        if (d1 > 0.f)
            w = expf(-(e.x / d1));
        else
            w = (e.x == 0.f) ? 1.f : 0.f;
        w_sum += w;
        wy_sum = __fmaf_rn(w, __fsub_rn(xs[__float_as_int(e.y) + Tp], mu), wy_sum);
    }
    const float a = wy_sum / w_sum;
    const float b = __fsub_rn(xs[t + Tp], mu);
    m[0] += a;
    m[1] += b;
    m[2] = __fmaf_rn(a, a, m[2]);
    m[3] = __fmaf_rn(b, b, m[3]);
    m[4] = __fmaf_rn(a, b, m[4]);
}

template <int CH, bool HEAD1>
__device__ __forceinline__ void sweep_row(const float *xs, int t, int hi, int E_max, int tau,
                                          int Tp, float mu, WarpScratch *ws, float2 *nb,
                                          float (&m)[5], unsigned keep, FallbackCount &fc) {
    static_assert(CH % 4 == 0, "4-slot cells");
    const int lane = lane_id();
    float s[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
        const int u = lane + 32 * j;
        s[j] = (u <= hi && u != t) ? 0.f : EDM_INF;
    }
    int E_row = 0;
    for (int E = 1; E <= E_max; ++E) {
        const int lo = (E - 1) * tau;
        if (t < lo || hi - lo + 1 < E + 2) break;
        const int K = E + 1;
        // extend every distance by the lag E-1; candidates below lo leave P_E
        // (HEAD1: lo < 32, so only slot 0 can hold them)
        const float qv = xs[t - lo];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int u = lane + 32 * j;
            if (!HEAD1 || j == 0) {
                const float d = __fsub_rn(qv, xs[max(u - lo, 0)]);
                const float v = __fmaf_rn(d, d, s[j]);
                s[j] = (u < lo) ? EDM_INF : v;
            } else {
                const float d = __fsub_rn(qv, xs[u - lo]);
                s[j] = __fmaf_rn(d, d, s[j]);
            }
        }
        int u_out = 0;
        float d_out = 0.f;
        fc.add(select_set_regs<CH>(s, xs, t, lo, hi, E, tau, K, ws, u_out, d_out, keep));
        if (lane < K) nb[nb_off(E) + lane] = make_float2(d_out, __int_as_float(u_out));
        E_row = E;
    }
    __syncwarp();
    // lane E-1: prediction and moments of E
    if (lane < E_row) predict_into_moments(nb + nb_off(lane + 1), lane + 2, xs, t, Tp, mu, m);
    __syncwarp();
}

// Dynamic shared memory of sweep_block: per-warp scratch and neighbour
// lists, the moment reduction buffer, the series mean partials, and the
// series (32*CH points, zero past its end) behind 32 points of padding.
inline size_t sweep_smem_bytes(int CH) {
    return SX_WARPS * sizeof(WarpScratch) + SX_WARPS * 32 * 5 * sizeof(float) +
           SX_WARPS * sizeof(double) + SX_WARPS * SX_NB * sizeof(float2) +
           sizeof(float) * (32 + 32 * static_cast<size_t>(CH));
}

// One CTA-sized block of work: series `series` (staged in shared memory,
// zero-padded to 32*CH points) and its query times rb*TB .. rb*TB+TB-1;
// warps take query times t = warp, warp + SX_WARPS, ...  Writes the block's
// FP64 partial moments and ends with a barrier, so the shared memory can be
// reused for the next block.
template <int CH, bool HEAD1>
__device__ __forceinline__ void sweep_block(uint8_t *smem, const float *__restrict__ X, int L,
                                            int E_max, int tau, int Tp, int TB, int nrb,
                                            int series, int rb, double *__restrict__ partial,
                                            unsigned long long *stats) {
    WarpScratch *wsa = reinterpret_cast<WarpScratch *>(smem);
    float *red = reinterpret_cast<float *>(smem + SX_WARPS * sizeof(WarpScratch));
    double *mu_s = reinterpret_cast<double *>(red + SX_WARPS * 32 * 5);
    float2 *nba = reinterpret_cast<float2 *>(mu_s + SX_WARPS);
    float *xs = reinterpret_cast<float *>(nba + SX_WARPS * SX_NB) + 32;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const float *xg = X + static_cast<size_t>(series) * L;
    double acc = 0.0;
    for (int i = threadIdx.x; i < L; i += blockDim.x) acc += static_cast<double>(xg[i]);
    acc = warp_sum_d(acc);
    if (lane == 0) mu_s[warp] = acc;
    for (int i = static_cast<int>(threadIdx.x) - 32; i < 32 * CH; i += blockDim.x)
        xs[i] = (i >= 0 && i < L) ? xg[i] : 0.f;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < SX_WARPS; ++w) tot += mu_s[w];
    const float mu = static_cast<float>(tot / L);
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    WarpScratch *ws = wsa + warp;
    float2 *nb = nba + warp * SX_NB;
    const int hi = L - 1 - Tp;
    const int t1 = min(hi + 1, (rb + 1) * TB);
    const unsigned keep = bitonic_keep_min_bits();
    FallbackCount fc;
    for (int t = rb * TB + warp; t < t1; t += SX_WARPS)
        sweep_row<CH, HEAD1>(xs, t, hi, E_max, tau, Tp, mu, ws, nb, m, keep, fc);
    fc.flush(stats);
#pragma unroll
    for (int j = 0; j < 5; ++j) red[(warp * 32 + lane) * 5 + j] = m[j];
    __syncthreads();
    for (int i = threadIdx.x; i < E_max * 5; i += blockDim.x) {
        const int e = i / 5, j = i % 5;
        double sum = 0.0;
        for (int w = 0; w < SX_WARPS; ++w) sum += static_cast<double>(red[(w * 32 + e) * 5 + j]);
        partial[((static_cast<size_t>(series) * nrb + rb) * E_max + e) * 5 + j] = sum;
    }
    __syncthreads();
}

// Two CTAs per SM up to 48 slots (the register file allows 128 registers a
// thread); the 64-slot sweep needs more than 200 and runs one CTA per SM.
constexpr int sweep_min_blocks(int CH) { return CH <= 48 ? 2 : 1; }

// One CTA per (series, block of query times).
template <int CH, bool HEAD1>
__global__ void __launch_bounds__(SX_WARPS * 32, sweep_min_blocks(CH))
    sweep_kernel(const float *__restrict__ X, int L, int E_max, int tau, int Tp, int TB, int nrb,
                 double *__restrict__ partial, unsigned long long *stats) {
    extern __shared__ __align__(16) uint8_t smem[];
    sweep_block<CH, HEAD1>(smem, X, L, E_max, tau, Tp, TB, nrb, blockIdx.x, blockIdx.y, partial,
                           stats);
}

// ---------------------------------------------------------------------------
// Incremental sweep for long series (more than 2,048 points).
//
// The candidates of a query time are visited in chunks of 1,024 (32 slots per
// lane in registers); within a chunk every E extends the distances by one lag
// exactly as in sweep_row.  Each E keeps, in the warp's shared memory, the
// running list of its R = E+2 smallest FP32 keys over the chunks seen so far,
// sorted.  A chunk only needs the values at or below the list's last key (or,
// while the list is not yet full, below the R-th smallest lane minimum of the
// chunk); those are compacted, merged with the list and ranked.  After the
// last chunk every E has its exact FP32 top-R, and the band check of
// knn_row's KNN_SET mode decides whether the FP64 ranking must be consulted.
// Each E's list then takes its K neighbours, and lane E-1 forms the
// prediction of E from them, as in sweep_row.

constexpr int LS_CH = 32;          // candidate slots per lane per chunk
constexpr int LS_LIST = 256;       // sum over E = 1..20 of (E+2) = 250 keys

__device__ __forceinline__ int ls_list_off(int E) { return (E - 1) * (E + 4) / 2; }

// FP32 squared distance with E a run-time value: the same operations in the
// same order as dist32<E>.
__device__ __forceinline__ float dist32_rt(const float *xs, int t, int u, int E, int tau) {
    float s = 0.f;
    for (int l = 0; l < E; ++l) {
        const float d = __fsub_rn(xs[t - l * tau], xs[u - l * tau]);
        s = __fmaf_rn(d, d, s);
    }
    return s;
}

struct LongScratch {
    WarpScratch ws;
    uint64_t list[LS_LIST];   // per E: its R smallest keys so far, ascending
};

// One chunk of 32*LS_CH candidates u = c0 + lane + 32 j for every E of the
// row.  In an interior chunk every candidate is a point of every P_E
// (c0 >= (E_row-1)tau and the chunk ends at or before hi), so the lagged
// reads need no clamp and no candidate leaves the set; only that update
// loop differs (a warp-uniform branch), the selection code is shared.
__device__ __forceinline__ void long_chunk(const float *xs, int L, int t, int hi, int E_row,
                                           int tau, int c0, bool interior, LongScratch *sc,
                                           int &cnt, int &degen) {
    const int lane = lane_id();
    WarpScratch *ws = &sc->ws;
    float s[LS_CH];
#pragma unroll
    for (int j = 0; j < LS_CH; ++j) {
        const int u = c0 + lane + 32 * j;
        s[j] = u <= hi && u != t ? 0.f : EDM_INF;
    }
    for (int E = 1; E <= E_row; ++E) {
        const int lo = (E - 1) * tau;
        const float qv = xs[t - lo];
        if (interior) {
            const float *xl = xs + (c0 + lane - lo);
#pragma unroll
            for (int j = 0; j < LS_CH; ++j) {
                const float d = __fsub_rn(qv, xl[32 * j]);
                s[j] = __fmaf_rn(d, d, s[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < LS_CH; ++j) {
                const int u = c0 + lane + 32 * j;
                const float d = __fsub_rn(qv, xs[min(max(u - lo, 0), L - 1)]);
                const float v = __fmaf_rn(d, d, s[j]);
                s[j] = (u < lo) ? EDM_INF : v;
            }
        }
        const int R = min(E + 2, hi - lo);
        uint64_t *list = sc->list + ls_list_off(E);
        const int have = __shfl_sync(FULL, cnt, E - 1);
        if (__shfl_sync(FULL, degen, E - 1)) continue;
        float gm[LS_CH / 4];
        group_minima<LS_CH>(s, gm);
        float bound = have == R ? key_s(list[R - 1]) : EDM_INF;
        if (have < R) {
            float lmin = EDM_INF;
#pragma unroll
            for (int g = 0; g < LS_CH / 4; ++g) lmin = fminf(lmin, gm[g]);
            bound = fminf(bound, warp_sorted_at_f(lmin, min(R, 32) - 1));
        }
        int c = bound == EDM_INF ? compact_le<LS_CH>(s, bound, ws, c0)
                                 : compact_le_groups<LS_CH>(s, gm, bound, ws, c0);
        if (c > KNN_CAP - 32) {
            // a loose bound (large E, first chunks): shrink it while the
            // chunk's values under it plus the list's still number >= R
            auto in_list = [&](float b) {
                const bool p = lane < have && key_s(list[lane]) <= b;
                return __popc(__ballot_sync(FULL, p));
            };
            const float b = shrink_bound<LS_CH>(s, bound, c, R, KNN_CAP - 32, in_list);
            if (b >= 0.f) c = compact_le_groups<LS_CH>(s, gm, b, ws, c0);
        }
        if (c > KNN_CAP - 32) {
            // more values tie at the bound than the buffer holds (long runs
            // of repeated values): this E is resolved in FP64 after the chunks
            if (lane == E - 1) degen = 1;
            continue;
        }
        if (c == 0) continue;
        // merge the collected keys with the list and keep the R smallest
        for (int e = lane; e < have; e += 32) ws->key[c + e] = list[e];
        __syncwarp();
        const int tot = c + have;
        rank_keys(ws, tot, min(R, tot));
        const int keep = min(R, tot);
        for (int e = lane; e < keep; e += 32) list[e] = ws->sel[e];
        __syncwarp();
        if (lane == E - 1) cnt = keep;
    }
}

__device__ void sweep_long_row(const float *xs, int L, int t, int hi, int E_max, int tau, int Tp,
                               float mu, LongScratch *sc, float (&m)[5], FallbackCount &fc) {
    const int lane = lane_id();
    WarpScratch *ws = &sc->ws;
    // last E for which t is a point of P_E with enough points
    int E_row = 0;
    for (int E = 1; E <= E_max; ++E) {
        const int lo = (E - 1) * tau;
        if (t < lo || hi - lo + 1 < E + 2) break;
        E_row = E;
    }
    int cnt = 0;    // lane e: keys held in the list of E = e+1
    int degen = 0;  // lane e: E = e+1 has too many ties for the list
    const int lo_max = (E_row - 1) * tau;
    for (int c0 = 0; c0 <= hi; c0 += 32 * LS_CH)
        long_chunk(xs, L, t, hi, E_row, tau, c0, c0 >= lo_max && c0 + 32 * LS_CH - 1 <= hi, sc,
                   cnt, degen);
    // every E now holds its exact FP32 top-R: band check, weights, moments
    for (int E = 1; E <= E_row; ++E) {
        const int lo = (E - 1) * tau, K = E + 1;
        const int R = min(E + 2, hi - lo);
        const uint64_t *list = sc->list + ls_list_off(E);
        int u_out = 0;
        float d_out = 0.f;
        const bool deg = __shfl_sync(FULL, degen, E - 1) != 0;
        const float edge = deg ? 0.f : band_edge(key_s(list[K - 1]), E);
        if (deg) {
            fc.add(KNN_USED_BAND | KNN_USED_BRUTE);
            brute_fp64(xs, t, lo, hi, E, tau, ws, K);
            if (lane < K) {
                u_out = ws->sel_u[lane];
                d_out = __double2float_rn(__dsqrt_rn(ws->sel_s64[lane]));
            }
        } else if (R <= K || key_s(list[K]) > edge) {
            if (lane < K) {
                u_out = key_u(list[lane]);
                d_out = sqrtf(key_s(list[lane]));
            }
        } else {
            if (lane == 0) ws->count = 0;
            __syncwarp();
            for (int u = lo + lane; u <= hi; u += 32) {
                if (u == t) continue;
                const float v = dist32_rt(xs, t, u, E, tau);
                if (v <= edge) {
                    const int pos = atomicAdd(&ws->count, 1);
                    if (pos < KNN_CAP) ws->key[pos] = mk_key(v, u);
                }
            }
            __syncwarp();
            const int c = ws->count;
            __syncwarp();
            fc.add(c <= KNN_CAP ? KNN_USED_BAND : KNN_USED_BAND | KNN_USED_BRUTE);
            if (c <= KNN_CAP)
                rank_band_fp64(xs, t, E, tau, ws, c, K);
            else
                brute_fp64(xs, t, lo, hi, E, tau, ws, K);
            if (lane < K) {
                u_out = ws->sel_u[lane];
                d_out = __double2float_rn(__dsqrt_rn(ws->sel_s64[lane]));
            }
        }
        __syncwarp();
        // the list of E is no longer needed: it now holds E's neighbours
        if (lane < K)
            reinterpret_cast<float2 *>(sc->list + ls_list_off(E))[lane] =
                make_float2(d_out, __int_as_float(u_out));
        __syncwarp();
    }
    // lane E-1: prediction and moments of E, as in sweep_row
    if (lane < E_row)
        predict_into_moments(reinterpret_cast<const float2 *>(sc->list + ls_list_off(lane + 1)),
                             lane + 2, xs, t, Tp, mu, m);
    __syncwarp();
}

template <bool SMEM>
__device__ __forceinline__ void sweep_long_block(uint8_t *smem, const float *__restrict__ X, int L,
                                                 int E_max, int tau, int Tp, int TB, int nrb,
                                                 int series, int rb, double *__restrict__ partial,
                                                 unsigned long long *stats) {
    LongScratch *sca = reinterpret_cast<LongScratch *>(smem);
    float *red = reinterpret_cast<float *>(smem + SX_WARPS * sizeof(LongScratch));
    double *mu_s = reinterpret_cast<double *>(red + SX_WARPS * 32 * 5);
    float *xs_s = reinterpret_cast<float *>(mu_s + SX_WARPS);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const float *xg = X + static_cast<size_t>(series) * L;
    double acc = 0.0;
    for (int i = threadIdx.x; i < L; i += blockDim.x) acc += static_cast<double>(xg[i]);
    acc = warp_sum_d(acc);
    if (lane == 0) mu_s[warp] = acc;
    const float *xs = xg;
    if (SMEM) {
        for (int i = threadIdx.x; i < L; i += blockDim.x) xs_s[i] = xg[i];
        xs = xs_s;
    }
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < SX_WARPS; ++w) tot += mu_s[w];
    const float mu = static_cast<float>(tot / L);
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int hi = L - 1 - Tp;
    const int t1 = min(hi + 1, (rb + 1) * TB);
    FallbackCount fc;
    for (int t = rb * TB + warp; t < t1; t += SX_WARPS)
        sweep_long_row(xs, L, t, hi, E_max, tau, Tp, mu, sca + warp, m, fc);
    fc.flush(stats);
#pragma unroll
    for (int j = 0; j < 5; ++j) red[(warp * 32 + lane) * 5 + j] = m[j];
    __syncthreads();
    for (int i = threadIdx.x; i < E_max * 5; i += blockDim.x) {
        const int e = i / 5, j = i % 5;
        double sum = 0.0;
        for (int w = 0; w < SX_WARPS; ++w) sum += static_cast<double>(red[(w * 32 + e) * 5 + j]);
        partial[((static_cast<size_t>(series) * nrb + rb) * E_max + e) * 5 + j] = sum;
    }
    __syncthreads();
}

template <bool SMEM>
__global__ void __launch_bounds__(SX_WARPS * 32, 2)
    sweep_long_kernel(const float *__restrict__ X, int L, int E_max, int tau, int Tp, int TB,
                      int nrb, double *__restrict__ partial, unsigned long long *stats) {
    extern __shared__ __align__(16) uint8_t smem[];
    sweep_long_block<SMEM>(smem, X, L, E_max, tau, Tp, TB, nrb, blockIdx.x, blockIdx.y, partial,
                           stats);
}

// ---------------------------------------------------------------------------
// Batched optimal E as a work queue (many uneven problems in one launch per
// kind of sweep).  A job is one problem; its work items are its (series,
// block of TB query times) pairs, numbered from item0 in the queue of its
// kind.  The launch is persistent: a grid sized to the resident CTAs takes
// items from one device counter until the queue is empty, so problems of
// every size share the GPU without a launch (and a tail) per problem.  Jobs
// are queued largest first.

struct SweepJob {
    const float *X;       // [N][L]
    double *partial;      // [N][nrb][E_max][5]
    int32_t *E_opt;       // [N]
    long long item0;      // first item of this job in its queue
    int N, L, tau, TB, nrb;
};

// The job of queue item g: the last job whose item0 <= g (jobs ascending).
__device__ __forceinline__ int job_of(const SweepJob *jobs, int njobs, long long g) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].item0 <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int CH, bool HEAD1>
__global__ void __launch_bounds__(SX_WARPS * 32, sweep_min_blocks(CH))
    sweep_queue_kernel(const SweepJob *__restrict__ jobs, int njobs, long long nitems,
                       unsigned long long *counter, int E_max, int Tp,
                       unsigned long long *stats) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ long long item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = static_cast<long long>(atomicAdd(counter, 1ull));
        __syncthreads();
        const long long g = item_s;
        __syncthreads();
        if (g >= nitems) break;
        const SweepJob J = jobs[job_of(jobs, njobs, g)];
        const long long local = g - J.item0;
        sweep_block<CH, HEAD1>(smem, J.X, J.L, E_max, J.tau, Tp, J.TB, J.nrb,
                               static_cast<int>(local / J.nrb), static_cast<int>(local % J.nrb),
                               J.partial, stats);
    }
}

__global__ void __launch_bounds__(SX_WARPS * 32, 2)
    sweep_long_queue_kernel(const SweepJob *__restrict__ jobs, int njobs, long long nitems,
                            unsigned long long *counter, int E_max, int Tp,
                            unsigned long long *stats) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ long long item_s;
    for (;;) {
        if (threadIdx.x == 0) item_s = static_cast<long long>(atomicAdd(counter, 1ull));
        __syncthreads();
        const long long g = item_s;
        __syncthreads();
        if (g >= nitems) break;
        const SweepJob J = jobs[job_of(jobs, njobs, g)];
        const long long local = g - J.item0;
        sweep_long_block<true>(smem, J.X, J.L, E_max, J.tau, Tp, J.TB, J.nrb,
                               static_cast<int>(local / J.nrb), static_cast<int>(local % J.nrb),
                               J.partial, stats);
    }
}

// Sum the partials of one series, rho per E, argmax.
__device__ __forceinline__ void finish_series(const double *__restrict__ partial, int series, int L,
                                              int E_max, int tau, int Tp, int nrb,
                                              int32_t *__restrict__ E_opt,
                                              float *__restrict__ rho_E) {
    int best_E = 1;
    double best = 0.0;
    bool have = false;
    for (int E = 1; E <= E_max; ++E) {
        const int n = L - (E - 1) * tau - Tp;
        double r = __longlong_as_double(0x7ff8000000000000LL);
        if (n >= E + 2) {
            double S[5] = {0, 0, 0, 0, 0};
            for (int rb = 0; rb < nrb; ++rb)
                for (int j = 0; j < 5; ++j)
                    S[j] += partial[((static_cast<size_t>(series) * nrb + rb) * E_max + (E - 1)) * 5 + j];
            r = pearson_from_moments(static_cast<double>(n), S[0], S[1], S[2], S[3], S[4]);
        }
        if (rho_E) rho_E[static_cast<size_t>(series) * E_max + (E - 1)] = static_cast<float>(r);
        if (!isnan(r) && (!have || r > best)) {
            best = r;
            best_E = E;
            have = true;
        }
    }
    E_opt[series] = best_E;
}

// One thread per series.
__global__ void simplex_finish_kernel(const double *__restrict__ partial, int N, int L, int E_max,
                                      int tau, int Tp, int nrb, int32_t *__restrict__ E_opt,
                                      float *__restrict__ rho_E) {
    const int series = blockIdx.x * blockDim.x + threadIdx.x;
    if (series >= N) return;
    finish_series(partial, series, L, E_max, tau, Tp, nrb, E_opt, rho_E);
}

// One thread per series of every job of a batched run: jobs[i] covers the
// global series series0[i] .. series0[i] + N - 1 (series0 ascending).
__global__ void simplex_finish_jobs_kernel(const SweepJob *__restrict__ jobs,
                                           const long long *__restrict__ series0, int njobs,
                                           long long total, int E_max, int Tp) {
    const long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (series0[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    const SweepJob J = jobs[lo];
    finish_series(J.partial, static_cast<int>(g - series0[lo]), J.L, E_max, J.tau, Tp, J.nrb,
                  J.E_opt, nullptr);
}

static void simplex_geometry(edm_ctx *ctx, int N, int L, int &TB, int &nrb) {
    const long long want_ctas = 8LL * ctx->num_sms;
    long long per_series = (want_ctas + N - 1) / N;
    TB = static_cast<int>((L + per_series - 1) / per_series);
    TB = std::max(TB, 4 * SX_WARPS);
    TB = std::min(TB, L);
    nrb = (L + TB - 1) / TB;
}

size_t simplex_workspace_bytes(edm_ctx *ctx, int N, int L, int E_max) {
    int TB, nrb;
    simplex_geometry(ctx, N, L, TB, nrb);
    return sizeof(double) * static_cast<size_t>(N) * nrb * E_max * 5;
}

edm_status launch_simplex(edm_ctx *ctx, const float *X, int N, int L, int E_max, int tau,
                          int Tp_sel, int32_t *E_opt, float *rho_E) {
    int TB, nrb;
    simplex_geometry(ctx, N, L, TB, nrb);
    edm_status st = ws_reserve(ctx, simplex_workspace_bytes(ctx, N, L, E_max));
    if (st != EDM_OK) return st;
    double *partial = static_cast<double *>(ctx->ws);
    dim3 grid(N, nrb);
    const int ch = (L + 31) / 32;
    if (ch <= 64) {
        // incremental sweep with register-resident distances
        const int CHs[] = {8, 16, 24, 32, 48, 64};
        int CH = 64;
        for (int c : CHs)
            if (c >= ch) { CH = c; break; }
        const size_t smem = sweep_smem_bytes(CH);
        void (*kern)(const float *, int, int, int, int, int, int, double *, unsigned long long *) = nullptr;
        const bool head1 = (E_max - 1) * tau < 32;
        switch (CH) {
        case 8: kern = head1 ? sweep_kernel<8, true> : sweep_kernel<8, false>; break;
        case 16: kern = head1 ? sweep_kernel<16, true> : sweep_kernel<16, false>; break;
        case 24: kern = head1 ? sweep_kernel<24, true> : sweep_kernel<24, false>; break;
        case 32: kern = head1 ? sweep_kernel<32, true> : sweep_kernel<32, false>; break;
        case 48: kern = head1 ? sweep_kernel<48, true> : sweep_kernel<48, false>; break;
        default: kern = head1 ? sweep_kernel<64, true> : sweep_kernel<64, false>; break;
        }
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        before_launch(ctx);
        kern<<<grid, SX_WARPS * 32, smem, ctx->stream>>>(X, L, E_max, tau, Tp_sel, TB, nrb, partial,
                                                          diag_stats(ctx));
        st = after_launch(ctx, "sweep_kernel");
        if (st != EDM_OK) return st;
    } else {
        // long series: chunked incremental sweep
        const size_t lfixed = SX_WARPS * sizeof(LongScratch) + SX_WARPS * 32 * 5 * sizeof(float) +
                              SX_WARPS * sizeof(double);
        const bool smem_series = sizeof(float) * static_cast<size_t>(L) <= SX_SERIES_SMEM_MAX;
        const size_t smem = lfixed + (smem_series ? align_up(sizeof(float) * L, 16) : 0);
        auto kern = smem_series ? sweep_long_kernel<true> : sweep_long_kernel<false>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        before_launch(ctx);
        kern<<<grid, SX_WARPS * 32, smem, ctx->stream>>>(X, L, E_max, tau, Tp_sel, TB, nrb, partial,
                                                          diag_stats(ctx));
        st = after_launch(ctx, "sweep_long_kernel");
        if (st != EDM_OK) return st;
    }
    before_launch(ctx);
    simplex_finish_kernel<<<(N + 127) / 128, 128, 0, ctx->stream>>>(partial, N, L, E_max, tau,
                                                                      Tp_sel, nrb, E_opt, rho_E);
    return after_launch(ctx, "simplex_finish_kernel");
}

// ---------------------------------------------------------------------------
// Batched optimal E through the work queues.
//
// Kinds of sweep: the register-resident sweep for each slot count CH (8, 16,
// 24, 32, 48, 64; HEAD1 when every lag offset is below 32) and the chunked
// sweep for series longer than 2,048 points.  Each kind with jobs gets one
// persistent launch; then one kernel finishes every series of every job.

constexpr int SQ_KINDS = 13;   // 6 slot counts x HEAD1 or not, + the long sweep
constexpr int SQ_LONG = 12;
constexpr int SQ_CH[6] = {8, 16, 24, 32, 48, 64};

static int sweep_kind(int L, int E_max, int tau) {
    const int ch = (L + 31) / 32;
    if (ch > 64) return SQ_LONG;
    int c = 5;
    for (int i = 0; i < 6; ++i)
        if (SQ_CH[i] >= ch) { c = i; break; }
    return 2 * c + ((E_max - 1) * tau < 32 ? 1 : 0);
}

using QueueKernel = void (*)(const SweepJob *, int, long long, unsigned long long *, int, int,
                             unsigned long long *);

static QueueKernel queue_kernel(int kind) {
    switch (kind) {
    case 0: return sweep_queue_kernel<8, false>;
    case 1: return sweep_queue_kernel<8, true>;
    case 2: return sweep_queue_kernel<16, false>;
    case 3: return sweep_queue_kernel<16, true>;
    case 4: return sweep_queue_kernel<24, false>;
    case 5: return sweep_queue_kernel<24, true>;
    case 6: return sweep_queue_kernel<32, false>;
    case 7: return sweep_queue_kernel<32, true>;
    case 8: return sweep_queue_kernel<48, false>;
    case 9: return sweep_queue_kernel<48, true>;
    case 10: return sweep_queue_kernel<64, false>;
    case 11: return sweep_queue_kernel<64, true>;
    default: return sweep_long_queue_kernel;
    }
}

static size_t queue_smem(int kind, int L_max) {
    const size_t red = SX_WARPS * 32 * 5 * sizeof(float) + SX_WARPS * sizeof(double);
    if (kind == SQ_LONG) return SX_WARPS * sizeof(LongScratch) + red + align_up(sizeof(float) * L_max, 16);
    return sweep_smem_bytes(SQ_CH[kind / 2]);
}

// Rows per work item of a kind: the tuned value if any, else 256.
static int queue_rows(edm_ctx *ctx, int kind) {
    if (ctx->tune) {
        auto it = ctx->tune->find(0x5157000000000000ull | static_cast<uint64_t>(kind));
        if (it != ctx->tune->end()) return it->second;
    }
    return 256;
}

struct SweepQueuePlan {
    int njobs = 0;
    std::vector<int> kinds;                  // kinds with jobs
    int job0[SQ_KINDS] = {}, njob[SQ_KINDS] = {};
    long long items[SQ_KINDS] = {};
    int L_max[SQ_KINDS] = {};
    long long series_total = 0;
    SweepJob *d_jobs = nullptr;
    long long *d_series0 = nullptr;
    unsigned long long *d_counters = nullptr;
    size_t bytes = 0;                        // workspace used
};

// Lay the batch out in the context's workspace: the job descriptors (grouped
// by kind, each kind's jobs largest first), their series offsets, one queue
// counter per kind, then the partial moments of every job.  rows[kind] is the
// query times per work item.  Copies the descriptors to the device (and
// synchronises the stream): call before any capture.
static edm_status plan_sweep_queue(edm_ctx *ctx, const edm_instance *inst, int n, int E_max,
                                   int32_t *const *E_out, const int *rows, SweepQueuePlan &P) {
    std::vector<int> order[SQ_KINDS];
    for (int i = 0; i < n; ++i) order[sweep_kind(inst[i].L, E_max, inst[i].tau)].push_back(i);
    std::vector<SweepJob> jobs;
    std::vector<long long> series0;
    size_t partial_doubles = 0;
    P = SweepQueuePlan();
    for (int k = 0; k < SQ_KINDS; ++k) {
        auto &o = order[k];
        if (o.empty()) continue;
        std::stable_sort(o.begin(), o.end(), [&](int a, int b) {
            return static_cast<double>(inst[a].N) * inst[a].L * inst[a].L >
                   static_cast<double>(inst[b].N) * inst[b].L * inst[b].L;
        });
        P.kinds.push_back(k);
        P.job0[k] = static_cast<int>(jobs.size());
        P.njob[k] = static_cast<int>(o.size());
        long long item = 0;
        for (int i : o) {
            const edm_instance &p = inst[i];
            SweepJob J;
            J.X = p.X;
            J.N = p.N;
            J.L = p.L;
            J.tau = p.tau;
            J.TB = std::min(std::max(rows[k], SX_WARPS), p.L);
            J.nrb = (p.L + J.TB - 1) / J.TB;
            J.E_opt = E_out[i];
            J.item0 = item;
            J.partial = reinterpret_cast<double *>(partial_doubles);  // offset for now
            partial_doubles += static_cast<size_t>(p.N) * J.nrb * E_max * 5;
            item += static_cast<long long>(p.N) * J.nrb;
            P.L_max[k] = std::max(P.L_max[k], p.L);
            jobs.push_back(J);
            series0.push_back(P.series_total);
            P.series_total += p.N;
        }
        P.items[k] = item;
    }
    P.njobs = static_cast<int>(jobs.size());
    const size_t jb = align_up(sizeof(SweepJob) * jobs.size(), 256);
    const size_t sb = align_up(sizeof(long long) * series0.size(), 256);
    const size_t cb = align_up(sizeof(unsigned long long) * SQ_KINDS, 256);
    P.bytes = jb + sb + cb + sizeof(double) * partial_doubles;
    edm_status st = ws_reserve(ctx, P.bytes);
    if (st != EDM_OK) return st;
    uint8_t *base = static_cast<uint8_t *>(ctx->ws);
    P.d_jobs = reinterpret_cast<SweepJob *>(base);
    P.d_series0 = reinterpret_cast<long long *>(base + jb);
    P.d_counters = reinterpret_cast<unsigned long long *>(base + jb + sb);
    double *partial = reinterpret_cast<double *>(base + jb + sb + cb);
    for (auto &J : jobs) J.partial = partial + reinterpret_cast<size_t>(J.partial);
    st = cuda_check(ctx, cudaMemcpyAsync(P.d_jobs, jobs.data(), sizeof(SweepJob) * jobs.size(),
                                         cudaMemcpyHostToDevice, ctx->stream), "queue jobs");
    if (st == EDM_OK)
        st = cuda_check(ctx, cudaMemcpyAsync(P.d_series0, series0.data(),
                                             sizeof(long long) * series0.size(),
                                             cudaMemcpyHostToDevice, ctx->stream), "queue jobs");
    // the host vectors must outlive the copies
    if (st == EDM_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "queue jobs");
    return st;
}

// Enqueue the planned batch on `stream`: reset the counters, one persistent
// launch per kind (times in ms per kind when `ms` is given, which
// synchronises), then the finish of every series.
static edm_status enqueue_sweep_queue(edm_ctx *ctx, const SweepQueuePlan &P, int E_max, int Tp_sel,
                                      cudaStream_t stream, float *ms) {
    edm_status st = cuda_check(ctx, cudaMemsetAsync(P.d_counters, 0,
                                                    sizeof(unsigned long long) * SQ_KINDS, stream),
                               "queue counters");
    if (st != EDM_OK) return st;
    for (int k : P.kinds) {
        QueueKernel kern = queue_kernel(k);
        const size_t smem = queue_smem(k, P.L_max[k]);
        st = cuda_check(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  static_cast<int>(smem)), "queue attribute");
        if (st != EDM_OK) return st;
        int per_sm = 0;
        st = cuda_check(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                                           SX_WARPS * 32, smem),
                        "queue occupancy");
        if (st != EDM_OK) return st;
        const long long want = static_cast<long long>(std::max(per_sm, 1)) * ctx->num_sms;
        const int grid = static_cast<int>(std::min<long long>(want, P.items[k]));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (ms) {
            st = cuda_check(ctx, cudaEventCreate(&e0), "queue timing");
            if (st == EDM_OK) st = cuda_check(ctx, cudaEventCreate(&e1), "queue timing");
            if (st == EDM_OK) st = cuda_check(ctx, cudaEventRecord(e0, stream), "queue timing");
            if (st != EDM_OK) return st;
        }
        before_launch(ctx);
        kern<<<grid, SX_WARPS * 32, smem, stream>>>(P.d_jobs + P.job0[k], P.njob[k], P.items[k],
                                                    P.d_counters + k, E_max, Tp_sel,
                                                    diag_stats(ctx));
        st = after_launch(ctx, k == SQ_LONG ? "sweep_long_queue_kernel" : "sweep_queue_kernel");
        if (ms) {
            edm_status t = cuda_check(ctx, cudaEventRecord(e1, stream), "queue timing");
            if (t == EDM_OK) t = cuda_check(ctx, cudaEventSynchronize(e1), "queue timing");
            if (t == EDM_OK) t = cuda_check(ctx, cudaEventElapsedTime(&ms[k], e0, e1), "queue timing");
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (st == EDM_OK) st = t;
        }
        if (st != EDM_OK) return st;
    }
    before_launch(ctx);
    simplex_finish_jobs_kernel<<<static_cast<unsigned>((P.series_total + 127) / 128), 128, 0,
                                 stream>>>(P.d_jobs, P.d_series0, P.njobs, P.series_total, E_max,
                                           Tp_sel);
    return after_launch(ctx, "simplex_finish_kernel");
}

// Autotuner of the queues (before any capture: it times launches): for every
// kind of this batch not tuned yet, run the batch with 128, 256 and 512
// query times per work item and keep, per kind, the fastest.
static edm_status tune_sweep_queue(edm_ctx *ctx, const edm_instance *inst, int n, int E_max,
                                   int Tp_sel, int32_t *const *E_out) {
    bool need = false;
    for (int i = 0; i < n; ++i) {
        const uint64_t key = 0x5157000000000000ull |
                             static_cast<uint64_t>(sweep_kind(inst[i].L, E_max, inst[i].tau));
        if (!ctx->tune->count(key)) need = true;
    }
    if (!need) return EDM_OK;
    const int cands[3] = {128, 256, 512};
    float best_ms[SQ_KINDS];
    int best_rows[SQ_KINDS];
    for (int k = 0; k < SQ_KINDS; ++k) {
        best_ms[k] = 0.f;
        best_rows[k] = 0;
    }
    for (int c : cands) {
        int rows[SQ_KINDS];
        for (int k = 0; k < SQ_KINDS; ++k) rows[k] = c;
        SweepQueuePlan P;
        edm_status st = plan_sweep_queue(ctx, inst, n, E_max, E_out, rows, P);
        if (st != EDM_OK) return st;
        float ms[SQ_KINDS] = {};
        st = enqueue_sweep_queue(ctx, P, E_max, Tp_sel, ctx->stream, ms);
        if (st != EDM_OK) return st;
        for (int k : P.kinds)
            if (best_rows[k] == 0 || ms[k] < best_ms[k]) {
                best_ms[k] = ms[k];
                best_rows[k] = c;
            }
    }
    for (int k = 0; k < SQ_KINDS; ++k)
        if (best_rows[k]) (*ctx->tune)[0x5157000000000000ull | static_cast<uint64_t>(k)] = best_rows[k];
    return EDM_OK;
}

edm_status launch_simplex_queue(edm_ctx *ctx, const edm_instance *inst, int n, int E_max,
                                int Tp_sel, int32_t *const *E_out, bool tune, bool capture) {
    if (tune && ctx->autotune) {
        edm_status st = tune_sweep_queue(ctx, inst, n, E_max, Tp_sel, E_out);
        if (st != EDM_OK) return st;
    }
    int rows[SQ_KINDS];
    for (int k = 0; k < SQ_KINDS; ++k) rows[k] = queue_rows(ctx, k);
    SweepQueuePlan P;
    edm_status st = plan_sweep_queue(ctx, inst, n, E_max, E_out, rows, P);
    if (st != EDM_OK) return st;
    if (!capture) return enqueue_sweep_queue(ctx, P, E_max, Tp_sel, ctx->stream, nullptr);
    // one graph of the whole batch, replayed while the batch and the tuned
    // values stay the same
    uint64_t key = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t b) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < b; ++i) key = (key ^ c[i]) * 1099511628211ull;
    };
    mix("sweepq", 6);
    mix(&E_max, sizeof(E_max));
    mix(&Tp_sel, sizeof(Tp_sel));
    mix(rows, sizeof(rows));
    for (int i = 0; i < n; ++i) {
        mix(&inst[i], sizeof(inst[i]));
        mix(&E_out[i], sizeof(E_out[i]));
    }
    mix(&P.d_jobs, sizeof(P.d_jobs));
    if (!ctx->qgraph_exec || ctx->qgraph_key != key) {
        if (ctx->qgraph_exec) cudaGraphExecDestroy(ctx->qgraph_exec);
        ctx->qgraph_exec = nullptr;
        if (!ctx->origin &&
            cudaStreamCreateWithFlags(&ctx->origin, cudaStreamNonBlocking) != cudaSuccess)
            return set_error(ctx, EDM_ERR_CUDA, "batch stream creation failed");
        if (cudaStreamBeginCapture(ctx->origin, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return set_error(ctx, EDM_ERR_CUDA, "graph capture could not begin");
        const uint64_t before = ctx->launches;
        st = enqueue_sweep_queue(ctx, P, E_max, Tp_sel, ctx->origin, nullptr);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(ctx->origin, &graph);
        if (st != EDM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ce != cudaSuccess || !graph) return cuda_check(ctx, ce, "graph capture");
        const cudaError_t ie = cudaGraphInstantiate(&ctx->qgraph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_check(ctx, ie, "graph instantiation");
        ctx->qgraph_key = key;
        ctx->qgraph_kernels = ctx->launches - before;
        ctx->launches = before;
    }
    if (!ctx->ev_fork)
        st = cuda_check(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming),
                        "batch event");
    if (st == EDM_OK && !ctx->ev_done)
        st = cuda_check(ctx, cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming),
                        "batch event");
    if (st == EDM_OK) st = cuda_check(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream), "batch order");
    if (st == EDM_OK)
        st = cuda_check(ctx, cudaStreamWaitEvent(ctx->origin, ctx->ev_fork, 0), "batch order");
    if (st == EDM_OK)
        st = cuda_check(ctx, cudaGraphLaunch(ctx->qgraph_exec, ctx->origin), "graph launch");
    if (st == EDM_OK) st = cuda_check(ctx, cudaEventRecord(ctx->ev_done, ctx->origin), "batch order");
    if (st == EDM_OK)
        st = cuda_check(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_done, 0), "batch order");
    if (st != EDM_OK) return st;
    ctx->launches += ctx->qgraph_kernels;
    return EDM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of edm_simplex_optimal_E (no counterpart in the
// paper).  Its only scratch memory -- the per-CTA partial moments that the
// sweep kernels write and the finishing kernel reads -- lives in the
// file-scope array below instead of a context workspace.  Every GPU that
// loads the library holds this array until the process exits.

constexpr size_t NOALLOC_SCRATCH_DOUBLES = size_t(1) << 19;  // 4 MiB
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

// Device address of g_noalloc_scratch on each device, looked up once per
// device (with that device current) on the first call there.
constexpr int NOALLOC_MAX_DEVICES = 64;
static double *g_noalloc_ptr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

static cudaError_t noalloc_scratch(int device, double **ptr) {
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = static_cast<double *>(p);
    }
    *ptr = g_noalloc_ptr[device];
    return cudaSuccess;
}

}  // namespace edm

extern "C" edm_status edm_simplex_optimal_E_noalloc(const float *X, int N, int L, int E_max,
                                                    int tau, int Tp_sel, int32_t *E_opt,
                                                    float *rho_E, void *cuda_stream) {
    using namespace edm;
    if (!X || !E_opt || N < 1 || L < 2 || L > EDM_L_MAX || E_max < 1 || E_max > EDM_E_MAX ||
        tau < 1 || Tp_sel < 0 || L - Tp_sel < 3)
        return EDM_ERR_INVALID_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int device = 0, num_sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return EDM_ERR_CUDA;
    // query times per CTA: the same split as the context path, widened until
    // the partial moments fit the static scratch
    const long long want_ctas = 8LL * num_sms;
    const long long per_series = (want_ctas + N - 1) / N;
    int TB = static_cast<int>((L + per_series - 1) / per_series);
    TB = std::min(std::max(TB, 4 * SX_WARPS), L);
    int nrb = (L + TB - 1) / TB;
    const size_t per_block = static_cast<size_t>(E_max) * 5;
    if (static_cast<size_t>(N) * nrb * per_block > NOALLOC_SCRATCH_DOUBLES) {
        // fewer, longer row blocks (never needed on a 152-SM GPU: there the
        // split above always fits whenever N * E_max is within capacity)
        TB = L;
        nrb = 1;
    }
    if (static_cast<size_t>(N) * nrb * per_block > NOALLOC_SCRATCH_DOUBLES)
        return EDM_ERR_INVALID_ARG;  // N * E_max above the scratch capacity
    double *partial = nullptr;
    if (noalloc_scratch(device, &partial) != cudaSuccess) return EDM_ERR_CUDA;
    // an error left pending by some earlier call is not this call's to report
    // or to clear
    if (cudaPeekAtLastError() != cudaSuccess) return EDM_ERR_CUDA;

    dim3 grid(N, nrb);
    const int ch = (L + 31) / 32;
    if (ch <= 64) {
        const int CHs[] = {8, 16, 24, 32, 48, 64};
        int CH = 64;
        for (int c : CHs)
            if (c >= ch) { CH = c; break; }
        const size_t smem = sweep_smem_bytes(CH);
        const bool head1 = (E_max - 1) * tau < 32;
        void (*kern)(const float *, int, int, int, int, int, int, double *, unsigned long long *) = nullptr;
        switch (CH) {
        case 8: kern = head1 ? sweep_kernel<8, true> : sweep_kernel<8, false>; break;
        case 16: kern = head1 ? sweep_kernel<16, true> : sweep_kernel<16, false>; break;
        case 24: kern = head1 ? sweep_kernel<24, true> : sweep_kernel<24, false>; break;
        case 32: kern = head1 ? sweep_kernel<32, true> : sweep_kernel<32, false>; break;
        case 48: kern = head1 ? sweep_kernel<48, true> : sweep_kernel<48, false>; break;
        default: kern = head1 ? sweep_kernel<64, true> : sweep_kernel<64, false>; break;
        }
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return EDM_ERR_CUDA;
        kern<<<grid, SX_WARPS * 32, smem, stream>>>(X, L, E_max, tau, Tp_sel, TB, nrb, partial,
                                                     nullptr);
    } else {
        // long series: the chunked incremental sweep of the context path
        const size_t lfixed = SX_WARPS * sizeof(LongScratch) + SX_WARPS * 32 * 5 * sizeof(float) +
                              SX_WARPS * sizeof(double);
        const bool smem_series = sizeof(float) * static_cast<size_t>(L) <= SX_SERIES_SMEM_MAX;
        const size_t smem = lfixed + (smem_series ? align_up(sizeof(float) * L, 16) : 0);
        auto kern = smem_series ? sweep_long_kernel<true> : sweep_long_kernel<false>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return EDM_ERR_CUDA;
        kern<<<grid, SX_WARPS * 32, smem, stream>>>(X, L, E_max, tau, Tp_sel, TB, nrb, partial,
                                                     nullptr);
    }
    // no error was pending before the launch, so one now is this call's
    if (cudaGetLastError() != cudaSuccess) return EDM_ERR_CUDA;
    simplex_finish_kernel<<<(N + 127) / 128, 128, 0, stream>>>(partial, N, L, E_max, tau, Tp_sel,
                                                                nrb, E_opt, rho_E);
    if (cudaGetLastError() != cudaSuccess) return EDM_ERR_CUDA;
    return EDM_OK;
}
