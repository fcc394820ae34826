// knn_core.cuh -- one warp finds the k nearest neighbours of one query point.
//
// kEDM section 2.1 step 2 and Algorithms 1-2: exhaustive distances from the
// query x(t) to every other library point (the embedding is never
// materialised: lagged values are read straight from the series), then the
// k smallest.  Instead of Algorithm 2's per-thread priority queues in shared
// memory, a warp
//   1. takes the minimum key (s, u) of each lane's candidates; the R-th
//      smallest of those 32 minima bounds the R-th smallest key of the row;
//   2. collects every key at or below that bound into a small per-warp
//      buffer (typically R..2R entries) and ranks them;
//   3. makes the FP32 ranking exact against an FP64 evaluation of the same
//      definition: every candidate whose FP64 key can belong to the k
//      nearest has an FP32 squared distance within the band
//      s32 <= s32_(k) (1 + 4 (E+3) 2^-24) + 3 * 2^-140
//      (|s32 - s| <= (E+2) u s for u = 2^-24 plus an absolute term for
//      subnormal squares, and the same for FP64 with u = 2^-53).  If the
//      collected candidates cover that band, ranking them by the FP64 key
//      (s64, u) gives exactly the FP64 neighbour set and order; otherwise
//      the band is collected and ranked in FP64, and in a degenerate row
//      (more than CAP candidates in the band) k FP64 arg-min sweeps are run.
// The FP64 squared distance uses the same operations in the same order as
// the definition: d = (double)a - (double)b, s = fma(d, d, s), l = 0..E-1.
#pragma once

#include "edm_internal.cuh"

namespace edm {

constexpr int KNN_CAP = 128;     // per-warp candidate buffer
constexpr int KNN_MARGIN = 8;    // extra FP32 candidates re-ranked in FP64
constexpr int KNN_CELLS = 64;    // per-warp buffer of 4-slot cells (select_set_regs)

// The cell buffer shares memory with the FP64 band buffers: cells are turned
// into keys before any band is resolved.
struct alignas(16) WarpScratch {
    uint64_t key[KNN_CAP];   // collected FP32 keys
    union {
        double s64[KNN_CAP];        // FP64 squared distances of the keys (band fallback)
        float4 cell_v[KNN_CELLS];   // the four values of a collected cell
    };
    uint64_t sel[32];        // the R smallest collected keys, ascending
    union {
        double sel_s64[32];         // exact ranking: FP64 distances by final rank
        int cell_u[KNN_CELLS];      // time index of the first value of a cell
    };
    int sel_u[32];
    int count;
    int pad;
};

enum KnnMode { KNN_SET = 0, KNN_ORDERED = 1 };

// Flags returned by knn_row (for statistics only).
enum { KNN_USED_BAND = 1, KNN_USED_BRUTE = 2 };

__device__ __forceinline__ uint64_t mk_key(float s, int u) {
    return (static_cast<uint64_t>(__float_as_uint(s)) << 32) | static_cast<uint32_t>(u);
}
__device__ __forceinline__ float key_s(uint64_t k) {
    return __uint_as_float(static_cast<uint32_t>(k >> 32));
}
__device__ __forceinline__ int key_u(uint64_t k) { return static_cast<int>(static_cast<uint32_t>(k)); }

// FP32 squared distance between query (held in q) and the point at time u,
// lag order 0..E-1, one fma per lag.
template <int E>
__device__ __forceinline__ float dist32(const float (&q)[E], const float *xs, int u, int tau) {
    float s = 0.f;
#pragma unroll
    for (int l = 0; l < E; ++l) {
        float d = __fsub_rn(q[l], xs[u - l * tau]);
        s = __fmaf_rn(d, d, s);
    }
    return s;
}

// FP64 squared distance, same operation sequence as the definition.
__device__ __forceinline__ double dist64(const float *xs, int t, int u, int E, int tau) {
    double s = 0.0;
    for (int l = 0; l < E; ++l) {
        double d = __dsub_rn(static_cast<double>(xs[t - l * tau]),
                             static_cast<double>(xs[u - l * tau]));
        s = __fma_rn(d, d, s);
    }
    return s;
}

// Upper edge of the band of FP32 squared distances that may hide an FP64
// neighbour, given the k-th smallest FP32 squared distance sK:
// sK (1 + 4 (E+3) 2^-24) + 3 * 2^-140, evaluated with upward rounding so the
// float result is never below the exact value.  4 (E+3) 2^-24 = (E+3) 2^-22
// is exact in float.
__device__ __forceinline__ float band_edge(float sK, int E) {
    const float factor = 1.0f + static_cast<float>(E + 3) * 0x1p-22f;
    return __fadd_ru(__fmul_ru(sK, factor), 3.0f * 0x1p-140f);
}

__device__ __forceinline__ bool less64(double sa, int ua, double sb, int ub) {
    return sa < sb || (sa == sb && ua < ub);
}

// Collect into ws->key every candidate key <= theta (at most KNN_CAP kept);
// returns how many there are in total.
template <int E>
__device__ __forceinline__ int filter_keys(const float (&q)[E], const float *xs, int t, int lo,
                                           int hi, int tau, uint64_t theta, WarpScratch *ws) {
    const int lane = lane_id();
    if (lane == 0) ws->count = 0;
    __syncwarp();
    for (int u = lo + lane; u <= hi; u += WARP) {
        if (u == t) continue;
        uint64_t key = mk_key(dist32<E>(q, xs, u, tau), u);
        if (key <= theta) {
            int pos = atomicAdd(&ws->count, 1);
            if (pos < KNN_CAP) ws->key[pos] = key;
        }
    }
    __syncwarp();
    int c = ws->count;
    __syncwarp();
    return c;
}

// Rank the c (<= KNN_CAP) keys of ws->key; write the R smallest, ascending,
// to ws->sel.  The buffer is padded to a multiple of four with keys above
// every real key (a real key's high word is a finite float), and read two
// keys per 16-byte load.
__device__ __forceinline__ void rank_keys(WarpScratch *ws, int c, int R) {
    const int lane = lane_id();
    const int c4 = (c + 3) & ~3;  // <= KNN_CAP, a multiple of four
    if (lane < c4 - c) ws->key[c + lane] = ~0ull;
    __syncwarp();
    const ulonglong2 *k2 = reinterpret_cast<const ulonglong2 *>(ws->key);
    // every lane runs every pass (no divergent loop); a lane past the last
    // key ranks a copy of key c4-1 and stores nothing
    for (int e0 = 0; e0 < c; e0 += WARP) {
        const int e = e0 + lane;
        const uint64_t ke = ws->key[min(e, c4 - 1)];
        int rank = 0;
        for (int e2 = 0; e2 < c4 / 2; e2 += 2) {
            const ulonglong2 a = k2[e2], b = k2[e2 + 1];
            rank += (a.x < ke) + (a.y < ke) + (b.x < ke) + (b.y < ke);
        }
        if (e < c && rank < R) ws->sel[rank] = ke;
    }
    __syncwarp();
}

// The key of rank r among the first c keys of ws->key (all lanes).
__device__ __forceinline__ uint64_t key_at_rank(WarpScratch *ws, int c, int r) {
    const int lane = lane_id();
    for (int e = lane; e < c; e += WARP) {
        uint64_t ke = ws->key[e];
        int rank = 0;
        for (int e2 = 0; e2 < c; ++e2) rank += ws->key[e2] < ke;
        if (rank == r) ws->sel[0] = ke;
    }
    __syncwarp();
    uint64_t v = ws->sel[0];
    __syncwarp();
    return v;
}

// Exact ranking of the c band candidates collected in ws->key by their FP64
// key; the K smallest go to ws->sel_u / ws->sel_s64 in order.
__device__ __forceinline__ void rank_band_fp64(const float *xs, int t, int E, int tau,
                                               WarpScratch *ws, int c, int K) {
    const int lane = lane_id();
    for (int e = lane; e < c; e += WARP) ws->s64[e] = dist64(xs, t, key_u(ws->key[e]), E, tau);
    __syncwarp();
    for (int e = lane; e < c; e += WARP) {
        double se = ws->s64[e];
        int ue = key_u(ws->key[e]);
        int rank = 0;
        for (int e2 = 0; e2 < c; ++e2) rank += less64(ws->s64[e2], key_u(ws->key[e2]), se, ue);
        if (rank < K) {
            ws->sel_s64[rank] = se;
            ws->sel_u[rank] = ue;
        }
    }
    __syncwarp();
}

// Degenerate rows: K sweeps, each taking the smallest FP64 key above the
// previous one.  O(K n E) FP64 work; only reached when more than KNN_CAP
// candidates fall in the band (long runs of repeated values).
static __device__ __noinline__ void brute_fp64(const float *xs, int t, int lo, int hi, int E, int tau,
                                        WarpScratch *ws, int K) {
    const int lane = lane_id();
    double last_s = -1.0;
    int last_u = -1;
    for (int r = 0; r < K; ++r) {
        double best_s = __longlong_as_double(0x7ff0000000000000LL);
        int best_u = 0x7fffffff;
        for (int u = lo + lane; u <= hi; u += WARP) {
            if (u == t) continue;
            double s = dist64(xs, t, u, E, tau);
            if (less64(last_s, last_u, s, u) && less64(s, u, best_s, best_u)) {
                best_s = s;
                best_u = u;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double os = __shfl_xor_sync(FULL, best_s, o);
            int ou = __shfl_xor_sync(FULL, best_u, o);
            if (less64(os, ou, best_s, best_u)) {
                best_s = os;
                best_u = ou;
            }
        }
        if (lane == 0) {
            ws->sel_s64[r] = best_s;
            ws->sel_u[r] = best_u;
        }
        last_s = best_s;
        last_u = best_u;
    }
    __syncwarp();
}

// The K nearest neighbours of the point at time t among the times lo..hi
// (t excluded).  Requires 1 <= K <= hi-lo and K + KNN_MARGIN <= 32 in
// KNN_ORDERED mode, K + 1 <= 32 in KNN_SET mode.  All lanes of the warp call
// it; on return lane r < K holds the r-th neighbour:
//   KNN_ORDERED: exact FP64 order (s64, u); d = (float)sqrt(s64).
//   KNN_SET:     the exact FP64 neighbour set; order and d from FP32 (the
//                exact FP64 values when the band had to be resolved).
// Returns KNN_USED_* flags.
template <int E, int MODE>
__device__ int knn_row(const float *xs, int t, int lo, int hi, int tau, int K, WarpScratch *ws,
                       int *out_u, float *out_d) {
    const int lane = lane_id();
    float q[E];
#pragma unroll
    for (int l = 0; l < E; ++l) q[l] = xs[t - l * tau];

    const int nc = hi - lo;  // number of candidates (the point itself excluded)
    const int R = (MODE == KNN_ORDERED) ? min(K + KNN_MARGIN, nc) : min(K + 1, nc);

    // 1. per-lane minimum key, then the R-th smallest of the 32 minima
    uint64_t kmin = ~0ull;
    for (int u = lo + lane; u <= hi; u += WARP) {
        if (u == t) continue;
        uint64_t key = mk_key(dist32<E>(q, xs, u, tau), u);
        kmin = key < kmin ? key : kmin;
    }
    uint64_t theta = warp_sorted_at(kmin, R - 1);

    // 2. collect keys <= theta; shrink theta while the buffer overflows
    int c = filter_keys<E>(q, xs, t, lo, hi, tau, theta, ws);
    while (c > KNN_CAP) {
        theta = key_at_rank(ws, KNN_CAP, R - 1);
        c = filter_keys<E>(q, xs, t, lo, hi, tau, theta, ws);
    }
    rank_keys(ws, c, R);  // ws->sel[0..R) ascending FP32 keys

    const float sK = key_s(ws->sel[K - 1]);
    const float edge = band_edge(sK, E);
    const bool all_taken = (R == nc);

    if (MODE == KNN_SET) {
        // exact set when the (K+1)-th FP32 key lies beyond the band
        if (R <= K || key_s(ws->sel[K]) > edge) {
            if (lane < K) {
                uint64_t k = ws->sel[lane];
                *out_u = key_u(k);
                *out_d = sqrtf(key_s(k));
            }
            __syncwarp();
            return 0;
        }
    } else {
        // FP64 re-rank of the R collected keys; valid when they cover the band
        if (all_taken || key_s(ws->sel[R - 1]) > edge) {
            double s64 = __longlong_as_double(0x7ff0000000000000LL);
            int u = 0x7fffffff;
            if (lane < R) {
                u = key_u(ws->sel[lane]);
                s64 = dist64(xs, t, u, E, tau);
            }
            int rank = 0;
            for (int j = 0; j < R; ++j) {
                double sj = __shfl_sync(FULL, s64, j);
                int uj = __shfl_sync(FULL, u, j);
                rank += less64(sj, uj, s64, u);
            }
            if (lane < R && rank < K) {
                ws->sel_s64[rank] = s64;
                ws->sel_u[rank] = u;
            }
            __syncwarp();
            if (lane < K) {
                *out_u = ws->sel_u[lane];
                *out_d = __double2float_rn(__dsqrt_rn(ws->sel_s64[lane]));
            }
            __syncwarp();
            return 0;
        }
    }

    // 3. band fallback: every candidate with s32 <= edge, ranked in FP64
    int flags = KNN_USED_BAND;
    c = filter_keys<E>(q, xs, t, lo, hi, tau, mk_key(edge, 0x7fffffff), ws);
    if (c <= KNN_CAP) {
        rank_band_fp64(xs, t, E, tau, ws, c, K);
    } else {
        brute_fp64(xs, t, lo, hi, E, tau, ws, K);
        flags |= KNN_USED_BRUTE;
    }
    if (lane < K) {
        *out_u = ws->sel_u[lane];
        *out_d = __double2float_rn(__dsqrt_rn(ws->sel_s64[lane]));
    }
    __syncwarp();
    return flags;
}

// ------------------------------------------ selection from register arrays
//
// A warp holds the FP32 squared distances of a query row in a register array
// s[CH] per lane: slot j of lane l is the candidate u0 + l + 32 j.  A 4-slot
// group g of lane l is a "cell": its first candidate is u0 + l + 128 g and
// value i of it is that plus 32 i.

#define EDM_INF __int_as_float(0x7f800000)

// Bit i of the result is set when this lane keeps the smaller value at
// compare-exchange stage i of the ascending 32-lane bitonic network (stages
// in the order of warp_sorted_at_f).  A per-lane constant: computed once.
__device__ __forceinline__ unsigned bitonic_keep_min_bits() {
    const int lane = lane_id();
    unsigned bits = 0;
    int st = 0;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1, ++st)
            if (((lane & k) == 0) == ((lane & j) == 0)) bits |= 1u << st;
    return bits;
}

// Ascending bitonic sort of one float per lane; value at position r.  keep
// is bitonic_keep_min_bits() of this lane.
__device__ __forceinline__ float warp_sorted_at_f(float v, int r, unsigned keep) {
    int st = 0;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1, ++st) {
            const float o = __shfl_xor_sync(FULL, v, j);
            v = (keep >> st) & 1u ? fminf(v, o) : fmaxf(v, o);
        }
    }
    return __shfl_sync(FULL, v, r);
}
__device__ __forceinline__ float warp_sorted_at_f(float v, int r) {
    return warp_sorted_at_f(v, r, bitonic_keep_min_bits());
}

// Compact the keys (s[j], u0+lane+32j) with s[j] <= bound (and finite, i.e. a
// candidate of P_E) into ws->key; returns
// how many there are (only the first KNN_CAP are stored).
template <int CH>
__device__ __forceinline__ int compact_le(const float (&s)[CH], float bound, WarpScratch *ws,
                                          int u0 = 0) {
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    int base = 0;
#pragma unroll
    for (int j = 0; j < CH; ++j) {
        const bool p = s[j] <= bound && s[j] != EDM_INF;
        const unsigned b = __ballot_sync(FULL, p);
        const int pos = base + __popc(b & lt);
        if (p && pos < KNN_CAP) ws->key[pos] = mk_key(s[j], u0 + lane + 32 * j);
        base += __popc(b);
    }
    __syncwarp();
    return base;
}


// Compact the keys (s[j], u0+lane+32j) with s[j] <= bound, a FINITE bound,
// into ws->key, visiting only the slot groups (4 slots each, minima in gm)
// in which some lane holds such a value; returns how many there are (only
// the first KNN_CAP are stored).  Finite bounds exclude the +inf
// non-candidates by themselves.
template <int CH>
__device__ __forceinline__ int compact_le_groups(const float (&s)[CH], const float (&gm)[CH / 4],
                                                 float bound, WarpScratch *ws, int u0 = 0) {
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    int base = 0;
#pragma unroll
    for (int g = 0; g < CH / 4; ++g) {
        if (__any_sync(FULL, gm[g] <= bound)) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int j = 4 * g + i;
                const bool p = s[j] <= bound;
                const unsigned b = __ballot_sync(FULL, p);
                const int pos = base + __popc(b & lt);
                if (p && pos < KNN_CAP) ws->key[pos] = mk_key(s[j], u0 + lane + 32 * j);
                base += __popc(b);
            }
        }
    }
    __syncwarp();
    return base;
}

// Compact the 4-slot cells (lane, group g) whose minimum gm[g] is at or below
// a FINITE bound into ws->cell_v / ws->cell_u: the lane writes the cell's four
// values and the time index of its first slot, u0 + lane + 128 g.
// Returns the number of cells (only the first KNN_CELLS are stored).  On this
// data nearly every value at or below the lane-minimum bound is the minimum
// of its cell, so a cell is written with one 16-byte store where a ballot per
// slot would be needed otherwise.  The code has no data-dependent branch:
// each lane marks its cells in a bit mask, an inclusive warp scan of the mask
// counts gives each lane its first position, and the stores are predicated.
// (A ballot per group with a branch over the active groups costs far more
// when the neighbours are scattered over many groups, as on chaotic series.)
template <int CH>
__device__ __forceinline__ int compact_cells(const float (&s)[CH], const float (&gm)[CH / 4],
                                             float bound, WarpScratch *ws, int u0 = 0) {
    constexpr int NG = CH / 4;
    const int lane = lane_id();
    unsigned mask = 0;
#pragma unroll
    for (int g = 0; g < NG; ++g) mask |= (gm[g] <= bound ? 1u : 0u) << g;
    const int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < WARP; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        incl += lane >= o ? v : 0;
    }
    const int M = __shfl_sync(FULL, incl, WARP - 1);
    int pos = incl - cnt;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
        const bool p = (mask >> g) & 1u;
        if (p && pos < KNN_CELLS) {
            ws->cell_v[pos] = make_float4(s[4 * g], s[4 * g + 1], s[4 * g + 2], s[4 * g + 3]);
            ws->cell_u[pos] = u0 + lane + 128 * g;
        }
        pos += p ? 1 : 0;
    }
    __syncwarp();
    return M;
}

// The keys of the values at or below `bound` in the first M (<= KNN_CELLS)
// cells, into ws->key; returns how many there are (at most 4 M; only the
// first KNN_CAP are stored).  Value i of a cell is the candidate 32 i past
// the cell's first one (ws->cell_u).
__device__ __forceinline__ int cells_to_keys(WarpScratch *ws, int M, float bound) {
    const int lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    int base = 0;
    for (int e0 = 0; e0 < M; e0 += WARP) {
        const int e = e0 + lane;
        float4 v = make_float4(EDM_INF, EDM_INF, EDM_INF, EDM_INF);
        int u0 = 0;
        if (e < M) {
            v = ws->cell_v[e];
            u0 = ws->cell_u[e];
        }
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool p = vv[i] <= bound;
            const unsigned b = __ballot_sync(FULL, p);
            const int pos = base + __popc(b & lt);
            if (p && pos < KNN_CAP) ws->key[pos] = mk_key(vv[i], u0 + 32 * i);
            base += __popc(b);
        }
    }
    __syncwarp();
    return base;
}

// Minima of the 4-slot groups of a register array.
template <int CH>
__device__ __forceinline__ void group_minima(const float (&s)[CH], float (&gm)[CH / 4]) {
    static_assert(CH % 4 == 0, "slots come in groups of four");
#pragma unroll
    for (int g = 0; g < CH / 4; ++g)
        gm[g] = fminf(fminf(s[4 * g], s[4 * g + 1]), fminf(s[4 * g + 2], s[4 * g + 3]));
}

// Warp-wide number of register slots with s <= b.
template <int CH>
__device__ __forceinline__ int warp_count_le(const float (&s)[CH], float b) {
    int c = 0;
#pragma unroll
    for (int j = 0; j < CH; ++j) c += s[j] <= b ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    return c;
}

// Shrink a bound that too many values lie under.  On entry `hi` is a bound
// with c_hi > cap values of s at or below it, and at least `need` values of
// s plus extra(b) lie at or below any accepted bound b (extra(b) counts
// values held elsewhere, e.g. a running list).  Bisection on the value (all
// values are >= 0) keeps that property and stops once at most `cap` values
// of s lie below the bound; returns the bound, or -1 when it cannot get there
// (more than `cap` values tie).  Used where the threshold taken from lane
// minima is loose: at large E the distances concentrate and the (E+2)-th
// smallest lane minimum can lie above half of all values.
template <int CH, class Extra>
__device__ __forceinline__ float shrink_bound(const float (&s)[CH], float hi, int c_hi, int need,
                                              int cap, Extra extra) {
    float lo = 0.f;
    for (int it = 0; it < 48 && c_hi > cap; ++it) {
        const float mid = 0.5f * (lo + hi);
        if (!(mid > lo && mid < hi)) break;  // no float left between the two
        const int cm = warp_count_le<CH>(s, mid);
        if (cm + extra(mid) >= need) {
            hi = mid;
            c_hi = cm;
        } else {
            lo = mid;
        }
    }
    return c_hi <= cap ? hi : -1.f;
}

// The K nearest candidates (exact FP64 neighbour set) of the query time t
// from the FP32 squared distances held in registers: s[j] is the distance to
// the candidate u = lane + 32 j, +inf when u is not a candidate.  Steps as in
// knn_row's KNN_SET mode: lane minima, the (K+1)-th smallest of them as a
// bound, compaction of the values at or below it (through 4-slot cells),
// exact ranking of the collected keys, then the band check (resolved in FP64
// when it fails).  On return lane r < K holds the r-th neighbour and its
// distance (other lanes hold values the caller must ignore).  keep:
// bitonic_keep_min_bits() of this lane.  Returns KNN_USED_* flags (the same
// in every lane).
template <int CH>
__device__ __forceinline__ int select_set_regs(const float (&s)[CH], const float *xs, int t,
                                               int lo, int hi, int E, int tau, int K,
                                               WarpScratch *ws, int &u_out, float &d_out,
                                               unsigned keep) {
    constexpr int NG = CH / 4;
    const int lane = lane_id();
    const int nc = hi - lo;
    const int R = min(K + 1, nc);
    // minima of the slot groups (4 slots each) and of the lane
    float gm[NG];
    group_minima<CH>(s, gm);
    float lmin = EDM_INF;
#pragma unroll
    for (int g = 0; g < NG; ++g) lmin = fminf(lmin, gm[g]);
    const float theta = warp_sorted_at_f(lmin, R - 1, keep);
    // a finite theta excludes the +inf non-candidates by itself
    int c;
    if (theta == EDM_INF) {
        c = compact_le<CH>(s, theta, ws);
    } else {
        const int M = compact_cells<CH>(s, gm, theta, ws);
        c = M <= KNN_CELLS ? cells_to_keys(ws, M, theta)
                           : compact_le_groups<CH>(s, gm, theta, ws);
    }
    if (c > KNN_CAP) {
        // a loose threshold: shrink it so that the values under it fit
        const float b = shrink_bound<CH>(s, theta, c, R, KNN_CAP, [](float) { return 0; });
        if (b >= 0.f) c = compact_le_groups<CH>(s, gm, b, ws);
    }
    int flags = 0;
    if (c <= KNN_CAP) {
        rank_keys(ws, c, R);
        const float edge = band_edge(key_s(ws->sel[K - 1]), E);
        if (R <= K || key_s(ws->sel[K]) > edge) {
            // all lanes (no divergence); lanes >= K repeat entry K-1
            const uint64_t k = ws->sel[min(lane, K - 1)];
            u_out = key_u(k);
            d_out = sqrtf(key_s(k));
            __syncwarp();
            return 0;
        }
        // resolve the band in FP64
        flags = KNN_USED_BAND;
        c = compact_le<CH>(s, edge, ws);
        if (c <= KNN_CAP) {
            rank_band_fp64(xs, t, E, tau, ws, c, K);
        } else {
            brute_fp64(xs, t, lo, hi, E, tau, ws, K);
            flags |= KNN_USED_BRUTE;
        }
    } else {
        // more than KNN_CAP values tie (long runs of repeats)
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

// Per-warp counts of the rows whose neighbour set needed the FP64 band
// (KNN_USED_BAND) and an FP64 brute-force scan (KNN_USED_BRUTE); lane 0 adds
// them to stats[0] / stats[1] once per warp when diagnostics are on.
struct FallbackCount {
    unsigned band = 0, brute = 0;
    __device__ __forceinline__ void add(int flags) {
        band += (flags & KNN_USED_BAND) ? 1u : 0u;
        brute += (flags & KNN_USED_BRUTE) ? 1u : 0u;
    }
    __device__ __forceinline__ void flush(unsigned long long *stats) const {
        if (stats && lane_id() == 0 && (band | brute)) {
            if (band) atomicAdd(stats, static_cast<unsigned long long>(band));
            if (brute) atomicAdd(stats + 1, static_cast<unsigned long long>(brute));
        }
    }
};

// Simplex weights of the K neighbours held one per lane (lane r < K holds
// distance d of rank r; lane 0 the nearest): w = exp(-d/d1) normalised, or
// the d1 == 0 limit.  Returns the normalised weight of this lane (0 for
// lanes >= K).
__device__ __forceinline__ float simplex_weight(float d, int K) {
    const int lane = lane_id();
    const float d1 = __shfl_sync(FULL, d, 0);
    float w = 0.f;
    if (lane < K) {
        if (d1 > 0.f)
            w = expf(-(d / d1));
        else
            w = (d == 0.f) ? 1.f : 0.f;
    }
    const float sum = warp_sum(w);
    return w / sum;
}

}  // namespace edm
