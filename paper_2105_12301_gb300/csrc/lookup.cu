// lookup.cu -- batched lookup with on-the-fly Pearson (kEDM section 2.1
// steps 3-4, Algorithm 3 and the closing paragraph of section 3.3).
//
// Targets are first stored transposed and centred, in tiles of 32 (FP32) or
// 64 (BF16) targets: Yt[tile][u][lane], one 128-byte row per time u.  One
// CTA owns one target tile (staged in shared memory by a bulk TMA copy) and
// a block of libraries.  A producer warp streams the libraries' neighbour
// tables through a ring of shared-memory stages (bulk TMA copies completing
// on mbarriers); sixteen consumer warps take one table row (one query time)
// at a time: the k (neighbour row, weight) pairs are warp-uniform broadcast
// reads (one 16-byte read for k <= 3), and lane l gathers target l's value
// at each neighbour row -- all 32 lanes read one 128-byte shared-memory row,
// so every gather is a single conflict-free wavefront.  The prediction never
// leaves registers; each lane accumulates the prediction's sum, its sum of
// squares and its cross product with the observation in FP32.  The target's
// own sums over the observation window are precomputed in FP64 per (target,
// E).  A finisher warp adds the consumers' partials and forms rho in FP64,
// handed over through a pair of mbarriers so that no consumer waits for it.
#include <cuda_bf16.h>

#include "edm_internal.cuh"

namespace edm {

// consumer warps: 24 with FP32 targets, 16 with BF16 (whose six moments
// per lane need a larger hand-over buffer next to the tile)
template <bool BF16> struct LkWarps {
    static constexpr int NC = BF16 ? 16 : 24;
    static constexpr int PRODUCER = NC;       // warp issuing the bulk copies
    static constexpr int FINISHER = NC + 1;   // warp turning moments into rho
    static constexpr int THREADS = (NC + 2) * 32;
};
constexpr int LK_STAGE_BYTES = 6144;           // table bytes per pipeline stage
constexpr int LK_MAX_STAGES = 8;
constexpr int LK_TILE_ROW = 128;               // bytes per time row of a tile

// ---------------------------------------------------------- target store

__global__ void target_mean_kernel(const float *__restrict__ Y, long long ld, int N, int L,
                                   double *__restrict__ mean) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = lane_id();
    if (warp >= N) return;
    const float *y = Y + static_cast<size_t>(warp) * ld;
    double s = 0.0;
    for (int i = lane; i < L; i += 32) s += static_cast<double>(y[i]);
    s = warp_sum_d(s);
    if (lane == 0) mean[warp] = s / L;
}

// FP32: Yt[tile][u][32] = Y[32 tile + lane][u] - mean; pad targets are 0.
// BF16: Yt[tile][u][64] bf16, lane l's 32-bit word holds targets 2l (low
// half) and 2l+1 (high half), each rounded to nearest even.
// Every tile has L+1 time rows; row L is all zeros (the dummy neighbour row
// of odd-length tables).
template <bool BF16>
__global__ void target_store_kernel(const float *__restrict__ Y, long long ld, int N, int L,
                                    const double *__restrict__ mean, uint8_t *__restrict__ Yt) {
    constexpr int TT = BF16 ? 64 : 32;  // targets per tile
    __shared__ float s[TT][33];
    const int tile = blockIdx.x, u0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int j = ty; j < TT; j += 8) {
        const int tgt = tile * TT + j, u = u0 + tx;
        float v = 0.f;
        if (tgt < N && u < L)
            v = static_cast<float>(static_cast<double>(Y[static_cast<size_t>(tgt) * ld + u]) -
                                   mean[tgt]);
        s[j][tx] = v;
    }
    __syncthreads();
    uint8_t *base = Yt + static_cast<size_t>(tile) * (L + 1) * LK_TILE_ROW;
    if (blockIdx.y == 0 && ty == 0)
        reinterpret_cast<uint32_t *>(base + static_cast<size_t>(L) * LK_TILE_ROW)[tx] = 0u;
    for (int r = ty; r < 32; r += 8) {
        const int u = u0 + r;
        if (u >= L) continue;
        if (BF16) {
            const unsigned lo = __bfloat16_as_ushort(__float2bfloat16_rn(s[2 * tx][r]));
            const unsigned hi = __bfloat16_as_ushort(__float2bfloat16_rn(s[2 * tx + 1][r]));
            reinterpret_cast<uint32_t *>(base + static_cast<size_t>(u) * LK_TILE_ROW)[tx] =
                lo | (hi << 16);
        } else {
            reinterpret_cast<float *>(base + static_cast<size_t>(u) * LK_TILE_ROW)[tx] = s[tx][r];
        }
    }
}

// The stored value of target tgt at time u, as the lookup reads it.
template <bool BF16>
__device__ __forceinline__ float stored_target(const uint8_t *Yt, int L, int tgt, int u) {
    constexpr int TT = BF16 ? 64 : 32;
    const uint32_t *row = reinterpret_cast<const uint32_t *>(
        Yt + (static_cast<size_t>(tgt / TT) * (L + 1) + u) * LK_TILE_ROW);
    if (!BF16) return __uint_as_float(row[tgt % 32]);
    const uint32_t v = row[(tgt % 64) >> 1];
    return __uint_as_float((tgt & 1) ? (v & 0xffff0000u) : (v << 16));
}

// One warp per target: FP64 sums of the stored values and their squares
// over the observation window of every E, times (E-1)tau+Tp .. L-1.  The
// windows are nested, so one pass over the longest suffix plus the pieces
// between consecutive starts gives all of them.
template <bool BF16>
__global__ void target_sums_kernel(const uint8_t *__restrict__ Yt, int N, int L, int tau, int Tp,
                                   double *__restrict__ ysum, double *__restrict__ yysum) {
    const int tgt = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = lane_id();
    if (tgt >= N) return;
    int e_top = EDM_E_MAX;
    while (e_top > 1 && (e_top - 1) * tau + Tp >= L) --e_top;
    const int start_top = (e_top - 1) * tau + Tp;
    double s1 = 0.0, s2 = 0.0;
    for (int u = start_top + lane; u < L; u += 32) {
        const double v = stored_target<BF16>(Yt, L, tgt, u);
        s1 += v;
        s2 += v * v;
    }
    s1 = warp_sum_d(s1);
    s2 = warp_sum_d(s2);
    if (lane != 0) return;
    for (int E = EDM_E_MAX; E >= 1; --E) {
        const int start = (E - 1) * tau + Tp;
        if (E < e_top) {
            // add times start .. start(E+1)-1
            for (int u = start; u < E * tau + Tp && u < L; ++u) {
                const double v = stored_target<BF16>(Yt, L, tgt, u);
                s1 += v;
                s2 += v * v;
            }
        }
        const bool valid = start < L;
        ysum[static_cast<size_t>(E - 1) * N + tgt] = valid ? s1 : 0.0;
        yysum[static_cast<size_t>(E - 1) * N + tgt] = valid ? s2 : 0.0;
    }
}

static int targets_per_tile(edm_precision prec) { return prec == EDM_BF16_TARGETS ? 64 : 32; }

size_t target_store_bytes(int N_tgt, int L, edm_precision prec) {
    const int tt = targets_per_tile(prec);
    const size_t tiles = (N_tgt + tt - 1) / tt;
    return align_up(tiles * (L + 1) * LK_TILE_ROW, 256);
}

edm_status launch_target_store(edm_ctx *ctx, const float *Y, long long ld, int N_tgt, int L,
                               int tau, int Tp, edm_precision prec, uint8_t *Yt, double *mean_ws,
                               double *ysum, double *yysum) {
    const int warps_blocks = (N_tgt * 32 + 255) / 256;
    before_launch(ctx);
    target_mean_kernel<<<warps_blocks, 256, 0, ctx->stream>>>(Y, ld, N_tgt, L, mean_ws);
    edm_status st = after_launch(ctx, "target_mean_kernel");
    if (st != EDM_OK) return st;
    const int tt = targets_per_tile(prec);
    dim3 grid((N_tgt + tt - 1) / tt, (L + 31) / 32), block(32, 8);
    const bool bf16 = prec == EDM_BF16_TARGETS;
    before_launch(ctx);
    if (bf16)
        target_store_kernel<true><<<grid, block, 0, ctx->stream>>>(Y, ld, N_tgt, L, mean_ws, Yt);
    else
        target_store_kernel<false><<<grid, block, 0, ctx->stream>>>(Y, ld, N_tgt, L, mean_ws, Yt);
    st = after_launch(ctx, "target_store_kernel");
    if (st != EDM_OK) return st;
    before_launch(ctx);
    if (bf16)
        target_sums_kernel<true><<<warps_blocks, 256, 0, ctx->stream>>>(Yt, N_tgt, L, tau, Tp, ysum, yysum);
    else
        target_sums_kernel<false><<<warps_blocks, 256, 0, ctx->stream>>>(Yt, N_tgt, L, tau, Tp, ysum, yysum);
    return after_launch(ctx, "target_sums_kernel");
}

// ------------------------------------------------------- lookup + Pearson

struct LookupArgs {
    const uint8_t *Yt;
    const uint8_t *tables;
    size_t slot_bytes;
    const int32_t *E_lib;  // indexed by library id
    const double *ysum;    // [EDM_E_MAX][N_tgt]
    const double *yysum;
    int lib0, nlib, LB;    // libraries [lib0, lib0+nlib) of this launch; LB per CTA
    int L, tau, Tp, N_tgt;
    int stages;
    float *rho;            // row of library lib0
    long long rho_ld;
    int *flags;
};

__device__ __forceinline__ bool lib_valid(int E, int L, int tau, int Tp) {
    return E >= 1 && E <= EDM_E_MAX && L - (E - 1) * tau - Tp >= E + 2;
}

// Row pairs of one table chunk: as many whole pair blocks as fit a stage.
__host__ __device__ constexpr int chunk_pairs(int K) { return LK_STAGE_BYTES / table_pair_bytes(K); }

template <bool BF16>
struct Moments {
    static constexpr int N = BF16 ? 6 : 3;  // per target: sum a, sum a^2, sum a*b
};

// Per-lane prediction moments: for each of the lane's targets, the sums of
// the prediction, of its square and of its product with the observation,
// kept as (row 2p, row 2p+1) pairs for the packed FP32x2 arithmetic.
template <bool BF16>
struct PairMoments {
    static constexpr int T = BF16 ? 2 : 1;  // targets per lane
    float2 s[T], ss[T], sy[T];
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// One table pair block (query times 2p and 2p+1) for this lane's target(s).
// For each row the prediction is y_last + sum_q w_q (y_q - y_last) over its
// K neighbour rows (the K-th weight is 1 minus the others); the two rows run
// side by side in FFMA2/FADD2 lanes.  y_q - y_last is formed as
// fma(y_last, -1, y_q): the exact difference rounded once, as a subtraction.
template <int K, bool BF16, bool SMEM_TILE>
__device__ __forceinline__ void lookup_pair(const uint8_t *blk, const uint32_t *tl, int yrow,
                                            PairMoments<BF16> &m) {
    constexpr int PB = table_pair_bytes(K);
    constexpr int NV = PB / 16;
    uint32_t wd[4 * NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const uint4 v = reinterpret_cast<const uint4 *>(blk)[q];
        wd[4 * q + 0] = v.x;
        wd[4 * q + 1] = v.y;
        wd[4 * q + 2] = v.z;
        wd[4 * q + 3] = v.w;
    }
    uint32_t gA[K], gB[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const uint32_t hA = wd[2 * (K - 1 + (q >> 1))], hB = wd[2 * (K - 1 + (q >> 1)) + 1];
        const uint32_t uA = (q & 1) ? (hA >> 16) : (hA & 0xffffu);
        const uint32_t uB = (q & 1) ? (hB >> 16) : (hB & 0xffffu);
        gA[q] = SMEM_TILE ? tl[uA * 32] : __ldg(tl + uA * 32);
        gB[q] = SMEM_TILE ? tl[uB * 32] : __ldg(tl + uB * 32);
    }
    const uint32_t yA = SMEM_TILE ? tl[yrow * 32] : __ldg(tl + yrow * 32);
    const uint32_t yB = SMEM_TILE ? tl[(yrow + 1) * 32] : __ldg(tl + (yrow + 1) * 32);
    const float2 m1 = f2(-1.f, -1.f);
#pragma unroll
    for (int c = 0; c < PairMoments<BF16>::T; ++c) {
        // c selects the lane's target: FP32 word, or BF16 low / high half
        auto val = [&](uint32_t v) {
            return __uint_as_float(BF16 ? (c == 0 ? (v << 16) : (v & 0xffff0000u)) : v);
        };
        const float2 yl = f2(val(gA[K - 1]), val(gB[K - 1]));
        float2 acc = yl;
#pragma unroll
        for (int q = 0; q < K - 1; ++q) {
            const float2 w = f2(__uint_as_float(wd[2 * q]), __uint_as_float(wd[2 * q + 1]));
            const float2 diff = __ffma2_rn(yl, m1, f2(val(gA[q]), val(gB[q])));
            acc = __ffma2_rn(w, diff, acc);
        }
        const float2 y = f2(val(yA), val(yB));
        m.s[c] = __fadd2_rn(m.s[c], acc);
        m.ss[c] = __ffma2_rn(acc, acc, m.ss[c]);
        m.sy[c] = __ffma2_rn(acc, y, m.sy[c]);
    }
}

// Gather + accumulate one library whose k = K is a compile-time value.
// Warps take pair blocks warp, warp + NC, ... of each chunk.
template <int K, bool BF16, bool SMEM_TILE>
__device__ __forceinline__ void consume_library(const LookupArgs &a, const uint8_t *tile,
                                                const uint8_t *stages, uint64_t *full,
                                                uint64_t *empty, int &seq, int n, int t0,
                                                PairMoments<BF16> &m) {
    constexpr int PB = table_pair_bytes(K);
    constexpr int CP = LK_STAGE_BYTES / PB;
    constexpr int LK_NC = LkWarps<BF16>::NC;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t *tl = reinterpret_cast<const uint32_t *>(tile) + lane;
    const int npairs = (n + 1) >> 1;
    for (int p0 = 0; p0 < npairs; p0 += CP) {
        const int s = seq % a.stages;
        const uint32_t par = (seq / a.stages) & 1;
        mbar_wait_bounded(&full[s], par, a.flags);
        const uint8_t *st = stages + static_cast<size_t>(s) * LK_STAGE_BYTES;
        const int pairs = min(CP, npairs - p0);
        const int ybase = t0 + a.Tp + 2 * p0;
        for (int p = warp; p < pairs; p += LK_NC)
            lookup_pair<K, BF16, SMEM_TILE>(st + p * PB, tl, ybase + 2 * p, m);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        ++seq;
    }
}

// rho from the prediction moments (FP32 partials of the consumer warps) and
// the target's FP64 window sums.
__device__ __forceinline__ float finish_rho(double n, double sa, double saa, double sab, double sb,
                                            double sbb) {
    return static_cast<float>(pearson_from_moments(n, sa, sb, saa, sbb, sab));
}

template <bool BF16, bool SMEM_TILE>
__global__ void __launch_bounds__(LkWarps<BF16>::THREADS, 1) lookup_kernel(const LookupArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int NM = Moments<BF16>::N;
    constexpr int LK_NC = LkWarps<BF16>::NC;
    constexpr int LK_PRODUCER = LkWarps<BF16>::PRODUCER;
    constexpr int LK_FINISHER = LkWarps<BF16>::FINISHER;
    constexpr int TT = BF16 ? 64 : 32;
    const int tile_id = blockIdx.x;
    const int lb0 = a.lib0 + blockIdx.y * a.LB;
    const int lb1 = min(a.lib0 + a.nlib, lb0 + a.LB);
    const size_t tile_bytes = static_cast<size_t>(a.L + 1) * LK_TILE_ROW;
    const uint8_t *tile_g = a.Yt + static_cast<size_t>(tile_id) * tile_bytes;
    uint8_t *tile_s = smem;
    uint8_t *stages = smem + (SMEM_TILE ? tile_bytes : 0);
    float *red = reinterpret_cast<float *>(stages + static_cast<size_t>(a.stages) * LK_STAGE_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(red + 2 * LK_NC * NM * 32);
    uint64_t *full = bars, *empty = bars + a.stages, *tbar = bars + 2 * a.stages;
    uint64_t *red_full = tbar + 1, *red_empty = tbar + 3;
    const int warp = threadIdx.x >> 5, lane = lane_id();

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], LK_NC);
        }
        mbar_init(tbar, 1);
        for (int p = 0; p < 2; ++p) {
            mbar_init(&red_full[p], LK_NC);
            mbar_init(&red_empty[p], 1);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == LK_PRODUCER) {
        // ---------------- producer: target tile, then the table stream
        if (lane == 0) {
            if (SMEM_TILE) {
                mbar_arrive_expect_tx(tbar, static_cast<uint32_t>(tile_bytes));
                for (size_t off = 0; off < tile_bytes; off += 32768)
                    bulk_copy_g2s(tile_s + off, tile_g + off,
                                  static_cast<uint32_t>(tile_bytes - off < 32768 ? tile_bytes - off : 32768),
                                  tbar);
            }
            int seq = 0;
            for (int lib = lb0; lib < lb1; ++lib) {
                const int E = a.E_lib[lib];
                if (!lib_valid(E, a.L, a.tau, a.Tp)) continue;
                const int n = a.L - (E - 1) * a.tau - a.Tp;
                const int npairs = (n + 1) >> 1;
                const int PB = table_pair_bytes(E + 1);
                const int CP = chunk_pairs(E + 1);
                const uint8_t *slot = a.tables + static_cast<size_t>(lib - a.lib0) * a.slot_bytes;
                for (int p0 = 0; p0 < npairs; p0 += CP) {
                    const int s = seq % a.stages, j = seq / a.stages;
                    if (j > 0) mbar_wait_bounded(&empty[s], (j - 1) & 1, a.flags);
                    const uint32_t bytes = static_cast<uint32_t>(min(CP, npairs - p0) * PB);
                    mbar_arrive_expect_tx(&full[s], bytes);
                    bulk_copy_g2s(stages + static_cast<size_t>(s) * LK_STAGE_BYTES,
                                  slot + static_cast<size_t>(p0) * PB, bytes, &full[s]);
                    ++seq;
                }
            }
        }
        return;
    }

    if (warp == LK_FINISHER) {
        // ---------------- finisher: rho of every library of this CTA
        int done = 0;
        for (int lib = lb0; lib < lb1; ++lib) {
            const int E = a.E_lib[lib];
            float *rho_row = a.rho + static_cast<long long>(lib - a.lib0) * a.rho_ld;
            if (!lib_valid(E, a.L, a.tau, a.Tp)) {
                for (int j = lane; j < TT; j += 32) {
                    const int tgt = tile_id * TT + j;
                    if (tgt < a.N_tgt) rho_row[tgt] = __int_as_float(0x7fc00000);
                }
                if (lane == 0 && blockIdx.x == 0) set_flag(a.flags, EDMF_BADARG);
                continue;
            }
            const int p = done & 1;
            mbar_wait_bounded(&red_full[p], (done >> 1) & 1, a.flags);
            const float *base = red + p * LK_NC * NM * 32;
            float S[NM];
#pragma unroll
            for (int j = 0; j < NM; ++j) S[j] = 0.f;
            for (int w = 0; w < LK_NC; ++w)
#pragma unroll
                for (int j = 0; j < NM; ++j) S[j] += base[(w * NM + j) * 32 + lane];
            __syncwarp();
            if (lane == 0) mbar_arrive(&red_empty[p]);
            const double dn = static_cast<double>(a.L - (E - 1) * a.tau - a.Tp);
            const size_t wo = static_cast<size_t>(E - 1) * a.N_tgt;
            if (!BF16) {
                const int tgt = tile_id * 32 + lane;
                if (tgt < a.N_tgt)
                    rho_row[tgt] = finish_rho(dn, S[0], S[1], S[2], a.ysum[wo + tgt], a.yysum[wo + tgt]);
            } else {
                const int tgt = tile_id * 64 + 2 * lane;
                if (tgt < a.N_tgt)
                    rho_row[tgt] = finish_rho(dn, S[0], S[1], S[2], a.ysum[wo + tgt], a.yysum[wo + tgt]);
                if (tgt + 1 < a.N_tgt)
                    rho_row[tgt + 1] = finish_rho(dn, S[3], S[4], S[5], a.ysum[wo + tgt + 1],
                                                  a.yysum[wo + tgt + 1]);
            }
            ++done;
        }
        return;
    }

    // -------------------- consumers
    const uint8_t *tile = SMEM_TILE ? tile_s : tile_g;
    if (SMEM_TILE) mbar_wait_bounded(tbar, 0, a.flags);
    int seq = 0, done = 0;
    PairMoments<BF16> pm;
    for (int lib = lb0; lib < lb1; ++lib) {
        const int E = a.E_lib[lib];
        if (!lib_valid(E, a.L, a.tau, a.Tp)) continue;
        const int n = a.L - (E - 1) * a.tau - a.Tp, t0 = (E - 1) * a.tau;
#pragma unroll
        for (int c = 0; c < PairMoments<BF16>::T; ++c)
            pm.s[c] = pm.ss[c] = pm.sy[c] = f2(0.f, 0.f);
        switch (E + 1) {
#define EDM_CASE(k) \
    case k: consume_library<k, BF16, SMEM_TILE>(a, tile, stages, full, empty, seq, n, t0, pm); break;
            EDM_CASE(2) EDM_CASE(3) EDM_CASE(4) EDM_CASE(5) EDM_CASE(6) EDM_CASE(7) EDM_CASE(8)
            EDM_CASE(9) EDM_CASE(10) EDM_CASE(11) EDM_CASE(12) EDM_CASE(13) EDM_CASE(14)
            EDM_CASE(15) EDM_CASE(16) EDM_CASE(17) EDM_CASE(18) EDM_CASE(19) EDM_CASE(20)
            EDM_CASE(21)
#undef EDM_CASE
        default: break;
        }
        // hand the partial moments to the finisher (double-buffered)
        const int p = done & 1;
        if (done >= 2) mbar_wait_bounded(&red_empty[p], ((done >> 1) - 1) & 1, a.flags);
        float *rb = red + (p * LK_NC + warp) * NM * 32;
#pragma unroll
        for (int c = 0; c < PairMoments<BF16>::T; ++c) {
            rb[(3 * c + 0) * 32 + lane] = pm.s[c].x + pm.s[c].y;
            rb[(3 * c + 1) * 32 + lane] = pm.ss[c].x + pm.ss[c].y;
            rb[(3 * c + 2) * 32 + lane] = pm.sy[c].x + pm.sy[c].y;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&red_full[p]);
        ++done;
    }
}

// Heuristic libraries per CTA: enough CTAs for balance (8 per SM), enough
// libraries per CTA to amortise the target tile load, at most 128.
int lookup_default_lb(edm_ctx *ctx, int nlib, int n_tiles) {
    const long long pairs = static_cast<long long>(nlib) * n_tiles;
    const long long lb = pairs / (8LL * ctx->num_sms);
    return static_cast<int>(std::max<long long>(1, std::min<long long>(128, lb)));
}

static int ceil_log2(long long v) {
    int b = 0;
    while ((1LL << b) < v) ++b;
    return b;
}

uint64_t lookup_bucket(int L, int N_tgt, int nlib, edm_precision prec) {
    const int tt = targets_per_tile(prec);
    const int n_tiles = (N_tgt + tt - 1) / tt;
    return (static_cast<uint64_t>(ceil_log2(L)) << 24) | (static_cast<uint64_t>(ceil_log2(n_tiles)) << 16) |
           (static_cast<uint64_t>(ceil_log2(nlib)) << 8) | static_cast<uint64_t>(prec);
}

edm_status launch_lookup(edm_ctx *ctx, const uint8_t *Yt, int N_tgt, int L, const uint8_t *tables,
                         size_t slot_bytes, const int32_t *E_lib, int lib0, int nlib, int tau,
                         int Tp, edm_precision prec, const double *ysum, const double *yysum,
                         float *rho, long long rho_ld) {
    const bool bf16 = prec == EDM_BF16_TARGETS;
    const int tt = targets_per_tile(prec);
    const int n_tiles = (N_tgt + tt - 1) / tt;
    const int nm = bf16 ? 6 : 3;
    const int LK_NC = bf16 ? LkWarps<true>::NC : LkWarps<false>::NC;
    const int threads = bf16 ? LkWarps<true>::THREADS : LkWarps<false>::THREADS;
    const size_t tile_bytes = static_cast<size_t>(L + 1) * LK_TILE_ROW;
    const size_t fixed = static_cast<size_t>(2) * LK_NC * nm * 32 * sizeof(float) +
                         (2 * LK_MAX_STAGES + 5) * sizeof(uint64_t);
    const size_t limit = static_cast<size_t>(ctx->max_smem_optin);
    const bool smem_tile =
        tile_bytes + fixed + 2 * LK_STAGE_BYTES <= limit && tile_bytes < (1u << 20);
    const size_t avail = limit - fixed - (smem_tile ? tile_bytes : 0);
    const int stages = static_cast<int>(std::min<size_t>(LK_MAX_STAGES, avail / LK_STAGE_BYTES));
    if (stages < 2) return set_error(ctx, EDM_ERR_INTERNAL, "lookup: no room for table stages");
    const size_t smem = (smem_tile ? tile_bytes : 0) + static_cast<size_t>(stages) * LK_STAGE_BYTES +
                        static_cast<size_t>(2) * LK_NC * nm * 32 * sizeof(float) +
                        (2 * stages + 5) * sizeof(uint64_t);

    // libraries per CTA: a fixed override, else the autotuned value of this
    // launch's bucket, else the heuristic
    long long lb = lookup_default_lb(ctx, nlib, n_tiles);
    if (ctx->lookup_lb > 0) {
        lb = std::min(ctx->lookup_lb, nlib);
    } else if (ctx->autotune && ctx->tune) {
        auto it = ctx->tune->find(lookup_bucket(L, N_tgt, nlib, prec));
        if (it != ctx->tune->end()) lb = std::min(it->second, nlib);
    }
    LookupArgs a;
    a.Yt = Yt;
    a.tables = tables;
    a.slot_bytes = slot_bytes;
    a.E_lib = E_lib;
    a.ysum = ysum;
    a.yysum = yysum;
    a.lib0 = lib0;
    a.nlib = nlib;
    a.LB = static_cast<int>(lb);
    a.L = L;
    a.tau = tau;
    a.Tp = Tp;
    a.N_tgt = N_tgt;
    a.stages = stages;
    a.rho = rho;
    a.rho_ld = rho_ld;
    a.flags = ctx->d_flags;
    dim3 grid(n_tiles, static_cast<unsigned>((nlib + lb - 1) / lb));
    void (*kern)(const LookupArgs);
    if (bf16)
        kern = smem_tile ? lookup_kernel<true, true> : lookup_kernel<true, false>;
    else
        kern = smem_tile ? lookup_kernel<false, true> : lookup_kernel<false, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    before_launch(ctx);
    kern<<<grid, threads, smem, ctx->stream>>>(a);
    return after_launch(ctx, "lookup_kernel");
}

}  // namespace edm
