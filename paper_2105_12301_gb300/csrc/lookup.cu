// lookup.cu -- batched lookup with on-the-fly Pearson (kEDM section 2.1
// steps 3-4, Algorithm 3 and the closing paragraph of section 3.3).
//
// Targets are first stored transposed and centred, in tiles of 32 (FP32) or
// 64 (BF16 or FP16, two per 32-bit word) targets: Yt[tile][u][lane], one
// 128-byte row per time u.  One
// CTA owns one target tile (staged in shared memory by a bulk TMA copy) and
// a block of library groups (libraries of equal E, see CcmGroups).  A
// producer warp streams the groups' interleaved neighbour tables through a
// ring of shared-memory stages (bulk TMA copies completing on mbarriers);
// sixteen consumer warps take one pair of query times at a time: they read
// the two observations once, then, for every member library, the pair's
// (neighbour row, weight) values as warp-uniform broadcast reads, and lane l
// gathers target l's value at each neighbour row -- all 32 lanes read one
// 128-byte shared-memory row, so every gather is a single conflict-free
// wavefront.  The prediction never leaves registers; each lane accumulates
// the prediction's sum, its sum of squares and its cross product with the
// observation in FP32, per member.  The target's own sums over the
// observation window are precomputed in FP64 per (target, E).  At the end of
// a group, consumer warp w+8 hands its partial moments to warp w, which adds
// them to its own in FP32 and passes the sum on; a finisher warp adds those
// eight with compensated (TwoSum) FP32 arithmetic, finishes the sums in FP64
// and forms rho in FP64 (a fixed summation order, handed over through
// mbarriers).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "edm_internal.cuh"

namespace edm {

// Target storage formats (the edm_precision values): FP32, or two 16-bit
// values per 32-bit tile word (BF16, or FP16 scaled per target by a power of
// two).  unpack_target gives value c (0: low half, 1: high half) of a word.
template <int FMT>
__device__ __forceinline__ float unpack_target(uint32_t v, int c) {
    if (FMT == EDM_FP32) return __uint_as_float(v);
    if (FMT == EDM_BF16_TARGETS) return __uint_as_float(c == 0 ? (v << 16) : (v & 0xffff0000u));
    return __half2float(__ushort_as_half(static_cast<unsigned short>(c == 0 ? (v & 0xffffu) : (v >> 16))));
}

// Warp roles of the lookup CTA; G libraries per group, NM FP32 moments per
// lane and library (3 per target: sum of the prediction, of its square and
// of its product with the observation).
template <int FMT> struct LkCfg {
    static constexpr bool PK = FMT != EDM_FP32;    // two targets per lane
    static constexpr int NC = 16;                  // consumer warps
    static constexpr int G = PK ? LK_GROUP_16 : LK_GROUP_FP32;
    static constexpr int NM = PK ? 6 : 3;
    static constexpr int PRODUCER = NC;            // warp issuing the bulk copies
    static constexpr int FINISHER = NC + 1;        // warp turning moments into rho
    static constexpr int THREADS = (NC + 2) * 32;
    static constexpr int HALF = NC / 2;            // hand-over slots
    static constexpr int RED_FLOATS = HALF * G * NM * 32;  // hand-over buffer
};
constexpr int LK_MAX_STAGES = 8;

// ---------------------------------------------------------- target store

// Row r of the target store is series rows[r] of Y (series r when rows is NULL).
__device__ __forceinline__ size_t target_row(const int32_t *rows, int r) {
    return static_cast<size_t>(rows ? rows[r] : r);
}

// mean[r]: the FP64 mean of stored target r; scale[r]: the power of two
// 2^(13 - floor(log2 B)), B = max|y| + |mean| >= max|y - mean|, so that the
// centred, scaled values of an FP16 store lie below 2^14 in magnitude with
// the largest of them at full FP16 precision (1 when B is 0 or not finite).
// Pearson's rho does not change when a target is scaled, so the scale is
// never undone.
__global__ void target_mean_kernel(const float *__restrict__ Y, long long ld,
                                   const int32_t *__restrict__ rows, int N, int L,
                                   double *__restrict__ mean, double *__restrict__ scale) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = lane_id();
    if (warp >= N) return;
    const float *y = Y + target_row(rows, warp) * ld;
    double s = 0.0;
    float amax = 0.f;
    for (int i = lane; i < L; i += 32) {
        s += static_cast<double>(y[i]);
        amax = fmaxf(amax, fabsf(y[i]));
    }
    s = warp_sum_d(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, o));
    if (lane == 0) {
        const double mu = s / L;
        mean[warp] = mu;
        const double B = static_cast<double>(amax) + fabs(mu);
        scale[warp] = (B > 0.0 && isfinite(B)) ? ldexp(1.0, 13 - ilogb(B)) : 1.0;
    }
}

// A tile row holds RW 32-bit words: RW = 32 (128-byte rows) normally, 16
// (64-byte rows) when a 32-word tile of the series length does not fit
// shared memory but a 16-word one does.  FP32: Yt[tile][u][RW] = Y[RW tile +
// w][u] - mean; BF16 / FP16: word w holds targets 2w (low half) and 2w+1
// (high half), each rounded to nearest even (FP16: after scaling by the
// target's power of two).  Pad targets are 0.  Every tile has L+1 time rows;
// row L is all zeros (the dummy neighbour row of odd-length tables).
template <int FMT, int RW>
__global__ void target_store_kernel(const float *__restrict__ Y, long long ld,
                                    const int32_t *__restrict__ rows, int N, int L,
                                    const double *__restrict__ mean,
                                    const double *__restrict__ scale, uint8_t *__restrict__ Yt) {
    constexpr bool PK = FMT != EDM_FP32;
    constexpr int TT = PK ? 2 * RW : RW;  // targets per tile
    __shared__ float s[TT][33];
    const int tile = blockIdx.x, u0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int j = ty; j < TT; j += 8) {
        const int tgt = tile * TT + j, u = u0 + tx;
        float v = 0.f;
        if (tgt < N && u < L) {
            double c = static_cast<double>(Y[target_row(rows, tgt) * ld + u]) - mean[tgt];
            if (FMT == EDM_FP16_TARGETS) c *= scale[tgt];
            v = static_cast<float>(c);
        }
        s[j][tx] = v;
    }
    __syncthreads();
    constexpr size_t ROW = 4 * RW;
    uint8_t *base = Yt + static_cast<size_t>(tile) * (L + 1) * ROW;
    if (blockIdx.y == 0 && ty == 0 && tx < RW)
        reinterpret_cast<uint32_t *>(base + static_cast<size_t>(L) * ROW)[tx] = 0u;
    if (tx >= RW) return;
    for (int r = ty; r < 32; r += 8) {
        const int u = u0 + r;
        if (u >= L) continue;
        if (FMT == EDM_BF16_TARGETS) {
            const unsigned lo = __bfloat16_as_ushort(__float2bfloat16_rn(s[2 * tx][r]));
            const unsigned hi = __bfloat16_as_ushort(__float2bfloat16_rn(s[2 * tx + 1][r]));
            reinterpret_cast<uint32_t *>(base + static_cast<size_t>(u) * ROW)[tx] = lo | (hi << 16);
        } else if (FMT == EDM_FP16_TARGETS) {
            const unsigned lo = __half_as_ushort(__float2half_rn(s[2 * tx][r]));
            const unsigned hi = __half_as_ushort(__float2half_rn(s[2 * tx + 1][r]));
            reinterpret_cast<uint32_t *>(base + static_cast<size_t>(u) * ROW)[tx] = lo | (hi << 16);
        } else {
            reinterpret_cast<float *>(base + static_cast<size_t>(u) * ROW)[tx] = s[tx][r];
        }
    }
}

// The stored value of target tgt at time u, as the lookup reads it.
template <int FMT, int RW>
__device__ __forceinline__ float stored_target(const uint8_t *Yt, int L, int tgt, int u) {
    constexpr int TT = FMT != EDM_FP32 ? 2 * RW : RW;
    const uint32_t *row = reinterpret_cast<const uint32_t *>(
        Yt + (static_cast<size_t>(tgt / TT) * (L + 1) + u) * (4 * RW));
    if (FMT == EDM_FP32) return __uint_as_float(row[tgt % TT]);
    return unpack_target<FMT>(row[(tgt % TT) >> 1], tgt & 1);
}

// One warp per target: FP64 sums of the stored values and their squares
// over the observation window of every E, times (E-1)tau+Tp .. L-1.  The
// windows are nested, so one pass over the longest suffix plus the pieces
// between consecutive starts gives all of them.
template <int FMT, int RW>
__global__ void target_sums_kernel(const uint8_t *__restrict__ Yt, int N, int L, int tau, int Tp,
                                   double *__restrict__ ysum, double *__restrict__ yysum) {
    const int tgt = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = lane_id();
    if (tgt >= N) return;
    int e_top = EDM_E_MAX;
    while (e_top > 1 && (e_top - 1) * tau + Tp >= L) --e_top;
    const int start_top = (e_top - 1) * tau + Tp;
    double s1 = 0.0, s2 = 0.0;
    for (int u = start_top + lane; u < L; u += 32) {
        const double v = stored_target<FMT, RW>(Yt, L, tgt, u);
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
                const double v = stored_target<FMT, RW>(Yt, L, tgt, u);
                s1 += v;
                s2 += v * v;
            }
        }
        const bool valid = start < L;
        ysum[static_cast<size_t>(E - 1) * N + tgt] = valid ? s1 : 0.0;
        yysum[static_cast<size_t>(E - 1) * N + tgt] = valid ? s2 : 0.0;
    }
}

// Shared memory a lookup CTA needs besides its tile: the hand-over buffer,
// at least two 4 KB table stages and the mbarriers.
static size_t lookup_fixed_bytes(edm_precision prec) {
    const size_t red = sizeof(float) * (prec != EDM_FP32 ? LkCfg<EDM_BF16_TARGETS>::RED_FLOATS
                                                          : LkCfg<EDM_FP32>::RED_FLOATS);
    // stage barriers (full, empty), the tile barrier, the three hand-over
    // barriers and the abort word: 2 stages + 5 words (6 reserved)
    return red + (2 * LK_MAX_STAGES + 6) * sizeof(uint64_t);
}

int lookup_row_words(edm_ctx *ctx, int L, edm_precision prec) {
    const size_t limit = static_cast<size_t>(ctx->max_smem_optin);
    const size_t need = lookup_fixed_bytes(prec) + 2 * 4096;
    if (static_cast<size_t>(L + 1) * 128 + need <= limit) return 32;
    if (static_cast<size_t>(L + 1) * 64 + need <= limit) return 16;
    return 32;  // the tile stays in global memory
}

static int targets_per_tile(edm_precision prec, int rw) {
    return prec != EDM_FP32 ? 2 * rw : rw;
}

size_t target_store_bytes(int N_tgt, int L, edm_precision prec, int rw) {
    const int tt = targets_per_tile(prec, rw);
    const size_t tiles = (N_tgt + tt - 1) / tt;
    return align_up(tiles * (L + 1) * 4 * rw, 256);
}

// The kernels of the target store for one storage format and row width.
template <int FMT, int RW>
static edm_status launch_store_fmt(edm_ctx *ctx, const float *Y, long long ld, const int32_t *rows,
                                   int N_tgt, int L, int tau, int Tp, uint8_t *Yt,
                                   const double *mean, const double *scale, double *ysum,
                                   double *yysum) {
    const int tt = FMT != EDM_FP32 ? 2 * RW : RW;
    dim3 grid((N_tgt + tt - 1) / tt, (L + 31) / 32), block(32, 8);
    before_launch(ctx);
    target_store_kernel<FMT, RW><<<grid, block, 0, ctx->stream>>>(Y, ld, rows, N_tgt, L, mean,
                                                                  scale, Yt);
    edm_status st = after_launch(ctx, "target_store_kernel");
    if (st != EDM_OK) return st;
    const int warps_blocks = (N_tgt * 32 + 255) / 256;
    before_launch(ctx);
    target_sums_kernel<FMT, RW><<<warps_blocks, 256, 0, ctx->stream>>>(Yt, N_tgt, L, tau, Tp,
                                                                      ysum, yysum);
    return after_launch(ctx, "target_sums_kernel");
}

edm_status launch_target_store(edm_ctx *ctx, const float *Y, long long ld, const int32_t *rows,
                               int N_tgt, int L, int tau, int Tp, edm_precision prec, int rw,
                               uint8_t *Yt, double *mean_ws, double *ysum, double *yysum) {
    // mean_ws holds the means [N_tgt] followed by the FP16 scales [N_tgt]
    double *scale = mean_ws + N_tgt;
    const int warps_blocks = (N_tgt * 32 + 255) / 256;
    before_launch(ctx);
    target_mean_kernel<<<warps_blocks, 256, 0, ctx->stream>>>(Y, ld, rows, N_tgt, L, mean_ws,
                                                              scale);
    edm_status st = after_launch(ctx, "target_mean_kernel");
    if (st != EDM_OK) return st;
    const bool half = rw == 16;
    switch (prec) {
    case EDM_BF16_TARGETS:
        return half ? launch_store_fmt<EDM_BF16_TARGETS, 16>(ctx, Y, ld, rows, N_tgt, L, tau, Tp, Yt, mean_ws, scale, ysum, yysum)
                    : launch_store_fmt<EDM_BF16_TARGETS, 32>(ctx, Y, ld, rows, N_tgt, L, tau, Tp, Yt, mean_ws, scale, ysum, yysum);
    case EDM_FP16_TARGETS:
        return half ? launch_store_fmt<EDM_FP16_TARGETS, 16>(ctx, Y, ld, rows, N_tgt, L, tau, Tp, Yt, mean_ws, scale, ysum, yysum)
                    : launch_store_fmt<EDM_FP16_TARGETS, 32>(ctx, Y, ld, rows, N_tgt, L, tau, Tp, Yt, mean_ws, scale, ysum, yysum);
    default:
        return half ? launch_store_fmt<EDM_FP32, 16>(ctx, Y, ld, rows, N_tgt, L, tau, Tp, Yt, mean_ws, scale, ysum, yysum)
                    : launch_store_fmt<EDM_FP32, 32>(ctx, Y, ld, rows, N_tgt, L, tau, Tp, Yt, mean_ws, scale, ysum, yysum);
    }
}

// ------------------------------------------------------- lookup + Pearson

struct LookupArgs {
    const uint8_t *Yt;
    const uint8_t *tables;
    CcmGroups grp;
    const double *ysum;    // [EDM_E_MAX][N_tgt]
    const double *yysum;
    int lib0, GB;          // rho row 0 is library lib0; GB groups per CTA
    int L, tau, Tp, N_tgt;
    int stages, stage_bytes;
    float *rho;
    long long rho_ld;
    const int32_t *rho_col;  // column of target tgt in rho (tgt itself when NULL)
    int *flags;
};

__device__ __forceinline__ long long rho_column(const LookupArgs &a, int tgt) {
    return a.rho_col ? a.rho_col[tgt] : tgt;
}

// Per-lane prediction moments of one library: for each of the lane's
// targets, the sums of the prediction, of its square and of its product with
// the observation, kept as (row 2p, row 2p+1) pairs for the packed FP32x2
// arithmetic.
template <bool PK>
struct PairMoments {
    static constexpr int T = PK ? 2 : 1;  // targets per lane
    float2 s[T], ss[T], sy[T];
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// One table pair block (query times 2p and 2p+1) of one library for this
// lane's target(s); yA / yB are the lane's stored observation words of the
// two times.  For each row the prediction is y_last + sum_q w_q (y_q -
// y_last) over its K neighbour rows (the K-th weight is 1 minus the others);
// the two rows run side by side in FFMA2/FADD2 lanes.  y_q - y_last is formed
// as fma(y_last, -1, y_q): the exact difference rounded once, as a
// subtraction.
template <int K, int FMT, bool SMEM_TILE>
__device__ __forceinline__ void lookup_pair(const uint8_t *blk, const uint32_t *tl, uint32_t yA,
                                            uint32_t yB, PairMoments<FMT != EDM_FP32> &m) {
    constexpr bool PK = FMT != EDM_FP32;
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
    const float2 m1 = f2(-1.f, -1.f);
#pragma unroll
    for (int c = 0; c < PairMoments<PK>::T; ++c) {
        // c selects the lane's target: FP32 word, or 16-bit low / high half
        auto val = [&](uint32_t v) { return unpack_target<FMT>(v, c); };
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

// Half-row layout (16-word tile rows): half-warp h = lane/16 takes row 2p+h
// of the pair block and lane l its tile word l%16, so one gather reads two
// rows of 16 words.  Same prediction formula as lookup_pair; the moments
// go to the .x lanes of the pair accumulators.
template <int K, int FMT>
__device__ __forceinline__ void lookup_pair_half(const uint8_t *blk, const uint32_t *tl, int h,
                                                 uint32_t yv, PairMoments<FMT != EDM_FP32> &m) {
    constexpr bool PK = FMT != EDM_FP32;
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
    uint32_t g[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const int iw = 2 * (K - 1 + (q >> 1));
        const uint32_t hw = h ? wd[iw + 1] : wd[iw];
        const uint32_t u = (q & 1) ? (hw >> 16) : (hw & 0xffffu);
        g[q] = tl[u * 16];
    }
#pragma unroll
    for (int c = 0; c < PairMoments<PK>::T; ++c) {
        auto val = [&](uint32_t v) { return unpack_target<FMT>(v, c); };
        const float yl = val(g[K - 1]);
        float acc = yl;
#pragma unroll
        for (int q = 0; q < K - 1; ++q) {
            const float w = __uint_as_float(h ? wd[2 * q + 1] : wd[2 * q]);
            acc = __fmaf_rn(w, __fmaf_rn(yl, -1.f, val(g[q])), acc);
        }
        m.s[c].x = __fadd_rn(m.s[c].x, acc);
        m.ss[c].x = __fmaf_rn(acc, acc, m.ss[c].x);
        m.sy[c].x = __fmaf_rn(acc, val(yv), m.sy[c].x);
    }
}

// Position in the ring of table stages: the stage and the parity of the
// ring's current pass (kept incrementally; the stage count is a run-time
// value, so no division per stage).
struct RingPos {
    int s = 0;
    uint32_t ph = 0;
    __device__ __forceinline__ void next(int stages) {
        if (++s == stages) {
            s = 0;
            ph ^= 1u;
        }
    }
};

// Gather + accumulate one group whose k = K is a compile-time value: warps
// take pairs warp, warp + NC, ... of each stage; a pair's observations are
// read once and serve every member of the group.  All G slots are processed
// (the empty slots of a partial group hold a copy of its first member).
template <int K, int FMT, bool SMEM_TILE, bool HALF>
__device__ __forceinline__ void consume_group(const LookupArgs &a, const uint8_t *tile,
                                              const uint8_t *stages, uint64_t *full,
                                              uint64_t *empty, RingPos &rp, int n, int t0,
                                              volatile int *a_abort,
                                              PairMoments<LkCfg<FMT>::PK> (&pm)[LkCfg<FMT>::G]) {
    using C = LkCfg<FMT>;
    constexpr int PB = table_pair_bytes(K);
    constexpr int GPB = C::G * PB;
    const int CP = a.stage_bytes / GPB;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t *tl = reinterpret_cast<const uint32_t *>(tile) + (HALF ? (lane & 15) : lane);
    const int h = lane >> 4;
    const int npairs = (n + 1) >> 1;
    if (HALF) {
        for (int p0 = 0; p0 < npairs; p0 += CP) {
            const int s = rp.s;
            const bool ok = mbar_wait_bounded(&full[s], rp.ph, a.flags, a_abort);
            const uint8_t *st = stages + static_cast<size_t>(s) * a.stage_bytes;
            const int pairs = ok ? min(CP, npairs - p0) : 0;  // no data: skip the stage
            const int ybase = t0 + a.Tp + 2 * p0 + h;
            for (int p = warp; p < pairs; p += C::NC) {
                const uint32_t yv = tl[(ybase + 2 * p) * 16];
                const uint8_t *blk = st + static_cast<size_t>(p) * GPB;
#pragma unroll
                for (int m = 0; m < C::G; ++m)
                    lookup_pair_half<K, FMT>(blk + m * PB, tl, h, yv, pm[m]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            rp.next(a.stages);
        }
        return;
    }
    for (int p0 = 0; p0 < npairs; p0 += CP) {
        const int s = rp.s;
        const bool ok = mbar_wait_bounded(&full[s], rp.ph, a.flags, a_abort);
        const uint8_t *st = stages + static_cast<size_t>(s) * a.stage_bytes;
        const int pairs = ok ? min(CP, npairs - p0) : 0;  // no data: skip the stage
        const int ybase = t0 + a.Tp + 2 * p0;
        for (int p = warp; p < pairs; p += C::NC) {
            const int yrow = ybase + 2 * p;
            const uint32_t yA = SMEM_TILE ? tl[yrow * 32] : __ldg(tl + yrow * 32);
            const uint32_t yB = SMEM_TILE ? tl[(yrow + 1) * 32] : __ldg(tl + (yrow + 1) * 32);
            const uint8_t *blk = st + static_cast<size_t>(p) * GPB;
#pragma unroll
            for (int m = 0; m < C::G; ++m)
                lookup_pair<K, FMT, SMEM_TILE>(blk + m * PB, tl, yA, yB, pm[m]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        rp.next(a.stages);
    }
}

// hi + lo += v, with hi + lo kept as an unevaluated sum of two floats: the
// rounding error of hi + v is recovered exactly (Knuth's TwoSum, six FP32
// operations, every one rounded to nearest) and added into lo.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// rho from the prediction moments (FP32 partials of the consumer warps) and
// the target's FP64 window sums.
__device__ __forceinline__ float finish_rho(double n, double sa, double saa, double sab, double sb,
                                            double sbb) {
    return static_cast<float>(pearson_from_moments(n, sa, sb, saa, sbb, sab));
}

// HALF: 16-word tile rows (see lookup_pair_half); only with the tile in
// shared memory.
template <int FMT, bool SMEM_TILE, bool HALF>
__global__ void __launch_bounds__(LkCfg<FMT>::THREADS, 1) lookup_kernel(const LookupArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    using C = LkCfg<FMT>;
    constexpr bool PK = C::PK;
    constexpr int RW = HALF ? 16 : 32;            // words per tile row
    constexpr int TT = PK ? 2 * RW : RW;          // targets per tile
    constexpr int G = C::G, NM = C::NM;
    const int g0 = blockIdx.y * a.GB;
    const int g1 = min(*a.grp.count, g0 + a.GB);
    if (g0 >= g1) return;  // every thread of the CTA leaves here together
    const int tile_id = blockIdx.x;
    const size_t tile_bytes = static_cast<size_t>(a.L + 1) * 4 * RW;
    const uint8_t *tile_g = a.Yt + static_cast<size_t>(tile_id) * tile_bytes;
    uint8_t *tile_s = smem;
    uint8_t *stages = smem + (SMEM_TILE ? tile_bytes : 0);
    float *red = reinterpret_cast<float *>(stages + static_cast<size_t>(a.stages) * a.stage_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(red + C::RED_FLOATS);
    uint64_t *full = bars, *empty = bars + a.stages, *tbar = bars + 2 * a.stages;
    // hand-over barriers, one phase per group each: half_full (warps 8..15
    // wrote their slots), red_full (warps 0..7 added theirs), red_empty (the
    // finisher read them)
    uint64_t *half_full = tbar + 1, *red_full = tbar + 2, *red_empty = tbar + 3;
    volatile int *abort_w = reinterpret_cast<volatile int *>(tbar + 4);
    const int warp = threadIdx.x >> 5, lane = lane_id();

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], C::NC);
        }
        mbar_init(tbar, 1);
        mbar_init(half_full, C::NC - C::HALF);
        mbar_init(red_full, C::HALF);
        mbar_init(red_empty, 1);
        *abort_w = 0;
        fence_barrier_init();
    }
    __syncthreads();

    if (warp == C::PRODUCER) {
        // ---------------- producer: target tile, then the table stream
        if (lane == 0) {
            if (SMEM_TILE) {
                mbar_arrive_expect_tx(tbar, static_cast<uint32_t>(tile_bytes));
                for (size_t off = 0; off < tile_bytes; off += 32768)
                    bulk_copy_g2s(tile_s + off, tile_g + off,
                                  static_cast<uint32_t>(tile_bytes - off < 32768 ? tile_bytes - off : 32768),
                                  tbar);
            }
            RingPos rp;
            bool first_pass = true;  // the stages are empty until the ring wraps
            bool stop = false;       // a wait gave up: issue no more copies
            for (int gi = g0; gi < g1 && !stop; ++gi) {
                const int E = a.grp.E[gi];
                if (E == 0) continue;
                const int n = a.L - (E - 1) * a.tau - a.Tp;
                const int npairs = (n + 1) >> 1;
                const int GPB = G * table_pair_bytes(E + 1);
                const int CP = a.stage_bytes / GPB;
                const uint8_t *src = a.tables + a.grp.off[gi];
                for (int p0 = 0; p0 < npairs; p0 += CP) {
                    const int s = rp.s;
                    if (!first_pass && !mbar_wait_bounded(&empty[s], rp.ph ^ 1u, a.flags, abort_w)) {
                        stop = true;
                        break;
                    }
                    const uint32_t bytes = static_cast<uint32_t>(min(CP, npairs - p0) * GPB);
                    mbar_arrive_expect_tx(&full[s], bytes);
                    bulk_copy_g2s(stages + static_cast<size_t>(s) * a.stage_bytes,
                                  src + static_cast<size_t>(p0) * GPB, bytes, &full[s]);
                    rp.next(a.stages);
                    if (rp.s == 0) first_pass = false;
                }
            }
            // the CTA's shared memory must outlive every copy issued into it:
            // wait (bounded, past any abort) for the last fill of each stage
            // and for the tile
            for (int s = 0; s < a.stages; ++s) {
                if (s < rp.s)
                    mbar_wait_bounded(&full[s], rp.ph, a.flags, nullptr);
                else if (!first_pass)
                    mbar_wait_bounded(&full[s], rp.ph ^ 1u, a.flags, nullptr);
            }
            if (SMEM_TILE) mbar_wait_bounded(tbar, 0, a.flags, nullptr);
        }
        return;
    }

    if (warp == C::FINISHER) {
        // ---------------- finisher: rho of every member of every group from
        // the HALF slots of FP32 partial moments (consumer warps w and w+8
        // added together), summed in slot order
        int done = 0;
        for (int gi = g0; gi < g1; ++gi) {
            const int E = a.grp.E[gi], nm = a.grp.n[gi];
            const int32_t *libs = a.grp.lib + static_cast<size_t>(gi) * G;
            if (E == 0) {
                for (int m = 0; m < nm; ++m) {
                    float *rho_row = a.rho + static_cast<long long>(libs[m] - a.lib0) * a.rho_ld;
                    for (int j = lane; j < TT; j += 32) {
                        const int tgt = tile_id * TT + j;
                        if (tgt < a.N_tgt) rho_row[rho_column(a, tgt)] = __int_as_float(0x7fc00000);
                    }
                }
                if (lane == 0 && blockIdx.x == 0) set_flag(a.flags, EDMF_BADARG);
                continue;
            }
            // the eight partials are summed exactly enough for FP64: each sum
            // is kept as an unevaluated pair hi + lo of floats (Knuth's
            // TwoSum: hi + lo equals the running sum to about 2^-48), which
            // the FP32 pipe does at full rate; FP64 runs at a small fraction
            // of that on this GPU and held the next group's hand-over up
            float Shi[G][NM], Slo[G][NM];
#pragma unroll
            for (int m = 0; m < G; ++m)
#pragma unroll
                for (int j = 0; j < NM; ++j) Shi[m][j] = Slo[m][j] = 0.f;
            const bool ok = mbar_wait_bounded(red_full, done & 1, a.flags, abort_w);
            for (int w = 0; w < C::HALF; ++w)
#pragma unroll
                for (int m = 0; m < G; ++m)
                    if (m < nm)
#pragma unroll
                        for (int j = 0; j < NM; ++j)
                            two_sum_acc(Shi[m][j], Slo[m][j], red[((w * G + m) * NM + j) * 32 + lane]);
            __syncwarp();
            if (lane == 0) mbar_arrive(red_empty);
            double S[G][NM];
#pragma unroll
            for (int m = 0; m < G; ++m)
#pragma unroll
                for (int j = 0; j < NM; ++j)
                    S[m][j] = static_cast<double>(Shi[m][j]) + static_cast<double>(Slo[m][j]);
            const double dn = static_cast<double>(a.L - (E - 1) * a.tau - a.Tp);
            const size_t wo = static_cast<size_t>(E - 1) * a.N_tgt;
            const float nan = __int_as_float(0x7fc00000);
#pragma unroll
            for (int m = 0; m < G; ++m) {
                if (m >= nm) continue;
                float *rho_row = a.rho + static_cast<long long>(libs[m] - a.lib0) * a.rho_ld;
                if (HALF && lane >= 16) continue;
                if (!PK) {
                    const int tgt = tile_id * TT + lane;
                    if (tgt < a.N_tgt)
                        rho_row[rho_column(a, tgt)] =
                            ok ? finish_rho(dn, S[m][0], S[m][1], S[m][2], a.ysum[wo + tgt],
                                            a.yysum[wo + tgt])
                               : nan;
                } else {
                    const int tgt = tile_id * TT + 2 * lane;
                    if (tgt < a.N_tgt)
                        rho_row[rho_column(a, tgt)] =
                            ok ? finish_rho(dn, S[m][0], S[m][1], S[m][2], a.ysum[wo + tgt],
                                            a.yysum[wo + tgt])
                               : nan;
                    if (tgt + 1 < a.N_tgt)
                        rho_row[rho_column(a, tgt + 1)] =
                            ok ? finish_rho(dn, S[m][3], S[m][4], S[m][5], a.ysum[wo + tgt + 1],
                                            a.yysum[wo + tgt + 1])
                               : nan;
                }
            }
            ++done;
        }
        return;
    }

    // -------------------- consumers
    const uint8_t *tile = SMEM_TILE ? tile_s : tile_g;
    if (SMEM_TILE) mbar_wait_bounded(tbar, 0, a.flags, abort_w);
    RingPos rp;
    int done = 0;
    PairMoments<PK> pm[G];
    for (int gi = g0; gi < g1; ++gi) {
        const int E = a.grp.E[gi];
        if (E == 0) continue;
        const int nm = a.grp.n[gi];
        const int n = a.L - (E - 1) * a.tau - a.Tp, t0 = (E - 1) * a.tau;
#pragma unroll
        for (int m = 0; m < G; ++m)
#pragma unroll
            for (int c = 0; c < PairMoments<PK>::T; ++c)
                pm[m].s[c] = pm[m].ss[c] = pm[m].sy[c] = f2(0.f, 0.f);
        switch (E + 1) {
#define EDM_CASE(k) \
    case k: consume_group<k, FMT, SMEM_TILE, HALF>(a, tile, stages, full, empty, rp, n, t0, abort_w, pm); break;
            EDM_CASE(2) EDM_CASE(3) EDM_CASE(4) EDM_CASE(5) EDM_CASE(6) EDM_CASE(7) EDM_CASE(8)
            EDM_CASE(9) EDM_CASE(10) EDM_CASE(11) EDM_CASE(12) EDM_CASE(13) EDM_CASE(14)
            EDM_CASE(15) EDM_CASE(16) EDM_CASE(17) EDM_CASE(18) EDM_CASE(19) EDM_CASE(20)
            EDM_CASE(21)
#undef EDM_CASE
        default: break;
        }
        // hand the partial moments over; group d = done is phase d of every
        // hand-over barrier.  Warp w+8 writes slot w once the finisher has
        // read the previous group (red_empty phase d-1); warp w waits for it
        // (half_full phase d), adds its own partials to the slot in FP32 and
        // signals the finisher (red_full).  No barrier can be more than one
        // phase past the one waited for (its next phase needs this warp's own
        // arrival first), so each parity test is unambiguous.
        const bool upper = warp >= C::HALF;
        float *rb0 = red + (upper ? warp - C::HALF : warp) * G * NM * 32;
        if (upper) {
            if (done > 0) mbar_wait_bounded(red_empty, (done - 1) & 1, a.flags, abort_w);
        } else {
            mbar_wait_bounded(half_full, done & 1, a.flags, abort_w);
        }
#pragma unroll
        for (int m = 0; m < G; ++m) {
            if (m >= nm) continue;
            float *rb = rb0 + m * NM * 32;
#pragma unroll
            for (int c = 0; c < PairMoments<PK>::T; ++c) {
                // row pairs: the two rows of a lane (FFMA2 lanes), or the
                // two half-warps (HALF)
                float v0, v1, v2;
                if (HALF) {
                    v0 = pm[m].s[c].x + __shfl_xor_sync(FULL, pm[m].s[c].x, 16);
                    v1 = pm[m].ss[c].x + __shfl_xor_sync(FULL, pm[m].ss[c].x, 16);
                    v2 = pm[m].sy[c].x + __shfl_xor_sync(FULL, pm[m].sy[c].x, 16);
                } else {
                    v0 = pm[m].s[c].x + pm[m].s[c].y;
                    v1 = pm[m].ss[c].x + pm[m].ss[c].y;
                    v2 = pm[m].sy[c].x + pm[m].sy[c].y;
                }
                if (!upper) {
                    v0 += rb[(3 * c + 0) * 32 + lane];
                    v1 += rb[(3 * c + 1) * 32 + lane];
                    v2 += rb[(3 * c + 2) * 32 + lane];
                }
                rb[(3 * c + 0) * 32 + lane] = v0;
                rb[(3 * c + 1) * 32 + lane] = v1;
                rb[(3 * c + 2) * 32 + lane] = v2;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(upper ? half_full : red_full);
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
    const int tt = targets_per_tile(prec, 32);
    const int n_tiles = (N_tgt + tt - 1) / tt;
    return (static_cast<uint64_t>(ceil_log2(L)) << 24) | (static_cast<uint64_t>(ceil_log2(n_tiles)) << 16) |
           (static_cast<uint64_t>(ceil_log2(nlib)) << 8) | static_cast<uint64_t>(prec);
}

edm_status launch_lookup(edm_ctx *ctx, const uint8_t *Yt, int N_tgt, int L, const uint8_t *tables,
                         const CcmGroups &g, int lib0, int nlib, int tau, int Tp,
                         edm_precision prec, int rw, const double *ysum, const double *yysum,
                         float *rho, long long rho_ld, const int32_t *rho_col) {
    const bool pk = prec != EDM_FP32;  // two 16-bit targets per word
    const bool half = rw == 16;
    const int tt = targets_per_tile(prec, rw);
    const int n_tiles = (N_tgt + tt - 1) / tt;
    const int threads = pk ? LkCfg<EDM_BF16_TARGETS>::THREADS : LkCfg<EDM_FP32>::THREADS;
    const int G = pk ? LkCfg<EDM_BF16_TARGETS>::G : LkCfg<EDM_FP32>::G;
    if (g.G != G) return set_error(ctx, EDM_ERR_INTERNAL, "lookup: group size mismatch");
    const size_t red_bytes =
        sizeof(float) * (pk ? LkCfg<EDM_BF16_TARGETS>::RED_FLOATS : LkCfg<EDM_FP32>::RED_FLOATS);
    const size_t tile_bytes = static_cast<size_t>(L + 1) * 4 * rw;
    const size_t fixed = red_bytes + (2 * LK_MAX_STAGES + 6) * sizeof(uint64_t);
    const size_t limit = static_cast<size_t>(ctx->max_smem_optin);
    // stages of 6 KB (4 KB when the tile leaves less room); at least two
    const size_t min_stage = 4096, big_stage = 6144;
    const bool smem_tile = tile_bytes + fixed + 2 * min_stage <= limit && tile_bytes < (1u << 20);
    if (half && !smem_tile) return set_error(ctx, EDM_ERR_INTERNAL, "lookup: half tile does not fit");
    const size_t avail = limit - fixed - (smem_tile ? tile_bytes : 0);
    const size_t stage_bytes = avail >= 2 * big_stage ? big_stage : min_stage;
    const int stages = static_cast<int>(std::min<size_t>(LK_MAX_STAGES, avail / stage_bytes));
    if (stages < 2) return set_error(ctx, EDM_ERR_INTERNAL, "lookup: no room for table stages");
    const size_t smem = (smem_tile ? tile_bytes : 0) + static_cast<size_t>(stages) * stage_bytes +
                        red_bytes + (2 * stages + 6) * sizeof(uint64_t);

    // libraries per CTA: a fixed override, else the autotuned value of this
    // launch's bucket, else the heuristic; a CTA takes lb / G groups
    long long lb = lookup_default_lb(ctx, nlib, n_tiles);
    if (ctx->lookup_lb > 0) {
        lb = std::min(ctx->lookup_lb, nlib);
    } else if (ctx->autotune && ctx->tune) {
        auto it = ctx->tune->find(lookup_bucket(L, N_tgt, nlib, prec));
        if (it != ctx->tune->end()) lb = std::min(it->second, nlib);
    }
    const int GB = static_cast<int>(std::max<long long>(1, lb / G));
    LookupArgs a;
    a.Yt = Yt;
    a.tables = tables;
    a.grp = g;
    a.ysum = ysum;
    a.yysum = yysum;
    a.lib0 = lib0;
    a.GB = GB;
    a.L = L;
    a.tau = tau;
    a.Tp = Tp;
    a.N_tgt = N_tgt;
    a.stages = stages;
    a.stage_bytes = static_cast<int>(stage_bytes);
    a.rho = rho;
    a.rho_ld = rho_ld;
    a.rho_col = rho_col;
    a.flags = ctx->d_flags;
    dim3 grid(n_tiles, static_cast<unsigned>((g.ngroups_max + GB - 1) / GB));
    void (*kern)(const LookupArgs);
    switch (prec) {
    case EDM_BF16_TARGETS:
        kern = half ? lookup_kernel<EDM_BF16_TARGETS, true, true>
                    : (smem_tile ? lookup_kernel<EDM_BF16_TARGETS, true, false>
                                 : lookup_kernel<EDM_BF16_TARGETS, false, false>);
        break;
    case EDM_FP16_TARGETS:
        kern = half ? lookup_kernel<EDM_FP16_TARGETS, true, true>
                    : (smem_tile ? lookup_kernel<EDM_FP16_TARGETS, true, false>
                                 : lookup_kernel<EDM_FP16_TARGETS, false, false>);
        break;
    default:
        kern = half ? lookup_kernel<EDM_FP32, true, true>
                    : (smem_tile ? lookup_kernel<EDM_FP32, true, false>
                                 : lookup_kernel<EDM_FP32, false, false>);
        break;
    }
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    before_launch(ctx);
    kern<<<grid, threads, smem, ctx->stream>>>(a);
    return after_launch(ctx, "lookup_kernel");
}

}  // namespace edm
