// predict.cu -- simplex predictions written out (kEDM Algorithm 3's output,
// section 2.1 step 3): for each library i and its target j, the prediction
// Yhat_j(t+Tp) = sum_r w_r Y_j[u_r+Tp] over the k = E_i+1 nearest neighbours
// u_r of x_i(t), for every t in P.  The neighbour tables are the CCM tables
// (exact neighbour sets, normalised weights) in their grouped layout; one
// thread per output time reads its table row and gathers the target.
#include "edm_internal.cuh"

namespace edm {

constexpr int PRED_THREADS = 256;

// pred[lib - lib0][v] for v in [0, L): the prediction of time v when
// v = t + Tp for a query time t of the library, else NaN.  A library whose E
// or target index is out of range gets a NaN row and raises the flag.
__global__ void __launch_bounds__(PRED_THREADS)
    predict_kernel(const float *__restrict__ Y, long long ld_tgt, int N_tgt,
                   const int32_t *__restrict__ tgt_of, int L, int tau, int Tp, const CcmGroups g,
                   const uint8_t *__restrict__ tables,
                   int lib0, float *__restrict__ pred, long long ld_pred, int *flags) {
    const int s = blockIdx.x;
    const int lib = g.lib[s];
    if (lib < 0) return;
    const int gi = s / g.G, m = s % g.G;
    if (m >= g.n[gi]) return;  // a repeated member of a partial group
    const int E = g.E[gi];
    float *out = pred + static_cast<long long>(lib - lib0) * ld_pred;
    const int v = blockIdx.y * PRED_THREADS + threadIdx.x;
    if (v >= L) return;
    const float nan = __int_as_float(0x7fc00000);
    const int j = tgt_of ? tgt_of[lib] : lib;
    if (E == 0 || j < 0 || j >= N_tgt) {
        out[v] = nan;
        if (v == 0) set_flag(flags, EDMF_BADARG);
        return;
    }
    const int t0 = (E - 1) * tau, n = L - t0 - Tp;
    const int i = v - Tp - t0;  // table row of query time v - Tp
    if (i < 0 || i >= n) {
        out[v] = nan;
        return;
    }
    const int K = E + 1;
    const int pb = table_pair_bytes(K);
    const uint32_t *blk = reinterpret_cast<const uint32_t *>(
        tables + g.off[gi] + (static_cast<size_t>(i >> 1) * g.G + m) * pb);
    const int h = i & 1;
    const float *y = Y + static_cast<long long>(j) * ld_tgt;
    // neighbour rows are stored shifted by Tp; the K-th weight is 1 minus the others
    auto nbr = [&](int q) {
        const uint32_t w = blk[2 * (K - 1 + (q >> 1)) + h];
        return static_cast<int>((q & 1) ? (w >> 16) : (w & 0xffffu));
    };
    const float y_last = y[nbr(K - 1)];
    float acc = y_last;
    for (int q = 0; q < K - 1; ++q) {
        const float w = __uint_as_float(blk[2 * q + h]);
        acc = __fmaf_rn(w, __fsub_rn(y[nbr(q)], y_last), acc);
    }
    out[v] = acc;
}

edm_status launch_predict(edm_ctx *ctx, const float *Y, long long ld_tgt, int N_tgt,
                          const int32_t *tgt_of, int L, int tau, int Tp, const CcmGroups &g,
                          const uint8_t *tables, int lib0, float *pred, long long ld_pred) {
    dim3 grid(g.ngroups_max * g.G, (L + PRED_THREADS - 1) / PRED_THREADS);
    before_launch(ctx);
    predict_kernel<<<grid, PRED_THREADS, 0, ctx->stream>>>(Y, ld_tgt, N_tgt, tgt_of, L, tau, Tp, g,
                                                           tables, lib0, pred, ld_pred, ctx->d_flags);
    return after_launch(ctx, "predict_kernel");
}

}  // namespace edm
