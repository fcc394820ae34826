/*
 * edm_oracle.c -- plain, slow FP64 CPU oracle for convergent cross mapping
 * (CCM) as stated in kEDM (Takahashi et al., PEARC'21), section 2.1
 * "Empirical Dynamic Modeling", steps 1-4, and the lookup-table reuse of
 * section 2.1's closing paragraph.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this code.  It shares nothing with the CUDA path:
 * no headers, no helpers, no tables.  Every function below is the plain
 * definition written out, one candidate at a time, in double precision.
 *
 * Conventions (readings of the paper, listed again in the design notes):
 *  - Inputs are float32 series; they are widened to double on read.
 *  - Embedding time labels: a point exists for t = (E-1)*tau .. L-1 and its
 *    l-th coordinate is X[t - l*tau], l = 0..E-1 (section 2.1 step 1).
 *  - The library set equals the prediction set:
 *      P = { t : (E-1)*tau <= t <= L-1-Tp },  n = |P| = L-(E-1)*tau-Tp.
 *    A query point is never its own neighbour (leave-one-out).
 *  - Distances are ranked on the squared distance s, accumulated in lag order
 *    l = 0..E-1 with fma(d, d, s); ties go to the lower time index.
 *  - k = E+1 neighbours; weights w_r = exp(-d_r / d_1) with d_1 the nearest
 *    distance (the paper's min over 1..E is read as the min over all
 *    neighbours); if d_1 == 0 then w_r = 1 for d_r == 0 and 0 otherwise.
 *  - Pearson's rho is two-pass; zero variance gives NaN.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math), so
 * that no multiply-add is fused except the explicit fma() calls.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* Number of points in P (section 2.1 steps 1-2 with the leave-one-out
 * library = prediction set reading).  Non-positive means "no points". */
int oracle_n_rows(int L, int E, int tau, int Tp)
{
    return L - (E - 1) * tau - Tp;
}

/* Section 2.1 step 1: time-delay embedding.
 * out is [L-(E-1)*tau][E] row-major, row i is the point at time t=(E-1)tau+i,
 * column l is X[t - l*tau]. */
int oracle_embed(const float *X, int L, int E, int tau, double *out)
{
    if (!X || !out || L < 1 || E < 1 || tau < 1)
        return ORACLE_EINVAL;
    int t0 = (E - 1) * tau;
    if (t0 >= L)
        return ORACLE_EINVAL;
    for (int t = t0; t < L; ++t)
        for (int l = 0; l < E; ++l)
            out[(size_t)(t - t0) * E + l] = (double)X[t - l * tau];
    return ORACLE_OK;
}

/* Section 2.1 step 2: squared Euclidean distance between the embedded points
 * at times t and u, lag order 0..E-1, one fma per lag. */
static double sq_dist(const float *X, int t, int u, int E, int tau)
{
    double s = 0.0;
    for (int l = 0; l < E; ++l) {
        double d = (double)X[t - l * tau] - (double)X[u - l * tau];
        s = fma(d, d, s);
    }
    return s;
}

/* Lexicographic order on (s, u): smaller distance first, then lower index. */
static int key_less(double sa, int ua, double sb, int ub)
{
    return sa < sb || (sa == sb && ua < ub);
}

/* Section 2.1 step 2 for one query time t: the k nearest points of P\{t},
 * ascending.  Selection is k passes of "smallest key greater than the last
 * one taken", which needs no sort and is plainly correct. */
static void knn_one_row(const float *X, int t, int lo, int hi, int E, int tau,
                        int k, double *s_all, int32_t *idx, double *dist)
{
    for (int u = lo; u <= hi; ++u)
        s_all[u - lo] = sq_dist(X, t, u, E, tau);
    double last_s = -1.0;
    int last_u = -1;
    for (int r = 0; r < k; ++r) {
        double best_s = INFINITY;
        int best_u = -1;
        for (int u = lo; u <= hi; ++u) {
            if (u == t)
                continue;
            double s = s_all[u - lo];
            if (r > 0 && !key_less(last_s, last_u, s, u))
                continue; /* already taken */
            if (best_u < 0 || key_less(s, u, best_s, best_u)) {
                best_s = s;
                best_u = u;
            }
        }
        idx[r] = best_u;
        dist[r] = sqrt(best_s);
        last_s = best_s;
        last_u = best_u;
    }
}

static int knn_args_ok(const float *X, int L, int E, int tau, int Tp, int k)
{
    if (!X || L < 2 || E < 1 || tau < 1 || Tp < 0 || k < 1)
        return 0;
    int n = oracle_n_rows(L, E, tau, Tp);
    return n >= 2 && k <= n - 1;
}

/* Section 2.1 step 2 (all-kNN table, precomputed once per library as in the
 * closing paragraph of section 2.1).  idx/dist are [n][k]; idx holds time
 * indices u, dist holds sqrt(s) in double. */
int oracle_knn(const float *X, int L, int E, int tau, int Tp, int k,
               int32_t *idx, double *dist)
{
    if (!knn_args_ok(X, L, E, tau, Tp, k) || !idx || !dist)
        return ORACLE_EINVAL;
    int lo = (E - 1) * tau, hi = L - 1 - Tp, n = hi - lo + 1;
    double *s_all = (double *)malloc(sizeof(double) * (size_t)n);
    if (!s_all)
        return ORACLE_ENOMEM;
    for (int t = lo; t <= hi; ++t)
        knn_one_row(X, t, lo, hi, E, tau, k, s_all, idx + (size_t)(t - lo) * k,
                    dist + (size_t)(t - lo) * k);
    free(s_all);
    return ORACLE_OK;
}

/* One row of oracle_knn, for sampling very long series. */
int oracle_knn_row(const float *X, int L, int E, int tau, int Tp, int k, int t,
                   int32_t *idx, double *dist)
{
    if (!knn_args_ok(X, L, E, tau, Tp, k) || !idx || !dist)
        return ORACLE_EINVAL;
    int lo = (E - 1) * tau, hi = L - 1 - Tp;
    if (t < lo || t > hi)
        return ORACLE_EINVAL;
    double *s_all = (double *)malloc(sizeof(double) * (size_t)(hi - lo + 1));
    if (!s_all)
        return ORACLE_ENOMEM;
    knn_one_row(X, t, lo, hi, E, tau, k, s_all, idx, dist);
    free(s_all);
    return ORACLE_OK;
}

/* Section 2.1 step 3: simplex weights of one row of ascending distances,
 * normalised to sum 1.  d_1 = dist[0] is the nearest distance. */
void oracle_weights(const double *dist, int k, double *w)
{
    double d1 = dist[0], sum = 0.0;
    for (int r = 0; r < k; ++r) {
        if (d1 > 0.0)
            w[r] = exp(-dist[r] / d1);
        else
            w[r] = (dist[r] == 0.0) ? 1.0 : 0.0;
        sum += w[r];
    }
    for (int r = 0; r < k; ++r)
        w[r] /= sum;
}

/* Section 2.1 step 3 (lookup): prediction of Y(t+Tp) for every t in P from
 * the neighbour table, and the observed value Y(t+Tp).  pred/obs are [n]. */
int oracle_predict(const int32_t *idx, const double *dist, int n, int k,
                   const float *Y, int t0, int Tp, double *pred, double *obs)
{
    if (!idx || !dist || !Y || !pred || !obs || n < 1 || k < 1)
        return ORACLE_EINVAL;
    double *w = (double *)malloc(sizeof(double) * (size_t)k);
    if (!w)
        return ORACLE_ENOMEM;
    for (int i = 0; i < n; ++i) {
        oracle_weights(dist + (size_t)i * k, k, w);
        double p = 0.0;
        for (int r = 0; r < k; ++r)
            p += w[r] * (double)Y[idx[(size_t)i * k + r] + Tp];
        pred[i] = p;
        obs[i] = (double)Y[t0 + i + Tp];
    }
    free(w);
    return ORACLE_OK;
}

/* Section 2.1 step 4: Pearson's correlation, two passes. */
double oracle_pearson(const double *a, const double *b, int n)
{
    if (n < 1)
        return NAN;
    double ma = 0.0, mb = 0.0;
    for (int i = 0; i < n; ++i) {
        ma += a[i];
        mb += b[i];
    }
    ma /= n;
    mb /= n;
    double sab = 0.0, saa = 0.0, sbb = 0.0;
    for (int i = 0; i < n; ++i) {
        double da = a[i] - ma, db = b[i] - mb;
        sab += da * db;
        saa += da * da;
        sbb += db * db;
    }
    if (saa == 0.0 || sbb == 0.0)
        return NAN;
    return sab / sqrt(saa * sbb);
}

/* Section 2.1 steps 1-4 for one library X and many targets Y[N_tgt][L]:
 * the kNN table of X is built once and reused for every target.
 * rho[j] = skill of X's manifold at predicting target j. */
int oracle_ccm_row(const float *X, const float *Y, int N_tgt, int L, int E,
                   int tau, int Tp, double *rho)
{
    int k = E + 1;
    if (!knn_args_ok(X, L, E, tau, Tp, k) || !Y || !rho || N_tgt < 0)
        return ORACLE_EINVAL;
    int n = oracle_n_rows(L, E, tau, Tp), t0 = (E - 1) * tau;
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * k);
    double *dist = (double *)malloc(sizeof(double) * (size_t)n * k);
    double *pred = (double *)malloc(sizeof(double) * (size_t)n);
    double *obs = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = ORACLE_ENOMEM;
    if (idx && dist && pred && obs) {
        rc = oracle_knn(X, L, E, tau, Tp, k, idx, dist);
        for (int j = 0; rc == ORACLE_OK && j < N_tgt; ++j) {
            rc = oracle_predict(idx, dist, n, k, Y + (size_t)j * L, t0, Tp,
                                pred, obs);
            if (rc == ORACLE_OK)
                rho[j] = oracle_pearson(pred, obs, n);
        }
    }
    free(idx);
    free(dist);
    free(pred);
    free(obs);
    return rc;
}

/* Simplex projection of a series onto itself: CCM with target = library. */
double oracle_simplex_rho(const float *X, int L, int E, int tau, int Tp)
{
    double rho = NAN;
    if (oracle_ccm_row(X, X, 1, L, E, tau, Tp, &rho) != ORACLE_OK)
        return NAN;
    return rho;
}

/* Argmax of the skills rho_E[0..E_max-1] of E = 1..E_max (section 3.3 names
 * the optimal E without defining it; the reading is argmax rho_E).  A NaN skill
 * ranks below every number; among equal skills the smallest E wins; when every
 * skill is NaN the result is 1. */
int oracle_argmax_E(const double *rho_E, int E_max)
{
    int best_E = 1;
    double best = NAN;
    for (int E = 1; E <= E_max; ++E) {
        double r = rho_E[E - 1];
        if (isnan(r))
            continue;
        if (isnan(best) || r > best) { /* strictly greater: ties keep the smaller E */
            best = r;
            best_E = E;
        }
    }
    return best_E;
}

/* Optimal embedding dimension by simplex projection over E = 1..E_max
 * (named but not specified in section 3.3; the reading is leave-one-out
 * simplex at horizon Tp_sel).  rho_E[E-1] receives each skill (NaN when E
 * leaves fewer than E+2 points); E_opt is oracle_argmax_E of them.  rho_E may
 * be NULL. */
int oracle_optimal_E(const float *X, int L, int E_max, int tau, int Tp_sel,
                     int32_t *E_opt, double *rho_E)
{
    if (!X || !E_opt || L < 2 || E_max < 1 || tau < 1 || Tp_sel < 0)
        return ORACLE_EINVAL;
    double *r = (double *)malloc(sizeof(double) * (size_t)E_max);
    if (!r)
        return ORACLE_ENOMEM;
    for (int E = 1; E <= E_max; ++E) {
        r[E - 1] = NAN;
        if (knn_args_ok(X, L, E, tau, Tp_sel, E + 1))
            r[E - 1] = oracle_simplex_rho(X, L, E, tau, Tp_sel);
        if (rho_E)
            rho_E[E - 1] = r[E - 1];
    }
    *E_opt = oracle_argmax_E(r, E_max);
    free(r);
    return ORACLE_OK;
}
