"""GPU parity of the embedding and the exhaustive kNN against the FP64 oracle.

Neighbour indices must match bit for bit (time index, order by (s, u));
distances must equal the oracle's FP64 distance rounded to float32.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_12301_gb300 import edm, inputs

pytestmark = pytest.mark.gpu


def gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check_knn(X, E, tau, Tp, k=None):
    X = np.atleast_2d(np.asarray(X, np.float32))
    k = E + 1 if k is None else k
    idx, dist = edm.edm_knn(gpu(X), E, tau, Tp, k)
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    for s in range(X.shape[0]):
        oi, od = oracle.knn(X[s], E, tau, Tp, k)
        np.testing.assert_array_equal(idx[s], oi, err_msg="series %d E=%d tau=%d Tp=%d k=%d"
                                      % (s, E, tau, Tp, k))
        np.testing.assert_array_equal(dist[s], od.astype(np.float32))


def test_embed_matches_oracle():
    x = inputs.logistic_16x200()[3]
    for E, tau in [(1, 1), (3, 1), (5, 7), (20, 2)]:
        out = edm.edm_embed(gpu(x), E, tau).cpu().numpy()
        np.testing.assert_array_equal(out, oracle.embed(x, E, tau).astype(np.float32))


@pytest.mark.parametrize("E", [1, 2, 3, 5, 8, 13, 20])
def test_knn_matches_oracle_across_E(E):
    X = inputs.logistic_16x200()[:3]
    check_knn(X, E, 1, 0)
    check_knn(X, E, 2, 1)


@pytest.mark.parametrize("L,tau,Tp,k", [(12, 1, 0, 1), (33, 3, 4, None), (57, 1, 1, 24),
                                        (97, 2, 0, 3), (1000, 1, 0, None)])
def test_knn_ragged_sizes_and_k(L, tau, Tp, k):
    X = inputs.coupled_logistic(2, L, 31)
    E = 3
    n = L - (E - 1) * tau - Tp
    kk = min(k, n - 1) if k is not None else None
    check_knn(X, E, tau, Tp, kk)


def test_knn_exact_ties_on_a_grid():
    rng = np.random.default_rng(5)
    for L in (16, 40, 130):
        x = (rng.integers(0, 4, L) * 0.5).astype(np.float32)
        for E in (1, 2, 4):
            check_knn(x, E, 1, 0)
            check_knn(x, E, 2, 1, k=min(E + 8, L - (E - 1) * 2 - 2))


def test_knn_constant_series_takes_lowest_indices():
    # every distance is 0: the band holds all points (brute-force FP64 path)
    x = np.full(300, 0.75, np.float32)
    check_knn(x, 2, 1, 0)


def test_knn_repeated_pattern_near_ties():
    # a period-7 pattern with tiny noise: many near-equal distances, exercises
    # the band re-rank
    t = np.arange(800)
    x = (np.sin(2 * np.pi * t / 7) + 1e-6 * np.random.default_rng(1).standard_normal(800))
    check_knn(x.astype(np.float32), 3, 1, 0)
    check_knn(x.astype(np.float32), 6, 1, 1)


def test_knn_many_series_full_table():
    X = inputs.logistic_noisy(N=24, L=300)
    check_knn(X, 4, 1, 0)


def test_knn_long_series_sampled_rows():
    # 30,000 points: the series is read from global memory (not staged)
    x = inputs.coupled_logistic(1, 30000, 77)[0]
    E, tau, Tp = 4, 1, 0
    idx, dist = edm.edm_knn(gpu(x[None]), E, tau, Tp)
    idx, dist = idx[0].cpu().numpy(), dist[0].cpu().numpy()
    for t in (3, 4, 999, 15000, 29999):
        oi, od = oracle.knn_row(x, E, tau, Tp, t)
        np.testing.assert_array_equal(idx[t - 3], oi)
        np.testing.assert_array_equal(dist[t - 3], od.astype(np.float32))


def test_knn_rejects_bad_arguments():
    X = gpu(inputs.logistic_16x200()[:1])
    with pytest.raises(edm.EdmError):
        edm.edm_knn(X, 21, 1, 0)          # E above EDM_E_MAX
    with pytest.raises(edm.EdmError):
        edm.edm_knn(X, 2, 1, 0, k=25)     # k above EDM_K_MAX
    with pytest.raises(edm.EdmError):
        edm.edm_knn(gpu(np.zeros((1, 4), np.float32)), 2, 1, 0, k=3)  # too few points


@pytest.mark.parametrize("E,tau,Tp,k", [(1, 1, 0, 2), (3, 2, 1, 4), (12, 1, 0, 13), (20, 1, 2, 24)])
def test_knn_chunked_long_series_exact_order(E, tau, Tp, k):
    # 2,048 < L: candidates in chunks of 1,024 against a running list; the
    # exact FP64 order, also for k != E+1 and at the largest k
    x = inputs.coupled_logistic(1, 5000, 300 + E)[0]
    x[1000:1010] = x[2000:2010]                      # exact repeats: ties
    idx, dist = edm.edm_knn(gpu(x[None]), E, tau, Tp, k=k)
    idx, dist = idx[0].cpu().numpy(), dist[0].cpu().numpy()
    lo = (E - 1) * tau
    for t in (lo, lo + 1, 1005, 2005, 4000, 5000 - 1 - Tp):
        oi, od = oracle.knn_row(x, E, tau, Tp, t, k=k)
        np.testing.assert_array_equal(idx[t - lo], oi)
        np.testing.assert_array_equal(dist[t - lo], od.astype(np.float32))


@pytest.mark.parametrize("L,E,tau,Tp", [(300, 1, 1, 0), (300, 3, 2, 1), (2100, 2, 1, 0),
                                         (2100, 7, 1, 0)])
def test_materialized_baseline_equals_fused_knn_and_oracle(L, E, tau, Tp):
    # the paper's two-kernel route (distance matrix in memory, then per-row
    # selection) gives exactly edm_knn's neighbours and distances, and the
    # oracle's on sampled rows
    X = inputs.coupled_logistic(3, L, 77 + L + E)
    Xg = gpu(X)
    i_f, d_f = edm.edm_knn(Xg, E, tau, Tp)
    i_m, d_m = edm.edm_knn_materialized(Xg, E, tau, Tp)
    edm.edm_ctx_sync()
    torch.testing.assert_close(i_m, i_f, rtol=0, atol=0)
    torch.testing.assert_close(d_m, d_f, rtol=0, atol=0)
    i_m = i_m.cpu().numpy()
    t0 = (E - 1) * tau
    n = L - t0 - Tp
    for s in range(3):
        for i in (0, 1, n // 2, n - 1):
            oi, _ = oracle.knn_row(X[s], E, tau, Tp, t0 + i)
            np.testing.assert_array_equal(i_m[s, i], oi)
