"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks the oracle against brute force on tiny inputs, a library
routine (scipy's KD-tree), closed forms, invariants, or the qualitative
behaviour the paper states for CCM (section 2.1).  Together they are chosen so
that a dropped term, a wrong sign, an off-by-one in the lag or time index, or
a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_12301_gb300 import inputs


# ---------------------------------------------------------------------------
# independent brute force (numpy): explicit embedding matrix, full sort
# ---------------------------------------------------------------------------

def brute_points(x, E, tau, Tp):
    """Explicit delay vectors of every point in P; row i is time t0+i."""
    x = np.asarray(x, np.float64)
    t0 = (E - 1) * tau
    ts = np.arange(t0, len(x) - Tp)
    pts = np.stack([x[ts - l * tau] for l in range(E)], axis=1)
    return ts, pts


def brute_knn(x, E, tau, Tp, k):
    ts, pts = brute_points(x, E, tau, Tp)
    idx = np.empty((len(ts), k), np.int64)
    dist = np.empty((len(ts), k))
    for i, t in enumerate(ts):
        s = ((pts - pts[i]) ** 2).sum(axis=1)
        order = np.lexsort((ts, s))          # by s, then by time index
        order = order[ts[order] != t][:k]    # the point itself is excluded
        idx[i] = ts[order]
        dist[i] = np.sqrt(s[order])
    return idx, dist


def brute_ccm(x_lib, y, E, tau, Tp):
    """Brute-force cross map skill: explicit kNN, weights, prediction, corrcoef."""
    idx, dist = brute_knn(x_lib, E, tau, Tp, E + 1)
    y = np.asarray(y, np.float64)
    d1 = dist[:, :1]
    with np.errstate(divide="ignore", invalid="ignore"):
        w = np.where(d1 > 0, np.exp(-dist / np.where(d1 > 0, d1, 1.0)),
                     (dist == 0).astype(float))
    w /= w.sum(axis=1, keepdims=True)
    pred = (w * y[idx + Tp]).sum(axis=1)
    t0 = (E - 1) * tau
    obs = y[t0 + Tp: len(y)][: len(pred)]
    return np.corrcoef(pred, obs)[0, 1]


# ---------------------------------------------------------------------------
# embedding
# ---------------------------------------------------------------------------

def test_embed_is_lagged_copies():
    x = np.arange(10, dtype=np.float32)
    emb = oracle.embed(x, 3, 2)
    # point at time t is (t, t-2, t-4): rows start at t0 = 4
    assert emb.shape == (6, 3)
    np.testing.assert_array_equal(emb[0], [4, 2, 0])
    np.testing.assert_array_equal(emb[-1], [9, 7, 5])


# ---------------------------------------------------------------------------
# kNN: brute force with exact ties, scipy KD-tree on continuous data
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_knn_brute_force_tiny_with_ties(seed):
    rng = np.random.default_rng(seed)
    for L in range(5, 13):
        # values on a coarse dyadic grid: many exact distance ties, all
        # arithmetic exact in both implementations
        x = (rng.integers(0, 4, L) * 0.5).astype(np.float32)
        for E in range(1, 5):
            for tau in (1, 2):
                for Tp in (0, 1):
                    n = L - (E - 1) * tau - Tp
                    if n < 3:
                        continue
                    for k in sorted({1, min(E + 1, n - 1), n - 1}):
                        idx, dist = oracle.knn(x, E, tau, Tp, k)
                        bidx, bdist = brute_knn(x, E, tau, Tp, k)
                        np.testing.assert_array_equal(idx, bidx)
                        np.testing.assert_array_equal(dist, bdist)


def test_knn_matches_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(7)
    x = rng.standard_normal(300).astype(np.float32)
    for E, tau, Tp in [(1, 1, 0), (2, 1, 1), (3, 2, 0), (5, 1, 2), (4, 3, 1)]:
        k = E + 1
        ts, pts = brute_points(x, E, tau, Tp)
        tree = spatial.cKDTree(pts)
        d, j = tree.query(pts, k=k + 1)       # includes the point itself
        idx, dist = oracle.knn(x, E, tau, Tp, k)
        assert np.all(j[:, 0] == np.arange(len(ts)))
        np.testing.assert_array_equal(idx, ts[j[:, 1:]])
        np.testing.assert_allclose(dist, d[:, 1:], rtol=1e-12, atol=1e-12)


def test_knn_row_equals_table_row():
    x = inputs.logistic_map(120)
    idx, dist = oracle.knn(x, 3, 2, 1)
    for t in (4, 50, 118):
        i2, d2 = oracle.knn_row(x, 3, 2, 1, t)
        np.testing.assert_array_equal(i2, idx[t - 4])
        np.testing.assert_array_equal(d2, dist[t - 4])


def test_knn_constant_series_ties_to_lowest_index():
    x = np.full(20, 1.5, np.float32)
    idx, dist = oracle.knn(x, 2, 1, 0)
    assert np.all(dist == 0)
    # row of time t takes the three lowest times of P other than t
    for i, t in enumerate(range(1, 20)):
        expect = [u for u in range(1, 20) if u != t][:3]
        assert list(idx[i]) == expect


def test_knn_rejects_too_few_points():
    with pytest.raises(ValueError):
        oracle.knn(np.zeros(5, np.float32), 3, 1, 1, k=4)


# ---------------------------------------------------------------------------
# weights (closed form) and the lookup
# ---------------------------------------------------------------------------

def test_weights_closed_form():
    w = oracle.weights([1.0, 2.0, 3.0])
    e = np.exp([-1.0, -2.0, -3.0])
    np.testing.assert_allclose(w, e / e.sum(), rtol=1e-15)
    # nearest at distance 0: all weight on the exact matches, shared equally
    np.testing.assert_array_equal(oracle.weights([0.0, 0.0, 1.0]), [0.5, 0.5, 0.0])
    # scale invariance: d / d_1 only depends on ratios
    np.testing.assert_allclose(oracle.weights([0.5, 1.0, 1.5]), e / e.sum(),
                               rtol=1e-15)


def test_lookup_closed_form_one_row():
    # E=1, tau=1, Tp=0: the point X=0 (time 0) has neighbours X=1 (time 1,
    # distance 1) and X=3 (time 2, distance 3); k = 2.
    x = np.array([0.0, 1.0, 3.0, 7.0, 15.0], np.float32)
    y = np.array([10.0, 20.0, 40.0, 80.0, 160.0], np.float32)
    idx, dist = oracle.knn(x, 1, 1, 0)
    assert list(idx[0]) == [1, 2]
    np.testing.assert_array_equal(dist[0], [1.0, 3.0])
    pred, obs = oracle.predict(idx, dist, y, 0, 0)
    w1, w2 = math.exp(-1.0), math.exp(-3.0)
    assert pred[0] == pytest.approx((w1 * 20 + w2 * 40) / (w1 + w2), rel=1e-15)
    assert obs[0] == 10.0


def test_lookup_horizon_shifts_both_prediction_and_observation():
    # with Tp=1 the neighbour values are read one step ahead and so is the
    # observation: on y = time index, every neighbour u contributes u+1
    x = inputs.logistic_map(60)
    y = np.arange(60, dtype=np.float32)
    idx, dist = oracle.knn(x, 2, 1, 1)
    pred, obs = oracle.predict(idx, dist, y, 1, 1)
    for i in range(len(pred)):
        w = oracle.weights(dist[i])
        assert pred[i] == pytest.approx((w * (idx[i] + 1)).sum(), rel=1e-14)
        assert obs[i] == 1 + i + 1


# ---------------------------------------------------------------------------
# Pearson
# ---------------------------------------------------------------------------

def test_pearson_matches_numpy_and_special_cases():
    rng = np.random.default_rng(3)
    for n in (2, 3, 17, 1000):
        a, b = rng.standard_normal((2, n))
        assert oracle.pearson(a, b) == pytest.approx(np.corrcoef(a, b)[0, 1],
                                                      abs=1e-14)
    a = rng.standard_normal(50)
    assert oracle.pearson(a, 3 * a + 2) == pytest.approx(1.0, abs=1e-15)
    assert oracle.pearson(a, -0.5 * a + 1) == pytest.approx(-1.0, abs=1e-15)
    assert math.isnan(oracle.pearson(a, np.full(50, 4.0)))


# ---------------------------------------------------------------------------
# whole pipeline
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("E,tau,Tp", [(1, 1, 0), (2, 1, 1), (3, 2, 0), (4, 1, 2)])
def test_ccm_matches_brute_force(E, tau, Tp):
    X = inputs.coupled_logistic(3, 40, 11)
    for i in range(3):
        rho = oracle.ccm_row(X[i], X, E, tau, Tp)
        for j in range(3):
            assert rho[j] == pytest.approx(brute_ccm(X[i], X[j], E, tau, Tp),
                                           abs=1e-12)


def test_simplex_logistic_map_high_skill():
    # noise-free logistic map, r=3.8, L=500: simplex E=2, Tp=1 predicts well
    x = inputs.logistic_map(500)
    assert oracle.simplex_rho(x, 2, 1, 1) > 0.99


def test_ccm_self_map_equals_simplex():
    X = inputs.logistic_16x200()
    for i in (0, 5):
        for E in (1, 3, 6):
            row = oracle.ccm_row(X[i], X[i], E, 1, 0)
            # simplex built step by step from the parts
            idx, dist = oracle.knn(X[i], E, 1, 0)
            pred, obs = oracle.predict(idx, dist, X[i], E - 1, 0)
            assert row[0] == oracle.pearson(pred, obs)
            assert row[0] == oracle.simplex_rho(X[i], E, 1, 0)


def test_ccm_affine_invariance_of_target():
    X = inputs.coupled_logistic(2, 150, 5)
    # dyadic grid so that a*y + b is exact in float32
    y = (np.round(X[1].astype(np.float64) * 1024) / 1024).astype(np.float32)
    base = oracle.ccm_row(X[0], y, 3, 1, 0)[0]
    for a, b in [(2.0, 0.25), (4.0, -1.0), (0.5, 3.0), (-2.0, 0.5)]:
        ya = (a * y.astype(np.float64) + b).astype(np.float32)
        assert np.array_equal(ya.astype(np.float64), a * y.astype(np.float64) + b)
        r = oracle.ccm_row(X[0], ya, 3, 1, 0)[0]
        # prediction and observation are both a*y + b: rho is unchanged even
        # for a < 0 (both signs flip)
        assert r == pytest.approx(base, abs=1e-12)


def test_shuffled_target_has_no_skill():
    X = inputs.logistic_pair(400, 3)
    rng = np.random.default_rng(0)
    rhos = []
    for _ in range(20):
        y = X[0][rng.permutation(400)]
        rhos.append(oracle.ccm_row(X[1], y, 2, 1, 0)[0])
    rhos = np.array(rhos)
    n = 399
    assert np.all(np.abs(rhos) < 5.0 / math.sqrt(n))
    assert abs(rhos.mean()) < 3.0 / math.sqrt(20 * n)
    # the unshuffled driver is recovered well
    assert oracle.ccm_row(X[1], X[0], 2, 1, 0)[0] > 0.5


def test_ccm_direction_and_convergence():
    # x drives y (b_yx = 0.1, b_xy = 0).  Section 2.1: high skill of library
    # Y's manifold at predicting X means "X CCM-causes Y".  So library y must
    # cross-map the driver x better than library x cross-maps y, and that
    # skill must grow with the library length.
    X = inputs.logistic_pair(400, 1)
    x, y = X[0], X[1]
    skill_yx, skill_xy = [], []
    for Lw in (25, 50, 100, 200, 400):
        skill_yx.append(oracle.ccm_row(y[:Lw], x[:Lw], 2, 1, 0)[0])
        skill_xy.append(oracle.ccm_row(x[:Lw], y[:Lw], 2, 1, 0)[0])
    assert skill_yx[-1] > skill_xy[-1] + 0.2
    assert skill_yx[-1] > skill_yx[0] + 0.1
    assert skill_yx[-1] > 0.8


def test_optimal_E_sine_needs_two_dimensions():
    t = np.arange(300)
    x = np.sin(2 * np.pi * t / 37.3).astype(np.float32)
    E, rho = oracle.optimal_E(x, 6, 1, 1)
    assert rho[1] > rho[0] + 0.01
    assert E >= 2


def test_optimal_E_logistic_one_dimension_suffices():
    x = inputs.logistic_map(400)
    E, rho = oracle.optimal_E(x, 5, 1, 1)
    assert rho[0] > 0.99
    assert rho[E - 1] == np.nanmax(rho)


def test_optimal_E_nan_and_ties():
    # a constant series has zero variance: every skill is NaN, E* = 1
    E, rho = oracle.optimal_E(np.ones(40, np.float32), 4, 1, 1)
    assert E == 1 and np.all(np.isnan(rho))
    # E too large for the series length gives NaN for those E only
    x = inputs.logistic_map(12)
    E, rho = oracle.optimal_E(x, 10, 1, 1)
    n = 12 - np.arange(10) - 1
    assert np.all(np.isnan(rho[n < np.arange(1, 11) + 2]))
    assert np.all(np.isfinite(rho[n >= np.arange(1, 11) + 2]))


def test_argmax_E_tie_and_nan_rule():
    # Hand-written skills with the expected E* from the stated rule: the
    # largest skill wins, a NaN ranks below every number, equal skills go to
    # the smaller E, and all-NaN gives 1.  Ties to the larger E (>=), a NaN
    # that wins, or a 0-based result each fail one of these.
    nan = float("nan")
    cases = [
        ([0.5, 0.5, 0.3], 1),
        ([0.1, 0.7, 0.7, 0.2], 2),
        ([0.2, 0.9, 0.4, 0.9, 0.9], 2),
        ([nan, 0.2, 0.2], 2),
        ([nan, nan, -0.3, -0.3], 3),
        ([-0.5, nan, -0.5], 1),
        ([0.3, nan, 0.8], 3),
        ([nan, nan, nan], 1),
        ([-1.0], 1),
        ([0.0, -0.0], 1),                   # -0.0 == 0.0 is a tie
        ([0.25, 0.25 + 2.0 ** -52, 0.25], 2),   # one ulp above is not a tie
    ]
    for rho, want in cases:
        assert oracle.argmax_E(np.array(rho)) == want, (rho, want)


def test_optimal_E_uses_the_argmax_rule():
    # the E* that oracle_optimal_E reports is the rule applied to the skills
    # it reports, on data with NaN skills at large E (short series)
    for seed, L in ((5, 14), (6, 40), (7, 200)):
        x = inputs.coupled_logistic(1, L, seed)[0]
        E, rho = oracle.optimal_E(x, 12, 1, 1)
        finite = np.where(np.isnan(rho), -np.inf, rho)
        want = int(np.flatnonzero(finite == finite.max())[0]) + 1 if np.isfinite(finite.max()) else 1
        assert E == want


def test_constant_target_gives_nan():
    X = inputs.coupled_logistic(1, 80, 2)
    assert math.isnan(oracle.ccm_row(X[0], np.full(80, 2.0, np.float32), 2, 1, 0)[0])
