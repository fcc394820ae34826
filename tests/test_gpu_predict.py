"""GPU parity of the written-out simplex predictions (edm_predict) against
the FP64 oracle's kNN + prediction (section 2.1 step 3, Algorithm 3)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_12301_gb300 import edm, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 weights and arithmetic against FP64, values of order 1


def gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check_predictions(X_lib, Y, E, tgt, tau, Tp):
    pred = edm.edm_predict(gpu(X_lib), gpu(Y), gpu(E), None if tgt is None else gpu(tgt), tau, Tp)
    edm.edm_ctx_sync()
    pred = pred.cpu().numpy()
    L = X_lib.shape[1]
    for i in range(X_lib.shape[0]):
        j = i if tgt is None else int(tgt[i])
        idx, dist = oracle.knn(X_lib[i], int(E[i]), tau, Tp)
        t0 = (int(E[i]) - 1) * tau
        ref, _ = oracle.predict(idx, dist, Y[j], t0, Tp)
        lo, hi = t0 + Tp, t0 + Tp + ref.shape[0]
        assert np.max(np.abs(pred[i, lo:hi] - ref)) <= TOL, i
        outside = np.r_[pred[i, :lo], pred[i, hi:L]]
        assert np.all(np.isnan(outside)), i


def test_self_forecast_matches_oracle():
    X = inputs.logistic_noisy(N=12, L=400)
    E = np.array([1, 2, 3, 4, 5, 6, 2, 3, 1, 8, 20, 2], np.int32)
    check_predictions(X, X, E, None, 1, 1)


def test_cross_forecast_with_target_map_tau_and_ragged_groups():
    X = inputs.coupled_logistic(9, 333, 91)
    Y = inputs.coupled_logistic(5, 333, 92)
    E = np.array([2, 2, 2, 2, 2, 3, 3, 1, 7], np.int32)   # a full group, partial groups
    tgt = np.array([4, 0, 3, 1, 2, 2, 0, 4, 1], np.int32)
    check_predictions(X, Y, E, tgt, 2, 0)
    check_predictions(X, Y, E, tgt, 1, 3)


def test_bad_target_index_gives_nan_row_and_error():
    X = inputs.logistic_16x200()[:3]
    E = gpu(np.array([2, 2, 2], np.int32))
    tgt = gpu(np.array([0, 7, 1], np.int32))   # 7 is out of range for 3 targets
    pred = edm.edm_predict(gpu(X), gpu(X), E, tgt, 1, 0)
    with pytest.raises(edm.EdmError):
        edm.edm_ctx_sync()
    p = pred.cpu().numpy()
    assert np.all(np.isnan(p[1])) and not np.all(np.isnan(p[0]))
