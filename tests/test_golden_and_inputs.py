"""Golden regression of the oracle on the 16 x 200 workload, and checks of the
seeded input generators (CPU only)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2105_12301_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "logistic_16x200_oracle.json")


def test_oracle_reproduces_golden_logistic_16x200():
    g = json.load(open(GOLDEN))
    X = inputs.logistic_16x200()
    E_opt, rho_E = oracle.optimal_E_many(X, g["E_max"], g["tau"], g["Tp_sel"])
    assert list(E_opt) == g["E_opt"]
    np.testing.assert_allclose(rho_E, np.array(g["rho_E"]), rtol=0, atol=1e-12)
    rho = oracle.ccm_matrix(X, X, E_opt, g["tau"], g["Tp"])
    np.testing.assert_allclose(rho, np.array(g["rho"]), rtol=0, atol=1e-12)


def test_generators_are_seeded_and_normalised():
    a = inputs.logistic_16x200()
    b = inputs.logistic_16x200()
    assert a.dtype == np.float32 and a.shape == (16, 200)
    assert np.array_equal(a, b)
    np.testing.assert_allclose(a.astype(np.float64).mean(axis=1), 0, atol=1e-6)
    np.testing.assert_allclose(a.astype(np.float64).std(axis=1), 1, atol=1e-5)
    c = inputs.calcium(N=64, L=300)
    assert c.shape == (64, 300) and np.all(np.isfinite(c))
    np.testing.assert_allclose(c.astype(np.float64).std(axis=1), 1, atol=1e-5)


def test_beta_row_cap_keeps_maps_bounded():
    X, info = inputs.coupled_logistic(400, 300, 9, 3.6, 3.9, 0.05, 0.1,
                                      return_info=True)
    assert np.all(np.isfinite(X))
    assert info["beta_rows_rescaled"] > 0
    assert np.all(info["beta"].sum(axis=1) <= inputs.BETA_ROW_CAP + 1e-12)
    assert np.all(np.diag(info["beta"]) == 0)


def test_uneven_batch_shapes_in_range():
    N, L = inputs.uneven_batch_shapes()
    assert len(N) == 256 and N.min() >= 32 and N.max() <= 2048
    assert L.min() >= 200 and L.max() <= 5000
