"""Failure detection without a GPU fault: every wait inside a libedm kernel is
bounded, records EDM_ERR_TIMEOUT in the context when it gives up, and lets
the kernel run to its end, so the context stays usable."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2105_12301_gb300 import edm, inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_stays_usable():
    edm.edm_ctx_sync()                      # start from a clean flag
    edm.edm_check_wait_timeout(50)          # a wait nothing completes, 50 ms limit
    with pytest.raises(edm.EdmError) as err:
        edm.edm_ctx_sync()
    assert err.value.status == 4            # EDM_ERR_TIMEOUT
    edm.edm_ctx_sync()                      # the flag was cleared by the read
    X = inputs.logistic_16x200()[:6]
    Xg = torch.from_numpy(X).cuda()
    E = np.array([2, 3, 1, 2, 4, 2], np.int32)
    rho = edm.edm_ccm_all(Xg, Xg, torch.from_numpy(E).cuda(), 1, 0, "fp32")
    edm.edm_ctx_sync()
    ref = oracle.ccm_matrix(X, X, E, 1, 0)
    assert np.max(np.abs(rho.cpu().numpy() - ref)) <= 1e-5


def test_waits_after_a_timeout_return_at_once():
    # the check kernel waits twice on a barrier nothing completes; the first
    # wait gives up after the limit and sets the CTA's abort word, so the
    # second returns at once: about one limit in all, not two
    edm.edm_ctx_sync()
    t0 = time.perf_counter()
    edm.edm_check_wait_timeout(400)
    with pytest.raises(edm.EdmError) as err:
        edm.edm_ctx_sync()
    dt = time.perf_counter() - t0
    assert err.value.status == 4
    assert 0.35 <= dt < 0.7, dt


def test_wait_check_rejects_bad_limits():
    with pytest.raises(edm.EdmError):
        edm.edm_check_wait_timeout(0)
    with pytest.raises(edm.EdmError):
        edm.edm_check_wait_timeout(20000)
