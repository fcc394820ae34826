"""The allocation-free optimal-E entry point (collected last on purpose).

edm_simplex_optimal_E_noalloc serves callers that may not allocate device
memory once running (latency-bound pipelines, plug-ins whose host owns the
GPU's memory): its scratch is a fixed array inside the library.  Its results
must equal those of edm_simplex_optimal_E, also on a second call in a row
(the shared scratch keeps the previous call's contents)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2105_12301_gb300 import edm, inputs

pytestmark = pytest.mark.gpu

TOL_RHO_E = 1e-5


def call_noalloc_abi(Xg, E_max, tau, Tp_sel):
    """Straight through the C ABI: device pointers and a stream, no context."""
    lib = edm.load()
    N, L = Xg.shape
    E_opt = torch.empty(N, dtype=torch.int32, device=Xg.device)
    rho_E = torch.empty((N, E_max), dtype=torch.float32, device=Xg.device)
    stream = torch.cuda.current_stream(Xg.device).cuda_stream
    st = lib.edm_simplex_optimal_E_noalloc(
        ctypes.c_void_p(Xg.data_ptr()), N, L, E_max, tau, Tp_sel,
        ctypes.c_void_p(E_opt.data_ptr()), ctypes.c_void_p(rho_E.data_ptr()),
        ctypes.c_void_p(stream))
    assert st == 0, st
    torch.cuda.synchronize(Xg.device)
    return E_opt.cpu().numpy(), rho_E.cpu().numpy()


def reference(Xg, E_max, tau, Tp_sel):
    E_opt, rho_E = edm.edm_simplex_optimal_E(Xg, E_max, tau, Tp_sel)
    edm.edm_ctx_sync(Xg.device)
    return E_opt.cpu().numpy(), rho_E.cpu().numpy()


def compare(got, ref):
    (e1, r1), (e2, r2) = got, ref
    np.testing.assert_array_equal(np.isnan(r1), np.isnan(r2))
    ok = ~np.isnan(r2)
    assert np.max(np.abs(r1[ok] - r2[ok]), initial=0.0) <= TOL_RHO_E
    for i in np.nonzero(e1 != e2)[0]:
        assert abs(r2[i, e1[i] - 1] - r2[i, e2[i] - 1]) <= 1e-5


def test_noalloc_matches_context_path_on_two_calls_in_a_row():
    A = torch.from_numpy(inputs.logistic_16x200()).cuda()                    # 16 x 200
    B = torch.from_numpy(inputs.logistic_noisy(N=300, L=700)).cuda()        # 300 x 700
    ref_a = reference(A, 10, 1, 1)
    ref_b = reference(B, 20, 1, 1)
    compare(call_noalloc_abi(A, 10, 1, 1), ref_a)
    compare(call_noalloc_abi(B, 20, 1, 1), ref_b)   # second call, other shape
    compare(call_noalloc_abi(A, 10, 1, 1), ref_a)   # and back


def test_noalloc_long_series_and_binding():
    # L = 2600 takes the non-register sweep; tau = 2
    X = torch.from_numpy(inputs.coupled_logistic(4, 2600, 61)).cuda()
    ref = reference(X, 5, 2, 1)
    E_opt = torch.empty(4, dtype=torch.int32, device="cuda")
    rho_E = torch.empty((4, 5), dtype=torch.float32, device="cuda")
    for _ in range(2):
        edm.edm_simplex_optimal_E_noalloc(X, E_opt, rho_E, 5, 2, 1)
        torch.cuda.synchronize()
        compare((E_opt.cpu().numpy(), rho_E.cpu().numpy()), ref)


def test_noalloc_rejects_requests_beyond_its_scratch():
    lib = edm.load()
    X = torch.zeros((6000, 64), dtype=torch.float32, device="cuda")
    E_opt = torch.empty(6000, dtype=torch.int32, device="cuda")
    st = lib.edm_simplex_optimal_E_noalloc(ctypes.c_void_p(X.data_ptr()), 6000, 64, 20, 1, 1,
                                           ctypes.c_void_p(E_opt.data_ptr()), None, None)
    assert st == 1   # EDM_ERR_INVALID_ARG: 6000 * 20 > 104,857
