"""GPU parity of optimal-E selection and all-to-all CCM against the FP64 oracle.

Tolerances: |rho_gpu - rho_oracle| <= 1e-5 with FP32 target storage,
<= 5e-4 with FP16 target storage, and with BF16 target storage <= 1e-3 when
the library has at least 300 points and <= 2e-3 below that (BF16 keeps 8
significant bits; the rounding of short targets alone moves rho by up to
about 1.5e-3); the skills rho_E of the simplex sweep within 1e-5; E* equal
to the oracle's unless the oracle's own skills of the two choices lie within
1e-5 of each other (a near-tie).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2105_12301_gb300 import edm, inputs

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_FP16 = 5e-4
TOL_BF16 = 1e-3
TOL_BF16_SHORT = 2e-3      # BF16 with fewer than 300 library points
TOL_RHO_E = 1e-5


def tol16(precision, L):
    """The bound of a 16-bit target storage at library length L."""
    if precision == "fp16":
        return TOL_FP16
    return TOL_BF16 if L >= 300 else TOL_BF16_SHORT


def gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check_optimal_E(X, E_max, tau=1, Tp_sel=1):
    E_gpu, rho_gpu = edm.edm_simplex_optimal_E(gpu(X), E_max, tau, Tp_sel)
    edm.edm_ctx_sync()
    E_gpu, rho_gpu = E_gpu.cpu().numpy(), rho_gpu.cpu().numpy()
    E_or, rho_or = oracle.optimal_E_many(X, E_max, tau, Tp_sel)
    np.testing.assert_array_equal(np.isnan(rho_gpu), np.isnan(rho_or))
    ok = ~np.isnan(rho_or)
    assert np.max(np.abs(rho_gpu[ok] - rho_or[ok]), initial=0.0) <= TOL_RHO_E
    for i in np.nonzero(E_gpu != E_or)[0]:
        gap = abs(rho_or[i, E_gpu[i] - 1] - rho_or[i, E_or[i] - 1])
        assert gap <= 1e-5, (i, E_gpu[i], E_or[i], gap)
    return E_gpu


def check_ccm(X_lib, Y, E_lib, tau, Tp, precision, tol, lib_rows=None):
    rho = edm.edm_ccm_all(gpu(X_lib), gpu(Y), gpu(E_lib.astype(np.int32)), tau, Tp, precision)
    edm.edm_ctx_sync()
    rho = rho.cpu().numpy()
    rows = np.arange(X_lib.shape[0]) if lib_rows is None else np.asarray(lib_rows)
    ref = oracle.ccm_matrix(X_lib, Y, E_lib, tau, Tp, lib_rows=rows)
    got = rho[rows]
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    err = np.max(np.abs(got[ok] - ref[ok]), initial=0.0)
    assert err <= tol, err
    return rho, err


def test_logistic_16x200_optimal_E_and_full_rho_matrix():
    X = inputs.logistic_16x200()
    E = check_optimal_E(X, 10)
    check_ccm(X, X, E, 1, 0, "fp32", TOL_FP32)
    check_ccm(X, X, E, 1, 0, "fp16", TOL_FP16)
    check_ccm(X, X, E, 1, 0, "bf16", tol16("bf16", 200))


def test_logistic_1000_full_matrix():
    # 1,000 x 1,000 coupled logistic with noise: E* of every series against
    # the oracle's, then all 10^6 rho values in every target storage
    X = inputs.logistic_noisy()
    E = check_optimal_E(X, 20)
    ref = oracle.ccm_matrix(X, X, E, 1, 0)
    ok = ~np.isnan(ref)
    for prec, tol in (("fp32", TOL_FP32), ("fp16", TOL_FP16), ("bf16", TOL_BF16)):
        rho = edm.edm_ccm_all(gpu(X), gpu(X), gpu(E), 1, 0, prec)
        edm.edm_ctx_sync()
        got = rho.cpu().numpy()
        np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
        err = np.abs(got[ok] - ref[ok])
        print("1000x1000 %s: max %.3g p99 %.3g over %d pairs"
              % (prec, err.max(), np.percentile(err, 99), err.size))
        assert err.max() <= tol, (prec, err.max())


def test_library_length_windows_1000_sampled_pairs():
    # 2,000 x 10,000 coupled logistic; E per library from the full-length
    # simplex; CCM on the windows [0, L_lib) with 1,000 sampled (library,
    # target) pairs per window checked against the oracle in every storage
    X = inputs.logistic_long()
    Xg = gpu(X)
    E_full, _ = edm.edm_simplex_optimal_E(Xg, 20, 1, 1, with_rho=False)
    E_np = E_full.cpu().numpy()
    rng = np.random.default_rng(105)
    lib_rows = np.sort(rng.choice(2000, 40, replace=False))
    tgts = np.sort(rng.choice(2000, 25, replace=False))
    for L_lib in (100, 300, 1000, 3000, 10000):
        Xw = np.ascontiguousarray(X[:, :L_lib])
        ref = oracle.ccm_matrix(Xw[lib_rows], Xw[tgts], E_np[lib_rows], 1, 0)
        ok = ~np.isnan(ref)
        assert ok.sum() >= 990
        for prec in ("fp32", "fp16", "bf16"):
            tol = TOL_FP32 if prec == "fp32" else tol16(prec, L_lib)
            rho = edm.edm_ccm_window(Xg, 0, L_lib, E_full, 1, 0, prec)
            edm.edm_ctx_sync()
            got = rho.cpu().numpy()[np.ix_(lib_rows, tgts)]
            del rho
            np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
            err = np.abs(got[ok] - ref[ok])
            print("window %d %s: max %.3g p99 %.3g over %d pairs"
                  % (L_lib, prec, err.max(), np.percentile(err, 99), err.size))
            assert err.max() <= tol, (L_lib, prec, err.max())


@pytest.mark.parametrize("E", [1, 2, 7, 20])
def test_every_K_specialisation(E):
    X = inputs.coupled_logistic(5, 180, 100 + E)
    E_lib = np.full(5, E, np.int32)
    check_ccm(X, X, E_lib, 1, 0, "fp32", TOL_FP32)


def test_ragged_counts_tau_and_horizon():
    X = inputs.coupled_logistic(3, 90, 8)
    Y = inputs.coupled_logistic(70, 90, 9)        # 70 targets: ragged tiles
    E_lib = np.array([2, 5, 3], np.int32)
    check_ccm(X, Y, E_lib, 3, 2, "fp32", TOL_FP32)
    check_ccm(X, Y, E_lib, 3, 2, "fp16", TOL_FP16)
    check_ccm(X, Y, E_lib, 3, 2, "bf16", tol16("bf16", 90))


def test_mixed_E_in_one_launch():
    X = inputs.logistic_noisy(N=40, L=400)
    E_lib = np.arange(40, dtype=np.int32) % 20 + 1
    check_ccm(X, X, E_lib, 1, 0, "fp32", TOL_FP32)


@pytest.mark.parametrize("L,N", [(1700, 37), (2500, 40), (3250, 21)])
def test_half_width_target_tiles(L, N):
    # 1,600 < L <= 3,300: a 32-word tile row no longer fits shared memory, a
    # 16-word one does (two half-warps take the two rows of a pair)
    X = inputs.coupled_logistic(N, L, 12 + L)
    E_lib = np.array([1, 2, 3, 4, 7] * 8, np.int32)[:N]
    check_ccm(X, X, E_lib, 1, 0, "fp32", TOL_FP32, lib_rows=[0, 13, N - 1])
    check_ccm(X, X, E_lib, 1, 0, "fp16", TOL_FP16, lib_rows=[0, 13, N - 1])
    check_ccm(X, X, E_lib, 1, 0, "bf16", TOL_BF16, lib_rows=[0, 13, N - 1])


def test_long_series_gathers_from_global_memory():
    # L = 3,600: not even a 16-word tile fits; gathers read global memory
    X = inputs.coupled_logistic(35, 3600, 13)
    E_lib = np.array([1, 2, 3, 4, 5] * 7, np.int32)
    check_ccm(X, X, E_lib, 1, 0, "fp32", TOL_FP32, lib_rows=[0, 13, 34])
    check_ccm(X, X, E_lib, 1, 0, "fp16", TOL_FP16, lib_rows=[0, 13, 34])
    check_ccm(X, X, E_lib, 1, 0, "bf16", TOL_BF16, lib_rows=[0, 13, 34])


def test_self_map_equals_simplex():
    X = inputs.logistic_16x200()
    E_gpu, rho_E = edm.edm_simplex_optimal_E(gpu(X), 6, 1, 0)
    rho = edm.edm_ccm_all(gpu(X), gpu(X), E_gpu, 1, 0).cpu().numpy()
    rho_E = rho_E.cpu().numpy()
    E_np = E_gpu.cpu().numpy()
    for i in range(16):
        assert abs(rho[i, i] - rho_E[i, E_np[i] - 1]) <= 2e-6


def test_constant_target_and_bad_E_give_nan():
    X = inputs.coupled_logistic(2, 100, 3)
    Y = np.vstack([X, np.full((1, 100), 1.5, np.float32)])
    rho = edm.edm_ccm_all(gpu(X), gpu(Y), gpu(np.array([2, 2], np.int32))).cpu().numpy()
    assert np.all(np.isnan(rho[:, 2])) and np.all(np.isfinite(rho[:, :2]))
    rho = edm.edm_ccm_all(gpu(X), gpu(Y), gpu(np.array([2, 33], np.int32)))
    with pytest.raises(edm.EdmError):
        edm.edm_ctx_sync()
    rho = rho.cpu().numpy()
    assert np.all(np.isnan(rho[1])) and np.all(np.isfinite(rho[0, :2]))


def test_batched_instances_match_single_calls():
    probs = []
    for i, (N, L) in enumerate([(33, 250), (70, 130), (5, 600)]):
        X = inputs.coupled_logistic(N, L, 200 + i)
        E = (np.arange(N) % 4 + 1).astype(np.int32)
        probs.append({"X": gpu(X), "E_lib": gpu(E), "tau": 1, "Tp": 0,
                      "lib_begin": 1, "lib_end": N})
    outs = edm.edm_ccm_batched(probs)
    for p, out in zip(probs, outs):
        ref = edm.edm_ccm_all(p["X"][1:].contiguous(), p["X"], p["E_lib"][1:].contiguous())
        torch.testing.assert_close(out, ref, rtol=0, atol=0, equal_nan=True)
    edm.edm_ctx_sync()


def test_full_size_calcium_workload_sampled():
    # 50,000 x 1,500 as timed by the bench: GPU runs everything, the oracle
    # checks sampled libraries against all 50,000 targets
    X = inputs.calcium()
    Xg = gpu(X)
    E_gpu, rho_E = edm.edm_simplex_optimal_E(Xg, 20, 1, 1)
    rows = [0, 17, 31337, 49999]
    E_np = E_gpu.cpu().numpy()
    E_or, rho_or = oracle.optimal_E_many(X[rows], 20, 1, 1)
    got = rho_E.cpu().numpy()[rows]
    assert np.max(np.abs(got - rho_or)) <= TOL_RHO_E
    for r, e in zip(rows, E_or):
        if E_np[r] != e:
            assert abs(rho_or[rows.index(r), E_np[r] - 1] - rho_or[rows.index(r), e - 1]) <= 1e-5
    rho = edm.edm_ccm_all(Xg, Xg, E_gpu, 1, 0, "fp32")
    edm.edm_ctx_sync()
    ref = oracle.ccm_matrix(X, X, E_np, 1, 0, lib_rows=rows)
    err = np.max(np.abs(rho[rows].cpu().numpy() - ref))
    assert err <= TOL_FP32, err
    del rho
    for prec, tol in (("fp16", TOL_FP16), ("bf16", TOL_BF16)):
        rho = edm.edm_ccm_all(Xg, Xg, E_gpu, 1, 0, prec)
        edm.edm_ctx_sync()
        err = np.max(np.abs(rho[rows].cpu().numpy() - ref))
        del rho
        assert err <= tol, (prec, err)


@pytest.mark.parametrize("L,tau", [(2048, 1), (2049, 1), (1000, 2), (700, 3)])
def test_register_path_boundaries(L, tau):
    # 2048 points: 64 candidate slots per lane (largest register path);
    # 2049: the generic path; tau > 1 with lag offsets beyond one slot
    X = inputs.coupled_logistic(6, L, 40 + L + tau)
    E = check_optimal_E(X[:3], 6, tau, 1)
    E_lib = np.array([2, 5, 1, 3, 4, 6], np.int32)
    E_lib[:3] = E
    check_ccm(X, X, E_lib, tau, 0, "fp32", TOL_FP32, lib_rows=[0, 4])


@pytest.mark.parametrize("L", [600, 1500, 3000])
def test_selection_through_long_runs_of_ties(L):
    # libraries on a coarse value grid (3 to 8 levels): long runs of exactly
    # tied squared distances drive the selection from registers (optimal-E
    # sweep, table builder; the chunked variants at 3,000 points) through its
    # rare paths: more collected values than the key buffer holds, the
    # bisection of the bound, the FP64 band and the full FP64 scan.  Series 3
    # is constant, so every distance ties and every skill is NaN (E* = 1); as
    # a library it still runs through the table builder, but its row of rho
    # is not compared: its nearly constant predictions make rho
    # ill-conditioned in FP32 moments.
    X = inputs.coupled_logistic(4, L, 900 + L)
    Xq = (np.round(X * 2.0) / 2.0).astype(np.float32)
    Xq[3] = 0.0
    edm.edm_set_option("diagnostics", 1)
    try:
        edm.edm_fallback_counts()
        E = check_optimal_E(Xq, 8)
        band, brute = edm.edm_fallback_counts()
        assert band > 0 and brute > 0, (band, brute)
        assert E[3] == 1
        check_ccm(Xq, X, E.astype(np.int32), 1, 0, "fp32", TOL_FP32, lib_rows=[0, 1, 2])
        band, brute = edm.edm_fallback_counts()
        assert band > 0 and brute > 0, (band, brute)
    finally:
        edm.edm_set_option("diagnostics", 0)


@pytest.mark.parametrize("L,tau,Tp_sel", [(3100, 1, 1), (2600, 2, 1), (4000, 1, 2)])
def test_optimal_E_long_series(L, tau, Tp_sel):
    # more than 2,048 points: the chunked incremental sweep
    X = inputs.coupled_logistic(3, L, 70 + L)
    check_optimal_E(X, 6, tau, Tp_sel)


def test_window_convergence_matches_oracle():
    # library-length windows [0, Lw) of longer series, as in the convergence sweep
    X = inputs.coupled_logistic(24, 1200, 91)
    Xg = gpu(X)
    E_full, _ = edm.edm_simplex_optimal_E(Xg, 8, 1, 1)
    E_np = E_full.cpu().numpy()
    for Lw in (100, 300, 1200):
        rho = edm.edm_ccm_window(Xg, 0, Lw, E_full, 1, 0, "fp32")
        edm.edm_ctx_sync()
        ref = oracle.ccm_matrix(X[:, :Lw], X[:, :Lw], E_np, 1, 0, lib_rows=[0, 7, 23])
        got = rho.cpu().numpy()[[0, 7, 23]]
        np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
        ok = ~np.isnan(ref)
        assert np.max(np.abs(got[ok] - ref[ok])) <= TOL_FP32
    # an offset window
    rho = edm.edm_ccm_window(Xg, 200, 500, E_full, 1, 0, "bf16").cpu().numpy()
    ref = oracle.ccm_matrix(X[:, 200:700], X[:, 200:700], E_np, 1, 0, lib_rows=[3])
    assert np.max(np.abs(rho[3] - ref[0])) <= TOL_BF16


def _uneven_problems(seed0=300):
    probs = []
    for i, (N, L) in enumerate([(40, 240), (96, 900), (33, 2300), (7, 180), (150, 600),
                                (64, 1500), (12, 3000), (200, 300)]):
        X = inputs.coupled_logistic(N, L, seed0 + i, 3.6, 3.9, 0.05, 0.1, noise=0.02)
        probs.append({"X": gpu(X), "tau": 1, "Tp": 0})
    return probs


def _check_batched_E(E, X, E_max):
    # the batched runs split query rows into other blocks than a single
    # call, so the FP64 sums of rho_E differ in the last bits: E* must equal
    # the single call's unless the two skills are a near-tie
    ref, rho = edm.edm_simplex_optimal_E(X, E_max, 1, 1)
    E, ref, rho = E.cpu().numpy(), ref.cpu().numpy(), rho.cpu().numpy()
    for i in np.nonzero(E != ref)[0]:
        assert abs(rho[i, E[i] - 1] - rho[i, ref[i] - 1]) <= 1e-5, (i, E[i], ref[i])


def test_batched_optimal_E_work_queues_and_streams():
    # the work-queue launches (default: tuned, graph-captured, replayed) and
    # the per-instance launches over streams both match single calls
    probs = _uneven_problems(seed0=340)
    for queue in (1, 0):
        edm.edm_set_option("batch_queue", queue)
        for _ in range(2):          # the second call replays the cached graph
            E_list = edm.edm_simplex_optimal_E_batched(probs, 12, 1)
            for p, E in zip(probs, E_list):
                _check_batched_E(E, p["X"], 12)
    edm.edm_set_option("batch_queue", 1)
    edm.edm_ctx_sync()


def test_batched_graph_and_streams_match_single_calls():
    probs = _uneven_problems()
    E_list = edm.edm_simplex_optimal_E_batched(probs, 8, 1)
    for p, E in zip(probs, E_list):
        _check_batched_E(E, p["X"], 8)
        p["E_lib"] = E
    singles = [edm.edm_ccm_all(p["X"], p["X"], p["E_lib"]) for p in probs]
    for graph in (0, 1):
        edm.edm_set_option("batch_graph", graph)
        for _ in range(2):          # the second graph call replays the cached graph
            outs = edm.edm_ccm_batched(probs)
            for out, ref in zip(outs, singles):
                torch.testing.assert_close(out, ref, rtol=0, atol=0, equal_nan=True)
    edm.edm_set_option("batch_graph", 1)
    edm.edm_ctx_sync()
    # and one instance against the oracle
    X = probs[2]["X"].cpu().numpy()
    E = probs[2]["E_lib"].cpu().numpy()
    ref = oracle.ccm_matrix(X, X, E, 1, 0, lib_rows=[0, 32])
    assert np.max(np.abs(outs[2].cpu().numpy()[[0, 32]] - ref)) <= TOL_FP32


def test_set_option_rejects_unknown():
    with pytest.raises(edm.EdmError):
        edm.edm_set_option("no_such_option", 1)
    with pytest.raises(edm.EdmError):
        edm.edm_set_option("batch_streams", 0)


def test_per_target_E_rule_matches_oracle():
    # section 3.3: each library is embedded at each target's E
    X = inputs.logistic_noisy(N=14, L=350)
    Y = inputs.coupled_logistic(11, 350, 5150)
    E_tgt = np.array([2, 1, 3, 2, 5, 20, 2, 1, 3, 7, 2], np.int32)
    for prec, tol in (("fp32", TOL_FP32), ("fp16", TOL_FP16), ("bf16", TOL_BF16)):
        rho = edm.edm_ccm_all_target_E(gpu(X), gpu(Y), gpu(E_tgt), 1, 0, prec)
        edm.edm_ctx_sync()
        rho = rho.cpu().numpy()
        ref = np.stack([[oracle.ccm_row(X[i], Y[j], int(E_tgt[j]), 1, 0)[0]
                         for j in range(Y.shape[0])] for i in range(X.shape[0])])
        assert np.max(np.abs(rho - ref)) <= tol
    # a single E equals the per-library call with that E everywhere
    E3 = np.full(Y.shape[0], 3, np.int32)
    a = edm.edm_ccm_all_target_E(gpu(X), gpu(Y), gpu(E3), 1, 0, "fp32")
    b = edm.edm_ccm_all(gpu(X), gpu(Y), gpu(np.full(X.shape[0], 3, np.int32)), 1, 0, "fp32")
    torch.testing.assert_close(a, b, rtol=0, atol=0)
    with pytest.raises(edm.EdmError):
        edm.edm_ccm_all_target_E(gpu(X), gpu(Y), gpu(np.full(Y.shape[0], 21, np.int32)))


def test_ccm_all_host_streams_rows_to_pinned_memory():
    X = inputs.logistic_noisy(N=300, L=400)
    E = check_optimal_E(X[:20], 8)
    E_lib = np.resize(E, 300).astype(np.int32)
    Xg = gpu(X)
    out = torch.empty((300, 300), dtype=torch.float32, device="cuda")
    host = torch.empty((300, 300), dtype=torch.float32).pin_memory()
    edm.edm_ccm_all_host(Xg, Xg, gpu(E_lib), out, host, 1, 0, "fp32")
    edm.edm_ctx_sync()
    ref = edm.edm_ccm_all(Xg, Xg, gpu(E_lib), 1, 0, "fp32")
    edm.edm_ctx_sync()
    torch.testing.assert_close(out, ref, rtol=0, atol=0, equal_nan=True)
    torch.testing.assert_close(host, ref.cpu(), rtol=0, atol=0, equal_nan=True)
    with pytest.raises(edm.EdmError):   # pageable host memory is refused
        edm.load()
        ctx = edm._ctx(Xg.device)
        st = edm.load().edm_ccm_all_host(ctx, edm._ptr(Xg), 300, edm._ptr(Xg), 300, 400,
                                         edm._ptr(gpu(E_lib)), 1, 0, 0, edm._ptr(out),
                                         edm._ptr(torch.empty((300, 300))))
        edm._check(ctx, st, "edm_ccm_all_host")


def test_random_library_windows_match_oracle():
    # several windows of one length (e.g. random starts for convergence curves)
    X = inputs.coupled_logistic(10, 900, 93)
    E = np.array([2, 3, 1, 2, 4, 2, 3, 5, 2, 1], np.int32)
    rng = np.random.default_rng(4)
    L_win = 250
    offs = sorted(rng.choice(900 - L_win + 1, 4, replace=False).tolist())
    rho = edm.edm_ccm_windows(gpu(X), offs, L_win, gpu(E), 1, 0, "fp32")
    edm.edm_ctx_sync()
    rho = rho.cpu().numpy()
    for w, o in enumerate(offs):
        Xw = np.ascontiguousarray(X[:, o:o + L_win])
        ref = oracle.ccm_matrix(Xw, Xw, E, 1, 0)
        assert np.max(np.abs(rho[w] - ref)) <= TOL_FP32, (w, o)
    with pytest.raises(edm.EdmError):
        edm.edm_ccm_windows(gpu(X), [700], L_win, gpu(E))   # runs past the end
