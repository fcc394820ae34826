"""Parity report of the GPU path against the FP64 oracle, one JSON line per
workload (needs a GPU; the oracle runs on all host cores).

    python tests/parity_report.py [--quick]

Per workload it reports:
  - neighbour-index mismatches of edm_knn against the oracle's exact kNN
    (ties to the lower time index) on sampled libraries at their E*;
  - E* agreement of edm_simplex_optimal_E, with the number of disagreements
    that are near-ties (the oracle's skills of the two choices within 1e-5);
  - max |rho_E gpu - rho_E oracle| of the simplex sweep;
  - max and 99th percentile of |rho gpu - rho oracle| of all-to-all CCM with
    FP32, FP16 and BF16 target storage (the oracle always takes the GPU's E*).
Like the tests, this script is test infrastructure: it is the only kind of
code besides tests that calls the oracle.
"""
import argparse
import json
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2105_12301_gb300 import edm, inputs  # noqa: E402


def gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def knn_mismatch(X, rows, E_np, tau, Tp):
    """Neighbour indices that differ from the oracle's, over every query row
    of the sampled libraries at their E."""
    bad = total = 0
    for i in rows:
        E = int(E_np[i])
        idx, _ = edm.edm_knn(gpu(X[i:i + 1]), E, tau, Tp)
        ref, _ = oracle.knn(X[i], E, tau, Tp)
        got = idx[0].cpu().numpy()
        bad += int(np.sum(got != ref))
        total += ref.size
    return bad, total


def optimal_E_report(X, rows, E_max, tau, Tp_sel):
    E_gpu, rho_gpu = edm.edm_simplex_optimal_E(gpu(X), E_max, tau, Tp_sel)
    E_gpu, rho_gpu = E_gpu.cpu().numpy(), rho_gpu.cpu().numpy()
    E_or, rho_or = oracle.optimal_E_many(X[rows], E_max, tau, Tp_sel)
    g = rho_gpu[rows]
    ok = ~np.isnan(rho_or)
    nan_match = bool(np.array_equal(np.isnan(g), np.isnan(rho_or)))
    diff = E_gpu[rows] != E_or
    near = 0
    for j in np.nonzero(diff)[0]:
        gap = abs(rho_or[j, E_gpu[rows][j] - 1] - rho_or[j, E_or[j] - 1])
        near += int(gap <= 1e-5)
    return E_gpu, {"series_checked": len(rows), "E_star_equal": int(np.sum(~diff)),
                   "E_star_near_ties": near, "E_star_other": int(np.sum(diff)) - near,
                   "rho_E_max_abs_diff": float(np.max(np.abs(g[ok] - rho_or[ok]), initial=0.0)),
                   "rho_E_nan_pattern_equal": nan_match}


def ccm_report(Xg, X, E_gpu, rows, tau, Tp, targets=None):
    out = {}
    Y = X if targets is None else X[targets]
    ref = oracle.ccm_matrix(X, Y, E_gpu, tau, Tp, lib_rows=rows)
    for prec in ("fp32", "fp16", "bf16"):
        rho = edm.edm_ccm_all(Xg, Xg, gpu(E_gpu.astype(np.int32)), tau, Tp, prec)
        edm.edm_ctx_sync()
        got = rho[rows].cpu().numpy()
        if targets is not None:
            got = got[:, targets]
        ok = ~np.isnan(ref)
        d = np.abs(got[ok] - ref[ok])
        out[prec] = {"pairs_checked": int(ok.sum()), "max_abs_diff": float(d.max(initial=0.0)),
                     "p99_abs_diff": float(np.percentile(d, 99)) if d.size else 0.0,
                     "nan_pattern_equal": bool(np.array_equal(np.isnan(got), np.isnan(ref)))}
        del rho
    return out


def emit(name, rec, t0):
    rec = dict(rec)
    rec["workload"] = name
    rec["seconds"] = round(time.time() - t0, 1)
    print(json.dumps(rec), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="fewer sampled libraries")
    args = ap.parse_args()
    q = args.quick
    rng = np.random.default_rng(2105)

    # 16 x 200 coupled logistic, E in 1..10, the full matrix
    t0 = time.time()
    X = inputs.logistic_16x200()
    rows = list(range(16))
    E_gpu, rep = optimal_E_report(X, rows, 10, 1, 1)
    rep["knn_mismatch"], rep["knn_checked"] = knn_mismatch(X, rows, E_gpu, 1, 0)
    rep["ccm"] = ccm_report(gpu(X), X, E_gpu, rows, 1, 0)
    emit("coupled logistic 16 x 200", rep, t0)

    # 1,000 x 1,000 coupled logistic + noise, E in 1..20
    t0 = time.time()
    X = inputs.logistic_noisy()
    rows = sorted(rng.choice(1000, 32 if q else 128, replace=False).tolist())
    E_gpu, rep = optimal_E_report(X, rows, 20, 1, 1)
    rep["knn_mismatch"], rep["knn_checked"] = knn_mismatch(X, rows[:16], E_gpu, 1, 0)
    rep["ccm"] = ccm_report(gpu(X), X, E_gpu, rows, 1, 0)
    emit("coupled logistic 1,000 x 1,000", rep, t0)

    # 50,000 x 1,500 calcium-shaped, sampled libraries against all targets
    t0 = time.time()
    X = inputs.calcium()
    rows = sorted(rng.choice(50000, 8 if q else 32, replace=False).tolist())
    E_gpu, rep = optimal_E_report(X, rows, 20, 1, 1)
    rep["knn_mismatch"], rep["knn_checked"] = knn_mismatch(X, rows[:8], E_gpu, 1, 0)
    Xg = gpu(X)
    rep["ccm"] = ccm_report(Xg, X, E_gpu, rows, 1, 0)
    del Xg
    torch.cuda.empty_cache()
    emit("calcium-shaped 50,000 x 1,500", rep, t0)

    # 2,000 x 10,000 coupled logistic: library-length windows, 1,000 sampled
    # (library, target) pairs per window, E from the full-length simplex
    t0 = time.time()
    X = inputs.logistic_long()
    Xg = gpu(X)
    E_full, _ = edm.edm_simplex_optimal_E(Xg, 20, 1, 1, with_rho=False)
    E_np = E_full.cpu().numpy()
    srows = sorted(rng.choice(2000, 8 if q else 40, replace=False).tolist())
    E_or, _ = oracle.optimal_E_many(X[srows], 20, 1, 1)
    rep = {"E_star_equal_sampled": int(np.sum(E_or == E_np[srows])),
           "E_star_sampled": len(srows), "windows": {}}
    lib_rows = sorted(rng.choice(2000, 10 if q else 40, replace=False).tolist())
    tgts = sorted(rng.choice(2000, 25, replace=False).tolist())
    for L_lib in (100, 300, 1000, 3000, 10000):
        w = {}
        Xw = np.ascontiguousarray(X[:, :L_lib])
        ref = oracle.ccm_matrix(Xw[lib_rows], Xw[tgts], E_np[lib_rows], 1, 0)
        for prec in ("fp32", "fp16", "bf16"):
            rho = edm.edm_ccm_window(Xg, 0, L_lib, E_full, 1, 0, prec)
            edm.edm_ctx_sync()
            got = rho.cpu().numpy()[np.ix_(lib_rows, tgts)]
            ok = ~np.isnan(ref)
            d = np.abs(got[ok] - ref[ok])
            w[prec] = {"pairs_checked": int(ok.sum()), "max_abs_diff": float(d.max(initial=0.0)),
                       "p99_abs_diff": float(np.percentile(d, 99)) if d.size else 0.0}
            del rho
        rep["windows"][str(L_lib)] = w
    emit("library-length windows 2,000 x 10,000", rep, t0)


if __name__ == "__main__":
    main()
