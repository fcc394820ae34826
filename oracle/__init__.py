"""FP64 CPU oracle for convergent cross mapping (kEDM section 2.1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (``paper_2105_12301_gb300``) never does.

The arithmetic lives in ``edm_oracle.c`` (plain C, double precision); this
module only marshals numpy arrays through ctypes.  ctypes releases the GIL
during a foreign call, so the ``*_many`` helpers run one library per Python
thread on all host cores.
"""
import ctypes
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        c_int = ctypes.c_int
        lib.oracle_n_rows.argtypes = [c_int] * 4
        lib.oracle_n_rows.restype = c_int
        lib.oracle_embed.argtypes = [f32p, c_int, c_int, c_int, f64p]
        lib.oracle_knn.argtypes = [f32p] + [c_int] * 5 + [i32p, f64p]
        lib.oracle_knn_row.argtypes = [f32p] + [c_int] * 6 + [i32p, f64p]
        lib.oracle_weights.argtypes = [f64p, c_int, f64p]
        lib.oracle_weights.restype = None
        lib.oracle_predict.argtypes = [i32p, f64p, c_int, c_int, f32p, c_int,
                                       c_int, f64p, f64p]
        lib.oracle_pearson.argtypes = [f64p, f64p, c_int]
        lib.oracle_pearson.restype = ctypes.c_double
        lib.oracle_ccm_row.argtypes = [f32p, f32p] + [c_int] * 5 + [f64p]
        lib.oracle_simplex_rho.argtypes = [f32p] + [c_int] * 4
        lib.oracle_simplex_rho.restype = ctypes.c_double
        lib.oracle_optimal_E.argtypes = [f32p] + [c_int] * 4 + [i32p, f64p]
        lib.oracle_argmax_E.argtypes = [f64p, c_int]
        lib.oracle_argmax_E.restype = c_int
        for name in ("oracle_embed", "oracle_knn", "oracle_knn_row",
                     "oracle_predict", "oracle_ccm_row", "oracle_optimal_E"):
            getattr(lib, name).restype = c_int
        _lib = lib
    return _lib


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed (rc=%d)" % (what, rc))


def n_rows(L, E, tau, Tp):
    return _load().oracle_n_rows(L, E, tau, Tp)


def embed(x, E, tau):
    x = _f32(x)
    L = x.shape[0]
    out = np.empty((L - (E - 1) * tau, E), np.float64)
    _check(_load().oracle_embed(x, L, E, tau, out), "embed")
    return out


def knn(x, E, tau, Tp, k=None):
    """All-kNN table of one series: (idx [n][k] int32 time indices,
    dist [n][k] float64), ascending, self excluded, ties to lower index."""
    x = _f32(x)
    k = E + 1 if k is None else k
    L = x.shape[0]
    n = n_rows(L, E, tau, Tp)
    if n < 2:
        raise ValueError("too few points")
    idx = np.empty((n, k), np.int32)
    dist = np.empty((n, k), np.float64)
    _check(_load().oracle_knn(x, L, E, tau, Tp, k, idx, dist), "knn")
    return idx, dist


def knn_row(x, E, tau, Tp, t, k=None):
    x = _f32(x)
    k = E + 1 if k is None else k
    idx = np.empty(k, np.int32)
    dist = np.empty(k, np.float64)
    _check(_load().oracle_knn_row(x, x.shape[0], E, tau, Tp, k, int(t), idx,
                                  dist), "knn_row")
    return idx, dist


def weights(dist_row):
    d = np.ascontiguousarray(dist_row, np.float64)
    w = np.empty_like(d)
    _load().oracle_weights(d, d.shape[0], w)
    return w


def predict(idx, dist, y, t0, Tp):
    idx = np.ascontiguousarray(idx, np.int32)
    dist = np.ascontiguousarray(dist, np.float64)
    n, k = idx.shape
    pred = np.empty(n, np.float64)
    obs = np.empty(n, np.float64)
    _check(_load().oracle_predict(idx, dist, n, k, _f32(y), t0, Tp, pred, obs),
           "predict")
    return pred, obs


def pearson(a, b):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    return _load().oracle_pearson(a, b, a.shape[0])


def simplex_rho(x, E, tau, Tp):
    x = _f32(x)
    return _load().oracle_simplex_rho(x, x.shape[0], E, tau, Tp)


def optimal_E(x, E_max, tau, Tp_sel):
    """(E_opt, rho_E[E_max]) for one series."""
    x = _f32(x)
    e = np.zeros(1, np.int32)
    rho = np.empty(E_max, np.float64)
    _check(_load().oracle_optimal_E(x, x.shape[0], E_max, tau, Tp_sel, e, rho),
           "optimal_E")
    return int(e[0]), rho


def argmax_E(rho_E):
    """E* (1-based) of the skills rho_E[E-1]: NaN below every number, ties to
    the smaller E, 1 when all are NaN."""
    r = np.ascontiguousarray(rho_E, np.float64)
    return int(_load().oracle_argmax_E(r, r.shape[0]))


def ccm_row(x_lib, Y, E, tau, Tp):
    """rho[j] for library x_lib (embedded at E) against every target row of Y."""
    x_lib = _f32(x_lib)
    Y = _f32(Y)
    if Y.ndim == 1:
        Y = Y[None, :]
    rho = np.empty(Y.shape[0], np.float64)
    _check(_load().oracle_ccm_row(x_lib, Y, Y.shape[0], Y.shape[1], E, tau, Tp,
                                  rho), "ccm_row")
    return rho


def _threads(threads):
    return threads or os.cpu_count() or 1


def optimal_E_many(X, E_max, tau, Tp_sel, threads=None):
    X = _f32(X)
    with ThreadPoolExecutor(_threads(threads)) as ex:
        res = list(ex.map(lambda i: optimal_E(X[i], E_max, tau, Tp_sel),
                          range(X.shape[0])))
    return (np.array([r[0] for r in res], np.int32),
            np.stack([r[1] for r in res]) if res else np.zeros((0, E_max)))


def ccm_matrix(X_lib, Y, E_lib, tau, Tp, lib_rows=None, threads=None):
    """rho[i][j] for the library rows lib_rows (default all) of X_lib."""
    X_lib = _f32(X_lib)
    Y = _f32(Y)
    rows = range(X_lib.shape[0]) if lib_rows is None else list(lib_rows)
    with ThreadPoolExecutor(_threads(threads)) as ex:
        res = list(ex.map(lambda i: ccm_row(X_lib[i], Y, int(E_lib[i]), tau, Tp),
                          rows))
    return np.stack(res) if res else np.zeros((0, Y.shape[0]))
