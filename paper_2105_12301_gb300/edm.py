"""ctypes binding of libedm (include/edm.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libedm.so.  Tensors must be CUDA tensors (float32 series, int32
E arrays), C-contiguous; results are allocated as CUDA tensors on the same
device.  Calls are enqueued on torch's current stream of that device.

There is no CPU path: if libedm.so is missing or no GPU is present, the
calls raise.
"""
import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libedm.so")

EDM_OK = 0
EDM_FP32 = 0
EDM_BF16_TARGETS = 1
EDM_FP16_TARGETS = 2
EDM_E_MAX = 20
EDM_K_MAX = 24
EDM_L_MAX = 65535

_STATUS = {0: "EDM_OK", 1: "EDM_ERR_INVALID_ARG", 2: "EDM_ERR_CUDA", 3: "EDM_ERR_OOM",
           4: "EDM_ERR_TIMEOUT", 5: "EDM_ERR_INTERNAL"}


class EdmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS.get(status, str(status)), message))
        self.status = status


class edm_instance(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int), ("L", ctypes.c_int),
                ("E_lib", ctypes.c_void_p), ("tau", ctypes.c_int), ("Tp", ctypes.c_int),
                ("rho", ctypes.c_void_p), ("lib_begin", ctypes.c_int),
                ("lib_end", ctypes.c_int)]


_lib = None
_lock = threading.Lock()
_ctxs = {}


def load():
    """Load libedm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libedm.so not found at %s: run "
                           "`python -m paper_2105_12301_gb300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci = ctypes.c_void_p, ctypes.c_int
    lib.edm_create.argtypes = [ctypes.POINTER(vp), ci, vp]
    lib.edm_destroy.argtypes = [vp]
    lib.edm_set_stream.argtypes = [vp, vp]
    lib.edm_ctx_sync.argtypes = [vp]
    lib.edm_status_string.argtypes = [ci]
    lib.edm_status_string.restype = ctypes.c_char_p
    lib.edm_last_error.argtypes = [vp]
    lib.edm_last_error.restype = ctypes.c_char_p
    lib.edm_kernel_launches.argtypes = [vp]
    lib.edm_kernel_launches.restype = ctypes.c_uint64
    lib.edm_embed.argtypes = [vp, vp, ci, ci, ci, vp]
    lib.edm_knn.argtypes = [vp, vp, ci, ci, ci, ci, ci, ci, vp, vp]
    lib.edm_simplex_optimal_E.argtypes = [vp, vp, ci, ci, ci, ci, ci, vp, vp]
    lib.edm_ccm_all.argtypes = [vp, vp, ci, vp, ci, ci, vp, ci, ci, ci, vp]
    lib.edm_ccm_batched.argtypes = [vp, ctypes.POINTER(edm_instance), ci, ci]
    lib.edm_ccm_window.argtypes = [vp, vp, ci, ci, ci, ci, vp, ci, ci, ci, vp]
    lib.edm_simplex_optimal_E_batched.argtypes = [vp, ctypes.POINTER(edm_instance), ci, ci, ci,
                                                  ctypes.POINTER(vp)]
    lib.edm_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_longlong]
    lib.edm_simplex_optimal_E_noalloc.argtypes = [vp, ci, ci, ci, ci, ci, vp, vp, vp]
    lib.edm_check_wait_timeout.argtypes = [vp, ci]
    lib.edm_predict.argtypes = [vp, vp, ci, vp, ci, ci, vp, vp, ci, ci, vp]
    lib.edm_ccm_all_target_E.argtypes = [vp, vp, ci, vp, ci, ci, vp, ci, ci, ci, vp]
    lib.edm_ccm_all_host.argtypes = [vp, vp, ci, vp, ci, ci, vp, ci, ci, ci, vp, vp]
    lib.edm_upload_series.argtypes = [vp, vp, ci, ci, vp]
    lib.edm_ccm_rows.argtypes = [vp, vp, ci, ci, ci, ci, vp, ci, ci, ci, vp]
    lib.edm_knn_materialized.argtypes = [vp, vp, ci, ci, ci, ci, ci, ci, vp, vp]
    lib.edm_fallback_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]
    lib.edm_ccm_windows.argtypes = [vp, vp, ci, ci, ctypes.POINTER(ci), ci, ci, vp, ci, ci, ci, vp]
    lib.edm_profile_enable.argtypes = [vp, ci]
    lib.edm_profile_read.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ci)]
    lib.edm_probe_smem_bandwidth.argtypes = [vp, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_double)]
    lib.edm_probe_l2_bandwidth.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    for f in ("edm_create", "edm_destroy", "edm_set_stream", "edm_ctx_sync", "edm_embed",
              "edm_knn", "edm_simplex_optimal_E", "edm_ccm_all", "edm_ccm_batched",
              "edm_profile_enable", "edm_profile_read", "edm_probe_smem_bandwidth",
              "edm_simplex_optimal_E_noalloc", "edm_ccm_window",
              "edm_simplex_optimal_E_batched", "edm_set_option", "edm_check_wait_timeout",
              "edm_predict", "edm_ccm_all_target_E", "edm_ccm_all_host", "edm_ccm_windows",
              "edm_upload_series", "edm_fallback_counts", "edm_ccm_rows",
              "edm_knn_materialized", "edm_probe_l2_bandwidth"):
        getattr(lib, f).restype = ci
    _lib = lib
    return lib


def _ctx(device):
    """The context of a CUDA device, bound to torch's current stream."""
    lib = load()
    dev = torch.device(device)
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    with _lock:
        ctx = _ctxs.get(idx)
        if ctx is None:
            p = ctypes.c_void_p()
            st = lib.edm_create(ctypes.byref(p), idx, None)
            if st != EDM_OK:
                raise EdmError(st, "edm_create(device=%d) failed" % idx)
            ctx = p
            _ctxs[idx] = ctx
    stream = torch.cuda.current_stream(idx).cuda_stream
    lib.edm_set_stream(ctx, ctypes.c_void_p(stream))
    return ctx


def _check(ctx, st, what):
    if st != EDM_OK:
        msg = load().edm_last_error(ctx).decode() if ctx else ""
        raise EdmError(st, "%s: %s" % (what, msg))


def _series(x, name, ndim):
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if x.dtype != torch.float32 or x.dim() != ndim or not x.is_contiguous():
        raise TypeError("%s must be a contiguous float32 tensor with %d dims" % (name, ndim))
    return x


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def edm_ctx_sync(device=None):
    """Wait for the device and raise the first device-side error since the
    previous sync (out-of-range E on the device, a timed-out wait)."""
    dev = device if device is not None else torch.cuda.current_device()
    ctx = _ctx(dev)
    _check(ctx, load().edm_ctx_sync(ctx), "edm_ctx_sync")


def edm_kernel_launches(device=None):
    dev = device if device is not None else torch.cuda.current_device()
    return int(load().edm_kernel_launches(_ctx(dev)))


def edm_profile_enable(on, device=None):
    """Start (clearing the record) or stop per-kernel CUDA-event timing."""
    dev = device if device is not None else torch.cuda.current_device()
    ctx = _ctx(dev)
    _check(ctx, load().edm_profile_enable(ctx, 1 if on else 0), "edm_profile_enable")


def edm_profile_read(kernel, device=None):
    """(summed milliseconds, launches) of the recorded launches of `kernel`."""
    dev = device if device is not None else torch.cuda.current_device()
    ctx = _ctx(dev)
    ms, n = ctypes.c_double(), ctypes.c_int()
    _check(ctx, load().edm_profile_read(ctx, kernel.encode(), ctypes.byref(ms), ctypes.byref(n)),
           "edm_profile_read")
    return ms.value, n.value


def edm_probe_smem_bandwidth(ms=200.0, device=None):
    """Measured shared-memory gather bandwidth of the GPU, bytes/s."""
    dev = device if device is not None else torch.cuda.current_device()
    ctx = _ctx(dev)
    bw = ctypes.c_double()
    _check(ctx, load().edm_probe_smem_bandwidth(ctx, float(ms), ctypes.byref(bw)),
           "edm_probe_smem_bandwidth")
    return bw.value


def edm_probe_l2_bandwidth(ms=200.0, device=None):
    """Measured L2 gather bandwidth of the GPU (128-byte rows at scattered
    indexes of an L2-resident buffer), bytes/s."""
    dev = device if device is not None else torch.cuda.current_device()
    ctx = _ctx(dev)
    bw = ctypes.c_double()
    _check(ctx, load().edm_probe_l2_bandwidth(ctx, float(ms), ctypes.byref(bw)),
           "edm_probe_l2_bandwidth")
    return bw.value


def edm_check_wait_timeout(ms=50, device=None):
    """Enqueue a bounded device-side wait that nothing completes; the next
    edm_ctx_sync raises EdmError(EDM_ERR_TIMEOUT)."""
    dev = device if device is not None else torch.cuda.current_device()
    ctx = _ctx(dev)
    _check(ctx, load().edm_check_wait_timeout(ctx, int(ms)), "edm_check_wait_timeout")


def edm_embed(x, E, tau=1):
    """Delay embedding of one series x [L] -> [L-(E-1)tau][E] float32."""
    _series(x, "x", 1)
    L = x.shape[0]
    out = torch.empty((max(L - (E - 1) * tau, 0), E), dtype=torch.float32, device=x.device)
    ctx = _ctx(x.device)
    _check(ctx, load().edm_embed(ctx, _ptr(x), L, E, tau, _ptr(out)), "edm_embed")
    return out


def edm_knn(X, E, tau=1, Tp=0, k=None, with_dist=True):
    """All-kNN of every series of X [N][L]: (idx [N][n][k] int32 time
    indices, dist [N][n][k] float32 or None)."""
    _series(X, "X", 2)
    N, L = X.shape
    k = E + 1 if k is None else k
    n = L - (E - 1) * tau - Tp
    idx = torch.empty((N, max(n, 0), k), dtype=torch.int32, device=X.device)
    dist = torch.empty((N, max(n, 0), k), dtype=torch.float32, device=X.device) if with_dist else None
    ctx = _ctx(X.device)
    _check(ctx, load().edm_knn(ctx, _ptr(X), N, L, E, tau, Tp, k, _ptr(idx), _ptr(dist)),
           "edm_knn")
    return idx, dist


def edm_knn_materialized(X, E, tau=1, Tp=0, k=None, with_dist=True):
    """edm_knn by the paper's two-kernel route (distance matrix written to
    memory, then per-row selection); the same results, kept as a baseline."""
    _series(X, "X", 2)
    N, L = X.shape
    k = E + 1 if k is None else k
    n = L - (E - 1) * tau - Tp
    idx = torch.empty((N, max(n, 0), k), dtype=torch.int32, device=X.device)
    dist = torch.empty((N, max(n, 0), k), dtype=torch.float32, device=X.device) if with_dist else None
    ctx = _ctx(X.device)
    _check(ctx, load().edm_knn_materialized(ctx, _ptr(X), N, L, E, tau, Tp, k, _ptr(idx),
                                            _ptr(dist)), "edm_knn_materialized")
    return idx, dist


def edm_simplex_optimal_E(X, E_max=EDM_E_MAX, tau=1, Tp_sel=1, with_rho=True):
    """(E_opt [N] int32, rho_E [N][E_max] float32 or None) for X [N][L]."""
    _series(X, "X", 2)
    N, L = X.shape
    E_opt = torch.empty(N, dtype=torch.int32, device=X.device)
    rho_E = torch.empty((N, E_max), dtype=torch.float32, device=X.device) if with_rho else None
    ctx = _ctx(X.device)
    _check(ctx, load().edm_simplex_optimal_E(ctx, _ptr(X), N, L, E_max, tau, Tp_sel,
                                             _ptr(E_opt), _ptr(rho_E)), "edm_simplex_optimal_E")
    return E_opt, rho_E


def edm_simplex_optimal_E_noalloc(X, E_opt, rho_E=None, E_max=EDM_E_MAX, tau=1, Tp_sel=1):
    """Optimal E into caller-allocated outputs, with no device allocation in
    the library (for callers that may not allocate once running; see
    include/edm.h).  E_opt: CUDA int32 [N]; rho_E: CUDA float32 [N][E_max]
    or None.  Runs on torch's current stream of X's device."""
    _series(X, "X", 2)
    N, L = X.shape
    if E_opt.dtype != torch.int32 or E_opt.shape != (N,) or not E_opt.is_cuda:
        raise TypeError("E_opt must be a CUDA int32 tensor of shape [N]")
    if rho_E is not None and (rho_E.dtype != torch.float32 or rho_E.shape != (N, E_max)
                              or not rho_E.is_contiguous()):
        raise TypeError("rho_E must be a contiguous CUDA float32 tensor of shape [N][E_max]")
    stream = torch.cuda.current_stream(X.device).cuda_stream
    with torch.cuda.device(X.device):
        st = load().edm_simplex_optimal_E_noalloc(_ptr(X), N, L, E_max, tau, Tp_sel, _ptr(E_opt),
                                                  _ptr(rho_E), ctypes.c_void_p(stream))
    if st != EDM_OK:
        raise EdmError(st, "edm_simplex_optimal_E_noalloc(N=%d, L=%d, E_max=%d)" % (N, L, E_max))
    return E_opt, rho_E


def _prec(precision):
    if precision in ("fp32", EDM_FP32):
        return EDM_FP32
    if precision in ("bf16", EDM_BF16_TARGETS):
        return EDM_BF16_TARGETS
    if precision in ("fp16", EDM_FP16_TARGETS):
        return EDM_FP16_TARGETS
    raise ValueError("precision must be 'fp32', 'bf16' or 'fp16'")


def edm_ccm_all(X_lib, Y_tgt, E_lib, tau=1, Tp=0, precision="fp32", out=None):
    """rho [N_lib][N_tgt]: skill of library i's manifold at predicting target j."""
    _series(X_lib, "X_lib", 2)
    _series(Y_tgt, "Y_tgt", 2)
    if X_lib.shape[1] != Y_tgt.shape[1]:
        raise ValueError("libraries and targets must have the same length")
    if E_lib.dtype != torch.int32 or not E_lib.is_cuda or E_lib.shape != (X_lib.shape[0],):
        raise TypeError("E_lib must be a CUDA int32 tensor of shape [N_lib]")
    E_lib = E_lib.contiguous()
    N_lib, L = X_lib.shape
    N_tgt = Y_tgt.shape[0]
    rho = out if out is not None else torch.empty((N_lib, N_tgt), dtype=torch.float32,
                                                  device=X_lib.device)
    if rho.shape != (N_lib, N_tgt) or rho.dtype != torch.float32 or not rho.is_contiguous():
        raise TypeError("out must be a contiguous float32 [N_lib][N_tgt] tensor")
    ctx = _ctx(X_lib.device)
    _check(ctx, load().edm_ccm_all(ctx, _ptr(X_lib), N_lib, _ptr(Y_tgt), N_tgt, L, _ptr(E_lib),
                                   tau, Tp, _prec(precision), _ptr(rho)), "edm_ccm_all")
    return rho


def edm_ccm_rows(X, lib_begin, lib_end, E_lib, tau=1, Tp=0, precision="fp32", out=None):
    """Rows lib_begin..lib_end-1 of the all-to-all rho matrix of the series X
    [N][L] (libraries and targets alike): [lib_end-lib_begin][N] float32."""
    _series(X, "X", 2)
    N, L = X.shape
    if not (0 <= lib_begin <= lib_end <= N):
        raise ValueError("need 0 <= lib_begin <= lib_end <= N")
    if E_lib.dtype != torch.int32 or not E_lib.is_cuda or E_lib.numel() != N:
        raise TypeError("E_lib must be a CUDA int32 tensor of N entries")
    rho = out if out is not None else torch.empty((lib_end - lib_begin, N), dtype=torch.float32,
                                                  device=X.device)
    ctx = _ctx(X.device)
    _check(ctx, load().edm_ccm_rows(ctx, _ptr(X), N, L, lib_begin, lib_end,
                                    _ptr(E_lib.contiguous()), tau, Tp, _prec(precision),
                                    _ptr(rho)), "edm_ccm_rows")
    return rho


def edm_ccm_all_host(X_lib, Y_tgt, E_lib, out, out_host, tau=1, Tp=0, precision="fp32"):
    """edm_ccm_all into the device tensor `out` [N_lib][N_tgt] and, block by
    block while the computation continues, into the pinned CPU tensor
    `out_host` of the same shape; both are complete once torch's current
    stream reaches this point."""
    _series(X_lib, "X_lib", 2)
    _series(Y_tgt, "Y_tgt", 2)
    if X_lib.shape[1] != Y_tgt.shape[1]:
        raise ValueError("libraries and targets must have the same length")
    N_lib, L = X_lib.shape
    N_tgt = Y_tgt.shape[0]
    if E_lib.dtype != torch.int32 or not E_lib.is_cuda or E_lib.shape != (N_lib,):
        raise TypeError("E_lib must be a CUDA int32 tensor of shape [N_lib]")
    for name, t, cuda in (("out", out, True), ("out_host", out_host, False)):
        if (t.shape != (N_lib, N_tgt) or t.dtype != torch.float32 or not t.is_contiguous()
                or t.is_cuda != cuda):
            raise TypeError("%s must be a contiguous float32 [N_lib][N_tgt] %s tensor"
                            % (name, "CUDA" if cuda else "CPU"))
    if not out_host.is_pinned():
        raise TypeError("out_host must be in pinned memory")
    ctx = _ctx(X_lib.device)
    _check(ctx, load().edm_ccm_all_host(ctx, _ptr(X_lib), N_lib, _ptr(Y_tgt), N_tgt, L,
                                        _ptr(E_lib.contiguous()), tau, Tp, _prec(precision),
                                        _ptr(out), _ptr(out_host)), "edm_ccm_all_host")
    return out, out_host


def edm_fallback_counts(device=None):
    """(band_rows, brute_rows) counted since the previous call while the
    option "diagnostics" is 1: query rows (per E) resolved in FP64 because a
    candidate fell in the band around the k-th distance, and rows that needed
    a full FP64 scan."""
    dev = device if device is not None else torch.cuda.current_device()
    ctx = _ctx(dev)
    band, brute = ctypes.c_uint64(), ctypes.c_uint64()
    _check(ctx, load().edm_fallback_counts(ctx, ctypes.byref(band), ctypes.byref(brute)),
           "edm_fallback_counts")
    return int(band.value), int(brute.value)


def edm_upload_series(X_host, out):
    """Copy the page-locked host series X_host [N][L] (float32) into the CUDA
    tensor `out` of the same shape, ordered on torch's current stream."""
    if not isinstance(X_host, torch.Tensor) or X_host.is_cuda or not X_host.is_pinned():
        raise TypeError("X_host must be a page-locked (pinned) CPU tensor")
    if X_host.dtype != torch.float32 or X_host.dim() != 2 or not X_host.is_contiguous():
        raise TypeError("X_host must be a contiguous float32 [N][L] tensor")
    _series(out, "out", 2)
    if tuple(out.shape) != tuple(X_host.shape):
        raise ValueError("out must have the shape of X_host")
    ctx = _ctx(out.device)
    N, L = X_host.shape
    _check(ctx, load().edm_upload_series(ctx, ctypes.c_void_p(X_host.data_ptr()), N, L,
                                         _ptr(out)), "edm_upload_series")
    return out


def edm_ccm_all_target_E(X_lib, Y_tgt, E_tgt, tau=1, Tp=0, precision="fp32", out=None):
    """rho [N_lib][N_tgt] with every library embedded at each target's E
    (E_tgt: CUDA int32 [N_tgt]); synchronises the stream once."""
    _series(X_lib, "X_lib", 2)
    _series(Y_tgt, "Y_tgt", 2)
    if X_lib.shape[1] != Y_tgt.shape[1]:
        raise ValueError("libraries and targets must have the same length")
    N_lib, L = X_lib.shape
    N_tgt = Y_tgt.shape[0]
    if E_tgt.dtype != torch.int32 or not E_tgt.is_cuda or E_tgt.shape != (N_tgt,):
        raise TypeError("E_tgt must be a CUDA int32 tensor of shape [N_tgt]")
    rho = out if out is not None else torch.empty((N_lib, N_tgt), dtype=torch.float32,
                                                  device=X_lib.device)
    if rho.shape != (N_lib, N_tgt) or rho.dtype != torch.float32 or not rho.is_contiguous():
        raise TypeError("out must be a contiguous float32 [N_lib][N_tgt] tensor")
    ctx = _ctx(X_lib.device)
    _check(ctx, load().edm_ccm_all_target_E(ctx, _ptr(X_lib), N_lib, _ptr(Y_tgt), N_tgt, L,
                                            _ptr(E_tgt.contiguous()), tau, Tp, _prec(precision),
                                            _ptr(rho)), "edm_ccm_all_target_E")
    return rho


def edm_predict(X_lib, Y_tgt, E_lib, tgt_of_lib=None, tau=1, Tp=0, out=None):
    """pred [N_lib][L]: simplex prediction of target tgt_of_lib[i] (target i
    when None) from library i's manifold at time t+Tp for every library point
    t; NaN elsewhere."""
    _series(X_lib, "X_lib", 2)
    _series(Y_tgt, "Y_tgt", 2)
    if X_lib.shape[1] != Y_tgt.shape[1]:
        raise ValueError("libraries and targets must have the same length")
    N_lib, L = X_lib.shape
    for name, a in (("E_lib", E_lib), ("tgt_of_lib", tgt_of_lib)):
        if a is not None and (a.dtype != torch.int32 or not a.is_cuda or a.shape != (N_lib,)):
            raise TypeError("%s must be a CUDA int32 tensor of shape [N_lib]" % name)
    pred = out if out is not None else torch.empty((N_lib, L), dtype=torch.float32,
                                                   device=X_lib.device)
    if pred.shape != (N_lib, L) or pred.dtype != torch.float32 or not pred.is_contiguous():
        raise TypeError("out must be a contiguous float32 [N_lib][L] tensor")
    tgt = tgt_of_lib.contiguous() if tgt_of_lib is not None else None
    ctx = _ctx(X_lib.device)
    _check(ctx, load().edm_predict(ctx, _ptr(X_lib), N_lib, _ptr(Y_tgt), Y_tgt.shape[0], L,
                                   _ptr(E_lib.contiguous()), _ptr(tgt), tau, Tp, _ptr(pred)),
           "edm_predict")
    return pred


def edm_ccm_window(X, offset, L_win, E_lib, tau=1, Tp=0, precision="fp32", out=None):
    """rho [N][N] of all-to-all CCM on the windows X[:, offset:offset+L_win]."""
    _series(X, "X", 2)
    N, ld = X.shape
    if E_lib.dtype != torch.int32 or not E_lib.is_cuda or E_lib.shape != (N,):
        raise TypeError("E_lib must be a CUDA int32 tensor of shape [N]")
    rho = out if out is not None else torch.empty((N, N), dtype=torch.float32, device=X.device)
    ctx = _ctx(X.device)
    _check(ctx, load().edm_ccm_window(ctx, _ptr(X), N, ld, offset, L_win, _ptr(E_lib.contiguous()),
                                      tau, Tp, _prec(precision), _ptr(rho)), "edm_ccm_window")
    return rho


def edm_ccm_windows(X, offsets, L_win, E_lib, tau=1, Tp=0, precision="fp32", out=None):
    """rho [n_windows][N][N]: all-to-all CCM on the windows
    X[:, o:o+L_win] for every offset o in `offsets` (a list of ints)."""
    _series(X, "X", 2)
    N, ld = X.shape
    if E_lib.dtype != torch.int32 or not E_lib.is_cuda or E_lib.shape != (N,):
        raise TypeError("E_lib must be a CUDA int32 tensor of shape [N]")
    offs = (ctypes.c_int * len(offsets))(*[int(o) for o in offsets])
    rho = out if out is not None else torch.empty((len(offsets), N, N), dtype=torch.float32,
                                                  device=X.device)
    if rho.shape != (len(offsets), N, N) or rho.dtype != torch.float32 or not rho.is_contiguous():
        raise TypeError("out must be a contiguous float32 [n_windows][N][N] tensor")
    ctx = _ctx(X.device)
    _check(ctx, load().edm_ccm_windows(ctx, _ptr(X), N, ld, offs, len(offsets), L_win,
                                       _ptr(E_lib.contiguous()), tau, Tp, _prec(precision),
                                       _ptr(rho)), "edm_ccm_windows")
    return rho


def edm_set_option(name, value, device=None):
    """Set an execution option of the device's context (see include/edm.h)."""
    dev = device if device is not None else torch.cuda.current_device()
    ctx = _ctx(dev)
    _check(ctx, load().edm_set_option(ctx, name.encode(), int(value)), "edm_set_option")


def _instances(problems):
    arr = (edm_instance * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        X = _series(p["X"], "X", 2)
        N, L = X.shape
        E_lib = p.get("E_lib")
        E_ptr = 0
        if E_lib is not None:
            E_lib = E_lib.contiguous()
            E_ptr = E_lib.data_ptr()
        rho = p.get("rho")
        arr[i] = edm_instance(X.data_ptr(), N, L, E_ptr, p.get("tau", 1), p.get("Tp", 0),
                              rho.data_ptr() if rho is not None else 0,
                              p.get("lib_begin", 0), p.get("lib_end", N))
        keep.append((X, E_lib, rho))
    return arr, keep


def edm_simplex_optimal_E_batched(problems, E_max=EDM_E_MAX, Tp_sel=1, out=None):
    """Optimal E of every series of every problem (dicts with X, tau).  `out`:
    optional list of CUDA int32 [N_i] tensors to write (the same tensors on
    every call let a captured batch be replayed)."""
    if not problems:
        return []
    arr, keep = _instances(problems)
    if out is None:
        outs = [torch.empty(p["X"].shape[0], dtype=torch.int32, device=p["X"].device)
                for p in problems]
    else:
        outs = list(out)
        for o, p in zip(outs, problems):
            if o.dtype != torch.int32 or o.shape != (p["X"].shape[0],) or not o.is_cuda:
                raise TypeError("out[i] must be a CUDA int32 tensor of shape [N_i]")
    ptrs = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
    ctx = _ctx(problems[0]["X"].device)
    _check(ctx, load().edm_simplex_optimal_E_batched(ctx, arr, len(problems), E_max, Tp_sel, ptrs),
           "edm_simplex_optimal_E_batched")
    return outs


def edm_ccm_batched(problems, precision="fp32"):
    """problems: list of dicts with X [N][L], E_lib [N] int32, tau, Tp, optional
    lib_begin/lib_end and optional preallocated rho; returns the rho blocks."""
    if not problems:
        return []
    rhos = []
    probs = []
    for p in problems:
        N = p["X"].shape[0]
        b, e = p.get("lib_begin", 0), p.get("lib_end", N)
        rho = p.get("rho")
        if rho is None:
            rho = torch.empty((e - b, N), dtype=torch.float32, device=p["X"].device)
        q = dict(p)
        q["rho"] = rho
        probs.append(q)
        rhos.append(rho)
    arr, keep = _instances(probs)
    ctx = _ctx(problems[0]["X"].device)
    _check(ctx, load().edm_ccm_batched(ctx, arr, len(probs), _prec(precision)),
           "edm_ccm_batched")
    return rhos
