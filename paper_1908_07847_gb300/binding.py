"""Thin ctypes binding of libmlp_gb300.so with the C ABI's names.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Device buffers are passed as integers (``tensor.data_ptr()``) and
streams as ``torch.cuda.current_stream().cuda_stream`` (or 0).  A missing or
unloadable library raises ``MLPError``; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

MLP_OK, MLP_EINVAL, MLP_ENOMEM, MLP_ECUDA, MLP_ETIMEOUT, MLP_ENONFINITE, MLP_EUNSUPPORTED = range(7)
MLP_FP32, MLP_BF16, MLP_FP64 = 0, 1, 2
MLP_ACT_SIGMOID, MLP_ACT_TANH = 0, 1
MLP_PATH_FUSED, MLP_PATH_TC_CLUSTER, MLP_PATH_PLAIN = 0, 1, 2
STATUS_NAMES = {0: "MLP_OK", 1: "MLP_EINVAL", 2: "MLP_ENOMEM", 3: "MLP_ECUDA", 4: "MLP_ETIMEOUT",
                5: "MLP_ENONFINITE", 6: "MLP_EUNSUPPORTED"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libmlp_gb300.so")

# Every symbol the header declares (checked by the CPU tests).
EXPORTS = [
    "mlp_create", "mlp_destroy", "mlp_set_weights", "mlp_get_weights", "mlp_weights_device",
    "mlp_forward", "mlp_backward", "mlp_update", "mlp_grad_sum", "mlp_step_plain", "mlp_train_epochs",
    "mlp_train_host", "mlp_train_path", "mlp_predict", "mlp_check", "mlp_workspace_bytes", "mlp_forward_w",
    "mlp_backward_w", "mlp_debug_skip_block", "mlp_set_rows_per_block", "mlp_set_clusters",
    "mlp_cluster_limit", "mlp_batch_train",
    "mlp_batch_create", "mlp_batch_run", "mlp_batch_check", "mlp_batch_destroy", "mlp_batch_create_host",
    "mlp_batch_run_host", "mlp_batch_set_shape", "mlp_batch_get_shape", "mlp_train_fused_noalloc",
    "mlp_zscore_workspace_bytes", "mlp_zscore", "mlp_unit_rates", "mlp_last_error", "mlp_version",
]


class MLPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class mlp_config(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int32), ("H", ctypes.c_int32), ("lr", ctypes.c_float),
                ("loss_mean", ctypes.c_int32), ("prec", ctypes.c_int32), ("act", ctypes.c_int32)]


class mlp_net_desc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("n", ctypes.c_int64), ("X", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("params", ctypes.c_void_p), ("loss_hist", ctypes.c_void_p),
                ("gnorm_hist", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load the library (raises MLPError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise MLPError(-1, "CUDA library not built: %s (run __graft_entry__.build())" % LIB_PATH)
        try:
            import torch  # noqa: F401  (loads the same libcudart first)
        except Exception:
            pass
        L = ctypes.CDLL(LIB_PATH)
        S, V, I32, I64, F, U64 = (ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_float, ctypes.c_uint64)
        sig = {
            "mlp_create": (S, [ctypes.POINTER(mlp_config), ctypes.POINTER(V)]),
            "mlp_destroy": (None, [V]),
            "mlp_set_weights": (S, [V, V, V, V, V]),
            "mlp_get_weights": (S, [V, V, V, V, V]),
            "mlp_weights_device": (S, [V, ctypes.POINTER(V)]),
            "mlp_forward": (S, [V, V, I64, V, V]),
            "mlp_backward": (S, [V, V, V, I64, V, V, V, V, V, V]),
            "mlp_update": (S, [V, V, V, V, V, V]),
            "mlp_step_plain": (S, [V, V, V, I64, V, V]),
            "mlp_train_epochs": (S, [V, V, V, I64, I32, I64, V, V, V]),
            "mlp_train_host": (S, [V, V, V, I64, I32, I64, V, V]),
            "mlp_train_path": (S, [V, I64, I64, ctypes.POINTER(I32)]),
            "mlp_predict": (S, [V, V, I64, V, V]),
            "mlp_check": (S, [V, V]),
            "mlp_workspace_bytes": (S, [I32, I32, I32, I64, ctypes.POINTER(U64)]),
            "mlp_forward_w": (S, [I32, I32, I32, I32, I64, V, V, V, V, V, V, V, V, U64, V]),
            "mlp_backward_w": (S, [I32, I32, I32, I32, I64, V, V, V, V, V, V, V, V, V, V, V, V, U64, V]),
            "mlp_debug_skip_block": (S, [V, I32]),
            "mlp_set_rows_per_block": (S, [V, I32]),
            "mlp_set_clusters": (S, [V, I32]),
            "mlp_grad_sum": (S, [V, V, I32, I64, F, ctypes.c_double, V, V, V]),
            "mlp_cluster_limit": (S, [I32, ctypes.POINTER(I32)]),
            "mlp_batch_train": (S, [I32, I32, I32, ctypes.POINTER(mlp_net_desc), I32, I32, F, I32, V]),
            "mlp_batch_create": (S, [I32, I32, I32, ctypes.POINTER(mlp_net_desc), I32, F, I32, ctypes.POINTER(V)]),
            "mlp_batch_run": (S, [V, I32, V]),
            "mlp_batch_check": (S, [V, V]),
            "mlp_batch_destroy": (None, [V]),
            "mlp_batch_create_host": (S, [I32, I32, I32, V, V, I32, I32, F, I32, ctypes.POINTER(V)]),
            "mlp_batch_run_host": (S, [V, V, V, V, V, V, I32, V]),
            "mlp_batch_set_shape": (S, [V, I32]),
            "mlp_batch_get_shape": (S, [V, ctypes.POINTER(I32)]),
            "mlp_train_fused_noalloc": (S, [I32, I32, I32, I64, V, V, V, F, I32, I32, I64, V, V, V]),
            "mlp_last_error": (ctypes.c_char_p, []),
            "mlp_version": (ctypes.c_char_p, []),
            "mlp_unit_rates": (S, [ctypes.POINTER(ctypes.c_double)] * 3),
            "mlp_zscore_workspace_bytes": (S, [I32, ctypes.POINTER(U64)]),
            "mlp_zscore": (S, [V, I64, I32, I64, I32, I32, V, V, V, V, U64, V]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _ck(status):
    if status != MLP_OK:
        raise MLPError(status, lib().mlp_last_error().decode())
    return status


def _p(x):
    """Device/host address of a torch tensor, numpy array, int or None.  The
    library reads and writes dense row-major buffers, so a tensor or array
    view that is not C-contiguous is refused rather than misread."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor is not contiguous (call .contiguous() first)")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array is not C-contiguous (use numpy.ascontiguousarray)")
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


# ----------------------------------------------------------------- handle API

def mlp_create(D, H, lr=0.1, loss_mean=1, prec=MLP_FP32, act=MLP_ACT_SIGMOID):
    cfg = mlp_config(D, H, lr, loss_mean, prec, act)
    h = ctypes.c_void_p()
    _ck(lib().mlp_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def mlp_destroy(h):
    lib().mlp_destroy(h)


def mlp_set_weights(h, W1, b1, w2, b2):
    return _ck(lib().mlp_set_weights(h, _p(W1), _p(b1), _p(w2), _p(b2)))


def mlp_get_weights(h, W1, b1, w2, b2):
    return _ck(lib().mlp_get_weights(h, _p(W1), _p(b1), _p(w2), _p(b2)))


def mlp_weights_device(h):
    p = ctypes.c_void_p()
    _ck(lib().mlp_weights_device(h, ctypes.byref(p)))
    return p.value


def mlp_forward(h, X, n, o, stream=0):
    return _ck(lib().mlp_forward(h, _p(X), n, _p(o), stream))


def mlp_backward(h, X, y, n, gW1, gb1, gw2, gb2, loss=None, stream=0):
    return _ck(lib().mlp_backward(h, _p(X), _p(y), n, _p(gW1), _p(gb1), _p(gw2), _p(gb2), _p(loss), stream))


def mlp_update(h, gW1, gb1, gw2, gb2, stream=0):
    return _ck(lib().mlp_update(h, _p(gW1), _p(gb1), _p(gw2), _p(gb2), stream))


def mlp_step_plain(h, X, y, n, loss=None, stream=0):
    return _ck(lib().mlp_step_plain(h, _p(X), _p(y), n, _p(loss), stream))


def mlp_train_epochs(h, X, y, n, epochs, minibatch=0, loss_hist=None, gnorm_hist=None, stream=0):
    return _ck(lib().mlp_train_epochs(h, _p(X), _p(y), n, epochs, minibatch, _p(loss_hist), _p(gnorm_hist),
                                      stream))


def mlp_train_host(h, X_host, y_host, n, epochs, minibatch=0, loss_hist_host=None, stream=0):
    return _ck(lib().mlp_train_host(h, _p(X_host), _p(y_host), n, epochs, minibatch, _p(loss_hist_host), stream))


def mlp_train_path(h, n, minibatch=0):
    """MLP_PATH_FUSED, MLP_PATH_TC_CLUSTER or MLP_PATH_PLAIN: the path
    mlp_train_epochs takes for this handle and size."""
    v = ctypes.c_int32()
    _ck(lib().mlp_train_path(h, n, minibatch, ctypes.byref(v)))
    return v.value


def mlp_predict(h, X, n, labels, stream=0):
    return _ck(lib().mlp_predict(h, _p(X), n, _p(labels), stream))


def mlp_check(h, stream=0):
    """Returns the status code (does not raise)."""
    return lib().mlp_check(h, stream)


def mlp_debug_skip_block(h, b):
    return _ck(lib().mlp_debug_skip_block(h, b))


def mlp_set_rows_per_block(h, rows):
    return _ck(lib().mlp_set_rows_per_block(h, rows))


def mlp_grad_sum(parts, loss_parts, nparts, length, scale, loss_scale, out, loss_acc, stream=0):
    """out = scale * rank-order sum of the nparts x length gradient rows in
    parts; loss_acc += loss_scale * rank-order sum of loss_parts."""
    return _ck(lib().mlp_grad_sum(_p(parts), _p(loss_parts), nparts, length, scale, loss_scale, _p(out),
                                  _p(loss_acc), stream))


def mlp_set_clusters(h, clusters):
    """Cap the bf16 wide-network kernel's cluster count (0 = the default)."""
    return _ck(lib().mlp_set_clusters(h, clusters))


def mlp_cluster_limit(H):
    """Most clusters of H/256 blocks the current device keeps resident."""
    k = ctypes.c_int32()
    _ck(lib().mlp_cluster_limit(H, ctypes.byref(k)))
    return k.value


# ------------------------------------------------------------ handle-free API

def mlp_workspace_bytes(prec, D, H, n):
    b = ctypes.c_uint64()
    _ck(lib().mlp_workspace_bytes(prec, D, H, n, ctypes.byref(b)))
    return b.value


def mlp_forward_w(prec, act, D, H, n, X, W1, b1, w2, b2, hid, o, ws, ws_bytes, stream=0):
    return _ck(lib().mlp_forward_w(prec, act, D, H, n, _p(X), _p(W1), _p(b1), _p(w2), _p(b2), _p(hid), _p(o),
                                   _p(ws), ws_bytes, stream))


def mlp_backward_w(prec, act, D, H, n, X, W1, w2, hid, o, dLdo, gW1, gb1, gw2, gb2, gX, ws, ws_bytes, stream=0):
    return _ck(lib().mlp_backward_w(prec, act, D, H, n, _p(X), _p(W1), _p(w2), _p(hid), _p(o), _p(dLdo),
                                    _p(gW1), _p(gb1), _p(gw2), _p(gb2), _p(gX), _p(ws), ws_bytes, stream))


def mlp_batch_train(prec, act, D, descs, epochs, lr, loss_mean=1, stream=0):
    arr = (mlp_net_desc * max(len(descs), 1))(*descs)
    return _ck(lib().mlp_batch_train(prec, act, D, arr, len(descs), epochs, lr, loss_mean, stream))


def mlp_batch_create(prec, act, D, descs, lr, loss_mean=1):
    arr = (mlp_net_desc * max(len(descs), 1))(*descs)
    b = ctypes.c_void_p()
    _ck(lib().mlp_batch_create(prec, act, D, arr, len(descs), lr, loss_mean, ctypes.byref(b)))
    return b.value


def mlp_batch_run(b, epochs, stream=0):
    return _ck(lib().mlp_batch_run(b, epochs, stream))


def mlp_batch_check(b, stream=0):
    """Returns the status code (does not raise)."""
    return lib().mlp_batch_check(b, stream)


def mlp_batch_destroy(b):
    lib().mlp_batch_destroy(b)


def mlp_batch_set_shape(b, shape):
    return _ck(lib().mlp_batch_set_shape(b, shape))


def mlp_batch_get_shape(b):
    v = ctypes.c_int32()
    _ck(lib().mlp_batch_get_shape(b, ctypes.byref(v)))
    return v.value


def mlp_batch_create_host(prec, act, D, Hs, ns, max_epochs, lr, loss_mean=1):
    """Plan owning device copies of every net's data (host layout: nets one
    after another); Hs and ns are sequences of ints."""
    import numpy as np
    H = np.ascontiguousarray(np.asarray(Hs, np.int32))
    n = np.ascontiguousarray(np.asarray(ns, np.int64))
    if H.shape != n.shape:
        raise ValueError("Hs and ns differ in length")
    b = ctypes.c_void_p()
    _ck(lib().mlp_batch_create_host(prec, act, D, _p(H), _p(n), len(H), max_epochs, lr, loss_mean, ctypes.byref(b)))
    return b.value


def mlp_batch_run_host(b, X_host, y_host, params_in_host, params_out_host, loss_hist_host, epochs, stream=0):
    return _ck(lib().mlp_batch_run_host(b, _p(X_host), _p(y_host), _p(params_in_host), _p(params_out_host),
                                        _p(loss_hist_host), epochs, stream))


def mlp_train_fused_noalloc(act, D, H, n, X, y, params, lr, loss_mean, epochs, minibatch=0, loss_hist=None,
                            status_out=None, stream=0):
    """Fused training that allocates no device memory (scratch in a fixed
    device array; D <= 64, H <= 128; overlapping calls race)."""
    return _ck(lib().mlp_train_fused_noalloc(act, D, H, n, _p(X), _p(y), _p(params), lr, loss_mean, epochs,
                                             minibatch, _p(loss_hist), _p(status_out), stream))


def mlp_last_error():
    return lib().mlp_last_error().decode()


def mlp_version():
    return lib().mlp_version().decode()


def mlp_unit_rates():
    """(FP32 FMA, tanh.approx.f32, ex2.approx.f32) instructions per second,
    measured on the current device."""
    v = [ctypes.c_double() for _ in range(3)]
    _ck(lib().mlp_unit_rates(*[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def mlp_zscore_workspace_bytes(D):
    b = ctypes.c_uint64()
    _ck(lib().mlp_zscore_workspace_bytes(D, ctypes.byref(b)))
    return b.value


def mlp_zscore(X, n, D, n_fit, out_prec, D_out, Y, mean, sdev, workspace, workspace_bytes, stream=0):
    return _ck(lib().mlp_zscore(_p(X), n, D, n_fit, out_prec, D_out, _p(Y), _p(mean), _p(sdev), _p(workspace),
                                workspace_bytes, stream))
