"""FP64 CPU oracle for the one-hidden-layer sigmoid network of arXiv 1908.07847.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA product
path never imports it and shares no code with it.

The arithmetic lives in ``mlp_oracle.c`` (plain serial C, doubles, compiled with
``-O2 -ffp-contract=off`` so that no multiply-add is fused).  This module only
compiles it and marshals numpy arrays in and out; every function converts its
inputs to float64 first, so callers may pass float32 arrays and get the exact
widening of those values.

Citations (the paper's sections): forward pass Sec. 2.2 with Eq. 1; backward
pass and gradient descent (lr 0.1, no momentum) Sec. 2.2; classification of the
test rows Sec. 2.2 / Fig. 2; separate male and female subsets Sec. 2.1.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

ACT_SIGMOID = 0
ACT_TANH = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc_mlp.so")
SOURCE = _SRC
_lock = threading.Lock()
_lib = None


def compile_c(src: str, out: str) -> str:
    """gcc -O2 -ffp-contract=off shared build of one C file (OpenMP if present)."""
    tmp = out + ".%d.tmp" % os.getpid()
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
            src, "-o", tmp]
    # OpenMP is used only to spread independent nets over host cores.
    r = subprocess.run(base + ["-fopenmp", "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base + ["-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile mlp_oracle.c into oracle/_build/liborc_mlp.so (gcc, C11)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    return compile_c(_SRC, _LIB)


def _bind(lib):
    d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
    lib.orc_sigmoid.restype = d
    lib.orc_sigmoid.argtypes = [d]
    lib.orc_forward.restype = None
    lib.orc_forward.argtypes = [i, i, l, p, p, p, p, d, i, p, p]
    lib.orc_backward.restype = None
    lib.orc_backward.argtypes = [i, i, l, p, p, p, p, d, i, p, p, p, p, p, p]
    lib.orc_mse_gradients.restype = d
    lib.orc_mse_gradients.argtypes = [i, i, l, p, p, p, p, p, d, i, i, p, p, p, p]
    lib.orc_update.restype = None
    lib.orc_update.argtypes = [i, i, d, p, p, p, p, p, p, p, d]
    lib.orc_train.restype = None
    lib.orc_train.argtypes = [i, i, l, p, p, p, p, p, p, i, i, d, i, l, p, p]
    lib.orc_predict.restype = None
    lib.orc_predict.argtypes = [i, i, l, p, p, p, p, d, i, p]
    lib.orc_zscore.restype = None
    lib.orc_zscore.argtypes = [l, i, l, p, p, p, p]
    lib.orc_batch_train.restype = None
    lib.orc_batch_train.argtypes = [i, p, p, p, p, p, p, p, p, p, i, i, d, i, l, p, i]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


@contextlib.contextmanager
def substituted_library(path: str):
    """Run the wrappers against another build of the oracle source (used by the
    test that plants mistakes in a copy of mlp_oracle.c)."""
    global _lib
    with _lock:
        saved = _lib
        _lib = _bind(ctypes.CDLL(path))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Params:
    """Network parameters in float64: W1 (H x D), b1 (H), w2 (H), b2 (scalar)."""

    def __init__(self, W1, b1, w2, b2):
        self.W1 = _f64(W1).copy()
        self.b1 = _f64(b1).copy()
        self.w2 = _f64(w2).copy()
        self.b2 = float(np.asarray(b2, dtype=np.float64).reshape(-1)[0])

    @property
    def H(self):
        return self.W1.shape[0]

    @property
    def D(self):
        return self.W1.shape[1]

    def copy(self):
        return Params(self.W1, self.b1, self.w2, self.b2)

    def flat(self):
        """Packed [W1, b1, w2, b2] vector of (D + 2) H + 1 values."""
        return np.concatenate([self.W1.ravel(), self.b1, self.w2, [self.b2]])


def sigmoid(x: float) -> float:
    """Eq. 1."""
    return _load().orc_sigmoid(float(x))


def forward(X, p: Params, act: int = ACT_SIGMOID):
    """Sec. 2.2 feed-forward; returns (hidden n x H, output n)."""
    lib = _load()
    X = _f64(X)
    n = X.shape[0]
    hid = np.zeros((n, p.H))
    o = np.zeros(n)
    lib.orc_forward(p.D, p.H, n, _ptr(X), _ptr(p.W1), _ptr(p.b1), _ptr(p.w2),
                    p.b2, act, _ptr(hid), _ptr(o))
    return hid, o


def backward(X, p: Params, dLdo, act: int = ACT_SIGMOID, want_gX: bool = False):
    """Sec. 2.2 backpropagation of an upstream gradient dL/do; returns
    (gW1, gb1, gw2, gb2[, gX])."""
    lib = _load()
    X = _f64(X)
    n = X.shape[0]
    dLdo = _f64(dLdo)
    gW1 = np.zeros((p.H, p.D))
    gb1 = np.zeros(p.H)
    gw2 = np.zeros(p.H)
    gb2 = ctypes.c_double(0.0)
    gX = np.zeros((n, p.D)) if want_gX else None
    lib.orc_backward(p.D, p.H, n, _ptr(X), _ptr(p.W1), _ptr(p.b1), _ptr(p.w2),
                     p.b2, act, _ptr(dLdo), _ptr(gW1), _ptr(gb1), _ptr(gw2),
                     ctypes.byref(gb2), _ptr(gX))
    out = (gW1, gb1, gw2, gb2.value)
    return out + (gX,) if want_gX else out


def mse_gradients(X, y, p: Params, loss_mean: bool = True, act: int = ACT_SIGMOID):
    """Squared-error gradients (Sec. 2.2); returns (gW1, gb1, gw2, gb2, loss)
    with loss = (c/2) * sum (o - y)^2."""
    lib = _load()
    X = _f64(X)
    y = _f64(y)
    n = X.shape[0]
    gW1 = np.zeros((p.H, p.D))
    gb1 = np.zeros(p.H)
    gw2 = np.zeros(p.H)
    gb2 = ctypes.c_double(0.0)
    sse = lib.orc_mse_gradients(p.D, p.H, n, _ptr(X), _ptr(y), _ptr(p.W1),
                                _ptr(p.b1), _ptr(p.w2), p.b2, act, int(loss_mean),
                                _ptr(gW1), _ptr(gb1), _ptr(gw2), ctypes.byref(gb2))
    c = (1.0 / n if n > 0 else 0.0) if loss_mean else 1.0
    return gW1, gb1, gw2, gb2.value, 0.5 * c * sse


def update(p: Params, grads, lr: float) -> Params:
    """Sec. 2.2 gradient-descent step (no momentum); returns a new Params."""
    lib = _load()
    q = p.copy()
    gW1, gb1, gw2, gb2 = [_f64(g) if i < 3 else float(g) for i, g in enumerate(grads[:4])]
    b2 = ctypes.c_double(q.b2)
    lib.orc_update(q.D, q.H, float(lr), _ptr(q.W1), _ptr(q.b1), _ptr(q.w2),
                   ctypes.byref(b2), _ptr(gW1), _ptr(gb1), _ptr(gw2), gb2)
    q.b2 = b2.value
    return q


def train(X, y, p: Params, lr: float, epochs: int, minibatch: int = 0,
          loss_mean: bool = True, act: int = ACT_SIGMOID):
    """Sec. 2.2 training loop; returns (trained Params, loss_hist, gnorm_hist)."""
    lib = _load()
    X = _f64(X)
    y = _f64(y)
    n = X.shape[0]
    q = p.copy()
    b2 = ctypes.c_double(q.b2)
    lh = np.zeros(max(epochs, 0))
    gh = np.zeros(max(epochs, 0))
    lib.orc_train(q.D, q.H, n, _ptr(X), _ptr(y), _ptr(q.W1), _ptr(q.b1),
                  _ptr(q.w2), ctypes.byref(b2), act, int(loss_mean), float(lr),
                  int(epochs), int(minibatch), _ptr(lh), _ptr(gh))
    q.b2 = b2.value
    return q, lh, gh


def predict(X, p: Params, act: int = ACT_SIGMOID):
    """Sec. 2.2 classification: int8 labels, 1 iff o >= 0.5."""
    lib = _load()
    X = _f64(X)
    n = X.shape[0]
    lab = np.zeros(n, dtype=np.int8)
    lib.orc_predict(p.D, p.H, n, _ptr(X), _ptr(p.W1), _ptr(p.b1), _ptr(p.w2),
                    p.b2, act, _ptr(lab))
    return lab


def batch_train(nets, lr: float, epochs: int, minibatch: int = 0,
                loss_mean: bool = True, act: int = ACT_SIGMOID, threads: int = 1):
    """Independent nets (Sec. 2.1's separate subsets, generalised).

    ``nets`` is a list of (X, y, Params).  Returns (list of trained Params,
    loss array n_nets x epochs)."""
    lib = _load()
    T = len(nets)
    Ds = np.array([p.D for _, _, p in nets], dtype=np.int32)
    Hs = np.array([p.H for _, _, p in nets], dtype=np.int32)
    ns = np.array([np.asarray(X).shape[0] for X, _, _ in nets], dtype=np.int64)
    Xs = [_f64(X).ravel() for X, _, _ in nets]
    ys = [_f64(y).ravel() for _, y, _ in nets]
    Ps = [p.flat() for _, _, p in nets]

    def offs(parts):
        o = np.zeros(len(parts), dtype=np.int64)
        if len(parts) > 1:
            o[1:] = np.cumsum([len(a) for a in parts[:-1]])
        return o

    x_off, y_off, p_off = offs(Xs), offs(ys), offs(Ps)
    X_all = np.concatenate(Xs) if T else np.zeros(1)
    y_all = np.concatenate(ys) if T else np.zeros(1)
    P_all = np.concatenate(Ps) if T else np.zeros(1)
    loss = np.zeros((T, max(epochs, 0)))
    lib.orc_batch_train(T, _ptr(Ds), _ptr(Hs), _ptr(ns), _ptr(X_all), _ptr(x_off),
                        _ptr(y_all), _ptr(y_off), _ptr(P_all), _ptr(p_off), act,
                        int(loss_mean), float(lr), int(epochs), int(minibatch),
                        _ptr(loss), int(threads))
    out = []
    for t in range(T):
        D, H = int(Ds[t]), int(Hs[t])
        P = P_all[p_off[t]:p_off[t] + (D + 2) * H + 1]
        out.append(Params(P[:H * D].reshape(H, D), P[H * D:H * D + H],
                          P[H * D + H:H * D + 2 * H], P[-1]))
    return out, loss


if __name__ == "__main__":  # pragma: no cover - manual build entry
    print(build(force="--force" in sys.argv))


def zscore(X, n_fit=None):
    """Column z-score with the statistics of the first n_fit rows (Sec. 2.2's
    normalisation, read as training-set mean and population deviation);
    returns (Y, mean, sdev)."""
    lib = _load()
    X = _f64(X)
    n, D = X.shape
    n_fit = n if n_fit is None else int(n_fit)
    mean = np.zeros(D)
    sdev = np.zeros(D)
    Y = np.zeros((n, D))
    lib.orc_zscore(n, D, n_fit, _ptr(X), _ptr(mean), _ptr(sdev), _ptr(Y))
    return Y, mean, sdev
