"""Helpers for the GPU parity tests: seeded inputs, handles, error measures.

Tolerances (the reading of the stated parity bar):
  forward      max_i |o_i - o*_i| / |o*_i|                      <= 1e-6  (FP32)
  gradients    max_p |g_p - g*_p| / max_p |g*_p|                 <= 1e-5  (FP32)
  weights      max_p |w_p - w*_p| / max_p |w*_p| after 100 epochs <= 1e-4 (FP32)
  BF16 math    gradients <= 2e-2 by the same measure
where * is the FP64 oracle run on the same (float32 or bf16-exact) inputs.
"""
import numpy as np

import oracle
from paper_1908_07847_gb300 import binding as B
from paper_1908_07847_gb300 import inputs as I

FWD_TOL = 1e-6
GRAD_TOL = 1e-5
W_TOL = 1e-4
BF16_GRAD_TOL = 2e-2


def torch_mod():
    import torch
    return torch


def stream():
    return torch_mod().cuda.current_stream().cuda_stream


def dev(a):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def lr32(lr=0.1):
    return float(np.float32(lr))


def labels_from_teacher(X, D):
    """Teacher-net labels computed by the oracle (Sec. 2.1's HbA1c control
    label stand-in)."""
    T = oracle.Params(*I.teacher_weights(D=D, Dpad=X.shape[1]))
    return oracle.predict(X, T).astype(np.float32)


def problem(seed, n, D, H, Dpad=None):
    X = I.features(seed, n, D, Dpad)
    y = labels_from_teacher(X, D)
    W = I.init_weights(seed + 1, D, H, Dpad)
    return X, y, W


def rel_err_norm(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def rel_err_elem(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


class Net:
    """Owns one library handle."""

    def __init__(self, D, H, lr=0.1, loss_mean=1, prec=B.MLP_FP32, act=B.MLP_ACT_SIGMOID):
        self.D, self.H, self.prec = D, H, prec
        self.dt = np.float64 if prec == B.MLP_FP64 else np.float32
        self.h = B.mlp_create(D, H, lr, loss_mean, prec, act)

    def set(self, W):
        W1, b1, w2, b2 = [np.ascontiguousarray(np.asarray(a, self.dt)) for a in W]
        B.mlp_set_weights(self.h, W1, b1, w2, b2)

    def get(self):
        W1 = np.zeros((self.H, self.D), self.dt)
        b1 = np.zeros(self.H, self.dt)
        w2 = np.zeros(self.H, self.dt)
        b2 = np.zeros(1, self.dt)
        B.mlp_get_weights(self.h, W1, b1, w2, b2)
        return W1, b1, w2, b2

    def flat(self):
        W1, b1, w2, b2 = self.get()
        return np.concatenate([W1.ravel(), b1, w2, b2]).astype(np.float64)

    def check(self):
        return B.mlp_check(self.h, stream())

    def close(self):
        if self.h:
            B.mlp_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
