"""torch.autograd.Function over the library's hand-written forward and backward
kernels (Sec. 2.2 of arXiv 1908.07847: feed-forward, then backpropagation of the
error through the sigmoid output and hidden layers).

``mlp(X, W1, b1, w2, b2)`` returns the network outputs o [n]; its backward runs
the library's backward kernel on the upstream gradient dL/do and returns the
gradients of X, W1, b1, w2 and b2.  float32 and float64 tensors on a CUDA device
are supported; the FP64 kernels are the ones to check against finite
differences.  Marshalling only: both directions run in the CUDA library.
"""
from __future__ import annotations

import torch

from . import binding as B

_PREC = {torch.float32: B.MLP_FP32, torch.float64: B.MLP_FP64}


def _workspace(prec, D, H, n, device):
    nbytes = B.mlp_workspace_bytes(prec, D, H, n)
    # torch's allocator returns blocks aligned to at least 512 bytes.
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device), nbytes


class MLPFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, W1, b1, w2, b2, act=B.MLP_ACT_SIGMOID):
        dt = X.dtype
        if dt not in _PREC or not X.is_cuda:
            raise TypeError("mlp: X must be a float32 or float64 CUDA tensor")
        for t in (W1, b1, w2, b2):
            if t.dtype != dt or t.device != X.device:
                raise TypeError("mlp: all tensors must share X's dtype and device")
        prec = _PREC[dt]
        X, W1, b1, w2, b2 = (t.contiguous() for t in (X, W1, b1, w2, b2))
        n, D = X.shape
        H = W1.shape[0]
        if W1.shape != (H, D) or b1.numel() != H or w2.numel() != H or b2.numel() != 1:
            raise ValueError("mlp: inconsistent shapes")
        hid = torch.empty((n, H), dtype=dt, device=X.device)
        o = torch.empty(n, dtype=dt, device=X.device)
        ws, nb = _workspace(prec, D, H, n, X.device)
        B.mlp_forward_w(prec, act, D, H, n, X, W1, b1, w2, b2, hid, o, ws, nb,
                        torch.cuda.current_stream(X.device).cuda_stream)
        ctx.save_for_backward(X, W1, w2, hid, o)
        ctx.act = act
        ctx.b2_shape = b2.shape
        return o

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, go):
        X, W1, w2, hid, o = ctx.saved_tensors
        prec = _PREC[X.dtype]
        n, D = X.shape
        H = W1.shape[0]
        go = go.contiguous().to(X.dtype)
        gW1 = torch.empty_like(W1)
        gb1 = torch.empty(H, dtype=X.dtype, device=X.device)
        gw2 = torch.empty(H, dtype=X.dtype, device=X.device)
        gb2 = torch.empty(1, dtype=X.dtype, device=X.device)
        gX = torch.empty_like(X) if ctx.needs_input_grad[0] else None
        ws, nb = _workspace(prec, D, H, n, X.device)
        B.mlp_backward_w(prec, ctx.act, D, H, n, X, W1, w2, hid, o, go, gW1, gb1, gw2, gb2, gX, ws, nb,
                         torch.cuda.current_stream(X.device).cuda_stream)
        return gX, gW1, gb1, gw2, gb2.reshape(ctx.b2_shape), None


def mlp(X, W1, b1, w2, b2, act=B.MLP_ACT_SIGMOID):
    """Network outputs o = sigmoid(f(X W1^T + b1) w2 + b2) (Eq. 1, Sec. 2.2)."""
    return MLPFunction.apply(X, W1, b1, w2, b2, act)


class MLP(torch.nn.Module):
    """One-hidden-layer network whose forward and backward run in the library."""

    def __init__(self, D, H, dtype=torch.float32, device="cuda", act=B.MLP_ACT_SIGMOID):
        super().__init__()
        self.act = act
        self.W1 = torch.nn.Parameter(torch.zeros((H, D), dtype=dtype, device=device))
        self.b1 = torch.nn.Parameter(torch.zeros(H, dtype=dtype, device=device))
        self.w2 = torch.nn.Parameter(torch.zeros(H, dtype=dtype, device=device))
        self.b2 = torch.nn.Parameter(torch.zeros(1, dtype=dtype, device=device))

    def forward(self, X):
        return mlp(X, self.W1, self.b1, self.w2, self.b2, self.act)
