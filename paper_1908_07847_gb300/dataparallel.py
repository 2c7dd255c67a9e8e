"""One network trained data-parallel across ranks (one process per GPU).

Mini-batch gradient descent (Sec. 2.2 of arXiv 1908.07847) updates with the
gradient of the batch's squared error, a sum over the batch's rows.  So the
rows of every mini-batch can be split across ranks: rank r takes the
contiguous shard [floor(r m / R), floor((r + 1) m / R)) of each batch of m
rows, computes the summed gradient of its shard on its own replica of the
network (the library's backward, on a handle built with loss_mean = 0), and
one exchange per mini-batch -- an all-gather of every rank's flat gradient
[gW1, gb1, gw2, gb2] and shard loss -- lets every rank add the R vectors in
rank order and scale them by 1/m for the mean loss (``mlp_grad_sum``), then
apply the same update (``mlp_update``).  Each rank adds the same numbers in the
same order, so the replicas stay bit-identical; the result depends on the
number of ranks only through the rounding of the partial sums.

Everything here is argument marshalling and the collective; the arithmetic
(shard gradients, the rank-order sum, the update) runs in the library.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np

from . import binding as B


def shard_rows(m: int, world: int, rank: int) -> Tuple[int, int]:
    """Rows [lo, hi) of a batch of m rows that rank `rank` of `world` takes."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank or world size")
    return (m * rank) // world, (m * (rank + 1)) // world


def batches(n: int, minibatch: int):
    """(start, rows) of each mini-batch of an epoch: contiguous slices in
    order, the whole set when minibatch <= 0 or >= n, the last one ragged."""
    mb = n if (minibatch <= 0 or minibatch >= n) else minibatch
    start = 0
    while start < n:
        m = min(mb, n - start)
        yield start, m
        start += m


class DataParallel:
    """Trains the replica `handle` (D inputs, H hidden units, FP32 or BF16
    rows, created with loss_mean = 0) together with the replicas of the other
    ranks of `group` (default: the whole world of torch.distributed).

    ``train`` runs `epochs` epochs over the rows X (device, n x D) and labels
    y (device, n floats) that every rank holds; a rank reads only its shards.
    The exchange runs on the device tensors' own backend (NCCL for CUDA
    tensors); under gloo the vectors go through host memory."""

    def __init__(self, handle, D: int, H: int, group=None):
        import torch
        import torch.distributed as dist
        self.h = handle
        self.D, self.H = D, H
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.host_exchange = dist.get_backend(group) == "gloo"
        self.len = (D + 2) * H + 1
        dev = torch.device("cuda", torch.cuda.current_device())
        f32, f64 = torch.float32, torch.float64
        self.flat = torch.zeros(self.len, dtype=f32, device=dev)       # this rank's summed gradient
        self.loss = torch.zeros(1, dtype=f64, device=dev)              # this rank's summed shard loss
        self.parts = torch.zeros((self.world, self.len), dtype=f32, device=dev)
        self.lparts = torch.zeros(self.world, dtype=f64, device=dev)
        self.sum = torch.zeros(self.len, dtype=f32, device=dev)
        HD = H * D
        self.views = [(self.flat[:HD], self.flat[HD:HD + H], self.flat[HD + H:HD + 2 * H], self.flat[HD + 2 * H:]),
                      (self.sum[:HD], self.sum[HD:HD + H], self.sum[HD + H:HD + 2 * H], self.sum[HD + 2 * H:])]

    def _gather(self):
        import torch
        import torch.distributed as dist
        if self.host_exchange:
            torch.cuda.current_stream().synchronize()
            parts = [torch.empty(self.len, dtype=torch.float32) for _ in range(self.world)]
            lparts = [torch.empty(1, dtype=torch.float64) for _ in range(self.world)]
            dist.all_gather(parts, self.flat.cpu(), group=self.group)
            dist.all_gather(lparts, self.loss.cpu(), group=self.group)
            self.parts.copy_(torch.stack(parts))
            self.lparts.copy_(torch.cat(lparts))
        else:
            dist.all_gather_into_tensor(self.parts, self.flat, group=self.group)
            dist.all_gather_into_tensor(self.lparts, self.loss, group=self.group)

    def step(self, X, y, start: int, m: int, loss_mean: bool, loss_acc, loss_scale: float, stream: int):
        """One mini-batch of m rows starting at row `start`: shard gradient,
        exchange, rank-order sum, update; loss_acc += loss_scale * batch loss."""
        lo, hi = shard_rows(m, self.world, self.rank)
        if hi > lo:
            gW1, gb1, gw2, gb2 = self.views[0]
            B.mlp_backward(self.h, X[start + lo:], y[start + lo:], hi - lo, gW1, gb1, gw2, gb2, self.loss, stream)
        else:
            self.flat.zero_()
            self.loss.zero_()
        self._gather()
        scale = float(np.float32(1.0 / m)) if loss_mean else 1.0
        B.mlp_grad_sum(self.parts, self.lparts, self.world, self.len, scale, loss_scale, self.sum, loss_acc, stream)
        B.mlp_update(self.h, *self.views[1], stream)

    def train(self, X, y, n: int, epochs: int, minibatch: int = 0, loss_mean: bool = True, loss_hist=None):
        """`epochs` epochs of mini-batch gradient descent over n rows;
        loss_hist (device doubles, one an epoch, or None) receives
        (C/2) sum (o - y)^2 over each epoch's rows before their updates,
        C = 1/n for the mean loss, else 1."""
        import torch
        stream = torch.cuda.current_stream().cuda_stream
        acc = torch.zeros(1, dtype=torch.float64, device=self.flat.device)
        lscale = (1.0 / n if n > 0 else 0.0) if loss_mean else 1.0
        for e in range(epochs):
            acc.zero_()
            for start, m in batches(n, minibatch):
                self.step(X, y, start, m, loss_mean, acc, lscale, stream)
            if loss_hist is not None:
                loss_hist[e:e + 1].copy_(acc)
