"""Many-nets workloads split across ranks (one process per GPU).

The nets of a batch are independent trainings (Sec. 2.1 of arXiv 1908.07847
trains its male and female subsets as separate networks; a sweep trains
thousands), so a rank needs no data from another while it trains.  The split
is by cost: nets are taken in decreasing cost (rows x hidden units) and each
goes to the rank with the least work so far (longest processing time first),
ties to the lower rank, so every rank computes the same assignment.  The only
exchange is the final gather of every net's trained weights and loss history
to rank 0, which puts them back in the global net order.

Everything here is host-side bookkeeping plus one ``torch.distributed``
gather; the training itself is the library's one-launch batch plan.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def partition_lpt(costs: Sequence[float], world: int) -> List[np.ndarray]:
    """Net indices of each rank, each list in increasing net order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(world)
    owner = np.empty(len(costs), dtype=np.int64)
    for t in order:
        r = int(np.argmin(load))          # first rank with the least work
        owner[t] = r
        load[r] += costs[t]
    return [np.flatnonzero(owner == r) for r in range(world)]


def packed_sizes(D: int, Hs: Sequence[int]) -> np.ndarray:
    """Floats of each net's packed weights [W1 (H x D), b1, w2, b2]."""
    return (D + 2) * np.asarray(Hs, dtype=np.int64) + 1


class Gather:
    """Gathers every rank's trained weights and loss histories to rank 0 in
    global net order.  Each rank holds its nets' packed weights one net after
    another in increasing net order (a flat float32 tensor) and their loss
    histories (len(part) x epochs float64).  The shares travel padded to the
    largest one, on the device the tensors live on (NCCL for CUDA tensors,
    gloo for CPU ones); rank 0 puts them in place with one indexed copy each,
    whose indices are computed once here."""

    def __init__(self, parts: List[np.ndarray], D: int, Hs: Sequence[int], epochs: int):
        self.parts = parts
        self.epochs = epochs
        sizes = packed_sizes(D, Hs)
        self.world = len(parts)
        self.pmax = max(int(sizes[p].sum()) for p in parts)
        self.lmax = max(len(p) for p in parts) * epochs
        offs = np.concatenate([[0], np.cumsum(sizes)])
        self.n_params = int(offs[-1])
        self.n_nets = len(sizes)
        # global position of every gathered element (rank r's share starts at
        # r * pmax in the gathered buffer)
        pidx = np.empty(self.n_params, dtype=np.int64)
        lidx = np.empty(self.n_nets * epochs, dtype=np.int64)
        for r, part in enumerate(parts):
            o = r * self.pmax
            for i, t in enumerate(part):
                sz = int(sizes[t])
                pidx[int(offs[t]):int(offs[t]) + sz] = np.arange(o, o + sz)
                o += sz
                lidx[t * epochs:(t + 1) * epochs] = r * self.lmax + i * epochs + np.arange(epochs)
        self._pidx, self._lidx = pidx, lidx
        self._dev_idx = {}

    def __call__(self, local_params, local_losses, group=None):
        """Returns (params [n_params], losses [n_nets x epochs]) on rank 0,
        None elsewhere."""
        import torch
        import torch.distributed as dist
        rank = dist.get_rank(group)
        dev = local_params.device
        pbuf = torch.zeros(self.pmax, dtype=torch.float32, device=dev)
        pbuf[:local_params.numel()] = local_params.reshape(-1)
        lbuf = torch.zeros(self.lmax, dtype=torch.float64, device=dev)
        lbuf[:local_losses.numel()] = local_losses.reshape(-1)
        root = 0 if group is None else dist.get_global_rank(group, 0)
        pall = torch.empty(self.world * self.pmax, dtype=torch.float32, device=dev) if rank == 0 else None
        lall = torch.empty(self.world * self.lmax, dtype=torch.float64, device=dev) if rank == 0 else None
        dist.gather(pbuf, list(pall.chunk(self.world)) if rank == 0 else None, dst=root, group=group)
        dist.gather(lbuf, list(lall.chunk(self.world)) if rank == 0 else None, dst=root, group=group)
        if rank != 0:
            return None
        if dev not in self._dev_idx:
            self._dev_idx[dev] = (torch.from_numpy(self._pidx).to(dev), torch.from_numpy(self._lidx).to(dev))
        pi, li = self._dev_idx[dev]
        return pall[pi], lall[li].reshape(self.n_nets, self.epochs)
