"""Autotuners for the training kernels' tile shapes.

* ``tune_fused``: rows per block of the fused single-network kernel.  It splits
  each step's rows over blocks; more blocks shorten the row phase but add
  cross-block traffic and barrier participants.
* ``tune_batched``: the kernel shape of an FP32 many-nets plan
  (mlp_batch_set_shape): one hidden unit a lane in blocks of 8 warps; two
  units a lane in blocks of 4 warps with one or two rows in flight; or
  register-tiled products over row chunks of 128, 64 or 32 rows (which trade
  shared memory for blocks an SM).  Which is fastest depends on the plan's mix
  of widths and row counts.
* ``tune_clusters``: the cluster count of the bf16 wide-network kernel
  (mlp_set_clusters): a step's 128-row tiles are dealt to the clusters, whose
  gradient slices are then summed; fewer clusters mean more tiles each but a
  shorter cross-cluster sum.

Each times its candidates on the caller's device and workload and caches the
fastest in a JSON file (``$MLP_GB300_TUNE_CACHE``, else
``~/.cache/mlp_gb300/tune.json``), keyed by device name and workload.  Timing
uses CUDA events on the launching stream; the library does the work.
"""
from __future__ import annotations

import json
import os
import threading

from . import binding as B

CANDIDATES = (8, 16, 24, 32, 48, 64, 96, 128)
_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("MLP_GB300_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "mlp_gb300", "tune.json")


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(table):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _key(device_name, D, H, n, mb, act):
    return "%s|fused|D=%d|H=%d|n=%d|mb=%d|act=%d" % (device_name, D, H, n, mb, act)


def tune_fused(X, y, D, H, n, minibatch=0, act=B.MLP_ACT_SIGMOID, candidates=CANDIDATES, reps=30,
               use_cache=True):
    """Best rows-per-block for mlp_train_epochs on (D, H, n, minibatch).

    X, y: device tensors of the shape to train (their values do not matter for
    timing; a throw-away handle with zero weights is trained).  Returns
    (rows_per_block, {candidate: microseconds per epoch})."""
    import torch
    dev_name = torch.cuda.get_device_name()
    key = _key(dev_name, D, H, n, minibatch, act)
    with _lock:
        table = _load() if use_cache else {}
        if key in table:
            return int(table[key]["rows_per_block"]), table[key]["us_per_epoch"]
    stream = torch.cuda.current_stream().cuda_stream
    h = B.mlp_create(D, H, 0.0, 1, B.MLP_FP32, act)   # lr 0: timing only, weights stay put
    times = {}
    try:
        for rows in candidates:
            B.mlp_set_rows_per_block(h, int(rows))
            for _ in range(3):
                B.mlp_train_epochs(h, X, y, n, 1, minibatch, None, None, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                B.mlp_train_epochs(h, X, y, n, 1, minibatch, None, None, stream)
            e1.record()
            torch.cuda.synchronize()
            times[int(rows)] = e0.elapsed_time(e1) * 1e3 / reps
        if B.mlp_check(h, stream) != B.MLP_OK:
            raise B.MLPError(B.MLP_ECUDA, "autotune run failed: " + B.mlp_last_error())
    finally:
        B.mlp_destroy(h)
    best = min(times, key=times.get)
    with _lock:
        table = _load() if use_cache else {}
        table[key] = {"rows_per_block": best, "us_per_epoch": {str(k): v for k, v in times.items()}}
        if use_cache:
            _store(table)
    return best, times


def configure(handle, X, y, D, H, n, minibatch=0, act=B.MLP_ACT_SIGMOID):
    """Tune (or read the cache) and set the handle's rows per block."""
    rows, _ = tune_fused(X, y, D, H, n, minibatch, act)
    B.mlp_set_rows_per_block(handle, rows)
    return rows


BATCH_SHAPES = (0, 1, 2, 3, 4, 5, 6)


def _batch_key(device_name, D, Hs, ns, act):
    import numpy as np
    Hs = np.asarray(Hs, np.int64)
    ns = np.asarray(ns, np.int64)
    return "%s|batched|D=%d|nets=%d|rows=%d|work=%d|act=%d" % (device_name, D, len(Hs), int(ns.sum()),
                                                              int((Hs * ns).sum()), act)


def tune_batched(plan, D, Hs, ns, params, act=B.MLP_ACT_SIGMOID, epochs=25, reps=3, shapes=BATCH_SHAPES,
                 use_cache=True):
    """Best kernel shape for an FP32 many-nets plan; sets it on the plan.

    plan: from mlp_batch_create; Hs, ns: its nets' widths and row counts (the
    cache key); params: the device tensor(s) holding the nets' packed weights,
    which the timed launches train and which are restored afterwards.  Each
    shape the plan's D takes is timed on `epochs`-epoch launches of the plan
    itself.  Returns (shape, {shape: milliseconds per epoch})."""
    import torch
    dev_name = torch.cuda.get_device_name()
    key = _batch_key(dev_name, D, Hs, ns, act)
    with _lock:
        table = _load() if use_cache else {}
        if key in table:
            best = int(table[key]["shape"])
            B.mlp_batch_set_shape(plan, best)
            return best, {int(k): v for k, v in table[key]["ms_per_epoch"].items()}
    stream = torch.cuda.current_stream().cuda_stream
    params = params if isinstance(params, (list, tuple)) else [params]
    saved = [p.clone() for p in params]
    before = B.mlp_batch_get_shape(plan)
    times = {}
    try:
        for shape in shapes:
            try:
                B.mlp_batch_set_shape(plan, int(shape))
            except B.MLPError:
                continue          # not available for this D
            B.mlp_batch_run(plan, epochs, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                B.mlp_batch_run(plan, epochs, stream)
            e1.record()
            torch.cuda.synchronize()
            times[int(shape)] = e0.elapsed_time(e1) / (reps * epochs)
        if B.mlp_batch_check(plan, stream) != B.MLP_OK:
            raise B.MLPError(B.MLP_ECUDA, "autotune run failed: " + B.mlp_last_error())
    finally:
        for p, q in zip(params, saved):
            p.copy_(q)
        torch.cuda.synchronize()
        B.mlp_batch_set_shape(plan, before)
    best = min(times, key=times.get)
    B.mlp_batch_set_shape(plan, best)
    with _lock:
        table = _load() if use_cache else {}
        table[key] = {"shape": best, "ms_per_epoch": {str(k): v for k, v in times.items()}}
        if use_cache:
            _store(table)
    return best, times


def _cluster_key(device_name, D, H, mb, act):
    return "%s|clusters|D=%d|H=%d|mb=%d|act=%d" % (device_name, D, H, mb, act)


def tune_clusters(X, y, D, H, n, minibatch, act=B.MLP_ACT_SIGMOID, candidates=None, steps=8, reps=3,
                  use_cache=True):
    """Best cluster count for the bf16 wide-network kernel (mlp_set_clusters)
    on mini-batches of `minibatch` rows of width D and H hidden units.

    X (bf16 rows, n >= minibatch) and y: device tensors; their values do not
    matter for timing (a throw-away handle with lr 0 trains `steps`
    mini-batches a launch).  Candidates default to the device limit and the
    six counts below it, plus half the limit.  Returns (clusters, {candidate:
    microseconds per mini-batch step})."""
    import torch
    dev_name = torch.cuda.get_device_name()
    key = _cluster_key(dev_name, D, H, minibatch, act)
    with _lock:
        table = _load() if use_cache else {}
        if key in table:
            return int(table[key]["clusters"]), {int(k): v for k, v in table[key]["us_per_step"].items()}
    kmax = B.mlp_cluster_limit(H)
    if candidates is None:
        candidates = sorted({k for k in range(max(1, kmax - 6), kmax + 1)} | {max(1, kmax // 2)})
    rows = min(int(n), int(steps) * int(minibatch))
    nsteps = (rows + minibatch - 1) // minibatch
    stream = torch.cuda.current_stream().cuda_stream
    h = B.mlp_create(D, H, 0.0, 1, B.MLP_BF16, act)   # lr 0: timing only
    times = {}
    try:
        if B.mlp_train_path(h, rows, minibatch) != B.MLP_PATH_TC_CLUSTER:
            raise ValueError("tune_clusters: this shape does not run on the wide-network kernel")
        for k in candidates:
            B.mlp_set_clusters(h, int(k))
            B.mlp_train_epochs(h, X, y, rows, 1, minibatch, None, None, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                B.mlp_train_epochs(h, X, y, rows, 1, minibatch, None, None, stream)
            e1.record()
            torch.cuda.synchronize()
            times[int(k)] = e0.elapsed_time(e1) * 1e3 / (reps * nsteps)
        if B.mlp_check(h, stream) != B.MLP_OK:
            raise B.MLPError(B.MLP_ECUDA, "autotune run failed: " + B.mlp_last_error())
    finally:
        B.mlp_destroy(h)
    best = min(times, key=times.get)
    with _lock:
        table = _load() if use_cache else {}
        table[key] = {"clusters": best, "us_per_step": {str(k): v for k, v in times.items()}}
        if use_cache:
            _store(table)
    return best, times


def configure_clusters(handle, X, y, D, H, n, minibatch, act=B.MLP_ACT_SIGMOID):
    """Tune (or read the cache) and set the handle's cluster count."""
    k, _ = tune_clusters(X, y, D, H, n, minibatch, act)
    B.mlp_set_clusters(handle, k)
    return k
