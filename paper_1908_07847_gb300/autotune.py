"""Autotuner for the fused training kernel's tile shape (rows per block).

The fused kernel splits each step's rows over blocks; more blocks shorten the
row phase but add cross-block traffic and barrier participants.  ``tune_fused``
times one-epoch launches for each candidate on the caller's device and shape and
caches the fastest in a JSON file (``$MLP_GB300_TUNE_CACHE``, else
``~/.cache/mlp_gb300/tune.json``), keyed by device name and shape.  Timing uses
CUDA events on the launching stream; the library does the work.
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
