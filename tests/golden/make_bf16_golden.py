"""Writes the stored oracle results of the two long bf16 runs
(c3_wide_net_20epochs.json, c4_sampled_nets_200epochs.json) that the GPU
tests compare the tensor-core paths with.  Calls only the FP64 oracle (and the
seeded input generators); nothing here touches the CUDA library.

    python tests/golden/make_bf16_golden.py [c3] [c4]

Both runs follow Sec. 2.2 (sigmoid units, squared error with the 1/n mean,
gradient descent without momentum, lr = float(0.1)); the wide net by
mini-batches of 8192 rows in order, the many nets by full batch.  Stored: the
loss and gradient-norm histories, the train and test accuracy of the trained
net (class 1 iff o >= 0.5), and a subsample of the trained weights.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import Params  # noqa: E402
from paper_1908_07847_gb300 import inputs as I  # noqa: E402
from tests import bf16_workloads as WL  # noqa: E402

LR = float(np.float32(0.1))


def teacher():
    return Params(*I.teacher_weights(D=WL.D_REAL, Dpad=WL.D_PAD))


def accuracy(X, y, p):
    return float((oracle.predict(X, p) == y).mean())


def make_c3():
    X = WL.c3_rows().astype(np.float64)
    y = oracle.predict(X, teacher()).astype(np.float64)
    Xtr, ytr, Xte, yte = X[:WL.C3_TRAIN], y[:WL.C3_TRAIN], X[WL.C3_TRAIN:], y[WL.C3_TRAIN:]
    t0 = time.time()
    q, lh, gh = oracle.train(Xtr, ytr, Params(*WL.c3_weights()), LR, WL.C3_EPOCHS, minibatch=WL.C3_MB)
    out = {"what": "48-2048-1 sigmoid net, first 49,152 of the first 65,536 rows of the 1M-row table, "
                   "mini-batch 8192, 20 epochs, lr float(0.1), mean squared error; FP64 oracle",
           "loss_hist": lh.tolist(), "gnorm_hist": gh.tolist(),
           "train_acc": accuracy(Xtr, ytr, q), "test_acc": accuracy(Xte, yte, q),
           "keep_every": WL.C3_KEEP_EVERY,
           "kept_params": WL.kept_params(q.W1, q.b1, q.w2, q.b2, WL.C3_KEEP_EVERY).tolist(),
           "oracle_seconds": time.time() - t0}
    with open(os.path.join(HERE, "c3_wide_net_20epochs.json"), "w") as f:
        json.dump(out, f)


def make_c4():
    ns = WL.c4_shapes()
    picks = WL.c4_picks(ns)
    T = teacher()
    nets, splits = [], []
    for t in picks:
        X = WL.c4_net_rows(ns, t).astype(np.float64)
        y = oracle.predict(X, T).astype(np.float64)
        ntr = I.split_count(X.shape[0])
        nets.append((X[:ntr], y[:ntr], Params(*WL.c4_weights(t))))
        splits.append((X, y, ntr))
    t0 = time.time()
    # the nets in parallel (ctypes releases the interpreter lock during the
    # oracle's C calls)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(len(nets)) as ex:
        runs = list(ex.map(lambda n: oracle.train(n[0], n[1], n[2], LR, WL.C4_EPOCHS), nets))
    dt = time.time() - t0
    per = []
    for t, (X, y, ntr), (q, lh, gh) in zip(picks, splits, runs):
        per.append({"net": t, "n": int(X.shape[0]), "n_train": ntr, "loss_hist": lh.tolist(),
                    "gnorm_hist": gh.tolist(), "train_acc": accuracy(X[:ntr], y[:ntr], q),
                    "test_acc": accuracy(X[ntr:], y[ntr:], q),
                    "kept_params": WL.kept_params(q.W1, q.b1, q.w2, q.b2, WL.C4_KEEP_EVERY).tolist()})
    out = {"what": "1024 nets 48-256-1 (n ~ U{4096..16384}), each trained on its first 75% of rows, full batch, "
                   "200 epochs, lr float(0.1), mean squared error; FP64 oracle on four of them",
           "keep_every": WL.C4_KEEP_EVERY, "nets": per, "oracle_seconds": dt}
    with open(os.path.join(HERE, "c4_sampled_nets_200epochs.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    which = sys.argv[1:] or ["c3", "c4"]
    if "c3" in which:
        make_c3()
    if "c4" in which:
        make_c4()
