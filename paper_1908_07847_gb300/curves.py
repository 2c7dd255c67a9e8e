"""Train and test accuracy against epochs on the synthetic sex-split cohort.

The paper (Sec. 3, Figs. 3 and 4) plots the accuracy of its network on the male
(61 participants) and female (59) subsets as training runs to 100,000 epochs,
each subset split 75 % / 25 % (Sec. 1).  The cohort itself is not available, so
this runs the same protocol on the synthetic stand-in: the 120-row feature
table, its first 61 rows as one subset and the remaining 59 as the other,
n_train = round(0.75 n) (46/15 and 44/15), teacher-net labels.  Both subsets are
trained as independent networks in one launch of the many-nets kernel per
checkpoint interval (full-batch gradient descent, lr 0.1, Sec. 2.2); accuracy
is measured with the library's classification call (o >= 0.5).

    python -m paper_1908_07847_gb300.curves [--hidden 16] [--epochs 100000] [--out curves.json]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import binding as B
from . import inputs as I

CHECKPOINTS = (1, 10, 100, 1000, 10000, 100000)


def subsets(labels):
    """(name, X, y, n_train) of the two subsets, rows in cohort order."""
    X = I.features(I.COHORT_SEED, I.N_PARTICIPANTS)
    out = []
    for name, r0, r1 in (("male", 0, I.N_MALE), ("female", I.N_MALE, I.N_PARTICIPANTS)):
        Xs, ys = X[r0:r1], labels[r0:r1]
        out.append((name, Xs, ys, I.split_count(r1 - r0)))
    return out


def teacher_labels_gpu(X):
    """Labels = the teacher net's class decisions, by the library's predict."""
    import torch
    T = I.teacher_weights()
    h = B.mlp_create(I.D_MARKERS, T[0].shape[0], 0.1, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    try:
        B.mlp_set_weights(h, *T)
        Xd = torch.from_numpy(X).cuda()
        lab = torch.zeros(X.shape[0], dtype=torch.int8, device="cuda")
        B.mlp_predict(h, Xd, X.shape[0], lab, torch.cuda.current_stream().cuda_stream)
        return lab.cpu().numpy().astype(np.float32)
    finally:
        B.mlp_destroy(h)


def accuracy_curve(hidden=16, checkpoints=CHECKPOINTS, lr=0.1, seed=I.INIT_SEED):
    """Returns {subset: [(epochs, train_acc, test_acc), ...]}."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    X = I.features(I.COHORT_SEED, I.N_PARTICIPANTS)
    labels = teacher_labels_gpu(X)
    parts = subsets(labels)
    keep, descs, params = [], [], []
    for k, (name, Xs, ys, ntr) in enumerate(parts):
        W = I.init_weights(seed + k, I.D_MARKERS, hidden)
        Xd = torch.from_numpy(np.ascontiguousarray(Xs[:ntr])).cuda()
        yd = torch.from_numpy(np.ascontiguousarray(ys[:ntr])).cuda()
        P = torch.from_numpy(np.concatenate([a.ravel() for a in W]).astype(np.float32)).cuda()
        keep += [Xd, yd]
        params.append(P)
        descs.append(B.mlp_net_desc(hidden, ntr, Xd.data_ptr(), yd.data_ptr(), P.data_ptr(), None))
    plan = B.mlp_batch_create(B.MLP_FP32, B.MLP_ACT_SIGMOID, I.D_MARKERS, descs, lr, 1)
    curves = {name: [] for name, _, _, _ in parts}
    h = B.mlp_create(I.D_MARKERS, hidden, lr, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    try:
        done = 0
        for cp in checkpoints:
            if cp > done:
                B.mlp_batch_run(plan, cp - done, stream)
                done = cp
            if B.mlp_batch_check(plan, stream) != B.MLP_OK:
                raise B.MLPError(B.MLP_ENONFINITE, B.mlp_last_error())
            for (name, Xs, ys, ntr), P in zip(parts, params):
                p = P.cpu().numpy()
                HD = hidden * I.D_MARKERS
                B.mlp_set_weights(h, p[:HD].reshape(hidden, I.D_MARKERS).copy(), p[HD:HD + hidden].copy(),
                                  p[HD + hidden:HD + 2 * hidden].copy(), p[-1:].copy())
                lab = torch.zeros(Xs.shape[0], dtype=torch.int8, device="cuda")
                B.mlp_predict(h, torch.from_numpy(np.ascontiguousarray(Xs)).cuda(), Xs.shape[0], lab, stream)
                pred = lab.cpu().numpy()
                tr = float((pred[:ntr] == ys[:ntr]).mean())
                te = float((pred[ntr:] == ys[ntr:]).mean())
                curves[name].append((cp, tr, te))
    finally:
        B.mlp_destroy(h)
        B.mlp_batch_destroy(plan)
    return curves


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--hidden", type=int, default=16)
    ap.add_argument("--epochs", type=int, default=100000)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    cps = tuple(c for c in CHECKPOINTS if c <= a.epochs)
    if not cps or cps[-1] != a.epochs:
        cps = cps + (a.epochs,)
    curves = accuracy_curve(a.hidden, cps)
    text = json.dumps({"hidden": a.hidden, "curves": curves}, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
