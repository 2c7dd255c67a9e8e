"""BF16 tensor-core (tcgen05) path of the many-nets plan against the FP64 oracle
(Sec. 2.2 of arXiv 1908.07847), on the same bf16-exact inputs.  Tolerance: the
gradient within 2e-2 (max-norm relative), as stated for bf16 arithmetic."""
import numpy as np
import pytest

import oracle
from oracle import Params
from paper_1908_07847_gb300 import binding as B
from paper_1908_07847_gb300 import inputs as I
from tests.gpu_util import BF16_GRAD_TOL, dev, host, lr32, rel_err_elem, rel_err_norm, stream

pytestmark = pytest.mark.gpu

D_REAL, D_PAD = 33, 48


def make_net(seed, n, H):
    X = I.bf16_round(I.features(seed, n, D_REAL, D_PAD))
    T = Params(*I.teacher_weights(D=D_REAL, Dpad=D_PAD))
    y = oracle.predict(X, T).astype(np.float32)
    W = I.init_weights(seed + 7, D_REAL, H, D_PAD)
    return X, y, W


def run_tc(nets, epochs, lr, act=B.MLP_ACT_SIGMOID, norms=False):
    import torch
    keep, descs, params, losses, gns = [], [], [], [], []
    for X, y, W in nets:
        Xd = dev(I.bf16_bits(X).view(np.int16))
        yd = dev(y)
        P = dev(np.concatenate([W[0].ravel(), W[1], W[2], W[3]]).astype(np.float32))
        L = torch.zeros(max(epochs, 1), dtype=torch.float64, device="cuda")
        G = torch.zeros(max(epochs, 1), dtype=torch.float64, device="cuda")
        keep += [Xd, yd]
        params.append(P)
        losses.append(L)
        gns.append(G)
        d = B.mlp_net_desc(W[0].shape[0], X.shape[0], Xd.data_ptr(), yd.data_ptr(), P.data_ptr(), L.data_ptr())
        if norms:
            d.gnorm_hist = G.data_ptr()
        descs.append(d)
    b = B.mlp_batch_create(B.MLP_BF16, act, D_PAD, descs, lr, 1)
    try:
        B.mlp_batch_run(b, epochs, stream())
        st = B.mlp_batch_check(b, stream())
    finally:
        B.mlp_batch_destroy(b)
    assert st == B.MLP_OK, B.mlp_last_error()
    out = [host(p).astype(np.float64) for p in params], [host(l)[:epochs] for l in losses]
    return out + ([host(g)[:epochs] for g in gns],) if norms else out


def flat(W):
    return np.concatenate([np.asarray(W[0]).ravel(), W[1], W[2], np.asarray(W[3]).ravel()]).astype(np.float64)


SHAPES = [(1, 128), (100, 128), (128, 256), (129, 256), (300, 128), (1000, 256)]


def test_one_epoch_gradient_matches_oracle():
    """With lr = 1 one epoch moves the weights by exactly -g (FP32 master)."""
    nets = [make_net(500 + i, n, H) for i, (n, H) in enumerate(SHAPES)]
    got, _ = run_tc(nets, 1, 1.0)
    for (X, y, W), P, (n, H) in zip(nets, got, SHAPES):
        g = flat(W) - P
        ref = oracle.mse_gradients(X, y, Params(*W))
        exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
        assert rel_err_norm(g, exp) <= BF16_GRAD_TOL, (n, H)
        HD = H * D_PAD
        assert rel_err_norm(g[HD:HD + H], ref[1]) <= BF16_GRAD_TOL, ("gb1", n, H)
        assert rel_err_norm(g[HD + H:HD + 2 * H], ref[2]) <= BF16_GRAD_TOL, ("gw2", n, H)
        assert abs(g[-1] - ref[3]) <= BF16_GRAD_TOL * max(abs(ref[3]), np.max(np.abs(exp))), ("gb2", n, H)
        # padded input columns never move
        assert np.all(P[:HD].reshape(H, D_PAD)[:, D_REAL:] == 0.0)


def test_training_tracks_oracle_and_accuracy():
    """30 epochs at lr 0.1: loss history within 2e-2 of the oracle's and the
    train accuracy within one point."""
    shapes = [(2000, 128), (3000, 256)]
    nets = [make_net(900 + i, n, H) for i, (n, H) in enumerate(shapes)]
    epochs = 30
    got, gl = run_tc(nets, epochs, lr32())
    for (X, y, W), P, L, (n, H) in zip(nets, got, gl, shapes):
        q, lh, _ = oracle.train(X, y, Params(*W), lr32(), epochs)
        assert rel_err_elem(L, lh) <= 2e-2, (n, H)
        HD = H * D_PAD
        pg = Params(P[:HD].reshape(H, D_PAD), P[HD:HD + H], P[HD + H:HD + 2 * H], P[-1])
        acc_gpu = (oracle.predict(X, pg) == y).mean()
        acc_ref = (oracle.predict(X, q) == y).mean()
        assert abs(acc_gpu - acc_ref) <= 0.01, (acc_gpu, acc_ref)


def test_tc_batch_is_deterministic_and_validates():
    nets = [make_net(1300 + i, n, H) for i, (n, H) in enumerate([(257, 128), (640, 256)])]
    a, la = run_tc(nets, 3, lr32())
    b, lb = run_tc(nets, 3, lr32())
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    import torch
    P = torch.zeros(1024, device="cuda")
    bad = B.mlp_net_desc(100, 5, P.data_ptr(), P.data_ptr(), P.data_ptr(), 0)
    with pytest.raises(B.MLPError) as e:
        B.mlp_batch_create(B.MLP_BF16, 0, D_PAD, [bad], 0.1, 1)
    assert e.value.status == B.MLP_EINVAL


@pytest.mark.parametrize("D_real,D_pad", [(5, 8), (13, 16), (33, 40), (50, 56)])
def test_one_epoch_gradient_over_input_widths(D_real, D_pad):
    """Every supported width class of the many-nets plan, H = 128 and 256."""
    import torch
    nets, shapes = [], [(300, 128), (513, 256)]
    for i, (n, H) in enumerate(shapes):
        X = I.bf16_round(I.features(5000 + 10 * D_pad + i, n, D_real, D_pad))
        y = (X[:, 0] + X[:, 1] > 0).astype(np.float32)
        nets.append((X, y, I.init_weights(5100 + 10 * D_pad + i, D_real, H, D_pad)))
    keep, descs, params = [], [], []
    for X, y, W in nets:
        Xd = dev(I.bf16_bits(X).view(np.int16))
        yd = dev(y)
        P = dev(np.concatenate([W[0].ravel(), W[1], W[2], W[3]]).astype(np.float32))
        keep += [Xd, yd]
        params.append(P)
        descs.append(B.mlp_net_desc(W[0].shape[0], X.shape[0], Xd.data_ptr(), yd.data_ptr(), P.data_ptr(), 0))
    b = B.mlp_batch_create(B.MLP_BF16, B.MLP_ACT_SIGMOID, D_pad, descs, 1.0, 1)
    try:
        B.mlp_batch_run(b, 1, stream())
        assert B.mlp_batch_check(b, stream()) == B.MLP_OK, B.mlp_last_error()
    finally:
        B.mlp_batch_destroy(b)
    for (X, y, W), P in zip(nets, params):
        got = host(P).astype(np.float64)
        g = flat(W) - got
        ref = oracle.mse_gradients(X, y, Params(*W))
        exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
        assert rel_err_norm(g, exp) <= BF16_GRAD_TOL, (D_pad, W[0].shape[0])
        H = W[0].shape[0]
        assert np.all(got[:H * D_pad].reshape(H, D_pad)[:, D_real:] == 0.0)


def test_gradient_norm_matches_oracle():
    """gnorm_hist on the bf16 path: the FP64 2-norm of the FP32 gradient each
    epoch's update applied, within the bf16 gradient bar of the oracle's."""
    nets = [make_net(1400 + i, n, H) for i, (n, H) in enumerate([(700, 128), (1500, 256)])]
    got, _, gn = run_tc(nets, 5, lr32(), norms=True)
    for (X, y, W), G in zip(nets, gn):
        _, _, gh = oracle.train(X, y, Params(*W), lr32(), 5)
        assert rel_err_elem(G, gh) <= BF16_GRAD_TOL


def test_tanh_one_epoch_gradient_and_training():
    """tanh hidden units (Sec. 2.2's other activation) on the tensor cores:
    the one-epoch gradient within the bf16 bar, and 30 epochs at lr 0.1 with
    the loss history within 2e-2 and train accuracy within one point."""
    nets = [make_net(1500 + i, n, H) for i, (n, H) in enumerate([(300, 128), (1000, 256)])]
    got, _ = run_tc(nets, 1, 1.0, act=B.MLP_ACT_TANH)
    for (X, y, W), P in zip(nets, got):
        ref = oracle.mse_gradients(X, y, Params(*W), act=oracle.ACT_TANH)
        exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
        assert rel_err_norm(flat(W) - P, exp) <= BF16_GRAD_TOL
    nets = [make_net(1600 + i, n, H) for i, (n, H) in enumerate([(2000, 128), (3000, 256)])]
    got, gl = run_tc(nets, 30, lr32(), act=B.MLP_ACT_TANH)
    for (X, y, W), P, L in zip(nets, got, gl):
        q, lh, _ = oracle.train(X, y, Params(*W), lr32(), 30, act=oracle.ACT_TANH)
        assert rel_err_elem(L, lh) <= 2e-2
        H = W[0].shape[0]
        HD = H * D_PAD
        pg = Params(P[:HD].reshape(H, D_PAD), P[HD:HD + H], P[HD + H:HD + 2 * H], P[-1])
        acc_gpu = (oracle.predict(X, pg, act=oracle.ACT_TANH) == y).mean()
        acc_ref = (oracle.predict(X, q, act=oracle.ACT_TANH) == y).mean()
        assert abs(acc_gpu - acc_ref) <= 0.01, (acc_gpu, acc_ref)


def test_config_1024_nets_200_epochs_against_stored_oracle_runs():
    """The 1024-net workload at full size (48-256-1, n ~ U{4096..16384}, 10.5M
    bf16 rows), every net trained on its first 75 % of rows for all 200
    epochs in one launch of the plan; four nets (the first, the largest, the
    smallest, the last) against the oracle's runs of the same 200 epochs
    (tests/golden/c4_sampled_nets_200epochs.json): train and test accuracy
    within one point, loss and gradient-norm histories within 2e-2, and the
    stored weights' change within 2e-2 (max-norm relative)."""
    import json
    import os
    import torch
    from tests import bf16_workloads as WL
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c4_sampled_nets_200epochs.json")))
    ns = WL.c4_shapes()
    picks = WL.c4_picks(ns)
    assert picks == [g["net"] for g in gold["nets"]]
    offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    total = int(offs[-1])
    D, H = WL.D_PAD, WL.C4_H
    T = Params(*I.teacher_weights(D=WL.D_REAL, Dpad=D))
    Xd = torch.zeros((total, D), dtype=torch.bfloat16, device="cuda")
    yd = torch.zeros(total, dtype=torch.float32, device="cuda")
    keep = {t: [] for t in picks}
    for r0, rows in WL.c4_chunks(ns):
        Xc = WL.c4_chunk(r0, rows)
        yc = oracle.predict(Xc, T).astype(np.float32)
        Xd[r0:r0 + rows] = torch.from_numpy(I.bf16_bits(Xc).view(np.int16)).to("cuda").view(torch.bfloat16)
        yd[r0:r0 + rows] = torch.from_numpy(yc).to("cuda")
        for t in picks:
            a, b = max(int(offs[t]), r0), min(int(offs[t + 1]), r0 + rows)
            if a < b:
                keep[t].append((Xc[a - r0:b - r0], yc[a - r0:b - r0]))
    W = [WL.c4_weights(t) for t in range(WL.C4_NETS)]
    P = torch.from_numpy(np.concatenate([np.concatenate([np.ravel(a) for a in w]) for w in W]).astype(np.float32)).cuda()
    Pp = (D + 2) * H + 1
    ntr = [I.split_count(int(n)) for n in ns]
    L = torch.zeros((WL.C4_NETS, WL.C4_EPOCHS), dtype=torch.float64, device="cuda")
    G = torch.zeros((WL.C4_NETS, WL.C4_EPOCHS), dtype=torch.float64, device="cuda")
    descs = []
    for t in range(WL.C4_NETS):
        d = B.mlp_net_desc(H, ntr[t], Xd[int(offs[t]):].data_ptr(), yd[int(offs[t]):].data_ptr(),
                           P[t * Pp:].data_ptr(), L[t].data_ptr())
        d.gnorm_hist = G[t].data_ptr()
        descs.append(d)
    b = B.mlp_batch_create(B.MLP_BF16, B.MLP_ACT_SIGMOID, D, descs, lr32(), 1)
    try:
        B.mlp_batch_run(b, WL.C4_EPOCHS, stream())
        assert B.mlp_batch_check(b, stream()) == B.MLP_OK, B.mlp_last_error()
    finally:
        B.mlp_batch_destroy(b)
    Ph, Lh, Gh = host(P).astype(np.float64), host(L), host(G)
    for t, g in zip(picks, gold["nets"]):
        X = np.concatenate([x for x, _ in keep[t]])
        y = np.concatenate([v for _, v in keep[t]])
        n1 = g["n_train"]
        assert X.shape[0] == ns[t] == g["n"] and n1 == ntr[t]
        p = Ph[t * Pp:(t + 1) * Pp]
        HD = H * D
        pg = Params(p[:HD].reshape(H, D), p[HD:HD + H], p[HD + H:HD + 2 * H], p[-1])
        acc_tr = (oracle.predict(X[:n1], pg) == y[:n1]).mean()
        acc_te = (oracle.predict(X[n1:], pg) == y[n1:]).mean()
        assert abs(acc_tr - g["train_acc"]) <= 0.01, (t, acc_tr, g["train_acc"])
        assert abs(acc_te - g["test_acc"]) <= 0.01, (t, acc_te, g["test_acc"])
        assert rel_err_elem(Lh[t], g["loss_hist"]) <= BF16_GRAD_TOL, t
        assert rel_err_elem(Gh[t], g["gnorm_hist"]) <= BF16_GRAD_TOL, t
        w0 = WL.kept_params(*W[t], WL.C4_KEEP_EVERY)
        got = WL.kept_params(pg.W1, pg.b1, pg.w2, pg.b2, WL.C4_KEEP_EVERY)
        assert rel_err_norm(got - w0, np.asarray(g["kept_params"]) - w0) <= BF16_GRAD_TOL, t
