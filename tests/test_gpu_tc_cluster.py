"""BF16 tensor-core (tcgen05) training of one wide network (clusters of H/256
blocks sharing z2 through distributed shared memory; Sec. 2.2 of arXiv
1908.07847: forward, output error, backpropagation, w <- w - lr g) against the
FP64 oracle on the same bf16-exact inputs.  Bars: the gradient within 2e-2
(max-norm relative), train and test accuracy within one point."""
import numpy as np
import pytest

import oracle
from oracle import Params
from paper_1908_07847_gb300 import binding as B
from paper_1908_07847_gb300 import inputs as I
from tests.gpu_util import BF16_GRAD_TOL, Net, dev, host, labels_from_teacher, lr32, rel_err_elem, rel_err_norm, \
    stream

pytestmark = pytest.mark.gpu

D_REAL, D_PAD = 33, 48


def make(seed, n, H):
    X = I.bf16_round(I.features(seed, n, D_REAL, D_PAD))
    y = labels_from_teacher(X, D_REAL)
    W = I.init_weights(seed + 1, D_REAL, H, D_PAD)
    return X, y, W


def flat(W):
    return np.concatenate([np.asarray(W[0]).ravel(), W[1], W[2], np.asarray(W[3]).ravel()]).astype(np.float64)


def unflat(p, H):
    HD = H * D_PAD
    return Params(p[:HD].reshape(H, D_PAD), p[HD:HD + H], p[HD + H:HD + 2 * H], p[-1])


def run(X, y, W, epochs, lr, mb=0, loss_mean=1, act=B.MLP_ACT_SIGMOID, norms=False):
    import torch
    H = W[0].shape[0]
    with Net(D_PAD, H, lr, loss_mean, B.MLP_BF16, act) as net:
        net.set(W)
        Xd = dev(I.bf16_bits(X).view(np.int16))
        yd = dev(y)
        L = torch.zeros(max(epochs, 1), dtype=torch.float64, device="cuda")
        G = torch.zeros(max(epochs, 1), dtype=torch.float64, device="cuda") if norms else None
        B.mlp_train_epochs(net.h, Xd, yd, X.shape[0], epochs, mb, L, G, stream())
        st = net.check()
        assert st == B.MLP_OK, B.mlp_last_error()
        out = net.flat(), host(L)[:epochs]
        return out + (host(G)[:epochs],) if norms else out


ONE_STEP = [(1, 256), (100, 256), (128, 512), (777, 768), (1000, 1024), (2500, 2048)]


@pytest.mark.parametrize("n,H", ONE_STEP)
def test_one_step_gradient_matches_oracle(n, H):
    """Full batch, lr = 1: one epoch moves the FP32 master weights by -g."""
    X, y, W = make(3000 + n + H, n, H)
    got, _ = run(X, y, W, 1, 1.0)
    g = flat(W) - got
    ref = oracle.mse_gradients(X, y, Params(*W))
    exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
    assert rel_err_norm(g, exp) <= BF16_GRAD_TOL
    HD = H * D_PAD
    assert rel_err_norm(g[HD:HD + H], ref[1]) <= BF16_GRAD_TOL, "gb1"
    assert rel_err_norm(g[HD + H:HD + 2 * H], ref[2]) <= BF16_GRAD_TOL, "gw2"
    assert abs(g[-1] - ref[3]) <= BF16_GRAD_TOL * max(abs(ref[3]), np.max(np.abs(exp))), "gb2"
    # padded input columns carry zero gradient
    assert np.all(got[:HD].reshape(H, D_PAD)[:, D_REAL:] == 0.0)


def test_sum_loss_gradient():
    """c = 1 (loss_mean = 0): the gradient is the plain sum over rows."""
    n, H = 3000, 512
    X, y, W = make(3100, n, H)
    lr = 1e-3
    got, _ = run(X, y, W, 1, lr, loss_mean=0)
    g = (flat(W) - got) / lr
    ref = oracle.mse_gradients(X, y, Params(*W), loss_mean=False)
    exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
    assert rel_err_norm(g, exp) <= BF16_GRAD_TOL


def test_minibatch_training_tracks_oracle():
    """Contiguous mini-batches with a ragged last one: loss history, weight
    change and accuracy against the oracle's run of the same schedule."""
    n, H, mb, epochs = 5000, 512, 2048, 4
    X, y, W = make(3200, n, H)
    got, L = run(X, y, W, epochs, lr32(), mb=mb)
    q, lh, _ = oracle.train(X, y, Params(*W), lr32(), epochs, minibatch=mb)
    assert rel_err_elem(L, lh) <= BF16_GRAD_TOL
    d_gpu, d_ref = got - flat(W), q.flat() - flat(W)
    assert rel_err_norm(d_gpu, d_ref) <= BF16_GRAD_TOL
    acc_gpu = (oracle.predict(X, unflat(got, H)) == y).mean()
    acc_ref = (oracle.predict(X, q) == y).mean()
    assert abs(acc_gpu - acc_ref) <= 0.01


def test_wide_net_train_and_test_accuracy():
    """48-2048-1, 75 / 25 split, mini-batch 1024: final train and test accuracy
    within one point of the oracle's."""
    n, H, mb, epochs = 8192, 2048, 1024, 3
    X, y, W = make(3300, n, H)
    ntr = I.split_count(n)
    got, L = run(X[:ntr], y[:ntr], W, epochs, lr32(), mb=mb)
    q, lh, _ = oracle.train(X[:ntr], y[:ntr], Params(*W), lr32(), epochs, minibatch=mb)
    assert rel_err_elem(L, lh) <= BF16_GRAD_TOL
    pg = unflat(got, H)
    for rows in (slice(0, ntr), slice(ntr, n)):
        a_gpu = (oracle.predict(X[rows], pg) == y[rows]).mean()
        a_ref = (oracle.predict(X[rows], q) == y[rows]).mean()
        assert abs(a_gpu - a_ref) <= 0.01, (rows, a_gpu, a_ref)


def test_deterministic_and_continues_across_calls():
    """Fixed-point cross-cluster sums: two runs agree bit for bit; two calls of
    one epoch each equal one call of two epochs."""
    n, H, mb = 2000, 768, 512
    X, y, W = make(3400, n, H)
    a, la = run(X, y, W, 2, lr32(), mb=mb)
    b, lb = run(X, y, W, 2, lr32(), mb=mb)
    assert np.array_equal(a, b) and np.array_equal(la, lb)
    import torch
    with Net(D_PAD, H, lr32(), 1, B.MLP_BF16) as net:
        net.set(W)
        Xd = dev(I.bf16_bits(X).view(np.int16))
        yd = dev(y)
        for _ in range(2):
            B.mlp_train_epochs(net.h, Xd, yd, n, 1, mb, None, None, stream())
        assert net.check() == B.MLP_OK
        assert np.array_equal(net.flat(), a)


def test_nonfinite_loss_is_reported():
    n, H = 300, 256
    X, y, W = make(3500, n, H)
    y = y.copy()
    y[7] = np.inf
    with Net(D_PAD, H, lr32(), 1, B.MLP_BF16) as net:
        net.set(W)
        B.mlp_train_epochs(net.h, dev(I.bf16_bits(X).view(np.int16)), dev(y), n, 2, 0, None, None, stream())
        assert net.check() == B.MLP_ENONFINITE


def test_wide_net_65536_row_subset_one_epoch():
    """The wide workload's own schedule on its first 65,536 rows: 48-2048-1,
    mini-batch 8192 (eight updates), against the oracle run of the same
    schedule: loss and weight change within 2e-2, accuracy within one point."""
    n, H, mb = 65536, 2048, 8192
    X, y, W = make(3600, n, H)
    got, L = run(X, y, W, 1, lr32(), mb=mb)
    q, lh, _ = oracle.train(X, y, Params(*W), lr32(), 1, minibatch=mb)
    assert rel_err_elem(L, lh) <= BF16_GRAD_TOL
    assert rel_err_norm(got - flat(W), q.flat() - flat(W)) <= BF16_GRAD_TOL
    acc_gpu = (oracle.predict(X, unflat(got, H)) == y).mean()
    acc_ref = (oracle.predict(X, q) == y).mean()
    assert abs(acc_gpu - acc_ref) <= 0.01


@pytest.mark.parametrize("D_real,D_pad", [(5, 8), (13, 16), (33, 40), (48, 48)])
def test_one_step_gradient_over_input_widths(D_real, D_pad):
    """Every supported width class: the forward covers D rounded up to 16
    columns, the gradient MMA carries the ones column at column D."""
    n, H = 700, 512
    X = I.bf16_round(I.features(3700 + D_pad, n, D_real, D_pad))
    y = (X[:, 0] + X[:, 1] > 0).astype(np.float32)
    W = I.init_weights(3800 + D_pad, D_real, H, D_pad)
    import torch
    with Net(D_pad, H, 1.0, 1, B.MLP_BF16) as net:
        net.set(W)
        B.mlp_train_epochs(net.h, dev(I.bf16_bits(X).view(np.int16)), dev(y), n, 1, 0, None, None, stream())
        assert net.check() == B.MLP_OK, B.mlp_last_error()
        got = net.flat()
    g = flat(W) - got
    ref = oracle.mse_gradients(X, y, Params(*W))
    exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
    assert rel_err_norm(g, exp) <= BF16_GRAD_TOL
    HD = H * D_pad
    assert rel_err_norm(g[HD:HD + H], ref[1]) <= BF16_GRAD_TOL, "gb1"
    assert np.all(got[:HD].reshape(H, D_pad)[:, D_real:] == 0.0)


@pytest.mark.parametrize("mb", [0, 1000])
def test_gradient_norm_matches_oracle(mb):
    """gnorm_hist on the cluster kernel (full batch, and mini-batches whose
    last one is ragged: the norm of each epoch's last update) within the bf16
    gradient bar of the oracle's."""
    n, H = 2600, 768
    X, y, W = make(3900 + mb, n, H)
    got, L, G = run(X, y, W, 3, lr32(), mb=mb, norms=True)
    q, lh, gh = oracle.train(X, y, Params(*W), lr32(), 3, minibatch=mb)
    assert rel_err_elem(G, gh) <= BF16_GRAD_TOL
    assert rel_err_elem(L, lh) <= BF16_GRAD_TOL


@pytest.mark.parametrize("n,H", [(300, 256), (1500, 1024)])
def test_tanh_one_step_gradient(n, H):
    """tanh hidden units (Sec. 2.2's other activation) on the cluster kernel:
    one full-batch step at lr = 1 moves the weights by -g within the bf16 bar."""
    X, y, W = make(4000 + n, n, H)
    got, _ = run(X, y, W, 1, 1.0, act=B.MLP_ACT_TANH)
    ref = oracle.mse_gradients(X, y, Params(*W), act=oracle.ACT_TANH)
    exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
    g = flat(W) - got
    assert rel_err_norm(g, exp) <= BF16_GRAD_TOL
    HD = H * D_PAD
    assert rel_err_norm(g[HD:HD + H], ref[1]) <= BF16_GRAD_TOL, "gb1"
    assert rel_err_norm(g[HD + H:HD + 2 * H], ref[2]) <= BF16_GRAD_TOL, "gw2"


def test_tanh_minibatch_training_accuracy():
    n, H, mb, epochs = 4000, 512, 1024, 4
    X, y, W = make(4100, n, H)
    got, L = run(X, y, W, epochs, lr32(), mb=mb, act=B.MLP_ACT_TANH)
    q, lh, _ = oracle.train(X, y, Params(*W), lr32(), epochs, minibatch=mb, act=oracle.ACT_TANH)
    assert rel_err_elem(L, lh) <= BF16_GRAD_TOL
    acc_gpu = (oracle.predict(X, unflat(got, H), act=oracle.ACT_TANH) == y).mean()
    acc_ref = (oracle.predict(X, q, act=oracle.ACT_TANH) == y).mean()
    assert abs(acc_gpu - acc_ref) <= 0.01


def test_wide_net_20_epochs_against_stored_oracle_run():
    """The wide workload's whole schedule on its first 65,536 rows: 48-2048-1,
    the first 49,152 rows (75 %) trained by mini-batches of 8192 for 20 epochs
    (120 updates), against the oracle's run of the same schedule
    (tests/golden/c3_wide_net_20epochs.json): train and test accuracy within
    one point, loss and gradient-norm histories within 2e-2, and the stored
    weights' change within 2e-2 (max-norm relative)."""
    import json
    import os
    from tests import bf16_workloads as WL
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c3_wide_net_20epochs.json")))
    X = WL.c3_rows()
    y = labels_from_teacher(X, D_REAL)
    W = WL.c3_weights()
    ntr = WL.C3_TRAIN
    got, L, G = run(X[:ntr], y[:ntr], W, WL.C3_EPOCHS, lr32(), mb=WL.C3_MB, norms=True)
    pg = unflat(got, WL.C3_H)
    acc_tr = (oracle.predict(X[:ntr], pg) == y[:ntr]).mean()
    acc_te = (oracle.predict(X[ntr:], pg) == y[ntr:]).mean()
    assert abs(acc_tr - gold["train_acc"]) <= 0.01, (acc_tr, gold["train_acc"])
    assert abs(acc_te - gold["test_acc"]) <= 0.01, (acc_te, gold["test_acc"])
    assert rel_err_elem(L, gold["loss_hist"]) <= BF16_GRAD_TOL
    assert rel_err_elem(G, gold["gnorm_hist"]) <= BF16_GRAD_TOL
    w0 = WL.kept_params(*W, WL.C3_KEEP_EVERY)
    w = WL.kept_params(pg.W1, pg.b1, pg.w2, pg.b2, WL.C3_KEEP_EVERY)
    assert rel_err_norm(w - w0, np.asarray(gold["kept_params"]) - w0) <= BF16_GRAD_TOL


def test_cluster_count_knob_and_tuner(tmp_path, monkeypatch):
    """The cluster count (mlp_set_clusters) changes how a step's tiles are
    dealt and the order of the cross-cluster sum, not the method: 1, 3 and
    the default cluster counts each train within the bf16 bar of the oracle.
    The tuner picks one of its candidates, caches it, and bad values are
    refused."""
    import torch
    from paper_1908_07847_gb300 import autotune
    monkeypatch.setenv("MLP_GB300_TUNE_CACHE", str(tmp_path / "tune.json"))
    H, n, mb, epochs, lr = 1024, 6000, 2048, 2, 0.5
    kmax = B.mlp_cluster_limit(H)
    assert kmax >= 1
    with pytest.raises(B.MLPError) as e:
        B.mlp_cluster_limit(300)
    assert e.value.status == B.MLP_EINVAL
    X, y, W = make(3900, n, H)
    q, _, _ = oracle.train(X, y, Params(*W), float(np.float32(lr)), epochs, minibatch=mb)
    dref = q.flat() - flat(W)
    Xd = dev(I.bf16_bits(X).view(np.int16))
    yd = dev(y)
    for k in (1, 3, 0):
        with Net(D_PAD, H, lr, 1, B.MLP_BF16, B.MLP_ACT_SIGMOID) as net:
            net.set(W)
            with pytest.raises(B.MLPError):
                B.mlp_set_clusters(net.h, -1)
            B.mlp_set_clusters(net.h, k)
            B.mlp_train_epochs(net.h, Xd, yd, n, epochs, mb, None, None, stream())
            assert net.check() == B.MLP_OK, B.mlp_last_error()
            assert rel_err_norm(net.flat() - flat(W), dref) <= BF16_GRAD_TOL, k
    cands = sorted({1, max(1, kmax - 1), kmax})
    best, times = autotune.tune_clusters(Xd, yd, D_PAD, H, n, mb, candidates=cands, steps=2, reps=1)
    assert best in cands and set(times) == set(cands)
    again, _ = autotune.tune_clusters(Xd, yd, D_PAD, H, n, mb, candidates=cands, steps=2, reps=1)
    assert again == best
    torch.cuda.synchronize()
