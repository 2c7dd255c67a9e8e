"""GPU parity of the many-nets kernel (one launch trains every net) against the
FP64 oracle run net by net (Sec. 2.1's separately trained subsets, generalised;
Sec. 2.2's full-batch gradient descent)."""
import numpy as np
import pytest

import oracle
from oracle import Params
from paper_1908_07847_gb300 import binding as B
from paper_1908_07847_gb300 import inputs as I
from tests.gpu_util import W_TOL, dev, host, lr32, rel_err_elem, rel_err_norm, stream

pytestmark = pytest.mark.gpu


def torch():
    import torch as t
    return t


def make_batch(seed, Hs, ns, D=33):
    nets = []
    for t, (H, n) in enumerate(zip(Hs, ns)):
        X = I.features(I.subseed(seed, 100 + t), int(n), D)
        y = oracle.predict(X, Params(*I.teacher_weights(D=D))).astype(np.float32)
        W = I.init_weights(I.subseed(seed, 200 + t), D, int(H))
        nets.append((X, y, W))
    return nets


def run_batch(nets, epochs, D=33, act=B.MLP_ACT_SIGMOID):
    t = torch()
    keep, descs, params, losses = [], [], [], []
    for X, y, W in nets:
        Xd, yd = dev(X), dev(y)
        P = dev(np.concatenate([W[0].ravel(), W[1], W[2], W[3]]).astype(np.float32))
        L = t.zeros(max(epochs, 1), dtype=t.float64, device="cuda")
        keep += [Xd, yd]
        params.append(P)
        losses.append(L)
        descs.append(B.mlp_net_desc(W[0].shape[0], X.shape[0], Xd.data_ptr(), yd.data_ptr(), P.data_ptr(),
                                    L.data_ptr()))
    b = B.mlp_batch_create(B.MLP_FP32, act, D, descs, lr32(), 1)
    try:
        B.mlp_batch_run(b, epochs, stream())
        assert B.mlp_batch_check(b, stream()) == B.MLP_OK
    finally:
        B.mlp_batch_destroy(b)
    return [host(p).astype(np.float64) for p in params], [host(l)[:epochs] for l in losses]


EDGE_H = [1, 3, 4, 5, 8, 9, 16, 17, 31, 32, 33, 40, 63, 64, 65, 100, 127, 128]
EDGE_N = [1, 2, 7, 50, 97, 120, 255, 256, 257, 300, 600]


def test_edge_shapes_match_oracle():
    rng = np.random.default_rng(1)
    Hs = EDGE_H + list(rng.integers(1, 129, 12))
    ns = [EDGE_N[i % len(EDGE_N)] for i in range(len(Hs))]
    nets = make_batch(5, Hs, ns)
    epochs = 15
    got, gl = run_batch(nets, epochs)
    ref, rl = oracle.batch_train([(X, y, Params(*W)) for X, y, W in nets], lr32(), epochs, threads=8)
    for t in range(len(nets)):
        assert rel_err_norm(got[t], ref[t].flat()) <= W_TOL, (t, Hs[t], ns[t])
        assert rel_err_elem(gl[t], rl[t]) <= 1e-5, (t, Hs[t], ns[t])


def test_tanh_batch_matches_oracle():
    nets = make_batch(6, [7, 48, 90], [60, 120, 200])
    got, _ = run_batch(nets, 10, act=B.MLP_ACT_TANH)
    ref, _ = oracle.batch_train([(X, y, Params(*W)) for X, y, W in nets], lr32(), 10, act=oracle.ACT_TANH,
                                threads=3)
    for t in range(3):
        assert rel_err_norm(got[t], ref[t].flat()) <= W_TOL


def test_config_4096_nets_500_epochs_sampled():
    """4096 nets, H ~ U{4..128}, n ~ U{50..120}, 500 epochs in one launch; 24
    nets spread over the H range are checked against the oracle."""
    Hs, ns = I.batched_shapes(2, 4096, (4, 128), (50, 120))
    nets = make_batch(2, Hs, ns)
    got, gl = run_batch(nets, 500)
    idx = np.argsort(Hs)[np.linspace(0, 4095, 24).astype(int)]
    sample = [(nets[i][0], nets[i][1], Params(*nets[i][2])) for i in idx]
    ref, rl = oracle.batch_train(sample, lr32(), 500, threads=8)
    for k, i in enumerate(idx):
        assert rel_err_norm(got[i], ref[k].flat()) <= 1e-3, (i, Hs[i], ns[i])
        assert rel_err_elem(gl[i][-1:], rl[k][-1:]) <= 1e-3


def test_batched_is_deterministic_and_matches_single_net_path():
    nets = make_batch(7, [64, 20, 100], [120, 77, 90])
    a, _ = run_batch(nets, 50)
    b, _ = run_batch(nets, 50)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    X, y, W = nets[0]
    h = B.mlp_create(33, 64, 0.1, 1, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    try:
        B.mlp_set_weights(h, *W)
        B.mlp_train_epochs(h, dev(X), dev(y), X.shape[0], 50, 0, None, None, stream())
        W1 = np.zeros((64, 33), np.float32)
        b1 = np.zeros(64, np.float32)
        w2 = np.zeros(64, np.float32)
        b2 = np.zeros(1, np.float32)
        B.mlp_get_weights(h, W1, b1, w2, b2)
        single = np.concatenate([W1.ravel(), b1, w2, b2]).astype(np.float64)
    finally:
        B.mlp_destroy(h)
    assert rel_err_norm(a[0], single) <= 1e-5


def test_empty_net_and_validation():
    t = torch()
    X, y, W = make_batch(8, [10], [40])[0]
    P = dev(np.concatenate([W[0].ravel(), W[1], W[2], W[3]]).astype(np.float32))
    L = t.full((3,), 5.0, dtype=t.float64, device="cuda")
    d0 = B.mlp_net_desc(10, 0, 0, 0, P.data_ptr(), L.data_ptr())
    before = host(P).copy()
    b = B.mlp_batch_create(B.MLP_FP32, 0, 33, [d0], lr32(), 1)
    B.mlp_batch_run(b, 3, stream())
    assert B.mlp_batch_check(b, stream()) == B.MLP_OK
    B.mlp_batch_destroy(b)
    assert np.array_equal(host(P), before) and (host(L) == 0).all()
    bad = B.mlp_net_desc(129, 5, P.data_ptr(), P.data_ptr(), P.data_ptr(), 0)
    with pytest.raises(B.MLPError) as e:
        B.mlp_batch_create(B.MLP_FP32, 0, 33, [bad], lr32(), 1)
    assert e.value.status == B.MLP_EINVAL
