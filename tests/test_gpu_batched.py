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


def run_batch(nets, epochs, D=33, act=B.MLP_ACT_SIGMOID, shape=None):
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
        if shape is not None:
            B.mlp_batch_set_shape(b, shape)
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
        assert rel_err_norm(got[i], ref[k].flat()) <= W_TOL, (i, Hs[i], ns[i])
        # the loss history follows the weights (same bar as the weights)
        assert rel_err_elem(gl[i], rl[k]) <= W_TOL, (i, Hs[i], ns[i])


def test_gradient_norm_history_matches_oracle():
    """gnorm_hist: the FP64 2-norm of each epoch's gradient, against the
    oracle's (Sec. 2.2's full-batch step; the norm is the convergence check)."""
    t = torch()
    nets = make_batch(9, [5, 40, 128], [70, 120, 300])
    keep, descs, params, norms = [], [], [], []
    for X, y, W in nets:
        Xd, yd = dev(X), dev(y)
        P = dev(np.concatenate([W[0].ravel(), W[1], W[2], W[3]]).astype(np.float32))
        G = t.zeros(20, dtype=t.float64, device="cuda")
        keep += [Xd, yd]
        params.append(P)
        norms.append(G)
        d = B.mlp_net_desc(W[0].shape[0], X.shape[0], Xd.data_ptr(), yd.data_ptr(), P.data_ptr(), None)
        d.gnorm_hist = G.data_ptr()
        descs.append(d)
    b = B.mlp_batch_create(B.MLP_FP32, B.MLP_ACT_SIGMOID, 33, descs, lr32(), 1)
    try:
        B.mlp_batch_run(b, 20, stream())
        assert B.mlp_batch_check(b, stream()) == B.MLP_OK
    finally:
        B.mlp_batch_destroy(b)
    for (X, y, W), P, G in zip(nets, params, norms):
        q, _, gh = oracle.train(X, y, Params(*W), lr32(), 20)
        assert rel_err_elem(host(G), gh) <= 1e-4
        assert rel_err_norm(host(P), q.flat()) <= W_TOL


def test_net_result_does_not_depend_on_the_batch():
    """A net trained alone and the same net trained among others (taken by
    another block, in another order) end bitwise equal: every net's arithmetic
    is its block's alone."""
    nets = make_batch(10, [17, 64, 100, 3, 128], [90, 120, 51, 77, 300])
    together, lt = run_batch(nets, 25)
    for i in (0, 2, 4):
        alone, la = run_batch([nets[i]], 25)
        assert np.array_equal(alone[0], together[i]) and np.array_equal(la[0], lt[i]), i


def test_host_buffer_plan_equals_device_plan():
    """mlp_batch_run_host (rows, labels and weights copied in, weights and
    losses copied out) trains exactly what the device-buffer plan trains;
    fewer epochs than the plan's maximum leave the loss layout n_nets x epochs."""
    t = torch()
    Hs, ns = [12, 64, 128, 33], [50, 120, 97, 260]
    nets = make_batch(11, Hs, ns)
    dev_w, dev_l = run_batch(nets, 30)
    X = np.concatenate([X for X, _, _ in nets])
    y = np.concatenate([y for _, y, _ in nets])
    P0 = np.concatenate([np.concatenate([W[0].ravel(), W[1], W[2], W[3]]) for _, _, W in nets]).astype(np.float32)
    Pout = np.zeros_like(P0)
    L = np.zeros((len(nets), 30))
    b = B.mlp_batch_create_host(B.MLP_FP32, B.MLP_ACT_SIGMOID, 33, Hs, ns, 40, lr32(), 1)
    try:
        B.mlp_batch_run_host(b, X, y, P0, Pout, L, 30, stream())
        B.mlp_batch_run_host(b, X, y, P0, Pout, L, 30, stream())    # a second call starts afresh
        with pytest.raises(B.MLPError) as e:
            B.mlp_batch_run_host(b, X, y, P0, Pout, L, 41, stream())
        assert e.value.status == B.MLP_EINVAL
    finally:
        B.mlp_batch_destroy(b)
    offs = np.concatenate([[0], np.cumsum([(33 + 2) * H + 1 for H in Hs])])
    for i in range(len(nets)):
        assert np.array_equal(Pout[offs[i]:offs[i + 1]].astype(np.float64), dev_w[i]), i
        assert np.array_equal(L[i], dev_l[i]), i
    # a plan made from device descriptors has no host copies to run
    Xd, yd = dev(nets[0][0]), dev(nets[0][1])
    P = dev(P0[:offs[1]])
    d = B.mlp_batch_create(B.MLP_FP32, 0, 33, [B.mlp_net_desc(Hs[0], ns[0], Xd.data_ptr(), yd.data_ptr(),
                                                               P.data_ptr(), None)], lr32(), 1)
    try:
        with pytest.raises(B.MLPError) as e:
            B.mlp_batch_run_host(d, X, y, P0, Pout, None, 1, stream())
        assert e.value.status == B.MLP_EINVAL
    finally:
        B.mlp_batch_destroy(d)


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
    # Not bitwise: the single-net kernel sums the gradient across blocks in
    # 64-bit fixed point (resolution 2^-40), the many-nets kernel in FP32 in
    # shared memory; both are within the FP32 bars of the oracle.
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


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5, 6])
def test_kernel_shapes_match_oracle(shape):
    """The other kernel shapes (two units a lane: segments of 2..32 lanes, one
    and two warps a row; register-tiled: 4 x 4 tiles over row chunks of 128,
    64 or 32 rows) over every width edge and row counts up to streamed ones,
    sigmoid and tanh, against the oracle at the FP32 bars."""
    rng = np.random.default_rng(2)
    Hs = EDGE_H + [2] + list(rng.integers(1, 129, 8))
    ns = [EDGE_N[i % len(EDGE_N)] for i in range(len(Hs))]
    nets = make_batch(12, Hs, ns)
    got, gl = run_batch(nets, 15, shape=shape)
    ref, rl = oracle.batch_train([(X, y, Params(*W)) for X, y, W in nets], lr32(), 15, threads=8)
    for t in range(len(nets)):
        assert rel_err_norm(got[t], ref[t].flat()) <= W_TOL, (shape, t, Hs[t], ns[t])
        assert rel_err_elem(gl[t], rl[t]) <= 1e-5, (shape, t, Hs[t], ns[t])
    tn = make_batch(13, [7, 48, 90, 128], [60, 120, 200, 33])
    got, _ = run_batch(tn, 10, act=B.MLP_ACT_TANH, shape=shape)
    ref, _ = oracle.batch_train([(X, y, Params(*W)) for X, y, W in tn], lr32(), 10, act=oracle.ACT_TANH, threads=4)
    for t in range(len(tn)):
        assert rel_err_norm(got[t], ref[t].flat()) <= W_TOL, ("tanh", shape, t)


@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5, 6])
def test_every_shape_on_plans_of_tiny_nets(shape):
    """Plans whose widest net has at most 4 hidden units and whose nets have
    at most 4 rows, on every kernel shape: in the register-tiled shapes the
    smallest h / d1 buffer still takes at least four rows a pass (the layout
    reserves four rows at the widest stride), against the oracle."""
    for Hs, ns in (([1, 2, 3, 4], [1, 2, 3, 4]), ([1, 1], [4, 3]), ([2], [1])):
        nets = make_batch(40 + len(Hs), Hs, ns)
        got, gl = run_batch(nets, 20, shape=shape)
        ref, rl = oracle.batch_train([(X, y, Params(*W)) for X, y, W in nets], lr32(), 20, threads=2)
        for t in range(len(nets)):
            assert rel_err_norm(got[t], ref[t].flat()) <= W_TOL, (shape, Hs[t], ns[t])
            assert rel_err_elem(gl[t], rl[t]) <= 1e-5, (shape, Hs[t], ns[t])


@pytest.mark.parametrize("shape", [1, 3])
@pytest.mark.parametrize("D", [1, 5, 8, 16, 20, 32, 35, 36])
def test_input_width_classes_of_the_other_shapes(D, shape):
    """Every input-width class of the two-units-a-lane shape (zero-padded
    row buffers for D below the class width) and of the tiled shape."""
    nets = make_batch(14 + D, [3, 40, 100], [50, 129, 90], D=D)
    got, _ = run_batch(nets, 12, D=D, shape=shape)
    ref, _ = oracle.batch_train([(X, y, Params(*W)) for X, y, W in nets], lr32(), 12, threads=3)
    for t in range(3):
        assert rel_err_norm(got[t], ref[t].flat()) <= W_TOL, (D, t)


def test_shape_validation_and_autotuner(tmp_path, monkeypatch):
    """Shape 2 needs D = 33, shapes 1-2 need D <= 36; the autotuner times the
    shapes a plan takes, keeps the fastest, restores the weights it trained,
    and the tuned plan trains what the default shape trains within the FP32
    bar."""
    import torch
    from paper_1908_07847_gb300 import autotune
    monkeypatch.setenv("MLP_GB300_TUNE_CACHE", str(tmp_path / "tune.json"))
    Hs, ns = I.batched_shapes(21, 200, (4, 128), (50, 120))
    nets = make_batch(21, Hs, ns)
    keep, descs = [], []
    P = torch.from_numpy(np.concatenate([np.concatenate([W[0].ravel(), W[1], W[2], W[3]]) for _, _, W in nets])
                         .astype(np.float32)).cuda()
    P0 = P.clone()
    o = 0
    for X, y, W in nets:
        Xd, yd = dev(X), dev(y)
        keep += [Xd, yd]
        descs.append(B.mlp_net_desc(W[0].shape[0], X.shape[0], Xd.data_ptr(), yd.data_ptr(), P[o:].data_ptr(), None))
        o += (33 + 2) * W[0].shape[0] + 1
    b = B.mlp_batch_create(B.MLP_FP32, B.MLP_ACT_SIGMOID, 33, descs, lr32(), 1)
    try:
        assert B.mlp_batch_get_shape(b) == 0
        shape, times = autotune.tune_batched(b, 33, Hs, ns, P, epochs=5, reps=1)
        assert set(times) == {0, 1, 2, 3, 4, 5, 6} and shape in times and B.mlp_batch_get_shape(b) == shape
        assert torch.equal(P, P0)                       # the tuner's launches were undone
        again, _ = autotune.tune_batched(b, 33, Hs, ns, P, epochs=5, reps=1)   # from the cache
        assert again == shape and torch.equal(P, P0)
        B.mlp_batch_run(b, 30, stream())
        assert B.mlp_batch_check(b, stream()) == B.MLP_OK
        tuned = host(P).astype(np.float64)
        P.copy_(P0)
        B.mlp_batch_set_shape(b, 0)
        B.mlp_batch_run(b, 30, stream())
        assert B.mlp_batch_check(b, stream()) == B.MLP_OK
        assert rel_err_norm(tuned, host(P)) <= W_TOL
    finally:
        B.mlp_batch_destroy(b)
    narrow = make_batch(22, [10], [40], D=40)[0]
    Xd, yd = dev(narrow[0]), dev(narrow[1])
    Pn = dev(np.concatenate([narrow[2][0].ravel(), narrow[2][1], narrow[2][2], narrow[2][3]]).astype(np.float32))
    b = B.mlp_batch_create(B.MLP_FP32, 0, 40, [B.mlp_net_desc(10, 40, Xd.data_ptr(), yd.data_ptr(), Pn.data_ptr(),
                                                              None)], lr32(), 1)
    try:
        for bad in (1, 2, 3, 4, 5, 6, 7, -1):
            with pytest.raises(B.MLPError) as e:
                B.mlp_batch_set_shape(b, bad)
            assert e.value.status == B.MLP_EINVAL
    finally:
        B.mlp_batch_destroy(b)
