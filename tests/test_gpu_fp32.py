"""GPU parity of the FP32 / FP64 / BF16-input paths against the FP64 oracle,
called through the C ABI (Sec. 2.2 and Eq. 1 of arXiv 1908.07847)."""
import numpy as np
import pytest

import oracle
from oracle import Params
from paper_1908_07847_gb300 import binding as B
from paper_1908_07847_gb300 import inputs as I
from tests.gpu_util import (BF16_GRAD_TOL, FWD_TOL, GRAD_TOL, W_TOL, Net, dev, host, lr32, problem,
                            rel_err_elem, rel_err_norm, stream)

pytestmark = pytest.mark.gpu


def torch():
    import torch as t
    return t


SHAPES = [(1, 1, 1), (17, 7, 16), (95, 33, 16), (96, 33, 17), (97, 33, 64), (300, 48, 33),
          (1000, 33, 64), (257, 64, 100), (130, 5, 130), (4096, 33, 64)]


@pytest.mark.parametrize("n,D,H", SHAPES)
def test_forward_matches_oracle(n, D, H):
    X, y, W = problem(100 + n, n, D, H)
    with Net(D, H) as net:
        net.set(W)
        o = torch().zeros(n, dtype=torch().float32, device="cuda")
        B.mlp_forward(net.h, dev(X), n, o, stream())
        _, o_ref = oracle.forward(X, Params(*W))
        assert rel_err_elem(host(o), o_ref) <= FWD_TOL


@pytest.mark.parametrize("n,D,H", SHAPES)
@pytest.mark.parametrize("loss_mean", [1, 0])
def test_gradients_match_oracle(n, D, H, loss_mean):
    X, y, W = problem(200 + n, n, D, H)
    t = torch()
    with Net(D, H, loss_mean=loss_mean) as net:
        net.set(W)
        g = [t.zeros((H, D), device="cuda"), t.zeros(H, device="cuda"), t.zeros(H, device="cuda"),
             t.zeros(1, device="cuda")]
        loss = t.zeros(1, dtype=t.float64, device="cuda")
        B.mlp_backward(net.h, dev(X), dev(y), n, *g, loss, stream())
        ref = oracle.mse_gradients(X, y, Params(*W), bool(loss_mean))
        # each block on its own (a wrong gb1 or gb2 cannot hide under gW1's
        # maximum): max-norm relative within the block, and every element
        # within 1e-4 of its own value above a floor of the block bar
        for name, a, r in zip(("gW1", "gb1", "gw2", "gb2"), g, ref[:4]):
            got, exp = host(a).astype(np.float64).ravel(), np.atleast_1d(np.asarray(r, np.float64)).ravel()
            scale = np.max(np.abs(exp))
            if scale == 0.0:
                assert np.max(np.abs(got)) <= 1e-12, name
                continue
            assert rel_err_norm(got, exp) <= GRAD_TOL, (name, rel_err_norm(got, exp))
            assert np.all(np.abs(got - exp) <= 1e-4 * np.abs(exp) + GRAD_TOL * scale), name
        assert float(host(loss)[0]) == pytest.approx(ref[4], rel=1e-5)


@pytest.mark.parametrize("n,D,H", [(96, 33, 16), (97, 33, 64), (1000, 7, 33), (4096, 33, 64), (513, 48, 40)])
def test_fused_train_100_epochs_matches_oracle(n, D, H):
    X, y, W = problem(300 + n, n, D, H)
    t = torch()
    epochs = 100
    with Net(D, H) as net:
        net.set(W)
        lh = t.zeros(epochs, dtype=t.float64, device="cuda")
        gh = t.zeros(epochs, dtype=t.float64, device="cuda")
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, epochs, 0, lh, gh, stream())
        assert net.check() == B.MLP_OK
        q, lh_ref, gh_ref = oracle.train(X, y, Params(*W), lr32(), epochs)
        assert rel_err_norm(net.flat(), q.flat()) <= W_TOL
        assert rel_err_elem(host(lh), lh_ref) <= 1e-5
        assert rel_err_elem(host(gh), gh_ref) <= 1e-4


def test_config0_1000_epochs():
    """33-16-1 on the 120-row synthetic cohort, first 96 rows train, 1000
    epochs, lr 0.1: weights and both accuracies agree with the oracle."""
    X = I.features(I.COHORT_SEED, 120)
    T = Params(*I.teacher_weights())
    y = oracle.predict(X, T).astype(np.float32)
    W = I.init_weights(I.INIT_SEED, 33, 16)
    t = torch()
    with Net(33, 16) as net:
        net.set(W)
        lh = t.zeros(1000, dtype=t.float64, device="cuda")
        B.mlp_train_epochs(net.h, dev(X[:96]), dev(y[:96]), 96, 1000, 0, lh, None, stream())
        lab = t.zeros(120, dtype=t.int8, device="cuda")
        B.mlp_predict(net.h, dev(X), 120, lab, stream())
        q, lh_ref, _ = oracle.train(X[:96], y[:96], Params(*W), lr32(), 1000)
        err = rel_err_norm(net.flat(), q.flat())
        assert err <= W_TOL, err
        assert rel_err_elem(host(lh), lh_ref) <= 1e-5
        lab_ref = oracle.predict(X, q)
        _, o_ref = oracle.forward(X, q)
        agree = (host(lab) == lab_ref) | (np.abs(o_ref - 0.5) < 1e-4)
        assert agree.all()


def test_plain_step_equals_one_epoch():
    n, D, H = 777, 33, 64
    X, y, W = problem(400, n, D, H)
    t = torch()
    with Net(D, H) as a, Net(D, H) as b:
        a.set(W)
        b.set(W)
        loss = t.zeros(1, dtype=t.float64, device="cuda")
        Xd, yd = dev(X), dev(y)
        B.mlp_step_plain(a.h, Xd, yd, n, loss, stream())
        B.mlp_train_epochs(b.h, Xd, yd, n, 1, 0, None, None, stream())
        q, lh_ref, _ = oracle.train(X, y, Params(*W), lr32(), 1)
        assert rel_err_norm(a.flat(), q.flat()) <= GRAD_TOL
        assert rel_err_norm(b.flat(), q.flat()) <= GRAD_TOL
        assert float(host(loss)[0]) == pytest.approx(lh_ref[0], rel=1e-6)


@pytest.mark.parametrize("mb", [1, 10, 64, 100, 1000])
def test_minibatch_matches_oracle(mb):
    n, D, H = 250, 33, 24
    X, y, W = problem(500, n, D, H)
    t = torch()
    with Net(D, H) as net:
        net.set(W)
        lh = t.zeros(5, dtype=t.float64, device="cuda")
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, 5, mb, lh, None, stream())
        q, lh_ref, _ = oracle.train(X, y, Params(*W), lr32(), 5, minibatch=mb)
        assert rel_err_norm(net.flat(), q.flat()) <= W_TOL
        assert rel_err_elem(host(lh), lh_ref) <= 1e-5


@pytest.mark.parametrize("H", [65, 130])
def test_plain_fallback_training_matches_oracle(H):
    n, D = 300, 33
    X, y, W = problem(600 + H, n, D, H)
    t = torch()
    with Net(D, H) as net:
        net.set(W)
        lh = t.zeros(20, dtype=t.float64, device="cuda")
        gh = t.zeros(20, dtype=t.float64, device="cuda")
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, 20, 64, lh, gh, stream())
        q, lh_ref, gh_ref = oracle.train(X, y, Params(*W), lr32(), 20, minibatch=64)
        assert rel_err_norm(net.flat(), q.flat()) <= W_TOL
        assert rel_err_elem(host(lh), lh_ref) <= 1e-5
        assert rel_err_elem(host(gh), gh_ref) <= 1e-4


def test_tanh_hidden_matches_oracle():
    n, D, H = 200, 33, 40
    X, y, W = problem(700, n, D, H)
    t = torch()
    with Net(D, H, act=B.MLP_ACT_TANH) as net:
        net.set(W)
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, 30, 0, None, None, stream())
        q, _, _ = oracle.train(X, y, Params(*W), lr32(), 30, act=oracle.ACT_TANH)
        assert rel_err_norm(net.flat(), q.flat()) <= W_TOL


def test_predict_matches_oracle_labels():
    n, D, H = 1001, 33, 16
    X, y, W = problem(800, n, D, H)
    t = torch()
    with Net(D, H) as net:
        net.set(W)
        lab = t.zeros(n, dtype=t.int8, device="cuda")
        B.mlp_predict(net.h, dev(X), n, lab, stream())
        lab_ref = oracle.predict(X, Params(*W))
        _, o_ref = oracle.forward(X, Params(*W))
        ok = (host(lab) == lab_ref) | (np.abs(o_ref - 0.5) < 1e-6)
        assert ok.all()
        zero = (np.zeros((H, D), np.float32), np.zeros(H, np.float32), np.zeros(H, np.float32),
                np.zeros(1, np.float32))
        net.set(zero)
        B.mlp_predict(net.h, dev(X), n, lab, stream())
        assert (host(lab) == 1).all()  # o = 1/2 exactly: ties go to class 1


def test_fp64_path_matches_oracle_tightly():
    n, D, H = 333, 33, 70
    X, y, W = problem(900, n, D, H)
    X = X.astype(np.float64)
    t = torch()
    with Net(D, H, prec=B.MLP_FP64) as net:
        net.set([a.astype(np.float64) for a in W])
        lh = t.zeros(10, dtype=t.float64, device="cuda")
        B.mlp_train_epochs(net.h, dev(X), dev(y.astype(np.float64)), n, 10, 0, lh, None, stream())
        q, lh_ref, _ = oracle.train(X, y, Params(*W), lr32(), 10)  # the handle stores lr as float
        assert rel_err_norm(net.flat(), q.flat()) <= 1e-12
        assert rel_err_elem(host(lh), lh_ref) <= 1e-12


def test_bf16_inputs_plain_path():
    n, D, Dp, H = 500, 33, 48, 64
    X = I.features(950, n, D, Dp)
    y = oracle.predict(X, Params(*I.teacher_weights(D=D, Dpad=Dp))).astype(np.float32)
    W = I.init_weights(951, D, H, Dp)
    Xb = I.bf16_round(X)
    t = torch()
    with Net(Dp, H, prec=B.MLP_BF16) as net:
        net.set(W)
        g = [t.zeros((H, Dp), device="cuda"), t.zeros(H, device="cuda"), t.zeros(H, device="cuda"),
             t.zeros(1, device="cuda")]
        B.mlp_backward(net.h, dev(I.bf16_bits(X)), dev(y), n, *g, None, stream())
        ref = oracle.mse_gradients(Xb, y, Params(*W))
        got = np.concatenate([host(a).ravel() for a in g])
        exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
        assert rel_err_norm(got, exp) <= GRAD_TOL
        assert np.all(host(g[0])[:, D:] == 0.0)


def test_empty_and_degenerate_inputs():
    t = torch()
    D, H = 33, 16
    W = I.init_weights(1, D, H)
    with Net(D, H) as net:
        net.set(W)
        before = net.flat()
        X = t.zeros((0, D), device="cuda")
        y = t.zeros(0, device="cuda")
        lh = t.full((3,), 7.0, dtype=t.float64, device="cuda")
        B.mlp_train_epochs(net.h, X, y, 0, 3, 0, lh, None, stream())
        assert np.array_equal(net.flat(), before)
        assert (host(lh) == 0).all()
        g = [t.ones((H, D), device="cuda"), t.ones(H, device="cuda"), t.ones(H, device="cuda"),
             t.ones(1, device="cuda")]
        B.mlp_backward(net.h, X, y, 0, *g, None, stream())
        assert all((host(a) == 0).all() for a in g)
        with pytest.raises(B.MLPError) as e:
            B.mlp_train_epochs(net.h, 0, 0, 5, 1, 0, None, None, stream())
        assert e.value.status == B.MLP_EINVAL


def test_fused_training_is_deterministic():
    n, D, H = 4096, 33, 64
    X, y, W = problem(1000, n, D, H)
    Xd, yd = dev(X), dev(y)
    res = []
    for _ in range(2):
        with Net(D, H) as net:
            net.set(W)
            B.mlp_train_epochs(net.h, Xd, yd, n, 50, 0, None, None, stream())
            res.append(net.flat())
    assert np.array_equal(res[0], res[1])


def test_host_buffer_entry_matches_device_entry():
    n, D, H = 4096, 33, 64
    X, y, W = problem(1100, n, D, H)
    t = torch()
    with Net(D, H) as a, Net(D, H) as b:
        a.set(W)
        b.set(W)
        lh = np.zeros(5)
        B.mlp_train_host(a.h, X, y, n, 5, 0, lh, stream())
        lhd = t.zeros(5, dtype=t.float64, device="cuda")
        B.mlp_train_epochs(b.h, dev(X), dev(y), n, 5, 0, lhd, None, stream())
        assert np.array_equal(a.flat(), b.flat())
        assert np.array_equal(lh, host(lhd))


def test_cross_block_wait_gives_up_with_status():
    """A block that never arrives makes the others give up after about a
    second; the launch records MLP_ETIMEOUT and the next run is normal."""
    import time
    n, D, H = 4096, 33, 64
    X, y, W = problem(1200, n, D, H)
    with Net(D, H) as net:
        net.set(W)
        B.mlp_debug_skip_block(net.h, 1)
        t0 = time.time()
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, 1, 0, None, None, stream())
        assert net.check() == B.MLP_ETIMEOUT
        assert time.time() - t0 < 30
        B.mlp_debug_skip_block(net.h, -1)
        net.set(W)
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, 1, 0, None, None, stream())
        assert net.check() == B.MLP_OK
        q, _, _ = oracle.train(X, y, Params(*W), lr32(), 1)
        assert rel_err_norm(net.flat(), q.flat()) <= GRAD_TOL


def test_nonfinite_loss_is_reported():
    n, D, H = 64, 4, 8
    X, y, W = problem(1300, n, D, H)
    X[3, 1] = np.nan
    with Net(D, H) as net:
        net.set(W)
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, 1, 0, None, None, stream())
        assert net.check() == B.MLP_ENONFINITE


def test_fp32_sigmoid_error_bound():
    """Eq. 1 in FP32 on the GPU (hidden activations of a 1-1 layer with unit
    weight) against the FP64 value: relative error <= 5e-7 over [-80, 80],
    exact limits at +-inf, NaN propagates."""
    from scipy.special import expit
    t = torch()
    x = np.concatenate([np.linspace(-80, 80, 400001), [0.0, -0.0, 1e-30, -1e-30, 1e-3, -1e-3, 103.9, -87.0]])
    x = x.astype(np.float32)
    n = x.size
    W1 = t.ones((1, 1), device="cuda")
    zero = t.zeros(1, device="cuda")
    hid = t.zeros((n, 1), device="cuda")
    o = t.zeros(n, device="cuda")
    nb = B.mlp_workspace_bytes(B.MLP_FP32, 1, 1, n)
    ws = t.empty(nb, dtype=t.uint8, device="cuda")
    B.mlp_forward_w(B.MLP_FP32, B.MLP_ACT_SIGMOID, 1, 1, n, dev(x.reshape(n, 1)), W1, zero, zero, zero, hid, o, ws,
                    nb, stream())
    got = host(hid)[:, 0].astype(np.float64)
    ref = expit(x.astype(np.float64))
    assert np.max(np.abs(got - ref) / ref) <= 5e-7
    assert np.all(host(o) == 0.5)
    special = np.array([np.inf, -np.inf, np.nan], np.float32).reshape(3, 1)
    h3 = t.zeros((3, 1), device="cuda")
    o3 = t.zeros(3, device="cuda")
    B.mlp_forward_w(B.MLP_FP32, B.MLP_ACT_SIGMOID, 1, 1, 3, dev(special), W1, zero, zero, zero, h3, o3, ws, nb,
                    stream())
    r = host(h3)[:, 0]
    assert r[0] == 1.0 and r[1] == 0.0 and np.isnan(r[2])


@pytest.mark.parametrize("n,D,H,mb", [(96, 33, 16, 0), (200, 33, 64, 0), (300, 7, 33, 100), (1, 1, 1, 0)])
def test_single_block_path_matches_oracle(n, D, H, mb):
    """A grid of one block (rows per block >= the rows of a step) sums and
    updates on chip: weights, loss and gradient-norm histories against the
    oracle, for full batch and mini-batches."""
    X, y, W = problem(1500 + n, n, D, H)
    t = torch()
    epochs = 50
    with Net(D, H) as net:
        net.set(W)
        B.mlp_set_rows_per_block(net.h, 512)
        lh = t.zeros(epochs, dtype=t.float64, device="cuda")
        gh = t.zeros(epochs, dtype=t.float64, device="cuda")
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, epochs, mb, lh, gh, stream())
        assert net.check() == B.MLP_OK, B.mlp_last_error()
        q, lh_ref, gh_ref = oracle.train(X, y, Params(*W), lr32(), epochs, minibatch=mb)
        assert rel_err_norm(net.flat(), q.flat()) <= W_TOL
        assert rel_err_elem(host(lh), lh_ref) <= 1e-5
        assert rel_err_elem(host(gh), gh_ref) <= 1e-4


def test_single_block_then_multi_block_on_one_handle():
    """The one-block path leaves the cross-block counters alone: a multi-block
    launch after it (and after it again) still meets its barriers, and the
    result is the oracle's for the whole schedule."""
    n, D, H = 700, 33, 64
    X, y, W = problem(1600, n, D, H)
    Xd, yd = dev(X), dev(y)
    with Net(D, H) as net:
        net.set(W)
        for rows in (1024, 32, 1024, 32):
            B.mlp_set_rows_per_block(net.h, rows)
            B.mlp_train_epochs(net.h, Xd, yd, n, 3, 0, None, None, stream())
            assert net.check() == B.MLP_OK, (rows, B.mlp_last_error())
        q, _, _ = oracle.train(X, y, Params(*W), lr32(), 12)
        assert rel_err_norm(net.flat(), q.flat()) <= W_TOL


def test_single_block_path_reports_nonfinite():
    n, D, H = 64, 4, 8
    X, y, W = problem(1700, n, D, H)
    X[5, 2] = np.nan
    with Net(D, H) as net:
        net.set(W)
        B.mlp_set_rows_per_block(net.h, 64)
        B.mlp_train_epochs(net.h, dev(X), dev(y), n, 1, 0, None, None, stream())
        assert net.check() == B.MLP_ENONFINITE


@pytest.mark.parametrize("mb", [0, 1000])
def test_host_entry_reads_page_locked_buffers_in_place(mb):
    """One-epoch calls on page-locked host buffers (read through the device's
    mapping, no staging copy) give the device entry's weights and losses bit
    for bit; pageable buffers take the staging copy and agree as well."""
    n, D, H = 4096, 33, 64
    X, y, W = problem(1800 + mb, n, D, H)
    t = torch()
    Xp = t.from_numpy(X).pin_memory()
    yp = t.from_numpy(y).pin_memory()
    lp = t.zeros(1, dtype=t.float64).pin_memory()
    with Net(D, H) as a, Net(D, H) as b, Net(D, H) as c:
        for net in (a, b, c):
            net.set(W)
        lhd = t.zeros(1, dtype=t.float64, device="cuda")
        lpg = np.zeros(1)
        for _ in range(3):
            B.mlp_train_host(a.h, Xp, yp, n, 1, mb, lp, stream())
            B.mlp_train_epochs(b.h, dev(X), dev(y), n, 1, mb, lhd, None, stream())
            B.mlp_train_host(c.h, X, y, n, 1, mb, lpg, stream())
            assert float(lp[0]) == float(host(lhd)[0]) == float(lpg[0])
        assert a.check() == B.MLP_OK
        assert np.array_equal(a.flat(), b.flat()) and np.array_equal(c.flat(), b.flat())


@pytest.mark.parametrize("prec,D,H", [(B.MLP_FP32, 33, 64), (B.MLP_FP64, 33, 16), (B.MLP_BF16, 48, 512)])
def test_empty_inputs_and_zero_epochs(prec, D, H):
    """n = 0 trains nothing and reports zero losses; epochs = 0 touches
    nothing; forward and predict of no rows succeed; negative sizes are
    rejected.  Every path: fused FP32, plain FP64, tensor-core bf16."""
    t = torch()
    _, _, W = problem(1900 + prec, 8, D, H)
    with Net(D, H, prec=prec) as net:
        net.set(W)
        before = net.flat()
        lh = t.full((4,), 7.0, dtype=t.float64, device="cuda")
        dummy = t.zeros(16, device="cuda")
        B.mlp_train_epochs(net.h, dummy, dummy, 0, 4, 0, lh, None, stream())
        assert net.check() == B.MLP_OK
        assert np.all(host(lh) == 0.0)
        lh.fill_(7.0)
        B.mlp_train_epochs(net.h, dummy, dummy, 5, 0, 0, lh, None, stream())
        assert np.all(host(lh) == 7.0)
        assert np.array_equal(net.flat(), before)
        o = t.zeros(1, device="cuda")
        B.mlp_forward(net.h, dummy, 0, o, stream())
        lab = t.zeros(1, dtype=t.int8, device="cuda")
        B.mlp_predict(net.h, dummy, 0, lab, stream())
        lhh = np.full(2, 7.0)
        B.mlp_train_host(net.h, np.zeros(1, np.float32), np.zeros(1, np.float32), 0, 2, 0, lhh, stream())
        assert np.all(lhh == 0.0)
        assert np.array_equal(net.flat(), before)
        with pytest.raises(B.MLPError) as e:
            B.mlp_train_epochs(net.h, dummy, dummy, -1, 1, 0, None, None, stream())
        assert e.value.status == B.MLP_EINVAL


def test_train_path_names_the_kernel_a_shape_takes():
    """The path query tells the fast kernels from the plain fallback."""
    cases = [((33, 64, B.MLP_FP32), B.MLP_PATH_FUSED), ((64, 128, B.MLP_FP32), B.MLP_PATH_FUSED),
             ((65, 64, B.MLP_FP32), B.MLP_PATH_PLAIN), ((33, 129, B.MLP_FP32), B.MLP_PATH_PLAIN),
             ((48, 2048, B.MLP_BF16), B.MLP_PATH_TC_CLUSTER), ((48, 300, B.MLP_BF16), B.MLP_PATH_PLAIN),
             ((33, 64, B.MLP_FP64), B.MLP_PATH_PLAIN)]
    for (D, H, prec), want in cases:
        with Net(D, H, prec=prec) as net:
            assert B.mlp_train_path(net.h, 1000, 0) == want, (D, H, prec)
