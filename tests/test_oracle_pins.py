"""Pins for the FP64 oracle against facts that do not come from the oracle itself.

The paper (arXiv 1908.07847) prints no worked example, so the oracle is pinned by
closed forms derived by hand, an independent symbolic differentiation (sympy),
central finite differences, an independent automatic differentiation (torch on
CPU, float64), textbook library routines, invariants of the method, and the
split arithmetic implied by the accuracies the paper prints (Abstract, Sec. 1).
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_1908_07847_gb300 import inputs as I

LN3 = math.log(3.0)
HERE = os.path.dirname(os.path.abspath(__file__))


def rand_params(rng, D, H, scale=0.5):
    return Params(rng.normal(0, scale, (H, D)), rng.normal(0, scale, H),
                  rng.normal(0, scale, H), rng.normal(0, scale))


def loss_only(X, y, p, loss_mean=True, act=oracle.ACT_SIGMOID):
    _, o = oracle.forward(X, p, act)
    c = 1.0 / len(y) if loss_mean else 1.0
    return 0.5 * c * float(np.sum((o - y) ** 2))


# --------------------------------------------------------------- Eq. 1 ------

def test_sigmoid_closed_values():
    """Eq. 1 at points with exact values: sigma(0) = 1/2, sigma(ln 3) = 3/4."""
    assert oracle.sigmoid(0.0) == 0.5
    assert abs(oracle.sigmoid(LN3) - 0.75) < 1e-16
    assert abs(oracle.sigmoid(-LN3) - 0.25) < 1e-16
    assert oracle.sigmoid(800.0) == 1.0
    assert oracle.sigmoid(-800.0) == 0.0


def test_sigmoid_matches_scipy_expit():
    from scipy.special import expit
    xs = np.linspace(-40, 40, 1001)
    for x in xs:
        s = oracle.sigmoid(x)
        assert abs(s - expit(x)) <= 4e-16 * max(1.0, abs(expit(x)))
        assert abs(s + oracle.sigmoid(-x) - 1.0) < 1e-15


# ----------------------------------------------- closed-form gradients ------

@pytest.mark.parametrize("loss_mean", [True, False])
def test_zero_weights_221_closed_form(loss_mean):
    """All weights 0: h = o = 1/2, d2 = c (1/2 - y) / 4, gw2 = gb2 / 2,
    hidden deltas vanish (w2 = 0) so gW1 = gb1 = 0."""
    X = np.array([[0.3, -1.2], [2.0, 0.5], [-0.7, 0.1]])
    y = np.array([1.0, 0.0, 1.0])
    p = Params(np.zeros((2, 2)), np.zeros(2), np.zeros(2), 0.0)
    c = 1.0 / 3 if loss_mean else 1.0
    gW1, gb1, gw2, gb2, loss = oracle.mse_gradients(X, y, p, loss_mean)
    exp_gb2 = c * sum((0.5 - yi) / 4.0 for yi in y)
    assert gb2 == pytest.approx(exp_gb2, abs=1e-16)
    np.testing.assert_allclose(gw2, [exp_gb2 / 2] * 2, atol=1e-16)
    assert np.all(gW1 == 0.0) and np.all(gb1 == 0.0)
    assert loss == pytest.approx(0.5 * c * sum((0.5 - yi) ** 2 for yi in y), abs=1e-16)
    hid, o = oracle.forward(X, p)
    assert np.all(hid == 0.5) and np.all(o == 0.5)


def ln3_case():
    """Hand-built 3-2-1 net whose activations are exact fractions.

    x = (1, 2, -1).  Row 0 of W1 = (ln3/3, 0, 0), b1_0 = 2 ln3/3  ->  z = ln 3,
    h_0 = 3/4.  Row 1 = (1, 1, 3), b1_1 = 0  ->  z = 0, h_1 = 1/2.
    w2 = (ln 3, ln3/2), b2 = 0  ->  z2 = 3 ln3/4 + ln3/4 = ln 3, o = 3/4.
    """
    X = np.array([[1.0, 2.0, -1.0]])
    W1 = np.array([[LN3 / 3, 0.0, 0.0], [1.0, 1.0, 3.0]])
    b1 = np.array([2 * LN3 / 3, 0.0])
    w2 = np.array([LN3, LN3 / 2])
    return X, Params(W1, b1, w2, 0.0)


def test_ln3_forward_exact():
    X, p = ln3_case()
    hid, o = oracle.forward(X, p)
    np.testing.assert_allclose(hid[0], [0.75, 0.5], atol=1e-15)
    assert o[0] == pytest.approx(0.75, abs=1e-15)


def test_ln3_gradients_closed_form():
    """y = 1, n = 1: dE/do = -1/4, d2 = -1/4 * 3/4 * 1/4 = -3/64.
    gw2 = d2 h = (-9/256, -3/128);  d1_0 = d2 ln3 (3/16) = -9 ln3/1024,
    d1_1 = d2 (ln3/2)(1/4) = -6 ln3/1024;  gW1_j = d1_j x;  gX = sum_j d1_j W1_j."""
    X, p = ln3_case()
    y = np.array([1.0])
    gW1, gb1, gw2, gb2, loss = oracle.mse_gradients(X, y, p, loss_mean=True)
    d2 = -3.0 / 64
    d1 = np.array([-9 * LN3 / 1024, -6 * LN3 / 1024])
    assert gb2 == pytest.approx(d2, abs=1e-16)
    np.testing.assert_allclose(gw2, [-9.0 / 256, -3.0 / 128], atol=1e-16)
    np.testing.assert_allclose(gb1, d1, atol=1e-16)
    np.testing.assert_allclose(gW1, np.outer(d1, X[0]), atol=1e-16)
    assert loss == pytest.approx(0.5 * (0.25 ** 2), abs=1e-17)
    # Upstream-gradient form with the same dL/do gives the same values plus gX.
    g = oracle.backward(X, p, np.array([-0.25]), want_gX=True)
    np.testing.assert_allclose(g[0], gW1, atol=1e-16)
    np.testing.assert_allclose(g[4][0], d1[0] * p.W1[0] + d1[1] * p.W1[1], atol=1e-16)


def test_gradients_match_sympy_symbolic():
    """Symbolic differentiation of the loss written from Sec. 2.2 / Eq. 1."""
    sp = pytest.importorskip("sympy")
    rng = np.random.default_rng(3)
    D, H, n = 3, 2, 4
    Xv = rng.integers(-3, 4, (n, D)) / 2.0
    yv = np.array([1.0, 0.0, 0.0, 1.0])
    Wv = rng.integers(-4, 5, (H, D)) / 4.0
    b1v = rng.integers(-2, 3, H) / 4.0
    w2v = rng.integers(-4, 5, H) / 3.0
    b2v = 0.25
    W = sp.Matrix(H, D, lambda j, k: sp.Symbol(f"W{j}{k}"))
    b1 = [sp.Symbol(f"b{j}") for j in range(H)]
    w2 = [sp.Symbol(f"v{j}") for j in range(H)]
    b2 = sp.Symbol("c")
    sig = lambda t: 1 / (1 + sp.exp(-t))
    E = 0
    for i in range(n):
        hs = [sig(sum(sp.Rational(Xv[i, k]).limit_denominator() * W[j, k] for k in range(D)) + b1[j])
              for j in range(H)]
        o = sig(sum(hs[j] * w2[j] for j in range(H)) + b2)
        E += (o - sp.Rational(yv[i]).limit_denominator()) ** 2
    E = E / (2 * n)
    subs = {W[j, k]: sp.Rational(Wv[j, k]).limit_denominator() for j in range(H) for k in range(D)}
    subs.update({b1[j]: sp.Rational(b1v[j]).limit_denominator() for j in range(H)})
    subs.update({w2[j]: sp.Rational(w2v[j]).limit_denominator() for j in range(H)})
    subs[b2] = sp.Rational(1, 4)
    p = Params(Wv, b1v, w2v, b2v)
    gW1, gb1, gw2, gb2, loss = oracle.mse_gradients(Xv, yv, p, loss_mean=True)
    assert float(E.subs(subs).evalf(30)) == pytest.approx(loss, rel=1e-13)
    for j in range(H):
        for k in range(D):
            ref = float(sp.diff(E, W[j, k]).subs(subs).evalf(30))
            assert gW1[j, k] == pytest.approx(ref, rel=1e-12, abs=1e-15)
        assert gb1[j] == pytest.approx(float(sp.diff(E, b1[j]).subs(subs).evalf(30)), rel=1e-12, abs=1e-15)
        assert gw2[j] == pytest.approx(float(sp.diff(E, w2[j]).subs(subs).evalf(30)), rel=1e-12, abs=1e-15)
    assert gb2 == pytest.approx(float(sp.diff(E, b2).subs(subs).evalf(30)), rel=1e-12, abs=1e-15)


# ------------------------------------------------ finite differences --------

def fd_grad(X, y, p, loss_mean, act, h=1e-6):
    flat = p.flat()
    D, H = p.D, p.H
    g = np.zeros_like(flat)
    for t in range(flat.size):
        for s, sgn in ((h, 1), (-h, -1)):
            q = flat.copy()
            q[t] += s
            pp = Params(q[:H * D].reshape(H, D), q[H * D:H * D + H], q[H * D + H:H * D + 2 * H], q[-1])
            g[t] += sgn * loss_only(X, y, pp, loss_mean, act)
        g[t] /= 2 * h
    return g


@pytest.mark.parametrize("seed,loss_mean,act", [(0, True, 0), (1, False, 0), (2, True, 1), (3, False, 1)])
def test_gradients_match_central_fd(seed, loss_mean, act):
    """Central differences, h = 1e-6, FP64, random 5-7-1 nets."""
    rng = np.random.default_rng(seed)
    D, H, n = 5, 7, 11
    X = rng.normal(size=(n, D))
    y = (rng.random(n) < 0.5).astype(np.float64)
    p = rand_params(rng, D, H)
    gW1, gb1, gw2, gb2, _ = oracle.mse_gradients(X, y, p, loss_mean, act)
    g = np.concatenate([gW1.ravel(), gb1, gw2, [gb2]])
    gfd = fd_grad(X, y, p, loss_mean, act)
    assert np.max(np.abs(g - gfd)) / np.max(np.abs(gfd)) < 1e-7


def test_backward_upstream_matches_torch_autograd():
    """Independent automatic differentiation (torch, CPU, float64) of an
    arbitrary weighted sum of outputs, including the input gradient."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    D, H, n = 6, 9, 13
    X = rng.normal(size=(n, D))
    p = rand_params(rng, D, H)
    u = rng.normal(size=n)
    tX = torch.tensor(X, requires_grad=True)
    tW1 = torch.tensor(p.W1, requires_grad=True)
    tb1 = torch.tensor(p.b1, requires_grad=True)
    tw2 = torch.tensor(p.w2, requires_grad=True)
    tb2 = torch.tensor(p.b2, dtype=torch.float64, requires_grad=True)
    o = torch.sigmoid(torch.sigmoid(tX @ tW1.T + tb1) @ tw2 + tb2)
    (o * torch.tensor(u)).sum().backward()
    gW1, gb1, gw2, gb2, gX = oracle.backward(X, p, u, want_gX=True)
    np.testing.assert_allclose(gW1, tW1.grad.numpy(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gb1, tb1.grad.numpy(), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gw2, tw2.grad.numpy(), rtol=1e-12, atol=1e-14)
    assert gb2 == pytest.approx(float(tb2.grad), rel=1e-12, abs=1e-14)
    np.testing.assert_allclose(gX, tX.grad.numpy(), rtol=1e-12, atol=1e-14)
    _, o_orc = oracle.forward(X, p)
    np.testing.assert_allclose(o_orc, o.detach().numpy(), rtol=1e-14)


# ------------------------------------------------------- update / train -----

def test_update_is_plain_gd_step():
    """Sec. 2.2: lr 0.1, no momentum: w_new = w - 0.1 g, param by param."""
    rng = np.random.default_rng(7)
    p = rand_params(rng, 4, 3)
    g = (rng.normal(size=(3, 4)), rng.normal(size=3), rng.normal(size=3), 0.37)
    q = oracle.update(p, g, 0.1)
    np.testing.assert_allclose(q.W1, p.W1 - 0.1 * g[0], rtol=0, atol=1e-16)
    np.testing.assert_allclose(q.b1, p.b1 - 0.1 * g[1], rtol=0, atol=1e-16)
    np.testing.assert_allclose(q.w2, p.w2 - 0.1 * g[2], rtol=0, atol=1e-16)
    assert q.b2 == pytest.approx(p.b2 - 0.037, abs=1e-16)


def test_one_epoch_equals_fd_gradient_step():
    rng = np.random.default_rng(8)
    D, H, n = 4, 5, 9
    X = rng.normal(size=(n, D))
    y = (rng.random(n) < 0.5).astype(float)
    p = rand_params(rng, D, H)
    q, lh, gh = oracle.train(X, y, p, lr=0.1, epochs=1)
    gfd = fd_grad(X, y, p, True, 0)
    np.testing.assert_allclose(q.flat(), p.flat() - 0.1 * gfd, rtol=0, atol=1e-9)
    assert lh[0] == pytest.approx(loss_only(X, y, p), rel=1e-15)
    assert gh[0] == pytest.approx(np.linalg.norm(gfd), rel=1e-7)


def test_loss_history_is_loss_before_each_update():
    rng = np.random.default_rng(9)
    X = rng.normal(size=(20, 6))
    y = (rng.random(20) < 0.5).astype(float)
    p = rand_params(rng, 6, 4)
    _, lh, _ = oracle.train(X, y, p, 0.1, 6)
    for e in range(6):
        q, _, _ = oracle.train(X, y, p, 0.1, e)
        assert lh[e] == pytest.approx(loss_only(X, y, q), rel=1e-14)


def test_descent_monotone_small_lr():
    X = I.features(11, 64, 8)
    rng = np.random.default_rng(10)
    y = (rng.random(64) < 0.4).astype(float)
    p = Params(*I.init_weights(3, 8, 6))
    _, lh, _ = oracle.train(X, y, p, lr=1e-3, epochs=200)
    assert np.all(np.diff(lh) <= 0.0)
    assert lh[-1] < lh[0]


def test_minibatch_is_sequence_of_full_batch_steps():
    """A mini-batch epoch equals full-batch steps on the contiguous slices in
    order, including a ragged last slice; m = n equals full batch."""
    rng = np.random.default_rng(12)
    X = rng.normal(size=(23, 5))
    y = (rng.random(23) < 0.5).astype(float)
    p = rand_params(rng, 5, 3)
    q, lh, _ = oracle.train(X, y, p, 0.1, 2, minibatch=10)
    r = p.copy()
    sse = 0.0
    for _ in range(2):
        sse = 0.0
        for s in range(0, 23, 10):
            r2, l2, _ = oracle.train(X[s:s + 10], y[s:s + 10], r, 0.1, 1)
            sse += 2 * l2[0] * len(y[s:s + 10])
            r = r2
    np.testing.assert_array_equal(q.flat(), r.flat())
    assert lh[1] == pytest.approx(0.5 * sse / 23, rel=1e-14)
    qa, la, _ = oracle.train(X, y, p, 0.1, 3, minibatch=23)
    qb, lb, _ = oracle.train(X, y, p, 0.1, 3, minibatch=0)
    np.testing.assert_array_equal(qa.flat(), qb.flat())
    np.testing.assert_array_equal(la, lb)


def test_online_step_equals_single_sample_full_batch():
    rng = np.random.default_rng(13)
    X = rng.normal(size=(5, 4))
    y = np.array([1.0, 0, 1, 1, 0])
    p = rand_params(rng, 4, 3)
    q, _, _ = oracle.train(X, y, p, 0.1, 1, minibatch=1)
    r = p.copy()
    for i in range(5):
        g = oracle.mse_gradients(X[i:i + 1], y[i:i + 1], r)
        r = oracle.update(r, g, 0.1)
    np.testing.assert_array_equal(q.flat(), r.flat())


# ------------------------------------------------------------ invariants ----

def test_hidden_permutation_equivariance():
    rng = np.random.default_rng(14)
    D, H, n = 5, 6, 17
    X = rng.normal(size=(n, D))
    y = (rng.random(n) < 0.5).astype(float)
    p = rand_params(rng, D, H)
    perm = rng.permutation(H)
    pp = Params(p.W1[perm], p.b1[perm], p.w2[perm], p.b2)
    g = oracle.mse_gradients(X, y, p)
    gp = oracle.mse_gradients(X, y, pp)
    np.testing.assert_allclose(gp[0], g[0][perm], rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(gp[1], g[1][perm], rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(gp[2], g[2][perm], rtol=1e-13, atol=1e-16)
    assert gp[3] == pytest.approx(g[3], rel=1e-13)


def test_identical_hidden_units_stay_identical():
    rng = np.random.default_rng(15)
    D, H, n = 4, 5, 12
    X = rng.normal(size=(n, D))
    y = (rng.random(n) < 0.5).astype(float)
    p = rand_params(rng, D, H)
    p.W1[3] = p.W1[1]
    p.b1[3] = p.b1[1]
    p.w2[3] = p.w2[1]
    q, _, _ = oracle.train(X, y, p, 0.1, 25)
    np.testing.assert_array_equal(q.W1[3], q.W1[1])
    assert q.b1[3] == q.b1[1] and q.w2[3] == q.w2[1]
    assert not np.array_equal(q.W1[1], p.W1[1])


def test_zero_padding_leaves_gradients_unchanged():
    """33 markers padded to 48 with zero columns and zero weights: the padded
    gradient columns are exactly 0 and everything else is bit-identical."""
    X = I.features(21, 30, 33).astype(np.float64)
    Xp = I.features(21, 30, 33, 48).astype(np.float64)
    rng = np.random.default_rng(16)
    y = (rng.random(30) < 0.5).astype(float)
    W1, b1, w2, b2 = I.init_weights(5, 33, 7)
    W1p, _, _, _ = I.init_weights(5, 33, 7, 48)
    g = oracle.mse_gradients(X, y, Params(W1, b1, w2, b2))
    gp = oracle.mse_gradients(Xp, y, Params(W1p, b1, w2, b2))
    assert np.all(gp[0][:, 33:] == 0.0)
    np.testing.assert_array_equal(gp[0][:, :33], g[0])
    np.testing.assert_array_equal(gp[2], g[2])
    assert gp[4] == g[4]


def test_full_batch_gradient_invariant_to_sample_order():
    rng = np.random.default_rng(17)
    X = rng.normal(size=(40, 5))
    y = (rng.random(40) < 0.5).astype(float)
    p = rand_params(rng, 5, 4)
    perm = rng.permutation(40)
    g = oracle.mse_gradients(X, y, p)
    gp = oracle.mse_gradients(X[perm], y[perm], p)
    for a, b in zip(g, gp):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)


def test_empty_input():
    p = rand_params(np.random.default_rng(18), 3, 2)
    X = np.zeros((0, 3))
    g = oracle.mse_gradients(X, np.zeros(0), p)
    assert np.all(g[0] == 0) and g[3] == 0.0 and g[4] == 0.0
    q, lh, _ = oracle.train(X, np.zeros(0), p, 0.1, 3)
    np.testing.assert_array_equal(q.flat(), p.flat())
    assert oracle.predict(X, p).shape == (0,)


# --------------------------------------------------------------- predict ----

def test_predict_threshold_and_tie():
    """Class 1 iff o >= 0.5; an all-zero net gives o = 1/2 exactly -> 1."""
    X = np.random.default_rng(19).normal(size=(7, 3))
    zero = Params(np.zeros((2, 3)), np.zeros(2), np.zeros(2), 0.0)
    assert np.all(oracle.predict(X, zero) == 1)
    neg = Params(np.zeros((2, 3)), np.zeros(2), np.zeros(2), -1e-9)
    assert np.all(oracle.predict(X, neg) == 0)
    p = rand_params(np.random.default_rng(20), 3, 4)
    _, o = oracle.forward(X, p)
    np.testing.assert_array_equal(oracle.predict(X, p), (o >= 0.5).astype(np.int8))


def test_teacher_recovery_sanity():
    """A 33-16-1 student learns the 33-8-1 teacher's labels on the synthetic
    cohort (sanity, not parity)."""
    X = I.features(I.COHORT_SEED, 120)
    y = oracle.predict(X, Params(*I.teacher_weights())).astype(float)
    p = Params(*I.init_weights(1, 33, 16))
    q, lh, _ = oracle.train(X[:96], y[:96], p, lr=1.0, epochs=2000)
    assert (oracle.predict(X[:96], q) == y[:96]).mean() >= 0.95
    assert lh[-1] < 0.1 * lh[0]


# -------------------------------------------------------- batch of nets -----

def test_batch_train_equals_independent_runs():
    rng = np.random.default_rng(21)
    nets = []
    for t in range(5):
        D, H, n = 4 + t % 2, 2 + t, 6 + 3 * t
        X = rng.normal(size=(n, D))
        y = (rng.random(n) < 0.5).astype(float)
        nets.append((X, y, rand_params(rng, D, H)))
    out, loss = oracle.batch_train(nets, 0.1, 7, threads=2)
    for t, (X, y, p) in enumerate(nets):
        q, lh, _ = oracle.train(X, y, p, 0.1, 7)
        np.testing.assert_array_equal(out[t].flat(), q.flat())
        np.testing.assert_array_equal(loss[t], lh)


# ---------------------------------------------------- paper's split rule ----

def test_split_rule_reproduces_paper_accuracies():
    """The Abstract's accuracies are k / n_train and k / n_test with
    n_train = round(0.75 n) (Sec. 1: 75 % / 25 %) on 61 male and 59 female
    participants (Sec. 1): 44/46, 13/15, 43/44, 10/15."""
    rows = []
    with open(os.path.join(HERE, "golden", "paper_split_accuracy.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, n, tr, te = line.split()
                rows.append((name, int(n), float(tr), float(te)))
    assert sum(r[1] for r in rows) == I.N_PARTICIPANTS
    for name, n, tr, te in rows:
        ntr = I.split_count(n)
        nte = n - ntr
        assert any(round(100.0 * k / ntr, 2) == tr for k in range(ntr + 1)), name
        assert any(round(100.0 * k / nte, 2) == te for k in range(nte + 1)), name
    assert (I.split_count(61), I.split_count(59)) == (46, 44)


# ------------------------------------------------- z-score normalisation ----

def _zdata(seed=11, n=400, D=7):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, D)) * rng.uniform(0.5, 4.0, D) + rng.uniform(-10, 10, D)
    X[:, 3] = 2.5   # a constant column
    return X


def test_zscore_statistics_match_numpy_population_moments():
    """Mean and population deviation (ddof 0) of the fit rows, as numpy
    computes them; the test rows use the fit rows' statistics."""
    X = _zdata()
    n_fit = 300
    Y, m, s = oracle.zscore(X, n_fit)
    np.testing.assert_allclose(m, X[:n_fit].mean(axis=0), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(s, X[:n_fit].std(axis=0, ddof=0), rtol=1e-12, atol=1e-15)
    ok = s > 0
    np.testing.assert_allclose(Y[:, ok], (X[:, ok] - m[ok]) / s[ok], rtol=1e-12, atol=1e-12)


def test_zscore_fit_rows_have_zero_mean_unit_deviation():
    X = _zdata(12)
    Y, m, s = oracle.zscore(X, 250)
    ok = s > 0
    np.testing.assert_allclose(Y[:250, ok].mean(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.sqrt((Y[:250, ok] ** 2).mean(axis=0)), 1.0, rtol=1e-12)


def test_zscore_affine_invariance_constant_column_and_test_rows():
    """Scaling a column by a > 0 and shifting it leaves the output unchanged; a
    constant column maps to 0; changing test rows changes no statistic."""
    X = _zdata(13)
    Y, m, s = oracle.zscore(X, 200)
    X2 = X * 3.0 + 7.0
    Y2, _, _ = oracle.zscore(X2, 200)
    np.testing.assert_allclose(Y2, Y, rtol=1e-9, atol=1e-9)
    assert s[3] == 0.0 and np.all(Y[:, 3] == 0.0)
    X3 = X.copy()
    X3[200:] = 1e6
    _, m3, s3 = oracle.zscore(X3, 200)
    np.testing.assert_array_equal(m3, m)
    np.testing.assert_array_equal(s3, s)
    Y1, m1, s1 = oracle.zscore(X[:5], 1)     # one fit row: no spread anywhere
    assert np.all(s1 == 0.0) and np.all(Y1 == 0.0)
