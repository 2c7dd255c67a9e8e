"""Autotuner of the fused kernel's tile shape, and the accuracy-vs-epochs
protocol of Sec. 3 (Figs. 3 and 4) on the synthetic sex-split cohort."""
import os

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_1908_07847_gb300 import binding as B
from paper_1908_07847_gb300 import inputs as I
from tests.gpu_util import W_TOL, Net, dev, lr32, problem, rel_err_norm, stream

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_training_stays_exact(tmp_path, monkeypatch):
    from paper_1908_07847_gb300 import autotune
    monkeypatch.setenv("MLP_GB300_TUNE_CACHE", str(tmp_path / "tune.json"))
    n, D, H = 4096, 33, 64
    X, y, W = problem(77, n, D, H)
    Xd, yd = dev(X), dev(y)
    rows, times = autotune.tune_fused(Xd, yd, D, H, n, candidates=(16, 32, 64), reps=5)
    assert rows in (16, 32, 64) and set(times) == {16, 32, 64}
    assert os.path.exists(tmp_path / "tune.json")
    again, _ = autotune.tune_fused(Xd, yd, D, H, n, candidates=(16, 32, 64), reps=5)
    assert again == rows  # served from the cache
    with Net(D, H) as net:
        net.set(W)
        assert autotune.configure(net.h, Xd, yd, D, H, n) == rows
        B.mlp_train_epochs(net.h, Xd, yd, n, 10, 0, None, None, stream())
        q, _, _ = oracle.train(X, y, Params(*W), lr32(), 10)
        assert rel_err_norm(net.flat(), q.flat()) <= W_TOL


def test_accuracy_curve_matches_oracle_protocol():
    from paper_1908_07847_gb300 import curves
    cps = (10, 100, 1000)
    got = curves.accuracy_curve(hidden=16, checkpoints=cps)
    X = I.features(I.COHORT_SEED, I.N_PARTICIPANTS)
    labels = oracle.predict(X, Params(*I.teacher_weights())).astype(np.float32)
    for k, (name, Xs, ys, ntr) in enumerate(curves.subsets(labels)):
        assert ntr == {"male": 46, "female": 44}[name]
        p = Params(*I.init_weights(I.INIT_SEED + k, 33, 16))
        done = 0
        for (cp, tr, te) in got[name]:
            p, _, _ = oracle.train(Xs[:ntr], ys[:ntr], p, lr32(), cp - done)
            done = cp
            pred = oracle.predict(Xs, p)
            assert abs(tr - (pred[:ntr] == ys[:ntr]).mean()) <= 1.0 / ntr + 1e-12, (name, cp)
            assert abs(te - (pred[ntr:] == ys[ntr:]).mean()) <= 1.0 / (len(ys) - ntr) + 1e-12, (name, cp)
