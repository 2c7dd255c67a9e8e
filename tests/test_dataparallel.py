"""One network trained data-parallel across ranks (host logic, CPU): the shard
and mini-batch splits, and two gloo ranks that each compute their shard's
summed gradient with the FP64 oracle, all-gather them, add them in rank order,
scale by 1/m and update, end with the single-process oracle's mini-batch
training (within FP64 rounding) and with bit-identical replicas."""
import os
import socket

import numpy as np
import pytest

from paper_1908_07847_gb300 import dataparallel as dp


def test_shard_rows_cover_each_batch_once():
    for m in (0, 1, 2, 7, 255, 256, 8192):
        for world in (1, 2, 3, 8):
            spans = [dp.shard_rows(m, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == m
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        dp.shard_rows(10, 2, 2)


def test_batches_are_contiguous_slices_in_order():
    assert list(dp.batches(769, 256)) == [(0, 256), (256, 256), (512, 256), (768, 1)]
    assert list(dp.batches(100, 0)) == [(0, 100)]
    assert list(dp.batches(100, 500)) == [(0, 100)]
    assert list(dp.batches(0, 8)) == []


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


N, D, H, MB, EPOCHS, LR = 769, 7, 9, 256, 3, 0.25


def _problem():
    import oracle
    from paper_1908_07847_gb300 import inputs as I
    X = I.features(I.subseed(91, 1), N, D)
    y = oracle.predict(X, oracle.Params(*I.teacher_weights(D=D, H=3))).astype(np.float64)
    return X, y, oracle.Params(*I.init_weights(92, D, H))


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X, y, p = _problem()
    hist = []
    for _ in range(EPOCHS):
        sse = 0.0
        for start, m in dp.batches(N, MB):
            lo, hi = dp.shard_rows(m, world, rank)
            if hi > lo:
                g = oracle.mse_gradients(X[start + lo:start + hi], y[start + lo:start + hi], p, loss_mean=False)
                flat = np.concatenate([g[0].ravel(), g[1], g[2], [g[3]], [g[4]]])
            else:
                flat = np.zeros(D * H + 2 * H + 2)
            parts = [torch.empty(flat.size, dtype=torch.float64) for _ in range(world)]
            dist.all_gather(parts, torch.from_numpy(flat))
            s = parts[0].numpy().copy()
            for t in parts[1:]:
                s += t.numpy()                          # rank order
            sse += s[-1]
            gs = s[:-1] / m                             # mean loss over the batch
            HD = D * H
            p = oracle.update(p, (gs[:HD].reshape(H, D), gs[HD:HD + H], gs[HD + H:HD + 2 * H], gs[-1]), LR)
        hist.append(sse / N)
    q.put((rank, p.flat(), np.array(hist)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process_minibatch_training():
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict((r, (w, h)) for r, w, h in (q.get(timeout=300) for _ in range(2)))
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][1], got[1][1])
    X, y, p0 = _problem()
    q1, lh, _ = oracle.train(X, y, p0, LR, EPOCHS, minibatch=MB)
    assert np.max(np.abs(got[0][0] - q1.flat())) <= 1e-12 * np.max(np.abs(q1.flat()))
    assert np.allclose(got[0][1], lh, rtol=1e-12, atol=0)
