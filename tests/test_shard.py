"""The many-nets workload split across ranks (host logic, CPU): the
longest-processing-time partition, and two gloo ranks that each train their
share with the FP64 oracle and gather to rank 0 reproduce the single-rank run
bit for bit."""
import os
import socket

import numpy as np
import pytest

from paper_1908_07847_gb300 import shard


def test_partition_covers_every_net_once_and_balances():
    rng = np.random.default_rng(3)
    costs = rng.integers(4, 129, 1000) * rng.integers(50, 121, 1000)
    for world in (1, 2, 3, 8):
        parts = shard.partition_lpt(costs, world)
        allv = np.sort(np.concatenate(parts))
        assert np.array_equal(allv, np.arange(1000))
        for p in parts:
            assert np.all(np.diff(p) > 0)            # increasing net order
        loads = [costs[p].sum() for p in parts]
        # LPT: no rank exceeds the mean by more than the largest single net
        assert max(loads) - np.mean(loads) <= costs.max()
        # every rank computes the same assignment
        assert all(np.array_equal(a, b) for a, b in zip(parts, shard.partition_lpt(costs, world)))


def test_partition_ties_and_small_cases():
    assert [list(p) for p in shard.partition_lpt([5, 5, 5, 5], 2)] == [[0, 2], [1, 3]]
    assert [list(p) for p in shard.partition_lpt([1], 3)] == [[0], [], []]
    with pytest.raises(ValueError):
        shard.partition_lpt([1, 2], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _nets():
    import oracle
    from paper_1908_07847_gb300 import inputs as I
    Hs, ns = I.batched_shapes(77, 9, (2, 12), (5, 30))
    T = oracle.Params(*I.teacher_weights(D=6, H=3))
    nets = []
    for t in range(9):
        X = I.features(I.subseed(77, 100 + t), int(ns[t]), 6)
        nets.append((X, oracle.predict(X, T).astype(np.float64), oracle.Params(*I.init_weights(t, 6, int(Hs[t])))))
    return Hs, ns, nets


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    Hs, ns, nets = _nets()
    parts = shard.partition_lpt(ns * Hs, world)
    mine = [nets[t] for t in parts[rank]]
    epochs = 7
    out, loss = oracle.batch_train(mine, 0.1, epochs) if mine else ([], np.zeros((0, epochs)))
    P = torch.from_numpy(np.concatenate([p.flat() for p in out]).astype(np.float32)) if out else torch.zeros(0)
    L = torch.from_numpy(np.asarray(loss, np.float64).reshape(len(mine), epochs))
    got = shard.Gather(parts, 6, Hs, epochs)(P, L)
    if rank == 0:
        q.put((got[0].numpy(), got[1].numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_single_rank_result():
    import torch.multiprocessing as mp

    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    P, L = q.get(timeout=300)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    Hs, ns, nets = _nets()
    out, loss = oracle.batch_train(nets, 0.1, 7)
    assert np.array_equal(P, np.concatenate([p.flat() for p in out]).astype(np.float32))
    assert np.array_equal(L, np.asarray(loss).reshape(9, 7))
