"""The many-nets workload split across two ranks on the GPU: two processes
(gloo for the gather; each runs its own independent training launch, no
kernel waits on another) train their cost-balanced shares of a batch with the
library's plan, and the gathered weights and loss histories equal those of a
single-process run of the whole batch bit for bit."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

D, EPOCHS = 33, 40


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _batch():
    import oracle
    from paper_1908_07847_gb300 import inputs as I
    Hs, ns = I.batched_shapes(31, 40, (4, 128), (50, 120))
    T = oracle.Params(*I.teacher_weights(D=D))
    nets = []
    for t in range(40):
        X = I.features(I.subseed(31, 100 + t), int(ns[t]), D)
        nets.append((X, oracle.predict(X, T).astype(np.float32), I.init_weights(I.subseed(31, 200 + t), D, int(Hs[t]))))
    return Hs, ns, nets


def _train(nets):
    """The library's one-launch plan on `nets`; (flat weights, losses) on the host."""
    import torch
    from paper_1908_07847_gb300 import binding as B
    keep, descs = [], []
    P = torch.from_numpy(np.concatenate([np.concatenate([W[0].ravel(), W[1], W[2], W[3]]) for _, _, W in nets])
                         .astype(np.float32) if nets else np.zeros(0, np.float32)).cuda()
    L = torch.zeros((len(nets), EPOCHS), dtype=torch.float64, device="cuda")
    o = 0
    for i, (X, y, W) in enumerate(nets):
        Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
        keep += [Xd, yd]
        descs.append(B.mlp_net_desc(W[0].shape[0], X.shape[0], Xd.data_ptr(), yd.data_ptr(), P[o:].data_ptr(),
                                    L[i].data_ptr()))
        o += (D + 2) * W[0].shape[0] + 1
    if nets:
        b = B.mlp_batch_create(B.MLP_FP32, B.MLP_ACT_SIGMOID, D, descs, float(np.float32(0.1)), 1)
        try:
            B.mlp_batch_run(b, EPOCHS, torch.cuda.current_stream().cuda_stream)
            assert B.mlp_batch_check(b, torch.cuda.current_stream().cuda_stream) == B.MLP_OK, B.mlp_last_error()
        finally:
            B.mlp_batch_destroy(b)
    return P.cpu(), L.cpu()


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_1908_07847_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    Hs, ns, nets = _batch()
    parts = shard.partition_lpt(ns * Hs, world)
    P, L = _train([nets[t] for t in parts[rank]])
    got = shard.Gather(parts, D, Hs, EPOCHS)(P, L)
    if rank == 0:
        q.put((got[0].numpy(), got[1].numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gather_the_single_process_result():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    P, L = q.get(timeout=600)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    _, _, nets = _batch()
    P1, L1 = _train(nets)
    assert np.array_equal(P, P1.numpy()) and np.array_equal(L, L1.numpy())
