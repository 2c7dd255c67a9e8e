"""One network trained data-parallel on the GPU: two processes (gloo for the
exchange; each runs its own kernels, no kernel waits on another) each hold a
replica, compute the summed gradient of their shard of every mini-batch with
the library's backward, all-gather, add in rank order and update
(mlp_grad_sum, mlp_update).  The replicas end bit for bit equal, and within
the FP32 bars of the FP64 oracle's mini-batch training of the whole batch,
loss history included; a ragged last mini-batch of one row leaves rank 0 an
empty shard.  Also the combine kernel alone against a plain sum."""
import os
import socket

import numpy as np
import pytest

from tests.gpu_util import W_TOL, rel_err_elem, rel_err_norm

pytestmark = pytest.mark.gpu

N, D, H, MB, EPOCHS, LR = 769, 33, 64, 256, 4, 0.1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem(prec):
    import oracle
    from paper_1908_07847_gb300 import inputs as I
    Dp = 48 if prec == "bf16" else D
    X = I.features(I.subseed(93, 1), N, D, Dp)
    if prec == "bf16":
        X = I.bf16_round(X)
    y = oracle.predict(X[:, :D], oracle.Params(*I.teacher_weights(D=D))).astype(np.float32)
    return X, y, I.init_weights(94, D, H, Dp)


def _worker(rank, world, port, prec, q):
    import torch
    import torch.distributed as dist
    from paper_1908_07847_gb300 import binding as B
    from paper_1908_07847_gb300 import dataparallel as dp
    from paper_1908_07847_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    X, y, W = _problem(prec)
    Dp = X.shape[1]
    if prec == "bf16":
        Xd = torch.from_numpy(I.bf16_bits(X).view(np.int16)).cuda()
        h = B.mlp_create(Dp, H, float(np.float32(LR)), 0, B.MLP_BF16, B.MLP_ACT_SIGMOID)
    else:
        Xd = torch.from_numpy(X).cuda()
        h = B.mlp_create(Dp, H, float(np.float32(LR)), 0, B.MLP_FP32, B.MLP_ACT_SIGMOID)
    try:
        B.mlp_set_weights(h, *[np.ascontiguousarray(np.asarray(a, np.float32)) for a in W])
        yd = torch.from_numpy(y).cuda()
        L = torch.zeros(EPOCHS, dtype=torch.float64, device="cuda")
        dp.DataParallel(h, Dp, H).train(Xd, yd, N, EPOCHS, MB, True, L)
        torch.cuda.synchronize()
        Wn = [np.zeros((H, Dp), np.float32), np.zeros(H, np.float32), np.zeros(H, np.float32),
              np.zeros(1, np.float32)]
        B.mlp_get_weights(h, *Wn)
        flat = np.concatenate([a.astype(np.float64).ravel() for a in Wn])
        q.put((rank, flat, L.cpu().numpy()))
    finally:
        B.mlp_destroy(h)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_two_ranks_train_one_network(prec):
    import torch.multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, prec, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict((r, (w, lh)) for r, w, lh in (q.get(timeout=600) for _ in range(2)))
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][1], got[1][1])
    X, y, W = _problem(prec)
    qo, lh, _ = oracle.train(X.astype(np.float64), y.astype(np.float64), oracle.Params(*W),
                             float(np.float32(LR)), EPOCHS, minibatch=MB)
    assert rel_err_norm(got[0][0], qo.flat()) <= W_TOL
    assert rel_err_elem(got[0][1], lh) <= 1e-5


def test_grad_sum_is_the_rank_order_sum():
    import torch
    from paper_1908_07847_gb300 import binding as B
    rng = np.random.default_rng(5)
    for nparts, length in ((1, 1), (2, 6849), (3, 100003), (8, 257)):
        parts = rng.standard_normal((nparts, length)).astype(np.float32)
        lp = rng.standard_normal(nparts)
        P, LP = torch.from_numpy(parts).cuda(), torch.from_numpy(lp).cuda()
        out = torch.zeros(length, dtype=torch.float32, device="cuda")
        acc = torch.full((1,), 0.25, dtype=torch.float64, device="cuda")
        B.mlp_grad_sum(P, LP, nparts, length, 0.125, 0.5, out, acc, torch.cuda.current_stream().cuda_stream)
        exp = parts[0].copy()
        for r in range(1, nparts):
            exp = exp + parts[r]                      # float32, rank order
        exp = exp * np.float32(0.125)
        assert np.array_equal(out.cpu().numpy(), exp)
        le = lp[0]
        for r in range(1, nparts):
            le = le + lp[r]
        assert acc.cpu().numpy()[0] == 0.25 + 0.5 * le
    with pytest.raises(B.MLPError):
        B.mlp_grad_sum(P, None, 0, 4, 1.0, 1.0, out, None)
    with pytest.raises(B.MLPError):
        B.mlp_grad_sum(P, LP, 1, 4, 1.0, 1.0, out, None)
