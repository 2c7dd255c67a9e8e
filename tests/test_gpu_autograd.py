"""The autograd.Function over the library's hand-written backward kernel:
FP64 gradcheck against central finite differences (h = 1e-6) and FP32 / FP64
gradients against the oracle (Sec. 2.2 backpropagation)."""
import numpy as np
import pytest

import oracle
from oracle import Params
from tests.gpu_util import GRAD_TOL, problem, rel_err_norm

pytestmark = pytest.mark.gpu


def tt(a, dtype, grad=False):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda", requires_grad=grad)


@pytest.mark.parametrize("act", [0, 1])
def test_gradcheck_fp64_small_with_input_gradient(act):
    import torch
    from paper_1908_07847_gb300.autograd import mlp
    X, y, W = problem(2024, 17, 5, 7)
    args = [tt(X, torch.float64, True)] + [tt(w, torch.float64, True) for w in W]
    assert torch.autograd.gradcheck(lambda *a: mlp(*a, act=act), args, eps=1e-6, atol=1e-8, rtol=1e-6)


def test_gradcheck_fp64_config_4096x33_h64():
    """The 33-64-1 network on 4096 rows, parameters only (fast mode: random
    projections of the Jacobian), central differences with h = 1e-6."""
    import torch
    from paper_1908_07847_gb300.autograd import mlp
    X, y, W = problem(2025, 4096, 33, 64)
    Xd = tt(X, torch.float64)
    args = [tt(w, torch.float64, True) for w in W]
    assert torch.autograd.gradcheck(lambda *a: mlp(Xd, *a), args, eps=1e-6, atol=1e-8, rtol=1e-6,
                                    fast_mode=True)


@pytest.mark.parametrize("dtype_name,tol", [("float32", GRAD_TOL), ("float64", 1e-12)])
def test_mse_gradients_through_autograd_match_oracle(dtype_name, tol):
    import torch
    from paper_1908_07847_gb300.autograd import mlp
    dt = getattr(torch, dtype_name)
    X, y, W = problem(2026, 4096, 33, 64)
    Wt = [tt(w, dt, True) for w in W]
    o = mlp(tt(X, dt), *Wt)
    loss = 0.5 * ((o - tt(y, dt)) ** 2).mean()
    loss.backward()
    ref = oracle.mse_gradients(X, y, Params(*W))
    got = np.concatenate([w.grad.double().cpu().numpy().ravel() for w in Wt])
    exp = np.concatenate([ref[0].ravel(), ref[1], ref[2], [ref[3]]])
    assert rel_err_norm(got, exp) <= tol
    assert float(loss) == pytest.approx(ref[4], rel=1e-6 if dtype_name == "float32" else 1e-13)


def test_upstream_gradient_and_input_gradient_match_oracle():
    import torch
    from paper_1908_07847_gb300.autograd import mlp
    X, y, W = problem(2027, 300, 33, 40)
    u = np.random.default_rng(0).normal(size=300)
    Xt = tt(X, torch.float64, True)
    Wt = [tt(w, torch.float64, True) for w in W]
    (mlp(Xt, *Wt) * tt(u, torch.float64)).sum().backward()
    gW1, gb1, gw2, gb2, gX = oracle.backward(X, Params(*W), u, want_gX=True)
    assert rel_err_norm(Wt[0].grad.cpu().numpy(), gW1) <= 1e-12
    assert rel_err_norm(Wt[1].grad.cpu().numpy(), gb1) <= 1e-12
    assert rel_err_norm(Wt[2].grad.cpu().numpy(), gw2) <= 1e-12
    assert abs(float(Wt[3].grad) - gb2) <= 1e-12 * max(1.0, abs(gb2))
    assert rel_err_norm(Xt.grad.cpu().numpy(), gX) <= 1e-12


def test_module_trains_with_torch_optimizer():
    """The module's parameters take plain SGD steps (lr 0.1, no momentum,
    Sec. 2.2) and follow the oracle's full-batch trajectory."""
    import torch
    from paper_1908_07847_gb300.autograd import MLP
    X, y, W = problem(2028, 512, 33, 16)
    m = MLP(33, 16, dtype=torch.float64)
    with torch.no_grad():
        for p, w in zip([m.W1, m.b1, m.w2, m.b2], W):
            p.copy_(torch.tensor(w, dtype=torch.float64))
    opt = torch.optim.SGD(m.parameters(), lr=0.1)
    Xd, yd = tt(X, torch.float64), tt(y, torch.float64)
    for _ in range(10):
        opt.zero_grad()
        (0.5 * ((m(Xd) - yd) ** 2).mean()).backward()
        opt.step()
    q, _, _ = oracle.train(X, y, Params(*W), 0.1, 10)
    got = np.concatenate([p.detach().cpu().numpy().ravel() for p in [m.W1, m.b1, m.w2, m.b2]])
    assert rel_err_norm(got, q.flat()) <= 1e-12
