"""The entry point that allocates no device memory (for callers that cannot
call cudaMalloc: a framework that serves all device memory from its own pool,
or a real-time loop that must not wait on the allocator) against the
handle-based training entry point, through the C ABI.  Collected last on
purpose, so that a run stopping at the first failure has run everything else."""
import numpy as np
import pytest

from paper_1908_07847_gb300 import binding as B
from tests.gpu_util import W_TOL, Net, dev, host, lr32, problem, rel_err_elem, rel_err_norm, stream

pytestmark = pytest.mark.gpu


def test_noalloc_matches_handle_path_on_two_calls_in_a_row():
    import torch
    n, D, H, epochs = 1000, 33, 64, 20
    X, y, W = problem(4321, n, D, H)
    Xd, yd = dev(X), dev(y)
    params = dev(np.concatenate([W[0].ravel(), W[1], W[2], W[3]]).astype(np.float32))
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    with Net(D, H) as ref:
        ref.set(W)
        for call in range(2):
            lh_ref = torch.zeros(epochs, dtype=torch.float64, device="cuda")
            lh = torch.zeros(epochs, dtype=torch.float64, device="cuda")
            B.mlp_train_epochs(ref.h, Xd, yd, n, epochs, 0, lh_ref, None, stream())
            B.mlp_train_fused_noalloc(B.MLP_ACT_SIGMOID, D, H, n, Xd, yd, params, lr32(), 1, epochs, 0, lh,
                                      status, stream())
            torch.cuda.synchronize()
            assert int(host(status)[0]) == 0
            assert ref.check() == B.MLP_OK
            assert rel_err_norm(host(params), ref.flat()) <= W_TOL, call
            assert rel_err_elem(host(lh), host(lh_ref)) <= 1e-5, call


def test_noalloc_largest_network_with_minibatches():
    """D = 64, H = 128 fills the static array exactly; mini-batches of 300 rows
    (the last one ragged) and the tanh activation, two calls in a row."""
    import torch
    n, D, H, epochs, mb = 1000, 64, 128, 5, 300
    X, y, W = problem(8765, n, D, H)
    Xd, yd = dev(X), dev(y)
    params = dev(np.concatenate([W[0].ravel(), W[1], W[2], W[3]]).astype(np.float32))
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    with Net(D, H, act=B.MLP_ACT_TANH) as ref:
        ref.set(W)
        for call in range(2):
            lh_ref = torch.zeros(epochs, dtype=torch.float64, device="cuda")
            lh = torch.zeros(epochs, dtype=torch.float64, device="cuda")
            B.mlp_train_epochs(ref.h, Xd, yd, n, epochs, mb, lh_ref, None, stream())
            B.mlp_train_fused_noalloc(B.MLP_ACT_TANH, D, H, n, Xd, yd, params, lr32(), 1, epochs, mb, lh,
                                      status, stream())
            torch.cuda.synchronize()
            assert int(host(status)[0]) == 0
            assert ref.check() == B.MLP_OK
            assert rel_err_norm(host(params), ref.flat()) <= W_TOL, call
            assert rel_err_elem(host(lh), host(lh_ref)) <= 1e-5, call


def test_noalloc_rejects_networks_beyond_its_array():
    import torch
    p = torch.zeros(1024, device="cuda")
    with pytest.raises(B.MLPError) as e:
        B.mlp_train_fused_noalloc(B.MLP_ACT_SIGMOID, 33, 129, 10, p, p, p, 0.1, 1, 1)
    assert e.value.status == B.MLP_EINVAL and "H <= 128" in str(e.value)
