"""Z-score normalisation on the GPU (Sec. 2.2 normalises the data; read as the
training rows' per-column mean and population deviation) against the oracle:
statistics within 1e-12 relative (FP64 sums in another order), FP32 outputs
within a few float ulps, bf16 outputs within one bf16 ulp; padding exactly 0."""
import numpy as np
import pytest

import oracle
from paper_1908_07847_gb300 import binding as B
from paper_1908_07847_gb300 import inputs as I
from tests.gpu_util import dev, host, stream

pytestmark = pytest.mark.gpu


def table(seed, n, D):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, D)) * rng.uniform(0.2, 5.0, D) + rng.uniform(-50.0, 50.0, D)
    X[:, min(3, D - 1)] = 7.25    # a constant column
    return X.astype(np.float32)


def run(X, n_fit, prec, D_out):
    import torch
    n, D = X.shape
    ws = B.mlp_zscore_workspace_bytes(D)
    W = torch.empty(ws, dtype=torch.uint8, device="cuda")
    Y = torch.full((n, D_out), 99, dtype=torch.float32 if prec == B.MLP_FP32 else torch.int16, device="cuda")
    m = torch.zeros(D, dtype=torch.float64, device="cuda")
    s = torch.zeros(D, dtype=torch.float64, device="cuda")
    B.mlp_zscore(dev(X), n, D, n_fit, prec, D_out, Y, m, s, W, ws, stream())
    torch.cuda.synchronize()
    return host(Y), host(m), host(s)


def bf16_to_float(bits):
    return (bits.astype(np.uint16).astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("n,D,n_fit", [(1, 5, 1), (100, 33, 75), (1000, 33, 1000), (5000, 33, 3750), (300, 300, 200)])
def test_fp32_output_and_statistics(n, D, n_fit):
    X = table(n + D, n, D)
    Y, m, s = run(X, n_fit, B.MLP_FP32, D)
    Yr, mr, sr = oracle.zscore(X.astype(np.float64), n_fit)
    np.testing.assert_allclose(m, mr, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(s, sr, rtol=1e-12, atol=1e-300)
    # FP32: the two-float mean keeps x - m within a float ulp of |x - m|, the
    # scaling adds one rounding: a few ulps of max(|y|, 1)
    tol = 4 * np.finfo(np.float32).eps * np.maximum(np.abs(Yr), 1.0)
    assert np.all(np.abs(Y - Yr) <= tol)
    assert np.all(Y[:, s == 0.0] == 0.0)


def test_bf16_padded_output_is_the_tensor_core_input():
    """33 columns normalised, converted to bf16 and zero-padded to 48."""
    n, D, n_fit = 65536, 33, I.split_count(65536)
    X = table(7, n, D)
    Yb, m, s = run(X, n_fit, B.MLP_BF16, 48)
    Yr, mr, sr = oracle.zscore(X.astype(np.float64), n_fit)
    got = bf16_to_float(Yb)
    assert np.all(Yb[:, D:] == 0)
    ref = I.bf16_round(Yr.astype(np.float32)).astype(np.float64)
    ulp = np.maximum(np.abs(ref), 2.0 ** -126) * 2.0 ** -7
    assert np.all(np.abs(got[:, :D] - ref) <= ulp)
    assert np.mean(got[:, :D] == ref) > 0.999


def test_deterministic_and_rejects_bad_arguments():
    X = table(3, 2000, 33)
    a = run(X, 1500, B.MLP_FP32, 33)
    b = run(X, 1500, B.MLP_FP32, 33)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    import torch
    ws = B.mlp_zscore_workspace_bytes(33)
    W = torch.empty(ws, dtype=torch.uint8, device="cuda")
    Y = torch.empty((10, 33), device="cuda")
    m = torch.empty(33, dtype=torch.float64, device="cuda")
    for n_fit, D_out, wsb in [(0, 33, ws), (11, 33, ws), (5, 32, ws), (5, 33, 8)]:
        with pytest.raises(B.MLPError) as e:
            B.mlp_zscore(dev(X[:10]), 10, 33, n_fit, B.MLP_FP32, D_out, Y, m, m, W, wsb, stream())
        assert e.value.status == B.MLP_EINVAL
