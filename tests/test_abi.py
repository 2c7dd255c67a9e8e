"""The C-ABI library loads and exports every symbol include/mlp_gb300.h
declares; host-side argument checks run without a GPU."""
import os
import re

import pytest

from paper_1908_07847_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mlp_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mlp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    return B.lib()


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(built):
    for name in declared_symbols():
        assert hasattr(built, name), name
    assert "sm_103a" in B.mlp_version()


def test_host_side_validation_without_gpu(built):
    # Rejected before any CUDA call: shape and precision checks.
    with pytest.raises(B.MLPError) as e:
        B.mlp_workspace_bytes(7, 33, 64, 10)
    assert e.value.status == B.MLP_EINVAL
    with pytest.raises(B.MLPError):
        B.mlp_workspace_bytes(B.MLP_FP32, 0, 64, 10)
    assert "mlp_workspace_bytes" in B.mlp_last_error()


def test_binding_refuses_non_contiguous_buffers():
    """The binding passes raw addresses: a strided view would be read as if it
    were dense, so it is refused; dense arrays, tensors, ints and None pass."""
    import numpy as np
    import torch
    a = np.zeros((4, 6), np.float32)
    assert B._p(a) == a.ctypes.data
    assert B._p(a[1:3]) == a[1:3].ctypes.data          # a row slice stays dense
    with pytest.raises(ValueError):
        B._p(a[:, :3])
    with pytest.raises(ValueError):
        B._p(a.T)
    t = torch.zeros(4, 6)
    assert B._p(t) == t.data_ptr()
    with pytest.raises(ValueError):
        B._p(t.t())
    assert B._p(None) is None and B._p(1234) == 1234
