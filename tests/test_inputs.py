"""Seeded input generators: published SplitMix64 vectors, distributions, bf16
rounding against torch's conversion, padding and shapes."""
import numpy as np
import pytest

from paper_1908_07847_gb300 import inputs as I


def test_splitmix64_published_vectors():
    # Reference outputs of SplitMix64 for seeds 0 and 1234567.
    assert [int(v) for v in I.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in I.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_counter_based_slices_agree():
    a = I.splitmix64(99, 100)
    b = I.splitmix64(99, 40, start=60)
    np.testing.assert_array_equal(a[60:], b)


def test_normal_moments():
    z = I.normal(5, 200_000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    u = I.uniform(6, 100_000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01


def test_features_padding_and_determinism():
    X = I.features(1908, 120, 33, 48)
    assert X.shape == (120, 48) and X.dtype == np.float32
    assert np.all(X[:, 33:] == 0)
    np.testing.assert_array_equal(X[:, :33], I.features(1908, 120, 33))
    assert not np.array_equal(X, I.features(1909, 120, 33, 48))


def test_init_weights_ranges():
    W1, b1, w2, b2 = I.init_weights(3, 33, 64, 48)
    assert W1.shape == (64, 48) and np.all(W1[:, 33:] == 0)
    assert np.abs(W1).max() <= 1 / np.sqrt(33) and np.abs(w2).max() <= 1 / 8
    assert np.all(b1 == 0) and b2[0] == 0


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([I.normal(8, 10000).astype(np.float32) * 7,
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -0.0, 65504.0, 3e38],
                                 dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(I.bf16_round(x), ref)
    bits = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(I.bf16_bits(x), bits)


def test_batched_shapes_ranges():
    Hs, ns = I.batched_shapes(2, 4096, (4, 128), (50, 120))
    assert Hs.min() == 4 and Hs.max() == 128 and ns.min() == 50 and ns.max() == 120
