"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method (no forward pass, no gradient, no
update).  It only draws random numbers and lays them out:

* ``splitmix64``: the SplitMix64 generator (Steele, Lea, Flood, "Fast
  splittable pseudorandom number generators", OOPSLA 2014; the finaliser
  constants as published by Vigna), used counter-style: value i of a stream with
  seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15).
* uniform doubles in [0, 1) from the top 53 bits; standard normals by the
  Box-Muller transform on pairs of uniforms.
* the cohort stand-in: the paper's 120 participants x 33 markers (Sec. 2.1) is
  not available, so features are i.i.d. N(0, 1) (already standardised), seed
  1908 + the workload index, optionally zero-padded on the right (33 -> 48).
* weight initialisation (the paper does not state one): W1 ~ U(-1/sqrt(D),
  1/sqrt(D)), w2 ~ U(-1/sqrt(H), 1/sqrt(H)), biases 0, padded W1 columns 0.
* teacher-net weights (33-8-1, N(0, 1), biases 0, seed 7847).  Labels are the
  teacher's class decisions; computing them runs the method's forward pass, so
  that happens on the caller's side (the oracle in tests, the library's own
  predict call in the benchmark), not here.
* bfloat16 rounding of features (round to nearest even), so that both sides
  see the same bf16 values.
* the 75 % / 25 % split rule (Sec. 1 and Sec. 2.2): n_train = round(0.75 n).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

COHORT_SEED = 1908
TEACHER_SEED = 7847
INIT_SEED = 4242
D_MARKERS = 33
D_PADDED = 48
N_PARTICIPANTS = 120
N_MALE = 61
N_FEMALE = 59


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Values start .. start+count-1 of the SplitMix64 stream with this seed."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + idx * _GOLDEN
        return _mix(z)


def subseed(seed: int, stream: int) -> int:
    """Independent child seed number ``stream`` of ``seed``."""
    return int(splitmix64(seed, 1, start=stream)[0])


def uniform(seed: int, count: int) -> np.ndarray:
    """float64 uniforms in [0, 1) (top 53 bits of each SplitMix64 value)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """float64 standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]          # in (0, 1], so the log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:count]


def uniform_int(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on [lo, hi] (inclusive)."""
    u = uniform(seed, count)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def features(seed: int, n: int, D: int = D_MARKERS, Dpad: int | None = None) -> np.ndarray:
    """n x Dpad float32 row-major features: N(0, 1) in the first D columns,
    zeros in the padding columns."""
    Dpad = D if Dpad is None else Dpad
    X = np.zeros((n, Dpad), dtype=np.float32)
    X[:, :D] = normal(seed, n * D).reshape(n, D).astype(np.float32)
    return X


def init_weights(seed: int, D: int, H: int, Dpad: int | None = None):
    """float32 (W1 H x Dpad, b1 H, w2 H, b2 1): U(+-1/sqrt(D)), U(+-1/sqrt(H)),
    zero biases, zero padding columns."""
    Dpad = D if Dpad is None else Dpad
    a1 = 1.0 / np.sqrt(D)
    a2 = 1.0 / np.sqrt(H)
    W1 = np.zeros((H, Dpad), dtype=np.float32)
    W1[:, :D] = ((2.0 * uniform(subseed(seed, 1), H * D) - 1.0) * a1).reshape(H, D).astype(np.float32)
    w2 = ((2.0 * uniform(subseed(seed, 2), H) - 1.0) * a2).astype(np.float32)
    return W1, np.zeros(H, np.float32), w2, np.zeros(1, np.float32)


def teacher_weights(seed: int = TEACHER_SEED, D: int = D_MARKERS, H: int = 8,
                    Dpad: int | None = None):
    """float32 teacher-net weights (W1 H x Dpad ~ N(0,1), b1 = 0, w2 ~ N(0,1),
    b2 = 0); padding columns are 0."""
    Dpad = D if Dpad is None else Dpad
    W1 = np.zeros((H, Dpad), dtype=np.float32)
    W1[:, :D] = normal(subseed(seed, 1), H * D).reshape(H, D).astype(np.float32)
    w2 = normal(subseed(seed, 2), H).astype(np.float32)
    return W1, np.zeros(H, np.float32), w2, np.zeros(1, np.float32)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returns
    float32 arrays holding exactly representable bf16 values."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(x)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).copy()
    out[nan] = np.nan
    return out.reshape(x.shape)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of bf16_round(x)."""
    return (bf16_round(x).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def split_count(n: int, train_frac: float = 0.75) -> int:
    """Rows in the training split: round half up of train_frac * n."""
    return int(np.floor(train_frac * n + 0.5))


def batched_shapes(seed: int, n_nets: int, H_range, n_range):
    """Per-net hidden widths and row counts, each uniform on its inclusive range."""
    Hs = uniform_int(subseed(seed, 11), n_nets, H_range[0], H_range[1])
    ns = uniform_int(subseed(seed, 12), n_nets, n_range[0], n_range[1])
    return Hs, ns
