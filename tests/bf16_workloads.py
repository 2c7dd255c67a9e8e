"""Seeded inputs of the two bf16 tensor-core workloads whose long runs are
checked against stored oracle results (tests/golden/*.json, written by
tests/golden/make_bf16_golden.py, which calls only the oracle).  Input
generation only: no arithmetic of the method here.

* wide net (48-2048-1, mini-batch 8192, 20 epochs): the first 65,536 rows of
  the 1,048,576-row table (33 N(0, 1) features zero-padded to 48, rounded to
  bf16), the first 75 % (49,152 rows, six mini-batches) for training and the
  rest (16,384 rows) for testing (Sec. 1 and Sec. 2.2: a 75 / 25 split);
* many nets (1024 nets 48-256-1, n ~ U{4096..16384}, 200 epochs): four of the
  nets (the first, the largest, the smallest, the last), each split 75 / 25.
Labels are the 33-8-1 teacher net's decisions; the callers compute them with
the oracle.
"""
import numpy as np

from paper_1908_07847_gb300 import inputs as I

D_REAL, D_PAD = 33, 48

# wide net
C3_SEED, C3_H, C3_MB, C3_EPOCHS, C3_ROWS = 1908, 2048, 8192, 20, 65536
C3_TRAIN = I.split_count(C3_ROWS)          # 49,152
C3_KEEP_EVERY = 16                         # stored hidden units: j % 16 == 0

# many nets
C4_SEED, C4_NETS, C4_H, C4_EPOCHS = 4, 1024, 256, 200
C4_KEEP_EVERY = 8
C4_CHUNK = 1 << 20


def c3_rows():
    """The 65,536 rows (bf16-exact float32, 48 wide)."""
    X = I.features(I.subseed(C3_SEED, 20_000), 1 << 18, D_REAL, D_PAD)[:C3_ROWS]
    return I.bf16_round(X)


def c3_weights():
    return I.init_weights(I.INIT_SEED + 3, D_REAL, C3_H, D_PAD)


def c4_shapes():
    _, ns = I.batched_shapes(C4_SEED, C4_NETS, (C4_H, C4_H), (4096, 16384))
    return ns


def c4_picks(ns):
    return sorted({0, int(np.argmax(ns)), int(np.argmin(ns)), C4_NETS - 1})


def c4_chunks(ns):
    """(first row, rows) of every 2^20-row chunk of the concatenated table."""
    total = int(np.sum(ns))
    return [(r0, min(C4_CHUNK, total - r0)) for r0 in range(0, total, C4_CHUNK)]


def c4_chunk(r0, rows):
    """Rows r0 .. r0 + rows - 1 of the concatenated table (bf16-exact)."""
    return I.bf16_round(I.features(I.subseed(C4_SEED, 10_000 + r0 // C4_CHUNK), rows, D_REAL, D_PAD))


def c4_net_rows(ns, t):
    """Net t's rows, assembled from the chunks it spans."""
    offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    a, b = int(offs[t]), int(offs[t + 1])
    parts = []
    for r0, rows in c4_chunks(ns):
        lo, hi = max(a, r0), min(b, r0 + rows)
        if lo < hi:
            parts.append(c4_chunk(r0, rows)[lo - r0:hi - r0])
    return np.concatenate(parts)


def c4_weights(t):
    return I.init_weights(I.subseed(C4_SEED, 200 + t), D_REAL, C4_H, D_PAD)


def kept_params(W1, b1, w2, b2, every):
    """The stored subsample of a net's weights: the rows of W1 (real columns),
    b1 and w2 of the hidden units j % every == 0, then b2."""
    W1, b1, w2 = np.asarray(W1), np.asarray(b1), np.asarray(w2)
    js = np.arange(0, W1.shape[0], every)
    return np.concatenate([W1[js, :D_REAL].ravel(), b1[js], w2[js], np.ravel(b2)]).astype(np.float64)
