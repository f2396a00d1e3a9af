"""ORACLE -- test infrastructure only.

Plain statement of the learned partitioner's data preparation: which key
values get a dedicated bucket (heavy keys), and the training set the network
is fitted to.  The sort that uses the partition is pinned by the plain
sort (its output must be identical); these functions pin the pieces the CUDA
path computes on the way.

Cells.  Key 0 is cell 0.  A key k >= 1 with highest set bit m lies in cell
1 + 1024 m + (the 10 bits just below bit m); the 32 bits below those are its
offset inside the cell.  A cell with m <= 10 holds exactly one key value
("exact" cell).

Heavy keys.  A key value is heavy when its sample count, scaled to the rows
the sample stands for, exceeds half the bucket capacity: count * n_rows >
(capacity / HEAVY_DIV) * m.  The heavy keys are taken in ascending order, at most
MAX_HEAVY of them (the smallest, if there are more).

Training set.  The non-heavy samples, sorted; row r of the set takes sorted
sample j = (r * P) mod m', with P the first integer >= 2654435761 mod m'
coprime to m'.  Its input is the key feature (``mlp.feature``) and its
target the midpoint of the key's empirical CDF step among the non-heavy
samples.
"""
from __future__ import annotations

import math

import numpy as np

from . import mlp

NCELL = 1 + 64 * 1024
EXACT_MAX_MSB = 10
MAX_HEAVY = 16384
HEAVY_DIV = 2


def cell_of(keys) -> np.ndarray:
    out = np.zeros(len(keys), dtype=np.int64)
    for i, k in enumerate(np.asarray(keys, dtype=np.uint64).tolist()):
        if k == 0:
            continue
        m = k.bit_length() - 1
        top = (k << (63 - m)) & 0xFFFFFFFFFFFFFFFF
        out[i] = 1 + 1024 * m + ((top >> 53) & 1023)
    return out


def cell_is_exact(c: int) -> bool:
    return c == 0 or (c - 1) // 1024 <= EXACT_MAX_MSB


def heavy_keys(sample, n_rows: int, capacity: int) -> np.ndarray:
    """The heavy key values, ascending (uint64), at most MAX_HEAVY."""
    sample = np.asarray(sample, dtype=np.uint64)
    m = sample.size
    counts = {}
    for k in sample.tolist():
        counts[k] = counts.get(k, 0) + 1
    heavy = sorted(k for k, c in counts.items() if c * n_rows > (capacity // HEAVY_DIV) * m)
    return np.array(heavy[:MAX_HEAVY], dtype=np.uint64)


def stride_multiplier(m: int) -> int:
    p = 2654435761 % m
    while math.gcd(p, m) != 1:
        p += 1
    return p


def training_set(sample, n_rows: int, capacity: int):
    """(x, t) in training order, as float64."""
    sample = np.asarray(sample, dtype=np.uint64)
    heavy = heavy_keys(sample, n_rows, capacity)
    srt = np.sort(sample)
    keep = ~np.isin(srt, heavy)
    nh = srt[keep]
    m = nh.size
    if m == 0:
        return np.zeros(0), np.zeros(0)
    lt = np.searchsorted(nh, nh, side="left")
    le = np.searchsorted(nh, nh, side="right")
    t = (lt + le).astype(np.float64) / (2.0 * m)
    x = mlp.feature(nh)
    P = stride_multiplier(m)
    j = (np.arange(m, dtype=np.uint64) * np.uint64(P)) % np.uint64(m)
    j = j.astype(np.int64)
    return x[j], t[j]
