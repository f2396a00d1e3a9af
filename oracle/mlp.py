"""ORACLE -- test infrastructure only.

FP64 statement of the learned partitioner's network: a 1-32-32-1 ReLU MLP
that maps a monotone feature of a 64-bit key to an estimate of the key's
empirical CDF, trained with mean squared error and Adam.  The paper has no
learned component (its Sort splits the KPA into chunks and sorts each chunk
in-core, Sec. 4.2 "Primitive Implementation"); this network only chooses MSD
bucket boundaries, and the sorted output it leads to is the plain sort.

Parameter layout (flat, 1153 values): W1[32], b1[32], W2[32][32] (row = output
unit), b2[32], w3[32], b3[1].

Pins: backward against FP64 central finite differences of ``loss``; forward
against closed-form networks; one Adam step against its closed form; the
feature against its bit-level definition on hand-picked keys.
"""
from __future__ import annotations

import numpy as np

H = 32
N_PARAMS = H + H + H * H + H + H + 1
SLICES = {
    "W1": slice(0, H),
    "b1": slice(H, 2 * H),
    "W2": slice(2 * H, 2 * H + H * H),
    "b2": slice(2 * H + H * H, 3 * H + H * H),
    "w3": slice(3 * H + H * H, 4 * H + H * H),
    "b3": slice(4 * H + H * H, 4 * H + H * H + 1),
}


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    return (p[SLICES["W1"]], p[SLICES["b1"]], p[SLICES["W2"]].reshape(H, H), p[SLICES["b2"]],
            p[SLICES["w3"]], p[SLICES["b3"]][0])


def feature(keys: np.ndarray) -> np.ndarray:
    """x(k) = (msb(k) + f/2^17) / 64, where msb(k) is the index of the highest
    set bit and f the 17 bits just below it (zero-padded); x(0) = 0.  The value
    has at most 23 significant bits, so it is exact in FP32, and it is
    non-decreasing in k."""
    keys = np.asarray(keys, dtype=np.uint64)
    x = np.zeros(keys.shape, dtype=np.float64)
    for i, k in enumerate(keys.tolist()):
        if k == 0:
            continue
        m = k.bit_length() - 1
        shifted = (k << (63 - m)) & 0xFFFFFFFFFFFFFFFF
        f = (shifted >> 46) & 0x1FFFF
        x[i] = (m + f / 131072.0) / 64.0
    return x


def cdf_targets(sample: np.ndarray) -> np.ndarray:
    """Target of each sample key: the midpoint of its empirical CDF step,
    (#samples < k + #samples <= k) / (2m)."""
    sample = np.asarray(sample, dtype=np.uint64)
    m = sample.size
    srt = np.sort(sample)
    lt = np.searchsorted(srt, sample, side="left")
    le = np.searchsorted(srt, sample, side="right")
    return (lt + le).astype(np.float64) / (2.0 * m)


def forward(p: np.ndarray, x: np.ndarray):
    """Returns y and the intermediates (a1, h1, a2, h2)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    a1 = x[:, None] * W1[None, :] + b1[None, :]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2[None, :]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    return y, (a1, h1, a2, h2)


def loss(p: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(p, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def backward(p: np.ndarray, x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Gradient of the mean squared error over the batch (ReLU'(0) = 0)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    y, (a1, h1, a2, h2) = forward(p, x)
    B = x.size
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / B
    g = np.zeros(N_PARAMS, dtype=np.float64)
    g[SLICES["w3"]] = h2.T @ dy
    g[SLICES["b3"]] = dy.sum()
    da2 = (dy[:, None] * w3[None, :]) * (a2 > 0)
    g[SLICES["W2"]] = (da2.T @ h1).reshape(-1)
    g[SLICES["b2"]] = da2.sum(axis=0)
    da1 = (da2 @ W2) * (a1 > 0)
    g[SLICES["W1"]] = da1.T @ x
    g[SLICES["b1"]] = da1.sum(axis=0)
    return g


def abs_terms(p: np.ndarray, x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Per parameter, the sum over rows of the magnitudes of the row terms
    whose sum is the gradient (each term of ``backward`` taken in absolute
    value before the sum over rows).  A sum of such terms computed in FP32
    is off by at most a small multiple of the unit roundoff times this, so it
    scales the tolerance of each parameter's gradient."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    y, (a1, h1, a2, h2) = forward(p, x)
    B = x.size
    dy = np.abs(2.0 * (y - np.asarray(t, dtype=np.float64)) / B)
    A = np.zeros(N_PARAMS, dtype=np.float64)
    A[SLICES["w3"]] = h2.T @ dy
    A[SLICES["b3"]] = dy.sum()
    da2 = (dy[:, None] * np.abs(w3)[None, :]) * (a2 > 0)
    A[SLICES["W2"]] = (da2.T @ h1).reshape(-1)
    A[SLICES["b2"]] = da2.sum(axis=0)
    # |da1| of each row is bounded by the sum of its terms' magnitudes
    da1 = (da2 @ np.abs(W2)) * (a1 > 0)
    A[SLICES["W1"]] = da1.T @ np.abs(x)
    A[SLICES["b1"]] = da1.sum(axis=0)
    return A


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update with bias correction (step counts from 1).  Returns
    new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v


def train(p0, x, t, steps, batch, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam on the training set in order: step j (from 0) uses the rows
    (j * batch + i) mod m for i < batch.  Returns the final parameters and the
    loss over the whole set after each step."""
    p = np.asarray(p0, dtype=np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = x.size
    losses = []
    for j in range(steps):
        idx = (np.arange(batch, dtype=np.int64) + j * batch) % n
        g = backward(p, x[idx], t[idx])
        p, m, v = adam_step(p, g, m, v, j + 1, lr, beta1, beta2, eps)
        losses.append(loss(p, x, t))
    return p, losses


def quantile_init(nh_sorted) -> np.ndarray:
    """Parameters that make the network the piecewise-linear interpolation of
    the training set's CDF at 33 quantiles (the start when no initial weights
    are given).  With m' sorted non-heavy samples, knot i (0..32) is sample
    j = floor(i (m' - 1) / 32): x = feature(key), F = its CDF target
    (#samples < key + #samples <= key) / (2 m').  Knots with the x of the
    previous kept knot are merged into it (it takes the later F).  Hidden unit
    u of the first layer kinks at kept knot u (W1 = 1, b1 = -x_u); the second
    layer passes it on (W2 = I, b2 = 0); w3_u is the change of slope at knot u
    and b3 the first knot's F, so the output passes through every kept knot.
    Units without a segment are zero."""
    nh = np.asarray(nh_sorted, dtype=np.uint64)
    m = nh.size
    p = np.zeros(N_PARAMS, dtype=np.float64)
    if m == 0:
        return p
    xs, fs = [], []
    for i in range(H + 1):
        j = (i * (m - 1)) // H
        k = nh[j]
        lt = int(np.searchsorted(nh, k, side="left"))
        le = int(np.searchsorted(nh, k, side="right"))
        x = float(feature(np.array([k], dtype=np.uint64))[0])
        f = (lt + le) / (2.0 * m)
        if xs and x <= xs[-1]:
            fs[-1] = f
        else:
            xs.append(x)
            fs.append(f)
    W1, b1, W2, b2, w3 = (np.zeros(H), np.zeros(H), np.eye(H), np.zeros(H), np.zeros(H))
    prev = 0.0
    for u in range(len(xs) - 1):
        slope = (fs[u + 1] - fs[u]) / (xs[u + 1] - xs[u])
        W1[u], b1[u], w3[u] = 1.0, -xs[u], slope - prev
        prev = slope
    p[SLICES["W1"]], p[SLICES["b1"]], p[SLICES["W2"]] = W1, b1, W2.reshape(-1)
    p[SLICES["b2"]], p[SLICES["w3"]], p[SLICES["b3"]] = b2, w3, fs[0]
    return p
