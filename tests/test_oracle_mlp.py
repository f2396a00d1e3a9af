"""Pins for the FP64 statement of the learned partitioner's network."""
import numpy as np
import pytest

import gen
from oracle import mlp


def _rand_params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.5, mlp.N_PARAMS)


def test_backward_matches_central_differences():
    p = _rand_params(1)
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, 16)
    t = rng.uniform(0, 1, 16)
    g = mlp.backward(p, x, t)
    h = 1e-6
    num = np.empty_like(g)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        num[i] = (mlp.loss(p + e, x, t) - mlp.loss(p - e, x, t)) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_forward_closed_form_spline():
    # W1 = 1, b1_j = -j/32: h1_j = relu(x - j/32); W2 = I, b2 = 0; y = sum_j w3_j relu(x - j/32) + b3,
    # a linear spline with knots at j/32.
    H = mlp.H
    p = np.zeros(mlp.N_PARAMS)
    p[mlp.SLICES["W1"]] = 1.0
    p[mlp.SLICES["b1"]] = -np.arange(H) / H
    p[mlp.SLICES["W2"]] = np.eye(H).reshape(-1)
    w3 = np.linspace(-1, 1, H)
    p[mlp.SLICES["w3"]] = w3
    p[mlp.SLICES["b3"]] = 0.25
    for x in (0.0, 0.03, 0.5, 0.99):
        exp = 0.25 + sum(w3[j] * (x - j / H) for j in range(H) if x > j / H)
        y, _ = mlp.forward(p, np.array([x]))
        assert abs(y[0] - exp) < 1e-12


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # step 1: mhat = g, vhat = g^2, so each parameter moves by lr * g / (|g| + eps)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_feature_bit_definition():
    M64 = (1 << 64) - 1
    keys = np.array([0, 1, 2, 3, 6, (1 << 17) + 1, 1 << 63, M64], dtype=np.uint64)
    x = mlp.feature(keys)
    exp = [0.0, 0.0, 1 / 64, 1.5 / 64, (2 + 0.5) / 64, (17 + 1 / 131072) / 64, 63 / 64,
           (63 + (131071 / 131072)) / 64]
    assert np.allclose(x, exp, rtol=0, atol=0)
    # exact in float32 and non-decreasing in the key
    ks = np.sort(gen.mixed_keys(20_000, seed=4))
    xs = mlp.feature(ks)
    assert np.all(np.diff(xs) >= 0)
    assert np.array_equal(xs.astype(np.float32).astype(np.float64), xs)


def test_cdf_targets():
    s = np.array([5, 1, 9, 3], dtype=np.uint64)
    # distinct keys: rank r (from 0) -> (2r + 1) / 2m
    assert np.allclose(mlp.cdf_targets(s), [5 / 8, 1 / 8, 7 / 8, 3 / 8])
    assert np.allclose(mlp.cdf_targets(np.full(7, 3, np.uint64)), 0.5)
    s = np.array([2, 2, 1, 4], dtype=np.uint64)
    assert np.allclose(mlp.cdf_targets(s), [(1 + 3) / 8, (1 + 3) / 8, (0 + 1) / 8, (3 + 4) / 8])


def test_training_learns_uniform_cdf():
    # keys whose feature is uniform on [0, 1): the CDF of the feature is the identity
    u = gen.unif01(8, 1, 4096)
    x = np.floor(u * 64 * 131072) / (64 * 131072)
    t = np.argsort(np.argsort(x, kind="stable"), kind="stable").astype(np.float64) / x.size + 0.5 / x.size
    p0 = gen.mlp_init().astype(np.float64)
    p, losses = mlp.train(p0, x, t, steps=400, batch=512, lr=1e-2)
    assert losses[-1] < 0.1 * losses[0]
    y, _ = mlp.forward(p, np.linspace(0.05, 0.95, 19))
    assert np.max(np.abs(y - np.linspace(0.05, 0.95, 19))) < 0.05


# ------------------------------------------------------------------ learned partition data
from oracle import learned  # noqa: E402


def test_cells_bit_definition():
    keys = np.array([0, 1, 2, 3, 1023, 1024, 1025, 2047, 2048, (1 << 40) + (5 << 30), (1 << 64) - 1], dtype=np.uint64)
    c = learned.cell_of(keys)
    # key 1: m = 0 -> cell 1; key 2: m = 1, next bits 0 -> 1 + 1024; key 3: next bit 1 -> bits '1000000000' = 512
    assert c[0] == 0 and c[1] == 1 and c[2] == 1 + 1024 and c[3] == 1 + 1024 + 512
    assert c[4] == 1 + 1024 * 9 + 1022       # 1023 = 2^10 - 1: m = 9, bits below = 1111111110 (zero-padded)
    assert c[5] == 1 + 1024 * 10 and c[6] == 1 + 1024 * 10 + 1 and c[7] == 1 + 1024 * 10 + 1023
    assert c[8] == 1 + 1024 * 11 and c[9] == 1 + 1024 * 40 + 5
    assert c[10] == learned.NCELL - 1
    # exact cells hold one key value: distinct keys below 2^11 never share a cell
    small = np.arange(0, 2048, dtype=np.uint64)
    assert np.unique(learned.cell_of(small)).size == 2048
    assert all(learned.cell_is_exact(int(x)) for x in learned.cell_of(small))
    assert not learned.cell_is_exact(1 + 1024 * 11)
    # cells are non-decreasing in the key
    ks = np.sort(gen.mixed_keys(5000, seed=9))
    assert np.all(np.diff(learned.cell_of(ks)) >= 0)


def test_heavy_keys_threshold():
    # 1000 samples standing for 100000 rows; capacity 2000 -> heavy above 1000 rows, i.e. > 10 samples
    s = np.concatenate([np.full(11, 7), np.full(10, 9), np.full(50, 5000), np.full(12, 1 << 60),
                        np.arange(100, 1017)]).astype(np.uint64)
    h = learned.heavy_keys(s, 100_000, 2000)
    # any key value counts, in or out of an exact cell; 9 (10 samples) is at the threshold
    assert h.tolist() == [7, 5000, 1 << 60]
    assert not learned.cell_is_exact(int(learned.cell_of(np.array([5000], dtype=np.uint64))[0]))
    # at most MAX_HEAVY, the smallest keys
    many = np.repeat(np.arange(1, learned.MAX_HEAVY + 11, dtype=np.uint64), 3)
    hm = learned.heavy_keys(many, many.size * 1000, 4000)  # 3 samples = 3000 rows > 2000
    assert hm.size == learned.MAX_HEAVY and hm[0] == 1 and hm[-1] == learned.MAX_HEAVY


def test_training_set_is_a_permutation_with_cdf_targets():
    s = np.array([5, 5, 1, 9, 7, 7, 7, 3], dtype=np.uint64)
    x, t = learned.training_set(s, 8, 1 << 20)  # huge capacity: nothing is heavy
    nh = np.sort(s)
    assert sorted(x.tolist()) == sorted(mlp.feature(nh).tolist())
    # targets of key 7 (three copies, four smaller samples): (4 + 7) / 16
    xt = dict(zip(x.tolist(), t.tolist()))
    assert xt[float(mlp.feature(np.array([7], np.uint64))[0])] == 11 / 16
    assert xt[float(mlp.feature(np.array([1], np.uint64))[0])] == 1 / 16
    P = learned.stride_multiplier(8)
    assert np.gcd(P, 8) == 1
    # heavy keys leave the set: with 1000 rows per sample and capacity 3000, a key
    # with two or more samples (>= 2000 rows > 1500) is heavy: 7 and 5 leave
    x2, t2 = learned.training_set(s, 8000, 3000)
    assert x2.size == 3
    # the targets are recomputed over the remaining samples {1, 3, 9}
    assert sorted(t2.tolist()) == [1 / 6, 3 / 6, 5 / 6]


def test_quantile_init_passes_through_its_knots():
    # the network is the interpolation of the CDF through the kept knots; merged
    # knots (equal x) keep the later CDF value
    keys = np.sort(np.concatenate([np.full(50, 3), np.arange(1000, 1300) ** 2, np.full(40, 1 << 40)])).astype(np.uint64)
    p = mlp.quantile_init(keys)
    m = keys.size
    seen = {}
    for i in range(mlp.H + 1):
        k = keys[(i * (m - 1)) // mlp.H]
        x = float(mlp.feature(np.array([k], np.uint64))[0])
        f = (np.searchsorted(keys, k, "left") + np.searchsorted(keys, k, "right")) / (2.0 * m)
        seen[x] = f
    xs = np.array(sorted(seen))
    y, _ = mlp.forward(p, xs)
    assert np.allclose(y, [seen[x] for x in xs], rtol=0, atol=1e-12)
    assert len(seen) < mlp.H + 1  # the repeated keys merged knots
    # between knots the output is linear (the midpoint of two kept knots)
    ym, _ = mlp.forward(p, (xs[:-1] + xs[1:]) / 2)
    fs = np.array([seen[x] for x in xs])
    assert np.allclose(ym, (fs[:-1] + fs[1:]) / 2, atol=1e-12)
    # a single key value: the constant network
    p1 = mlp.quantile_init(np.full(10, 7, dtype=np.uint64))
    assert np.allclose(mlp.forward(p1, np.array([0.0, 0.5, 1.0]))[0], 0.5)


def test_abs_terms_bound_the_gradient():
    # the sum of the row terms' magnitudes is at least the magnitude of their
    # sum (every parameter), and equals it when every term has one sign
    rng = np.random.default_rng(7)
    p = rng.normal(0, 0.5, mlp.N_PARAMS)
    x = rng.random(300)
    t = rng.random(300)
    g = mlp.backward(p, x, t)
    A = mlp.abs_terms(p, x, t)
    assert np.all(A + 1e-15 >= np.abs(g))
    assert np.any(A > 10 * np.abs(g))  # cancellation happens: A is the scale, not g
    y, _ = mlp.forward(p, x)
    g2 = mlp.backward(p, x, y + 1.0)  # every residual -1: the b3 and w3 terms have one sign
    A2 = mlp.abs_terms(p, x, y + 1.0)
    sl = mlp.SLICES
    assert np.allclose(A2[sl["b3"]], np.abs(g2[sl["b3"]])) and np.allclose(A2[sl["w3"]], np.abs(g2[sl["w3"]]))
