"""The seeded generators: deterministic, thread-count independent, and drawing
the stated distributions."""
import numpy as np

import gen


def test_deterministic_and_thread_independent(monkeypatch):
    a = gen.mixed_keys(300_000)
    monkeypatch.setattr(gen, "_threads", lambda: 1)
    b = gen.mixed_keys(300_000)
    assert np.array_equal(a, b)
    # a prefix of a longer draw equals the shorter draw
    c = gen.mixed_keys(100_000)
    assert np.array_equal(a[:100_000], c)


def test_zipf_head_probability():
    n_ids, s = 1 << 24, 1.1
    z = gen.zipf(1, 2, 2_000_000, s, n_ids)
    assert z.min() >= 1 and z.max() <= n_ids
    r = np.arange(1, 200_001, dtype=np.float64)
    # generalized harmonic number: partial sum plus the integral tail
    Hn = (r ** -s).sum() + ((200_000.5) ** (1 - s) - (n_ids + 0.5) ** (1 - s)) / (s - 1)
    for k in (1, 2, 10):
        p = k ** -s / Hn
        emp = (z == k).mean()
        assert abs(emp - p) < 5 * np.sqrt(p * (1 - p) / z.size)


def test_mixture_shape():
    k = gen.mixed_keys(1_000_000)
    small = (k >= 1) & (k <= (1 << 24))
    assert abs(small.mean() - 0.7) < 0.01          # Zipf part (lognormal rarely lands below 2^24)
    big = np.log(k[k > (1 << 24)].astype(np.float64))
    assert abs(np.median(big) - 30.0) < 0.2        # lognormal median exp(mu)


def test_uniform_range_and_window_sizes():
    w = gen.tumbling_window(100_000)
    assert w["keys"].max() < (1 << 20) and w["vals"].max() < (1 << 16)
    b = gen.batched_windows(512, 8)
    sizes = np.diff(b["offsets"].astype(np.int64))
    assert sizes.min() >= 1000 and sizes.max() <= 4_000_000
    assert abs(np.log(np.median(sizes)) - 10.4) < 0.2
