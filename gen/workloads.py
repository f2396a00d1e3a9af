"""Workload recipes: the synthetic stand-ins for the paper's 64-bit random
integer streams (Sec. 7, "Benchmarks"), at the five workload shapes of the
KPA grouping path.  Every function takes a size so tests can draw scaled-down
versions of the same distributions.

Streams (draw streams of the counter-based generator) are fixed per column so
that a column never depends on another column's size.
"""
from __future__ import annotations

import numpy as np

from . import SEED_BASE, lognormal_sizes, unif01, uniform, zipf, zipf_lognormal_mix

__all__ = ["tumbling_window", "mixed_keys", "batched_windows", "join_streams", "tiny_kpa", "mlp_init", "ad_events",
           "SEED_TUMBLING", "SEED_MIXED", "SEED_BATCHED", "SEED_JOIN", "SEED_ADS"]

SEED_TUMBLING = SEED_BASE + 1
SEED_MIXED = SEED_BASE + 2
SEED_BATCHED = SEED_BASE + 3
SEED_JOIN = SEED_BASE + 4
SEED_ADS = SEED_BASE + 6


def tumbling_window(n: int = 1_000_000, key_bits: int = 20, seed: int = SEED_TUMBLING):
    """One tumbling window of 3-column records: key u64 ~ U[0, 2^key_bits),
    value u32 ~ U[0, 2^16), ts u32 = row index (strictly increasing)."""
    keys = uniform(seed, 1, n, 0, 1 << key_bits, np.uint64)
    vals = uniform(seed, 2, n, 0, 1 << 16, np.uint32)
    ts = np.arange(n, dtype=np.uint32)
    return {"keys": keys, "vals": vals, "ts": ts}


def mixed_keys(n: int = 256_000_000, seed: int = SEED_MIXED, zipf_frac: float = 0.7, s: float = 1.1,
               n_ids: int = 1 << 24, mu: float = 30.0, sigma: float = 4.0, out=None, hashed: bool = False) -> np.ndarray:
    """Skewed 64-bit keys: 70% Zipf(1.1) ranks over 2^24 ids, 30%
    floor(lognormal(30, 4)) redrawn until below 2^64.  hashed: the Zipf ranks
    pass through mix64 (the robustness variant: same multiplicities, keys
    spread over all 64 bits)."""
    return zipf_lognormal_mix(seed, n, zipf_frac, s, n_ids, mu, sigma, out=out, hashed=hashed)


def batched_windows(n_windows: int = 4096, n_streams: int = 64, seed: int = SEED_BATCHED,
                    size_mu: float = 10.4, size_sigma: float = 1.5, size_lo: int = 1000,
                    size_hi: int = 4_000_000, s: float = 1.0, n_ids: int = 10_000_000):
    """Many uneven tumbling windows laid end to end: window sizes
    clamp(lognormal(size_mu, size_sigma), size_lo, size_hi); keys Zipf(s) ranks
    over n_ids; values u64 uniform.  Window w belongs to stream w % n_streams.
    Returns row offsets (n_windows + 1), keys, values, stream ids."""
    sizes = lognormal_sizes(seed, 1, n_windows, size_mu, size_sigma, size_lo, size_hi)
    offsets = np.zeros(n_windows + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    n = int(offsets[-1])
    keys = zipf(seed, 2, n, s, n_ids)
    vals = uniform(seed, 3, n, 0, 0, np.uint64)
    stream = (np.arange(n_windows, dtype=np.uint32) % n_streams).astype(np.uint32)
    return {"offsets": offsets, "keys": keys, "vals": vals, "stream": stream}


def join_streams(n: int = 128_000_000, key_space: int = 1 << 24, seed: int = SEED_JOIN):
    """Two streams L and R of 3-column records: key u64 ~ U[0, key_space),
    ts u64 = row index, payload u64 (never read by the join)."""
    out = {}
    for side, base in (("L", 10), ("R", 20)):
        out[side] = {
            "keys": uniform(seed, base + 1, n, 0, key_space, np.uint64),
            "ts": np.arange(n, dtype=np.uint64),
        }
    return out


def tiny_kpa(n: int, key_space: int, seed: int, stream: int = 1, val_span: int = 16, val_bytes: int = 8):
    """Small inputs with many duplicates for brute-force checks."""
    keys = uniform(seed, stream, n, 0, key_space, np.uint64)
    vals = uniform(seed, stream + 100, n, 0, val_span, np.uint64 if val_bytes == 8 else np.uint32)
    return keys, vals


def mlp_init(seed: int = SEED_MIXED, hidden: int = 32) -> np.ndarray:
    """Initial weights of the 1-hidden-hidden-1 network as float32 (flat layout
    W1, b1, W2 row-major, b2, w3, b3).  W1 ~ U(-sqrt 6, sqrt 6); b1 = -W1 * c
    with c ~ U[0, 1), so each first-layer unit turns on somewhere in [0, 1);
    W2, w3 ~ U(-sqrt(6/hidden), sqrt(6/hidden)); b2 = 0; b3 = 0.5."""
    h = hidden
    u = unif01(seed, 50, 2 * h + h * h + h)
    w1 = (2.0 * u[:h] - 1.0) * np.sqrt(6.0)
    c = u[h:2 * h]
    w2 = (2.0 * u[2 * h:2 * h + h * h] - 1.0) * np.sqrt(6.0 / h)
    w3 = (2.0 * u[2 * h + h * h:] - 1.0) * np.sqrt(6.0 / h)
    w1 = w1.astype(np.float32)
    b1 = (-(w1.astype(np.float64)) * c).astype(np.float32)
    p = np.concatenate([w1, b1, w2.astype(np.float32), np.zeros(h, np.float32), w3.astype(np.float32),
                        np.array([0.5], np.float32)])
    return p.astype(np.float32)


def ad_events(n: int = 64_000_000, n_ads: int = 1000, n_campaigns: int = 100, events_per_s: float = 1e7,
              seed: int = SEED_ADS):
    """A 7-column ad-event stream with the shape of an advertising-analytics
    benchmark (our own seeded draws, not any benchmark's generator): user,
    page and ad ids, ad type (0..4), event type (0 view, 1 click, 2
    purchase), event time in ns (increasing, events_per_s on average) and an
    IPv4 address; plus the ad -> campaign table (each ad in one of
    n_campaigns campaigns)."""
    gaps = np.floor(-np.log1p(-unif01(seed, 8, n)) * (1e9 / events_per_s)).astype(np.uint64)
    cols = {
        "user_id": uniform(seed, 1, n, 0, 0, np.uint64),
        "page_id": uniform(seed, 2, n, 0, 0, np.uint64),
        "ad_id": uniform(seed, 3, n, 0, n_ads, np.uint64),
        "ad_type": uniform(seed, 4, n, 0, 5, np.uint64),
        "event_type": uniform(seed, 5, n, 0, 3, np.uint64),
        "event_time": np.cumsum(gaps, dtype=np.uint64),
        "ip": uniform(seed, 6, n, 0, 1 << 32, np.uint64),
    }
    campaign_of_ad = uniform(seed, 7, n_ads, 0, n_campaigns, np.uint64)
    return cols, campaign_of_ad
