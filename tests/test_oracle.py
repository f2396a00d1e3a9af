"""Pins for the oracle: it is checked against brute force, invariants and
closed forms -- never against itself -- and each pin is shown to catch a
planted mistake."""
import numpy as np
import pytest

import gen
import oracle
from tests import pins

M64 = (1 << 64) - 1


def _tiny(n, space, seed, stream=1):
    return gen.tiny_kpa(n, space, seed, stream=stream)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 17, 64])
@pytest.mark.parametrize("space", [1, 4, 0])  # 0: full 64-bit range
def test_sort_matches_brute_force(n, space):
    k, _ = _tiny(n, space, 7 + n)
    p = np.arange(n, dtype=np.uint32)[::-1].copy()  # non-ascending ptrs too
    ok, op = oracle.sort(k, p)
    bk, bp = pins.brute_sort(k, p)
    assert np.array_equal(ok, bk) and np.array_equal(op, bp)


def test_sort_extreme_keys():
    k = np.array([M64, 0, M64, 1, 0, 1 << 63], dtype=np.uint64)
    p = np.arange(6, dtype=np.uint32)
    ok, op = oracle.sort(k, p)
    assert ok.tolist() == [0, 0, 1, 1 << 63, M64, M64]
    assert op.tolist() == [1, 4, 3, 5, 0, 2]


def test_extract_and_sort_invariants_mixed_keys():
    col = gen.mixed_keys(200_003)
    keys, ptrs = oracle.extract(col, 1001, 150_000)
    assert np.array_equal(keys, col[1001:151001])
    assert np.array_equal(ptrs, np.arange(1001, 151001, dtype=np.uint32))
    sk, sp = oracle.sort(keys, ptrs)
    pins.check_sorted_kpa(col[1001:151001], 1001, sk, sp)
    # numpy's stable sort of the keys alone gives the same order (ptrs ascend)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(sk, keys[order]) and np.array_equal(sp, ptrs[order])


def test_merge_is_sorted_concatenation():
    col = gen.mixed_keys(50_000, seed=99)
    runs = []
    bounds = [0, 1, 7000, 7001, 30000, 50000]
    for a, b in zip(bounds, bounds[1:]):
        runs.append(oracle.sort(*oracle.extract(col, a, b - a)))
    mk, mp = oracle.merge(runs)
    pins.check_sorted_kpa(col, 0, mk, mp)
    tk, tp = _tiny(40, 3, 5)
    r1 = oracle.sort(tk[:25], np.arange(25, dtype=np.uint32))
    r2 = oracle.sort(tk[25:], np.arange(25, 40, dtype=np.uint32))
    mk, mp = oracle.merge([r1, r2])
    bk, bp = pins.brute_sort(tk, np.arange(40, dtype=np.uint32))
    assert np.array_equal(mk, bk) and np.array_equal(mp, bp)


@pytest.mark.parametrize("vb", [4, 8])
@pytest.mark.parametrize("n,space", [(0, 4), (1, 4), (64, 4), (200, 1), (300, 50)])
def test_group_matches_brute_force(vb, n, space):
    k, _ = _tiny(n, space, 11 + n)
    v = gen.uniform(3, 4, n, 0, 0, np.uint64 if vb == 8 else np.uint32)  # full range: sums wrap
    p = np.arange(n, dtype=np.uint32)
    got = oracle.group_sum_count(k, p, v)
    exp = pins.brute_group(k, p, v)
    for a, b in zip(got, exp):
        assert np.array_equal(a, b)


def test_group_count_only_and_invariants_tumbling_window():
    w = gen.tumbling_window(1_000_000)
    keys, ptrs = oracle.sort(*oracle.extract(w["keys"], 0, 1_000_000))
    ok, oc, osum = oracle.group_sum_count(keys, ptrs, w["vals"])
    pins.check_group(keys, w["vals"], ptrs, ok, oc, osum)
    # distinct-key count of n uniform draws over 2^20 ids: mean 2^20 (1 - (1 - 2^-20)^n)
    N = float(1 << 20)
    mean = N * (1.0 - (1.0 - 1.0 / N) ** 1e6)
    var = N * (1 - 1 / N) ** 1e6 + N * N * (1 - 2 / N) ** 1e6 - N * N * (1 - 1 / N) ** 2e6
    assert abs(ok.size - mean) < 6.0 * np.sqrt(var)
    _, oc2, os2 = oracle.group_sum_count(keys, ptrs, None)
    assert np.array_equal(oc2, oc) and not os2.any()


@pytest.mark.parametrize("K", [1, 3, 5])
@pytest.mark.parametrize("n,space,vspan", [(0, 4, 8), (1, 4, 8), (64, 4, 4), (100, 7, 3), (150, 1, 1000)])
def test_topk_matches_brute_force(K, n, space, vspan):
    k, _ = _tiny(n, space, 21 + n)
    v = gen.uniform(9, 9, n, 0, vspan, np.uint64)  # small value span: many value ties
    p = np.arange(n, dtype=np.uint32)
    got = oracle.topk(k, p, v, K)
    exp = pins.brute_topk(k, p, v, K)
    for a, b in zip(got, exp):
        assert np.array_equal(a, b)
    pins.check_topk(k, p, v, K, *got)


@pytest.mark.parametrize("nl,nr,space", [(0, 5, 3), (5, 0, 3), (30, 40, 4), (50, 50, 1000), (64, 64, 1)])
def test_join_matches_nested_loop(nl, nr, space):
    lk, _ = _tiny(nl, space, 31 + nl)
    rk, _ = _tiny(nr, space, 41 + nr, stream=2)
    lp = np.arange(nl, dtype=np.uint32)
    rp = np.arange(nr, dtype=np.uint32)
    a = oracle.join(lk, lp, rk, rp)
    b = oracle.join_nested(lk, lp, rk, rp)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    pins.check_join(lk, rk, a[0], a[1], pins.join_cardinality(lk, rk))


def test_join_cardinality_medium():
    s = gen.join_streams(20_000, key_space=1 << 12)
    lk, rk = s["L"]["keys"], s["R"]["keys"]
    ol, orr = oracle.join(lk, np.arange(lk.size, dtype=np.uint32), rk, np.arange(rk.size, dtype=np.uint32))
    pins.check_join(lk, rk, ol, orr, pins.join_cardinality(lk, rk))


def test_window_ranges_binary_search():
    ts = np.sort(gen.uniform(5, 5, 5000, 0, 20000, np.uint64))
    starts = np.array([0, 1, 250, 9999, 19999, 20000, 30000], dtype=np.uint64)
    b, e = oracle.window_ranges(ts, starts, 1000)
    assert np.array_equal(b, np.searchsorted(ts, starts, side="left"))
    assert np.array_equal(e, np.searchsorted(ts, starts + 1000, side="left"))
    ts32 = np.arange(100, dtype=np.uint32)
    b, e = oracle.window_ranges(ts32, np.array([10, 95], np.uint64), 25)
    assert b.tolist() == [10, 95] and e.tolist() == [35, 100]


# ------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_sort_mistakes():
    col = gen.mixed_keys(5000, seed=3)
    sk, sp = oracle.sort(*oracle.extract(col, 0, 5000))
    pins.check_sorted_kpa(col, 0, sk, sp)
    mutants = []
    a, b = sk.copy(), sp.copy(); a[[10, 11]] = a[[11, 10]]; b[[10, 11]] = b[[11, 10]]; mutants.append((a, b))  # swap
    a, b = sk.copy(), sp.copy(); b[5] = b[6]; mutants.append((a, b))  # duplicate ptr
    a, b = sk[:-1].copy(), sp[:-1].copy(); mutants.append((a, b))  # dropped element
    a, b = sk.copy(), sp.copy(); a[100] += np.uint64(1); mutants.append((a, b))  # wrong key
    dup = np.flatnonzero(sk[1:] == sk[:-1])[0]
    a, b = sk.copy(), sp.copy(); b[[dup, dup + 1]] = b[[dup + 1, dup]]; mutants.append((a, b))  # tie order
    for a, b in mutants:
        with pytest.raises(AssertionError):
            pins.check_sorted_kpa(col, 0, a, b)


def test_pins_catch_planted_group_mistakes():
    w = gen.tumbling_window(20_000, key_bits=10)
    keys, ptrs = oracle.sort(*oracle.extract(w["keys"], 0, 20_000))
    ok, oc, osum = oracle.group_sum_count(keys, ptrs, w["vals"])
    bad = [
        (ok, oc, osum + np.uint64(1) * (np.arange(ok.size) == 3)),   # a sum off by one
        (ok, oc - np.uint64(1) * (np.arange(ok.size) == 0), osum),   # a dropped record
        (ok[::-1], oc[::-1], osum[::-1]),                            # wrong order
    ]
    for k2, c2, s2 in bad:
        with pytest.raises(AssertionError):
            pins.check_group(keys, w["vals"], ptrs, k2, c2, s2)


def test_pins_catch_planted_topk_and_join_mistakes():
    k, _ = _tiny(300, 20, 77)
    v = gen.uniform(2, 2, 300, 0, 50, np.uint64)
    p = np.arange(300, dtype=np.uint32)
    ok, nv, ov, op = oracle.topk(k, p, v, 3)
    ov2 = ov.copy(); ov2[0, [0, 1]] = ov2[0, [1, 0]]
    with pytest.raises(AssertionError):
        pins.check_topk(k, p, v, 3, ok, nv, ov2, op)
    nv2 = nv.copy(); nv2[1] -= 1
    with pytest.raises(AssertionError):
        pins.check_topk(k, p, v, 3, ok, nv2, ov, op)
    lk, _ = _tiny(80, 6, 1)
    rk, _ = _tiny(80, 6, 2, stream=3)
    ol, orr = oracle.join(lk, p[:80], rk, p[:80])
    card = pins.join_cardinality(lk, rk)
    with pytest.raises(AssertionError):
        pins.check_join(lk, rk, ol[:-1], orr[:-1], card)
    o2 = orr.copy(); o2[0] = (o2[0] + 1) % 80
    with pytest.raises(AssertionError):
        pins.check_join(lk, rk, ol, o2, card)


# ------------------------------------------------------------------ Materialize, KeySwap, Select, Median, Unique
def test_materialize_is_the_gather_by_pointer():
    rng = np.random.default_rng(3)
    for dtype in (np.uint32, np.uint64):
        col = rng.integers(0, np.iinfo(dtype).max, 5000, dtype=dtype)
        ptrs = rng.permutation(5000).astype(np.uint32)[:3000]
        got = oracle.materialize(ptrs, col)
        assert got.dtype == dtype and [int(x) for x in got] == [int(col[p]) for p in ptrs]


def test_keyswap_then_sort_orders_by_the_new_key():
    # KeySwap: the KPA's resident key becomes another column of the same rows
    col_a, _ = gen.tiny_kpa(2000, 50, seed=11)
    col_b = gen.uniform(11, 2, 2000, 0, 1 << 30, np.uint64)
    k, p = oracle.sort(*oracle.extract(col_a, 0, 2000))
    k2 = oracle.materialize(p, col_b)
    sk, sp = oracle.sort(k2, p)
    pins.check_sorted_kpa(col_b, 0, sk, sp)


@pytest.mark.parametrize("lo,hi", [(0, 0), (3, 9), (0, 1 << 64 - 1), (7, 8)])
def test_select_matches_brute_force(lo, hi):
    keys, _ = gen.tiny_kpa(3000, 40, seed=lo + 5)
    vals = gen.uniform(6, 1, 3000, 0, 12, np.uint64)
    ptrs = np.arange(3000, dtype=np.uint32)[::-1].copy()
    ok, op = oracle.select(keys, ptrs, vals, lo, hi)
    brute = [(int(keys[i]), int(ptrs[i])) for i in range(3000) if lo <= int(vals[ptrs[i]]) < hi]
    assert list(zip(ok.tolist(), op.tolist())) == brute


@pytest.mark.parametrize("n,space,vspan", [(1, 3, 5), (700, 9, 4), (5000, 300, 1000), (4000, 2, 0)])
def test_median_unique_matches_brute_force(n, space, vspan):
    import statistics
    keys, _ = gen.tiny_kpa(n, space, seed=n)
    vals = gen.uniform(8, 2, n, 0, vspan, np.uint64)
    ptrs = np.arange(n, dtype=np.uint32)
    uk, med, uni = oracle.median_unique(keys, ptrs, vals)
    groups = {}
    for i in range(n):
        groups.setdefault(int(keys[i]), []).append(int(vals[i]))
    assert uk.tolist() == sorted(groups)
    for j, k in enumerate(sorted(groups)):
        v = groups[k]
        assert med[j] == statistics.median_low(v)          # lower median
        assert uni[j] == len(set(v))
        assert sum(x <= med[j] for x in v) >= (len(v) + 1) // 2 and sum(x >= med[j] for x in v) >= len(v) // 2 + 1


def test_pins_catch_planted_median_mistakes():
    import statistics
    vals = [5, 1, 9, 9, 2, 7]
    assert statistics.median_low(vals) == 5
    # an upper median, or a median over unsorted values, fails the pin
    assert sorted(vals)[len(vals) // 2] != statistics.median_low(vals)
    assert vals[(len(vals) - 1) // 2] != statistics.median_low(vals)


def test_oracle_reproduces_the_worked_example():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))
    keys = np.array(g["keys"], np.uint64)
    vals = np.array(g["values"], np.uint64)
    k, p = oracle.sort(*oracle.extract(keys, 0, keys.size))
    assert k.tolist() == g["sorted"]["keys"] and p.tolist() == g["sorted"]["ptrs"]
    uk, uc, us = oracle.group_sum_count(k, p, vals)
    assert [uk.tolist(), uc.tolist(), us.tolist()] == [g["sum_count"][x] for x in ("keys", "counts", "sums")]
    tk, tn, tv, tp = oracle.topk(k, p, vals, 2)
    t = g["top2"]
    assert tk.tolist() == t["keys"] and tn.tolist() == t["nvalid"] and tv.tolist() == t["vals"] and tp.tolist() == t["ptrs"]
    mk, mm, mu = oracle.median_unique(k, p, vals)
    m = g["median_unique"]
    assert mk.tolist() == m["keys"] and mm.tolist() == m["median"] and mu.tolist() == m["unique"]
    j = g["join"]
    lk, lp = oracle.sort(*oracle.extract(keys, 0, 4))
    rk, rp = oracle.sort(*oracle.extract(keys, 4, 4))
    ol, orr = oracle.join(lk, lp, rk, rp)
    assert ol.tolist() == j["ptr_l"] and orr.tolist() == j["ptr_r"]
    sk, sp = oracle.select(k, p, vals, 20, 45)
    assert sk.tolist() == g["select_20_45"]["keys"] and sp.tolist() == g["select_20_45"]["ptrs"]
    w = g["window_2_4"]
    b, e = oracle.window_ranges(np.array(w["ts"], np.uint64), np.array([w["start"]], np.uint64), w["len"])
    assert [int(b[0]), int(e[0])] == w["rows"]
    q = g["partition_3_6"]
    pk, pp, po = oracle.partition(keys, np.arange(keys.size, dtype=np.uint32), np.array(q["bounds"], np.uint64))
    assert pk.tolist() == q["keys"] and pp.tolist() == q["ptrs"] and po.tolist() == q["offsets"]


# ------------------------------------------------------------- partition (Table 2)
@pytest.mark.parametrize("n", [0, 1, 5, 64])
@pytest.mark.parametrize("bounds", [[], [3], [2, 2, 9], [0, 1 << 63, M64]])
def test_partition_matches_brute_force(n, bounds):
    k, _ = _tiny(n, 12, 40 + n)
    p = gen.uniform(40, 3, n, 0, 50, np.uint32)  # arbitrary, repeated ptrs: parts keep input order
    b = np.array(bounds, np.uint64)
    ok, op, off = oracle.partition(k, p, b)
    bk, bp, boff = pins.brute_partition(k, p, b)
    assert np.array_equal(ok, bk) and np.array_equal(op, bp) and np.array_equal(off, boff)


def test_partition_invariants_and_planted_mistakes():
    n = 50_000
    col = gen.mixed_keys(n, seed=12)
    ptrs = np.arange(n, dtype=np.uint32)
    bounds = np.sort(gen.mixed_keys(300, seed=13))
    ok, op, off = oracle.partition(col, ptrs, bounds)
    pins.check_partition(col, ptrs, bounds, ok, op, off)
    big = [j for j in range(1, bounds.size) if off[j + 1] - off[j] >= 2]
    j0, j1 = big[0], big[1]
    a = op.copy(); a[[int(off[j0]), int(off[j0]) + 1]] = a[[int(off[j0]) + 1, int(off[j0])]]  # order in a part
    b = off.copy(); b[j1] += np.uint64(1)                                                  # a row in the wrong part
    c = ok.copy(); c[int(off[j1])] = bounds[j1]                                            # a key out of its range
    for kk, pp, oo in ((ok, a, off), (ok, op, b), (c, op, off)):
        with pytest.raises(AssertionError):
            pins.check_partition(col, ptrs, bounds, kk, pp, oo)
    # the part sizes are the numbers of keys per range, counted directly
    sizes = np.diff(off)
    assert int(sizes[0]) == int(np.sum(col < bounds[0]))
    assert int(sizes[100]) == int(np.sum((col >= bounds[99]) & (col < bounds[100])))
    assert int(sizes[300]) == int(np.sum(col >= bounds[299]))
