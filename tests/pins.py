"""Independent checks that pin the oracle (and, at sizes the oracle cannot
reach, the CUDA path) to what the definitions fix: brute force on tiny
inputs, and invariants that hold at any size.  Nothing here calls the oracle
or the CUDA library."""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1


# ------------------------------------------------------------- brute force
def brute_sort(keys, ptrs):
    """O(n^2) selection sort of (key, ptr) pairs, in plain Python."""
    items = list(zip([int(k) for k in keys], [int(p) for p in ptrs]))
    out = []
    while items:
        best = 0
        for i in range(1, len(items)):
            if items[i] < items[best]:
                best = i
        out.append(items.pop(best))
    return (np.array([k for k, _ in out], dtype=np.uint64), np.array([p for _, p in out], dtype=np.uint32))


def brute_group(keys, ptrs, vals):
    """Per distinct key (ascending): count and sum mod 2^64, one scan per key."""
    keys = [int(k) for k in keys]
    ptrs = [int(p) for p in ptrs]
    distinct = sorted(set(keys))
    counts, sums = [], []
    for d in distinct:
        c = 0
        s = 0
        for k, p in zip(keys, ptrs):
            if k == d:
                c += 1
                if vals is not None:
                    s = (s + int(vals[p])) & M64
        counts.append(c)
        sums.append(s)
    return (np.array(distinct, dtype=np.uint64), np.array(counts, dtype=np.uint64), np.array(sums, dtype=np.uint64))


def brute_topk(keys, ptrs, vals, K):
    """Per distinct key: repeatedly take the largest remaining value (smallest
    ptr on ties) K times."""
    keys = [int(k) for k in keys]
    ptrs = [int(p) for p in ptrs]
    distinct = sorted(set(keys))
    nvalid = np.zeros(len(distinct), np.uint8)
    ov = np.zeros((len(distinct), K), np.uint64)
    op = np.full((len(distinct), K), 0xFFFFFFFF, np.uint32)
    for j, d in enumerate(distinct):
        pool = [(int(vals[p]), p) for k, p in zip(keys, ptrs) if k == d]
        for s in range(K):
            if not pool:
                break
            best = 0
            for i in range(1, len(pool)):
                if pool[i][0] > pool[best][0] or (pool[i][0] == pool[best][0] and pool[i][1] < pool[best][1]):
                    best = i
            v, p = pool.pop(best)
            ov[j, s] = v
            op[j, s] = p
            nvalid[j] = s + 1
    return np.array(distinct, dtype=np.uint64), nvalid, ov, op


# ------------------------------------------------------------- invariants
def check_sorted_kpa(key_col_rows, ptr_base, keys, ptrs):
    """A sorted KPA of rows [ptr_base, ptr_base + n): ordered by (key, ptr),
    every row exactly once, and key[i] = key_col[ptr[i]].  Raises
    AssertionError naming the first violated property."""
    keys = np.asarray(keys, dtype=np.uint64)
    ptrs = np.asarray(ptrs, dtype=np.uint32)
    n = keys.size
    assert ptrs.size == n, "length"
    if n == 0:
        return
    rel = ptrs.astype(np.int64) - int(ptr_base)
    assert rel.min() >= 0 and rel.max() < n, "ptr out of range"
    seen = np.zeros(n, dtype=bool)
    seen[rel] = True
    assert seen.all(), "not a permutation"
    assert np.array_equal(np.asarray(key_col_rows, dtype=np.uint64)[rel], keys), "key does not match its row"
    dk = keys[1:] > keys[:-1]
    eq = keys[1:] == keys[:-1]
    assert np.all(dk | eq), "keys not ascending"
    assert np.all(~eq | (ptrs[1:] > ptrs[:-1])), "equal keys not in ptr order"


def check_group(keys_sorted, vals_by_ptr, ptrs_sorted, out_keys, out_counts, out_sums):
    """Group output invariants: distinct keys ascending, counts sum to n, sums
    add up to the total mod 2^64, and each count matches the run length."""
    n = len(keys_sorted)
    out_keys = np.asarray(out_keys, dtype=np.uint64)
    assert np.all(out_keys[1:] > out_keys[:-1]), "keys not strictly ascending"
    assert int(np.asarray(out_counts, dtype=np.uint64).sum()) == n, "counts do not sum to n"
    if vals_by_ptr is not None:
        tot = int(np.asarray(vals_by_ptr, dtype=np.uint64)[np.asarray(ptrs_sorted, dtype=np.int64)].sum(dtype=np.uint64))
        assert int(np.asarray(out_sums, dtype=np.uint64).sum(dtype=np.uint64)) == tot, "sums do not add up"
    uk, uc = np.unique(np.asarray(keys_sorted, dtype=np.uint64), return_counts=True)
    assert np.array_equal(uk, out_keys), "distinct keys differ"
    assert np.array_equal(uc.astype(np.uint64), np.asarray(out_counts, dtype=np.uint64)), "run lengths differ"


def check_topk(keys, ptrs, vals, K, out_keys, nvalid, ov, op):
    """Top-K invariants: size = min(K, count); kept (value desc, ptr asc);
    every kept value >= every dropped value of the key; pads are (0, ~0)."""
    keys = np.asarray(keys, dtype=np.uint64)
    ptrs = np.asarray(ptrs, dtype=np.int64)
    v = np.asarray(vals, dtype=np.uint64)[ptrs]
    uk, start, cnt = np.unique(keys, return_index=True, return_counts=True)
    order = np.lexsort((ptrs, keys))
    assert np.array_equal(uk, out_keys), "distinct keys differ"
    for j in range(uk.size):
        rows = order[np.nonzero(keys[order] == uk[j])[0]]
        assert int(nvalid[j]) == min(K, int(cnt[j])), "n_valid"
        kept = [(int(ov[j, s]), int(op[j, s])) for s in range(int(nvalid[j]))]
        for a, b in zip(kept, kept[1:]):
            assert a[0] > b[0] or (a[0] == b[0] and a[1] < b[1]), "kept order"
        kept_p = {p for _, p in kept}
        for r in rows:
            assert int(v[r]) == int(np.asarray(vals, dtype=np.uint64)[ptrs[r]])
        dropped = [int(v[r]) for r in rows if int(ptrs[r]) not in kept_p]
        if kept and dropped:
            assert min(x for x, _ in kept) >= max(dropped), "a dropped value beats a kept one"
        for s in range(int(nvalid[j]), K):
            assert int(ov[j, s]) == 0 and int(op[j, s]) == 0xFFFFFFFF, "pad"


def join_cardinality(lkeys, rkeys):
    """sum over keys of count_L(k) * count_R(k)."""
    lu, lc = np.unique(np.asarray(lkeys, dtype=np.uint64), return_counts=True)
    ru, rc = np.unique(np.asarray(rkeys, dtype=np.uint64), return_counts=True)
    common, li, ri = np.intersect1d(lu, ru, return_indices=True)
    return int((lc[li].astype(np.int64) * rc[ri].astype(np.int64)).sum())


def check_join(lkeys_by_ptr, rkeys_by_ptr, out_l, out_r, cardinality):
    """Join invariants: cardinality, key equality of every pair, (key, ptrL,
    ptrR) order, no duplicate pair."""
    out_l = np.asarray(out_l, dtype=np.int64)
    out_r = np.asarray(out_r, dtype=np.int64)
    assert out_l.size == cardinality, "cardinality"
    if cardinality == 0:
        return
    kl = np.asarray(lkeys_by_ptr, dtype=np.uint64)[out_l]
    kr = np.asarray(rkeys_by_ptr, dtype=np.uint64)[out_r]
    assert np.array_equal(kl, kr), "pair keys differ"
    order = np.lexsort((out_r, out_l, kl))
    assert np.array_equal(order, np.arange(out_l.size)), "pair order"
    packed = out_l * (1 << 32) + out_r
    assert np.unique(packed).size == packed.size, "duplicate pair"


def brute_partition(keys, ptrs, bounds):
    """Partition by key ranges in plain Python: one pass over the parts, each
    collecting, in input order, the records whose key lies in its range."""
    keys = [int(k) for k in keys]
    ptrs = [int(p) for p in ptrs]
    bounds = [int(b) for b in bounds]
    ok, op, off = [], [], []
    for j in range(len(bounds) + 1):
        lo = bounds[j - 1] if j > 0 else None
        hi = bounds[j] if j < len(bounds) else None
        off.append(len(ok))
        for k, p in zip(keys, ptrs):
            if (lo is None or k >= lo) and (hi is None or k < hi):
                ok.append(k)
                op.append(p)
    off.append(len(ok))
    return np.array(ok, np.uint64), np.array(op, np.uint32), np.array(off, np.uint64)


def check_partition(keys, ptrs, bounds, out_keys, out_ptrs, offsets):
    """Invariants of a partition at any size: the offsets cut the output into
    one part per range, every part's keys lie in its range, each part lists
    exactly the input records of its range in their input order."""
    keys, ptrs = np.asarray(keys, np.uint64), np.asarray(ptrs, np.uint32)
    bounds, offsets = np.asarray(bounds, np.uint64), np.asarray(offsets, np.uint64)
    assert offsets.size == bounds.size + 2 and offsets[0] == 0 and int(offsets[-1]) == keys.size
    assert np.all(offsets[1:] >= offsets[:-1])
    part = np.searchsorted(bounds, keys, side="right")  # bounds not above the key
    for j in range(bounds.size + 1):
        a, b = int(offsets[j]), int(offsets[j + 1])
        sel = part == j
        assert np.array_equal(out_keys[a:b], keys[sel]), f"part {j} keys"
        assert np.array_equal(out_ptrs[a:b], ptrs[sel]), f"part {j} ptrs"
