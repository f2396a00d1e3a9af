"""The window pipelines on the GPU against the oracle, window by window:
many uneven tumbling windows (per-key count, sum and top-3 in each; both
schedules) and the sliding-window temporal join over panes (key columns in
page-locked host memory).  Small cases check every window; the full-size
workloads check sampled windows."""
import numpy as np
import pytest
import torch

import gen
import oracle
from tests.gpu_util import cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import pipeline
    return pipeline


def _oracle_window(keys, vals, lo, m, K):
    k, p = oracle.sort(*oracle.extract(keys, lo, m))
    uk, uc, us = oracle.group_sum_count(k, p, vals)
    tk, tn, tv, tp = oracle.topk(k, p, vals, K)
    assert np.array_equal(tk, uk)
    return uk, uc, us, tn, tv, tp


def _check_window(res, w, keys, vals, offsets, K):
    got = res.window(w)
    exp = _oracle_window(keys, vals, int(offsets[w]), int(offsets[w + 1] - offsets[w]), K)
    for g, e in zip(got, exp):
        assert np.array_equal(g, e.reshape(g.shape)), f"window {w}"


@pytest.mark.parametrize("schedule", ["batched", "loop"])
def test_batched_windows_every_window(P, schedule):
    b = gen.batched_windows(48, 8, size_hi=60_000)
    keys, vals, off = b["keys"], b["vals"], b["offsets"]
    res = P.batched_windows(cuda(keys), cuda(vals), off, K=3, schedule=schedule)
    for w in range(off.size - 1):
        _check_window(res, w, keys, vals, off, 3)


def test_batched_windows_edge_cases(P):
    # one window; an empty window; windows that are one row; a heavy key
    keys = np.concatenate([np.full(5000, 7, np.uint64), gen.uniform(3, 1, 3000, 0, 100, np.uint64)])
    vals = gen.uniform(3, 2, keys.size, 0, 0, np.uint64)
    for off in (np.array([0, keys.size], np.uint64), np.array([0, 1, 1, 2, 4000, keys.size], np.uint64)):
        for schedule in ("batched", "loop"):
            res = P.batched_windows(cuda(keys), cuda(vals), off, K=3, schedule=schedule)
            for w in range(off.size - 1):
                _check_window(res, w, keys, vals, off, 3)


def test_batched_windows_falls_back_when_keys_use_window_bits(P):
    b = gen.batched_windows(16, 4, size_hi=20_000)
    keys, vals, off = b["keys"].copy(), b["vals"], b["offsets"]
    keys[5] |= np.uint64(1) << np.uint64(63)
    res = P.batched_windows(cuda(keys), cuda(vals), off, K=3, schedule="batched")
    assert res.shift == 64  # the loop ran
    for w in (0, 15):
        _check_window(res, w, keys, vals, off, 3)


def test_batched_windows_full_size_sampled(P):
    # 4096 windows (64 streams), sizes lognormal(10.4, 1.5) in [1K, 4M],
    # keys Zipf(1.0) over 10M: the batched schedule, sampled windows checked
    b = gen.batched_windows()
    keys, vals, off = b["keys"], b["vals"], b["offsets"]
    res = P.batched_windows(cuda(keys), cuda(vals), off, K=3, schedule="batched")
    sizes = np.diff(off)
    for w in {0, int(np.argmax(sizes)), int(np.argmin(sizes)), 4095}:
        _check_window(res, w, keys, vals, off, 3)
    # every window's counts add up to its size
    cnt = res.counts[: int(res.end[-1])].cpu().numpy()
    per = np.add.reduceat(cnt, res.begin.astype(np.int64)) if cnt.size else cnt
    assert np.array_equal(per.astype(np.uint64), sizes)


def _pinned(a):
    t = torch.from_numpy(a.astype(np.int64, copy=False).view(np.int64)).pin_memory()
    return t.view(torch.uint64)


def _check_join(res, i, w, lcol, rcol, window, stride):
    gl, gr = res.window(i)
    lo = w * stride
    lk, lp = oracle.sort(*oracle.extract(lcol, lo, window))
    rk, rp = oracle.sort(*oracle.extract(rcol, lo, window))
    ol, orr = oracle.join(lk, lp, rk, rp)
    assert np.array_equal(gl, ol) and np.array_equal(gr, orr), f"window {w}"


def test_sliding_join_every_window(P):
    s = gen.join_streams(3_000_000, key_space=1 << 20)
    lcol, rcol = s["L"]["keys"], s["R"]["keys"]
    res, wl = P.sliding_join(_pinned(lcol), _pinned(rcol), 3_000_000, pair_cap=1 << 21)
    assert wl == list(range(9))
    for i, w in enumerate(wl):
        _check_join(res, i, w, lcol, rcol, 1_000_000, 250_000)


def test_sliding_join_full_size_sampled(P):
    # 2 x 128M rows in page-locked host memory, 509 windows of 1M rows
    s = gen.join_streams()
    lcol, rcol = s["L"]["keys"], s["R"]["keys"]
    res, wl = P.sliding_join(_pinned(lcol), _pinned(rcol), lcol.size)
    assert len(wl) == 509
    for w in (0, 254, 508):
        _check_join(res, w, w, lcol, rcol, 1_000_000, 250_000)
    # pair counts near 10^12 / 2^24 per window
    assert abs(float(res.npairs.mean()) - 1e12 / (1 << 24)) < 0.02 * 1e12 / (1 << 24)


def test_ad_campaign_counts_chain(P):
    # Extract -> Select(view) -> KeySwap(ad -> campaign) -> Sort -> count, per
    # 100 ms window, against the oracle's steps and a direct count
    n = 3_000_000
    cols, camp = gen.ad_events(n, events_per_s=1e7)
    dcols = {k: cuda(v) for k, v in cols.items()}
    res = P.ad_campaign_counts(dcols, cuda(camp), 100_000_000)
    ts, et, ad = cols["event_time"], cols["event_type"], cols["ad_id"]
    assert len(res) == int(ts[-1] // 100_000_000) + 1
    for w, ck, cc in res:
        lo, hi = np.searchsorted(ts, [w * 100_000_000, (w + 1) * 100_000_000])
        k, p = oracle.extract(et, int(lo), int(hi - lo))
        sk, sp = oracle.select(k, p, et, 0, 1)
        ads = oracle.materialize(sp, ad)
        c = oracle.materialize(ads.astype(np.uint32), camp)
        ok, oc, _ = oracle.group_sum_count(*oracle.sort(c, sp), None)
        assert np.array_equal(ck, ok) and np.array_equal(cc, oc)
        direct = np.bincount(camp[ad[lo:hi][et[lo:hi] == 0]].astype(np.int64), minlength=100)
        assert np.array_equal(direct[direct > 0], oc)


def test_keyswap_lookup_misses(P):
    from paper_1901_01328_b300 import sbh
    col = np.array([0, 5, 2, 9, 1], np.uint64)
    table = np.array([10, 11, 12, 13, 14, 15], np.uint64)
    ptrs = np.array([4, 3, 2, 1, 0], np.uint32)
    out = torch.empty(5, dtype=torch.uint64, device="cuda")
    miss = torch.zeros(1, dtype=torch.uint64, device="cuda")
    sbh.sbh_kpa_keyswap_lookup(cuda(ptrs), cuda(col), cuda(table), out, miss)
    assert out.cpu().numpy().tolist() == [11, 2**64 - 1, 12, 15, 10] and int(miss.item()) == 1


def test_sliding_join_batched_equals_loop_schedule(P):
    s = gen.join_streams(2_000_000, key_space=1 << 18)
    lcol, rcol = s["L"]["keys"], s["R"]["keys"]
    a, wa = P.sliding_join(cuda(lcol), cuda(rcol), 2_000_000, window=500_000, stride=125_000, schedule="batched")
    b, wb = P.sliding_join(cuda(lcol), cuda(rcol), 2_000_000, window=500_000, stride=125_000, schedule="loop",
                           pair_cap=1 << 21)
    assert wa == wb == list(range(13))
    for i in range(13):
        ga, gb = a.window(i), b.window(i)
        assert np.array_equal(ga[0], gb[0]) and np.array_equal(ga[1], gb[1])
    _check_join(a, 12, 12, lcol, rcol, 500_000, 125_000)


def _sorted_runs(col, starts, lens):
    out = []
    for st, ln in zip(starts, lens):
        out.append(oracle.sort(*oracle.extract(col, st, ln)))
    return out


def test_merge_segments_parity():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import sbh
    # A and B: concatenations of sorted runs of uneven length (empty ones,
    # ragged tails, one long run), merged pairwise, in a shuffled order of
    # segments that also reuse runs
    col = gen.mixed_keys(3_000_000, seed=41)
    lens = [0, 1, 2047, 2048, 2049, 100_003, 5, 700_000, 0, 31_111]
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    runs = _sorted_runs(col, starts, lens)
    ak = np.concatenate([r[0] for r in runs]); ap = np.concatenate([r[1] for r in runs])
    segs = [(0, 1), (2, 3), (4, 5), (7, 6), (9, 3), (8, 8), (5, 5), (1, 7)]
    a_start = [int(starts[i]) for i, _ in segs]; a_len = [lens[i] for i, _ in segs]
    b_start = [int(starts[j]) for _, j in segs]; b_len = [lens[j] for _, j in segs]
    total = sum(a_len) + sum(b_len)
    ok = torch.empty(total, dtype=torch.uint64, device="cuda")
    op = torch.empty(total, dtype=torch.uint32, device="cuda")
    A = (cuda(ak), cuda(ap))
    sbh.sbh_kpa_merge_segments(A, A, a_start, a_len, b_start, b_len, ok, op)
    gk, gp = ok.cpu().numpy(), op.cpu().numpy()
    o = 0
    for (i, j), la, lb in zip(segs, a_len, b_len):
        ek, ep = oracle.merge([runs[i], runs[j]])
        assert np.array_equal(gk[o:o + la + lb], ek) and np.array_equal(gp[o:o + la + lb], ep), (i, j)
        o += la + lb


@pytest.mark.parametrize("reuse", [False, True])
def test_join_segments_parity(reuse):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import sbh
    lcol = gen.uniform(42, 1, 900_000, 0, 1 << 12, np.uint64)
    rcol = gen.uniform(42, 2, 800_000, 0, 1 << 12, np.uint64)
    l_lens = [0, 5, 4097, 300_000, 1, 595_897]
    r_specs = [(0, 10), (0, 800_000), (100, 4096), (0, 0), (700_000, 100_000), (250_000, 300_000)]  # overlapping
    l_off = np.concatenate([[0], np.cumsum(l_lens)]).astype(np.int64)
    Lr = _sorted_runs(lcol, l_off[:-1], l_lens)
    Rr = _sorted_runs(rcol, [a for a, _ in r_specs], [b for _, b in r_specs])
    lk = np.concatenate([r[0] for r in Lr]); lp = np.concatenate([r[1] for r in Lr])
    # R segments are sorted runs laid out where their specs say (overlapping specs share rows)
    rk, rp = oracle.sort(*oracle.extract(rcol, 0, 800_000))
    r_start, r_len = [], []
    rk_all, rp_all = [rk], [rp]
    base = 800_000
    for (a, b), run in zip(r_specs, Rr):
        r_start.append(base); r_len.append(b)
        rk_all.append(run[0]); rp_all.append(run[1])
        base += b
    RK, RP = np.concatenate(rk_all), np.concatenate(rp_all)
    npairs = torch.empty(1, dtype=torch.uint64, device="cuda")
    seg = torch.empty(len(l_lens) + 1, dtype=torch.uint64, device="cuda")
    L, R = (cuda(lk), cuda(lp)), (cuda(RK), cuda(RP))
    scr = sbh.sbh_join_segments(L, l_off, R, r_start, r_len, None, None, 0, npairs, seg)
    total = int(npairs.item())
    ol = torch.empty(max(1, total), dtype=torch.uint32, device="cuda")
    orr = torch.empty(max(1, total), dtype=torch.uint32, device="cuda")
    # reuse: the pairs from the first call's counts, without searching again
    sbh.sbh_join_segments(L, l_off, R, r_start, r_len, ol, orr, total, npairs, seg, scratch=scr, reuse_counts=reuse)
    so = seg.cpu().numpy().astype(np.int64)
    gl, gr = ol.cpu().numpy(), orr.cpu().numpy()
    assert so[0] == 0 and so[-1] == total
    for g in range(len(l_lens)):
        el, er = oracle.join(Lr[g][0], Lr[g][1], Rr[g][0], Rr[g][1])
        assert np.array_equal(gl[so[g]:so[g + 1]], el) and np.array_equal(gr[so[g]:so[g + 1]], er), g
