"""Window pipelines composed of the C ABI calls (orchestration only: every
step runs in the kernels of libsbh.so).

batched_windows  per-key count, sum and top-K inside each of many tumbling
    windows laid end to end (Sec. 4.2 "Windowing" and "Keyed Aggregation";
    the TopK Per Key and Sum Per Key benchmarks of Sec. 7).  Two schedules
    with identical results:
      "batched"  one pass over all windows: Extract writes composite keys
                 (window << (64 - window_bits)) | key, so one sort, one keyed
                 reduction and one top-K group every window at once; window
                 w's results are the output keys in [w << shift, (w + 1) <<
                 shift), found by binary search (the window-range kernel).
      "loop"     one Extract, Sort, keyed reduction and top-K per window.
sliding_join  the temporal join of two streams over sliding windows built
    from panes (Sec. 4.2 "Temporal Join" and "Windowing"): every pane of
    every stream is extracted (from page-locked host memory when the key
    column lives there) and sorted once; the windows' panes are merged and
    the two sides joined, for all windows at once (a few launches per merge
    level and one segmented join) or window by window.
ad_campaign_counts  a chain of operators over a 7-column ad-event stream
    (Extract -> Select -> KeySwap through a lookup table -> Sort -> Keyed
    count per window), the kind of pipeline the paper's declarative API
    builds (Sec. 4.3), composed from operators.py, with Materialize fused
    into the key swap.
"""
from __future__ import annotations

import numpy as np
import torch

from . import operators, sbh


def _u64(n, dev):
    return torch.empty(max(1, n), dtype=torch.uint64, device=dev)


def _u32(n, dev):
    return torch.empty(max(1, n), dtype=torch.uint32, device=dev)


class WindowResults:
    """Per-window grouping results held on the device.

    For window w, rows [begin[w], end[w]) of keys / counts / sums and of the
    top-K arrays belong to it, in key order.  keys hold the raw keys (window
    bits removed) once `window()` is called."""

    def __init__(self, keys, counts, sums, nvalid, tvals, tptrs, begin, end, shift, K):
        self.keys, self.counts, self.sums = keys, counts, sums
        self.nvalid, self.tvals, self.tptrs = nvalid, tvals, tptrs
        self.begin, self.end, self.shift, self.K = begin, end, shift, K

    def window(self, w):
        """(keys, counts, sums, nvalid, top values [m, K], top ptrs [m, K]) as host arrays."""
        b, e = int(self.begin[w]), int(self.end[w])
        mask = np.uint64((1 << self.shift) - 1) if self.shift < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        keys = self.keys[b:e].cpu().numpy() & mask
        K = self.K
        return (keys, self.counts[b:e].cpu().numpy(), self.sums[b:e].cpu().numpy(), self.nvalid[b:e].cpu().numpy(),
                self.tvals[b * K:e * K].cpu().numpy().reshape(-1, K), self.tptrs[b * K:e * K].cpu().numpy().reshape(-1, K))


def batched_windows(key_col, val_col, offsets, K=3, schedule="batched"):
    """key_col, val_col: device uint64 columns; offsets: host array of
    nwin + 1 non-decreasing row offsets.  Returns WindowResults.  The
    batched schedule needs every key below 2^(64 - window_bits(nwin)) and
    falls back to the loop when one is not."""
    offsets = np.asarray(offsets, dtype=np.uint64)
    nwin = offsets.size - 1
    if schedule == "batched":
        res = _batched(key_col, val_col, offsets, K)
        if res is not None:
            return res
    return _loop(key_col, val_col, offsets, K)


def _batched(key_col, val_col, offsets, K):
    dev = key_col.device
    nwin = offsets.size - 1
    row0, n = int(offsets[0]), int(offsets[-1] - offsets[0])
    shift = 64 - sbh.window_bits(nwin)
    d_off = torch.from_numpy(offsets.astype(np.int64)).to(dev).view(torch.uint64)
    keys, ptrs, key_or = _u64(n, dev), _u32(n, dev), _u64(1, dev)
    sbh.sbh_kpa_extract_windows(key_col, d_off, row0, n, keys, ptrs, key_or)
    if shift < 64 and int(key_or.item()) >> shift:
        return None  # some key uses the window bits
    sk, sp = _u64(n, dev), _u32(n, dev)
    sbh.sbh_kpa_sort(keys[:n], ptrs[:n], sk, sp)
    del keys, ptrs
    ok, oc, osum, nk = _u64(n, dev), _u64(n, dev), _u64(n, dev), _u64(1, dev)
    sbh.sbh_group_reduce(sk[:n], sp[:n], val_col, ok, oc, osum, n, nk)
    tk, tnv, tv, tp, nkt = (_u64(n, dev), torch.empty(max(1, n), dtype=torch.uint8, device=dev), _u64(n * K, dev),
                            _u32(n * K, dev), _u64(1, dev))
    sbh.sbh_topk(sk[:n], sp[:n], val_col, K, tk, tnv, tv, tp, n, nkt)
    m = int(nk.item())
    starts = (torch.arange(nwin, dtype=torch.int64, device=dev) << shift).view(torch.uint64) if shift < 64 else \
        torch.zeros(1, dtype=torch.uint64, device=dev)
    rb, re_ = _u64(nwin, dev), _u64(nwin, dev)
    if shift < 64:
        sbh.sbh_window_ranges(ok[:m], starts, 1 << shift, rb[:nwin], re_[:nwin])
        begin, end = rb[:nwin].cpu().numpy(), re_[:nwin].cpu().numpy()
    else:
        begin, end = np.zeros(1, np.uint64), np.array([m], np.uint64)
    return WindowResults(ok, oc, osum, tnv, tv, tp, begin, end, shift, K)


def _loop(key_col, val_col, offsets, K):
    dev = key_col.device
    nwin = offsets.size - 1
    row0, n = int(offsets[0]), int(offsets[-1] - offsets[0])
    sizes = np.diff(offsets).astype(np.int64)
    big = int(sizes.max()) if nwin else 0
    keys, ptrs, sk, sp = _u64(big, dev), _u32(big, dev), _u64(big, dev), _u32(big, dev)
    sort_scr = torch.empty(max(1, sbh.sort_scratch_bytes(big)), dtype=torch.uint8, device=dev)
    ok, oc, osum = _u64(n, dev), _u64(n, dev), _u64(n, dev)
    tk, tnv, tv, tp = _u64(n, dev), torch.empty(max(1, n), dtype=torch.uint8, device=dev), _u64(n * K, dev), \
        _u32(n * K, dev)
    nk, nkt = _u64(nwin, dev), _u64(nwin, dev)
    red_scr = top_scr = None
    for w in range(nwin):
        o, m = int(offsets[w]) - row0, int(sizes[w])
        if m == 0:
            nk[w:w + 1].zero_()
            nkt[w:w + 1].zero_()
            continue
        sbh.sbh_kpa_extract(key_col, row0 + o, m, keys, ptrs)
        sbh.sbh_kpa_sort(keys[:m], ptrs[:m], sk, sp, scratch=sort_scr)
        red_scr = sbh.sbh_group_reduce(sk[:m], sp[:m], val_col, ok[o:], oc[o:], osum[o:], m, nk[w:w + 1],
                                       scratch=_fit(red_scr, sbh.group_reduce_scratch_bytes(m, 8), dev))
        top_scr = sbh.sbh_topk(sk[:m], sp[:m], val_col, K, tk[o:], tnv[o:], tv[o * K:], tp[o * K:], m, nkt[w:w + 1],
                               scratch=_fit(top_scr, sbh.topk_scratch_bytes(m, K, 8), dev))
    begin = offsets[:-1] - offsets[0]
    end = begin + nk.cpu().numpy()[:nwin]
    return WindowResults(ok, oc, osum, tnv, tv, tp, begin, end, 64, K)


def _fit(buf, nbytes, dev):
    if buf is None or buf.numel() < nbytes:
        return torch.empty(max(1, nbytes), dtype=torch.uint8, device=dev)
    return buf


class JoinResults:
    """Pairs of every window: window i's pairs are rows [begin[i], end[i]) of
    ptr_l / ptr_r, in (key, ptrL, ptrR) order."""

    def __init__(self, ptr_l, ptr_r, begin, end):
        self.ptr_l, self.ptr_r = ptr_l, ptr_r
        self.begin, self.end = np.asarray(begin, np.int64), np.asarray(end, np.int64)
        self.npairs = self.end - self.begin

    def window(self, i):
        b, e = int(self.begin[i]), int(self.end[i])
        return self.ptr_l[b:e].cpu().numpy(), self.ptr_r[b:e].cpu().numpy()


def sliding_join(lkey_col, rkey_col, n_rows, window=1_000_000, stride=250_000, pair_cap=262_144, windows=None,
                 schedule="batched"):
    """Equi-join of L and R inside every sliding window [w * stride, w *
    stride + window) of the first n_rows rows (ts = row index).  Key columns
    may be device tensors or page-locked host tensors.  Returns (JoinResults,
    the windows joined).

    "batched" (when window / stride is a power of two and every window is
    joined): each side's key column crosses the host link once, a group of
    windows at a time, while the windows before are joined; a group's panes
    are sorted by one sort of composite (pane, key) keys and merged level by
    level, every merge of a level in one launch (run i of level r + 1 merges
    runs i and i + 2^r of level r, so the last level holds every window's
    merged KPA); one segmented join joins every window of the group.
    "loop" (or `windows` given: only those windows are joined): the panes are
    sorted one by one and each window merges and joins on its own, at most
    pair_cap pairs per window."""
    per = window // stride
    if window % stride:
        raise ValueError("window must be a multiple of stride")
    if schedule == "batched" and windows is None and per & (per - 1) == 0:
        res = _sliding_join_batched(lkey_col, rkey_col, n_rows, window, stride)
        if res is not None:
            return res
    return _sliding_join_loop(lkey_col, rkey_col, n_rows, window, stride, pair_cap, windows)


def window_groups(nwin, per, stride, groups):
    """The batched sliding join's groups of windows: for group g, (first
    window, end window, first pane, end pane, first row to copy, end row to
    copy).  Window w covers panes [w, w + per); a group's panes are its
    windows' panes; the rows to copy are the group's rows that no earlier
    group copied, so the copy ranges tile [0, (nwin + per - 1) * stride)."""
    ngroups = max(1, min(groups, nwin))
    wb = [nwin * g // ngroups for g in range(ngroups + 1)]
    out, done = [], 0
    for g in range(ngroups):
        p0, p1 = wb[g], wb[g + 1] + per - 1
        out.append((wb[g], wb[g + 1], p0, p1, done, p1 * stride))
        done = p1 * stride
    return out


def _sliding_join_batched(lkey_col, rkey_col, n_rows, window, stride, groups=8):
    dev = torch.device("cuda")
    per = window // stride
    npanes = n_rows // stride
    nwin = npanes - per + 1
    if nwin <= 0:
        return JoinResults(_u32(0, dev), _u32(0, dev), [], []), []
    rows = npanes * stride
    # The windows go in `groups` groups; group g joins windows [wb[g],
    # wb[g + 1]) from panes [wb[g], wb[g + 1] + per - 1), each pane sorted
    # and merged within its group (a group shares per - 1 panes with the
    # next).  Host columns cross the link group by group on a copy stream,
    # each row once, so the work of a group overlaps the copies of the next:
    # the whole-column copies of both sides (2 GB) no longer come before
    # every kernel.  For 2 x 128M rows (509 windows): 63 ms with one group,
    # 51, 44.5, 42.2 and 44.9 ms with 2, 4, 8 and 16; the link alone takes
    # 37 ms for the 2 GB.
    main = torch.cuda.current_stream(dev)
    copy_st = torch.cuda.Stream(dev)
    copy_st.wait_stream(main)
    grp = window_groups(nwin, per, stride, groups)
    cols, copied = [], [[None, None] for _ in grp]
    for col in (lkey_col, rkey_col):
        cols.append(col[:rows] if col.is_cuda else _u64(rows, dev))
    for g, (_, _, _, _, c0, c1) in enumerate(grp):
        for si, col in enumerate((lkey_col, rkey_col)):
            if not col.is_cuda:
                with torch.cuda.stream(copy_st):
                    cols[si][c0:c1].copy_(col[c0:c1], non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(copy_st)
                copied[g][si] = ev
    for c, col in zip(cols, (lkey_col, rkey_col)):
        if not col.is_cuda:
            c.record_stream(copy_st)  # written on the copy stream
    key_ors, parts = [], []
    for g, (w0, w1, p0, p1, _, _) in enumerate(grp):
        nwg, npg = w1 - w0, p1 - p0
        r0, ng = p0 * stride, (p1 - p0) * stride
        offs = (torch.arange(p0, p1 + 1, dtype=torch.int64, device=dev) * stride).view(torch.uint64)
        sides = []
        for si in range(2):
            if copied[g][si] is not None:
                main.wait_event(copied[g][si])
            ck, cp, key_or = _u64(ng, dev), _u32(ng, dev), _u64(1, dev)
            sbh.sbh_kpa_extract_windows(cols[si], offs, r0, ng, ck, cp, key_or)
            key_ors.append((key_or, 64 - sbh.window_bits(npg)))
            sbh.sbh_kpa_sort(ck, cp, ck, cp)  # every pane sorted, pane after pane
            sbh.sbh_kpa_keyswap(cp, cols[si], ck)  # the plain keys back
            run_k, run_p, run_len, nruns = ck, cp, stride, npg
            gap = 1
            while gap < per:
                nnext = nruns - gap
                ok, op = _u64(nnext * 2 * run_len, dev), _u32(nnext * 2 * run_len, dev)
                a_start = [i * run_len for i in range(nnext)]
                b_start = [(i + gap) * run_len for i in range(nnext)]
                lens = [run_len] * nnext
                sbh.sbh_kpa_merge_segments((run_k, run_p), (run_k, run_p), a_start, lens, b_start, lens, ok, op)
                run_k, run_p, run_len, nruns = ok, op, 2 * run_len, nnext
                gap *= 2
            sides.append((run_k, run_p))
        l_off = [w * window for w in range(nwg + 1)]
        r_start, r_len = l_off[:-1], [window] * nwg
        npairs, seg = _u64(1, dev), _u64(nwg + 1, dev)
        scr = sbh.sbh_join_segments(sides[0], l_off, sides[1], r_start, r_len, None, None, 0, npairs, seg)
        parts.append((sides, l_off, r_start, r_len, npairs, seg, scr, nwg))
    if any(sh < 64 and int(o.item()) >> sh for o, sh in key_ors):
        return None  # a key uses the pane bits: the loop schedule instead
    totals = [int(x[4].item()) for x in parts]
    out_l, out_r = _u32(sum(totals), dev), _u32(sum(totals), dev)
    base = 0
    for (sides, l_off, r_start, r_len, npairs, seg, scr, nwg), tot in zip(parts, totals):
        sbh.sbh_join_segments(sides[0], l_off, sides[1], r_start, r_len, out_l[base:base + tot],
                              out_r[base:base + tot], tot, npairs, seg, scratch=scr, reuse_counts=True)
        base += tot
    begin, end, base = [], [], 0
    for (_, _, _, _, _, seg, _, nwg), tot in zip(parts, totals):
        off = seg[: nwg + 1].cpu().numpy().astype(np.int64) + base
        begin.extend(off[:-1])
        end.extend(off[1:])
        base += tot
    return JoinResults(out_l, out_r, begin, end), list(range(nwin))


def _sliding_join_loop(lkey_col, rkey_col, n_rows, window, stride, pair_cap, windows):
    dev = torch.device("cuda")
    per = window // stride
    npanes = n_rows // stride
    nwin = max(0, npanes - per + 1)
    sides = []
    for col in (lkey_col, rkey_col):
        keys, ptrs = _u64(npanes * stride, dev), _u32(npanes * stride, dev)
        sbh.sbh_kpa_extract(col, 0, npanes * stride, keys, ptrs)
        scr = torch.empty(max(1, sbh.sort_scratch_bytes(stride)), dtype=torch.uint8, device=dev)
        for p in range(npanes):
            seg = slice(p * stride, (p + 1) * stride)
            sbh.sbh_kpa_sort(keys[seg], ptrs[seg], keys[seg], ptrs[seg], scratch=scr)  # in place
        sides.append((keys, ptrs))
    wl = list(range(nwin)) if windows is None else list(windows)
    ml, mlp, mr, mrp = _u64(window, dev), _u32(window, dev), _u64(window, dev), _u32(window, dev)
    out_l, out_r = _u32(len(wl) * pair_cap, dev), _u32(len(wl) * pair_cap, dev)
    npairs = _u64(len(wl), dev)
    join_scr = None
    for i, w in enumerate(wl):
        merged = []
        for (keys, ptrs), mk, mp in ((sides[0], ml, mlp), (sides[1], mr, mrp)):
            runs = [(keys[(w + j) * stride:(w + j + 1) * stride], ptrs[(w + j) * stride:(w + j + 1) * stride])
                    for j in range(per)]
            sbh.sbh_kpa_merge(runs, mk, mp)
            merged.append((mk, mp))
        join_scr = sbh.sbh_join(*merged[0], *merged[1], out_l[i * pair_cap:], out_r[i * pair_cap:], pair_cap,
                                npairs[i:i + 1], scratch=_fit(join_scr, sbh.join_scratch_bytes(window, window), dev))
    counts = npairs.cpu().numpy()[:len(wl)].astype(np.int64)
    if len(wl) and counts.max() > pair_cap:
        over = [w for w, c in zip(wl, counts) if c > pair_cap]
        raise RuntimeError(f"windows {over[:4]} have more than pair_cap={pair_cap} pairs; raise pair_cap")
    begin = np.arange(len(wl), dtype=np.int64) * pair_cap
    return JoinResults(out_l, out_r, begin, begin + counts), wl


def ad_campaign_counts(cols, campaign_of_ad, window_ns, view=0, trace=None):
    """A chained pipeline over a 7-column ad-event stream (device columns;
    event_time non-decreasing): per tumbling window of event time, the
    number of view events of every campaign.  Built from the operator layer
    (operators.py), whose Listing 2 rule inserts the steps: per window,
    Extract (a KPA keyed by event type) -> Select (event type == view) ->
    KeySwap to the campaign (the ad column gathered through the ad ->
    campaign table: Materialize fused with the Extract of the new key,
    Sec. 4.3) -> Sort -> Keyed count.  Returns [(window, campaigns,
    counts)] as host arrays."""
    b = operators.Bundle(cols)
    campaign = operators.Lookup("campaign_id", "ad_id", campaign_of_ad)
    out = []
    for w, wb in b.windows("event_time", window_ns, trace):
        views = operators.select(wb, "event_type", view, view + 1, trace)
        k, c = operators.count_per_key(views, campaign, trace)
        out.append((w, k, c))
    return out
