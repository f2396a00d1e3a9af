"""The operator layer (Listing 2 of Sec. 4.3: Extract a bundle, KeySwap a
KPA whose resident column is not the grouping column, then group) on the
GPU, on the 7-column ad-event stream: three chains, each against the
oracle's step-by-step statement of the same chain, window by window, and
the steps the rule inserted."""
import numpy as np
import pytest
import torch

import gen
import oracle
from tests.gpu_util import cuda

pytestmark = pytest.mark.gpu

W = 100_000_000  # 100 ms windows


@pytest.fixture(scope="module")
def O():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import operators
    return operators


@pytest.fixture(scope="module")
def ads():
    cols, camp = gen.ad_events(1_500_000, events_per_s=1e7)
    return cols, camp, {k: cuda(v) for k, v in cols.items()}, cuda(camp)


def _window_rows(ts, w, length):
    lo, hi = np.searchsorted(ts, [w * length, (w + 1) * length])
    return int(lo), int(hi)


def test_bundle_straight_into_a_count_extracts_and_needs_no_keyswap(O, ads):
    cols, camp, dcols, dcamp = ads
    trace = []
    b = O.Bundle(dcols)
    k, c = O.count_per_key(b, "ad_type", trace)
    ok, oc, _ = oracle.group_sum_count(*oracle.sort(*oracle.extract(cols["ad_type"], 0, b.n)), None)
    assert np.array_equal(k, ok) and np.array_equal(c, oc)
    assert [s[0] for s in trace] == ["Extract", "Sort", "Keyed"]


def test_chain_views_per_campaign(O, ads):
    # Window -> Select(view) -> [KeySwap(ad -> campaign, fused gather)] -> Sort -> count
    cols, camp, dcols, dcamp = ads
    ts, et, ad = cols["event_time"], cols["event_type"], cols["ad_id"]
    campaign = O.Lookup("campaign_id", "ad_id", dcamp)
    wins = O.Bundle(dcols).windows("event_time", W)
    assert len(wins) == int(ts[-1] // W) + 1
    for w, wb in wins:
        trace = []
        views = O.select(wb, "event_type", 0, 1, trace)
        k, c = O.count_per_key(views, campaign, trace)
        assert [s[0] for s in trace] == ["Extract", "Select", "KeySwap", "Sort", "Keyed"]
        lo, hi = _window_rows(ts, w, W)
        # the oracle's chain, step by step
        ek, ep = oracle.extract(et, lo, hi - lo)
        sk, sp = oracle.select(ek, ep, et, 0, 1)
        ck = oracle.materialize(oracle.materialize(sp, ad).astype(np.uint32), camp)
        ok, oc, _ = oracle.group_sum_count(*oracle.sort(ck, sp), None)
        assert np.array_equal(k, ok) and np.array_equal(c, oc), f"window {w}"


def test_chain_latest_clicks_per_ad(O, ads):
    # Window -> Select(click) -> [KeySwap(ad)] -> Sort -> top-3 by event time
    cols, camp, dcols, dcamp = ads
    ts, et, ad = cols["event_time"], cols["event_type"], cols["ad_id"]
    for w, wb in O.Bundle(dcols).windows("event_time", W):
        trace = []
        clicks = O.select(wb, "event_type", 1, 2, trace)
        got = O.topk_per_key(clicks, "ad_id", "event_time", 3, trace)
        assert [s[0] for s in trace] == ["Extract", "Select", "KeySwap", "Sort", "TopK"]
        lo, hi = _window_rows(ts, w, W)
        ek, ep = oracle.extract(et, lo, hi - lo)
        sk, sp = oracle.select(ek, ep, et, 1, 2)
        exp = oracle.topk(*oracle.sort(oracle.materialize(sp, ad), sp), ts, 3)
        for g, e in zip(got, exp):
            assert np.array_equal(g, e), f"window {w}"


def test_chain_view_click_pairs_per_campaign(O, ads):
    # 1 ms windows: Select(view) and Select(click) -> [KeySwap both to the
    # campaign] -> Sort both -> Join
    cols, camp, dcols, dcamp = ads
    ts, et, ad = cols["event_time"], cols["event_type"], cols["ad_id"]
    campaign = O.Lookup("campaign_id", "ad_id", dcamp)
    wins = O.Bundle(dcols).windows("event_time", 1_000_000)
    for w, wb in wins[:: max(1, len(wins) // 12)]:
        trace = []
        views = O.select(wb, "event_type", 0, 1, trace)
        clicks = O.select(O.extract(wb, campaign, trace), "event_type", 1, 2, trace)
        pl, pr = O.join(views, clicks, campaign, trace)
        # the click side was extracted on the campaign already: one KeySwap only
        assert [s[0] for s in trace] == ["Extract", "Select", "Extract+Materialize", "Select", "KeySwap", "Sort",
                                         "Sort", "Join"]
        lo, hi = _window_rows(ts, w, 1_000_000)
        vk, vp = oracle.select(*oracle.extract(et, lo, hi - lo), et, 0, 1)
        ck, cp = oracle.select(*oracle.extract(et, lo, hi - lo), et, 1, 2)
        to_c = lambda p: oracle.materialize(oracle.materialize(p, ad).astype(np.uint32), camp)
        el, er = oracle.join(*oracle.sort(to_c(vp), vp), *oracle.sort(to_c(cp), cp))
        assert np.array_equal(pl, el) and np.array_equal(pr, er), f"window {w}"
        assert pl.size > 0
