"""The learned partition sort on the GPU: its network's forward pass and
gradient against the FP64 oracle (tolerances, not bit-exact: FP32 sums), the
training set against the oracle's (exact inputs, FP32 targets), and the
sorted output, which must equal the plain sort bit for bit.  The last test
shows what the trained network gains over the untrained one."""
import numpy as np
import pytest
import torch

import gen
import oracle
from oracle import learned as olearned
from oracle import mlp as omlp
from tests.gpu_util import cuda, host, same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_01328_b300 import sbh
    return sbh


def _params(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.5, omlp.N_PARAMS).astype(np.float32)


def test_mlp_forward_matches_oracle(S):
    p = _params(1)
    x = gen.unif01(3, 1, 10_000).astype(np.float32)
    y = torch.empty(x.size, dtype=torch.float32, device="cuda")
    S.sbh_mlp_forward(cuda(p), cuda(x), y)
    ref, _ = omlp.forward(p.astype(np.float64), x.astype(np.float64))
    # FP32 evaluation of 32-term sums: error well below 1e-5 of the output scale
    assert np.max(np.abs(host(y) - ref)) <= 2e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("m", [1, 255, 256, 4097, 20_000])
def test_mlp_grad_matches_oracle(S, m):
    p = _params(2)
    x = gen.unif01(4, 1, m).astype(np.float32)
    t = gen.unif01(4, 2, m).astype(np.float32)
    g = torch.empty(S.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    S.sbh_mlp_grad(cuda(p), cuda(x), cuda(t), g, loss)
    p64, x64, t64 = p.astype(np.float64), x.astype(np.float64), t.astype(np.float64)
    ref = omlp.backward(p64, x64, t64)
    got = host(g).astype(np.float64)
    # Each gradient is a sum over rows of terms computed in FP32 (32-term dot
    # products forward and back, then sums over the rows in a fixed order);
    # its rounding error is at most a few hundred units of roundoff (2^-24)
    # times the sum of its terms' magnitudes A.  The bound is 2^-16 A per
    # parameter (256 units of roundoff), which means a relative error below
    # 1e-4 wherever the terms do not cancel to under a sixth of A.
    A = omlp.abs_terms(p64, x64, t64)
    err = np.abs(got - ref)
    assert np.all(err <= 2.0 ** -16 * A)
    wide = np.abs(ref) >= A / 6
    assert np.all(err[wide] <= 1e-4 * np.abs(ref[wide]))
    ref_loss = omlp.loss(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(float(host(loss)[0]) - ref_loss) <= 1e-4 * ref_loss
    # repeated calls give identical bits
    g2 = torch.empty_like(g)
    S.sbh_mlp_grad(cuda(p), cuda(x), cuda(t), g2)
    assert torch.equal(g, g2)


def _sample(n, seed=gen.SEED_MIXED, hashed=False):
    col = gen.mixed_keys(n, seed=seed, hashed=hashed)
    return col, col[::100].copy()


@pytest.mark.parametrize("hashed", [False, True])
def test_training_set_and_heavy_keys_match_oracle(S, hashed):
    n = 4_000_000
    col, sample = _sample(n, hashed=hashed)
    init = gen.mlp_init()
    model = torch.zeros(S.LEARNED_MODEL_BYTES, dtype=torch.uint8, device="cuda")
    tx = torch.zeros(sample.size, dtype=torch.float32, device="cuda")
    tt = torch.zeros(sample.size, dtype=torch.float32, device="cuda")
    S.sbh_learned_train(cuda(sample), n, cuda(init), 0, 4096, 1e-2, model, None, tx, tt)
    torch.cuda.synchronize()
    heavy = olearned.heavy_keys(sample, n, S.LEARNED_CAPACITY)
    ox, ot = olearned.training_set(sample, n, S.LEARNED_CAPACITY)
    blob = host(model)
    words = blob.view(np.uint32)
    hdr = omlp.N_PARAMS
    assert heavy.size > 10  # Zipf ranks: heavy keys in and (hashed) out of exact cells
    assert words[hdr + 1] == heavy.size and words[hdr + 2] == ox.size
    got_heavy = blob[(hdr + 5) * 4: (hdr + 5) * 4 + 8 * heavy.size].view(np.uint64)
    assert np.array_equal(got_heavy, heavy)
    m2 = ox.size
    assert np.array_equal(host(tx)[:m2], ox.astype(np.float32))  # features are exact in FP32
    assert np.max(np.abs(host(tt)[:m2] - ot)) <= 1e-6
    # the weights are the initial ones when no step runs
    assert np.array_equal(blob[: hdr * 4].view(np.float32), init)


def test_training_follows_oracle_first_steps_and_learns(S):
    n = 4_000_000
    col, sample = _sample(n)
    init = gen.mlp_init()
    ox, ot = olearned.training_set(sample, n, S.LEARNED_CAPACITY)
    # one step: Adam's first update against the FP64 statement, on parameters
    # whose gradient is not near zero (the first step moves by lr * sign(g))
    model1, _ = S.learned_train(cuda(sample), n, cuda(init), steps=1, batch=4096, lr=1e-3)
    p1 = host(S.model_params(model1)).astype(np.float64)
    g = omlp.backward(init.astype(np.float64), ox[:4096], ot[:4096])
    e1, _, _ = omlp.adam_step(init.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    big = np.abs(g) > 1e-2 * np.max(np.abs(g))
    assert np.max(np.abs(p1[big] - e1[big])) <= 1e-5
    # many steps: the batch loss falls by more than 20x
    model, losses = S.learned_train(cuda(sample), n, cuda(init), steps=150, batch=4096, lr=2e-2)
    L = host(losses)
    assert L[-10:].mean() < L[:3].mean() / 20


@pytest.mark.parametrize("hashed", [False, True])
def test_quantile_start_matches_oracle_and_training_refines_it(S, hashed):
    n = 4_000_000
    col, sample = _sample(n, hashed=hashed)
    d_sample = cuda(sample)
    m0, _ = S.learned_train(d_sample, n, None, steps=0, batch=16384, lr=3e-5)
    p0 = host(S.model_params(m0)).astype(np.float64)
    heavy = olearned.heavy_keys(sample, n, S.LEARNED_CAPACITY)
    srt = np.sort(sample)
    nh = srt[~np.isin(srt, heavy)]
    ref = omlp.quantile_init(nh)
    # FP32 knots and slopes against the FP64 statement: the kinks exactly, the
    # network's output within FP32 rounding of a sum of 32 slope terms
    diffs = {k: float(np.max(np.abs(p0[sl] - ref[sl]))) for k, sl in omlp.SLICES.items()}
    for k in ("W1", "b1", "W2", "b2"):
        assert diffs[k] <= 1e-7, diffs
    xs = np.linspace(0.0, 1.0, 4097)
    assert np.max(np.abs(omlp.forward(p0, xs)[0] - omlp.forward(ref, xs)[0])) <= 2e-4, diffs
    ox, ot = olearned.training_set(sample, n, S.LEARNED_CAPACITY)
    loss0 = omlp.loss(p0, ox, ot)
    assert loss0 < 1e-4  # the interpolated CDF is already close
    m1, _ = S.learned_train(d_sample, n, None, steps=40, batch=16384, lr=3e-5)
    p1 = host(S.model_params(m1)).astype(np.float64)
    assert omlp.loss(p1, ox, ot) < loss0


@pytest.mark.parametrize("start", ["seeded", "quantile"])
@pytest.mark.parametrize("n,kind", [(1, "mixed"), (5000, "mixed"), (3_000_017, "mixed"), (2_500_000, "uniform"),
                                    (2_100_000, "equal"), (2_200_000, "highbyte"), (3_000_001, "hashed"),
                                    (600_011, "smallkeys"), (2_000_003, "smallkeys")])
def test_learned_sort_equals_plain_sort(S, n, kind, start):
    if kind == "mixed":
        col = gen.mixed_keys(n, seed=7)
    elif kind == "hashed":  # Zipf ranks through mix64: the same multiplicities over all 64 bits
        col = gen.mixed_keys(n, seed=7, hashed=True)
    elif kind == "uniform":
        col = gen.uniform(7, 1, n, 0, 0, np.uint64)
    elif kind == "equal":
        col = np.full(n, 12345, dtype=np.uint64)
    elif kind == "smallkeys":  # 4096 key values, exact cells: ids below 256, one pass
        col = gen.uniform(7, 3, n, 0, 4096, np.uint64)
    else:
        col = gen.uniform(7, 2, n, 0, 256, np.uint64) << np.uint64(56)
    sample = col[::100].copy()
    if start == "seeded":
        model, _ = S.learned_train(cuda(sample), n, cuda(gen.mlp_init()), steps=150, batch=4096, lr=2e-2)
    else:  # the bench's training: quantile-knot start (also all-heavy and one-sample samples)
        model, _ = S.learned_train(cuda(sample), n, None, steps=40, batch=4096, lr=3e-4)
    keys, ptrs = S.extract(cuda(col), 0, n)
    sk, sp, stats = S.sort_learned(keys, ptrs, model)
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)
    assert stats["overflow_rows"] <= n
    if kind in ("mixed", "hashed") and n >= 3_000_000:  # both id bytes vary: the second pass runs
        assert stats["bucket_ids"] > 256


@pytest.mark.parametrize("n,kind,offset", [(1, "mixed", 0), (4097, "mixed", 0), (3_000_017, "mixed", 0),
                                           (3_000_017, "mixed", 1), (2_000_003, "smallkeys", 0),
                                           (2_100_000, "equal", 0)])
def test_learned_sort_of_a_key_column_without_extract(S, n, kind, offset):
    # ptrs_in = None: the learned sort reads the key column itself and row
    # i's ptr is i; it trains on the column's samples (no Extract at all).
    # offset 1: the column starts 8 bytes past a 16-byte boundary (no bulk
    # copies of its tiles)
    if kind == "mixed":
        col = gen.mixed_keys(n + offset, seed=8)
    elif kind == "smallkeys":
        col = gen.uniform(8, 3, n + offset, 0, 4096, np.uint64)
    else:
        col = np.full(n + offset, 777, dtype=np.uint64)
    d = cuda(col)[offset:]
    model, _ = S.learned_train(S.sample(d, 100), n, None, steps=40, batch=4096, lr=3e-4)
    sk, sp, st = S.sort_learned(d, None, model)
    ok, op = oracle.sort(*oracle.extract(col[offset:], 0, n))
    assert same(sk, ok) and same(sp, op)
    if kind == "mixed" and n > 1_000_000:
        # the most frequent key (about 8% of the rows) has a bucket of its own,
        # the largest one
        assert st["largest_bucket"] == int(np.unique(col[offset:], return_counts=True)[1].max())


@pytest.mark.parametrize("hashed", [False, True])
def test_learned_sort_mixed_keys_32m_and_trained_vs_untrained(S, hashed):
    n = 32_000_000
    col, sample = _sample(n, hashed=hashed)
    d_sample, init = cuda(sample), cuda(gen.mlp_init())
    # the bench's training: quantile-knot start, 40 small Adam steps
    trained, _ = S.learned_train(d_sample, n, None, steps=40, batch=16384, lr=3e-5)
    untrained, _ = S.learned_train(d_sample, n, init, steps=0, batch=4096, lr=2e-2)
    keys, ptrs = S.extract(cuda(col), 0, n)
    sk, sp, st_tr = S.sort_learned(keys, ptrs, trained)
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)
    sk2, sp2, st_un = S.sort_learned(keys, ptrs, untrained)
    assert same(sk2, ok) and same(sp2, op)
    # the trained network keeps far more rows out of the fallback sort
    assert st_tr["overflow_rows"] < 0.05 * n
    assert st_un["overflow_rows"] > 5 * max(st_tr["overflow_rows"], 1)


@pytest.mark.parametrize("ptr_kind", ["shuffled", "duplicates"])
def test_learned_sort_keeps_input_order_of_ties(S, ptr_kind):
    # pointers that do not ascend (a permutation) or repeat: equal keys keep
    # their input order, as in the plain sort (the stable sort by key alone)
    n = 3_000_017
    col = gen.mixed_keys(n, seed=9)
    if ptr_kind == "shuffled":
        ptrs = np.argsort(gen.uniform(9, 4, n, 0, 0, np.uint64), kind="stable").astype(np.uint32)
    else:
        ptrs = gen.uniform(9, 5, n, 0, 1000, np.uint32)
    model, _ = S.learned_train(cuda(col[::100].copy()), n, None, steps=40, batch=4096, lr=3e-4)
    keys, d_ptrs = cuda(col), cuda(ptrs)
    sk, sp, stats = S.sort_learned(keys, d_ptrs, model)
    order = np.argsort(col, kind="stable")
    assert same(sk, col[order]) and same(sp, ptrs[order])
    pk, pp = S.sort(keys, d_ptrs)
    assert torch.equal(sk, pk) and torch.equal(sp, pp)
    assert stats["sorted_buckets"] > 0 and stats["radix_buckets"] > 0  # both in-bucket sorts ran


@pytest.mark.parametrize("hashed", [False, True])
def test_learned_sort_headline_window_256m(S, hashed):
    # the benchmark's exact step at full size: 256M mixed keys, the 0.25%
    # sample read from the column, quantile start, 40 Adam steps of 4096 rows
    # at lr 3e-4, then the learned sort of the key column (the extract fused
    # into its first pass); its output equals an explicit extract followed by
    # the plain sort and satisfies every sorted-KPA invariant (bit-exact
    # parity with the oracle at this size is out of the oracle's reach;
    # sampled ranks are checked below)
    from tests.gpu_util import sorted_kpa_on_device
    n = 256_000_000
    col_h = torch.empty(n, dtype=torch.uint64)
    gen.mixed_keys(n, out=col_h.numpy(), hashed=hashed)
    col = col_h.cuda()
    del col_h
    model, _ = S.learned_train(S.sample(col, 400), n, None, steps=40, batch=4096, lr=3e-4)
    lk, lp, stats = S.sort_learned(col, None, model)
    assert S.sync_status() == S.SBH_OK
    assert stats["bucket_ids"] > 256 and stats["overflow_rows"] < 0.05 * n
    keys, ptrs = S.extract(col, 0, n)
    pk, pp = S.sort(keys, ptrs)
    assert torch.equal(lk, pk) and torch.equal(lp, pp)
    del pk, pp, keys, ptrs
    torch.cuda.empty_cache()
    sorted_kpa_on_device(col, 0, lk, lp)
    # sampled rows: the rank of (key, ptr) among all rows is its output index
    sk = col.view(torch.int64) ^ torch.iinfo(torch.int64).min
    rows = torch.arange(n, device="cuda")
    for i in np.linspace(0, n - 1, 9).astype(np.int64):
        kk, pv = sk[int(lp[i])], int(lp[i])
        below = int((sk < kk).sum()) + int(((sk == kk) & (rows < pv)).sum())
        assert below == int(i)


@pytest.mark.parametrize("fused", [False, True])
def test_learned_step_replays_as_a_cuda_graph(S, fused):
    # extract + training + learned sort + per-key count queue their work
    # without host synchronisation, so the whole step is captured once and
    # replayed; every replay equals the plain sort and the eager count
    # (fused: the benchmark's step, the sample read from the column and the
    # sort reading the column itself)
    n = 3_000_017
    col = cuda(gen.mixed_keys(n, seed=17))
    keys = torch.empty(n, dtype=torch.uint64, device="cuda")
    ptrs = torch.empty(n, dtype=torch.uint32, device="cuda")
    samples = torch.empty((n + 99) // 100, dtype=torch.uint64, device="cuda")
    model = torch.zeros(S.LEARNED_MODEL_BYTES, dtype=torch.uint8, device="cuda")
    sk, sp = torch.empty_like(keys), torch.empty_like(ptrs)
    ok_, oc_ = torch.empty_like(keys), torch.empty_like(keys)
    nk = torch.zeros(1, dtype=torch.uint64, device="cuda")
    st = torch.zeros(len(S.LEARNED_STATS), dtype=torch.uint64, device="cuda")
    lscr = torch.empty(S.sort_learned_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    rscr = torch.empty(S.group_reduce_scratch_bytes(n, 8), dtype=torch.uint8, device="cuda")
    tscr = {}

    def step():
        if fused:
            S.sbh_kpa_extract(col, 0, n, None, None, None, samples, 100)
        else:
            S.sbh_kpa_extract(col, 0, n, keys, ptrs, None, samples, 100)
        tscr["t"] = S.sbh_learned_train(samples, n, None, 40, 4096, 3e-4, model)
        S.sbh_kpa_sort_learned(col if fused else keys, None if fused else ptrs, sk, sp, model, st, scratch=lscr)
        S.sbh_group_reduce(sk, None, None, ok_, oc_, None, n, nk, scratch=rscr)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    pk, pp = S.sort(*S.extract(col, 0, n))
    ek, ec, _ = S.group_reduce(pk, pp, None)
    for _ in range(2):
        sk.zero_()
        oc_.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(sk, pk) and torch.equal(sp, pp)
        m = int(nk.item())
        assert m == ek.numel() and torch.equal(ok_[:m], ek) and torch.equal(oc_[:m], ec)
    assert S.sync_status() == S.SBH_OK


@pytest.mark.parametrize("thr", [0, 1 << 16, 1 << 23, 1 << 40])
def test_overflow_sort_takes_either_path_on_the_device(S, thr):
    # the rows of oversized buckets are sorted with their count known only on
    # the device: below the chunked threshold by the onesweep kernels, from
    # it by the chunked ones (an untrained network overflows ~half the rows)
    n = 3_000_017
    col = gen.mixed_keys(n, seed=19)
    untrained, _ = S.learned_train(cuda(col[::100].copy()), n, cuda(gen.mlp_init()), steps=0, batch=4096, lr=1e-3)
    old = S.get_knob(S.KNOB_SORT_CHUNKED_MIN)
    S.set_knob(S.KNOB_SORT_CHUNKED_MIN, thr)
    try:
        keys, ptrs = S.extract(cuda(col), 0, n)
        sk, sp, st = S.sort_learned(keys, ptrs, untrained)
    finally:
        S.set_knob(S.KNOB_SORT_CHUNKED_MIN, old)
    assert st["overflow_rows"] > 1 << 16
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)


@pytest.mark.parametrize("bins", ["one_key", "two_keys"])
@pytest.mark.parametrize("span_bits", [30, 50])
def test_learned_sort_uneven_wide_buckets(S, bins, span_bits):
    # spread keys plus keys repeated 60-150 times: every bucket holding one
    # is uneven (a fine bin over 32 rows).  Spanning 30 bits, it takes the
    # radix passes on the key; spanning ~44 bits (50-bit keys), it is sorted
    # by a 16-bit group of the key and ranked, unless a group of over 32 rows
    # holds two keys: then it joins the overflow rows.  A repeated key and its
    # neighbour always share a group; a spread key shares one with a
    # repeated key now and then
    rng_keys = gen.uniform(23, 1, 300_000, 0, 1 << span_bits, np.uint64)
    reps = gen.uniform(23, 2, 400, 0, 1 << span_bits, np.uint64)
    parts = [rng_keys, np.repeat(reps, 150)]
    if bins == "two_keys":
        parts.append(np.repeat(reps + np.uint64(1), 60))  # a neighbour key in the same fine bin
    col = np.concatenate(parts)
    col = col[np.argsort(gen.uniform(23, 3, col.size, 0, 0, np.uint64), kind="stable")]
    n = col.size
    model, _ = S.learned_train(cuda(col[::100].copy()), n, None, steps=40, batch=4096, lr=3e-4)
    keys, ptrs = S.extract(cuda(col), 0, n)
    sk, sp, st = S.sort_learned(keys, ptrs, model)
    ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
    assert same(sk, ok) and same(sp, op)
    if span_bits == 30:
        assert st["radix_buckets"] > 0 and st["wide_rows"] == 0
    elif bins == "two_keys":
        assert st["wide_rows"] >= 400 * 210 and st["wide_buckets"] > 0
    else:  # every bucket holds a repeated key: without the group sort all would be wide
        assert st["radix_rows"] > n // 2 and st["wide_rows"] < n // 3
        # runs of several buckets whose group sort failed were retried bucket by bucket
        assert st["retried_buckets"] > 0


def test_learned_sort_ids_sharing_their_low_byte(S):
    # a model trained on uniform 32-bit keys, applied to a window of two keys
    # (2M rows: about 490 buckets): for some second key both keys' bucket ids
    # have the same low byte, so only the pass on the ids' high byte runs,
    # and its chunk counts read the high bytes of the input ids.  The sweep
    # over the second key crosses such ids (found at j = 133-136 of these
    # steps); every window must sort exactly
    n = 2_000_000
    train = cuda(gen.uniform(41, 1, n, 0, 1 << 32, np.uint64))
    model, _ = S.learned_train(train[::100].contiguous(), n, None, steps=40, batch=4096, lr=3e-4)
    order = np.argsort(gen.uniform(41, 2, n, 0, 0, np.uint64), kind="stable")
    k1 = np.uint64(int(0.1 * 2**32))
    step = 2**32 / 488 / 4
    high_only = 0
    for j in range(128, 142):
        k2 = np.uint64(int(0.55 * 2**32 + j * step))
        col = np.where(np.arange(n) < n // 2, k1, k2).astype(np.uint64)[order]
        sk, sp, st = S.sort_learned(cuda(col), None, model)
        assert st["id_passes"] in (2, 3) and st["bucket_ids"] > 256
        if st["id_passes"] == 2:
            high_only += 1
            ok, op = oracle.sort(col, np.arange(n, dtype=np.uint32))
            assert same(sk, ok) and same(sp, op)
        else:  # two keys, stable: each key's rows in input order
            assert same(sp, np.concatenate([np.flatnonzero(col == k1), np.flatnonzero(col == k2)]).astype(np.uint32))
            assert same(sk, np.sort(col))
    assert high_only > 0
