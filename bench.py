"""Benchmark of the KPA grouping path on B300.

One step = one pass of the hot path over one window of the mixed-key
workload: a 0.25% key sample (every 400th key) read from a device key column
of 256M uint64 keys, training of the learned partitioner's network on that
sample, the learned partition sort of the window's (key, row) pairs (the
Extract fused into its first pass: it reads the column and makes each ptr
from its row number), and per-key count (Keyed reduction).  The plain radix sort step is timed on the same window for the
comparison (--sort radix makes it the headline).  Keys are the seeded
mixture of 70% Zipf(1.1) ranks over 2^24 ids and 30% floor(lognormal(30, 4))
below 2^64.  The KPA (3 GB) is larger than the 126 MB L2, so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank sorts its own window (windows are independent:
weak scaling, no collective on the data path); rank 0 prints one JSON line.
The reference arm (--impl reference) times the oracle -- the plain CPU
statement of the same path -- on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FULL = 256_000_000
PAIR_BYTES = 12            # uint64 key + uint32 ptr
WORKLOAD = "mixed_keys_256m"
WORKLOAD_TEXT = ("256M KPA pairs (uint64 key, uint32 row): 70% Zipf(s=1.1) over 2^24 ids, "
                 "30% floor(lognormal(30, 4)) < 2^64; extract + sort + per-key count (the extract fused into "
                 "the sort's first pass: it reads the key column and makes each ptr from its row number)")
METRIC = "records/s grouped"
UNIT = "records/s"
CPU_SAMPLE = 4_000_000
# DRAM bytes per row of one launch (ncu, dram__bytes_read.sum +
# dram__bytes_write.sum on the 16M-row mixed-key window; for the carried-id
# scatter the mean of its two passes, for the radix scatter the mean of the
# second and third passes of a plain sort).
# Traffic grows in proportion to the rows, so a launch on n rows moves about
# n times these.
DRAM_BYTES_PER_ROW = {"learned_ids_scatter": 23.29, "sort_scatter": 23.65}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def window_seed(base, rank):
    """Each rank sorts its own window: the seed of rank r's keys."""
    return base + rank


def max_over_ranks_on(x, ws, device):
    """The largest x over the ranks (every rank gets it)."""
    if ws > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([x], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


def whole_job_rate(steps, rows_per_rank, ws, ms_max):
    """Records per second of the whole job: every rank's rows over the
    slowest rank's time."""
    return steps * rows_per_rank * ws / (ms_max / 1e3)


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU arm
def cpu_oracle_step(col: np.ndarray):
    import oracle
    keys, ptrs = oracle.extract(col, 0, col.size)
    sk, sp = oracle.sort(keys, ptrs)
    uk, uc, _ = oracle.group_sum_count(sk, sp, None)
    return uk.size


def cpu_baseline(sample_rows=CPU_SAMPLE):
    """The oracle on one host thread, and on all host cores (up to 64) with one
    independent window of sample_rows per thread (the oracle's C calls release
    the GIL, so the threads run in parallel)."""
    from concurrent.futures import ThreadPoolExecutor

    import gen
    col = gen.mixed_keys(sample_rows)
    t0 = time.perf_counter()
    cpu_oracle_step(col)
    dt = time.perf_counter() - t0
    cores = max(1, min(64, os.cpu_count() or 1))
    cols = [gen.mixed_keys(sample_rows, seed=window_seed(gen.SEED_MIXED, 1 + i)) for i in range(cores)]
    with ThreadPoolExecutor(cores) as ex:
        t0 = time.perf_counter()
        list(ex.map(cpu_oracle_step, cols))
        dt_all = time.perf_counter() - t0
    return {"value": sample_rows / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {sample_rows:,} rows of the same seeded mixed-key column; std::sort + std::map count, "
                      f"one thread",
            "all_cores": {"value": cores * sample_rows / dt_all, "unit": UNIT, "cores": cores,
                          "sample": f"{cores} independent windows of {sample_rows:,} rows of the same distribution, "
                                    f"one per thread"}}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import gen
    col = gen.mixed_keys(CPU_SAMPLE)
    for _ in range(args.warmup):
        cpu_oracle_step(col[: CPU_SAMPLE // 8])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_step(col)
    dt = time.perf_counter() - t0
    value = args.steps * CPU_SAMPLE / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "text": WORKLOAD_TEXT, "rows_per_step": CPU_SAMPLE,
                   "note": "the oracle on a bounded sample of the workload (one window of 4M rows per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {CPU_SAMPLE:,} rows of the seeded mixed-key column per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
SAMPLE_STRIDE = 400        # 0.25% sample for the learned partitioner (1%: 0.3 ms more a step, more overflow rows)
TRAIN = dict(steps=30, batch=4096, lr=3e-4, init="quantile knots")


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import gen
    from paper_1901_01328_b300 import sbh

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    n = args.rows
    m = (n + SAMPLE_STRIDE - 1) // SAMPLE_STRIDE

    # ---- inputs: each rank draws its own window (seed offset by rank)
    col_h = torch.empty(n, dtype=torch.uint64).pin_memory()
    gen.mixed_keys(n, seed=window_seed(gen.SEED_MIXED, rank), out=col_h.numpy())
    col = col_h.to(dev)
    init = None  # start from the CDF interpolated between 33 sample quantiles
    keys = torch.empty(n, dtype=torch.uint64, device=dev)
    ptrs = torch.empty(n, dtype=torch.uint32, device=dev)
    samples = torch.empty(m, dtype=torch.uint64, device=dev)
    sk = torch.empty(n, dtype=torch.uint64, device=dev)
    sp = torch.empty(n, dtype=torch.uint32, device=dev)
    sort_scratch = torch.empty(sbh.sort_scratch_bytes(n), dtype=torch.uint8, device=dev)
    lsort_scratch = torch.empty(sbh.sort_learned_scratch_bytes(n), dtype=torch.uint8, device=dev)
    model = torch.zeros(sbh.LEARNED_MODEL_BYTES, dtype=torch.uint8, device=dev)
    out_keys = torch.empty(n, dtype=torch.uint64, device=dev)
    out_counts = torch.empty(n, dtype=torch.uint32, device=dev)  # a count is below 2^32: 4 bytes hold it
    nkeys = torch.zeros(1, dtype=torch.uint64, device=dev)
    scr = {}
    stats_d = torch.zeros(len(sbh.LEARNED_STATS), dtype=torch.uint64, device=dev)
    stream = torch.cuda.current_stream(dev)

    outs0 = (out_keys, out_counts, nkeys)

    # Extract is fused into each sort's first pass: the sort reads the key
    # column and makes each row's ptr from its row number (ptrs_in = None),
    # the same KPA an Extract of the window would write; the learned step
    # trains on every SAMPLE_STRIDE-th key of the column
    def step_learned(src=col, outs=outs0):
        sbh.sbh_kpa_extract(src, 0, n, None, None, None, samples, SAMPLE_STRIDE)
        scr["train"] = sbh.sbh_learned_train(samples, n, init, TRAIN["steps"], TRAIN["batch"], TRAIN["lr"], model)
        sbh.sbh_kpa_sort_learned(src, None, sk, sp, model, stats_d, scratch=lsort_scratch)
        scr["red"] = sbh.sbh_group_reduce(sk, None, None, outs[0], outs[1], None, n, outs[2], scratch=scr.get("red"))

    def step_plain(src=col, outs=outs0):
        sbh.sbh_kpa_sort(src, None, sk, sp, scratch=sort_scratch)
        scr["red"] = sbh.sbh_group_reduce(sk, None, None, outs[0], outs[1], None, n, outs[2], scratch=scr.get("red"))

    step = step_plain if args.sort == "radix" else step_learned

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        return max_over_ranks_on(x, ws, dev)

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1))

    def profiled(fn, steps):
        sbh.profile_enable(True)
        for _ in range(steps):
            fn()
        recs = sbh.profile_collect()
        sbh.profile_enable(False)
        per = {}
        for name, t in recs:
            per.setdefault(name, []).append(t)
        return per, len(recs) / steps

    for _ in range(args.warmup):
        step()
    assert sbh.sync_status() == sbh.SBH_OK
    n_unique = int(nkeys.item())

    def verify(src):
        """Outside the timed region: an explicit Extract followed by the plain
        sort gives the KPA the plain step sorts from the column, and the
        learned step's sorted KPA and per-key counts equal the plain step's
        on the same window."""
        sbh.sbh_kpa_extract(src, 0, n, keys, ptrs)
        sbh.sbh_kpa_sort(keys, ptrs, sk, sp, scratch=sort_scratch)
        unfused = (sk.clone(), sp.clone())
        step_plain(src)
        m = int(nkeys.item())
        ref = (sk.clone(), sp.clone(), out_keys[:m].clone(), out_counts[:m].clone())
        same_unfused = torch.equal(unfused[0], ref[0]) and torch.equal(unfused[1], ref[1])
        del unfused
        step_learned(src)
        ok = (same_unfused and sbh.sync_status() == sbh.SBH_OK and int(nkeys.item()) == m and torch.equal(sk, ref[0])
              and torch.equal(sp, ref[1]) and torch.equal(out_keys[:m], ref[2])
              and torch.equal(out_counts[:m], ref[3]))
        del ref
        torch.cuda.empty_cache()
        return bool(ok)

    verified = {"mixed_keys": verify(col)}

    # ---- the step as one CUDA graph: every call of the step only queues work
    # on the stream (no host synchronisation), so it is captured once and
    # replayed; the replay's output is checked against the eager step's
    graphs = {}
    graph_note = None

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            fn()  # allocations the step makes happen before the capture
        stream.wait_stream(side)
        torch.cuda.synchronize(dev)
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize(dev)
        return g

    if not args.no_graph:
        try:
            for name, fn in (("learned", step_learned), ("plain", step_plain)):
                step_plain()
                m = int(nkeys.item())
                ref = (sk.clone(), sp.clone(), out_keys[:m].clone(), out_counts[:m].clone())
                graphs[name] = capture(fn)
                sk.zero_()
                sp.zero_()
                out_counts.zero_()
                graphs[name].replay()
                torch.cuda.synchronize(dev)
                ok = (int(nkeys.item()) == m and torch.equal(sk, ref[0]) and torch.equal(sp, ref[1])
                      and torch.equal(out_keys[:m], ref[2]) and torch.equal(out_counts[:m], ref[3]))
                del ref
                if not ok:
                    raise RuntimeError(f"the replayed {name} graph differs from the eager step")
                verified[f"{name}_graph"] = True
        except Exception as e:  # capture refused: time the eager steps
            graphs = {}
            graph_note = f"eager (capture failed: {type(e).__name__}: {str(e)[:160]})"
        torch.cuda.empty_cache()
    timed_learned = (lambda: graphs["learned"].replay()) if "learned" in graphs else step_learned
    timed_plain = (lambda: graphs["plain"].replay()) if "plain" in graphs else step_plain
    headline = timed_plain if args.sort == "radix" else timed_learned

    # ---- device-resident timing of the headline step
    with Clocks(local) as clk:
        ms = timed(headline, args.steps)
    clocks = clk.summary()
    value = whole_job_rate(args.steps, n, ws, ms)
    assert sbh.sync_status() == sbh.SBH_OK
    stats = sbh.stats_dict(stats_d) if step is step_learned else {}

    # ---- the other sort path on the same window, for the comparison
    other = step_plain if step is step_learned else step_learned
    timed_other = timed_plain if step is step_learned else timed_learned
    for _ in range(2):
        timed_other()
    ms_other = timed(timed_other, args.steps)
    if other is step_learned:
        stats = sbh.stats_dict(stats_d)

    # ---- robustness variant and an external library sort, on the same window size
    variants = None
    if not args.no_rows:
        variants = {}
        # the Zipf ranks through mix64: the same multiplicities, spread over all 64 bits
        col2 = torch.from_numpy(gen.mixed_keys(n, seed=window_seed(gen.SEED_MIXED, rank), hashed=True)).to(dev)
        verified["hashed_zipf"] = verify(col2)
        for _ in range(2):
            step_learned(col2)
        ms_l2 = timed(lambda: step_learned(col2), args.steps)
        st2 = sbh.stats_dict(stats_d)
        for _ in range(2):
            step_plain(col2)
        ms_p2 = timed(lambda: step_plain(col2), args.steps)
        per2, _ = profiled(lambda: step_learned(col2), args.steps)
        assert sbh.sync_status() == sbh.SBH_OK
        variants["hashed_zipf"] = {
            "learned_ms_per_step": ms_l2 / args.steps, "radix_ms_per_step": ms_p2 / args.steps,
            "speedup": ms_p2 / ms_l2, "learned_stats": st2, "overflow_row_rate": st2.get("overflow_rows", 0) / n,
            "stages_ms": {k: sum(v) / args.steps for k, v in per2.items() if sum(v) / args.steps >= 0.05},
            "text": "the headline window with each Zipf rank r replaced by mix64(r) (SplitMix64 output function); "
                    "both steps launched eagerly"}
        del col2
        # a library sort for context: PyTorch's stable sort of the same keys, mapped order-preservingly
        # to int64 (top bit flipped), with int64 indices (16 B per pair against the KPA's 12)
        sbh.sbh_kpa_extract(col, 0, n, keys, ptrs)
        k64 = (keys.view(torch.int64) ^ torch.iinfo(torch.int64).min)
        ts = []
        for r in range(3 + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.sort(k64, stable=True)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if r:
                ts.append(e0.elapsed_time(e1))
        variants["library_sort_ms"] = {"ms": statistics.median(ts),
                                       "text": "torch.sort(stable=True) on the 256M keys as int64 (values and int64 "
                                               "indices out); our sorts on the same keys: see learned_vs_radix stages"}
        del k64
        torch.cuda.empty_cache()

    # ---- per-kernel breakdown (separate, profiled runs of the same steps)
    per, launches_per_step = profiled(step, args.steps)
    tot = {k: sum(v) for k, v in per.items()}
    dominant = max(tot, key=tot.get)
    algo_bytes = {"sort_scatter": PAIR_BYTES * 2 * n, "sort_onesweep": PAIR_BYTES * 2 * n,
                  "sort_count": 8 * n, "extract": (8 + PAIR_BYTES) * n, "sort_upsweep": 8 * n,
                  "keyed_tile_agg": 8 * n, "keyed_emit": 8 * n + 16 * n_unique,
                  # a scatter pass of the learned sort moves a pair in and out (24 B/row); the
                  # kernel's own carried id bytes (the first pass reads 2 and writes 1, the last
                  # reads 1) are not counted
                  "learned_ids_scatter": PAIR_BYTES * 2 * n, "learned_ids_count": 1 * n,
                  "learned_ids_upsweep": (8 + 2) * n, "learned_bucket_sort": PAIR_BYTES * 2 * n}
    peak, peak_kind = _peaks()
    dom_avg_ms = statistics.mean(per[dominant])
    achieved = algo_bytes.get(dominant, 0) / (dom_avg_ms / 1e3) / 1e9
    traffic = DRAM_BYTES_PER_ROW.get(dominant)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                "algorithmic_bytes_per_row": algo_bytes.get(dominant, 0) / n,
                "launch_ms": dom_avg_ms,
                "traffic": traffic * n if traffic else None,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on 16M rows, "
                                   "per row, times the rows of a launch" if traffic else None),
                "algorithmic_bytes_per_launch": algo_bytes.get(dominant)}
    def stage_table(per):
        tot = {k: sum(v) for k, v in per.items()}
        st = {k: {"launches_per_step": len(v) / args.steps, "ms_per_step": sum(v) / args.steps,
                  "share": sum(v) / sum(tot.values())} for k, v in per.items()}
        for k, b in algo_bytes.items():
            if k in per:
                st[k]["gbs"] = b / (statistics.mean(per[k]) / 1e3) / 1e9
        return st

    stages = stage_table(per)
    other_stages = stage_table(profiled(other, args.steps)[0])

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(step, col, col_h, outs0, n, args.steps, dev, barrier, max_over_ranks, ws)

    if rank == 0:
        learned_ms = ms if step is step_learned else ms_other
        radix_ms = ms if step is step_plain else ms_other
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "text": WORKLOAD_TEXT, "rows_per_gpu": n, "sort": args.sort,
                       "launch": ("one CUDA graph per step (captured once, replayed; output checked against the "
                                  "eager step)" if graphs else (graph_note or "eager")),
                       "distinct_keys": n_unique, "l2": "inputs larger than L2 (3 GB KPA per step)",
                       "parallelism": f"replicas{ws}", "train": TRAIN, "sample_stride": SAMPLE_STRIDE},
            "verified": all(verified.values()),
            "verified_detail": {"check": "an explicit extract + plain sort equals the plain step's fused sort, "
                                         "and the learned step's sorted KPA and per-key counts equal the plain "
                                         "radix step's on the same window (torch.equal, outside the timed region)",
                                **verified},
            "roofline": roofline,
            "cpu_baseline": cpu_baseline() if ws == 1 and not args.no_cpu else None,
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clocks,
            "learned_vs_radix": {"learned_ms_per_step": learned_ms / args.steps,
                                 "radix_ms_per_step": radix_ms / args.steps,
                                 "speedup": radix_ms / learned_ms,
                                 "learned_stats": stats,
                                 "overflow_row_rate": stats.get("overflow_rows", 0) / n,
                                 "other_stages": other_stages,
                                 "variants": variants},
            "stages": stages,
            "rows": row_suite(peak) if ws == 1 and not args.no_rows else None,
            "serving": (serving_rows([float(x) for x in args.serve_loads.split(",")], args.serve_windows,
                                     n_windows_rest=args.serve_windows_rest)
                        if ws == 1 and not args.no_rows else None),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def end_to_end(step, col, col_h, outs0, n, steps, dev, barrier, max_over_ranks, ws):
    """The step through the public API with the key column in page-locked
    host memory and the grouped result (distinct keys and their 4-byte
    counts) read back, every step.  Steps are pipelined over three streams: the copy-in of
    step i + 1 and the copy-out of step i - 1 run while step i computes (the
    input column and the outputs are double-buffered)."""
    import torch

    cur = torch.cuda.current_stream(dev)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    cols = [col, torch.empty_like(col)]
    outs = [outs0, tuple(torch.empty_like(t) for t in outs0)]
    res_k = torch.empty(n, dtype=torch.uint64).pin_memory()
    res_c = torch.empty(n, dtype=outs0[1].dtype).pin_memory()
    nk_h = torch.empty(2, dtype=torch.uint64).pin_memory()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    d2h = [0]

    def copy_in(i):
        b = i % 2
        with torch.cuda.stream(s_in):
            if i >= 2:
                s_in.wait_event(ev_done[b])  # step i - 2 has finished reading this buffer
            cols[b].copy_(col_h, non_blocking=True)
            ev_in[b].record(s_in)

    def copy_out(i):
        b = i % 2
        ev_done[b].synchronize()
        m = int(nk_h[b])
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[b])
            res_k[:m].copy_(outs[b][0][:m], non_blocking=True)
            res_c[:m].copy_(outs[b][1][:m], non_blocking=True)
            ev_out[b].record(s_out)
        d2h[0] += 8 + (8 + outs[b][1].element_size()) * m

    barrier()
    t0 = time.perf_counter()
    copy_in(0)
    for i in range(steps):
        b = i % 2
        if i + 1 < steps:
            copy_in(i + 1)
        if i >= 1:
            copy_out(i - 1)
        cur.wait_event(ev_in[b])
        if i >= 2:
            cur.wait_event(ev_out[b])  # the copy-out of step i - 2 has read these outputs
        step(cols[b], outs[b])
        nk_h[b:b + 1].copy_(outs[b][2], non_blocking=True)
        ev_done[b].record(cur)
    copy_out(steps - 1)
    torch.cuda.synchronize(dev)
    barrier()
    dt = max_over_ranks(time.perf_counter() - t0)
    return {"value": steps * n * ws / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
            "d2h_bytes_per_step": d2h[0] // steps, "pipelined": "copy-in of step i+1 and copy-out of step i-1 "
                                                                 "overlap step i (three streams)"}


def serving_rows(loads, n_windows, budget=40e9, n_windows_rest=None):
    """The serving loop in real time: Poisson bundles of U[64K, 1M]
    rows (keys Zipf(0.8) over 50M, u64 values, 5% of rows up to 100 ms
    late), 1 s tumbling windows closed by watermark, per-key sum, count and
    top-3 of every window copied back, memory planned for a 40 GB HBM
    budget.  p50 / p99 window-close latency over the full windows."""
    import torch

    import gen
    from paper_1901_01328_b300 import serve

    win, late = 1_000_000_000, 100_000_000
    seed = gen.SEED_BASE + 5
    pool = serve.BundlePool(gen, 48, 65_536, 1_048_576, 0.8, 50_000_000, 0.05, late, seed)
    mean = float(pool.sizes.mean())
    out = {}
    for li, load in enumerate(loads):
        nw = n_windows if li == 0 or n_windows_rest is None else n_windows_rest
        # the in-place radix close: the keys (Zipf ranks over 50M, 26 bits)
        # take four radix passes, which the learned close does not beat (30.6
        # against 27.4 ms of device time per 250M-row window)
        sort = "radix"
        slot_rows, arena_rows, out_rows = serve.plan(budget, load, win, late, 50_000_000)
        server = serve.WindowServer(win, late, slot_rows, arena_rows, 1_048_576, K=3, keep=False, out_rows=out_rows,
                                    idle_ns=200_000_000, sort=sort)
        arr = serve.poisson_schedule(gen, seed + int(load // 1e6), (nw + 1) * win, load, mean)
        torch.cuda.synchronize()
        wall = serve.run_loop(server, pool, arr, realtime=True, t0_ns=10 * win)
        res = [r for r in server.results if r.rows]
        full = res[1:-1] if len(res) > 2 else res  # the first window starts mid-way; the last closes at the end
        lat = np.array([r.latency_s for r in full]) * 1e3
        dlat = np.array([r.device_latency_s for r in full]) * 1e3
        st = server.stats()
        offered = int(pool.sizes[np.arange(arr.size) % len(pool.bundles)].sum())
        out[f"{load / 1e6:g}M_rows_per_s"] = {
            "offered_rows_per_s": load, "windows": len(full), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "p99_note": (f"np.percentile over {len(full)} closed windows" +
                         (" (fewer than 100: close to the maximum)" if len(full) < 100 else "")),
            "p50_device_ms": float(np.percentile(dlat, 50)), "p99_device_ms": float(np.percentile(dlat, 99)),
            "admitted_rows_per_s": st["admitted_rows"] / (arr[-1] * 1e-9) if arr.size else 0.0,
            "shed_fraction": st["shed_rows"] / max(1, offered), "wall_s": wall, "sort": sort,
            "slot_rows": slot_rows, "arena_rows": arena_rows, **st}
        del server
        torch.cuda.empty_cache()
    out["early_aggregation"] = early_aggregation_rows()
    return out


def early_aggregation_rows(load=2.5e8, seed_off=5):
    """Early per-bundle aggregation (Sec. 4.2 "Keyed Aggregation": each
    bundle's KPA is sorted and aggregated before the window closes, and the
    partial results are merged at the close) against the serving loop's
    design (bundles only appended; one sort of the whole window at the
    close), on one 1 s window of the serving workload at `load` rows/s.
    Early: per bundle, sort + keyed sum/count + top-3 (the partials: one row
    per distinct key of the bundle, and the top-3 rows of each key as
    candidates); at the close, sort the partial rows and reduce their counts
    and sums, sort the candidates and take the top-3 against the values.
    Both closes are timed on the device (CUDA events) and must give the same
    results."""
    import torch

    import gen
    from paper_1901_01328_b300 import sbh, serve

    dev = torch.device("cuda")
    late = 100_000_000
    pool = serve.BundlePool(gen, 48, 65_536, 1_048_576, 0.8, 50_000_000, 0.05, late, gen.SEED_BASE + seed_off)
    sizes = [int(x) for x in pool.sizes]
    nb, W = 0, 0
    while W + sizes[nb % len(sizes)] <= load:
        W += sizes[nb % len(sizes)]
        nb += 1
    # (int64 / int32 views for the concatenation and the index ramps)
    keys = torch.cat([pool.get(i)[0].view(torch.int64).to(dev) for i in range(nb)]).view(torch.uint64)
    vals = torch.cat([pool.get(i)[1].view(torch.int64).to(dev) for i in range(nb)]).view(torch.uint64)
    ptrs = torch.arange(W, dtype=torch.int32, device=dev).view(torch.uint32)
    K = 3

    def ev_ms(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # the loop's close: one sort of the window, keyed sum/count, top-3
    sk, sp = torch.empty_like(keys), torch.empty_like(ptrs)
    sort_scr = torch.empty(sbh.sort_scratch_bytes(W), dtype=torch.uint8, device=dev)
    rk, rc, rs = (torch.empty(W, dtype=torch.uint64, device=dev) for _ in range(3))
    rn = torch.empty(1, dtype=torch.uint64, device=dev)
    tk, tn = torch.empty(W, dtype=torch.uint64, device=dev), torch.empty(W, dtype=torch.uint8, device=dev)
    tv, tp = torch.empty(W * K, dtype=torch.uint64, device=dev), torch.empty(W * K, dtype=torch.uint32, device=dev)
    tnk = torch.empty(1, dtype=torch.uint64, device=dev)
    scr = {}

    def close_raw():
        sbh.sbh_kpa_sort(keys, ptrs, sk, sp, scratch=sort_scr)
        scr["r"] = sbh.sbh_group_reduce(sk, sp, vals, rk, rc, rs, W, rn, scratch=scr.get("r"))
        scr["t"] = sbh.sbh_topk(sk, sp, vals, K, tk, tn, tv, tp, W, tnk, scratch=scr.get("t"))

    close_raw()
    raw_ms = statistics.median(ev_ms(close_raw) for _ in range(3))
    m = int(rn.item())
    ref = (rk[:m].clone(), rc[:m].clone(), rs[:m].clone(), tn[:m].clone(), tv[:m * K].clone(), tp[:m * K].clone())

    # early: per-bundle partials (their device time summed), then the close
    pk, pc, ps = (torch.empty(W, dtype=torch.uint64, device=dev) for _ in range(3))
    ck, cp = torch.empty(W, dtype=torch.uint64, device=dev), torch.empty(W, dtype=torch.uint32, device=dev)
    bk, bp = torch.empty(1 << 20, dtype=torch.uint64, device=dev), torch.empty(1 << 20, dtype=torch.uint32, device=dev)
    bnk, btk = torch.empty(1, dtype=torch.uint64, device=dev), torch.empty(1 << 20, dtype=torch.uint64, device=dev)
    btnk = torch.empty(1, dtype=torch.uint64, device=dev)
    btn = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    btv = torch.empty(K << 20, dtype=torch.uint64, device=dev)
    btp = torch.empty(K << 20, dtype=torch.uint32, device=dev)
    bscr = torch.empty(sbh.sort_scratch_bytes(1 << 20), dtype=torch.uint8, device=dev)
    scr["br"] = torch.empty(sbh.group_reduce_scratch_bytes(1 << 20, 8), dtype=torch.uint8, device=dev)
    scr["bt"] = torch.empty(sbh.topk_scratch_bytes(1 << 20, K, 8), dtype=torch.uint8, device=dev)
    P = C = 0
    per_bundle_ms = 0.0
    o = 0
    for b in range(nb):
        n = sizes[b % len(sizes)]

        def partial():
            sbh.sbh_kpa_sort(keys[o:o + n], ptrs[o:o + n], bk[:n], bp[:n], scratch=bscr)
            sbh.sbh_group_reduce(bk[:n], bp[:n], vals, pk[P:], pc[P:], ps[P:], n, bnk, scratch=scr["br"])
            sbh.sbh_topk(bk[:n], bp[:n], vals, K, btk, btn, btv, btp, n, btnk, scratch=scr["bt"])
        per_bundle_ms += ev_ms(partial)
        u = int(bnk.item())
        # candidates: each key's valid top-3 slots, as (key, ptr) rows (host-side glue of this measurement)
        valid = (torch.arange(K, device=dev)[None, :] < btn[:u, None].to(torch.int64)).flatten()
        cand_k = btk[:u].view(torch.int64).repeat_interleave(K)[valid]
        cand_p = btp[:u * K].view(torch.int32)[valid]
        c = cand_k.numel()
        ck[C:C + c].view(torch.int64).copy_(cand_k)
        cp[C:C + c].view(torch.int32).copy_(cand_p)
        P += u
        C += c
        o += n
    pidx = torch.arange(P, dtype=torch.int32, device=dev).view(torch.uint32)
    qk, qp = torch.empty(P, dtype=torch.uint64, device=dev), torch.empty(P, dtype=torch.uint32, device=dev)
    xk, xp = torch.empty(C, dtype=torch.uint64, device=dev), torch.empty(C, dtype=torch.uint32, device=dev)
    ek, ec, es = (torch.empty(P, dtype=torch.uint64, device=dev) for _ in range(3))
    en = torch.empty(1, dtype=torch.uint64, device=dev)
    e2 = torch.empty(P, dtype=torch.uint64, device=dev)
    fk, fn_ = torch.empty(C, dtype=torch.uint64, device=dev), torch.empty(C, dtype=torch.uint8, device=dev)
    fv, fp = torch.empty(C * K, dtype=torch.uint64, device=dev), torch.empty(C * K, dtype=torch.uint32, device=dev)
    fnk = torch.empty(1, dtype=torch.uint64, device=dev)

    def close_early():
        sbh.sbh_kpa_sort(pk[:P], pidx, qk, qp, scratch=sort_scr)
        sbh.sbh_group_reduce(qk, qp, pc[:P], ek, e2, ec, P, en)   # counts: the sum of the partial counts
        sbh.sbh_group_reduce(qk, qp, ps[:P], ek, e2, es, P, en)   # sums: the sum of the partial sums
        sbh.sbh_kpa_sort(ck[:C], cp[:C], xk, xp, scratch=sort_scr)
        sbh.sbh_topk(xk, xp, vals, K, fk, fn_, fv, fp, C, fnk)

    close_early()
    early_ms = statistics.median(ev_ms(close_early) for _ in range(3))
    me = int(en.item())
    same = (me == m and torch.equal(ek[:m], ref[0]) and torch.equal(ec[:m], ref[1]) and torch.equal(es[:m], ref[2])
            and torch.equal(fn_[:m], ref[3]) and torch.equal(fv[:m * K], ref[4]) and torch.equal(fp[:m * K], ref[5]))
    out = {"load_rows_per_s": load, "bundles": nb, "window_rows": W, "distinct_keys": m,
           "partial_rows": P, "candidate_rows": C, "partial_fraction": P / W,
           "close_ms_one_sort": raw_ms, "close_ms_early": early_ms, "per_bundle_ms_total_early": per_bundle_ms,
           "same_results": bool(same),
           "text": "one 1 s window of the serving workload; device time of the window close, and of the "
                   "per-bundle partial aggregation that early aggregation adds during the window"}
    del keys, vals, ptrs, sk, sp, sort_scr, rk, rc, rs, tk, tn, tv, tp, pk, pc, ps, ck, cp, qk, qp, xk, xp
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ per-row measurements
def row_suite(peak):
    """Each remaining row of the path on its workload shape: device time by
    CUDA events (the call captured in a CUDA graph, the median of 9 replays,
    each after a 256 MB write that flushes L2: device time from HBM, without
    the host's per-call work), algorithmic GB/s against the HBM peak, and the
    oracle on the same input (one host thread)."""
    import torch

    import gen
    import oracle
    from paper_1901_01328_b300 import sbh

    dev = torch.device("cuda")
    out = {}

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # twice the L2

    def dev_ms(fn, reps=9):
        """Device time of one call: the call (which only queues work) is
        captured once in a CUDA graph and replayed, so that the host's
        per-call work (argument marshalling, launches) is not timed; the
        median of reps replays, each after an L2 flush."""
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            fn()  # first-call work (scratch sizing) outside the capture
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        g.replay()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            flush.zero_()  # L2 flushed: every replay reads its inputs from HBM
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        del g
        return statistics.median(ts)

    def cpu_ms(fn):
        t0 = time.perf_counter()
        fn()
        return 1e3 * (time.perf_counter() - t0)

    def entry(ms, nbytes, shape, oms):
        gbs = nbytes / (ms / 1e3) / 1e9 if nbytes else None
        return {"ms": ms, "algorithmic_gbs": gbs, "frac_of_hbm": (gbs / peak if gbs else None), "shape": shape,
                "oracle_ms": oms}

    # A1 window ranges: 509 sliding windows (1M rows, stride 250K) over 128M timestamps
    nrow = 128_000_000
    ts = torch.arange(nrow, dtype=torch.int64, device=dev).to(torch.uint64)
    starts = torch.arange(0, 509 * 250_000, 250_000, dtype=torch.int64, device=dev).to(torch.uint64)
    rb = torch.empty(509, dtype=torch.uint64, device=dev)
    re_ = torch.empty_like(rb)
    ms = dev_ms(lambda: sbh.sbh_window_ranges(ts, starts, 1_000_000, rb, re_))
    ts_h = np.arange(4_000_000, dtype=np.uint64)
    oms = cpu_ms(lambda: oracle.window_ranges(ts_h, np.array([0, 250_000, 500_000, 750_000], np.uint64), 1_000_000))
    out["A1_window_ranges"] = entry(ms, None, "509 windows over 128M u64 timestamps (oracle: 4 windows over 4M rows)",
                                    oms)
    del ts

    # A5 merge: one window of the join workload = 4 sorted panes of 250K rows
    s = gen.join_streams(1_000_000)
    col = s["L"]["keys"]
    d_col = torch.from_numpy(col).to(dev)
    panes = [sbh.sort(*sbh.extract(d_col, i * 250_000, 250_000)) for i in range(4)]
    total = 1_000_000
    mk = torch.empty(total, dtype=torch.uint64, device=dev)
    mp = torch.empty(total, dtype=torch.uint32, device=dev)
    ms = dev_ms(lambda: sbh.sbh_kpa_merge(panes, mk, mp))
    hp = [(p[0].cpu().numpy(), p[1].cpu().numpy()) for p in panes]
    oms = cpu_ms(lambda: oracle.merge(hp))
    out["A5_merge"] = entry(ms, 2 * 24 * total, "4 sorted panes x 250K -> 1M (two rounds of pairwise merges)", oms)
    # and a large two-run merge
    big = 128_000_000
    bcol = gen.uniform(5, 5, big, 0, 1 << 40, np.uint64)
    d_b = torch.from_numpy(bcol).to(dev)
    r1 = sbh.sort(*sbh.extract(d_b, 0, big // 2))
    r2 = sbh.sort(*sbh.extract(d_b, big // 2, big // 2))
    bk = torch.empty(big, dtype=torch.uint64, device=dev)
    bp = torch.empty(big, dtype=torch.uint32, device=dev)
    ms = dev_ms(lambda: sbh.sbh_kpa_merge([r1, r2], bk, bp))
    out["A5_merge_large"] = entry(ms, 24 * big, "2 sorted runs x 64M -> 128M", None)
    del d_b, r1, r2, bk, bp

    # A6 keyed sum/count: the tumbling window (1M rows, u32 values)
    w = gen.tumbling_window(1_000_000)
    sk, sp = sbh.sort(*sbh.extract(torch.from_numpy(w["keys"]).to(dev), 0, 1_000_000))
    vals = torch.from_numpy(w["vals"]).to(dev)
    ok = torch.empty(1_000_000, dtype=torch.uint64, device=dev)
    oc = torch.empty_like(ok)
    osum = torch.empty_like(ok)
    nk = torch.empty(1, dtype=torch.uint64, device=dev)
    red_scr = torch.empty(sbh.group_reduce_scratch_bytes(1_000_000, 4), dtype=torch.uint8, device=dev)
    ms = dev_ms(lambda: sbh.sbh_group_reduce(sk, sp, vals, ok, oc, osum, 1_000_000, nk, scratch=red_scr))
    hk, hp_ = sk.cpu().numpy(), sp.cpu().numpy()
    oms = cpu_ms(lambda: oracle.group_sum_count(hk, hp_, w["vals"]))
    nkeys = int(nk.item())
    out["A6_keyed_sum_count"] = entry(ms, 1_000_000 * (12 + 4) + 24 * nkeys,
                                      "1M-row tumbling window, u32 values (L2-resident)", oms)

    # A7 top-3: one 4M-row window of the batched workload (Zipf(1.0) keys, u64 values)
    nb_ = 4_000_000
    bk_ = gen.zipf(gen.SEED_BATCHED, 2, nb_, 1.0, 10_000_000)
    bv_ = gen.uniform(gen.SEED_BATCHED, 3, nb_, 0, 0, np.uint64)
    tsk, tsp = sbh.sort(*sbh.extract(torch.from_numpy(bk_).to(dev), 0, nb_))
    tv = torch.from_numpy(bv_).to(dev)
    K = 3
    tk = torch.empty(nb_, dtype=torch.uint64, device=dev)
    tn = torch.empty(nb_, dtype=torch.uint8, device=dev)
    tvo = torch.empty(nb_ * K, dtype=torch.uint64, device=dev)
    tpo = torch.empty(nb_ * K, dtype=torch.uint32, device=dev)
    tnk = torch.empty(1, dtype=torch.uint64, device=dev)
    ms = dev_ms(lambda: sbh.sbh_topk(tsk, tsp, tv, K, tk, tn, tvo, tpo, nb_, tnk))
    hk, hp_ = tsk.cpu().numpy(), tsp.cpu().numpy()
    oms = cpu_ms(lambda: oracle.topk(hk, hp_, bv_, K))
    m = int(tnk.item())
    out["A7_topk"] = entry(ms, nb_ * (12 + 8) + m * (8 + 1 + K * 12), "4M-row window, K=3, Zipf(1.0) keys", oms)

    # A8 join: one 1M x 1M sliding window of the two join streams
    lcol, rcol = s["L"]["keys"], s["R"]["keys"]
    L = sbh.sort(*sbh.extract(torch.from_numpy(lcol).to(dev), 0, 1_000_000))
    R = sbh.sort(*sbh.extract(torch.from_numpy(rcol).to(dev), 0, 1_000_000))
    cap = 1 << 20
    jl = torch.empty(cap, dtype=torch.uint32, device=dev)
    jr = torch.empty(cap, dtype=torch.uint32, device=dev)
    npairs = torch.empty(1, dtype=torch.uint64, device=dev)
    ms = dev_ms(lambda: sbh.sbh_join(L[0], L[1], R[0], R[1], jl, jr, cap, npairs))
    lh, rh = (L[0].cpu().numpy(), L[1].cpu().numpy()), (R[0].cpu().numpy(), R[1].cpu().numpy())
    oms = cpu_ms(lambda: oracle.join(lh[0], lh[1], rh[0], rh[1]))
    pairs = int(npairs.item())
    out["A8_join"] = entry(ms, 2 * 1_000_000 * 12 + pairs * 8, f"1M x 1M window, keys U[0,2^24), {pairs} pairs", oms)

    # Table 2 record primitives and per-key statistics, on the 4M-row top-K window
    mat = torch.empty(nb_, dtype=torch.uint64, device=dev)
    ms = dev_ms(lambda: sbh.sbh_kpa_materialize(tsp, tv, mat))
    hp_ = tsp.cpu().numpy()
    oms = cpu_ms(lambda: oracle.materialize(hp_, bv_))
    out["materialize"] = entry(ms, nb_ * (4 + 32 + 8), "4M ptrs, u64 column gathered (a 32-byte sector per row)", oms)
    lo_, hi_ = 0, 1 << 63
    sel_k = torch.empty(nb_, dtype=torch.uint64, device=dev)
    sel_p = torch.empty(nb_, dtype=torch.uint32, device=dev)
    sel_n = torch.empty(1, dtype=torch.uint64, device=dev)
    scr_sel = sbh.sbh_kpa_select(tsk, tsp, tv, lo_, hi_, sel_k, sel_p, nb_, sel_n)
    ms = dev_ms(lambda: sbh.sbh_kpa_select(tsk, tsp, tv, lo_, hi_, sel_k, sel_p, nb_, sel_n, scratch=scr_sel))
    kept = int(sel_n.item())
    hk_ = tsk.cpu().numpy()
    oms = cpu_ms(lambda: oracle.select(hk_, hp_, bv_, lo_, hi_))
    out["select"] = entry(ms, 2 * nb_ * (4 + 32) + kept * 12, f"4M rows, values in [0, 2^63): {kept} kept", oms)
    mk_ = torch.empty(nb_, dtype=torch.uint64, device=dev)
    mm_ = torch.empty(nb_, dtype=torch.uint64, device=dev)
    mu_ = torch.empty(nb_, dtype=torch.uint64, device=dev)
    mn_ = torch.empty(1, dtype=torch.uint64, device=dev)
    scr_mu = sbh.sbh_median_unique(tsk, tsp, tv, mk_, mm_, mu_, nb_, mn_)
    ms = dev_ms(lambda: sbh.sbh_median_unique(tsk, tsp, tv, mk_, mm_, mu_, nb_, mn_, scratch=scr_mu))
    oms = cpu_ms(lambda: oracle.median_unique(hk_, hp_, bv_))
    out["median_unique"] = entry(ms, None, "4M-row window, Zipf(1.0) keys: lower median and distinct values per key "
                                 "(two stable radix sorts)", oms)
    del L, R, jl, jr, tsk, tsp, tv, tk, tn, tvo, tpo, mat, sel_k, sel_p, mk_, mm_, mu_, scr_sel, scr_mu, flush
    out.update(pipeline_rows())
    return out


def pipeline_rows():
    """The two window pipelines on their full workloads, wall-clock (each
    includes its host synchronisations), with the oracle on sampled windows."""
    import torch

    import gen
    import oracle
    from paper_1901_01328_b300 import pipeline

    dev = torch.device("cuda")
    out = {}

    def wall_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(1e3 * (time.perf_counter() - t0))
        return statistics.median(ts)

    # batched windows: 4096 tumbling windows, per-key count, sum and top-3
    b = gen.batched_windows()
    keys, vals, off = b["keys"], b["vals"], b["offsets"]
    n = int(off[-1])
    kd, vd = torch.from_numpy(keys).to(dev), torch.from_numpy(vals).to(dev)
    ms_b = wall_ms(lambda: pipeline.batched_windows(kd, vd, off, K=3, schedule="batched"))
    ms_l = wall_ms(lambda: pipeline.batched_windows(kd, vd, off, K=3, schedule="loop"), reps=1)
    sample = range(0, 4096, 512)
    rows_s = int(sum(off[w + 1] - off[w] for w in sample))
    t0 = time.perf_counter()
    for w in sample:
        k, p = oracle.sort(*oracle.extract(keys, int(off[w]), int(off[w + 1] - off[w])))
        oracle.group_sum_count(k, p, vals)
        oracle.topk(k, p, vals, 3)
    oms = 1e3 * (time.perf_counter() - t0)
    out["batched_windows_4096"] = {
        "rows": n, "windows": 4096, "batched_ms": ms_b, "loop_ms": ms_l,
        "batched_rows_per_s": n / (ms_b / 1e3), "loop_rows_per_s": n / (ms_l / 1e3),
        "oracle_rows_per_s": rows_s / (oms / 1e3), "oracle_sample": f"8 windows, {rows_s} rows, one thread",
        "shape": "4096 windows, sizes lognormal(10.4, 1.5) in [1K, 4M], Zipf(1.0) keys over 10M, u64 values, K=3"}
    del kd, vd, b, keys, vals
    torch.cuda.empty_cache()

    # sliding-window temporal join: 2 x 128M rows in page-locked host memory
    s = gen.join_streams()
    lcol, rcol = s["L"]["keys"], s["R"]["keys"]
    lh = torch.from_numpy(lcol.view(np.int64)).pin_memory().view(torch.uint64)
    rh = torch.from_numpy(rcol.view(np.int64)).pin_memory().view(torch.uint64)
    res = {}

    def run():
        res["r"] = pipeline.sliding_join(lh, rh, lcol.size)

    ms_j = wall_ms(run, reps=1)
    pairs = int(res["r"][0].npairs.sum())
    res.clear()
    torch.cuda.empty_cache()
    ms_loop = wall_ms(lambda: res.__setitem__("r", pipeline.sliding_join(lh, rh, lcol.size, schedule="loop")), reps=1)
    assert int(res["r"][0].npairs.sum()) == pairs
    res.clear()
    t0 = time.perf_counter()
    lk, lp = oracle.sort(*oracle.extract(lcol, 0, 1_000_000))
    rk, rp = oracle.sort(*oracle.extract(rcol, 0, 1_000_000))
    oracle.join(lk, lp, rk, rp)
    oms = 1e3 * (time.perf_counter() - t0)
    out["sliding_join_509"] = {
        "rows_per_side": int(lcol.size), "windows": 509, "ms": ms_j, "windows_per_s": 509 / (ms_j / 1e3),
        "loop_ms": ms_loop,
        "schedule": "batched, in eight groups of windows whose host copies overlap the earlier groups' work: per "
                    "group and side one composite-key sort of its panes, one segmented merge launch per level, one "
                    "segmented join for its windows (loop_ms: per-pane sorts and per-window merge + join)",
        "pairs": pairs, "h2d_bytes": 2 * 8 * int(lcol.size), "oracle_ms_per_window": oms,
        "shape": "2 x 128M keys U[0, 2^24) in pinned host memory; 1M-row windows, stride 250K; panes sorted once"}

    # a chained pipeline: 64M ad events, 1 s windows, views per campaign
    del lh, rh, res
    torch.cuda.empty_cache()
    cols, camp = gen.ad_events(64_000_000)
    dcols = {k: torch.from_numpy(v).to(dev) for k, v in cols.items()}
    dcamp = torch.from_numpy(camp).to(dev)
    ms_a = wall_ms(lambda: pipeline.ad_campaign_counts(dcols, dcamp, 1_000_000_000), reps=3)
    ts, et, ad = cols["event_time"], cols["event_type"], cols["ad_id"]
    lo, hi = np.searchsorted(ts, [0, 1_000_000_000])
    t0 = time.perf_counter()
    k, p = oracle.extract(et, int(lo), int(hi - lo))
    sk, sp = oracle.select(k, p, et, 0, 1)
    c = oracle.materialize(oracle.materialize(sp, ad).astype(np.uint32), camp)
    oracle.group_sum_count(*oracle.sort(c, sp), None)
    oms = 1e3 * (time.perf_counter() - t0)
    out["ad_campaign_chain"] = {
        "events": 64_000_000, "windows": int(ts[-1] // 1_000_000_000) + 1, "ms": ms_a,
        "events_per_s": 64e6 / (ms_a / 1e3), "oracle_events_per_s": float(hi - lo) / (oms / 1e3),
        "shape": "7-column ad events at 1e7/s; Extract -> Select(view) -> KeySwap(ad -> campaign) -> Sort -> "
                 "count, per 1 s window (wall clock, a synchronisation per window)"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sbh", choices=["sbh", "reference"])
    ap.add_argument("--rows", type=int, default=N_FULL)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time the eager steps instead of one CUDA graph per step")
    ap.add_argument("--sort", default="learned", choices=["learned", "radix"])
    ap.add_argument("--no-rows", action="store_true", help="skip the per-row measurements")
    ap.add_argument("--serve-windows", type=int, default=62,
                    help="1 s windows at the first offered load (serving loop; the first and last are not counted)")
    ap.add_argument("--serve-windows-rest", type=int, default=6, help="1 s windows at each further offered load")
    ap.add_argument("--serve-loads", default="2.5e8,1e9", help="offered loads, rows/s")
    ap.add_argument("--serve-only", action="store_true", help="print only the serving-loop measurement")
    args = ap.parse_args()
    if args.serve_only:
        loads = [float(x) for x in args.serve_loads.split(",")]
        print(json.dumps({"metric": "window-close latency", "unit": "ms",
                          "serving": serving_rows(loads, args.serve_windows, n_windows_rest=args.serve_windows_rest)}),
              flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
