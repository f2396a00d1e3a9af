"""Benchmark of the KPA grouping path on B300.

One step = one pass of the hot path over one window of the mixed-key
workload: Extract of 256M (uint64 key, uint32 row) pairs from a device key
column with a 1% key sample, training of the learned partitioner's network on
that sample, the learned partition sort, and per-key count (Keyed
reduction).  The plain radix sort step is timed on the same window for the
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
                 "30% floor(lognormal(30, 4)) < 2^64; extract + sort + per-key count")
METRIC = "records/s grouped"
UNIT = "records/s"
CPU_SAMPLE = 4_000_000


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
    import gen
    col = gen.mixed_keys(sample_rows)
    t0 = time.perf_counter()
    cpu_oracle_step(col)
    dt = time.perf_counter() - t0
    return {"value": sample_rows / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {sample_rows:,} rows of the same seeded mixed-key column; std::sort + std::map count, "
                      f"one thread"}


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
SAMPLE_STRIDE = 100        # 1% sample for the learned partitioner
TRAIN = dict(steps=40, batch=16384, lr=4e-2)


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
    gen.mixed_keys(n, seed=gen.SEED_MIXED + rank, out=col_h.numpy())
    col = col_h.to(dev)
    init = torch.from_numpy(gen.mlp_init()).to(dev)
    keys = torch.empty(n, dtype=torch.uint64, device=dev)
    ptrs = torch.empty(n, dtype=torch.uint32, device=dev)
    samples = torch.empty(m, dtype=torch.uint64, device=dev)
    sk = torch.empty(n, dtype=torch.uint64, device=dev)
    sp = torch.empty(n, dtype=torch.uint32, device=dev)
    sort_scratch = torch.empty(sbh.sort_scratch_bytes(n), dtype=torch.uint8, device=dev)
    lsort_scratch = torch.empty(sbh.sort_learned_scratch_bytes(n), dtype=torch.uint8, device=dev)
    model = torch.zeros(sbh.LEARNED_MODEL_BYTES, dtype=torch.uint8, device=dev)
    out_keys = torch.empty(n, dtype=torch.uint64, device=dev)
    out_counts = torch.empty(n, dtype=torch.uint64, device=dev)
    nkeys = torch.zeros(1, dtype=torch.uint64, device=dev)
    scr = {}
    stats = {}
    stream = torch.cuda.current_stream(dev)

    def step_learned(src=col):
        sbh.sbh_kpa_extract(src, 0, n, keys, ptrs, None, samples, SAMPLE_STRIDE)
        scr["train"] = sbh.sbh_learned_train(samples, n, init, TRAIN["steps"], TRAIN["batch"], TRAIN["lr"], model)
        stats.update(sbh.sbh_kpa_sort_learned(keys, ptrs, sk, sp, model, scratch=lsort_scratch))
        scr["red"] = sbh.sbh_group_reduce(sk, None, None, out_keys, out_counts, None, n, nkeys,
                                          scratch=scr.get("red"))

    def step_plain(src=col):
        sbh.sbh_kpa_extract(src, 0, n, keys, ptrs)
        sbh.sbh_kpa_sort(keys, ptrs, sk, sp, scratch=sort_scratch)
        scr["red"] = sbh.sbh_group_reduce(sk, None, None, out_keys, out_counts, None, n, nkeys,
                                          scratch=scr.get("red"))

    step = step_plain if args.sort == "radix" else step_learned

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        if ws > 1:
            t = torch.tensor([x], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        return x

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

    # ---- device-resident timing of the headline step
    with Clocks(local) as clk:
        ms = timed(step, args.steps)
    clocks = clk.summary()
    value = args.steps * n * ws / (ms / 1e3)
    assert sbh.sync_status() == sbh.SBH_OK

    # ---- the other sort path on the same window, for the comparison
    other = step_plain if step is step_learned else step_learned
    for _ in range(2):
        other()
    ms_other = timed(other, args.steps)

    # ---- per-kernel breakdown (separate, profiled runs of the same steps)
    per, launches_per_step = profiled(step, args.steps)
    tot = {k: sum(v) for k, v in per.items()}
    dominant = max(tot, key=tot.get)
    algo_bytes = {"sort_scatter": PAIR_BYTES * 2 * n, "sort_onesweep": PAIR_BYTES * 2 * n,
                  "sort_count": 8 * n, "extract": (8 + PAIR_BYTES) * n, "sort_upsweep": 8 * n,
                  "keyed_tile_agg": 8 * n, "keyed_emit": 8 * n + 16 * n_unique,
                  "learned_ids_scatter": PAIR_BYTES * 2 * n, "learned_ids_count": 8 * n,
                  "learned_ids_upsweep": 8 * n, "learned_bucket_sort": PAIR_BYTES * 2 * n,
                  "learned_bounds": 8 * n}
    peak, peak_kind = _peaks()
    dom_avg_ms = statistics.mean(per[dominant])
    achieved = algo_bytes.get(dominant, 0) / (dom_avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                "algorithmic_bytes_per_launch": algo_bytes.get(dominant)}
    stages = {k: {"launches_per_step": len(v) / args.steps, "ms_per_step": sum(v) / args.steps,
                  "share": sum(v) / sum(tot.values())} for k, v in per.items()}
    for k, b in algo_bytes.items():
        if k in per:
            stages[k]["gbs"] = b / (statistics.mean(per[k]) / 1e3) / 1e9

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        res_k = torch.empty(n, dtype=torch.uint64).pin_memory()
        res_c = torch.empty(n, dtype=torch.uint64).pin_memory()
        nk_h = torch.empty(1, dtype=torch.uint64).pin_memory()
        d2h = 0
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            col.copy_(col_h, non_blocking=True)
            step()
            nk_h.copy_(nkeys, non_blocking=True)
            torch.cuda.synchronize(dev)
            mk = int(nk_h[0])
            res_k[:mk].copy_(out_keys[:mk], non_blocking=True)
            res_c[:mk].copy_(out_counts[:mk], non_blocking=True)
            d2h += 8 + 16 * mk
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": args.steps * n * ws / dt, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": d2h // args.steps}

    if rank == 0:
        learned_ms = ms if step is step_learned else ms_other
        radix_ms = ms if step is step_plain else ms_other
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "text": WORKLOAD_TEXT, "rows_per_gpu": n, "sort": args.sort,
                       "distinct_keys": n_unique, "l2": "inputs larger than L2 (3 GB KPA per step)",
                       "parallelism": f"replicas{ws}", "train": TRAIN, "sample_stride": SAMPLE_STRIDE},
            "roofline": roofline,
            "cpu_baseline": cpu_baseline() if ws == 1 and not args.no_cpu else None,
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clocks,
            "learned_vs_radix": {"learned_ms_per_step": learned_ms / args.steps,
                                 "radix_ms_per_step": radix_ms / args.steps,
                                 "speedup": radix_ms / learned_ms,
                                 "learned_stats": stats,
                                 "overflow_row_rate": stats.get("overflow_rows", 0) / n},
            "stages": stages,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sbh", choices=["sbh", "reference"])
    ap.add_argument("--rows", type=int, default=N_FULL)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--sort", default="learned", choices=["learned", "radix"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
