"""The multi-GPU path's host logic on CPU: two gloo ranks, as torchrun would
launch them, agree on the slowest rank's time, draw different windows, and
compute the whole-job rate from all ranks' rows (weak scaling, replicas: no
collective touches the data)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    import gen

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ws_, r_, _ = bench._dist()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    slowest = bench.max_over_ranks_on(ms, ws_, "cpu")
    keys = gen.mixed_keys(1000, seed=bench.window_seed(gen.SEED_MIXED, r_))
    q.put((r_, slowest, bench.whole_job_rate(3, 1000, ws_, slowest), int(keys.sum() % (1 << 62))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_time_and_draw_distinct_windows():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, v0, k0), (r1, s1, v1, k1) = out
    assert (r0, r1) == (0, 1)
    assert s0 == s1 == 15.0                       # max over ranks
    assert v0 == v1 == 3 * 1000 * 2 / 0.015       # all ranks' rows over the slowest time
    assert k0 != k1                               # each rank sorts its own window
