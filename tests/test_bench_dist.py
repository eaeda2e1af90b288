"""Host logic of the multi-GPU benchmark (one independent instance per rank, weak scaling), run as
world-size-2 gloo process groups on the CPU: the slowest rank's time is what every rank reports,
the whole-job value counts every rank's work, and the reference arm runs on rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.dist_env()
        t_rank = [0.25, 0.75][rank]                 # rank 1 is the slow one
        t = bench.max_over_ranks(t_rank, w, torch.device("cpu"))
        units = 2.0 * 1000 * 50                     # 2 N Nt of one rank's instance
        value = bench.aggregate_gpts(units, w, t)
        # the reference arm prints its line on rank 0 only; the other ranks return silently
        buf = io.StringIO()

        class A:
            workload, steps, warmup, gpus = "disc2d_168", 1, 0, w

        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(A)
        dist.barrier()
        q.put((rank, (w, r, lr), t, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_the_whole_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, env, t, value, out = q.get(timeout=120)
        res[rank] = (env, t, value, out)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        env, t, value, out = res[rank]
        assert env == (world, rank, rank)
        assert t == 0.75                                     # max over ranks
        assert abs(value - 2 * 2.0 * 1000 * 50 / 0.75 / 1e9) < 1e-18
    assert res[1][3] == ""                                   # no reference line on rank 1


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.aggregate_gpts(2e9, 1, 2.0) == 1.0
    assert json.dumps(bench.dist_env()) is not None


def test_cpu_baseline_all_cores_counts_every_replica():
    """The all-cores oracle leg: spawned single-thread replicas of the same bounded sample, the
    value counting every replica's grid-point-steps over the span from the first start to the
    last end, so it is at most the replicas' count times one replica's rate."""
    sys.path.insert(0, ROOT)
    import bench

    r = bench.cpu_baseline_all_cores("disc2d_168", 60, cores=2, timeout_s=120.0)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["unit"] == bench.UNIT
    assert r["span_s"] > 0
    units = 2 * 2.0 * 168 * 168 * 60     # 2 replicas x 2 N Nt_s
    assert r["value"] == pytest.approx(units / r["span_s"] / 1e9, rel=1e-12)


def test_cpu_baseline_all_cores_fails_fast_when_a_replica_fails():
    """A replica that raises (here: a workload name whose grid size does not parse) ends the leg
    with an error at once instead of leaving the others waiting at the start barrier."""
    import time

    sys.path.insert(0, ROOT)
    import bench

    t0 = time.perf_counter()
    with pytest.raises(RuntimeError):
        bench.cpu_baseline_all_cores("tube3d_x", 2, cores=2, timeout_s=60.0)
    assert time.perf_counter() - t0 < 45.0
