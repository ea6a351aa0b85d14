"""The benchmark's multi-rank host logic on CPU: two gloo ranks.

Replicas only (the path needs no exchange): every rank prices the same
request on its own random stream, the step time is the slowest rank's, the
throughput counts the units of all ranks, and the reference arm runs on
rank 0 alone."""
import contextlib
import io
import json
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2206_03719_gb300 import workloads

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = bench.replica_workload(workloads.PAPER_FP64, rank)
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, dist, "cpu")
        value = bench.job_throughput(world, wl.n_greeks, ms_max)

        # the reference arm: the oracle timing replaced by a fixed figure
        bench.oracle_sample_rate = lambda w, n, threads=None: (0.25, 1.0, 4)
        buf = io.StringIO()
        sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world),
                    "--steps", "2", "--warmup", "1"]
        with contextlib.redirect_stdout(buf):
            bench.run_reference(bench.parse(), wl)
        dist.barrier()
        json.dump({"stream": wl.stream, "ms_max": ms_max, "value": value,
                   "n_greeks": wl.n_greeks, "stdout": buf.getvalue()},
                  open(os.path.join(out_dir, "rank%d.json" % rank), "w"))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [json.load(open(tmp_path / ("rank%d.json" % i))) for i in range(world)]
    # independent replicas: distinct random streams, rank 0 on the stored one
    assert r[0]["stream"] == 0 and r[1]["stream"] == 1
    # the slowest rank's time on every rank, units of both ranks counted
    assert r[0]["ms_max"] == r[1]["ms_max"] == 15.0
    assert r[0]["value"] == r[1]["value"] == world * r[0]["n_greeks"] / 0.015
    # the reference arm prints one line, on rank 0
    assert r[1]["stdout"] == ""
    lines = r[0]["stdout"].strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == world
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 == line["e2e"]["d2h_bytes_per_step"]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2206_03719_gb300 import workloads
    assert bench.replica_workload(workloads.PAPER_FP64, 0) is workloads.PAPER_FP64
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(1, 10, 20.0) == 500.0
