"""The multi-GPU path is replicas (independent operators per rank, no exchange
on the data path): the benchmark's step time is the slowest rank's and its
throughput counts every rank's units.  These host-side pieces run here as two
`gloo` ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (t, bench.replica_rate(1000.0, world, t))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time_and_every_rank_counts():
    world = 2
    times = [0.25, 0.4]
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, v = res[rank]
        assert t == max(times)
        assert v == pytest.approx(1000.0 * world / max(times))


def test_single_process_is_unchanged():
    assert bench.max_over_ranks(0.5, None, "cpu") == 0.5
    assert bench.replica_rate(10.0, 1, 0.5) == 20.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse
    import json
    args = argparse.Namespace(workload="ico3", r=0, steps=1, warmup=0)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
    bench.run_reference(args, rank=0, world=2)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
