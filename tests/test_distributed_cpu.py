"""The replica path of bench.py for N > 1 (one independent problem per rank, no
data-path collective): the barrier and the max-over-ranks timing, run as two
gloo ranks on the CPU.  Also the reference arm: only rank 0 runs it, and its
JSON line on a small cube carries the arm's keys."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    import bench
    dist.init_process_group(backend="gloo", rank=rank, world_size=world)
    bench.barrier(world)
    # each rank "timed" a different duration; the job time is the slowest rank's
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    out[rank] = t
    dist.destroy_process_group()


def test_replica_timing_takes_max_over_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_reference_arm_rank_gating(capsys):
    # --impl reference under N > 1: only rank 0 runs and prints
    import bench

    class A:
        pass
    a = A()
    assert bench.run_reference(a, 2, 1) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_a_small_workload(capsys):
    # rank 0 at N = 1: the oracle timed on a small cube prints one JSON line
    # with the arm's keys (e2e without host copies, the cpu_baseline of this run)
    import json

    import bench

    class A:
        size, rank, solve, steps, warmup, gpus = 24, 3, "qr", 2, 1, 1
    bench.run_reference(A(), 1, 0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["dims"] == [24, 24, 24] and d["config"]["rank"] == 3
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and "2 full sweeps" in cb["sample"]
