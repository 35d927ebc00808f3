"""The replica path of bench.py for N > 1 (one independent problem per rank, no
data-path collective): the barrier and the max-over-ranks timing, run as two
gloo ranks on the CPU."""
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
