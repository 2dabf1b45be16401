"""The multi-rank logic of bench.py on CPU: two gloo ranks with different
step times agree on the slowest rank's time and on the whole-job
throughput; only rank 0 runs the reference arm."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [0.010, 0.030][rank]                 # seconds per step on this rank
    value, s = bench.job_throughput(1000, local, world, dist)
    out[rank] = (value, s)
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        value, s = res[rank]
        assert s == 0.030
        assert abs(value - 2 * 1000 / 0.030) < 1e-6


def test_single_rank_throughput_and_reference_rank_gate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(500, 0.5, 1) == (1000.0, 0.5)
    # a rank other than 0 leaves the reference arm at once, without work or output
    assert bench.run_reference(None, bench.WORKLOADS["sbm"], 1, 2) == 0
