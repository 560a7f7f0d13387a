"""The multi-rank logic of the benchmark on CPU (gloo, world size 2): every rank reports its own
step time and the job's time is the maximum over ranks; the per-GPU work is fixed (each rank
images its own copy of the workload), so the job's throughput is world x units / max time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [3.0, 5.0][rank]                       # this rank's measured step time
    job_ms = bench.max_over_ranks([ms], world, torch.device("cpu"))[0]
    w, r, _ = bench.dist_setup()
    out[rank] = (job_ms, w, r, bench.job_throughput(1000, w, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        job_ms, w, r, value = out[rank]
        assert job_ms == 5.0 and w == world and r == rank
        assert abs(value - world * 1000 / 5e-3) < 1e-6
