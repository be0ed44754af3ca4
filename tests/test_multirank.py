"""The N > 1 path of the benchmark (replicas: one independent solve per GPU, no data-path
collective) on CPU with two gloo ranks: the whole-job number takes the slowest rank's
timed region and every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r: 10 (r + 1) ms for (r + 1) million cell updates
    ms, updates, value = bench.whole_job(10.0 * (rank + 1), 1e6 * (rank + 1), world, "cpu")
    q.put((rank, ms, updates, value))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, updates, value in got:
        assert ms == 20.0 and updates == 3e6
        assert abs(value - 3e6 / 20e-3 / 1e6) < 1e-9


def test_whole_job_single_rank():
    import bench

    assert bench.whole_job(4.0, 8e6, 1, "cpu") == (4.0, 8e6, 8e6 / 4e-3 / 1e6)
