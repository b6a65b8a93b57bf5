"""Host logic of the multi-replica benchmark on CPU (gloo, world size 2).

With N > 1 every rank steps its own replica of the domain (weak scaling, no
collective on the data path); the job's time is the slowest rank's and its
throughput the units of all ranks over that time.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [0.5, 2.0, 1.0, 1.5][rank]
    s_max, thr = bench.job_throughput(dist, local, 1000)
    # the reference arm runs on rank 0 only: the others return at once
    ref_rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 1})(), rank, world) if rank else None
    out.put((rank, s_max, thr, ref_rc))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_job_throughput_is_max_over_ranks(world):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([0.5, 2.0, 1.0, 1.5][:world])
    for rank, s_max, thr, ref_rc in res:
        assert s_max == slowest
        assert thr == pytest.approx(world * 1000 / slowest)
        if rank:
            assert ref_rc == 0
    del torch


def test_job_throughput_single_process():
    import bench
    assert bench.job_throughput(None, 0.25, 500) == (0.25, 2000.0)
