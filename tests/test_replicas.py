"""Multi-GPU runs are replicas only (independent copies of the workload, no
collective on the data path); the host-side logic that combines them is the
max-over-ranks time and the summed throughput.  Checked here with two gloo
ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 5.0 * rank          # the slower replica sets the job time
    t = bench.reduce_max(local_ms, world)
    v = bench.job_value(cells=1000, steps=4, world=world, total_ms_max=t)
    # the reference arm does no work on ranks other than 0
    rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "n": 8, "nu": 1, "gpus": world})(), rank,
                             world) if rank != 0 else None
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v, rc))


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    port = 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, rc in out:
        assert t == 15.0                          # max over ranks
        assert v == pytest.approx(1000 * 4 * 2 / 15e-3)
    assert out[1][3] == 0                         # rank 1 skips the reference arm
