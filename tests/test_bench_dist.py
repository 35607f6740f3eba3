"""The multi-rank (torchrun) path of bench.py on CPU: two gloo ranks on
127.0.0.1 check the max-over-ranks timing and the whole-job aggregation.
Each rank runs an independent replica, so there is no data-path collective to
test; only the timing reduction crosses ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.reduce_max(10.0 + 5.0 * rank, dist, device="cpu")
    v = bench.job_mlups(world, 1000, 50, ms / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, v))


def test_two_rank_timing_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]          # max over ranks on every rank
    assert all(abs(r[2] - 2 * 1000 * 50 / 0.015 / 1e6) < 1e-9 for r in res)


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_max(3.5, None) == 3.5
    assert abs(bench.job_mlups(1, 256 ** 3, 100, 0.1) - 256 ** 3 * 1000 / 1e6) < 1e-6
