"""The multi-rank bookkeeping of bench.py with two gloo ranks on the CPU: disjoint
per-rank batches, the max-over-ranks timing and the whole-job throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1310_1871_gb300 import inputs as I
    seeds = [x.seed for x in I.batch_sweep(4, seed0=bench.rank_seed0(rank))]
    my_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    worst = bench.max_over_ranks(my_ms, world)
    mlups = bench.job_mlups(1000, 50, worst, world)
    out.put((rank, seeds, worst, mlups))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
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
    (r0, s0, w0, m0), (r1, s1, w1, m1) = res
    assert set(s0).isdisjoint(s1)  # independent problems per rank
    assert w0 == w1 == 20.0        # both ranks see the slowest time
    assert m0 == m1 == pytest.approx(2 * 1000 * 50 / 20e-3 / 1e6)
