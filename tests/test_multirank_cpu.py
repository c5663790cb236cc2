"""The multi-rank bookkeeping of bench.py with two gloo ranks on the CPU.  Each rank
builds its instance list exactly as bench.py's run_gpu does (the 64-drop sweep
recipe with the rank's first seed); the lists are disjoint, together they hold
64 x world instances whose site counts add up to the job's, and the timing is
the max over ranks.  (The sharding has no collective on the data path; it is
measured on one GPU only, since the pool offers one GPU per run.)"""
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
    inst = I.batch_sweep(64, seed0=bench.rank_seed0(rank))  # as run_gpu builds it
    seeds = [x.seed for x in inst]
    shapes = [(x.Nz, x.Nr, x.tau, x.G) for x in inst]
    sites = sum(x.Nz * x.Nr for x in inst)
    total = bench.sum_over_ranks(sites, world)  # the job's site count
    my_ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    worst = bench.max_over_ranks(my_ms, world)
    mlups = bench.job_mlups(total, 50, worst)
    out.put((rank, seeds, shapes, sites, total, worst, mlups))
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
    (r0, s0, sh0, n0, t0, w0, m0), (r1, s1, sh1, n1, t1, w1, m1) = res
    assert len(s0) == len(s1) == 64
    assert set(s0).isdisjoint(s1)              # independent problems per rank
    assert len(set(s0) | set(s1)) == 2 * 64    # the job holds 64 x world instances
    assert sh0 != sh1                          # different lattices, not a replica
    assert t0 == t1 == n0 + n1                 # site counts add up to the job's
    assert w0 == w1 == 20.0                    # both ranks see the slowest time
    # bench's whole-job throughput: all ranks' sites over the slowest time
    assert m0 == m1 == pytest.approx((n0 + n1) * 50 / 20e-3 / 1e6)
