"""The multi-GPU form is replicas (one independent realisation per rank, no
data exchanged); its host logic -- the cross-rank reductions bench.py uses
for the timed region and the end-to-end rate, and the whole-job value --
runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as tdist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r measured (r + 1) * 100 ms for its replica and a rate of 10 / (r + 1)
        t = bench.rank_reduce([(rank + 1) * 100.0], "max")[0]
        e = bench.rank_reduce([10.0 / (rank + 1)], "min")[0]
        s = bench.rank_reduce([1.0, rank], "sum")
        tdist.barrier()
        out.put((rank, t, e, s, bench.replicas_value(1000, 50, t, world)))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    import torch.multiprocessing as tmp

    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, e, s, v in res:
        assert t == 200.0          # the slowest replica bounds the timed region
        assert e == 5.0            # the slowest replica's rate
        assert s == [2.0, 1.0]
        assert v == pytest.approx(2 * 1000 * 50 / 0.2)  # all ranks' work / slowest time
