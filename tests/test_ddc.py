"""Domain decomposition (Sec. 2.2, Sec. 6): one 1-d system split into slabs,
one rank each, ghosts exchanged with the neighbours every step.  The slab
logic (ghost selection, hand-over, ownership after the move) runs here on
the CPU, with the oracle as each rank's local step, and must reproduce the
undivided oracle run: positions bit for bit, masses to 1e-12 (with the same
summation order they agree exactly), every particle owned by exactly one
rank.  Two gloo ranks exchange through torch.distributed; three slabs are
also run in one process (the middle slab has two neighbours)."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import ddc, synth

N, L, STEPS, K = 2400, 2400.0, 25, 29
V, D = 0.5, 0.1


def _setup():
    po = O.params(L=(L,), v=(V,), D_mt=D, D_rw=D, dt=1.0, frac_bits=K)
    x = O.dequantize(O.quantize(synth.uniform_positions(N, L, seed=51), K), K)[0]
    A, B = synth.uniform_masses(N, seed=51)
    xi = synth.normals(STEPS, 1, N, seed=52)[:, 0, :]
    return po, x, A, B, xi


def _oracle_local_step(po, xi):
    import torch

    def step(parts, s):
        gid = parts.gid.numpy()
        X = O.quantize(parts.x.numpy()[None, :], K)
        X2, A2, B2 = O.step(po, X, xi[s][gid][None, :], parts.A.numpy().copy(),
                            parts.B.numpy().copy())
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
        return ddc.Particles(parts.gid, t(O.dequantize(X2, K)[0]), t(A2), t(B2))
    return step


def _initial(x, A, B):
    import torch

    return ddc.Particles(torch.arange(N, dtype=torch.int64), torch.from_numpy(x.copy()),
                         torch.from_numpy(A.copy()), torch.from_numpy(B.copy()))


def _reference(po, x, A, B, xi):
    X, a, b = O.quantize(x[None, :], K), A.copy(), B.copy()
    for s in range(STEPS):
        X, a, b = O.step(po, X, xi[s][None, :], a, b)
    return O.dequantize(X, K)[0], a, b


def _check(parts, ref):
    gx, ga, gb = ddc.gather(parts, N)
    rx, ra, rb = ref
    assert np.array_equal(gx, rx), "positions differ from the undivided run"
    for g, r in ((ga, ra), (gb, rb)):
        err = np.abs(g - r) / np.maximum(np.abs(r), 0.5)
        assert err.max() <= 1e-12


def test_pad_covers_two_cutoffs_and_a_step():
    p = ddc.ghost_pad(1.8974, 0.5, 0.1, 1.0, xi_max=5.78)
    assert p == pytest.approx(2 * 1.8974 + 0.5 + np.sqrt(0.2) * 5.78, abs=1e-8)
    assert ddc.slab_bounds(10.0, 4) == [0.0, 2.5, 5.0, 7.5, 10.0]


def test_three_slabs_in_one_process_equal_the_undivided_run():
    po, x, A, B, xi = _setup()
    pad = ddc.ghost_pad(po.smax, V, D, 1.0, xi_max=float(np.abs(xi).max()))
    bounds = ddc.slab_bounds(L, 3)
    step = _oracle_local_step(po, xi)
    slabs = [ddc.Slab(bounds, r, pad, step, _initial(x, A, B)) for r in range(3)]
    assert sum(len(s.own) for s in slabs) == N
    moved = 0
    for s in range(STEPS):
        before = [set(sl.own.gid.tolist()) for sl in slabs]
        ddc.step_in_process(slabs, s)
        moved += sum(len(b - set(sl.own.gid.tolist())) for b, sl in zip(before, slabs))
    assert moved > 0, "no particle crossed a slab edge: migration untested"
    _check([s.own for s in slabs], _reference(po, x, A, B, xi))


def test_slab_narrower_than_the_pad_is_refused():
    po, x, A, B, xi = _setup()
    with pytest.raises(ValueError):
        ddc.Slab([0.0, 5.0, L], 0, 8.0, _oracle_local_step(po, xi), _initial(x, A, B))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        po, x, A, B, xi = _setup()
        pad = ddc.ghost_pad(po.smax, V, D, 1.0, xi_max=float(np.abs(xi).max()))
        slab = ddc.Slab(ddc.slab_bounds(L, world), rank, pad, _oracle_local_step(po, xi),
                        _initial(x, A, B))
        for s in range(STEPS):
            ddc.step_distributed(slab, s)
        dist.barrier()
        o = slab.own
        q.put((rank, o.gid.numpy(), o.x.numpy(), o.A.numpy(), o.B.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_undivided_run():
    import torch
    import torch.multiprocessing as tmp

    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = [ddc.Particles(*(torch.from_numpy(a) for a in r[1:])) for r in res]
    assert all(len(p) > 0 for p in parts)
    po, x, A, B, xi = _setup()
    _check(parts, _reference(po, x, A, B, xi))
