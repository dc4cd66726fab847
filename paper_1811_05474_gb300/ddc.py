"""Domain decomposition of one 1-d system into slabs (the paper's DDC with
ghost particles, Sec. 2.2 and Sec. 6): one rank per slab, one GPU each.

The domain [0, L] is cut into P contiguous slabs [a_r, a_{r+1}) (the last
closed at L).  Rank r owns the particles whose position lies in its slab.
One time step on rank r:

1. ghosts: each rank sends its neighbours copies (index, position, masses)
   of its particles within ``pad`` of the shared edge, pad = 2 s_max + the
   largest displacement of one step (the drift plus the walk's bound);
2. local step: the rank advances its owned particles and the received
   ghosts together through one step of the library (move, cell-list search,
   transfer, reaction).  Every particle takes the walk it takes in the
   undivided system, because the normals are drawn by its index in the
   whole system (``mt_walk_normals``), so a ghost moves on both ranks exactly
   as on its owner;
3. ownership: the rank keeps the particles that ended inside its slab.  A
   particle that crossed an edge is picked up by the neighbour, which moved
   it as a ghost: migration needs no message of its own.

After the move, every particle within 2 s_max of the slab was within pad of
it before, so each owned particle sees all its neighbours and each of those
sees all of theirs: its row sums (Eq. 3), its exchange (Eq. 4, 7) and its
reaction are those of the undivided system.  The results of ghosts far from
the slab are incomplete and are dropped.

The exchange is point to point with the two neighbours (torch.distributed:
NCCL between GPUs, gloo on CPUs), into local receive buffers, one message
per neighbour per step.  The local step is a callable, so the same slab
logic runs with the CUDA library (``gpu_local_step``) or, in tests, with
any other implementation of the step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable

import numpy as np

# largest |normal| the built-in generator draws: sqrt(-2 ln 2^-24) < 5.78
WALK_BOUND = 5.78


def slab_bounds(L: float, parts: int) -> list[float]:
    """Edges of `parts` equal slabs of [0, L]."""
    return [L * r / parts for r in range(parts)] + [float(L)]


def ghost_pad(cutoff: float, v: float, D_rw: float, dt: float, xi_max: float = WALK_BOUND,
              frac_bits: int = 29) -> float:
    """Width of the ghost layer: 2 s_max plus the largest displacement of one
    step (|v| dt + sqrt(2 D_rw dt) xi_max), plus two grid ticks of rounding."""
    return 2.0 * cutoff + abs(v) * dt + math.sqrt(2.0 * D_rw * dt) * xi_max + 2.0 ** (1 - frac_bits)


@dataclass
class Particles:
    """Particles of a rank: their indices in the whole system and their
    state (torch tensors, all on one device)."""
    gid: object  # int64
    x: object    # float64
    A: object    # float64
    B: object    # float64

    def __len__(self):
        return int(self.gid.numel())

    def take(self, mask):
        return Particles(self.gid[mask], self.x[mask], self.A[mask], self.B[mask])

    def pack(self):
        """One float64 tensor [4, n] (indices < 2^53 are exact)."""
        import torch

        return torch.stack([self.gid.to(torch.float64), self.x, self.A, self.B])

    @staticmethod
    def unpack(t):
        import torch

        return Particles(t[0].to(torch.int64), t[1].contiguous(), t[2].contiguous(),
                         t[3].contiguous())

    @staticmethod
    def cat(parts):
        import torch

        return Particles(*(torch.cat([getattr(p, f) for p in parts])
                           for f in ("gid", "x", "A", "B")))


LocalStep = Callable[[Particles, int], Particles]


class Slab:
    """Rank `rank` of a system split at `bounds` (P + 1 edges)."""

    def __init__(self, bounds, rank: int, pad: float, local_step: LocalStep, own: Particles):
        self.bounds = [float(b) for b in bounds]
        self.P = len(self.bounds) - 1
        self.rank = rank
        self.pad = float(pad)
        self.local_step = local_step
        self.a, self.b = self.bounds[rank], self.bounds[rank + 1]
        if self.P > 1 and min(self.bounds[i + 1] - self.bounds[i] for i in range(self.P)) < pad:
            raise ValueError("every slab must be at least as wide as the ghost pad")
        self.own = own.take(self.inside(own.x))

    def inside(self, x):
        last = self.rank == self.P - 1
        return (x >= self.a) & ((x <= self.b) if last else (x < self.b))

    def outgoing(self):
        """Copies of the particles within pad of each shared edge: (to the
        left neighbour, to the right neighbour); None where there is none."""
        x = self.own.x
        left = self.own.take(x < self.a + self.pad) if self.rank > 0 else None
        right = self.own.take(x >= self.b - self.pad) if self.rank < self.P - 1 else None
        return left, right

    def advance(self, from_left: Particles | None, from_right: Particles | None, step: int):
        """One step over owned particles and ghosts; keep what ends inside."""
        parts = [self.own] + [g for g in (from_left, from_right) if g is not None and len(g)]
        local = Particles.cat(parts) if len(parts) > 1 else self.own
        out = self.local_step(local, step)
        self.own = out.take(self.inside(out.x))
        return self


def step_in_process(slabs: list[Slab], step: int) -> None:
    """One step of all slabs of a system held in one process (the exchange
    is a hand-over of tensors; used where the ranks are emulated)."""
    out = [s.outgoing() for s in slabs]
    for r, s in enumerate(slabs):
        from_left = out[r - 1][1] if r > 0 else None
        from_right = out[r + 1][0] if r < len(slabs) - 1 else None
        s.advance(from_left, from_right, step)


def step_distributed(slab: Slab, step: int, group=None) -> None:
    """One step of this rank's slab: ghosts exchanged with the neighbour
    ranks by point-to-point messages (counts first, then one packed tensor
    per neighbour), then the local step."""
    import torch
    import torch.distributed as dist

    to_left, to_right = slab.outgoing()
    dev = slab.own.x.device
    nb = [(slab.rank - 1, to_left), (slab.rank + 1, to_right)]
    nb = [(r, p) for r, p in nb if 0 <= r < slab.P]
    counts_out = {r: torch.tensor([len(p)], dtype=torch.int64, device=dev) for r, p in nb}
    counts_in = {r: torch.zeros(1, dtype=torch.int64, device=dev) for r, _ in nb}
    ops = []
    for r, _ in nb:
        ops.append(dist.P2POp(dist.isend, counts_out[r], r, group))
        ops.append(dist.P2POp(dist.irecv, counts_in[r], r, group))
    for w in dist.batch_isend_irecv(ops) if ops else []:
        w.wait()
    bufs_in = {r: torch.empty((4, int(counts_in[r].item())), dtype=torch.float64, device=dev)
               for r, _ in nb}
    ops = []
    for r, p in nb:
        if len(p):
            ops.append(dist.P2POp(dist.isend, p.pack().contiguous(), r, group))
        if bufs_in[r].shape[1]:
            ops.append(dist.P2POp(dist.irecv, bufs_in[r], r, group))
    for w in dist.batch_isend_irecv(ops) if ops else []:
        w.wait()
    got = {r: Particles.unpack(bufs_in[r]) for r, _ in nb}
    slab.advance(got.get(slab.rank - 1), got.get(slab.rank + 1), step)


def gpu_local_step(params, device="cuda", stream=None) -> LocalStep:
    """The local step on the GPU through the C ABI: a handle for the rank's
    current particles (the system's resolved grid, cutoff and coefficients;
    its own particle count), the walk's normals drawn by index in the whole
    system, one step, positions and masses read back on the device.  The
    handle lives for one step (its particle count changes from step to step)
    and launches its kernels directly."""
    import torch

    from . import mt

    g = mt.mt_resolve(params)
    dev = torch.device(device)
    st = stream if stream is not None else torch.cuda.Stream(device=dev)

    def local(parts: Particles, step: int) -> Particles:
        n = len(parts)
        p = mt.mt_params_init()
        for f, _ in mt.mt_params._fields_:
            setattr(p, f, getattr(g, f))
        p.n, p.observe_cap, p.cell_shift, p.seg_target = n, 0, 0, 0
        ws = torch.empty(max(mt.mt_workspace_bytes(p), 256), dtype=torch.uint8, device=dev)
        gid = parts.gid.to(dev).contiguous()
        x = parts.x.to(dev).contiguous()
        A = parts.A.to(dev).contiguous()
        B = parts.B.to(dev).contiguous()
        xi = torch.empty(max(n, 1) * int(p.dim), dtype=torch.float32, device=dev)
        out = [torch.empty(max(n, 1), dtype=torch.float64, device=dev) for _ in range(3)]
        st.wait_stream(torch.cuda.current_stream(dev))
        h = mt.mt_create(p, ws.data_ptr(), ws.numel(), st.cuda_stream)
        try:
            mt.mt_walk_normals(p, gid.data_ptr(), n, step, xi.data_ptr(), st.cuda_stream)
            mt.mt_set_noise(h, xi.data_ptr())
            mt.mt_set_profiling(h, True)
            mt.mt_upload(h, x.data_ptr(), A.data_ptr(), B.data_ptr(), mt.MT_MEM_DEVICE)
            mt.mt_step(h)
            mt.mt_read_positions(h, out[0].data_ptr(), mt.MT_MEM_DEVICE)
            mt.mt_read_masses(h, out[1].data_ptr(), out[2].data_ptr(), mt.MT_MEM_DEVICE)
            mt.mt_sync(h)
        finally:
            mt.mt_destroy(h)
        torch.cuda.current_stream(dev).wait_stream(st)
        return Particles(gid, out[0][:n], out[1][:n], out[2][:n])

    return local


def gather(parts: list[Particles], n: int):
    """The whole system from the ranks' owned particles, by index:
    (x, A, B) numpy arrays; checks that every index is owned exactly once."""
    gid = np.concatenate([p.gid.cpu().numpy() for p in parts])
    if len(gid) != n or not np.array_equal(np.sort(gid), np.arange(n)):
        raise AssertionError("the slabs do not own every particle exactly once")
    out = []
    for f in ("x", "A", "B"):
        v = np.empty(n)
        v[gid] = np.concatenate([getattr(p, f).cpu().numpy() for p in parts])
        out.append(v)
    return tuple(out)
