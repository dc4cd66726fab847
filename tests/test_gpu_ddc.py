"""Domain decomposition on the GPU through the C ABI (Sec. 2.2, Sec. 6):
the slabs of one system, each advanced by its own library handle with the
walk drawn by particle index (mt_walk_normals), against one handle over the
whole system with the built-in generator.  The ranks are emulated one after
another in this process (the exchange is a hand-over of device tensors; no
kernel waits on another).  Positions bit for bit, masses to the parity
tolerance, every particle owned once."""
import numpy as np
import pytest

from paper_1811_05474_gb300 import ddc, mt, synth

from .test_gpu_parity import TOL, assert_masses

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("parts,precision", [(2, mt.MT_FP64), (3, mt.MT_FP64), (3, mt.MT_MIXED)])
def test_slabs_equal_one_handle(parts, precision):
    import torch

    n, L, steps = 30000, 30000.0, 12
    p = mt.mt_params_init(n=n, L=(L,), v=(0.5,), precision=precision, seed=77, realisation=3)
    x = synth.uniform_positions(n, L, seed=61)
    A, B = synth.uniform_masses(n, seed=61)
    whole = mt.Simulation(p)
    whole.upload(x, A, B)
    whole.run(steps)
    wx = whole.positions()[0]
    wa, wb = whole.masses()
    whole.close()

    g = mt.mt_resolve(p)
    dev = torch.device("cuda")
    init = ddc.Particles(torch.arange(n, dtype=torch.int64, device=dev),
                         torch.tensor(x[0], device=dev), torch.tensor(A, device=dev),
                         torch.tensor(B, device=dev))
    pad = ddc.ghost_pad(g.cutoff, 0.5, g.D_rw, g.dt, frac_bits=int(g.frac_bits))
    step = ddc.gpu_local_step(p)
    slabs = [ddc.Slab(ddc.slab_bounds(L, parts), r, pad, step, init) for r in range(parts)]
    for s in range(steps):
        ddc.step_in_process(slabs, s)
    gx, ga, gb = ddc.gather([s.own for s in slabs], n)
    assert np.array_equal(gx, wx), "positions differ from the undivided handle"
    assert_masses(ga, wa, TOL[precision], "A")
    assert_masses(gb, wb, TOL[precision], "B")


def test_walk_normals_are_the_built_in_generator():
    """mt_walk_normals gives the normals a handle's built-in generator uses:
    one step of a handle with them injected equals one step without."""
    import torch

    n, L = 5000, 5000.0
    p = mt.mt_params_init(n=n, L=(L,), seed=5, realisation=9)
    x = synth.uniform_positions(n, L, seed=3)
    A, B = synth.uniform_masses(n, seed=3)
    runs = []
    for inject in (False, True):
        sim = mt.Simulation(p)
        sim.upload(x, A, B)
        sim.run(2)
        if inject:
            gid = torch.arange(n, dtype=torch.int64, device="cuda")
            xi = torch.empty(n, dtype=torch.float32, device="cuda")
            mt.mt_walk_normals(p, gid.data_ptr(), n, 2, xi.data_ptr(), None)
            torch.cuda.synchronize()
            sim.set_noise(xi.cpu().numpy()[None, :])
        sim.step()
        runs.append(sim.ticks())
        sim.close()
    assert np.array_equal(runs[0], runs[1])
