"""Failure detection on the GPU without a GPU fault: a bounded device wait
that runs out returns MT_ERR_TIMEOUT, and a device-side index check that
fails returns MT_ERR_DEVICE; in both cases the process and the CUDA context
stay usable and the next run is correct."""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import mt, synth

from .test_gpu_parity import assert_masses, oracle_params

pytestmark = pytest.mark.gpu


def _one_checked_step(sim, x, A, B, seed):
    """Upload, one step with injected noise, compare with the oracle."""
    po = oracle_params(sim)
    sim.upload(x, A, B)
    xi = synth.normals(1, sim.dim, sim.n, seed=seed)[0]
    sim.set_noise(xi)
    sim.step()
    X, a, b = O.step(po, O.quantize(np.asarray(x).reshape(sim.dim, -1), int(sim.params.frac_bits)),
                     xi, A.copy(), B.copy())
    assert np.array_equal(sim.ticks(), X)
    ga, gb = sim.masses()
    assert_masses(ga, a, 1e-12, "A")
    assert_masses(gb, b, 1e-12, "B")


def test_scan_wait_runs_out_and_reports_timeout():
    """The multi-kernel pipeline's look-back scan waits for earlier tiles'
    status words with a bounded poll loop.  The test hook withholds the
    first tile's word (a flag that nothing sets), so the others give up
    after 2^14 polls: the step must come back as MT_ERR_TIMEOUT, not hang.
    2-d, 64 particles, cells of two units on a 1000 x 1000 domain: 250 000
    cells, 62 scan tiles, every later kernel bounded by the 64 particles."""
    n, L = 64, (1000.0, 1000.0)
    p = mt.mt_params_init(dim=2, n=n, L=L, precision=mt.MT_FP64, seed=3)
    k = int(mt.mt_resolve(p).frac_bits)
    p.cell_shift = k + 1  # 2-unit cells, wider than the 1.9-unit cutoff
    sim = mt.Simulation(p)
    x = synth.uniform_positions(n, L, dim=2, seed=3)
    A, B = synth.uniform_masses(n, seed=3)
    sim.upload(x, A, B)
    mt.mt_test_hold_scan(sim.h, 1, 1 << 14)
    with pytest.raises(mt.MtError) as e:
        sim.step()
        sim.sync()
    assert e.value.status == mt.MT_ERR_TIMEOUT
    assert "gave up" in mt.mt_last_error()
    with pytest.raises(mt.MtError):
        mt.mt_test_hold_scan(sim.h, 2, 0)
    # the context is intact: a fresh upload clears the hook and the error
    _one_checked_step(sim, x, A, B, seed=4)
    sim.close()


def test_bad_index_reports_device_error():
    """A particle id outside [0, n), written by the host into the handle's
    id array, is caught by the read-back kernel's index check (which skips
    the access): MT_ERR_DEVICE.  The next upload runs normally."""
    import torch

    n, L = 1000, 1000.0
    sim = mt.Simulation(mt.mt_params_init(n=n, L=(L,), precision=mt.MT_FP64))
    # sorted positions: the upload's cell sort then keeps the caller's order,
    # and the id array holds 0, 1, ..., n - 1
    x = np.sort(synth.uniform_positions(n, L, seed=8), axis=1)
    A, B = synth.uniform_masses(n, seed=8)
    sim.upload(x, A, B)
    sim.sync()
    ws = sim.workspace.cpu().numpy()
    w = ws[:ws.size // 4 * 4].view(np.int32).copy()
    ids = np.arange(n, dtype=np.int32)
    hits = [o for o in np.flatnonzero(w[:w.size - n + 1] == 0) if np.array_equal(w[o:o + n], ids)]
    assert hits, "the id array was not found in the workspace"
    for o in hits:  # both ping-pong id buffers hold the identity after the upload's sort
        w[o + 500] = n + 7
    bad = ws.copy()
    bad[:w.size * 4] = w.view(np.uint8)
    sim.workspace.copy_(torch.from_numpy(bad).to(sim.workspace.device))
    torch.cuda.synchronize()
    with pytest.raises(mt.MtError) as e:
        sim.masses()
    assert e.value.status == mt.MT_ERR_DEVICE
    assert "index check" in mt.mt_last_error()
    _one_checked_step(sim, x, A, B, seed=9)
    sim.close()
