"""The observables (the conservative components of Sec. 3: sum A, sum B,
sum (A - B), mean A) against the exact sums of the masses read back
(math.fsum), with masses over 25 decades and of both signs, on the
one-kernel step and on the general pipeline, in every precision: within
the error bound of a summation of depth 40 (16 terms per thread in order,
the shuffle and block trees, the chunk sums) in the precision's own
arithmetic, 40 u sum |m| with u = 2^-53 (binary64) or 2^-48
(double-binary32); an infinite mass gives non-finite sums."""
import math

import numpy as np
import pytest

from paper_1811_05474_gb300 import mt, synth

from .test_gpu_parity import PRECISIONS, make

pytestmark = pytest.mark.gpu


def _exact(a, b):
    return math.fsum(a), math.fsum(b), math.fsum(np.concatenate([a, -b]))


UNIT = {mt.MT_FP64: 2.0 ** -53, mt.MT_MIXED: 2.0 ** -53, mt.MT_MIXED_DF32: 2.0 ** -48}


def _masses(n, seed):
    """Masses spread over 25 decades, both signs, some exact zeros."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(2):
        m = 10.0 ** rng.uniform(-20.0, 5.0, n) * rng.choice([-1.0, 1.0], n)
        m[rng.integers(0, n, n // 50)] = 0.0
        out.append(m)
    return out


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("dim", [1, 2])
def test_observables_are_the_rounded_exact_sums(precision, dim):
    n = 50000  # 13 chunks, the last one ragged
    L = 50000.0 if dim == 1 else (250.0, 200.0)
    x = synth.uniform_positions(n, L, dim=dim, seed=31)
    A, B = _masses(n, 32)
    sim = make(n, L, dim=dim, precision=precision, react=0, observe_cap=4, seed=3,
               v=(0.5, 0.0))
    sim.upload(x, A, B)
    sim.run(2)
    obs = sim.observables()
    a, b = sim.masses()
    sim.close()
    sa, sb, sd = _exact(a, b)
    row = obs[-1]
    ma, mb = math.fsum(np.abs(a)), math.fsum(np.abs(b))
    bound = {0: ma, 1: mb, 2: ma + mb, 3: ma / n}
    for k, e in enumerate((sa, sb, sd, sa / n)):
        tol = 40 * UNIT[precision] * bound[k] + 2 * math.ulp(e)
        assert abs(row[k] - e) <= tol, (k, row[k], e, tol)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_non_finite_mass_gives_non_finite_sums(precision):
    n, L = 20000, 20000.0
    x = synth.uniform_positions(n, L, seed=33)
    A, B = synth.uniform_masses(n, seed=33)
    A[12345] = np.inf
    sim = make(n, L, precision=precision, react=0, observe_cap=4, seed=4)
    sim.upload(x, A, B)
    sim.run(1)
    row = sim.observables()[-1]
    sim.close()
    assert not np.isfinite(row[0]) and not np.isfinite(row[2])
    assert np.isfinite(row[1])  # B holds no infinity after one step


@pytest.mark.parametrize("precision", PRECISIONS)
def test_pipelined_row_copies_equal_the_ring(precision):
    """Each step's row copied one step late (the step that computes it
    beside itself was just enqueued), the last one after the loop: the rows
    equal those read from the ring, on a system large enough for the
    predicted-segment kernel (where the observables run beside the next
    step) and on a small one."""
    import torch

    for n in (300000, 20000):
        L = float(n)
        x = synth.uniform_positions(n, L, seed=41)
        A, B = synth.uniform_masses(n, seed=41)
        steps = 12
        sim = make(n, L, precision=precision, observe_cap=steps, seed=6, v=(0.5, 0.0))
        sim.upload(x, A, B)
        rows = torch.zeros((steps, 4), dtype=torch.float64).pin_memory()
        for s in range(steps):
            mt.mt_run(sim.h, 1)
            if s >= 1:
                mt.mt_copy_observables_row_async(sim.h, rows[s - 1].data_ptr(), s)
        mt.mt_copy_observables_row_async(sim.h, rows[steps - 1].data_ptr(), steps)
        sim.sync()
        ring = sim.observables()
        sim.close()
        assert np.array_equal(rows.numpy(), ring)
    # a step that was not enqueued has no row
    sim = make(1000, 1000.0, precision=precision, observe_cap=2)
    sim.upload(synth.uniform_positions(1000, 1000.0, seed=1), *synth.uniform_masses(1000, seed=1))
    sim.run(3)
    buf = torch.zeros(4, dtype=torch.float64).pin_memory()
    for bad in (0, 1, 4):  # 1 left the ring of two rows
        with pytest.raises(mt.MtError):
            mt.mt_copy_observables_row_async(sim.h, buf.data_ptr(), bad)
    sim.close()
