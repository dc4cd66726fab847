"""Checkpoint and resume: a handle loaded from a checkpoint continues bit for
bit like the handle that saved it (positions, masses and observables; the
counter-based walk is keyed by the saved step counter), on the one-kernel step with its second tiers busy, on
the multi-kernel pipeline with extra species, and for a batch; foreign or
damaged checkpoints are refused and leave the state unchanged."""
import numpy as np
import pytest

from paper_1811_05474_gb300 import mt, synth

pytestmark = pytest.mark.gpu


def state(sim, S=2):
    return (sim.ticks(), *[sim.species(s) for s in range(S)], sim.observables())


def assert_same(a, b):
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def clustered(n, L, seed):
    """Uniform positions with a dense cluster near the left wall, so that the
    one-kernel step sends segments to its second tiers."""
    x = synth.uniform_positions(n, L, seed=seed)
    k = n // 100
    x[0, :k] = np.random.default_rng(seed).uniform(0.0, 4.0, k)
    return x


@pytest.mark.parametrize("precision", [mt.MT_MIXED, mt.MT_FP64])
def test_resume_is_bit_identical_one_kernel_step(tmp_path, precision):
    n, L = 400000, 4.0e5
    p = mt.mt_params_init(n=n, L=(L,), v=(0.5,), precision=precision, seed=11, observe_cap=64)
    x = clustered(n, L, 3)
    A, B = synth.uniform_masses(n, seed=3)
    a = mt.Simulation(p)
    assert a.params.seg_target > 0
    a.upload(x, A, B)
    a.run(15)
    a.step(2)  # direct launches too
    ck = tmp_path / "a.ckpt"
    a.save(ck)
    a.run(20)
    ref = state(a)
    assert mt.mt_checkpoint_params(ck).seg_target == a.params.seg_target
    b = mt.Simulation(mt.mt_checkpoint_params(ck))
    b.load(ck)
    assert mt.mt_steps_done(b.h) == 17
    b.run(20)
    assert_same(state(b), ref)
    a.close()
    b.close()


def test_resume_multi_kernel_pipeline_with_species(tmp_path):
    n = 3000
    L = (150.0, 120.0)
    p = mt.mt_params_init(dim=2, n=n, L=L, v=(0.3, -0.2), precision=mt.MT_FP64, species=3,
                          seed=5, observe_cap=16)
    x = synth.uniform_positions(n, L, dim=2, seed=8)
    A, B = synth.uniform_masses(n, seed=8)
    a = mt.Simulation(p)
    a.upload(x, A, B)
    a.set_species(2, np.linspace(0.0, 1.0, n))
    a.run(7)
    ck = tmp_path / "b.ckpt"
    a.save(ck)
    a.run(9)
    ref = state(a, 3)
    b = mt.Simulation(p)
    b.load(ck)
    b.run(9)
    assert_same(state(b, 3), ref)


def test_resume_batch_and_refusals(tmp_path):
    ns, Ls = [3000, 1500, 5000], [3000.0, 1500.0, 5000.0]
    p = mt.mt_params_init(dim=1, L=(1.0,), precision=mt.MT_MIXED, seed=2, observe_cap=8)
    bt = mt.make_batch(ns, Ls)
    xs = np.concatenate([synth.uniform_positions(n, L, seed=i)[0] for i, (n, L) in
                         enumerate(zip(ns, Ls))])[None, :]
    A, B = synth.uniform_masses(sum(ns), seed=4)
    a = mt.Simulation(p, batch=bt)
    a.upload(xs, A, B)
    a.run(6)
    ck = tmp_path / "c.ckpt"
    a.save(ck)
    a.run(6)
    ref = state(a)
    b = mt.Simulation(p, batch=bt)
    b.load(ck)
    b.run(6)
    assert_same(state(b), ref)
    # other realisations, other parameters, damaged file: refused, state kept
    other = mt.Simulation(p, batch=mt.make_batch([3000, 1500, 5000], [3000.0, 1600.0, 5000.0]))
    with pytest.raises(mt.MtError) as e:
        other.load(ck)
    assert e.value.status == mt.MT_ERR_INVALID
    c = mt.Simulation(mt.mt_params_init(n=100, L=(100.0,)))
    with pytest.raises(mt.MtError) as e:
        c.save(tmp_path / "never.ckpt")
    assert e.value.status == mt.MT_ERR_STATE
    c.upload(np.linspace(1, 99, 100), np.ones(100), np.zeros(100))
    before = state(c)
    for bad in (ck, tmp_path / "missing.ckpt"):
        with pytest.raises(mt.MtError):
            c.load(bad)
    cut = tmp_path / "cut.ckpt"
    cut.write_bytes(ck.read_bytes()[:-100])
    with pytest.raises(mt.MtError):
        b.load(cut)
    assert_same(state(c), before)
    assert_same(state(b), ref)
