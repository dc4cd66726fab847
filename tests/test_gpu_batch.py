"""Batches of independent 1-d realisations in one handle, against the oracle
run on each realisation alone and against single handles.

Every realisation has its own domain [0, L_r], walls and random-walk
counter word; a batch step advances all of them with one fused kernel.
"""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import mt, synth

from .test_gpu_parity import PRECISIONS, TOL, assert_masses

pytestmark = pytest.mark.gpu


def batch_params(precision=mt.MT_FP64, observe_cap=0, frac_bits=0, v=(0.0, 0.0), D_rw=0.1,
                 cell_shift=0, seg_target=0, seed=0):
    return mt.mt_params_init(dim=1, L=(1.0,), v=v, D_rw=D_rw, D_mt=0.1, dt=1.0,
                             precision=precision, observe_cap=observe_cap, frac_bits=frac_bits,
                             cell_shift=cell_shift, seg_target=seg_target, seed=seed)


def batch_inputs(ns, Ls, seed):
    xs, As, Bs = [], [], []
    for r, (n, L) in enumerate(zip(ns, Ls)):
        xs.append(synth.uniform_positions(n, L, seed=seed + r)[0])
        a, b = synth.uniform_masses(n, seed=seed + r)
        As.append(a)
        Bs.append(b)
    return xs, As, Bs


def split(v, ns):
    return np.split(np.asarray(v), np.cumsum(ns)[:-1])


def oracle_for(sim, L):
    r = sim.params
    return O.params(dim=1, frac_bits=r.frac_bits, L=(L,), v=tuple(r.v), D_mt=r.D_mt,
                    D_rw=r.D_rw, dt=r.dt, smax=r.cutoff, search=O.SEARCH_CUTOFF, norm=r.norm,
                    react=r.react)


def run_batch_vs_oracle(sim, ns, Ls, xs, As, Bs, steps, seed, check_every=1):
    k = int(sim.params.frac_bits)
    sim.upload(np.concatenate(xs)[None, :], np.concatenate(As), np.concatenate(Bs))
    Xs = [O.quantize(x[None, :], k) for x in xs]
    a = [A.copy() for A in As]
    b = [B.copy() for B in Bs]
    po = [oracle_for(sim, L) for L in Ls]
    tol = TOL[int(sim.params.precision)]
    xi = synth.normals(steps, 1, int(sum(ns)), seed=seed)
    for s in range(steps):
        sim.set_noise(xi[s])
        sim.step()
        parts = split(xi[s][0], ns)
        for r in range(len(ns)):
            Xs[r], a[r], b[r] = O.step(po[r], Xs[r], parts[r][None, :], a[r], b[r])
        if (s + 1) % check_every == 0 or s == steps - 1:
            T = split(sim.ticks()[0], ns)
            ga, gb = sim.masses()
            ga, gb = split(ga, ns), split(gb, ns)
            for r in range(len(ns)):
                assert np.array_equal(T[r], Xs[r][0]), f"realisation {r} positions, step {s}"
                assert_masses(ga[r], a[r], tol, f"realisation {r} A step {s}")
                assert_masses(gb[r], b[r], tol, f"realisation {r} B step {s}")
    return Xs, a, b, po


@pytest.mark.parametrize("precision", PRECISIONS)
def test_batch_matches_oracle_per_realisation(precision):
    """Uneven realisations (1 to 3000 particles, density 1 and denser ones)
    with observables and pair sets per realisation."""
    ns = [1, 2, 33, 1000, 3000, 257, 64, 5]
    Ls = [3.0, 10.0, 33.0, 1000.0, 3000.0, 50.0, 64.0, 2.0]
    xs, As, Bs = batch_inputs(ns, Ls, seed=7)
    steps = 12
    sim = mt.Simulation(batch_params(precision, observe_cap=steps), batch=mt.make_batch(ns, Ls))
    assert sim.n == sum(ns) and sim.nreal == len(ns)
    Xs, a, b, po = run_batch_vs_oracle(sim, ns, Ls, xs, As, Bs, steps, seed=8, check_every=3)
    obs = sim.observables()
    assert obs.shape == (steps, len(ns), 4)
    for r in range(len(ns)):
        np.testing.assert_allclose(obs[-1, r], O.observables(a[r], b[r]),
                                   rtol=TOL[precision] * 10, atol=1e-12 * ns[r])
    gi, gj = sim.pairs()
    got = set(zip(gi.tolist(), gj.tolist()))
    want = set()
    off = 0
    for r in range(len(ns)):
        oi, oj = O.pairs_brute(po[r], Xs[r])
        want |= set(zip((oi + off).tolist(), (oj + off).tolist()))
        off += ns[r]
    assert len(got) == len(gi) and got == want


def test_batch_positions_in_own_domains_and_walls():
    """Strong advection piles particles against each realisation's own wall
    at x = L_r; positions read back stay in [0, L_r]."""
    ns = [500, 40, 900]
    Ls = [100.0, 5.0, 300.0]
    xs, As, Bs = batch_inputs(ns, Ls, seed=3)
    sim = mt.Simulation(batch_params(mt.MT_MIXED, v=(2.0, 0.0), D_rw=0.3),
                        batch=mt.make_batch(ns, Ls))
    run_batch_vs_oracle(sim, ns, Ls, xs, As, Bs, 30, seed=4, check_every=10)
    x = split(sim.positions()[0], ns)
    for r in range(len(ns)):
        assert x[r].min() >= 0.0 and x[r].max() <= Ls[r]


@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_batch_equals_single_handles(precision):
    """With the built-in generator, realisation r of a batch is the run of
    a single handle with realisation = r (same frac_bits): positions bit for
    bit, masses to the tolerance, observables too."""
    ns = [700, 1500, 90, 2600]
    Ls = [700.0, 1500.0, 90.0, 2600.0]
    xs, As, Bs = batch_inputs(ns, Ls, seed=11)
    steps = 40
    p = batch_params(precision, observe_cap=steps, frac_bits=29, seed=5)
    sim = mt.Simulation(p, batch=mt.make_batch(ns, Ls, realisation=[10, 11, 12, 13]))
    sim.upload(np.concatenate(xs)[None, :], np.concatenate(As), np.concatenate(Bs))
    sim.run(steps)
    T = split(sim.ticks()[0], ns)
    ga, gb = sim.masses()
    ga, gb = split(ga, ns), split(gb, ns)
    obs = sim.observables()
    for r in range(len(ns)):
        q = mt.mt_params_init(dim=1, n=ns[r], L=(Ls[r],), D_rw=0.1, D_mt=0.1, dt=1.0,
                              precision=precision, observe_cap=steps, frac_bits=29, seed=5,
                              realisation=10 + r)
        one = mt.Simulation(q)
        one.upload(xs[r][None, :], As[r], Bs[r])
        one.run(steps)
        assert np.array_equal(one.ticks()[0], T[r])
        a1, b1 = one.masses()
        assert_masses(ga[r], a1, TOL[precision] / 10, f"A realisation {r}")
        assert_masses(gb[r], b1, TOL[precision] / 10, f"B realisation {r}")
        np.testing.assert_allclose(obs[:, r], one.observables(), rtol=1e-9, atol=1e-9)
        one.close()


@pytest.mark.parametrize("cluster", [300, 5000])
def test_batch_with_dense_realisation_uses_second_tier(cluster):
    """A realisation with a dense cluster: pair-heavy (second tier) or too big
    for it (general pipeline); the others are unaffected."""
    ns = [2000, 2000 + cluster, 1000]
    Ls = [2000.0, 2000.0, 1000.0]
    xs, As, Bs = batch_inputs(ns, Ls, seed=21)
    xs[1][:cluster] = 1000.0 + synth.uniform_positions(cluster, 1.0, seed=22)[0]
    sim = mt.Simulation(batch_params(mt.MT_FP64, observe_cap=4, D_rw=0.01),
                        batch=mt.make_batch(ns, Ls))
    Xs, a, b, _ = run_batch_vs_oracle(sim, ns, Ls, xs, As, Bs, 3, seed=23)
    mt.mt_set_profiling(sim.h, True)
    sim.set_noise(None)
    sim.step()
    names = [k for k, _ in mt.mt_read_profile(sim.h)]
    assert "fused_step" in names and ("fused_pred" in names or "fused_big" in names)
    if cluster == 5000:
        assert "move" in names  # the general pipeline redid the step
    assert names[-1] == "observables"  # after every step, whichever path ran it
    obs = sim.observables()
    assert obs.shape[1:] == (3, 4)
    for r in range(3):  # sum (A - B) is conserved by transfer and reaction
        np.testing.assert_allclose(obs[-1, r, 2], np.sum(a[r] - b[r]), rtol=1e-10, atol=1e-9)


def test_batch_graph_run_matches_step_loop():
    ns = [3000, 1200, 4500]
    Ls = [3000.0, 1200.0, 4500.0]
    xs, As, Bs = batch_inputs(ns, Ls, seed=31)
    out = []
    for mode in ("run", "step"):
        sim = mt.Simulation(batch_params(mt.MT_MIXED, observe_cap=8), batch=mt.make_batch(ns, Ls))
        sim.upload(np.concatenate(xs)[None, :], np.concatenate(As), np.concatenate(Bs))
        if mode == "run":
            sim.run(8)
        else:
            sim.step(8)
        out.append((sim.ticks(), *sim.masses(), sim.observables()))
    for u, v in zip(out[0], out[1]):
        assert np.array_equal(u, v)


def test_batch_of_256_log_uniform_realisations_invariants():
    """The ensemble shape of the batched workload at reduced size: 256
    realisations, N log-uniform in [1e3, 1e4], domain [0, N]; per
    realisation sum (A - B) stays exactly as the oracle's invariant says,
    and a sampled realisation matches the oracle after one step."""
    ns = synth.ensemble_sizes(256, 1e3, 1e4)
    Ls = [float(n) for n in ns]
    xs, As, Bs = batch_inputs(ns, Ls, seed=100)
    sim = mt.Simulation(batch_params(mt.MT_MIXED, observe_cap=20), batch=mt.make_batch(ns, Ls))
    sim.upload(np.concatenate(xs)[None, :], np.concatenate(As), np.concatenate(Bs))
    d0 = np.array([np.sum(As[r] - Bs[r]) for r in range(256)])
    sim.run(20)
    obs = sim.observables()
    assert obs.shape == (20, 256, 4)
    tot = np.array([np.sum(As[r] + Bs[r]) for r in range(256)])
    assert np.all(np.abs(obs[-1, :, 2] - d0) <= 1e-9 * tot)
    ga, gb = sim.masses()
    ga, gb = split(ga, ns), split(gb, ns)
    for r in range(256):
        np.testing.assert_allclose(obs[-1, r, 0], ga[r].sum(), rtol=1e-9)
        np.testing.assert_allclose(obs[-1, r, 3], ga[r].mean(), rtol=1e-9)


def test_autotune_picks_a_candidate_and_results_do_not_depend_on_it():
    """The tuner returns a resolved parameter set from its candidate list;
    the cell width and segment size change the schedule, not the results
    (positions bit for bit, masses to the tolerance)."""
    ns = synth.ensemble_sizes(16, 1e3, 2e4, seed0=40)
    Ls = [float(n) for n in ns]
    xs, As, Bs = batch_inputs(ns, Ls, seed=41)
    b = mt.make_batch(ns, Ls)
    p = batch_params(mt.MT_MIXED, observe_cap=4)
    x, A, B = np.concatenate(xs)[None, :], np.concatenate(As), np.concatenate(Bs)
    best, ms = mt.autotune(p, x, A, B, batch=b, warmup=2, steps=4)
    assert ms > 0.0
    auto = mt.mt_batch_resolve(p, b)
    assert abs(best.cell_shift - auto.cell_shift) <= 2 and 16 <= best.seg_target <= 1024
    out = []
    for q in (auto, best):
        sim = mt.Simulation(q, batch=b)
        sim.upload(x, A, B)
        sim.run(6)
        out.append((sim.ticks(), *sim.masses()))
    assert np.array_equal(out[0][0], out[1][0])
    assert_masses(out[1][1], out[0][1], 1e-6)
    assert_masses(out[1][2], out[0][2], 1e-6)


def test_autotune_single_system():
    n = 50000
    x = synth.uniform_positions(n, float(n), seed=50)
    A, B = synth.uniform_masses(n, seed=50)
    p = mt.mt_params_init(n=n, L=(float(n),), precision=mt.MT_MIXED)
    best, ms = mt.autotune(p, x, A, B, warmup=2, steps=3)
    assert ms > 0.0 and best.n == n and best.seg_target > 0
