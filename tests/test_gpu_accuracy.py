"""The paper's accuracy test problem (Sec. 3) on the GPU, as batches of
realisations: parity with the oracle per realisation, and the error against
the exact solution over 75 realisations."""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import accuracy as acc
from paper_1811_05474_gb300 import mt, synth

pytestmark = pytest.mark.gpu


def batch_sim(ns, precision, norm=mt.MT_NORM_SYM, seed=11):
    kw = acc.params_kw()
    p = mt.mt_params_init(dim=1, L=(1.0,), D_mt=kw["D_mt"], D_rw=kw["D_rw"], dt=kw["dt"],
                          react=0, precision=precision, norm=norm, frac_bits=29, seed=seed)
    return mt.Simulation(p, batch=mt.make_batch(ns, [acc.L] * len(ns)))


def split(v, ns):
    return np.split(np.asarray(v), np.cumsum(ns)[:-1])


@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_paper_problem_batch_equals_oracle_per_realisation(precision):
    ns = [500] * 6 + [1000] * 2
    ins = [acc.inputs(n, 300 + r) for r, n in enumerate(ns)]
    sim = batch_sim(ns, precision)
    sim.upload(np.concatenate([i[0][0] for i in ins])[None, :], np.concatenate([i[1] for i in ins]),
               np.concatenate([i[2] for i in ins]))
    kw = acc.params_kw()
    po = O.params(frac_bits=29, **kw)
    X = [O.quantize(i[0], 29) for i in ins]
    c1 = [i[1].copy() for i in ins]
    c2 = [i[2].copy() for i in ins]
    xi = synth.normals(acc.STEPS, 1, sum(ns), seed=5)
    for s in range(acc.STEPS):
        sim.set_noise(xi[s])
        sim.step()
        parts = split(xi[s][0], ns)
        for r in range(len(ns)):
            X[r], c1[r], c2[r] = O.step(po, X[r], parts[r][None, :], c1[r], c2[r])
    T = split(sim.ticks()[0], ns)
    g1, g2 = (split(v, ns) for v in sim.masses())
    tol = 1e-12 if precision == mt.MT_FP64 else 1e-6
    for r in range(len(ns)):
        assert np.array_equal(T[r], X[r][0])
        assert np.max(np.abs(g1[r] - c1[r])) <= tol
        assert np.max(np.abs(g2[r] - c2[r])) <= tol


@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_paper_problem_error_against_exact_solution(precision):
    """75 realisations each of N = 500 and N = 2500 in one batch (built-in
    generator): error and fitted D in the bands the oracle shows, falling
    with N, C1 conserved."""
    ns = [500] * acc.REALISATIONS + [2500] * acc.REALISATIONS
    ins = [acc.inputs(n, 1000 + r) for r, n in enumerate(ns)]
    sim = batch_sim(ns, precision)
    sim.upload(np.concatenate([i[0][0] for i in ins])[None, :], np.concatenate([i[1] for i in ins]),
               np.concatenate([i[2] for i in ins]))
    sim.run(acc.STEPS)
    xs = split(sim.positions()[0], ns)
    c1 = split(sim.masses()[0], ns)
    R = acc.REALISATIONS
    e500 = [acc.rmse(xs[r], c1[r]) for r in range(R)]
    e2500 = [acc.rmse(xs[r], c1[r]) for r in range(R, 2 * R)]
    assert 0.015 < np.mean(e500) < 0.032
    assert 0.007 < np.mean(e2500) < 0.016
    assert np.mean(e2500) < np.mean(e500)
    assert 0.85 <= acc.fitted_d(xs[:R], c1[:R]) <= 1.02
    assert 0.85 <= acc.fitted_d(xs[R:], c1[R:]) <= 1.02
    for r in range(2 * R):
        assert abs(c1[r].sum() - ins[r][1].sum()) <= 1e-9 * ns[r]


def test_cutoff_width_and_full_matrix_on_the_paper_problem():
    """75 realisations of N = 500 (the same inputs and built-in walks for
    each variant): a 2-sigma cutoff damps the transfer visibly against
    3 sigma (fitted D), and the full matrix, run as one handle per
    realisation, gives the cell list's RMSE and fitted D."""
    R, n = acc.REALISATIONS, 500
    ns = [n] * R
    ins = [acc.inputs(n, 2000 + r) for r in range(R)]
    x = np.concatenate([i[0][0] for i in ins])[None, :]
    c1 = np.concatenate([i[1] for i in ins])
    c2 = np.concatenate([i[2] for i in ins])
    sig = np.sqrt(4 * 0.5 * acc.DT)
    out = {}
    for name, cutoff in (("3s", 3 * sig), ("2s", 2 * sig)):
        kw = acc.params_kw()
        p = mt.mt_params_init(dim=1, L=(1.0,), D_mt=kw["D_mt"], D_rw=kw["D_rw"], dt=kw["dt"],
                              react=0, precision=mt.MT_MIXED, frac_bits=29, seed=17, cutoff=cutoff)
        sim = mt.Simulation(p, batch=mt.make_batch(ns, [acc.L] * R))
        sim.upload(x, c1, c2)
        sim.run(acc.STEPS)
        out[name] = (split(sim.positions()[0], ns), split(sim.masses()[0], ns))
        sim.close()
    xs, cs = [], []
    for r in range(R):
        kw = acc.params_kw()
        p = mt.mt_params_init(n=n, L=(acc.L,), D_mt=kw["D_mt"], D_rw=kw["D_rw"], dt=kw["dt"], react=0,
                              precision=mt.MT_MIXED, frac_bits=29, seed=17, realisation=r,
                              search=mt.MT_SEARCH_FULL)
        sim = mt.Simulation(p)
        sim.upload(ins[r][0], ins[r][1], ins[r][2])
        sim.run(acc.STEPS)
        xs.append(sim.positions()[0])
        cs.append(sim.masses()[0])
        sim.close()
    out["full"] = (xs, cs)
    d = {k: acc.fitted_d(*v) for k, v in out.items()}
    e = {k: np.mean([acc.rmse(a, b) for a, b in zip(*v)]) for k, v in out.items()}
    assert d["2s"] < d["3s"] - 0.05
    assert abs(d["full"] - d["3s"]) < 0.03
    assert e["2s"] > e["3s"]
    assert abs(e["full"] - e["3s"]) < 0.1 * e["3s"]
