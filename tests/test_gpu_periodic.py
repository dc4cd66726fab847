"""Periodic walls on the GPU against the oracle: the wrapping move, minimum-
image pairs and weights, for the cell lists (1-d general pipeline; 2-d with
wrapped cell neighbourhoods, including partial last cells and grids of two
cells a side) and the all-pairs forms in 1-d and 2-d."""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import mt, synth

from .test_gpu_parity import TOL, assert_masses

pytestmark = pytest.mark.gpu


def make(n, L, dim, search, precision, v=(0.7, -0.4), D_rw=0.3):
    Ls = tuple(L) if dim == 2 else (float(L),)
    p = mt.mt_params_init(dim=dim, n=n, L=Ls, v=v[:dim] if dim == 2 else (v[0],), D_rw=D_rw,
                          search=search, precision=precision, walls=mt.MT_WALLS_PERIODIC,
                          observe_cap=8)
    return mt.Simulation(p)


def oracle_of(sim):
    r = sim.params
    return O.params(dim=r.dim, frac_bits=r.frac_bits, L=tuple(r.L)[: r.dim], v=tuple(r.v)[: r.dim],
                    D_mt=r.D_mt, D_rw=r.D_rw, dt=r.dt, smax=r.cutoff,
                    search=O.SEARCH_FULL if r.search == mt.MT_SEARCH_FULL else O.SEARCH_CUTOFF,
                    norm=r.norm, react=r.react, walls=O.WALLS_PERIODIC)


CASES = [
    (3000, 2000.0, 1, mt.MT_SEARCH_CELL, 12),
    (500, 300.0, 1, mt.MT_SEARCH_BRUTE, 6),
    (500, 300.0, 1, mt.MT_SEARCH_FULL, 3),
    (400, (30.0, 20.0), 2, mt.MT_SEARCH_BRUTE, 6),
    (3000, (120.0, 90.0), 2, mt.MT_SEARCH_CELL, 8),
    (500, (9.0, 7.1), 2, mt.MT_SEARCH_CELL, 6),    # a few cells a side, partial last cells
    (300, (4.0, 3.9), 2, mt.MT_SEARCH_CELL, 4),    # two cells a side: the wrapped pieces meet
    (300, (20.0, 12.0), 2, mt.MT_SEARCH_FULL, 3),
]


@pytest.mark.parametrize("n,L,dim,search,steps", CASES)
@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_periodic_matches_oracle(n, L, dim, search, steps, precision):
    sim = make(n, L, dim, search, precision)
    assert sim.params.seg_target == 0  # no one-kernel step with periodic walls
    po = oracle_of(sim)
    k = int(sim.params.frac_bits)
    x = synth.uniform_positions(n, L, dim=dim, seed=n + dim)
    A, B = synth.uniform_masses(n, seed=n)
    sim.upload(x, A, B)
    X = O.quantize(x.reshape(dim, -1), k)
    a, b = A.copy(), B.copy()
    xi = synth.normals(steps, dim, n, seed=77)
    Lq = [O.quantize(np.array([[v]]), k)[0, 0] for v in (L if dim == 2 else (L,))]
    for s in range(steps):
        sim.set_noise(xi[s])
        sim.step()
        X, a, b = O.step(po, X, xi[s], a, b)
        T = sim.ticks()
        assert np.array_equal(T, X), f"positions at step {s}"
        for ax in range(dim):
            assert T[ax].min() >= 0 and T[ax].max() < Lq[ax]
    ga, gb = sim.masses()
    assert_masses(ga, a, TOL[precision], "A")
    assert_masses(gb, b, TOL[precision], "B")
    if search != mt.MT_SEARCH_FULL:
        gi, gj = sim.pairs()
        oi, oj = O.pairs_brute(po, X)
        got = set(zip(gi.tolist(), gj.tolist()))
        assert len(got) == len(gi) and got == set(zip(oi.tolist(), oj.tolist()))


def test_periodic_pair_across_the_wall():
    """Two particles 0.2 apart through the wall exchange mass like an
    interior pair; with reflecting walls they do not interact."""
    x = np.array([[19.9, 0.1]])
    A = np.array([1.0, 0.0])
    B = np.array([0.0, 1.0])
    out = []
    for walls in (mt.MT_WALLS_PERIODIC, mt.MT_WALLS_REFLECT):
        p = mt.mt_params_init(n=2, L=(20.0,), D_rw=0.0, react=0, walls=walls)
        sim = mt.Simulation(p)
        sim.upload(x, A, B)
        sim.step()
        out.append(sim.masses()[0])
    assert 0.0 < out[0][1] < 0.5
    assert out[1][1] == 0.0


@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_periodic_batch_each_realisation_wraps_on_its_own(precision):
    """A batch with periodic walls: every realisation wraps on its own domain
    (its walks go around its own slot range) and equals the oracle of that
    realisation alone; the pair sets never join two realisations."""
    ns, Ls = [800, 1500, 300], [600.0, 1500.0, 250.0]
    k = 29
    p = mt.mt_params_init(dim=1, L=(1.0,), v=(0.6,), D_rw=0.3, precision=precision, frac_bits=k,
                          walls=mt.MT_WALLS_PERIODIC, observe_cap=4)
    sim = mt.Simulation(p, batch=mt.make_batch(ns, Ls))
    assert sim.params.seg_target == 0
    xs = [synth.uniform_positions(n, L, seed=60 + i) for i, (n, L) in enumerate(zip(ns, Ls))]
    AB = [synth.uniform_masses(n, seed=61 + i) for i, n in enumerate(ns)]
    sim.upload(np.concatenate([x[0] for x in xs])[None, :], np.concatenate([a for a, _ in AB]),
               np.concatenate([b for _, b in AB]))
    offs = np.cumsum([0] + ns)
    cur = []
    for i, L in enumerate(Ls):
        po = O.params(frac_bits=k, L=(L,), v=(0.6,), D_rw=0.3, walls=O.WALLS_PERIODIC)
        cur.append([O.quantize(xs[i], k), AB[i][0].copy(), AB[i][1].copy(), po])
    xi = synth.normals(6, 1, sum(ns), seed=62)
    for s in range(6):
        sim.set_noise(xi[s])
        sim.step()
        for i, c in enumerate(cur):
            c[0], c[1], c[2] = O.step(c[3], c[0], xi[s][:, offs[i]:offs[i + 1]], c[1], c[2])
    T = sim.ticks()[0]
    ga, gb = sim.masses()
    for i, c in enumerate(cur):
        sl = slice(offs[i], offs[i + 1])
        assert np.array_equal(T[sl], c[0][0]), f"realisation {i} positions"
        assert_masses(ga[sl], c[1], TOL[precision], f"A of realisation {i}")
        assert_masses(gb[sl], c[2], TOL[precision], f"B of realisation {i}")
    gi, gj = sim.pairs()
    got = set(zip(gi.tolist(), gj.tolist()))
    want = set()
    for i, c in enumerate(cur):
        oi, oj = O.pairs_brute(c[3], c[0])
        want |= set(zip((oi + offs[i]).tolist(), (oj + offs[i]).tolist()))
    assert len(got) == len(gi) and got == want
