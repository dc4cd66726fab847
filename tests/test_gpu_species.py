"""More than two species on the GPU against the oracle (Sec. 1.1: the same
transfer weights act on every species; only A and B react): the 1-d and 2-d
cell lists and the all-pairs forms, FP64 and MIXED, an odd and an even count
of extra species, reflecting and periodic walls."""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import mt, synth

from .test_gpu_parity import TOL, assert_masses
from .test_oracle_species import oracle_step_species, species_masses

pytestmark = pytest.mark.gpu


def make(n, L, dim, search, precision, S, walls=mt.MT_WALLS_REFLECT, react=1):
    Ls = tuple(L) if dim == 2 else (float(L),)
    v = (0.4, -0.3)[:dim]
    p = mt.mt_params_init(dim=dim, n=n, L=Ls, v=v, D_rw=0.2, D_mt=0.15, search=search,
                          precision=precision, species=S, walls=walls, react=react,
                          observe_cap=8)
    return mt.Simulation(p)


def oracle_of(sim):
    r = sim.params
    return O.params(dim=r.dim, frac_bits=r.frac_bits, L=tuple(r.L)[: r.dim], v=tuple(r.v)[: r.dim],
                    D_mt=r.D_mt, D_rw=r.D_rw, dt=r.dt, smax=r.cutoff,
                    search=O.SEARCH_FULL if r.search == mt.MT_SEARCH_FULL else O.SEARCH_CUTOFF,
                    norm=r.norm, react=r.react, walls=r.walls)


CASES = [  # n, L, dim, search, S, steps
    (5000, 4000.0, 1, mt.MT_SEARCH_CELL, 3, 10),
    (3000, 2000.0, 1, mt.MT_SEARCH_CELL, 8, 6),
    (2000, (150.0, 120.0), 2, mt.MT_SEARCH_CELL, 5, 6),
    (600, 500.0, 1, mt.MT_SEARCH_BRUTE, 4, 5),
    (400, (30.0, 25.0), 2, mt.MT_SEARCH_BRUTE, 3, 4),
    (400, 300.0, 1, mt.MT_SEARCH_FULL, 5, 3),
]


def run_both(sim, n, L, dim, S, steps, seed):
    po = oracle_of(sim)
    k = int(sim.params.frac_bits)
    x = synth.uniform_positions(n, L, dim=dim, seed=seed)
    Ms = species_masses(n, S, seed=seed + 1)
    sim.upload(x, Ms[0], Ms[1])
    for s in range(2, S):
        sim.set_species(s, Ms[s])
    X = O.quantize(x.reshape(dim, -1), k)
    cur = [m.copy() for m in Ms]
    xi = synth.normals(steps, dim, n, seed=seed + 2)
    for s in range(steps):
        sim.set_noise(xi[s])
        sim.step()
        X, cur = oracle_step_species(po, X, xi[s], cur)
        assert np.array_equal(sim.ticks(), X), f"positions at step {s}"
    return Ms, cur


@pytest.mark.parametrize("n,L,dim,search,S,steps", CASES)
@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_species_match_oracle(n, L, dim, search, S, steps, precision):
    sim = make(n, L, dim, search, precision, S)
    assert sim.params.species == S and sim.params.seg_target == 0
    _, cur = run_both(sim, n, L, dim, S, steps, seed=n + S)
    for s in range(S):
        assert_masses(sim.species(s), cur[s], TOL[precision], f"species {s}")
    ga, gb = sim.masses()
    assert np.array_equal(ga, sim.species(0)) and np.array_equal(gb, sim.species(1))
    # A and B's observables are those of the two-species step
    obs = sim.observables()
    assert abs(obs[-1][0] - cur[0].sum()) <= 1e-9 * n


def test_species_with_periodic_walls():
    n, L, S = 3000, 2500.0, 4
    sim = make(n, L, 1, mt.MT_SEARCH_CELL, mt.MT_FP64, S, walls=mt.MT_WALLS_PERIODIC, react=0)
    Ms, cur = run_both(sim, n, L, 1, S, 8, seed=21)
    for s in range(S):
        got = sim.species(s)
        assert_masses(got, cur[s], TOL[mt.MT_FP64], f"species {s}")
        assert abs(got.sum() - Ms[s].sum()) <= 1e-10 * n


def test_two_species_path_unchanged_and_species_io():
    """species = 2 keeps the one-kernel step; species 0 and 1 read and set
    through the species calls are A and B; setting a species between steps
    takes effect at the next step."""
    n, L = 4000, 4000.0
    x = synth.uniform_positions(n, L, seed=5)
    A, B = synth.uniform_masses(n, seed=5)
    p2 = mt.mt_params_init(n=n, L=(L,), precision=mt.MT_FP64)
    s2 = mt.Simulation(p2)
    assert s2.params.seg_target > 0
    s2.upload(x, A, B)
    s2.run(3)
    p3 = mt.mt_params_init(n=n, L=(L,), precision=mt.MT_FP64, species=3)
    s3 = mt.Simulation(p3)
    s3.upload(x, A, B)
    assert np.array_equal(s3.species(2), np.zeros(n))  # upload zeroes the extra species
    s3.run(3)
    a2, b2 = s2.masses()
    a3, b3 = s3.masses()
    assert_masses(a3, a2, 1e-12, "A")
    assert_masses(b3, b2, 1e-12, "B")
    # set A through the species call; a second handle with the same A agrees
    newA = np.linspace(0.0, 1.0, n)
    s3.set_species(0, newA)
    assert np.array_equal(s3.species(0), newA)
    s2.set_species(0, newA)
    s3.run(2)
    s2.run(2)
    assert_masses(s3.masses()[0], s2.masses()[0], 1e-12, "A after set")
    with pytest.raises(mt.MtError):
        s3.set_species(3, newA)
    with pytest.raises(mt.MtError):
        s2.species(2)
    s2.close()
    s3.close()


def test_server_requests_with_more_species():
    """A request carrying three species, served beside a two-species one,
    equals its run alone in every species; the two-species call refuses it."""
    n, L, S = 3000, 3000.0, 3
    p3 = mt.mt_params_init(n=n, L=(L,), species=S, precision=mt.MT_MIXED, seed=9, observe_cap=5)
    x = synth.uniform_positions(n, L, seed=9)
    Ms = species_masses(n, S, seed=9)
    p2 = mt.mt_params_init(n=2000, L=(2000.0,), precision=mt.MT_MIXED, seed=10)
    x2 = synth.uniform_positions(2000, 2000.0, seed=10)
    A2, B2 = synth.uniform_masses(2000, seed=10)
    srv = mt.Server(pool_bytes=2 ** 26, max_active=2, chunk_steps=4)
    with pytest.raises(mt.MtError) as e:
        srv.submit(p3, x, Ms[0], Ms[1], 10)
    assert e.value.status == mt.MT_ERR_INVALID
    rid3 = srv.submit_species(p3, x, Ms, 10)
    srv.submit(p2, x2, A2, B2, 10)
    srv.drain()
    alone = mt.Simulation(p3)
    alone.upload(x, Ms[0], Ms[1])
    alone.set_species(2, Ms[2])
    alone.run(10)
    for s in range(S):
        assert np.array_equal(srv.result_species(rid3, s), alone.species(s)), f"species {s}"
    gA, gB, gobs = srv.result(rid3)
    assert np.array_equal(gA, alone.species(0)) and np.array_equal(gobs, alone.observables())
    with pytest.raises(mt.MtError):
        srv.result_species(rid3, S)
    srv.close()
    alone.close()


@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_species_in_a_batch(precision):
    """A batch of realisations carrying four species runs the multi-kernel
    pipeline; every realisation matches the oracle on its own, and species 2
    and 3 of each realisation are read back in the caller's order."""
    ns, Ls = [700, 1500, 400], [700.0, 1200.0, 500.0]
    S = 4
    k = 28  # cutoff 3 sqrt(4 D_mt dt) = 2.32: 2.32 2^k < 2^30
    p = mt.mt_params_init(dim=1, L=(1.0,), D_mt=0.15, D_rw=0.2, precision=precision, species=S,
                          frac_bits=k, observe_cap=4)
    sim = mt.Simulation(p, batch=mt.make_batch(ns, Ls))
    assert sim.params.seg_target == 0
    xs = [synth.uniform_positions(n, L, seed=70 + i) for i, (n, L) in enumerate(zip(ns, Ls))]
    Ms = [species_masses(n, S, seed=80 + i) for i, n in enumerate(ns)]
    sim.upload(np.concatenate([x[0] for x in xs])[None, :], np.concatenate([m[0] for m in Ms]),
               np.concatenate([m[1] for m in Ms]))
    for s in range(2, S):
        sim.set_species(s, np.concatenate([m[s] for m in Ms]))
    offs = np.cumsum([0] + ns)
    cur = []
    for i, (n, L) in enumerate(zip(ns, Ls)):
        po = O.params(frac_bits=k, L=(L,), D_mt=0.15, D_rw=0.2)
        cur.append([O.quantize(xs[i], k), [m.copy() for m in Ms[i]], po])
    xi = synth.normals(4, 1, sum(ns), seed=90)
    for s in range(4):
        sim.set_noise(xi[s])
        sim.step()
        for i, c in enumerate(cur):
            c[0], c[1] = oracle_step_species(c[2], c[0], xi[s][:, offs[i]:offs[i + 1]], c[1])
    T = sim.ticks()[0]
    got = [sim.species(s) for s in range(S)]
    for i, c in enumerate(cur):
        sl = slice(offs[i], offs[i + 1])
        assert np.array_equal(T[sl], c[0][0])
        for s in range(S):
            assert_masses(got[s][sl], c[1][s], TOL[precision], f"realisation {i} species {s}")
    obs = sim.observables()
    for i in range(len(ns)):  # each realisation's row sums its own A and B
        sl = slice(offs[i], offs[i + 1])
        np.testing.assert_allclose(obs[-1, i, :2], [got[0][sl].sum(), got[1][sl].sum()],
                                   rtol=1e-12)
