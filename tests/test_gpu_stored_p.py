"""The SPaM form (Sec. 6: the step's sparse transfer matrix stored once and
applied to the masses) on the GPU: parity with the oracle at the headline
density and at the paper's density, with a band wide enough and one so
narrow that most weights are recomputed past it, reflecting and periodic
walls, more than two species; and agreement with the on-the-fly form."""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import mt, synth

from .test_gpu_parity import TOL, assert_masses
from .test_oracle_species import oracle_step_species, species_masses

pytestmark = pytest.mark.gpu


def make(n, L, precision, stored_p, D_mt=0.1, dt=1.0, walls=mt.MT_WALLS_REFLECT, S=2, v=0.3):
    p = mt.mt_params_init(n=n, L=(float(L),), v=(v,), D_mt=D_mt, D_rw=D_mt, dt=dt,
                          precision=precision, stored_p=stored_p, walls=walls, species=S,
                          observe_cap=8)
    return mt.Simulation(p)


def oracle_of(sim):
    r = sim.params
    return O.params(frac_bits=r.frac_bits, L=(r.L[0],), v=(r.v[0],), D_mt=r.D_mt, D_rw=r.D_rw,
                    dt=r.dt, smax=r.cutoff, norm=r.norm, react=r.react, walls=r.walls)


CASES = [  # n, L, D_mt, dt, stored_p, walls, S, steps
    (20000, 20000.0, 0.1, 1.0, 1, mt.MT_WALLS_REFLECT, 2, 8),      # rho = 1, auto band
    (20000, 20000.0, 0.1, 1.0, 2, mt.MT_WALLS_REFLECT, 2, 8),      # band of 2: many recomputed
    (6000, 30.0, 0.5, 0.1, 1, mt.MT_WALLS_REFLECT, 2, 4),          # paper density, auto band
    (6000, 30.0, 0.5, 0.1, 100, mt.MT_WALLS_REFLECT, 2, 4),        # paper density, narrow band
    (8000, 6000.0, 0.1, 1.0, 1, mt.MT_WALLS_PERIODIC, 2, 8),
    (8000, 6000.0, 0.1, 1.0, 3, mt.MT_WALLS_PERIODIC, 3, 6),
    (5000, 40.0, 0.5, 0.1, 1, mt.MT_WALLS_REFLECT, 5, 3),
    (77, 0.4, 0.5, 0.1, 1, mt.MT_WALLS_REFLECT, 2, 3),        # all within reach, band = n
    (1000, 700.0, 0.1, 1.0, 1, mt.MT_WALLS_PERIODIC, 2, 4),   # ragged last warp tile
]


@pytest.mark.parametrize("n,L,D_mt,dt,stored_p,walls,S,steps", CASES)
@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_stored_p_matches_oracle(n, L, D_mt, dt, stored_p, walls, S, steps, precision):
    sim = make(n, L, precision, stored_p, D_mt=D_mt, dt=dt, walls=walls, S=S)
    assert sim.params.stored_p >= 2 and sim.params.seg_target == 0
    po = oracle_of(sim)
    k = int(sim.params.frac_bits)
    x = synth.uniform_positions(n, L, seed=n + S)
    Ms = species_masses(n, S, seed=n)
    sim.upload(x, Ms[0], Ms[1])
    for s in range(2, S):
        sim.set_species(s, Ms[s])
    X = O.quantize(x.reshape(1, -1), k)
    cur = [m.copy() for m in Ms]
    xi = synth.normals(steps, 1, n, seed=31)
    for s in range(steps):
        sim.set_noise(xi[s])
        sim.step()
        X, cur = oracle_step_species(po, X, xi[s], cur)
        assert np.array_equal(sim.ticks(), X), f"positions at step {s}"
    for s in range(S):
        assert_masses(sim.species(s), cur[s], TOL[precision], f"species {s}")


@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_stored_p_equals_on_the_fly(precision):
    """At the paper's density the stored form agrees with the on-the-fly form
    (FP64 to rounding), a run with one directly launched (profiled) step
    equals a graph-replayed run, and the profile shows the three SPaM
    kernels."""
    n, L = 50000, 250.0  # 200 per unit length, about 270 neighbours a side
    x = synth.uniform_positions(n, L, seed=3)
    c1, c2 = synth.segregated_masses(x, L)
    out = {}
    for sp in (0, 1):
        sim = make(n, L, precision, sp, D_mt=0.5, dt=0.1, v=0.0)
        sim.upload(x, c1, c2)
        sim.run(5)
        out[sp] = sim.masses()
        if sp:
            mt.mt_set_profiling(sim.h, True)
            sim.step()
            names = [k for k, _ in mt.mt_read_profile(sim.h)]
            assert ["band_build", "band_rowsum", "band_exchange"] == [
                k for k in names if k.startswith("band")]
            sim2 = make(n, L, precision, sp, D_mt=0.5, dt=0.1, v=0.0)
            sim2.upload(x, c1, c2)
            sim2.step(6)
            for a, b in zip(sim.masses(), sim2.masses()):
                assert np.array_equal(a, b)
    tol = 1e-12 if precision == mt.MT_FP64 else 1e-6
    for a, b in zip(out[0], out[1]):
        assert_masses(b, a, tol, "stored vs on the fly")


@pytest.mark.parametrize("walls", [mt.MT_WALLS_REFLECT, mt.MT_WALLS_PERIODIC])
@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_stored_p_in_a_batch(walls, precision):
    """The SPaM form for a batch: realisations at the paper's density side by
    side (periodic: each wraps on its own ring), each equal to the oracle of
    that realisation alone, with a band narrow enough that some weights are
    recomputed past it."""
    ns, Ls = [1500, 900, 2400], [7.5, 4.5, 12.0]
    k = 29
    p = mt.mt_params_init(dim=1, L=(1.0,), D_mt=0.5, D_rw=0.5, dt=0.1, precision=precision,
                          frac_bits=k, walls=walls, stored_p=200, observe_cap=4)
    sim = mt.Simulation(p, batch=mt.make_batch(ns, Ls))
    assert sim.params.stored_p == 200 and sim.params.seg_target == 0
    xs = [synth.uniform_positions(n, L, seed=40 + i) for i, (n, L) in enumerate(zip(ns, Ls))]
    AB = [synth.uniform_masses(n, seed=50 + i) for i, n in enumerate(ns)]
    sim.upload(np.concatenate([x[0] for x in xs])[None, :], np.concatenate([a for a, _ in AB]),
               np.concatenate([b for _, b in AB]))
    offs = np.cumsum([0] + ns)
    cur = []
    for i, L in enumerate(Ls):
        po = O.params(frac_bits=k, L=(L,), D_mt=0.5, D_rw=0.5, dt=0.1, walls=walls)
        cur.append([O.quantize(xs[i], k), AB[i][0].copy(), AB[i][1].copy(), po])
    xi = synth.normals(3, 1, sum(ns), seed=55)
    for s in range(3):
        sim.set_noise(xi[s])
        sim.step()
        for i, c in enumerate(cur):
            Xo, Ms = oracle_step_species(c[3], c[0], xi[s][:, offs[i]:offs[i + 1]], [c[1], c[2]])
            c[0], c[1], c[2] = Xo, Ms[0], Ms[1]
    T = sim.ticks()[0]
    ga, gb = sim.masses()
    for i, c in enumerate(cur):
        sl = slice(offs[i], offs[i + 1])
        assert np.array_equal(T[sl], c[0][0])
        assert_masses(ga[sl], c[1], TOL[precision], f"A of realisation {i}")
        assert_masses(gb[sl], c[2], TOL[precision], f"B of realisation {i}")
