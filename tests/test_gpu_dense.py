"""Dense 1-d neighbourhoods (the paper's densities, Sec. 3 and Sec. 6: hundreds
to thousands of neighbours per particle) on the GPU: the transfer passes
over shared-memory tiles, against the oracle for single systems, batches,
more species, and a density whose neighbourhoods span many staged chunks."""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import mt, synth

from .test_gpu_parity import PRECISIONS, TOL, assert_masses
from .test_oracle_species import oracle_step_species, species_masses

pytestmark = pytest.mark.gpu


def oracle_of(r):
    return O.params(frac_bits=r.frac_bits, L=(r.L[0],), v=(r.v[0],), D_mt=r.D_mt, D_rw=r.D_rw,
                    dt=r.dt, smax=r.cutoff, norm=r.norm, react=r.react)


def profile_names(sim):
    mt.mt_set_profiling(sim.h, True)
    sim.step()
    names = [k for k, _ in mt.mt_read_profile(sim.h)]
    mt.mt_set_profiling(sim.h, False)
    return names


@pytest.mark.parametrize("n,L,S,steps", [
    (20000, 100.0, 2, 3),     # 200 per unit length: ~270 neighbours a side
    (12000, 6.0, 2, 2),       # 2000 per unit length: ~2700 a side, many chunks
    (9000, 45.0, 3, 3),       # three species
    (77, 0.4, 2, 3),          # one partial CTA, every particle within reach of every other
    (1000, 3.3, 2, 3),        # four CTAs, a ragged last one
])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_dense_tiles_match_oracle(n, L, S, steps, precision):
    p = mt.mt_params_init(n=n, L=(L,), v=(0.05,), D_mt=0.5, D_rw=0.5, dt=0.1,
                          precision=precision, species=S, observe_cap=4)
    sim = mt.Simulation(p)
    assert sim.params.seg_target == 0
    po = oracle_of(sim.params)
    k = int(sim.params.frac_bits)
    x = synth.uniform_positions(n, L, seed=n)
    Ms = species_masses(n, S, seed=n + 1)
    sim.upload(x, Ms[0], Ms[1])
    for s in range(2, S):
        sim.set_species(s, Ms[s])
    X = O.quantize(x.reshape(1, -1), k)
    cur = [m.copy() for m in Ms]
    xi = synth.normals(steps + 1, 1, n, seed=4)
    for s in range(steps):
        sim.set_noise(xi[s])
        sim.step()
        X, cur = oracle_step_species(po, X, xi[s], cur)
        assert np.array_equal(sim.ticks(), X), f"positions at step {s}"
    for s in range(S):
        assert_masses(sim.species(s), cur[s], TOL[precision], f"species {s}")
    sim.set_noise(xi[steps])
    names = profile_names(sim)
    assert "rowsum_tile" in names and "exchange_tile" in names
    assert "rowsum_walk" not in names


@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_dense_tiles_in_a_batch(precision):
    """Realisations at the paper's density side by side: the tiles never
    pair particles of different realisations."""
    ns = [3000, 1700, 4100, 2500]
    Ls = [15.0, 8.5, 20.5, 12.5]
    p = mt.mt_params_init(dim=1, L=(1.0,), D_mt=0.5, D_rw=0.5, dt=0.1, react=1,
                          precision=precision, frac_bits=29)
    sim = mt.Simulation(p, batch=mt.make_batch(ns, Ls))
    assert sim.params.seg_target == 0
    xs = [synth.uniform_positions(n, L, seed=50 + i) for i, (n, L) in enumerate(zip(ns, Ls))]
    As = [synth.uniform_masses(n, seed=60 + i) for i, n in enumerate(ns)]
    sim.upload(np.concatenate([x[0] for x in xs])[None, :], np.concatenate([a for a, _ in As]),
               np.concatenate([b for _, b in As]))
    xi = synth.normals(3, 1, sum(ns), seed=8)
    cur = []
    for i, (n, L) in enumerate(zip(ns, Ls)):
        po = O.params(frac_bits=29, L=(L,), D_mt=0.5, D_rw=0.5, dt=0.1, react=1)
        cur.append([O.quantize(xs[i], 29), As[i][0].copy(), As[i][1].copy(), po])
    offs = np.cumsum([0] + ns)
    for s in range(3):
        sim.set_noise(xi[s])
        sim.step()
        for i, c in enumerate(cur):
            c[0], c[1], c[2] = O.step(c[3], c[0], xi[s][:, offs[i]:offs[i + 1]], c[1], c[2])
    T = sim.ticks()[0]
    ga, gb = sim.masses()
    for i, c in enumerate(cur):
        sl = slice(offs[i], offs[i + 1])
        assert np.array_equal(T[sl], c[0][0])
        assert_masses(ga[sl], c[1], TOL[precision], f"A of realisation {i}")
        assert_masses(gb[sl], c[2], TOL[precision], f"B of realisation {i}")
    assert "rowsum_tile" in profile_names(sim)


@pytest.mark.parametrize("stored_p", [0, 1])
def test_paper_density_full_size_step(stored_p):
    """The paper-density workload at full size (N = 1e6 on [0, 5000], ~270
    neighbours a side, MIXED) in the benchmark's launch configuration (CUDA
    graph, built-in generator) for 5 steps, on the fly (tiles) and in the
    SPaM form; then one injected-noise step from the read-back state against
    the oracle element by element (sorted-window search), C1 and C2
    conserved."""
    n, L = 10 ** 6, 5000.0
    p = mt.mt_params_init(n=n, L=(L,), D_mt=0.5, D_rw=0.5, dt=0.1, react=0,
                          precision=mt.MT_MIXED, seed=3, stored_p=stored_p)
    sim = mt.Simulation(p)
    x = synth.uniform_positions(n, L, seed=9)
    c1, c2 = synth.segregated_masses(x, L)
    sim.upload(x, c1, c2)
    sim.run(5)
    X0 = sim.ticks()
    a0, b0 = sim.masses()
    assert abs(a0.sum() - c1.sum()) <= 1e-9 * n and abs(b0.sum() - c2.sum()) <= 1e-9 * n
    xi = synth.normals(1, 1, n, seed=77)[0]
    sim.set_noise(xi)
    sim.step()
    X1, a1, b1 = O.step(oracle_of(sim.params), X0, xi, a0, b0)
    assert np.array_equal(sim.ticks(), X1)
    ga, gb = sim.masses()
    assert_masses(ga, a1, TOL[mt.MT_MIXED], "C1")
    assert_masses(gb, b1, TOL[mt.MT_MIXED], "C2")
    sim.close()
