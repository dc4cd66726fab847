"""The oracle with more than two species (Sec. 1.1: one system of Eq. 4 per
species, all with the same transfer weights; cost linear in the species
count).  Pins the multi-species transfer against what the mathematics fixes:
species do not interact (each equals its transfer alone, bit for bit), the
transfer is linear in the masses, the dense matrix form (Eq. 5-6) agrees,
symmetric normalisation conserves every species, and a uniform species stays
uniform.  The step with S species is the paper's order (move, transfer,
reaction of A and B only), written here from the oracle's pieces and checked
against the oracle's own two-species step."""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import synth

K = 27


def species_masses(n, S, seed):
    g = np.random.default_rng(seed)
    return [g.uniform(0.0, 1.0, n) for _ in range(S)]


def oracle_step_species(p, X, xi, Ms):
    """Move, transfer all species with the same weights, then A + B -> E on
    species 0 and 1; returns (X, Ms)."""
    X = O.move(p, X, xi)
    if p.dim == 1 and p.search == O.SEARCH_CUTOFF and p.walls == O.WALLS_REFLECT:
        Ms = O.mass_transfer_sorted_1d(p, X, Ms)
    else:
        Ms = O.mass_transfer(p, X, Ms)
    if p.react:
        a, b = O.react(Ms[0], Ms[1])
        Ms = [a, b] + list(Ms[2:])
    return X, Ms


@pytest.mark.parametrize("dim,search", [(1, O.SEARCH_CUTOFF), (2, O.SEARCH_CUTOFF),
                                        (1, O.SEARCH_FULL)])
def test_species_do_not_interact(dim, search):
    n = 400
    L = (400.0,) if dim == 1 else (40.0, 40.0)
    p = O.params(dim=dim, L=L, frac_bits=K, search=search, D_mt=0.5)
    X = O.quantize(synth.uniform_positions(n, L if dim == 2 else L[0], dim=dim, seed=1), K)
    Ms = species_masses(n, 5, seed=2)
    out = O.mass_transfer(p, X, Ms)
    for s in range(5):
        alone = O.mass_transfer(p, X, [Ms[s]])[0]
        assert np.array_equal(out[s], alone), f"species {s}"


def test_transfer_is_linear_in_the_masses():
    n = 500
    p = O.params(L=(300.0,), frac_bits=K, D_mt=0.4)
    X = O.quantize(synth.uniform_positions(n, 300.0, seed=3), K)
    a, b = species_masses(n, 2, seed=4)
    c = 0.3 * a - 1.7 * b
    oa, ob, oc = O.mass_transfer(p, X, [a, b, c])
    assert np.max(np.abs(oc - (0.3 * oa - 1.7 * ob))) <= 1e-13


def test_matrix_form_agrees_for_four_species():
    n = 300
    p = O.params(L=(200.0,), frac_bits=K, D_mt=0.5)
    X = O.quantize(synth.uniform_positions(n, 200.0, seed=5), K)
    Ms = species_masses(n, 4, seed=6)
    loop = O.mass_transfer(p, X, Ms)
    mat = O.mass_transfer_matrix(p, X, Ms)
    for s in range(4):
        assert np.max(np.abs(loop[s] - mat[s])) <= 1e-13


def test_every_species_is_conserved_and_uniform_stays_uniform():
    n = 600
    p = O.params(L=(500.0,), frac_bits=K, D_mt=0.5, D_rw=0.2, react=0)
    X = O.quantize(synth.uniform_positions(n, 500.0, seed=7), K)
    Ms = species_masses(n, 3, seed=8) + [np.full(n, 0.25)]
    xi = synth.normals(4, 1, n, seed=9)
    cur = [m.copy() for m in Ms]
    for s in range(4):
        X, cur = oracle_step_species(p, X, xi[s], cur)
    for m0, m in zip(Ms, cur):
        assert abs(m.sum() - m0.sum()) <= 1e-11 * n
    assert np.max(np.abs(cur[3] - 0.25)) <= 1e-15


def test_composed_step_equals_the_two_species_step():
    n = 700
    p = O.params(L=(700.0,), frac_bits=K, D_mt=0.3, D_rw=0.3, v=(0.2, 0.0))
    X = O.quantize(synth.uniform_positions(n, 700.0, seed=10), K)
    A, B = synth.uniform_masses(n, seed=10)
    xi = synth.normals(3, 1, n, seed=11)
    Xa, Ms = X.copy(), [A.copy(), B.copy()]
    Xb, a, b = X.copy(), A.copy(), B.copy()
    for s in range(3):
        Xa, Ms = oracle_step_species(p, Xa, xi[s], Ms)
        Xb, a, b = O.step(p, Xb, xi[s], a, b)
    assert np.array_equal(Xa, Xb)
    assert np.array_equal(Ms[0], a) and np.array_equal(Ms[1], b)
