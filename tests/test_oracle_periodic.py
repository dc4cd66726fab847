"""The oracle with periodic walls (a variant of Sec. 3's reflecting ones): the
move wraps, separations are minimum images, and the transfer is invariant
under translation on the ring."""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import synth

K = 29


def per(L=20.0, **kw):
    kw.setdefault("D_mt", 0.1)
    return O.params(L=(L,), frac_bits=K, walls=O.WALLS_PERIODIC, **kw)


def test_move_wraps_around():
    p = per(L=20.0, v=(0.3,), D_rw=0.0, dt=1.0)
    X = O.quantize(np.array([[19.9, 0.05, 10.0]]), K)
    X2 = O.move(p, X, np.zeros((1, 3), dtype=np.float32))
    drift = O.quantize(np.array([[0.3]]), K)[0, 0]
    Lq = O.quantize(np.array([[20.0]]), K)[0, 0]
    assert X2[0].tolist() == [(X[0, 0] + drift) % Lq, X[0, 1] + drift, X[0, 2] + drift]


def test_pair_across_the_wall_equals_the_same_pair_inside():
    p = per(L=20.0)
    A = np.array([1.0, 0.0])
    B = np.array([0.0, 1.0])
    X_edge = O.quantize(np.array([[19.9, 0.1]]), K)   # 0.2 apart through the wall
    X_mid = O.quantize(np.array([[10.0, 10.2]]), K)
    a1, b1 = O.mass_transfer(p, X_edge, [A, B])
    a2, b2 = O.mass_transfer(p, X_mid, [A, B])
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    assert 0.0 < a1[1] < 0.5  # mass did move across the wall
    i, j = O.pairs_brute(p, X_edge)
    assert list(zip(i.tolist(), j.tolist())) == [(0, 1)]
    # with reflecting walls the two are 19.8 apart: no pair, no transfer
    q = O.params(L=(20.0,), frac_bits=K, D_mt=0.1)
    assert len(O.pairs_brute(q, X_edge)[0]) == 0
    a3, _ = O.mass_transfer(q, X_edge, [A, B])
    assert np.array_equal(a3, A)


@pytest.mark.parametrize("search", [O.SEARCH_CUTOFF, O.SEARCH_FULL])
def test_translation_on_the_ring_changes_nothing(search):
    n, L = 300, 60.0
    p = per(L=L, search=search)
    X = O.quantize(synth.uniform_positions(n, L, seed=3), K)
    A, B = synth.uniform_masses(n, seed=3)
    Lq = O.quantize(np.array([[L]]), K)[0, 0]
    a1, b1 = O.mass_transfer(p, X, [A, B])
    for shift in (1, Lq // 3, Lq - 7):
        Xs = (X + shift) % Lq
        a2, b2 = O.mass_transfer(p, Xs, [A, B])
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)


def test_periodic_transfer_conserves_and_step_runs():
    n, L = 400, 40.0
    p = per(L=L, v=(0.7,), D_rw=0.2, react=0)
    X = O.quantize(synth.uniform_positions(n, L, seed=5), K)
    A, B = synth.uniform_masses(n, seed=5)
    xi = synth.normals(5, 1, n, seed=6)
    a, b = A.copy(), B.copy()
    Lq = O.quantize(np.array([[L]]), K)[0, 0]
    for s in range(5):
        X, a, b = O.step(p, X, xi[s], a, b)
        assert X.min() >= 0 and X.max() < Lq
    assert abs(a.sum() - A.sum()) <= 1e-11 * n and abs(b.sum() - B.sum()) <= 1e-11 * n


def test_periodic_needs_cutoff_below_half_the_domain():
    p = per(L=3.0)  # s_max = 1.897 > L / 2
    X = O.quantize(np.array([[0.5, 2.5]]), K)
    with pytest.raises(ValueError):
        O.mass_transfer(p, X, [np.ones(2), np.zeros(2)])
