"""Pins for the CPU oracle: each test checks it against something other than
itself -- a closed form worked by hand or in high-precision arithmetic, an
exhaustive listing on a tiny input, an invariant the paper states, a second
formulation, or a statistical law with a known value.

Paper references: Eq. 2 (move), Eq. 3 (weights), Sec. 1.1 (row
normalisation), Eq. 4-7 (exchange and its matrix form), Sec. 2.1 (fixed-radius
search), Sec. 3 (walls, D split, A + B -> E), Sec. 4 (pad width numbers).
"""
import itertools
import math

import mpmath as mp
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import synth

K = 29  # fractional bits of the position grid used throughout


def q1(xs):
    return O.quantize(np.asarray(xs, dtype=np.float64).reshape(1, -1), K)


# --------------------------------------------------------------- closed forms

@pytest.mark.parametrize("norm", [O.NORM_SYM, O.NORM_ROW])
def test_two_particles_closed_form(norm):
    """P-1: two particles at distance s: q = exp(-s^2/(8 D dt)), r = 1 + q,
    dM_1 = 1/2 q/(1+q) (M_2 - M_1) = -dM_2 under either normalisation."""
    p = O.params(L=(10.0,), norm=norm, react=0)
    s = 0.75
    X = q1([2.0, 2.0 + s])
    A = np.array([0.9, 0.2])
    B = np.array([0.1, 0.7])
    A2, B2 = O.mass_transfer(p, X, [A, B])
    mp.mp.dps = 40
    qq = mp.exp(-mp.mpf(s) ** 2 / (8 * mp.mpf(0.1) * 1))
    f = mp.mpf(1) / 2 * qq / (1 + qq)
    for M, M2 in ((A, A2), (B, B2)):
        d = f * (mp.mpf(M[1]) - mp.mpf(M[0]))
        assert abs(M2[0] - float(mp.mpf(M[0]) + d)) < 2e-16
        assert abs(M2[1] - float(mp.mpf(M[1]) - d)) < 2e-16


@pytest.mark.parametrize("norm", [O.NORM_SYM, O.NORM_ROW])
def test_three_collinear_closed_form(norm):
    """P-2: particles at 0, a, 2a, all in range.  Row sums r_end = 1 + q + q^4,
    r_mid = 1 + 2q.  ROW and SYM give different, hand-derivable answers, which
    also fixes the 1/2 of Eq. 4."""
    a = 0.5
    p = O.params(L=(10.0,), norm=norm, react=0)
    X = q1([3.0, 3.0 + a, 3.0 + 2 * a])
    M = np.array([1.0, 0.0, 0.25])
    (M2,) = O.mass_transfer(p, X, [M])
    mp.mp.dps = 40
    qq = mp.exp(-mp.mpf(a) ** 2 / (8 * mp.mpf(0.1)))
    q4 = qq ** 4
    r0, r1, r2 = 1 + qq + q4, 1 + 2 * qq, 1 + qq + q4
    w = {(0, 1): qq, (1, 2): qq, (0, 2): q4}
    r = [r0, r1, r2]
    Mm = [mp.mpf(v) for v in M]

    def Pn(i, j):
        wij = w[(min(i, j), max(i, j))]
        if norm == O.NORM_ROW:
            return wij / r[i]
        return (wij / r[i] + wij / r[j]) / 2

    # dM_0 by hand
    d0 = (Pn(0, 1) * (Mm[1] - Mm[0]) + Pn(0, 2) * (Mm[2] - Mm[0])) / 2
    d1 = (Pn(1, 0) * (Mm[0] - Mm[1]) + Pn(1, 2) * (Mm[2] - Mm[1])) / 2
    d2 = (Pn(2, 0) * (Mm[0] - Mm[2]) + Pn(2, 1) * (Mm[1] - Mm[2])) / 2
    exp = [float(Mm[0] + d0), float(Mm[1] + d1), float(Mm[2] + d2)]
    np.testing.assert_allclose(M2, exp, rtol=0, atol=4e-16)
    if norm == O.NORM_SYM:
        assert abs(M2.sum() - M.sum()) < 1e-15
    else:
        # the literal row normalisation does not conserve mass here
        assert abs(M2.sum() - M.sum()) > 1e-6


def test_row_and_sym_differ_only_when_row_sums_differ():
    """Equal row sums (two-particle and lattice interior) make ROW == SYM."""
    X = q1([1.0, 1.5])
    A = np.array([0.3, 0.8])
    (a1,) = O.mass_transfer(O.params(L=(10.0,), norm=O.NORM_SYM), X, [A])
    (a2,) = O.mass_transfer(O.params(L=(10.0,), norm=O.NORM_ROW), X, [A])
    np.testing.assert_allclose(a1, a2, rtol=0, atol=1e-16)


@pytest.mark.parametrize("norm", [O.NORM_SYM, O.NORM_ROW])
def test_coincident_cloud_halves_deviation(norm):
    """P-3: n particles at one point: P_ij = 1/n, so M' - mean = (M - mean)/2
    each step, exactly in real arithmetic."""
    n = 37
    X = q1(np.full(n, 12.25))
    M = synth.uniform_masses(n, seed=3)[0]
    mean = M.mean()
    cur = M
    for stepno in range(1, 4):
        (cur,) = O.mass_transfer(O.params(L=(50.0,), norm=norm), X, [cur])
        np.testing.assert_allclose(cur - mean, (M - mean) / 2 ** stepno, rtol=0, atol=2e-15)


def test_isolated_particles_unchanged_bitwise():
    """P-4: no pair within s_max -> P = I and masses unchanged bit for bit."""
    p = O.params(L=(100.0,))
    S = O.cutoff_ticks(p)
    X = np.array([[0, S + 1, 2 * S + 2, 3 * S + 3, 5 * S]], dtype=np.int64)
    A, B = synth.uniform_masses(5, seed=1)
    A2, B2 = O.mass_transfer(p, X, [A, B])
    assert np.array_equal(A2, A) and np.array_equal(B2, B)


# -------------------------------------------------- second formulations

@pytest.mark.parametrize("norm", [O.NORM_SYM, O.NORM_ROW])
@pytest.mark.parametrize("search", [O.SEARCH_CUTOFF, O.SEARCH_FULL])
@pytest.mark.parametrize("dim", [1, 2])
def test_loop_equals_matrix_form(norm, search, dim):
    """P-5: Eq. 4 as a loop and Eq. 5-6 (sign as Eq. 4) as a dense matvec."""
    n = 300
    L = (150.0, 15.0) if dim == 2 else (150.0,)
    p = O.params(dim=dim, L=L, norm=norm, search=search)
    X = O.quantize(synth.uniform_positions(n, L, dim=dim, seed=5), K)
    A, B = synth.uniform_masses(n, seed=5)
    a1, b1 = O.mass_transfer(p, X, [A, B])
    a2, b2 = O.mass_transfer_matrix(p, X, [A, B])
    np.testing.assert_allclose(a1, a2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(b1, b2, rtol=0, atol=1e-14)


@pytest.mark.parametrize("norm", [O.NORM_SYM, O.NORM_ROW])
def test_sorted_window_equals_all_pairs(norm):
    n = 3000
    p = O.params(L=(1500.0,), norm=norm)
    X = O.quantize(synth.uniform_positions(n, 1500.0, seed=6), K)
    A, B = synth.uniform_masses(n, seed=6)
    a1, b1 = O.mass_transfer(p, X, [A, B])
    a2, b2 = O.mass_transfer_sorted_1d(p, X, [A, B])
    np.testing.assert_allclose(a1, a2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(b1, b2, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [1, 2])
def test_sample_equals_all_pairs(dim):
    n = 800
    L = (400.0, 20.0) if dim == 2 else (400.0,)
    p = O.params(dim=dim, L=L)
    X = O.quantize(synth.uniform_positions(n, L, dim=dim, seed=8), K)
    A, B = synth.uniform_masses(n, seed=8)
    a1, b1 = O.mass_transfer(p, X, [A, B])
    idx = np.array([0, 5, 17, 399, 799])
    a2, b2 = O.mass_transfer_sample(p, X, [A, B], idx)
    np.testing.assert_allclose(a2, a1[idx], rtol=0, atol=1e-16)
    np.testing.assert_allclose(b2, b1[idx], rtol=0, atol=1e-16)


# ----------------------------------------------------------------- invariants

def test_sym_conserves_mass_and_row_obeys_maximum_principle():
    """P-6: SYM makes Eq. 4 an antisymmetric flux (sum dM = 0); ROW makes
    M_i' a convex combination of the old masses (sum_j P_ij = 1)."""
    n = 2000
    X = O.quantize(synth.uniform_positions(n, 1000.0, seed=9), K)
    A, B = synth.uniform_masses(n, seed=9)
    a, b = O.mass_transfer(O.params(L=(1000.0,)), X, [A, B])
    assert abs(a.sum() - A.sum()) <= 1e-13 * A.sum()
    assert abs(b.sum() - B.sum()) <= 1e-13 * B.sum()
    a, b = O.mass_transfer(O.params(L=(1000.0,), norm=O.NORM_ROW), X, [A, B])
    assert a.min() >= A.min() and a.max() <= A.max()
    assert abs(a.sum() - A.sum()) > 1e-9  # and does not conserve mass


def test_sym_weights_are_symmetric():
    """Moving a unit mass from i shows up at j with the same weight as the
    reverse: dM_j(e_i) = S_ji / 2 = S_ij / 2 = dM_i(e_j)."""
    n = 60
    X = O.quantize(synth.uniform_positions(n, 30.0, seed=10), K)
    p = O.params(L=(30.0,))
    G = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        (m,) = O.mass_transfer(p, X, [e])
        G[:, i] = m - e
    off = G - np.diag(np.diag(G))
    np.testing.assert_allclose(off, off.T, rtol=0, atol=1e-16)
    assert np.count_nonzero(off) > n  # the pairs really interact


def test_permutation_equivariance():
    n = 500
    X = O.quantize(synth.uniform_positions(n, 250.0, seed=11), K)
    A, B = synth.uniform_masses(n, seed=11)
    perm = synth.rng(11, 9).permutation(n)
    p = O.params(L=(250.0,))
    a, b = O.mass_transfer(p, X, [A, B])
    a2, b2 = O.mass_transfer(p, X[:, perm], [A[perm], B[perm]])
    np.testing.assert_allclose(a2, a[perm], rtol=0, atol=1e-15)
    np.testing.assert_allclose(b2, b[perm], rtol=0, atol=1e-15)


def test_react_invariants():
    """A + B -> E: min(A', B') = 0 exactly and A - B unchanged exactly."""
    A, B = synth.uniform_masses(10000, seed=12)
    B[:10] = A[:10]
    a, b = O.react(A, B)
    assert np.all(np.minimum(a, b) == 0.0)
    assert np.array_equal(a - b, A - B)
    assert np.all(a[:10] == 0) and np.all(b[:10] == 0)


# ----------------------------------------------------------------- truncation

@pytest.mark.parametrize("norm", [O.NORM_SYM, O.NORM_ROW])
def test_cutoff_within_truncation_bound(norm):
    """P-7: the cutoff result differs from the full matrix by no more than the
    neglected weight allows.  With rho_i = r_i^F - r_i^C, tau_i = rho_i/r_i^F
    and R the range of M:  ROW |dM^F - dM^C| <= tau_i R / 2;
    SYM <= R (tau_i + tau_max r_i^C + rho_i) / 4."""
    n = 1500
    L = 1500.0
    X = O.quantize(synth.uniform_positions(n, L, seed=13), K)
    A, _ = synth.uniform_masses(n, seed=13)
    pc = O.params(L=(L,), norm=norm)
    pf = O.params(L=(L,), norm=norm, search=O.SEARCH_FULL)
    (ac,) = O.mass_transfer(pc, X, [A])
    (af,) = O.mass_transfer(pf, X, [A])
    rc, rf = O.row_sums(pc, X), O.row_sums(pf, X)
    rho = rf - rc
    tau = rho / rf
    R = A.max() - A.min()
    bound = tau * R / 2 if norm == O.NORM_ROW else R * (tau + tau.max() * rc + rho) / 4
    diff = np.abs(af - ac)
    assert np.all(diff <= bound * (1 + 1e-12) + 1e-15)
    assert diff.max() > 0  # the cutoff really drops weight


def test_row_sum_means_match_gaussian_integrals():
    """For a uniform density rho, E[r^F - 1] = rho sqrt(8 pi D dt) and the
    expected weight beyond s_max is rho sqrt(8 pi D dt) erfc(s_max/sqrt(8 D dt));
    at the 3-sigma cutoff that is erfc(3/sqrt 2) of the total (Eq. 3's width)."""
    n, L = 8000, 8000.0
    X = O.quantize(synth.uniform_positions(n, L, seed=14), K)
    lo, hi = O.quantize(np.array([20.0, L - 20.0]), K)
    interior = (X[0] > lo) & (X[0] < hi)
    rc = O.row_sums(O.params(L=(L,)), X)
    rf = O.row_sums(O.params(L=(L,), search=O.SEARCH_FULL), X)
    tot = math.sqrt(8 * math.pi * 0.1)
    m_full = (rf - 1.0)[interior].mean()
    m_neg = (rf - rc)[interior].mean()
    assert abs(m_full - tot) < 0.04 * tot
    exp_neg = tot * math.erfc(3 / math.sqrt(2))
    assert abs(m_neg - exp_neg) < 0.1 * exp_neg


# -------------------------------------------------------- exhaustive pairs

def _pairs_by_hand(X, S, dim):
    n = X.shape[1]
    out = []
    for i, j in itertools.combinations(range(n), 2):
        dx = int(X[0, j]) - int(X[0, i])
        if dim == 1:
            ok = abs(dx) <= S
        else:
            dy = int(X[1, j]) - int(X[1, i])
            ok = dx * dx + dy * dy <= S * S
        if ok:
            out.append((i, j))
    return out


@pytest.mark.parametrize("dim", [1, 2])
def test_pairs_exhaustive_tiny(dim):
    """P-8: every pair of a tiny input checked with exact integers."""
    for seed in range(5):
        n = 64
        L = (40.0, 6.0) if dim == 2 else (40.0,)
        p = O.params(dim=dim, L=L)
        X = O.quantize(synth.uniform_positions(n, L, dim=dim, seed=seed), K)
        pi, pj = O.pairs_brute(p, X)
        assert list(zip(pi.tolist(), pj.tolist())) == _pairs_by_hand(X, O.cutoff_ticks(p), dim)


def test_pairs_edge_cases():
    """s exactly s_max (in), one tick more (out), particles at 0 and L, and a
    2-d pair at distance exactly Smax along a 3-4-5 diagonal (in)."""
    p = O.params(L=(100.0,))
    S = O.cutoff_ticks(p)
    Lq = O.quantize(np.array([100.0]), K)[0]
    X = np.array([[0, S, 2 * S + 1, Lq - S, Lq]], dtype=np.int64)
    pi, pj = O.pairs_brute(p, X)
    assert list(zip(pi.tolist(), pj.tolist())) == [(0, 1), (3, 4)]
    p2 = O.params(dim=2, L=(100.0, 100.0), smax=5.0 * 2 ** -20)
    S2 = O.cutoff_ticks(p2)
    assert S2 == 5 * 2 ** 9
    m = 2 ** 9
    X2 = np.array([[0, 3 * m, 3 * m + 1], [0, 4 * m, 4 * m]], dtype=np.int64)
    pi, pj = O.pairs_brute(p2, X2)
    assert list(zip(pi.tolist(), pj.tolist())) == [(0, 1), (1, 2)]


def test_sorted_pairs_equal_brute_pairs():
    n = 4000
    p = O.params(L=(2000.0,))
    X = O.quantize(synth.uniform_positions(n, 2000.0, seed=21), K)
    X[0, 100:110] = X[0, 100]  # coincident particles
    a = set(zip(*[v.tolist() for v in O.pairs_brute(p, X)]))
    b = set(zip(*[v.tolist() for v in O.pairs_sorted_1d(p, X)]))
    assert a == b and len(a) > n


# ---------------------------------------------------------------------- move

def test_move_drift_rounding_and_reflection():
    """Eq. 2 on the grid: drift rint(v dt 2^k), displacement rint(b xi),
    mirrored at 0 and at L (Sec. 3)."""
    p = O.params(L=(10.0,), v=(0.5,), D_rw=0.5, dt=1.0)  # b = sqrt(2*0.5*1) = 1
    X = q1([0.1, 5.0, 9.9])
    xi = np.array([[-0.7, 0.25, 0.3]], dtype=np.float32)
    X2 = O.move(p, X, xi)
    # b = 1 unit = 2^K ticks, so b xi is exact: the nearest tick by hand
    disp = [round(float(mp.mpf(float(v)) * 2 ** K)) for v in xi[0]]
    drift = int(0.5 * 2 ** K)
    Lq = 10 * 2 ** K
    raw = [int(X[0, i]) + drift + disp[i] for i in range(3)]
    exp = [raw[0] if raw[0] >= 0 else -raw[0], raw[1],
           raw[2] if raw[2] <= Lq else 2 * Lq - raw[2]]
    assert X2[0].tolist() == exp
    assert raw[2] > Lq  # the last particle really crossed the wall


@pytest.mark.parametrize("D_rw,dt,k", [(0.1, 1.0, 29), (0.5, 0.1, 33), (0.037, 0.25, 40)])
def test_move_displacement_is_eq2_in_binary64(D_rw, dt, k):
    """Eq. 2's random-walk displacement sqrt(2 D_rw dt) xi, evaluated in
    40-digit arithmetic and rounded to the nearest tick, for 400 normals:
    the oracle's displacement must equal it exactly.  A displacement formed
    as a binary32 product (the square root or the product rounded to 24
    bits, about 2^-24 relative, i.e. tens of ticks at k = 29) fails this pin,
    which the second half checks on the same values."""
    L = 2.0 ** 20
    p = O.params(L=(L,), v=(0.0,), D_rw=D_rw, dt=dt, frac_bits=k)
    n = 400
    xi = synth.normals(1, 1, n, seed=77)[0]
    xi[0, :4] = np.array([5.7, -5.7, 1e-3, 0.0], dtype=np.float32)
    X = np.full((1, n), 2 ** (k + 19), dtype=np.int64)  # mid-domain, no wall
    got = O.move(p, X, xi)[0] - X[0]
    mp.mp.dps = 40
    b = mp.sqrt(2 * mp.mpf(D_rw) * mp.mpf(dt)) * mp.mpf(2) ** k
    want = [int(mp.nint(b * mp.mpf(float(v)))) for v in xi[0]]
    assert got.tolist() == want
    # the same pin rejects a binary32 displacement
    b32 = np.float32(math.ldexp(math.sqrt(2.0 * D_rw * dt), k))
    f32 = [int(np.rint(np.float32(b32 * v))) for v in xi[0]]
    assert sum(a != w for a, w in zip(f32, want)) > n // 4


def test_move_statistics():
    """P-9: displacement mean v dt and variance 2 D_rw dt per axis."""
    n = 200000
    L = 1e6
    for dim in (1, 2):
        p = O.params(dim=dim, L=(L, L), v=(0.5, -0.25), D_rw=0.1, dt=1.0)
        X = O.quantize(np.full((dim, n), L / 2), K)
        xi = synth.normals(1, dim, n, seed=31)[0]
        d = (O.move(p, X, xi) - X) * 2.0 ** -K
        for ax, v in zip(range(dim), (0.5, -0.25)):
            assert abs(d[ax].mean() - v) < 5 * math.sqrt(0.2 / n)
            assert abs(d[ax].var() - 0.2) < 5 * 0.2 * math.sqrt(2 / n)


def test_move_stays_in_domain_with_large_steps():
    n = 5000
    p = O.params(L=(3.0,), D_rw=2.0)  # steps of ~2 units on a 3-unit domain
    X = O.quantize(synth.uniform_positions(n, 3.0, seed=32), K)
    xi = synth.normals(1, 1, n, seed=32)[0] * 3
    X2 = O.move(p, X, xi)
    assert X2.min() >= 0 and X2.max() <= 3 * 2 ** K


# ----------------------------------------------------------- physics pins

@pytest.mark.parametrize("norm", [O.NORM_SYM, O.NORM_ROW])
def test_pulse_variance_grows_by_2Ddt(norm):
    """P-9: on a dense regular lattice Eq. 3-4 is diffusion with D_mt: the
    variance of a mass pulse grows by exactly 2 D_mt dt per step (the 1/2 of
    Eq. 4 times the kernel variance 4 D_mt dt).  Pins the 8 D dt of Eq. 3, the
    1/2 of Eq. 4 and the sign."""
    h = 0.05
    n = 2001
    x = np.arange(n) * h
    X = q1(x)
    p = O.params(L=(x[-1],), norm=norm, search=O.SEARCH_FULL)
    M = np.exp(-((x - x.mean()) ** 2) / (2 * 0.3 ** 2))
    M /= M.sum()

    def var(m):
        mu = (m * x).sum() / m.sum()
        return (m * (x - mu) ** 2).sum() / m.sum()

    v0 = var(M)
    (M1,) = O.mass_transfer(p, X, [M])
    (M2,) = O.mass_transfer(p, X, [M1])
    assert abs((var(M1) - v0) - 2 * 0.1 * 1.0) < 1e-9
    assert abs((var(M2) - var(M1)) - 0.2) < 1e-9


def test_react_mean_of_uniform_masses():
    """A, B ~ U[0,1] -> E[A'] = E[(A - B)^+] = 1/6."""
    n = 400000
    A, B = synth.uniform_masses(n, seed=41)
    a, _ = O.react(A, B)
    assert abs(a.mean() - 1 / 6) < 5 * math.sqrt(1 / 18 - 1 / 36) / math.sqrt(n)


def test_step_order_move_transfer_react():
    """mto_step = move, then transfer on the moved positions, then react."""
    n = 400
    p = O.params(L=(200.0,))
    X = O.quantize(synth.uniform_positions(n, 200.0, seed=51), K)
    A, B = synth.uniform_masses(n, seed=51)
    xi = synth.normals(1, 1, n, seed=51)[0]
    X2, A2, B2 = O.step(p, X, xi, A, B)
    Xm = O.move(p, X, xi)
    assert np.array_equal(X2, Xm)
    a, b = O.mass_transfer(p, Xm, [A, B])
    a, b = O.react(a, b)
    np.testing.assert_allclose(A2, a, rtol=0, atol=1e-15)
    np.testing.assert_allclose(B2, b, rtol=0, atol=1e-15)


def test_sorted_window_edges_at_exactly_smax():
    """Window scan and all-pairs agree when pairs sit exactly at s_max (in)
    and one tick beyond (out), including ties in position."""
    p = O.params(L=(100.0,))
    S = O.cutoff_ticks(p)
    base = [0, S, 2 * S, 3 * S + 1, 3 * S + 1, 4 * S + 1, 6 * S + 3, 7 * S + 3]
    X = np.array([base[::-1]], dtype=np.int64)
    a = set(zip(*[v.tolist() for v in O.pairs_brute(p, X)]))
    b = set(zip(*[v.tolist() for v in O.pairs_sorted_1d(p, X)]))
    assert a == b and len(a) == 6
    A, B = synth.uniform_masses(len(base), seed=61)
    for u, v in zip(O.mass_transfer(p, X, [A, B]), O.mass_transfer_sorted_1d(p, X, [A, B])):
        np.testing.assert_allclose(u, v, rtol=0, atol=1e-16)


def test_observables_closed_form():
    """sum A, sum B, sum (A - B) and mean A of A = 1..n, B = n..1."""
    n = 1000
    A = np.arange(1, n + 1, dtype=np.float64)
    B = A[::-1].copy()
    o = O.observables(A, B)
    assert o.tolist() == [n * (n + 1) / 2, n * (n + 1) / 2, 0.0, (n + 1) / 2]


def test_sorted_window_threads_do_not_change_results():
    """The all-cores CPU baseline runs the sorted-window transfer's
    per-particle loops on several threads: bit-identical to one thread."""
    n = 20000
    p = O.params(L=(20000.0,), v=(0.5,))
    X = O.quantize(synth.uniform_positions(n, 20000.0, seed=41), K)
    A, B = synth.uniform_masses(n, seed=41)
    one = O.mass_transfer_sorted_1d(p, X, [A, B])
    try:
        O.set_threads(4)
        four = O.mass_transfer_sorted_1d(p, X, [A, B])
    finally:
        O.set_threads(1)
    for u, w in zip(one, four):
        assert np.array_equal(u, w)
