"""GPU path vs the CPU oracle, through the C ABI.

Every test injects the same random-walk normals into both sides, so the
positions must agree bit for bit (they are integers on the grid), the pair
set must be identical, and the masses must agree to 1e-12 (FP64) or 1e-6
(MIXED) relative, with relative taken against max(|m_oracle|, m_ref) where
m_ref = 0.5 is the mean initial mass (late-time values after the reaction
cancel towards zero).
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import mt, synth

pytestmark = pytest.mark.gpu

TOL = {mt.MT_FP64: 1e-12, mt.MT_MIXED: 1e-6, mt.MT_MIXED_DF32: 1e-6}
PRECISIONS = [mt.MT_FP64, mt.MT_MIXED, mt.MT_MIXED_DF32]
MREF = 0.5


def make(n, L, *, dim=1, search=mt.MT_SEARCH_CELL, precision=mt.MT_FP64,
         norm=mt.MT_NORM_SYM, react=1, v=(0.0, 0.0), D_rw=0.1, D_mt=0.1, dt=1.0,
         cutoff=0.0, observe_cap=0, seed=0, frac_bits=0, cell_shift=0):
    Ls = tuple(L) if isinstance(L, (tuple, list)) else (float(L),)
    p = mt.mt_params_init(dim=dim, n=n, L=Ls, v=v, D_rw=D_rw, D_mt=D_mt, dt=dt,
                          cutoff=cutoff, search=search, precision=precision, norm=norm,
                          react=react, observe_cap=observe_cap, seed=seed,
                          frac_bits=frac_bits, cell_shift=cell_shift)
    return mt.Simulation(p)


def oracle_params(sim):
    r = sim.params
    return O.params(dim=r.dim, frac_bits=r.frac_bits, L=tuple(r.L), v=tuple(r.v),
                    D_mt=r.D_mt, D_rw=r.D_rw, dt=r.dt, smax=r.cutoff,
                    search=O.SEARCH_FULL if r.search == mt.MT_SEARCH_FULL else O.SEARCH_CUTOFF,
                    norm=r.norm, react=r.react)


def assert_masses(g, o, tol, what=""):
    err = np.abs(g - o) / np.maximum(np.abs(o), MREF)
    assert err.max(initial=0.0) <= tol, f"{what} max rel err {err.max():.3e} (tol {tol})"


def run_both(sim, x, A, B, steps, seed=0, check_every=True, pairs=True):
    po = oracle_params(sim)
    k = int(sim.params.frac_bits)
    sim.upload(x, A, B)
    X = O.quantize(np.asarray(x).reshape(sim.dim, -1), k)
    a, b = np.array(A, dtype=np.float64), np.array(B, dtype=np.float64)
    xi = synth.normals(steps, sim.dim, sim.n, seed=seed + 1000)
    tol = TOL[int(sim.params.precision)]
    for s in range(steps):
        sim.set_noise(xi[s])
        sim.step()
        X, a, b = O.step(po, X, xi[s], a, b)
        if check_every or s == steps - 1:
            assert np.array_equal(sim.ticks(), X), f"positions differ at step {s}"
            ga, gb = sim.masses()
            assert_masses(ga, a, tol, f"A step {s}")
            assert_masses(gb, b, tol, f"B step {s}")
    if pairs and sim.params.search != mt.MT_SEARCH_FULL:
        gi, gj = sim.pairs()
        oi, oj = O.pairs_brute(po, X)
        got = set(zip(gi.tolist(), gj.tolist()))
        assert len(got) == len(gi), "a pair was reported twice"
        assert got == set(zip(oi.tolist(), oj.tolist())), "pair sets differ"
    return X, a, b


# ------------------------------------------------------------ workload 1 --

@pytest.mark.parametrize("search", [mt.MT_SEARCH_CELL, mt.MT_SEARCH_BRUTE, mt.MT_SEARCH_FULL])
def test_1d_n1000_100_steps_fp64(search):
    """N = 1000 uniform on [0, 1000], D = 0.1, dt = 1, cutoff 3 sigma,
    100 steps, FP64: cell list, cutoff brute force and the full matrix."""
    n, L, steps = 1000, 1000.0, 100
    x = synth.uniform_positions(n, L, seed=0)
    A, B = synth.uniform_masses(n, seed=0)
    sim = make(n, L, search=search, observe_cap=steps)
    X, a, b = run_both(sim, x, A, B, steps, check_every=(search != mt.MT_SEARCH_FULL))
    obs = sim.observables()
    assert obs.shape == (steps, 4)
    o = O.observables(a, b)
    np.testing.assert_allclose(obs[-1], o, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("search", [mt.MT_SEARCH_CELL, mt.MT_SEARCH_BRUTE, mt.MT_SEARCH_FULL])
@pytest.mark.parametrize("precision", [mt.MT_MIXED, mt.MT_MIXED_DF32])
def test_1d_n1000_100_steps_mixed(search, precision):
    n, L, steps = 1000, 1000.0, 100
    x = synth.uniform_positions(n, L, seed=0)
    A, B = synth.uniform_masses(n, seed=0)
    sim = make(n, L, search=search, precision=precision, observe_cap=steps)
    run_both(sim, x, A, B, steps, check_every=False)


# ------------------------------------------------------------ edge cases --

@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 255, 256, 257, 4099])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_sizes_and_ragged_tails(n, precision):
    L = max(4.0, n * 0.8)
    x = synth.uniform_positions(n, L, seed=n)
    A, B = synth.uniform_masses(n, seed=n)
    for search in (mt.MT_SEARCH_CELL, mt.MT_SEARCH_BRUTE):
        sim = make(n, L, search=search, precision=precision)
        run_both(sim, x, A, B, 4, seed=n)


def test_empty_state():
    sim = make(0, 100.0, observe_cap=4)
    sim.upload(np.zeros((1, 0)), np.zeros(0), np.zeros(0))
    sim.step(3)
    sim.sync()
    A, B = sim.masses()
    assert A.shape == (0,) and sim.steps_done() == 3


@pytest.mark.parametrize("search", [mt.MT_SEARCH_CELL, mt.MT_SEARCH_BRUTE])
def test_exact_cutoff_walls_and_coincident(search):
    """Pairs exactly s_max apart (in), one tick more (out), particles on both
    walls, coincident particles and particles on cell edges; no random walk so
    the geometry is kept."""
    sim = make(16, 50.0, search=search, D_rw=0.0, react=0)
    k = int(sim.params.frac_bits)
    S = int(np.floor(sim.params.cutoff * 2.0 ** k))
    c = 2 ** int(sim.params.cell_shift) if search == mt.MT_SEARCH_CELL else 2 ** (k + 2)
    Lq = int(50.0 * 2 ** k)
    ticks = [0, S, 2 * S + 1, 3 * S + 1, 3 * S + 1, 3 * S + 1, Lq - S, Lq, Lq,
             5 * c, 5 * c - 1, 5 * c + S, 7 * c - S - 1, 7 * c, 9 * c + 3, 9 * c + 3 + S]
    x = np.array(ticks, dtype=np.float64) * 2.0 ** -k
    assert np.array_equal(O.quantize(x, k), np.array(ticks))
    A, B = synth.uniform_masses(16, seed=5)
    run_both(sim, x.reshape(1, -1), A, B, 3)


@pytest.mark.parametrize("cluster", [40, 3000])
def test_large_cells(cluster):
    """A coincident cluster larger than the per-thread cell sort (40) and
    larger than the shared-memory sort (3000) goes through the large-cell
    paths and still gives the oracle's result."""
    n = 5000
    x = synth.uniform_positions(n, 2000.0, seed=9)
    x[0, :cluster] = 1000.0
    A, B = synth.uniform_masses(n, seed=9)
    sim = make(n, 2000.0, D_rw=0.0)
    run_both(sim, x, A, B, 2, pairs=(cluster < 1000))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_segments_beyond_the_pair_list(precision):
    """Segments of 900 particles at density 1.25 stage about 920 particles
    (within the staging) but list about 2150 pairs, beyond the first tier's
    pair list (2048): they go to the cluster tier; every step still equals
    the oracle, and the pair set is exact."""
    n, L = 75000, 60000.0
    x = synth.uniform_positions(n, L, seed=13)
    A, B = synth.uniform_masses(n, seed=13)
    p = mt.mt_params_init(n=n, L=(L,), v=(0.3,), precision=precision, seg_target=900, seed=1)
    sim = mt.Simulation(p)
    run_both(sim, x, A, B, 3, seed=13)
    mt.mt_set_profiling(sim.h, True)
    sim.step()
    names = [k for k, _ in mt.mt_read_profile(sim.h)]
    assert "fused_step" in names and "fused_big" in names and "move" not in names


# ------------------------------------------------------------------ 2-d --

@pytest.mark.parametrize("search", [mt.MT_SEARCH_CELL, mt.MT_SEARCH_BRUTE, mt.MT_SEARCH_FULL])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_2d(search, precision):
    n, L = 1500, (60.0, 40.0)
    x = synth.uniform_positions(n, L, dim=2, seed=3)
    A, B = synth.uniform_masses(n, seed=3)
    sim = make(n, L, dim=2, search=search, precision=precision, v=(0.3, -0.2))
    run_both(sim, x, A, B, 6, check_every=False)


# ---------------------------------------------------------- normalisation --

@pytest.mark.parametrize("precision", PRECISIONS)
def test_row_normalisation(precision):
    n, L = 2000, 1000.0
    x = synth.uniform_positions(n, L, seed=4)
    A, B = synth.uniform_masses(n, seed=4)
    sim = make(n, L, norm=mt.MT_NORM_ROW, precision=precision)
    run_both(sim, x, A, B, 10, check_every=False)


def test_no_reaction_and_advection():
    n, L = 3000, 1500.0
    x = synth.uniform_positions(n, L, seed=6)
    A, B = synth.uniform_masses(n, seed=6)
    sim = make(n, L, react=0, v=(0.5, 0.0))
    run_both(sim, x, A, B, 20, check_every=False)


# ---------------------------------------------------------- determinism --

@pytest.mark.parametrize("precision", PRECISIONS)
def test_bitwise_deterministic(precision):
    n, L = 20000, 20000.0
    x = synth.uniform_positions(n, L, seed=11)
    A, B = synth.uniform_masses(n, seed=11)
    outs = []
    for _ in range(2):
        sim = make(n, L, precision=precision, seed=123, v=(0.5, 0.0))
        sim.upload(x, A, B)
        sim.run(30)
        outs.append((sim.ticks(), *sim.masses()))
        sim.close()
    for u, w in zip(*outs):
        assert np.array_equal(u, w)


def test_observables_bitwise_deterministic_on_a_large_system():
    """More than one wave of segments (the first tier takes them by ticket)
    and the predicted-segment kernel beside it: two runs give the same
    observables bit for bit, and equal to the sums of the masses read back."""
    n, L = 400000, 4.0e5
    x = synth.uniform_positions(n, L, seed=12)
    x[0, :4000] = np.random.default_rng(12).uniform(0.0, 4.0, 4000)
    A, B = synth.uniform_masses(n, seed=12)
    outs = []
    for _ in range(2):
        sim = make(n, L, precision=mt.MT_MIXED, seed=5, v=(0.5, 0.0), observe_cap=40)
        assert sim.params.seg_target > 0
        sim.upload(x, A, B)
        sim.run(30)
        outs.append((sim.observables(), *sim.masses()))
        sim.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    a, b = outs[0][1], outs[0][2]
    np.testing.assert_allclose(outs[0][0][-1], O.observables(a, b), rtol=1e-12, atol=1e-8)


def test_run_graph_equals_step_loop():
    n, L = 5000, 5000.0
    x = synth.uniform_positions(n, L, seed=12)
    A, B = synth.uniform_masses(n, seed=12)
    res = []
    for use_run in (True, False):
        sim = make(n, L, precision=mt.MT_MIXED, seed=5, observe_cap=16)
        sim.upload(x, A, B)
        if use_run:
            sim.run(16)
        else:
            sim.step(16)
        res.append((sim.ticks(), *sim.masses(), sim.observables()))
    for u, w in zip(*res):
        assert np.array_equal(u, w)


# ------------------------------------------------------------- generator --

def test_philox_known_answers_and_reference():
    from tests.philox_ref import load_kat, philox4x32_10
    import torch

    sim = make(10, 100.0)
    out = torch.zeros(4 * 64, dtype=torch.int32, device="cuda")
    for ctr, key, exp in load_kat():
        mt.mt_philox(sim.h, ctr, key, 1, out.data_ptr())
        sim.sync()
        got = tuple(int(v) & 0xFFFFFFFF for v in out[:4].cpu().tolist())
        assert got == exp
    ctr = (7, 123456, 0, 42)
    key = (0xDEADBEEF, 0x01234567)
    mt.mt_philox(sim.h, ctr, key, 64, out.data_ptr())
    sim.sync()
    got = [int(v) & 0xFFFFFFFF for v in out.cpu().tolist()]
    for i in range(64):
        assert tuple(got[4 * i:4 * i + 4]) == philox4x32_10(((ctr[0] + i) & 0xFFFFFFFF, *ctr[1:]), key)


@pytest.mark.parametrize("dim", [1, 2])
def test_builtin_noise_statistics(dim):
    """Built-in Philox / Box-Muller walk: displacement mean v dt and
    variance 2 D_rw dt per axis, uncorrelated axes."""
    n, L = 10 ** 6, 1e7
    sim = make(n, (L, L) if dim == 2 else L, dim=dim, v=(0.5, -0.25), seed=77,
               search=mt.MT_SEARCH_CELL, precision=mt.MT_MIXED, react=0)
    x = L / 2 + synth.uniform_positions(n, 2000.0, dim=dim, seed=1) - 1000.0
    A, B = synth.uniform_masses(n, seed=1)
    sim.upload(x, A, B)
    x0 = sim.positions()
    sim.run(1)
    d = sim.positions() - x0
    for ax, v in zip(range(dim), (0.5, -0.25)):
        assert abs(d[ax].mean() - v) < 5 * np.sqrt(0.2 / n)
        assert abs(d[ax].var() - 0.2) < 5 * 0.2 * np.sqrt(2 / n)
        kurt = ((d[ax] - d[ax].mean()) ** 4).mean() / d[ax].var() ** 2
        assert abs(kurt - 3.0) < 0.05
    if dim == 2:
        assert abs(np.corrcoef(d[0], d[1])[0, 1]) < 5 / np.sqrt(n)


# ------------------------------------------------------- full-size checks --

@pytest.mark.parametrize("precision", [mt.MT_MIXED, mt.MT_FP64])
@pytest.mark.parametrize("before", [20, 1000])
def test_full_size_step_after_graph_run(precision, before):
    """N = 1e6 on [0, 1e6], v = 0.5, in the benchmark's launch configuration
    (CUDA graph, built-in generator) for 20 or 1000 steps (by then the drift
    has piled ~500 particles against the wall at x = L, a pair-heavy layer
    the cluster kernel takes beside the first tier); then one injected-noise
    step from the read-back state, compared with the oracle element by
    element (sorted-window search)."""
    n, L = 10 ** 6, 1e6
    sim = make(n, L, v=(0.5, 0.0), precision=precision, seed=3, observe_cap=64)
    x = synth.uniform_positions(n, L, seed=2)
    A, B = synth.uniform_masses(n, seed=2)
    sim.upload(x, A, B)
    sim.run(before)
    X0 = sim.ticks()
    a0, b0 = sim.masses()
    assert X0.min() >= 0 and X0.max() <= int(L * 2 ** int(sim.params.frac_bits))
    xi = synth.normals(1, 1, n, seed=99)[0]
    sim.set_noise(xi)
    sim.step()
    X1, a1, b1 = O.step(oracle_params(sim), X0, xi, a0, b0)
    assert np.array_equal(sim.ticks(), X1)
    ga, gb = sim.masses()
    assert_masses(ga, a1, TOL[precision], "A")
    assert_masses(gb, b1, TOL[precision], "B")
    obs = sim.observables()
    assert obs.shape[0] == min(before + 1, 64)
    np.testing.assert_allclose(obs[-1], O.observables(ga, gb), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("precision", [mt.MT_FP64, mt.MT_MIXED])
def test_invariants_at_scale(precision):
    """Symmetric normalisation conserves each species' total; the reaction
    conserves sum(A - B) and leaves min(A, B) = 0; positions stay in [0, L]."""
    n, L = 10 ** 6, 1e6
    x = synth.uniform_positions(n, L, seed=21)
    A, B = synth.uniform_masses(n, seed=21)
    for react in (0, 1):
        sim = make(n, L, precision=precision, react=react, seed=8, observe_cap=50)
        sim.upload(x, A, B)
        sim.run(50)
        a, b = sim.masses()
        obs = sim.observables()
        if react == 0:
            assert abs(a.sum() - A.sum()) <= 1e-11 * A.sum()
            assert abs(b.sum() - B.sum()) <= 1e-11 * B.sum()
            np.testing.assert_allclose(obs[:, 0], A.sum(), rtol=1e-11)
        else:
            assert abs((a - b).sum() - (A - B).sum()) <= 1e-11 * np.abs(A - B).sum()
            assert np.all(np.minimum(a, b) == 0.0)
            # sum(A - B) is a small difference of two ~5e5 totals: bound its
            # drift relative to the total mass
            np.testing.assert_allclose(obs[:, 2], (A - B).sum(), rtol=0,
                                       atol=1e-11 * (A.sum() + B.sum()))
        X = sim.ticks()
        assert X.min() >= 0 and X.max() <= int(L * 2 ** int(sim.params.frac_bits))


# -------------------------------------------------------- API behaviour --

def test_device_pointer_io_matches_host_io():
    import torch

    n, L = 4000, 4000.0
    x = synth.uniform_positions(n, L, seed=31)
    A, B = synth.uniform_masses(n, seed=31)
    sim = make(n, L, precision=mt.MT_MIXED, seed=4)
    xd = torch.tensor(x, device="cuda").contiguous()
    Ad = torch.tensor(A, device="cuda")
    Bd = torch.tensor(B, device="cuda")
    torch.cuda.synchronize()
    mt.mt_upload(sim.h, xd.data_ptr(), Ad.data_ptr(), Bd.data_ptr(), mt.MT_MEM_DEVICE)
    sim.run(5)
    oA = torch.empty(n, dtype=torch.float64, device="cuda")
    oB = torch.empty(n, dtype=torch.float64, device="cuda")
    mt.mt_read_masses(sim.h, oA.data_ptr(), oB.data_ptr(), mt.MT_MEM_DEVICE)
    ha, hb = sim.masses()
    assert np.array_equal(oA.cpu().numpy(), ha) and np.array_equal(oB.cpu().numpy(), hb)


def test_step_before_upload_and_bad_positions():
    sim = make(10, 10.0)
    with pytest.raises(mt.MtError) as e:
        sim.step()
    assert e.value.status == mt.MT_ERR_STATE
    x = np.linspace(0, 12.0, 10).reshape(1, -1)  # beyond L = 10
    with pytest.raises(mt.MtError) as e:
        sim.upload(x, np.ones(10), np.ones(10))
        sim.sync()
    assert e.value.status == mt.MT_ERR_INVALID


def test_profiling_events_in_graph_and_direct_steps():
    n, L = 100000, 100000.0
    x = synth.uniform_positions(n, L, seed=41)
    A, B = synth.uniform_masses(n, seed=41)
    sim = make(n, L, precision=mt.MT_MIXED)
    sim.upload(x, A, B)
    mt.mt_set_profiling(sim.h, True)
    for runner in (lambda: sim.run(3), lambda: sim.step(1)):
        runner()
        prof = mt.mt_read_profile(sim.h)
        names = [k for k, _ in prof]
        assert names == ["fused_step"]  # one kernel per step, no fallback
        assert all(ms > 0 for _, ms in prof)
    mt.mt_set_profiling(sim.h, False)
    sim.run(2)
    sim.sync()
    # 2-d and brute force keep the multi-kernel pipeline
    sim2 = make(1000, (50.0, 50.0), dim=2)
    sim2.upload(synth.uniform_positions(1000, (50.0, 50.0), dim=2, seed=1), *synth.uniform_masses(1000))
    mt.mt_set_profiling(sim2.h, True)
    sim2.step()
    names = [k for k, _ in mt.mt_read_profile(sim2.h)]
    assert names[0] == "move" and names[-1] == "exchange_cell2"


@pytest.mark.parametrize("cluster,tiers", [
    (1500, ["fused_step", "fused_big"]),
    (5000, ["fused_step", "fused_big", "move"]),
])
def test_fused_tiers_on_clustered_segments(cluster, tiers):
    """A segment whose staged particles exceed the first tier's shared memory
    goes to the second tier; one that exceeds the second tier too makes the
    step fall back to the general pipeline (visible in the kernel list).
    Results match the oracle either way."""
    n = 9000
    x = synth.uniform_positions(n, 9000.0, seed=13)
    x[0, :cluster] = 4500.0 + synth.uniform_positions(cluster, 1.0, seed=14)[0]
    A, B = synth.uniform_masses(n, seed=13)
    sim = make(n, 9000.0)
    run_both(sim, x, A, B, 2, pairs=False)
    mt.mt_set_profiling(sim.h, True)
    sim.step()
    names = [k for k, _ in mt.mt_read_profile(sim.h)]
    # the heavy segment goes to a cluster kernel: the predicted-segment
    # kernel (it was heavy last step) or the second tier (newly heavy)
    assert "fused_step" in names
    assert ("fused_pred" in names) or ("fused_big" in names)
    if "move" in tiers:
        assert names[-1] == "fused_prep"
    else:
        assert "move" not in names


def test_fused_segments_many_steps_with_drift_and_walls():
    """Long run on the fused path with advection against a reflecting wall
    (density piles up near x = L), checked against the oracle every 25
    steps; exercises the segment boundaries that each step hands to the
    next."""
    n, L = 20000, 20000.0
    x = synth.uniform_positions(n, L, seed=17)
    A, B = synth.uniform_masses(n, seed=17)
    sim = make(n, L, v=(3.0, 0.0), D_rw=0.5, precision=mt.MT_MIXED)
    po = oracle_params(sim)
    k = int(sim.params.frac_bits)
    sim.upload(x, A, B)
    X = O.quantize(x, k)
    a, b = A.copy(), B.copy()
    xi = synth.normals(100, 1, n, seed=18)
    for s in range(100):
        sim.set_noise(xi[s])
        sim.step()
        X, a, b = O.step(po, X, xi[s], a, b)
        if s % 25 == 24:
            assert np.array_equal(sim.ticks(), X)
            ga, gb = sim.masses()
            assert_masses(ga, a, TOL[mt.MT_MIXED], f"A step {s}")
            assert_masses(gb, b, TOL[mt.MT_MIXED], f"B step {s}")


@pytest.mark.parametrize("cluster,tiers", [(40, ["fused_step"]), (300, ["fused_step", "fused_big"])])
def test_fused_dense_bins_sorted_in_place(cluster, tiers):
    """A cluster denser than a cell (particles piled up like at a wall) is
    sorted in place by the whole CTA; a small one (40 particles, 780 pairs:
    within the first tier's pair list) stays in the first tier, a pair-heavy
    one (O(n^2) work) goes to the second tier, whose exchange is split
    across several CTAs.  Results match the oracle."""
    n = 5000
    x = synth.uniform_positions(n, 5000.0, seed=23)
    x[0, :cluster] = 2500.0 + synth.uniform_positions(cluster, 1.0, seed=24)[0]
    A, B = synth.uniform_masses(n, seed=23)
    sim = make(n, 5000.0, D_rw=0.01)
    run_both(sim, x, A, B, 3, pairs=True)
    mt.mt_set_profiling(sim.h, True)
    sim.step()
    names = [k for k, _ in mt.mt_read_profile(sim.h)]
    if tiers == ["fused_step"]:
        assert names == ["fused_step"]
    else:  # a cluster kernel took the pair-heavy segment
        assert "fused_step" in names and ("fused_pred" in names or "fused_big" in names)
        assert "move" not in names


@pytest.mark.parametrize("precision", PRECISIONS)
def test_workload2_n1e5_1000_steps_oracle_on_strided_steps(precision):
    """N = 1e5 uniform on [0, 1e5], no advection, 1000 steps on the built-in
    generator; every 100th step is taken from the GPU's own state with
    injected noise on both sides and checked against one oracle step from
    that identical state (positions bit for bit, masses to the tolerance)."""
    n, L = 100000, 1e5
    x = synth.uniform_positions(n, L, seed=0)
    A, B = synth.uniform_masses(n, seed=0)
    sim = make(n, L, precision=precision, observe_cap=1000)
    po = oracle_params(sim)
    sim.upload(x, A, B)
    tol = TOL[precision]
    for block in range(10):
        sim.run(99)
        X = sim.ticks()
        a, b = sim.masses()
        xi = synth.normals(1, 1, n, seed=700 + block)[0]
        sim.set_noise(xi)
        sim.step()
        sim.set_noise(None)
        Xo, ao, bo = O.step(po, X, xi, a, b)
        assert np.array_equal(sim.ticks(), Xo), f"positions at step {100 * block + 99}"
        ga, gb = sim.masses()
        assert_masses(ga, ao, tol, f"A at step {100 * block + 99}")
        assert_masses(gb, bo, tol, f"B at step {100 * block + 99}")
    assert sim.steps_done() == 1000
    obs = sim.observables()
    assert obs.shape == (1000, 4)
    np.testing.assert_allclose(obs[-1, 2], np.sum(A - B), rtol=0, atol=1e-10 * np.sum(A + B))


def test_async_observables_copy_matches_synchronous_read():
    """Rows copied behind each step into page-locked host memory (no wait
    between steps) equal the synchronous read; several rows across the
    ring's wrap; bad row counts refused."""
    import torch

    n, L = 5000, 5000.0
    sim = make(n, L, precision=mt.MT_MIXED, seed=4, observe_cap=5)
    sim.upload(synth.uniform_positions(n, L, seed=4), *synth.uniform_masses(n, seed=4))
    rows = torch.zeros((12, 4), dtype=torch.float64).pin_memory().numpy()
    for s in range(12):
        sim.run(1)
        mt.mt_copy_observables_async(sim.h, rows[s:].ctypes.data_as(ctypes.c_void_p), 1)
    sim.sync()
    assert np.array_equal(rows[-5:], sim.observables())
    wrap = np.zeros((4, 4))
    sim.run(3)  # the ring's newest row is now at index 0 again after a wrap
    mt.mt_copy_observables_async(sim.h, wrap.ctypes.data_as(ctypes.c_void_p), 4)
    sim.sync()
    assert np.array_equal(wrap, sim.observables()[-4:])
    for bad in (0, 6):
        with pytest.raises(mt.MtError):
            mt.mt_copy_observables_async(sim.h, wrap.ctypes.data_as(ctypes.c_void_p), bad)
    sim.close()
