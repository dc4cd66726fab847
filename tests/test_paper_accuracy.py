"""The oracle on the paper's accuracy test problem (Sec. 3): the C1 profile
after t = 10 against the exact solution of the diffusion equation.

Pins the whole step -- move, transfer with the D split, walls -- against a
closed form: the profile's fitted diffusion coefficient is D = 1 less the
scheme's known damping (the self weight in r_i and the 3-sigma cutoff take
a few per cent off the transfer's half), and a wrong split is far outside
the band (doubling D_mt gives about 1.25, doubling D_rw about 1.45, halving
D_mt about 0.7).  Symmetric normalisation conserves C1; row normalisation
(the literal Sec. 1.1 form) does not.
"""
import numpy as np
import pytest

import oracle as O
from paper_1811_05474_gb300 import accuracy as acc
from paper_1811_05474_gb300 import synth


def run(n, seed, norm=O.NORM_SYM, **over):
    kw = dict(acc.params_kw())
    kw.update(over)
    p = O.params(frac_bits=29, norm=norm, **kw)
    x, c1, c2 = acc.inputs(n, seed)
    X = O.quantize(x, 29)
    xi = synth.normals(acc.STEPS, 1, n, seed=seed + 1)
    for s in range(acc.STEPS):
        X, c1, c2 = O.step(p, X, xi[s], c1, c2)
    return O.dequantize(X, 29)[0], c1, c2


@pytest.fixture(scope="module")
def sym500():
    return [run(500, s) for s in range(8)]


def test_profile_matches_the_exact_solution(sym500):
    xs = [r[0] for r in sym500]
    cs = [r[1] for r in sym500]
    assert 0.85 <= acc.fitted_d(xs, cs) <= 1.02
    e = [acc.rmse(x, c) for x, c in zip(xs, cs)]
    assert np.mean(e) < 0.035
    # the initial step is far from the exact profile at t = 10
    x0, c10, _ = acc.inputs(500, 0)
    assert acc.rmse(x0[0], c10) > 0.1


def test_rmse_falls_with_particle_count(sym500):
    e500 = np.mean([acc.rmse(x, c) for x, c, _ in sym500])
    e1500 = np.mean([acc.rmse(x, c) for x, c, _ in (run(1500, s) for s in range(4))])
    assert e1500 < e500


def test_wrong_diffusion_split_is_detected():
    runs = [run(500, s, D_mt=1.0) for s in range(4)]
    assert acc.fitted_d([r[0] for r in runs], [r[1] for r in runs]) > 1.1


def test_symmetric_normalisation_conserves_row_does_not(sym500):
    for s, (x, c1, c2) in enumerate(sym500[:4]):
        _, c10, c20 = acc.inputs(500, s)
        assert abs(c1.sum() - c10.sum()) <= 1e-11 * c10.size
        assert abs(c2.sum() - c20.sum()) <= 1e-11 * c20.size
    x, c1, _ = run(500, 0, norm=O.NORM_ROW)
    _, c10, _ = acc.inputs(500, 0)
    assert abs(c1.sum() - c10.sum()) > 1e-3


def test_narrower_pad_damps_more_and_full_matrix_agrees(sym500):
    """Sec. 5's observations with the same inputs and walks: a 2-sigma cutoff
    truncates more of Eq. 3's kernel than 3 sigma and damps the transfer
    visibly (fitted D well below), while the full matrix (no cutoff) gives
    the 3-sigma result within a few per cent."""
    sig = np.sqrt(4 * 0.5 * acc.DT)
    d3 = acc.fitted_d([r[0] for r in sym500], [r[1] for r in sym500])
    two = [run(500, s, smax=2 * sig) for s in range(8)]
    full = [run(500, s, search=O.SEARCH_FULL) for s in range(8)]
    d2 = acc.fitted_d([r[0] for r in two], [r[1] for r in two])
    dfull = acc.fitted_d([r[0] for r in full], [r[1] for r in full])
    assert d2 < d3 - 0.05
    assert abs(dfull - d3) < 0.03
    e3 = np.mean([acc.rmse(x, c) for x, c, _ in sym500])
    e2 = np.mean([acc.rmse(x, c) for x, c, _ in two])
    efull = np.mean([acc.rmse(x, c) for x, c, _ in full])
    assert e2 > e3
    assert abs(efull - e3) < 0.1 * e3
