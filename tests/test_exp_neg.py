"""The binary64 exp(-t) of the MT_FP64 weights (Eq. 3; Tang's table-driven
method, csrc/mt_pair.cuh): its constants are the correctly rounded
mathematical values (checked against 200-bit evaluations), and the recipe,
replayed operation by operation with exact rounding (tests/exp_neg_replay.py),
stays within 1.1 units in the last place of the exact exponential over the
weights' range and beyond.  The GPU test compares the kernel with the
replay bit for bit."""
import math
from fractions import Fraction

import numpy as np
import pytest

from .exp_neg_replay import consts as _consts, replay

mp = pytest.importorskip("mpmath")


@pytest.fixture(scope="module")
def consts():
    mp.mp.prec = 200
    return _consts()

def test_constants_are_the_rounded_mathematical_values(consts):
    tab, c = consts
    assert len(tab) == 32
    for j, v in enumerate(tab):
        assert v == float(mp.power(2, mp.mpf(j) / 32)), j
    ln2_32 = mp.log(2) / 32
    assert c["inv"] == float(1 / ln2_32)
    # the head has at most 37 significant bits (k * head exact for |k| < 2^16)
    m, e = math.frexp(c["head"])
    assert (Fraction(m) * 2 ** 37).denominator == 1
    # the tail is the rest rounded once: within half its last place
    assert abs(mp.mpf(c["head"]) + mp.mpf(c["tail"]) - ln2_32) <= mp.mpf(math.ulp(c["tail"])) / 2
    for k, key in ((6, "c6"), (5, "c5"), (4, "c4"), (3, "c3")):
        assert c[key] == float(1 / mp.factorial(k)), key


def _ulps(got: float, t: float) -> float:
    exact = mp.exp(-mp.mpf(t))
    return float(abs(mp.mpf(got) - exact) / mp.mpf(math.ulp(float(exact))))


def test_replay_within_about_one_ulp(consts):
    tab, c = consts
    rng = np.random.default_rng(7)
    ts = np.concatenate([rng.uniform(0.0, 5.0, 1500), rng.uniform(0.0, 40.0, 500),
                         rng.uniform(40.0, 700.0, 200), [0.0, 1e-300, 2.0 ** -60, 1e-8, 0.5,
                                                         math.log(2) / 64, 4.5, 18.0, 700.0]])
    worst = max(_ulps(replay(float(t), tab, c), float(t)) for t in ts)
    assert worst <= 1.1, worst


def test_replay_edges(consts):
    tab, c = consts
    assert replay(0.0, tab, c) == 1.0
    assert replay(746.0, tab, c) == 0.0
    assert replay(math.inf, tab, c) == 0.0
    assert math.isnan(replay(math.nan, tab, c))
    # the subnormal range: within a few subnormal steps of the exact value
    for t in (709.0, 720.0, 740.0):
        exact = float(mp.exp(-mp.mpf(t)))
        assert abs(replay(t, tab, c) - exact) <= 4 * 5e-324 + 2 * math.ulp(exact)
