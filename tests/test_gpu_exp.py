"""The weights' binary64 exp(-t) on the GPU (mt_test_exp_neg) equals the
operation-by-operation replay of its recipe (tests/exp_neg_replay.py) bit
for bit, over the weights' range, beyond it, and at the edges."""
import math

import numpy as np
import pytest

from paper_1811_05474_gb300 import mt

from .exp_neg_replay import consts, replay

pytestmark = pytest.mark.gpu


def test_exp_neg_equals_its_replay_bit_for_bit():
    import torch

    rng = np.random.default_rng(11)
    t = np.concatenate([rng.uniform(0.0, 5.0, 3000), rng.uniform(0.0, 60.0, 1000),
                        rng.uniform(60.0, 745.0, 500),
                        [0.0, 1e-300, 2.0 ** -60, 0.5, math.log(2) / 64, 4.5, 708.5, 720.0,
                         745.0, 746.0, 1e300, math.inf, math.nan]])
    dt = torch.tensor(t, dtype=torch.float64, device="cuda")
    out = torch.empty_like(dt)
    mt.mt_test_exp_neg(dt.data_ptr(), out.data_ptr(), dt.numel())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    tab, c = consts()
    want = np.array([replay(float(v), tab, c) for v in t])
    same = (got == want) | (np.isnan(got) & np.isnan(want))
    assert same.all(), (t[~same][:5], got[~same][:5], want[~same][:5])
    # and close to the library's exponential
    ok = np.isfinite(t) & (t < 700)
    rel = np.abs(got[ok] - np.exp(-t[ok])) / np.exp(-t[ok])
    assert rel.max() <= 4e-16
