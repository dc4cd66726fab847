"""The paper's accuracy test problem (Sec. 3) and its error metrics.

1-d domain [0, 50] with reflecting walls, D = 1 applied half by the mass
transfer and half by the random walk (D_mt = D_rw = 1/2), dt = 0.1 up to
t = 10 (100 steps), positions uniform, and a segregated initial state: the
conservative component C1 = A + E is 1 on the left half and 0 on the right,
C2 = B + E the opposite.  Both diffuse without reacting (E = min(C1, C2) at
any time), so the simulation transfers C1 and C2 with the reaction off.

The error is measured against the solution of the diffusion equation from a
step at x0 = L/2 (boundary effects are negligible at t = 10): C1(x, t) =
erfc((x - x0) / sqrt(4 D t)) / 2, at the particles' final positions.  The
printed formula in Sec. 3 squares the argument and drops the root; this is
the standard solution it stands for.

These are evaluation helpers (inputs and metrics), not part of the step.
"""
from __future__ import annotations

import numpy as np

from . import synth

L = 50.0
D = 1.0
DT = 0.1
T_END = 10.0
STEPS = 100
X0 = 0.5 * L
SIZES = (500, 1000, 2500, 5000, 10000, 25000)  # particle counts of Sec. 3
REALISATIONS = 75


def params_kw() -> dict:
    """Keyword arguments for mt_params_init / the oracle's params."""
    return dict(L=(L,), D_mt=0.5 * D, D_rw=0.5 * D, dt=DT, react=0)


def inputs(n: int, seed: int):
    """Positions (1, n) uniform on [0, L] and the segregated C1, C2."""
    x = synth.uniform_positions(n, L, seed=seed)
    c1, c2 = synth.segregated_masses(x, L)
    return x, c1, c2


def c1_exact(x, t: float = T_END, d: float = D):
    from scipy.special import erfc

    return 0.5 * erfc((np.asarray(x) - X0) / np.sqrt(4.0 * d * t))


def rmse(x, c1, t: float = T_END) -> float:
    """Root-mean-square error of C1 at the particles against c1_exact."""
    return float(np.sqrt(np.mean((np.asarray(c1) - c1_exact(x, t)) ** 2)))


def fitted_d(xs, cs, t: float = T_END) -> float:
    """The diffusion coefficient whose exact profile fits the pooled
    particles (x, C1) best in least squares."""
    from scipy.optimize import minimize_scalar

    x = np.concatenate([np.ravel(v) for v in xs])
    c = np.concatenate([np.ravel(v) for v in cs])
    f = lambda d: float(np.sum((c - c1_exact(x, t, d)) ** 2))
    return float(minimize_scalar(f, bounds=(0.05, 10.0), method="bounded").x)
