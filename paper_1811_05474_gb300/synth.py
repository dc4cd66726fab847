"""Seeded synthetic inputs for the mass-transfer particle-tracking step.

The paper's test problems use uniform random particle positions on a bounded
domain and per-particle species masses (Sec. 3); every workload here is
synthetic in that shape.  This module only draws random numbers with numpy:
it holds none of the method's arithmetic, so the oracle, the CUDA path's tests
and the benchmark can all take their inputs from it.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Independent generator per (seed, stream)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, stream])))


def uniform_positions(n: int, L, dim: int = 1, seed: int = 0) -> np.ndarray:
    """(dim, n) float64 positions, i.i.d. uniform on [0, L_d] per axis."""
    Ls = [float(v) for v in np.atleast_1d(np.asarray(L, dtype=np.float64))]
    Ls = Ls + [Ls[-1]] * (2 - len(Ls))
    g = rng(seed, 1)
    return np.stack([g.uniform(0.0, Ls[d], size=n) for d in range(dim)]).astype(np.float64)


def uniform_masses(n: int, seed: int = 0):
    """A, B masses i.i.d. uniform on [0, 1)."""
    g = rng(seed, 2)
    return g.uniform(0.0, 1.0, size=n), g.uniform(0.0, 1.0, size=n)


def segregated_masses(x: np.ndarray, L: float):
    """Unit A on the left half, unit B on the right half (Sec. 3 initial state)."""
    x0 = np.asarray(x)[0] if np.ndim(x) == 2 else np.asarray(x)
    A = (x0 < 0.5 * L).astype(np.float64)
    return A, 1.0 - A


def normals(steps: int, dim: int, n: int, seed: int = 0) -> np.ndarray:
    """(steps, dim, n) float32 standard normals for injected random-walk noise."""
    g = rng(seed, 3)
    return g.standard_normal(size=(steps, dim, n), dtype=np.float32)


def ensemble_sizes(count: int = 256, lo: float = 1e3, hi: float = 1e5, seed0: int = 0) -> np.ndarray:
    """Realisation r draws N_r = floor(10^U(log10 lo, log10 hi)) from seed seed0 + r."""
    out = np.empty(count, dtype=np.int64)
    for r in range(count):
        u = rng(seed0 + r, 4).uniform(np.log10(lo), np.log10(hi))
        out[r] = int(np.floor(10.0 ** u))
    return out


def poisson_requests(count: int, rate: float = 200.0, seed: int = 0,
                     n_lo: float = 1e3, n_hi: float = 1e6, steps_lo: int = 100,
                     steps_hi: int = 1000):
    """Simulation requests arriving as a Poisson process of the given rate.

    Each request: arrival time (s), particle count N log-uniform in
    [n_lo, n_hi], dimension 1 or 2 with equal probability, a step count uniform
    in [steps_lo, steps_hi], and its own seed.  2-d requests live on the square
    [0, sqrt(N) * 10]^2 and 1-d ones on [0, N]."""
    g = rng(seed, 5)
    t = np.cumsum(g.exponential(1.0 / rate, size=count))
    n = np.floor(10.0 ** g.uniform(np.log10(n_lo), np.log10(n_hi), size=count)).astype(np.int64)
    dim = g.integers(1, 3, size=count)
    steps = g.integers(steps_lo, steps_hi + 1, size=count)
    reqs = []
    for i in range(count):
        L = float(np.sqrt(n[i]) * 10.0) if dim[i] == 2 else float(n[i])
        reqs.append(dict(t=float(t[i]), n=int(n[i]), dim=int(dim[i]), L=L,
                         steps=int(steps[i]), seed=int(seed * 100003 + i)))
    return reqs
