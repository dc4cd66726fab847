"""CPU FP64 oracle for the mass-transfer particle-tracking step (arXiv 1811.05474).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain C code in ``mt_oracle.c``
(declared in ``mt_oracle.h``); this module compiles it with gcc and wraps it
with ctypes.  Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it.  It shares no code with the CUDA library and
never imports the product package.

Which passage each function follows is stated in ``mt_oracle.h``: Eq. 2 (move,
Sec. 3 walls), Eq. 3 (weights), the row normalisation of Sec. 1.1 and its
symmetric part, Eq. 4 and Eq. 7 (exchange), Eq. 5-6 (matrix form, sign as in
Eq. 4), the A + B -> E reaction of Sec. 3 and Sec. 7, and the fixed-radius
search of Sec. 2.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "mt_oracle.c"
HDR = HERE / "mt_oracle.h"
BUILD_DIR = HERE / "_build"
LIB = BUILD_DIR / "libmt_oracle.so"

SEARCH_CUTOFF = 0
SEARCH_FULL = 2
NORM_SYM = 0
NORM_ROW = 1
WALLS_REFLECT = 0
WALLS_PERIODIC = 1


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("frac_bits", ctypes.c_int32),
        ("L", ctypes.c_double * 2),
        ("v", ctypes.c_double * 2),
        ("D_mt", ctypes.c_double),
        ("D_rw", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("smax", ctypes.c_double),
        ("search", ctypes.c_int32),
        ("norm", ctypes.c_int32),
        ("react", ctypes.c_int32),
        ("walls", ctypes.c_int32),
    ]


def params(*, dim=1, frac_bits=29, L=(1000.0, 0.0), v=(0.0, 0.0), D_mt=0.1,
           D_rw=0.1, dt=1.0, smax=None, search=SEARCH_CUTOFF, norm=NORM_SYM,
           react=1, walls=0) -> Params:
    """Problem parameters.  ``smax`` defaults to three standard deviations of
    Eq. 3's Gaussian, 3 * sqrt(4 D_mt dt).  ``walls``: WALLS_REFLECT (Sec. 3)
    or WALLS_PERIODIC (a wrapping domain, minimum-image separations)."""
    if smax is None:
        smax = 3.0 * np.sqrt(4.0 * D_mt * dt)
    Lv = list(L) + [0.0] * (2 - len(L))
    vv = list(v) + [0.0] * (2 - len(v))
    return Params(dim, frac_bits, (ctypes.c_double * 2)(*Lv),
                  (ctypes.c_double * 2)(*vv), D_mt, D_rw, dt, float(smax),
                  search, norm, react, walls)


def build(force: bool = False) -> Path:
    """Compile the oracle into a shared library (gcc, no FMA contraction)."""
    BUILD_DIR.mkdir(exist_ok=True)
    newer = LIB.exists() and LIB.stat().st_mtime >= max(SRC.stat().st_mtime,
                                                         HDR.stat().st_mtime)
    if newer and not force:
        return LIB
    tmp = BUILD_DIR / f"libmt_oracle.{os.getpid()}.so"
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-o", str(tmp), str(SRC), "-lm"]
    # OpenMP (for the all-cores baseline) where the compiler has it
    if subprocess.run(base + ["-fopenmp"], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None
_P = ctypes.POINTER


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build()))
        pp = _P(Params)
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        vp = ctypes.c_void_p
        L.mto_quantize.argtypes = [f64, i32]; L.mto_quantize.restype = i64
        L.mto_dequantize.argtypes = [i64, i32]; L.mto_dequantize.restype = f64
        L.mto_quantize_n.argtypes = [i64, vp, i32, vp]; L.mto_quantize_n.restype = None
        L.mto_dequantize_n.argtypes = [i64, vp, i32, vp]; L.mto_dequantize_n.restype = None
        L.mto_cutoff_ticks.argtypes = [pp]; L.mto_cutoff_ticks.restype = i64
        L.mto_move.argtypes = [pp, i64, vp, vp]; L.mto_move.restype = None
        L.mto_row_sums.argtypes = [pp, i64, vp, vp]; L.mto_row_sums.restype = None
        for name in ("mto_mass_transfer", "mto_mass_transfer_matrix",
                     "mto_mass_transfer_sorted_1d"):
            f = getattr(L, name)
            f.argtypes = [pp, i64, vp, i32, vp, vp]
            f.restype = ctypes.c_int
        L.mto_mass_transfer_sample.argtypes = [pp, i64, vp, i32, vp, i64, vp, vp]
        L.mto_mass_transfer_sample.restype = ctypes.c_int
        L.mto_react.argtypes = [i64, vp, vp]; L.mto_react.restype = None
        for name in ("mto_pairs_brute", "mto_pairs_sorted_1d"):
            f = getattr(L, name)
            f.argtypes = [pp, i64, vp, i64, vp, vp]
            f.restype = i64
        L.mto_step.argtypes = [pp, i64, vp, vp, vp, vp]; L.mto_step.restype = ctypes.c_int
        L.mto_observables.argtypes = [i64, vp, vp, vp]; L.mto_observables.restype = None
        L.mto_set_threads.argtypes = [i32]; L.mto_set_threads.restype = ctypes.c_int
        L.mto_set_threads(1)
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def quantize(x, k: int) -> np.ndarray:
    """Positions (dim, n) or (n,) as doubles -> int64 ticks."""
    x = _c(x, np.float64)
    X = np.empty(x.shape, dtype=np.int64)
    lib().mto_quantize_n(x.size, _ptr(x), k, _ptr(X))
    return X


def dequantize(X, k: int) -> np.ndarray:
    X = _c(X, np.int64)
    x = np.empty(X.shape, dtype=np.float64)
    lib().mto_dequantize_n(X.size, _ptr(X), k, _ptr(x))
    return x


def cutoff_ticks(p: Params) -> int:
    return int(lib().mto_cutoff_ticks(ctypes.byref(p)))


def move(p: Params, X: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Returns the moved copy of X (shape (dim, n) int64); xi float32 same shape."""
    X2 = _c(X, np.int64).reshape(p.dim, -1).copy()
    xi = _c(xi, np.float32).reshape(p.dim, -1)
    assert xi.shape == X2.shape
    lib().mto_move(ctypes.byref(p), X2.shape[1], _ptr(X2), _ptr(xi))
    return X2


def row_sums(p: Params, X: np.ndarray) -> np.ndarray:
    X = _c(X, np.int64).reshape(p.dim, -1)
    r = np.empty(X.shape[1], dtype=np.float64)
    lib().mto_row_sums(ctypes.byref(p), X.shape[1], _ptr(X), _ptr(r))
    return r


def _mt(fname, p: Params, X, Ms):
    X = _c(X, np.int64).reshape(p.dim, -1)
    n = X.shape[1]
    Ms = [_c(m, np.float64) for m in Ms]
    outs = [np.empty(n, dtype=np.float64) for _ in Ms]
    inp = (ctypes.c_void_p * len(Ms))(*[m.ctypes.data for m in Ms])
    out = (ctypes.c_void_p * len(Ms))(*[o.ctypes.data for o in outs])
    rc = getattr(lib(), fname)(ctypes.byref(p), n, _ptr(X), len(Ms), inp, out)
    if rc != 0:
        raise ValueError(f"{fname} rejected its arguments")
    return outs


def mass_transfer(p, X, Ms):
    """Eq. 3, 4, 7 by plain all-pairs loops; returns the new mass arrays."""
    return _mt("mto_mass_transfer", p, X, Ms)


def mass_transfer_matrix(p, X, Ms):
    """Eq. 5-6 dense matrix form (sign as in Eq. 4)."""
    return _mt("mto_mass_transfer_matrix", p, X, Ms)


def mass_transfer_sorted_1d(p, X, Ms):
    """Sec. 2.1 fixed-radius search via sorted windows (1-d, cutoff only)."""
    return _mt("mto_mass_transfer_sorted_1d", p, X, Ms)


def mass_transfer_sample(p, X, Ms, idx):
    X = _c(X, np.int64).reshape(p.dim, -1)
    Ms = [_c(m, np.float64) for m in Ms]
    idx = _c(idx, np.int64)
    outs = [np.empty(len(idx), dtype=np.float64) for _ in Ms]
    inp = (ctypes.c_void_p * len(Ms))(*[m.ctypes.data for m in Ms])
    out = (ctypes.c_void_p * len(Ms))(*[o.ctypes.data for o in outs])
    rc = lib().mto_mass_transfer_sample(ctypes.byref(p), X.shape[1], _ptr(X),
                                        len(Ms), inp, len(idx), _ptr(idx), out)
    if rc != 0:
        raise ValueError("mto_mass_transfer_sample rejected its arguments")
    return outs


def react(A, B):
    A = _c(A, np.float64).copy()
    B = _c(B, np.float64).copy()
    lib().mto_react(len(A), _ptr(A), _ptr(B))
    return A, B


def _pairs(fname, p, X):
    X = _c(X, np.int64).reshape(p.dim, -1)
    n = X.shape[1]
    f = getattr(lib(), fname)
    cnt = f(ctypes.byref(p), n, _ptr(X), 0, None, None)
    if cnt < 0:
        raise ValueError(f"{fname} rejected its arguments")
    pi = np.empty(max(cnt, 1), dtype=np.int32)
    pj = np.empty(max(cnt, 1), dtype=np.int32)
    f(ctypes.byref(p), n, _ptr(X), cnt, _ptr(pi), _ptr(pj))
    return pi[:cnt], pj[:cnt]


def pairs_brute(p, X):
    """All unordered pairs i < j inside the cutoff, by testing every pair."""
    return _pairs("mto_pairs_brute", p, X)


def pairs_sorted_1d(p, X):
    """The same set via sort + window scan (1-d)."""
    return _pairs("mto_pairs_sorted_1d", p, X)


def step(p, X, xi, A, B):
    """One time step (move, transfer, react); returns new (X, A, B)."""
    X2 = _c(X, np.int64).reshape(p.dim, -1).copy()
    xi = _c(xi, np.float32).reshape(p.dim, -1)
    A2 = _c(A, np.float64).copy()
    B2 = _c(B, np.float64).copy()
    rc = lib().mto_step(ctypes.byref(p), X2.shape[1], _ptr(X2), _ptr(xi),
                        _ptr(A2), _ptr(B2))
    if rc != 0:
        raise ValueError("mto_step rejected its arguments")
    return X2, A2, B2


def observables(A, B):
    A = _c(A, np.float64)
    B = _c(B, np.float64)
    out = np.empty(4, dtype=np.float64)
    lib().mto_observables(len(A), _ptr(A), _ptr(B), _ptr(out))
    return out


def set_threads(threads: int) -> int:
    """Threads of the sorted-window transfer's per-particle loops (OpenMP
    builds; the results do not depend on the count).  Returns the count in
    effect: 1 when the oracle was built without OpenMP."""
    return int(lib().mto_set_threads(int(threads)))
