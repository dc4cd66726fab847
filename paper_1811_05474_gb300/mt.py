"""ctypes binding of libmt (include/mt.h).

Functions keep the C names and only marshal arguments; every step of the
computation runs in the library's CUDA kernels.  ``Simulation`` bundles a
handle with a PyTorch-allocated device workspace and stream.  Loading fails
loudly (``RuntimeError``) when the compiled library is missing: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from .build import LIB

MT_OK = 0
MT_ERR_INVALID = -1
MT_ERR_WORKSPACE = -2
MT_ERR_CUDA = -3
MT_ERR_DEVICE = -4
MT_ERR_TIMEOUT = -5
MT_ERR_STATE = -6

MT_SEARCH_CELL, MT_SEARCH_BRUTE, MT_SEARCH_FULL = 0, 1, 2
MT_FP64, MT_MIXED, MT_MIXED_DF32 = 0, 1, 2
MT_NORM_SYM, MT_NORM_ROW = 0, 1
MT_MEM_HOST, MT_MEM_DEVICE = 0, 1
MT_WALLS_REFLECT, MT_WALLS_PERIODIC = 0, 1
MT_MAX_SPECIES = 8


class mt_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("frac_bits", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("L", ctypes.c_double * 2),
        ("v", ctypes.c_double * 2),
        ("D_mt", ctypes.c_double),
        ("D_rw", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("cutoff", ctypes.c_double),
        ("search", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("norm", ctypes.c_int32),
        ("react", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("realisation", ctypes.c_uint64),
        ("observe_cap", ctypes.c_int32),
        ("cell_shift", ctypes.c_int32),
        ("seg_target", ctypes.c_int32),
        ("walls", ctypes.c_int32),
        ("species", ctypes.c_int32),
        ("stored_p", ctypes.c_int32),
    ]


class mt_batch(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("n", ctypes.POINTER(ctypes.c_int64)),
        ("L", ctypes.POINTER(ctypes.c_double)),
        ("realisation", ctypes.POINTER(ctypes.c_uint64)),
    ]


def make_batch(n, L, realisation=None) -> mt_batch:
    """An mt_batch over Python sequences; the arrays are kept alive on the
    returned object."""
    R = len(n)
    b = mt_batch()
    b._n = (ctypes.c_int64 * R)(*[int(v) for v in n])
    b._L = (ctypes.c_double * R)(*[float(v) for v in L])
    b.count = R
    b.n = ctypes.cast(b._n, ctypes.POINTER(ctypes.c_int64))
    b.L = ctypes.cast(b._L, ctypes.POINTER(ctypes.c_double))
    if realisation is not None:
        b._r = (ctypes.c_uint64 * R)(*[int(v) for v in realisation])
        b.realisation = ctypes.cast(b._r, ctypes.POINTER(ctypes.c_uint64))
    return b


MT_REQ_QUEUED, MT_REQ_RUNNING, MT_REQ_DONE, MT_REQ_FAILED = 0, 1, 2, 3


class mt_server_config(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int32), ("chunk_steps", ctypes.c_int32),
                ("backfill", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class mt_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("steps_done", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("gpu_ms", ctypes.c_double), ("footprint", ctypes.c_size_t)]


class mt_server_summary(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("done", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("pool_used", ctypes.c_size_t), ("pool_peak", ctypes.c_size_t),
                ("step_samples", ctypes.c_int64)]


class MtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmt status {status}: {msg}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p


def lib(path: Path | None = None):
    """Load libmt (once).  Raises RuntimeError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB
    if not p.exists():
        raise RuntimeError(f"libmt is not built ({p} missing); run __graft_entry__.build()")
    L = ctypes.CDLL(str(p))
    P = ctypes.POINTER(mt_params)
    BP = ctypes.POINTER(mt_batch)
    H = ctypes.c_void_p
    i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "mt_params_init": [P],
        "mt_resolve": [P, P],
        "mt_workspace_bytes": [P, ctypes.POINTER(ctypes.c_size_t)],
        "mt_create": [P, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(H)],
        "mt_batch_resolve": [P, BP, P],
        "mt_batch_workspace_bytes": [P, BP, ctypes.POINTER(ctypes.c_size_t)],
        "mt_batch_create": [P, BP, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(H)],
        "mt_autotune_workspace_bytes": [P, BP, ctypes.POINTER(ctypes.c_size_t)],
        "mt_autotune": [P, BP, _vp, _vp, _vp, i32, _vp, ctypes.c_size_t, _vp, i32, i32, P,
                        ctypes.POINTER(ctypes.c_float)],
        "mt_upload": [H, _vp, _vp, _vp, i32],
        "mt_set_noise": [H, _vp],
        "mt_step": [H],
        "mt_run": [H, i64],
        "mt_sync": [H],
        "mt_read_masses": [H, _vp, _vp, i32],
        "mt_set_species": [H, i32, _vp, i32],
        "mt_save": [H, ctypes.c_char_p],
        "mt_checkpoint_params": [ctypes.c_char_p, P],
        "mt_load": [H, ctypes.c_char_p],
        "mt_read_species": [H, i32, _vp, i32],
        "mt_read_positions": [H, _vp, i32],
        "mt_read_ticks": [H, _vp, i32],
        "mt_read_observables": [H, _vp, i64, ctypes.POINTER(i64)],
        "mt_read_pairs": [H, _vp, _vp, i64, ctypes.POINTER(i64)],
        "mt_copy_observables_async": [H, _vp, i64],
        "mt_copy_observables_row_async": [H, _vp, i64],
        "mt_steps_done": [H, ctypes.POINTER(i64)],
        "mt_philox": [H, u32, u32, u32, u32, u32, u32, i64, _vp],
        "mt_set_profiling": [H, i32],
        "mt_test_hold_scan": [H, i32, i64],
        "mt_walk_normals": [P, _vp, i64, ctypes.c_uint64, _vp, _vp],
        "mt_probe_rate": [i32, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(ctypes.c_double)],
        "mt_test_exp_neg": [_vp, _vp, i64, _vp],
        "mt_transfer_1d_noalloc": [_vp, _vp, _vp, _vp, _vp, i64, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, i32, i32,
                                   _vp],
        "mt_read_profile": [H, _vp, i32, ctypes.POINTER(i32)],
        "mt_server_footprint": [P, ctypes.POINTER(ctypes.c_size_t)],
        "mt_server_create": [ctypes.POINTER(mt_server_config), _vp, ctypes.c_size_t,
                             ctypes.POINTER(H)],
        "mt_server_submit": [H, P, _vp, _vp, _vp, i64, ctypes.POINTER(i64)],
        "mt_server_poll": [H, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "mt_server_info": [H, i64, ctypes.POINTER(mt_request_info)],
        "mt_server_result": [H, i64, _vp, _vp, _vp, i64, ctypes.POINTER(i64)],
        "mt_server_submit_species": [H, P, _vp, _vp, i64, ctypes.POINTER(i64)],
        "mt_server_result_species": [H, i64, i32, _vp],
        "mt_server_release": [H, i64],
        "mt_server_stats": [H, ctypes.POINTER(mt_server_summary), _vp, i64],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.mt_profile_name.argtypes = [H, i32]
    L.mt_profile_name.restype = ctypes.c_char_p
    L.mt_last_error.argtypes = []
    L.mt_last_error.restype = ctypes.c_char_p
    L.mt_destroy.argtypes = [H]
    L.mt_destroy.restype = None
    L.mt_server_destroy.argtypes = [H]
    L.mt_server_destroy.restype = None
    _lib = L
    return L


def mt_last_error() -> str:
    return lib().mt_last_error().decode(errors="replace")


def check(status: int) -> None:
    if status != MT_OK:
        raise MtError(status, mt_last_error())


# ------------------------------------------------------------ thin wrappers --

def mt_params_init(**kw) -> mt_params:
    p = mt_params()
    check(lib().mt_params_init(ctypes.byref(p)))
    for k, v in kw.items():
        if k in ("L", "v"):
            vals = list(v) + [0.0] * (2 - len(v))
            setattr(p, k, (ctypes.c_double * 2)(*vals))
        else:
            setattr(p, k, v)
    return p


def mt_resolve(p: mt_params) -> mt_params:
    out = mt_params()
    check(lib().mt_resolve(ctypes.byref(p), ctypes.byref(out)))
    return out


def mt_workspace_bytes(p: mt_params) -> int:
    b = ctypes.c_size_t(0)
    check(lib().mt_workspace_bytes(ctypes.byref(p), ctypes.byref(b)))
    return int(b.value)


def mt_create(p: mt_params, workspace_ptr: int, workspace_bytes: int, stream_ptr: int | None):
    h = ctypes.c_void_p(0)
    check(lib().mt_create(ctypes.byref(p), workspace_ptr, workspace_bytes, stream_ptr or None,
                          ctypes.byref(h)))
    return h


def _bref(b):
    return ctypes.byref(b) if b is not None else None


def mt_batch_resolve(p: mt_params, b: mt_batch | None) -> mt_params:
    out = mt_params()
    check(lib().mt_batch_resolve(ctypes.byref(p), _bref(b), ctypes.byref(out)))
    return out


def mt_batch_workspace_bytes(p: mt_params, b: mt_batch | None) -> int:
    n = ctypes.c_size_t(0)
    check(lib().mt_batch_workspace_bytes(ctypes.byref(p), _bref(b), ctypes.byref(n)))
    return int(n.value)


def mt_batch_create(p: mt_params, b: mt_batch | None, workspace_ptr: int, workspace_bytes: int,
                    stream_ptr: int | None):
    h = ctypes.c_void_p(0)
    check(lib().mt_batch_create(ctypes.byref(p), _bref(b), workspace_ptr, workspace_bytes,
                                stream_ptr or None, ctypes.byref(h)))
    return h


def mt_autotune_workspace_bytes(p: mt_params, b: mt_batch | None) -> int:
    n = ctypes.c_size_t(0)
    check(lib().mt_autotune_workspace_bytes(ctypes.byref(p), _bref(b), ctypes.byref(n)))
    return int(n.value)


def mt_autotune(p: mt_params, b: mt_batch | None, x_ptr, A_ptr, B_ptr, mem: int,
                workspace_ptr: int, workspace_bytes: int, stream_ptr, warmup: int, steps: int):
    """Returns (best resolved mt_params, ms per step)."""
    best = mt_params()
    ms = ctypes.c_float(0.0)
    check(lib().mt_autotune(ctypes.byref(p), _bref(b), x_ptr, A_ptr, B_ptr, mem, workspace_ptr,
                            workspace_bytes, stream_ptr or None, warmup, steps, ctypes.byref(best),
                            ctypes.byref(ms)))
    return best, float(ms.value)


def autotune(params: mt_params, x, A, B, batch: mt_batch | None = None, warmup: int = 3,
             steps: int = 10, device="cuda"):
    """mt_autotune on host arrays with a torch-allocated workspace and
    stream; returns (best params, ms per step)."""
    import torch

    x = np.ascontiguousarray(x, dtype=np.float64)
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    nbytes = mt_autotune_workspace_bytes(params, batch)
    ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
    stream = torch.cuda.Stream(device=device)
    try:
        return mt_autotune(params, batch, _ptr(x), _ptr(A), _ptr(B), MT_MEM_HOST, ws.data_ptr(),
                           ws.numel(), stream.cuda_stream, warmup, steps)
    finally:
        stream.synchronize()
        del ws


def mt_upload(h, x_ptr, A_ptr, B_ptr, mem: int) -> None:
    check(lib().mt_upload(h, x_ptr, A_ptr, B_ptr, mem))


def mt_set_noise(h, xi_ptr) -> None:
    check(lib().mt_set_noise(h, xi_ptr))


def mt_step(h) -> None:
    check(lib().mt_step(h))


def mt_run(h, nsteps: int) -> None:
    check(lib().mt_run(h, nsteps))


def mt_sync(h) -> None:
    check(lib().mt_sync(h))


def mt_read_masses(h, A_ptr, B_ptr, mem: int) -> None:
    check(lib().mt_read_masses(h, A_ptr, B_ptr, mem))


def mt_set_species(h, s: int, M_ptr, mem: int) -> None:
    check(lib().mt_set_species(h, s, M_ptr, mem))


def mt_save(h, path: str) -> None:
    check(lib().mt_save(h, str(path).encode()))


def mt_checkpoint_params(path: str) -> mt_params:
    p = mt_params()
    check(lib().mt_checkpoint_params(str(path).encode(), ctypes.byref(p)))
    return p


def mt_load(h, path: str) -> None:
    check(lib().mt_load(h, str(path).encode()))


def mt_read_species(h, s: int, M_ptr, mem: int) -> None:
    check(lib().mt_read_species(h, s, M_ptr, mem))


def mt_read_positions(h, x_ptr, mem: int) -> None:
    check(lib().mt_read_positions(h, x_ptr, mem))


def mt_read_ticks(h, X_ptr, mem: int) -> None:
    check(lib().mt_read_ticks(h, X_ptr, mem))


def mt_copy_observables_async(h, out_ptr, rows: int) -> None:
    check(lib().mt_copy_observables_async(h, out_ptr, rows))


def mt_copy_observables_row_async(h, out_ptr, step: int) -> None:
    """Enqueue the copy of step `step`'s observables row (see include/mt.h)."""
    check(lib().mt_copy_observables_row_async(h, out_ptr, step))


def mt_read_observables(h, out_ptr, cap: int) -> int:
    cnt = ctypes.c_int64(0)
    check(lib().mt_read_observables(h, out_ptr, cap, ctypes.byref(cnt)))
    return int(cnt.value)


def mt_read_pairs(h, pi_ptr, pj_ptr, cap: int) -> int:
    cnt = ctypes.c_int64(0)
    check(lib().mt_read_pairs(h, pi_ptr, pj_ptr, cap, ctypes.byref(cnt)))
    return int(cnt.value)


def mt_steps_done(h) -> int:
    s = ctypes.c_int64(0)
    check(lib().mt_steps_done(h, ctypes.byref(s)))
    return int(s.value)


def mt_philox(h, ctr, key, n: int, out_ptr) -> None:
    check(lib().mt_philox(h, *[int(c) & 0xFFFFFFFF for c in ctr],
                          *[int(k) & 0xFFFFFFFF for k in key], n, out_ptr))


def mt_set_profiling(h, on: bool) -> None:
    check(lib().mt_set_profiling(h, 1 if on else 0))


def mt_read_profile(h):
    """[(kernel name, ms), ...] for the last profiled step."""
    ms = (ctypes.c_float * 16)()
    cnt = ctypes.c_int32(0)
    check(lib().mt_read_profile(h, ms, 16, ctypes.byref(cnt)))
    n = min(int(cnt.value), 16)
    return [(mt_profile_name(h, i), float(ms[i])) for i in range(n)]


def mt_profile_name(h, idx: int) -> str:
    return lib().mt_profile_name(h, idx).decode()


def mt_walk_normals(p: mt_params, gid_ptr, n: int, step: int, out_ptr, stream_ptr=None) -> None:
    """Built-in walk normals of particles gid at a step (see include/mt.h)."""
    check(lib().mt_walk_normals(ctypes.byref(p), gid_ptr, n, step, out_ptr, stream_ptr))


PROBE_DFMA, PROBE_FFMA, PROBE_EXPF, PROBE_EXP, PROBE_EXP_NEG = 0, 1, 2, 3, 4


def mt_probe_rate(which: int, device="cuda") -> float:
    """Operations per second of one device pipe (see include/mt.h)."""
    import torch

    scratch = torch.empty(64 * 1024, dtype=torch.uint8, device=device)
    out = ctypes.c_double(0.0)
    check(lib().mt_probe_rate(which, scratch.data_ptr(), scratch.numel(), None,
                              ctypes.byref(out)))
    return float(out.value)


def mt_test_exp_neg(t_ptr, out_ptr, n: int, stream_ptr=None) -> None:
    """Test hook: the weights' binary64 exp(-t) on device arrays (see include/mt.h)."""
    check(lib().mt_test_exp_neg(t_ptr, out_ptr, n, stream_ptr))


def mt_test_hold_scan(h, hold: int, spin_limit: int = 0) -> None:
    """Test hook: withhold the scan's first status word (see include/mt.h)."""
    check(lib().mt_test_hold_scan(h, hold, spin_limit))


def mt_transfer_1d_noalloc(x_ptr, A_ptr, B_ptr, Ao_ptr, Bo_ptr, n: int, L: float, D_mt: float,
                           dt: float, cutoff: float, norm: int, react: int,
                           stream_ptr=None) -> None:
    """Device pointers in and out; see include/mt.h (no device allocation)."""
    check(lib().mt_transfer_1d_noalloc(x_ptr, A_ptr, B_ptr, Ao_ptr, Bo_ptr, n, L, D_mt, dt,
                                       cutoff, norm, react, stream_ptr))


def mt_destroy(h) -> None:
    lib().mt_destroy(h)


def mt_server_footprint(p: mt_params) -> int:
    b = ctypes.c_size_t(0)
    check(lib().mt_server_footprint(ctypes.byref(p), ctypes.byref(b)))
    return int(b.value)


def mt_server_create(cfg: mt_server_config, pool_ptr: int, pool_bytes: int):
    s = ctypes.c_void_p(0)
    check(lib().mt_server_create(ctypes.byref(cfg), pool_ptr, pool_bytes, ctypes.byref(s)))
    return s


def mt_server_submit(s, p: mt_params, x_ptr, A_ptr, B_ptr, steps: int) -> int:
    rid = ctypes.c_int64(0)
    check(lib().mt_server_submit(s, ctypes.byref(p), x_ptr, A_ptr, B_ptr, steps,
                                 ctypes.byref(rid)))
    return int(rid.value)


def mt_server_poll(s):
    q, r = ctypes.c_int32(0), ctypes.c_int32(0)
    check(lib().mt_server_poll(s, ctypes.byref(q), ctypes.byref(r)))
    return int(q.value), int(r.value)


def mt_server_info(s, rid: int) -> mt_request_info:
    info = mt_request_info()
    check(lib().mt_server_info(s, rid, ctypes.byref(info)))
    return info


def mt_server_result(s, rid: int, A_ptr, B_ptr, obs_ptr, cap: int) -> int:
    rows = ctypes.c_int64(0)
    check(lib().mt_server_result(s, rid, A_ptr, B_ptr, obs_ptr, cap, ctypes.byref(rows)))
    return int(rows.value)


def mt_server_submit_species(s, p, x_ptr, M_ptr, steps: int) -> int:
    rid = ctypes.c_int64(0)
    check(lib().mt_server_submit_species(s, ctypes.byref(p), x_ptr, M_ptr, steps, ctypes.byref(rid)))
    return int(rid.value)


def mt_server_result_species(s, rid: int, sp: int, out_ptr) -> None:
    check(lib().mt_server_result_species(s, rid, sp, out_ptr))


def mt_server_release(s, rid: int) -> None:
    check(lib().mt_server_release(s, rid))


def mt_server_stats(s, step_ms_ptr=None, cap: int = 0) -> mt_server_summary:
    out = mt_server_summary()
    check(lib().mt_server_stats(s, ctypes.byref(out), step_ms_ptr, cap))
    return out


def mt_server_destroy(s) -> None:
    lib().mt_server_destroy(s)


# -------------------------------------------------------------- Simulation --

def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Simulation:
    """A handle plus its device workspace (a torch uint8 tensor) and stream.

    Host-array helpers copy through the C ABI with MT_MEM_HOST; the ``*_dev``
    variants take torch CUDA tensors.
    """

    def __init__(self, params: mt_params, device="cuda", stream=None, batch: mt_batch | None = None):
        import torch

        self.torch = torch
        self.batch = batch
        self.nreal = int(batch.count) if batch is not None else 1
        self.params = mt_batch_resolve(params, batch)
        self.device = torch.device(device)
        self.nbytes = mt_batch_workspace_bytes(params, batch)
        self.workspace = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.h = mt_batch_create(params, batch, self.workspace.data_ptr(), self.workspace.numel(),
                                 self.stream.cuda_stream)
        self._noise = None

    @property
    def n(self) -> int:
        return int(self.params.n)

    @property
    def dim(self) -> int:
        return int(self.params.dim)

    def close(self):
        if getattr(self, "h", None):
            mt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state in / out (host numpy)
    def upload(self, x: np.ndarray, A: np.ndarray, B: np.ndarray) -> None:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.dim, self.n)
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        assert A.shape == (self.n,) and B.shape == (self.n,)
        mt_upload(self.h, _ptr(x), _ptr(A), _ptr(B), MT_MEM_HOST)

    def masses(self):
        A = np.empty(self.n, dtype=np.float64)
        B = np.empty(self.n, dtype=np.float64)
        mt_read_masses(self.h, _ptr(A), _ptr(B), MT_MEM_HOST)
        return A, B

    def set_species(self, s: int, M: np.ndarray) -> None:
        M = np.ascontiguousarray(M, dtype=np.float64)
        assert M.shape == (self.n,)
        mt_set_species(self.h, s, _ptr(M), MT_MEM_HOST)

    def species(self, s: int) -> np.ndarray:
        M = np.empty(self.n, dtype=np.float64)
        mt_read_species(self.h, s, _ptr(M), MT_MEM_HOST)
        return M

    def save(self, path) -> None:
        mt_save(self.h, path)

    def load(self, path) -> None:
        mt_load(self.h, path)

    def positions(self) -> np.ndarray:
        x = np.empty((self.dim, self.n), dtype=np.float64)
        mt_read_positions(self.h, _ptr(x), MT_MEM_HOST)
        return x

    def ticks(self) -> np.ndarray:
        X = np.empty((self.dim, self.n), dtype=np.int64)
        mt_read_ticks(self.h, _ptr(X), MT_MEM_HOST)
        return X

    def observables(self) -> np.ndarray:
        """(steps, 4) rows; (steps, realisations, 4) for a batch."""
        cap = int(self.params.observe_cap)
        out = np.zeros((max(cap, 1), self.nreal, 4), dtype=np.float64)
        cnt = mt_read_observables(self.h, _ptr(out), cap)
        return out[:cnt] if self.batch is not None else out[:cnt, 0]

    def set_noise(self, xi: np.ndarray | None) -> None:
        """Inject standard normals (dim, n) for the following steps; None
        returns to the built-in generator."""
        if xi is None:
            self._noise = None
            mt_set_noise(self.h, None)
            return
        t = self.torch.as_tensor(np.ascontiguousarray(xi, dtype=np.float32).reshape(-1))
        dev = t.to(self.device)
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        dev.record_stream(self.stream)  # the handle's stream reads it
        self._noise = dev
        mt_set_noise(self.h, dev.data_ptr())

    def step(self, n: int = 1) -> None:
        for _ in range(n):
            mt_step(self.h)

    def run(self, n: int) -> None:
        mt_run(self.h, n)

    def sync(self) -> None:
        mt_sync(self.h)

    def pairs(self):
        cnt = mt_read_pairs(self.h, None, None, 0)
        torch = self.torch
        pi = torch.empty(max(cnt, 1), dtype=torch.int32, device=self.device)
        pj = torch.empty(max(cnt, 1), dtype=torch.int32, device=self.device)
        cnt2 = mt_read_pairs(self.h, pi.data_ptr(), pj.data_ptr(), cnt)
        assert cnt2 == cnt
        return pi[:cnt].cpu().numpy(), pj[:cnt].cpu().numpy()

    def steps_done(self) -> int:
        return mt_steps_done(self.h)


# ------------------------------------------------------------------ Server --

class Server:
    """An mt_server over a torch-allocated device pool of pool_bytes."""

    def __init__(self, pool_bytes: int, max_active: int = 16, chunk_steps: int = 25,
                 backfill: bool = True, device="cuda"):
        import torch

        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=device)
        cfg = mt_server_config(max_active=max_active, chunk_steps=chunk_steps,
                               backfill=1 if backfill else 0)
        self.s = mt_server_create(cfg, self.pool.data_ptr(), self.pool.numel())
        self.params = {}

    def submit(self, p: mt_params, x, A, B, steps: int) -> int:
        r = mt_resolve(p)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        assert x.size == r.dim * r.n and A.size == r.n and B.size == r.n
        rid = mt_server_submit(self.s, p, _ptr(x), _ptr(A), _ptr(B), steps)
        self.params[rid] = r
        return rid

    def submit_species(self, p: mt_params, x, Ms, steps: int) -> int:
        """A request carrying len(Ms) species (Ms[0] = A, Ms[1] = B, ...)."""
        r = mt_resolve(p)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        M = np.ascontiguousarray(np.stack([np.asarray(m, dtype=np.float64) for m in Ms]))
        assert x.size == r.dim * r.n and M.shape == (r.species, r.n)
        rid = mt_server_submit_species(self.s, p, _ptr(x), _ptr(M), steps)
        self.params[rid] = r
        return rid

    def result_species(self, rid: int, sp: int) -> np.ndarray:
        r = self.params[rid]
        out = np.empty(int(r.n))
        mt_server_result_species(self.s, rid, sp, _ptr(out))
        return out

    def poll(self):
        return mt_server_poll(self.s)

    def drain(self, sleep: float = 0.0):
        import time

        while True:
            q, r = self.poll()
            if q == 0 and r == 0:
                return
            if sleep:
                time.sleep(sleep)

    def info(self, rid: int) -> mt_request_info:
        return mt_server_info(self.s, rid)

    def result(self, rid: int):
        r = self.params.get(rid)
        if r is None:  # unknown here: let the server report it
            mt_server_result(self.s, rid, None, None, None, 0)
            raise MtError(MT_ERR_INVALID, f"unknown request {rid}")
        A = np.empty(int(r.n))
        B = np.empty(int(r.n))
        cap = int(r.observe_cap)
        obs = np.zeros((max(cap, 1), 4))
        rows = mt_server_result(self.s, rid, _ptr(A), _ptr(B), _ptr(obs), cap)
        return A, B, obs[:rows]

    def release(self, rid: int):
        mt_server_release(self.s, rid)
        self.params.pop(rid, None)

    def stats(self):
        st = mt_server_stats(self.s)
        ms = np.zeros(max(int(st.step_samples), 1), dtype=np.float32)
        st = mt_server_stats(self.s, _ptr(ms), int(st.step_samples))
        return st, ms[:int(st.step_samples)]

    def close(self):
        if getattr(self, "s", None):
            mt_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
