#!/usr/bin/env python
"""Benchmark of the mass-transfer particle-tracking hot path on GB300.

One step = one time step of the whole path (random-walk move, cell-list
search, weight normalisation, mass exchange, A + B -> E reaction, per-step
observables) for every particle of the workload.  Workload: 1-d, N = 1e6
particles uniform on [0, 1e6], A and B masses uniform on [0, 1), D = 0.1,
dt = 1, advection v = 0.5, cutoff 3 sigma of the co-location kernel,
synthetic and seeded.  The headline runs the MIXED precision path (binary32
weights and exponentials; binary64 masses, flux terms, sums, update and
reaction).  The same line carries the binary64 path ("fp64"), the
double-binary32 variant ("mixed_df32"), the two smaller workloads
("workloads": N = 1e3 with the cell list, the cutoff brute force and the
full matrix; N = 1e5 in each precision), the batched, serving, accuracy
and paper-density forms, and the CPU oracle on one core and on all cores.

Timing: W warm-up steps, then K steps each replayed from a CUDA graph and
bracketed by CUDA events on the simulation's stream, with a 512 MiB write
(then read, so no dirty line is left) between steps to flush L2 (129 MB);
value = particles * K / sum of step times, max over ranks.  Per-kernel
durations come from a second pass of the same steps with events recorded
between the step's kernels inside the graph.

``--impl reference`` times the CPU oracle (single thread) on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 10 ** 6
L = 1e6
V = 0.5
D = 0.1
DT = 1.0
WORKLOAD = "1d_uniform_n1e6_L1e6_v0.5_D0.1_dt1_cutoff3sigma"

# Algorithmic bytes per particle for each kernel (what the kernel's job must
# read and write at minimum; sort scaffolding, ids and 1/r are overhead).
ALGO_BYTES = {
    "move": 16,            # x in, x out
    "scan": 0,
    "scatter": 16,         # x in, x out (sorted)
    "cellsort": 0,
    "bigsort": 0,
    "rowsum_walk": 8,      # x in
    "exchange_walk": 40,   # x, A, B in; A, B out
    "fused_step": 48,      # the whole step in one kernel: x, A, B in and out
    "step": 48,            # whole step: x, A, B in and out
}

CSRC = os.path.join(ROOT, "paper_1811_05474_gb300", "csrc")

DTYPES = {
    "mixed": "mixed: f32 weights and exp, f64 masses, flux terms, sums, update and reaction; "
             "i64 positions",
    "fp64": "f64 weights, masses and arithmetic; i64 positions",
    "df32": "mixed_df32: f32 weights, f32x2 (double-binary32) masses and compensated sums; "
            "i64 positions",
}


def prec_code(name: str) -> int:
    from paper_1811_05474_gb300 import mt

    return {"mixed": mt.MT_MIXED, "fp64": mt.MT_FP64, "df32": mt.MT_MIXED_DF32}[name]


def config_dict(precision: str) -> dict:
    """The headline workload's description, identical in both arms."""
    return {"workload": WORKLOAD, "n_particles": N, "L": L, "v": V, "D_mt": D, "D_rw": D,
            "dt": DT, "steps_per_run": 1000, "cutoff": "3*sqrt(4*D_mt*dt)",
            "normalisation": "symmetric", "precision": precision,
            "l2": "flushed between timed steps (512 MiB write, then read)"}


# The sources of the one-kernel step's device code: its translation unit and
# the internal headers it includes (the public header adds only the MT_*
# constants and the host API's declarations).
FUSED_SOURCES = ("paper_1811_05474_gb300/csrc/mt_fused.cu", "paper_1811_05474_gb300/csrc/mt_pair.cuh",
                 "paper_1811_05474_gb300/csrc/mt_internal.cuh")


def source_hash(files=None) -> str:
    """Hash of the given sources (paths relative to the repository), or of
    every file under csrc/."""
    if files is None:
        files = [os.path.relpath(os.path.join(CSRC, f), ROOT) for f in sorted(os.listdir(CSRC))]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(os.path.basename(f).encode() + fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "df32"])
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the binary64 and double-binary32 objects")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the N = 1e3 and N = 1e5 workloads")
    ap.add_argument("--detail", default=None,
                    help="also write the full result (every per-kernel list) to this JSON file")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ncu", action="store_true",
                    help="profiling mode: upload, W graph steps, then K direct steps, nothing else")
    ap.add_argument("--n", type=int, default=N, help="particles (profiling mode only)")
    ap.add_argument("--ncu-search", default="cell", choices=["cell", "full", "dense", "dense_spam"],
                    help="profiling mode: the cell list (headline), the full matrix, or the "
                         "paper's density on the fly or in the SPaM form")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble object")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision report")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving object")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the paper's accuracy problem")
    ap.add_argument("--no-dense", action="store_true", help="skip the paper-density workload")
    ap.add_argument("--no-brute", action="store_true", help="skip the all-pairs forms")
    ap.add_argument("--no-species", action="store_true", help="skip the species-count sweep")
    ap.add_argument("--serve-requests", type=int, default=64, help="requests in the serving run")
    return ap.parse_args()


def rank_reduce(vals, op: str, device=None):
    """All-reduce a list of floats over the ranks of the default process
    group ('max', 'min' or 'sum'); any backend (NCCL on GPUs, gloo in the
    CPU tests)."""
    import torch
    import torch.distributed as tdist

    ops = {"max": tdist.ReduceOp.MAX, "min": tdist.ReduceOp.MIN, "sum": tdist.ReduceOp.SUM}
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=ops[op])
    return [float(v) for v in t.tolist()]


def replicas_value(particles_per_rank: int, steps: int, max_total_ms: float, ranks: int) -> float:
    """Whole-job particle-steps/s of independent replicas (one realisation
    per rank, no data exchanged): all ranks' work over the slowest rank's
    timed region."""
    return ranks * particles_per_rank * steps / (max_total_ms * 1e-3)


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples (every 20 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu=timestamp,{self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.split(", ") for r in self.tmp.read().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        mine = [r for r in rows if len(r) >= 11 and (self.uuid is None or r[2].strip() == self.uuid)]
        if not mine and rows:
            idx0 = rows[0][1]
            mine = [r for r in rows if len(r) >= 11 and r[1] == idx0]
        self.rows = mine
        return self.summary(self.t0, self.t1)

    def summary(self, t0, t1):
        """Median SM clock, max clock and throttle reasons of the samples
        taken between t0 and t1 (all samples if no window is given)."""
        mine = getattr(self, "rows", [])
        if t0 is not None and t1 is not None:
            from datetime import datetime

            def ts(r):
                try:
                    return datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    return None

            inside = [r for r in mine if (ts(r) or 0) >= t0 - 0.05 and (ts(r) or 0) <= t1 + 0.05]
            if inside:
                mine = inside
        sm = [float(r[3]) for r in mine if r[3].replace(".", "").isdigit()]
        mx = [float(r[4]) for r in mine if r[4].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in mine for i in range(4) if r[7 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle --

def cpu_oracle_rate(n: int, steps: int, seed: int = 0):
    """Time the oracle (single thread) for `steps` steps of an n-particle,
    density-1 sample of the workload; returns particle-steps/s."""
    import oracle as O
    from paper_1811_05474_gb300 import synth

    Ln = float(n) * (L / N)
    p = O.params(L=(Ln,), v=(V,), D_mt=D, D_rw=D, dt=DT, frac_bits=29)
    X = O.quantize(synth.uniform_positions(n, Ln, seed=seed), 29)
    A, B = synth.uniform_masses(n, seed=seed)
    xi = synth.normals(steps, 1, n, seed=seed + 1)
    t0 = time.perf_counter()
    for s in range(steps):
        X, A, B = O.step(p, X, xi[s], A, B)
    dt = time.perf_counter() - t0
    return n * steps / dt, dt


def run_reference(args):
    """The reference arm: the CPU oracle as it stands (sorted-window search,
    one thread) on a bounded sample of the headline workload, each step of
    the run timed on an n-particle density-1 piece of it, n chosen so the
    whole run takes about two minutes."""
    ws, rank, _ = dist()
    if rank != 0:
        return 0
    per_particle = 0.7e-6
    budget = 120.0
    n = int(min(N, max(10 ** 4, budget / max(args.steps + args.warmup, 1) / per_particle)))
    cpu_oracle_rate(n, max(args.warmup, 0))
    rate, secs = cpu_oracle_rate(n, args.steps, seed=1)
    info = cpu_info()
    line = {
        "impl": "reference", "metric": "particle-steps/s", "value": rate,
        "unit": "particle-steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / max(args.steps, 1) * (N / n), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args.precision),
        "cpu_baseline": {"value": rate, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps of a {n}-particle density-1 piece of the "
                                   f"workload (sorted-window search, one thread)", **info},
        "e2e": {"value": rate, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU --

def gpu_run(args, precision: str, steps: int, warmup: int, local: int, realisation: int,
            sampler: ClockSampler | None):
    import torch

    from paper_1811_05474_gb300 import mt, synth

    dev = torch.device("cuda", local)
    prec = prec_code(precision)
    p = mt.mt_params_init(n=N, L=(L,), v=(V, 0.0), D_mt=D, D_rw=D, dt=DT,
                          search=mt.MT_SEARCH_CELL, precision=prec, norm=mt.MT_NORM_SYM,
                          react=1, seed=2024, realisation=realisation,
                          observe_cap=steps + warmup)
    sim = mt.Simulation(p, device=dev)
    x = synth.uniform_positions(N, L, seed=realisation)
    A, B = synth.uniform_masses(N, seed=realisation)
    sim.upload(x, A, B)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    flush_sum = torch.empty((), dtype=torch.int64, device=dev)
    s = sim.stream

    def flush_l2():
        # write 512 MiB (evicts the state), then read it back so the lines
        # left in L2 are clean and no write-back lands in the timed step
        with torch.cuda.stream(s):
            flush.zero_()
            torch.sum(flush.view(torch.int64), dim=0, out=flush_sum)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for _ in range(warmup):
        flush_l2()
        sim.run(1)
    sim.sync()
    # timed region: steps enqueued back to back (no host sync inside), each
    # bracketed by events after its L2 flush
    t_start = time.time()
    if sampler:
        sampler.mark("t0")
    for i in range(steps):
        flush_l2()
        e0[i].record(s)
        sim.run(1)
        e1[i].record(s)
    torch.cuda.synchronize(dev)
    t_end = time.time()
    if sampler:
        sampler.mark("t1")
    step_ms = [e0[i].elapsed_time(e1[i]) for i in range(steps)]
    npairs = mt.mt_read_pairs(sim.h, None, None, 0)
    # kernel breakdown: the same run again from the same state, every
    # stride-th step of the timed range launched directly with CUDA events
    # between its kernels (the others from the graph), so that the kernel
    # times average over the same steps as the timed region (the wall layer
    # grows over the run); the first tier and the predicted-segment kernel
    # run one after the other there, so the transfer phase of a sampled step
    # is the longer of the two
    sim.upload(x, A, B)
    stride = max(1, steps // 200)
    kernel_ms = {}
    order = []
    phase = []
    nprof = 0
    for i in range(warmup + steps):
        flush_l2()
        sampled = i >= warmup and (i - warmup) % stride == 0
        if sampled:
            mt.mt_set_profiling(sim.h, True)
        sim.run(1)
        if sampled:
            nprof += 1
            got = mt.mt_read_profile(sim.h)
            mt.mt_set_profiling(sim.h, False)
            for name, ms in got:
                if name not in kernel_ms:
                    kernel_ms[name] = []
                    order.append(name)
                kernel_ms[name].append(ms)
            tr = [ms for name, ms in got if name in ("fused_step", "fused_pred")]
            if tr:
                phase.append(max(tr))
    sim.sync()
    kernels = [{"name": k, "ms": sum(kernel_ms[k]) / len(kernel_ms[k]),
                "launches_per_step": len(kernel_ms[k]) / nprof,
                "ms_per_step": sum(kernel_ms[k]) / nprof} for k in order]
    launches_per_step = sum(len(v) for v in kernel_ms.values()) / nprof
    obs = sim.observables()
    sim.close()
    del flush
    return {"total_ms": sum(step_ms), "step_ms": step_ms, "kernels": kernels,
            "phase_ms": sum(phase) / len(phase) if phase else None, "profiled_steps": nprof,
            "launches_per_step": launches_per_step, "npairs": npairs,
            "mean_A_last": float(obs[-1, 3]) if len(obs) else None,
            "t0": t_start, "t1": t_end}


def e2e_run(steps: int, local: int, realisation: int, precision: str = "mixed"):
    """Through the public API with host buffers: upload from pinned host
    memory, then every step enqueue it and the copy of an observables row
    into pinned host memory -- the previous step's, which the step just
    enqueued computes beside itself (mt_copy_observables_row_async), and
    the last step's after the loop -- with no wait between steps, then read
    the final masses (which waits for all of it).  Wall-clock."""
    import numpy as np
    import torch

    from paper_1811_05474_gb300 import mt, synth

    dev = torch.device("cuda", local)
    p = mt.mt_params_init(n=N, L=(L,), v=(V, 0.0), D_mt=D, D_rw=D, dt=DT,
                          precision=prec_code(precision), seed=7, realisation=realisation,
                          observe_cap=2)
    sim = mt.Simulation(p, device=dev)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    x = pin(synth.uniform_positions(N, L, seed=realisation))
    A, B = (pin(v) for v in synth.uniform_masses(N, seed=realisation))
    oa, ob = pin(np.empty(N)), pin(np.empty(N))
    rows = pin(np.zeros((steps, 4)))
    last = np.empty((1, 4))
    ptr = mt._ptr
    sim.upload(x, A, B)  # warm the graph and the pages
    sim.run(2)
    sim.masses()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    mt.mt_upload(sim.h, ptr(x), ptr(A), ptr(B), mt.MT_MEM_HOST)
    for s in range(steps):
        mt.mt_run(sim.h, 1)
        if s >= 1:
            mt.mt_copy_observables_row_async(sim.h, ptr(rows[s - 1]), s)
    mt.mt_copy_observables_row_async(sim.h, ptr(rows[steps - 1]), steps)
    mt.mt_read_masses(sim.h, ptr(oa), ptr(ob), mt.MT_MEM_HOST)
    secs = time.perf_counter() - t0
    last = np.empty((2, 4))
    mt.mt_read_observables(sim.h, ptr(last), 2)
    assert np.array_equal(rows[-2:], last) and np.all(rows[:, 0] > 0), "observables rows"
    sim.close()
    return {"value": N * steps / secs, "unit": "particle-steps/s",
            "h2d_bytes_per_step": (24 * N) / steps, "d2h_bytes_per_step": 32 + (16 * N) / steps}


BATCH_R = 256
BATCH_WORKLOAD = "batch_256x1d_N_loguniform_1e3_1e5_L_eq_N_D0.1_dt1_cutoff3sigma"


def batch_inputs():
    """256 realisations, N_r = floor(10^U(3, 5)) from seed r, uniform on
    [0, N_r] (density 1), masses U[0, 1) from seed r."""
    import numpy as np

    from paper_1811_05474_gb300 import synth

    ns = synth.ensemble_sizes(BATCH_R, 1e3, 1e5)
    Ls = [float(n) for n in ns]
    xs, As, Bs = [], [], []
    for r, n in enumerate(ns):
        xs.append(synth.uniform_positions(int(n), Ls[r], seed=r)[0])
        a, b = synth.uniform_masses(int(n), seed=r)
        As.append(a)
        Bs.append(b)
    return ns, Ls, xs, As, Bs, (np.concatenate(xs)[None, :], np.concatenate(As),
                                np.concatenate(Bs))


def timed_steps(sim, steps: int, warmup: int, flush_l2=None):
    """Sum of per-step CUDA-event times over `steps` graph steps (after
    `warmup` untimed ones), each step bracketed on the simulation's stream."""
    import torch

    s = sim.stream
    for _ in range(warmup):
        if flush_l2:
            flush_l2(s)
        sim.run(1)
    sim.sync()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        if flush_l2:
            flush_l2(s)
        e0[i].record(s)
        sim.run(1)
        e1[i].record(s)
    sim.sync()
    return sum(e0[i].elapsed_time(e1[i]) for i in range(steps))


def batch_run(local: int, steps: int, peak: float):
    """The batched form: 256 uneven realisations in one handle, one fused
    kernel per step replayed from a CUDA graph, cell width and segment size
    picked by mt_autotune; MIXED, then FP64, then the same realisations as
    separate single handles run one after another (FP64 and MIXED)."""
    import numpy as np
    import torch

    from paper_1811_05474_gb300 import mt

    dev = torch.device("cuda", local)
    ns, Ls, xs, As, Bs, (x, A, B) = batch_inputs()
    ntot = int(sum(ns))
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    fsum = torch.empty((), dtype=torch.int64, device=dev)

    def flush_l2(s):
        with torch.cuda.stream(s):
            flush.zero_()
            torch.sum(flush.view(torch.int64), dim=0, out=fsum)

    b = mt.make_batch(ns, Ls)
    out = {"workload": BATCH_WORKLOAD, "realisations": BATCH_R, "particles": ntot,
           "n_min": int(min(ns)), "n_max": int(max(ns)), "unit": "particle-steps/s"}
    res = {}
    for prec, name in ((mt.MT_MIXED, "mixed"), (mt.MT_FP64, "fp64")):
        p = mt.mt_params_init(dim=1, L=(1.0,), D_mt=D, D_rw=D, dt=DT, precision=prec, seed=2024,
                              observe_cap=16)
        t0 = time.perf_counter()
        best, tune_ms = mt.autotune(p, x, A, B, batch=b, warmup=2, steps=5, device=dev)
        tune_s = time.perf_counter() - t0
        auto = mt.mt_batch_resolve(p, b)
        sim = mt.Simulation(best, device=dev, batch=b)
        sim.upload(x, A, B)
        k = steps if prec == mt.MT_MIXED else max(10, steps // 5)
        ms = timed_steps(sim, k, 3, flush_l2)
        mt.mt_set_profiling(sim.h, True)
        prof = {}
        for _ in range(20):
            sim.run(1)
            for kn, kms in mt.mt_read_profile(sim.h):
                prof[kn] = prof.get(kn, 0.0) + kms / 20
        mt.mt_set_profiling(sim.h, False)
        sim.close()
        fused_ms = prof.get("fused_step", 0.0)
        achieved = 48.0 * ntot / (fused_ms * 1e-3) / 1e9 if fused_ms > 0 else 0.0
        res[name] = {"value": ntot * k / (ms * 1e-3), "ms_per_step": ms / k, "steps": k,
                     "kernels_ms_per_step": prof,
                     "tuned": {"cell_shift": int(best.cell_shift), "seg_target": int(best.seg_target),
                               "resolver_cell_shift": int(auto.cell_shift),
                               "resolver_seg_target": int(auto.seg_target),
                               "tuned_ms_per_step": tune_ms, "tuner_seconds": tune_s},
                     "roofline": {"bound": "hbm", "kernel": "fused_step", "achieved": achieved,
                                  "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                  "algo_bytes_per_launch": 48 * ntot}}
    out.update(res["mixed"])
    out["fp64"] = res["fp64"]
    # the same realisations one handle at a time (each its own graph)
    for prec, name in ((mt.MT_FP64, "sequential_fp64"), (mt.MT_MIXED, "sequential_mixed")):
        k = 10
        tot_ms = 0.0
        for r in range(BATCH_R):
            q = mt.mt_params_init(dim=1, n=int(ns[r]), L=(Ls[r],), D_mt=D, D_rw=D, dt=DT,
                                  precision=prec, seed=2024, realisation=r, observe_cap=16)
            sim = mt.Simulation(q, device=dev)
            sim.upload(xs[r][None, :], As[r], Bs[r])
            tot_ms += timed_steps(sim, k, 2)
            sim.close()
        out[name] = {"value": ntot * k / (tot_ms * 1e-3), "ms_per_step": tot_ms / k, "steps": k,
                     "note": "256 single handles, one after another, 10 graph steps each"}
    del flush
    return out


SERVE_WORKLOAD = "poisson_200_per_s_N_loguniform_1e3_1e6_d1_or_2_steps_100_1000_mixed"


def serve_run(local: int, count: int, pool_gb: float = 8.0, max_active: int = 16,
              chunk_steps: int = 25):
    """The serving form: `count` requests with Poisson arrivals (200/s),
    N log-uniform in [1e3, 1e6], d in {1, 2} (2-d on [0, sqrt(N) 10]^2),
    100 to 1000 steps, MIXED, submitted at their arrival times to an
    mt_server with a `pool_gb` device pool; host arrays in, host results out.
    Step latency: per resident chunk, its CUDA-event time / its steps."""
    import numpy as np
    import torch

    from paper_1811_05474_gb300 import mt, synth

    torch.cuda.set_device(local)
    reqs = synth.poisson_requests(count, rate=200.0, seed=0)
    inputs = []
    for r in reqs:
        L = (float(np.sqrt(r["n"]) * 10.0),) * 2 if r["dim"] == 2 else (float(r["n"]),)
        p = mt.mt_params_init(dim=r["dim"], n=r["n"], L=L, D_mt=D, D_rw=D, dt=DT,
                              precision=mt.MT_MIXED, seed=r["seed"], observe_cap=1)
        x = synth.uniform_positions(r["n"], L if r["dim"] == 2 else L[0], dim=r["dim"],
                                    seed=r["seed"])
        A, B = synth.uniform_masses(r["n"], seed=r["seed"])
        inputs.append((p, x, A, B, r["steps"]))
    srv = mt.Server(pool_bytes=int(pool_gb * 2 ** 30), max_active=max_active,
                    chunk_steps=chunk_steps, device=torch.device("cuda", local))
    ids = []
    t0 = time.perf_counter()
    for r, (p, x, A, B, steps) in zip(reqs, inputs):
        while time.perf_counter() - t0 < r["t"]:
            srv.poll()
        ids.append(srv.submit(p, x, A, B, steps))
        srv.poll()
    srv.drain()
    wall = time.perf_counter() - t0
    st, step_ms = srv.stats()
    infos = [srv.info(i) for i in ids]
    lat = np.array([i.t_done - i.t_submit for i in infos])
    wait = np.array([i.t_admit - i.t_submit for i in infos])
    work = sum(r["n"] * r["steps"] for r in reqs)
    span = max(i.t_done for i in infos) - min(i.t_submit for i in infos)
    srv.close()
    pct = lambda a, q: float(np.percentile(a, q))
    return {"workload": SERVE_WORKLOAD, "requests": count,
            "requests_1d": sum(1 for r in reqs if r["dim"] == 1),
            "requests_2d": sum(1 for r in reqs if r["dim"] == 2),
            "arrival_span_s": reqs[-1]["t"], "pool_bytes": int(pool_gb * 2 ** 30),
            "max_active": max_active, "chunk_steps": chunk_steps, "admission": "first fit, backfill",
            "done": int(st.done), "failed": int(st.failed),
            "p50_step_ms": pct(step_ms, 50), "p99_step_ms": pct(step_ms, 99),
            "p50_request_s": pct(lat, 50), "p99_request_s": pct(lat, 99),
            "p50_queue_s": pct(wait, 50), "p99_queue_s": pct(wait, 99),
            "particle_steps_per_s": work / span, "requests_per_s": count / span,
            "makespan_s": span, "wall_s": wall, "pool_peak_bytes": int(st.pool_peak)}


SFU_EX2_PER_SM_CLK = 16  # MUFU ex2 results per SM per clock (4 quadrants x 4)


def dense_run(local: int, steps: int = 10, sm_mhz: float | None = None, peak_gbs: float = 0.0):
    """The paper's own density (Sec. 6): N = 1e6 on [0, 5000] (200 particles
    per unit length, about 270 neighbours within the cutoff), D = 1 split,
    dt = 0.1, segregated C1/C2, MIXED, in two forms.  On the fly, each pass
    evaluates its weights (4 exponentials per unordered pair: two passes,
    both sides), reported against the SFU's ex2 rate from its unit count and
    clock.  The SPaM form (Sec. 6's stored sparse matrix) evaluates each
    pair's weight once, stores it in the band and reads it back in both
    passes, reported against HBM: the band's bytes written once and read by
    each of the two passes."""
    import torch

    from paper_1811_05474_gb300 import mt, synth

    dev = torch.device("cuda", local)
    n, Ld = 10 ** 6, 5000.0
    x = synth.uniform_positions(n, Ld, seed=9)
    c1, c2 = synth.segregated_masses(x, Ld)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    fsum = torch.empty((), dtype=torch.int64, device=dev)

    def flush_l2(s):
        with torch.cuda.stream(s):
            flush.zero_()
            torch.sum(flush.view(torch.int64), dim=0, out=fsum)

    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_mhz or 2070.0
    sfu_peak = nsm * SFU_EX2_PER_SM_CLK * mhz * 1e6
    out = {"workload": "paper_sec6_density_1d_n1e6_L5000_D1_dt0.1_mixed", "steps": steps,
           "l2": "flushed between timed steps (512 MiB write, then read)"}
    for form, stored in (("on_the_fly", 0), ("spam", 1)):
        p = mt.mt_params_init(n=n, L=(Ld,), D_mt=0.5, D_rw=0.5, dt=0.1, react=0,
                              precision=mt.MT_MIXED, seed=3, stored_p=stored)
        sim = mt.Simulation(p, device=dev)
        sim.upload(x, c1, c2)
        ms = timed_steps(sim, steps, 3, flush_l2) / steps
        npairs = mt.mt_read_pairs(sim.h, None, None, 0)
        mt.mt_set_profiling(sim.h, True)
        sim.run(1)
        kernels = mt.mt_read_profile(sim.h)
        band = int(sim.params.stored_p)
        sim.close()
        r = {"ms_per_step": ms, "particle_steps_per_s": n / (ms * 1e-3),
             "pairs_per_step": npairs, "pair_interactions_per_s": npairs / (ms * 1e-3),
             "kernels": [{"name": k, "ms": v} for k, v in kernels]}
        if stored:
            t = sum(v for k, v in kernels if k.startswith("band"))
            bb = 3.0 * 4.0 * npairs  # band: written once, read by both passes (binary32)
            r["band_per_particle"] = band
            r["exponentials_per_step"] = npairs
            r["roofline"] = {"bound": "hbm", "kernels": "band_build + band_rowsum + band_exchange",
                             "achieved": bb / (t * 1e-3) / 1e9, "peak": peak_gbs, "unit": "GB/s",
                             "frac": bb / (t * 1e-3) / 1e9 / peak_gbs if peak_gbs else None,
                             "algo_bytes_per_step": bb,
                             "note": "band bytes only (3 x 4 B per unordered pair); "
                                     "per-particle arrays add about 0.1 GB"}
        else:
            exps = 4.0 * npairs
            r["exponentials_per_step"] = exps
            r["roofline"] = {"bound": "sfu", "achieved": exps / (ms * 1e-3), "peak": sfu_peak,
                             "unit": "exp/s", "frac": exps / (ms * 1e-3) / sfu_peak,
                             "peak_kind": f"derived: {nsm} SMs x {SFU_EX2_PER_SM_CLK} ex2/clk x "
                                          f"{mhz:.0f} MHz"}
        out[form] = r
    del flush
    return out


def species_run(local: int, steps: int = 50, counts=(2, 3, 4, 6, 8)):
    """Cost against the species count (Sec. 2: linear in it) at the N = 1e6
    workload's shape (1-d, [0, 1e6], MIXED): two species run the one-kernel
    step; more run the multi-kernel pipeline, whose row sums and A/B pass
    are shared and each further pair of species adds one exchange pass with
    the same weights."""
    import torch

    from paper_1811_05474_gb300 import mt, synth

    dev = torch.device("cuda", local)
    n, Ld = 10 ** 6, 1.0e6
    x = synth.uniform_positions(n, Ld, seed=13)
    A, B = synth.uniform_masses(n, seed=13)
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    fsum = torch.empty((), dtype=torch.int64, device=dev)

    def flush_l2(s):
        with torch.cuda.stream(s):
            flush.zero_()
            torch.sum(flush.view(torch.int64), dim=0, out=fsum)

    rows = []
    for S in counts:
        p = mt.mt_params_init(n=n, L=(Ld,), v=(0.5,), precision=mt.MT_MIXED, species=S, seed=5)
        sim = mt.Simulation(p, device=dev)
        sim.upload(x, A, B)
        for s in range(2, S):
            sim.set_species(s, A if s % 2 == 0 else B)
        ms = timed_steps(sim, steps, 3, flush_l2) / steps
        mt.mt_set_profiling(sim.h, True)
        sim.run(1)
        kernels = mt.mt_read_profile(sim.h)
        path = "one-kernel step" if sim.params.seg_target > 0 else "multi-kernel pipeline"
        sim.close()
        rows.append({"species": S, "path": path, "ms_per_step": ms,
                     "particle_steps_per_s": n / (ms * 1e-3),
                     "kernels": [{"name": k, "ms": v} for k, v in kernels]})
    return {"workload": "1d_uniform_n1e6_L1e6_v0.5_D0.1_dt1_cutoff3sigma_mixed", "steps": steps,
            "l2": "flushed between timed steps (512 MiB write, then read)",
            "per_species_count": rows}


def brute_run(local: int, n: int = 100000, steps: int = 2, sm_mhz: float | None = None):
    """The all-pairs forms at the N = 1e5 workload's shape (1-d, [0, 1e5],
    MIXED): the full matrix (every pair's exponential, the paper's
    reference) and the cutoff brute force (every pair tested).  Per pass:
    kernel time, pairs per second, and for the full matrix the exponentials
    per second against the SFU's ex2 rate."""
    import torch

    from paper_1811_05474_gb300 import mt, synth

    dev = torch.device("cuda", local)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_mhz or 2070.0
    peak = nsm * SFU_EX2_PER_SM_CLK * mhz * 1e6
    x = synth.uniform_positions(n, float(n), seed=0)
    A, B = synth.uniform_masses(n, seed=0)
    out = {"workload": f"1d_uniform_n{n}_L{n}_D0.1_dt1_mixed", "steps": steps}
    for name, search in (("full_matrix", mt.MT_SEARCH_FULL), ("brute_cutoff", mt.MT_SEARCH_BRUTE)):
        p = mt.mt_params_init(n=n, L=(float(n),), search=search, precision=mt.MT_MIXED, seed=1)
        sim = mt.Simulation(p, device=dev)
        sim.upload(x, A, B)
        sim.run(1)
        sim.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.run(steps)
        e1.record(sim.stream)
        sim.sync()
        ms = e0.elapsed_time(e1) / steps
        mt.mt_set_profiling(sim.h, True)
        sim.run(1)
        prof = dict(mt.mt_read_profile(sim.h))
        sim.close()
        pairs = float(n) * n
        rk, xk = ("rowsum_full", "exchange_full") if search == mt.MT_SEARCH_FULL else \
                 ("rowsum_brute", "exchange_brute")
        r = {"ms_per_step": ms, "pair_evaluations_per_step": 2 * pairs,
             "pairs_per_s": 2 * pairs / (ms * 1e-3),
             "rowsum_ms": prof.get(rk), "exchange_ms": prof.get(xk)}
        if search == mt.MT_SEARCH_FULL:
            # one exponential per ordered pair in each pass (self included)
            rate = pairs / (prof[rk] * 1e-3)
            r["rowsum_roofline"] = {"bound": "sfu", "achieved": rate, "peak": peak, "unit": "exp/s",
                                    "frac": rate / peak,
                                    "peak_kind": f"derived: {nsm} SMs x {SFU_EX2_PER_SM_CLK} ex2/clk x {mhz:.0f} MHz"}
            rate = pairs / (prof[xk] * 1e-3)
            r["exchange_roofline"] = {"bound": "sfu", "achieved": rate, "peak": peak, "unit": "exp/s",
                                      "frac": rate / peak}
        out[name] = r
    return out


def accuracy_run(local: int):
    """The paper's accuracy test problem (Sec. 3): 75 realisations at each
    N in {500, 1000, 2500, 5000, 10000, 25000}, all in one batch handle,
    100 steps of dt = 0.1 on [0, 50] with D = 1 split between transfer and
    walk, C1 and C2 transferred without reaction; error of C1 against the
    exact step solution at t = 10 (mean RMSE per N), fitted D, and the
    conservation of C1.  FP64 and MIXED with symmetric normalisation, and
    MIXED with the literal row normalisation (which does not conserve)."""
    import numpy as np
    import torch

    from paper_1811_05474_gb300 import accuracy as acc
    from paper_1811_05474_gb300 import mt

    dev = torch.device("cuda", local)
    ns, ins = [], []
    for n in acc.SIZES:
        for r in range(acc.REALISATIONS):
            ns.append(n)
            ins.append(acc.inputs(n, 100000 * (1 + acc.SIZES.index(n)) + r))
    x = np.concatenate([i[0][0] for i in ins])[None, :]
    c1 = np.concatenate([i[1] for i in ins])
    c2 = np.concatenate([i[2] for i in ins])
    b = mt.make_batch(ns, [acc.L] * len(ns))
    kw = acc.params_kw()
    out = {"workload": "paper_sec3_L50_D1_dt0.1_t10_segregated", "realisations_per_N": acc.REALISATIONS,
           "sizes": list(acc.SIZES), "particles": int(sum(ns)), "steps": acc.STEPS}
    for name, prec, norm in (("fp64_sym", mt.MT_FP64, mt.MT_NORM_SYM),
                             ("mixed_sym", mt.MT_MIXED, mt.MT_NORM_SYM),
                             ("mixed_row", mt.MT_MIXED, mt.MT_NORM_ROW)):
        p = mt.mt_params_init(dim=1, L=(1.0,), D_mt=kw["D_mt"], D_rw=kw["D_rw"], dt=kw["dt"],
                              react=0, precision=prec, norm=norm, seed=2024)
        sim = mt.Simulation(p, device=dev, batch=b)
        sim.upload(x, c1, c2)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.run(acc.STEPS)
        e1.record(sim.stream)
        sim.sync()
        ms = e0.elapsed_time(e1)
        xs = np.split(sim.positions()[0], np.cumsum(ns)[:-1])
        g1 = np.split(sim.masses()[0], np.cumsum(ns)[:-1])
        sim.close()
        per = {}
        k = 0
        for n in acc.SIZES:
            R = acc.REALISATIONS
            e = [acc.rmse(xs[k + r], g1[k + r]) for r in range(R)]
            cons = max(abs(g1[k + r].sum() - ins[k + r][1].sum()) for r in range(R))
            per[str(n)] = {"rmse_mean": float(np.mean(e)), "rmse_sd": float(np.std(e)),
                           "fitted_D": acc.fitted_d(xs[k:k + R], g1[k:k + R]),
                           "max_abs_change_sum_C1": float(cons)}
            k += R
        out[name] = {"per_N": per, "gpu_ms": ms,
                     "particle_steps_per_s": sum(ns) * acc.STEPS / (ms * 1e-3)}
    return out


def precision_report(local: int, steps: int):
    """MIXED and double-binary32 against the binary64 GPU path on the
    headline workload: all run `steps` steps from the same state with the
    same random walk (positions are identical integers), then masses and the
    mean-A series are compared.  (Each path's error against the CPU oracle
    is asserted by the parity tests: 1e-12 binary64, 1e-6 the mixed forms.)"""
    import numpy as np
    import torch

    from paper_1811_05474_gb300 import mt, synth

    dev = torch.device("cuda", local)
    x = synth.uniform_positions(N, L, seed=5)
    A0, B0 = synth.uniform_masses(N, seed=5)
    rel = lambda g, o: float(np.max(np.abs(g - o) / np.maximum(np.abs(o), 0.5)))
    res = {}
    for name in ("fp64", "mixed", "df32"):
        p = mt.mt_params_init(n=N, L=(L,), v=(V, 0.0), D_mt=D, D_rw=D, dt=DT,
                              precision=prec_code(name), seed=99, observe_cap=steps)
        sim = mt.Simulation(p, device=dev)
        sim.upload(x, A0, B0)
        sim.run(steps)
        res[name] = (sim.ticks(), *sim.masses(), sim.observables())
        sim.close()
    X64, a64, b64, o64 = res["fp64"]
    d0 = float(np.sum(A0 - B0))
    out = {"workload": WORKLOAD, "steps": steps,
           "relative_to": "max(|m_fp64|, 0.5) per particle (0.5 = mean initial mass)",
           "sum_A_plus_B_initial": float(np.sum(A0 + B0)),
           "fp64": {"mean_A_last": float(o64[-1, 3]),
                    "sum_A_minus_B_drift": float(abs(o64[-1, 2] - d0))}}
    for name in ("mixed", "df32"):
        X, a, b, o = res[name]
        out[name] = {"positions_identical": bool(np.array_equal(X64, X)),
                     "vs_fp64_max_rel_err_A": rel(a, a64), "vs_fp64_max_rel_err_B": rel(b, b64),
                     "mean_A_series_max_abs_diff": float(np.max(np.abs(o[:, 3] - o64[:, 3]))),
                     "mean_A_last": float(o[-1, 3]),
                     "sum_A_minus_B_drift": float(abs(o[-1, 2] - d0))}
    return out


def make_flush(dev):
    """A function that flushes L2 on a stream: write 512 MiB, then read it
    back so the lines left are clean."""
    import torch

    buf = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    acc = torch.empty((), dtype=torch.int64, device=dev)

    def flush_l2(s):
        with torch.cuda.stream(s):
            buf.zero_()
            torch.sum(buf.view(torch.int64), dim=0, out=acc)
    return flush_l2


def workloads_run(local: int, flush_l2):
    """The two smaller workloads, timed like the headline (graph steps,
    events on the simulation's stream, L2 flushed between steps).
    N = 1e3 uniform on [0, 1e3], 100 steps, binary64: the cell list, the
    cutoff brute force (every pair tested) and the full matrix (every
    pair's weight, the paper's reference).  N = 1e5 uniform on [0, 1e5],
    1000 steps, no advection: binary64, MIXED and double-binary32.
    pair-interactions/s counts the unordered pairs within the cutoff (the
    full matrix: every unordered pair it evaluates, labelled as such)."""
    import torch

    from paper_1811_05474_gb300 import mt, synth

    dev = torch.device("cuda", local)
    out = {}
    n1, steps1 = 1000, 100
    x1 = synth.uniform_positions(n1, 1000.0, seed=0)
    A1, B1 = synth.uniform_masses(n1, seed=0)
    w1 = {"workload": "1d_uniform_n1e3_L1e3_D0.1_dt1_cutoff3sigma_fp64", "steps": steps1}
    for name, search in (("cell", mt.MT_SEARCH_CELL), ("brute", mt.MT_SEARCH_BRUTE),
                         ("full", mt.MT_SEARCH_FULL)):
        p = mt.mt_params_init(n=n1, L=(1000.0,), D_mt=D, D_rw=D, dt=DT, search=search,
                              precision=mt.MT_FP64, seed=0)
        sim = mt.Simulation(p, device=dev)
        sim.upload(x1, A1, B1)
        ms = timed_steps(sim, steps1, 3, flush_l2)
        if search == mt.MT_SEARCH_FULL:
            pairs, label = n1 * (n1 - 1) // 2, "all unordered pairs (evaluated)"
        else:
            pairs, label = mt.mt_read_pairs(sim.h, None, None, 0), "unordered pairs within the cutoff"
        sim.close()
        w1[name] = {"value": n1 * steps1 / (ms * 1e-3), "unit": "particle-steps/s",
                    "ms_per_step": ms / steps1, "pairs_per_step": int(pairs), "pairs": label,
                    "pair_interactions_per_s": pairs * steps1 / (ms * 1e-3)}
    out["n1e3"] = w1
    n2, steps2 = 10 ** 5, 1000
    x2 = synth.uniform_positions(n2, 1e5, seed=0)
    A2, B2 = synth.uniform_masses(n2, seed=0)
    w2 = {"workload": "1d_uniform_n1e5_L1e5_D0.1_dt1_cutoff3sigma", "steps": steps2,
          "search": "cell list (one-kernel step)"}
    for name in ("fp64", "mixed", "df32"):
        p = mt.mt_params_init(n=n2, L=(1e5,), D_mt=D, D_rw=D, dt=DT, precision=prec_code(name),
                              seed=0)
        sim = mt.Simulation(p, device=dev)
        sim.upload(x2, A2, B2)
        ms = timed_steps(sim, steps2, 3, flush_l2)
        pairs = mt.mt_read_pairs(sim.h, None, None, 0)
        sim.close()
        w2[name] = {"value": n2 * steps2 / (ms * 1e-3), "unit": "particle-steps/s",
                    "ms_per_step": ms / steps2, "dtype": DTYPES[name],
                    "pair_interactions_per_s": pairs * steps2 / (ms * 1e-3)}
    out["n1e5"] = w2
    return out


def cpu_info():
    """Host core count and CPU model (for the CPU baseline's record)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def cpu_baselines(n: int = N, steps: int = 10):
    """The CPU oracle on the host: (i) the sorted-window step (Sec. 2.1's
    fixed-radius search without a tree) on the headline workload, on one
    core and on all cores (the oracle's per-particle loops on OpenMP
    threads; its sort stays on one core), `steps` steps each, per-step time
    extrapolated to the 1000-step run; (ii) the full-matrix transfer (every
    pair, the paper's reference): N = 1e3 for 100 steps, and N = 1e4 for one
    step, whose per-pair rate extrapolates one step at N = 1e5 (1e10
    pairs), stated as extrapolated."""
    import oracle as O
    from paper_1811_05474_gb300 import synth

    info = cpu_info()
    cores = info["nproc"] or 1
    single, secs1 = cpu_oracle_rate(n, steps, seed=0)
    used = O.set_threads(cores)
    try:
        multi, secsm = cpu_oracle_rate(n, steps, seed=0)
    finally:
        O.set_threads(1)
    full = {}
    for nf, sf in ((1000, 100), (10000, 1)):
        p = O.params(L=(float(nf),), D_mt=D, D_rw=D, dt=DT, frac_bits=29, search=O.SEARCH_FULL)
        X = O.quantize(synth.uniform_positions(nf, float(nf), seed=0), 29)
        A, B = synth.uniform_masses(nf, seed=0)
        xi = synth.normals(sf, 1, nf, seed=1)
        t0 = time.perf_counter()
        for k in range(sf):
            X, A, B = O.step(p, X, xi[k], A, B)
        dt = time.perf_counter() - t0
        full[f"n{nf}"] = {"steps": sf, "seconds": dt, "particle_steps_per_s": nf * sf / dt,
                          "pair_evaluations_per_s": 2.0 * nf * nf * sf / dt}
    per_pair = full["n10000"]["seconds"] / (2.0 * 10000 * 10000)
    full["n1e5_one_step_seconds_extrapolated"] = per_pair * 2.0 * 1e5 * 1e5
    return {"value": single, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of the full {n}-particle workload, single thread, "
                      f"sorted-window search ({secs1:.1f} s; 1000 steps extrapolate to "
                      f"{secs1 * 1000 / steps:.0f} s)",
            **info,
            "all_cores": {"value": multi, "unit": "particle-steps/s", "cores": used,
                          "kind": "oracle",
                          "sample": f"{steps} steps, per-particle loops on {used} OpenMP threads "
                                    f"({secsm:.1f} s; 1000 steps extrapolate to "
                                    f"{secsm * 1000 / steps:.0f} s)"},
            "full_matrix": full}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def load_issue(kernel: str, launch_ms: float, sm_mhz: float | None):
    """The kernel's instruction-issue rate: warp instructions per launch from
    the committed ncu capture (if taken on the kernel's current sources) over
    the event-timed launch duration, against the issue peak of one warp
    instruction per clock per SM sub-partition (4 per SM)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            k = json.load(f)["kernels"][kernel]
        if k["source_hash"] != source_hash(k["sources"]):
            return None
        inst = float(k["warp_instructions"])
    except (OSError, ValueError, KeyError, TypeError):
        return None
    import torch

    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or 2070.0
    achieved = inst / (launch_ms * 1e-3)
    peak = nsm * 4 * mhz * 1e6
    return {"bound": "issue", "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "warp instructions/s", "frac": achieved / peak,
            "warp_instructions_per_launch": inst,
            "peak_kind": f"derived: {nsm} SMs x 4 issue slots/clk x {mhz:.0f} MHz"}


def load_traffic(kernel: str):
    """dram bytes per launch from a committed ncu summary, if it was taken on
    the kernel's current sources (the hash of its translation unit)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        k = t["kernels"][kernel]
        if k["source_hash"] != source_hash(k["sources"]):
            return None
        return float(k["bytes"])
    except (OSError, ValueError, KeyError, TypeError):
        return None


def run_ncu(args):
    """Minimal run for ncu: the workload's state, W steps replayed from the
    CUDA graph, then K directly launched steps (profiling mode)."""
    import torch

    from paper_1811_05474_gb300 import mt, synth

    n = args.n
    prec = prec_code(args.precision)
    if args.ncu_search.startswith("dense"):
        # the paper's density (200 per unit length, D = 1 split, dt = 0.1)
        Ln = float(n) * 5000.0 / 1e6
        p = mt.mt_params_init(n=n, L=(Ln,), D_mt=0.5, D_rw=0.5, dt=0.1, react=0, precision=prec,
                              seed=3, stored_p=1 if args.ncu_search == "dense_spam" else 0)
        x = synth.uniform_positions(n, Ln, seed=9)
        sim = mt.Simulation(p)
        sim.upload(x, *synth.segregated_masses(x, Ln))
    else:
        Ln = float(n) * (L / N)
        search = mt.MT_SEARCH_FULL if args.ncu_search == "full" else mt.MT_SEARCH_CELL
        p = mt.mt_params_init(n=n, L=(Ln,), v=(V, 0.0), D_mt=D, D_rw=D, dt=DT, precision=prec,
                              search=search, seed=2024, observe_cap=args.steps + args.warmup)
        sim = mt.Simulation(p)
        sim.upload(synth.uniform_positions(n, Ln, seed=0), *synth.uniform_masses(n, seed=0))
    sim.run(args.warmup)
    # direct launches (ncu does not profile kernels inside graphs that
    # contain conditional nodes)
    mt.mt_set_profiling(sim.h, True)
    sim.run(args.steps)
    sim.sync()
    torch.cuda.synchronize()
    return 0


def compact_kernels(kernels):
    ksum = sum(k["ms_per_step"] for k in kernels)
    return [{"name": k["name"], "ms": round(k["ms"], 5), "launches_per_step": k["launches_per_step"],
             "share": round(k["ms_per_step"] / ksum, 4) if ksum else None} for k in kernels]


def fp64_ops_per_step(npairs: int, n: int) -> float:
    """Binary64 pipe instructions (per lane) the step needs with binary64
    masses (MIXED and FP64), the unit of the measured FMA rate: per ordered
    pair within the cutoff and species, the difference M_j - M_i and one
    fused multiply-add of it with P into the accumulator (2 x 2 species x 2
    orders per unordered pair); per particle and species the update (one
    fused multiply-add), per particle the reaction (a comparison and one
    subtraction: the smaller mass becomes exactly 0) and the walk's product
    (1)."""
    return 8.0 * npairs + 5.0 * n


def alu_roofline(r, n: int, dfma_peak: float):
    """The transfer phase against the binary64 pipe: the first tier and the
    predicted-segment kernel run side by side in the step's graph, so the
    phase lasts the longer of the two (per step, averaged over the sampled
    steps of the run); achieved = the step's algorithmic binary64 operations
    over that time; peak = the measured binary64 FMA rate (lane operations
    per second)."""
    t = r.get("phase_ms") or 0.0
    if t <= 0:
        return None
    ops = fp64_ops_per_step(r["npairs"], n)
    achieved = ops / (t * 1e-3)
    return {"bound": "alu", "kernel": "fused_step || fused_pred (concurrent)", "achieved": achieved,
            "peak": dfma_peak, "unit": "binary64 instr/s", "frac": achieved / dfma_peak,
            "peak_kind": "measured (mt_probe_rate: binary64 FMA, lane operations per second)",
            "algo_ops_per_launch": ops, "launch_ms": t,
            "algo": "8 per unordered pair within the cutoff + 5 per particle "
                    "(an FMA counts once, as in the peak)"}


def state_kernel(kernels):
    """The kernel whose launch reads and writes the whole state (48 B per
    particle): the first tier on the one-kernel path, else the longest."""
    for k in kernels:
        if k["name"] == "fused_step":
            return k
    return max(kernels, key=lambda k: k["ms_per_step"])


def variant_object(r, steps: int, name: str, peak: float, peak_kind: str, clocks, exp_peak,
                   dfma_peak=None):
    """A precision's own result on the headline workload: rate, its
    state kernel against HBM (48 B per particle-step) and, with binary64
    weights, the transfer phase against the measured binary64 exponential
    rate (one exponential per unordered pair within the cutoff, the method's
    minimum)."""
    dom = state_kernel(r["kernels"])
    achieved = ALGO_BYTES.get(dom["name"], 48) * N / (dom["ms"] * 1e-3) / 1e9
    obj = {"value": N * steps / (r["total_ms"] * 1e-3), "unit": "particle-steps/s",
           "ms_per_step": r["total_ms"] / steps, "steps": steps, "dtype": DTYPES[name],
           "pair_interactions_per_s": r["npairs"] * steps / (r["total_ms"] * 1e-3),
           "roofline": {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak,
                        "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                        "algo_bytes_per_launch": ALGO_BYTES.get(dom["name"], 48) * N,
                        "traffic": load_traffic(dom["name"] + ("" if name == "mixed" else "_" + name))},
           "clocks": clocks, "kernels": compact_kernels(r["kernels"])}
    if name in ("fp64", "mixed") and dfma_peak:
        obj["alu_roofline"] = alu_roofline(r, N, dfma_peak)
    if name == "fp64" and exp_peak and r.get("phase_ms"):
        rate = r["npairs"] / (r["phase_ms"] * 1e-3)
        obj["exp_roofline"] = {"bound": "alu", "kernel": "fused_step || fused_pred (concurrent)",
                               "achieved": rate,
                               "peak": exp_peak, "unit": "binary64 exp/s", "frac": rate / exp_peak,
                               "peak_kind": "measured (mt_probe_rate: the weights' binary64 "
                                            "exp(-t), exp_neg)",
                               "algo": "one exponential per unordered pair within the cutoff"}
    return obj


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu:
        return run_ncu(args)
    import torch

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
    from paper_1811_05474_gb300 import build as _b

    if rank == 0:
        _b.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_1811_05474_gb300 import mt

    dev = torch.device("cuda", local)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    sampler.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    main_run = gpu_run(args, args.precision, args.steps, max(args.warmup, 3), local, rank, sampler)
    total_ms = main_run["total_ms"]
    if ws > 1:
        total_ms = rank_reduce([total_ms], "max", device="cuda")[0]
        torch.distributed.barrier()
    peak, peak_kind = load_peaks()
    probes = None
    if rank == 0:
        probes = {"binary64_fma_per_s": mt.mt_probe_rate(mt.PROBE_DFMA, dev),
                  "binary32_fma_per_s": mt.mt_probe_rate(mt.PROBE_FFMA, dev),
                  "binary32_fast_exp_per_s": mt.mt_probe_rate(mt.PROBE_EXPF, dev),
                  "binary64_exp_per_s": mt.mt_probe_rate(mt.PROBE_EXP, dev),
                  "binary64_exp_neg_per_s": mt.mt_probe_rate(mt.PROBE_EXP_NEG, dev),
                  "how": "mt_probe_rate: 8 independent chains per thread, 8 CTAs x 256 threads "
                         "per SM, fastest of 3 event-timed launches"}
    variants = {}
    if not args.no_fp64 and rank == 0:
        for name in ("fp64", "mixed", "df32"):
            if name != args.precision:
                k = args.steps  # the same steps as the headline (the wall layer grows)
                variants[name] = (gpu_run(args, name, k, 3, local, rank, None), k)
    flush_l2 = make_flush(dev)
    workloads = None
    if not args.no_workloads and rank == 0:
        workloads = workloads_run(local, flush_l2)
    e2e = e2e_run(args.steps, local, rank, args.precision)
    batched = None
    if not args.no_batch and rank == 0:
        batched = batch_run(local, args.steps, peak)
    precision = None
    if not args.no_precision and rank == 0:
        precision = precision_report(local, args.steps)
    serving = None
    if not args.no_serve and rank == 0:
        serving = serve_run(local, args.serve_requests)
    accuracy = None
    if not args.no_accuracy and rank == 0:
        accuracy = accuracy_run(local)
    sm_now = None
    brute = None
    if not args.no_brute and rank == 0:
        brute = brute_run(local, sm_mhz=sm_now)
    dense = None
    if not args.no_dense and rank == 0:
        dense = dense_run(local, sm_mhz=sm_now, peak_gbs=peak)
    species = None
    if not args.no_species and rank == 0:
        species = species_run(local)
    sampler.stop()
    clocks = sampler.summary(main_run["t0"], main_run["t1"])
    if ws > 1:
        # the slowest replica's rate times the replicas
        e2e["value"] = rank_reduce([e2e["value"]], "min", device="cuda")[0] * ws
    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    K = args.steps
    value = replicas_value(N, K, total_ms, ws)
    ms_step = total_ms / K
    kernels = main_run["kernels"]
    dom = state_kernel(kernels)
    dom_bytes = ALGO_BYTES.get(dom["name"], 0) * N
    achieved = dom_bytes / (dom["ms"] * 1e-3) / 1e9 if dom["ms"] > 0 else 0.0
    step_bytes = ALGO_BYTES["step"] * N
    path_achieved = step_bytes / (ms_step * 1e-3) / 1e9
    exp_peak = probes["binary64_exp_neg_per_s"] if probes else None
    dfma_peak = probes["binary64_fma_per_s"] if probes else None
    objs = {name: variant_object(r, k, name, peak, peak_kind,
                                 sampler.summary(r["t0"], r["t1"]), exp_peak, dfma_peak)
            for name, (r, k) in variants.items()}
    cpu = None
    if ws == 1 and not args.no_cpu:
        cpu = cpu_baselines()
    traffic_key = dom["name"] + ("" if args.precision == "mixed" else "_" + args.precision)
    # the headline kernel's roofline: binary64 masses make the transfer
    # binary64-bound on this GPU (MIXED and FP64); the double-binary32 form
    # is compared with HBM
    hbm_roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                    "algo_bytes_per_launch": dom_bytes, "traffic": load_traffic(traffic_key)}
    roofline = hbm_roofline
    if args.precision in ("mixed", "fp64") and dfma_peak:
        alu = alu_roofline(main_run, N, dfma_peak)
        if alu:
            alu["traffic"] = hbm_roofline["traffic"]
            roofline = alu
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
        "n_gpus": ws, "steps": K, "warmup": max(args.warmup, 3), "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic: seeded uniform positions and U[0,1) masses",
        "config": config_dict(args.precision),
        "pair_interactions_per_s": ws * main_run["npairs"] * K / (total_ms * 1e-3),
        "pairs_per_step": main_run["npairs"],
        "roofline": roofline,
        "hbm_roofline": hbm_roofline,
        "gpu_launches": int(round(K * main_run["launches_per_step"])),
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "fp64": objs.get("fp64"),
        "mixed": objs.get("mixed"),
        "mixed_df32": objs.get("df32"),
        "workloads": workloads,
        "path_roofline": {"bound": "hbm", "achieved": path_achieved, "peak": peak, "unit": "GB/s",
                          "frac": path_achieved / peak, "algo_bytes_per_step": step_bytes},
        "issue_roofline": load_issue(traffic_key, dom["ms"], clocks.get("sm_mhz") if clocks else None),
        "kernels": compact_kernels(kernels),
        "probes": probes,
        "precision": precision,
        "batched": batched,
        "serving": serving,
        "paper_density": dense,
        "brute_force": brute,
        "accuracy": accuracy,
        "species": species,
        "mean_A_last_step": main_run["mean_A_last"],
    }
    if args.detail:
        with open(args.detail, "w") as f:
            json.dump(line, f, indent=1)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
