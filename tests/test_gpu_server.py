"""The request server: admission by device footprint, overlapping resident
requests, and results that are the same alone and in the mix."""
import numpy as np
import pytest

from paper_1811_05474_gb300 import mt, synth

pytestmark = pytest.mark.gpu


def request(n, dim, seed, precision=mt.MT_MIXED, observe_cap=0):
    L = (float(np.sqrt(n) * 10.0),) * 2 if dim == 2 else (float(n),)
    p = mt.mt_params_init(dim=dim, n=n, L=L, precision=precision, seed=seed, realisation=seed,
                          observe_cap=observe_cap)
    x = synth.uniform_positions(n, L if dim == 2 else L[0], dim=dim, seed=seed)
    A, B = synth.uniform_masses(n, seed=seed)
    return p, x, A, B


def alone(p, x, A, B, steps):
    sim = mt.Simulation(p)
    sim.upload(x, A, B)
    sim.run(steps)
    out = (*sim.masses(), sim.observables())
    sim.close()
    return out


MIX = [  # (n, dim, steps, precision)
    (1200, 1, 37, mt.MT_MIXED), (20000, 1, 23, mt.MT_MIXED), (900, 2, 18, mt.MT_MIXED),
    (5000, 2, 30, mt.MT_FP64), (333, 1, 51, mt.MT_FP64), (60000, 1, 12, mt.MT_MIXED),
    (2500, 2, 9, mt.MT_MIXED), (7000, 1, 44, mt.MT_FP64),
]


def test_server_results_equal_alone_runs():
    reqs = [request(n, d, 40 + i, prec, observe_cap=steps) + (steps,)
            for i, (n, d, steps, prec) in enumerate(MIX)]
    foot = [mt.mt_server_footprint(r[0]) for r in reqs]
    # room for about three of the larger requests at once
    srv = mt.Server(pool_bytes=3 * max(foot) + 4096, max_active=3, chunk_steps=7)
    ids = []
    for i, (p, x, A, B, steps) in enumerate(reqs):
        ids.append(srv.submit(p, x, A, B, steps))
        if i % 3 == 2:  # later arrivals join while others are resident
            for _ in range(5):
                srv.poll()
    srv.drain()
    st, step_ms = srv.stats()
    assert st.done == len(reqs) and st.failed == 0 and st.running == 0 and st.queued == 0
    assert st.pool_peak <= srv.pool.numel() and st.pool_used == 0
    assert len(step_ms) > 0 and np.all(step_ms > 0)
    for rid, (p, x, A, B, steps) in zip(ids, reqs):
        info = srv.info(rid)
        assert info.state == mt.MT_REQ_DONE and info.steps_done == steps
        assert info.t_submit <= info.t_admit <= info.t_done and info.gpu_ms > 0
        gA, gB, gobs = srv.result(rid)
        aA, aB, aobs = alone(p, x, A, B, steps)
        assert np.array_equal(gA, aA) and np.array_equal(gB, aB), f"request {rid}"
        assert np.array_equal(gobs, aobs)
        srv.release(rid)
    srv.close()


def test_server_admits_by_footprint_and_keeps_order_without_backfill():
    small = [request(1000, 1, 70 + i) for i in range(4)]
    big = request(200000, 1, 80)
    f_small = mt.mt_server_footprint(small[0][0])
    f_big = mt.mt_server_footprint(big[0])
    assert f_big > 4 * f_small
    pool = f_big + f_small  # the big one leaves room for one small one
    for backfill in (False, True):
        srv = mt.Server(pool_bytes=pool, max_active=4, chunk_steps=5, backfill=backfill)
        order = [small[0], big, small[1], small[2], small[3]]
        ids = [srv.submit(p, x, A, B, 20) for (p, x, A, B) in order]
        srv.drain()
        st, _ = srv.stats()
        assert st.done == 5 and st.pool_peak <= pool
        t_admit = [srv.info(i).t_admit for i in ids]
        if not backfill:
            assert t_admit == sorted(t_admit)  # arrival order
        srv.close()


def test_server_refuses_bad_requests_and_handles_zero_steps():
    p, x, A, B = request(500, 1, 90)
    srv = mt.Server(pool_bytes=mt.mt_server_footprint(p) + 256, max_active=2, chunk_steps=4)
    bad = mt.mt_params_init(dim=3, n=10)
    with pytest.raises(mt.MtError) as e:
        srv.submit(bad, np.zeros(30), np.zeros(10), np.zeros(10), 5)
    assert e.value.status == mt.MT_ERR_INVALID
    p2, x2, A2, B2 = request(100000, 1, 91)
    with pytest.raises(mt.MtError) as e:
        srv.submit(p2, x2, A2, B2, 5)
    assert e.value.status == mt.MT_ERR_WORKSPACE
    # zero steps returns the uploaded masses (exactly in FP64; MIXED keeps
    # them as double-binary32)
    p64, x64, A64, B64 = request(500, 1, 92, precision=mt.MT_FP64)
    rid = srv.submit(p64, x64, A64, B64, 0)
    srv.drain()
    gA, gB, _ = srv.result(rid)
    assert np.array_equal(gA, A64) and np.array_equal(gB, B64)
    with pytest.raises(mt.MtError):
        srv.result(rid + 100)
    srv.close()


def test_server_poisson_mix_matches_alone_on_sampled_requests():
    """The serving workload's request mix at reduced sizes (N up to 3e4, 20
    to 60 steps): Poisson arrival order, 1-d and 2-d, MIXED; every request
    finishes and three sampled ones equal their alone runs."""
    reqs = synth.poisson_requests(24, rate=200.0, seed=3, n_hi=3e4, steps_lo=20, steps_hi=60)
    srv = mt.Server(pool_bytes=512 * 2 ** 20, max_active=8, chunk_steps=10)
    ids = []
    inputs = []
    for r in reqs:
        p, x, A, B = request(r["n"], r["dim"], r["seed"])
        inputs.append((p, x, A, B, r["steps"]))
        ids.append(srv.submit(p, x, A, B, r["steps"]))
        srv.poll()
    srv.drain()
    st, _ = srv.stats()
    assert st.done == len(reqs) and st.failed == 0
    for k in (0, len(reqs) // 2, len(reqs) - 1):
        p, x, A, B, steps = inputs[k]
        gA, gB, _ = srv.result(ids[k])
        aA, aB, _ = alone(p, x, A, B, steps)
        assert np.array_equal(gA, aA) and np.array_equal(gB, aB)
    srv.close()


def test_served_requests_equal_the_oracle():
    """Served results against the CPU oracle, not only against the library
    run alone.  The requests have no random walk (D_rw = 0) and a constant
    drift, so every position is fixed by Eq. 2 and the walls alone and the
    oracle reproduces each whole served run: 1-d and 2-d, two and three
    species, all three precisions, served side by side with chunks that
    interleave on the device.  Positions are compared through the masses
    (a moved particle would change its neighbours), masses per particle to
    1e-12 (FP64) or 1e-6 (mixed forms) relative to max(|m|, 0.5)."""
    import oracle as O

    from .test_gpu_parity import TOL, assert_masses
    from .test_oracle_species import oracle_step_species, species_masses

    specs = [  # (n, dim, species, steps, precision, v)
        (3000, 1, 2, 25, mt.MT_FP64, (0.3, 0.0)),
        (5000, 1, 3, 20, mt.MT_MIXED, (-0.4, 0.0)),
        (1600, 2, 2, 12, mt.MT_MIXED, (0.25, -0.15)),
        (2500, 1, 2, 30, mt.MT_MIXED_DF32, (0.5, 0.0)),
        (900, 2, 3, 10, mt.MT_FP64, (0.0, 0.2)),
    ]
    srv = mt.Server(pool_bytes=2 ** 28, max_active=3, chunk_steps=4)
    runs = []
    for i, (n, dim, S, steps, prec, v) in enumerate(specs):
        L = (float(np.sqrt(n) * 10.0),) * 2 if dim == 2 else (float(n),)
        p = mt.mt_params_init(dim=dim, n=n, L=L, v=v, D_rw=0.0, precision=prec, species=S,
                              seed=200 + i)
        x = synth.uniform_positions(n, L if dim == 2 else L[0], dim=dim, seed=200 + i)
        Ms = species_masses(n, S, seed=300 + i)
        rid = srv.submit_species(p, x, Ms, steps) if S > 2 else srv.submit(p, x, *Ms, steps)
        runs.append((rid, mt.mt_resolve(p), x, Ms, steps))
        srv.poll()
    srv.drain()
    for rid, r, x, Ms, steps in runs:
        po = O.params(dim=r.dim, frac_bits=r.frac_bits, L=tuple(r.L), v=tuple(r.v), D_mt=r.D_mt,
                      D_rw=0.0, dt=r.dt, smax=r.cutoff, norm=r.norm, react=r.react)
        X = O.quantize(np.asarray(x).reshape(r.dim, -1), int(r.frac_bits))
        xi = np.zeros((r.dim, r.n), dtype=np.float32)
        cur = [np.array(m, dtype=np.float64) for m in Ms]
        for _ in range(steps):
            X, cur = oracle_step_species(po, X, xi, cur)
        tol = TOL[int(r.precision)]
        for s in range(int(r.species)):
            got = srv.result_species(rid, s) if r.species > 2 else srv.result(rid)[s]
            assert_masses(got, cur[s], tol, f"request {rid} species {s}")
    srv.close()
