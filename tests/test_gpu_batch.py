"""The batch engine (continuous batching of steady solves) through the C ABI.

- a batch solve agrees with the single-lattice solve of the same request (same checks), and
  with the FP64 oracle within the steady-field tolerances;
- a request's result is the same alone and in a mix of other requests, bit for bit;
- admission respects the memory budget and first-come-first-served order;
- the engine thread admits requests that arrive while others run;
- bad requests are refused.
"""
import numpy as np
import pytest

import mfc_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-4


@pytest.fixture(scope="module")
def P():
    from paper_1802_07525_gb300 import build
    build.build()
    import paper_1802_07525_gb300 as P
    return P


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def kw(w):
    return dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)


def mix():
    """Uneven 2-D and 3-D requests (porous anodes and electrodes, seeded)."""
    return [mi.anode_2d(96, 48, seed=21), mi.anode_2d(200, 40, seed=22),
            mi.electrode_3d(24, 20, 32, seed=23), mi.anode_2d(130, 70, seed=24),
            mi.electrode_3d(16, 16, 40, seed=25), mi.anode_2d(64, 64, seed=26)]


def solve_in_batch(P, works, K=100, block=128, tol=1e-6, max_steps=3000, **bopts):
    b = P.Batch(check_every=K, block=block, **bopts)
    tickets = [b.submit(w.shape, w.cls, tol_flow=tol, tol_ade=tol, max_steps=max_steps, **kw(w))
               for w in works]
    b.run()
    out = [b.poll(t) for t in tickets]
    stats = b.stats()
    b.close()
    return out, stats


def test_batch_matches_single_lattice_solves(P):
    """Every request of an uneven 2-D/3-D mix ends at the same check as the single-lattice
    solve with check_every = K, with the same fields (FP32 roundoff) and residuals."""
    works = mix()
    out, stats = solve_in_batch(P, works)
    assert stats["completed"] == len(works) and stats["check_every"] == 100
    for w, r in zip(works, out):
        g = P.Lattice(w.shape, **kw(w))
        g.set_geometry(w.cls)
        s = g.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=1e-6, tol_ade=1e-6, max_steps=3000,
                           check_every=100)
        rho, u, c, cur = g.read_fields()
        g.close()
        assert r["status"] == s.status, w.name
        assert r["steps_flow"] == s.steps_flow, w.name
        assert rel_l2(r["u"], u) < 1e-5 and rel_l2(r["c"], c) < 1e-5, w.name
        assert r["current"] == pytest.approx(s.current, rel=1e-5)
        assert r["res_flow"] == pytest.approx(s.res_flow, rel=1e-2, abs=1e-12)


def test_batch_solve_matches_oracle(P):
    """The 128x64 channel solved in a batch: steady fields within 1e-4 relative L2 and the
    current within 1e-4 of the FP64 oracle run with the same checks."""
    w = mi.channel_128x64()
    out, _ = solve_in_batch(P, [w], K=100, tol=1e-7, max_steps=6000)
    r = out[0]
    o = oracle.Oracle(w.shape, w.cls, **kw(w))
    ro = o.solve_steady(mode=oracle.CONCURRENT, tol_flow=1e-7, tol_ade=1e-7, max_steps=6000,
                        check_every=100)
    assert rel_l2(r["u"], o.u) < FIELD_TOL
    assert rel_l2(r["c"], o.conc) < FIELD_TOL
    assert abs(r["current"] - ro.current) / ro.current < FIELD_TOL
    assert r["steps_flow"] == ro.steps_flow or r["status"] == P.MFC_NOT_CONVERGED


def test_result_same_alone_and_in_the_mix(P):
    """A request solved alone and among five others of other sizes and dimensions gives the
    same fields and sums bit for bit (same K and block)."""
    works = mix()
    probe = works[3]
    alone, _ = solve_in_batch(P, [probe])
    mixed, _ = solve_in_batch(P, works)
    a, m = alone[0], mixed[3]
    for k in ("status", "steps_flow", "res_flow", "res_ade", "current", "mass", "substrate"):
        assert a[k] == m[k], k
    for k in ("rho", "u", "c"):
        assert np.array_equal(a[k], m[k]), k
    # a 3-D request too
    alone3, _ = solve_in_batch(P, [works[2]])
    assert np.array_equal(alone3[0]["u"], mixed[2]["u"])
    assert alone3[0]["current"] == mixed[2]["current"]


def test_admission_within_budget_first_come_first_served(P):
    """With room for about two requests at a time, six requests all finish, the memory in use
    never exceeds the budget, and requests are admitted in submission order."""
    works = [mi.anode_2d(256, 128, seed=30 + i) for i in range(6)]
    one = P.lattice_bytes(works[0].shape) + 4 * works[0].nodes * 8 + 32 * 2 ** 20
    budget = int(2.5 * one)
    out, stats = solve_in_batch(P, works, tol=1e-5, max_steps=1000, budget_bytes=budget)
    assert stats["completed"] == 6
    assert stats["bytes_peak"] <= budget
    admits = [r["t_admit"] for r in out]
    assert admits == sorted(admits)
    # at most two at a time: the third waited for one of the first two to finish
    assert admits[2] >= min(out[0]["t_done"], out[1]["t_done"]) - 1e-6


def test_engine_thread_admits_requests_arriving_while_others_run(P):
    """Continuous batching: a request submitted while another has already run blocks is set up
    during a running block and joins between blocks; the first request keeps running (it
    finishes after the second was admitted, with no restart), and each result is bit-identical
    to the same request solved alone (same K and block)."""
    import time
    first, second = mi.anode_2d(160, 80, seed=41), mi.electrode_3d(20, 16, 24, seed=42)
    opts = dict(tol_flow=0.0, tol_ade=0.0)  # run to the cap: a known number of blocks
    b = P.Batch(check_every=100, block=128)
    b.start()
    t1 = b.submit(first.shape, first.cls, max_steps=6000, **opts, **kw(first))
    deadline = time.monotonic() + 60.0
    while b.stats()["blocks"] < 3 and time.monotonic() < deadline:
        time.sleep(0.001)
    blocks_before = b.stats()["blocks"]
    assert blocks_before >= 3, "the first request never ran"
    t2 = b.submit(second.shape, second.cls, max_steps=3000, **opts, **kw(second))
    r2 = b.wait(t2, timeout_s=120.0)
    r1 = b.wait(t1, timeout_s=120.0)
    st = b.stats()
    b.stop()
    b.close()
    assert r1 is not None and r2 is not None
    # the second was admitted after the first had run blocks, while the first was running, and
    # the first went on to its cap without interruption
    assert r2["t_admit"] > r1["t_admit"] and r2["t_admit"] < r1["t_done"]
    assert r1["steps_flow"] == 6000 and r2["steps_flow"] == 3000
    assert r1["status"] == r2["status"] == P.MFC_NOT_CONVERGED
    # blocks ran both together: fewer blocks than running them one after the other
    assert st["blocks"] < 60 + 30
    # bit for bit the results of the same requests alone
    alone1, _ = solve_in_batch(P, [first], max_steps=6000, tol=0.0)
    alone2, _ = solve_in_batch(P, [second], max_steps=3000, tol=0.0)
    for a, m in ((alone1[0], r1), (alone2[0], r2)):
        for k in ("steps_flow", "res_flow", "res_ade", "current", "mass", "substrate"):
            assert a[k] == m[k], k
        for k in ("rho", "u", "c"):
            assert np.array_equal(a[k], m[k]), k


def test_bad_requests_are_refused(P):
    w = mi.anode_2d(64, 32, seed=3)
    b = P.Batch(check_every=100, block=128, budget_bytes=64 * 2 ** 20)
    with pytest.raises(P.MfcError) as e:  # larger than the whole budget
        big = mi.anode_2d(2048, 1024)
        b.submit(big.shape, big.cls, **kw(big))
    assert e.value.status == P.MFC_ERR_OOM_BUDGET
    with pytest.raises(P.MfcError) as e:  # tau <= 1/2
        b.submit(w.shape, w.cls, tau=0.5)
    assert e.value.status == P.MFC_ERR_ARG
    with pytest.raises(P.MfcError) as e:  # population arrays past 32-bit element offsets
        shape = (512, 512, 430)  # 19 x the pitched plane > 2^31 elements; no fields requested
        b.submit(shape, np.zeros(shape, np.uint8), fields=False, u_in=0.01)
    assert e.value.status == P.MFC_ERR_ARG
    bad = w.cls.copy()
    bad[5] = 9
    with pytest.raises(P.MfcError):
        b.submit(w.shape, bad, **kw(w))
    t = b.submit(w.shape, w.cls, max_steps=200, **kw(w))
    assert b.poll(t) is None  # queued, no engine has run
    b.run()
    assert b.poll(t)["steps_flow"] == 200
    with pytest.raises(P.MfcError):
        b.poll(t)  # the ticket was released
    b.close()


@pytest.mark.parametrize("shape,bc", [
    ((150, 37), (2, 1)),          # inlet/outlet along x, periodic y
    ((96, 40), (1, 1)),           # fully periodic
    ((20, 13, 30), (1, 0, 2)),    # periodic x, walls y, inlet/outlet along z
])
def test_batch_boundaries_match_oracle(P, shape, bc):
    """The batch step takes inlet and transport-outlet values at the pulling node and writes only
    periodic images and flow outlet values; after 200 fused steps its fields equal the FP64
    oracle's within the per-step population tolerance."""
    N = int(np.prod(shape))
    rng = np.random.default_rng(N)
    r = rng.random(N)
    cls = np.where(r < 0.12, 3, np.where(r < 0.22, 4, 0)).astype(np.uint8)
    kw = dict(tau=0.8, tau_c=0.7, u_in=0.02, c_in=1.0, k_sink=0.01)
    b = P.Batch(check_every=50, block=128)
    t = b.submit(shape, cls, bc=bc, tol_flow=0.0, tol_ade=0.0, max_steps=200, **kw)
    b.run()
    res = b.poll(t)
    b.close()
    o = oracle.Oracle(shape, cls, bc=bc, **kw)
    o.step_coupled(200)
    assert res["steps_flow"] == 200
    assert np.max(np.abs(res["u"] - o.u)) < 1e-5
    assert np.max(np.abs(res["c"] - o.conc)) < 1e-5
    assert np.max(np.abs(res["rho"] - o.rho)) < 1e-5


def test_batch_monod_consumption_matches_single_lattice(P):
    """A request with the saturating consumption (k_half) ends at the same check as the
    single-lattice solve, with the same current."""
    w = mi.anode_2d(96, 48, seed=21)
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=0.02, k_half=0.05)
    b = P.Batch(check_every=100, block=128)
    t = b.submit(w.shape, w.cls, tol_flow=1e-6, tol_ade=1e-6, max_steps=3000, **kw)
    b.run()
    r = b.poll(t)
    b.close()
    g = P.Lattice(w.shape, **kw)
    g.set_geometry(w.cls)
    s = g.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=1e-6, tol_ade=1e-6, max_steps=3000,
                       check_every=100)
    g.close()
    assert r["steps_flow"] == s.steps_flow
    assert r["current"] == pytest.approx(s.current, rel=1e-5)
