"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on seeded synthetic inputs.

Tolerances (FP32 storage and arithmetic against the FP64 oracle):
  - populations over the first 1000 steps: max-abs 1e-5;
  - steady velocity and concentration fields: relative L2 1e-4; integrated current: relative 1e-4;
  - integer work (link masks via node classes, biofilm growth): bit-exact.
"""
import numpy as np
import pytest

import mfc_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
FIELD_TOL = 1e-4


@pytest.fixture(scope="module")
def P():
    from paper_1802_07525_gb300 import build
    build.build()
    import paper_1802_07525_gb300 as P
    return P


def pair(P, shape, cls, bc=None, precision=0, **kw):
    """A GPU lattice and an oracle lattice with the same geometry and parameters."""
    dim = len(shape)
    if bc is None:
        bc = (2, 0) if dim == 2 else (0, 0, 2)
    g = P.Lattice(shape, bc=bc, precision=precision, **kw)
    g.set_geometry(cls, reset_fields=True)
    o = oracle.Oracle(shape, cls, bc=bc, **kw)
    return g, o


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def channel_kw(w):
    return dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)


# ------------------------------------------------------------------------------------------
# Per-step populations
# ------------------------------------------------------------------------------------------

def test_channel_128x64_coupled_populations_first_1000_steps(P):
    """Fused flow + transport on the 128x64 channel: populations within 1e-5 of the oracle
    at steps 1, 10, 100, 1000."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, **channel_kw(w))
    done = 0
    for target in (1, 10, 100, 1000):
        g.step_coupled(target - done)
        o.step_coupled(target - done)
        done = target
        assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL, target
        assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL, target
    rho, u, c, _ = g.read_fields()
    assert maxabs(rho, o.rho) < POP_TOL
    assert maxabs(u, o.u) < POP_TOL
    assert maxabs(c, o.conc) < POP_TOL


def test_channel_128x64_sequential_populations(P):
    """Flow steps, then transport steps with that velocity frozen (the paper's order)."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, **channel_kw(w))
    g.step_flow(300)
    o.step_flow(300)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL
    assert maxabs(g.read_populations(P.MFC_FIELD_VELOCITY), o.u) < POP_TOL
    g.step_ade(300)
    o.step_ade(300)
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL
    assert maxabs(g.read_fields()[2], o.conc) < POP_TOL


@pytest.mark.parametrize("shape,bc", [
    ((37, 23), (2, 0)),          # ragged: not a multiple of the warp or block width
    ((300, 9), (2, 1)),          # periodic cross axis, two column blocks with a ragged tail
    ((20, 16), (1, 1)),          # fully periodic
    ((17, 11), (0, 0)),          # closed box
    ((1, 5), (0, 0)),            # one column
    ((3, 1), (2, 1)),            # one row, periodic
])
def test_2d_boundary_kinds_and_ragged_sizes(P, shape, bc):
    N = int(np.prod(shape))
    rng = np.random.default_rng(N)
    r = rng.random(N)
    cls = np.where(r < 0.15, 3, np.where(r < 0.3, 4, np.where(r < 0.35, 5, 0))).astype(np.uint8)
    g, o = pair(P, shape, cls, bc=bc, tau=0.7, tau_c=0.9, u_in=0.03, c_in=0.8, k_sink=0.01)
    if bc[0] != 2:
        # no inlet: start from a perturbed state so something moves
        f = o.f.copy()
        open_ = (cls & 1) == 0
        for k in np.nonzero(open_)[0]:
            f[:, k] = oracle.flow_equilibrium(2, 1.0 + 0.01 * rng.standard_normal(),
                                              0.02 * rng.standard_normal(2))
        gg = np.where((cls & 2) == 0, rng.random((5, N)) * 0.2, 0.0)
        o.f[:] = f
        o.g[:] = gg
        g.write_populations(P.MFC_POP_FLOW, f)
        g.write_populations(P.MFC_POP_ADE, gg)
    g.step_coupled(200)
    o.step_coupled(200)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL


def test_dirichlet_outlet_and_velocity_scale(P):
    shape = (40, 12)
    cls = mi.mark_sink_layer(shape, mi.bernoulli_block(shape, 0.2, 5, block=(10, 30)), mi.SINK)
    kw = dict(tau=0.8, tau_c=0.75, u_in=0.02, c_in=1.0, c_out=0.25, k_sink=5e-3, u_scale=2.5,
              ade_outlet=1)
    g, o = pair(P, shape, cls, **kw)
    g.step_flow(150)
    o.step_flow(150)
    g.step_ade(150)
    o.step_ade(150)
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL


@pytest.mark.parametrize("shape,bc", [((24, 20, 32), (0, 0, 2)), ((19, 13, 11), (1, 0, 2)),
                                      ((12, 10, 9), (1, 1, 1))])
def test_3d_populations(P, shape, bc):
    cls = mi.overlapping_balls(shape, 3, 0.7, 31)
    cls = mi.mark_sink_layer(shape, cls, mi.SINK)
    kw = dict(tau=0.7, tau_c=0.6, u_in=0.005, c_in=1.0, k_sink=5e-4)
    g, o = pair(P, shape, cls, bc=bc, **kw)
    if bc[2] != 2:
        rng = np.random.default_rng(3)
        gg = np.where((cls & 2) == 0, rng.random((7, g.N)) * 0.1, 0.0)
        o.g[:] = gg
        g.write_populations(P.MFC_POP_ADE, gg)
    g.step_coupled(100)
    o.step_coupled(100)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL


# ------------------------------------------------------------------------------------------
# Steady state, residuals, current
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [0, 1])
def test_channel_128x64_steady_fields_and_current(P, mode):
    """Solve to tol 1e-8 or 10^4 steps with a residual check every 100 steps, on both sides;
    fields within 1e-4 relative L2, current within 1e-4 relative."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, **channel_kw(w))
    rg = g.solve_steady(mode=mode, tol_flow=w.tol, tol_ade=w.tol, max_steps=w.max_steps,
                        check_every=100)
    ro = o.solve_steady(mode=mode, tol_flow=w.tol, tol_ade=w.tol, max_steps=w.max_steps,
                        check_every=100)
    rho, u, c, cur = g.read_fields()
    assert rel_l2(u, o.u) < FIELD_TOL
    assert rel_l2(c, o.conc) < FIELD_TOL
    assert abs(rg.current - ro.current) / ro.current < FIELD_TOL
    assert abs(cur - ro.current) / ro.current < FIELD_TOL
    assert abs(rg.mass - ro.mass) / ro.mass < 1e-6
    # same stopping decisions, or both at the cap
    assert rg.steps_flow == ro.steps_flow or max(rg.res_flow, ro.res_flow) < 3 * w.tol
    assert rg.status in (P.MFC_OK, P.MFC_NOT_CONVERGED)


def test_residual_sums_match_oracle_sums(P):
    """The FP64 reductions of a check step agree with the oracle's sums of the same fields:
    400 fused steps (fields stored at 400), then a 2-step solve block that compares the fields
    of step 402 with those of step 400; its residuals are per step."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, **channel_kw(w))
    g.step_coupled(400)
    r = g.solve_steady(mode=1, tol_flow=0.0, tol_ade=0.0, max_steps=2, check_every=2)
    o.step_coupled(400)
    u1, c1 = o.u.copy(), o.conc.copy()
    o.step_coupled(2)
    s = o.sums(u1, c1)
    assert r.status == P.MFC_NOT_CONVERGED and r.steps_flow == 2
    assert r.res_flow == pytest.approx(np.sqrt(s[0] / s[1]) / 2, rel=1e-3)
    assert r.res_ade == pytest.approx(np.sqrt(s[3] / s[4]) / 2, rel=1e-3)
    assert r.current == pytest.approx(s[6], rel=1e-5)
    assert r.mass == pytest.approx(s[2], rel=1e-7)
    assert r.substrate == pytest.approx(s[5], rel=1e-5)


def test_solve_statuses_and_host_injected_nonfinite(P):
    w = mi.channel_128x64()
    g = P.Lattice(w.shape, **channel_kw(w))
    g.set_geometry(w.cls)
    r = g.solve_steady(mode=1, tol_flow=1e-30, tol_ade=1e-30, max_steps=10, check_every=4)
    assert r.status == P.MFC_NOT_CONVERGED and r.steps_flow == 10
    r = g.solve_steady(mode=1, tol_flow=1e-30, tol_ade=1e-30, max_steps=10**7, check_every=100,
                       timeout_s=0.05)
    assert r.status == P.MFC_ERR_TIMEOUT
    # inject a NaN into the populations on the host; the residual check reports it
    f = g.read_populations(P.MFC_POP_FLOW)
    k = int(np.nonzero((w.cls & 1) == 0)[0][100])
    f[3, k] = np.nan
    g.write_populations(P.MFC_POP_FLOW, f)
    r = g.solve_steady(mode=1, tol_flow=1e-8, tol_ade=1e-8, max_steps=100, check_every=10)
    assert r.status == P.MFC_ERR_NONFINITE and r.steps_flow == 10
    # the lattice stays usable after a reset
    g.set_geometry(w.cls, reset_fields=True)
    g.step_coupled(5)
    assert np.isfinite(g.read_fields()[1]).all()


# ------------------------------------------------------------------------------------------
# Geometry updates and the biofilm rule
# ------------------------------------------------------------------------------------------

def test_biofilm_growth_bit_exact_and_warm_start(P):
    """The GPU growth pass equals the oracle's rule applied to the GPU's own concentration
    field (the threshold is decided in the same precision); the warm-started step after the
    mask change matches the oracle stepping from the same state."""
    shape = (96, 48)
    cls = mi.mark_sink_layer(shape, mi.overlapping_balls(shape, 4, 0.75, 12), mi.SINK)
    kw = dict(tau=0.8, tau_c=0.7, u_in=0.02, c_in=1.0, k_sink=1e-3)
    g, o = pair(P, shape, cls, **kw)
    g.step_coupled(2500)  # the substrate front has passed the first biofilm by then
    c_gpu = g.read_fields()[2]
    f_gpu = g.read_populations(P.MFC_POP_FLOW)
    g_gpu = g.read_populations(P.MFC_POP_ADE)
    for cycle in range(3):
        new_o, n_o = o.biofilm_convert(77, cycle, prob=0.3, c_thresh=0.5, conc=c_gpu)
        n_g = g.biofilm_grow(77, cycle, prob=0.3, c_thresh=0.5)
        assert n_g == n_o and n_o > 0
        o.cls[:] = new_o
        # the GPU's flow-blocked set (populations read as 0 there) equals the oracle's mask
        fb = np.all(g.read_populations(P.MFC_POP_FLOW) == 0.0, axis=0)
        assert np.array_equal(fb, (o.cls & 1) > 0)
        c_gpu = g.read_fields()[2]
    # warm start: oracle steps from the GPU's populations with the grown mask
    o2 = oracle.Oracle(shape, o.cls, **kw)
    newly_solid = (o.cls & 1) & ~(cls & 1)
    f0 = f_gpu.copy()
    f0[:, newly_solid > 0] = 0.0
    o2.f[:] = f0
    o2.g[:] = g_gpu
    # the GPU kept the same populations (no steps since the read)
    o2.step_coupled(20)
    g.step_coupled(20)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o2.f) < POP_TOL
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o2.g) < POP_TOL


def test_set_geometry_warm_start_opens_and_closes_nodes(P):
    shape = (40, 20)
    rng = np.random.default_rng(1)
    cls1 = np.where(rng.random(800) < 0.2, 3, 0).astype(np.uint8)
    cls2 = np.where(rng.random(800) < 0.2, 3, 0).astype(np.uint8)
    g, o = pair(P, shape, cls1, tau=0.9, tau_c=0.8, u_in=0.02)
    g.step_coupled(50)
    o.step_coupled(50)
    g.set_geometry(cls2, reset_fields=False)
    # oracle: keep populations where open in both, rest state where newly open, drop newly blocked
    f = o.f.copy()
    gg = o.g.copy()
    opened_f = ((cls1 & 1) > 0) & ((cls2 & 1) == 0)
    opened_a = ((cls1 & 2) > 0) & ((cls2 & 2) == 0)
    wf = oracle.flow_equilibrium(2, 1.0, [0, 0])
    f[:, opened_f] = wf[:, None]
    gg[:, opened_a] = 0.0
    f[:, (cls2 & 1) > 0] = 0.0
    gg[:, (cls2 & 2) > 0] = 0.0
    o2 = oracle.Oracle(shape, cls2, tau=0.9, tau_c=0.8, u_in=0.02)
    o2.f[:] = f
    o2.g[:] = gg
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o2.f) < POP_TOL
    g.step_coupled(30)
    o2.step_coupled(30)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o2.f) < POP_TOL
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o2.g) < POP_TOL
    assert g.active_nodes() == (int(((cls2 & 1) == 0).sum()), int(((cls2 & 2) == 0).sum()))


# ------------------------------------------------------------------------------------------
# Full size, in the launch configuration the benchmark times
# ------------------------------------------------------------------------------------------

def test_anode_2048x1024_one_step_parity_at_full_size(P):
    """2048x1024 porous anode after 300 fused steps: one more GPU step equals one oracle step
    taken from the GPU's own state (every node), and the check-step sums equal the oracle's."""
    w = mi.anode_2d()
    g = P.Lattice(w.shape, **channel_kw(w))
    g.set_geometry(w.cls)
    g.step_coupled(300)
    f = g.read_populations(P.MFC_POP_FLOW)
    gg = g.read_populations(P.MFC_POP_ADE)
    o = oracle.Oracle(w.shape, w.cls, **channel_kw(w))
    o.f[:] = f
    o.g[:] = gg
    o.step_coupled(1)
    g.step_coupled(1)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < 1e-6
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < 1e-6
    rho, u, c, _ = g.read_fields()
    assert maxabs(u, o.u) < 1e-6 and maxabs(c, o.conc) < 1e-6


def test_electrode_256x128x128_one_step_parity_at_full_size(P):
    """The 256x128x128 porous electrode after 100 fused steps: one more GPU step (the step
    kernel and launch shape the benchmark times) equals one oracle step taken from the GPU's
    own state, at every node, and so do the velocity and concentration fields."""
    w = mi.electrode_3d()
    g = P.Lattice(w.shape, **channel_kw(w))
    g.set_geometry(w.cls)
    g.step_coupled(100)
    o = oracle.Oracle(w.shape, w.cls, **channel_kw(w))
    o.f[:] = g.read_populations(P.MFC_POP_FLOW)
    o.g[:] = g.read_populations(P.MFC_POP_ADE)
    o.step_coupled(1)
    g.step_coupled(1)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < 1e-6
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < 1e-6
    rho, u, c, _ = g.read_fields()
    assert maxabs(u, o.u) < 1e-6 and maxabs(c, o.conc) < 1e-6
    g.close()


def test_fp16_deviation_storage_error_is_bounded(P):
    """FP16 deviation storage (FP32 arithmetic): the error against the FP64 oracle after 1000
    fused steps is stated rather than held to the FP32 bound; FP16 keeps about 3 significant
    digits of each stored deviation."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, precision=1, **channel_kw(w))
    g.step_coupled(1000)
    o.step_coupled(1000)
    rho, u, c, _ = g.read_fields()
    eu, ec = rel_l2(u, o.u), rel_l2(c, o.conc)
    print(f"FP16 storage after 1000 steps: rel L2 u {eu:.3e}, C {ec:.3e}, "
          f"max |f - f_oracle| {maxabs(g.read_populations(P.MFC_POP_FLOW), o.f):.3e}")
    assert eu < 2e-2
    assert ec < 1e-2


# ------------------------------------------------------------------------------------------
# Launch variants: every variant computes the same arithmetic; the results agree to FP32
# rounding (the compiler may contract multiply-adds differently in each variant)
# ------------------------------------------------------------------------------------------

def _variants(dim):
    return [dict(block=128), dict(block=256), dict(block=128, offsets32=0),
            dict(block=256, offsets32=0)]


@pytest.mark.parametrize("shape,bc,prec", [
    ((300, 37), (2, 0), 0),      # ragged strip and row tails, inlet/outlet, walls
    ((133, 20), (2, 1), 0),      # periodic cross axis
    ((64, 24), (1, 1), 0),       # fully periodic
    ((45, 9), (0, 0), 0),        # closed box
    ((300, 37), (2, 0), 1),      # FP16 storage
    ((23, 11, 17), (0, 0, 2), 0),
    ((16, 9, 10), (1, 1, 1), 0),
])
def test_launch_variants_agree(P, shape, bc, prec):
    dim = len(shape)
    N = int(np.prod(shape))
    rng = np.random.default_rng(N + prec)
    r = rng.random(N)
    cls = np.where(r < 0.15, 3, np.where(r < 0.3, 4, np.where(r < 0.35, 5, 0))).astype(np.uint8)
    kw = dict(tau=0.7, tau_c=0.9, u_in=0.03, c_in=0.8, k_sink=0.01)
    f0 = g0 = None
    if bc[0] != 2 and (dim == 2 or bc[2] != 2):
        o = oracle.Oracle(shape, cls, bc=bc, **kw)
        for k in np.nonzero((cls & 1) == 0)[0]:
            o.f[:, k] = oracle.flow_equilibrium(dim, 1.0 + 0.01 * rng.standard_normal(),
                                                0.02 * rng.standard_normal(dim))
        f0 = o.f.copy()
        g0 = np.where((cls & 2) == 0, rng.random((o.qa, N)) * 0.2, 0.0)
    ref = None
    for v in _variants(dim):
        g = P.Lattice(shape, bc=bc, precision=prec, **kw)
        g.set_geometry(cls)
        g.set_launch(**v)
        if f0 is not None:
            g.write_populations(P.MFC_POP_FLOW, f0)
            g.write_populations(P.MFC_POP_ADE, g0)
        g.step_coupled(37)
        r1 = g.solve_steady(mode=1, tol_flow=0.0, tol_ade=0.0, max_steps=6, check_every=6)
        g.step_flow(5)
        g.step_ade(4)
        out = (g.read_populations(P.MFC_POP_FLOW), g.read_populations(P.MFC_POP_ADE),
               g.read_fields()[1], (r1.res_flow, r1.res_ade, r1.current, r1.mass))
        g.close()
        if ref is None:
            ref = out
            continue
        tol = 2e-6 if prec == 0 else 2e-3
        assert maxabs(out[0], ref[0]) < tol, v
        assert maxabs(out[1], ref[1]) < tol, v
        assert maxabs(out[2], ref[2]) < tol, v
        assert np.allclose(out[3], ref[3], rtol=1e-3 if prec else 1e-5, atol=1e-12), v


@pytest.mark.parametrize("shape,bc,k_half", [
    ((300, 37), (2, 0), 0.0),       # inlet/outlet, walls; odd ny: the last pair has one row
    ((133, 20), (2, 1), 0.0),       # periodic cross axis
    ((64, 24), (1, 1), 0.0),        # fully periodic
    ((45, 9), (0, 0), 0.05),        # closed box, saturating consumption
    ((23, 11, 17), (0, 0, 2), 0.0),  # 3-D inlet/outlet along z, odd ny
    ((16, 9, 10), (1, 1, 1), 0.05),
])
def test_paired_plain_steps_agree_with_single_node_steps(P, shape, bc, k_half):
    """FP16 storage: plain coupled steps of two rows per thread (paired FP32 arithmetic, 32-bit
    offsets) against single-node plain steps (64-bit offsets) from the same state.  The two group
    the FP32 operations differently, so a stored FP16 value may round to the neighbouring one:
    after one step every population agrees within two FP16 spacings of the largest, after 50
    steps within the FP16 bound of the launch-variant test."""
    dim = len(shape)
    N = int(np.prod(shape))
    rng = np.random.default_rng(N + 7)
    r = rng.random(N)
    cls = np.where(r < 0.15, 3, np.where(r < 0.3, 4, np.where(r < 0.35, 5, 0))).astype(np.uint8)
    kw = dict(tau=0.7, tau_c=0.9, u_in=0.03, c_in=0.8, k_sink=0.01, k_half=k_half)
    f0 = g0 = None
    if bc[0] != 2 and (dim == 2 or bc[2] != 2):
        o = oracle.Oracle(shape, cls, bc=bc, **{k: v for k, v in kw.items() if k != "k_half"})
        for k in np.nonzero((cls & 1) == 0)[0]:
            o.f[:, k] = oracle.flow_equilibrium(dim, 1.0 + 0.01 * rng.standard_normal(),
                                                0.02 * rng.standard_normal(dim))
        f0 = o.f.copy()
        g0 = np.where((cls & 2) == 0, rng.random((o.qa, N)) * 0.2, 0.0)
    lats = []
    for off32 in (1, 0):
        g = P.Lattice(shape, bc=bc, precision=P.MFC_FP16_DEV, **kw)
        g.set_geometry(cls)
        g.set_launch(block=128, offsets32=off32)
        if f0 is not None:
            g.write_populations(P.MFC_POP_FLOW, f0)
            g.write_populations(P.MFC_POP_ADE, g0)
        else:
            g.step_coupled(20)  # a developed, non-uniform state from the inlet
        lats.append(g)
    a, b = lats
    # the same starting state in both (the warm-up steps above may differ by FP16 roundings)
    for which in (P.MFC_POP_FLOW, P.MFC_POP_ADE):
        b.write_populations(which, a.read_populations(which))
    for n, rel in ((1, 2.0 ** -10), (49, None)):
        a.step_coupled_plain(n)
        b.step_coupled_plain(n)
        for which in (P.MFC_POP_FLOW, P.MFC_POP_ADE):
            pa, pb = a.read_populations(which), b.read_populations(which)
            tol = rel * np.abs(pb).max() + 1e-7 if rel else 2e-3
            assert maxabs(pa, pb) <= tol, (n, which, maxabs(pa, pb), tol)
    # solve blocks: paired plain steps between single-node stored-field and check steps (the two
    # kernels must leave each other the ghost values they read) against single-node steps only
    for g in lats:
        g.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0, max_steps=60, check_every=10)
    for which in (P.MFC_POP_FLOW, P.MFC_POP_ADE):
        pa, pb = a.read_populations(which), b.read_populations(which)
        assert maxabs(pa, pb) <= 2e-3, ("solve blocks", which, maxabs(pa, pb))
    for g in lats:
        g.close()


def test_fp16_3d_solve_blocks_against_oracle(P):
    """FP16 storage on a 3-D electrode with an inlet and an outlet along z: 200 steps as
    mfc_solve_steady runs them (paired plain steps, a stored-field and a check step every 20)
    against 200 steps of the FP64 oracle, within the FP16 bound of the launch-variant test."""
    w = mi.electrode_3d(20, 16, 24, seed=21)
    g, o = pair(P, w.shape, w.cls, precision=P.MFC_FP16_DEV, **channel_kw(w))
    g.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0, max_steps=200, check_every=20)
    o.step_coupled(200)
    ef = maxabs(g.read_populations(P.MFC_POP_FLOW), o.f)
    eg = maxabs(g.read_populations(P.MFC_POP_ADE), o.g)
    print(f"FP16 3-D, 200 steps in solve blocks: max |df| {ef:.2e}, max |dg| {eg:.2e}")
    assert ef < 2e-3 and eg < 2e-3, (ef, eg)


# ------------------------------------------------------------------------------------------
# Paper-literal transport: D2Q9 with the equilibrium of Eq. 5 (C in place of rho)
# ------------------------------------------------------------------------------------------

def test_d2q9_transport_channel_populations_first_1000_steps(P):
    """Fused flow + D2Q9 transport on the 128x64 channel: populations within 1e-5 of the
    oracle's D2Q9 transport at steps 1, 10, 100, 1000."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, ade_q=9, **channel_kw(w))
    assert g.qa == 9 and o.qa == 9
    done = 0
    for target in (1, 10, 100, 1000):
        g.step_coupled(target - done)
        o.step_coupled(target - done)
        done = target
        assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL, target
        assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL, target
    _, u, c, _ = g.read_fields()
    assert maxabs(c, o.conc) < POP_TOL


@pytest.mark.parametrize("shape,bc,outlet", [
    ((150, 37), (2, 1), 0),   # inlet/outlet along x, periodic y, ragged rows
    ((133, 20), (2, 0), 1),   # walls, Dirichlet transport outlet
    ((64, 24), (1, 1), 0),    # fully periodic
])
def test_d2q9_transport_boundary_kinds(P, shape, bc, outlet):
    N = int(np.prod(shape))
    rng = np.random.default_rng(N + 9)
    r = rng.random(N)
    cls = np.where(r < 0.12, 3, np.where(r < 0.22, 4, np.where(r < 0.26, 5, 0))).astype(np.uint8)
    kw = dict(tau=0.75, tau_c=0.8, u_in=0.03, c_in=1.0, c_out=0.25, k_sink=0.01, ade_outlet=outlet)
    g, o = pair(P, shape, cls, bc=bc, ade_q=9, **kw)
    g.step_coupled(300)
    o.step_coupled(300)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL


def test_d2q9_transport_steady_fields_and_current(P):
    """Both sides to tol 1e-7 (cap 10^4, a check every 100 steps): steady fields within 1e-4
    relative L2 and the current within 1e-4."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, ade_q=9, **channel_kw(w))
    rg = g.solve_steady(mode=1, tol_flow=1e-7, tol_ade=1e-7, max_steps=10000, check_every=100)
    ro = o.solve_steady(mode=1, tol_flow=1e-7, tol_ade=1e-7, max_steps=10000, check_every=100)
    _, u, c, _ = g.read_fields()
    assert rel_l2(u, o.u) < FIELD_TOL
    assert rel_l2(c, o.conc) < FIELD_TOL
    assert abs(rg.current - ro.current) / ro.current < FIELD_TOL


def test_d2q9_transport_launch_shapes_agree_and_fp16_bound(P):
    w = mi.channel_128x64()
    out = []
    for block in (128, 256):
        g = P.Lattice(w.shape, ade_q=9, **channel_kw(w))
        g.set_geometry(w.cls)
        g.set_launch(block=block)
        g.step_coupled(500)
        out.append(g.read_populations(P.MFC_POP_ADE))
        g.close()
    assert maxabs(out[0], out[1]) < 2e-6
    g, o = pair(P, w.shape, w.cls, precision=1, ade_q=9, **channel_kw(w))
    g.step_coupled(1000)
    o.step_coupled(1000)
    _, u, c, _ = g.read_fields()
    assert rel_l2(u, o.u) < 2e-2 and rel_l2(c, o.conc) < 1e-2


# ------------------------------------------------------------------------------------------
# Saturating consumption (Eq. 16's substrate factor, k_half = K_s)
# ------------------------------------------------------------------------------------------

MONOD = dict(tau=0.8, tau_c=0.7, u_in=0.01, c_in=1.0, k_sink=0.02, k_half=0.05)


def test_monod_consumption_channel_populations_and_current(P):
    """The 128x64 channel with consumption k C K_s / (K_s + C) (K_s = 0.05, about the paper's
    K_s / C_in = 20 / 410): populations within 1e-5 of the oracle at steps 1, 10, 100, 1000;
    the check-step current equals the oracle's sum of the same consumption."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, **MONOD)
    done = 0
    for target in (1, 10, 100, 1000):
        g.step_coupled(target - done)
        o.step_coupled(target - done)
        done = target
        assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL, target
        assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL, target
    r = g.solve_steady(mode=1, tol_flow=0.0, tol_ade=0.0, max_steps=2, check_every=2)
    o.step_coupled(2)
    s = o.sums()
    assert r.current == pytest.approx(s[6], rel=1e-5)


def test_monod_consumption_steady_current(P):
    """Steady solve with the saturating consumption: same stopping check as the oracle, fields
    and current within 1e-4."""
    w = mi.channel_128x64()
    g, o = pair(P, w.shape, w.cls, **MONOD)
    rg = g.solve_steady(mode=1, tol_flow=w.tol, tol_ade=w.tol, max_steps=w.max_steps,
                        check_every=100)
    ro = o.solve_steady(mode=1, tol_flow=w.tol, tol_ade=w.tol, max_steps=w.max_steps,
                        check_every=100)
    rho, u, c, cur = g.read_fields()
    assert rel_l2(c, o.conc) < FIELD_TOL
    assert abs(rg.current - ro.current) / ro.current < FIELD_TOL
    assert rg.steps_flow == ro.steps_flow or max(rg.res_flow, ro.res_flow) < 3 * w.tol


def test_monod_consumption_3d(P):
    shape = (19, 13, 11)
    cls = mi.mark_sink_layer(shape, mi.overlapping_balls(shape, 3, 0.7, 31), mi.SINK)
    kw = dict(tau=0.7, tau_c=0.6, u_in=0.005, c_in=1.0, k_sink=0.05, k_half=0.1)
    g, o = pair(P, shape, cls, bc=(1, 0, 2), **kw)
    g.step_coupled(150)
    o.step_coupled(150)
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL


def test_monod_consumption_d2q9_transport_and_fp16(P):
    """The saturating-consumption kernels of the D2Q9 transport (FP32) and of FP16 storage:
    populations against the oracle within the FP32 bound (D2Q9) and the FP16 bound of the
    first-order kernels (max-abs 5e-3 over 300 steps)."""
    shape = (150, 37)
    N = int(np.prod(shape))
    rng = np.random.default_rng(N)
    r = rng.random(N)
    cls = np.where(r < 0.12, 3, np.where(r < 0.3, 4, 0)).astype(np.uint8)
    kw = dict(tau=0.8, tau_c=0.7, u_in=0.02, c_in=1.0, k_sink=0.05, k_half=0.05)
    g, o = pair(P, shape, cls, bc=(2, 1), ade_q=9, **kw)
    g.step_coupled(300)
    o.step_coupled(300)
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL
    g.close()
    g, o = pair(P, shape, cls, bc=(2, 1), precision=P.MFC_FP16_DEV, **kw)
    g.step_coupled(300)
    o.step_coupled(300)
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < 5e-3
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < 5e-3
    g.close()


# ------------------------------------------------------------------------------------------
# 3-D electrode: populations over 1000 steps, steady fields and current
# ------------------------------------------------------------------------------------------

def electrode_kw(w):
    return dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)


def test_3d_electrode_populations_first_1000_steps(P):
    """Fused D3Q19 + D3Q7 on a 24x20x32 porous electrode (spheres of radius 4, flow along z):
    populations within 1e-5 of the oracle at steps 1, 10, 100 and 1000."""
    w = mi.electrode_3d(24, 20, 32, seed=9)
    g, o = pair(P, w.shape, w.cls, **electrode_kw(w))
    done = 0
    for target in (1, 10, 100, 1000):
        g.step_coupled(target - done)
        o.step_coupled(target - done)
        done = target
        assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL, target
        assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL, target
    _, u, c, _ = g.read_fields()
    assert maxabs(u, o.u) < POP_TOL
    assert maxabs(c, o.conc) < POP_TOL
    g.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_3d_electrode_steady_fields_and_current(P, mode):
    """The 16x16x24 electrode solved to 1e-7 (checks every 100 steps) in both modes on both
    sides: velocity and concentration within 1e-4 relative L2, current within 1e-4 relative,
    the same stopping checks."""
    w = mi.electrode_3d(16, 16, 24, seed=9)
    g, o = pair(P, w.shape, w.cls, **electrode_kw(w))
    rg = g.solve_steady(mode=mode, tol_flow=w.tol, tol_ade=w.tol, max_steps=w.max_steps,
                        check_every=100)
    ro = o.solve_steady(mode=mode, tol_flow=w.tol, tol_ade=w.tol, max_steps=w.max_steps,
                        check_every=100)
    _, u, c, cur = g.read_fields()
    assert rg.status == P.MFC_OK and ro.converged
    assert rel_l2(u, o.u) < FIELD_TOL
    assert rel_l2(c, o.conc) < FIELD_TOL
    assert abs(rg.current - ro.current) / ro.current < FIELD_TOL
    assert abs(cur - ro.current) / ro.current < FIELD_TOL
    assert abs(rg.steps_flow - ro.steps_flow) <= 100 and abs(rg.steps_ade - ro.steps_ade) <= 100
    g.close()


# ------------------------------------------------------------------------------------------
# Range guard: a solve whose flow reaches the lattice sound speed stops with its own status
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_flow_at_the_sound_speed_ends_the_solve_at_the_first_check(P, dim):
    """A uniform flow written through mfc_write_populations into a periodic box is a fixed
    point of the scheme.  At 0.6 (above the sound speed 0.577) the solve ends at its first check
    with MFC_ERR_UNSTABLE, as the oracle's does; at 0.55 it runs to its step cap."""
    shape = (64, 32) if dim == 2 else (32, 16, 16)
    N = int(np.prod(shape))
    for speed, expect in ((0.6, P.MFC_ERR_UNSTABLE), (0.55, P.MFC_NOT_CONVERGED)):
        u = [0.0] * dim
        u[0] = speed
        f = np.repeat(oracle.flow_equilibrium(dim, 1.0, u)[:, None], N, axis=1)
        g = P.Lattice(shape, bc=(1,) * dim, tau=0.8)
        g.set_geometry(np.zeros(N, np.uint8))
        g.write_populations(P.MFC_POP_FLOW, f)
        r = g.solve_steady(mode=1, tol_flow=0.0, tol_ade=0.0, max_steps=50, check_every=10)
        assert r.status == expect
        assert r.steps_flow == (10 if expect == P.MFC_ERR_UNSTABLE else 50)
        o = oracle.Oracle(shape, bc=(1,) * dim, tau=0.8)
        o.f[:] = f
        ro = o.solve_steady(mode=1, tol_flow=0.0, tol_ade=0.0, max_steps=50, check_every=10)
        assert ro.unstable == int(expect == P.MFC_ERR_UNSTABLE) and ro.steps_flow == r.steps_flow
        g.close()


# ------------------------------------------------------------------------------------------
# The paper's units (Table 1): tau = 0.6706, tau_D = 0.5036, and the transport velocity
# scaled by the ratio of the two lattices' time steps, 17.66
# ------------------------------------------------------------------------------------------

# Table 1: V = 1.758e-2 mm/s, nu = 1.004 mm^2/s at tau = 0.6706 with dx = 1 mm, so the flow
# time step is ((tau - 1/2) / 3) / nu = 0.05664 s and the inlet speed in flow lattice units
# V * dt / dx = 9.957e-4; D = 0.0012 mm^2/s at tau_D = 0.5036 gives a transport time step of 1 s,
# 17.66 flow steps.
PAPER_U_IN = 1.758e-2 * ((0.6706 - 0.5) / 3.0) / 1.004


def paper_kw(q, u_scale):
    return dict(tau=0.6706, tau_c=0.5036, u_in=PAPER_U_IN, c_in=1.0, k_sink=1e-3,
                u_scale=u_scale), (9 if q == 9 else 0)


@pytest.mark.parametrize("q", [9, 5])
@pytest.mark.parametrize("u_scale", [17.66, 1.0])
def test_paper_units_transport_populations_first_1000_steps(P, q, u_scale):
    """The 128x64 channel in Table 1's units, with the paper-literal D2Q9 transport (the
    equilibrium of Eq. 5) and with D2Q5: populations within 1e-5 of the oracle at steps 1, 10,
    100 and 1000, with transport at the scaled velocity (17.66) and unscaled (1)."""
    w = mi.channel_128x64()
    kw, aq = paper_kw(q, u_scale)
    g = P.Lattice(w.shape, ade_q=aq, **kw)
    g.set_geometry(w.cls)
    o = oracle.Oracle(w.shape, w.cls, ade_q=q, **kw)
    done = 0
    for target in (1, 10, 100, 1000):
        g.step_coupled(target - done)
        o.step_coupled(target - done)
        done = target
        assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < POP_TOL, target
        assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < POP_TOL, target
    g.close()


@pytest.mark.parametrize("q", [9, 5])
def test_paper_units_transport_stability(P, q):
    """tau_D = 0.5036 is close to the BGK limit 1/2.  With the transport velocity scaled to its
    own time step (u_scale 17.66, a grid Peclet number of 30 to 75 in the pores) the transport
    of the 128x64 channel grows without bound after about 2,500 steps, on the GPU as in the
    oracle; read in the flow's units (u_scale 1) it stays bounded, with the concentration within
    [-0.01, 1.05] after 20,000 steps."""
    w = mi.channel_128x64()
    for u_scale, bounded in ((1.0, True), (17.66, False)):
        kw, aq = paper_kw(q, u_scale)
        g = P.Lattice(w.shape, ade_q=aq, **kw)
        g.set_geometry(w.cls)
        g.step_coupled(20000 if bounded else 10000)
        _, _, c, _ = g.read_fields()
        c = c[(w.cls & 2) == 0]
        if bounded:
            assert c.min() > -0.01 and c.max() < 1.05
        else:
            assert not (np.isfinite(c).all() and np.abs(c).max() < 10.0)
        g.close()
