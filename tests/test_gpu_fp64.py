"""Parity of the FP64 instantiation of the CUDA kernels (MFC_FP64: FP64 storage, arithmetic and
fields) with the FP64 oracle, through the C ABI.

The two sides compute the same method in the same precision, with different rounding orders:
the kernels store deviations from rest (f_i - w_i), close the rest population from the
conserved total and may contract multiply-adds, the oracle stores f_i and rounds every
operation.  Each step differs by a few units in the last place of O(1) values (~1e-16), and
BGK relaxation (|1 - 1/tau| < 1) does not amplify differences, so over n steps they stay below
n * 1e-15: the tolerance is 1e-12 for populations and fields over up to 1000 steps.  These are
the brute-force tiny-lattice checks (4x3 in 2-D, 5x4x3 in 3-D) and the 128x64 channel of the
method's small configuration, run in FP64 on the GPU.
"""
import numpy as np
import pytest

import mfc_inputs as mi
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def P():
    from paper_1802_07525_gb300 import build
    build.build()
    import paper_1802_07525_gb300 as P
    return P


def pair(P, shape, cls, bc, ade_q=0, **kw):
    g = P.Lattice(shape, bc=bc, precision=P.MFC_FP64, ade_q=ade_q, **kw)
    g.set_geometry(cls, reset_fields=True)
    o = oracle.Oracle(shape, cls, bc=bc, ade_q=ade_q or None, **kw)
    return g, o


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


def perturb(P, g, o, cls, rng, qa):
    """A random non-rest start (flow near equilibrium, random substrate) on both sides."""
    dim, N = o.dim, o.f.shape[1]
    f = o.f.copy()
    for k in np.nonzero((cls & 1) == 0)[0]:
        f[:, k] = oracle.flow_equilibrium(dim, 1.0 + 0.01 * rng.standard_normal(),
                                          0.02 * rng.standard_normal(dim))
    gg = np.where((cls & 2) == 0, rng.random((qa, N)) * 0.2, 0.0)
    o.f[:] = f
    o.g[:] = gg
    g.write_populations(P.MFC_POP_FLOW, f)
    g.write_populations(P.MFC_POP_ADE, gg)


def random_classes(shape, seed):
    N = int(np.prod(shape))
    r = np.random.default_rng(seed).random(N)
    # electrode (flow + transport blocked), biofilm (flow blocked, sink), sink on a fluid node
    return np.where(r < 0.15, 3, np.where(r < 0.3, 5, np.where(r < 0.35, 4, 0))).astype(np.uint8)


@pytest.mark.parametrize("shape,bc", [
    ((4, 3), (2, 0)),          # inlet/outlet along x, walls in y
    ((4, 3), (2, 1)),          # inlet/outlet, periodic y
    ((4, 3), (1, 1)),          # fully periodic
    ((4, 3), (0, 0)),          # closed box
    ((5, 4, 3), (0, 0, 2)),    # walls in x and y, inlet/outlet along z
    ((5, 4, 3), (1, 0, 2)),
    ((5, 4, 3), (1, 1, 1)),
])
def test_tiny_lattices_brute_force(P, shape, bc):
    """Every boundary kind on the smallest lattices, every node class, 300 fused steps from a
    perturbed start: populations within 1e-12 of the oracle at steps 1, 30 and 300."""
    cls = random_classes(shape, int(np.prod(shape)) + sum(bc))
    kw = dict(tau=0.7, tau_c=0.9, u_in=0.03, c_in=0.8, k_sink=0.01)
    g, o = pair(P, shape, cls, bc, **kw)
    perturb(P, g, o, cls, np.random.default_rng(7), o.qa)
    done = 0
    for target in (1, 30, 300):
        g.step_coupled(target - done)
        o.step_coupled(target - done)
        done = target
        assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < TOL64, target
        assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < TOL64, target
    g.close()


def test_channel_128x64_coupled_1000_steps(P):
    """The porous channel of the small configuration: populations and fields within 1e-12 of
    the oracle at steps 1, 100 and 1000."""
    w = mi.channel_128x64()
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    g, o = pair(P, w.shape, w.cls, (2, 0), **kw)
    done = 0
    for target in (1, 100, 1000):
        g.step_coupled(target - done)
        o.step_coupled(target - done)
        done = target
        assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < TOL64, target
        assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < TOL64, target
    rho, u, c, _ = g.read_fields()
    assert maxabs(rho, o.rho) < TOL64
    assert maxabs(u, o.u) < TOL64
    assert maxabs(c, o.conc) < TOL64
    g.close()


def test_sequential_order_and_dirichlet_outlet(P):
    """Flow steps, then transport steps on the frozen (FP64) velocity with u_scale and a
    Dirichlet outlet."""
    shape = (40, 12)
    cls = mi.mark_sink_layer(shape, mi.bernoulli_block(shape, 0.2, 5, block=(10, 30)), mi.SINK)
    kw = dict(tau=0.8, tau_c=0.75, u_in=0.02, c_in=1.0, c_out=0.25, k_sink=5e-3, u_scale=2.5,
              ade_outlet=1)
    g, o = pair(P, shape, cls, (2, 0), **kw)
    g.step_flow(300)
    o.step_flow(300)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < TOL64
    assert maxabs(g.read_populations(P.MFC_FIELD_VELOCITY), o.u) < TOL64
    g.step_ade(300)
    o.step_ade(300)
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < TOL64
    assert maxabs(g.read_fields()[2], o.conc) < TOL64
    g.close()


@pytest.mark.parametrize("shape,bc", [((24, 20, 32), (0, 0, 2)), ((19, 13, 11), (1, 0, 2))])
def test_3d_electrode_populations(P, shape, bc):
    cls = mi.mark_sink_layer(shape, mi.overlapping_balls(shape, 3, 0.7, 31), mi.SINK)
    kw = dict(tau=0.7, tau_c=0.6, u_in=0.005, c_in=1.0, k_sink=5e-4)
    g, o = pair(P, shape, cls, bc, **kw)
    g.step_coupled(200)
    o.step_coupled(200)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < TOL64
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < TOL64
    g.close()


@pytest.mark.parametrize("shape,bc", [((37, 23), (2, 0)), ((20, 16), (1, 1))])
def test_d2q9_transport_populations(P, shape, bc):
    """The paper-literal D2Q9 transport (the equilibrium of Eq. 5) in FP64."""
    cls = random_classes(shape, 91)
    kw = dict(tau=0.8, tau_c=0.7, u_in=0.02, c_in=1.0, k_sink=0.01)
    g, o = pair(P, shape, cls, bc, ade_q=9, **kw)
    if bc[0] != 2:
        perturb(P, g, o, cls, np.random.default_rng(11), 9)
    g.step_coupled(300)
    o.step_coupled(300)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < TOL64
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < TOL64
    g.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_channel_steady_solve_same_stop_and_current(P, mode):
    """Steady solve to 1e-8 with a check every 100 steps on both sides: the same stopping step,
    fields within 1e-10 relative, current and mass within 1e-10 relative."""
    w = mi.channel_128x64()
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    g, o = pair(P, w.shape, w.cls, (2, 0), **kw)
    rg = g.solve_steady(mode=mode, tol_flow=w.tol, tol_ade=w.tol, max_steps=w.max_steps,
                        check_every=100)
    ro = o.solve_steady(mode=mode, tol_flow=w.tol, tol_ade=w.tol, max_steps=w.max_steps,
                        check_every=100)
    assert rg.steps_flow == ro.steps_flow and rg.steps_ade == ro.steps_ade
    rho, u, c, cur = g.read_fields()
    assert np.linalg.norm(u - o.u) / np.linalg.norm(o.u) < 1e-10
    assert np.linalg.norm(c - o.conc) / np.linalg.norm(o.conc) < 1e-10
    assert abs(rg.current - ro.current) / ro.current < 1e-10
    assert abs(rg.mass - ro.mass) / ro.mass < 1e-12
    assert rg.res_flow == pytest.approx(ro.res_flow, rel=1e-6)
    g.close()


def test_check_step_sums_in_fp64(P):
    """The check-step sums of the FP64 instantiation (per-node and per-block terms in FP64)
    against the oracle's sums of the same fields."""
    w = mi.channel_128x64()
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    g, o = pair(P, w.shape, w.cls, (2, 0), **kw)
    g.step_coupled(400)
    r = g.solve_steady(mode=1, tol_flow=0.0, tol_ade=0.0, max_steps=2, check_every=2)
    o.step_coupled(400)
    u1, c1 = o.u.copy(), o.conc.copy()
    o.step_coupled(2)
    s = o.sums(u1, c1)
    assert r.res_flow == pytest.approx(np.sqrt(s[0] / s[1]) / 2, rel=1e-8)
    assert r.res_ade == pytest.approx(np.sqrt(s[3] / s[4]) / 2, rel=1e-8)
    assert r.current == pytest.approx(s[6], rel=1e-12)
    assert r.mass == pytest.approx(s[2], rel=1e-13)
    assert r.substrate == pytest.approx(s[5], rel=1e-12)
    g.close()



def test_monod_consumption_fp64(P):
    """The saturating consumption in the FP64 instantiation: populations and the check-step
    current within rounding of the oracle."""
    w = mi.channel_128x64()
    kw = dict(tau=0.8, tau_c=0.7, u_in=0.01, c_in=1.0, k_sink=0.02, k_half=0.05)
    g, o = pair(P, w.shape, w.cls, (2, 0), **kw)
    g.step_coupled(300)
    o.step_coupled(300)
    assert maxabs(g.read_populations(P.MFC_POP_FLOW), o.f) < TOL64
    assert maxabs(g.read_populations(P.MFC_POP_ADE), o.g) < TOL64
    r = g.solve_steady(mode=1, tol_flow=0.0, tol_ade=0.0, max_steps=2, check_every=2)
    o.step_coupled(2)
    assert r.current == pytest.approx(o.sums()[6], rel=1e-12)
    g.close()
