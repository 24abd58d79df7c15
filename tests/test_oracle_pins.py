"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: values printed in the paper
(tests/golden), closed-form solutions, exact conservation laws, symmetry, or published generator
outputs.  A dropped term, a wrong sign or index, or a transposed table entry fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import BC_INOUT, BC_PERIODIC, BC_WALL, FLOW_SOLID, ADE_SOLID, SINK

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ------------------------------------------------------------------------------------------
# Velocity sets and equilibria
# ------------------------------------------------------------------------------------------

def test_d2q9_matches_eqs_1_to_3_and_eq_11():
    """Velocities of Eqs. 1-3, weights of Eqs. 6-8 and the south-wall pairs of Eq. 11."""
    gd = golden("eq11_south_wall.json")
    c, opp, w = oracle.velocity_set(9)
    assert tuple(c[0]) == (0, 0, 0)
    for i, v in gd["axis_velocities"].items():
        assert tuple(c[int(i)][:2]) == tuple(v)
    assert all(abs(c[i][0]) == 1 and abs(c[i][1]) == 1 for i in range(5, 9))
    for a, b in gd["south_wall_pairs"]:
        assert opp[a] == b and opp[b] == a
        # the populations set at a south wall point north, their sources point south
        assert c[a][1] == 1 and c[b][1] == -1
    ww = gd["weights_over_rho0"]
    assert w[0] == pytest.approx(ww["0"], abs=1e-16)
    assert np.allclose(w[1:5], ww["1-4"], atol=1e-16)
    assert np.allclose(w[5:9], ww["5-8"], atol=1e-16)


@pytest.mark.parametrize("q,cs2,order4", [(9, 1 / 3, True), (19, 1 / 3, True), (5, 1 / 3, False),
                                          (7, 1 / 4, False)])
def test_velocity_set_isotropy(q, cs2, order4):
    c, opp, w = oracle.velocity_set(q)
    c = c.astype(float)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert len({tuple(v) for v in c}) == q
    for i in range(q):
        assert np.all(c[opp[i]] == -c[i])
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    dim = 2 if q in (5, 9) else 3
    m2 = np.einsum("i,ia,ib->ab", w, c, c)[:dim, :dim]
    assert np.allclose(m2, cs2 * np.eye(dim), atol=1e-15)
    if order4:
        m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)[:dim, :dim, :dim, :dim]
        d = np.eye(dim)
        iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                          + np.einsum("ad,bc->abcd", d, d))
        assert np.allclose(m4, iso, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_flow_equilibrium_moments(dim):
    """Eq. 5 has density rho, momentum rho u and momentum flux rho (u u + I/3)."""
    q = 9 if dim == 2 else 19
    c, _, _ = oracle.velocity_set(q)
    c = c[:, :dim].astype(float)
    rng = np.random.default_rng(7)
    for _ in range(5):
        rho = 1.0 + 0.2 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(dim)
        f = oracle.flow_equilibrium(dim, rho, u)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        assert np.allclose(c.T @ f, rho * u, atol=1e-15)
        pi = np.einsum("i,ia,ib->ab", f, c, c)
        assert np.allclose(pi, rho * (np.outer(u, u) + np.eye(dim) / 3.0), atol=1e-15)


@pytest.mark.parametrize("q", [5, 7, 9])
def test_transport_equilibrium_moments(q):
    """The transport equilibrium carries concentration C and flux C u."""
    dim = 3 if q == 7 else 2
    c, _, _ = oracle.velocity_set(q)
    c = c[:, :dim].astype(float)
    cs2 = 0.25 if q == 7 else 1 / 3
    rng = np.random.default_rng(3)
    for _ in range(5):
        C = rng.uniform(0.1, 2.0)
        u = 0.05 * rng.standard_normal(dim)
        g = oracle.ade_equilibrium(q, C, u)
        assert g.sum() == pytest.approx(C, rel=1e-14)
        assert np.allclose(c.T @ g, C * u, atol=1e-15)
        if q != 9:
            pi = np.einsum("i,ia,ib->ab", g, c, c)
            assert np.allclose(pi, cs2 * C * np.eye(dim), atol=1e-15)


# ------------------------------------------------------------------------------------------
# Flow: viscosity, conservation, fixed points, Poiseuille, symmetry
# ------------------------------------------------------------------------------------------

def _shear_wave_nu(tau, dim, L=64, t1=200, t2=1200):
    shape = (L, 1) if dim == 2 else (L, 1, 1)
    o = oracle.Oracle(shape, bc=(BC_PERIODIC,) * 3, tau=tau)
    x = np.arange(L)
    s = np.sin(2 * np.pi * x / L)
    for k in range(L):
        o.f[:, k] = oracle.flow_equilibrium(dim, 1.0, [0.0, 1e-4 * s[k], 0.0][:dim])
    o.step_flow(t1)
    a1 = (o.u[1] * s).sum() / (s * s).sum()
    o.step_flow(t2 - t1)
    a2 = (o.u[1] * s).sum() / (s * s).sum()
    kk = 2 * np.pi / L
    return math.log(a1 / a2) / (kk * kk * (t2 - t1))


@pytest.mark.parametrize("dim,tau", [(2, 0.8), (2, 1.2), (3, 0.8)])
def test_shear_wave_viscosity(dim, tau):
    """A decaying shear wave gives nu = (tau - 1/2)/3."""
    nu = _shear_wave_nu(tau, dim)
    assert nu == pytest.approx((tau - 0.5) / 3.0, rel=1e-3)


def test_residual_is_mean_change_per_step_since_last_check():
    """The steady-state residual of a decaying wave has a closed form.  With v^n = a e^(-lam n) s
    (flow: shear wave, lam = nu k^2; transport: C = C0 + a e^(-lam n) s on a fluid at rest,
    lam = D k^2), the residual over the checks at 100, 200 and the cap 250 is, at n = 251 steps
    after the start (one step run before the solve), ||v^251 - v^201|| / (50 ||v^251||)."""
    L, K, cap = 64, 100, 250
    x = np.arange(L)
    s = np.sin(2 * np.pi * x / L)
    kk = 2 * np.pi / L
    # flow
    tau = 0.8
    o = oracle.Oracle((L, 1), bc=(BC_PERIODIC,) * 3, tau=tau)
    for k in range(L):
        o.f[:, k] = oracle.flow_equilibrium(2, 1.0, [0.0, 1e-4 * s[k]])
    o.step_flow(1)
    r = o.solve_steady(mode=oracle.SEQUENTIAL, tol_flow=0.0, tol_ade=0.0, max_steps=cap,
                       check_every=K)
    lam = (tau - 0.5) / 3.0 * kk * kk
    assert r.steps_flow == cap
    assert r.res_flow == pytest.approx((math.exp(50 * lam) - 1.0) / 50, rel=5e-3)
    # transport
    tau_c, c0, a0 = 0.7, 1.0, 0.1
    o = oracle.Oracle((L, 1), bc=(BC_PERIODIC,) * 3, tau=0.8, tau_c=tau_c)
    for k in range(L):
        o.g[:, k] = oracle.ade_equilibrium(5, c0 + a0 * s[k], [0.0, 0.0])
    o.step_coupled(1)
    r = o.solve_steady(mode=oracle.CONCURRENT, tol_flow=0.0, tol_ade=0.0, max_steps=cap,
                       check_every=K)
    lam = (tau_c - 0.5) / 3.0 * kk * kk
    a = a0 * math.exp(-lam * 251)
    ss = float((s * s).sum())
    expect = a * (math.exp(50 * lam) - 1.0) * math.sqrt(ss) / (50 * math.sqrt(L * c0 * c0 + a * a * ss))
    assert r.res_ade == pytest.approx(expect, rel=5e-3)
    assert r.res_flow == 0.0  # a fluid at rest: no change and no velocity


def test_table1_flow_relaxation_time():
    """Table 1's tau = 0.6706 runs at the lattice viscosity (tau - 1/2)/3 = 0.05687."""
    t1 = golden("table1.json")
    nu = _shear_wave_nu(t1["tau"], 2)
    assert nu == pytest.approx((t1["tau"] - 0.5) / 3.0, rel=1e-3)


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_conserved_periodic_with_obstacles(dim):
    """Periodic box with solid obstacles: the total mass is constant to 1e-12 (FP64)."""
    shape = (24, 20) if dim == 2 else (12, 10, 8)
    N = int(np.prod(shape))
    rng = np.random.default_rng(11)
    cls = np.where(rng.random(N) < 0.2, FLOW_SOLID | ADE_SOLID, 0).astype(np.uint8)
    o = oracle.Oracle(shape, cls, bc=(BC_PERIODIC,) * 3, tau=0.7)
    for k in range(N):
        if cls[k] == 0:
            u = 0.03 * rng.standard_normal(dim)
            o.f[:, k] = oracle.flow_equilibrium(dim, 1.0 + 0.05 * rng.standard_normal(), u)
    m0 = o.f.sum()
    o.step_flow(10000 if dim == 2 else 2000)
    assert abs(o.f.sum() - m0) / m0 < 1e-12
    assert abs(o.rho.sum() - m0) / m0 < 1e-12


def test_rest_state_is_fixed_point_in_closed_box():
    shape = (16, 12)
    rng = np.random.default_rng(2)
    cls = np.where(rng.random(192) < 0.25, FLOW_SOLID, 0).astype(np.uint8)
    o = oracle.Oracle(shape, cls, bc=(BC_WALL, BC_WALL), tau=0.9)
    f0 = o.f.copy()
    o.step_flow(50)
    assert np.allclose(o.f, f0, atol=1e-15, rtol=0)
    assert np.abs(o.u).max() < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_inflow_is_steady_without_walls(dim):
    """With periodic cross axes and no obstacles, uniform flow at the inlet velocity and the
    outlet density is a fixed point of the inlet, the outlet and the interior."""
    shape = (12, 5) if dim == 2 else (4, 3, 12)
    u_in = 0.02
    o = oracle.Oracle(shape, bc=(BC_PERIODIC,) * 3 if dim == 3 else (BC_INOUT, BC_PERIODIC),
                      u_in=u_in, tau=0.75)
    if dim == 3:
        o.p.bc[2] = BC_INOUT
    u = [u_in, 0.0] if dim == 2 else [0.0, 0.0, u_in]
    feq = oracle.flow_equilibrium(dim, 1.0, u)
    o.f[:] = feq[:, None]
    o.step_flow(20)
    assert np.allclose(o.f, feq[:, None], atol=1e-15, rtol=0)
    fa = 0 if dim == 2 else 2
    assert np.allclose(o.u[fa], u_in, atol=1e-15, rtol=0)


def _poiseuille(H, tau, u_in=0.01):
    nx = 4 * H
    o = oracle.Oracle((nx, H), tau=tau, u_in=u_in)
    r = o.solve_steady(mode=oracle.SEQUENTIAL, tol_flow=1e-11, tol_ade=1.0, max_steps=100000,
                       check_every=100)
    return o, r, nx


@pytest.mark.slow
def test_poiseuille_profile_flux_and_pressure_drop():
    """Inlet-driven channel of width H (walls half-way outside the first and last rows):
    - the flux through every cross-section equals the injected flux u_in (H - 1/3) (the two
      inlet corner links cross a wall and bounce back without injection);
    - the developed profile is the parabola with zeros at the walls: error of second order
      in H, and nearly exact at tau = 1/2 + sqrt(3)/4 where half-way bounce-back is exact;
    - the pressure gradient is d rho/dx = -36 nu rho Ubar / H^2."""
    errs = {}
    for H, tau in [(8, 0.8), (16, 0.8), (8, 0.5 + math.sqrt(3) / 4)]:
        o, r, nx = _poiseuille(H, tau)
        assert r.converged
        ux = o.u[0].reshape(H, nx)
        rho = o.rho.reshape(H, nx)
        flux = (rho * ux).sum(axis=0)
        assert np.allclose(flux, 0.01 * (H - 1 / 3), rtol=1e-8, atol=0)
        xm = nx // 2
        y = np.arange(H)
        par = (y + 0.5) * (H - 0.5 - y)
        prof = ux[:, xm]
        amp = (prof * par).sum() / (par * par).sum()
        errs[(H, tau)] = np.abs(prof - amp * par).max() / prof.max()
        nu = (tau - 0.5) / 3
        rbar = rho[:, xm].mean()
        ubar = flux[xm] / H / rbar
        drdx = (rho[:, xm + 1].mean() - rho[:, xm - 1].mean()) / 2
        assert drdx == pytest.approx(-36 * nu * rbar * ubar / H ** 2, rel=0.02)
    assert errs[(8, 0.5 + math.sqrt(3) / 4)] < 1e-4
    assert errs[(8, 0.8)] < 1e-2
    assert 3.0 < errs[(8, 0.8)] / errs[(16, 0.8)] < 5.0


@pytest.mark.parametrize("dim", [2, 3])
def test_mirror_symmetric_geometry_gives_mirror_symmetric_fields(dim):
    """A geometry symmetric about the channel mid-plane gives u_x, rho, C symmetric and the
    cross velocity antisymmetric (catches a wrong opposite or a transposed direction)."""
    if dim == 2:
        shape = (20, 10)
    else:
        shape = (6, 8, 14)
    N = int(np.prod(shape))
    rng = np.random.default_rng(5)
    g = (rng.random(shape[::-1]) < 0.15)
    g = g | g[..., ::-1, :] if dim == 3 else g | g[::-1, :]  # symmetric in y
    cls = np.where(g.reshape(-1), FLOW_SOLID | ADE_SOLID, 0).astype(np.uint8)
    o = oracle.Oracle(shape, cls, tau=0.8, tau_c=0.7, u_in=0.02, k_sink=1e-2)
    o.step_coupled(200)
    ax = 0 if dim == 2 else 1  # numpy axis of y in the [z][y][x] / [y][x] view

    def mirror(a):
        v = a.reshape(shape[::-1])
        return np.flip(v, axis=ax).reshape(-1)

    fa = 0 if dim == 2 else 2
    assert np.allclose(o.u[fa], mirror(o.u[fa]), atol=1e-14)
    assert np.allclose(o.u[1], -mirror(o.u[1]), atol=1e-14)
    assert np.allclose(o.rho, mirror(o.rho), atol=1e-13)
    assert np.allclose(o.conc, mirror(o.conc), atol=1e-13)
    assert np.abs(o.u[fa]).max() > 1e-3


# ------------------------------------------------------------------------------------------
# Transport: diffusion, advection, Dirichlet exponential, sink, balance
# ------------------------------------------------------------------------------------------

def _gaussian(sig0, dim=2, q=None, tau_c=0.8, u=(0.0, 0.0, 0.0), u_scale=1.0, v_expect=None):
    """Error of a Gaussian advected by the frozen field u, which transport sees as u_scale * u,
    against the closed form moving at v_expect (default u_scale * u); and the relative change
    of its mass."""
    L = int(16 * sig0)
    shape = (L, L) if dim == 2 else (L, L, L)
    q = q or (5 if dim == 2 else 7)
    cs2 = 0.25 if q == 7 else 1 / 3
    D = cs2 * (tau_c - 0.5)
    t = int(3 * sig0 * sig0 / D / 4)
    o = oracle.Oracle(shape, bc=(BC_PERIODIC,) * 3, tau_c=tau_c, k_sink=0.0, ade_q=q,
                      u_scale=u_scale)
    k = np.arange(o.N)
    x, y, z = k % L, (k // L) % L, k // (L * L)
    c0 = L // 2
    r2 = (x - c0) ** 2 + (y - c0) ** 2 + ((z - c0) ** 2 if dim == 3 else 0)
    C0 = np.exp(-r2 / (2 * sig0 ** 2))
    uu = np.zeros((dim, o.N))
    for a in range(dim):
        uu[a] = u[a]
    for kk in range(o.N):
        o.g[:, kk] = oracle.ade_equilibrium(q, C0[kk], list(u_scale * uu[:, kk]))
    o.step_ade(t, u=uu)
    s2 = sig0 ** 2 + 2 * D * t
    v = [u_scale * ua for ua in u] if v_expect is None else list(v_expect)
    rr = (x - c0 - v[0] * t) ** 2 + (y - c0 - v[1] * t) ** 2
    if dim == 3:
        rr = rr + (z - c0 - v[2] * t) ** 2
    ex = C0.sum() / (2 * np.pi * s2) ** (dim / 2) * np.exp(-rr / (2 * s2))
    return np.abs(o.conc - ex).max() / ex.max(), o.conc.sum() / C0.sum() - 1.0


def test_gaussian_diffusion_second_order():
    """C(x,t) = M/(2 pi (s0^2 + 2 D t)) exp(-|x|^2 / (2 (s0^2 + 2 D t))), D = (tau_c - 1/2)/3;
    the error falls by ~4 when the initial width doubles; mass is conserved."""
    e4, m4 = _gaussian(4)
    e8, m8 = _gaussian(8)
    assert e4 < 8e-3 and abs(m4) < 1e-13 and abs(m8) < 1e-13
    assert 3.3 < e4 / e8 < 4.7


def test_gaussian_advection_and_3d_and_d2q9():
    e_adv, _ = _gaussian(4, u=(0.05, 0.02, 0.0))
    assert e_adv < 5e-3
    e9, _ = _gaussian(4, q=9)
    assert e9 < 8e-3
    e3, m3 = _gaussian(3, dim=3)
    assert e3 < 2e-2 and abs(m3) < 1e-13


@pytest.mark.parametrize("q", [5, 9])
def test_velocity_scale_moves_the_gaussian_at_the_scaled_speed(q):
    """Transport sees the flow velocity times u_scale (the factor between the time steps of
    the two lattices in the paper's units, Table 1).  A Gaussian in a frozen field u with
    u_scale = 2.5 moves at 2.5 u: it matches the closed form at the scaled speed as closely as
    the unscaled Gaussian at that same speed, and is far from the closed form at u itself."""
    e_scaled, m = _gaussian(4, q=q, u=(0.02, 0.008, 0.0), u_scale=2.5)
    e_direct, _ = _gaussian(4, q=q, u=(0.05, 0.02, 0.0))
    assert e_scaled < 8e-3 and abs(m) < 1e-13
    assert e_scaled == pytest.approx(e_direct, rel=1e-6)
    # against the closed form at the unscaled speed the same run is far off: over t steps its
    # centre has moved 1.5 u t further
    e_unscaled, _ = _gaussian(4, q=q, u=(0.02, 0.008, 0.0), u_scale=2.5, v_expect=(0.02, 0.008, 0.0))
    assert e_unscaled > 20 * e_scaled


def _late_diffusivity(tau_c, q, t1=1000, t2=3000, sig0=4.0, L=64):
    o = oracle.Oracle((L, L), bc=(BC_PERIODIC,) * 3, tau_c=tau_c, k_sink=0.0, ade_q=q)
    k = np.arange(o.N)
    x, y = k % L, k // L
    c0 = L // 2
    C0 = np.exp(-((x - c0) ** 2 + (y - c0) ** 2) / (2 * sig0 ** 2))
    for kk in range(o.N):
        o.g[:, kk] = oracle.ade_equilibrium(q, C0[kk], [0.0, 0.0])
    uu = np.zeros((2, o.N))

    def var(C):
        return ((x - c0) ** 2 * C).sum() / C.sum()

    o.step_ade(t1, u=uu)
    va = var(o.conc)
    o.step_ade(t2 - t1, u=uu)
    return (var(o.conc) - va) / (2 * (t2 - t1))


@pytest.mark.parametrize("q", [5, 9])
def test_table1_diffusion_coefficient(q):
    """Table 1 prints tau_D = 0.5036 with D = 0.0012 mm^2/s.  With dx^2/dt = 1 mm^2/s the
    oracle's measured diffusivity (variance growth 2 D t) reproduces that D."""
    t1 = golden("table1.json")
    D = _late_diffusivity(t1["tau_D"], q)
    assert D == pytest.approx(t1["D_mm2_per_s"], rel=1e-6)


@pytest.mark.parametrize("Pe", [1.0, 10.0])
def test_steady_advection_diffusion_exponential(Pe):
    """1-D steady ADE with C = 1 at the inlet ghost and C = 0 at the outlet ghost (distance
    L = nx + 1): C = (exp(Pe xi) - exp(Pe)) / (1 - exp(Pe)); second-order in 1/L."""
    errs = []
    for nx in (31, 63):
        tau_c = 1.0
        D = (tau_c - 0.5) / 3
        L = nx + 1
        u = Pe * D / L
        o = oracle.Oracle((nx, 1), bc=(BC_INOUT, BC_PERIODIC), ade_outlet=1, c_in=1.0, c_out=0.0,
                          u_in=u, tau_c=tau_c, k_sink=0.0)
        uu = np.zeros((2, nx))
        uu[0] = u
        o.step_ade(int(5 * L * L / D), u=uu)
        xi = (np.arange(nx) + 1) / L
        ex = (np.exp(Pe * xi) - np.exp(Pe)) / (1 - np.exp(Pe))
        errs.append(np.abs(o.conc - ex).max())
    assert errs[0] < (2e-5 if Pe == 1.0 else 5e-3)
    assert 3.5 < errs[0] / errs[1] < 4.5


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_sink_decays_geometrically(dim):
    """Every node consumes at rate k, no flow: C^t = C0 (1-k)^(t-1) and the current is
    N k C^t, exactly (the streamed moment of step t sees t-1 consumptions)."""
    shape = (8, 6) if dim == 2 else (4, 3, 5)
    N = int(np.prod(shape))
    k_sink, C0 = 0.1, 0.7
    o = oracle.Oracle(shape, np.full(N, SINK, np.uint8), bc=(BC_PERIODIC,) * 3, k_sink=k_sink,
                      tau_c=0.9)
    o.g[:] = oracle.ade_equilibrium(o.qa, C0, [0.0] * dim)[:, None]
    uu = np.zeros((dim, N))
    for t in range(1, 30):
        o.step_ade(1, u=uu)
        expect = C0 * (1 - k_sink) ** (t - 1)
        assert np.allclose(o.conc, expect, rtol=1e-13, atol=0)
        s = o.sums()
        assert s[6] == pytest.approx(N * k_sink * expect, rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("K,C0", [(5.0, 0.1), (0.4, 0.4), (0.02, 0.4)])
def test_uniform_monod_sink_follows_the_scalar_map(dim, K, C0):
    """Eq. 16's substrate factor on every node, no flow: a uniform state stays uniform, and
    its concentration follows the scalar map C <- C - k K C / (K + C), iterated here on its own,
    from well below K (near first order) to far above it (near zero order); the current is
    N k K C / (K + C)."""
    shape = (8, 6) if dim == 2 else (4, 3, 5)
    N = int(np.prod(shape))
    k = 0.1
    o = oracle.Oracle(shape, np.full(N, SINK, np.uint8), bc=(BC_PERIODIC,) * 3, k_sink=k,
                      k_half=K, tau_c=0.9)
    o.g[:] = oracle.ade_equilibrium(o.qa, C0, [0.0] * dim)[:, None]
    uu = np.zeros((dim, N))
    c = C0
    for t in range(1, 30):
        o.step_ade(1, u=uu)
        assert np.allclose(o.conc, c, rtol=1e-13, atol=0), t
        assert o.sums()[6] == pytest.approx(N * k * K * c / (K + c), rel=1e-13)
        c = c - k * K * c / (K + c)


def test_monod_sink_limits():
    """Saturated (C >> K): each step removes k K C / (K + C), between k K - k K^2 / (K + C)
    and k K, so the concentration falls linearly: C^t lies above C0 - (t - 1) k K, and by at
    most (t - 1) k K^2 / (K + C).
    K -> infinity: the first-order sink k C (geometric decay)."""
    shape = (6, 5)
    N = 30
    k, K, C0 = 0.2, 1e-3, 1.0
    o = oracle.Oracle(shape, np.full(N, SINK, np.uint8), bc=(BC_PERIODIC,) * 3, k_sink=k,
                      k_half=K, tau_c=0.8)
    o.g[:] = oracle.ade_equilibrium(5, C0, [0.0, 0.0])[:, None]
    uu = np.zeros((2, N))
    for t in range(1, 40):
        o.step_ade(1, u=uu)
        lin = C0 - (t - 1) * k * K
        # each step removes less than k K, and more than k K - k K^2 / (K + C); 1e-15 allows
        # for the rounding of the moment of the stored populations
        assert o.conc.min() >= lin - 1e-15
        assert o.conc.max() - lin <= (t - 1) * k * K * K / (K + o.conc.min()) + 1e-15
    big = oracle.Oracle(shape, np.full(N, SINK, np.uint8), bc=(BC_PERIODIC,) * 3, k_sink=k,
                        k_half=1e15, tau_c=0.8)
    big.g[:] = oracle.ade_equilibrium(5, C0, [0.0, 0.0])[:, None]
    for t in range(1, 20):
        big.step_ade(1, u=uu)
        assert np.allclose(big.conc, C0 * (1 - k) ** (t - 1), rtol=1e-12, atol=0)


@pytest.mark.parametrize("k_half", [0.0, 0.3])
def test_substrate_balance_closed_box(k_half):
    """Closed box with obstacles, sinks and an arbitrary frozen velocity: each step the total
    substrate falls by exactly the consumption, sum C^(t+1) = sum C^t - I^t (first-order and
    saturating consumption)."""
    shape = (14, 11)
    N = 154
    rng = np.random.default_rng(9)
    r = rng.random(N)
    cls = np.where(r < 0.15, FLOW_SOLID | ADE_SOLID, np.where(r < 0.35, SINK, 0)).astype(np.uint8)
    cls[(r > 0.9)] = FLOW_SOLID | SINK
    o = oracle.Oracle(shape, cls, bc=(BC_WALL, BC_WALL), k_sink=0.05, tau_c=0.65, k_half=k_half)
    o.g[:] = rng.random(o.g.shape)
    o.g[:, (cls & ADE_SOLID) > 0] = 0.0
    uu = 0.05 * rng.standard_normal((2, N))
    o.step_ade(1, u=uu)
    for _ in range(40):
        s_prev = o.sums()
        o.step_ade(1, u=uu)
        s = o.sums()
        assert s[5] == pytest.approx(s_prev[5] - s_prev[6], rel=1e-13)


@pytest.mark.parametrize("k_half", [0.0, 0.1])
def test_substrate_balance_channel_fluxes(k_half):
    """Open channel (D2Q5): the change of total substrate equals inlet inflow minus what
    leaves through the inlet and outlet planes plus what the zero-gradient outlet returns,
    minus the consumption, to round-off."""
    nx, ny = 12, 7
    N = nx * ny
    rng = np.random.default_rng(4)
    cls = np.zeros(N, np.uint8)
    inner = rng.random(N) < 0.2
    xs = np.arange(N) % nx
    cls[inner & (xs > 1) & (xs < nx - 2)] = FLOW_SOLID | ADE_SOLID
    cls[(cls == 0) & (rng.random(N) < 0.3)] = SINK
    u_in, c_in = 0.03, 0.8
    o = oracle.Oracle((nx, ny), cls, u_in=u_in, c_in=c_in, k_sink=0.02, tau_c=0.7, k_half=k_half)
    uu = 0.02 * rng.standard_normal((2, N))
    o.step_ade(25, u=uu)
    geq_in = oracle.ade_equilibrium(5, c_in, [u_in, 0.0])
    open_ = (cls & ADE_SOLID) == 0
    for _ in range(10):
        s_prev = o.sums()
        gs = o.g.copy()  # post-collision populations of the previous step
        o.step_ade(1, u=uu)
        s = o.sums()
        rows = np.arange(ny)
        k0 = rows * nx
        k1 = rows * nx + nx - 1
        inflow = geq_in[1] * open_[k0].sum()
        out_inlet = gs[3, k0][open_[k0]].sum()      # moving -x at x = 0 leaves
        out_outlet = gs[1, k1][open_[k1]].sum()     # moving +x at x = nx-1 leaves
        back = gs[3, k1][open_[k1]].sum()           # zero-gradient ghost returns the -x ones
        expect = s_prev[5] - s_prev[6] + inflow - out_inlet - out_outlet + back
        assert s[5] == pytest.approx(expect, rel=1e-13)


def test_concurrent_and_sequential_reach_the_same_steady_state():
    """Both solve orders converge to the same fixed point of the coupled problem."""
    import mfc_inputs as mi
    shape = (40, 16)
    cls = mi.mark_sink_layer(shape, mi.bernoulli_block(shape, 0.25, 3, block=(12, 28)), SINK)
    kw = dict(tau=0.9, tau_c=0.8, u_in=0.02, k_sink=2e-3)
    a = oracle.Oracle(shape, cls, **kw)
    ra = a.solve_steady(oracle.SEQUENTIAL, 1e-11, 1e-11, 200000, 50)
    b = oracle.Oracle(shape, cls, **kw)
    rb = b.solve_steady(oracle.CONCURRENT, 1e-11, 1e-11, 200000, 50)
    assert ra.converged and rb.converged
    assert np.linalg.norm(a.u - b.u) / np.linalg.norm(a.u) < 1e-7
    assert np.linalg.norm(a.conc - b.conc) / np.linalg.norm(a.conc) < 1e-7
    assert ra.current == pytest.approx(rb.current, rel=1e-7)


# ------------------------------------------------------------------------------------------
# Biofilm rule and the counter-based generator
# ------------------------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    gd = golden("splitmix64.json")
    gamma = 0x9E3779B97F4A7C15
    for k, want in enumerate(gd["outputs"], start=1):
        x = (k * gamma - gamma) & 0xFFFFFFFFFFFFFFFF
        assert oracle.splitmix64(x) == int(want, 16)


def test_input_generator_splitmix64_published_outputs():
    import mfc_inputs as mi
    gd = golden("splitmix64.json")
    gamma = 0x9E3779B97F4A7C15
    xs = np.array([(k * gamma - gamma) & 0xFFFFFFFFFFFFFFFF for k in range(1, 5)], np.uint64)
    got = mi.splitmix64(xs)
    assert [int(v) for v in got] == [int(w, 16) for w in gd["outputs"]]


def test_biofilm_rule_cases():
    """Hand-built cases: eligibility (open node, a sink neighbour, C strictly above the
    threshold), the draw threshold pinned by the first published splitmix64 output, and
    decisions taken on the classes from before the pass."""
    nx, ny = 6, 4
    N = nx * ny
    cls = np.zeros(N, np.uint8)
    cls[1] = SINK            # node (1,0) is biofilm
    cls[23] = FLOW_SOLID | ADE_SOLID
    o = oracle.Oracle((nx, ny), cls)
    conc = np.full(N, 0.9)
    # node 0 (neighbour of the sink) with seed 0, cycle 0: h = splitmix64(0) = 0xe220a8397b1dcdaf
    u0 = (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53          # ~0.8833
    out, n = o.biofilm_convert(0, 0, prob=u0 - 1e-6, c_thresh=0.5, conc=conc)
    assert out[0] == 0
    out, n = o.biofilm_convert(0, 0, prob=u0 + 1e-6, c_thresh=0.5, conc=conc)
    assert out[0] == (FLOW_SOLID | SINK)
    # prob 1: exactly the open nodes next to the original sink convert (no chaining)
    out, n = o.biofilm_convert(0, 0, prob=1.0, c_thresh=0.5, conc=conc)
    expect = {0, 2, 6, 7, 8}
    assert set(np.nonzero(out != cls)[0]) == expect and n == len(expect)
    # threshold is strict; prob 0 converts nothing
    out, n = o.biofilm_convert(0, 0, prob=1.0, c_thresh=0.9, conc=conc)
    assert n == 0
    out, n = o.biofilm_convert(0, 0, prob=0.0, c_thresh=0.5, conc=conc)
    assert n == 0


def test_biofilm_rule_cases_3d():
    """3-D: the neighbours are the 18 moving directions of the D3Q19 flow set, i.e. the six
    face and twelve edge neighbours of the 3x3x3 cube around a node, never its eight corners.
    With prob 1, every open node among them converts; a blocked face neighbour and an open
    corner neighbour do not."""
    n = 5
    N = n ** 3

    def k(x, y, z):
        return x + n * (y + n * z)

    cls = np.zeros(N, np.uint8)
    cls[k(2, 2, 2)] = SINK
    cls[k(3, 2, 2)] = FLOW_SOLID | ADE_SOLID  # a blocked face neighbour
    o = oracle.Oracle((n, n, n), cls)
    conc = np.full(N, 0.9)
    out, cnt = o.biofilm_convert(7, 3, prob=1.0, c_thresh=0.5, conc=conc)
    faces = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    edges = [(1, 1, 0), (1, -1, 0), (-1, 1, 0), (-1, -1, 0), (1, 0, 1), (1, 0, -1), (-1, 0, 1),
             (-1, 0, -1), (0, 1, 1), (0, 1, -1), (0, -1, 1), (0, -1, -1)]
    expect = {k(2 + a, 2 + b, 2 + c) for a, b, c in faces + edges} - {k(3, 2, 2)}
    assert len(expect) == 17
    assert set(np.nonzero(out != cls)[0]) == expect and cnt == 17
    assert all(out[j] == (FLOW_SOLID | SINK) for j in expect)
    assert out[k(3, 3, 3)] == 0 and out[k(1, 1, 1)] == 0  # corners are not neighbours
    # the first node scanned is still decided by its own draw: (2,2,1) = node 37, seed 7,
    # cycle 3: h = splitmix64(7 ^ (3 << 32) ^ 37)
    h = oracle.splitmix64(7 ^ (3 << 32) ^ k(2, 2, 1))
    u = (h >> 11) / 2.0 ** 53
    out, _ = o.biofilm_convert(7, 3, prob=u - 1e-9, c_thresh=0.5, conc=conc)
    assert out[k(2, 2, 1)] == 0
    out, _ = o.biofilm_convert(7, 3, prob=u + 1e-9, c_thresh=0.5, conc=conc)
    assert out[k(2, 2, 1)] == (FLOW_SOLID | SINK)


def test_biofilm_rule_rate():
    """On many eligible nodes the converted fraction is prob within binomial bounds."""
    nx, ny = 200, 3
    cls = np.zeros(nx * ny, np.uint8)
    cls[nx:2 * nx] = SINK
    o = oracle.Oracle((nx, ny), cls)
    conc = np.ones(nx * ny)
    out, n = o.biofilm_convert(12345, 7, prob=0.05, c_thresh=0.5, conc=conc)
    m = 2 * nx
    assert abs(n - 0.05 * m) < 4 * math.sqrt(m * 0.05 * 0.95)
    out2, n2 = o.biofilm_convert(12345, 8, prob=0.05, c_thresh=0.5, conc=conc)
    assert not np.array_equal(out, out2)


def test_steady_rest_populations_closed_form():
    """The rest populations never stream, so at a steady state they are fixed points of their
    own collision: F_0 = F_0^(0)(rho, u) on every open node, and G_0 = w_0 C (1 - k tau_c) on
    consumption nodes (w_0 C elsewhere).  This fixes the sink's split over the directions."""
    import mfc_inputs as mi
    shape = (36, 14)
    cls = mi.mark_sink_layer(shape, mi.bernoulli_block(shape, 0.25, 8, block=(10, 26)), SINK)
    tau, tau_c, k = 0.9, 0.8, 5e-3
    o = oracle.Oracle(shape, cls, tau=tau, tau_c=tau_c, u_in=0.02, k_sink=k)
    r = o.solve_steady(oracle.CONCURRENT, 1e-12, 1e-12, 300000, 50)
    assert r.converged
    w0f = oracle.flow_equilibrium(2, 1.0, [0.0, 0.0])[0]
    w0a = oracle.ade_equilibrium(5, 1.0, [0.0, 0.0])[0]
    open_f = (cls & FLOW_SOLID) == 0
    uu = o.u[0] ** 2 + o.u[1] ** 2
    f0 = w0f * o.rho * (1 - 1.5 * uu)
    assert np.allclose(o.f[0, open_f], f0[open_f], rtol=1e-8, atol=0)
    open_a = (cls & ADE_SOLID) == 0
    sink = (cls & SINK) > 0
    g0 = w0a * o.conc * np.where(sink, 1 - k * tau_c, 1.0)
    assert np.allclose(o.g[0, open_a], g0[open_a], rtol=1e-8, atol=1e-15)


# ------------------------------------------------------------------------------------------
# Range guard of the solve (no counterpart in the paper: it stops a solve whose flow has left
# the low-Mach range of the equilibrium of Eq. 5)
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_flow_at_the_sound_speed_stops_the_solve_at_the_first_check(dim):
    """A uniform flow in a periodic box is a fixed point of stream and collide at any speed.
    Above the sound speed 1/sqrt(3) = 0.577 the solve stops at its first check with the range
    flag; every open node counts.  Just below it, the same box runs to the step cap."""
    shape = (12, 6) if dim == 2 else (6, 4, 5)
    N = int(np.prod(shape))
    for speed, out in ((0.6, True), (0.55, False)):
        o = oracle.Oracle(shape, bc=(BC_PERIODIC,) * dim, tau=0.8)
        u = [0.0] * dim
        u[0] = speed
        o.f[:] = oracle.flow_equilibrium(dim, 1.0, u)[:, None]
        r = o.solve_steady(mode=oracle.CONCURRENT, tol_flow=0.0, tol_ade=0.0, max_steps=50,
                           check_every=10)
        assert np.allclose(o.u[0], speed, atol=1e-14, rtol=0)
        assert r.unstable == int(out) and not r.converged
        assert r.steps_flow == (10 if out else 50)
        assert o.sums()[8] == (N if out else 0)


def test_range_guard_counts_fast_and_non_positive_density_nodes():
    """The count of the guard over hand-set fields: nodes with |u|^2 >= 1/3 (on the boundary
    too) or rho <= 0 among the flow-open nodes; blocked nodes never count, nor does a high
    density (the 128x64 channel's steady state has rho near 2 upstream of its block)."""
    shape = (8, 4)
    cls = np.zeros(32, np.uint8)
    cls[5] = FLOW_SOLID | ADE_SOLID
    o = oracle.Oracle(shape, cls, bc=(BC_PERIODIC, BC_PERIODIC))
    o.rho[:] = 1.0
    o.u[:] = 0.0
    o.u[0, 1] = 0.6                        # above the sound speed
    o.u[0, 2], o.u[1, 2] = 0.4, 0.42       # |u|^2 = 0.3364 >= 1/3 by its two components
    o.u[0, 3] = math.sqrt(1.0 / 3.0) - 1e-9  # just below
    o.rho[4] = 0.0                         # non-positive density
    o.u[0, 5] = 0.9                        # blocked: not counted
    o.rho[6] = 1e-12                       # small but positive
    o.rho[7] = 2.5                         # high density: not out of range
    assert o.sums()[8] == 3


# ------------------------------------------------------------------------------------------
# Agent-based biofilm (Sec. 3.3): attachment, growth, spreading
# ------------------------------------------------------------------------------------------

def _electrode_only(shape, seed):
    import mfc_inputs as mi
    cls = mi.overlapping_balls(shape, 4 if len(shape) == 3 else 6, 0.7, seed)
    return np.where((cls & 3) == 3, 3, 0).astype(np.uint8)


def _front(o):
    """The front by brute force over the 3x3(x3) neighbourhood: open nodes without biomass with
    an electrode node among their neighbours along the flow set's directions."""
    c, _, _ = oracle.velocity_set(9 if o.dim == 2 else 19)
    shape = o.shape if o.dim == 3 else (o.shape[0], o.shape[1], 1)
    cls = o.cls.reshape(shape[::-1])
    out = set()
    for z in range(shape[2]):
        for y in range(shape[1]):
            for x in range(shape[0]):
                if cls[z, y, x] != 0:
                    continue
                for d in c[1:]:
                    sx, sy, sz = x + d[0], y + d[1], z + d[2]
                    if 0 <= sx < shape[0] and 0 <= sy < shape[1] and 0 <= sz < shape[2] \
                            and cls[sz, sy, sx] == 3:
                        out.add(x + shape[0] * (y + shape[1] * z))
                        break
    return out


@pytest.mark.parametrize("shape", [(40, 24), (14, 12, 10)])
def test_agent_attachment_count_and_choice(shape):
    """Exactly k_ata front nodes attach, at C_0^bio, and they are the k_ata front nodes with the
    smallest keys (top 32 bits of the published splitmix64 hash, then the node index); with
    fewer front nodes than k_ata, all of them attach."""
    cls = _electrode_only(shape, 5)
    o = oracle.Oracle(shape, cls)
    front = _front(o)
    assert len(front) > 30
    bio = np.zeros(o.N)
    a = oracle.agent_table1(seed=11, k_ata=30, mu=0.0, Cmax_bio=1e9)
    s = o.agent_step(a, 4, bio, conc=np.zeros(o.N))
    assert s["attached"] == 30 and s["front"] == len(front)
    got = set(np.nonzero(bio)[0])
    assert got <= front and np.all(bio[list(got)] == 450.0)
    base = oracle.splitmix64(11 ^ 0x6174746163680000)
    keys = sorted(((oracle.splitmix64(base ^ (4 << 32) ^ k) >> 32) << 32 | k) for k in front)
    assert got == {k & 0xFFFFFFFF for k in keys[:30]}
    # more than the front: everything attaches; the classes follow the biomass
    o2 = oracle.Oracle(shape, cls)
    bio2 = np.zeros(o2.N)
    s2 = o2.agent_step(oracle.agent_table1(k_ata=10 ** 6, mu=0.0, Cmax_bio=1e9), 0, bio2,
                       conc=np.zeros(o2.N))
    assert s2["attached"] == len(front) and set(np.nonzero(bio2)[0]) == front
    assert np.all(o2.cls[list(front)] == (FLOW_SOLID | SINK))


def test_agent_growth_follows_the_monod_closed_form():
    """Uniform substrate C: after n steps a node's biomass is C_0 (1 + mu C / (C + K_s))^n, and
    a node at C <= 0 does not grow."""
    shape = (16, 8)
    cls = np.zeros(128, np.uint8)
    cls[:16] = 3                      # an electrode row along y = 0
    o = oracle.Oracle(shape, cls)
    bio = np.zeros(128)
    bio[40] = 100.0
    bio[41] = 100.0
    conc = np.full(128, 0.3)
    conc[41] = -0.01
    a = oracle.agent_table1(k_ata=0, mu=0.25, K_s=0.1, Cmax_bio=1e12)
    for n in range(1, 6):
        o.agent_step(a, n, bio, conc=conc)
        assert bio[40] == pytest.approx(100.0 * (1 + 0.25 * 0.3 / 0.4) ** n, rel=1e-14)
        assert bio[41] == 100.0


@pytest.mark.parametrize("shape", [(48, 32), (16, 12, 10)])
def test_agent_spreading_conserves_biomass(shape):
    """Spreading only moves biomass: over steps with no attachment and no growth the total is
    kept (to rounding), every spreading node ends with (1 - fr_spr) of what it had, and walks
    through a dense biofilm happen and end on free cells."""
    cls = _electrode_only(shape, 9)
    o = oracle.Oracle(shape, cls)
    rng = np.random.default_rng(2)
    bio = np.where(cls == 0, rng.uniform(0, 1000, o.N) * (rng.random(o.N) < 0.6), 0.0)
    total = bio.sum()
    a = oracle.agent_table1(seed=5, k_ata=0, mu=0.0, fr_spr=0.4, max_walk=2000)
    walked = 0
    for cyc in range(4):
        before = bio.copy()
        s = o.agent_step(a, cyc, bio, conc=np.zeros(o.N))
        walked += s["walk_steps"]
        assert bio.sum() == pytest.approx(total, rel=1e-13)
        assert s["total_biomass"] == pytest.approx(total, rel=1e-13)
        assert np.all(bio >= 0.0)
        assert np.all(bio[cls == 3] == 0.0)
        assert s["spread"] > 0
        # nodes that spread were above the threshold, and a new node holding biomass takes
        # at most fr_spr of the largest value (its donor's) or a shoved value
        assert np.count_nonzero(bio) == np.count_nonzero(before) + s["spread"]
    assert walked > 0


def test_agent_spreading_hand_cases():
    """A lone node above C_max^bio with free neighbours gives fr_spr of its biomass to the one the
    first draw picks; a node boxed in by biofilm shoves the chain along its walk."""
    shape = (7, 7)
    cls = np.zeros(49, np.uint8)
    o = oracle.Oracle(shape, cls)
    bio = np.zeros(49)
    k = 3 + 7 * 3
    bio[k] = 600.0
    a = oracle.agent_table1(seed=1, k_ata=0, mu=0.0)
    s = o.agent_step(a, 2, bio, conc=np.zeros(49))
    c, _, _ = oracle.velocity_set(9)
    nbrs = [(3 + d[0]) + 7 * (3 + d[1]) for d in c[1:]]  # all eight are free, in direction order
    d0 = oracle.splitmix64(oracle.splitmix64(1 ^ 0x7370726561640000 ^ (2 << 32)) ^ 0)
    j = nbrs[(d0 >> 32) % 8]
    assert s["spread"] == 1 and s["walk_steps"] == 0
    assert bio[k] == 600.0 - 0.4 * 600.0 and bio[j] == 0.4 * 600.0
    assert np.count_nonzero(bio) == 2
    # boxed in: the 3x3 block around k full of biomass below the threshold
    o = oracle.Oracle(shape, np.zeros(49, np.uint8))
    bio = np.zeros(49)
    for d in c:
        bio[(3 + d[0]) + 7 * (3 + d[1])] = 100.0
    bio[k] = 600.0
    s = o.agent_step(a, 2, bio, conc=np.zeros(49))
    assert s["spread"] == 1 and s["walk_steps"] >= 2
    assert bio.sum() == pytest.approx(600.0 + 800.0, rel=1e-15)
    assert bio[k] == 360.0 and np.count_nonzero(bio) == 10
    assert sorted(bio[bio > 0].tolist()) == [100.0] * 8 + [240.0, 360.0]
