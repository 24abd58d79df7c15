"""Slab decomposition (one lattice split along its flow axis) against the whole lattice.

Slabs held by one process on one GPU, exchanging halos through device buffers after every step,
compute exactly what the whole lattice computes: the same kernels on the same values.  Checked on
the populations after many steps (bit for bit in FP32), on the summed check sums (to the FP32
rounding of their per-block partials, whose node ranges differ), and on a steady solve.
"""
import numpy as np
import pytest

import mfc_inputs as mi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1802_07525_gb300 import build
    build.build()
    import paper_1802_07525_gb300 as P
    return P


def split(P, w, nslab, bc, precision=0, **kw):
    """The whole lattice and its slabs along the flow axis (x in 2-D, z in 3-D)."""
    from paper_1802_07525_gb300 import slab as S
    dim = w.dim
    fa = 0 if dim == 2 else 2
    n = w.shape[fa]
    cls = w.cls.reshape(w.shape[::-1])  # [z][y][x] or [y][x]
    whole = P.Lattice(w.shape, bc=bc, precision=precision, **kw)
    whole.set_geometry(w.cls)
    slabs = []
    for r in range(nslab):
        lo, hi = S.slab_bounds(n, nslab, r)
        shape = list(w.shape)
        shape[fa] = hi - lo
        part = cls[..., lo:hi] if dim == 2 else cls[lo:hi]
        g = P.Lattice(tuple(shape), bc=bc, precision=precision, cut=(r > 0, r < nslab - 1), **kw)
        g.set_geometry(np.ascontiguousarray(part).reshape(-1))
        if r > 0:
            g.set_halo_classes(0, cls[..., lo - 1] if dim == 2 else cls[lo - 1])
        if r < nslab - 1:
            g.set_halo_classes(1, cls[..., hi] if dim == 2 else cls[hi])
        slabs.append(g)
    return whole, slabs, S.LocalSlabs(slabs)


def joined(P, w, slabs, which):
    """Populations of the slabs reassembled into the whole lattice's layout."""
    dim = w.dim
    parts = [s.read_populations(which).reshape((-1,) + s.shape[::-1]) for s in slabs]
    return np.concatenate(parts, axis=-1 if dim == 2 else 1).reshape(parts[0].shape[0], -1)


CASES = [
    ("anode_2d", (2, 0), 2),
    ("anode_2d", (2, 1), 3),        # periodic cross axis
    ("electrode_3d", (0, 0, 2), 2),
    ("electrode_3d", (1, 0, 2), 3),  # periodic x
]


@pytest.mark.parametrize("name,bc,nslab", CASES)
def test_slabs_compute_what_the_whole_lattice_computes(P, name, bc, nslab):
    w = mi.anode_2d(150, 40, seed=12) if name == "anode_2d" else mi.electrode_3d(20, 16, 36, seed=13)
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    whole, slabs, local = split(P, w, nslab, bc, **kw)
    for target in (1, 7, 150):
        done = getattr(local, "_done", 0)
        local.step(target - done)
        whole.step_coupled_plain(target - done)  # the slabs' steps keep the stored fields too
        local._done = target
        for which in (P.MFC_POP_FLOW, P.MFC_POP_ADE):
            a, b = joined(P, w, slabs, which), whole.read_populations(which)
            assert np.array_equal(a, b), (target, which, float(np.abs(a - b).max()))
    # a check step: the sums over the slabs are the whole lattice's sums, to the FP32 rounding of
    # the per-block partial sums (the slabs' blocks cover other node ranges)
    s_local = local.check(20)
    s_whole = whole.step_check_sums(20)
    assert np.allclose(s_local, s_whole, rtol=1e-6, atol=1e-300)
    for g in slabs + [whole]:
        g.close()


@pytest.mark.parametrize("name,bc,nslab", [("anode_2d", (2, 0), 2), ("electrode_3d", (0, 0, 2), 3)])
def test_fp16_slabs_compute_what_the_whole_lattice_computes(P, name, bc, nslab):
    """FP16 storage: plain steps two rows per thread, rows paired along y, which no cut divides;
    the halos carry the stored FP16 values.  Populations bit for bit."""
    w = mi.anode_2d(150, 40, seed=12) if name == "anode_2d" else mi.electrode_3d(20, 16, 36, seed=13)
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    whole, slabs, local = split(P, w, nslab, bc, precision=P.MFC_FP16_DEV, **kw)
    done = 0
    for target in (1, 7, 150):
        local.step(target - done)
        whole.step_coupled_plain(target - done)
        done = target
        for which in (P.MFC_POP_FLOW, P.MFC_POP_ADE):
            a, b = joined(P, w, slabs, which), whole.read_populations(which)
            assert np.array_equal(a, b), (target, which, float(np.abs(a - b).max()))
    for g in slabs + [whole]:
        g.close()


def test_slab_steady_solve_matches_the_whole_lattice(P):
    from paper_1802_07525_gb300 import slab as S
    w = mi.electrode_3d(16, 16, 24, seed=9)
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    whole, slabs, local = split(P, w, 3, (0, 0, 2), **kw)
    r = local.solve_steady(w.tol, w.tol, w.max_steps, 100)
    rw = whole.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=w.tol, tol_ade=w.tol,
                            max_steps=w.max_steps, check_every=100)
    assert r["status"] == "converged" and rw.status == P.MFC_OK
    assert r["steps"] == rw.steps_flow
    # the sums agree to the FP32 rounding of the per-block partials
    assert r["current"] == pytest.approx(rw.current, rel=1e-6)
    assert r["res_flow"] == pytest.approx(rw.res_flow, rel=1e-4)
    assert np.array_equal(joined(P, w, slabs, P.MFC_POP_ADE), whole.read_populations(P.MFC_POP_ADE))
    assert S.residuals(r["sums"], 100)[0] == pytest.approx(r["res_flow"])
    for g in slabs + [whole]:
        g.close()


def test_cut_arguments_are_checked(P):
    with pytest.raises(P.MfcError):  # a cut on a periodic flow axis
        P.Lattice((32, 8), bc=(1, 0), cut=(1, 0))
    g = P.Lattice((32, 8), bc=(2, 0), cut=(0, 1))
    g.set_geometry(np.zeros(256, np.uint8))
    with pytest.raises(P.MfcError):  # side 0 is not a cut
        g.halo_bytes(0)
    assert g.halo_bytes(1) == (3 + 1) * 8 * 4  # three D2Q9 and one D2Q5 direction cross, FP32
    g.close()
