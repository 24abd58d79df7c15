"""The allocation-free sums entry point (for callers that cannot call cudaMalloc).

It is checked through the C ABI against the check-step reduction of mfc_solve_steady on the
same fields, on two calls in a row.  This file is collected last on purpose, so that a run that
stops at the first failure has run every other test before it.
"""
import ctypes

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


def _dev(torch, a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("case", ["channel_128x64", "electrode_64x32x32"])
def test_field_sums_noalloc_matches_solve_check(P, case):
    torch = pytest.importorskip("torch")
    # the 2-D channel, and a 3-D electrode whose velocity has three component planes
    w = mi.channel_128x64() if case == "channel_128x64" else mi.electrode_3d(64, 32, 32, seed=11)
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    a = P.Lattice(w.shape, **kw)  # steps one by one and hands its fields to the new entry point
    b = P.Lattice(w.shape, **kw)  # reaches the same steps through mfc_solve_steady's check
    a.set_geometry(w.cls)
    b.set_geometry(w.cls)
    L = P.lib()
    cls = _dev(torch, w.cls, torch.uint8)
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    done = 0
    for n in (300, 800):  # two calls in a row, the second on later fields
        a.step_coupled(n - done)
        _, u_prev, c_prev, _ = a.read_fields()
        a.step_coupled(2)
        rho, u, c, _ = a.read_fields()
        b.step_coupled(n - done)
        r = b.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0, max_steps=2,
                           check_every=2)
        done = n + 2
        out.fill_(-1.0)
        # keep every device tensor referenced until the call's work is done
        d = {k: _dev(torch, v, torch.float64)
             for k, v in dict(rho=rho, u=u, u_prev=u_prev, c=c, c_prev=c_prev).items()}
        st = L.mfc_field_sums_noalloc(w.nodes, w.dim, cls.data_ptr(), d["rho"].data_ptr(),
                                      d["u"].data_ptr(), d["u_prev"].data_ptr(), d["c"].data_ptr(),
                                      d["c_prev"].data_ptr(), w.k_sink, out.data_ptr(),
                                      stream.cuda_stream)
        assert st == P.MFC_OK
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert o[7] == 0.0
        # the tolerances of the other reduction tests: the two lattices run different
        # instantiations of the step at the compared steps, which may round FP32 differently;
        # the solve's residual is the change over its two steps per step
        assert o[8] / 2 == pytest.approx(r.res_flow, rel=1e-3)
        assert o[9] / 2 == pytest.approx(r.res_ade, rel=1e-3)
        assert o[6] == pytest.approx(r.current, rel=1e-5)
        assert o[2] == pytest.approx(r.mass, rel=1e-7)
        assert o[5] == pytest.approx(r.substrate, rel=1e-5)
    a.close()
    b.close()


def test_field_sums_noalloc_rejects_sizes_beyond_its_scratch(P):
    L = P.lib()
    z = ctypes.c_void_p(8)  # never dereferenced: the size check comes first
    assert L.mfc_field_sums_noalloc(2097152 + 1, 2, z, z, z, z, z, z, 1e-3, z, None) == P.MFC_ERR_ARG
    assert L.mfc_field_sums_noalloc(0, 2, z, z, z, z, z, z, 1e-3, z, None) == P.MFC_ERR_ARG
    assert L.mfc_field_sums_noalloc(100, 4, z, z, z, z, z, z, 1e-3, z, None) == P.MFC_ERR_ARG
