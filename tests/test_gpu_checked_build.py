"""The checking build (MFC_CHECK_BOUNDS): every element offset of the step kernels tested against
its array, guard regions around every device buffer.

A child process loads the checking library (MFC_LIBRARY=check) and drives every kind of work
through it: 2-D and 3-D lattices in FP32, FP16 and FP64, every boundary kind, mixed node classes,
D2Q9 transport, flow-only, transport-only and fused steps, steady solves, reads and writes of
populations, the agent model, slabs exchanging halos, and a batch.  No call may report an offset
out of range and no guard byte may change.  (This stands in for a memory checker, which is not
available here.)
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _classes(shape, seed):
    rng = np.random.default_rng(seed)
    r = rng.random(int(np.prod(shape)))
    return np.where(r < 0.15, 3, np.where(r < 0.3, 4, np.where(r < 0.35, 5, 0))).astype(np.uint8)


def _exercise():
    sys.path.insert(0, ROOT)
    import mfc_inputs as mi
    import paper_1802_07525_gb300 as P
    assert P.lib().mfc_check_build() == 1
    kw = dict(tau=0.7, tau_c=0.9, u_in=0.03, c_in=0.8, k_sink=0.01)
    cases = [((37, 11), (2, 0), 0, 0), ((33, 20), (2, 1), 1, 0), ((16, 9), (1, 1), 2, 0),
             ((29, 13), (0, 0), 0, 9), ((41, 10), (2, 0), 1, 9), ((13, 11, 17), (0, 0, 2), 0, 0),
             ((9, 10, 12), (1, 1, 1), 1, 0), ((7, 6, 9), (1, 0, 2), 2, 0), ((300, 5), (2, 0), 0, 0)]
    for shape, bc, prec, aq in cases:
        N = int(np.prod(shape))
        g = P.Lattice(shape, bc=bc, precision=prec, ade_q=aq, **kw)
        g.set_geometry(_classes(shape, N))
        for block in (128, 256):
            g.set_launch(block=block, offsets32=1)
            g.step_coupled(9)
            g.set_launch(block=block, offsets32=0)
            g.step_coupled(4)
            g.step_flow(3)
            g.step_ade(3)
        g.solve_steady(mode=1, tol_flow=0.0, tol_ade=0.0, max_steps=40, check_every=10)
        g.solve_steady(mode=0, tol_flow=0.0, tol_ade=0.0, max_steps=20, check_every=10)
        f = g.read_populations(P.MFC_POP_FLOW)
        g.write_populations(P.MFC_POP_FLOW, f)
        g.read_fields()
        g.set_geometry(_classes(shape, N + 1), reset_fields=False)
        g.step_coupled(5)
        g.synchronize()
        assert g.check_canaries() == 0, shape
        g.close()
    # the agent model
    w = mi.anode_2d(64, 32, seed=3)
    g = P.Lattice(w.shape, tau=0.8, tau_c=0.7)
    g.set_geometry(np.where((w.cls & 3) == 3, 3, 0).astype(np.uint8))
    g.step_coupled(50)
    for cyc in range(3):
        g.agent_step(P.agent_params(seed=1, k_ata=50, growth=0.4, max_walk=200), cyc)
        g.step_coupled(20)
    g.synchronize()
    assert g.check_canaries() == 0
    g.close()
    # slabs exchanging halos
    import torch
    from paper_1802_07525_gb300 import slab as S
    for dim in (2, 3):
        shape = (40, 12) if dim == 2 else (10, 8, 24)
        fa = 0 if dim == 2 else 2
        slabs = []
        for r in range(2):
            s = list(shape)
            s[fa] //= 2
            gl = P.Lattice(tuple(s), bc=(2, 1) if dim == 2 else (1, 0, 2), cut=(r == 1, r == 0), **kw)
            gl.set_geometry(_classes(tuple(s), 7 + r))
            slabs.append(gl)
        loc = S.LocalSlabs(slabs)
        loc.step(10)
        loc.check(5)
        for gl in slabs:
            gl.synchronize()
            assert gl.check_canaries() == 0
            gl.close()
    # a batch of two instances
    b = P.Batch(check_every=10, block=64)
    t1 = b.submit((50, 20), _classes((50, 20), 1), tol_flow=0.0, tol_ade=0.0, max_steps=40, **kw)
    t2 = b.submit((10, 9, 14), _classes((10, 9, 14), 2), tol_flow=0.0, tol_ade=0.0, max_steps=40,
                  bc=(0, 0, 2), **kw)
    b.run()
    assert b.poll(t1)["steps_flow"] == 40 and b.poll(t2)["steps_flow"] == 40
    b.close()
    print("checked build: no offset out of range, guards intact")


def test_checked_build_finds_no_out_of_range_access():
    from paper_1802_07525_gb300 import build
    build.build(check_bounds=True)
    env = dict(os.environ, MFC_LIBRARY="check")
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no offset out of range" in r.stdout


if __name__ == "__main__":
    _exercise()
