"""The agent-based biofilm (Sec. 3.3) on the GPU against the oracle, bit for bit.

Each cycle the lattice advances its flow and transport, then one biofilm step runs on the GPU
and on the oracle, the oracle reading the GPU's own concentration field (so both take every
decision on the same values).  Attachment, the spreading walks and the class update are integer
decisions, and growth and the spreading split are FP64 without contraction on both sides, so the
biomass must agree exactly.
"""
import numpy as np
import pytest

import mfc_inputs as mi
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1802_07525_gb300 import build
    build.build()
    import paper_1802_07525_gb300 as P
    return P


def electrode_only(w):
    return np.where((w.cls & 3) == 3, 3, 0).astype(np.uint8)


@pytest.mark.parametrize("case", ["anode_96x48", "electrode_24x20x32"])
def test_agent_biofilm_bit_exact_over_three_cycles(P, case):
    if case == "anode_96x48":
        w = mi.anode_2d(96, 48, seed=5)
    else:
        w = mi.electrode_3d(24, 20, 32, seed=9)
    cls = electrode_only(w)
    kw = dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    g = P.Lattice(w.shape, **kw)
    g.set_geometry(cls)
    o = oracle.Oracle(w.shape, cls)
    bio_o = np.zeros(w.nodes)
    # Table 1's k_ata, C_0^bio, C_max^bio and fr_spr; growth 0.3 per cycle so that cells pass the
    # threshold in the first cycle and spreading (with walks) starts at once
    pg = P.agent_params(seed=17, growth=0.3, k_half=0.05, max_walk=500)
    po = oracle.agent_table1(seed=17, mu=0.3, K_s=0.05, max_walk=500)
    electrode = int(np.count_nonzero(cls == 3))
    attached = spread = 0
    for cyc in range(3):
        g.step_coupled(300)
        _, _, c, _ = g.read_fields()
        sg = g.agent_step(pg, cyc)
        so = o.agent_step(po, cyc, bio_o, conc=c)
        bio_g = g.read_biomass()
        assert np.array_equal(bio_g, bio_o), (cyc, int(np.count_nonzero(bio_g != bio_o)))
        for k in ("attached", "front", "spread", "walks_failed", "walk_steps", "biofilm_nodes"):
            assert sg[k] == so[k], (cyc, k, sg[k], so[k])
        assert sg["total_biomass"] == pytest.approx(so["total_biomass"], rel=1e-12)
        # the classes followed the biomass: biofilm is closed to the flow
        flow_open, ade_open = g.active_nodes()
        assert flow_open == w.nodes - electrode - so["biofilm_nodes"]
        assert ade_open == w.nodes - electrode
        attached += so["attached"]
        spread += so["spread"]
    # every part of the model ran: attachment (until the front was covered) and spreading
    assert attached > 0 and spread > 0
    g.close()


def test_agent_write_read_and_bad_parameters(P):
    w = mi.anode_2d(64, 32, seed=3)
    g = P.Lattice(w.shape, tau=0.8, tau_c=0.7)
    g.set_geometry(electrode_only(w))
    assert not g.read_biomass().any()
    v = np.linspace(0.0, 5.0, w.nodes)
    g.write_biomass(v)
    assert np.array_equal(g.read_biomass(), v)
    with pytest.raises(P.MfcError):
        g.write_biomass(-v - 1.0)
    for bad in (dict(k_half=0.0), dict(fr_spr=1.5), dict(max_walk=0), dict(growth=-1.0),
                dict(k_ata=-1)):
        with pytest.raises(P.MfcError):
            g.agent_step(P.agent_params(**bad), 0)
    g.close()
