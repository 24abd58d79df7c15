"""The bio-electrochemical model of the anode (Sec. 3.2, Eqs. 14-21), lumped over the anode.

Oracle pins (against closed forms, limits and the paper's reported output), then the library's
host entry point mfc_electro_update against the oracle through the C ABI (no GPU needed).
The oracle finds the implicit current of Eq. 20 by bisection; the library uses its closed form.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F = 96485.33212
R = 8.314462618


def run(S=0.8, C_bio=450.0, M_ox=0.02, **over):
    over.setdefault("dt", 0.0)
    over.setdefault("substeps", 1)
    return oracle.electro_update(oracle.electro_table1(**over), S, C_bio, M_ox)


def test_without_losses_the_current_is_ohms_law():
    """M_ox = 0 leaves no concentration overpotential (M_red = M_total) and no activation
    overpotential (Eq. 19 carries M_ox); with eps = 0, Eq. 20 is I = E_0 / (R_int + R_ext)."""
    r = run(M_ox=0.0, eps=0.0)
    assert r["n_conc"] == 0.0 and r["n_act"] == 0.0
    assert r["i_cell"] == pytest.approx(0.7 / 720.0, rel=1e-15)
    assert r["v_cell"] == pytest.approx(0.35, rel=1e-15)  # equal resistances: half of E_0


@pytest.mark.parametrize("M_ox", [0.001, 0.02, 0.045])
def test_kirchhoff_eq17_holds_when_eps_is_zero(M_ox):
    """Eq. 17 (Kirchhoff's voltage law) and Eq. 20 coincide when eps = 0: the current the
    oracle finds from Eq. 20 satisfies I R_ext = E_0 - I R_int - n_conc - n_act."""
    r = run(M_ox=M_ox, eps=0.0)
    lhs = r["i_cell"] * 360.0
    rhs = 0.7 - r["i_cell"] * 360.0 - r["n_conc"] - r["n_act"]
    assert lhs == pytest.approx(rhs, rel=1e-13)
    assert r["i_cell"] > 0.0


def test_nernst_concentration_overpotential():
    """Eq. 18 at M_red = M_total / e is R T / F (25.69 mV at 298.15 K), and 0 at M_ox = 0."""
    r = run(M_ox=0.05 * (1.0 - 1.0 / math.e))
    assert r["n_conc"] == pytest.approx(R * 298.15 / F, rel=1e-12)
    assert r["n_conc"] == pytest.approx(0.0256926, rel=1e-5)


def test_activation_overpotential_scaling():
    """Eq. 19: n_act / I is proportional to M_ox / M_red, to T and to 1 / (A_a I_0 m)."""
    a = run(M_ox=0.01)
    b = run(M_ox=0.03)
    ra, rb = a["n_act"] / a["i_cell"], b["n_act"] / b["i_cell"]
    assert ra / rb == pytest.approx((0.01 / 0.04) / (0.03 / 0.02), rel=1e-12)
    c = run(M_ox=0.01, A_a=2 * 0.048 * 0.065)
    assert (c["n_act"] / c["i_cell"]) / ra == pytest.approx(0.5, rel=1e-12)
    d = run(M_ox=0.01, m=4.0, T=2 * 298.15)
    assert (d["n_act"] / d["i_cell"]) / ra == pytest.approx(1.0, rel=1e-12)


def test_open_circuit_limit():
    """R_ext -> infinity: no current flows, and the voltage across the load tends to the
    open-circuit voltage less the concentration overpotential, scaled by M_red/(eps + M_red)."""
    r = run(M_ox=0.02, R_ext=1e13)
    s = 0.03 / (0.01 + 0.03)
    assert abs(r["i_cell"]) < 1e-12
    assert r["v_cell"] == pytest.approx((0.7 - r["n_conc"]) * s, rel=1e-9)


def test_double_monod_consumption():
    """Eq. 16: half the maximum rate at M_ox = K_Mox with saturated substrate; the two Monod
    factors multiply."""
    r = run(S=1.0, M_ox=0.02 * 0.05)
    assert r["q_a"] == pytest.approx(8.48 / 2, rel=1e-15)
    r = run(S=0.5, M_ox=0.02 * 0.05)
    assert r["q_a"] == pytest.approx(8.48 / 4, rel=1e-15)
    assert run(S=0.0)["q_a"] == 0.0


def test_mediator_step_conservation_and_fixed_point():
    """Eq. 14: M_ox + M_red = M_total after every call.  Eq. 15 as one explicit step of dt:
    the change of M_ox is dt (-Y q_a / 86400 + gamma I / (m F V_a C_bio)).  Iterated, the
    balance settles where the mediator reduced by consumption equals the mediator oxidised by
    the current."""
    V_a = 17 * 60 * 65 * 1e-6
    r0 = run(M_ox=0.02)
    r1 = run(M_ox=0.02, dt=1.0)
    expect = 0.02 + 1.0 * (-0.5687 * r0["q_a"] / 86400 + 663400 * r0["i_cell"] / (2 * F) / (V_a * 450.0))
    assert r1["m_ox"] == pytest.approx(expect, rel=1e-14)
    assert r1["m_ox"] + r1["m_red"] == pytest.approx(0.05, rel=1e-15)
    r = run(M_ox=0.02, dt=1.0, substeps=20000)
    assert r["m_ox"] + r["m_red"] == pytest.approx(0.05, rel=1e-15)
    consumed = 0.5687 * r["q_a"] / 86400
    oxidised = 663400 * r["i_cell"] / (2 * F) / (V_a * 450.0)
    assert consumed == pytest.approx(oxidised, rel=1e-9)


def test_reported_voltage_is_current_times_external_resistance():
    """Sec. 4 reports about 330 mV at 0.91 mA with R_ext = R_int = 360 ohm: that is the
    voltage across the load, I R_ext = 327.6 mV, not Eq. 21 as printed, I (R_int + R_ext)
    = 655 mV.  The oracle returns the former as the cell voltage and the latter beside it."""
    with open(os.path.join(GOLDEN, "sec4_cell_output.json")) as fh:
        g = json.load(fh)
    assert g["current_A"] * g["R_ext_ohm"] == pytest.approx(g["voltage_V"], rel=0.01)
    assert abs(g["current_A"] * (g["R_ext_ohm"] + g["R_int_ohm"]) - g["voltage_V"]) > 0.3
    r = run(M_ox=0.01)
    assert r["v_cell"] == pytest.approx(r["i_cell"] * g["R_ext_ohm"], rel=1e-15)
    assert r["v_eq21"] == pytest.approx(r["i_cell"] * (g["R_ext_ohm"] + g["R_int_ohm"]), rel=1e-15)


# ------------------------------------------------------------------------------------------
# The library's entry point against the oracle (host call through the C ABI; no GPU)
# ------------------------------------------------------------------------------------------

KEYS = ("m_ox", "m_red", "q_a", "n_conc", "n_act", "i_cell", "v_cell", "v_eq21")
LIB_OF = {"M_total": "m_total", "Y": "mediator_yield", "gamma": "gamma", "m": "m_electrons",
          "q_max": "q_max", "K_Mox": "k_mox", "I_0": "i0", "E_0": "e0", "R_ext": "r_ext",
          "R_int": "r_int", "eps": "epsilon", "A_a": "area", "T": "temperature", "V_a": "volume",
          "dt": "dt", "substeps": "substeps"}


@pytest.fixture(scope="module")
def P():
    from paper_1802_07525_gb300 import build
    build.build()
    import paper_1802_07525_gb300 as P
    return P


def test_library_defaults_are_table1(P):
    p = P.electro_params()
    e = oracle.electro_table1()
    for ok, lk in LIB_OF.items():
        assert getattr(p, lk) == pytest.approx(getattr(e, ok), rel=1e-15), lk


@pytest.mark.parametrize("seed", range(6))
def test_library_matches_oracle(P, seed):
    """Random constants and states: one step and one hour of 1-s steps agree with the oracle
    (closed form against bisection) to 1e-12, and 1e-9 after 3600 steps."""
    rng = np.random.default_rng(seed)
    over = dict(eps=10 ** rng.uniform(-4, -1), A_a=10 ** rng.uniform(-3, -1),
                T=rng.uniform(280, 320), R_ext=rng.uniform(10, 2000), R_int=rng.uniform(10, 500),
                E_0=rng.uniform(0.3, 0.9), q_max=rng.uniform(1, 20))
    S, C_bio, M_ox = rng.uniform(0, 1), rng.uniform(100, 2000), rng.uniform(0, 0.049)
    for dt, n, tol in ((0.0, 1, 1e-12), (1.0, 1, 1e-12), (1.0, 3600, 1e-9)):
        over.update(dt=dt, substeps=n)
        ro = oracle.electro_update(oracle.electro_table1(**over), S, C_bio, M_ox)
        p = P.electro_params(**{LIB_OF[k]: v for k, v in over.items()})
        rl = P.electro_update(p, S, C_bio, M_ox)
        for k in KEYS:
            assert rl[k] == pytest.approx(ro[k], rel=tol, abs=1e-18), (k, dt, n)


def test_library_rejects_bad_arguments(P):
    p = P.electro_params()
    for args in ((1.5, 450.0, 0.01), (0.5, 0.0, 0.01), (0.5, 450.0, 0.05), (0.5, 450.0, -1e-3)):
        with pytest.raises(P.MfcError):
            P.electro_update(p, *args)
    bad = P.electro_params(substeps=0)
    with pytest.raises(P.MfcError):
        P.electro_update(bad, 0.5, 450.0, 0.01)
