"""FP64 CPU oracle for the coupled flow + advection-diffusion LBM (arXiv 1802.07525, Sec. 3.1).

TEST INFRASTRUCTURE ONLY.  The C source ``mfc_oracle.c`` is a plain restatement of the paper's
equations in double precision; this module compiles it with gcc (no FMA contraction) and wraps
it with ctypes.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
it.  It shares no code with the CUDA library and imports nothing from it.

Arrays follow the oracle's conventions: node index k = x + nx*(y + ny*z); populations SoA
``f[i, k]``; velocity ``u[a, k]``; node classes uint8 with bits 1 = flow-blocked,
2 = transport-blocked, 4 = consumption (sink).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mfc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

BC_WALL, BC_PERIODIC, BC_INOUT = 0, 1, 2
FLOW_SOLID, ADE_SOLID, SINK = 1, 2, 4
SEQUENTIAL, CONCURRENT = 0, 1


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 3), ("ade_q", ctypes.c_int), ("ade_outlet", ctypes.c_int),
        ("tau", ctypes.c_double), ("tau_c", ctypes.c_double), ("u_in", ctypes.c_double),
        ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double), ("c_in", ctypes.c_double),
        ("c_out", ctypes.c_double),
        ("k_sink", ctypes.c_double), ("u_scale", ctypes.c_double), ("k_half", ctypes.c_double),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("steps_flow", ctypes.c_long), ("steps_ade", ctypes.c_long),
        ("res_flow", ctypes.c_double), ("res_ade", ctypes.c_double),
        ("current", ctypes.c_double), ("mass", ctypes.c_double), ("substrate", ctypes.c_double),
        ("converged", ctypes.c_int), ("unstable", ctypes.c_int),
    ]


class Agent(ctypes.Structure):
    """Parameters of the agent-based biofilm of Sec. 3.3 (Table 1 gives k_ata, C_0^bio,
    C_max^bio and fr_spr)."""
    _fields_ = [("seed", ctypes.c_uint64), ("k_ata", ctypes.c_int), ("C0_bio", ctypes.c_double),
                ("Cmax_bio", ctypes.c_double), ("fr_spr", ctypes.c_double), ("mu", ctypes.c_double),
                ("K_s", ctypes.c_double), ("max_walk", ctypes.c_int)]


def agent_table1(**over) -> Agent:
    """Table 1's k_ata = 200, C_0^bio = 450, C_max^bio = 512.5, fr_spr = 0.4; mu = 0.1,
    K_s = 0.05 and max_walk = 1000 unless given."""
    a = Agent()
    vals = dict(seed=0, k_ata=200, C0_bio=450.0, Cmax_bio=512.5, fr_spr=0.4, mu=0.1, K_s=0.05,
                max_walk=1000)
    vals.update(over)
    for k, v in vals.items():
        setattr(a, k, v)
    return a


class Electro(ctypes.Structure):
    """Constants of the bio-electrochemical model (Sec. 3.2, Table 1), in the oracle's units."""
    _fields_ = [(n, ctypes.c_double) for n in
                ("M_total", "Y", "gamma", "m", "q_max", "K_Mox", "I_0", "E_0", "R_ext", "R_int",
                 "eps", "A_a", "T", "V_a", "dt")] + [("substeps", ctypes.c_int)]


def electro_table1(**over) -> Electro:
    """Table 1's values; eps, A_a and T (not in the paper) and the step as given in ``over``,
    defaulting to eps 0.01, A_a 0.048 x 0.065 m^2, T 298.15 K, V_a 17 x 60 x 65 mm, and one
    hour as 3600 steps of 1 s."""
    e = Electro()
    vals = dict(M_total=0.05, Y=0.5687, gamma=663400.0, m=2.0, q_max=8.48, K_Mox=0.02 * 0.05,
                I_0=0.001, E_0=0.7, R_ext=360.0, R_int=360.0, eps=0.01, A_a=0.048 * 0.065,
                T=298.15, V_a=17 * 60 * 65 * 1e-6, dt=1.0, substeps=3600)
    vals.update(over)
    for k, v in vals.items():
        setattr(e, k, v)
    return e


def electro_update(e: Electro, S: float, C_bio: float, M_ox: float) -> dict:
    """One call of the oracle's bio-electrochemical update (e.substeps steps of Eq. 15)."""
    out = np.zeros(8)
    lib().orc_electro_update(ctypes.byref(e), S, C_bio, M_ox, _d(out))
    return dict(zip(("m_ox", "m_red", "q_a", "n_conc", "n_act", "i_cell", "v_cell", "v_eq21"),
                    out.tolist()))


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, -ffp-contract=off)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def build_omp(force: bool = False):
    """Compile the timing-only OpenMP build ``oracle/_build/liboracle_omp.so`` (the same source
    and flags plus -fopenmp); returns its path, or None when the compiler has no OpenMP."""
    with _lock:
        if not force and os.path.exists(_LIB_OMP) and \
                os.path.getmtime(_LIB_OMP) >= os.path.getmtime(_SRC):
            return _LIB_OMP
        os.makedirs(os.path.dirname(_LIB_OMP), exist_ok=True)
        tmp = _LIB_OMP + f".{os.getpid()}.tmp"
        r = subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                            "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _LIB_OMP)
        return _LIB_OMP


def _declare(L):
    dp = ctypes.POINTER(ctypes.c_double)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    pp = ctypes.POINTER(Params)
    L.orc_flow_step.argtypes = [pp, u8p, dp, dp, dp, dp]
    L.orc_ade_step.argtypes = [pp, u8p, dp, dp, dp, dp]
    return L


def lib_omp():
    """The OpenMP timing build (None where it cannot be built).  Its steps give the same results
    as the plain build's; only the CPU-baseline timing uses it."""
    global _lib_omp
    if _lib_omp is None:
        path = build_omp()
        if path is None:
            return None
        _lib_omp = _declare(ctypes.CDLL(path))
    return _lib_omp


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        pp = ctypes.POINTER(Params)
        L.orc_flow_step.argtypes = [pp, u8p, dp, dp, dp, dp]
        L.orc_ade_step.argtypes = [pp, u8p, dp, dp, dp, dp]
        L.orc_sums.argtypes = [pp, u8p, dp, dp, dp, dp, dp, dp]
        L.orc_init_state.argtypes = [pp, u8p, dp, dp]
        L.orc_solve_steady.argtypes = [pp, u8p, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_long, ctypes.c_int,
                                       ctypes.POINTER(Result)]
        L.orc_solve_steady.restype = ctypes.c_int
        L.orc_flow_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_ade_equilibrium.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_velocity_set.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int), dp]
        L.orc_velocity_set.restype = ctypes.c_int
        L.orc_splitmix64.argtypes = [ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_biofilm_convert.argtypes = [pp, u8p, dp, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_double, ctypes.c_double, u8p]
        L.orc_biofilm_convert.restype = ctypes.c_long
        L.orc_agent_step.argtypes = [pp, u8p, dp, ctypes.POINTER(Agent), ctypes.c_uint64, dp, u8p,
                                     dp]
        L.orc_agent_size.restype = ctypes.c_int
        assert L.orc_agent_size() == ctypes.sizeof(Agent)
        L.orc_electro_update.argtypes = [ctypes.POINTER(Electro), ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, dp]
        L.orc_electro_size.restype = ctypes.c_int
        assert L.orc_electro_size() == ctypes.sizeof(Electro)
        L.orc_params_size.restype = ctypes.c_int
        L.orc_result_size.restype = ctypes.c_int
        assert L.orc_params_size() == ctypes.sizeof(Params)
        assert L.orc_result_size() == ctypes.sizeof(Result)
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def velocity_set(q: int):
    """(c[q,3], opp[q], w[q]) of the oracle's velocity set with q directions (5, 7, 9, 19)."""
    c = (ctypes.c_int * 57)()
    o = (ctypes.c_int * 19)()
    w = (ctypes.c_double * 19)()
    n = lib().orc_velocity_set(q, c, o, w)
    return (np.array(c[:3 * n]).reshape(n, 3), np.array(o[:n]), np.array(w[:n]))


def flow_equilibrium(dim: int, rho: float, u) -> np.ndarray:
    q = 9 if dim == 2 else 19
    uu = np.zeros(3)
    uu[:len(u)] = u
    out = np.zeros(q)
    lib().orc_flow_equilibrium(dim, rho, _d(uu), _d(out))
    return out


def ade_equilibrium(q: int, conc: float, u) -> np.ndarray:
    uu = np.zeros(3)
    uu[:len(u)] = u
    out = np.zeros(q)
    lib().orc_ade_equilibrium(q, conc, _d(uu), _d(out))
    return out


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


class Oracle:
    """A lattice held by the oracle: classes, flow state f, transport state g and fields."""

    def __init__(self, shape, cls=None, *, bc=None, ade_q=None,
                 ade_outlet=0, tau=0.8, tau_c=0.7, u_in=0.01, rho_in=1.0, rho_out=1.0, c_in=1.0, c_out=0.0,
                 k_sink=1e-3, u_scale=1.0, k_half=0.0, parallel=False):
        """parallel: step with the OpenMP timing build (CPU-baseline timing only)."""
        self._steps = lib_omp() if parallel else None
        if parallel and self._steps is None:
            raise RuntimeError("the OpenMP build of the oracle is not available")
        shape = tuple(int(s) for s in shape)
        self.dim = len(shape)
        nx, ny = shape[0], shape[1]
        nz = shape[2] if self.dim == 3 else 1
        self.shape = shape
        self.N = nx * ny * nz
        self.qf = 9 if self.dim == 2 else 19
        self.qa = ade_q or (5 if self.dim == 2 else 7)
        p = Params()
        p.dim, p.nx, p.ny, p.nz = self.dim, nx, ny, nz
        if bc is None:  # channel: inlet/outlet along the flow axis, walls across it
            bc = (BC_INOUT, BC_WALL) if self.dim == 2 else (BC_WALL, BC_WALL, BC_INOUT)
        bcs = list(bc) + [BC_WALL] * (3 - len(bc))
        if self.dim == 2:
            bcs[2] = BC_PERIODIC
        for a in range(3):
            p.bc[a] = bcs[a]
        p.ade_q, p.ade_outlet = self.qa, ade_outlet
        p.tau, p.tau_c, p.u_in, p.rho_in, p.rho_out = tau, tau_c, u_in, rho_in, rho_out
        p.c_in, p.c_out, p.k_sink, p.u_scale, p.k_half = c_in, c_out, k_sink, u_scale, k_half
        self.p = p
        if cls is None:
            cls = np.zeros(self.N, np.uint8)
        self.cls = np.ascontiguousarray(np.asarray(cls, np.uint8).reshape(-1))
        assert self.cls.size == self.N
        self.f = np.zeros((self.qf, self.N))
        self.g = np.zeros((self.qa, self.N))
        self.rho = np.zeros(self.N)
        self.u = np.zeros((self.dim, self.N))
        self.conc = np.zeros(self.N)
        lib().orc_init_state(ctypes.byref(p), _u8(self.cls), _d(self.f), _d(self.g))
        self._f2 = np.zeros_like(self.f)
        self._g2 = np.zeros_like(self.g)

    def step_flow(self, n: int = 1):
        L = self._steps or lib()
        for _ in range(n):
            L.orc_flow_step(ctypes.byref(self.p), _u8(self.cls), _d(self.f), _d(self._f2),
                            _d(self.rho), _d(self.u))
            self.f, self._f2 = self._f2, self.f

    def step_ade(self, n: int = 1, u=None):
        """Transport steps with the velocity ``u`` (default: the stored flow velocity)."""
        L = self._steps or lib()
        uu = self.u if u is None else np.ascontiguousarray(np.asarray(u, float).reshape(self.dim, self.N))
        for _ in range(n):
            L.orc_ade_step(ctypes.byref(self.p), _u8(self.cls), _d(self.g), _d(self._g2), _d(uu),
                           _d(self.conc))
            self.g, self._g2 = self._g2, self.g

    def step_coupled(self, n: int = 1):
        for _ in range(n):
            self.step_flow(1)
            self.step_ade(1)

    def sums(self, u_prev=None, c_prev=None):
        out = np.zeros(9)
        up = self.u if u_prev is None else np.ascontiguousarray(u_prev)
        cp = self.conc if c_prev is None else np.ascontiguousarray(c_prev)
        lib().orc_sums(ctypes.byref(self.p), _u8(self.cls), _d(self.rho), _d(self.u), _d(up),
                       _d(self.conc), _d(cp), _d(out))
        return out

    def solve_steady(self, mode=SEQUENTIAL, tol_flow=1e-8, tol_ade=1e-8, max_steps=10000,
                     check_every=1) -> Result:
        r = Result()
        lib().orc_solve_steady(ctypes.byref(self.p), _u8(self.cls), _d(self.f), _d(self.g),
                               _d(self.rho), _d(self.u), _d(self.conc), mode, tol_flow, tol_ade,
                               max_steps, check_every, ctypes.byref(r))
        return r

    def agent_step(self, agent: Agent, cycle: int, bio, conc=None):
        """One agent-based biofilm step (attachment, growth, spreading) on the biomass array
        ``bio`` (N doubles, updated in place); the classes become the new ones.  ``conc``
        defaults to the oracle's own concentration field.  Returns the statistics."""
        c = self.conc if conc is None else np.ascontiguousarray(np.asarray(conc, float).reshape(-1))
        assert bio.dtype == np.float64 and bio.flags.c_contiguous and bio.size == self.N
        out = np.zeros_like(self.cls)
        st = np.zeros(7)
        lib().orc_agent_step(ctypes.byref(self.p), _u8(self.cls), _d(c), ctypes.byref(agent), cycle,
                             _d(bio), _u8(out), _d(st))
        self.cls = out
        return dict(zip(("attached", "front", "spread", "walks_failed", "walk_steps",
                         "biofilm_nodes", "total_biomass"), st.tolist()))

    def biofilm_convert(self, seed: int, cycle: int, prob: float = 0.05, c_thresh: float = 0.5,
                        conc=None):
        """Apply the biofilm growth rule; ``conc`` defaults to the oracle's own field."""
        c = self.conc if conc is None else np.ascontiguousarray(np.asarray(conc, float).reshape(-1))
        out = np.zeros_like(self.cls)
        n = lib().orc_biofilm_convert(ctypes.byref(self.p), _u8(self.cls), _d(c), seed, cycle,
                                      prob, c_thresh, _u8(out))
        return out, int(n)
