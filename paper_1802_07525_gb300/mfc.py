"""Thin ctypes binding of the C ABI in ``include/mfc.h`` (argument marshalling only).

Every computation runs in the sm_103a library ``_lib/libmfc.so``; this module only converts
NumPy arrays and Python numbers into the C structures and pointers the library takes.  There
is no CPU fallback: if the library is missing, :func:`lib` raises.

The raw entry points are available under their C names (``mfc_create_lattice``,
``mfc_set_geometry``, ``mfc_step_flow``, ``mfc_step_ade``, ``mfc_step_coupled``,
``mfc_solve_steady``, ``mfc_read_fields``, ...); :class:`Lattice` wraps them for NumPy users.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MFC_LIBRARY=check selects the checking build (element offsets and guard regions checked)
LIB_PATH = os.path.join(_HERE, "_lib", "libmfc_check.so" if os.environ.get("MFC_LIBRARY") == "check"
                        else "libmfc.so")

MFC_OK, MFC_ERR_ARG, MFC_ERR_OOM, MFC_ERR_OOM_BUDGET, MFC_ERR_CUDA = 0, 1, 2, 3, 4
MFC_NOT_CONVERGED, MFC_ERR_NONFINITE, MFC_ERR_TIMEOUT, MFC_ERR_STATE, MFC_PENDING = 5, 6, 7, 8, 9
MFC_ERR_UNSTABLE = 10
MFC_BC_WALL, MFC_BC_PERIODIC, MFC_BC_INOUT = 0, 1, 2
MFC_FP32, MFC_FP16_DEV, MFC_FP64 = 0, 1, 2
MFC_SEQUENTIAL, MFC_CONCURRENT = 0, 1
MFC_OUTLET_ZERO_GRADIENT, MFC_OUTLET_DIRICHLET = 0, 1
MFC_POP_FLOW, MFC_POP_ADE, MFC_FIELD_VELOCITY = 0, 1, 2


class LatticeDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("bc", ctypes.c_int * 3), ("precision", ctypes.c_int),
                ("ade_q", ctypes.c_int), ("cut", ctypes.c_int * 2), ("stream", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("tau_c", ctypes.c_double), ("u_in", ctypes.c_double),
                ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double),
                ("c_in", ctypes.c_double), ("c_out", ctypes.c_double),
                ("k_sink", ctypes.c_double), ("u_scale", ctypes.c_double),
                ("ade_outlet", ctypes.c_int), ("k_half", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol_flow", ctypes.c_double), ("tol_ade", ctypes.c_double),
                ("max_steps", ctypes.c_long), ("check_every", ctypes.c_int),
                ("mode", ctypes.c_int), ("timeout_s", ctypes.c_double)]


class SolveResult(ctypes.Structure):
    _fields_ = [("steps_flow", ctypes.c_long), ("steps_ade", ctypes.c_long),
                ("res_flow", ctypes.c_double), ("res_ade", ctypes.c_double),
                ("current", ctypes.c_double), ("mass", ctypes.c_double),
                ("substrate", ctypes.c_double), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Launch(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("offsets32", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("precision", ctypes.c_int),
                ("check_every", ctypes.c_int), ("block", ctypes.c_int),
                ("max_instances", ctypes.c_int), ("stream", ctypes.c_void_p)]


class BatchResult(ctypes.Structure):
    _fields_ = [("result", SolveResult), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class BatchStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("running", ctypes.c_longlong), ("queued", ctypes.c_longlong),
                ("blocks", ctypes.c_longlong), ("instance_steps", ctypes.c_longlong),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("check_every", ctypes.c_int),
                ("block", ctypes.c_int), ("grid", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AgentParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("k_ata", ctypes.c_int), ("c0_bio", ctypes.c_double),
                ("c_max_bio", ctypes.c_double), ("fr_spr", ctypes.c_double),
                ("growth", ctypes.c_double), ("k_half", ctypes.c_double), ("max_walk", ctypes.c_int)]


class AgentStats(ctypes.Structure):
    _fields_ = [("attached", ctypes.c_longlong), ("front", ctypes.c_longlong),
                ("spread", ctypes.c_longlong), ("walks_failed", ctypes.c_longlong),
                ("walk_steps", ctypes.c_longlong), ("biofilm_nodes", ctypes.c_longlong),
                ("total_biomass", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def agent_params(seed=0, k_ata=200, c0_bio=450.0, c_max_bio=512.5, fr_spr=0.4, growth=0.1,
                 k_half=0.05, max_walk=1000) -> AgentParams:
    """Agent-model parameters; the defaults are Table 1's k_ata, C_0^bio, C_max^bio and fr_spr,
    with a growth of 0.1 per call and K_s = 0.05 (the paper's 20 mg/L against 410 mg/L)."""
    return AgentParams(seed, k_ata, c0_bio, c_max_bio, fr_spr, growth, k_half, max_walk)


class ElectroParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("m_total", "mediator_yield", "gamma", "m_electrons", "q_max", "k_mox", "i0", "e0", "r_ext",
                 "r_int", "epsilon", "area", "temperature", "volume", "dt")] + \
               [("substeps", ctypes.c_int)]


class ElectroResult(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("m_ox", "m_red", "q_a", "n_conc", "n_act", "i_cell", "v_cell", "v_eq21")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MfcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)} ({status}): {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "mfc_create_lattice": (ctypes.c_int, [ctypes.POINTER(LatticeDesc), ctypes.POINTER(Params),
                                          ctypes.POINTER(_vp)]),
    "mfc_destroy_lattice": (ctypes.c_int, [_vp]),
    "mfc_set_params": (ctypes.c_int, [_vp, ctypes.POINTER(Params)]),
    "mfc_set_geometry": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int]),
    "mfc_step_flow": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mfc_step_ade": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mfc_step_coupled": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mfc_step_coupled_plain": (ctypes.c_int, [_vp, ctypes.c_int]),
    "mfc_solve_steady": (ctypes.c_int, [_vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveResult)]),
    "mfc_biofilm_grow": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_long)]),
    "mfc_read_fields": (ctypes.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "mfc_read_populations": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    "mfc_write_populations": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    "mfc_synchronize": (ctypes.c_int, [_vp]),
    "mfc_set_launch": (ctypes.c_int, [_vp, ctypes.POINTER(Launch)]),
    "mfc_get_launch": (ctypes.c_int, [_vp, ctypes.POINTER(Launch)]),
    "mfc_check_build": (ctypes.c_int, []),
    "mfc_check_canaries": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "mfc_field_sums_noalloc": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_int, _vp, _vp, _vp, _vp,
                                              _vp, _vp, ctypes.c_double, _vp, _vp]),
    "mfc_agent_step": (ctypes.c_int, [_vp, ctypes.POINTER(AgentParams), ctypes.c_uint64,
                                      ctypes.POINTER(AgentStats)]),
    "mfc_read_biomass": (ctypes.c_int, [_vp, _dp]),
    "mfc_write_biomass": (ctypes.c_int, [_vp, _dp]),
    "mfc_halo_bytes": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "mfc_halo_pack": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "mfc_halo_unpack": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "mfc_set_halo_classes": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8)]),
    "mfc_step_check_sums": (ctypes.c_int, [_vp, ctypes.c_int, _dp]),
    "mfc_electro_default_params": (ctypes.c_int, [ctypes.POINTER(ElectroParams)]),
    "mfc_electro_update": (ctypes.c_int, [ctypes.POINTER(ElectroParams), ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(ElectroResult)]),
    "mfc_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchOpts), ctypes.POINTER(_vp)]),
    "mfc_batch_destroy": (ctypes.c_int, [_vp]),
    "mfc_batch_submit": (ctypes.c_int, [_vp, ctypes.POINTER(LatticeDesc), ctypes.POINTER(Params),
                                        ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(SolveOpts),
                                        _dp, _dp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "mfc_batch_poll": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.POINTER(BatchResult)]),
    "mfc_batch_wait": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_double,
                                      ctypes.POINTER(BatchResult)]),
    "mfc_batch_run": (ctypes.c_int, [_vp]),
    "mfc_batch_start": (ctypes.c_int, [_vp]),
    "mfc_batch_stop": (ctypes.c_int, [_vp]),
    "mfc_batch_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(BatchStats)]),
    "mfc_batch_last_error": (ctypes.c_char_p, [_vp]),
    "mfc_clock": (ctypes.c_double, []),
    "mfc_active_nodes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_long),
                                        ctypes.POINTER(ctypes.c_long)]),
    "mfc_device_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "mfc_lattice_bytes": (ctypes.c_size_t, [ctypes.POINTER(LatticeDesc)]),
    "mfc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mfc_last_error": (ctypes.c_char_p, [_vp]),
    "mfc_version": (ctypes.c_char_p, []),
}
EXPORTED = tuple(_SIGS)


def lib():
    """Load libmfc.so (built by ``paper_1802_07525_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(
                        f"CUDA library not built: {LIB_PATH} is missing; run "
                        "`python -m paper_1802_07525_gb300.build` (needs nvcc)")
                L = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in _SIGS.items():
                    fn = getattr(L, name)
                    fn.restype = res
                    fn.argtypes = args
                _lib = L
    return _lib


def __getattr__(name):
    if name in _SIGS:
        return getattr(lib(), name)
    raise AttributeError(name)


def status_string(s: int) -> str:
    return lib().mfc_status_string(s).decode()


def _ptr(a, ct=ctypes.c_double):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def make_params(tau=0.8, tau_c=0.7, u_in=0.01, rho_in=1.0, rho_out=1.0, c_in=1.0, c_out=0.0,
                k_sink=1e-3, u_scale=1.0, ade_outlet=MFC_OUTLET_ZERO_GRADIENT, k_half=0.0) -> Params:
    return Params(tau, tau_c, u_in, rho_in, rho_out, c_in, c_out, k_sink, u_scale, ade_outlet, k_half)


def make_desc(shape, bc=None, precision=MFC_FP32, stream=None, ade_q=0, cut=(0, 0)) -> LatticeDesc:
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    if bc is None:
        bc = (MFC_BC_INOUT, MFC_BC_WALL) if dim == 2 else (MFC_BC_WALL, MFC_BC_WALL, MFC_BC_INOUT)
    bcs = list(bc) + [MFC_BC_PERIODIC] * (3 - len(bc))
    d = LatticeDesc()
    d.dim = dim
    d.nx, d.ny = shape[0], shape[1]
    d.nz = shape[2] if dim == 3 else 1
    for a in range(3):
        d.bc[a] = bcs[a]
    d.precision = precision
    d.ade_q = ade_q
    d.cut[0], d.cut[1] = int(cut[0]), int(cut[1])
    d.stream = stream
    return d


def lattice_bytes(shape, bc=None, precision=MFC_FP32, ade_q=0) -> int:
    return int(lib().mfc_lattice_bytes(ctypes.byref(make_desc(shape, bc, precision, None, ade_q))))


class Lattice:
    """One lattice resident on the current CUDA device (see ``include/mfc.h``)."""

    def __init__(self, shape, *, bc=None, precision=MFC_FP32, stream=None, ade_q=0, cut=(0, 0),
                 **params):
        """ade_q: 0 for the default transport set (D2Q5 / D3Q7), 9 for D2Q9 with the equilibrium
        of Eq. 5 (2-D).  cut: the low / high faces of the flow axis that are cuts to neighbouring
        slabs."""
        self.shape = tuple(int(s) for s in shape)
        self.dim = len(self.shape)
        self.N = int(np.prod(self.shape))
        self.qf = 9 if self.dim == 2 else 19
        self.qa = (9 if ade_q == 9 else 5) if self.dim == 2 else 7
        self._L = lib()
        self.desc = make_desc(self.shape, bc, precision, stream, ade_q, cut)
        self.params = make_params(**params)
        h = ctypes.c_void_p()
        st = self._L.mfc_create_lattice(ctypes.byref(self.desc), ctypes.byref(self.params),
                                        ctypes.byref(h))
        if st != MFC_OK:
            raise MfcError(st, self._L.mfc_last_error(None).decode())
        self.handle = h

    def _check(self, st, ok=(MFC_OK,)):
        if st not in ok:
            raise MfcError(st, self._L.mfc_last_error(self.handle).decode())
        return st

    def close(self):
        if getattr(self, "handle", None):
            self._L.mfc_destroy_lattice(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, **params):
        self.params = make_params(**params)
        self._check(self._L.mfc_set_params(self.handle, ctypes.byref(self.params)))

    def set_geometry(self, node_class, reset_fields=True):
        c = np.ascontiguousarray(np.asarray(node_class, dtype=np.uint8).reshape(-1))
        if c.size != self.N:
            raise ValueError(f"node_class has {c.size} entries, lattice has {self.N}")
        self._check(self._L.mfc_set_geometry(self.handle, _ptr(c, ctypes.c_uint8),
                                             int(bool(reset_fields))))

    def step_flow(self, n=1):
        self._check(self._L.mfc_step_flow(self.handle, int(n)))

    def step_ade(self, n=1):
        self._check(self._L.mfc_step_ade(self.handle, int(n)))

    def step_coupled_plain(self, n=1):
        """Fused steps that leave the stored fields as they are (see mfc_step_coupled_plain)."""
        self._check(self._L.mfc_step_coupled_plain(self.handle, n))

    def step_coupled(self, n=1):
        self._check(self._L.mfc_step_coupled(self.handle, int(n)))

    def solve_steady(self, mode=MFC_SEQUENTIAL, tol_flow=1e-8, tol_ade=1e-8, max_steps=10000,
                     check_every=100, timeout_s=0.0) -> SolveResult:
        o = SolveOpts(tol_flow, tol_ade, int(max_steps), int(check_every), mode, timeout_s)
        r = SolveResult()
        # the result is filled for these outcomes; its status field says which one it was
        self._check(self._L.mfc_solve_steady(self.handle, ctypes.byref(o), ctypes.byref(r)),
                    ok=(MFC_OK, MFC_NOT_CONVERGED, MFC_ERR_TIMEOUT, MFC_ERR_NONFINITE,
                        MFC_ERR_UNSTABLE))
        return r

    def biofilm_grow(self, seed, cycle, prob=0.05, c_thresh=0.5) -> int:
        n = ctypes.c_long(0)
        self._check(self._L.mfc_biofilm_grow(self.handle, seed, cycle, prob, c_thresh,
                                             ctypes.byref(n)))
        return int(n.value)

    # ---- slab decomposition ----------------------------------------------------------------

    def halo_bytes(self, side: int) -> int:
        n = ctypes.c_size_t()
        self._check(self._L.mfc_halo_bytes(self.handle, side, ctypes.byref(n)))
        return int(n.value)

    def halo_pack(self, side: int, dev_ptr: int):
        """Queue the populations leaving through face `side` into device memory at dev_ptr."""
        self._check(self._L.mfc_halo_pack(self.handle, side, ctypes.c_void_p(dev_ptr)))

    def halo_unpack(self, side: int, dev_ptr: int):
        """Queue a neighbour's packed populations into the ghost layer beyond face `side`."""
        self._check(self._L.mfc_halo_unpack(self.handle, side, ctypes.c_void_p(dev_ptr)))

    def set_halo_classes(self, side: int, plane):
        p = np.ascontiguousarray(np.asarray(plane, np.uint8).reshape(-1))
        self._check(self._L.mfc_set_halo_classes(self.handle, side, _ptr(p, ctypes.c_uint8)))

    def step_check_sums(self, nsteps: int = 1) -> np.ndarray:
        """nsteps fused steps, the last a check step; its nine FP64 sums over this lattice."""
        s = np.zeros(9)
        self._check(self._L.mfc_step_check_sums(self.handle, nsteps, _ptr(s)))
        return s

    def agent_step(self, params: AgentParams, cycle: int) -> dict:
        """One agent-based biofilm step (attachment, growth, spreading, class update)."""
        s = AgentStats()
        self._check(lib().mfc_agent_step(self.handle, ctypes.byref(params), cycle, ctypes.byref(s)))
        return s.as_dict()

    def read_biomass(self) -> np.ndarray:
        out = np.empty(self.N, np.float64)
        self._check(lib().mfc_read_biomass(self.handle, _ptr(out)))
        return out

    def write_biomass(self, values):
        v = np.ascontiguousarray(np.asarray(values, np.float64).reshape(-1))
        assert v.size == self.N
        self._check(lib().mfc_write_biomass(self.handle, _ptr(v)))

    def read_fields(self):
        rho = np.empty(self.N)
        u = np.empty((self.dim, self.N))
        c = np.empty(self.N)
        cur = np.zeros(1)
        self._check(self._L.mfc_read_fields(self.handle, _ptr(rho), _ptr(u), _ptr(c), _ptr(cur)))
        return rho, u, c, float(cur[0])

    def read_populations(self, which=MFC_POP_FLOW):
        q = {MFC_POP_FLOW: self.qf, MFC_POP_ADE: self.qa, MFC_FIELD_VELOCITY: self.dim}[which]
        out = np.empty((q, self.N))
        self._check(self._L.mfc_read_populations(self.handle, which, _ptr(out)))
        return out

    def write_populations(self, which, values):
        q = {MFC_POP_FLOW: self.qf, MFC_POP_ADE: self.qa, MFC_FIELD_VELOCITY: self.dim}[which]
        v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(q, self.N))
        self._check(self._L.mfc_write_populations(self.handle, which, _ptr(v)))

    def set_launch(self, block=128, offsets32=1):
        v = Launch(int(block), int(offsets32))
        self._check(self._L.mfc_set_launch(self.handle, ctypes.byref(v)))

    def get_launch(self) -> dict:
        v = Launch()
        self._check(self._L.mfc_get_launch(self.handle, ctypes.byref(v)))
        return v.as_dict()

    def check_canaries(self) -> int:
        """Guard bytes found changed (checking builds; 0 in other builds)."""
        n = ctypes.c_longlong()
        self._check(self._L.mfc_check_canaries(self.handle, ctypes.byref(n)))
        return int(n.value)

    def synchronize(self):
        self._check(self._L.mfc_synchronize(self.handle))

    def active_nodes(self):
        a, b = ctypes.c_long(), ctypes.c_long()
        self._check(self._L.mfc_active_nodes(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def device_bytes(self):
        b = ctypes.c_size_t()
        self._check(self._L.mfc_device_bytes(self.handle, ctypes.byref(b)))
        return int(b.value)


class Batch:
    """Many steady solves sharing the GPU with continuous batching (``mfc_batch_*``).

    ``submit`` queues a solve and returns a ticket; the engine runs on the caller's thread
    (``run``) or on a library thread (``start`` / ``stop``).  ``poll`` and ``wait`` return
    ``None`` while the request is pending, else a dict with the solve result, the time stamps
    (``mfc_clock`` seconds) and, when asked for, the fields ``rho``, ``u``, ``c``."""

    def __init__(self, *, budget_bytes=0, precision=MFC_FP32, check_every=0, block=0,
                 max_instances=0, stream=None):
        self._L = lib()
        o = BatchOpts(int(budget_bytes), precision, int(check_every), int(block),
                      int(max_instances), stream)
        h = ctypes.c_void_p()
        st = self._L.mfc_batch_create(ctypes.byref(o), ctypes.byref(h))
        if st != MFC_OK:
            raise MfcError(st, "mfc_batch_create")
        self.handle = h
        self.precision = precision
        self._pending = {}  # ticket -> (shape, host buffers kept alive until the solve ends)

    def submit(self, shape, node_class, *, bc=None, tol_flow=1e-7, tol_ade=1e-7,
               max_steps=100000, timeout_s=0.0, fields=True, **params) -> int:
        shape = tuple(int(v) for v in shape)
        n = int(np.prod(shape))
        dim = len(shape)
        cls = np.ascontiguousarray(np.asarray(node_class, dtype=np.uint8).reshape(-1))
        if cls.size != n:
            raise ValueError("node_class must hold one class per node")
        bufs = (np.empty(n), np.empty((dim, n)), np.empty(n)) if fields else (None, None, None)
        desc = make_desc(shape, bc, self.precision)
        prm = make_params(**params)
        opts = SolveOpts(tol_flow, tol_ade, int(max_steps), 0, MFC_CONCURRENT, timeout_s)
        t = ctypes.c_longlong(0)
        st = self._L.mfc_batch_submit(self.handle, ctypes.byref(desc), ctypes.byref(prm),
                                      _ptr(cls, ctypes.c_uint8), ctypes.byref(opts),
                                      _ptr(bufs[0]), _ptr(bufs[1]), _ptr(bufs[2]), ctypes.byref(t))
        if st != MFC_OK:
            raise MfcError(st, "mfc_batch_submit")
        self._pending[t.value] = (shape, bufs)
        return t.value

    def _result(self, ticket, st, r):
        if st == MFC_PENDING:
            return None
        if st == MFC_ERR_ARG and ticket not in self._pending:
            raise MfcError(st, f"unknown ticket {ticket}")
        _, bufs = self._pending.pop(ticket)
        out = r.result.as_dict()
        out.update(t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done, ticket=ticket)
        if bufs[0] is not None and st not in (MFC_ERR_CUDA,):
            out.update(rho=bufs[0], u=bufs[1], c=bufs[2])
        return out

    def poll(self, ticket):
        r = BatchResult()
        st = self._L.mfc_batch_poll(self.handle, ticket, ctypes.byref(r))
        return self._result(ticket, st, r)

    def wait(self, ticket, timeout_s=-1.0):
        r = BatchResult()
        st = self._L.mfc_batch_wait(self.handle, ticket, float(timeout_s), ctypes.byref(r))
        return self._result(ticket, st, r)

    def run(self):
        st = self._L.mfc_batch_run(self.handle)
        if st != MFC_OK:
            raise MfcError(st, self._L.mfc_batch_last_error(self.handle).decode())

    def start(self):
        st = self._L.mfc_batch_start(self.handle)
        if st != MFC_OK:
            raise MfcError(st, "mfc_batch_start")

    def stop(self):
        self._L.mfc_batch_stop(self.handle)

    def stats(self) -> dict:
        s = BatchStats()
        self._L.mfc_batch_get_stats(self.handle, ctypes.byref(s))
        return s.as_dict()

    def close(self):
        if self.handle:
            self._L.mfc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def electro_params(**over) -> ElectroParams:
    """The library's defaults (Table 1 and the chosen constants), with fields replaced by
    ``over`` (``mediator_yield`` is Y)."""
    p = ElectroParams()
    st = lib().mfc_electro_default_params(ctypes.byref(p))
    if st != MFC_OK:
        raise MfcError(st, "mfc_electro_default_params")
    for k, v in over.items():
        setattr(p, k, v)
    return p


def electro_update(params: ElectroParams, substrate_factor: float, c_bio: float,
                   m_ox: float) -> dict:
    """One call of mfc_electro_update: the mediator balance and the cell's current and voltage
    after params.substeps steps (Eqs. 14-21)."""
    r = ElectroResult()
    st = lib().mfc_electro_update(ctypes.byref(params), substrate_factor, c_bio, m_ox,
                                  ctypes.byref(r))
    if st != MFC_OK:
        raise MfcError(st, "mfc_electro_update")
    return r.as_dict()


def clock() -> float:
    """Seconds on the library's monotonic clock (the clock of the batch time stamps)."""
    return float(lib().mfc_clock())
