"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This module generates geometry (node-class masks) and workload descriptions only; it holds
none of the lattice Boltzmann arithmetic.  Randomness comes from a counter-based splitmix64
(Steele, Lea and Flood, OOPSLA 2014, in the form published by Vigna), so every mask is a pure
function of (shape, parameters, seed).

Node classes are uint8 bit flags, x fastest (k = x + nx*(y + ny*z)):
  1 = blocked for the flow lattice, 2 = blocked for the transport lattice, 4 = consumption
  (biofilm sink).  Electrode material is 1|2; the initial biofilm layer is 4 on the open nodes
  next to the electrode; biofilm grown later is 1|4 (impermeable to flow, still transported).

The paper's own anode (a 60x65 lattice of random shapes, porosity 0.874) is shown only as a
figure, so these generators stand in for it with the shapes, porosities and sizes of the
workloads the method is run on.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FLOW_SOLID, ADE_SOLID, SINK = 1, 2, 4
ELECTRODE = FLOW_SOLID | ADE_SOLID
BIOFILM = FLOW_SOLID | SINK

_M64 = 0xFFFFFFFFFFFFFFFF


def splitmix64(x):
    """splitmix64 finaliser of (x + golden gamma), vectorised over uint64 arrays."""
    z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counter):
    """Uniform doubles in [0, 1) from counter-based draws of stream ``seed``."""
    key = np.uint64((int(seed) * 0x632BE59BD9B4E019) & _M64)
    h = splitmix64(key ^ np.asarray(counter, dtype=np.uint64))
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _block_bounds(n_flow: int, lo=None, hi=None):
    """The porous block along the flow axis: [lo, hi), default the middle half."""
    return (n_flow // 4 if lo is None else lo, (3 * n_flow) // 4 if hi is None else hi)


def bernoulli_block(shape, p_solid: float, seed: int, block=None) -> np.ndarray:
    """2-D/3-D mask with electrode nodes drawn Bernoulli(p_solid) inside the porous block."""
    shape = tuple(shape)
    dim = len(shape)
    N = int(np.prod(shape))
    cls = np.zeros(N, np.uint8)
    idx = np.arange(N, dtype=np.uint64)
    solid = uniform01(seed, idx) < p_solid
    coord = _axis_coord(shape, 0 if dim == 2 else 2)
    lo, hi = block if block is not None else _block_bounds(shape[0 if dim == 2 else 2])
    solid &= (coord >= lo) & (coord < hi)
    cls[solid] = ELECTRODE
    return cls


def _axis_coord(shape, axis):
    nx = shape[0]
    ny = shape[1]
    k = np.arange(int(np.prod(shape)))
    if axis == 0:
        return k % nx
    if axis == 1:
        return (k // nx) % ny
    return k // (nx * ny)


def overlapping_balls(shape, radius: int, porosity: float, seed: int, block=None) -> np.ndarray:
    """Random overlapping discs (2-D) or spheres (3-D) of ``radius`` inside the porous block,
    added one at a time until the solid fraction of the block reaches 1 - porosity.
    A node is inside a ball when its squared distance to the centre is <= radius^2."""
    shape = tuple(int(s) for s in shape)
    dim = len(shape)
    fa = 0 if dim == 2 else 2
    lo, hi = block if block is not None else _block_bounds(shape[fa])
    grid = np.zeros(shape[::-1], dtype=bool)  # [z][y][x] or [y][x]
    lens = list(shape)
    lens[fa] = hi - lo
    block_nodes = int(np.prod(lens))
    target = math.ceil((1.0 - porosity) * block_nodes)
    r = int(radius)
    offs = np.arange(-r, r + 1)
    if dim == 2:
        dy, dx = np.meshgrid(offs, offs, indexing="ij")
        stamp = (dx * dx + dy * dy) <= r * r
    else:
        dz, dy, dx = np.meshgrid(offs, offs, offs, indexing="ij")
        stamp = (dx * dx + dy * dy + dz * dz) <= r * r
    solid = 0
    j = 0
    while solid < target:
        u = uniform01(seed, np.arange(dim * j, dim * (j + 1), dtype=np.uint64))
        cen = [int(u[a] * shape[a]) for a in range(dim)]
        cen[fa] = lo + int(u[fa] * (hi - lo))
        j += 1
        # window of the stamp clipped to the block (flow axis) and the lattice (other axes)
        sl_g, sl_s = [], []
        for a in range(dim):
            a_lo = lo if a == fa else 0
            a_hi = hi if a == fa else shape[a]
            g0 = max(cen[a] - r, a_lo)
            g1 = min(cen[a] + r + 1, a_hi)
            sl_g.append(slice(g0, g1))
            sl_s.append(slice(g0 - (cen[a] - r), g1 - (cen[a] - r)))
        sl_g = tuple(sl_g[::-1])
        sl_s = tuple(sl_s[::-1])
        win = grid[sl_g]
        new = stamp[sl_s] & ~win
        solid += int(new.sum())
        win |= stamp[sl_s]
    cls = np.zeros(grid.size, np.uint8)
    cls[grid.reshape(-1)] = ELECTRODE
    return cls


def mark_sink_layer(shape, cls: np.ndarray, biofilm_class: int = SINK) -> np.ndarray:
    """Mark the open nodes next to electrode material (any of the 8 neighbours in 2-D, 18 in
    3-D, inside the lattice) with ``biofilm_class``: SINK (consumption on a flow-open node)
    or BIOFILM (impermeable biofilm)."""
    shape = tuple(shape)
    dim = len(shape)
    g = (cls.reshape(shape[::-1]) & FLOW_SOLID).astype(bool)
    near = np.zeros_like(g)
    rng = (-1, 0, 1)
    if dim == 2:
        for dy in rng:
            for dx in rng:
                if dx == 0 and dy == 0:
                    continue
                near |= _shifted(g, (dy, dx))
    else:
        for dz in rng:
            for dy in rng:
                for dx in rng:
                    n1 = abs(dx) + abs(dy) + abs(dz)
                    if n1 == 0 or n1 == 3:
                        continue
                    near |= _shifted(g, (dz, dy, dx))
    out = cls.copy()
    sel = near.reshape(-1) & (cls == 0)
    out[sel] = biofilm_class
    return out


def _shifted(g, d):
    """s[idx] = g[idx + d] where inside, else False."""
    s = np.zeros_like(g)
    src, dst = [], []
    for a, da in enumerate(d):
        n = g.shape[a]
        if da >= 0:
            src.append(slice(da, n))
            dst.append(slice(0, n - da))
        else:
            src.append(slice(0, n + da))
            dst.append(slice(-da, n))
    s[tuple(dst)] = g[tuple(src)]
    return s


# --------------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    shape: tuple
    cls: np.ndarray
    tau: float
    tau_c: float
    u_in: float
    c_in: float = 1.0
    k_sink: float = 1e-3
    tol: float = 1e-8
    max_steps: int = 10000

    @property
    def dim(self):
        return len(self.shape)

    @property
    def nodes(self):
        return int(np.prod(self.shape))


def channel_128x64(seed: int = 1) -> Workload:
    """2-D plain channel: 128x64, porous block x in [32, 96) of Bernoulli(0.3) electrode nodes,
    sink on the open nodes next to them, tau 0.8 / 0.7, inlet u 0.01, k 1e-3, tol 1e-8, 10^4."""
    shape = (128, 64)
    cls = bernoulli_block(shape, 0.3, seed, block=(32, 96))
    cls = mark_sink_layer(shape, cls, SINK)
    return Workload("channel_128x64", shape, cls, 0.8, 0.7, 0.01, 1.0, 1e-3, 1e-8, 10000)


def anode_2d(nx: int = 2048, ny: int = 1024, seed: int = 2, porosity: float = 0.7,
             radius: int = 6) -> Workload:
    """2-D porous anode: random overlapping discs of radius 6 at porosity 0.7 in the middle
    half of the channel, sink layer next to the discs; tau 0.8 / 0.7, u 0.01, k 1e-3, tol 1e-7."""
    shape = (nx, ny)
    cls = overlapping_balls(shape, radius, porosity, seed)
    cls = mark_sink_layer(shape, cls, SINK)
    return Workload(f"anode_2d_{nx}x{ny}", shape, cls, 0.8, 0.7, 0.01, 1.0, 1e-3, 1e-7, 100000)


def electrode_3d(nx: int = 256, ny: int = 128, nz: int = 128, seed: int = 3,
                 porosity: float = 0.6, radius: int = 4) -> Workload:
    """3-D porous electrode: random overlapping spheres of radius 4 at porosity 0.6, flow along
    z; D3Q19 tau 0.7, D3Q7 tau_c 0.6, inlet u_z 0.005, k 5e-4."""
    shape = (nx, ny, nz)
    cls = overlapping_balls(shape, radius, porosity, seed)
    cls = mark_sink_layer(shape, cls, SINK)
    return Workload(f"electrode_3d_{nx}x{ny}x{nz}", shape, cls, 0.7, 0.6, 0.005, 1.0, 5e-4,
                    1e-7, 100000)


def batch_instances(count: int = 64, seed: int = 4, nx_range=(256, 1024), ny_range=(128, 512),
                    porosity_range=(0.5, 0.9), tau_range=(0.6, 1.0),
                    u_range=(0.002, 0.02)) -> list:
    """Uneven batch: instance i uses seed + i; sizes uniform over the integer ranges,
    porosity, tau and inlet speed uniform over their intervals; discs of radius 6."""
    out = []
    for i in range(count):
        s = seed + i
        u = uniform01(10_000 + s, np.arange(5, dtype=np.uint64))
        nx = nx_range[0] + int(u[0] * (nx_range[1] - nx_range[0] + 1))
        ny = ny_range[0] + int(u[1] * (ny_range[1] - ny_range[0] + 1))
        por = porosity_range[0] + u[2] * (porosity_range[1] - porosity_range[0])
        tau = tau_range[0] + u[3] * (tau_range[1] - tau_range[0])
        uin = u_range[0] + u[4] * (u_range[1] - u_range[0])
        cls = overlapping_balls((nx, ny), 6, por, s)
        cls = mark_sink_layer((nx, ny), cls, SINK)
        # the workload names no step cap; 3e5 lets every instance reach 1e-7 in FP32
        out.append(Workload(f"batch{i}_{nx}x{ny}", (nx, ny), cls, float(tau), 0.7, float(uin),
                            1.0, 1e-3, 1e-7, 300000))
    return out


SERVING_MAX_STEPS = 1_000_000


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    shape: tuple
    seed: int
    porosity: float

    def workload(self) -> Workload:
        # tolerance 1e-7 as in the batched workload; the cap is 1e6 steps because the longest
        # 2-D channels (2048 nodes along the flow at inlet speed 0.01) take more than the batched
        # workload's 3e5 steps to settle to 1e-7
        if len(self.shape) == 2:
            cls = overlapping_balls(self.shape, 6, self.porosity, self.seed)
            cls = mark_sink_layer(self.shape, cls, SINK)
            return Workload(f"req{self.rid}", self.shape, cls, 0.8, 0.7, 0.01, 1.0, 1e-3, 1e-7,
                            SERVING_MAX_STEPS)
        cls = overlapping_balls(self.shape, 4, self.porosity, self.seed)
        cls = mark_sink_layer(self.shape, cls, SINK)
        return Workload(f"req{self.rid}", self.shape, cls, 0.7, 0.6, 0.005, 1.0, 5e-4, 1e-7,
                        SERVING_MAX_STEPS)


def serving_stream(count: int = 2000, rate_per_s: float = 200.0, seed: int = 5,
                   frac_2d: float = 0.7, size_2d=((512, 2048), (256, 1024)),
                   size_3d=((64, 192), (64, 96), (64, 96)), porosity=(0.5, 0.9)) -> list:
    """Poisson arrivals of steady-solve requests: 70% 2-D, 30% 3-D, sizes uniform per axis."""
    out = []
    t = 0.0
    for i in range(count):
        u = uniform01(20_000 + seed, np.arange(6 * i, 6 * i + 6, dtype=np.uint64))
        t += -math.log(1.0 - u[0]) / rate_per_s
        if u[1] < frac_2d:
            nx = size_2d[0][0] + int(u[2] * (size_2d[0][1] - size_2d[0][0] + 1))
            ny = size_2d[1][0] + int(u[3] * (size_2d[1][1] - size_2d[1][0] + 1))
            shape = (nx, ny)
        else:
            shape = tuple(size_3d[a][0] + int(u[2 + a] * (size_3d[a][1] - size_3d[a][0] + 1))
                          for a in range(3))
        por = porosity[0] + u[5] * (porosity[1] - porosity[0])
        out.append(Request(i, t, shape, seed * 1_000_003 + i, float(por)))
    return out
