"""Slab decomposition of one lattice along its flow axis (argument marshalling and orchestration;
every population update and copy runs in the library's kernels).

A lattice too large for one GPU is split along the flow axis into slabs, slab r on rank r, in
flow-axis order.  Each slab is a lattice whose faces towards its neighbours are cuts
(``cut=(r > 0, r < world - 1)``).  One step of the whole lattice is one step of every slab
followed by the halo exchange: each slab packs the populations leaving it through a cut face
(``mfc_halo_pack``), they travel to the neighbour, which unpacks them into its ghost layer
(``mfc_halo_unpack``).  A check step's nine FP64 sums are summed over the slabs, then the
residuals follow as for a whole lattice (the mean relative change per step since the previous
check).  The exchange runs over a ``torch.distributed`` process group (NCCL between GPUs, gloo on
CPU), or, for slabs held by one process, as direct device copies (:func:`exchange_local`).

Any object with ``halo_bytes(side)``, ``halo_pack(side, ptr)``, ``halo_unpack(side, ptr)``,
``step_coupled_plain(n)`` (steps that keep the stored fields, so that a check compares with the
previous check), ``step_check_sums(n)`` and ``synchronize()`` can be a slab; :class:`~.mfc.Lattice`
is one.
"""
from __future__ import annotations

import math

import numpy as np

SUM_DU2, SUM_U2, SUM_MASS, SUM_DC2, SUM_C2, SUM_C, SUM_CURRENT, SUM_BAD, SUM_FAST = range(9)


def slab_bounds(n: int, world: int, rank: int):
    """[lo, hi) of slab `rank` when n layers split into `world` slabs as evenly as possible."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def residuals(sums, nsteps: int):
    """Flow and transport residuals of summed check sums, per step over nsteps steps."""
    rf = math.sqrt(sums[SUM_DU2] / sums[SUM_U2]) if sums[SUM_U2] > 0 else (
        math.inf if sums[SUM_DU2] > 0 else 0.0)
    ra = math.sqrt(sums[SUM_DC2] / sums[SUM_C2]) if sums[SUM_C2] > 0 else (
        math.inf if sums[SUM_DC2] > 0 else 0.0)
    return rf / nsteps, ra / nsteps


def _buffers(slab, torch, device, dtype):
    out = {}
    for side in (0, 1):
        try:
            n = slab.halo_bytes(side)
        except Exception:
            continue
        out[side] = (torch.empty(n, dtype=torch.uint8, device=device),
                     torch.empty(n, dtype=torch.uint8, device=device))
    return out


def exchange_local(slabs, bufs):
    """One halo exchange among slabs held by this process, in flow-axis order: the populations
    leaving slab r upwards go into slab r + 1's low ghost layer and those leaving slab r + 1
    downwards into slab r's high ghost layer.  bufs[r] = (buffer, buffer) per neighbour pair.
    Each slab works on its own stream, so the packs wait for every slab's step and the unpacks
    for every pack."""
    for s in slabs:
        s.synchronize()
    for r in range(len(slabs) - 1):
        up, down = bufs[r]
        slabs[r].halo_pack(1, up.data_ptr())
        slabs[r + 1].halo_pack(0, down.data_ptr())
    for s in slabs:
        s.synchronize()
    for r in range(len(slabs) - 1):
        up, down = bufs[r]
        slabs[r + 1].halo_unpack(0, up.data_ptr())
        slabs[r].halo_unpack(1, down.data_ptr())


class LocalSlabs:
    """Slabs of one lattice held by one process (one GPU), stepped together with exchanges."""

    def __init__(self, slabs):
        import torch
        self.slabs = list(slabs)
        self.bufs = []
        for r in range(len(self.slabs) - 1):
            n = self.slabs[r].halo_bytes(1)
            assert n == self.slabs[r + 1].halo_bytes(0)
            self.bufs.append((torch.empty(n, dtype=torch.uint8, device="cuda"),
                              torch.empty(n, dtype=torch.uint8, device="cuda")))

    def exchange(self):
        exchange_local(self.slabs, self.bufs)

    def step(self, n: int = 1):
        for _ in range(n):
            for s in self.slabs:
                s.step_coupled_plain(1)
            self.exchange()

    def check(self, nsteps: int):
        """nsteps steps, the last a check step: the sums over every slab."""
        self.step(nsteps - 1)
        total = np.zeros(9)
        for s in self.slabs:
            total += s.step_check_sums(1)
        self.exchange()
        return total

    def solve_steady(self, tol_flow, tol_ade, max_steps, check_every):
        return _solve(self.check, tol_flow, tol_ade, max_steps, check_every)


class DistributedSlab:
    """This rank's slab of a lattice split across the ranks of a process group (rank order is
    flow-axis order).  Halos travel by point-to-point send/receive, check sums by an all-reduce in
    FP64."""

    def __init__(self, slab, dist, group=None, device="cuda"):
        import torch
        self.slab, self.dist, self.group = slab, dist, group
        self.torch = torch
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = device
        self.bufs = {}
        for side, peer in ((0, self.rank - 1), (1, self.rank + 1)):
            if 0 <= peer < self.world:
                n = slab.halo_bytes(side)
                self.bufs[side] = (torch.empty(n, dtype=torch.uint8, device=device),
                                   torch.empty(n, dtype=torch.uint8, device=device))

    def _peer(self, side):
        return self.rank - 1 if side == 0 else self.rank + 1

    def exchange(self):
        """Pack both cut faces, swap with the neighbours, unpack what arrived."""
        dist = self.dist
        if self.device == "cuda":
            self.torch.cuda.current_stream().synchronize()
        ops = []
        for side, (out, inn) in self.bufs.items():
            self.slab.halo_pack(side, out.data_ptr())
        if self.device == "cuda":
            self.slab.synchronize()
        for side, (out, inn) in self.bufs.items():
            peer = dist.get_global_rank(self.group, self._peer(side)) if self.group else self._peer(side)
            ops.append(dist.P2POp(dist.isend, out, peer, self.group))
            ops.append(dist.P2POp(dist.irecv, inn, peer, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if self.device == "cuda":
            self.torch.cuda.current_stream().synchronize()
        for side, (out, inn) in self.bufs.items():
            self.slab.halo_unpack(side, inn.data_ptr())

    def step(self, n: int = 1):
        for _ in range(n):
            self.slab.step_coupled_plain(1)
            self.exchange()

    def check(self, nsteps: int):
        self.step(nsteps - 1)
        local = self.slab.step_check_sums(1)
        self.exchange()
        t = self.torch.tensor(local, dtype=self.torch.float64,
                              device=self.device if self.device != "cpu" else "cpu")
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def solve_steady(self, tol_flow, tol_ade, max_steps, check_every):
        return _solve(self.check, tol_flow, tol_ade, max_steps, check_every)


def _solve(check, tol_flow, tol_ade, max_steps, check_every):
    """The steady-state loop of mfc_solve_steady over summed check sums (concurrent mode): a check
    every check_every steps and at the cap; stop at the first check with both residuals below
    tolerance, at a non-finite or out-of-range check, or at the cap."""
    steps = 0
    out = {"status": "not_converged"}
    while steps < max_steps:
        n = min(check_every, max_steps - steps)
        s = check(n)
        steps += n
        rf, ra = residuals(s, n)
        out = {"steps": steps, "res_flow": rf, "res_ade": ra, "current": float(s[SUM_CURRENT]),
               "mass": float(s[SUM_MASS]), "substrate": float(s[SUM_C]), "sums": s}
        if s[SUM_BAD] > 0 or not np.isfinite(s[SUM_MASS]) or not np.isfinite(s[SUM_C]):
            out["status"] = "nonfinite"
            return out
        if s[SUM_FAST] > 0:
            out["status"] = "unstable"
            return out
        if rf < tol_flow and ra < tol_ade:
            out["status"] = "converged"
            return out
        out["status"] = "not_converged"
    return out
