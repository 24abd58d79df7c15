"""The slab-decomposition driver over a real two-rank process group (gloo, CPU).

Each rank holds one slab of a small stand-in lattice (a 1-D three-velocity BGK model with the same
halo interface as the library's lattices: pull streaming, an inlet and an outlet at the ends of
the whole domain, cut faces between slabs).  Stepped through DistributedSlab, with its halo
exchange and the FP64 all-reduce of the check sums, the two slabs must reproduce the whole
domain stepped alone, exactly, and the summed check sums and residuals must be the whole
domain's.  No GPU is involved: this covers the slab driver's ordering and reductions on two
processes; the kernels' side is covered on one GPU with slabs in one process.
"""
import ctypes
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


class ChainSlab:
    """A 1-D D1Q3 BGK lattice (velocities 0, +1, -1) on nodes [0, n) with a ghost on each side.
    The low end of the whole domain is an inlet (the right-moving ghost at equilibrium at rho 1,
    velocity u_in), the high end an outlet (zero gradient); a cut face takes its ghost from the
    neighbouring slab."""

    W = (2 / 3, 1 / 6, 1 / 6)

    def __init__(self, n, cut=(False, False), tau=0.8, u_in=0.05, x0=0):
        self.n, self.cut, self.omega, self.u_in = n, cut, 1.0 / tau, u_in
        x = np.arange(x0, x0 + n)
        rho = 1.0 + 0.1 * np.sin(0.3 * x)  # a non-uniform start, the same for any split
        self.f = np.zeros((3, n + 2))
        for i in range(3):
            self.f[i, 1:-1] = self.W[i] * rho
        self.rho = rho.copy()
        self.u = np.zeros(n)
        self.rho_prev, self.u_prev = self.rho.copy(), self.u.copy()
        self._boundaries()

    def _boundaries(self):
        if not self.cut[0]:
            self.f[1, 0] = self.W[1] * (1.0 + 3.0 * self.u_in)
        if not self.cut[1]:
            self.f[2, -1] = self.f[2, -2]

    def synchronize(self):
        pass

    def step_coupled_plain(self, n=1):
        self.step_coupled(n)

    def step_coupled(self, n=1):
        for _ in range(n):
            g = self.f.copy()
            g[1, 1:-1] = self.f[1, :-2]
            g[2, 1:-1] = self.f[2, 2:]
            fin = g[:, 1:-1]
            rho = fin.sum(0)
            u = (fin[1] - fin[2]) / rho
            for i, c in enumerate((0, 1, -1)):
                feq = self.W[i] * rho * (1 + 3 * c * u + 4.5 * (c * u) ** 2 - 1.5 * u * u)
                fin[i] += self.omega * (feq - fin[i])
            self.f = g
            self.rho, self.u = rho, u
            self._boundaries()

    def step_check_sums(self, n=1):
        self.step_coupled(n)
        s = np.zeros(9)
        s[0] = ((self.u - self.u_prev) ** 2).sum()
        s[1] = (self.u ** 2).sum()
        s[2] = self.rho.sum()
        s[3] = ((self.rho - self.rho_prev) ** 2).sum()
        s[4] = (self.rho ** 2).sum()
        s[5] = self.rho.sum()
        s[6] = 1e-3 * self.rho.sum()
        self.rho_prev, self.u_prev = self.rho.copy(), self.u.copy()
        return s

    # halo interface: one double per face
    def halo_bytes(self, side):
        if not self.cut[side]:
            raise ValueError("not a cut")
        return 8

    def halo_pack(self, side, ptr):
        v = np.array([self.f[1, -2] if side == 1 else self.f[2, 1]])
        ctypes.memmove(ptr, v.ctypes.data, 8)

    def halo_unpack(self, side, ptr):
        v = np.zeros(1)
        ctypes.memmove(v.ctypes.data, ptr, 8)
        if side == 0:
            self.f[1, 0] = v[0]
        else:
            self.f[2, -1] = v[0]


def _rank_main(rank, world, port, n, q):
    import torch.distributed as dist
    from paper_1802_07525_gb300 import slab as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = S.slab_bounds(n, world, rank)
        mine = ChainSlab(hi - lo, cut=(rank > 0, rank < world - 1), x0=lo)
        ds = S.DistributedSlab(mine, dist, device="cpu")
        ref = ChainSlab(n)
        ds.exchange()  # the ghosts of the start state
        ds.step(37)
        ref.step_coupled(37)
        ok_state = np.array_equal(mine.f[:, 1:-1], ref.f[:, 1 + lo:1 + hi])
        sums = ds.check(10)
        ref_sums = ref.step_check_sums(10)
        ok_sums = np.allclose(sums, ref_sums, rtol=1e-13, atol=0.0)
        r = ds.solve_steady(1e-9, 1e-9, 3000, 50)
        ref2 = ChainSlab(n)
        ref2.step_coupled(47)
        rr = S._solve(ref2.step_check_sums, 1e-9, 1e-9, 3000, 50)
        ok_solve = r["steps"] == rr["steps"] and r["status"] == rr["status"] and \
            abs(r["res_flow"] - rr["res_flow"]) <= 1e-12 * max(rr["res_flow"], 1e-300)
        ok_final = np.array_equal(mine.f[:, 1:-1], ref2.f[:, 1 + lo:1 + hi])
        q.put((rank, bool(ok_state), bool(ok_sums), bool(ok_solve), bool(ok_final), r["status"]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_slabs_reproduce_the_whole_domain(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, 61, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ok_state, ok_sums, ok_solve, ok_final, status in res:
        assert ok_state and ok_sums and ok_solve and ok_final, (rank, ok_state, ok_sums, ok_solve,
                                                                 ok_final, status)
    assert res[0][-1] == "converged"


def test_slab_bounds_cover_the_axis():
    from paper_1802_07525_gb300 import slab as S
    for n, w in ((61, 2), (61, 3), (128, 8), (7, 7)):
        b = [S.slab_bounds(n, w, r) for r in range(w)]
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(b[r][1] == b[r + 1][0] for r in range(w - 1))
        assert max(h - l for l, h in b) - min(h - l for l, h in b) <= 1
