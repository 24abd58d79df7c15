#!/usr/bin/env python3
"""Benchmark of the coupled flow + substrate-transport lattice Boltzmann hot path on GB300.

Workload: the 2048x1024 porous anode (random overlapping discs of radius 6, porosity 0.7 in the
middle half of the channel, seeded), D2Q9 flow + D2Q5 transport, FP32 storage and arithmetic
(FP64 reductions).  One step is one fused update of every node of both lattices; steps run in
CUDA-graph blocks of K (default 200) that end with the residual/current reduction and the
host-side convergence decision, exactly as a steady solve runs them (tolerance 0, so every
block is taken).  The working set (2 x 14 planes x 4 B x 2.1 M nodes = 235 MB of populations)
is larger than the 129 MB L2, so no explicit flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) are independent replicas, one lattice
per GPU, each with its own seed (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled flow+ADE MLUPS & % of HBM roofline; served solves/s with p50/p99 latency"
WORKLOAD = "anode_2d_2048x1024_fused_d2q9_d2q5"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=2000)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--check-every", type=int, default=200)
    ap.add_argument("--precision", choices=["fp32", "fp16"], default="fp32")
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=1000,
                    help="lattice updates per end-to-end step (upload, solve block, read back)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, seconds_target=10.0):
    """The FP64 oracle as it stands, one thread, on a bounded sample: fused steps of the full
    2048x1024 anode from rest, as many as fit about ten seconds."""
    import numpy as np  # noqa: F401
    import oracle
    o = oracle.Oracle(w.shape, w.cls, tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in,
                      k_sink=w.k_sink)
    t0 = time.perf_counter()
    o.step_coupled(1)
    t1 = time.perf_counter() - t0
    n = max(1, int(seconds_target / max(t1, 1e-6)))
    t0 = time.perf_counter()
    o.step_coupled(n)
    dt = time.perf_counter() - t0
    return {"value": w.nodes * n / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{n} fused D2Q9+D2Q5 steps of the full {w.shape[0]}x{w.shape[1]} anode "
                      f"from rest, FP64 C oracle, 1 thread ({dt:.1f} s)"}


def traffic_record(kernel):
    """DRAM bytes per launch of the kernel from the committed ncu summary, if it was taken
    on the kernel code that is built now (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    from paper_1802_07525_gb300 import build
    rec = d.get(kernel)
    if not rec or rec.get("kernel_digest") != build.kernel_digest(rec["translation_unit"]):
        return None
    return rec.get("dram_bytes_per_launch_full")


def run_reference(args, rank, world):
    """The oracle as the reference arm: every step is one fused FP64 update of a slab of the
    workload's rows, sized so that the whole run ends within a few minutes."""
    if rank != 0:
        return
    import numpy as np
    import mfc_inputs as mi
    import oracle
    w = mi.anode_2d(args.nx, args.ny)
    total = args.steps + args.warmup
    budget = 150.0 / max(total, 1)
    # calibrate on a 16-row slab
    rows = 16

    def slab(r):
        y0 = w.shape[1] // 2 - r // 2
        cls = w.cls.reshape(w.shape[1], w.shape[0])[y0:y0 + r].reshape(-1)
        return oracle.Oracle((w.shape[0], r), cls, tau=w.tau, tau_c=w.tau_c, u_in=w.u_in,
                             c_in=w.c_in, k_sink=w.k_sink)

    o = slab(rows)
    t0 = time.perf_counter()
    o.step_coupled(2)
    per_row = (time.perf_counter() - t0) / (2 * rows)
    rows = int(max(1, min(w.shape[1], budget / max(per_row, 1e-9))))
    o = slab(rows)
    o.step_coupled(args.warmup)
    t0 = time.perf_counter()
    o.step_coupled(args.steps)
    dt = time.perf_counter() - t0
    nodes = w.shape[0] * rows
    value = nodes * args.steps / dt / 1e6
    sample = (f"each step one fused FP64 update of a {w.shape[0]}x{rows} slab of the "
              f"{w.shape[0]}x{w.shape[1]} anode (middle rows), 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nodes": w.nodes, "sample_nodes": nodes},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        # one GPU per rank: the library and torch both see it as device 0
        os.environ["CUDA_VISIBLE_DEVICES"] = str(local)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import mfc_inputs as mi
    import paper_1802_07525_gb300 as P
    from paper_1802_07525_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)
        pg = dist

    w = mi.anode_2d(args.nx, args.ny, seed=2 + rank)
    prec = P.MFC_FP16_DEV if args.precision == "fp16" else P.MFC_FP32
    stream = torch.cuda.Stream()
    lat = P.Lattice(w.shape, precision=prec, stream=stream.cuda_stream, tau=w.tau,
                    tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)
    lat.set_geometry(w.cls)
    flow_open, ade_open = lat.active_nodes()
    K = args.check_every

    def run(nsteps):
        r = lat.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0,
                             max_steps=nsteps, check_every=K)
        assert r.status == P.MFC_NOT_CONVERGED, P.status_string(r.status)
        return r

    # warm-up (builds and instantiates the graph)
    run(max(args.warmup, 3))
    torch.cuda.synchronize()

    # timed region
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:  # nvidia-smi takes the UUID, which does not depend on CUDA_VISIBLE_DEVICES
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        gpu_id = str(local)
    with ClockSampler(gpu_id) as clocks:
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        res = run(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
    ms = ev0.elapsed_time(ev1)
    if pg:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    total_nodes = w.nodes * world
    value = total_nodes * args.steps / (ms * 1e-3) / 1e6

    # dominant kernel: the plain fused step, timed alone on the same stream
    M = 400
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat.step_coupled(20)
    e0.record(stream)
    lat.step_coupled(M)
    e1.record(stream)
    torch.cuda.synchronize()
    kern_ms = e0.elapsed_time(e1) / M
    sb = 2 if prec == P.MFC_FP16_DEV else 4
    bytes_per_launch = 2 * sb * (9 * flow_open + 5 * ade_open)
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / (kern_ms * 1e-3) / 1e9
    kname = "lbm_step_kernel<2,%s,true,true,0>" % ("half" if sb == 2 else "float")
    traffic = traffic_record(kname)

    # end to end through the public API with host buffers: upload classes from pinned memory,
    # one solve block of e2e_steps updates, read rho, u, C and the current back to pinned memory
    n_e2e = 3
    cls_h = torch.from_numpy(w.cls).pin_memory()
    rho_h = torch.empty(w.nodes, dtype=torch.float64).pin_memory()
    u_h = torch.empty(2 * w.nodes, dtype=torch.float64).pin_memory()
    c_h = torch.empty(w.nodes, dtype=torch.float64).pin_memory()
    cur_h = torch.empty(1, dtype=torch.float64).pin_memory()
    import ctypes
    L = P.lib()
    dp = ctypes.POINTER(ctypes.c_double)

    def e2e_step():
        st = L.mfc_set_geometry(lat.handle, ctypes.cast(cls_h.data_ptr(),
                                                        ctypes.POINTER(ctypes.c_uint8)), 1)
        assert st == 0
        r = lat.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0,
                             max_steps=args.e2e_steps, check_every=K)
        assert r.status == P.MFC_NOT_CONVERGED
        st = L.mfc_read_fields(lat.handle, ctypes.cast(rho_h.data_ptr(), dp),
                               ctypes.cast(u_h.data_ptr(), dp), ctypes.cast(c_h.data_ptr(), dp),
                               ctypes.cast(cur_h.data_ptr(), dp))
        assert st == 0

    e2e_step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if pg:
        t = torch.tensor([e2e_s], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = total_nodes * args.e2e_steps * n_e2e / e2e_s / 1e6
    assert np.isfinite(c_h.numpy()).all()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if rank == 0:
        launches = args.steps + (args.steps + K - 1) // K
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if sb == 4 else "f16-storage/f32-math", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": args.nx, "ny": args.ny,
                       "nodes_per_gpu": w.nodes, "flow_open": flow_open, "ade_open": ade_open,
                       "check_every": K, "parallelism": f"replicas{world}",
                       "l2": "working set 235 MB > 129 MB L2, no flush",
                       "mflups_flow_open": flow_open * world * args.steps / (ms * 1e-3) / 1e6},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel": kname, "kernel_ms": kern_ms,
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": int(w.nodes),
                    "d2h_bytes_per_step": int(w.nodes * 8 * 4 + 8),
                    "updates_per_step": args.e2e_steps},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "final": {"res_flow": res.res_flow, "res_ade": res.res_ade, "current": res.current},
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
