#!/usr/bin/env python3
"""Benchmark of the coupled flow + substrate-transport lattice Boltzmann hot path on GB300.

Headline workload: the 256x128x128 porous electrode (random overlapping spheres of radius 4,
porosity 0.6 in the middle half of the flow axis z, seeded), D3Q19 flow + D3Q7 transport, FP32
storage and arithmetic (FP64 reductions): the largest single-GPU configuration.  One step is one
fused update of every node of both lattices; steps run in CUDA-graph blocks of K that end with
the residual/current reduction and the host-side convergence decision, exactly as a steady solve
runs them (tolerance 0, so every block is taken).  K is the largest divisor of --steps that is
at most --check-every, so the timed region is whole graph replays however few steps are asked
for.  The working set (2 x 26 planes x 4 B x 4.2 M nodes = 872 MB of populations) is larger
than the 129 MB L2, so no explicit flush is needed between steps.  --workload anode2d times the
2048x1024 anode (D2Q9 + D2Q5) instead.

Further legs on one GPU (rank 0 of a 1-GPU run), each reported in the same JSON line:
  variants  - the 2048x1024 anode (FP32), the FP16-storage 2-D step, the 2-D step with the
              paper-literal D2Q9 transport and with the saturating consumption, and the 3-D
              electrode with FP16 storage: MLUPS and fraction of the HBM roofline;
  accuracy  - FP32 and FP16 results against the FP64 oracle (populations after a fixed number
              of steps, steady fields and current), the oracle running in spawned processes
              while the GPU legs run;
  batch     - 64 uneven 2-D instances solved to 1e-7 by the batch engine against the same
              solves one at a time (solves/s at equal accuracy);
  serve     - a Poisson stream of 2-D/3-D steady-solve requests through the batch engine's
              thread: capacity at the offered rate of 200/s, then p50/p99 latency at 0.8x the
              measured capacity;
  biofilm   - (only when asked for: it takes minutes) the 2048x1024 anode through 50 biofilm
              cycles: each cycle solves flow and transport to steady state (1e-7, at most 1e5
              steps), advances the cell's electrical model one hour, then grows biofilm by the
              seeded rule and warm-starts the next;
  model     - (only when asked for) the paper's whole loop on the 2048x1024 anode, one iteration
              per hour: steady flow and transport, the electrical model, the agent-based biofilm.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--legs ...]

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) are independent replicas, one lattice
per GPU, each with its own seed (weak scaling, no data-path collective); they run the headline
leg only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled flow+ADE MLUPS & % of HBM roofline; served solves/s with p50/p99 latency"
WORKLOADS = {"anode2d": "anode_2d_2048x1024_fused_d2q9_d2q5",
             "electrode3d": "electrode_3d_256x128x128_fused_d3q19_d3q7"}
DEFAULT_WORKLOAD = "electrode3d"
ALL_LEGS = "main,variants,accuracy,batch,serve"
EXTRA_LEGS = "biofilm,model"


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
    ap.add_argument("--legs", default=ALL_LEGS,
                    help="comma-separated subset of " + ALL_LEGS + "," + EXTRA_LEGS)
    ap.add_argument("--biofilm-cycles", type=int, default=50)
    ap.add_argument("--model-hours", type=int, default=24,
                    help="hours of the full model loop (the 'model' leg)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD,
                    help="lattice of the headline leg (electrode3d: the 256x128x128 electrode; "
                         "anode2d: the --nx x --ny anode)")
    ap.add_argument("--batch-max-steps", type=int, default=0,
                    help="step cap of the batch leg's solves (0: the workload's own cap)")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--serve-count", type=int, default=24, help="requests per serving phase")
    return ap.parse_args()


def max_over_ranks(x, pg, device):
    """The largest value of x over the ranks of the process group (x itself without one)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def check_interval(steps, k_max):
    """The largest divisor of steps that is at most k_max, so that `steps` steps are whole
    blocks of that many; where that divisor is small (a step count with no divisor near k_max),
    k_max itself, with a last, shorter block."""
    steps = max(int(steps), 1)
    top = max(1, min(k_max, steps))
    best = next(k for k in range(top, 0, -1) if steps % k == 0)
    return best if 4 * best >= top else top


def aggregate_mlups(nodes_per_rank, world, updates, seconds):
    """Whole-job lattice updates per second (millions): every rank's nodes, the slowest rank's
    time (weak scaling: each rank advances its own lattice)."""
    return nodes_per_rank * world * updates / seconds / 1e6


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


class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml of the installed NVIDIA driver): SM clock, its maximum,
    power draw and the active clock-event reasons of one GPU, named by UUID."""

    SM = 1  # NVML_CLOCK_SM
    # reason bits of nvmlDeviceGetCurrentClocksEventReasons
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
            "hw_thermal_slowdown": 0x40}

    def __init__(self, uuid):
        import ctypes
        self.c = ctypes
        L = ctypes.CDLL("libnvidia-ml.so.1")
        if L.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.L = L
        self.h = ctypes.c_void_p()
        if L.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle for " + uuid)
        fn = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn or L.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        c = self.c
        sm, mx, mw, rs = c.c_uint(), c.c_uint(), c.c_uint(), c.c_ulonglong()
        if self.L.nvmlDeviceGetClockInfo(self.h, self.SM, c.byref(sm)) != 0:
            return None
        self.L.nvmlDeviceGetMaxClockInfo(self.h, self.SM, c.byref(mx))
        self.L.nvmlDeviceGetPowerUsage(self.h, c.byref(mw))
        self.reasons_fn(self.h, c.byref(rs))
        return (float(sm.value), float(mx.value), mw.value / 1000.0,
                [n for n, b in self.BITS.items() if rs.value & b])


class ClockSampler:
    """SM clocks, power and throttle reasons sampled during the timed region: through NVML every
    2 ms (so that a region of a few milliseconds is sampled too), else nvidia-smi every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.nvml = None
        self.lines = []
        self.samples = []
        self.stop = threading.Event()

    def __enter__(self):
        try:
            self.nvml = _Nvml(self.uuid)
        except (OSError, AttributeError):
            self.nvml = None
        if self.nvml is not None:
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.uuid)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _poll(self):
        while True:
            x = self.nvml.sample()
            if x is not None:
                self.samples.append(x)
            if self.stop.wait(0.002):
                return

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        self.stop.set()
        if self.nvml is not None:
            self.t.join(timeout=5)
            x = self.nvml.sample()  # one sample at the end of the region
            if x is not None:
                self.samples.append(x)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for c, m, _, rs in self.samples:
            sm.append(c)
            mx.append(m)
            reasons.update(rs)
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(self.NAMES, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        src = "nvml" if self.nvml is not None else "nvidia-smi"
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "source": src}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": src}


def wkw(w):
    return dict(tau=w.tau, tau_c=w.tau_c, u_in=w.u_in, c_in=w.c_in, k_sink=w.k_sink)


# ---- oracle side (CPU) -----------------------------------------------------------------------

def _oracle_steps_per_s(w, parallel, seconds_target):
    """Fused FP64 oracle steps of the whole workload from rest, as many as fit about
    seconds_target (calibrated on one step): (steps, seconds)."""
    import oracle
    o = oracle.Oracle(w.shape, w.cls, parallel=parallel, **wkw(w))
    t0 = time.perf_counter()
    o.step_coupled(1)
    t1 = time.perf_counter() - t0
    n = max(1, int(seconds_target / max(t1, 1e-6)))
    t0 = time.perf_counter()
    o.step_coupled(n)
    dt = time.perf_counter() - t0
    del o
    return n, dt


def _lattice_name(w):
    kind = "anode" if w.dim == 2 else "electrode"
    sets = "D2Q9+D2Q5" if w.dim == 2 else "D3Q19+D3Q7"
    return kind, sets, "x".join(str(s) for s in w.shape)


def cpu_baseline(w, seconds_target=10.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload: fused steps of the
    whole lattice from rest, as many as fit about ten seconds, on all host cores (the OpenMP
    timing build, whose results are identical to the plain build's) and on one thread."""
    import oracle
    kind, sets, size = _lattice_name(w)
    cores = os.cpu_count() or 1
    out = {}
    n1, dt1 = _oracle_steps_per_s(w, False, seconds_target)
    one = {"value": w.nodes * n1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": f"{n1} fused {sets} steps of the full {size} {kind} from rest, FP64 C oracle, "
                     f"1 thread ({dt1:.1f} s)"}
    if oracle.lib_omp() is not None and cores > 1:
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
        n, dt = _oracle_steps_per_s(w, True, seconds_target)
        out = {"value": w.nodes * n / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{n} fused {sets} steps of the full {size} {kind} from rest, FP64 C "
                         f"oracle built with OpenMP over rows, {cores} threads ({dt:.1f} s); "
                         f"host nproc {cores}",
               "single_thread": one}
        return out
    return one


# The accuracy cases: (name, workload factory and arguments, steps or "steady").
ACC_CASES = [
    ("2d_256x128_1000_steps", ("anode_2d", (256, 128), {"seed": 2}), 1000),
    ("2d_64x32_steady", ("anode_2d", (64, 32), {"seed": 7}), "steady"),
    ("3d_48x32x32_200_steps", ("electrode_3d", (48, 32, 32), {"seed": 3}), 200),
    ("3d_16x16x24_steady", ("electrode_3d", (16, 16, 24), {"seed": 9}), "steady"),
]
ACC_K = 100
# FP16 storage's residual floor (mean change per step over K = 100 steps) is 1e-6 to 6e-6 on these
# lattices, against about 2e-9 in FP32: an FP16 steady solve stops at this tolerance instead
FP16_TOL = 1e-5


def _acc_workload(spec):
    import mfc_inputs as mi
    fn, shape, kw = spec
    return getattr(mi, fn)(*shape, **kw)


def oracle_case(case):
    """One accuracy reference on the FP64 oracle (run in a spawned process)."""
    import oracle
    name, spec, steps = case
    w = _acc_workload(spec)
    o = oracle.Oracle(w.shape, w.cls, **wkw(w))
    t0 = time.perf_counter()
    if steps == "steady":
        r = o.solve_steady(mode=oracle.CONCURRENT, tol_flow=w.tol, tol_ade=w.tol,
                           max_steps=w.max_steps, check_every=ACC_K)
        extra = {"steps": int(r.steps_flow), "current": float(r.current),
                 "converged": int(r.converged)}
    else:
        o.step_coupled(steps)
        extra = {"steps": steps}
    extra["oracle_s"] = time.perf_counter() - t0
    return name, {"f": o.f.copy(), "g": o.g.copy(), "u": o.u.copy(), "c": o.conc.copy(), **extra}


def start_oracle_pool():
    """Spawned worker processes (started before the first GPU call) computing the references."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    oracle.build()  # once, before the workers import it
    ex = cf.ProcessPoolExecutor(max_workers=len(ACC_CASES), mp_context=mp.get_context("spawn"))
    return ex, [ex.submit(oracle_case, c) for c in ACC_CASES]


def reference_workload(args):
    import mfc_inputs as mi
    if args.workload == "electrode3d":
        return mi.electrode_3d()
    return mi.anode_2d(args.nx, args.ny)


def run_reference(args, rank, world):
    """The oracle as the reference arm: every step is one fused FP64 update of a slab of the
    workload (the middle rows of the 2-D anode, the middle planes across the flow axis of the 3-D
    electrode), sized so that the whole run ends within a few minutes, on all host cores (the
    OpenMP timing build; one thread where it cannot be built)."""
    if rank != 0:
        return
    import oracle
    w = reference_workload(args)
    parallel = oracle.lib_omp() is not None and (os.cpu_count() or 1) > 1
    cores = (os.cpu_count() or 1) if parallel else 1
    if parallel:
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    total = args.steps + args.warmup
    budget = 150.0 / max(total, 1)
    # the slab: rows (2-D) or planes (3-D) across the flow axis, taken from the middle of the
    # porous block
    layers_all = w.shape[1] if w.dim == 2 else w.shape[2]
    per_layer_nodes = w.nodes // layers_all

    def slab(r):
        if w.dim == 2:
            y0 = w.shape[1] // 2 - r // 2
            cls = w.cls.reshape(w.shape[1], w.shape[0])[y0:y0 + r].reshape(-1)
            shape = (w.shape[0], r)
        else:
            z0 = w.shape[2] // 2 - r // 2
            cls = w.cls.reshape(w.shape[2], w.shape[1] * w.shape[0])[z0:z0 + r].reshape(-1)
            shape = (w.shape[0], w.shape[1], r)
        return oracle.Oracle(shape, cls, parallel=parallel, **wkw(w)), shape

    rows = min(16, layers_all)  # calibrate on a 16-layer slab
    o, _ = slab(rows)
    t0 = time.perf_counter()
    o.step_coupled(2)
    per_row = (time.perf_counter() - t0) / (2 * rows)
    rows = int(max(1, min(layers_all, budget / max(per_row, 1e-9))))
    o, shape = slab(rows)
    o.step_coupled(args.warmup)
    t0 = time.perf_counter()
    o.step_coupled(args.steps)
    dt = time.perf_counter() - t0
    nodes = per_layer_nodes * rows
    value = nodes * args.steps / dt / 1e6
    kind, sets, size = _lattice_name(w)
    sample = (f"each step one fused FP64 {sets} update of a {'x'.join(map(str, shape))} slab of "
              f"the {size} {kind} (middle {'rows' if w.dim == 2 else 'planes'}), "
              f"{cores} thread{'s' if cores > 1 else ''}"
              f"{' (OpenMP timing build)' if parallel else ''}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "nodes": w.nodes,
                       "sample_nodes": nodes},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    if not rec or "translation_unit" not in rec or \
            rec.get("kernel_digest") != build.kernel_digest(rec["translation_unit"]):
        return None
    return rec.get("dram_bytes_per_launch_full")


# ---- GPU legs --------------------------------------------------------------------------------

def time_plain_steps(P, lat, stream, M=400):
    """Average duration of the plain fused step kernel, in ms, two ways, each bracketed by CUDA
    events on the lattice stream: (1) launched as mfc_solve_steady launches it, one CUDA graph of
    M steps (M - 1 plain steps and one check step, then the two sum kernels), the block's time
    over M: an upper bound on the plain launch's duration, since the rest takes longer than a
    plain step; (2) M direct launches (mfc_step_coupled), which adds each launch's gap."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    solve = dict(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0, max_steps=M, check_every=M)
    lat.solve_steady(**solve)  # captures the graph
    e0.record(stream)
    lat.solve_steady(**solve)
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / M
    lat.step_coupled(20)
    e0.record(stream)
    lat.step_coupled(M)
    e1.record(stream)
    torch.cuda.synchronize()
    return graph_ms, e0.elapsed_time(e1) / M


def step_bytes(dim, prec_bytes, flow_open, ade_open, ade_q=0):
    """Algorithmic bytes of one fused step: every population of every open node read once and
    written once."""
    qf, qa = (9, 5) if dim == 2 else (19, 7)
    if ade_q:
        qa = ade_q
    return 2 * prec_bytes * (qf * flow_open + qa * ade_open)


def leg_variants(P, peak):
    """The 2048x1024 anode in FP32, the FP16-storage 2-D step, the D2Q9 transport, the
    saturating consumption of Eq. 16 and the 3-D electrode in FP32 and FP16: MLUPS over graph
    blocks and the plain kernel's fraction of the HBM roofline."""
    import torch
    import mfc_inputs as mi
    out = {}
    # the FP16 2-D case runs on 4096x1024: its 2048x1024 working set (118 MB) would fit the L2
    cases = [("2d_2048x1024_fp32", mi.anode_2d(), P.MFC_FP32, 10000),
             ("2d_4096x1024_fp16", mi.anode_2d(4096, 1024), P.MFC_FP16_DEV, 10000),
             ("2d_2048x1024_d2q9_transport_fp32", mi.anode_2d(), P.MFC_FP32, 10000),
             # K_s = 0.05: the paper's K_s / C_in = 20 / 410 with C_in = 1
             ("2d_2048x1024_monod_consumption_fp32", mi.anode_2d(), P.MFC_FP32, 10000),
             ("3d_256x128x128_fp32", mi.electrode_3d(), P.MFC_FP32, 5000),
             ("3d_256x128x128_fp16", mi.electrode_3d(), P.MFC_FP16_DEV, 5000)]
    for name, w, prec, steps in cases:
        stream = torch.cuda.Stream()
        aq = 9 if "d2q9" in name else 0
        kw = dict(wkw(w), k_half=0.05) if "monod" in name else wkw(w)
        lat = P.Lattice(w.shape, precision=prec, stream=stream.cuda_stream, ade_q=aq, **kw)
        lat.set_geometry(w.cls)
        fo, ao = lat.active_nodes()
        lat.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0, max_steps=1000,
                         check_every=200)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0, max_steps=steps,
                         check_every=200)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kern_ms, kern_direct_ms = time_plain_steps(P, lat, stream)
        # the same kernel with 64-bit element offsets, for comparison
        lat.set_launch(block=lat.get_launch()["block"], offsets32=0)
        kern64_ms, _ = time_plain_steps(P, lat, stream)
        lat.set_launch(block=lat.get_launch()["block"], offsets32=1)
        sb = 2 if prec == P.MFC_FP16_DEV else 4
        byt = step_bytes(w.dim, sb, fo, ao, aq)
        ach = byt / (kern_ms * 1e-3) / 1e9
        out[name] = {"mlups": w.nodes * steps / (ms * 1e-3) / 1e6, "steps": steps,
                     "kernel_ms": kern_ms, "kernel_ms_direct": kern_direct_ms,
                     "kernel_ms_offsets64": kern64_ms,
                     "algorithmic_bytes_per_launch": byt,
                     "achieved_gbs": ach, "roofline_frac": ach / peak,
                     "bytes_per_node": byt / w.nodes}
        lat.close()
    return out


def gpu_case(P, case, prec):
    name, spec, steps = case
    w = _acc_workload(spec)
    g = P.Lattice(w.shape, precision=prec, **wkw(w))
    g.set_geometry(w.cls)
    res = {}
    if steps == "steady":
        tol = max(w.tol, FP16_TOL) if prec == P.MFC_FP16_DEV else w.tol
        r = g.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=tol, tol_ade=tol,
                           max_steps=w.max_steps, check_every=ACC_K)
        res.update(steps=int(r.steps_flow), current=float(r.current), status=int(r.status), tol=tol)
    else:
        g.step_coupled(steps)
    _, u, c, _ = g.read_fields()
    res.update(f=g.read_populations(P.MFC_POP_FLOW), g=g.read_populations(P.MFC_POP_ADE), u=u, c=c)
    g.close()
    return res


def leg_accuracy(P, futures):
    """FP32 and FP16 results against the FP64 oracle references."""
    import numpy as np

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    refs = dict(f.result() for f in futures)
    out = {}
    for prec_name, prec in (("fp32", P.MFC_FP32), ("fp16", P.MFC_FP16_DEV)):
        d = {}
        for case in ACC_CASES:
            name, _, steps = case
            ref = refs[name]
            got = gpu_case(P, case, prec)
            e = {"u_rel_l2": rel(got["u"], ref["u"]), "c_rel_l2": rel(got["c"], ref["c"])}
            if steps == "steady":
                e.update(current_rel=abs(got["current"] - ref["current"]) / abs(ref["current"]),
                         steps=got["steps"], oracle_steps=ref["steps"], status=got["status"],
                         tol=got["tol"])
            else:
                e.update(pop_flow_maxabs=float(np.abs(got["f"] - ref["f"]).max()),
                         pop_ade_maxabs=float(np.abs(got["g"] - ref["g"]).max()), steps=steps)
            d[name] = e
        out[prec_name] = d
    out["oracle_seconds"] = {k: v["oracle_s"] for k, v in refs.items()}
    out["check_every"] = ACC_K
    return out


def leg_batch(P, count, max_steps=0):
    """The uneven batch (64 instances of 256..1024 x 128..512, porosity, tau and inlet speed
    drawn per instance) solved to 1e-7 by the batch engine, then the same solves one at a time
    with the same K; wall-clock solves/s of both and the agreement of their results."""
    import numpy as np
    import mfc_inputs as mi
    works = mi.batch_instances(count)
    b = P.Batch()
    t0 = time.perf_counter()
    tickets = [b.submit(w.shape, w.cls, tol_flow=w.tol, tol_ade=w.tol,
                        max_steps=max_steps or w.max_steps, **wkw(w)) for w in works]
    b.run()
    tb = time.perf_counter() - t0
    rb = [b.poll(t) for t in tickets]
    st = b.stats()
    b.close()
    K = st["check_every"]
    t0 = time.perf_counter()
    rs = []
    for w in works:
        g = P.Lattice(w.shape, **wkw(w))
        g.set_geometry(w.cls)
        r = g.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=w.tol, tol_ade=w.tol,
                           max_steps=max_steps or w.max_steps, check_every=K)
        _, u, c, _ = g.read_fields()
        rs.append((r, u, c))
        g.close()
    ts = time.perf_counter() - t0
    # field agreement over the solves that ended with finite fields in both arms
    bad = (P.MFC_ERR_NONFINITE, P.MFC_ERR_UNSTABLE)
    fin = [(x, y) for x, y in zip(rb, rs) if x["status"] not in bad and y[0].status not in bad]
    du = max(float(np.linalg.norm(x["u"] - u) / np.linalg.norm(u)) for x, (_, u, _) in fin)
    dc = max(float(np.linalg.norm(x["c"] - c) / np.linalg.norm(c)) for x, (_, _, c) in fin)
    upd = sum(x["steps_flow"] * w.nodes for x, w in zip(rb, works))
    return {"instances": count, "nodes": int(sum(w.nodes for w in works)), "tol": works[0].tol,
            "batched_s": tb, "batched_solves_per_s": count / tb,
            "one_at_a_time_s": ts, "one_at_a_time_solves_per_s": count / ts,
            "speedup": ts / tb, "check_every": K, "block": st["block"], "grid": st["grid"],
            "converged": sum(x["status"] == P.MFC_OK for x in rb),
            "at_cap": sum(x["status"] == P.MFC_NOT_CONVERGED for x in rb),
            "nonfinite": sum(x["status"] == P.MFC_ERR_NONFINITE for x in rb),
            "unstable": [{"instance": i, "shape": list(w.shape), "tau": w.tau, "u_in": w.u_in,
                          "steps": int(x["steps_flow"]), "alone_steps": int(r.steps_flow)}
                         for i, (x, w, (r, _, _)) in enumerate(zip(rb, works, rs))
                         if x["status"] == P.MFC_ERR_UNSTABLE],
            "same_status": sum(x["status"] == r.status for x, (r, _, _) in zip(rb, rs)),
            "same_stop_step": sum(x["steps_flow"] == r.steps_flow for x, (r, _, _) in zip(rb, rs)),
            "max_rel_l2_u_batch_vs_alone": du, "max_rel_l2_c_batch_vs_alone": dc,
            "batched_mlups": upd / tb / 1e6, "mean_steps": upd / sum(w.nodes for w in works)}


def serve_phase(P, reqs, works, rate_scale):
    """Submit each request at its arrival time (scaled) to the batch engine's thread; return
    per-request latency (submission to result) and the achieved solves/s."""
    b = P.Batch(budget_bytes=150 * 10 ** 9)
    b.start()
    t0 = P.clock()
    tickets = []
    for r, w in zip(reqs, works):
        delay = t0 + r.arrival_s * rate_scale - P.clock()
        if delay > 0:
            time.sleep(delay)
        tickets.append(b.submit(w.shape, w.cls, tol_flow=w.tol, tol_ade=w.tol,
                                max_steps=w.max_steps, **wkw(w)))
    res = [b.wait(t, timeout_s=3600.0) for t in tickets]
    b.stop()
    st = b.stats()
    b.close()
    def pct(v, q):
        return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))] if v else None

    lat = sorted(x["t_done"] - x["t_submit"] for x in res)
    conv = sorted(x["t_done"] - x["t_submit"] for x in res if x["status"] == P.MFC_OK)
    sc = sorted(x["steps_flow"] for x in res if x["status"] == P.MFC_OK)
    span = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
    first, last = min(x["t_submit"] for x in res), max(x["t_submit"] for x in res)
    return {"requests": len(res), "solves_per_s": len(res) / span, "span_s": span,
            "offered_per_s": (len(res) - 1) / max(last - first, 1e-9),
            "converged": len(conv),
            "at_cap": sum(x["status"] == P.MFC_NOT_CONVERGED for x in res),
            "other_status": sum(x["status"] not in (P.MFC_OK, P.MFC_NOT_CONVERGED) for x in res),
            # time to converged solution: submission to result, over the converged requests
            "p50_converged_s": pct(conv, 0.5), "p99_converged_s": pct(conv, 0.99),
            "p50_all_s": pct(lat, 0.5), "p99_all_s": pct(lat, 0.99), "max_s": lat[-1],
            "mean_steps": statistics.mean(x["steps_flow"] for x in res),
            "steps_converged_p50_p99_max": ([pct(sc, 0.5), pct(sc, 0.99), sc[-1]] if sc else None),
            # the requests that did not converge: shape and steps
            "not_converged": [[list(w.shape), x["steps_flow"], x["status"]]
                              for w, x in zip(works, res) if x["status"] != P.MFC_OK],
            "check_every": st["check_every"], "block": st["block"],
            "peak_bytes": st["bytes_peak"]}


def leg_serve(P, count):
    """Serving: Poisson arrivals of 2-D (512..2048 x 256..1024) and 3-D (64^3..192x96x96)
    steady-solve requests (tol 1e-7, cap 1e6 steps), 150 GB admission budget.  Phase 1 offers
    the stream at 200/s (capacity); phase 2 offers a second stream at 0.8x that capacity.
    Latencies are time to converged solution (submission to result, converged requests), with
    the requests that ended otherwise counted beside them."""
    import mfc_inputs as mi
    reqs1 = mi.serving_stream(count, 200.0, seed=5)
    works1 = [r.workload() for r in reqs1]
    p1 = serve_phase(P, reqs1, works1, 1.0)
    rate2 = 0.8 * p1["solves_per_s"]
    reqs2 = mi.serving_stream(count, 200.0, seed=6)
    works2 = [r.workload() for r in reqs2]
    p2 = serve_phase(P, reqs2, works2, 200.0 / rate2)
    return {"offered_200_per_s": p1, "offered_0.8x_capacity": p2,
            "mix": "70% 2-D, 30% 3-D by request", "requests_per_phase": count}


def leg_biofilm(P, cycles):
    """The biofilm-cycle workload: steady solve, growth, warm restart, `cycles` times, with the
    saturating consumption of Eq. 16 (K_s = 0.05, the paper's 20 mg/L against C_in = 410 mg/L).
    After each solve the anode's electrical model advances one model hour (Eqs. 14-21,
    mfc_electro_update) from the mean substrate factor over the biofilm, current / (k K_s n),
    and the mean biomass concentration 450 mg/L x (biofilm nodes / nodes); the cycle records the
    cell current and voltage."""
    import torch
    import mfc_inputs as mi
    w = mi.anode_2d()
    ks = 0.05
    stream = torch.cuda.Stream()
    lat = P.Lattice(w.shape, stream=stream.cuda_stream, k_half=ks, **wkw(w))
    lat.set_geometry(w.cls)
    n_sink = int(((w.cls & 4) != 0).sum())
    ep = P.electro_params()
    m_ox = 0.5 * ep.m_total
    per = []
    t0 = time.perf_counter()
    steps = 0
    for cyc in range(cycles):
        r = lat.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=w.tol, tol_ade=w.tol,
                             max_steps=w.max_steps, check_every=200)
        s_bar = min(1.0, max(0.0, r.current / (w.k_sink * ks * n_sink)))
        el = P.electro_update(ep, s_bar, 450.0 * n_sink / w.nodes, m_ox)
        m_ox = min(el["m_ox"], ep.m_total * (1 - 1e-9))
        n = lat.biofilm_grow(seed=2, cycle=cyc, prob=0.05, c_thresh=0.5)
        n_sink += n
        steps += r.steps_flow
        per.append({"steps": int(r.steps_flow), "status": int(r.status), "current": r.current,
                    "res_flow": r.res_flow, "res_ade": r.res_ade, "converted": n,
                    "substrate_factor": s_bar, "i_cell_mA": el["i_cell"] * 1e3,
                    "v_cell_mV": el["v_cell"] * 1e3, "m_ox": el["m_ox"]})
    dt = time.perf_counter() - t0
    lat.close()
    return {"cycles": cycles, "seconds": dt, "steps": steps,
            "mlups": w.nodes * steps / dt / 1e6,
            "converged": sum(c["status"] == P.MFC_OK for c in per),
            "converted_total": sum(c["converted"] for c in per),
            "current_first": per[0]["current"], "current_last": per[-1]["current"],
            "i_cell_mA_last": per[-1]["i_cell_mA"], "v_cell_mV_last": per[-1]["v_cell_mV"],
            "per_cycle": per}


def leg_model(P, hours):
    """The paper's model loop (Sec. 3, Sec. 4: one iteration per hour) on the 2048x1024 anode
    with its electrode only: each hour the flow and the transport are solved to steady state
    (1e-7, saturating consumption with K_s = 0.05), the electrical model advances one hour from the
    mean substrate factor over the biofilm, and the agent-based biofilm (Table 1's k_ata, C_0^bio,
    C_max^bio and fr_spr, growth 0.1 per hour) attaches, grows and spreads; the lattice warm-starts
    from the previous hour."""
    import numpy as np
    import torch
    import mfc_inputs as mi
    w = mi.anode_2d()
    cls = np.where((w.cls & 3) == 3, 3, 0).astype(np.uint8)
    ks = 0.05
    stream = torch.cuda.Stream()
    lat = P.Lattice(w.shape, stream=stream.cuda_stream, k_half=ks, **wkw(w))
    lat.set_geometry(cls)
    ep = P.electro_params()
    ap = P.agent_params(seed=7, growth=0.1, k_half=ks)
    m_ox = 0.5 * ep.m_total
    n_bio, total = 0, 0.0
    per = []
    t0 = time.perf_counter()
    steps = 0
    for hour in range(hours):
        r = lat.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=w.tol, tol_ade=w.tol,
                             max_steps=w.max_steps, check_every=200)
        steps += r.steps_flow
        s_bar = min(1.0, max(0.0, r.current / (w.k_sink * ks * n_bio))) if n_bio else 0.0
        c_bio = max(total / w.nodes, 1e-9)  # mean biomass concentration over the compartment
        el = P.electro_update(ep, s_bar, c_bio, m_ox)
        m_ox = min(el["m_ox"], ep.m_total * (1 - 1e-9))
        ag = lat.agent_step(ap, hour)
        n_bio, total = ag["biofilm_nodes"], ag["total_biomass"]
        per.append({"hour": hour + 1, "steps": int(r.steps_flow), "status": int(r.status),
                    "lattice_current": r.current, "substrate_factor": s_bar,
                    "i_cell_mA": el["i_cell"] * 1e3, "v_cell_mV": el["v_cell"] * 1e3,
                    "m_ox": el["m_ox"], "attached": ag["attached"], "spread": ag["spread"],
                    "biofilm_nodes": n_bio, "total_biomass": total})
    dt = time.perf_counter() - t0
    lat.close()
    return {"hours": hours, "seconds": dt, "steps": steps, "mlups": w.nodes * steps / dt / 1e6,
            "converged": sum(h["status"] == P.MFC_OK for h in per),
            "biofilm_nodes_last": per[-1]["biofilm_nodes"], "i_cell_mA_last": per[-1]["i_cell_mA"],
            "v_cell_mV_last": per[-1]["v_cell_mV"], "per_hour": per}


def main():
    args = parse()
    rank, world, local = dist_env()
    legs = set(args.legs.split(","))
    if world > 1:
        # one GPU per rank: the library and torch both see it as device 0
        os.environ["CUDA_VISIBLE_DEVICES"] = str(local)
        legs &= {"main"}
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    pool = futures = None
    if "accuracy" in legs and rank == 0:
        pool, futures = start_oracle_pool()  # before the first GPU call

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

    if args.workload == "electrode3d":
        w = mi.electrode_3d(seed=3 + rank)
    else:
        w = mi.anode_2d(args.nx, args.ny, seed=2 + rank)
    prec = P.MFC_FP16_DEV if args.precision == "fp16" else P.MFC_FP32
    stream = torch.cuda.Stream()
    lat = P.Lattice(w.shape, precision=prec, stream=stream.cuda_stream, **wkw(w))
    lat.set_geometry(w.cls)
    flow_open, ade_open = lat.active_nodes()
    # K: the largest divisor of the timed steps not above --check-every, so that the timed
    # region is whole graph replays of K steps and their checks, as a steady solve runs them
    K = check_interval(args.steps, args.check_every)

    def run(nsteps, k=K):
        r = lat.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0,
                             max_steps=nsteps, check_every=k)
        assert r.status == P.MFC_NOT_CONVERGED, P.status_string(r.status)
        return r

    # warm-up: at least W steps, rounded up to whole blocks (two for an odd K, whose graph
    # alternates between the two buffer parities), so every graph the timed region replays is
    # captured and instantiated before it starts
    blk = K if K % 2 == 0 else 2 * K
    warm = max(args.warmup, 3)
    warm = (warm + blk - 1) // blk * blk
    run(warm)
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
    ms = max_over_ranks(ev0.elapsed_time(ev1), pg, "cuda")
    value = aggregate_mlups(w.nodes, world, args.steps, ms * 1e-3)

    # dominant kernel: the plain fused step, timed alone on the same stream
    kern_ms, kern_direct_ms = time_plain_steps(P, lat, stream)
    # the same kernel inside the timed region: its share of the step (the rest is the check
    # step, the two sum kernels and the host round trip of each block)
    sb = 2 if prec == P.MFC_FP16_DEV else 4
    qf, qa = (9, 5) if w.dim == 2 else (19, 7)
    working_set = 2 * sb * (qf + qa) * w.nodes
    bytes_per_launch = step_bytes(w.dim, sb, flow_open, ade_open)
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_launch / (kern_ms * 1e-3) / 1e9
    # FP16 storage steps two rows per thread with paired FP32 arithmetic (lbm_pair_kernel)
    kname = ("lbm_pair_kernel<%d,half,0>" % w.dim if sb == 2 else
             "lbm_step_kernel<%d,float,true,true,0>" % w.dim)
    traffic = traffic_record(kname)

    # end to end through the public API with host buffers: upload classes from pinned memory,
    # one solve block of e2e_steps updates, read rho, u, C and the current back to pinned memory
    n_e2e = 3
    cls_h = torch.from_numpy(w.cls).pin_memory()
    rho_h = torch.empty(w.nodes, dtype=torch.float64).pin_memory()
    u_h = torch.empty(w.dim * w.nodes, dtype=torch.float64).pin_memory()
    c_h = torch.empty(w.nodes, dtype=torch.float64).pin_memory()
    cur_h = torch.empty(1, dtype=torch.float64).pin_memory()
    import ctypes
    L = P.lib()
    dp = ctypes.POINTER(ctypes.c_double)

    K_e2e = check_interval(args.e2e_steps, args.check_every)

    def e2e_step():
        st = L.mfc_set_geometry(lat.handle, ctypes.cast(cls_h.data_ptr(),
                                                        ctypes.POINTER(ctypes.c_uint8)), 1)
        assert st == 0
        r = lat.solve_steady(mode=P.MFC_CONCURRENT, tol_flow=0.0, tol_ade=0.0,
                             max_steps=args.e2e_steps, check_every=K_e2e)
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
    e2e_s = max_over_ranks(time.perf_counter() - t0, pg, "cuda")
    e2e_value = aggregate_mlups(w.nodes, world, args.e2e_steps * n_e2e, e2e_s)
    assert np.isfinite(c_h.numpy()).all()
    lat.close()

    extra = {}
    leg_s = {}
    if rank == 0 and world == 1:
        for name, fn in (("variants", lambda: leg_variants(P, peak)),
                         ("accuracy", lambda: leg_accuracy(P, futures)),
                         ("batch", lambda: leg_batch(P, args.batch_count, args.batch_max_steps)),
                         ("serve", lambda: leg_serve(P, args.serve_count)),
                         ("biofilm", lambda: leg_biofilm(P, args.biofilm_cycles)),
                         ("model", lambda: leg_model(P, args.model_hours))):
            if name in legs:
                t0 = time.perf_counter()
                extra[name] = fn()
                leg_s[name] = time.perf_counter() - t0
    if pool:
        pool.shutdown()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if rank == 0:
        nblocks = (args.steps + K - 1) // K
        # per block: K step kernels and the two sum kernels
        launches = args.steps + 2 * nblocks
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if sb == 4 else "f16-storage/f32-math", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "shape": list(w.shape),
                       "nodes_per_gpu": w.nodes, "flow_open": flow_open, "ade_open": ade_open,
                       "check_every": K, "warmup_steps_run": warm,
                       "parallelism": f"replicas{world}",
                       "l2": f"populations {working_set / 1e6:.0f} MB (both buffers) "
                             f"{'>' if working_set > 129e6 else '<='} 129 MB L2"
                             f"{', no flush' if working_set > 129e6 else ' (L2-resident: not a valid HBM number)'}",
                       "mflups_flow_open": flow_open * world * args.steps / (ms * 1e-3) / 1e6},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "kernel": kname, "kernel_ms": kern_ms,
                         "kernel_ms_timing": "mean step of a 400-step CUDA graph as mfc_solve_steady "
                                             "runs it (399 plain steps, 1 check step, 2 sum kernels): "
                                             "an upper bound on the plain launch",
                         "kernel_ms_direct": kern_direct_ms,
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": int(w.nodes),
                    "d2h_bytes_per_step": int(w.nodes * 8 * (2 + w.dim) + 8),
                    "updates_per_step": args.e2e_steps, "check_every": K_e2e,
                    "path": "mfc_set_geometry (pinned host classes) + mfc_solve_steady + "
                            "mfc_read_fields (rho, u, C, current into pinned host buffers)"},
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "final": {"res_flow": res.res_flow, "res_ade": res.res_ade, "current": res.current},
        }
        if "serve" in extra:
            s = extra["serve"]
            p2 = s["offered_0.8x_capacity"]
            line["serving"] = {"solves_per_s": s["offered_200_per_s"]["solves_per_s"],
                               "p50_s": p2["p50_converged_s"], "p99_s": p2["p99_converged_s"],
                               "converged": p2["converged"], "requests": p2["requests"],
                               **extra.pop("serve")}
        line.update(extra)
        if leg_s:
            line["leg_seconds"] = leg_s
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
