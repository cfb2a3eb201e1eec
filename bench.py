#!/usr/bin/env python3
"""Benchmark of the lattice step: MLUPS and HBM-roofline fraction on GB300.

A step is one full pass of the coupled update (chemical potentials, collide-
stream with particle bounce-back, psi/phi transport, particle update,
covering).  The default workload is the 256^3 eight-sphere box (spheres R=6
at seeded positions in the slab 20 < z < 60 below a flat interface at
z=128, tanh width 2, contact angle 90 degrees, phoretic mobility 0.1, cap
production 1e-3), FP32 arithmetic and storage; ``--precision fp16``/``bf16``
stores the populations as 16-bit deviations, ``--workload interface`` runs
the 128^3 single-sphere interface box instead.  Inputs are synthetic and
seeded; the state (several GB) is larger than L2, so no L2 flush is needed.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle (the
reference implementation written from the paper) on the host cores instead.
Multi-GPU runs (torchrun) are independent replicas: the boxes do not share
data, so there is no collective on the data path.

``--form batched`` times 64 uneven boxes (edges 32..96, one sphere each)
advanced together through the batched kernels and CUDA graphs after
autotuning, against the same boxes run one by one with the single-box path;
``--form served`` replays a seeded Poisson request stream through the
continuous-batching server and reports p50/p99 time-to-result and sims/hour,
against a one-by-one FIFO server.  The default form is the single box.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# algorithmic bytes per node and step (populations read+write, psi/phi
# read+write): FP32 19*4*2 + 2*4*2
ALG_BYTES_STEP = {"fp64": 336, "fp32": 168, "fp16": 92, "bf16": 92}
# algorithmic bytes per node of the fused kernel (chemical potentials, force,
# collide-stream): the part of the step's algorithmic bytes it carries, the
# populations read and written and psi, phi read
ALG_BYTES_FUSED = {"fp64": 19 * 8 * 2 + 16, "fp32": 19 * 4 * 2 + 8, "fp16": 19 * 2 * 2 + 8,
                   "bf16": 19 * 2 * 2 + 8}
# bytes per node the transport kernel moves by design (not algorithmic: mu and
# u are intermediates of the step): psi, phi, mu_psi, mu_phi, u read, psi, phi
# written
DESIGN_BYTES_SCALARS = {"fp64": 9 * 8, "fp32": 9 * 4, "fp16": 9 * 4, "bf16": 9 * 4}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f16-storage/f32", "bf16": "bf16-storage/f32"}
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--workload", default="precision", choices=["precision", "interface"],
                    help="precision: 256^3, 8 spheres R=6 below an interface; interface: 128^3, one "
                         "sphere R=8 straddling it")
    ap.add_argument("--edge", type=int, default=0, help="box edge (default 256 / 128 by workload)")
    ap.add_argument("--scalar-scheme", type=int, default=0, choices=[0, 1],
                    help="psi/phi transport: 0 finite differences, 1 D3Q7 lattice Boltzmann")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="single form: keep the size heuristic's z chunks")
    ap.add_argument("--form", default="single", choices=["single", "batched", "served"])
    ap.add_argument("--boxes", type=int, default=64, help="batched form: number of boxes")
    ap.add_argument("--graph-steps", type=int, default=16,
                    help="batched form: steps per captured CUDA graph (more than --steps: plain launches)")
    ap.add_argument("--requests", type=int, default=32, help="served form: number of requests")
    ap.add_argument("--rate", type=float, default=20.0, help="served form: mean arrivals per second")
    return ap.parse_args()


# physical settings of each bench workload (reported in the JSON config)
WORKLOAD_SETTINGS = {
    "precision": {"theta_c_deg": 90.0, "solubility_ratio": 1.0, "mobility": 0.1, "spheres": "8 x R=6",
                  "default_edge": 256},
    "interface": {"theta_c_deg": 60.0, "solubility_ratio": 2.0, "mobility": 0.1, "spheres": "1 x R=8",
                  "default_edge": 128},
}


def edge_of(args):
    return args.edge if args.edge > 0 else WORKLOAD_SETTINGS[args.workload]["default_edge"]


def workload(kind, edge, scalar_scheme=0):
    from paper_2202_01631_gb300 import workloads as W
    if kind == "precision":
        wl = W.precision(seed=0, edge=edge)
    else:
        wl = W.interface(theta_c_deg=60.0, solubility_ratio=2.0, mobility=0.1, seed=0, edge=edge)
    if scalar_scheme:
        wl.params = dict(wl.params, scalar_scheme=scalar_scheme)
    return wl


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    group = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        group = dist
    return world, rank, local, group


def barrier(group):
    if group is not None:
        import torch
        if torch.cuda.is_available():
            group.barrier(device_ids=[torch.cuda.current_device()])
        else:
            group.barrier()


def max_over_ranks(value, group):
    """Largest value over ranks (the job time is the slowest rank's)."""
    if group is None:
        return value
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    group.all_reduce(t, op=group.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled during a region.

    Polls NVML through ctypes every 2 ms (the timed region of a short run
    lasts tens of milliseconds); falls back to ``nvidia-smi -lms 20`` where
    the NVML library cannot be loaded.  Reading clocks changes nothing.
    """

    # NVML clock-event reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_s=0.002):
        self.index = self._nvml_index(index)
        self.period = period_s
        self.samples = []          # (sm_mhz, reason bits)
        self.max_mhz = None
        self.source = None
        self.proc = None
        self.lines = []
        self._stop = threading.Event()
        self._nvml = None

    @staticmethod
    def _nvml_index(local):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if ids and local < len(ids) and ids[local].isdigit():
            return int(ids[local])
        return local

    def _open_nvml(self):
        import ctypes
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                lib = None
        if lib is None or lib.nvmlInit_v2() != 0:
            return False
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
            return False
        mx = ctypes.c_uint(0)
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:   # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
        self._nvml = (ctypes, lib, h, reasons)
        return True

    def _poll(self):
        ctypes, lib, h, reasons = self._nvml
        clk = ctypes.c_uint(0)
        bits = ctypes.c_ulonglong(0)
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                r = 0
                if reasons is not None and reasons(h, ctypes.byref(bits)) == 0:
                    r = bits.value
                self.samples.append((float(clk.value), r))
            time.sleep(self.period)

    def __enter__(self):
        try:
            ok = self._open_nvml()
        except (OSError, AttributeError):
            ok = False
        if ok:
            self.source = "nvml %.0f ms" % (self.period * 1e3)
            self.t = threading.Thread(target=self._poll, daemon=True)
            self.t.start()
            time.sleep(3 * self.period)   # first samples before the region starts
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi 20 ms"
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        self._stop.set()
        if self._nvml is not None:
            self.t.join(timeout=1.0)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, reasons = [], set()
        mx = self.max_mhz
        if self._nvml is not None:
            for mhz, bits in self.samples:
                sm.append(mhz)
                for b, nm in self.REASONS.items():
                    if bits & b:
                        reasons.add(nm)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0, "source": self.source}
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm), "source": self.source}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def traffic_record(kernel, precision, workload_name):
    """DRAM bytes per launch of a kernel from the committed ncu summary, valid
    only while the kernel sources are unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            recs = json.load(f)
    except (OSError, ValueError):
        return None
    src = source_hash()
    for r in recs:
        if (r.get("kernel") == kernel and r.get("precision") == precision and r.get("workload") == workload_name
                and r.get("source_sha") == src):
            return float(r["bytes_per_launch"])
    return None


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2202_01631_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def build_box(wl, precision, stream):
    from paper_2202_01631_gb300.lbdp import Box
    box = Box(precision=precision, stream=stream, **wl.params)
    box.set_fields(**wl.fields)
    for p in wl.particles:
        box.add_particle(**p)
    return box


def _oracle_for(wl):
    from oracle.lbref import Oracle
    ref = Oracle(wl.params)
    ref.set_fields(**wl.fields)
    for p in wl.particles:
        ref.add_particle(**p)
    return ref


def _time_oracle(ref, budget_s, max_steps=20):
    """One untimed step, then as many steps as fit in budget_s (at least one,
    at most max_steps); returns (steps, seconds)."""
    t0 = time.perf_counter()
    ref.step(1)
    per = time.perf_counter() - t0
    k = max(1, min(max_steps, int(budget_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    ref.step(k)
    return k, time.perf_counter() - t0


def cpu_baseline(wl, budget_s=10.0):
    """The FP64 oracle as it stands on the host cores, on a bounded number of
    steps of the same workload: all cores (the reported figure) and one
    thread (alongside)."""
    from oracle import lbref
    ref = _oracle_for(wl)
    cores = lbref.set_threads(0)
    k, dt = _time_oracle(ref, budget_s)
    lbref.set_threads(1)
    k1, dt1 = _time_oracle(ref, budget_s)
    lbref.set_threads(0)
    edge = "%dx%dx%d" % (wl.params["nx"], wl.params["ny"], wl.params["nz"])
    return {"value": wl.nodes * k / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": "%d steps of the %s workload (after 1 untimed step), FP64, %d threads"
                      % (k, edge, cores),
            "single_thread": {"value": wl.nodes * k1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                              "sample": "%d steps of the same box (after 1 untimed step), FP64, 1 thread"
                                        % k1}}


def run_reference(args):
    """The FP64 oracle written from the paper (the paper ships no code) on the
    host cores, on the same workload as our arm: W warm-up steps (at most
    one) and K timed steps, bounded so that the run ends within about three
    minutes (the sample is stated in the line)."""
    world, rank, local, group = dist_setup(args)
    if rank != 0:
        return 0
    from oracle import lbref
    wl = workload(args.workload, edge_of(args))
    ref = _oracle_for(wl)
    cores = lbref.set_threads(0)
    t0 = time.perf_counter()
    ref.step(1 if args.warmup > 0 else 0)
    per = max(time.perf_counter() - t0, 1e-6) if args.warmup > 0 else None
    if per is None:
        t0 = time.perf_counter()
        ref.step(1)
        per = max(time.perf_counter() - t0, 1e-6)
    k = max(1, min(args.steps, int(150.0 / per)))
    t0 = time.perf_counter()
    ref.step(k)
    dt = time.perf_counter() - t0
    mlups = wl.nodes * k / dt / 1e6
    edge = "%dx%dx%d" % (wl.params["nx"], wl.params["ny"], wl.params["nz"])
    sample = ("%d of the %d requested steps of the %s workload after %d warm-up step (FP64 oracle, %d threads)"
              % (k, args.steps, edge, min(args.warmup, 1), cores))
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / k * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(workload_config(args, wl), precision="fp64", timed_steps=k),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "nproc": os.cpu_count(), "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args, wl):
    st = WORKLOAD_SETTINGS[args.workload]
    return {"workload": wl.name, "nodes": wl.nodes, "particles": len(wl.particles),
            "spheres": st["spheres"], "theta_c_deg": st["theta_c_deg"],
            "solubility_ratio": st["solubility_ratio"], "mobility": st["mobility"],
            "scalar_scheme": args.scalar_scheme}


def run_ours(args):
    import torch
    world, rank, local, group = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    from paper_2202_01631_gb300 import build
    build.build()
    from paper_2202_01631_gb300 import lbdp

    wl = workload(args.workload, edge_of(args), args.scalar_scheme)
    N = wl.nodes
    stream = torch.cuda.Stream()
    box = build_box(wl, args.precision, stream.cuda_stream)
    box.step(args.warmup)
    box.sync()
    # z chunk length of the two bulk kernels, timed on this machine (not timed)
    if args.no_tune:
        planes, tune_ms = box.planes(), None
    else:
        planes, tune_ms = box.tune(reps=5)

    # ---- device-resident throughput -------------------------------------
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(group)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        box.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(group)
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, group)
    box.sync()
    launches = lbdp.lb_step_launches(box.h, args.steps)
    value = N * args.steps * world / (ms * 1e-3) / 1e6

    # ---- per-kernel split (separate pass, events around every kernel) ----
    nprof = min(args.steps, 400)
    split, _ = lbdp.lb_profile_step(box.h, nprof)
    box.sync()
    peak, peak_kind = measured_peak()
    # the two bulk kernels, each timed alone in the split (events on the
    # launching stream); the roofline object reports the dominant one, the
    # fused kernel, against the algorithmic bytes it carries
    per_kernel = {}
    for name, cls, bpn, kind in (("kz_fused", "k_fused", ALG_BYTES_FUSED, "algorithmic"),
                                 ("kz_scalars", "k_scalars", DESIGN_BYTES_SCALARS, "design")):
        kms = split[cls] / nprof
        kb = bpn[args.precision] * N
        per_kernel[name] = {"avg_launch_ms": kms, "bytes_per_launch": kb, "bytes": kind,
                            "achieved": kb / (kms * 1e-3) / 1e9}
    coll_name = "kz_fused"
    coll_ms = per_kernel[coll_name]["avg_launch_ms"]
    coll_bytes = per_kernel[coll_name]["bytes_per_launch"]
    achieved = per_kernel[coll_name]["achieved"]
    step_ms = ms / args.steps
    step_gbs = ALG_BYTES_STEP[args.precision] * N / (step_ms * 1e-3) / 1e9

    # ---- end to end through host buffers --------------------------------
    host = {k: torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).pin_memory()
            for k, v in wl.fields.items()}
    outs = {k: torch.empty_like(v).pin_memory() for k, v in host.items()}
    e2e_steps = args.steps
    box2 = build_box(wl, args.precision, stream.cuda_stream)
    box2.set_planes(planes["k_fused"], planes["k_scalars"])
    box2.sync()
    barrier(group)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbdp.lb_set_fields(box2.h, *[host[k].numpy() for k in ("rho", "u", "psi", "phi")])
    box2.step(e2e_steps)
    lbdp.lb_read_fields(box2.h, *[outs[k].numpy() for k in ("rho", "u", "psi", "phi")])
    parts = box2.particles()
    dt = time.perf_counter() - t0
    dt = max_over_ranks(dt, group)
    h2d = sum(v.numel() * 8 for v in host.values())
    d2h = sum(v.numel() * 8 for v in outs.values()) + len(parts) * 18 * 8
    e2e = {"value": N * e2e_steps * world / dt / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
           "job": "upload initial fields from pinned host memory, %d steps, read back fields "
                  "and particles" % e2e_steps}
    box2.close()

    if rank != 0:
        box.close()
        return 0
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(wl)
    traffic = traffic_record(coll_name, args.precision, wl.name)
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": dict(workload_config(args, wl), precision=args.precision,
                       parallelism="replicas" if world > 1 else "single",
                       l2="state %.2f GB > L2 (129 MB); no flush" % (lbdp.lb_device_bytes(box.params) / 1e9),
                       z_planes=planes, z_tune_ms=tune_ms),
        "roofline": {"bound": "hbm", "kernel": coll_name, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": traffic,
                     "alg_bytes_per_launch": coll_bytes, "avg_launch_ms": coll_ms},
        "kernel_rooflines": {k: {"achieved": v["achieved"], "frac": v["achieved"] / peak,
                                 "avg_launch_ms": v["avg_launch_ms"], "unit": "GB/s", "bytes": v["bytes"]}
                             for k, v in per_kernel.items()},
        "step_roofline": {"alg_bytes_per_node": ALG_BYTES_STEP[args.precision], "achieved": step_gbs,
                          "peak": peak, "unit": "GB/s", "frac": step_gbs / peak},
        "kernel_ms_per_step": {k: v / nprof for k, v in split.items()},
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": launches,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    box.close()
    return 0


def _setup_member(box, wl):
    box.set_fields(**wl.fields)
    for p in wl.particles:
        box.add_particle(**p)


def run_batched(args):
    """64 uneven boxes in one batch vs the same boxes one by one."""
    import torch
    world, rank, local, group = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_2202_01631_gb300 import build
    build.build()
    from paper_2202_01631_gb300 import lbdp
    from paper_2202_01631_gb300 import workloads as W

    wls = W.batched(seed=0, n_boxes=args.boxes)
    target = wls[0].steps                        # steps per simulation (5000)
    nodes = sum(w.nodes for w in wls)
    stream = torch.cuda.Stream()
    batch = lbdp.Batch(precision=args.precision, arena_bytes=0, graph_steps=args.graph_steps,
                       stream=stream.cuda_stream)
    boxes = []
    for wl in wls:
        b = batch.add_box(**wl.params)
        _setup_member(b, wl)
        boxes.append(b)
    for b in boxes:
        batch.set_steps(b, args.warmup)
    batch.run(args.warmup)
    cfg, tune_ms = batch.tune(reps=5)
    for b in boxes:
        batch.set_steps(b, args.steps)
    batch.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(group)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        launches = batch.run(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(group)
    ms = max_over_ranks(ev0.elapsed_time(ev1), group)
    batch.sync()
    step_ms = ms / args.steps
    mlups = nodes * args.steps * world / (ms * 1e-3) / 1e6
    sims_h = len(wls) * world * 3600.0 / (step_ms * 1e-3 * target)
    peak, peak_kind = measured_peak()
    step_gbs = ALG_BYTES_STEP[args.precision] * nodes / (step_ms * 1e-3) / 1e9

    # ---- the same boxes one by one, single-box path -----------------------
    k1 = min(args.steps, 200)
    alone_ms = 0.0
    for wl in wls:
        b = lbdp.Box(precision=args.precision, stream=stream.cuda_stream, **wl.params)
        _setup_member(b, wl)
        b.step(10)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(k1)
        e1.record(stream)
        torch.cuda.synchronize()
        alone_ms += e0.elapsed_time(e1) / k1
        b.close()
    alone_sims_h = len(wls) * world * 3600.0 / (alone_ms * 1e-3 * target)

    # ---- end to end: host fields in, steps, psi/phi and particles out -----
    e2e_steps = min(args.steps, 500)
    host = [{k: torch.from_numpy(np.ascontiguousarray(wl.fields[k], dtype=np.float64)).pin_memory()
             for k in ("psi", "phi")} for wl in wls]
    outs = [{k: torch.empty_like(h[k]).pin_memory() for k in h} for h in host]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b, h in zip(boxes, host):
        lbdp.lb_set_fields(b.h, None, None, h["psi"].numpy(), h["phi"].numpy())
        batch.set_steps(b, e2e_steps)
    batch.run(e2e_steps)
    for b, o in zip(boxes, outs):
        lbdp.lb_read_fields(b.h, None, None, o["psi"].numpy(), o["phi"].numpy())
        b.particles()
    dt = max_over_ranks(time.perf_counter() - t0, group)
    h2d = sum(v.numel() * 8 for h in host for v in h.values())
    d2h = sum(v.numel() * 8 for o in outs for v in o.values()) + len(wls) * 18 * 8
    e2e = {"value": nodes * e2e_steps * world / dt / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
           "job": "upload psi, phi of every box from pinned host memory, %d batched steps, read back "
                  "psi, phi and particles" % e2e_steps}
    shapes = [lbdp.lbb_config_shape(c) for c in cfg]
    batch.close()
    if rank != 0:
        return 0
    line = {
        "metric": "batched sims/hour", "value": sims_h, "unit": "sims/hour", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": "batched_%d_boxes_32-96" % len(wls), "nodes": nodes, "precision": args.precision,
                   "steps_per_sim": target, "spheres_per_box": 1,
                   "tuned": {nc: {"threads": t, "planes_per_block": z, "ms": m}
                             for nc, (t, z), m in zip(lbdp.BATCH_KERNEL_CLASSES, shapes, tune_ms)},
                   "l2": "state %.1f GB > L2 (129 MB); no flush" % (batch_bytes(lbdp, wls, args.precision) / 1e9)},
        "mlups": mlups,
        "one_by_one": {"sims_per_hour": alone_sims_h, "ms_per_step_all_boxes": alone_ms,
                       "speedup": sims_h / alone_sims_h},
        "step_roofline": {"alg_bytes_per_node": ALG_BYTES_STEP[args.precision], "achieved": step_gbs,
                          "peak": peak, "unit": "GB/s", "frac": step_gbs / peak, "peak_kind": peak_kind},
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_bytes(lbdp, wls, precision):
    return sum(lbdp.lb_device_bytes(lbdp.box_params(precision, None, **w.params)) for w in wls)


def _percentile(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if v else None


def run_served(args):
    """A seeded Poisson request stream through the continuous-batching server,
    against a FIFO server that runs one request at a time."""
    import torch
    world, rank, local, group = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_2202_01631_gb300 import build
    build.build()
    from paper_2202_01631_gb300 import lbdp
    from paper_2202_01631_gb300 import workloads as W

    reqs = W.serving_requests(seed=rank, n=args.requests, rate=args.rate)
    stream = torch.cuda.Stream()
    srv = lbdp.Server(precision=args.precision, arena_bytes=48 << 30, chunk_steps=64,
                      stream=stream.cuda_stream)
    # warm the kernels and tune on a small mix first (not timed)
    warm = W.batched(seed=99, n_boxes=4, edge_range=(32, 48))
    for wl in warm:
        b = srv.batch.add_box(**wl.params)
        _setup_member(b, wl)
        srv.batch.set_steps(b, 20)
    srv.batch.run(20)
    srv.batch.tune(reps=3)
    for b in list(srv.batch.boxes):
        b.close()
    torch.cuda.synchronize()

    outs = {}
    done = {}
    nxt = 0
    rounds = 0
    barrier(group)
    t0 = time.perf_counter()
    with ClockSampler(local) as clk:
        while len(done) < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt][0] <= now:
                t_arr, wl = reqs[nxt]
                shape = (wl.params["nz"], wl.params["ny"], wl.params["nx"])
                outs[nxt] = (np.empty(shape), np.empty(shape))
                srv.submit(wl.params, wl.particles, psi=wl.fields["psi"], phi=wl.fields["phi"], steps=wl.steps,
                           arrival=t_arr, out_psi=outs[nxt][0], out_phi=outs[nxt][1])
                nxt += 1
            active, queued = srv.pump(time.perf_counter() - t0)
            rounds += 1
            for r in srv.poll():
                done[r["id"]] = r
            if active == 0 and queued == 0 and nxt < len(reqs):
                time.sleep(max(0.0, reqs[nxt][0] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    srv.close()
    lat = [done[i]["done"] - done[i]["arrival"] for i in sorted(done)]
    # a sustainable rate keeps the latency of late arrivals at that of early ones
    half = len(lat) // 2
    failed = sum(1 for i in done if done[i]["status"] != 0)   # ended early: reported, not hidden
    work = sum(wl.nodes * wl.steps for _, wl in reqs)
    span = max(done[i]["done"] for i in done) - reqs[0][0]
    sims_h = len(reqs) * 3600.0 / span

    # ---- one by one: each request alone (service time from a timed sample of
    # its steps), FIFO queue over the same arrivals --------------------------
    service = []
    for _, wl in reqs:
        b = lbdp.Box(precision=args.precision, stream=stream.cuda_stream, **wl.params)
        _setup_member(b, wl)
        k = min(wl.steps, 200)
        b.step(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        service.append(e0.elapsed_time(e1) * 1e-3 / k * wl.steps)
        b.close()
    t_free, lat1, last = 0.0, [], 0.0
    for (t_arr, _), sv in zip(reqs, service):
        start = max(t_arr, t_free)
        t_free = start + sv
        lat1.append(t_free - t_arr)
        last = t_free
    sims_h1 = len(reqs) * 3600.0 / (last - reqs[0][0])
    if rank != 0:
        return 0
    line = {
        "metric": "served p99 time-to-result", "value": _percentile(lat, 99), "unit": "s", "n_gpus": world,
        "steps": int(sum(wl.steps for _, wl in reqs)), "warmup": 20, "ms_per_step": None,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic",
        "config": {"workload": "served_poisson_%d_requests_rate_%g" % (len(reqs), args.rate),
                   "edges": "24..128", "steps": "log-uniform 500..20000", "spheres": "1..4",
                   "precision": args.precision, "chunk_steps": 64, "arena_gb": 48,
                   "l2": "resident states exceed L2 (129 MB); no flush"},
        "p50_s": _percentile(lat, 50), "p99_s": _percentile(lat, 99), "sims_per_hour": sims_h,
        "p50_first_half_s": _percentile(lat[:half], 50), "p50_second_half_s": _percentile(lat[half:], 50),
        "arrival_rate_per_h": args.rate * 3600.0,
        "mlups": work / wall / 1e6, "wall_s": wall, "rounds": rounds, "failed_requests": failed,
        "one_by_one": {"p50_s": _percentile(lat1, 50), "p99_s": _percentile(lat1, 99), "sims_per_hour": sims_h1,
                       "method": "each request timed alone on a sample of its steps; FIFO over the same arrivals"},
        "clocks": clk.summary(),
        "e2e": {"value": _percentile(lat, 99), "unit": "s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "job": "requests carry host psi/phi in and get host psi/phi and particles back"},
        "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "batched":
        return run_batched(args)
    if args.form == "served":
        return run_served(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
