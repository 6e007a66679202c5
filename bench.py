"""Benchmark: grid-point updates/s of the AT RK-stage right-hand side on GB300.

One step = one full Runge-Kutta step (every stage) over the whole domain of
the workload, inputs resident in HBM.  Default workload: the reactive-Euler
detonation, N = 2^24 FP64 points (4 fields, 512 MiB of state, larger than
L2) in 16,384 virtual PEs of 1024, WENO5 + AT-WENO5 with local
Lax-Friedrichs splitting, RK3-TVD, delays geometric (p = 0.5) on {0..4}
(Philox seed 0): the largest configuration that fits one GPU.  The timed
region is one at_step(K) call.  Workloads whose state fits in L2 flush it (a
256 MiB write) right before the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...      # the CPU oracle on host cores

Prints one JSON line (rank 0).  Under torchrun every rank runs an
independent replica (instance = rank): weak scaling, no collective.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (builder kwargs, description)
    "rns-flame-n16384": dict(kind="rns", case="flame", n=16384, pe_size=64, mode="at", k_max=4, seed=0, dt=0.003),
    "rns-ignition-n16384": dict(kind="rns", case="ignition", n=16384, pe_size=64, mode="at", k_max=4, seed=0,
                                dt=0.003),
    "advdiff-n2048": dict(kind="advdiff", n=2048, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075),
    # mid-size: the step-fused path with all steps in one cooperative launch
    "advdiff-n16384": dict(kind="advdiff", n=16384, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075),
    "advdiff-n134217728": dict(kind="advdiff", n=1 << 27, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075),
    # a quarter of the HBM run, for counter captures (inputs still larger than L2)
    "advdiff-n33554432": dict(kind="advdiff", n=1 << 25, pe_size=64, mode="at", k_max=3, seed=0, cfl=0.075),
    "detonation-n16777216": dict(kind="detonation", n=1 << 24, pe_size=1024, mode="at", k_max=4, seed=0),
    # half of it, for counter captures (inputs still larger than L2)
    "detonation-n8388608": dict(kind="detonation", n=1 << 23, pe_size=1024, mode="at", k_max=4, seed=0),
    "rns-flame-n16777216": dict(kind="rns", case="flame", n=1 << 24, pe_size=64, mode="at", k_max=4, seed=0,
                                dt=0.003),
    # half of it, for counter captures (inputs still larger than L2)
    "rns-flame-n8388608": dict(kind="rns", case="flame", n=1 << 23, pe_size=64, mode="at", k_max=4, seed=0,
                               dt=0.003),
    # 4,096 reacting instances, N log-uniform in [256, 8192] (9.4 M points), one batched launch
    "batched-rns-4096": dict(kind="batched", count=4096, seed=0),
    # Poisson arrivals at 2,000 requests/s of the three problem types, N log-uniform in
    # [512, 262,144], 100..5,000 steps: a burst of --serve-requests requests
    "serving-mixed": dict(kind="serving", rate=2000.0, seed=0),
}
DEFAULT = "detonation-n16777216"
NOMINAL_FP64_TFLOPS = 1.25  # GB300 FP64 (vector and tensor), nominal, at 2070 MHz boost

# FP64 flops per point per stage (FMA = 2, add/mul = 1) that the timed kernel
# executes: ncu's DFMA/DADD/DMUL thread-instruction counts of one launch on
# the large-N workloads (the persistent kernel on N = 16,384) divided by the
# point-stages of the launch.  They include the AT halo work and the
# instruction sequences of exp and the reciprocals, so achieved / peak is the
# share of the FP64 roof the kernel's own arithmetic uses.
FLOPS_PER_POINT_STAGE = {
    ("rns", "stage"): 165.7,         # central6 + AT6, 4 variables (RK4 stage 1 counted)
    ("rns", "persistent"): 165.8,    # same work, all K steps of one launch
    ("detonation", "stage"): 500.3,  # WENO5 + AT-WENO5, 8 reconstructions per edge (RK3 stage 0)
    ("advdiff", "stage"): 13.56,     # 5-tap merged stencil + RK4 update, mean of the 4 stages
    ("advdiff", "persistent"): 13.56,
    ("advdiff", "fused"): 13.56,     # the method's work only (13.65 as executed, with the recomputed edge points)
    ("rns", "fused"): 165.7,         # the method's work only (the tile-fused kernel also recomputes the strips)
    ("detonation", "fused"): 500.3,  # likewise: the per-stage kernel's count
}
# The method's own FP64 work per point per stage, by operation count (a
# divide, square root or exponential counts as one operation): the
# detonation's WENO5 + AT-WENO5 stage ~550 flops + 8 divides + 1 sqrt + 1 exp
# (two reconstructions per variable and edge, the splitting, the Arrhenius
# source, the update); the reacting flow's central6 stage ~150 flops + 4
# divides + 1 exp; advection-diffusion 52 flops per RK4 step.  The executed
# counts above also hold the instruction sequences of exp and the
# reciprocals and the AT halo work; achieved / peak on this count is
# roofline.frac_algorithmic.
ALG_FLOPS_PER_POINT_STAGE = {"detonation": 560.0, "rns": 155.0, "advdiff": 13.0}
# Algorithmic HBM bytes per point per stage of the per-stage path: the arrays
# a step reads and writes (RK4: 17 arrays, RK3-TVD: 8) x nvar x 8 B / stages.
BYTES_PER_POINT_STAGE = {"rns": 17 * 4 * 8 / 4, "detonation": 8 * 4 * 8 / 3, "advdiff": 17 * 8 / 4}
# the step-fused path reads u^n and writes u^{n+1} once per step (+ the ring)
BYTES_PER_POINT_STAGE_FUSED = {"advdiff": 2 * 8 / 4, "rns": 2 * 4 * 8 / 4, "detonation": 2 * 4 * 8 / 3}
# DRAM bytes per launch of the timed kernel (dram__bytes_read.sum +
# dram__bytes_write.sum) from the ncu captures of the current kernels, by
# workload and path; the advection-diffusion kernels were captured at
# N = 2^25 and are scaled by 4 for N = 2^27.
TRAFFIC_PER_LAUNCH = {
    ("rns-flame-n16384", "persistent"): 2.5541e+06,  # state and rings read once, writes stay in L2
    ("rns-flame-n16777216", "stage"): 2 * (8.3054e+08 + 5.2048e+08),  # captured at N = 2^23, x2
    ("rns-flame-n8388608", "stage"): 8.3054e+08 + 5.2048e+08,
    ("detonation-n8388608", "stage"): 2.7371e+08 + 2.2617e+08,
    ("detonation-n16777216", "stage"): 2 * (2.7371e+08 + 2.2617e+08),  # captured at N = 2^23, x2
    ("advdiff-n134217728", "stage"): 4 * (8.7076e+08 + 5.1195e+08),
    ("advdiff-n33554432", "stage"): 8.7076e+08 + 5.1195e+08,
    ("advdiff-n134217728", "fused"): 4 * (4.6988e+08 + 3.0293e+08),  # one step: u^n, u^{n+1}, the ring
    ("advdiff-n33554432", "fused"): 4.6988e+08 + 3.0293e+08,
    ("advdiff-n2048", "persistent"): 8.0384e+04,  # one-cluster launch: state and ring read once
    ("advdiff-n16384", "fused"): 2.8877e+05,  # cooperative fused launch: state and ring read once
    ("rns-flame-n16777216", "fused"): 2 * (2.6860e+08 + 3.1804e+08),  # tile-fused step, captured at N = 2^23, x2
    ("rns-flame-n8388608", "fused"): 2.6860e+08 + 3.1804e+08,
    ("detonation-n16777216", "fused"): 2 * (2.7574e+08 + 2.3274e+08),  # tile-fused step, captured at N = 2^23, x2
    ("detonation-n8388608", "fused"): 2.7574e+08 + 2.3274e+08,
}


# The kernel sources the captured counts above were taken from, per
# (workload, path): sha256 of the files that define the timed kernel (sorted
# by name, concatenated).  When they change, the counts may no longer hold:
# the roofline is then marked stale and its traffic is reported as null
# until the capture is redone.  A key without an entry is stale.
KERNEL_FILES = {
    "stage": ("at_device.cuh", "at_stage.cu"),
    "persistent": ("at_cluster.cu", "at_device.cuh", "at_persist.cu"),
    "fused": ("at_device.cuh", "at_fused.cu", "at_tilefused.cu"),
}
_SHA_STAGE = "0cecc1445fec100af6a8261ff949636d13abda82401f91c538bf46eea741a1e2"
_SHA_PERSISTENT = "b9e03fe76cc5c2182917044ff8965c8a015a4d4ab02a7bc7eaf4e2134e28dab4"
_SHA_FUSED = "ec36d6c3395c55e85546f641189d941abc7c206c5373b137cce2035fad616f1a"
PROFILED_SHA256 = {
    ("detonation-n16777216", "stage"): _SHA_STAGE,
    ("detonation-n8388608", "stage"): _SHA_STAGE,
    ("rns-flame-n16777216", "stage"): _SHA_STAGE,
    ("rns-flame-n8388608", "stage"): _SHA_STAGE,
    ("advdiff-n134217728", "stage"): _SHA_STAGE,
    ("advdiff-n33554432", "stage"): _SHA_STAGE,
    ("rns-flame-n16384", "persistent"): _SHA_PERSISTENT,
    ("advdiff-n2048", "persistent"): _SHA_PERSISTENT,
    ("advdiff-n134217728", "fused"): _SHA_FUSED,
    ("advdiff-n33554432", "fused"): _SHA_FUSED,
    ("advdiff-n16384", "fused"): _SHA_FUSED,
    ("rns-flame-n16777216", "fused"): _SHA_FUSED,
    ("rns-flame-n8388608", "fused"): _SHA_FUSED,
    ("detonation-n16777216", "fused"): _SHA_FUSED,
    ("detonation-n8388608", "fused"): _SHA_FUSED,
}


def sources_sha256(path: str) -> str:
    import hashlib
    d = os.path.join(ROOT, "paper_2204_01133_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(KERNEL_FILES[path]):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def kernel_label(kind, path, pb, arrival=False):
    """The kernel the library runs for this workload and path (the same rule
    as the library: small advection-diffusion problems take the one-cluster
    kernel on the persistent path)."""
    if path == "fused":
        return "step_fused_" + kind if kind == "advdiff" else "tile_fused_" + kind
    if path == "persistent" and kind == "advdiff" and not arrival and pb["pe_size"] in (32, 64, 128, 256):
        P = pb["n"] // pb["pe_size"]
        if any(P % c == 0 and P // c <= 4 for c in range(min(P, 16), 0, -1)):
            return "cluster_advdiff"
    return ("persist_" if path == "persistent" else "stage_") + kind


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # the profiling recipe's fallback copy bandwidth


def build_workload(name: str):
    from paper_2204_01133_gb300 import workloads as W
    kw = dict(WORKLOADS[name])
    kind = kw.pop("kind")
    if kind == "rns":
        return kind, W.rns(**kw)
    if kind == "advdiff":
        return kind, W.advdiff(**kw)
    return kind, W.detonation(**kw)


class Clocks:
    """nvidia-smi sampler running while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def fp64_probe(device: int):
    import ctypes

    import torch
    path = os.path.join(ROOT, "paper_2204_01133_gb300", "libat_probe.so")
    L = ctypes.CDLL(path)
    L.at_probe_fp64_fma.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    tf, ms = ctypes.c_double(), ctypes.c_double()
    st = torch.cuda.current_stream().cuda_stream
    rc = L.at_probe_fp64_fma(device, ctypes.c_void_p(st), 4000, 5, ctypes.byref(tf), ctypes.byref(ms))
    return tf.value if rc == 0 else None


def dist_env():
    from paper_2204_01133_gb300 import shard
    return shard.env()


def run_reference(args):
    """The CPU oracle, as it stands, on this host's cores (OpenMP over PEs,
    every core)."""
    import oracle
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = oracle.set_threads(0)
    if WORKLOADS[args.workload]["kind"] == "batched":
        from paper_2204_01133_gb300 import workloads as W
        cfg = WORKLOADS[args.workload]
        inst = W.batched_rns(count=cfg["count"], seed=cfg["seed"], nsteps=args.steps)
        rng = np.random.default_rng(1)
        sample = sorted(rng.choice(len(inst), size=8, replace=False).tolist())
        t0 = time.perf_counter()
        for i in sample:
            pb, init, n = inst[i]
            o = oracle.Oracle(pb, init)
            o.run(n)
        dt = time.perf_counter() - t0
        value = len(sample) / dt
        what = "%d random instances of the batch, %d RK4 steps each, %d threads" % (len(sample), args.steps, cores)
        print(json.dumps({
            "impl": "reference", "metric": "batched solves/s", "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "instances": cfg["count"]},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": what},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return
    if WORKLOADS[args.workload]["kind"] == "serving":
        from paper_2204_01133_gb300 import workloads as W
        cfg = WORKLOADS[args.workload]
        stream = W.serving_stream(rate=cfg["rate"], duration=1e9, seed=cfg["seed"], max_requests=args.serve_requests)
        # bounded sample: the first requests, each run for at most 50 of its steps
        t0, pts, nreq = time.perf_counter(), 0, 0
        for d in stream[:3]:
            pb, init = W.serving_request(d["kind"], d["n"], d["seed"], d["id"])
            st = min(50, d["steps"])
            o = oracle.Oracle(pb, init)
            o.run(st)
            pts += pb["n"] * st
            nreq += st / d["steps"]
        dt = time.perf_counter() - t0
        value = nreq / dt
        what = "first 3 requests of the stream, up to 50 of their steps each, %d threads" % cores
        print(json.dumps({
            "impl": "reference", "metric": "served solves/s", "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": None, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": what,
                             "grid_pt_updates_per_s": pts / dt},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return
    kind, (pb, init) = build_workload(args.workload)
    wl = describe(args.workload, pb)
    n = pb["n"]
    sample = "full domain, one oracle RK step per step"
    if n > 65536:
        # bounded sample: a window of whole PEs with the global PE indices
        B = pb["pe_size"]
        npe = max(1, 65536 // B)
        pb = dict(pb, n=npe * B, pe_base=0, pe_total=n // B)
        init = init[:, :npe * B].copy()
        sample = "window of %d PEs (%d points) of the %d-point domain, one oracle RK step per step" % (
            npe, npe * B, n)
    sample += ", %d threads (OpenMP over PEs)" % cores
    o = oracle.Oracle(pb, init)
    o.run(args.warmup)
    t0 = time.perf_counter()
    o.run(args.steps)
    dt = time.perf_counter() - t0
    pts = pb["n"]
    value = pts * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": "grid-pt updates/s", "value": value, "unit": "updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": wl,
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def describe(name, pb):
    d = {"workload": name, "n": pb["n"], "pe_size": pb["pe_size"], "pes": pb["n"] // pb["pe_size"],
         "pde": pb["pde"], "rk": pb["rk"], "mode": pb["mode"], "k_max": pb["k_max"], "dist": pb["dist"],
         "seed": pb["seed"], "dt": pb["dt"]}
    if pb["pde"] in ("advdiff", "rns"):
        d["order"] = pb["order"]
    else:
        d["scheme"] = "weno5"
    return d


def cpu_baseline(pb, init, budget_s=10.0):
    """The oracle, as it stands, on this host: one thread, then every core
    (OpenMP over PEs; the arithmetic per point is the same).  Each leg runs a
    bounded number of RK steps (about ``budget_s`` seconds) on a window of
    whole PEs for large domains."""
    import oracle
    n = pb["n"]
    sample_pb, sample_init, what = pb, init, "full domain"
    if n > 65536:
        B = pb["pe_size"]
        npe = max(1, 65536 // B)
        sample_pb = dict(pb, n=npe * B, pe_base=0, pe_total=n // B)
        sample_init = init[:, :npe * B].copy()
        what = "window of %d PEs (%d points) of the %d-point domain, global PE indices" % (npe, npe * B, n)
    legs = []
    for threads in (1, 0):
        used = oracle.set_threads(threads)
        o = oracle.Oracle(sample_pb, sample_init)
        t0 = time.perf_counter()
        o.run(2)
        per = (time.perf_counter() - t0) / 2
        steps = max(2, min(2000, int(budget_s / max(per, 1e-6))))
        t0 = time.perf_counter()
        o.run(steps)
        dt = time.perf_counter() - t0
        legs.append({"value": sample_pb["n"] * steps / dt, "cores": used, "steps": steps})
    oracle.set_threads(0)
    one, allc = legs
    return {"value": allc["value"], "unit": "updates/s", "cores": allc["cores"], "kind": "oracle",
            "sample": "%s, %d RK steps on %d threads (OpenMP over PEs)" % (what, allc["steps"], allc["cores"]),
            "single_thread": {"value": one["value"], "cores": 1,
                              "sample": "%s, %d RK steps, one thread" % (what, one["steps"])}}


def run_batched(args):
    """4,096 uneven reacting instances advanced together through the batch
    ABI (one graph-replayed launch for the K timed steps), against the same
    instances solved one after another through contexts (the plain
    per-instance launch path), on a random sample of them."""
    import torch
    from paper_2204_01133_gb300 import api, build
    from paper_2204_01133_gb300 import batch as BT
    from paper_2204_01133_gb300 import workloads as W
    from paper_2204_01133_gb300 import shard
    build.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = WORKLOADS[args.workload]
    count = args.batch_count or cfg["count"]
    tune_steps = len(BT.CANDIDATES)
    total = args.warmup + tune_steps + args.steps
    # weak scaling: every rank runs a batch of its own (seed per rank)
    inst = W.batched_rns(count=count, seed=cfg["seed"] + 7919 * rank, nsteps=total)
    points = sum(pb["n"] for pb, _, _ in inst)
    b = BT.Batch(capacity=count, device=local)
    for i, (pb, init, n) in enumerate(inst):
        b.bind(i, pb, init, n)
    b.run(args.warmup)
    tune = BT.autotune(b, chunk=1, use_cache=False)
    torch.cuda.synchronize()
    peak_meas = fp64_probe(local)
    l2 = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    l2.zero_()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record()
    b.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = shard.max_over_ranks(e0.elapsed_time(e1))
    clk = clocks.stop()
    for i in range(0, count, 512):
        assert b.query(i).left == 0
    solves_s = world * count / (ms * 1e-3)
    upd_s = world * points * args.steps / (ms * 1e-3)
    # plain per-instance path on a random sample (same instances, same steps)
    rng = np.random.default_rng(1)
    sample = sorted(rng.choice(count, size=min(args.plain_sample, count), replace=False).tolist())
    solvers = []
    for i in sample:
        pb, init, _ = inst[i]
        solvers.append(api.Solver(pb, init, device=local))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in solvers:
        s.step(args.steps)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_solves_s = len(sample) / plain_s
    sample_pts = sum(inst[i][0]["n"] for i in sample)
    # e2e: host states in, K steps, host states out (pinned), through the batch ABI
    host = [torch.from_numpy(np.ascontiguousarray(init)).pin_memory() for _, init, _ in inst]
    b2 = BT.Batch(capacity=count, device=local)
    b2.set_config(*b.config)
    outs = [torch.empty_like(h).pin_memory() for h in host]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, (pb, _, _) in enumerate(inst):
        b2.bind(i, pb, host[i], args.steps)
    b2.step(args.steps)
    for i in range(count):
        outs[i].copy_(b2.state(i), non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    state_bytes = sum(8 * 4 * pb["n"] for pb, _, _ in inst)
    fl = FLOPS_PER_POINT_STAGE[("rns", "stage")] * points * 4 * args.steps
    achieved = fl / (ms * 1e-3) / 1e12
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    print(json.dumps({
        "metric": "batched solves/s", "value": solves_s, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "instances": count, "points": points,
                   "solve": "one instance advanced %d RK4 steps" % args.steps, "pde": "rns", "order": 6,
                   "mode": "at", "k_max": "2..4 per instance", "pe_size": "32|64 per instance",
                   "l2": "flushed before the timed region",
                   "tuned": {"mode": ["instance", "flat"][tune["mode"]], "block": tune["block"],
                             "ctas_per_sm": tune["ctas_per_sm"]}},
        "grid_pt_updates_per_s": upd_s,
        "plain": {"solves_per_s": plain_solves_s, "sample_instances": len(sample), "sample_points": sample_pts,
                  "path": "one context per instance, at_step(K) each, one stream", "speedup": solves_s / plain_solves_s},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / NOMINAL_FP64_TFLOPS, "traffic": None,
                     "kernel": ["batch_run<RNS,3>", "batch_stage<RNS,3>"][tune["mode"]],
                     "peak_measured": peak_meas},
        "e2e": {"value": count / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": state_bytes / args.steps,
                "d2h_bytes_per_step": state_bytes / args.steps},
        "gpu_launches": 2 if tune["mode"] == 0 else 5 * args.steps + 1, "clocks": clk,
    }))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serving(args):
    """A burst of the serving stream (arrivals at 2,000 requests/s) served
    with continuous batching, then the same requests one at a time through a
    context each; solves/s over the makespan and p50/p99 latency for both."""
    import torch
    from paper_2204_01133_gb300 import build
    from paper_2204_01133_gb300 import workloads as W
    from paper_2204_01133_gb300.serve import Server, serve_plain, summarize
    build.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    cfg = WORKLOADS[args.workload]
    stream = W.serving_stream(rate=cfg["rate"], duration=1e9, seed=cfg["seed"], max_requests=args.serve_requests)
    # warm-up: a few small requests through both paths (module loads, first launches)
    warm = W.serving_stream(rate=1e4, duration=1e9, seed=99, n_min=512, n_max=2048, steps_min=10, steps_max=20,
                            max_requests=4)
    Server(mem_budget=args.serve_budget_gb << 30).run(warm)
    serve_plain(warm)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    srv = Server(mem_budget=args.serve_budget_gb << 30, capacity=1024, chunk=args.serve_chunk)
    done, elapsed = srv.run(stream)
    clk = clocks.stop()
    served = summarize(done, elapsed)
    pdone, pel = serve_plain(stream)
    plain = summarize(pdone, pel)
    work = sum(r.n * r.steps for r in done)
    # the FP64 work of the burst as the kernels execute it, and the fastest
    # any schedule could finish it at the FP64 peak
    per_step = {"advdiff": 4 * FLOPS_PER_POINT_STAGE[("advdiff", "stage")],
                "rns": 4 * FLOPS_PER_POINT_STAGE[("rns", "stage")],
                "detonation": 3 * FLOPS_PER_POINT_STAGE[("detonation", "stage")]}
    fl = sum(r.n * r.steps * per_step[r.kind] for r in done)
    floor_s = fl / (NOMINAL_FP64_TFLOPS * 1e12)
    print(json.dumps({
        "metric": "served solves/s", "value": served["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
        "steps": None, "warmup": len(warm), "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "requests": len(stream), "arrival_rate_per_s": cfg["rate"],
                   "mix": "advdiff | rns | detonation, N log-uniform [512, 262144], steps 100..5000",
                   "budget_gb": args.serve_budget_gb, "chunk_steps": args.serve_chunk,
                   "batch_mode": "flat", "ticks": srv.ticks,
                   "offered_point_steps": work},
        "served": served, "plain": plain, "speedup_solves_per_s": served["solves_per_s"] / plain["solves_per_s"],
        "saturation": {"fp64_work_tflop": fl / 1e12, "floor_s_at_fp64_peak": floor_s,
                       "max_speedup_vs_plain": plain["elapsed_s"] / floor_s,
                       "served_tflops": fl / 1e12 / served["elapsed_s"]},
        "latency_p50_s": served["latency_p50_s"], "latency_p99_s": served["latency_p99_s"],
        "e2e": {"value": served["solves_per_s"], "unit": "solves/s",
                "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "initial states are uploaded at admission; results stay on the device"},
        "clocks": clk,
    }))


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2204_01133_gb300 import api, build
    build.build()
    kind, (pb, init) = build_workload(args.workload)
    pb = dict(pb, instance=rank)
    n = pb["n"]
    S = api.STAGES[pb["rk"]]
    nvar = api.NVAR[pb["pde"]]
    state_bytes = 8 * nvar * n

    s = api.Solver(pb, init, device=local, path=args.path)
    if args.arrival:  # delays by arrival order (persistent path): not reproducible, reported beside
        s.set_option(api.OPT_ARRIVAL, 1)
    l2_flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush = state_bytes < (512 << 20)
    for _ in range(max(args.warmup, 3)):
        if flush:
            l2_flush.zero_()
        s.step(1)
    torch.cuda.synchronize()

    peak_meas = fp64_probe(local) if rank == 0 else None

    clocks = Clocks(local)
    clocks.start()
    launched0 = s.stats().kernels_launched
    s.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if flush:
        l2_flush.zero_()  # cold L2 when the timed region starts
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0.record()
    s.step(args.steps)  # K steps in one call, as a user would run them
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    st = s.stats()
    s.profile(False)
    clk = clocks.stop()
    launches = st.kernels_launched - launched0
    path = {1: "stage", 2: "persistent", 3: "fused"}.get(st.path, "?")
    launch_ms = st.stage_ms / max(st.launches_timed, 1)
    # point-stages per launch: all K steps (persistent; fused when its CTAs
    # fit one cooperative launch: one timed launch per call), one step (fused
    # otherwise), one stage
    fused_steps = max(1, round(args.steps / max(st.launches_timed, 1))) if path == "fused" else 1
    units_per_launch = n * (S * args.steps if path == "persistent" else S * fused_steps if path == "fused" else 1)
    from paper_2204_01133_gb300 import shard
    ms = shard.max_over_ranks(ms)
    value = world * n * args.steps / (ms * 1e-3)

    # end to end through the C ABI with host buffers: upload, steps, download
    import ctypes
    host_init = torch.from_numpy(np.ascontiguousarray(init)).pin_memory()
    host_out = torch.empty_like(host_init).pin_memory()
    e2e_steps = args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.check(api.lib().at_set_problem(s._h, ctypes.byref(s._pbs), ctypes.c_void_p(s.u.data_ptr()),
                                       ctypes.c_void_p(host_init.data_ptr()), 0, ctypes.c_void_p(s.ws.data_ptr()),
                                       s.ws.numel()))
    s.set_delays()
    s.run(e2e_steps)
    api.check(api.lib().at_read(s._h, api.READ_STATE, ctypes.c_void_p(host_out.data_ptr()), state_bytes, 0))
    e2e_s = time.perf_counter() - t0
    e2e_val = world * n * e2e_steps / shard.max_over_ranks(e2e_s)

    if rank == 0:
        fl = FLOPS_PER_POINT_STAGE[(kind, path)] * units_per_launch  # per launch
        achieved = fl / (launch_ms * 1e-3) / 1e12
        stale = PROFILED_SHA256.get((args.workload, path)) != sources_sha256(path)
        alg = ALG_FLOPS_PER_POINT_STAGE[kind] * units_per_launch / (launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / NOMINAL_FP64_TFLOPS,
                "traffic": None if stale else TRAFFIC_PER_LAUNCH.get((args.workload, path)),
                "stale": stale,
                "achieved_algorithmic": alg, "frac_algorithmic": alg / NOMINAL_FP64_TFLOPS,
                "alg_flops_per_point_stage": ALG_FLOPS_PER_POINT_STAGE[kind],
                "exec_flops_per_point_stage": FLOPS_PER_POINT_STAGE[(kind, path)],
                "kernel": ("steps_fused_" + kind) if path == "fused" and fused_steps > 1
                          else kernel_label(kind, path, pb, args.arrival),
                "avg_launch_ms": launch_ms, "launches_timed": int(st.launches_timed),
                "flops_per_launch": fl, "peak_kind": "nominal FP64 (1.25 TFLOP/s); see peak_measured",
                "peak_measured": peak_meas, "frac_of_measured": (achieved / peak_meas) if peak_meas else None}
        if path in ("stage", "fused"):  # HBM share (the persistent path keeps the state on chip)
            hbm_peak = measured_hbm_gbs()
            bpps = (BYTES_PER_POINT_STAGE if path == "stage" else BYTES_PER_POINT_STAGE_FUSED)[kind]
            gbs = bpps * units_per_launch / (launch_ms * 1e-3) / 1e9
            roof["hbm"] = {"achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                           "bytes_per_launch": bpps * units_per_launch,
                           "peak_kind": "measured copy bandwidth (MEASURED_PEAKS.json)"}
        out = {
            "metric": "grid-pt updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(describe(args.workload, pb), path=path,
                           delays="arrival order (not reproducible)" if args.arrival else "Philox draws",
                           l2="flushed before the timed region (K steps in one at_step call)" if flush
                           else "inputs larger than L2", parallelism="replicas" if world > 1 else "single"),
            "roofline": roof,
            "e2e": {"value": e2e_val, "unit": "updates/s", "h2d_bytes_per_step": state_bytes / e2e_steps,
                    "d2h_bytes_per_step": state_bytes / e2e_steps,
                    "note": "at_set_problem from pinned host + at_set_delays + at_run(K) + at_read to host"},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline(pb, init)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--plain-sample", type=int, default=256, help="instances timed on the plain path (batched)")
    ap.add_argument("--batch-count", type=int, default=0, help="instances of the batched workload (0: 4,096)")
    ap.add_argument("--serve-requests", type=int, default=48, help="requests in the served burst (serving)")
    ap.add_argument("--serve-budget-gb", type=int, default=16, help="device-memory budget of the server (GB)")
    ap.add_argument("--serve-chunk", type=int, default=50, help="steps per serving tick")
    ap.add_argument("--path", default="auto", choices=["auto", "stage", "persistent", "fused"],
                    help="execution path of the library (auto: persistent when the PEs fit on the GPU)")
    ap.add_argument("--arrival", action="store_true",
                    help="delays by arrival order instead of Philox draws (persistent path, not reproducible)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif WORKLOADS[args.workload]["kind"] == "batched":
        run_batched(args)
    elif WORKLOADS[args.workload]["kind"] == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
