#!/usr/bin/env python
"""Throughput of the DGSEM RK3 step: DOF-stage-updates/s on one GB300.

Workload (the metric's configuration): compressible Navier-Stokes
Taylor-Green vortex, Ma 0.1, Re 1600, Pr 0.72, periodic [-pi,pi]^3 with 16^3
curved hexahedra (every node moved by 0.05 sin x sin y sin z), N = 3
(64^3 nodes), Chandrashekar split-form volume term + Roe surface flux + BR1,
Williamson RK3 with the CFL-0.5 time step recomputed on the device each
step.  A step is one RK3 step (three residual evaluations + updates) of the
whole mesh.  value = nodes * 3 stages * K / (sum of the K step times), for
the mixed path (FP32 flux arithmetic, FP64 state / geometry / RK); the
FP64 path is reported beside it with its own throughput, and each path
states its L2 difference.

The state (~70 MB with geometry and scratch) fits in the 129 MB L2, so L2 is
flushed (a 512 MB buffer is written) between timed steps; each step is timed
with CUDA events on the launching stream and the flush is outside the events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl hs3d|reference]

--impl reference times the FP64 CPU oracle on this machine's host cores on the
same workload (a bounded sample per step), as the reference arm.
Under torchrun (N > 1) every rank runs an independent replica (the path is
a single-GPU solver; replicas only) and rank 0 prints the aggregate.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# workload
EX = EY = EZ = 16
N = 3
AMP = 0.05
MA, RE, PR, GAMMA, CFL = 0.1, 1600.0, 0.72, 1.4, 0.5
NODES = EX * EY * EZ * (N + 1) ** 3
VOLUME_FORM = "ec"
PHYSICS = "ns"
SURFACE_FLUX = "roe"
METRIC = "DOF-stage-updates/s"
WORKLOAD = ("NS Taylor-Green vortex Ma 0.1 Re 1600, [-pi,pi]^3, 16^3 curved hex (amp 0.05), N=3 (64^3 DOF), "
            "EC split form + Roe + BR1, Williamson RK3 CFL 0.5")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hs3d", choices=["hs3d", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=512, help="requests in the batched-serving stream (0: skip)")
    ap.add_argument("--mesh", type=int, default=16,
                    help="elements per direction (16 = the metric's workload; larger sizes for profiling only)")
    ap.add_argument("--stress", type=int, default=16, help="requests in the memory-admission stress run (0: skip)")
    ap.add_argument("--stress-budget-gb", type=float, default=8.0,
                    help="server device budget of the stress run; 0: 90%% of the device's free memory")
    ap.add_argument("--stress-emax", type=int, default=40)
    ap.add_argument("--stress-precisions", default="mixed32,fp64",
                    help="comma-separated precisions of the stress run, each on its own server")
    ap.add_argument("--no-workloads", dest="workloads", action="store_false",
                    help="skip the larger configurations reported beside the line")
    ap.add_argument("--only", choices=["mixed32", "mixed_tc", "fp64"], default=None,
                    help="time one precision only (profiling runs)")
    ap.add_argument("--order", type=int, default=None, help="profiling runs: polynomial order N (default 3)")
    ap.add_argument("--volume", default=None, help="profiling runs: volume form (default ec)")
    ap.add_argument("--physics", default=None, choices=["euler", "ns"], help="profiling runs: equations (default ns)")
    ap.add_argument("--surface", default=None, help="profiling runs: surface flux (default roe)")
    ap.add_argument("--aniso-profile", type=int, default=0, metavar="E",
                    help="profiling run only: 2 FP64 RK3 steps of the E^3 TGV with per-direction degrees 2..5 "
                         "(NS, EC + Roe), then exit")
    ap.add_argument("--pmesh-profile", type=int, default=0, metavar="E",
                    help="profiling run only: 3 mixed RK3 steps of the E^3 TGV with per-element degrees 2..5 "
                         "(NS, EC + Roe), then exit")
    args = ap.parse_args()
    if any(x is not None for x in (args.order, args.volume, args.physics, args.surface)) and not args.only:
        ap.error("--order, --volume, --physics and --surface select a profiling case: give --only too")
    global EX, EY, EZ, NODES, N, VOLUME_FORM, PHYSICS, SURFACE_FLUX
    EX = EY = EZ = args.mesh
    if args.order is not None:
        N = args.order
    if args.volume is not None:
        VOLUME_FORM = args.volume
    if args.physics is not None:
        PHYSICS = args.physics
    if args.surface is not None:
        SURFACE_FLUX = args.surface
    NODES = EX * EY * EZ * (N + 1) ** 3
    return args


# ------------------------------------------------------------------ distributed plumbing (replicas only)

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("HS3D_DIST_BACKEND", "nccl")
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(units_local, seconds_local, world):
    """Whole-job throughput: units all ranks processed / slowest rank's time."""
    units = reduce_sum(units_local, world)
    secs = reduce_max(seconds_local, world)
    return units / secs, secs


# ------------------------------------------------------------------ clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the sampler is running (first line in) before the timed region starts
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


# ------------------------------------------------------------------ measured DRAM traffic of the dominant kernel

# dram__bytes_read.sum + dram__bytes_write.sum per launch of k_volume_dev<3,NS,EC> on this workload,
# from one ncu capture (profiles/k_volume_mixed_ec_ns_N3_tgv16_traffic.md), and the digest of the
# kernel's sources at the time of the capture: the figure is reported only while they are unchanged.
VOLUME_TRAFFIC = {"bytes_per_launch": 56759979,
                  "sources_sha256": "995828b015ba9ee08d81b45f7f68b5945df2668c13662a1abe90444a4063f6ac"}
VOLUME_SOURCES = ["volume_dev.cuh", "lowmach.cuh", "volume_ec.cu", "physics.cuh", "internal.cuh"]


def volume_sources_digest():
    import hashlib
    h = hashlib.sha256()
    for f in VOLUME_SOURCES:
        with open(os.path.join(ROOT, "paper_2206_09733_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_volume_traffic():
    t = VOLUME_TRAFFIC
    if t["bytes_per_launch"] is None or t["sources_sha256"] != volume_sources_digest():
        return None
    return t["bytes_per_launch"]


# ------------------------------------------------------------------ algorithmic cost model (per launch)

def kernel_bytes(kernel, prec, E=None, n=N + 1):
    """Compulsory DRAM bytes of one launch of each kernel.  FP64 path: state,
    metric terms, 1/J and scratch in FP64.  Mixed path: every kernel reads
    the FP64 state (it forms the deviations from it) and FP32 copies of Ja,
    1/J and the face normals; the element kernel also reads the FP32 low
    part of Ja (the float-float mass divergence), keeps the RK register in
    FP32 and reads and rewrites each element's 112-byte reference state,
    which the gradient kernel reads too; the face kernel writes one flux
    block per side of each face; scratch in FP32."""
    E = EX * EY * EZ if E is None else E
    n2, n3 = n * n, n ** 3
    if prec == "fp64":
        s, geo, jal, sides, reg, anc = 8, 72 + 8, 0, 1, 8, 0
    else:
        s, geo, jal, sides, reg, anc = 4, 36 + 4, 36, 2, 4, 112
    if kernel == "volume":     # u, metrics (+ low part), 1/J, grads, this element's 6 face blocks, reference
        #                        state in and out; g in/out, u out
        return E * (40 * n3 + (geo + jal) * n3 + 12 * n3 * s + 6 * 5 * n2 * s + 2 * anc + 2 * 5 * reg * n3 + 40 * n3)
    if kernel == "face":       # two FP64 traces, face normal, two gradient traces in; flux (per side) out
        return 3 * E * (2 * 40 * n2 + 3 * n2 * s + 2 * 12 * n2 * s + sides * 5 * n2 * s)
    if kernel == "grad":       # own FP64 state, metrics, 1/J, 6 neighbour FP64 traces, reference state in;
        #                        gradients out
        return E * (40 * n3 + geo * n3 + 6 * 40 * n2 + anc + 12 * n3 * s)
    return 0


def volume_flops(E=None, n=N + 1):
    """Algorithmic flops of one launch of the split-form NS element kernel
    (an FMA counts 2, a divide / sqrt / log 1 each), counted from the
    formulas the kernel evaluates:
      primitives 14, three Euler fluxes 3*13, three viscous fluxes 3*40,
      two-point fluxes 3*(n-1) * 63 (two log means 2*14, averages 14,
      flux 21) plus the 5-term axpy 10 each, diagonal 3*10,
      viscous D-contraction 3*n*8, surface lift <= 3*10, scale + RK 5*5."""
    E = EX * EY * EZ if E is None else E
    per_node = 14 + 3 * 13 + 3 * 40 + 3 * (n - 1) * (63 + 10) + 3 * 10 + 3 * n * 8 + 30 + 25
    return E * n ** 3 * per_node


# ------------------------------------------------------------------ the hs3d arm

def run_hs3d(args, world, rank, local):
    import numpy as np
    import torch

    import paper_2206_09733_gb300 as hs
    from paper_2206_09733_gb300 import build as hsbuild

    if rank == 0 or not os.path.exists(hs.LIB_PATH):
        hsbuild.build()
    barrier(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    lo, hi = (-np.pi,) * 3, (np.pi,) * 3
    mesh = hs.Mesh(EX, EY, EZ, N, lo=lo, hi=hi, amp=AMP)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def cfg(prec):
        return hs.solver_cfg(PHYSICS, SURFACE_FLUX, VOLUME_FORM, prec, gamma=GAMMA, Re=RE, Pr=PR, Ma=MA, cfl=CFL)

    def fresh():
        u = mesh.init_state(mesh.empty_state(), "tgv", GAMMA, MA)
        return u, torch.zeros_like(u)

    # launch shapes chosen by the library's autotuner (outside every timed region;
    # profiling runs keep the default shapes so that captures see no tuning launches)
    tuned = {} if args.only else {prec: mesh.autotune(cfg(prec)) for prec in ("mixed32", "fp64")}

    def timed_steps(prec, K, W, sampler=None):
        u, g = fresh()
        c = cfg(prec)
        for _ in range(W):
            mesh.rk3_run(c, u, g, 1)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier(world)
        torch.cuda.synchronize()
        for a, b in evs:
            flush.fill_(1.0)                  # evict the working set from L2 between steps
            a.record(stream)
            # one step continuing the run (dt < 0): exactly a step of one longer run, the dt
            # maxima coming from the previous step's last stage
            mesh.rk3_run(c, u, g, 1, dt=-1.0)
            b.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms, u

    # --- headline: mixed path, then FP64 path, K timed steps each
    if args.only:
        # profiling run: one precision, no extras
        ms, _ = timed_steps(args.only, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"profiling_run": True, "precision": args.only, "mesh": EX, "steps": args.steps,
                              "ms_per_step": round(ms / args.steps, 4)}), flush=True)
        return
    with ClockSampler(local) as clk:
        ms32, u32 = timed_steps("mixed32", args.steps, args.warmup)
        ms64, u64 = timed_steps("fp64", args.steps, args.warmup)
    clocks = clk.summary()
    v32, s32 = aggregate(NODES * 3 * args.steps, ms32 * 1e-3, world)
    v64, s64 = aggregate(NODES * 3 * args.steps, ms64 * 1e-3, world)
    # both paths advanced W + K steps from the same initial state
    d = (u32 - u64).double()
    l2_32_vs_64 = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(u64))
    t64, steps64 = mesh.clock()

    # --- per-kernel attribution (eager steps with events between kernels)
    prof = {}
    for prec in ("mixed32", "fp64"):
        u, g = fresh()
        acc = {"dt": 0.0, "grad": 0.0, "face": 0.0, "volume": 0.0, "step": 0.0}
        reps = min(args.steps, 20)
        for _ in range(3):
            mesh.rk3_step_profiled(cfg(prec), u, g)
        for _ in range(reps):
            flush.fill_(1.0)
            r = mesh.rk3_step_profiled(cfg(prec), u, g)
            for k in acc:
                acc[k] += r[k] / reps
        prof[prec] = acc
    peaks = hs.alu_peaks()

    # --- e2e: the C-ABI with HOST buffers.  Every step copies its input state
    # from pinned host memory into a device buffer (H2D), runs one RK3 step on
    # it (hs3d_rk3_run) and copies the result back to pinned host memory (D2H).
    # Two device state buffers alternate (the library keeps a captured graph
    # for each), and the copies run on their own streams, so the H2D of step
    # k+1 and the D2H of step k overlap step k's kernels on the compute stream.
    pin_in = torch.empty(mesh.shape, dtype=torch.float64, pin_memory=True)
    pin_out = [torch.empty(mesh.shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    u, g = fresh()
    pin_in.copy_(u.cpu())
    ub = [u, torch.empty_like(u)]
    c = cfg("mixed32")
    s_h2d, s_d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_step = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]
    for b in (0, 1):
        ev_out[b].record(stream)

    def e2e_steps(K):
        for k in range(K):
            b = k & 1
            s_h2d.wait_event(ev_out[b])            # buffer b read out by step k-2
            with torch.cuda.stream(s_h2d):
                ub[b].copy_(pin_in, non_blocking=True)
                ev_in[b].record(s_h2d)
            stream.wait_event(ev_in[b])
            mesh.rk3_run(c, ub[b], g, 1, stream=stream)
            ev_step[b].record(stream)
            s_d2h.wait_event(ev_step[b])
            with torch.cuda.stream(s_d2h):
                pin_out[b].copy_(ub[b], non_blocking=True)
                ev_out[b].record(s_d2h)
        for b in (0, 1):
            stream.wait_event(ev_out[b])

    e2e_steps(max(args.warmup, 2))
    torch.cuda.synchronize()
    K_e2e = args.steps
    barrier(world)
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    s_h2d.wait_event(e_start)
    s_d2h.wait_event(e_start)
    e2e_steps(K_e2e)
    e_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = e_start.elapsed_time(e_end)
    # every step started from the same host state: its results agree bitwise
    assert K_e2e < 2 or torch.equal(pin_out[0], pin_out[1])
    e2e_val, _ = aggregate(NODES * 3 * K_e2e, e2e_ms * 1e-3, world)
    state_bytes = NODES * 5 * 8

    # --- roofline of the dominant kernel of the mixed path
    p32 = prof["mixed32"]
    dom = max(("grad", "face", "volume"), key=lambda k: p32[k])
    per_launch_ms = p32[dom] / 3.0
    hbm_peak = measured_hbm_peak()
    achieved_gbs = kernel_bytes(dom, "mixed32") / (per_launch_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved_gbs, 1), "peak": hbm_peak[0], "unit": "GB/s",
            "frac": round(achieved_gbs / hbm_peak[0], 4),
            "traffic": measured_volume_traffic() if dom == "volume" else None,
            "algorithmic_bytes_per_launch": kernel_bytes(dom, "mixed32"),
            "kernel": "k_volume_dev<3,NS,EC>" if dom == "volume" else dom, "peak_source": hbm_peak[1]}
    p64 = prof["fp64"]
    fp64_ach = volume_flops() / (p64["volume"] / 3.0 * 1e-3) / 1e12
    # the same element kernel of the mixed path against the FP32 pipe (algorithmic flops)
    fp32_ach = volume_flops() / (per_launch_ms * 1e-3) / 1e12 if dom == "volume" else None
    if fp32_ach is not None:
        roof["fp32_alu"] = {"achieved": round(fp32_ach, 3), "peak": round(peaks["fp32_tflops"], 3), "unit": "TFLOP/s",
                            "frac": round(fp32_ach / peaks["fp32_tflops"], 4),
                            "peak_source": "measured FP32 FMA-chain kernel (hs3d_alu_peaks)"}
    fp64_roof = {"bound": "alu", "kernel": "k_volume<3,double,NS,EC>", "achieved": round(fp64_ach, 3),
                 "peak": round(peaks["fp64_tflops"], 3), "unit": "TFLOP/s",
                 "frac": round(fp64_ach / peaks["fp64_tflops"], 4),
                 "peak_source": "measured FP64 FMA-chain kernel (hs3d_alu_peaks)"}

    extra = {}
    if args.workloads and args.mesh == 16:
        extra["tgv_32cubed_N7_standard_roe_br1"] = run_workload("cfg3", 32, 7, "ns", "roe", "standard", 5, 2,
                                                                precisions=("mixed32", "fp64"))
        extra["tgv_64cubed_N3_standard_lf_euler"] = run_workload("sweep", 64, 3, "euler", "lf", "standard", 5, 2,
                                                                 precisions=("mixed32", "fp64"))
        extra["tgv_52cubed_N4_standard_lf_euler"] = run_workload("sweep", 52, 4, "euler", "lf", "standard", 5, 2)
        extra["tgv_64cubed_N3_standard_roe_br1"] = run_workload("sweep", 64, 3, "ns", "roe", "standard", 5, 2)
        for vol, surf, tm in (("kg", "roe", "rk4"), ("pirozzoli", "roe", "rk3"), ("ducros", "roe", "rk3"),
                              ("morinishi", "ldroe", "rk3"), ("ir", "matrix", "rk3")):
            extra[f"tgv_32cubed_N3_{vol}_{surf}_br1_{tm}"] = run_workload("split", 32, 3, "ns", surf, vol, 5, 2,
                                                                          time=tm)
        extra["tgv_32cubed_N3_gauss_standard_roe_br1"] = run_workload("gauss", 32, 3, "ns", "roe", "standard", 5, 2,
                                                                       nodes="gauss")
        extra["tgv_32cubed_degrees2to5_ec_roe_br1_mortar"] = run_pworkload(32, 2, 5, "ns", "roe", "ec", 5, 2)
        extra["tgv_16cubed_aniso_degrees2to5_ec_roe_br1_fp64"] = run_aworkload(16, 2, 5, "ns", "roe", "ec", 3, 2)

    if args.stress > 0:
        extra["admission_stress"] = {p: run_stress(args.stress, args.stress_budget_gb, args.stress_emax, p)
                                     for p in args.stress_precisions.split(",")}

    serving = None
    if args.serving > 0:
        serving = run_serving(args.serving)
        # below saturation: 32 requests at a twentieth of the rate
        serving["below_saturation"] = run_serving(32, rate_scale=20.0, baselines=False)

    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # both headline paths advanced W + K steps from the initial condition
        cpu, errors = cpu_baseline(finals={"mixed32": u32.cpu().numpy(), "fp64": u64.cpu().numpy()},
                                   compare_steps=args.warmup + args.steps)

    launches_per_step = 1 + 3 * 3   # dt finalize, 3 x (grad, face, element) (continuing steps: no priming pass)
    line = {
        "metric": METRIC, "value": round(v32, 1), "unit": "DOF-stage-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(s32 * 1e3 / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (analytic Taylor-Green initial condition)",
        "config": {"workload": WORKLOAD, "E": EX * EY * EZ, "N": N, "nodes": NODES,
                   "precision": "mixed32: FP32 flux arithmetic on deviations from a per-element reference state "
                                "(deviations formed in FP64 from the FP64 state), mass divergence in float-float "
                                "(FP32 pairs), FP32 copies of Ja (+ FP32 low part), 1/J and face normals; FP64 "
                                "state and RK accumulation, FP32 RK register",
                   "l2": "flushed between timed steps (512 MB write outside the step events)",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "timing": "sum of per-step CUDA-event times on the launching stream, CUDA-graph replay"},
        "l2_rel_vs_fp64_gpu": l2_32_vs_64,
        "error_vs_oracle": errors,
        "fp64": {"value": round(v64, 1), "ms_per_step": round(s64 * 1e3 / args.steps, 4), "dtype": "f64",
                 "sim_time_after_all_steps": t64, "roofline": fp64_roof},
        "kernel_ms_per_step": {k: {kk: round(vv, 5) for kk, vv in v.items()} for k, v in prof.items()},
        "alu_peaks_measured": {k: round(v, 3) for k, v in peaks.items()},
        "autotuned_elems_per_cta": {k: {"grad": v[0], "element": v[1]} for k, v in tuned.items()},
        "roofline": roof,
        "e2e": {"value": round(e2e_val, 1), "unit": "DOF-stage-updates/s", "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes,
                "how": "per step: H2D copy of the state from pinned host memory, one RK3 step (hs3d_rk3_run), "
                       "D2H copy of the result to pinned host memory; two device state buffers alternate and the "
                       "copies run on two copy streams, overlapping the neighbouring steps' kernels"},
        "gpu_launches": launches_per_step * args.steps * 2,
        "clocks": clocks,
    }
    if extra:
        line["workloads"] = extra
    if serving is not None:
        line["serving"] = serving
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy, burst)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


# ------------------------------------------------------------------ further workloads (reported beside the line)

def step_bytes(prec, physics, E, n, stages=3):
    """Compulsory DRAM bytes of one RK step: `stages` stages of (BR1
    gradients,) face fluxes and the element kernel (the dt maxima are fused
    into the last stage)."""
    per_stage = kernel_bytes("face", prec, E, n) + kernel_bytes("volume", prec, E, n)
    if physics == "ns":
        per_stage += kernel_bytes("grad", prec, E, n)
    else:   # no gradients are read by the face and element kernels
        s = 8 if prec == "fp64" else 4
        per_stage -= E * 12 * n ** 3 * s + 3 * E * 24 * n * n * s
    return stages * per_stage


def run_workload(name, Ed, Nd, physics, surface, volume, steps, warmup, precisions=("mixed32", "fp64"), time="rk3",
                 nodes="lobatto"):
    """DOF-stage-updates/s of one curved TGV configuration (Ma 0.1, Re 1600,
    amp 0.05, CFL 0.5), CUDA-event timed per step; the state exceeds L2 so no
    flush is needed.  Also the algorithmic HBM throughput of the step."""
    import numpy as np
    import torch

    import paper_2206_09733_gb300 as hs
    mesh = hs.Mesh(Ed, Ed, Ed, Nd, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=AMP, nodes=nodes)
    n = Nd + 1
    npts = Ed ** 3 * n ** 3
    stages = 5 if time == "rk4" else 3
    out = {"E": Ed ** 3, "N": Nd, "nodes": npts,
           "scheme": f"{physics} {surface} surface, {volume} volume, {time} ({stages} stages), {nodes} nodes"}
    stream = torch.cuda.current_stream()
    finals = {}
    for prec in precisions:
        cfg = hs.solver_cfg(physics, surface, volume, prec, gamma=GAMMA, Re=RE, Pr=PR, Ma=MA, cfl=CFL, time=time)
        mesh.autotune(cfg)
        u = mesh.init_state(mesh.empty_state(), "tgv", GAMMA, MA)
        g = torch.zeros_like(u)
        mesh.rk3_run(cfg, u, g, warmup)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mesh.rk3_run(cfg, u, g, steps)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[prec] = {"value": round(npts * stages / (ms * 1e-3), 1), "ms_per_step": round(ms, 3)}
        if nodes == "lobatto":   # the byte model counts Gauss-Lobatto traces (one node per face point)
            gbs = step_bytes(prec, physics, Ed ** 3, n, stages) / (ms * 1e-3) / 1e9
            out[prec].update({"hbm_gbs_algorithmic": round(gbs, 1), "hbm_frac": round(gbs / measured_hbm_peak()[0], 4)})
        finals[prec] = u
        del g
    # every precision ran warmup + steps steps from the same initial state
    if "fp64" in finals:
        ref = finals["fp64"]
        for prec, u in finals.items():
            if prec != "fp64":
                out[prec]["l2_rel_vs_fp64_gpu"] = float(torch.linalg.vector_norm(u - ref) / torch.linalg.vector_norm(ref))
    del finals, mesh
    torch.cuda.empty_cache()
    return out


def pstep_bytes(prec, physics, deg, ex, ey, ez, stages=3):
    """Compulsory DRAM bytes of one RK step on a mesh with per-element
    degrees: per degree bucket the element (and BR1 gradient) kernel bytes of
    the conforming model, the gradient kernel reading the mortar's interface
    values (4 n^2 per face) instead of neighbour traces; per face the mortar
    kernels read both sides' traces at their own degree (+ gradients for the
    viscous flux, + the face metric of the side of the larger degree) and
    write each side's projected block."""
    import numpy as np
    s, st = (8, 40) if prec == "fp64" else (4, 20)
    ns = physics == "ns"
    deg = np.asarray(deg)
    n = deg + 1
    per_stage = 0
    for N in np.unique(deg):
        E = int((deg == N).sum())
        per_stage += kernel_bytes("volume", prec, E, int(N) + 1)
        if ns:
            nn = int(N) + 1
            per_stage += kernel_bytes("grad", prec, E, nn) - E * 6 * st * nn * nn + E * 6 * 4 * nn * nn * s
    if not ns:
        per_stage -= int(((12 * n ** 3 * s) * 1).sum())
    e = np.arange(deg.size)
    a, b, c = e % ex, (e // ex) % ey, e // (ex * ey)
    for d in range(3):
        ab = [a.copy(), b.copy(), c.copy()]
        ab[d] = (ab[d] + 1) % (ex, ey, ez)[d]
        r = ab[0] + ex * (ab[1] + ey * ab[2])
        nL2, nR2 = n ** 2, n[r] ** 2
        nH2 = np.maximum(nL2, nR2)
        flux = (nL2 + nR2) * (st + 5 * s + (12 * s if ns else 0)) + 3 * nH2 * s
        per_stage += int(flux.sum())
        if ns:
            per_stage += int(((nL2 + nR2) * (st + 4 * s)).sum())
    return stages * per_stage


def run_pworkload(Ed, dlo, dhi, physics, surface, volume, steps, warmup, precisions=("mixed32", "fp64"), seed=7):
    """DOF-stage-updates/s of the curved TGV (Ma 0.1, Re 1600, amp 0.05,
    CFL 0.5) on an Ed^3 mesh whose elements carry seeded degrees uniform in
    [dlo, dhi], coupled by mortars (hs3d_pmesh_run), CUDA-event timed; the
    state exceeds L2."""
    import numpy as np
    import torch

    import paper_2206_09733_gb300 as hs
    deg = np.random.default_rng(seed).integers(dlo, dhi + 1, size=Ed ** 3).astype(np.int32)
    pm = hs.PMesh(Ed, Ed, Ed, deg, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=AMP)
    npts = int(((deg + 1) ** 3).sum())
    out = {"E": Ed ** 3, "degrees": f"uniform in {dlo}..{dhi} (numpy default_rng({seed}))", "nodes": npts,
           "geometry_degree": pm.Ngeo,
           "scheme": f"{physics} {surface} surface, {volume} volume, rk3, mortars of degree max(N_L, N_R)",
           "counts": {int(k): int((deg == k).sum()) for k in range(dlo, dhi + 1)}}
    stream = torch.cuda.current_stream()
    finals = {}
    for prec in precisions:
        cfg = hs.solver_cfg(physics, surface, volume, prec, gamma=GAMMA, Re=RE, Pr=PR, Ma=MA, cfl=CFL)
        u = pm.init_state(pm.empty_state(), "tgv", GAMMA, MA)
        g = torch.zeros_like(u)
        pm.run(cfg, u, g, warmup)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pm.run(cfg, u, g, steps, dt=-1.0)   # continuing the warm-up run: every timed step a graph replay
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        gbs = pstep_bytes(prec, physics, deg, Ed, Ed, Ed) / (ms * 1e-3) / 1e9
        out[prec] = {"value": round(npts * 3 / (ms * 1e-3), 1), "ms_per_step": round(ms, 3),
                     "hbm_gbs_algorithmic": round(gbs, 1), "hbm_frac": round(gbs / measured_hbm_peak()[0], 4)}
        finals[prec] = u
        del g
    if "fp64" in finals:
        ref = finals["fp64"]
        for prec, u in finals.items():
            if prec != "fp64":
                out[prec]["l2_rel_vs_fp64_gpu"] = float(torch.linalg.vector_norm(u - ref) / torch.linalg.vector_norm(ref))
    del finals, pm
    torch.cuda.empty_cache()
    return out


def run_aworkload(Ed, dlo, dhi, physics, surface, volume, steps, warmup, seed=7):
    """DOF-stage-updates/s of the curved TGV (Ma 0.1, Re 1600, amp 0.05,
    CFL 0.5) on an Ed^3 mesh whose elements carry seeded degrees (P_x, P_y,
    P_z), each uniform in [dlo, dhi], coupled by mortars of per-direction
    degree (hs3d_pmesh_create3 + hs3d_pmesh_run, FP64: the anisotropic path
    computes in FP64 only), CUDA-event timed."""
    import numpy as np
    import torch

    import paper_2206_09733_gb300 as hs
    deg = np.random.default_rng(seed).integers(dlo, dhi + 1, size=(Ed ** 3, 3)).astype(np.int32)
    pm = hs.PMesh(Ed, Ed, Ed, deg, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=AMP)
    npts = int(np.prod(deg + 1, axis=1).sum())
    out = {"E": Ed ** 3, "degrees": f"(P_x, P_y, P_z) each uniform in {dlo}..{dhi} (numpy default_rng({seed}))",
           "nodes": npts, "geometry_degree": pm.Ngeo,
           "isotropic_elements": int(np.all(deg == deg[:, :1], axis=1).sum()),
           "scheme": f"{physics} {surface} surface, {volume} volume, rk3, mortars of degree max(P_L, P_R) "
                     f"per tangential direction"}
    stream = torch.cuda.current_stream()
    cfg = hs.solver_cfg(physics, surface, volume, "fp64", gamma=GAMMA, Re=RE, Pr=PR, Ma=MA, cfl=CFL)
    u = pm.init_state(pm.empty_state(), "tgv", GAMMA, MA)
    g = torch.zeros_like(u)
    pm.run(cfg, u, g, warmup)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    pm.run(cfg, u, g, steps, dt=-1.0)   # continuing the warm-up run: every timed step a graph replay
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    out["fp64"] = {"value": round(npts * 3 / (ms * 1e-3), 1), "ms_per_step": round(ms, 3)}
    del u, g, pm
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ serving (continuous batching)

def serving_requests(count, seed=0):
    """The batched-serving request stream: periodic cubes [0,10]^3 with E^3
    elements, E ~ U{4..24}, N ~ U{2..7}, isentropic vortex with centre ~
    U(box), strength ~ U[1,5], Mach ~ U[0.1,0.8], integrated to t = 1.0 at
    CFL 0.5; Poisson arrivals at 200 requests/s."""
    import numpy as np
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for _ in range(count):
        E = int(rng.integers(4, 25))
        N = int(rng.integers(2, 8))
        xc, yc = rng.uniform(0, 10, size=2)
        beta = float(rng.uniform(1, 5))
        Ma = float(rng.uniform(0.1, 0.8))
        t += float(rng.exponential(1 / 200.0))
        reqs.append(dict(E=E, N=N, xc=float(xc), yc=float(yc), beta=beta, Ma=Ma, arrival=t))
    return reqs


def serving_sample(reqs, t_final):
    """A stratified sample of the request stream: for every N in 2..7 and every
    third of the E range (4-10, 11-17, 18-24), the first request of the
    stream in that stratum (18 requests), each integrated to t_final."""
    picked = {}
    for k, r in enumerate(reqs):
        key = (r["N"], 0 if r["E"] <= 10 else 1 if r["E"] <= 17 else 2)
        if key not in picked:
            picked[key] = k
    return [dict(reqs[k], t_final=t_final) for k in sorted(picked.values())]


def serve(reqs, precision, mode, rate_scale=1.0, finals=None, launch_mode="grid"):
    """Run requests through one server.  mode "stream": submitted at their
    arrival times (rate_scale stretches them); "batch": all at once;
    "sequential": one at a time, each submitted when the previous finished
    (the library's single-solve path: graph replay, device dt, last step
    clipped at t_final, no host work per step).  Returns per-request
    (status, latency, t_done, t_submit, dof-stage updates) and the span."""
    import paper_2206_09733_gb300 as hs

    def descs(r):
        mesh = hs.mesh_desc(r["E"], r["E"], r["E"], r["N"], lo=(0, 0, 0), hi=(10, 10, 10))
        cfg = hs.solver_cfg("euler", "lf", "ec", precision, gamma=GAMMA, cfl=CFL)
        ic = hs.ic_desc("vortex", GAMMA, r["Ma"], r["beta"], r["xc"], r["yc"])
        return mesh, cfg, ic

    srv = hs.Server(launch_mode=launch_mode)
    m, c, i = descs(reqs[0])                      # warm-up: one short request
    t = srv.submit(m, c, i, t_final=0.05)
    while srv.poll(t)[0] == hs.PENDING:
        time.sleep(0.001)
    done = {}

    def wait(tk):
        while True:
            st, res = srv.poll(tk)
            if st != hs.PENDING:
                done[tk] = (st, res.t_done - res.t_submit, res.t_done, res.t_submit, res.dof * res.steps * 3)
                return
            time.sleep(0.0005)

    tickets = []
    t0 = time.perf_counter()
    for k, r in enumerate(reqs):
        if mode == "stream":
            while time.perf_counter() - t0 < r["arrival"] * rate_scale:
                time.sleep(0.0002)
        m, c, i = descs(r)
        res = finals[k] if finals is not None else None
        tickets.append(srv.submit(m, c, i, t_final=r.get("t_final", 1.0), result=res))
        if mode == "sequential":
            wait(tickets[-1])
    for tk in tickets:
        if tk not in done:
            wait(tk)
    srv.close()
    return [done[tk] for tk in tickets]


def serving_summary(rows, extra=None):
    import numpy as np
    ok = [v for v in rows if v[0] == 0]
    lat = np.array([v[1] for v in ok]) if ok else np.array([0.0])
    span = (max(v[2] for v in ok) - min(v[3] for v in ok)) if ok else 1.0
    out = {"requests": len(rows), "completed": len(ok), "solves_per_s": round(len(ok) / span, 3),
           "dof_stage_per_s": round(sum(v[4] for v in ok) / span, 1),
           "latency_p50_s": round(float(np.percentile(lat, 50)), 4),
           "latency_p99_s": round(float(np.percentile(lat, 99)), 4)}
    if extra:
        out.update(extra)
    return out


def run_serving(count, rate_scale=1.0, sample_t_final=0.25, baselines=True):
    """The batched server (mixed FP32 flux arithmetic, FP64 state) on `count`
    requests arriving as a Poisson stream, and, on a stratified sample of
    the stream, the same engine in four arms that separate the batching and
    precision effects: sequential FP64 per-solve, sequential mixed, batched
    FP64 and batched mixed (sample submitted at once), with the largest
    rel-L2 difference between the batched mixed final states and the
    sequential FP64 ones."""
    import numpy as np
    import paper_2206_09733_gb300 as hs
    reqs = serving_requests(count)
    designs = {}
    for launch_mode in ("grid", "persistent"):
        rows = serve(reqs, "mixed32", "stream", rate_scale, launch_mode=launch_mode)
        failed = {}
        for v in rows:
            if v[0] != hs.OK:
                nm = hs.STATUS_NAMES.get(v[0], str(v[0]))
                failed[nm] = failed.get(nm, 0) + 1
        designs[launch_mode] = serving_summary(
            rows, {"failed": failed, "arrivals": f"Poisson {200 / rate_scale:g} req/s",
                   "scheme": "Euler, LF + EC split form, mixed32, to t=1.0 at CFL 0.5",
                   "launch_design": launch_mode})
    out = dict(designs["grid"])
    out["launch_designs"] = {
        "grid": "a CTA per tile, binary search over the group's item table",
        "persistent": "work table (request of every element) + persistent grids walking the tiles",
        "persistent_run": designs["persistent"]}
    if not baselines:
        return out
    sample = serving_sample(reqs, sample_t_final)
    sizes = [r["E"] ** 3 * 5 * (r["N"] + 1) ** 3 for r in sample]
    fin = {}
    arms = {}
    for prec in ("fp64", "mixed32"):
        for mode in ("sequential", "batch"):
            fin[(prec, mode)] = [np.empty(n) for n in sizes]
            rows = serve(sample, prec, mode, finals=fin[(prec, mode)])
            arms[f"{mode}_{prec}"] = serving_summary(rows)
    ref = fin[("fp64", "sequential")]
    l2 = [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(fin[("mixed32", "batch")], ref)]
    l2b = [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(fin[("fp64", "batch")], ref)]
    out["sample"] = {"requests": len(sample), "t_final": sample_t_final,
                     "strata": "every N in 2..7 x every third of E in 4..24, the first request of each stratum",
                     "arms": arms,
                     "batching_gain_mixed": round(arms["batch_mixed32"]["solves_per_s"] /
                                                  arms["sequential_mixed32"]["solves_per_s"], 3),
                     "batching_gain_fp64": round(arms["batch_fp64"]["solves_per_s"] /
                                                 arms["sequential_fp64"]["solves_per_s"], 3),
                     "precision_gain_batched": round(arms["batch_mixed32"]["solves_per_s"] /
                                                     arms["batch_fp64"]["solves_per_s"], 3),
                     "server_mixed_vs_sequential_fp64": round(arms["batch_mixed32"]["solves_per_s"] /
                                                              arms["sequential_fp64"]["solves_per_s"], 3),
                     "l2_rel_batched_mixed_vs_sequential_fp64_max": max(l2),
                     "l2_rel_batched_fp64_vs_sequential_fp64_max": max(l2b)}
    return out


def stress_requests(count, seed=1, emax=64):
    """Memory-admission stress stream: NS Taylor-Green solves on E^3 curved
    cubes, E ~ U{16..emax}, N ~ U{3..6}, perturbation amplitude ~ U[0, 0.1],
    Re ~ U[400, 3200], 50 RK3 steps each, all submitted at once."""
    import numpy as np
    rng = np.random.default_rng(seed)
    return [dict(E=int(rng.integers(16, emax + 1)), N=int(rng.integers(3, 7)), amp=float(rng.uniform(0, 0.1)),
                 Re=float(rng.uniform(400, 3200))) for _ in range(count)]


def run_stress(count, budget_gb, emax, precision):
    """Submit the stress stream to a server whose device budget is smaller
    than the requests' total footprint; report throughput, queueing delay
    (admission - submission) and latency percentiles."""
    import numpy as np

    import paper_2206_09733_gb300 as hs
    reqs = stress_requests(count, emax=emax)
    budget = int(budget_gb * 2 ** 30)
    srv = hs.Server(hbm_budget_bytes=budget)        # 0: the library takes 90% of the free device memory
    if budget == 0:
        free, _ = __import__("torch").cuda.mem_get_info()
        budget = int(0.9 * free)
    tickets, total_bytes = [], 0
    t0 = time.perf_counter()
    for r in reqs:
        m = hs.mesh_desc(r["E"], r["E"], r["E"], r["N"], lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=r["amp"])
        c = hs.solver_cfg("ns", "roe", "ec", precision, gamma=GAMMA, Re=r["Re"], Pr=PR, Ma=MA, cfl=CFL)
        i = hs.ic_desc("tgv", GAMMA, MA)
        tickets.append(srv.submit(m, c, i, n_steps=50))
    peak = 0
    res = {}
    while len(res) < len(tickets):
        peak = max(peak, srv.stats()["bytes_in_use"])
        for t in tickets:
            if t not in res:
                st, rr = srv.poll(t)
                if st != hs.PENDING:
                    res[t] = (st, rr.t_submit, rr.t_admit, rr.t_done, rr.dof * rr.steps * 3, rr.device_bytes)
        time.sleep(0.002)
    wall = time.perf_counter() - t0
    srv.close()
    ok = [v for v in res.values() if v[0] == hs.OK]
    total_bytes = sum(v[5] for v in res.values())
    lat = np.array([v[3] - v[1] for v in ok])
    wait = np.array([v[2] - v[1] for v in ok])
    return {"requests": count, "completed": len(ok), "precision": precision,
            "budget_bytes": budget, "sum_of_footprints_bytes": total_bytes, "peak_bytes_in_use": peak,
            "dof_stage_per_s": round(sum(v[4] for v in ok) / wall, 1), "solves_per_s": round(len(ok) / wall, 3),
            "queueing_delay_p50_s": round(float(np.percentile(wait, 50)), 3),
            "queueing_delay_p99_s": round(float(np.percentile(wait, 99)), 3),
            "latency_p50_s": round(float(np.percentile(lat, 50)), 3),
            "latency_p99_s": round(float(np.percentile(lat, 99)), 3),
            "scheme": f"NS TGV, Roe + EC split form + BR1, 50 steps, E in 16..{emax}, N in 3..6"}


# ------------------------------------------------------------------ the oracle on the host cores

def rel_errors(a, b):
    """rel-L2 = |a - b|_2 / |b|_2 over all nodes and variables; rel-Linf =
    max |a - b| / max |b|."""
    import numpy as np
    d = np.asarray(a) - np.asarray(b)
    return {"l2_rel": float(np.linalg.norm(d) / np.linalg.norm(b)),
            "linf_rel": float(np.abs(d).max() / np.abs(b).max())}


def cpu_baseline(finals=None, compare_steps=0, budget_s=15.0):
    """Time the FP64 CPU oracle (as it stands) on this workload: RK3 steps
    from the initial condition until ~budget_s of CPU work (at most 200).
    finals: {precision: host state of the GPU path after compare_steps RK3
    steps from the same initial condition}; each is compared with the
    oracle's state after the same number of steps (each side with its own
    CFL time step)."""
    import numpy as np

    import oracle as O
    om = O.Mesh(EX, EY, EZ, N, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=AMP)
    oc = O.Cfg("ns", "roe", "ec", gamma=GAMMA, Re=RE, Pr=PR, cfl=CFL)
    u = om.ic_tgv(GAMMA, MA)
    g = np.zeros_like(u)
    steps = 0
    t_sim = 0.0
    errors = None
    t0 = time.perf_counter()
    while True:
        t_sim += om.rk3_step(oc, u, g)
        steps += 1
        if finals and steps == compare_steps:
            errors = {"steps": steps, "oracle_sim_time": t_sim,
                      "how": "GPU state after W+K RK3 steps vs the FP64 CPU oracle after as many steps from the "
                             "same initial condition (each with its own CFL time step)"}
            for prec, a in finals.items():
                errors[prec] = rel_errors(a, u)
        el = time.perf_counter() - t0
        if (el > budget_s and steps >= compare_steps) or steps >= max(200, compare_steps):
            break
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": round(NODES * 3 * steps / el, 1), "unit": "DOF-stage-updates/s", "cores": cores,
           "kind": "oracle", "sample": f"{steps} RK3 steps of the full 16^3 N=3 workload from t=0 "
                                       f"({el:.1f} s, OpenMP over elements)"}
    # the same oracle on one thread (a fresh process, so that OpenMP starts with one thread)
    code = ("import os, sys, time, numpy as np; sys.path.insert(0, %r); import oracle as O; "
            "om = O.Mesh(%d, %d, %d, %d, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=%r); "
            "oc = O.Cfg('ns', 'roe', 'ec', gamma=%r, Re=%r, Pr=%r, cfl=%r); u = om.ic_tgv(%r, %r); g = np.zeros_like(u); "
            "t0 = time.perf_counter(); om.rk3_step(oc, u, g); om.rk3_step(oc, u, g); "
            "print(time.perf_counter() - t0)" % (ROOT, EX, EY, EZ, N, AMP, GAMMA, RE, PR, CFL, GAMMA, MA))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                           env=dict(os.environ, OMP_NUM_THREADS="1"))
        el1 = float(r.stdout.strip().splitlines()[-1])
        out["single_thread"] = {"value": round(NODES * 3 * 2 / el1, 1), "cores": 1,
                                "sample": f"2 RK3 steps of the same workload ({el1:.1f} s)"}
    except (subprocess.SubprocessError, ValueError, IndexError) as exc:
        out["single_thread"] = {"unavailable": str(exc)[:200]}
    return out, errors


def run_reference(args, world, rank):
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    O.build()
    om = O.Mesh(EX, EY, EZ, N, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=AMP)
    oc = O.Cfg("ns", "roe", "ec", gamma=GAMMA, Re=RE, Pr=PR, cfl=CFL)
    u = om.ic_tgv(GAMMA, MA)
    g = np.zeros_like(u)
    for _ in range(args.warmup):
        om.rk3_step(oc, u, g)
    # each timed step is one full oracle RK3 step; cap the run near two minutes
    K = args.steps
    t0 = time.perf_counter()
    done = 0
    for _ in range(K):
        om.rk3_step(oc, u, g)
        done += 1
        if time.perf_counter() - t0 > 120.0:
            break
    el = time.perf_counter() - t0
    val = NODES * 3 * done / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 1), "unit": "DOF-stage-updates/s",
            "n_gpus": world, "steps": done, "warmup": args.warmup, "ms_per_step": round(el * 1e3 / done, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (analytic Taylor-Green initial condition)",
            "config": {"workload": WORKLOAD, "E": EX * EY * EZ, "N": N, "nodes": NODES},
            "cpu_baseline": {"value": round(val, 1), "unit": "DOF-stage-updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"{done} full RK3 steps (of {K} requested) after {args.warmup} warm-up steps"},
            "e2e": {"value": round(val, 1), "unit": "DOF-stage-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def pmesh_profile(E):
    """The p-mesh kernels alone, for an ncu launch list or capture: mesh set-up,
    one initial condition and 3 mixed RK3 steps (per stage 4 + 4 mortar
    launches, one gradient and one element kernel per degree)."""
    import numpy as np
    import torch

    import paper_2206_09733_gb300 as hs
    deg = np.random.default_rng(7).integers(2, 6, size=E ** 3).astype(np.int32)
    pm = hs.PMesh(E, E, E, deg, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=AMP)
    cfg = hs.solver_cfg("ns", "roe", "ec", "mixed32", gamma=GAMMA, Re=RE, Pr=PR, Ma=MA, cfl=CFL)
    u = pm.init_state(pm.empty_state(), "tgv", GAMMA, MA)
    g = torch.zeros_like(u)
    pm.run(cfg, u, g, 3)
    torch.cuda.synchronize()
    print(json.dumps({"pmesh_profile": E, "clock": pm.clock()}))


def aniso_profile(E):
    """The anisotropic-degree kernels alone, for an ncu launch list or
    capture: mesh set-up, one initial condition and 2 FP64 RK3 steps (per
    stage two mortar launches, then the gradient and element kernels of
    every node-count class)."""
    import numpy as np
    import torch

    import paper_2206_09733_gb300 as hs
    deg = np.random.default_rng(7).integers(2, 6, size=(E ** 3, 3)).astype(np.int32)
    pm = hs.PMesh(E, E, E, deg, lo=(-np.pi,) * 3, hi=(np.pi,) * 3, amp=AMP)
    cfg = hs.solver_cfg("ns", "roe", "ec", "fp64", gamma=GAMMA, Re=RE, Pr=PR, Ma=MA, cfl=CFL)
    u = pm.init_state(pm.empty_state(), "tgv", GAMMA, MA)
    g = torch.zeros_like(u)
    pm.run(cfg, u, g, 2)
    torch.cuda.synchronize()
    print(json.dumps({"aniso_profile": E, "clock": pm.clock()}))


def main():
    args = parse()
    if args.pmesh_profile:
        pmesh_profile(args.pmesh_profile)
        return
    if args.aniso_profile:
        aniso_profile(args.aniso_profile)
        return
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_hs3d(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
