"""Benchmark of the hybrid LB step (MLUPS and fraction of the HBM roofline).

Workload: one 3D active cholesteric droplet, 128^3 periodic box, R = 32, pitch 32,
zeta = 0.005 (A0 = 1, chi_in = 3, K = 0.04, Gamma_Q = 0.3, xi = 0.7, a = b = 0.07,
M = 0.1, tau = 1), FP32 with populations shifted by w_i rho0; synthetic seeded initial
state (tanh droplet, cholesteric helix + 1e-3 noise).  The plain FP64 GPU path is timed
on the same workload for the FP32/FP64 speedup.

One JSON line on rank 0.  `value` is whole-job site updates per second (MLUPS) with the
state resident in HBM; `e2e` is the same metric through the public API with host
buffers (state uploaded and read back every step).  `--impl reference` times the FP64
CPU oracle on the host cores instead.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hybrid-step MLUPS & % of HBM roofline, FP32 vs plain FP64 at stated error"
BYTES_PER_SITE = {"fp32": 200, "fp64": 400}
# fused-step schedules offered to the autotuner, in candidate order
TILE_NAMES = ["32x8", "32x16", "64x8", "32x8-pipelined-8+8", "32x8-pipelined-6+10", "32x6-pipelined-9+7",
              "32x6-pipelined-10+6"]


def workload_params(L, n, prec, **kw):
    kw.setdefault("zeta", 0.005)
    return L.default_params((n, n, n), R=n / 4.0, p0=n / 4.0, precision=prec, **kw)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources that define the step kernels: an ncu figure is current only while these are
# unchanged since the capture (the profile records their fingerprint)
STEP_SOURCES = ["lbcad_fused.cuh", "lbcad_kernels.cuh", "lbcad_internal.h", "lbcad_f32.cu"]
STEP_SOURCES_FP64 = ["lbcad_fused.cuh", "lbcad_kernels.cuh", "lbcad_internal.h", "lbcad_f64.cu"]


def kernel_source_sha(sources=None):
    import hashlib
    h = hashlib.sha256()
    for f in sources or STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2011_00287_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_is_current(name="lbcad_step_fp32_128cube.md", sources=None):
    """True when the committed ncu summary was taken of the kernels as they are now."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return False
    for line in open(p):
        if line.startswith("kernel_source_sha:"):
            return line.split(":", 1)[1].strip().split()[0] == kernel_source_sha(sources)
    return False


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def measured_alu_peaks(device=0):
    """FP64 and FP32 dense FMA throughput of this GPU (TFLOP/s), measured by the FMA-chain
    probe (csrc/peaks.cu); None where the probe fails."""
    import ctypes
    from paper_2011_00287_gb300 import build as B
    try:
        lib = ctypes.CDLL(B.PEAKS_LIB)
    except OSError:
        return None, None
    out = []
    for fn, iters in ((lib.peak_fp64_tflops, 256), (lib.peak_fp32_tflops, 8192)):
        fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        v = ctypes.c_double()
        out.append(v.value if fn(device, iters, ctypes.byref(v)) == 0 else None)
    return out[0], out[1]


def add_latencies(device=0):
    """Cycles of one dependent FP64 and FP32 addition on this GPU (chain probe, csrc/peaks.cu)."""
    import ctypes
    from paper_2011_00287_gb300 import build as B
    try:
        lib = ctypes.CDLL(B.PEAKS_LIB)
    except OSError:
        return None
    out = {}
    for name, fn in (("fp64", lib.add_latency_fp64_cycles), ("fp32", lib.add_latency_fp32_cycles)):
        fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        v = ctypes.c_double()
        out[name] = v.value if fn(device, ctypes.byref(v)) == 0 else None
    return out


def committed_profile_value(key, name="lbcad_step_fp32_128cube.md"):
    """A figure ('key: value ...') from a committed ncu summary of the step."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith(key + ":"):
            try:
                return float(line.split(":", 1)[1].split()[0])
            except ValueError:
                return None
    return None


def committed_traffic():
    """DRAM bytes per site-update of the step kernels from the committed ncu summary."""
    return committed_profile_value("traffic_bytes_per_site")


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, dist, device="cuda"):
    """Max of a per-rank number (the step time) over all ranks."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist, device="cuda"):
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_mlups(sites, world, ms):
    """Site updates per second of all ranks (each advances `sites`) per step time `ms`."""
    return world * sites / (ms * 1e-3) / 1e6


def time_steps(sim, torch, K):
    """Device time of K steps on the library's stream (CUDA events), ms per step."""
    st = sim.torch_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sim.sync()
    torch.cuda.synchronize()
    e0.record(st)
    sim.step(K)
    e1.record(st)
    e1.synchronize()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / K


def cpu_oracle_rate(n, budget_s=12.0, max_steps=None, omp=False):
    """Oracle site updates per second on a bounded sample of the workload (1 thread, or all
    host cores with the oracle's OpenMP build)."""
    from oracle import oracle as O
    O.build(omp=omp)
    p = O.default_params((n, n, n), R=n / 4.0, p0=n / 4.0, zeta=0.005)
    s = O.State((n, n, n), p, seed=1, omp=omp)
    steps, t0 = 0, time.perf_counter()
    while True:
        s.step(1)
        s.observables()  # a6 of every step, as the GPU step forms them
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps and steps >= max_steps):
            break
    return n ** 3 * steps / el, steps, el


def config0_leg(L, torch, local):
    """The small workload in full: FP64 droplet 32^3, R = 8, pitch 16, 200 steps with the a6 sums of
    every step, on the oracle (one thread, and all cores) and on the GPU's FP64 path."""
    from oracle import oracle as O
    n, K = 32, 200
    out = {"workload": "droplet 32^3, R = 8, pitch 16, zeta = 0.005, FP64, %d steps, a6 sums every step" % K}
    for omp in (False, True):
        O.build(omp=omp)
        s = O.State((n, n, n), O.default_params((n, n, n), R=8.0, p0=16.0, zeta=0.005), seed=1, omp=omp)
        t0 = time.perf_counter()
        for _ in range(K):
            s.step(1)
            s.observables()
        el = time.perf_counter() - t0
        out["oracle_all_cores" if omp else "oracle_single_thread"] = {
            "seconds": el, "mlups": n ** 3 * K / el / 1e6, "threads": O.num_threads(True) if omp else 1}
    sim = L.Simulation([(n, n, n)], [L.default_params((n, n, n), R=8.0, p0=16.0, precision=L.FP64, zeta=0.005)],
                       seed=1, device=local)
    sim.step(3)
    ms = time_steps(sim, torch, K)
    out["gpu_fp64"] = {"seconds": ms * K / 1e3, "mlups": n ** 3 / (ms * 1e-3) / 1e6}
    sim.close()
    return out


def run_reference(args):
    """--impl reference: the FP64 CPU oracle, as it stands, on all of this host's cores (its
    OpenMP build: the same per-site arithmetic, stage loops split over z)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    from oracle import oracle as O
    O.build(omp=True)
    threads = O.num_threads(True)
    K, W = args.steps, args.warmup
    # each step is one oracle step on the largest droplet box (same workload family,
    # R = n/4, pitch n/4) whose K + W steps fit in about two minutes
    rate_probe, _, _ = cpu_oracle_rate(32, budget_s=1.0, omp=True)
    n = 32
    for cand in (128, 96, 64, 48, 32):
        if cand ** 3 * (K + W) / rate_probe <= 120.0:
            n = cand
            break
    p = O.default_params((n, n, n), R=n / 4.0, p0=n / 4.0, zeta=0.005)
    s = O.State((n, n, n), p, seed=1, omp=True)
    s.step(W)
    t0 = time.perf_counter()
    for _ in range(K):  # each step with its a6 sums, as the GPU step forms them
        s.step(1)
        s.observables()
    el = time.perf_counter() - t0
    mlups = n ** 3 * K / el / 1e6
    sample = ("oracle FP64 on %d threads (OpenMP over z in each stage loop), %d^3 droplet (R=%d, pitch %d), %d "
              "timed steps (each with its conserved and centroid sums) after %d warm-up") % (
                  threads, n, n // 4, n // 4, K, W)
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": 1, "steps": K,
            "warmup": W, "ms_per_step": el / K * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "active cholesteric droplet %d^3 (CPU sample of 128^3, R=32, pitch 32)" % n,
                       "box": [n, n, n]},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batch_leg(torch, L, steps=100, warmup=3):
    """64 independent droplets (edges from {48, 64, 80, 96}, seed 7) advanced together by one
    persistent launch per step, replayed from a CUDA graph: aggregate MLUPS."""
    from paper_2011_00287_gb300 import workloads as WL
    work = WL.batch_uneven(seed=7, count=64)
    prms = [L.default_params(w["grid"], R=w["R"], p0=w["p0"], zeta=w["zeta"], precision=L.FP32) for w in work]
    sim = L.Simulation([w["grid"] for w in work], prms, seed=7)
    cfg, tms = sim.autotune(3)
    sim.set_graph(50)
    sim.step(max(warmup, 3))
    K = max(50, (steps // 50) * 50)
    with ClockSampler(0) as clk:
        ms = time_steps(sim, torch, K)
    sites = sim.sites()
    out = {"mlups": sites / (ms * 1e-3) / 1e6, "ms_per_step": ms, "steps": K, "sites": sites,
           "tiles": {"chosen": TILE_NAMES[cfg], "ms_per_cfg": dict(zip(TILE_NAMES, tms))},
           "workload": "64 droplets, edges from {48,64,80,96}, R = edge/4, zeta in [0.001, 0.01], pitch in "
                       "[12, 40], seed 7, FP32, one launch per step replayed from a CUDA graph, a6 sums fused",
           "clocks": clk.summary()}
    sim.close()
    return out


def run_batch(args):
    """--workload batch64: the batched leg alone, as its own JSON line."""
    import torch
    import paper_2011_00287_gb300 as L
    from paper_2011_00287_gb300 import build as B
    B.build()
    b = batch_leg(torch, L, args.steps, args.warmup)
    print(json.dumps({"metric": METRIC + " (batched 64 uneven droplets)", "value": b["mlups"], "unit": "MLUPS",
                      "n_gpus": 1, "steps": b["steps"], "ms_per_step": b["ms_per_step"], "sites": b["sites"],
                      "dtype": "f32", "data": "synthetic", "tiles": b["tiles"],
                      "config": {"workload": b["workload"]}, "clocks": b["clocks"]}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lbcad", choices=["lbcad", "reference"])
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--tiles", type=int, default=None,
                    help="fixed fused tile shape (index into the autotuner's candidates) instead of autotuning")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-staged", action="store_true",
                    help="skip the sync / Heun, LB-variant and bulk legs")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg (64^3, 500 steps)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-droplet leg")
    ap.add_argument("--no-large", action="store_true", help="skip the 256^3 droplet leg")
    ap.add_argument("--min-timed-s", type=float, default=1.0,
                    help="repeat the K-step timed region until this much device time has passed")
    ap.add_argument("--workload", default="droplet", choices=["droplet", "batch64"],
                    help="droplet: the 128^3 benchmark line; batch64: 64 uneven droplets in one launch")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)

    import torch
    import paper_2011_00287_gb300 as L
    from paper_2011_00287_gb300 import build as B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    B.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    n = args.size
    N = n ** 3
    K, W = args.steps, args.warmup
    # replicas: each rank advances its own copy of the workload (weak scaling)
    sim = L.Simulation([(n, n, n)], [workload_params(L, n, L.FP32)], seed=1 + rank, device=local)
    if args.tiles is None:
        tile_cfg, tile_ms = sim.autotune(5)
    else:  # a fixed tile shape (profiling runs): no autotuning launches
        sim.set_tiles(args.tiles)
        tile_cfg, tile_ms = args.tiles, [None] * len(TILE_NAMES)
    sim.step(W)
    sim.sync()
    if dist:
        dist.barrier()
    # every timed step is the whole hot path: stencils, fields, stress and force, the order-
    # parameter update, the LB collision and streaming, and the FP64 conserved and centroid
    # sums of the new state (fused into the same kernel; the library default).  The region of
    # exactly K steps is timed repeatedly (the same count on every rank) until about a second of
    # device time has passed, so that the clock sampler sees it; the step time is the median.
    ms_probe = time_steps(sim, torch, K)
    reps = max(1, int(math.ceil(args.min_timed_s / max(K * ms_probe * 1e-3, 1e-9))))
    if dist:
        reps = int(max_over_ranks(reps, dist))
    region_ms = []
    with ClockSampler(local) as clk:
        for _ in range(reps):
            if dist:
                dist.barrier()
            region_ms.append(time_steps(sim, torch, K))
    ms = statistics.median(region_ms)
    if dist:
        ms = max_over_ranks(ms, dist)
    obs = sim.observables(0)
    finite = all(math.isfinite(v) for v in obs)
    value = whole_job_mlups(N, world, ms)
    # the same step kernel without the sums (for runs that read observables rarely; each
    # read then costs a separate pass)
    sim.set_observe(False)
    sim.step(3)
    ms_nosums = time_steps(sim, torch, min(K, 1000))
    sim.set_observe(True)
    sim.step(1)
    without_sums = {"mlups": whole_job_mlups(N, world, ms_nosums), "ms_per_step": ms_nosums,
                    "note": "same step kernel without the fused FP64 sums (lbcad_set_observe(0))"}

    # plain FP64 GPU path on the same workload
    fp64 = None
    if not args.no_fp64:
        s64 = L.Simulation([(n, n, n)], [workload_params(L, n, L.FP64)], seed=1 + rank, device=local)
        s64.step(3)
        ms64 = time_steps(s64, torch, args.fp64_steps)
        fp64 = {"mlups": N / (ms64 * 1e-3) / 1e6, "ms_per_step": ms64, "steps": args.fp64_steps}
        # bound by the FP64 pipe: flops per site from the committed ncu counters, peak the FP64
        # FMA throughput measured on this GPU by the FMA-chain probe
        fp64_current = profile_is_current("lbcad_step_fp64_128cube.md", STEP_SOURCES_FP64)
        fl = committed_profile_value("fp64_flops_per_site", "lbcad_step_fp64_128cube.md") if fp64_current else None
        p64, p32 = measured_alu_peaks(local)
        fp64["measured_peak_tflops"] = {"fp64": p64, "fp32": p32,
                                        "how": "FMA-chain probe (csrc/peaks.cu), best of 5 launches on every SM"}
        fp64["add_latency_cycles"] = add_latencies(local)
        if fl and p64:
            ach = fl * N / (ms64 * 1e-3) / 1e12
            fp64["roofline"] = {"bound": "alu", "achieved": ach, "peak": p64, "unit": "TFLOP/s", "frac": ach / p64,
                                "peak_kind": "measured DFMA throughput of this GPU", "flops_per_site": fl,
                                "fp64_pipe_active_pct": committed_profile_value(
                                    "fp64_pipe_active_pct", "lbcad_step_fp64_128cube.md")}
        s64.close()

    # Sec. 3's sync coupling and predictor-corrector on the same workload, on the fused split
    # (the LB half in the fused kernel, then the order-parameter kernels) and on the staged path
    staged = None
    if not args.no_staged:
        staged = {}
        for name, integ, coup, path, launches in (
                ("euler_sync", L.EULER, L.SYNC, "fused LB half + order-parameter kernel", 2),
                ("euler_sync_staged", L.EULER, L.SYNC, "staged", 3),
                ("heun_sync", L.HEUN, L.SYNC, "fused LB half + predictor, fields, corrector", 4),
                ("heun_sync_staged", L.HEUN, L.SYNC, "staged", 5)):
            sv = L.Simulation([(n, n, n)], [workload_params(L, n, L.FP32, integrator=integ, coupling=coup)],
                              seed=1 + rank, device=local)
            if path == "staged":
                sv.set_path(L.lbcad.PATH_STAGED)
            sv.step(3)
            msv = time_steps(sv, torch, 20)
            staged[name] = {"mlups": N / (msv * 1e-3) / 1e6, "ms_per_step": msv, "kernels_per_step": launches,
                            "path": path}
            sv.close()

    # the other LB variants of Sec. 3 on the same workload: D3Q15 and the Eq. 9-11 form on the
    # fused kernels (autotuned over their two tile shapes), each at a tau where it is stable
    # on the droplet; the radius-2 stencils on the staged path
    variants = None
    if not args.no_staged:
        variants = {}
        for name, kw, steps in (("d3q15", dict(lattice=L.D3Q15, tau=1.0), 100),
                                ("stress_eq", dict(lb_form=L.LB_STRESS_EQ, tau=1.5), 100),
                                ("d3q15_stress_eq", dict(lattice=L.D3Q15, lb_form=L.LB_STRESS_EQ, tau=2.5), 50),
                                ("r2_stencils", dict(stencil=L.STENCIL_R2), 20)):
            sv = L.Simulation([(n, n, n)], [workload_params(L, n, L.FP32, **kw)], seed=1 + rank, device=local)
            cfg = None
            if name != "r2_stencils":
                cfg, _ = sv.autotune(3)
            sv.step(3)
            msv = time_steps(sv, torch, steps)
            variants[name] = {"mlups": N / (msv * 1e-3) / 1e6, "ms_per_step": msv, "tau": kw["tau"] if "tau" in kw else 1.0,
                              "path": "staged" if cfg is None else "fused " + TILE_NAMES[cfg]}
            sv.close()

    # second workload: bulk active nematic (no droplet, psi = 1), same kernel and schedule
    bulk = None
    if not args.no_staged:
        from paper_2011_00287_gb300 import workloads as WL
        sb = L.Simulation([(n, n, n)], [workload_params(L, n, L.FP32, zeta=0.008, q0=0.0)], seed=1 + rank,
                          device=local)
        sb.set_fields(0, WL.bulk_order((n, n, n), q0=0.0, noise=1e-3, seed=3))
        sb.set_tiles(tile_cfg)
        sb.step(3)
        msb = time_steps(sb, torch, 200)
        bulk = {"mlups": N / (msb * 1e-3) / 1e6, "ms_per_step": msb,
                "workload": "bulk active nematic %d^3, psi = 1, zeta = 0.008 (spontaneous-flow regime)" % n}
        sb.close()

    # the larger droplet workload: 256^3, R = 64, pitch 48, FP32 with the fused sums (the step of the
    # 128^3 line at 8x the sites)
    large = None
    if not args.no_large and world == 1:
        nl = 256
        sl = L.Simulation([(nl, nl, nl)], [L.default_params((nl, nl, nl), R=64.0, p0=48.0, precision=L.FP32,
                                                            zeta=0.005)], seed=1 + rank, device=local)
        sl.set_tiles(tile_cfg)
        sl.step(3)
        msl = time_steps(sl, torch, 50)
        ach = BYTES_PER_SITE["fp32"] * nl ** 3 / (msl * 1e-3) / 1e9
        pk, _ = measured_peaks()
        large = {"mlups": nl ** 3 / (msl * 1e-3) / 1e6, "ms_per_step": msl, "achieved_gbs": ach,
                 "frac_of_hbm_roofline": ach / pk if pk else None,
                 "workload": "droplet 256^3, R = 64, pitch 48, zeta = 0.005, FP32, a6 sums fused, %s" %
                             TILE_NAMES[tile_cfg]}
        sl.close()

    # adjoint of J = |centroid drift|^2 / 2 over 500 steps of a 64^3 droplet (R = 16, pitch 16),
    # checkpoints every 50 steps: wall time of the whole gradient against the forward run alone
    adjoint = None
    if not args.no_adjoint:
        na = 64
        pa = L.default_params((na, na, na), R=16.0, p0=16.0, precision=L.FP32, zeta=0.005)
        sf = L.Simulation([(na, na, na)], [pa], seed=1 + rank, device=local)
        sf.step(5)
        sf.sync()
        t0 = time.perf_counter()
        sf.step(500)
        sf.sync()
        t_fwd = time.perf_counter() - t0
        sf.close()
        sa = L.Simulation([(na, na, na)], [pa], seed=1 + rank, device=local)
        sa.adjoint(20, 10)  # warm-up (allocations)
        t0 = time.perf_counter()
        Ja, dz, dq, _ = sa.adjoint(500, 50)
        t_adj = time.perf_counter() - t0
        sa.close()
        adjoint = {"workload": "droplet 64^3, R = 16, pitch 16, 500 steps, checkpoints every 50, FP32",
                   "seconds": t_adj, "forward_seconds": t_fwd, "ratio_to_forward": t_adj / t_fwd,
                   "site_steps_per_s": na ** 3 * 500 / t_adj, "dJ_dzeta": dz, "finite": bool(math.isfinite(dz))}

    # batched sweep: 64 uneven droplets in one launch per step (CUDA graph)
    batch = None
    if not args.no_batch and world == 1:
        batch = batch_leg(torch, L)

    # end to end through the public API with host buffers: every step sets the whole state
    # from pinned host memory (lbcad_set_state, the storage precision), advances one step and
    # reads the whole state back (lbcad_get_state)
    e2e = None
    if not args.no_e2e:
        nb = sim.state_bytes(0)
        host_in = torch.empty(nb, dtype=torch.uint8).pin_memory()
        host_out = torch.empty(nb, dtype=torch.uint8).pin_memory()
        sim.get_state(0, out=host_in)
        sim.set_state(0, host_in)
        sim.step(1)
        sim.get_state(0, out=host_out)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            sim.set_state(0, host_in)
            sim.step(1)
            sim.get_state(0, out=host_out)
        el = time.perf_counter() - t0
        e2e = {"value": N * args.e2e_steps / el / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb,
               "note": "per step: whole state (populations, Q, psi, u in the storage precision, FP32) set from "
                       "pinned host memory, one step, whole state read back to pinned host memory"}

    peak, peak_kind = measured_peaks()
    achieved = BYTES_PER_SITE["fp32"] * N / (ms * 1e-3) / 1e9
    current = profile_is_current()
    traffic_site = committed_traffic() if current else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (traffic_site * N) if traffic_site else None,
                "kernel": "k_step_pipe (one launch = one whole hybrid step, a6 sums included)",
                "algorithmic_bytes_per_site": 200,
                "peak_kind": peak_kind,
                # the design floor also moves u in and out (224 B per site)
                "design_bytes_per_site": 224, "design_frac": 224 * N / (ms * 1e-3) / 1e9 / peak,
                "ncu_dram_throughput_pct": committed_profile_value("dram_throughput_pct") if current else None,
                "ncu_fma_pipe_active_pct": committed_profile_value("fma_pipe_active_pct") if current else None,
                "ncu_capture_current": current}

    # the bound the step actually meets: warp-instruction issue (one per cycle per SM
    # sub-partition, 4 per SM, 152 SMs) at the SM clock sampled during the timed region
    ipsite = committed_profile_value("warp_instructions_per_site") if current else None
    csum = clk.summary()
    roofline_issue = None
    if ipsite and csum.get("sm_mhz"):
        peak_i = 152 * 4 * csum["sm_mhz"] * 1e6
        ach_i = ipsite * N / (ms * 1e-3)
        roofline_issue = {"bound": "issue", "achieved": ach_i / 1e12, "peak": peak_i / 1e12,
                          "unit": "T warp-instructions/s", "frac": ach_i / peak_i,
                          "warp_instructions_per_site": ipsite}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        from oracle import oracle as O
        threads = O.num_threads(True)
        rate_n, steps_n, el_n = cpu_oracle_rate(n, budget_s=10.0, omp=True)
        rate, steps, el = cpu_oracle_rate(n, budget_s=10.0)
        cpu = {"value": rate_n / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": "FP64 oracle on %d threads (OpenMP over z in each stage loop), %d step(s) of the same %d^3 "
                         "droplet workload, each with its a6 sums (%.1f s)" % (threads, steps_n, n, el_n),
               "nproc": os.cpu_count(), "cpu_model": cpu_model(),
               "single_thread": {"value": rate / 1e6, "unit": "MLUPS", "cores": 1,
                                 "sample": "FP64 oracle, single thread, %d step(s) of the same workload (%.1f s)" % (
                                     steps, el)},
               "small_workload_in_full": config0_leg(L, torch, local)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "active cholesteric droplet 128^3, R=32, pitch 32, zeta=0.005, FP32 "
                                       "shifted populations" if n == 128 else "droplet %d^3" % n,
                           "box": [n, n, n], "parallelism": "replicas" if world > 1 else "single",
                           "l2": "state %.0f MB per step > 129 MB L2, no flush" % (224 * N / 1e6),
                           "a6": "FP64 mass, psi, momentum and centroid sums of every step, fused"},
                "roofline": roofline, "roofline_issue": roofline_issue, "cpu_baseline": cpu, "e2e": e2e,
                "tiles": {"chosen": TILE_NAMES[tile_cfg], "ms_per_cfg": dict(zip(TILE_NAMES, tile_ms))},
                "timing": {"regions": len(region_ms), "steps_per_region": K, "median_ms_per_step": ms,
                           "min_ms_per_step": min(region_ms), "max_ms_per_step": max(region_ms)},
                "gpu_launches": K, "clocks": csum, "batch64": batch, "step_without_sums": without_sums, "fp64_gpu": fp64, "integrators_fp32": staged, "lb_variants_fp32": variants, "bulk_fp32": bulk, "droplet_256_fp32": large, "adjoint_fp32": adjoint,
                "speedup_fp32_vs_fp64": (value / world / fp64["mlups"]) if fp64 else None,
                "observables_finite": finite}
        print(json.dumps(line))
    sim.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
