#!/usr/bin/env python3
"""Throughput of the porous lattice Boltzmann time step on one GB300.

Workload (default): the shale matrix with fractures, 4096 x 4096 D2Q9
lattice, matrix eps ~ U(0.05, 0.1), log10 k_i ~ N(-6, 0.3), 40 straight
fractures (eps 0.9, k_i 1e-2), Kn from the local pressure (0.5 at the
inlet), pressure-driven in x (rho 1.0005 -> 0.9995), periodic in y,
tau 0.8, Forchheimer drag on.  FP32-stored populations are the headline;
the FP16-stored run is reported beside it.

One JSON line on rank 0:
  value     lattice updates per second (GLUPS) of ``lbmp_step`` with the
            lattice resident in HBM (1.3 GB FP32 working set >> 129 MB L2);
            the median of five timed regions of K steps
  e2e       the same metric through the public API from host buffers:
            lbmp_set_fields from host arrays + K steps + lbmp_permeability
  roofline  the fused step kernel against the measured HBM copy bandwidth
            (and the data-sheet figure)
  cpu_baseline  the FP64 CPU oracle on the host cores, on a bounded sample,
            and on one core
  k_g_vs_oracle  k_g of FP32 and FP16 storage against the oracle's, on the
            oracle's own run (a crop of the workload from rest)
  adjoint   one gradient of k_g (lbmp_permeability_gradient) over 20000
            steps of the 1024^2 two-component medium, with its backward
            sweep against the HBM roofline
  batch     a subset of the batched sweep (two-component media of uneven
            sizes x Knudsen numbers), FP16 and FP32, tuned launch shape

``--impl reference`` times the FP64 CPU oracle instead (the reference arm).
With torchrun and N > 1 ranks every rank runs an independent replica (the
step needs no exchange between replicas); the value is the sum of their
lattice updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9 porous-LBM GLUPS & %HBM peak, FP32 vs FP16-stored at <=1e-3 k_a err"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0   # HBM3e of a GB300, the data-sheet figure


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--storage", choices=["fp32", "fp16"], default=None,
                    help="storage of the headline value (default fp32; fp16 for the batch "
                         "workload); the other one is reported beside it")
    ap.add_argument("--no-other", action="store_true", help="skip the second storage run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--fp16-rounding", choices=["stochastic", "nearest"], default="stochastic")
    ap.add_argument("--workload", choices=["shale", "batch", "adjoint"], default="shale",
                    help="shale: the 4096^2 fractured shale (default); batch: the batched sweep "
                         "of two-component media of uneven sizes x Knudsen numbers; adjoint: "
                         "gradient of k_g on the 1024^2 two-component medium (a step is one "
                         "gradient evaluation)")
    ap.add_argument("--adjoint-steps", type=int, default=20000,
                    help="time steps of the run the adjoint differentiates")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint object of the default line")
    ap.add_argument("--no-dynamic", action="store_true",
                    help="skip the dynamic-Kn object of the default line")
    ap.add_argument("--batch-media", type=int, default=256)
    ap.add_argument("--batch-kn", type=int, default=8)
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-sweep object of the default line")
    ap.add_argument("--batch-object-media", type=int, default=32,
                    help="media of the default line's batched-sweep object (x --batch-kn "
                         "Knudsen numbers)")
    ap.add_argument("--batch-object-steps", type=int, default=300)
    ap.add_argument("--kernel", choices=["auto", "staged", "direct"], default="auto",
                    help="implementation of the step kernel (auto: direct for FP32 storage, "
                         "staged for FP16)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(size: int):
    from paper_1411_7051_gb300 import media
    med = media.shale_fractures(n=size, seed=3, n_fractures=40 if size >= 1024 else 4,
                                length=(200.0, 2000.0) if size >= 2048 else
                                (size / 20, size / 2))
    cfg = dict(nx=size, ny=size, tau=0.8, bc_x=1, bc_y=0, rho_in=1.0005, rho_out=0.9995,
               forchheimer=1)
    return med, cfg


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(kernel_tag: str, source_hash: str):
    """DRAM bytes per launch from the committed ncu summary, or None when
    the summary was taken on a different build of the kernels."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(kernel_tag)
    if not e or e.get("source_hash") != source_hash:
        return None
    return e


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 power=float(parts[3]) if parts[3] not in ("[N/A]", "") else None,
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            if r["hw"] == "Active":
                reasons.add("hw_slowdown")
            if r["hwt"] == "Active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"] == "Active":
                reasons.add("sw_thermal_slowdown")
            if r["pcap"] == "Active":
                reasons.add("sw_power_cap")
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------ CPU (oracle)
def oracle_rate(med, cfg, seconds: float, crop: int = 1024, threads: int = 0):
    """FP64 oracle lattice updates per second on a crop of the workload, on
    all host cores (threads = 0) or on `threads` of them.  Also returns the
    oracle's k_g at the end of the run and the steps taken from rest."""
    from oracle import oracle
    n = min(crop, cfg["nx"])
    sub = med.crop(n, n)
    p = oracle.make_params(n, n, tau=cfg["tau"], bc_x=cfg["bc_x"], bc_y=cfg["bc_y"],
                           rho_in=cfg["rho_in"], rho_out=cfg["rho_out"],
                           forchheimer=cfg["forchheimer"])
    all_cores = oracle.max_threads()
    used = threads if threads > 0 else all_cores
    oracle.set_threads(used)
    try:
        sim = oracle.OracleSim(p)
        sim.set_fields(sub.eps, sub.k_i, sub.kn)
        sim.step(1)
        t0 = time.perf_counter()
        sim.step(1)
        per = time.perf_counter() - t0
        steps = max(2, int(seconds / max(per, 1e-6)))
        t0 = time.perf_counter()
        sim.step(steps)
        dt = time.perf_counter() - t0
        kg, _ = sim.permeability()
    finally:
        oracle.set_threads(all_cores)
    return dict(rate=n * n * steps / dt, steps=steps, n=n, cores=used, k_g=kg,
                total_steps=steps + 2)


def gpu_crop_kg(lbmp, med, cfg, n: int, steps: int, storage: str, rounding: str) -> float:
    """k_g of the GPU path (AUTO kernel) on the n x n crop after `steps`
    steps from rest, for the comparison with the oracle's run."""
    sub = med.crop(n, n)
    sc = lbmp.SimConfig(n, n, tau=cfg["tau"], bc_x=cfg["bc_x"], bc_y=cfg["bc_y"],
                        rho_in=cfg["rho_in"], rho_out=cfg["rho_out"],
                        forchheimer=cfg["forchheimer"],
                        storage=lbmp.STORE_FP32 if storage == "fp32" else lbmp.STORE_FP16,
                        fp16_rounding=(lbmp.ROUND_STOCHASTIC if rounding == "stochastic"
                                       else lbmp.ROUND_NEAREST))
    with lbmp.Sim(sc) as sim:
        sim.set_fields(sub.eps, sub.k_i, sub.kn)
        sim.step(steps)
        kg, _ = sim.permeability()
    return kg


def run_reference(args, ws, rank):
    if rank != 0:
        return
    med, cfg = workload(args.size)
    from oracle import oracle
    n = min(1024, args.size)
    sub = med.crop(n, n)
    p = oracle.make_params(n, n, tau=cfg["tau"], bc_x=cfg["bc_x"], bc_y=cfg["bc_y"],
                           rho_in=cfg["rho_in"], rho_out=cfg["rho_out"],
                           forchheimer=cfg["forchheimer"])
    sim = oracle.OracleSim(p)
    sim.set_fields(sub.eps, sub.k_i, sub.kn)
    sim.step(max(3, args.warmup))
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    glups = n * n * args.steps / dt / 1e9
    sample = f"{n}x{n} crop of the {args.size}x{args.size} workload, {args.steps} steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, cfg, "fp64 oracle (CPU)",
                              "wall clock of each step's bounded oracle sample on the host "
                              "cores"),
        "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": oracle.max_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(args, cfg, storage, timed_region=None):
    return {"workload": f"shale matrix with 40 fractures, {args.size}x{args.size} D2Q9, "
                        "pressure-driven x, periodic y, Forchheimer on",
            "nx": cfg["nx"], "ny": cfg["ny"], "tau": cfg["tau"], "storage": storage,
            "l2": "inputs larger than L2 (working set > 129 MB), no flush",
            "timed_region": timed_region or (
                "K steps on the device (CUDA events), submitted behind a ~1 ms spin "
                "kernel; median of %d regions" % REPEATS)}


# ------------------------------------------------------------- GPU (ours)
def kn_beta_for(cfg, p_ratio: float = 2.0) -> float:
    """beta of the dynamic Kn that makes the inlet pressure p_ratio times
    the outlet one (p / p0 = 1 + beta (rho - rho0), rho0 = 1)."""
    a, b = cfg["rho_in"] - 1.0, cfg["rho_out"] - 1.0
    return (p_ratio - 1.0) / (a - p_ratio * b)


REPEATS = 5   # timed K-step regions per measurement; the median is reported


# A spin of about 1 ms (torch's cycle-count sleep kernel) queued ahead of
# the start event: the host has submitted the K steps before the device
# reaches the event, so the region times the device's work and not the
# host's submission latency (the "blocking kernel" of NVBench).
HOLD_CYCLES = 2_000_000


def hold_stream(torch, stream):
    sleep = getattr(torch.cuda, "_sleep", None)
    if sleep is None:
        return False
    with torch.cuda.stream(stream):
        sleep(HOLD_CYCLES)
    return True


def time_storage(lbmp, torch, med, cfg, storage, K, W, kernel, rounding="stochastic",
                 kn_beta=0.0, repeats=REPEATS):
    st = lbmp.STORE_FP32 if storage == "fp32" else lbmp.STORE_FP16
    sc = lbmp.SimConfig(cfg["nx"], cfg["ny"], tau=cfg["tau"], bc_x=cfg["bc_x"],
                        bc_y=cfg["bc_y"], rho_in=cfg["rho_in"], rho_out=cfg["rho_out"],
                        forchheimer=cfg["forchheimer"], storage=st,
                        kernel={"auto": lbmp.KERNEL_AUTO, "staged": lbmp.KERNEL_STAGED,
                                "direct": lbmp.KERNEL_DIRECT}[kernel],
                        fp16_rounding=(lbmp.ROUND_STOCHASTIC if rounding == "stochastic"
                                       else lbmp.ROUND_NEAREST), kn_beta=kn_beta)
    sim = lbmp.Sim(sc)
    sim.set_fields(med.eps, med.k_i, med.kn)
    sim.step(W)
    sim.step(K)   # untimed: builds the step graphs a K-step call replays
    sim.synchronize()
    info0 = sim.info()
    samples = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        torch.cuda.synchronize()
        hold_stream(torch, sim.stream)
        e0.record(sim.stream)
        sim.step(K)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        samples.append(e0.elapsed_time(e1))
    ms = statistics.median(samples)
    info1 = sim.info()
    kg, um = sim.permeability()
    out = dict(ms=ms, ms_samples=samples, launches=int(info1.launches - info0.launches) // repeats,
               nodes=int(info1.fluid_nodes), bpu=float(info1.bytes_per_update),
               scale=float(info1.fp16_scale), k_g=kg)
    sim.close()
    return out


def time_e2e(lbmp, torch, med, cfg, K):
    sc = lbmp.SimConfig(cfg["nx"], cfg["ny"], tau=cfg["tau"], bc_x=cfg["bc_x"],
                        bc_y=cfg["bc_y"], rho_in=cfg["rho_in"], rho_out=cfg["rho_out"],
                        forchheimer=cfg["forchheimer"], storage=lbmp.STORE_FP32)
    sim = lbmp.Sim(sc)
    import numpy as np
    # the inputs sit in pinned host memory, as a serving process keeps them
    eps, k_i, kn = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                    for a in (med.eps, med.k_i, med.kn))
    sim.set_fields(eps, k_i, kn)  # warm the allocator and the graphs
    sim.step(64)
    sim.permeability()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.set_fields(eps, k_i, kn)
    sim.step(K)
    kg, _ = sim.permeability()
    dt = time.perf_counter() - t0
    sim.close()
    n = cfg["nx"] * cfg["ny"]
    return dict(s=dt, h2d=3 * 8 * n, d2h=6 * 8 + 4)


def reduce_max(value: float, device) -> float:
    """Max over the ranks of the process group (the value itself for one rank)."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([float(value)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return float(value)


def whole_job_glups(world_size: int, nodes_per_rank: int, steps: int, ms_slowest: float) -> float:
    """Lattice updates of all replicas over the slowest rank's time (weak
    scaling: every rank runs its own lattice of the same size)."""
    return world_size * nodes_per_rank * steps / (ms_slowest * 1e-3) / 1e9


def kernel_name(kernel: str, tag: str) -> str:
    staged = kernel == "staged" or (kernel == "auto" and tag == "StoreF16")
    return f"lbmp::staged_step_kernel<{tag}>" if staged else f"lbmp::step_kernel<{tag}>"


def run_ours(args, ws, rank, local):
    import torch
    from paper_1411_7051_gb300 import build as lbuild, lbmp
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the product path has no CPU fallback)")
    torch.cuda.set_device(local)
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    lbmp.load()
    K, W = args.steps, max(3, args.warmup)
    med, cfg = workload(args.size)
    primary = args.storage or "fp32"
    args.storage = primary
    other = "fp16" if primary == "fp32" else "fp32"

    with ClockSampler(local) as clk:
        res = time_storage(lbmp, torch, med, cfg, primary, K, W, args.kernel, args.fp16_rounding)
    clocks = clk.summary()
    res_other = None
    if not args.no_other:
        res_other = time_storage(lbmp, torch, med, cfg, other, K, W, args.kernel,
                                 args.fp16_rounding)
    e2e = None if args.no_e2e else time_e2e(lbmp, torch, med, cfg, K)
    dyn = dyn16 = None
    if not args.no_dynamic:
        dyn = time_storage(lbmp, torch, med, cfg, "fp32", K, W, "auto",
                           kn_beta=kn_beta_for(cfg))
        dyn16 = time_storage(lbmp, torch, med, cfg, "fp16", K, W, "auto", args.fp16_rounding,
                             kn_beta=kn_beta_for(cfg))
    adj = None if args.no_adjoint else adjoint_time(lbmp, torch, args.adjoint_steps)
    batch = None if args.no_batch else batch_object(lbmp, torch, args)

    # slowest rank decides
    ms = reduce_max(res["ms"], "cuda")
    if e2e:
        e2e["s"] = reduce_max(e2e["s"], "cuda")
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    nodes = res["nodes"]
    glups = whole_job_glups(ws, nodes, K, ms)
    peak, peak_kind = measured_peaks()
    src = lbuild.kernel_hash()

    def roofline(r, tag):
        per_launch_s = r["ms"] * 1e-3 / K          # one step kernel per time step
        alg = r["bpu"] * r["nodes"]                 # algorithmic bytes per launch
        achieved = alg / per_launch_s / 1e9
        tr = profiled_traffic(tag, src)
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": f"of {peak_kind}",
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                "bytes_per_update": r["bpu"],
                "traffic": (tr["dram_bytes_per_launch"] if tr else None),
                "traffic_per_update": (tr["dram_bytes_per_launch"] / r["nodes"] if tr else None),
                "achieved_dram": (tr["dram_bytes_per_launch"] / per_launch_s / 1e9 if tr else None),
                "kernel": kernel_name(args.kernel, tag)}

    line = {
        "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**config_dict(args, cfg, primary), "kernel": args.kernel,
                   "fp16_rounding": args.fp16_rounding,
                   "timing": f"median of {REPEATS} timed regions of K steps, CUDA events"},
        "ms_per_step_samples": [t / K for t in res["ms_samples"]],
        "roofline": roofline(res, "StoreF32" if primary == "fp32" else "StoreF16"),
        "gpu_launches": res["launches"],
        "clocks": clocks,
        "k_g": res["k_g"],
    }
    if res_other:
        g2 = ws * res_other["nodes"] * K / (res_other["ms"] * 1e-3) / 1e9
        line[f"{other}_stored"] = {
            "value": g2, "unit": "GLUPS", "ms_per_step": res_other["ms"] / K,
            "ms_per_step_samples": [t / K for t in res_other["ms_samples"]],
            "ratio_fp16_over_fp32": (g2 / glups) if other == "fp16" else (glups / g2),
            "roofline": roofline(res_other, "StoreF32" if other == "fp32" else "StoreF16"),
            "fp16_scale": res_other["scale"], "k_g": res_other["k_g"],
        }
    if e2e:
        line["e2e"] = {"value": ws * nodes * K / e2e["s"] / 1e9, "unit": "GLUPS",
                       "h2d_bytes_per_step": e2e["h2d"] / K, "d2h_bytes_per_step": e2e["d2h"] / K,
                       "what": "lbmp_set_fields from pinned host float64 arrays + K steps + "
                               "lbmp_permeability to host, wall clock"}
    if dyn:
        g3 = ws * dyn["nodes"] * K / (dyn["ms"] * 1e-3) / 1e9
        r = roofline(dyn, "StoreF32")
        r["traffic"] = r["traffic_per_update"] = r["achieved_dram"] = None  # static kernel only
        r["kernel"] = "lbmp::step_kernel<StoreF32, false, true> (dynamic Kn)"
        line["fp32_dynamic_kn"] = {
            "value": g3, "unit": "GLUPS", "ms_per_step": dyn["ms"] / K,
            "what": "same workload with Kn per node and step from the local pressure "
                    f"(p/p0 = 1 + beta (rho - rho0), beta {kn_beta_for(cfg):.1f}: inlet "
                    "pressure twice the outlet one; the medium's Kn taken at p0), f_c of "
                    "Eq. 6-7 in FP32 at every step",
            "ratio_to_static": g3 / glups, "roofline": r, "k_g": dyn["k_g"]}
    if dyn and dyn16:
        g4 = ws * dyn16["nodes"] * K / (dyn16["ms"] * 1e-3) / 1e9
        r = roofline(dyn16, "StoreF16")
        r["traffic"] = r["traffic_per_update"] = r["achieved_dram"] = None
        r["kernel"] = "lbmp::staged_step_kernel<StoreF16, SR, true> (dynamic Kn)"
        line["fp16_dynamic_kn"] = {
            "value": g4, "unit": "GLUPS", "ms_per_step": dyn16["ms"] / K,
            "what": "the FP32 dynamic-Kn object with FP16-stored populations (48 B per "
                    "update: the Kn plane at p0 staged beside the medium)",
            "ratio_fp16_over_fp32": g4 / (ws * dyn["nodes"] * K / (dyn["ms"] * 1e-3) / 1e9),
            "roofline": r, "fp16_scale": dyn16["scale"], "k_g": dyn16["k_g"]}
    if adj:
        line["adjoint"] = adjoint_object(adj, peak, peak_kind)
    if batch:
        line["batch"] = batch
    if not args.no_cpu and ws == 1:
        o = oracle_rate(med, cfg, args.cpu_seconds)
        o1 = oracle_rate(med, cfg, args.cpu_seconds / 3, crop=256, threads=1)
        line["cpu_baseline"] = {
            "value": o["rate"] / 1e9, "unit": "GLUPS", "cores": o["cores"], "kind": "oracle",
            "sample": f"{o['n']}x{o['n']} crop of the workload, {o['steps']} FP64 steps",
            "single_thread": {"value": o1["rate"] / 1e9, "unit": "GLUPS", "cores": 1,
                              "sample": f"{o1['n']}x{o1['n']} crop of the workload, "
                                        f"{o1['steps']} FP64 steps"}}
        # each storage against the oracle's k_g on the oracle's own run: the
        # crop, from rest, the same number of steps
        n, S = o["n"], o["total_steps"]
        errs = {"sample": f"{n}x{n} crop of the workload, {S} steps from rest",
                "k_g_oracle": o["k_g"]}
        for st in ("fp32", "fp16"):
            kg = gpu_crop_kg(lbmp, med, cfg, n, S, st, args.fp16_rounding)
            errs[st] = {"k_g": kg, "rel_err": abs(kg / o["k_g"] - 1.0)}
        line["k_g_vs_oracle"] = errs
        line["k_g_err_vs_oracle"] = errs[primary]["rel_err"]
        if res_other:
            line[f"{other}_stored"]["k_g_err_vs_oracle"] = errs[other]["rel_err"]
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ adjoint
# algorithmic bytes per node and time step of the backward sweep (see
# adjoint_time()): the recompute step (the forward step's 80 plus 12 of
# moments) and the reverse step (109.5)
ADJOINT_RECOMPUTE_BYTES = 80 + 12
ADJOINT_REVERSE_BYTES = 36 + 12 + 8 + 16 + 36 + 48 / 32
ADJOINT_BYTES_PER_NODE = ADJOINT_RECOMPUTE_BYTES + ADJOINT_REVERSE_BYTES


def adjoint_case(lbmp, n: int = 1024):
    """The adjoint workload: two-component medium (correlation length 32,
    matrix eps 0.2 / k_i 1e-5, inclusions eps 0.6 / k_i 1e-3, seed 2),
    Kn = 0.1, pressure-driven in x, plates in y, Forchheimer on."""
    from paper_1411_7051_gb300 import media
    med = media.two_component(n, seed=2, kn=0.1)
    cfg = lbmp.SimConfig(n, n, tau=0.8, bc_x=lbmp.BCX_PRESSURE, bc_y=lbmp.BCY_WALLS,
                         rho_in=1.0005, rho_out=0.9995, forchheimer=1)
    return med, cfg


def adjoint_time(lbmp, torch, N: int, evals: int = 1, warm: int = 1, n: int = 1024):
    """Times lbmp_permeability_gradient (N steps from rest) with CUDA events
    on the library's stream (median of `evals`), and the plain N-step run
    beside it.  The backward sweep is the gradient time minus the forward
    pass (one timed forward run): per node and time step it recomputes the
    forward step, storing the moments (80 + 12 bytes), and runs the reverse
    step: mu^{t+1} gathered 36, moments of f^t 12, medium 8, FP32
    accumulators read + written 16, mu^t written 36, plus the FP64 fold
    (8 + 32 + 8 bytes every 32 steps)."""
    import math
    med, cfg = adjoint_case(lbmp, n)
    sim = lbmp.Sim(cfg)
    sim.set_fields(med.eps, med.k_i, med.kn)
    for _ in range(warm):
        sim.permeability_gradient(min(N, 256))
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(sim.stream)
    sim.set_fields(med.eps, med.k_i, med.kn)
    sim.step(N)
    e1.record(sim.stream)
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1)
    l0 = sim.info().launches
    t_grad = []
    for _ in range(evals):
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        e0.record(sim.stream)
        kg, gl, ge = sim.permeability_gradient(N)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        t_grad.append(e0.elapsed_time(e1))
    launches = (sim.info().launches - l0) // evals
    nodes = int(sim.info().fluid_nodes)
    pitch = int(sim.info().pitch)
    sim.close()
    every = math.ceil(math.sqrt(N))
    nseg = math.ceil(N / every)
    state = 9 * 4 * pitch * n
    tg = statistics.median(t_grad)
    t_back = tg - t_fwd
    return dict(ms_gradient=tg, ms_forward=t_fwd, ms_backward=t_back, nodes=nodes, N=N,
                every=every, checkpoints=nseg, launches=int(launches), k_g=kg,
                sum_abs_dlogk=float(gl.abs().sum()), sum_abs_deps=float(ge.abs().sum()),
                device_bytes=(nseg + 4) * state + every * state // 3 + 24 * state // 36)


def adjoint_object(r, peak, peak_kind):
    from paper_1411_7051_gb300 import build as lbuild
    back_s = r["ms_backward"] * 1e-3
    achieved = ADJOINT_BYTES_PER_NODE * r["nodes"] * r["N"] / back_s / 1e9
    tr = profiled_traffic("adjoint", lbuild.kernel_hash(lbuild.ADJOINT_KERNEL_FILES))
    return {
        "workload": "two-component 1024x1024 (corr. length 32, matrix eps 0.2 / k_i 1e-5, "
                    "inclusions eps 0.6 / k_i 1e-3), Kn 0.1, pressure x, plates y, Forchheimer; "
                    f"J = k_g after {r['N']} steps from rest; d/d ln k_i and d/d eps of every node",
        "ms_per_gradient": r["ms_gradient"], "ms_forward_run": r["ms_forward"],
        "ratio_to_forward_run": r["ms_gradient"] / r["ms_forward"],
        "gradient_glups": r["nodes"] * r["N"] / (r["ms_gradient"] * 1e-3) / 1e9,
        "checkpoint_every": r["every"], "checkpoints": r["checkpoints"],
        "device_bytes": r["device_bytes"], "gpu_launches": r["launches"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"of {peak_kind}",
                     "bytes_per_update": ADJOINT_BYTES_PER_NODE,
                     "traffic": None,
                     "reverse_kernel": {
                         "bytes_per_update": ADJOINT_REVERSE_BYTES,
                         "traffic": (tr["dram_bytes_per_launch"] if tr else None),
                         "traffic_per_update": (tr["dram_bytes_per_launch"] / tr["nodes"]
                                                if tr else None)},
                     "kernel": "lbmp::step_kernel<StoreF32, 0, 0, 1> (recompute with moments) + "
                               "lbmp::adjoint_step_kernel<false> (+ fold)",
                     "timing": "backward sweep (recompute + reverse) = gradient minus the "
                               "forward pass, CUDA events"},
        "k_g": r["k_g"],
    }


def run_adjoint(args, ws, rank, local):
    """--workload adjoint: K gradient evaluations after W warm-up ones."""
    import torch
    from paper_1411_7051_gb300 import lbmp
    torch.cuda.set_device(local)
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    K, W = args.steps, max(3, args.warmup)
    with ClockSampler(local) as clk:
        r = adjoint_time(lbmp, torch, args.adjoint_steps, evals=K, warm=W)
    ms = reduce_max(r["ms_gradient"], "cuda")
    if rank == 0:
        peak, kind = measured_peaks()
        line = {
            "metric": METRIC, "value": ws * r["nodes"] * r["N"] / (ms * 1e-3) / 1e9,
            "unit": "GLUPS", "n_gpus": ws, "steps": K, "warmup": W, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "adjoint: gradient of k_g, one step = one gradient "
                                   f"evaluation over {r['N']} time steps (forward, recompute, "
                                   "reverse); value = time steps x nodes / gradient time",
                       "nx": 1024, "ny": 1024, "l2": "working set > L2 per sweep, no flush"},
            "adjoint": adjoint_object(r, peak, kind),
            "gpu_launches": r["launches"] * K, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


BATCH_SIDES = (256, 384, 512, 768, 1024)


def batch_media(n_media: int, seed0: int = 1000):
    """Seeded two-component media (correlation length 32, matrix eps 0.2 /
    k_i 1e-5, inclusions eps 0.6 / k_i 1e-3) with sides drawn uniformly from
    BATCH_SIDES; Kn is set per instance."""
    import numpy as np
    from paper_1411_7051_gb300 import media
    rng = np.random.Generator(np.random.PCG64(seed0))
    sides = rng.choice(BATCH_SIDES, size=n_media)
    return [media.two_component(int(n), seed=seed0 + m, corr_len=32.0) for m, n in enumerate(sides)]


def batch_measure(lbmp, torch, n_media: int, n_kn: int, storage: str, K: int, W: int,
                  rounding: str = "stochastic", repeats: int = REPEATS, clocks_index=None):
    """Builds the batched sweep (n_media media x n_kn Knudsen numbers), tunes
    its launch shape, and times K steps `repeats` times (median) with CUDA
    events on the batch's stream."""
    import numpy as np
    t0 = time.perf_counter()
    meds = batch_media(n_media)
    kns = np.logspace(-3, 1, n_kn)
    sizes = [(m.eps.shape[1], m.eps.shape[0]) for m in meds for _ in kns]
    st = lbmp.STORE_FP32 if storage == "fp32" else lbmp.STORE_FP16
    cfg = lbmp.SimConfig(1, 1, tau=0.8, bc_x=lbmp.BCX_PRESSURE, bc_y=lbmp.BCY_WALLS,
                         rho_in=1.0005, rho_out=0.9995, forchheimer=1, storage=st,
                         fp16_rounding=(lbmp.ROUND_STOCHASTIC if rounding == "stochastic"
                                        else lbmp.ROUND_NEAREST))
    b = lbmp.Batch(cfg, sizes)
    j = 0
    for m in meds:
        for kn in kns:
            b.set_fields(j, m.eps, m.k_i, np.full(m.eps.shape, kn))
            j += 1
    setup_s = time.perf_counter() - t0
    chosen, tune_ms = b.tune(steps=5)
    b.step(W)
    b.synchronize()
    samples = []
    clk = ClockSampler(clocks_index) if clocks_index is not None else None
    if clk:
        clk.__enter__()
    l0 = b.info().launches
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0.record(b.stream)
        b.step(K)
        e1.record(b.stream)
        torch.cuda.synchronize()
        samples.append(e0.elapsed_time(e1))
    if clk:
        clk.__exit__(None, None, None)
    info = b.info()
    kg, _ = b.permeability()
    b.close()
    return dict(ms=statistics.median(samples), ms_samples=samples, nodes=int(info.total_nodes),
                instances=len(sizes), bpu=float(info.bytes_per_update),
                shape=[info.shape_threads, info.shape_nodes_per_thread,
                       {0: "one block per item", 1: "persistent",
                        2: "staged (bulk-copy tiles)"}[int(info.persistent)]],
                staged=int(info.persistent) == 2, launches=int(info.launches - l0) // repeats,
                setup_s=setup_s, chosen=chosen, tune_ms=tune_ms,
                k_g_range=[float(np.min(kg)), float(np.max(kg))],
                clocks=clk.summary() if clk else None)


def batch_roofline(r, K, peak, kind, storage):
    """Roofline of the batched step; `traffic` from the committed ncu figures
    when they were taken on the current batched-kernel sources and on the
    same set of instances (the same node count)."""
    from paper_1411_7051_gb300 import build as lbuild
    per_launch_s = r["ms"] * 1e-3 / K
    achieved = r["bpu"] * r["nodes"] / per_launch_s / 1e9
    tr = None
    if r["staged"]:
        tr = profiled_traffic(f"batch_{storage}", lbuild.kernel_hash(lbuild.BATCH_KERNEL_FILES))
        if tr and tr.get("nodes") != r["nodes"]:
            tr = None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": f"of {kind}",
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
            "bytes_per_update": r["bpu"],
            "traffic": (tr["dram_bytes_per_launch"] if tr else None),
            "traffic_per_update": (tr["dram_bytes_per_launch"] / r["nodes"] if tr else None),
            "achieved_dram": (tr["dram_bytes_per_launch"] / per_launch_s / 1e9 if tr else None),
            "kernel": ("lbmp::batch_staged_kernel" if r["staged"] else "lbmp::batch_step_kernel")}


def batch_object(lbmp, torch, args):
    """The default line's batched-sweep object: a subset of the sweep (the
    first --batch-object-media media x --batch-kn Knudsen numbers), FP16
    (stochastic rounding) and FP32 storage."""
    peak, kind = measured_peaks()
    K, W = args.batch_object_steps, 10
    out = {"workload": f"batched sweep subset: {args.batch_object_media} two-component media "
                       f"(sides {list(BATCH_SIDES)}, corr. length 32) x {args.batch_kn} Kn in "
                       "[1e-3, 10], pressure x, walls y, Forchheimer on; one launch per step "
                       f"over all instances; median of {REPEATS} regions of {K} steps",
           "steps": K}
    for st in ("fp16", "fp32"):
        r = batch_measure(lbmp, torch, args.batch_object_media, args.batch_kn, st, K, W,
                          args.fp16_rounding)
        out[st] = {"value": r["nodes"] * K / (r["ms"] * 1e-3) / 1e9, "unit": "GLUPS",
                   "ms_per_step": r["ms"] / K, "instances": r["instances"], "nodes": r["nodes"],
                   "shape": r["shape"], "tuned_shape_index": r["chosen"],
                   "roofline": batch_roofline(r, K, peak, kind, st), "gpu_launches": r["launches"],
                   "k_g_range": r["k_g_range"], "setup_s": r["setup_s"]}
    return out


def run_batch(args, ws, rank, local):
    """One persistent launch per step over every (medium, Kn) instance."""
    import torch
    from paper_1411_7051_gb300 import lbmp
    torch.cuda.set_device(local)
    if ws > 1:
        torch.distributed.init_process_group("nccl")
    K, W = args.steps, max(3, args.warmup)
    storage = args.storage or "fp16"
    r = batch_measure(lbmp, torch, args.batch_media, args.batch_kn, storage, K, W,
                      args.fp16_rounding, clocks_index=local)
    ms = reduce_max(r["ms"], "cuda")
    if rank == 0:
        glups = whole_job_glups(ws, r["nodes"], K, ms)
        peak, kind = measured_peaks()
        line = {
            "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": ws, "steps": K,
            "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched sweep: {args.batch_media} two-component media "
                                   f"(sides {list(BATCH_SIDES)}) x {args.batch_kn} Kn in [1e-3, 10], "
                                   "pressure x, walls y, Forchheimer on, one persistent launch per step",
                       "instances": r["instances"], "nodes": r["nodes"], "storage": storage,
                       "shape": r["shape"], "l2": "inputs larger than L2, no flush",
                       "timing": f"median of {REPEATS} timed regions of K steps, CUDA events"},
            "ms_per_step_samples": [t / K for t in r["ms_samples"]],
            "roofline": batch_roofline(r, K, peak, kind, storage),
            "gpu_launches": r["launches"], "clocks": r["clocks"],
            "setup_s": r["setup_s"], "tuned_shape_index": r["chosen"],
            "tune_ms_per_step": r["tune_ms"], "k_g_range": r["k_g_range"],
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batch":
        run_batch(args, ws, rank, local)
    elif args.workload == "adjoint":
        run_adjoint(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
