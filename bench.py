#!/usr/bin/env python
"""Benchmark of the compressible Navier-Stokes RHS + RK4 hot path on GB300.

Workload: decaying isotropic turbulence on a 512^3 triply periodic grid (FP64,
rho = 1, p = 1/gamma, u0 = 0.3, k0 = 4, mu_eff for Re_lambda = 50, dt at CFL 0.4),
one step = one classical RK4 step (4 right-hand-side evaluations) plus the
statistics (kinetic energy, enstrophy, conservation sums, CFL) of the new state,
as in a run that logs them every step.  Metric: grid-point RHS evaluations per
second (Gpts/s) = points * 4 * steps / time, summed over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The same line carries the comparison modes: the all-FP64 form, FP32-bulk over 100
steps from the same state (speed and error against FP64), the adjoint (Taylor-Green
64^3 gradient), the 48-instance ensemble (50 steps per schedule) and 1024^3 with
SSP-RK3 on one GPU.

--impl reference times the FP64 CPU oracle on the host cores (per step, the RHS of a
periodic 72-plane z-slab of the same 512^3 state).  Multi-GPU: independent replicas,
one per rank (no collective on the data path), barrier + max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-point RHS evals/sec (Gpts/s) and HBM roofline fraction; FP32-bulk/adjoint vs FP64"
UNIT = "Gpts/s"
RK_STAGES = 4
# FP64 lane operations (FP64 instructions per thread, an FMA counting once) per grid point of
# one direction pass, counted from each formulation without the halo's share:
#  NS3D_FP64 (double-float weights, offsets, interface jumps, Roe dissipation and viscous
#   divergence): point fluxes 5, first differences 9, per flux component the interface sum
#   2 P_i + (g + dL + dR) 2 x 5 and the combination (fhat_L + fhat_R - diss)/(2 dx) 2 x 5, flux
#   difference 5, adding the double-float viscous divergence 2 x 4.
#  NS3D_FP64_STRICT: point fluxes 5, smoothness indicators 9 x 14, candidates and weighted sums
#   (with the division sequence) 9 x 50, Roe flux ~100 (two divisions, a square root), 26.
OPS_DIR_FP64 = 5 + 9 + 10 + 10 + 5 + 8
OPS_DIR_STRICT = 5 + 9 * 14 + 9 * 50 + 100 + 26
OPS_RK_EPI = 15            # RK4 stage update in the z pass (5 components x 3)
# The method's FP64 flops per point and pass (FMA = 2) in its all-FP64 form, for context.
FLOPS_DIR = 6 + 9 * 20 + 9 * 46 + 96 + 34
SMS, FP64_LANES_PER_SM, SM_MAX_MHZ, ISSUE_PER_SM = 152, 2, 2070.0, 4
FP64_LANEOPS_PEAK_T = SMS * FP64_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12          # 0.629 T lane-ops/s
ISSUE_PEAK_G = SMS * ISSUE_PER_SM * SM_MAX_MHZ * 1e6 / 1e9                       # 1258.6 G warp-instr/s
FP64_PEAK_TFLOPS = SMS * FP64_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 1.2586 (FMA = 2 flops)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512, help="grid points per direction")
    ap.add_argument("--cfl", type=float, default=0.4)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--compare-steps", type=int, default=100,
                    help="steps of the FP64 vs FP32-bulk comparison (from the same state and dt)")
    ap.add_argument("--parity-points", type=int, default=64,
                    help="sampled points of the headline's RHS checked against the oracle")
    ap.add_argument("--ens-steps", type=int, default=50, help="steps per schedule of the 48-instance ensemble")
    ap.add_argument("--big", type=int, default=1024, help="grid of the SSP-RK3 single-GPU run (0: skip)")
    ap.add_argument("--big-steps", type=int, default=3)
    ap.add_argument("--big-points", type=int, default=512, help="sampled oracle windows of the big run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-strict", action="store_true", help="skip the all-FP64 comparison run")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-bulk comparison run")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 48-instance ensemble measurement")
    ap.add_argument("--ens-count", type=int, default=0,
                    help="--study ensemble: only this many instances (sizes --ens-sizes), e.g. for a profiler")
    ap.add_argument("--ens-sizes", type=str, default="32,48", help="comma-separated grid sizes for --ens-count")
    ap.add_argument("--precision", choices=["fp64", "strict"], default="fp64",
                    help="context precision of --study vjp (NS3D_FP64 or NS3D_FP64_STRICT)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (Taylor-Green 64^3) measurement")
    ap.add_argument("--study", choices=["fp32", "ensemble", "adjoint", "vjp", "big", "oracle"], default=None,
                    help="fp32: FP64 vs FP32-bulk over --steps steps at --n^3 (KE/enstrophy every step); "
                         "ensemble: 48 uneven realisations, --steps steps per schedule")
    return ap.parse_args()


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if os.environ.get("NS3D_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_device() -> str:
    import torch.distributed as dist
    return "cpu" if dist.get_backend() == "gloo" else "cuda"


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="ns3d_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


KDIR_SOURCES = ("k_dir.cu", "k_dir_impl.cuh", "k_dir_common.cuh", "k_point_impl.cuh", "df.cuh", "df2.cuh")
KDIR32_SOURCES = ("k_dir32.cu", "k_dir_common.cuh", "df.cuh")


def kernel_source_sha(names=KDIR_SOURCES) -> str:
    """sha256 prefix over the code of the sources that make up the direction-pass kernel
    (comments and blank space removed, so that a comment edit keeps the profiled figures)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for nm in names:
        src = open(os.path.join(ROOT, "paper_2211_16718_gb300", "csrc", nm)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def _profile_line(tag: str, kernel: str, field: str, sha: str):
    """(value, file, grid) of the committed ncu figure `tag kernel field=value grid=G ...
    source_sha256=sha` under profiles/ taken on the largest grid, or None if no line matches the
    current kernel code."""
    import glob
    import re
    best = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            m = re.match(rf"{tag} {kernel} {field}=([0-9.]+) grid=(\d+) \S+ source_sha256=(\w+)", line)
            if m and m.group(3) == sha and (best is None or int(m.group(2)) > best[2]):
                best = (float(m.group(1)), os.path.basename(path), int(m.group(2)))
    return best


def ncu_traffic_per_point(kernel: str, sha: str):
    """DRAM bytes per grid point of one launch (dram__bytes_read.sum + dram__bytes_write.sum
    from a committed ncu summary under profiles/), or None if the kernel sources have changed
    since the counters were taken."""
    return _profile_line("TRAFFIC", kernel, "bytes_per_point", sha)


def ncu_issue_per_point(kernel: str, sha: str):
    """Warp instructions issued per grid point of one launch (smsp__inst_executed.sum from a
    committed ncu summary), or None if the kernel sources have changed since."""
    return _profile_line("ISSUE", kernel, "warp_instr_per_point", sha)


def measured_peaks() -> dict:
    """HBM copy bandwidth of this GPU pool (MEASURED_PEAKS.json, written by the driver of the
    measurement runs), else the fallback figure of one earlier GB300 measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json: STREAM-style copy)"}
    except (OSError, ValueError, KeyError):
        return {"hbm_gbs": 6800.0, "source": "fallback (6.8 TB/s, one earlier GB300 copy measurement)"}


def hit_state(n: int):
    """Host state of the decaying-turbulence problem (hit_velocity(n, seed 0)), for the
    CPU-side studies and the small adjoint kernel comparison."""
    from paper_2211_16718_gb300 import inputs as I
    return I.isotropic_turbulence(n, seed=0), I.hit_mu_eff()


HIT_NBASE = 64  # base grid of the device-built turbulence field (spectral interpolant, exact up to ~1e-52)


def workload_config(n: int, cfl: float, mu: float, dt: float) -> dict:
    return {"workload": f"decaying isotropic turbulence {n}^3, FP64, RK4 + KE/enstrophy each step",
            "grid": [n, n, n], "domain": "[0,2pi)^3 periodic", "integrator": "classical RK4",
            "rhs_per_step": RK_STAGES, "u0": 0.3, "k0": 4, "re_lambda": 50, "mu_eff": mu, "cfl": cfl,
            "dt": dt, "seed": 0,
            "initial_field": f"rho = 1, p = 1/gamma, velocity hit_velocity({HIT_NBASE}, seed 0) spectrally "
                             f"interpolated to {n}^3 (E(k) ~ k^4 exp(-2 (k/k0)^2), all shells < {HIT_NBASE // 2})",
            "l2": f"inputs larger than L2: state {5 * n ** 3 * 8 / 1e6:.0f} MB, working set "
                  f"{(5 * 4 + 7 + 12) * n ** 3 * 8 / 1e9:.2f} GB vs 129 MB L2; L2 flushed before the timed region",
            "parallelism": "replicas (one independent grid per GPU)"}


def cpu_oracle_sample(u0, mu, n, dt, full_step: bool):
    """Time the oracle as it stands on all host cores: one RK4 step (or one RHS)."""
    from oracle import oracle as O
    O.build()
    threads = os.cpu_count() or 1
    O.set_threads(threads)
    P = O.Params(n, n, n, mu_eff=mu)
    t0 = time.perf_counter()
    if full_step:
        O.rk_step(P, u0, dt, 1)
        pts = n ** 3 * RK_STAGES
        what = f"one RK4 step (4 RHS) of the {n}^3 state"
    else:
        O.rhs(P, u0)
        pts = n ** 3
        what = f"one RHS of the {n}^3 state"
    el = time.perf_counter() - t0
    return pts / el / 1e9, el, O.get_threads() if O.has_openmp() else 1, what


def run_study_oracle():
    """Timing table of the CPU oracle as it stands (FP64 C, OpenMP over lines/points): one RHS and
    one RK4 step of the isotropic-turbulence state at 32^3 .. 256^3 on one thread (256^3: the RHS
    only) and on all host cores, the 32^3 Taylor-Green case (10 RK4 steps) end to end, and one
    RHS at 512^3 on all cores.  CPU work only (the CPU baseline); the GPU is not used."""
    from oracle import oracle as O
    from paper_2211_16718_gb300 import inputs as I
    O.build()
    allc = os.cpu_count() or 1
    rows = []

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    for n in (32, 64, 128, 256):
        u0, mu = hit_state(n)
        P = O.Params(n, n, n, mu_eff=mu)
        for th in (1, allc):
            O.set_threads(th)
            t_rhs = timed(lambda: O.rhs(P, u0))
            row = {"grid": n, "threads": O.get_threads() if O.has_openmp() else 1,
                   "rhs_s": t_rhs, "rhs_gpts": n ** 3 / t_rhs / 1e9}
            if th > 1 or n < 256:  # a single-threaded 256^3 RK4 step would take minutes
                t_rk = timed(lambda: O.rk_step(P, u0, 1e-3, 1))
                row.update({"rk4_step_s": t_rk, "rk4_gpts": n ** 3 * RK_STAGES / t_rk / 1e9})
            rows.append(row)
    O.set_threads(allc)
    u = I.taylor_green(32)
    P = O.Params(32, 32, 32, mu_eff=6.25e-5)
    t_tgv = timed(lambda: O.rk_step(P, u, 0.089, 10))
    u0, mu = hit_state(512)
    P = O.Params(512, 512, 512, mu_eff=mu)
    t_512 = timed(lambda: O.rhs(P, u0))
    return {"study": "oracle", "host_cores": allc, "openmp": O.has_openmp(), "table": rows,
            "taylor_green_32_10_rk4_steps_s": t_tgv,
            "hit512_one_rhs_all_cores": {"s": t_512, "gpts": 512 ** 3 / t_512 / 1e9}}


REF_SLAB = 64     # planes of the workload per reference step ...
REF_HALO = 4      # ... plus the 4-plane reach of the stencil on each side (WENO5 3, viscous composite 4)


def run_reference(args, world, rank):
    """The oracle as it stands on the host cores, on a bounded sample of the workload per step:
    the right-hand side of a periodic slab of REF_SLAB + 2 REF_HALO z-planes of the n^3 state
    (every x-y plane of the slab is a full n x n plane of the workload; the inner REF_SLAB planes
    equal the n^3 RHS exactly, since the stencil reaches 4 planes).  value = points evaluated
    (all planes of the slab) / time."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2211_16718_gb300 import inputs as I
    n = args.n
    mu = I.hit_mu_eff()
    nzs = min(n, REF_SLAB + 2 * REF_HALO)
    slab = I.isotropic_turbulence_planes(n, seed=0, z0=n // 2 - nzs // 2, count=nzs, nbase=min(HIT_NBASE, n))
    O.build()
    O.set_threads(os.cpu_count() or 1)
    h = 2 * math.pi / n
    P = O.Params(n, n, nzs, lx=2 * math.pi, ly=2 * math.pi, lz=nzs * h, mu_eff=mu)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.rhs(P, slab)
        el = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(el)
    tot = sum(times)
    pts = n * n * nzs
    value = pts * len(times) / tot / 1e9
    cores = O.get_threads() if O.has_openmp() else 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(n, args.cfl, mu, None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step: one RHS of a {n}x{n}x{nzs} periodic z-slab of the {n}^3 state "
                                       f"(plain FP64 C oracle, OpenMP over lines/points; {pts} points per step)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _guard(name: str, fn):
    """Run one comparison mode; a failure is recorded in the line instead of ending the run."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        import torch
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return {"error": f"{type(e).__name__}: {e}"[:400], "mode": name}


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_2211_16718_gb300 import build as B
    B.build()
    from paper_2211_16718_gb300 import inputs as I
    from paper_2211_16718_gb300 import ns3d

    n = args.n
    N = n ** 3
    mu = I.hit_mu_eff()
    u0_dev = I.isotropic_turbulence_device(n, seed=0, nbase=min(HIT_NBASE, n))
    torch.cuda.synchronize()
    K, W = args.steps, args.warmup
    n_cmp = max(args.compare_steps, W + K)  # steps of the FP64 / FP32-bulk comparison (config: 100)
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()
    HBM = peaks["hbm_gbs"]
    solver0 = ns3d.Solver(n, n, n, mu_eff=mu)
    dt = solver0.dt_from_cfl(u0_dev, args.cfl)
    solver0.close()

    def timed_loop(precision: int, K: int, W: int, sample_clocks: bool, total: int):
        """W untimed + K timed steps (RK4 step + statistics into a device log), then untimed steps
        up to `total` (statistics logged every step), all from the same initial state and dt."""
        solver = ns3d.Solver(n, n, n, mu_eff=mu, precision=precision)
        ud = u0_dev.clone()
        total = max(total, W + K)
        stats_buf = torch.zeros((total + 1, ns3d.NS3D_STATS_NDOUBLE), dtype=torch.float64, device="cuda")
        solver.stats_async(ud, stats_buf[0])

        def step(i):
            solver.rk_step(ud, dt, 1)
            solver.stats_async(ud, stats_buf[i + 1])

        for i in range(W):
            step(i)
        torch.cuda.synchronize()
        # flush L2 before the timed region (the state alone exceeds L2 every step)
        flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device="cuda")
        flush.fill_(1.0)
        del flush
        solver.timing_enable(True)
        clocks = ClockSampler(local) if sample_clocks else None
        if clocks:
            clocks.start()
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(W, W + K):
            step(i)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clk = clocks.stop() if clocks else None
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        ktimes = solver.timing_read()
        solver.timing_enable(False)
        for i in range(W + K, total):
            step(i)
        torch.cuda.synchronize()
        st = stats_buf.cpu().numpy()
        return solver, ud, ms, ktimes, st, clk

    # headline: NS3D_FP64 (FP64 values, double-float WENO weights)
    solver, ud, ms, ktimes, st, clk = timed_loop(ns3d.NS3D_FP64, K, W, True, n_cmp)
    pts_total = sum_over_ranks(float(N * RK_STAGES * K), world)
    value = pts_total / (ms * 1e-3) / 1e9
    status_ok = bool(np.all(st[:, 10] == 0))
    launches = int(sum(c for _, c in ktimes.values()))

    def roofline_of(kt, ops_dir, form):
        # dominant kernel: the direction pass (x, y, z launches of the same kernel)
        dir_ms = sum(kt[k][0] for k in ("dir_x", "dir_y", "dir_z"))
        dir_launches = sum(kt[k][1] for k in ("dir_x", "dir_y", "dir_z"))
        avg_launch_s = dir_ms / dir_launches * 1e-3
        ops_pt = ops_dir + OPS_RK_EPI / 3.0
        achieved = ops_pt * N / avg_launch_s / 1e12
        step_ms_total = sum(v[0] for v in kt.values())
        return {"bound": "alu", "kernel": f"k_dir ({form}: fused WENO5 + Roe + difference + viscous divergence)",
                "achieved": achieved, "peak": FP64_LANEOPS_PEAK_T,
                "unit": "T FP64 lane-ops/s (FP64 instructions per thread; FMA = 1)",
                "frac": achieved / FP64_LANEOPS_PEAK_T, "traffic": None,
                "peak_source": "152 SMs x 2 FP64 lanes/clk x 2070 MHz (unit counts, max clock; "
                               "ns3d_alu_probe measures 626 G DFMA lane-ops/s)",
                "fp64_ops_per_point": ops_pt, "avg_launch_ms": avg_launch_s * 1e3,
                "share_of_device_time": dir_ms / step_ms_total if step_ms_total > 0 else None}

    fp64_view = roofline_of(ktimes, OPS_DIR_FP64, "NS3D_FP64")
    avg_launch_s = fp64_view["avg_launch_ms"] * 1e-3
    fp64_pipe = {k: fp64_view[k] for k in ("achieved", "peak", "unit", "frac", "peak_source", "fp64_ops_per_point")}
    iss = ncu_issue_per_point("k_dir", kernel_source_sha())
    if iss is not None:
        # NS3D_FP64 runs most of its FP64-accurate arithmetic as double-float on the FP32 pipe,
        # so the FP64 pipe is not the binding unit: instruction issue is.  The primary roofline
        # is the issue rate (warp instructions of this formulation per point, from the ncu
        # capture tied to the kernel source hash, x points per launch / live launch time).
        ipp, src, grid = iss
        ach = ipp * N / avg_launch_s / 1e9
        roofline = {"bound": "alu", "resource": "instruction issue",
                    "kernel": fp64_view["kernel"], "achieved": ach, "peak": ISSUE_PEAK_G,
                    "unit": "G warp instructions/s", "frac": ach / ISSUE_PEAK_G, "traffic": None,
                    "peak_source": "152 SMs x 4 schedulers x 1 issue/clk x 2070 MHz (unit counts, max clock)",
                    "warp_instr_per_point": ipp,
                    "per_unit_source": f"ncu smsp__inst_executed.sum per launch at {grid}^3 ({src})",
                    "fp64_pipe": fp64_pipe}
    else:
        roofline = dict(fp64_view)
        roofline["resource"] = "FP64 pipe (issue view unavailable: kernel sources changed since the ncu capture)"
    for k in ("avg_launch_ms", "share_of_device_time"):
        roofline[k] = fp64_view[k]
    # the method's own work per launch, beside the issue view: the scope table's algorithmic bytes
    # (a fused RK4 stage reads U_s, U_n, acc and writes acc, U_s+1: 200 B/pt, 160 B/pt in the
    # first and last stage, so 720 B/pt per step over 12 direction launches) and the method's
    # all-FP64 flops, with the pipe each part of them runs on in this formulation
    step_bytes = 160 + 200 + 200 + 160
    launch_bytes = step_bytes / 12.0
    step_ms = ms / K
    roofline["method"] = {
        "algorithmic_bytes_per_point_per_launch": launch_bytes,
        "algorithmic_bytes_source": "fused RK4 stage: read U_s, U_n, acc, write acc, U_s+1 (200 B/pt; stages 1 "
                                    "and 4: 160 B/pt) = 720 B/pt per step over 3 x 4 direction launches",
        "method_hbm_gbs": launch_bytes * N / avg_launch_s / 1e9,
        "method_hbm_frac": launch_bytes * N / avg_launch_s / 1e9 / HBM,
        "step_method_hbm_frac": (step_bytes + 40) * N / (step_ms * 1e-3) / 1e9 / HBM,
        "hbm_peak_gbs": HBM, "hbm_peak_source": peaks["source"],
        "method_flops_per_point_per_launch": FLOPS_DIR + 5,
        "method_flops_source": "all-FP64 form of one direction pass (FMA = 2): point fluxes 6, smoothness "
                               "indicators 9 x 20, candidates and weighted sums 9 x 46, Roe flux 96, "
                               "difference + viscous divergence 34, RK epilogue 5",
        "method_tflops": (FLOPS_DIR + 5) * N / avg_launch_s / 1e12,
        "method_fp64_frac": (FLOPS_DIR + 5) * N / avg_launch_s / 1e12 / FP64_PEAK_TFLOPS,
        "fp64_peak_tflops": FP64_PEAK_TFLOPS,
        "pipes": {"fp64_pipe_lane_ops_per_point": OPS_DIR_FP64 + OPS_RK_EPI / 3.0,
                  "fp64_pipe_part": "point values, first differences, point fluxes, interface-flux sums, flux "
                                    "difference, RK update",
                  "fp32_pipe_part": "WENO weights and offsets, interface jumps, Roe dissipation, viscous "
                                    "fluxes and divergence, as double-float; the differences, indicators and "
                                    "reconstructions of two lines per packed FP32 instruction"},
        "note": "method_fp64_frac above 1 means the formulation runs the method faster than the FP64 pipe "
                "could in all-FP64 arithmetic; instruction issue (frac), the FP64 pipe (~46 % busy, ncu) "
                "and the phase barriers bound it together"}
    tr = ncu_traffic_per_point("k_dir", kernel_source_sha())
    if tr is not None:
        bpp, src, grid = tr
        roofline["traffic"] = bpp * N
        roofline["traffic_note"] = (f"ncu dram read+write per launch at {grid}^3 ({src}), {bpp:.1f} B/point"
                                    + ("" if grid == n else f" scaled to {n}^3 (streaming kernel: traffic ~ points)"))
        roofline["hbm_frac_measured"] = bpp * N / avg_launch_s / 1e9 / HBM

    # sampled parity of the headline's initial right-hand side against the oracle
    parity = _guard("parity", lambda: _sampled_parity(solver, u0_dev, mu, args.parity_points))

    # end to end through the C ABI with host buffers (pinned): H2D state, RK4 step,
    # statistics, D2H state + statistics, every step
    e2e = _guard("e2e", lambda: _e2e(solver, u0_dev, dt, args.e2e_steps, world, step_ms))

    solver.close()
    del solver

    modes = {"fp64": {"value": value, "ms_per_step": ms / K,
                      "weights": "double-float (FP32 pairs), all else FP64"}}
    if not args.no_strict:
        def strict():
            Ks, Ws = 2, 1
            s2, u2, ms2, kt2, _, _ = timed_loop(ns3d.NS3D_FP64_STRICT, Ks, Ws, False, Ws + Ks)
            s2.close()
            del u2
            v2 = sum_over_ranks(float(N * RK_STAGES * Ks), world) / (ms2 * 1e-3) / 1e9
            return {"value": v2, "ms_per_step": ms2 / Ks, "steps": Ks, "weights": "FP64",
                    "speed_vs_fp64": v2 / value, "roofline": roofline_of(kt2, OPS_DIR_STRICT, "NS3D_FP64_STRICT")}
        modes["fp64_strict"] = _guard("fp64_strict", strict)
    torch.cuda.empty_cache()
    if not args.no_fp32:
        modes["fp32_bulk"] = _guard("fp32_bulk", lambda: _fp32_compare(timed_loop, ud, st, n_cmp, K, W, value,
                                                                       world, N, ns3d))
    del ud
    torch.cuda.empty_cache()
    if not args.no_adjoint:
        modes["adjoint"] = _guard("adjoint", run_adjoint)
    torch.cuda.empty_cache()
    if not args.no_ensemble:
        modes["ensemble_48"] = _guard("ensemble_48", lambda: run_ensemble(args.ens_steps, args.cfl))
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def cpu_leg():
            u0_host = u0_dev.cpu().numpy()
            g, el_cpu, cores, what = cpu_oracle_sample(u0_host, mu, n, dt, full_step=False)
            return {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle",
                    "sample": f"{what} (the headline's initial state), {el_cpu:.1f} s on the host cores "
                              f"(plain FP64 C oracle, OpenMP over lines/points)"}
        cpu = _guard("cpu_baseline", cpu_leg)
    del u0_dev
    torch.cuda.empty_cache()
    if args.big > 0:
        modes["big_1024"] = _guard("big_1024", lambda: run_big(args.big, args.big_steps, args.cfl,
                                                               n_sample=args.big_points))
        torch.cuda.empty_cache()

    if rank == 0:
        cfg = workload_config(n, args.cfl, mu, dt)
        cfg["precision"] = "NS3D_FP64: FP64 state/candidates/values/Roe/viscous/RK, WENO weights double-float"
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": cfg,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "kernel_ms": {k: v[0] for k, v in ktimes.items()}, "clocks": clk, "parity_rhs_sampled": parity,
                "modes": modes,
                "final_stats": {"after_steps": W + K, "ke": float(st[W + K, 5]), "enstrophy": float(st[W + K, 6]),
                                "status_ok": status_ok}}
        print(json.dumps(line), flush=True)


def _sampled_parity(solver, u_dev, mu, points: int) -> dict:
    import torch
    if points <= 0:
        return None
    rhs = torch.empty_like(u_dev)
    solver.rhs(u_dev, rhs)
    solver.check()
    out = window_oracle_check(u_dev, rhs, mu, points)
    del rhs
    torch.cuda.empty_cache()
    return out


def _e2e(solver, u0_dev, dt, steps: int, world: int, device_step_ms: float) -> dict:
    """ns3d_step_host with a pinned host state: H2D, one RK4 step, statistics, D2H every step;
    with the pinned-copy bandwidth of this machine and the share of the copy time hidden behind
    the kernels."""
    import torch
    from paper_2211_16718_gb300 import ns3d
    n = u0_dev.shape[-1]
    uh_t = u0_dev.cpu().pin_memory()
    uh = uh_t.numpy()
    solver.step_host(uh, dt, 1)  # warm-up (allocates the device copy and the copy stream)
    barrier(world)
    solver.timing_enable(True)
    t0 = time.perf_counter()
    for _ in range(steps):
        solver.step_host(uh, dt, 1)
    el = max_over_ranks(time.perf_counter() - t0, world)
    kt = solver.timing_read()
    solver.timing_enable(False)
    kernel_ms = sum(v[0] for v in kt.values()) / steps
    pts = sum_over_ranks(float(n ** 3 * RK_STAGES * steps), world)
    state_bytes = 5 * n ** 3 * 8
    # pinned-copy bandwidth of this machine, one whole state each way
    dev = torch.empty_like(u0_dev)
    stream = torch.cuda.current_stream()
    bw = {}
    for name, (dst, src) in (("h2d", (dev, uh_t)), ("d2h", (uh_t, dev))):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        bw[name] = 3 * state_bytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del dev
    # the same call with no step: the state in and out (serial copies) and the statistics
    solver.step_host(uh, dt, 0)
    t0 = time.perf_counter()
    for _ in range(3):
        solver.step_host(uh, dt, 0)
    t_call_copies = (time.perf_counter() - t0) / 3
    t_copy = state_bytes / (bw["h2d"] * 1e9) + state_bytes / (bw["d2h"] * 1e9)
    t_step = el / steps
    serial = device_step_ms * 1e-3 + t_copy
    return {"value": pts / el / 1e9, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
            "d2h_bytes_per_step": state_bytes + 8 * ns3d.NS3D_STATS_NDOUBLE,
            "call": "ns3d_step_host (pinned host state in, 1 RK4 step + statistics, state out)",
            "steps": steps, "ms_per_step": t_step * 1e3, "timer": "host perf_counter around the synchronising calls",
            "pinned_copy_gbs": bw, "copy_ms_per_step_serial": t_copy * 1e3,
            "call_without_steps_ms": t_call_copies * 1e3,
            "device_ms_per_step": device_step_ms,
            "kernel_ms_per_step_during_e2e": kernel_ms,
            "copy_time_hidden_frac": max(0.0, min(1.0, (serial - t_step) / t_copy)) if t_copy > 0 else None}


def _fp32_compare(timed_loop, u64, st64, n_cmp, K, W, value64, world, N, ns3d) -> dict:
    """FP32-bulk over the same steps from the same state and dt: speed, and its error against
    the FP64 path after n_cmp steps (KE and enstrophy every step, field max-norm at the end)."""
    import numpy as np
    s3, u3, ms3, kt3, st3, _ = timed_loop(ns3d.NS3D_FP32_BULK, K, W, False, n_cmp)
    s3.close()
    v3 = sum_over_ranks(float(N * RK_STAGES * K), world) / (ms3 * 1e-3) / 1e9
    a, b = st64[: n_cmp + 1], st3[: n_cmp + 1]
    diff = (u3 - u64).abs().reshape(5, -1).amax(dim=1).cpu().numpy()
    scale = u64.abs().reshape(5, -1).amax(dim=1).cpu().numpy()
    del u3
    return {"value": v3, "ms_per_step": ms3 / K, "speedup_vs_fp64": v3 / value64,
            "arithmetic": "FP32 indicators, weights, interface values, Roe flux; FP64 state, difference, "
                          "viscous terms, RK, reductions",
            "steps_compared": n_cmp, "dt": "the FP64 headline's",
            "ke_rel_err_max_over_steps": float((np.abs(b[:, 5] - a[:, 5]) / np.abs(a[:, 5])).max()),
            "enstrophy_rel_err_max_over_steps": float((np.abs(b[:, 6] - a[:, 6]) / np.abs(a[:, 6])).max()),
            "ke_final": [float(a[-1, 5]), float(b[-1, 5])], "enstrophy_final": [float(a[-1, 6]), float(b[-1, 6])],
            "field_maxnorm_rel_err": float(diff.max() / scale.max()),
            "field_maxnorm_rel_err_per_variable": (diff / scale).tolist(),
            "mass_rel_drift": float(abs(b[-1, 0] - b[0, 0]) / abs(b[0, 0])),
            "energy_rel_drift": float(abs(b[-1, 4] - b[0, 4]) / abs(b[0, 4])),
            "status_ok": bool(np.all(b[:, 10] == 0)),
            "kernel_ms_per_step": {k: v[0] / K for k, v in kt3.items() if v[1] > 0},
            "roofline": _fp32_roofline(kt3, N)}


def _fp32_roofline(kt, N) -> dict:
    """Roofline of the FP32-bulk direction pass (k_dir32): DRAM traffic (ncu, per point, keyed
    to the kernel code) and the method's algorithmic bytes over the live average launch time,
    against the measured HBM copy peak; the issue rate against the issue peak."""
    dir_ms = sum(kt[k][0] for k in ("dir_x", "dir_y", "dir_z"))
    launches = sum(kt[k][1] for k in ("dir_x", "dir_y", "dir_z"))
    avg_s = dir_ms / launches * 1e-3
    hbm = measured_peaks()["hbm_gbs"]
    out = {"kernel": "k_dir32 (FP32-bulk direction pass)", "avg_launch_ms": avg_s * 1e3,
           "method_hbm_frac": 60.0 * N / avg_s / 1e9 / hbm, "hbm_peak_gbs": hbm, "bound": None}
    sha = kernel_source_sha(KDIR32_SOURCES)
    tr = ncu_traffic_per_point("k_dir32", sha)
    if tr is not None:
        out["traffic"] = tr[0] * N
        out["hbm_frac_measured"] = tr[0] * N / avg_s / 1e9 / hbm
        out["traffic_source"] = f"ncu dram read+write per launch at {tr[2]}^3 ({tr[1]})"
    iss = ncu_issue_per_point("k_dir32", sha)
    if iss is not None:
        out["issue_frac"] = iss[0] * N / avg_s / 1e9 / ISSUE_PEAK_G
    if tr is not None and iss is not None:
        out["bound"] = "alu" if out["issue_frac"] >= out["hbm_frac_measured"] else "hbm"
    return out


ADJ_N, ADJ_STEPS, ADJ_EVERY, ADJ_MU, ADJ_CFL, ADJ_FD_DIRS, ADJ_FD_EPS = 64, 256, 16, 2.5e-4, 0.5, 8, 1e-6


def fd_direction(u, seed: int):
    """Seeded Gaussian direction, each field scaled to that field's RMS (the three momentum
    components share the RMS of |rho v|, so that the zero w-momentum of the vortex is
    perturbed too)."""
    import numpy as np
    g = np.random.default_rng(seed).normal(size=u.shape)
    rms = lambda a: float(np.sqrt(np.mean(a * a)))
    s_m = float(np.sqrt(np.mean(u[1] ** 2 + u[2] ** 2 + u[3] ** 2)))
    scales = [rms(u[0]), s_m, s_m, s_m, rms(u[4])]
    for v in range(5):
        g[v] *= scales[v] / rms(g[v])
    return g


def run_adjoint(n: int = ADJ_N, nsteps: int = ADJ_STEPS, every: int = ADJ_EVERY, n_fd: int = ADJ_FD_DIRS,
                oracle_steps: int = 16, kernel_sizes=(ADJ_N,)) -> dict:
    """Gradient of the mean kinetic energy at step nsteps with respect to the initial
    state of a Taylor-Green vortex (Re = 400: mu_eff = 2.5e-4 at Mach 0.1), by the
    checkpointed reverse sweep; its cost against the forward path, central differences
    of the GPU forward path along seeded directions, and the oracle's forward-mode
    derivative over the first oracle_steps steps."""
    import numpy as np
    import torch
    from oracle import dual_oracle as DO
    from oracle import oracle as O
    from paper_2211_16718_gb300 import inputs as I
    from paper_2211_16718_gb300 import ns3d

    u0 = I.taylor_green(n, v0=0.1)
    s = ns3d.Solver(n, n, n, mu_eff=ADJ_MU)
    ud = torch.from_numpy(u0.copy()).cuda()
    dt = s.dt_from_cfl(ud, ADJ_CFL)
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # warm-up (kernels, adjoint buffers, checkpoints)
    x = ud.clone()
    s.traj_forward(x, dt, 4, 2)
    g = torch.empty_like(x)
    s.functional(x, "ke", grad=g, value=False)
    s.traj_vjp(g)
    torch.cuda.synchronize()

    x = ud.clone()
    ms_fwd = timed(lambda: s.rk_step(x, dt, nsteps))
    x = ud.clone()
    ms_rec = timed(lambda: s.traj_forward(x, dt, nsteps, every))
    J, g = s.functional(x, "ke", grad=True)
    ms_adj = timed(lambda: s.traj_vjp(g))
    s.check()
    grad = g.cpu().numpy()

    def J_of(y):
        xd = torch.from_numpy(y).cuda()
        s.rk_step(xd, dt, nsteps)
        return s.functional(xd, "ke")[0]

    fd = []
    for seed in range(n_fd):
        w = fd_direction(u0, seed)
        d_fd = (J_of(u0 + ADJ_FD_EPS * w) - J_of(u0 - ADJ_FD_EPS * w)) / (2 * ADJ_FD_EPS)
        d_ad = float((grad * w).sum())
        fd.append({"seed": seed, "fd": d_fd, "adjoint": d_ad, "rel_diff": abs(d_fd - d_ad) / abs(d_ad)})

    # the oracle's forward-mode derivative of KE after oracle_steps steps along direction 0
    w0 = fd_direction(u0, 0)
    x = ud.clone()
    s.traj_forward(x, dt, oracle_steps, every)
    _, g2 = s.functional(x, "ke", grad=True)
    s.traj_vjp(g2)
    d_gpu = float((g2.cpu().numpy() * w0).sum())
    DO.build()
    DO.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    xN, dN = DO.rk_step_jvp(O.Params(n, n, n, mu_eff=ADJ_MU), u0, w0, dt, oracle_steps, "rk4")
    d_or = float(DO.stats_jvp(O.Params(n, n, n, mu_eff=ADJ_MU), xN, dN)[1][5])
    t_or = time.perf_counter() - t0

    # kernel level: one RHS against one RHS vector-Jacobian product
    kern = {}
    for m in kernel_sizes:
        um, mu_m = (I.taylor_green(m, v0=0.1), ADJ_MU) if m == n else hit_state(m)
        sm = ns3d.Solver(m, m, m, mu_eff=mu_m)
        a = torch.from_numpy(um).cuda()
        lam = a.flip(1)  # any non-constant field (J^T applied to a constant is zero)
        out = torch.empty_like(a)
        for _ in range(3):
            sm.rhs(a, out)
            sm.rhs_vjp(a, lam, out)
        reps = 10
        ms_r = timed(lambda: [sm.rhs(a, out) for _ in range(reps)]) / reps
        ms_v = timed(lambda: [sm.rhs_vjp(a, lam, out) for _ in range(reps)]) / reps
        sm.timing_enable(True)
        sm.rhs_vjp(a, lam, out)
        kt = sm.timing_read()
        sm.timing_enable(False)
        kern[f"{m}^3"] = {"rhs_ms": ms_r, "rhs_vjp_ms": ms_v, "vjp_over_rhs": ms_v / ms_r,
                          "rhs_vjp_gpts": m ** 3 / (ms_v * 1e-3) / 1e9,
                          "vjp_kernel_ms": {k: v[0] for k, v in kt.items() if v[1] > 0}}
        sm.close()
        del a, lam, out
    s.close()
    errs = [f["rel_diff"] for f in fd]
    return {"workload": f"Taylor-Green vortex {n}^3, Mach 0.1, mu_eff {ADJ_MU} (Re 400), RK4, dt at CFL "
                        f"{ADJ_CFL}; J = mean kinetic energy at step {nsteps}; gradient w.r.t. the 5 initial fields",
            "dt": dt, "steps": nsteps, "checkpoint_every": every, "J": J,
            "forward_ms": ms_fwd, "forward_recorded_ms": ms_rec, "adjoint_ms": ms_adj,
            "adjoint_over_forward": ms_adj / ms_fwd,
            "adjoint_ms_per_step": ms_adj / nsteps, "forward_ms_per_step": ms_fwd / nsteps,
            "fd_check": {"directions": n_fd, "eps": ADJ_FD_EPS,
                         "direction": "seeded Gaussian, each field scaled to its RMS (momenta: RMS of |rho v|)",
                         "max_rel_diff": max(errs), "median_rel_diff": statistics.median(errs), "per_direction": fd},
            "oracle_check": {"steps": oracle_steps, "direction_seed": 0, "adjoint": d_gpu, "oracle_forward_mode": d_or,
                             "rel_diff": abs(d_gpu - d_or) / abs(d_or), "oracle_seconds": t_or},
            "kernels": kern}


def window_oracle_check(u_dev, rhs_dev, mu: float, n_sample: int, seed: int = 0, tile: int = 24) -> dict:
    """Compare the GPU right-hand side at sampled points of an n^3 grid with the oracle
    evaluated on the 11^3 periodic window centred on each point: the RHS at a point
    reads the state within 4 points of it along the axes, so the window's own
    periodic wrap never reaches the centre's stencil and the oracle's value is exact.
    Besides the random points: the grid corners and points on the periodic seams and on
    the tile edges of the direction passes (multiples of `tile` along each axis)."""
    import numpy as np
    import torch
    from oracle import oracle as O
    n = u_dev.shape[-1]
    r, w = 5, 11
    h = 2 * math.pi / n
    P = O.Params(w, w, w, lx=w * h, ly=w * h, lz=w * h, mu_eff=mu)
    scale = float(rhs_dev.abs().max().item())
    rng = np.random.default_rng(seed)
    edge = sorted({0, 1, n - 1, n - 2, tile - 1, tile, tile + 1, n // 2, (n // tile) * tile % n,
                   ((n // tile) * tile - 1) % n})
    special = [(a, b, c) for a in (0, n - 1) for b in (0, n - 1) for c in (0, n - 1)]
    special += [(int(rng.choice(edge)), int(rng.choice(edge)), int(rng.integers(0, n))) for _ in range(n_sample // 8)]
    special += [(int(rng.integers(0, n)), int(rng.choice(edge)), int(rng.choice(edge))) for _ in range(n_sample // 8)]
    nrand = max(0, n_sample - len(special))
    pts = np.concatenate([np.array(special, dtype=np.int64).reshape(-1, 3),
                          rng.integers(0, n, size=(nrand, 3))])[:max(n_sample, 8)]
    off = np.arange(-r, r + 1)
    ix = (pts[:, 0:1] + off) % n
    iy = (pts[:, 1:2] + off) % n
    iz = (pts[:, 2:3] + off) % n
    flat = (iz[:, :, None, None] * n + iy[:, None, :, None]) * n + ix[:, None, None, :]  # [P, w, w, w]
    fi = torch.from_numpy(flat.reshape(-1)).to(u_dev.device)
    wins = u_dev.reshape(5, -1)[:, fi].reshape(5, len(pts), w, w, w).cpu().numpy()
    ci = torch.from_numpy(((pts[:, 2] * n + pts[:, 1]) * n + pts[:, 0]).astype(np.int64)).to(u_dev.device)
    got = rhs_dev.reshape(5, -1)[:, ci].cpu().numpy()
    worst = 0.0
    for q in range(len(pts)):
        ref = O.rhs_points(P, np.ascontiguousarray(wins[:, q]), [(r * w + r) * w + r])[0]
        worst = max(worst, float(np.abs(got[:, q] - ref).max()) / scale)
    return {"points": int(len(pts)), "special_points": int(min(len(special), len(pts))),
            "window": "11^3 periodic, centred", "max_rel_err": worst,
            "normalisation": "max |R| over the whole grid (all 5 variables)",
            "special": "grid corners, periodic seams and direction-pass tile edges"}


def run_big(n: int, steps: int, cfl: float, n_sample: int = 24) -> dict:
    """The decaying-turbulence problem on an n^3 grid (1024^3: 43 GB per state) with
    SSP-RK3: storage chosen automatically (viscous fluxes one direction at a time when
    the full scratch would not fit), one RHS checked against the oracle on sampled
    windows, then timed steps with statistics every step."""
    import numpy as np
    import torch
    from paper_2211_16718_gb300 import inputs as I
    from paper_2211_16718_gb300 import ns3d
    t0 = time.perf_counter()
    u = I.isotropic_turbulence_device(n, seed=0)
    torch.cuda.synchronize()
    t_ic = time.perf_counter() - t0
    torch.cuda.empty_cache()
    mu = I.hit_mu_eff()
    s = ns3d.Solver(n, n, n, mu_eff=mu, rk=ns3d.NS3D_SSPRK3)
    info0 = s.storage_info()
    rhs = torch.empty_like(u)
    s.rhs(u, rhs)
    s.check()
    parity = window_oracle_check(u, rhs, mu, n_sample)
    del rhs
    torch.cuda.empty_cache()
    dt = s.dt_from_cfl(u, cfl)
    st0 = s.stats(u)
    s.rk_step(u, dt, 1)  # allocates the stage states
    torch.cuda.synchronize()
    stats_buf = torch.zeros((steps, ns3d.NS3D_STATS_NDOUBLE), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    s.timing_enable(True)
    clocks.start()
    e0.record(stream)
    for i in range(steps):
        s.rk_step(u, dt, 1)
        s.stats_async(u, stats_buf[i])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    kt = s.timing_read()
    s.timing_enable(False)
    st = stats_buf.cpu().numpy()
    st1 = s.stats(u)
    info1 = s.storage_info()
    free_b, total_b = torch.cuda.mem_get_info()
    s.close()
    drift = {k: abs(st1[k] - st0[k]) / max(abs(st0[k]), 1e-300) for k in ("mass", "energy")}
    drift["momentum_abs"] = max(abs(st1[k] - st0[k]) for k in ("momx", "momy", "momz"))
    return {"workload": f"decaying isotropic turbulence {n}^3, FP64, SSP-RK3, dt at CFL {cfl}",
            "grid": n, "steps": steps, "dt": dt, "gpts": n ** 3 * 3 * steps / (ms * 1e-3) / 1e9,
            "ms_per_step": ms / steps, "rhs_per_step": 3,
            "storage": "lean" if info1["storage"] == ns3d.NS3D_STORAGE_LEAN else "full",
            "library_bytes_after_init": info0["device_bytes"], "library_bytes": info1["device_bytes"],
            "state_bytes": 5 * 8 * n ** 3, "device_free_bytes": free_b, "device_total_bytes": total_b,
            "ic_seconds": t_ic, "ic": "hit_velocity(64, seed 0) spectrally interpolated on the device",
            "parity_rhs_sampled": parity, "conservation_drift": drift,
            "ke": [float(st0["ke"])] + [float(x) for x in st[:, 5]],
            "enstrophy": [float(st0["enstrophy"])] + [float(x) for x in st[:, 6]],
            "status_ok": bool(np.all(st[:, 10] == 0)), "clocks": clk,
            "kernel_ms_per_step": {k: v[0] / steps for k, v in kt.items() if v[1] > 0}}


def run_study_fp32(args, local):
    """FP64 path vs FP32-bulk mode on the decaying-turbulence workload: same initial state
    and dt, --steps RK4 steps each, KE and enstrophy logged every step on the device."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_2211_16718_gb300 import build as B
    B.build()
    from paper_2211_16718_gb300 import ns3d

    n, K = args.n, args.steps
    u0, mu = hit_state(n)
    res, finals, dt = {}, {}, None
    for name, prec in (("fp64", ns3d.NS3D_FP64), ("fp32_bulk", ns3d.NS3D_FP32_BULK)):
        s = ns3d.Solver(n, n, n, mu_eff=mu, precision=prec)
        ud = torch.from_numpy(u0.copy()).cuda()
        if dt is None:
            dt = s.dt_from_cfl(ud, args.cfl)
        log = torch.zeros((K + 1, ns3d.NS3D_STATS_NDOUBLE), dtype=torch.float64, device="cuda")
        s.stats_async(ud, log[0])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(K):
            s.rk_step(ud, dt, 1)
            s.stats_async(ud, log[i + 1])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = {"ms_per_step": ms / K, "gpts": n ** 3 * RK_STAGES * K / (ms * 1e-3) / 1e9,
                     "log": log.cpu().numpy()}
        s.close()
        finals[name] = ud.cpu().numpy()
        del ud
    a, b = res["fp64"]["log"], res["fp32_bulk"]["log"]
    diff = np.abs(finals["fp32_bulk"] - finals["fp64"]).reshape(5, -1).max(axis=1)
    scale = np.abs(finals["fp64"]).reshape(5, -1).max(axis=1)
    out = {"study": "fp32_bulk vs fp64", "workload": f"decaying isotropic turbulence {n}^3, seed 0, CFL {args.cfl}",
           "steps": K, "dt": dt,
           "fp64": {k: res["fp64"][k] for k in ("ms_per_step", "gpts")},
           "fp32_bulk": {k: res["fp32_bulk"][k] for k in ("ms_per_step", "gpts")},
           "speedup": res["fp64"]["ms_per_step"] / res["fp32_bulk"]["ms_per_step"],
           "ke_rel_err_max_over_steps": float((np.abs(b[:, 5] - a[:, 5]) / np.abs(a[:, 5])).max()),
           "enstrophy_rel_err_max_over_steps": float((np.abs(b[:, 6] - a[:, 6]) / np.abs(a[:, 6])).max()),
           "ke_final": [float(a[-1, 5]), float(b[-1, 5])], "enstrophy_final": [float(a[-1, 6]), float(b[-1, 6])],
           "field_maxnorm_rel_err_final": float(diff.max() / scale.max()),
           "field_maxnorm_rel_err_per_variable": (diff / scale).tolist(),
           "conservation_mass_rel_drift_fp32": float(abs(b[-1, 0] - b[0, 0]) / b[0, 0]),
           "conservation_energy_rel_drift_fp32": float(abs(b[-1, 4] - b[0, 4]) / b[0, 4])}
    print(json.dumps(out), flush=True)


ENSEMBLE_SIZES = (32, 48, 64, 96, 128)


def run_ensemble(steps: int, cfl: float, count: int = 48, cache_path=None, sizes_cycle=ENSEMBLE_SIZES) -> dict:
    """Ensemble of `count` decaying-turbulence realisations (seed i, grid sizes_cycle[i % len]^3,
    dt_i from CFL `cfl` of its own initial state): `steps` RK4 steps in each schedule (from
    the same initial states), after the autotuner has picked the tile shape per grid size and
    the graph's branch count."""
    import numpy as np
    import torch
    from paper_2211_16718_gb300 import inputs as I
    from paper_2211_16718_gb300 import ns3d

    sizes = [sizes_cycle[i % len(sizes_cycle)] for i in range(count)]
    host = [I.isotropic_turbulence(n, seed=i) for i, n in enumerate(sizes)]
    params = [ns3d.default_params(n, n, n, mu_eff=I.hit_mu_eff()) for n in sizes]
    pts = sum(n ** 3 for n in sizes)
    b = ns3d.Batch(params)
    states = [torch.from_numpy(h.copy()).cuda() for h in host]
    b.set_states(states)
    b.set_dt_from_cfl(cfl)
    t0 = time.perf_counter()
    tune = b.autotune(cache_path)
    tune_s = time.perf_counter() - t0
    shapes = {0: "24x4", 1: "16x4", 2: "40x2"}
    per_size = {}
    for i, n in enumerate(sizes):
        per_size.setdefault(f"{n}^3", {"tile_shape": shapes[tune["variants"][i]],
                                       "ms_per_step_by_shape": dict(zip(shapes.values(), tune["ms_variants"][i]))})
    out = {"instances": count, "sizes": f"seed i: {tuple(sizes_cycle)}[i % {len(sizes_cycle)}]^3", "points": pts,
           "steps": steps, "autotune": {"per_size": per_size, "graph_branches": tune["branches"],
                                        "ms_per_step_by_branches": {str(k + 1): m for k, m in
                                                                    enumerate(tune["ms_branches"]) if m > 0},
                                        "seconds": tune_s}}
    finals = {}
    for schedule in ("sequential", "graph", "persistent"):
        for s, h in zip(states, host):
            s.copy_(torch.from_numpy(h))
        b.step(1, schedule)  # warm-up (and graph capture)
        for s, h in zip(states, host):
            s.copy_(torch.from_numpy(h))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(steps, schedule)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[schedule] = {"ms": ms, "gpts": pts * RK_STAGES * steps / (ms * 1e-3) / 1e9}
        finals[schedule] = [s.cpu().numpy() for s in states[:5]]
    b.check()
    info = b.info()
    out["persistent_in_graph"] = info["persistent_in_graph"]
    out["persistent_ctas_per_sm"] = info["persistent_ctas_per_sm"]
    out["persistent_tile_shape"] = shapes[info["variant"]]
    out["schedules_bitwise_equal"] = all(np.array_equal(a, c) for k in ("graph", "persistent")
                                         for a, c in zip(finals[k], finals["sequential"]))
    out["speedup_persistent_vs_sequential"] = out["persistent"]["gpts"] / out["sequential"]["gpts"]
    out["speedup_graph_vs_sequential"] = out["graph"]["gpts"] / out["sequential"]["gpts"]
    b.close()
    return out


def main():
    args = parse()
    if args.study == "ensemble":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2211_16718_gb300 import build as B
        B.build()
        if args.ens_count > 0:
            sizes = tuple(int(x) for x in args.ens_sizes.split(","))
            print(json.dumps({"study": "ensemble", "custom": run_ensemble(args.steps, args.cfl, count=args.ens_count,
                                                                           sizes_cycle=sizes)}), flush=True)
            return
        print(json.dumps({"study": "ensemble", "ensemble_48_uneven": run_ensemble(args.steps, args.cfl),
                          "small_instances": run_ensemble(args.steps, args.cfl, count=256,
                                                          sizes_cycle=(12, 16, 20, 24))}), flush=True)
        return
    if args.study == "fp32":
        run_study_fp32(args, int(os.environ.get("LOCAL_RANK", "0")))
        return
    if args.study == "oracle":
        print(json.dumps(run_study_oracle()), flush=True)
        return
    if args.study == "big":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2211_16718_gb300 import build as B
        B.build()
        print(json.dumps({"study": "big", "result": run_big(args.big, args.steps, args.cfl, n_sample=args.big_points)}),
              flush=True)
        return
    if args.study == "vjp":
        # --steps K right-hand-side vector-Jacobian products of the --n^3 turbulence state
        # (a small, fixed launch sequence for profilers)
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2211_16718_gb300 import build as B
        B.build()
        from paper_2211_16718_gb300 import ns3d
        u, mu = hit_state(args.n)
        prec = ns3d.NS3D_FP64_STRICT if args.precision == "strict" else ns3d.NS3D_FP64
        sv = ns3d.Solver(args.n, args.n, args.n, mu_eff=mu, precision=prec)
        a = torch.from_numpy(u).cuda()
        lam = a.flip(1)  # any non-constant field (J^T applied to a constant is zero)
        out = torch.empty_like(a)
        for _ in range(args.steps):
            sv.rhs_vjp(a, lam, out)
        sv.check()
        torch.cuda.synchronize()
        print(json.dumps({"study": "vjp", "n": args.n, "calls": args.steps,
                          "out_maxabs": float(out.abs().max().item())}), flush=True)
        sv.close()
        return
    if args.study == "adjoint":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2211_16718_gb300 import build as B
        B.build()
        print(json.dumps({"study": "adjoint", "taylor_green_64_ke_gradient": run_adjoint(kernel_sizes=(ADJ_N, 256))}),
              flush=True)
        return
    if args.impl == "reference":
        # the oracle runs on the host of rank 0 only; other ranks exit without work
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_init()
    run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
