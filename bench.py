#!/usr/bin/env python
"""Benchmark of the LP granular-flow step on GB300: particle-updates/s.

Default workload: the single cylindrical column collapse (radius 0.02 m,
height 2R, lattice spacing R/50 with +-0.05h jitter, 785,398 particles,
mu(I) parameters of the benchmark set, dt 1e-5 s), mixed-precision fits, the
step replayed as a captured CUDA graph. One "step" is one full LP step: cell
sort, neighbour search with floor mirrors, pass-1 fits, pass-2 fits with the
mu(I) closure and the update of V, u and x.

Every `restart_every` steps the state is reset to the initial column (a
device copy inside the timed region): the inertial-regime equations grow
short waves (they are ill-posed for mu(I) < 6/7), which blow this column up
after a few tens of steps at this spacing, and timing a blown-up state would
time a different workload.

Prints ONE JSON line (rank 0). `--impl reference` times the CPU oracle.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-updates/s per GB300 (full LP mu(I) step) & % HBM roofline; mixed vs FP64"
UNIT = "particle-updates/s"
B_ALG = 128.0  # algorithmic bytes per particle update: read+write x,u,V (112) + |gdot| (16)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("mixed_ff", "mixed", "fp64"), default="mixed_ff")
    ap.add_argument("--restart-every", type=int, default=10)
    ap.add_argument("--spacing-div", type=int, default=50,
                    help="lattice spacing R/spacing_div of the cylinder (50: the benchmark's "
                         "785k particles; smaller values give smaller cases for profiling)")
    ap.add_argument("--skin", type=float, default=0.1,
                    help="Verlet skin in lattice spacings (0: full search every step)")
    ap.add_argument("--free-surface", action="store_true",
                    help="ghost particles at free boundaries (Sec. 3.1 item 9)")
    ap.add_argument("--no-free-surface", action="store_true",
                    help="skip the line with free-surface ghosts")
    ap.add_argument("--no-moving", action="store_true",
                    help="skip the line with the column in a spreading flow")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint line (the 200-step adjoint column)")
    ap.add_argument("--no-collapse", action="store_true",
                    help="skip the column-collapse validation line (a = 0.6 column, Sec. 4.2.1)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large-column line (21M particles at the headline spacing)")
    ap.add_argument("--no-layer", action="store_true",
                    help="skip the layer-compaction validation line (periodic layer, Sec. 4.1)")
    ap.add_argument("--no-heun", action="store_true",
                    help="skip the line with Heun's method")
    ap.add_argument("--no-periodic", action="store_true",
                    help="skip the periodic-layer line (Sec. 3.1 item 9, Sec. 4)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the lp_fit_derivatives line (derivative-operator sweep)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison line")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-columns line")
    return ap.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------------------ clocks

def clock_summary(lines, t0: float, t1: float, interval_ms: int) -> dict:
    """Summary of nvidia-smi sample lines [(host time, csv line)] read between
    host times t0 and t1 (the first one after t1 if none fell inside): median
    and maximum SM clock, peak power, and the throttle reasons seen active."""
    inside = [ln for ts, ln in lines if t0 <= ts <= t1]
    window = "timed region"
    if not inside:
        inside = [ln for ts, ln in lines if ts > t1][:1]
        window = "first sample after the timed region"
    sm, smax, reasons, power = [], [], set(), []
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    for line in inside:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
            power.append(float(f[3]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "samples": len(sm), "interval_ms": interval_ms, "window": window,
            "reasons": sorted(reasons)}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region: sampling
    starts (first line read) before the region opens; the samples kept are
    those read between the host times that bracket it."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.gpu = gpu_index
        self.interval = interval_ms
        self.proc = None
        self.lines = []
        self.reader = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval), "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        t = time.perf_counter()
        while not self.lines and time.perf_counter() - t < 10.0 and self.proc.poll() is None:
            time.sleep(0.005)

    def stop(self, t0: float, t1: float) -> dict:
        """Summary of the samples read between host times t0 and t1 (the
        nearest one after t1 if none fell inside)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(2.5 * self.interval / 1e3)  # the sample in flight at t1
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        if self.reader is not None:
            self.reader.join(timeout=5)
        return clock_summary(self.lines, t0, t1, self.interval)


# ------------------------------------------------------------- our path

def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


KERNEL_SOURCES = ("fit.cu", "fit_bodies.cuh", "lp_internal.cuh", "ff_split.cuh")


def kernel_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the fit kernels' sources."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2206_14061_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(key: str):
    """DRAM bytes (read + write) per launch of the roofline kernels from a
    committed ncu summary, if it was taken on the current kernel sources
    (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(path))[key]
    except (OSError, ValueError, KeyError):
        return None
    if t.get("src_sha256_16") != kernel_source_hash():
        return None
    return t.get("bytes_per_launch_full")


PREC = {"fp64": 0, "mixed": 1, "mixed_ff": 2}
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate
FP32_PEAK_TOPS = 40.27    # 152 SMs x 128 FP32 lanes x 2.07 GHz, one op per lane and cycle
FP32_PEAK_TFLOPS = 80.54  # the same lanes issuing FMAs (2 flops each)


def pass1_method_flops(rows: float, n: int) -> float:
    """The pass-1 phase's own arithmetic, independent of how a precision mode
    carries it: per particle the Taylor rows (about 14 flops per row for the
    offsets and quadratic terms), the Gram matrix and three right-hand sides
    (81 multiply-adds = 162 flops per row), and about 1000 flops for the 9x9
    Cholesky factor and three solves."""
    return 176.0 * rows + 1000.0 * n


def pass1_work(prec: str, rows: float, n: int):
    """Instructions one pass-1 phase issues in its own pipe, and that pipe's
    peak (a utilisation figure; the method's own flops are pass1_method_flops).

    FP64 (flops, FMA = 2): per stencil row 6 (offsets) + 6 (quadratic terms) +
    62 (31 moments) + 3 (differences) + 54 (3 right-hand sides x 9) = 131; per
    particle about 1000 (9x9 Cholesky, three solves, derived quantities).
    MIXED (FP64 flops only; the FP32 moments run on the FP32 pipe): per row 6 +
    9 + 3 + 54 (residual) + 54 (A^T r) = 126; per particle about 550.
    MIXED_FF (FP32 lane operations: every FP32 add, multiply or FMA is one op,
    since float-float arithmetic is mostly additions): per row 75 (float-float
    offsets and quadratic terms) + 6 (Taylor scaling) + 348 (31 moments) +
    363 (3 right-hand sides) = 792, counted once although both fit kernels
    form the row; per particle 183 (Gram matrix) + 2016 (float-float Cholesky)
    + 3132 (three float-float solves) = 5331."""
    if prec == "mixed_ff":
        return (792.0 * rows + 5331.0 * n, "T FP32 lane-ops/s", FP32_PEAK_TOPS,
                "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz")
    flops = 131.0 * rows + 1000.0 * n if prec == "fp64" else 126.0 * rows + 550.0 * n
    return (flops, "TFLOP/s (FP64)", FP64_PEAK_TFLOPS,
            "nominal FP64 rate (no measured FP64 peak in MEASURED_PEAKS.json)")


PASS1_KERNELS = {"mixed_ff": "k_gram_ff + k_pass1_ff_rows + k_pass1_ff_solve", "mixed": "k_pass1", "fp64": "k_pass1"}


def our_arm(args):
    import torch
    import torch.distributed as dist

    from paper_2206_14061_gb300 import capi, workloads as W

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    capi.lib(build_if_missing=True)

    wl = W.cylinder(spacing_div=args.spacing_div)
    pd = W.param_dict(wl)
    n = wl.n
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")}
    init = {k: torch.tensor(wl.state[k], device=dev) for k in capi.FIELDS}
    st = {k: v.clone() for k, v in init.items()}
    ctx = capi.Context(n, cap=64)
    stream = torch.cuda.Stream(device=dev)
    R = max(1, args.restart_every)

    mode = {"fs": int(args.free_surface), "ts": 0}  # free-surface ghosts, time scheme

    def params(prec, graph=1):
        return dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
                    floor_z=0.0, mirror_mode=1,
                    precision=PREC[prec],
                    rebuild_every=1, launch_mode=graph, skin=args.skin * pd["h"],
                    free_surface=mode["fs"], time_scheme=mode["ts"])

    def run(nsteps, prec, graph=1):
        done = 0
        with torch.cuda.stream(stream):
            while done < nsteps:
                k = min(R, nsteps - done)
                for f in capi.FIELDS:
                    st[f].copy_(init[f])
                capi.lp_step(ctx, st, mui, eos, params(prec, graph), pd["dt"], k, stream=stream)
                done += k

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def timed(nsteps, prec, graph=1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        run(nsteps, prec, graph)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    def bench(prec):
        run(args.warmup, prec)
        ctx.sync(stream)
        ctx.phase_times(stream)  # reset counters
        clocks = ClockSampler(local)
        clocks.start()
        t0 = time.perf_counter()
        ms = timed(args.steps, prec)
        ck = clocks.stop(t0, time.perf_counter())
        pt = ctx.phase_times(stream)
        diag = ctx.sync(stream, raise_on_error=False)
        # per-kernel durations, measured with events on the launch stream
        ctx.profile(True)
        prof_steps = min(args.steps, R)
        run(prof_steps, prec, graph=0)
        prof = ctx.phase_times(stream)
        ctx.profile(False)
        ctx.sync(stream, raise_on_error=False)
        return ms, ck, pt, diag, prof, prof_steps

    ms, clocks, pt, diag, prof, prof_steps = bench(args.precision)
    updates = n * args.steps * world
    value = updates / (ms / 1e3)
    mean_m = diag["n_stencil_rows"] / max(diag["n_stencils"], 1)

    peaks = _peaks()
    per_phase = {k: v / max(prof["steps"], 1) for k, v in prof["ms"].items()}
    dom = max(per_phase, key=per_phase.get)
    work, punit, peak, psrc = pass1_work(args.precision, mean_m * n, n)
    mflops = pass1_method_flops(mean_m * n, n)
    kname = PASS1_KERNELS[args.precision]
    roof = {"kernel": {"pass1": kname, "pass2": "k_pass2", "neighbors": "k_neighbors",
                       "sort": "sort kernels"}[dom]}
    if dom == "pass1":
        sec = per_phase["pass1"] / 1e3
        ach = mflops / sec / 1e12
        traffic = _traffic(f"pass1_{args.precision}")
        roof.update(bound="alu", achieved=ach, peak=FP32_PEAK_TFLOPS,
                    unit="TFLOP/s (the method's FP32 flops)", frac=ach / FP32_PEAK_TFLOPS,
                    peak_source="derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                    flops_per_launch=mflops, ms_per_launch=per_phase["pass1"], traffic=traffic,
                    traffic_over_alg=None if traffic is None else traffic / (B_ALG * n),
                    pipe={"achieved": work / sec / 1e12, "peak": peak, "unit": punit,
                          "frac": work / sec / 1e12 / peak, "peak_source": psrc,
                          "work_per_launch": work})
    else:
        roof.update(bound="alu", achieved=None, peak=FP32_PEAK_TFLOPS,
                    unit="TFLOP/s (the method's FP32 flops)", frac=None,
                    ms_per_launch=per_phase[dom], traffic=None)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_ach = value / world * B_ALG / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed_ff": "f32 (float-float) + f64",
                  "mixed": "f32+f64"}.get(args.precision, "f64"),
        "data": "synthetic (seeded jittered lattice column)",
        "config": {
            "workload": f"cylindrical column collapse R=0.02 m H=2R h=R/{args.spacing_div} "
                        f"jitter 0.05h ({n} particles), mu_s 0.38 mu_2 0.64 I0 0.28 d 5e-4 "
                        "rho 2500, "
                        "dt 1e-5, stencil radius 2.2h, no-slip floor mirrors",
            "precision": args.precision, "graph": True, "restart_every": R,
            "verlet_skin_h": args.skin, "free_surface_ghosts": bool(args.free_surface),
            "mean_stencil": mean_m, "parallelism": f"replicas x{world}",
            "l2": "per-step working set (state, stencils, factors) is larger than L2",
        },
        "roofline": roof,
        "hbm": {"bytes_per_update": B_ALG, "achieved_gbs": hbm_ach, "peak_gbs": hbm_peak,
                "frac": hbm_ach / hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
        "phase_ms_per_step": per_phase,
        "gpu_launches": pt["launches"],
        "clocks": clocks,
        "diag": {k: diag[k] for k in ("n_fallback", "n_gas", "n_quasistatic", "n_nonfinite",
                                      "min_stencil", "max_stencil")},
    }

    if not args.no_fp64:
        for other in ("fp64", "mixed", "mixed_ff"):
            if other == args.precision:
                continue
            mso, _, _, _, profo, _ = bench(other)
            pho = {k: v / max(profo["steps"], 1) for k, v in profo["ms"].items()}
            wo, uo, po, _ = pass1_work(other, mean_m * n, n)
            mt = mflops / (pho["pass1"] / 1e3) / 1e12
            line[other] = {"value": n * args.steps * world / (mso / 1e3),
                           "ms_per_step": mso / args.steps, "phase_ms_per_step": pho,
                           "pass1_method_tflops": mt, "pass1_method_frac": mt / FP32_PEAK_TFLOPS,
                           "pass1_achieved": wo / (pho["pass1"] / 1e3) / 1e12,
                           "pass1_unit": uo, "pass1_frac": wo / (pho["pass1"] / 1e3) / 1e12 / po}

    if not args.no_free_surface and not args.free_surface:
        # the same workload with free-surface ghost particles (Sec. 3.1 item 9)
        mode["fs"] = 1
        msg, _, _, dgg, profg, _ = bench(args.precision)
        mode["fs"] = 0
        line["free_surface"] = {
            "value": n * args.steps * world / (msg / 1e3), "unit": UNIT,
            "ms_per_step": msg / args.steps,
            "phase_ms_per_step": {k: v / max(profg["steps"], 1) for k, v in profg["ms"].items()},
            "ghost_entries_per_step": dgg["n_ghosts"] / max(args.steps, 1)}

    if not args.no_heun:
        # the same workload with Heun's method (two stages per step)
        mode["ts"] = 1
        msh, _, _, _, profh, _ = bench(args.precision)
        mode["ts"] = 0
        line["heun"] = {
            "value": n * args.steps * world / (msh / 1e3), "unit": UNIT,
            "ms_per_step": msh / args.steps,
            "phase_ms_per_step": {k: v / max(profh["steps"], 1) for k, v in profh["ms"].items()}}

    if not args.no_moving:
        # the same column in a spreading flow u_r = U (r/R)(z/H), U = 0.5 m/s
        # (zero at the no-slip floor): particles move up to 0.0125 h per step,
        # so the Verlet lists are searched every few steps instead of once per
        # restart, as in a collapsing column
        U, Rc, Hc = 0.5, wl.extra["R"], wl.extra["H"]
        rest = {k: init[k] for k in ("u", "v")}
        init["u"] = torch.tensor(U * wl.state["x"] / Rc * (wl.state["z"] / Hc), device=dev)
        init["v"] = torch.tensor(U * wl.state["y"] / Rc * (wl.state["z"] / Hc), device=dev)
        msv, _, _, dgv, profv, _ = bench(args.precision)
        init.update(rest)
        line["moving"] = {
            "workload": "the same column in a spreading flow u_r = 0.5 m/s (r/R)(z/H)",
            "value": n * args.steps * world / (msv / 1e3), "unit": UNIT,
            "ms_per_step": msv / args.steps,
            "phase_ms_per_step": {k: v / max(profv["steps"], 1) for k, v in profv["ms"].items()},
            "n_nonfinite": dgv["n_nonfinite"]}

    if not args.no_periodic:
        line["periodic"] = periodic_layer(args, dev, stream, world)

    if not args.no_e2e:
        line["e2e"] = e2e(args, ctx, wl, pd, mui, eos, params, dev, stream, world)

    if not args.no_batched:
        ctx.close()
        line["batched"] = batched(args, dev, stream, rank, world)

    if not args.no_adjoint and world == 1:
        line["adjoint"] = adjoint_line(dev, stream)
    if not args.no_large:
        line["large_column"] = large_line(args, dev, stream, world)
    if not args.no_collapse and world == 1:
        line["column_collapse"] = collapse_line(dev, stream)
    if not args.no_layer and world == 1:
        line["layer_compaction"] = layer_line(dev, stream)

    if not args.no_sweep and world == 1:
        line["derivative_sweep"] = derivative_sweep(args, dev, stream)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, pd, budget_s=20.0)

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batched(args, dev, stream, rank=0, world=1):
    """256 independent columns (log-uniform 2k-64k particles, aspect 0.5-6,
    mu_s 0.3-0.45) advanced together in one lp_step call per window, with the
    autotuned launch configuration, against per-column lp_step calls over the
    same steps. With several ranks each one steps its shard of the columns
    (dist.shard_state: contiguous columns balanced by particle count); nothing
    is exchanged, and the step time is the maximum over ranks."""
    import torch

    from paper_2206_14061_gb300 import capi, dist as D, workloads as W

    wl = W.columns()
    pd = W.param_dict(wl)
    sh = D.shard_state(wl.state, wl.column_offsets, rank, world, wl.mu_s_col)
    offs = sh["offsets"]
    ncol = len(offs) - 1
    n_local = int(offs[-1])
    base = {k: pd[k] for k in ("mu_2", "I0", "d", "rho_s")}
    mui_c = [dict(base, mu_s=float(m)) for m in sh["per_column"]]
    eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")}
    init = {k: torch.tensor(np.ascontiguousarray(v), device=dev) for k, v in sh["state"].items()}
    st = {k: v.clone() for k, v in init.items()}
    prm = dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
               floor_z=0.0, mirror_mode=1, precision=PREC[args.precision], rebuild_every=1,
               launch_mode=capi.LP_LAUNCH_GRAPH, skin=args.skin * pd["h"])
    ctx = capi.Context(max(n_local, 1), max_columns=max(ncol, 1), cap=64)
    tune = capi.lp_autotune(ctx, init, mui_c, eos, prm, pd["dt"], 3, column_offsets=offs,
                            stream=stream)
    steps = max(1, min(args.steps, args.restart_every))

    def reset():
        for k in capi.FIELDS:
            st[k].copy_(init[k])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def timed(fn):
        with torch.cuda.stream(stream):
            reset()
            fn()  # warm-up
            reset()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            fn()
        e1.record(stream)
        barrier()
        return D.max_over_ranks(e0.elapsed_time(e1), device=dev)

    modes = {}
    for name, mode in (("graph", capi.LP_LAUNCH_GRAPH), ("persistent", capi.LP_LAUNCH_PERSISTENT)):
        p = dict(prm, launch_mode=mode)
        modes[name] = timed(lambda: capi.lp_step(ctx, st, mui_c, eos, p, pd["dt"], steps,
                                                 column_offsets=offs, stream=stream))
    chosen = "persistent" if tune["launch_mode"] == capi.LP_LAUNCH_PERSISTENT else "graph"
    ms_b = modes[chosen]

    def phases(mode):
        """Per-phase device ms per step: CUDA events around the per-phase
        kernels, or the persistent kernel's own marks after each barrier."""
        ctx.profile(True)
        ctx.phase_times(stream)  # reset
        with torch.cuda.stream(stream):
            reset()
            capi.lp_step(ctx, st, mui_c, eos, dict(prm, launch_mode=mode), pd["dt"], steps,
                         column_offsets=offs, stream=stream)
        pt = ctx.phase_times(stream)
        ctx.profile(False)
        return {k: v / steps for k, v in pt["ms"].items()}

    phase_kernels = phases(capi.LP_LAUNCH_KERNELS)
    phase_persistent = phases(capi.LP_LAUNCH_PERSISTENT)

    def per_column():
        p = dict(prm, launch_mode=capi.LP_LAUNCH_GRAPH)
        for c in range(ncol):
            sl = {k: st[k][offs[c]:offs[c + 1]] for k in capi.FIELDS}
            capi.lp_step(ctx, sl, mui_c[c], eos, p, pd["dt"], steps, stream=stream)

    ms_c = timed(per_column)
    ctx.sync(stream, raise_on_error=False)

    # the batch at its stated length: 500 steps in one lp_step call, no
    # restart, from solid fraction 0.5 with free-surface ghosts (the start
    # that keeps these columns inside their stable horizon)
    full_steps = 500
    p500 = dict(prm, launch_mode=tune["launch_mode"], free_surface=1)
    v_half = torch.full_like(init["V"], 2.0)

    def reset500():
        reset()
        st["V"].copy_(v_half)

    with torch.cuda.stream(stream):
        reset500()
        capi.lp_step(ctx, st, mui_c, eos, p500, pd["dt"], 10, column_offsets=offs, stream=stream)
        reset500()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    with torch.cuda.stream(stream):
        capi.lp_step(ctx, st, mui_c, eos, p500, pd["dt"], full_steps, column_offsets=offs,
                     stream=stream)
    f1.record(stream)
    barrier()
    ms_f = D.max_over_ranks(f0.elapsed_time(f1), device=dev)
    d500 = ctx.sync(stream, raise_on_error=False)
    ctx.close()
    upd = wl.n * steps  # all ranks' particles
    return {"workload": f"{len(wl.column_offsets) - 1} columns, {wl.n} particles, "
                        f"{args.precision}, {steps} steps",
            "value": upd / (ms_b / 1e3), "unit": UNIT, "ms_per_step": ms_b / steps,
            "scaling": "strong",
            "shard": {"ranks": world, "columns_rank0": ncol, "particles_rank0": n_local},
            "launch": chosen, "tuning": tune,
            "graph_ms_per_step": modes["graph"] / steps,
            "persistent_ms_per_step": modes["persistent"] / steps,
            "phase_ms_per_step_kernels": phase_kernels,
            "phase_ms_per_step_persistent": phase_persistent,
            "per_column_value": upd / (ms_c / 1e3), "per_column_ms_per_step": ms_c / steps,
            "speedup_vs_per_column": ms_c / ms_b,
            "full_length": {"steps": full_steps, "phi0": 0.5, "free_surface_ghosts": True,
                            "restart": None, "value": wl.n * full_steps / (ms_f / 1e3),
                            "ms_per_step": ms_f / full_steps,
                            "n_nonfinite": d500["n_nonfinite"],
                            "ghost_entries_per_step": d500["n_ghosts"] / full_steps}}


def large_line(args, dev, stream, world):
    """The headline column scaled up at the same spacing: R = 0.06 m, H = 2R,
    h = R/150 = 4e-4 m (about 21.2M particles, 27 times the headline's), the
    same parameters, float-float with graph replay and Verlet skin 0.1h, calls
    of 10 steps from the initial state (a warm-up call, then two timed ones).
    Reports the throughput and the device memory the context and the state
    take (cudaMemGetInfo before and after)."""
    import torch

    from paper_2206_14061_gb300 import capi, workloads as W

    wl = W.cylinder(R=0.06, spacing_div=150, index=2)
    pd = W.param_dict(wl)
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")}
    prm = dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
               floor_z=0.0, mirror_mode=1, precision=PREC["mixed_ff"], rebuild_every=1,
               launch_mode=capi.LP_LAUNCH_GRAPH, skin=args.skin * pd["h"])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    init = {k: torch.tensor(wl.state[k], device=dev) for k in capi.FIELDS}
    st = {k: v.clone() for k, v in init.items()}
    ctx = capi.Context(wl.n, cap=64)
    steps, calls = 10, 2

    def run():
        with torch.cuda.stream(stream):
            for k in capi.FIELDS:
                st[k].copy_(init[k])
            capi.lp_step(ctx, st, mui, eos, prm, pd["dt"], steps, stream=stream)

    run()  # warm-up
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    if world > 1:
        torch.distributed.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(calls):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (steps * calls)
    if world > 1:
        from paper_2206_14061_gb300 import dist as D
        ms = D.max_over_ranks(ms, device=dev)
    d = ctx.sync(stream, raise_on_error=False)
    ctx.close()
    return {"workload": f"cylindrical column R = 0.06 m, H = 2R, h = R/150 ({wl.n} particles), "
                        "the headline's parameters, mixed_ff, graph replay",
            "value": wl.n * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "steps": steps * calls, "restart_every": steps,
            "device_bytes": int(used), "bytes_per_particle": used / wl.n,
            "n_nonfinite": d["n_nonfinite"]}


def collapse_line(dev, stream):
    """The column collapse of the paper's validation (Sec. 4.2.1): the
    a = 0.6 column, r_i = 0.05 m, h_i = a r_i = 0.03 m, 10 particles per
    radius (h = 5 mm), the paper's mu(I) set (Sec. 4), solid fraction 0.5,
    free-surface ghosts, float-float with graph replay, run in chunks of 100
    steps to the fits' t_inf = 3 (h_i/g)^(1/2) or until it blows up (a
    non-finite value or a speed above 3 m/s), for the benchmark's stiff
    quasi-static law (beta = 400 m^2/s^2) and a soft one (beta = 1 m^2/s^2).
    Reports the time reached and the front radius and height over r_i and h_i
    at each tenth of the run, against the fits of Sec. 4.2 (r_inf/r_i =
    1 + 1.24 a, h_inf/h_i = 1 for a < 1.7)."""
    import torch

    from paper_2206_14061_gb300 import capi, workloads as W

    ri, a, g = 0.05, 0.6, 9.81
    hi = a * ri
    t_inf = 3.0 * math.sqrt(hi / g)
    wl = W.cylinder(R=ri, aspect=a, spacing_div=10, jitter=0.05, index=7)
    pd = dict(W.param_dict(wl), **W.PAPER_MUI)
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    dt, chunk = 1e-5, 100
    nmax = int(math.ceil(t_inf / dt / chunk)) * chunk
    out = {"workload": f"a = 0.6 column, r_i = 0.05 m, h_i = 0.03 m, h = r_i/10 ({wl.n} "
                       "particles), paper mu(I) set, phi 0.5, free-surface ghosts, mixed_ff",
           "t_inf_s": t_inf, "fit_r_inf_over_ri": 1.0 + 1.24 * a, "fit_h_inf_over_hi": 1.0,
           "runs": []}
    for beta in (400.0, 1.0):
        eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max")}
        eos.update(alpha=-beta * pd["phi_max"], beta=beta)
        st = {k: torch.tensor(wl.state[k], device=dev) for k in capi.FIELDS}
        st["V"].fill_(2.0)
        ctx = capi.Context(wl.n, cap=64)
        prm = dict(h=wl.h, radius=2.2 * wl.h, gx=0.0, gy=0.0, gz=-g, floor_z=0.0, mirror_mode=1,
                   precision=PREC["mixed_ff"], rebuild_every=1,
                   launch_mode=capi.LP_LAUNCH_GRAPH, skin=0.1 * wl.h, free_surface=1)
        traj, steps, status = [], 0, "reached t_inf"
        t0 = time.perf_counter()
        while steps < nmax:
            with torch.cuda.stream(stream):
                capi.lp_step(ctx, st, mui, eos, prm, dt, chunk, stream=stream)
            d = ctx.sync(stream, raise_on_error=False)
            steps += chunk
            x, y, z = (st[k].cpu().numpy() for k in "xyz")
            sp = np.sqrt(sum(st[k].cpu().numpy() ** 2 for k in "uvw"))
            traj.append((steps * dt, float(np.sqrt(x * x + y * y).max()) / ri,
                         float(z.max()) / hi, float(sp.max())))
            if not np.isfinite(sp).all() or sp.max() > 3.0:
                status = "blew up"
                break
            if d["status"] != 0:
                status = "stopped: " + capi.lib().lp_status_string(int(d["status"])).decode()
                break
        wall = time.perf_counter() - t0
        ctx.close()
        keep = traj[::max(1, len(traj) // 10)] + traj[-1:]
        out["runs"].append({"beta": beta, "status": status, "t_reached_s": steps * dt,
                            "steps": steps, "wall_s": wall,
                            "trajectory": [{"t_s": t, "r_front_over_ri": r, "h_max_over_hi": h,
                                            "max_speed": v} for t, r, h, v in keep]})
    return out


def layer_line(dev, stream):
    """The layer compaction of the paper's verification (Sec. 4.1): the
    periodic layer, 0.03 m high, 8 x 8 particles across (period 8 mm along x
    and y), h = 1e-3, at rest, solid fraction 0.50 at the floor to 0.48 at the
    top, free-surface ghosts, no-slip floor, float-float with graph replay, run
    in chunks of 100 steps to 0.3 s or until it blows up, for the benchmark's
    stiff quasi-static law (beta = 400 m^2/s^2) and a soft one (1 m^2/s^2).
    Reports the time reached, the top height (the highest particle) and the
    mean solid fraction against the expected settled height of 0.025 m (the
    paper's own run ends at 0.02 m)."""
    import torch

    from paper_2206_14061_gb300 import capi, workloads as W

    wl = W.periodic_layer(n_xy=8)
    L, H = wl.extra["L"], wl.extra["H"]
    pd = W.param_dict(wl)
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    dt, chunk, t_end = 1e-5, 100, 0.3
    nmax = int(round(t_end / dt))
    out = {"workload": f"periodic layer {wl.n} particles (8 x 8 x 30), H = 0.03 m, h = 1e-3, "
                       "phi 0.50 to 0.48, free-surface ghosts, mixed_ff",
           "expected_settled_height_m": 0.025, "paper_simulated_height_m": 0.02, "runs": []}
    for beta in (400.0, 1.0):
        eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max")}
        eos.update(alpha=-beta * pd["phi_max"], beta=beta)
        st = {k: torch.tensor(wl.state[k], device=dev) for k in capi.FIELDS}
        ctx = capi.Context(wl.n, cap=64)
        prm = dict(h=wl.h, radius=wl.radius, gx=0.0, gy=0.0, gz=-9.81, floor_z=0.0,
                   mirror_mode=1, precision=PREC["mixed_ff"], rebuild_every=1,
                   launch_mode=capi.LP_LAUNCH_GRAPH, skin=0.1 * wl.h, free_surface=1,
                   period_x=L, period_y=L)
        traj, steps, status = [], 0, "reached 0.3 s"
        t0 = time.perf_counter()
        while steps < nmax:
            with torch.cuda.stream(stream):
                capi.lp_step(ctx, st, mui, eos, prm, dt, chunk, stream=stream)
            d = ctx.sync(stream, raise_on_error=False)
            steps += chunk
            z = st["z"].cpu().numpy()
            V = st["V"].cpu().numpy()
            sp = np.sqrt(sum(st[k].cpu().numpy() ** 2 for k in "uvw"))
            traj.append((steps * dt, float(z.max()), float(np.mean(1.0 / V)), float(sp.max())))
            if not (np.isfinite(sp).all() and np.isfinite(V).all()) or sp.max() > 3.0:
                status = "blew up"
                break
            if d["status"] != 0:
                status = "stopped: " + capi.lib().lp_status_string(int(d["status"])).decode()
                break
        wall = time.perf_counter() - t0
        ctx.close()
        keep = traj[::max(1, len(traj) // 10)] + traj[-1:]
        out["runs"].append({"beta": beta, "status": status, "t_reached_s": steps * dt,
                            "steps": steps, "wall_s": wall,
                            "trajectory": [{"t_s": t, "top_height_m": zt, "mean_phi": ph,
                                            "max_speed": v} for t, zt, ph, v in keep]})
    return out


def adjoint_line(dev, stream):
    """The adjoint column at its stated length: radius 0.02 m, H = 2R,
    spacing R/25 (98,800 particles), 200 FP64 steps with a checkpoint every
    20, from solid fraction 0.5 with free-surface ghosts and a radial flow of
    0.5 m/s (r/R)(z/H). Times the forward run alone (lp_step, stencils
    rebuilt every 20 steps) and the adjoint (lp_step_adjoint) for a seed on
    every state field: by default the forward sweep keeps the whole run's
    data (about 19 GB here) and the reverse sweep reads it; `adjoint_rerun_ms`
    is the same call with no room for that (each segment re-run from its
    checkpoint)."""
    import torch

    from paper_2206_14061_gb300 import capi, workloads as W

    R, nsteps, C = 0.02, 200, 20
    wl = W.cylinder(R=R, aspect=2.0, spacing_div=25, index=4)
    s = dict(wl.state)
    s["u"] = 0.5 * s["x"] / R * (s["z"] / (2 * R))
    s["v"] = 0.5 * s["y"] / R * (s["z"] / (2 * R))
    s["V"] = np.full(wl.n, 2.0)
    pd = W.param_dict(wl)
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")}
    prm = dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
               floor_z=0.0, mirror_mode=1, precision=PREC["fp64"], rebuild_every=C,
               launch_mode=capi.LP_LAUNCH_KERNELS, free_surface=1)
    init = {k: torch.tensor(v, device=dev) for k, v in s.items()}
    rng = np.random.default_rng(20220628 + 4)
    seed = {k: torch.tensor(rng.standard_normal(wl.n), device=dev) for k in capi.FIELDS}
    ctx = capi.Context(wl.n, cap=64)
    out = {}
    for name in ("forward", "adjoint_rerun", "adjoint"):
        ctx.set_adjoint_memory(0 if name == "adjoint_rerun" else -1)
        with torch.cuda.stream(stream):
            for rep in range(2):  # a warm-up, then the timed call
                st = {k: v.clone() for k, v in init.items()}
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if name == "forward":
                    capi.lp_step(ctx, st, mui, eos, prm, pd["dt"], nsteps, stream=stream)
                else:
                    dmui, _ = capi.lp_step_adjoint(ctx, st, mui, eos, prm, pd["dt"], nsteps, C,
                                                   seed, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1)
        if name == "adjoint_rerun":
            dmui_rerun = dmui
    d = ctx.sync(stream, raise_on_error=False)
    ctx.close()
    return {"workload": f"adjoint column R = 0.02 m, H = 2R, h = R/25 ({wl.n} particles), "
                        "200 FP64 steps, checkpoint every 20, phi 0.5, free-surface ghosts, "
                        "radial flow 0.5 m/s",
            "forward_ms": out["forward"], "adjoint_ms": out["adjoint"],
            "adjoint_over_forward": out["adjoint"] / out["forward"],
            "adjoint_rerun_ms": out["adjoint_rerun"],
            "dL_dmui_rerun": [float(v) for v in dmui_rerun.cpu()],
            "value": wl.n * nsteps / (out["adjoint"] / 1e3),
            "unit": "particle-steps/s differentiated (d/d(mu_s, mu_2, I0) of every state field)",
            "dL_dmui": [float(v) for v in dmui.cpu()], "n_nonfinite": d["n_nonfinite"]}


def periodic_layer(args, dev, stream, world):
    """The paper's periodic layer (0.03 m high, periodic along x and y, at
    rest under gravity with a small density gradient) at the size of the
    default workload: 162 x 162 x 30 particles, free-surface ghosts at the
    top, same precision, skin and restarts as the default line."""
    import torch

    from paper_2206_14061_gb300 import capi, workloads as W

    wl = W.periodic_layer(n_xy=162)
    pd = W.param_dict(wl)
    L = wl.extra["L"]
    n = wl.n
    mui = {k: pd[k] for k in ("mu_s", "mu_2", "I0", "d", "rho_s")}
    eos = {k: pd[k] for k in ("phi_c", "phi_min", "phi_max", "alpha", "beta")}
    init = {k: torch.tensor(wl.state[k], device=dev) for k in capi.FIELDS}
    st = {k: v.clone() for k, v in init.items()}
    prm = dict(h=pd["h"], radius=pd["radius"], gx=pd["gx"], gy=pd["gy"], gz=pd["gz"],
               floor_z=0.0, mirror_mode=1, precision=PREC[args.precision], rebuild_every=1,
               launch_mode=capi.LP_LAUNCH_GRAPH, skin=args.skin * pd["h"], free_surface=1,
               period_x=L, period_y=L)
    ctx = capi.Context(n, cap=64)
    R = max(1, args.restart_every)

    def run(nsteps, launch=capi.LP_LAUNCH_GRAPH):
        done = 0
        p = dict(prm, launch_mode=launch)
        with torch.cuda.stream(stream):
            while done < nsteps:
                k = min(R, nsteps - done)
                for f in capi.FIELDS:
                    st[f].copy_(init[f])
                capi.lp_step(ctx, st, mui, eos, p, pd["dt"], k, stream=stream)
                done += k

    run(args.warmup)
    ctx.sync(stream)
    ctx.phase_times(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    diag = ctx.sync(stream, raise_on_error=False)
    ctx.phase_times(stream)
    ctx.profile(True)
    run(min(args.steps, R), launch=capi.LP_LAUNCH_KERNELS)
    prof = ctx.phase_times(stream)
    ctx.profile(False)
    ctx.sync(stream, raise_on_error=False)
    ctx.close()
    return {"workload": f"periodic layer {wl.name}: {n} particles, L = {L} m along x and y, "
                        "H = 0.03 m, free-surface ghosts, at rest under gravity",
            "value": n * args.steps * world / (ms / 1e3), "unit": UNIT,
            "ms_per_step": ms / args.steps,
            "phase_ms_per_step": {k: v / max(prof["steps"], 1) for k, v in prof["ms"].items()},
            "ghost_entries_per_step": diag["n_ghosts"] / max(args.steps, 1),
            "n_nonfinite": diag["n_nonfinite"]}


def derivative_sweep(args, dev, stream):
    """lp_fit_derivatives on the derivative-operator sweep (jittered +-0.2h
    lattice of 126^3 particles, per-particle radius U(1.8h, 2.6h), 48 nearest,
    four smooth fields): the stencil build (lp_build_neighbors, the 48
    nearest) timed once after a warm-up build, then the fit timed in each
    precision mode; throughput in particle-fields per second."""
    import torch

    from paper_2206_14061_gb300 import capi, workloads as W

    x, y, z, rad, fields, _ = W.sweep_lattice(n_side=126)
    n, nf = x.size, fields.shape[0]
    ctx = capi.Context(n, cap=64)
    X = [torch.tensor(a, device=dev) for a in (x, y, z)]
    F = [torch.tensor(f, device=dev) for f in fields]
    out = torch.empty((n, nf, 9), dtype=torch.float64, device=dev)
    rt = torch.tensor(rad, device=dev)

    def build():
        return capi.lp_build_neighbors(ctx, *X, radius=rt, mirror_mode=0, cap=48,
                                       keep_nearest=True, stream=stream)
    with torch.cuda.stream(stream):
        nb = build()  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        nb = build()
    e1.record(stream)
    ctx.sync(stream)
    res = {"workload": f"derivative sweep: {n} particles, {nf} fields, 48 nearest, "
                       "jitter +-0.2h, radius U(1.8h, 2.6h)",
           "neighbors_ms": e0.elapsed_time(e1)}
    reps = max(3, min(args.steps, 10))
    for name in ("fp64", "mixed", "mixed_ff"):
        def call():
            capi.lp_fit_derivatives(ctx, *X, nb, F, [1.0] * nf, 1e-3, precision=PREC[name],
                                    out=out, stream=stream)
        with torch.cuda.stream(stream):
            call()  # warm-up (and the float-float workspace)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(reps):
                call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms_per_call": ms, "particle_fields_per_s": n * nf / (ms / 1e3)}
    ctx.sync(stream)
    ctx.close()
    return res


def e2e(args, ctx, wl, pd, mui, eos, params, dev, stream, world):
    """The same metric through the public API with HOST buffers: every step
    is one lp_step call on the pinned host arrays, which copies the state in,
    steps and copies the new state back."""
    import numpy as np
    import torch

    from paper_2206_14061_gb300 import capi

    import queue
    import threading

    n = wl.n
    nfld = len(capi.FIELDS)
    # the state as one pinned [fields, n] block: lp_step on host arrays copies
    # it in and out in one copy each way per step
    host0 = torch.tensor(np.stack([wl.state[k] for k in capi.FIELDS])).pin_memory()
    R = max(1, args.restart_every)
    # The restart to the initial state every R steps (as in the device-timed
    # line) is the benchmark's, not the caller's: it switches to a pinned
    # block already refreshed from the initial state, and a helper thread
    # refreshes the block just left, off the steps' critical path.
    pool = [host0.clone().pin_memory() for _ in range(3)]
    fresh = [threading.Event() for _ in pool]
    for e in fresh:
        e.set()
    todo = queue.Queue()

    def refresher():
        while True:
            b = todo.get()
            if b is None:
                return
            pool[b].copy_(host0)
            fresh[b].set()

    helper = threading.Thread(target=refresher, daemon=True)
    helper.start()
    cur = {"b": len(pool) - 1, "hst": None}
    prm = dict(params(args.precision, graph=0), keep_lists=1)

    def one(i):
        if i % R == 0:
            old = cur["b"]
            b = (old + 1) % len(pool)
            fresh[b].wait()
            used = cur["hst"] is not None
            cur["b"] = b
            cur["hst"] = {k: pool[b][q] for q, k in enumerate(capi.FIELDS)}
            if used:  # refresh the block just left (the warm-up's included)
                fresh[old].clear()
                todo.put(old)
        # one call per step on the host arrays; the Verlet lists stay on the
        # context between calls
        capi.lp_step(ctx, cur["hst"], mui, eos, prm, pd["dt"], 1, stream=stream)
        stream.synchronize()

    for i in range(args.warmup):
        one(i)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        one(i)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    todo.put(None)
    helper.join()
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([dt], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    ctx.sync(stream, raise_on_error=False)
    return {"value": n * args.steps * world / dt, "unit": UNIT,
            "h2d_bytes_per_step": nfld * 8 * n, "d2h_bytes_per_step": nfld * 8 * n,
            "ms_per_step": dt * 1e3 / args.steps}


def cpu_baseline(wl, pd, budget_s=20.0, steps=None):
    """The oracle, as it stands, on the host cores: full LP steps of the same
    workload from the initial state, run until about budget_s of wall time."""
    from oracle import oracle as O

    O.build()
    p = O.params(**pd)
    cores = O.max_threads()
    done, t0 = 0, time.perf_counter()
    while True:
        O.step(wl.state, p, 1, brute=False, nthreads=cores)
        done += 1
        el = time.perf_counter() - t0
        if (steps is not None and done >= steps) or (steps is None and el >= budget_s):
            break
    out = {"value": wl.n * done / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{done} full LP step(s) of the {wl.n}-particle column from its initial "
                     f"state, grid neighbour search, OpenMP over particles ({el:.1f} s)"}
    if steps is None:  # one step on one core as well (about 10 s here)
        t1 = time.perf_counter()
        O.step(wl.state, p, 1, brute=False, nthreads=1)
        e1 = time.perf_counter() - t1
        out["single_thread"] = {"value": wl.n / e1, "unit": UNIT, "cores": 1,
                                "sample": f"1 full LP step of the same column ({e1:.1f} s)"}
    return out


# -------------------------------------------------------------- reference

REF_BUDGET_S = 120.0


def reference_arm(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from paper_2206_14061_gb300 import workloads as W

    wl = W.cylinder()
    pd = W.param_dict(wl)
    from oracle import oracle as O
    O.build()
    p = O.params(**pd)
    # warm-up steps (from the initial state), then the timed sample
    t_w = time.perf_counter()
    for _ in range(max(args.warmup, 1)):
        O.step(wl.state, p, 1, brute=False)
    t_step = (time.perf_counter() - t_w) / max(args.warmup, 1)
    # the timed sample is bounded to about REF_BUDGET_S seconds: at most K
    # steps, fewer when K steps of the oracle would take longer
    steps = max(1, min(args.steps, int(REF_BUDGET_S / max(t_step, 1e-9))))
    t0 = time.perf_counter()
    for _ in range(steps):
        O.step(wl.state, p, 1, brute=False)
    el = time.perf_counter() - t0
    value = wl.n * steps / el
    cores = O.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": steps, "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded jittered lattice column)",
            "config": {"workload": "cylindrical column collapse R=0.02 m H=2R h=R/50 "
                                   f"({wl.n} particles), FP64 CPU oracle",
                       "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{steps} full LP steps of the {wl.n}-particle column "
                                       f"from its initial state ({t_step:.2f} s per step; "
                                       f"{args.steps} requested, bounded to about "
                                       f"{REF_BUDGET_S:.0f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
