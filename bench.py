"""Benchmark: MWDG2 active-cell updates/s on the 1024 x 1024 fractal-valley
workload (dx = 10 m, L = 10, epsilon = 1e-3, Manning n = 0.035, triangular
inflow peaking at 400 m^3/s at 30 min on the west edge), FP32 free-surface
path, with the FP64 path, the FP32-vs-FP64 depth error and CSI, the
roofline of the dominant kernel and the CPU oracle beside it.

One step = one full MWDG2 time step (MRA encode, threshold, regularise,
decode, CFL dt, friction, both RK2 stages) on the state reached after a
spin-up of `--spinup` simulated seconds; one update = one active leaf
advanced one step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs one independent replica per GPU (launched with
torch.distributed.run); the per-replica work is fixed (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MWDG2/DG2 active-cell updates/s & % HBM roofline, FP32 vs FP64 at <=1e-3 m"
UNIT = "active-cell updates/s"
def workload(n=1024, kind="MWDG2"):
    """the valley workload's description at side n (L = log2 n)"""
    return (f"{kind} {n}x{n} fractal valley, dx=10 m, L={n.bit_length() - 1}, eps=1e-3, n=0.035, "
            "400 m3/s inflow")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--spinup", type=float, default=1800.0, help="simulated seconds before timing")
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="instead: the batched ensemble of this many seeded valleys (sides 256-1024)")
    ap.add_argument("--no-tune", action="store_true", help="ensemble: keep the default launch shapes")
    ap.add_argument("--grid", default="adaptive", choices=["adaptive", "uniform", "static"],
                    help="DG2 grid: adaptive MWDG2 (the headline), the uniform finest grid, or the static graded grid")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the FP64 DG2 adjoint: one checkpoint segment forward and backward")
    ap.add_argument("--adjoint-steps", type=int, default=200, help="adjoint: steps per checkpoint segment")
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"],
                    help="precision of the timed arm (f32: the free-surface FP32 path, the headline; f64: the "
                         "FP64 path, which then needs no separate FP64 leg)")
    ap.add_argument("--urban", type=int, default=1,
                    help="1: add the slow-to-gradual urban configuration (static vs uniform DG2) to the line; "
                         "2: with its whole 3 h run (static and uniform, FP32; minutes)")
    ap.add_argument("--scheme", default="dg2", choices=["dg2", "fv1", "acc"],
                    help="solver: DG2 (MWDG2, the headline), FV1 (HWFV1 on the adaptive grid) or ACC "
                         "(static graded grid from the same MRA of the topography)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def host_cpu():
    """the host's CPU model and logical core count"""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"model": model or "unknown", "nproc": os.cpu_count()}


def _oracle_window(n_full):
    """the 256 x 256 window (L = 8) of the valley through the inflow, as an
    oracle simulation at t = 0"""
    import oracle as O
    from paper_2107_02750_gb300 import synth as S
    full = S.valley(n=n_full, L=n_full.bit_length() - 1)
    p = S.crop(full, 0, n_full // 2 - 128, 256, 256, L=8)
    s = O.Sim(M=p.M, N=p.N, L=p.L, R=p.dx, mode=p.mode, eps=p.eps, bc=p.bc,
              inflow_edge=p.inflow_edge, inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1,
              limiter=p.limiter, dt_max=p.dt_max)
    s.load_dem(p.z_vert)
    s.load_roughness(p.n_cell())
    s.load_initial(p.h_vert, p.qx_vert, p.qy_vert, p.is_eta)
    s.set_inflow(p.inflow_t, p.inflow_Q)
    s.init_grid()
    return s


def _oracle_sample(job):
    """MWDG2 steps of the oracle on the valley window from t = 0: either a
    time budget (budget_s > 0) or warm-up + a step count; returns (updates,
    seconds, steps)"""
    n_full, budget_s, warmup, steps = job
    s = _oracle_window(n_full)
    for _ in range(warmup):
        s.step()
    upd = k = 0
    t0 = time.perf_counter()
    while (time.perf_counter() - t0 < budget_s) if budget_s > 0 else (k < steps):
        s.step()
        upd += len(s.leaves()[0])
        k += 1
    return upd, time.perf_counter() - t0, k


def oracle_all_cores(n_full, budget_s=0.0, warmup=0, steps=0):
    """the same sample in one process per logical core (spawned), all at
    once: whole-host throughput of the oracle as it stands"""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_sample, [(n_full, budget_s, warmup, steps)] * cores)
    upd = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return upd, el, cores, sum(r[2] for r in res)


def cpu_baseline(n_full, budget_s=10.0):
    """The FP64 oracle, as it stands, on this host: the 256 x 256 window (L = 8)
    of the same valley through the inflow, MWDG2 from t = 0, for about
    budget_s seconds on one thread, then the same in one process per core."""
    upd1, el1, k1 = _oracle_sample((n_full, budget_s, 0, 0))
    updN, elN, cores, kN = oracle_all_cores(n_full, budget_s)
    cpu = host_cpu()
    return {"value": updN / elN, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, 256x256 window (L=8) of the valley through the inflow, MWDG2 from t=0: "
                      f"one process per core ({cores}), {kN} steps ({updN} updates) in {elN:.1f} s",
            "cpu_model": cpu["model"], "nproc": cpu["nproc"],
            "single_thread": {"value": upd1 / el1, "unit": UNIT, "cores": 1,
                              "sample": f"the same window on 1 thread: {k1} steps ({upd1} updates) in {el1:.1f} s"}}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def make_solver(p, precision, stream):
    import paper_2107_02750_gb300 as M
    return M.solver_from_problem(p, precision=precision, stream=stream)


def timed_steps(solver, K, W, flush, stream, prof=False, profiler_range=False):
    """W untimed steps, then K steps each bracketed by CUDA events on the
    solver's stream with an L2 flush before each (no host synchronisation
    inside the loop); returns (ms per step, active-leaf updates, launches in
    the timed region, kernel times).  With profiler_range the K steps are the
    range an external profiler started with --profile-from-start off records."""
    import torch
    for _ in range(W):
        solver.run_steps(1)
    torch.cuda.synchronize()
    _, u0 = solver.get_counters()
    l0 = solver.launch_count()
    if profiler_range:
        torch.cuda.profiler.start()
    if prof:
        solver.profile(True)
    evs = []
    for _ in range(K):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        solver.run_steps(1)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    if profiler_range:
        torch.cuda.profiler.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    _, u1 = solver.get_counters()
    kt = solver.kernel_times() if prof else {}
    if prof:
        solver.profile(False)
    launches = solver.launch_count() - l0
    return ms, u1 - u0, launches, kt


def reduce_over_ranks(total_ms, updates, world, device):
    """Whole-job figures of independent replicas: the slowest rank's timed
    milliseconds and the updates of all ranks (no data-path collective; the
    replicas exchange only these two numbers)."""
    if world <= 1:
        return float(total_ms), float(updates)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], device=device, dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_gpu(args, rank, world):
    import torch
    import paper_2107_02750_gb300 as M
    from paper_2107_02750_gb300 import synth as S

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    p = S.valley(n=args.n, L=args.n.bit_length() - 1)
    if args.grid != "adaptive":
        from dataclasses import replace
        p = replace(p, mode=S.UNIFORM if args.grid == "uniform" else S.STATIC)
    if args.scheme == "fv1":
        p = S.fv1(p)  # HWFV1 on the adaptive grid
    elif args.scheme == "acc":
        from dataclasses import replace
        p = S.acc(replace(p, mode=S.STATIC))  # static graded grid from the MRA of the topography
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # FP32 free-surface path (headline)
    prec = M.F64 if args.precision == "f64" else M.F32
    s32 = make_solver(p, prec, sptr)
    s32.run_to_time(args.spinup)
    t_spin, _ = s32.get_time()
    ckpt = s32.save_state()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        ms, upd, launches, _ = timed_steps(s32, args.steps, args.warmup, flush, stream, prof=False,
                                           profiler_range=True)
    # per-kernel durations: steps again with CUDA events between the kernels
    # on the solver's stream (direct launches)
    kms, kupd, _, kt = timed_steps(s32, min(args.steps, 200), 0, flush, stream, prof=True)
    total_ms = sum(ms)
    updates = upd
    total_ms, updates_all = reduce_over_ranks(total_ms, updates, world, "cuda")
    value = updates_all / (total_ms * 1e-3)

    # roofline of the dominant kernel: the kernel with the longest average
    # launch (each MRA level is its own launch).  `frac` uses the algorithmic
    # bytes of the step's definition (a fused uniform stage: stage 1 reads 13
    # values and writes 9, stage 2 reads 22 and writes 9); the bytes this
    # design's kernel moves by construction (its flux-view record, stored
    # views, list entry and neighbour codes) are reported beside it
    peak_gbs, peak_kind = peaks()
    per_launch = {k: v[0] / v[1] for k, v in kt.items() if v[1]}
    dom_name = max(per_launch, key=per_launch.get)
    dom_ms, dom_n = kt[dom_name]
    mean_leaves = kupd / len(kms)
    elem = 8 if prec == M.F64 else 4
    bpl = kernel_bytes_per_leaf(dom_name, elem, args.scheme, args.grid)
    alg = STAGE_VALUES.get(dom_name) if args.scheme == "dg2" else None
    abpl = alg * elem if alg else bpl
    launch_s = dom_ms / dom_n * 1e-3
    achieved = (abpl * mean_leaves) / launch_s / 1e9 if abpl else None
    roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak_gbs,
                "unit": "GB/s", "frac": (achieved / peak_gbs) if achieved else None,
                "traffic": (TRAFFIC.get(dom_name) if (args.grid, args.scheme, args.precision, args.n) ==
                            ("adaptive", "dg2", "f32", 1024) else None),
                "peak_kind": peak_kind, "algorithmic_bytes_per_leaf": abpl,
                "design_bytes_per_leaf": bpl,
                "design_frac": (bpl * mean_leaves / launch_s / 1e9 / peak_gbs) if bpl else None,
                "launches": dom_n, "mean_leaves_per_launch": mean_leaves,
                "share_of_step": dom_ms / max(sum(v[0] for v in kt.values()), 1e-9),
                "step_ms_by_class": {k: round(v[0] / len(kms), 5) for k, v in kt.items() if v[1]},
                "ms_per_launch": {k: round(v, 5) for k, v in per_launch.items()}}
    if args.scheme == "dg2":
        # the whole step on the step's algorithmic bytes per update: the DG2
        # step (53 values) plus, on the adaptive grid, the MRA's per leaf
        wb = DG2_STEP_VALUES * elem + (MRA_BYTES_PER_LEAF[elem] if args.grid == "adaptive" else 0)
        roofline["whole_step"] = {"bytes_per_update": wb, "achieved": wb * value / 1e9,
                                  "frac": wb * value / 1e9 / peak_gbs, "unit": "GB/s"}

    # end to end through the public API: resume from a host checkpoint in
    # pinned memory, E2E_STEPS steps, depth and velocity maps back to the host
    pinned = torch.from_numpy(ckpt).pin_memory()
    hbuf = [torch.empty((p.ny, p.nx), dtype=torch.float64).pin_memory() for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s32.load_state(pinned)
    n_e2e = 0
    _, u0 = s32.get_counters()
    s32.run_steps(E2E_STEPS)
    _, u1 = s32.get_counters()
    n_e2e = u1 - u0
    import ctypes as C
    st = s32._lib.mwdg_read_fields(s32._h, *(C.cast(C.c_void_p(b.data_ptr()), C.POINTER(C.c_double)) for b in hbuf), 0)
    if st:
        raise RuntimeError("mwdg_read_fields failed")
    e2e_s = time.perf_counter() - t0
    e2e = {"value": n_e2e / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(ckpt.nbytes // E2E_STEPS),
           "d2h_bytes_per_step": int(3 * p.nx * p.ny * 8 // E2E_STEPS), "steps": E2E_STEPS,
           "what": f"mwdg_load_state from pinned host checkpoint + {E2E_STEPS} x mwdg_dg2_step + "
                   f"mwdg_read_fields to pinned host"}

    out = {"value": value, "ms_per_step": total_ms / len(ms), "updates": updates_all,
           "mean_active": updates / len(ms), "roofline": roofline, "clocks": clk.summary(), "e2e": e2e,
           "gpu_launches": int(launches) * world, "t_spinup": t_spin}
    if rank == 0 and args.grid == "adaptive" and args.scheme == "dg2":
        out["uniform_dg2"] = uniform_leg(p, stream, flush, args.steps, args.warmup, args.spinup)

    # FP64 path, and FP32 against FP64 at the same simulated times
    if not args.no_fp64 and rank == 0:
        s64 = make_solver(p, M.F64, sptr)
        s64.run_to_time(args.spinup)
        ms64, upd64, _, _ = timed_steps(s64, max(4, args.steps // 4), 2, flush, stream)
        v64 = upd64 / (sum(ms64) * 1e-3)
        fma64 = M.fma_rate(M.F64, sptr)
        fma32 = M.fma_rate(M.F32, sptr)
        out["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": sum(ms64) / len(ms64), "dtype": "f64",
                       "alu": {"bound": "alu", "peak": fma64 / 1e12, "unit": "TFLOP/s",
                               "peak_kind": "measured (FP64 FMA chains, CUDA events)",
                               "flops_per_update": FP64_FLOPS_PER_UPDATE,
                               "achieved": (v64 * FP64_FLOPS_PER_UPDATE / 1e12) if FP64_FLOPS_PER_UPDATE else None,
                               "frac": (v64 * FP64_FLOPS_PER_UPDATE / fma64) if FP64_FLOPS_PER_UPDATE else None,
                               # the FMA peak counts FMAs; the FP64 pipe's occupancy, measured by ncu,
                               # is the binding figure for this add/multiply/compare mix
                               "pipe_busy_pct_of_active_cycles": FP64_PIPE_BUSY},
                       "hbm": {"bytes_per_update": DG2_STEP_VALUES * 8 + MRA_BYTES_PER_LEAF[8],
                               "frac": (DG2_STEP_VALUES * 8 + MRA_BYTES_PER_LEAF[8]) * v64 / 1e9 / peak_gbs}}
        out["fma_peaks_tflops"] = {"fp64": fma64 / 1e12, "fp32": fma32 / 1e12}
        tcmp = max(s64.get_time()[0], s32.get_time()[0]) + 1.0
        a32, a64 = make_solver(p, M.F32, sptr), make_solver(p, M.F64, sptr)
        # the method's own sensitivity: a second FP64 run whose only
        # difference is one extra stop (one shortened step) at 150.5 s
        b64 = make_solver(p, M.F64, sptr)
        acc, self64 = [], []
        for t in (60.0, 300.0, 900.0, tcmp):
            a32.run_to_time(t)
            a64.run_to_time(t)
            acc.append(compare_depths(a32, a64, t))
            if t == 60.0:
                b64.run_to_time(60.0)
                b64.run_to_time(150.5)
            elif t in (300.0, 900.0):
                b64.run_to_time(t)
                self64.append(compare_depths(b64, a64, t))
        out["accuracy_f32_vs_f64"] = acc
        out["fp64_vs_fp64_one_extra_stop"] = self64
        out["accuracy_f32_on_fp64_steps"] = fixed_step_accuracy(p, sptr)
        out["run_average_2h"] = {"f32": run_average(p, M.F32, sptr, 7200.0),
                                 "f64": run_average(p, M.F64, sptr, 7200.0)}
    return out


def uniform_leg(p, stream, flush, K, W, spinup):
    """The same DG2 step on the uniform finest grid of the valley (one fused
    kernel per RK2 stage), FP32, after the same spin-up: updates/s and the
    roofline of each stage kernel and of the whole step on the step's
    algorithmic bytes (stage 1: 13 values read, 9 written; stage 2: 22 read,
    9 written; 212 B a cell and step in all)"""
    import torch
    import paper_2107_02750_gb300 as M
    from dataclasses import replace
    from paper_2107_02750_gb300 import synth as S
    q = replace(p, mode=S.UNIFORM)
    s = make_solver(q, M.F32, stream.cuda_stream)
    s.run_to_time(spinup)
    ms, upd, _, _ = timed_steps(s, K, W, flush, stream)
    kms, kupd, _, kt = timed_steps(s, min(K, 100), 0, flush, stream, prof=True)
    value = upd / (sum(ms) * 1e-3)
    peak, kind = peaks()
    cells = kupd / len(kms)
    stages = {}
    for name, vals in STAGE_VALUES.items():
        if name in kt and kt[name][1]:
            t = kt[name][0] / kt[name][1] * 1e-3
            stages[name] = {"ms_per_launch": t * 1e3, "algorithmic_bytes_per_cell": vals * 4,
                            "achieved": vals * 4 * cells / t / 1e9, "frac": vals * 4 * cells / t / 1e9 / peak}
    wb = DG2_STEP_VALUES * 4
    # the instruction-issue ceiling (four warp schedulers per SM, one warp
    # instruction each per cycle, at the maximum SM clock) with the stage
    # kernels' instruction counts from ncu: the bound these kernels meet first
    ipeak = torch.cuda.get_device_properties(0).multi_processor_count * 4 * ISSUE_CLOCK_MHZ * 1e6 / 1e9
    for name, st in stages.items():
        ipc = UNI_WARP_INSTR_PER_CELL.get(name)
        if ipc is not None:
            a = ipc * cells / (st["ms_per_launch"] * 1e-3) / 1e9
            st["issue"] = {"warp_instr_per_cell": ipc, "achieved": a, "peak": ipeak, "unit": "G warp instr/s",
                           "frac": a / ipeak}
    ipc_step = sum(UNI_WARP_INSTR_PER_CELL.values())
    return {"value": value, "unit": UNIT, "ms_per_step": sum(ms) / len(ms), "cells": cells,
            "roofline": {"bound": "hbm", "peak": peak, "peak_kind": kind, "unit": "GB/s", "stages": stages,
                         "whole_step": {"bytes_per_update": wb, "achieved": wb * value / 1e9,
                                        "frac": wb * value / 1e9 / peak}},
            "issue_roofline": {"bound": "alu", "unit": "G warp instr/s", "peak": ipeak,
                               "peak_kind": f"derived: SMs x 4 schedulers x 1 warp instruction/cycle x {ISSUE_CLOCK_MHZ} MHz",
                               "warp_instr_per_cell_step": ipc_step, "achieved": ipc_step * value / 1e9,
                               "frac": ipc_step * value / 1e9 / ipeak},
            "what": f"uniform DG2 on the valley's finest grid ({int(cells):,} cells), FP32, fused stage kernels, "
                    "L2 flushed before every timed step"}


def fixed_step_accuracy(p, sptr, marks=(120.0, 300.0, 900.0)):
    """FP32 against FP64 with the FP32 run taking the FP64 run's time steps
    (mwdg_dg2_step_dt): the FP32 arithmetic error alone, without the
    divergence of two trajectories that choose their own CFL steps"""
    import paper_2107_02750_gb300 as M
    a = make_solver(p, M.F64, sptr)
    b = make_solver(p, M.F32, sptr)
    out, t = [], 0.0
    for mark in marks:
        while t < mark:
            dt = a.dg2_step()
            b.dg2_step_dt(dt)
            t += dt
        r = compare_depths(b, a, t)
        r["steps"] = a.get_time()[1]
        r["n_clip_f32"] = b.get_volume()["n_clip"]
        out.append(r)
    return out


def run_average(p, precision, sptr, t_end):
    """the whole simulated run of the configuration from t = 0 (mwdg_run_to_time,
    CUDA events around it, no flush): active-cell updates/s averaged over the
    run, with the mass budget and the clipped volume at its end"""
    import torch
    import paper_2107_02750_gb300 as M
    s = make_solver(p, precision, sptr)
    stream = torch.cuda.ExternalStream(sptr)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s.run_to_time(t_end)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    steps, upd = s.get_counters()
    v = s.get_volume()
    return {"value": upd / (ms * 1e-3), "unit": UNIT, "simulated_s": s.get_time()[0], "steps": steps,
            "ms": ms, "mean_active": upd / max(steps, 1), "dtype": "f64" if precision == M.F64 else "f32",
            "n_clip": v["n_clip"], "v_clip_m3": v["v_clip"], "v_in_m3": v["v_in"],
            "budget_error_rel": abs(v["volume"] - (v["v_in"] - v["v_out"] + v["v_rain"])) / max(v["volume"], 1.0)}


def run_urban(stream, flush, K, W, spinup=1800.0, t_cmp=600.0, full=False):
    """The slow-to-gradual configuration: 2048 x 2048 urban-like DEM at dx =
    2 m, 8 m blocks off a 100 m road grid (n = 0.013 on roads, 0.035 else),
    50 mm/h of rain for 1 h.  Static non-uniform DG2 (one MRA of the
    topography at eps = 1e-2, reflux rule) against uniform DG2, both FP32
    with FP64 time and volume sums: K flushed steps each after `spinup`
    simulated seconds, and the static FP32 depth against the static FP64
    depth at t_cmp."""
    import paper_2107_02750_gb300 as M
    from dataclasses import replace
    from paper_2107_02750_gb300 import synth as S
    sptr = stream.cuda_stream
    p = S.urban()
    p.iface_rule = 1
    res = {}
    for name, q in (("static", p), ("uniform", replace(p, mode=S.UNIFORM))):
        s = make_solver(q, M.F32, sptr)
        s.run_to_time(spinup)
        ms, upd, _, _ = timed_steps(s, K, W, flush, stream)
        steps, _ = s.get_counters()
        res[name] = {"value": upd / (sum(ms) * 1e-3), "unit": UNIT, "ms_per_step": sum(ms) / len(ms),
                     "active_leaves": upd / len(ms), "steps_to_spinup": steps - K - W}
    a32, a64 = make_solver(p, M.F32, sptr), make_solver(p, M.F64, sptr)
    a32.run_to_time(t_cmp)
    a64.run_to_time(t_cmp)
    res["accuracy_f32_vs_f64_static"] = compare_depths(a32, a64, t_cmp)
    res["speedup_static_over_uniform_s_per_simulated_s"] = (
        (res["uniform"]["ms_per_step"]) / res["static"]["ms_per_step"])
    res["config"] = ("2048x2048 urban DEM, dx=2 m, blocks 10-40 m x 8 m at 25 % cover, roads every 100 m, "
                     f"rain 50 mm/h for 1 h; static grid eps=1e-2 (reflux rule); timed after {spinup:.0f} s, "
                     f"FP32 vs FP64 at {t_cmp:.0f} s")
    if full:
        # the configuration's whole 3 h from t = 0, FP32, static and uniform
        res["run_3h"] = {name: run_average(q, M.F32, sptr, 3.0 * 3600.0)
                         for name, q in (("static", p), ("uniform", replace(p, mode=S.UNIFORM)))}
    return res


def average_raster(s):
    """finest raster of the active leaves' average depths"""
    lev, ii, jj, co = s.read_active()
    out = np.zeros((s.ny, s.nx))
    for l in np.unique(lev):
        m = lev == l
        w = 1 << (s.levels - int(l))
        grid = np.full((s.ny // w, s.nx // w), np.nan)
        grid[jj[m], ii[m]] = co[m, 0]
        up = np.repeat(np.repeat(grid, w, axis=0), w, axis=1)
        sel = ~np.isnan(up)
        out[sel] = up[sel]
    return out


def compare_depths(s32, s64, t):
    """FP32 against FP64 depth: on the leaves' planes at the finest cells and
    on the leaves' averages; wet extent (depth > 0.01 m) CSI on both"""
    def scores(h32, h64):
        d = np.abs(h32 - h64)
        wet32, wet64 = h32 > 0.01, h64 > 0.01
        A = int(np.sum(wet32 & wet64)); B = int(np.sum(wet32 & ~wet64)); Cc = int(np.sum(~wet32 & wet64))
        wet = wet32 | wet64
        return {"max_m": float(d.max()), "p99_m": float(np.quantile(d, 0.99)),
                "rmse_wet_m": float(np.sqrt(np.mean(d[wet] ** 2))) if wet.any() else 0.0,
                "csi": A / max(A + B + Cc, 1)}
    h32, _, _ = s32.read_fields()
    h64, _, _ = s64.read_fields()
    return {"t": t, "planes": scores(h32, h64), "averages": scores(average_raster(s32), average_raster(s64))}


def reference_arm(args):
    """The reference arm is the FP64 CPU oracle as it stands, on all host
    cores (one spawned process per core, each the same sample): W untimed
    then K timed MWDG2 steps on the 256 x 256 window (L = 8) of the same
    valley through the inflow, from t = 0."""
    upd, el, cores, k = oracle_all_cores(args.n, 0.0, args.warmup, args.steps)
    v = upd / el
    cpu = host_cpu()
    sample = (f"FP64 oracle, one process per core ({cores}): {args.steps} MWDG2 steps each ({upd} updates in all) "
              f"of a 256x256 window (L=8) of the valley through the inflow, from t=0, in {el:.1f} s")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload(args.n)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu["model"], "nproc": cpu["nproc"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def kernel_bytes_per_leaf(name, ts, scheme="dg2", grid="adaptive"):
    """Algorithmic HBM bytes per active leaf of a kernel class: values of ts
    bytes, the 8-byte active-list entry and the leaf's 32-byte neighbour
    codes where the kernel reads them (not on uniform grids, whose kernels
    form both from the thread index); neighbour values served from L2 are
    not counted.  MRA classes are per node, not per leaf: None."""
    if scheme == "acc":  # discharges, then continuity (values, entry, codes)
        vals = {"dg2_update_stage1": (3 + 4 + 4, 40),   # h, z, n, old q read; new q written
                "dg2_update_stage2": (4 + 1 + 4 + 3, 40)}  # new q, h read; h, qx, qy, q written
    elif scheme == "fv1":  # one forward-Euler stage (labelled stage 2)
        vals = {"dg2_update_stage2": (12 + 9 + 9, 40), "limit": (9 + 3 + 9 + 12, 40)}
    elif grid == "uniform":  # one fused kernel per stage (limiter, interfaces and update)
        vals = {
            "dg2_update_stage1": (9 + 3 + 1 + 9 + 9, 0),  # U^n, bed, Manning n read; Wn, U_int written
            "dg2_update_stage2": (9 + 3 + 9 + 9, 0),      # U_int, bed, Wn read; U^{n+1} written
        }
    else:
        vals = {
            "dg2_update_stage1": (12 + 9 + 9, 40),      # FZ record, Wn read; Ui written
            "dg2_update_stage2": (12 + 9 + 9 + 9, 40),  # FZ record, Wi, Wn read; U written
            "limit": (9 + 3 + 9 + 12, 40),              # X, Z read; Wst, FZ record written
        }
    if name not in vals:
        return None
    n, extra = vals[name]
    if grid == "uniform" and scheme != "acc":
        extra = 0
    return n * ts + extra


# Algorithmic values per active-cell update of the DG2 step (a fused uniform
# stage keeps neighbour reads on chip): stage 1 reads U^n (9), the bed (3) and
# Manning n (1) and writes U_int (9); stage 2 reads U_int, U^n, the bed and n
# and writes U^{n+1}: 22 + 31 = 53 values, 212 B in FP32, 424 B in FP64.
STAGE_VALUES = {"dg2_update_stage1": 22, "dg2_update_stage2": 31}
DG2_STEP_VALUES = 53
# The MRA's algorithmic bytes per active leaf and step (adaptive grid): the
# leaf's state (9 values) and bed planes (3) read, the parents' scale
# coefficients written (9 values per refined node, about one node per three
# leaves: 3 values), and its flag byte
MRA_BYTES_PER_LEAF = {4: (9 + 3 + 3) * 4 + 1, 8: (9 + 3 + 3) * 8 + 1}
# FP64 floating-point operations per active-cell update of the FP64 MWDG2
# step (adds, multiplies, 2 per fused multiply-add; divisions and square
# roots as the instructions they expand to), counted by ncu over the ten
# kernels of one step on this workload after 1800 s: 3.249e8 operations for
# 244,945 leaves (profiles/fp64_flops_valley1024_mwdg2.md)
FP64_FLOPS_PER_UPDATE = 1326
E2E_STEPS = 200
# DRAM bytes (read + write) per launch measured by ncu for a kernel of the
# headline workload (FP32 MWDG2), when the kernel has not changed since
# (profiles/mwdg2_valley1024_f32_launches.md); absent while it has
TRAFFIC = {"dg2_update_stage2": 58_214_912 + 2_988_544}


def run_ensemble(args):
    """Batched ensemble: seeded valleys of sides 256, 512, 768, 1024 (M 2^L,
    M in {1, 3}), per-member Manning n and inflow scale, FP32 MWDG2 at
    eps = 1e-3.  All members run to the spin-up time, the launch shapes are
    autotuned (unless --no-tune), then K ensemble steps (one graph launch
    each, the members in batched launches over a (member, block) work list)
    are timed with CUDA events, bracketed by an L2 flush.  For comparison,
    K steps of the same ensemble with one graph branch per member, and K
    steps with the members queued one after another (each its own graph)."""
    import torch
    import paper_2107_02750_gb300 as M
    from paper_2107_02750_gb300 import synth as S
    probs = S.ensemble(count=args.ensemble)
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream
    members = [make_solver(p, M.F32, sptr) for p in probs]
    ens = M.Ensemble(members, stream=sptr)
    ens.run_to_time(args.spinup)
    chosen = None if args.no_tune else ens.tune(steps=8).tolist()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        ens.step(args.warmup)
        torch.cuda.synchronize()
        u0 = sum(m.get_counters()[1] for m in members)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
        flush.fill_(1.0)
        ev[0][0].record(stream)
        ens.step(args.steps)
        ev[0][1].record(stream)
        torch.cuda.synchronize()
        u1 = sum(m.get_counters()[1] for m in members)
        flush.fill_(2.0)
        ev[1][0].record(stream)
        for _ in range(args.steps):
            for m in members:
                m.run_steps(1)
        ev[1][1].record(stream)
        torch.cuda.synchronize()
        u2 = sum(m.get_counters()[1] for m in members)
        # batched groups of g members (one launch per kernel and group)
        batched = {}
        for grp in (4, 8, 16, 64):
            ens.set_batch(grp)
            ens.step(args.warmup)
            torch.cuda.synchronize()
            ua = sum(m.get_counters()[1] for m in members)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(float(grp))
            e0.record(stream)
            ens.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ub = sum(m.get_counters()[1] for m in members)
            ms = e0.elapsed_time(e1)
            batched[str(grp)] = {"value": (ub - ua) / (ms * 1e-3), "ms_per_step": ms / args.steps}
        ens.set_batch(0)
    ms_ens = ev[0][0].elapsed_time(ev[0][1])
    ms_seq = ev[1][0].elapsed_time(ev[1][1])
    sides = [p.nx for p in probs]
    return {"metric": "MWDG2 ensemble active-cell updates/s (batched scenarios, one graph per step)",
            "value": (u1 - u0) / (ms_ens * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_ens / args.steps, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(probs)} seeded fractal valleys, sides {sorted(set(sides))} "
                                   f"(total {sum(x * x for x in sides)} finest cells), eps=1e-3",
                       "spinup_s": args.spinup, "tuned_shapes": chosen},
            "batched_groups": {"unit": UNIT, "by_group_size": batched,
                               "what": "the same ensemble with its members in batched groups of g (one launch "
                                       "per kernel over a (member, block) work list per group, groups on "
                                       "parallel branches)"},
            "sequential": {"value": (u2 - u1) / (ms_seq * 1e-3), "unit": UNIT,
                           "ms_per_step": ms_seq / args.steps,
                           "what": "the same steps with members queued one after another"}}


def run_adjoint(args):
    """Differentiable DG2 (discrete adjoint, uniform grid): the squared depth
    misfit at 16 seeded gauge cells after one checkpoint segment of
    --adjoint-steps steps on the n x n valley (seed 1, with a flowing start and
    a 60-knot hydrograph), differentiated with respect to Manning n, the bed
    planes, the knots and the initial state, in FP32 (the line's value) and in
    FP64 (the bit-exact reference path, reported beside it).  Timed with CUDA
    events on the library's stream: the segment's forward sweep (CFL steps
    recorded) and its backward sweep (recomputation from the checkpoint, then
    the reverse kernels).  One unit = one cell carried through one step forward
    and back."""
    import torch
    import paper_2107_02750_gb300 as M
    from paper_2107_02750_gb300 import synth as S
    from paper_2107_02750_gb300.adjoint import Dg2Adjoint, dg2_run
    K = args.adjoint_steps
    p, gauges = S.adjoint_reach(n=args.n, crop_of=args.n)
    cells = p.nx * p.ny

    def measure(precision, prof=False):
        adj = Dg2Adjoint(p.nx, p.ny, p.dx, cfl=p.cfl, dt_max=p.dt_max, limiter=p.limiter, bc=tuple(p.bc),
                         inflow_edge=p.inflow_edge, inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1, max_steps=K,
                         precision=precision, tape_views=True)
        dev = adj.device
        U0 = torch.cat([adj.project(p.h_vert), adj.project(p.qx_vert), adj.project(p.qy_vert)])
        z = adj.project(p.z_vert)
        n = torch.tensor(p.n_cell(), dtype=adj.dtype, device=dev)
        kt = torch.tensor(p.inflow_t, dtype=torch.float64, device=dev)
        kQ = torch.tensor(p.inflow_Q, dtype=torch.float64, device=dev)
        gj = torch.tensor(gauges[:, 0], device=dev)
        gi = torch.tensor(gauges[:, 1], device=dev)
        h_obs = U0[0, gj, gi] + 0.05   # synthetic observations

        def segment(steps):
            leaves = [x.clone().requires_grad_(True) for x in (U0, z, n, kQ)]
            UK, d, t = dg2_run(adj, leaves[0], leaves[1], leaves[2], leaves[3], kt, 0.0, steps)
            return leaves, ((UK[0, gj, gi] - h_obs) ** 2).sum(), t

        for _ in range(max(3, args.warmup)):
            leaves, J, _ = segment(min(K, 20))
            J.backward()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with Clocks(dev.index) as clk:
            ev[0].record()
            leaves, J, t_seg = segment(K)
            ev[1].record()
            J.backward()
            ev[2].record()
            torch.cuda.synchronize()
        ms_f, ms_b = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        times = None
        if prof:
            # the same segment again with a CUDA event pair around every
            # launch group, for the per-kernel roofline (the events cost
            # about 10 % of the segment, so the line's value is the run above)
            adj.profile(40 * K + 64)
            _, J2, _ = segment(K)
            J2.backward()
            torch.cuda.synchronize()
            times = adj.kernel_times()
            adj.profile(0)
        grads = {k: float(x.grad.abs().max()) for k, x in zip(("U0", "z", "n", "Q"), leaves)}
        return {"value": cells * K / ((ms_f + ms_b) * 1e-3), "ms_per_step": (ms_f + ms_b) / K,
                "forward_ms": ms_f, "backward_ms": ms_b, "simulated_s": t_seg, "max_abs_grad": grads,
                "clocks": clk.summary(), "kernel_ms": times}

    r32 = measure(M.F32, prof=True)
    r64 = None if args.no_fp64 else measure(M.F64)
    frozen = run_adjoint_frozen(args, min(K, 100))
    roof = adjoint_roofline(r32.pop("kernel_ms"), cells, 4)
    cb = None if args.no_cpu else adjoint_cpu_baseline(args.n)
    line = {"metric": "DG2 adjoint cell-steps/s (forward + reverse sweep of one checkpoint segment)",
            "value": r32["value"], "unit": "cell-steps/s", "n_gpus": 1, "steps": K,
            "warmup": max(3, args.warmup), "ms_per_step": r32["ms_per_step"], "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"DG2 adjoint, {p.nx}x{p.ny} uniform valley (seed 1), dx=10 m, flowing start, "
                                   f"60-knot hydrograph, 16 gauges, squared depth misfit, segment {K} steps",
                       "inputs": "tape and state arrays far larger than L2",
                       "tape": "each step's state, stage inputs and flux views (51 coefficients per cell)"},
            "forward_ms": r32["forward_ms"], "backward_ms": r32["backward_ms"], "simulated_s": r32["simulated_s"],
            "max_abs_grad": r32["max_abs_grad"], "gpu_launches": 18 * K + 1, "clocks": r32["clocks"],
            "roofline": roof, "fp64": r64, "cpu_baseline": cb, "frozen_mwdg2": frozen}
    if r64 is not None:
        r64.pop("kernel_ms", None)
    return line


def run_adjoint_frozen(args, K):
    """The adjoint on the benchmark workload's own MWDG2 grid, frozen: the
    1024 x 1024 valley's active leaves and state after 1800 s of the FP32
    solver, one checkpoint segment of K steps from there (CFL steps over the
    leaves), the squared depth misfit at 16 seeded wet leaves, forward and
    backward sweeps timed with CUDA events, FP32 and FP64.  One unit = one
    active leaf carried through one step forward and back."""
    import torch
    import paper_2107_02750_gb300 as M
    from paper_2107_02750_gb300 import synth as S
    from paper_2107_02750_gb300.adjoint import Dg2Adjoint, dg2_run
    p = S.valley(n=args.n, L=args.n.bit_length() - 1)
    sol = make_solver(p, M.F32, torch.cuda.current_stream().cuda_stream)
    sol.run_to_time(1800.0)
    t0 = sol.get_time()[0]
    lev, ii, jj, co = sol.read_active()
    del sol
    nl = len(lev)
    nodes = sum((p.M << l) * (p.N << l) for l in range(p.L + 1))
    pick = np.random.default_rng(3).choice(np.flatnonzero(co[:, 0] > 0.5), size=16, replace=False)
    res = {"workload": f"{p.nx}x{p.ny} valley (seed 1), MWDG2 eps={p.eps} grid and state of the FP32 solver at "
                       f"t={t0:.0f} s, frozen; segment {K} CFL steps; squared depth misfit at 16 wet leaves",
           "leaves": nl, "level_nodes": nodes, "unit": "leaf-steps/s"}
    for name, prec in (("f32", M.F32), ("f64", M.F64)):
        if prec == M.F64 and args.no_fp64:
            continue
        adj = Dg2Adjoint.frozen(p.M, p.N, p.L, p.dx, M.ADAPTIVE, lev, ii, jj, cfl=p.cfl, dt_max=p.dt_max,
                                limiter=p.limiter, bc=tuple(p.bc), inflow_edge=p.inflow_edge,
                                inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1, rain_rate=p.rain_rate,
                                rain_t_end=p.rain_t_end, max_steps=K, precision=prec, tape_views=True)
        dev = adj.device
        U0 = torch.tensor(np.ascontiguousarray(co.T), dtype=adj.dtype, device=dev)
        z = adj.project(p.z_vert)
        n = torch.tensor(p.n_cell(), dtype=adj.dtype, device=dev)
        kt = torch.tensor(p.inflow_t, dtype=torch.float64, device=dev)
        kQ = torch.tensor(p.inflow_Q, dtype=torch.float64, device=dev)
        gidx = torch.tensor(pick, device=dev)
        h_obs = U0[0, gidx] + 0.05

        def segment(steps):
            leaves = [x.clone().requires_grad_(True) for x in (U0, z, n, kQ)]
            UK, d, t = dg2_run(adj, leaves[0], leaves[1], leaves[2], leaves[3], kt, t0, steps)
            return leaves, ((UK[0, gidx] - h_obs) ** 2).sum(), t

        for _ in range(max(3, args.warmup)):
            _, J, _ = segment(min(K, 10))
            J.backward()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        with Clocks(dev.index) as clk:
            ev[0].record()
            leaves, J, t_seg = segment(K)
            ev[1].record()
            J.backward()
            ev[2].record()
            torch.cuda.synchronize()
        ms_f, ms_b = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        res[name] = {"value": nl * K / ((ms_f + ms_b) * 1e-3), "ms_per_step": (ms_f + ms_b) / K,
                     "forward_ms": ms_f, "backward_ms": ms_b, "simulated_s": t_seg - t0,
                     "max_abs_grad": {k: float(x.grad.abs().max()) for k, x in zip(("U0", "z", "n", "Q"), leaves)},
                     "clocks": clk.summary()}
        del adj
    return res


# algorithmic coefficients moved per cell by one launch of each adjoint kernel
# class (reads + writes of unique data, neighbour re-reads not counted; the
# two stages averaged where they differ; the interface class per cell covers
# its two faces), and the bytes of the clip flags
ADJ_VALUES_PER_CELL = {"friction": 19, "limit": 33, "update": 34.5, "cfl": 3, "rev_face": 49, "rev_limit": 67,
                       "rev_gather": 32, "rev_friction": 30}
ADJ_FLAG_BYTES = {"update": 1, "rev_face": 1, "rev_limit": 1}
# warp instructions executed per cell by the uniform grid's fused stage
# kernels, counted by ncu at this workload
# (profiles/issue_rate_valley1024_f32.md), while those kernels are unchanged;
# the SM clock of the issue ceiling (GB300's maximum, which the benchmark's
# clock record shows under load)
UNI_WARP_INSTR_PER_CELL = {"dg2_update_stage1": 28.43, "dg2_update_stage2": 34.09}
ISSUE_CLOCK_MHZ = 2070
# FP64 pipe busy (% of active cycles) over the FP64 step's kernels, from ncu
# (profiles/fp64_pipe_valley512_mwdg2.md), while those kernels are unchanged
# (the encode's and the flux views' figures were taken before their tile
# slot offsets became a closed form, an integer-only change that left their
# FP64 instructions as they were)
FP64_PIPE_BUSY = {"min": 57.4, "max": 72.0, "stage_update": 72.0, "significance_encode": 62.1}

# DRAM bytes (read + write) per launch measured by ncu for the FP32 adjoint
# kernels at this workload, while the kernel is unchanged (see profiles/)
# (captured before the interfaces' outflow limit was added to these kernels:
# none is current, so the adjoint line reports no traffic)
ADJ_TRAFFIC = {}


def adjoint_roofline(times, cells, elem):
    """roofline of the adjoint kernel class with the largest time in the timed
    segment: algorithmic bytes per launch / its mean event-timed duration"""
    peak, src = peaks()
    cls = max((c for c in times if c in ADJ_VALUES_PER_CELL), key=lambda c: times[c][0])
    ms, cnt = times[cls]
    per_launch = cells * (ADJ_VALUES_PER_CELL[cls] * elem + ADJ_FLAG_BYTES.get(cls, 0))
    achieved = per_launch / (ms / cnt * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": cls, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": src, "traffic": ADJ_TRAFFIC.get(cls),
            "bytes_per_launch": per_launch, "launches": cnt, "mean_ms": ms / cnt,
            "share_of_segment": ms / sum(v[0] for v in times.values()),
            "step_ms_by_class": {c: v[0] for c, v in times.items() if v[1]}}


def adjoint_cpu_baseline(n_full, budget_s=10.0):
    """The adjoint oracle (PyTorch CPU autograd over the restated step) on a
    64 x 64 crop of the same valley, as many steps as fit the budget."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import oracle as O
    from oracle import dg2_adjoint as A
    from paper_2107_02750_gb300 import synth as S
    from util import oracle_sim
    p, gauges = S.adjoint_reach(n=64, crop_of=n_full)
    s = oracle_sim(p)
    _, _, _, co = s.leaves()
    U0 = co.T.reshape(9, p.ny, p.nx).copy()
    z = s.z_level(0)[0].reshape(3, p.ny, p.nx)
    P = A.Grid(nx=p.nx, ny=p.ny, dx=p.dx, limiter=p.limiter, bc=tuple(p.bc), inflow_edge=p.inflow_edge,
               inflow_c0=p.inflow_c0, inflow_c1=p.inflow_c1, knot_t=list(map(float, p.inflow_t)))
    seed = np.zeros((9, p.ny, p.nx))
    for j, i in gauges:
        seed[0, j, i] = 1.0
    K, spent = 5, 0.0
    while True:
        dts = [s.step() for _ in range(K)]
        t0 = time.perf_counter()
        A.gradients(U0, z, p.n_cell(), p.inflow_Q, dts, 0.0, P, seed)
        spent = time.perf_counter() - t0
        if spent > budget_s / 4 or K >= 80:
            break
        s = oracle_sim(p)
        K *= 2
    return {"value": p.nx * p.ny * K / spent, "unit": "cell-steps/s", "cores": torch.get_num_threads(),
            "kind": "oracle", "sample": f"64x64 crop, {K} steps, forward + autograd reverse"}


def main():
    args = parse()
    if args.adjoint:
        print(json.dumps(run_adjoint(args)))
        return
    if args.scheme != "dg2":  # the other solvers: throughput line only
        args.no_fp64 = True
        args.no_cpu = True
    if args.ensemble > 0:
        print(json.dumps(run_ensemble(args)))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(args)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_gpu(args, rank, world)
    if rank == 0:
        cb = None if args.no_cpu else cpu_baseline(args.n)
        line = {"metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": out["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": workload(args.n, ({"adaptive": "MWDG2", "uniform": "uniform DG2",
                                                          "static": "static DG2"}[args.grid]
                                                         if args.scheme == "dg2" else
                                                         {"fv1": "HWFV1", "acc": "static-grid ACC"}[args.scheme])),
                           "nx": args.n, "ny": args.n, "L": args.n.bit_length() - 1,
                           "eps": 1e-3, "spinup_s": out["t_spinup"], "mean_active_leaves": out["mean_active"],
                           "l2": "flushed (256 MB write) before every timed step",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": out["roofline"], "cpu_baseline": cb, "e2e": out["e2e"], "clocks": out["clocks"],
                "gpu_launches": out["gpu_launches"]}
        for k in ("uniform_dg2", "fp64", "fma_peaks_tflops", "accuracy_f32_vs_f64", "accuracy_f32_on_fp64_steps",
                  "fp64_vs_fp64_one_extra_stop", "run_average_2h"):
            if k in out:
                line[k] = out[k]
        if args.urban and args.scheme == "dg2" and args.grid == "adaptive" and not args.no_fp64:
            import torch
            flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
            line["urban_static_vs_uniform"] = run_urban(torch.cuda.current_stream(), flush,
                                                        max(5, args.steps), args.warmup, full=args.urban >= 2)
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
