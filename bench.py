#!/usr/bin/env python3
"""Benchmark of the GB300 IB-GM time step (Wiens & Stockie, arxiv 1305.3976).

Workload (one "step" = one full IB-GM time step, Sec. 3.4 Steps 1a-3f): 3D
ellipsoidal membrane in the periodic unit cube, 128^3 MAC grid, rho = 1,
mu = 0.05, semi-axes 0.2/0.25/0.3, icosahedral nu = 64 mesh (40962 markers,
122880 force connections, sigma = 1), dt = 5e-4; FP32 fields, FP64 markers.
Synthetic, seeded inputs.  L2 is flushed (a 256 MiB write) before every timed
step; each step is timed with CUDA events on the stream that launches it.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the same workload instead (rank 0 only; other ranks exit without work).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IB steps/s & cell-updates/s FP32 vs FP64 on one GB300; line-solve HBM GB/s"


def workload(n=128, nu=64, fields="FP32 fields"):
    """The benchmark workload by name (defaults: the 128^3 configuration)."""
    nm, ne = 10 * nu * nu + 2, 30 * nu * nu
    return (f"3D ellipsoidal membrane, {n}^3 periodic MAC grid, rho=1, mu=0.05, semi-axes 0.2/0.25/0.3, "
            f"icosahedral nu={nu} mesh ({nm} markers, {ne} springs, sigma=1), dt=5e-4, {fields}, FP64 markers")


WORKLOAD = workload()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--nu", type=int, default=64)
    ap.add_argument("--quick", action="store_true", help="skip the FP64, line-solve, e2e and CPU legs")
    ap.add_argument("--line-solve-only", action="store_true",
                    help="run only the line-solve microbench (one JSON line with its table), e.g. under a profiler")
    ap.add_argument("--sweep-config", default=None,
                    help="comma-separated line-solve configuration ids per axis (as printed under "
                         "sweep_configs) to use instead of autotuning, e.g. to profile a run's choice")
    ap.add_argument("--profile-one-step", type=int, nargs="?", const=0, default=None, metavar="I",
                    help="bracket per-kernel profiling step I (default 0; the steps rotate the split order) "
                         "with cudaProfilerStart/Stop, so that a profiler started with --profile-from-start off "
                         "captures exactly that step's kernels")
    return ap.parse_args()


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x, world, device=None):
    """Maximum of a per-rank float over all ranks (identity when world == 1).
    Works with any initialised torch.distributed backend (NCCL on GPUs, gloo
    on CPU)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells, steps, world, total_ms_max):
    """Whole-job cell-updates/s of `world` independent replicas, each
    advancing `cells` cells by `steps` steps, timed by the slowest rank."""
    return cells * steps * world / (total_ms_max * 1e-3)


def scene(args):
    from paper_1305_3976_gb300 import inputs as I
    return I.ellipsoid_3d(n=args.n, nu=args.nu)


# --------------------------------------------------------------------------
# clocks sampled during the timed region


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        load = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": float(np.median(load)) if load else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# algorithmic bytes per launch of each kernel slot (3D, w bytes per field word)


def kernel_bytes(name, cells, nm, ne, w, d=3):
    """HBM bytes of one launch: the arrays a kernel must stream from or to
    DRAM.  The 4^d grid nodes that interpolation gathers and spreading updates
    per marker and component are not counted: neighbouring markers share most
    of them and they are served by L1/L2 (ncu: interpolation and spreading move
    8.3 and 8.4 MB of DRAM per 128^3 step, their marker arrays being 7.9 MB);
    spreading is reported in atomic updates per second instead
    (stencil_updates)."""
    m = {
        # locations of X^n (d slots per component: index + 4 weights), U^n out
        "interp": nm * d * (d * (4 + 4 * w) + w),
        # X, U, U^{n-1} in; X^{n+1}, X^{n+1/2}, U^{n-1}, both location sets out
        "update": nm * (d * 8 + 2 * d * w + 2 * d * 8 + d * w + 2 * 2 * d * (4 + 4 * w)),
        # own and neighbour X^{n+1/2}, CSR row/col/kappa/rest, G out
        "force": nm * (d * 8 + 16 + d * w) + 2 * ne * (d * 8 + 4 + 16),
        # locations of X^{n+1/2}, G in
        "spread": nm * d * (d * (4 + 4 * w) + w),
        # u(3), p, psi, N(u^{n-1})(3) in; R(3), N(u^n)(3) out
        "rhs": cells * w * (3 * d + 5),
        "mom_sweep_1": cells * w * 2 * d,
        "mom_sweep_2": cells * w * 2 * d,
        "mom_sweep_3": cells * w * 3 * d,   # e in, u^n in/out
        "psi_sweep_1": cells * w * (d + 5), # u(3), div, p in; psi, div, p out
        "psi_sweep_2": cells * w * 2,
        "psi_sweep_3": cells * w * 4,       # psi, p in; psi, p out
    }
    return m[name]


def stencil_updates(nm, d=3):
    """Grid-node updates of one spreading launch (and node reads of one
    interpolation launch): 4^d nodes per marker and component."""
    return nm * d * 4 ** d


def survey_step_bytes(cells, w, d=3):
    """The per-pass byte model of a 3D step with one field round trip per
    sweep: right-hand side 17w + force clear 3w, six x/y momentum sweeps 12w,
    three z sweeps with u^n 9w, divergence 4w, psi x/y sweeps 4w, psi z sweep
    with the pressure update 6w: 55 words per cell."""
    assert d == 3
    return 55 * w * cells


def fp64_ops(name, cells):
    """FP64 instructions of one launch of the FP64 right-hand side or of one
    FP64 line-solve sweep, counted from the arithmetic: per cell and velocity
    component 30 (Laplacian 2 + 2 per axis, skew advection 5 per axis, p* 2,
    the R and N assembly 5); per line element 4 (the local recurrence and the
    correction of each of the two factors)."""
    return {"rhs": 90 * cells, "sweep": 4 * cells}[name]


STEP_SLOTS = ("interp", "update", "force", "rhs", "spread", "mom_sweep_1", "mom_sweep_2", "mom_sweep_3",
              "psi_sweep_1", "psi_sweep_2", "psi_sweep_3")


def step_bytes(cells, nm, ne, w, d=3):
    """Algorithmic bytes of one whole step: the sum over its kernels."""
    return sum(kernel_bytes(k, cells, nm, ne, w, d) for k in STEP_SLOTS)


def source_hash():
    """Hash of the CUDA sources without their // comments and blank lines, so
    that a counter file stays valid across comment edits but not code edits."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1305_3976_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            for line in open(os.path.join(csrc, f), encoding="utf-8"):
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_traffic(kernel, tag):
    """dram bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources and on workload `tag`."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        t = json.load(open(p))
    except Exception:
        return None
    if t.get("source_hash") != source_hash() or t.get("workload") != tag:
        return None
    return t.get("kernels", {}).get(kernel)


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def line_solve_leg(ib, torch, dev, flush, hbm, sizes=(128, 256, 512), precisions=("f32", "f64"), fp64_ops_peak=None):
    """Sec. 6.1's Poisson-comparison problem: (1 - D_xx)(1 - D_yy)(1 - D_zz) psi
    = f with f = sin 2 pi x cos 2 pi y cos 2 pi z at the cell centres of the
    unit cube, three line-solve sweeps through ib_split_solve.  r = 1/h^2 (the
    psi operator) everywhere, plus the momentum operator's r = mu dt / (2 rho
    h^2) of the benchmark workload at 512^3 FP32.  L2 is flushed before every
    timed solve; bytes = 3 sweeps x (read + write) of the field."""
    rows = []
    for N in sizes:
        for prec in precisions:
            dtype = torch.float32 if prec == "f32" else torch.float64
            c = (torch.arange(N, device=dev, dtype=torch.float64) + 0.5) / N
            z, y, x = torch.meshgrid(c, c, c, indexing="ij")
            f = (torch.sin(2 * torch.pi * x) * torch.cos(2 * torch.pi * y) * torch.cos(2 * torch.pi * z)).to(dtype)
            del x, y, z
            psi = torch.empty_like(f)
            kinds = [("psi", float(N * N))]
            if N == 512 and prec == "f32":
                kinds.append(("momentum", 0.05 * 5e-4 / 2.0 * N * N))
            for kind, rr in kinds:
                r = (rr,) * 3
                pcode = ib.IB_FP32 if prec == "f32" else ib.IB_FP64
                for _ in range(3):
                    ib.ib_split_solve(pcode, 3, (N, N, N), r, f, psi)
                torch.cuda.synchronize()
                reps, tot = 10, 0.0
                for _ in range(reps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    ib.ib_split_solve(pcode, 3, (N, N, N), r, f, psi)
                    e1.record()
                    torch.cuda.synchronize()
                    tot += e0.elapsed_time(e1)
                ms = tot / reps
                nbytes = 3 * 2 * f.element_size() * N ** 3
                gbs = nbytes / (ms * 1e-3) / 1e9
                row = {"n": N, "dtype": prec, "r": kind, "ms": round(ms, 5), "GB_per_s": round(gbs, 1),
                       "frac": round(gbs / hbm, 4), "cell_updates_per_s": N ** 3 / (ms * 1e-3)}
                if prec == "f64" and fp64_ops_peak:
                    ops = 3 * fp64_ops("sweep", N ** 3)
                    row["alu_frac"] = round(ops / (ms * 1e-3) / fp64_ops_peak, 4)
                rows.append(row)
            del f, psi
    return rows


# --------------------------------------------------------------------------


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle as O
    sc = scene(args)
    P = O.params(3, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel, rotate=True)
    sim = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
    # each oracle step takes about 2 s at 128^3 on one core: one untimed step
    # (the first step takes the n = 0 branch) and at most 5 timed ones
    steps = max(1, min(args.steps, 5))
    warm = min(args.warmup, 1)
    sim.step(warm)
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    cells = sc.cells
    val = cells * steps / dt
    sample = f"{steps} oracle step(s) of the {args.n}^3 workload (requested --steps {args.steps})"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "cell-updates/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args.n, args.nu, "FP64 fields (oracle)"), "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model()},
        "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import torch
    import paper_1305_3976_gb300 as ib

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    if args.line_solve_only:
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        hbm, _ = peaks()
        sizes = (args.n,) if args.n != 128 else (128, 256, 512)
        rows = line_solve_leg(ib, torch, dev, flush, hbm, sizes=sizes,
                              precisions=("f32",) if args.precision == "fp32" else ("f64",))
        if rank == 0:
            print(json.dumps({"metric": "line-solve HBM GB/s", "line_solve_table": rows}), flush=True)
        return 0
    sc = scene(args)
    cells, nm, ne = sc.cells, sc.X.shape[0], sc.edges.shape[0]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > 129 MB L2

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def make_grid(prec):
        g = ib.Grid(3, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, precision=prec, kernel=sc.kernel,
                    rotate_split=True)
        g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
        if args.sweep_config and prec == args.precision:
            g.fix_sweep_configs([int(x) for x in args.sweep_config.split(",")])
        return g

    def timed_steps(g, K, W):
        g.step(W)
        barrier()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for i in range(K):
            flush.zero_()
            starts[i].record()
            g.step(1)
            ends[i].record()
        barrier()
        return sum(s.elapsed_time(e) for s, e in zip(starts, ends))   # ms

    def max_over_ranks(x):
        return reduce_max(x, world, dev)

    prec = args.precision
    w = 4 if prec == "fp32" else 8
    # ceilings of the kernels not bound by HBM, measured on this GPU
    unit_peaks = {"fp64_flops": ib.ib_measure_peak(ib.IB_PEAK_FP64_FMA),
                  "fp32_flops": ib.ib_measure_peak(ib.IB_PEAK_FP32_FMA),
                  "l2_atomics_per_s": ib.ib_measure_peak(ib.IB_PEAK_L2_ATOMIC)}
    g = make_grid(prec)
    clocks = Clocks(local)
    clocks.start()
    tot_ms = timed_steps(g, args.steps, args.warmup)
    clk = clocks.stop()
    tot_ms = max_over_ranks(tot_ms)
    ms_step = tot_ms / args.steps
    value = job_value(cells, args.steps, world, tot_ms)

    # per-kernel durations: every kernel launched on its own, CUDA events on
    # the launching stream, L2 flushed before each step
    prof = {}
    nprof = 6
    for i in range(nprof):
        flush.zero_()
        torch.cuda.synchronize()
        bracket = args.profile_one_step is not None and i == args.profile_one_step
        if bracket:
            torch.cuda.profiler.start()
        for k, v in g.profile(1).items():
            prof[k] = prof.get(k, 0.0) + v
        if bracket:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
    per_launch = {k: v / nprof for k, v in prof.items()}
    dom = max(per_launch, key=per_launch.get)
    hbm, peak_kind = peaks()
    ab = kernel_bytes(dom, cells, nm, ne, w)
    achieved = ab / (per_launch[dom] * 1e-3) / 1e9
    sb = step_bytes(cells, nm, ne, w)
    diag = g.diagnostics()
    tuned = g.sweep_configs()
    g.close()

    out = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": workload(args.n, args.nu, "FP32 fields" if prec == "fp32" else "FP64 fields"),
                   "cells": cells, "markers": nm, "springs": ne,
                   "l2": "flushed (256 MiB write) before every timed step", "parallelism": f"replicas x{world}"},
        "steps_per_s": 1e3 / ms_step * world,
        "kernels_ms_per_launch": {k: round(v, 5) for k, v in per_launch.items()},
        "sweep_configs": {"x": {"id": tuned[0][0], "ctas_per_sm": tuned[0][3]},
                          **{ax: {"id": t[0], "vector": t[1], "chunk": t[2], "warps_per_line": t[3]}
                             for ax, t in zip(("y", "z"), tuned[1:])}},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": ab, "traffic": measured_traffic(dom, f"ellipsoid{args.n}_{prec}" if args.nu == 64 else None)},
        "step_roofline": {"algorithmic_bytes": sb, "GB_per_s": sb / (ms_step * 1e-3) / 1e9,
                          "frac": sb / (ms_step * 1e-3) / 1e9 / hbm,
                          "what": "sum of the kernels' HBM byte models per step / ms_per_step",
                          "survey_model": {"bytes": survey_step_bytes(cells, w),
                                           "GB_per_s": survey_step_bytes(cells, w) / (ms_step * 1e-3) / 1e9,
                                           "frac": survey_step_bytes(cells, w) / (ms_step * 1e-3) / 1e9 / hbm,
                                           "what": "55 words per cell (one field round trip per sweep)"}},
        "spreading": {"bound": "l2_atomic", "updates_per_launch": stencil_updates(nm),
                      "ms": per_launch["spread"],
                      "updates_per_s": stencil_updates(nm) / (per_launch["spread"] * 1e-3),
                      "peak": unit_peaks["l2_atomics_per_s"],
                      "frac": stencil_updates(nm) / (per_launch["spread"] * 1e-3) / unit_peaks["l2_atomics_per_s"],
                      "unit": "atomic updates/s"},
        "measured_unit_peaks": unit_peaks,
        "gpu_launches": args.steps * (11 if nm else 7),
        "clocks": clk,
        "state_check": {"volume": diag["volume"], "div_l2": diag["div_l2"], "kinetic": diag["kinetic"]},
    }

    if not args.quick:
        # FP64 fields on the same workload
        if prec == "fp32":
            g64 = make_grid("fp64")
            k64 = max(5, args.steps // 2)
            ms64 = max_over_ranks(timed_steps(g64, k64, args.warmup)) / k64
            p64 = {}
            for _ in range(3):
                flush.zero_()
                torch.cuda.synchronize()
                for k, v in g64.profile(1).items():
                    p64[k] = p64.get(k, 0.0) + v / 3
            g64.close()
            fp64_ops_peak = unit_peaks["fp64_flops"] / 2.0     # FP64 instructions/s (one FMA = 2 FLOP)
            alu = {}
            for slot, kind in (("rhs", "rhs"), ("mom_sweep_1", "sweep"), ("psi_sweep_2", "sweep")):
                ops = fp64_ops(kind, cells) * (3 if slot.startswith("mom") else 1)
                alu[slot] = {"fp64_ops": ops, "ms": p64[slot], "achieved": ops / (p64[slot] * 1e-3),
                             "peak": fp64_ops_peak, "frac": ops / (p64[slot] * 1e-3) / fp64_ops_peak,
                             "unit": "FP64 instructions/s"}
            out["fp64"] = {"value": cells * world / (ms64 * 1e-3), "unit": "cell-updates/s", "ms_per_step": ms64,
                           "steps_per_s": 1e3 / ms64 * world, "steps": k64,
                           "alu_roofline": {"bound": "alu", "kernels": alu,
                                            "what": "FP64 instructions counted from the arithmetic / ms, against "
                                                    "the measured FP64 FMA issue rate (ib_measure_peak)"},
                           "kernels_ms_per_launch": {k: round(v, 5) for k, v in p64.items()}}
        from paper_1305_3976_gb300 import inputs as I
        # line-solve microbench: the paper's Poisson-comparison problem
        out["line_solve_table"] = line_solve_leg(ib, torch, dev, flush, hbm,
                                                 fp64_ops_peak=unit_peaks["fp64_flops"] / 2.0)
        head = [r for r in out["line_solve_table"] if r["n"] == 512 and r["dtype"] == "f32" and r["r"] == "psi"][0]
        out["line_solve"] = {"workload": "(1-D_xx)(1-D_yy)(1-D_zz) psi = f, 512^3 FP32, r = N^2, 3 sweeps",
                             "ms": head["ms"], "GB_per_s": head["GB_per_s"], "frac": head["frac"],
                             "cell_updates_per_s": head["cell_updates_per_s"]}
        # the 512^3 precision-scaling scene: 8 randomly oriented ellipsoids of
        # 64002 markers each, mu = 0.01, dt = 3.125e-5; FP32 and FP64 fields
        sc3 = I.random_ellipsoids_3d()
        cells3, nm3, ne3 = sc3.cells, sc3.X.shape[0], sc3.edges.shape[0]
        big = {}
        for prec3, k3 in (("fp32", 10), ("fp64", 3)):
            g3 = ib.Grid(3, sc3.n, rho=sc3.rho, mu=sc3.mu, dt=sc3.dt, chi=sc3.chi, precision=prec3,
                         kernel=sc3.kernel, rotate_split=True)
            g3.add_fiber(sc3.X, sc3.edges, sc3.kappa, sc3.rest, sc3.tris)
            ms3 = max_over_ranks(timed_steps(g3, k3, 3)) / k3
            flush.zero_()
            torch.cuda.synchronize()
            p3 = g3.profile(1)
            g3.close()
            w3 = 4 if prec3 == "fp32" else 8
            sb3 = step_bytes(cells3, nm3, ne3, w3)
            dom3 = max(p3, key=p3.get)
            ab3 = kernel_bytes(dom3, cells3, nm3, ne3, w3)
            big[prec3] = {"ms_per_step": ms3, "value": cells3 * world / (ms3 * 1e-3), "unit": "cell-updates/s",
                          "steps": k3, "step_GB_per_s": sb3 / (ms3 * 1e-3) / 1e9,
                          "step_frac": sb3 / (ms3 * 1e-3) / 1e9 / hbm,
                          "dominant_kernel": {"kernel": dom3, "ms": p3[dom3],
                                              "GB_per_s": ab3 / (p3[dom3] * 1e-3) / 1e9,
                                              "frac": ab3 / (p3[dom3] * 1e-3) / 1e9 / hbm},
                          "kernels_ms_per_launch": {k: round(v, 5) for k, v in p3.items()}}
        out["step_512"] = {"workload": "8 randomly oriented ellipsoidal membranes (semi-axes U[0.05,0.1], "
                                       "icosahedral nu=80, 64002 markers each), 512^3, mu=0.01, dt=3.125e-5",
                           "cells": cells3, "markers": nm3, "springs": ne3,
                           "l2": "inputs larger than L2; also flushed before every timed step", **big}
        # batched ensemble: 48 independent runs (N in {48, 64, 96, 128}, sigma
        # log-uniform in [0.1, 10], mu uniform in [0.01, 0.1]), one graph
        # launch per ensemble step, against the same members stepped one by one
        members = I.ensemble_members(count=48)
        grids = []
        for sc_m in members:
            gm = ib.Grid(3, sc_m.n, rho=sc_m.rho, mu=sc_m.mu, dt=sc_m.dt, precision="fp32", rotate_split=True)
            gm.add_fiber(sc_m.X, sc_m.edges, sc_m.kappa, sc_m.rest, sc_m.tris)
            grids.append(gm)
        ens = ib.Ensemble(grids)
        ens.step(args.warmup)
        ke = 100
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ens.step(ke)
        e1.record()
        barrier()
        ms_e = max_over_ranks(e0.elapsed_time(e1)) / ke
        e0.record()
        for _ in range(ke):
            for gm in grids:
                gm.step(1)
        e1.record()
        barrier()
        ms_s = max_over_ranks(e0.elapsed_time(e1)) / ke
        cells_e = sum(int(np.prod(sc_m.n)) for sc_m in members)
        ens.close()
        for gm in grids:
            gm.close()
        out["ensemble"] = {"workload": "48 independent 3D runs, N uniform in {48,64,96,128}, one ellipsoidal "
                                       "membrane each (nu = N/2), sigma log-uniform [0.1,10], mu uniform "
                                       "[0.01,0.1], FP32 fields",
                           "members": len(members), "cells": cells_e,
                           "markers": int(sum(sc_m.X.shape[0] for sc_m in members)), "steps": ke,
                           "ms_per_step": ms_e, "value": cells_e * world / (ms_e * 1e-3),
                           "unit": "cell-updates/s",
                           "survey_model_frac": survey_step_bytes(cells_e, 4) / (ms_e * 1e-3) / 1e9 / hbm,
                           "one_by_one_ms_per_step": ms_s,
                           "one_by_one_value": cells_e * world / (ms_s * 1e-3)}
        # stiffness gradient by the discrete adjoint: 96^3 FP32 fields, 7842
        # markers, one stiffness per connection, 200 steps, checkpoints every
        # 20 steps (forward, replay of every segment, reverse sweep), against
        # the same 200 forward steps alone
        sc_a = I.stiffness_fit_3d()
        adj = {}
        for prec_a in ("fp32", "fp64"):
            ga = ib.Grid(3, sc_a.n, rho=sc_a.rho, mu=sc_a.mu, dt=sc_a.dt, chi=sc_a.chi, precision=prec_a,
                         kernel=sc_a.kernel, rotate_split=True)
            ga.add_fiber(sc_a.X, sc_a.edges, sc_a.kappa, sc_a.rest, sc_a.tris)
            ga.adjoint(20, sc_a.extra["target"], 20)              # warm-up: setup, autotune, graphs
            barrier()
            t0 = time.perf_counter()
            loss_a, _ = ga.adjoint(sc_a.steps, sc_a.extra["target"], 20)
            barrier()
            ta = max_over_ranks(time.perf_counter() - t0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ga.step(sc_a.steps)
            e1.record()
            barrier()
            tf = max_over_ranks(e0.elapsed_time(e1)) * 1e-3
            ga.close()
            adj[prec_a] = {"s": ta, "forward_s": tf, "ratio_to_forward": ta / tf, "loss": loss_a}
        out["adjoint"] = {"workload": "d loss / d kappa for 23520 connection stiffnesses, 96^3, 7842 markers, "
                                      "200 steps, checkpoints every 20 steps",
                          **{k: {kk: (round(vv, 6) if kk != "loss" else vv) for kk, vv in v.items()}
                             for k, v in adj.items()}}
        # the paper's timed 3D problem (Sec. 6, Table 9): the cylindrical shell
        # (N_s = 19N/4 x N_r = 3N markers, dt = 0.04/N, mu = 0.01) at N = 128
        # and 256 for 100 steps, FP32 and FP64 fields, L2 flushed before every
        # step; the paper's wall times are quoted as context only
        cyl = {}
        for N in (128, 256):
            scN = I.cylinder_3d(n=N)
            row = {"markers": int(scN.X.shape[0]), "connections": int(scN.edges.shape[0])}
            for precN in ("fp32", "fp64"):
                gN = ib.Grid(3, scN.n, rho=scN.rho, mu=scN.mu, dt=scN.dt, chi=scN.chi, precision=precN,
                             kernel=scN.kernel, rotate_split=True)
                gN.add_fiber(scN.X, scN.edges, scN.kappa, scN.rest)
                msN = max_over_ranks(timed_steps(gN, 100, 3))
                gN.close()
                row[precN] = {"s_per_100_steps": msN * 1e-3, "ms_per_step": msN / 100,
                              "steps_per_s": 100 / (msN * 1e-3), "cell_updates_per_s": N ** 3 * 100 / (msN * 1e-3)}
            cyl[str(N)] = row
        out["cylinder"] = {"workload": "cylindrical elastic shell of Sec. 6 (axial rest length 1, closed through the "
                                       "periodic box), N^3 grid, 100 steps, dt = 0.04/N",
                           "rows": cyl,
                           "paper_table9_context": {"hardware": "Intel Xeon X5650 cluster (WestGrid Bugaboo), "
                                                                "precision unstated",
                                                    "128": {"1_core_s": 401.0, "128_cores_s": 7.76},
                                                    "256": {"1_core_s": 2600.0, "128_cores_s": 30.2}}}
        # marker re-sorting: the tiled thin ellipses of Sec. 6.3 on 8 x 8 tiles
        # of 64^2 (512^2, 33 152 markers, raised by 0.3 so that the top row
        # straddles the periodic boundary), FP32 fields; interpolation and
        # spreading per launch at the start, after 300 steps of transport in
        # the initial numbering, and after re-numbering by current position
        sct = I.tiled_ellipses_2d(tiles=8, n_per_tile=64, dt=1e-3)
        gt = ib.Grid(2, sct.n, H=sct.H, rho=sct.rho, mu=sct.mu, dt=sct.dt, chi=sct.chi, precision="fp32",
                     kernel=sct.kernel, rotate_split=True)
        gt.add_fiber(sct.X + np.array([0.0, 0.3]), sct.edges, sct.kappa, sct.rest)
        gt.set_velocity(sct.extra["u0"])

        def marker_ms():
            acc = {"interp": 0.0, "spread": 0.0}
            for _ in range(5):
                flush.zero_()
                torch.cuda.synchronize()
                p = gt.profile(1)
                for k in acc:
                    acc[k] += p[k] / 5
            return {k: round(v, 5) for k, v in acc.items()}

        rs = {"start": marker_ms()}
        gt.step(300)
        rs["after_300_steps"] = marker_ms()
        gt.resort_markers()
        rs["after_resort"] = marker_ms()
        gt.close()
        out["marker_resort"] = {"workload": "tiled thin ellipses (Sec. 6.3), 8 x 8 tiles of 64^2, 33152 markers, "
                                            "background flow (1/2, sqrt(3)/2), dt = 1e-3, FP32 fields",
                                "ms_per_launch": rs}
        # the 2D ellipse workload: 64^2, 256 markers, FP64 fields, both kernels,
        # 100 steps (latency-bound: throughput only)
        c1 = {}
        for kern in ("cos4", "peskin4"):
            sc1 = I.thin_ellipse_2d(n=64, ns=256, kernel=kern)
            g1 = ib.Grid(2, sc1.n, rho=sc1.rho, mu=sc1.mu, dt=sc1.dt, chi=sc1.chi, precision="fp64", kernel=kern,
                         rotate_split=True)
            g1.add_fiber(sc1.X, sc1.edges, sc1.kappa, sc1.rest)
            ms1 = max_over_ranks(timed_steps(g1, 100, 3))
            g1.close()
            c1[kern] = {"ms_per_step": ms1 / 100, "steps_per_s": 100 / (ms1 * 1e-3),
                        "cell_updates_per_s": 64 * 64 * 100 / (ms1 * 1e-3)}
        out["ellipse_2d"] = {"workload": "2D elliptical membrane, 64^2, 256 markers, rho=1, mu=0.1, sigma=1, "
                                         "dt=1e-3, FP64 fields, 100 steps", **c1}
        # end to end through the C ABI with host buffers: every step the marker
        # positions come from pinned host memory and go back to it
        ge = make_grid(prec)
        ge.step(args.warmup)
        Xh = torch.empty((nm, 3), dtype=torch.float64, pin_memory=True).numpy()
        ib.ib_read_markers(ge.h, Xh)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ib.ib_set_markers(ge.h, Xh)
            ib.ib_step(ge.h, 1)
            ib.ib_read_markers(ge.h, Xh)
        barrier()
        te = max_over_ranks(time.perf_counter() - t0)
        ge.close()
        out["e2e"] = {"value": cells * args.steps * world / te, "unit": "cell-updates/s",
                      "h2d_bytes_per_step": nm * 3 * 8, "d2h_bytes_per_step": nm * 3 * 8,
                      "what": "per step: ib_set_markers from pinned host memory, ib_step, ib_read_markers to host"}
        # the oracle on this host's cores: one warm-up step (the n = 0 branch),
        # then the median of 3 single steps of the same workload
        if rank == 0 and world == 1:
            import oracle as O
            P = O.params(3, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, chi=sc.chi, kernel=sc.kernel, rotate=True)
            sim = O.Simulation(P, sc.X, sc.edges, sc.kappa, sc.rest)
            sim.step(1)
            ts = []
            for _ in range(3):
                t0 = time.perf_counter()
                sim.step(1)
                ts.append(time.perf_counter() - t0)
            tc = float(np.median(ts))
            out["cpu_baseline"] = {"value": cells / tc, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                                   "cpu": cpu_model(),
                                   "sample": f"median of 3 single steps of the {args.n}^3 workload after one "
                                             f"warm-up step ({tc:.2f} s per step, FP64, one thread)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
