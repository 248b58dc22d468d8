"""Throughput benchmark of the sector-integrand Monte-Carlo hot path.

One step = one pass of the whole hot path over one workload.  Default: the
two-loop massless planar double box at s = t = -1 (orders eps^-4..eps^0, 293
sectors of 6 dimensions, 1141 (sector, eps order) integrands), one unit per
sector evaluating all its orders at every point (--fuse 0: one unit per sector
and order), one Vegas iteration of 10^7 Philox points per sector, binary64:
point generation, Vegas map, bytecode evaluation, reduction, grid refinement
and the per-order assembly.  The metric counts evaluations of (sector, order)
integrands.  --workload box|bubble|box_physical|stress selects the other
configurations.

Prints one JSON line (rank 0).  After the timed region the line also carries
``time_to_1e-4``: GPU-seconds to 1e-4 relative error on every order, plain
binary64 Vegas against the faster forms (randomised QMC, AUTO precision with
point allocation, the learned flow on the double box, the cubature on the
box), measured live (--no-tta skips it).  ``--mode tta`` runs the comparison
with more forms on any workload, ``--mode cuhre`` the cubature's evaluation
rate.  ``--impl reference`` times the oracle (the plain CPU restatement of the
method) on a bounded sample of the same workload.
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
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (points per unit per iteration, iterations, rng)
    "box": (1_000_000, 10, "philox"),
    "bubble": (100_000, 10, "philox"),
    "box_physical": (1_000_000, 10, "philox"),
    "double_box": (10_000_000, 1, "philox"),
    "stress": (1 << 20, 1, "sobol"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="double_box", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "auto"])
    ap.add_argument("--points", type=int, default=0, help="points per unit per iteration (0: workload default)")
    ap.add_argument("--iters", type=int, default=0, help="Vegas iterations per step (0: workload default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tta", action="store_true", help="skip the live time-to-1e-4 comparison")
    ap.add_argument("--fuse", type=int, default=1, help="1: one unit per sector carrying all its eps orders")
    ap.add_argument("--forms", default="fp64,auto,fp32,fp64_alloc,auto_alloc,rqmc_fp64,flow_fp32,cuhre_fp64",
                    help="tta mode: comma-separated forms to run")
    ap.add_argument("--threads", type=int, default=256, help="kernel mode: threads per block")
    ap.add_argument("--ppt", type=int, default=8, help="kernel mode: points per thread per work item")
    ap.add_argument("--units", type=int, default=0, help="kernel mode, stress: the first N integrands (0: all)")
    ap.add_argument("--stress-orders", default="one", choices=["one", "all"],
                    help="stress: one eps coefficient per integrand (10 000 units) or every one of eps^0..eps^2")
    ap.add_argument("--launch-shape", default="",
                    help="throughput mode: threads,points_per_thread,wide_threads instead of the autotuner's")
    ap.add_argument("--wide-threads", type=int, default=0,
                    help="kernel mode: split the fused units by slot count, the few-slot group at this block size")
    ap.add_argument("--min-slots", type=int, default=0, help="kernel mode: only units with at least this many slots")
    ap.add_argument("--max-slots", type=int, default=0,
                    help="kernel mode: only the units whose programs need at most this many slots (0: all)")
    ap.add_argument("--mode", default="throughput", choices=["throughput", "tta", "cuhre", "kernel", "flow"],
                    help="tta: GPU-seconds to 1e-4 relative error per eps order, each precision policy")
    ap.add_argument("--target", type=float, default=1e-4)
    ap.add_argument("--max-iters", type=int, default=400, help="tta mode: Vegas iteration cap per form")
    ap.add_argument("--cap-s", type=float, default=0.0, help="tta mode: GPU-seconds cap per form (0: none)")
    ap.add_argument("--small-x32", type=float, default=-1.0,
                    help="tta mode: binary64 below this coordinate in binary32 units (-1: the binding default)")
    return ap.parse_args()


STRESS_ALL_ORDERS = False      # --stress-orders all: every integrand's eps^0..eps^2 coefficients


def prepared(workload, fuse=False, mix=1, terms=False):
    import workloads as W
    from paper_1511_03614_gb300 import prepare_feynman, prepare_direct
    if workload == "stress":
        return prepare_direct(W.stress_suite(all_orders=STRESS_ALL_ORDERS), "stress")
    return prepare_feynman(getattr(W, workload)(), fuse_orders=bool(fuse), mix_sectors=mix,
                           separate_terms=bool(terms))


def dist_setup(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def op_costs(peaks):
    """FMA-equivalents of each opcode from the measured pipe rates (the interpreter's log)."""
    fma_rate = peaks[0] * 1e12 / 2.0                 # binary64 FMA per second
    log_c = fma_rate / (peaks[6] * 1e9)
    div_c = fma_rate / (peaks[2] * 1e9)
    atan_c = fma_rate / (peaks[7] * 1e9) if len(peaks) > 7 and peaks[7] > 0 else log_c
    inv_c = fma_rate / (peaks[8] * 1e9) if len(peaks) > 8 and peaks[8] > 0 else div_c
    return {"LOG": log_c, "DIV": div_c, "INV": inv_c, "ATAN2": atan_c}


def unit_work(prog, costs, dim, n_out):
    """Work per point of one unit: (algorithmic flops, FMA-equivalent pipe slots,
    flops of the integrand body alone).

    Flops follow the survey's count: ADD SUB MUL NEG ADDC MULC = 1, MAC MACC (fused
    multiply-add) = 2, POWI = its multiplies, and LOG DIV INV ATAN2 converted at their
    measured cost (FMA slots x 2 flops; ``op_costs``); plus the Vegas map (4 per
    coordinate) and the reduction (3 per result: v = f J, sum v, sum v^2).  Pipe slots
    count every instruction of the body as one FMA slot (the special operations at
    their measured cost), so slots x 2 / time is the pipe's occupancy, a different
    figure from the flop rate.
    """
    c = prog.counts
    powi = 0
    for w in prog.code.tolist():
        if (w & 0xFF) == 12:
            e = (w >> 24) & 0xFF
            e = e - 256 if e >= 128 else e
            m = abs(e)
            powi += max(m.bit_length() - 1 + bin(m).count("1") - 1, 0) + (1 if e < 0 else 0)
    special = sum(costs[k] * c.get(k, 0) for k in ("LOG", "DIV", "INV", "ATAN2"))
    body = prog.flops() + powi + 2.0 * special
    slots = prog.flops() - (c.get("MAC", 0) + c.get("MACC", 0)) + powi + special
    extra = 4 * dim + 3 * n_out
    return body + extra, slots + extra, body


def op_costs32(peaks):
    """binary32 FMA-equivalents of logf and of the binary32 divide (atan2f: as logf)."""
    fma_rate = peaks[3] * 1e12 / 2.0
    log_c = fma_rate / (peaks[4] * 1e9)
    div_c = fma_rate / (peaks[5] * 1e9)
    return {"LOG": log_c, "DIV": div_c, "INV": div_c, "ATAN2": log_c}


# DRAM bytes (read + write) per launch of the evaluation kernel from ncu captures, by
# (workload, precision, fused); the kernel stages programs, constants and grids in shared
# memory, so this does not grow with the number of points.  None: not captured for
# the current kernel.
TRAFFIC = {("double_box", "fp64", True): (
    41406976 + 41015552 + 1403392,
    "ncu dram__bytes_read.sum + dram__bytes_write.sum of the two k_eval<double, Philox, 6, registers> launches of "
    "one evaluation pass at the bench's size and shapes (bench.py --mode kernel --workload double_box --points "
    "10000000 --threads 384 --ppt 8 --wide-threads 384): mostly the (unit, chunk) partial sums of the fixed-order "
    "reduction, written back once they outgrow L2, and the sector fills of those 48-byte records")}


def roofline_of(prep, res, peaks, pts, pass_s, args, iters):
    """Roofline of the evaluation kernel (alu-bound: the binary64 pipe for binary64
    units; for binary32 units the binary32 pipe carries the body and the map, the
    binary64 pipe the reduction).  achieved = algorithmic flops per pass / pass time on
    the binding pipe; the other pipe's utilisation and the binary64 FMA-slot occupancy
    are reported beside it."""
    costs, costs32 = op_costs(peaks), op_costs32(peaks)
    prec = {}
    if res is not None:
        for d in res.per_unit:
            prec[d["unit"]] = d["precision"]
    f64 = f32 = slots64 = 0.0
    for k, u in enumerate(prep.units):
        if prec.get(k, "fp64") == "fp32":
            _, _, body = unit_work(u.program, costs32, u.dim, u.n_out)
            f32 += body + 4 * u.dim
            f64 += 3 * u.n_out
            slots64 += 3 * u.n_out
        else:
            fl, sl, _ = unit_work(u.program, costs, u.dim, u.n_out)
            f64 += fl
            slots64 += sl
    f64, f32, slots64 = f64 * pts, f32 * pts, slots64 * pts
    t64 = f64 / (peaks[0] * 1e12)
    t32 = f32 / (peaks[3] * 1e12)
    fp64_bound = t64 >= t32
    achieved = (f64 if fp64_bound else f32) / pass_s * 1e-12
    peak = peaks[0] if fp64_bound else peaks[3]
    key = (args.workload, args.precision, bool(args.fuse))
    traffic = TRAFFIC.get(key)
    return {"bound": "alu", "pipe": "fp64" if fp64_bound else "fp32", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic[0] if traffic else None, "traffic_source": traffic[1] if traffic else None,
            "kernel": "k_eval",
            "work": "flops per evaluation pass: add/sub/mul 1, fma 2, log/div/atan2 at their measured cost in "
                    "FMA slots x 2, map 4 per coordinate, reduction 3 per result",
            "peak_source": "measured in-process (fiesta_probe_peaks): binary64 / binary32 FMA rate",
            "nominal_fp64_tflops": 1.25,
            "pipes": {"fp64": {"tflop_per_pass": f64 * 1e-12, "utilisation": t64 / pass_s},
                      "fp32": {"tflop_per_pass": f32 * 1e-12, "utilisation": t32 / pass_s}},
            "fma_slot_occupancy": 2.0 * slots64 / pass_s / (peaks[0] * 1e12),
            "eval_ms_per_pass": pass_s * 1e3,
            "eval_launches_per_pass": res.stats["eval_launches"] // max(iters, 1) if res else None,
            "peaks_measured": {"fp64_tflops": peaks[0], "fp64_log_cuda_gps": peaks[1], "fp64_div_gps": peaks[2],
                               "fp32_tflops": peaks[3], "fp32_log_gps": peaks[4], "fp32_div_gps": peaks[5],
                               "fp64_log_table_gps": peaks[6], "fp64_atan2_gps": peaks[7],
                               "fp64_recip_gps": peaks[8]},
            "op_costs_fma_slots": {"fp64": costs, "fp32": costs32}}


def run_ours(args):
    import numpy as np
    import torch
    from paper_1511_03614_gb300 import Integrator, _native as N
    import ctypes as C

    rank, world, local = dist_setup(args)
    torch.cuda.set_device(local)
    pts, iters, rng = WORKLOADS[args.workload]
    pts = args.points or pts
    iters = args.iters or iters
    prep = prepared(args.workload, args.fuse)
    lib = N.load()
    peaks = (C.c_double * 9)()
    N.check(lib.fiesta_probe_peaks(peaks, 9))
    peaks = list(peaks)
    integ = Integrator(prep)
    # replicas: every rank integrates every unit with its own point streams (weak scaling)
    # one iteration per step refines the grid after it (adapt=2), so every step runs
    # every row of the path: points, map, evaluation, reduction, refinement, assembly
    kw = dict(n_iter=iters, points=pts, seed=1 + rank, rng=rng, precision=args.precision,
              adapt=2 if iters == 1 else True)
    if args.launch_shape:               # pin the autotuner's choice (e.g. for a profiler run)
        t, q, w = (int(v) for v in args.launch_shape.split(","))
        kw.update(threads=t, points_per_thread=q, wide_threads=w)
    for _ in range(args.warmup):
        integ.integrate(**kw)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2
    clocks = Clocks(local)
    stream = integ.stream
    times, eval_ms, launches, eval_iters, points = [], 0.0, 0, 0, 0
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    res = None
    for s in range(args.steps):
        flush.fill_(float(s))                          # evict L2 between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = integ.integrate(**kw)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        eval_ms += res.stats["eval_ms"]
        launches += res.stats["kernels_launched"]
        eval_iters += iters             # one evaluation pass (all its launches) per iteration
        points += res.stats["unit_points"]          # evaluations of (sector, order) integrands
    torch.cuda.synchronize()
    barrier(world)
    ck = clocks.stop()
    total_ms = sum(times)
    t_max = max_over_ranks(total_ms, world)
    all_points = sum_over_ranks(points, world)
    value = all_points / (t_max * 1e-3)

    # roofline of the evaluation kernel (dominant): algorithmic work per evaluation pass
    # (one pass per iteration) over the pass's mean CUDA-event duration
    roofline = roofline_of(prep, res, peaks, pts, eval_ms / max(eval_iters, 1) * 1e-3, args, iters)

    # end to end through the public API with host buffers: upload programs, integrate,
    # read the per-order results back; the copies are inside the timed region.
    e2e = None
    if not args.no_e2e:
        h2d = sum(u.program.code.nbytes + u.program.consts.nbytes for u in prep.units) + 64 * len(prep.units)
        d2h = 16 * len(prep.units) * iters + 8 * len(prep.units)
        e_times = []
        e_points = 0
        for s in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ig = Integrator(prep)
            r = ig.integrate(**kw)
            _ = [r.assembled[n] for n in r.assembled] if r.assembled else None
            ig.close()
            torch.cuda.synchronize()
            e_times.append(time.perf_counter() - t0)
            e_points += r.stats["unit_points"]
        et = max_over_ranks(sum(e_times), world)
        e2e = {"value": sum_over_ranks(e_points, world) / et, "unit": "points/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    cpu = onp = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        units = _oracle_units(args.workload)
        cpu = cpu_baseline(args.workload, 12.0, units)
        onp = oracle_numpy_rate(args.workload, 6.0, units)

    # the metric's second part, measured live on the same GPU after the timed region:
    # GPU-seconds to 1e-4 relative error on every eps order, plain binary64 Vegas against
    # the faster forms (randomised QMC, per-unit binary32 with allocation, cubature)
    tta = None
    if rank == 0 and world == 1 and not args.no_tta and args.workload in ("box", "bubble", "box_physical",
                                                                         "double_box"):
        tta = time_to_accuracy(args.workload, 1e-4)
        base = tta.get("fp64_vegas", {})
        if cpu and base.get("points") and cpu.get("value"):
            # the compiled CPU baseline at the same points and Vegas spec: the plain binary64
            # run's point count (scaled to the target when it was capped) at the CPU's rate
            need = base["points"] * (1.0 if base.get("converged") else base.get("error_over_target", 1.0) ** 2)
            cpu["time_to_1e-4_s"] = need / cpu["value"]
            cpu["time_to_1e-4_basis"] = ("points of the GPU's plain binary64 Vegas run"
                                         + ("" if base.get("converged") else ", extrapolated to the target")
                                         + " at the measured CPU rate")

    if rank == 0:
        line = {
            "metric": "sampling points/s", "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32 body, f64 map/sums/grid",
                      "auto": "per unit f32 or f64 body, f64 map/sums/grid"}[args.precision],
            "data": "synthetic",
            "config": {"workload": {"box": "one-loop massless box s=-1 t=-2, eps^-2..eps^0, 12 sectors x 3 dims "
                                           "(32 units), Vegas 10 it x 1e6 Philox points per unit",
                                    "bubble": "one-loop massless bubble p^2=-1 to eps^2, 8 units, 10 x 1e5",
                                    "box_physical": "one-loop massless box at the physical point s=3 t=-1 (F changes "
                                                    "sign): contour deformation, complex results, eps^-2..eps^0, "
                                                    "12 sectors x 3 dims, Vegas 10 it x 1e6 Philox points per unit",
                                    "double_box": "two-loop massless planar double box s=t=-1, eps^-4..eps^0, "
                                                  "293 sectors x 6 dims (1141 sector-order integrands), Vegas 1 it "
                                                  "x 1e7 Philox points per sector per step, grid refined after it "
                                                  "(20 steps: 2e8 points per sector)",
                                    "stress": ("10000 seeded synthetic integrands, dims 3..8, "
                                               + ("each expanded to eps^0..eps^2 (one unit per coefficient), "
                                                  if STRESS_ALL_ORDERS else "one eps coefficient each, ")
                                               + "2^20 Sobol points per unit")
                                    }[args.workload],
                       "units": len(prep.units), "points_per_unit_per_iter": pts, "iterations": iters,
                       "fused_orders": bool(args.fuse) and args.workload != "stress",
                       "results_per_point": sum(u.n_out for u in prep.units) / len(prep.units),
                       "units_fp32": res.stats.get("units_fp32") if res else None,
                       "launch_shape": {"threads": res.stats.get("threads"),
                                        "points_per_thread": res.stats.get("points_per_thread"),
                                        "wide_threads": res.stats.get("wide_threads"),
                                        "wide_points_per_thread": res.stats.get("wide_points_per_thread"),
                                        "eval_groups": res.stats.get("eval_groups")} if res else None,
                       "precision": args.precision, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MB write)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "oracle_numpy": onp,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": ck,
            "results": {str(n): [_num(res.assembled[n]), _num(res.assembled_errors[n])] for n in res.assembled}
            if res and res.assembled else None,
            "time_to_1e-4": tta,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def time_to_accuracy(workload, target, cap_s=15.0):
    """GPU-seconds (the library's device time) to `target` relative error on every eps
    order: plain binary64 Vegas (one unit per sector and order) against the faster forms.
    Box-sized workloads: randomised QMC on the adapted grids, AUTO precision with point
    allocation, and the cubature (fused units).  Double box: randomised QMC, AUTO with
    allocation and the learned flow (fused units, binary32 body); forms that do not
    converge within ``cap_s`` GPU-seconds report the device time spent, the worst
    error/target ratio and an extrapolation gpu_s * ratio^2 (errors fall as the inverse
    square root of the points once the grids have settled), labelled as such.  Errors
    are reported, not raised: this is an addition to the line."""
    from paper_1511_03614_gb300 import Integrator
    from paper_1511_03614_gb300.api import run_to_accuracy, run_to_accuracy_rqmc, run_cuhre_to_accuracy, run_flow
    out = {"target": target, "unit": "GPU-s", "workload": workload}
    if workload == "double_box":
        cap = dict(max_gpu_s=cap_s)
        runs = (("fp64_vegas", False, lambda ig: run_to_accuracy(ig, target=target, points=2_000_000,
                                                                 max_iters=400, **cap)),
                ("rqmc_fp64", True, lambda ig: run_to_accuracy_rqmc(ig, target=target, points=1 << 18,
                                                                    max_points=1 << 22)),
                ("rqmc_fp64_terms", "terms", lambda ig: run_to_accuracy_rqmc(ig, target=target, points=1 << 18,
                                                                             max_points=1 << 22)),
                ("auto_alloc", False, lambda ig: run_to_accuracy(ig, target=target, points=2_000_000,
                                                                 max_iters=400, precision="auto", allocate=True,
                                                                 **cap)),
                ("flow_fp32", True, lambda ig: run_flow(ig, target=target, points=2_000_000, keep=4096,
                                                        train_rounds=8, steps_per_round=20, max_rounds=300,
                                                        precision="fp32", **cap)))
    else:
        runs = (("fp64_vegas", False, lambda ig: run_to_accuracy(ig, target=target, points=1_000_000,
                                                                 max_iters=200)),
                ("rqmc_fp64", True, lambda ig: run_to_accuracy_rqmc(ig, target=target, points=1 << 18,
                                                                    max_points=1 << 22)),
                ("auto_alloc", False, lambda ig: run_to_accuracy(ig, target=target, points=1_000_000,
                                                                 max_iters=200, precision="auto", allocate=True)),
                ("cuhre_fp64", True, lambda ig: run_cuhre_to_accuracy(ig, target=target)))
    for name, fuse, fn in runs:
        try:
            t0 = time.perf_counter()
            ig = Integrator(prepared(workload, fuse=bool(fuse), terms=fuse == "terms"))
            r = fn(ig)
            rec = {"gpu_s": r["gpu_s"], "converged": r["converged"], "wall_s": time.perf_counter() - t0,
                   "points": r.get("points")}
            if not r["converged"] and r.get("ratio"):
                rec["error_over_target"] = r["ratio"]
                rec["extrapolated_gpu_s"] = r["gpu_s"] * r["ratio"] ** 2
            rec["values"] = {str(n): [_num(r["values"][n]), _num(r["errors"][n])] for n in r["values"]}
            out[name] = rec
            ig.close()
        except Exception as e:          # noqa: BLE001 - reported in the line instead
            out[name] = {"error": str(e)[:200]}
    base = out.get("fp64_vegas", {})
    base_s = base.get("gpu_s") if base.get("converged") else base.get("extrapolated_gpu_s")
    out["speedup_vs_fp64_vegas"] = {k: base_s / v["gpu_s"] for k, v in out.items()
                                    if isinstance(v, dict) and v.get("converged") and base_s and k != "fp64_vegas"}
    if base_s and not base.get("converged"):
        out["speedup_basis"] = "fp64_vegas extrapolated from its capped run"
    return out


def _oracle_lam(workload):
    """Contour-deformation parameter for the oracle's physical-point workloads (the
    value the preprocessor picks for every sector of the physical box)."""
    return 1.0 if workload == "box_physical" else None


def _real_f(unit):
    """The oracle unit's integrand as a real function for the timing loop: a complex
    unit is evaluated in full and its real part sampled."""
    if getattr(unit, "complex", False):
        import numpy as np
        return lambda X: np.real(unit.f_numpy(X))
    return unit.f_numpy


def _oracle_units(workload, n_stress=200):
    import workloads as W
    from oracle import pipeline as P
    if workload == "stress":
        return [P.direct_problem(p).units[0] for p in W.stress_suite(n_stress)]
    return P.feynman_problem(getattr(W, workload)(), lam=_oracle_lam(workload)).units


def cpu_baseline(workload, budget_s, units=None):
    """The timed CPU baseline: per-unit straight-line C++ generated from the oracle's
    expression trees (oracle/cbaseline.py), g++ -O3 (-mcpu=native on aarch64), OpenMP
    over units on every host core, binary64, the same Philox points and Vegas spec
    (map, v^2 histogram, refinement), on a bounded sample of the workload's units and
    points.  Complex (deformed-contour) units are left out: the generated code is real."""
    import numpy as np
    from oracle.cbaseline import Baseline, cpu_model
    units = units if units is not None else _oracle_units(workload)
    units = [u for u in units if not getattr(u, "complex", False)]
    if not units:
        return None
    step = max(1, len(units) // 96)
    sample = units[::step]
    b = Baseline(sample)
    n = 2000
    while True:                       # calibrate: grow the sample until a pass takes >= 0.5 s
        t0 = time.perf_counter()
        b.iterate(n, seed=1, iteration=0)
        dt = time.perf_counter() - t0
        if dt >= 0.5 or n >= 1 << 22:
            break
        n *= 4
    b.refine()
    n = int(min(max(n * budget_s / max(dt, 1e-6), 4096), 1 << 24))
    t0 = time.perf_counter()
    b.iterate(n, seed=1, iteration=1)
    b.refine()
    dt = time.perf_counter() - t0
    return {"value": n * len(sample) / dt, "unit": "points/s", "cores": b.threads, "kind": "compiled",
            "sample": f"{len(sample)} of {len(units)} {workload} sector-order integrands (every {step}th), one "
                      f"Vegas iteration of {n} Philox points each with refinement; C++ generated from the oracle's "
                      f"expression trees, binary64, OpenMP over units",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(), "compile_s": b.compile_s,
            "flags": " ".join(__import__("oracle.cbaseline", fromlist=["compile_flags"]).compile_flags())}


def oracle_numpy_rate(workload, budget_s, units=None):
    """The oracle as it stands (numpy float64, one thread) on a bounded sample."""
    from oracle import vegas as V
    units = units if units is not None else _oracle_units(workload)
    n = 20000
    done = 0
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < budget_s and k < 10 * len(units):
        u = units[k % len(units)]
        V.integrate_unit(_real_f(u), u.dim, 1, n, 1, k % len(units), rng="philox" if workload != "stress" else "sobol")
        done += n
        k += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} unit-iterations x {n} points of the {workload} units (numpy float64, one thread)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import workloads as W
    from oracle import pipeline as P, vegas as V
    pts, iters, rng = WORKLOADS[args.workload]
    if args.workload == "stress":
        units = [P.direct_problem(p).units[0] for p in W.stress_suite(100)]
    else:
        units = P.feynman_problem(getattr(W, args.workload)(), lam=_oracle_lam(args.workload)).units
    n = 20000
    for _ in range(args.warmup):
        V.integrate_unit(_real_f(units[0]), units[0].dim, 1, 2000, 1, 0, rng=rng)
    times = []
    done = 0
    for s in range(args.steps):
        t0 = time.perf_counter()
        for k, u in enumerate(units[:32]):
            V.integrate_unit(_real_f(u), u.dim, 1, n, 1 + s, k, rng=rng)
            done += n
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = done / total
    line = {"impl": "reference", "metric": "sampling points/s", "value": value, "unit": "points/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": f"{min(32, len(units))} units x {n} points per step"},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                             "sample": f"{min(32, len(units))} units x {n} Philox/Sobol points per step, one Vegas "
                                       "iteration each (numpy float64)"},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


class _Skip(Exception):
    """A tta form left out by --forms."""


def _num(z):
    """A JSON-able number: complex values as [re, im]."""
    return [z.real, z.imag] if isinstance(z, complex) else z


def run_tta(args):
    """GPU-seconds to the target relative error per eps order: plain binary64 Vegas
    against the per-unit mixed precision policy, binary32, variance-driven point
    allocation across units (*_alloc), binary64 for the points near the boundary of
    binary32 units (*_mixed: small_x32 = 1e-2), randomised quasi-Monte Carlo on the adapted
    grids (rqmc_*), the learned flow and the cubature."""
    import torch
    from paper_1511_03614_gb300 import Integrator
    from paper_1511_03614_gb300.api import run_to_accuracy
    torch.cuda.set_device(0)
    pts = args.points or {"box": 1_000_000, "double_box": 2_000_000, "bubble": 200_000}.get(args.workload, 1_000_000)
    prep = prepared(args.workload)
    out = {"mode": "tta", "workload": args.workload, "target": args.target, "points_per_unit_per_iter": pts,
           "units": len(prep.units), "runs": {}}
    from paper_1511_03614_gb300._native import FiestaError
    forms = set(args.forms.split(","))
    for form in ("fp64", "auto", "fp32", "fp64_alloc", "auto_alloc", "fp32_alloc", "auto_mixed",
                 "auto_mixed_alloc"):
        if form not in forms:
            continue
        prec = form.split("_")[0]
        integ = Integrator(prep)
        try:
            integ.integrate(n_iter=1, points=min(pts, 100_000), precision=prec)      # warm-up and autotuning
            sx = 1e-2 if "_mixed" in form else (None if args.small_x32 < 0 else args.small_x32)
            r = run_to_accuracy(integ, target=args.target, points=pts, precision=prec, max_iters=args.max_iters,
                                allocate=form.endswith("_alloc"), small_x32=sx, max_gpu_s=args.cap_s or None)
        except FiestaError as e:
            out["runs"][form] = {"error": str(e)}
            integ.close()
            continue
        out["runs"][form] = {"gpu_s": r["gpu_s"], "points": r["points"], "iterations": r["iterations"],
                             "converged": r["converged"], "error_over_target": r.get("ratio"),
                             "values": {str(n): [_num(r["values"][n]), _num(r["errors"][n])] for n in r["values"]}}
        integ.close()
    # learned proposal: flow sampling with training rounds, binary32 integrand
    from paper_1511_03614_gb300.api import run_flow
    integ = Integrator(prepared(args.workload, fuse=True))       # one flow per sector, all orders
    try:
        if "flow_fp32" not in forms:
            raise _Skip()
        r = run_flow(integ, target=args.target, points=pts, keep=4096, train_rounds=8, steps_per_round=20,
                     max_rounds=300, precision="fp32")
        out["runs"]["flow_fp32"] = {"gpu_s": r["gpu_s"], "points": r["points"], "rounds": r["rounds"],
                                    "converged": r["converged"],
                                    "values": {str(n): [_num(r["values"][n]), _num(r["errors"][n])] for n in r["values"]}}
    except FiestaError as e:
        out["runs"]["flow_fp32"] = {"error": str(e)}
    except _Skip:
        pass
    integ.close()
    # randomised quasi-Monte Carlo on adapted Vegas grids (Sobol replicates), fused units
    from paper_1511_03614_gb300.api import run_to_accuracy_rqmc
    for form in ("rqmc_fp64", "rqmc_fp64_mix4", "rqmc_fp64_terms"):
        if form not in forms:
            continue
        # *_mix4: four sectors of equal dimension summed into one program (MixSectors);
        # *_terms: every separately integrable term its own unit (SeparateTerms)
        integ = Integrator(prepared(args.workload, fuse=True, mix=4 if form.endswith("mix4") else 1,
                                    terms=form.endswith("terms")))
        try:
            prec = form.split("_")[1]
            integ.integrate(n_iter=1, points=min(pts, 100_000), precision=prec)      # warm-up and autotuning
            r = run_to_accuracy_rqmc(integ, target=args.target, points=1 << 18, precision=prec, max_points=1 << 22)
            out["runs"][form] = {"gpu_s": r["gpu_s"], "points": r["points"], "rounds": r["rounds"],
                                 "points_per_replicate": r["points_per_replicate"], "converged": r["converged"],
                                 "values": {str(n): [_num(r["values"][n]), _num(r["errors"][n])]
                                            for n in r["values"]}}
        except FiestaError as e:
            out["runs"][form] = {"error": str(e)}
        integ.close()
    # deterministic cubature (Genz-Malik rule, binary64), its error bound against the target
    from paper_1511_03614_gb300.api import run_cuhre_to_accuracy
    integ = Integrator(prepared(args.workload, fuse=True))
    try:
        if "cuhre_fp64" not in forms:
            raise _Skip()
        integ.cuhre(rel_tol=1e-2, max_passes=2)                                   # warm-up
        r = run_cuhre_to_accuracy(integ, target=args.target)
        out["runs"]["cuhre_fp64"] = {"gpu_s": r["gpu_s"], "points": r["points"], "rounds": r["rounds"],
                                     "rel_tol": r["rel_tol"], "converged": r["converged"],
                                     "values": {str(n): [_num(r["values"][n]), _num(r["errors"][n])]
                                                for n in r["values"]}}
    except FiestaError as e:
        out["runs"]["cuhre_fp64"] = {"error": str(e)}
    except _Skip:
        pass
    integ.close()
    base = out["runs"].get("fp64", {}).get("gpu_s")
    out["speedup_vs_fp64"] = {k: base / v["gpu_s"] for k, v in out["runs"].items() if base and "gpu_s" in v}
    print(json.dumps(out))


def run_cuhre(args):
    """Throughput of the adaptive cubature: one fiesta_cuhre call per step on the fused
    units of the workload at relative tolerance --target, reported as integrand
    evaluations per second (a fused unit's evaluation yields all its orders), with the
    evaluation kernels' share of the device time.  Not the headline line."""
    import torch
    from paper_1511_03614_gb300 import Integrator
    torch.cuda.set_device(0)
    prep = prepared(args.workload, fuse=True)
    integ = Integrator(prep)
    for _ in range(args.warmup):
        integ.cuhre(rel_tol=args.target)
    gpu_ms = eval_ms = 0.0
    pts = 0
    res = None
    for _ in range(args.steps):
        res = integ.cuhre(rel_tol=args.target)
        gpu_ms += res.stats["gpu_ms"]
        eval_ms += res.stats["eval_ms"]
        pts += res.stats["points"]
    print(json.dumps({"mode": "cuhre", "workload": args.workload, "rel_tol": args.target, "steps": args.steps,
                      "evaluations_per_s": pts / (gpu_ms * 1e-3), "eval_kernel_share": eval_ms / gpu_ms,
                      "gpu_ms_per_step": gpu_ms / args.steps, "evaluations_per_step": pts // args.steps,
                      "regions": sum({d["unit"]: d["n_regions"] for d in res.per_unit}.values()),
                      "converged_units": sum(d["converged"] for d in res.per_unit),
                      "results": {str(n): [_num(res.assembled[n]), _num(res.assembled_errors[n])]
                                  for n in res.assembled}}))


def run_kernel(args):
    """Two evaluation passes at a fixed launch shape (no autotuner, no graph): the second
    is the launch a profiler captures with -k regex:k_eval -s 1 -c 1.  Prints the pass's
    device time and rate.  Not a bench line."""
    import torch
    import workloads as W
    from paper_1511_03614_gb300 import Integrator, prepare_direct
    torch.cuda.set_device(0)
    if args.workload == "stress":
        prep = prepare_direct(W.stress_suite(args.units or 10_000), "stress")
        rng = "sobol"
    else:
        prep = prepared(args.workload, args.fuse)
        rng = "philox"
    if args.max_slots or args.min_slots:
        import dataclasses
        hi = args.max_slots or 1 << 30
        prep = dataclasses.replace(prep, units=[u for u in prep.units if args.min_slots <= u.program.n_slots <= hi])
    pts = args.points or 200_000
    ig = Integrator(prep)
    for s in range(2):
        r = ig.integrate(n_iter=1, points=pts, seed=1 + s, rng=rng, adapt=2, threads=args.threads,
                         points_per_thread=args.ppt, precision=args.precision, graph=False,
                         wide_threads=args.wide_threads,
                         accumulate="registers" if args.workload != "stress" else "auto")
    print(json.dumps({"mode": "kernel", "workload": args.workload, "precision": args.precision, "points": pts,
                      "units": len(prep.units), "threads": args.threads, "ppt": args.ppt,
                      "wide_threads": args.wide_threads, "eval_groups": r.stats["eval_groups"],
                      "eval_ms": r.stats["eval_ms"],
                      "unit_points_per_s": r.stats["unit_points"] / (r.stats["eval_ms"] * 1e-3)}))


# multiply-adds of one training point (4 coupling layers, MLP 16 -> 64 -> 64 -> 16): the
# forward pass, the reverse pass's recomputation, the three reverse products
# (dH2 = dout W3^T, dH1 = dH2 W2^T, d(input) = dH1 W1^T) and the three weight-gradient
# products (dW3 = H2^T dout, dW2 = H1^T dH2, dW1 = In^T dH1)
FLOW_LAYER_MACS = 16 * 64 + 64 * 64 + 64 * 16
FLOW_TRAIN_FLOPS_PER_POINT = 2 * 4 * (1 + 1 + 1 + 1) * FLOW_LAYER_MACS     # 196 608


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops (cuBLAS, burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s bf16"


def run_flow_kernels(args):
    """The learned proposal's kernels on the workload's fused units (one flow per
    sector): per step one sampling pass of --points points per sector that keeps 4096
    training points per sector, then 20 Adam steps of tensor-core training on them.
    Reports device time per pass and per training step, and the training kernel's
    tensor roofline (algorithmic BF16 flops of the MLP products over the measured
    cuBLAS BF16 peak).  Not the headline line."""
    import torch
    from paper_1511_03614_gb300 import Integrator
    torch.cuda.set_device(0)
    prep = prepared(args.workload, fuse=True)
    integ = Integrator(prep)
    integ.flow_init(seed=3)
    pts, keep, tsteps = args.points or 200_000, 4096, 20
    sample_ms, train_ms = [], []
    for s in range(args.warmup + args.steps):
        _, _, st = integ.flow_sample(pts, seed=1, iteration=s, keep=keep)
        _, tt = integ.flow_train(tsteps, lr=2e-3, power=1)
        if s >= args.warmup:
            sample_ms.append(st["gpu_ms"])
            train_ms.append(tt["gpu_ms"])
    nu = len(prep.units)
    step_s = statistics.median(train_ms) * 1e-3 / tsteps
    achieved = nu * keep * FLOW_TRAIN_FLOPS_PER_POINT / step_s * 1e-12
    peak, src = _bf16_peak()
    print(json.dumps({"mode": "flow", "workload": args.workload, "units": nu, "points_per_unit": pts,
                      "keep_per_unit": keep, "sample_ms_per_pass": statistics.median(sample_ms),
                      "sample_points_per_s": nu * pts / (statistics.median(sample_ms) * 1e-3),
                      "train_ms_per_adam_step": step_s * 1e3,
                      "train_roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                         "frac": achieved / peak, "peak_source": src,
                                         "work": f"{FLOW_TRAIN_FLOPS_PER_POINT} BF16 flops per training point"}}))


def main():
    global STRESS_ALL_ORDERS
    args = parse()
    STRESS_ALL_ORDERS = args.stress_orders == "all"
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "kernel":
        run_kernel(args)
    elif args.mode == "tta":
        run_tta(args)
    elif args.mode == "cuhre":
        run_cuhre(args)
    elif args.mode == "flow":
        run_flow_kernels(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
