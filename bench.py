#!/usr/bin/env python
"""Benchmark of the pCT simulator hot path on GB300.

One step = one whole simulation of the workload: phantom raster (x_true),
per-proton path + traversal count, int64 row-pointer scan, nnz read-back,
and the fill of col / val / b (WEPL with noise), all through the C ABI.

Metric: proton paths per second (whole job), with the CSR bytes per second
and the fill kernel's achieved HBM bandwidth against the measured peak.

  python bench.py [--gpus N --steps K --warmup W] [--precision mixed|f64]
                  [--impl ours|reference] [--workload head_3d_spline]

The default workload is the 3D head: 200x200x160 voxels of 1 mm, 90 angles x
200,000 cubic-spline paths with MCS draws, 1 % WEPL noise (18M rows).  After
the timed loop the line also carries the all-FP64 form's step time on the
same workload (the mixed form's speedup) and the max / RMS errors of A and b
against the CPU oracle on a row sample, for both forms.

Under torchrun (N > 1) the ranks split one acquisition into contiguous angle
blocks (Sec. IV), each block keyed by its global first row so that the blocks
are exactly the rows of the single-GPU run: strong scaling, no collective on
the data path (one all-gather of the blocks' nonzero counts places them in
the global CSR).  `--impl reference` times the CPU oracle on a bounded sample
of the same workload (rank 0 only).
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
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2108_12369_gb300 import workloads as W  # noqa: E402

METRIC = "proton paths/s (CSR generation, whole job)"
UNIT = "paths/s"
KERNEL_FILES = {
    "mixed": ["pct_mixed.cu", "pct_mixed.cuh", "pct_coop.cuh", "pct_walk.cuh", "pct_device.cuh"],
    "f64": ["pct_f64.cu", "pct_device.cuh"],
}
FILL_KERNEL = {"mixed": "k_fill_mixed", "f64": "k_fill_f64"}
# angles per block of the end-to-end leg's pct_simulate_host (9 blocks of the 3D head)
E2E_ANGLES_PER_BLOCK = 10
# our kernels launched per step: raster, path set-up + lead segments + count (mixed) or count (f64), 3 scan passes, fill
LAUNCHES_PER_STEP = {"mixed": 8, "f64": 6}


def workload(name: str, angles: int = 0, paths_per_angle: int = 0):
    """The named workload; angles / paths_per_angle > 0 shrink it (profiling)."""
    w = {"neo2_2d_spline": W.neo2_2d_spline, "neo1_2d_straight": W.neo1_2d_straight,
         "head_3d_spline": W.head_3d_spline}[name]()
    if angles > 0:
        w["angles"] = W.angles(angles)
    if paths_per_angle > 0:
        w["paths_per_angle"] = paths_per_angle
    return w


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_hash(prec: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_FILES[prec]:
        fp = ROOT / "paper_2108_12369_gb300" / "csrc" / f
        if fp.exists():
            h.update(fp.read_bytes())
    return h.hexdigest()[:16]


def recorded_traffic(prec: str, wname: str):
    """DRAM bytes per fill launch from a committed ncu summary, if it was
    taken on the current kernel source; else None."""
    p = ROOT / "profiles" / f"{FILL_KERNEL[prec]}_{wname}.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text())
    if d.get("kernel_hash") != kernel_hash(prec):
        return None
    return d.get("traffic_bytes_per_launch")


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in Path(self.path).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(w, target_s: float = 15.0):
    """The oracle as it stands, all host cores, on a stride sample of the rows."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    n_rows = W.n_rows(w)
    ph = O.Phantom(w["phantom"])
    t0 = time.perf_counter()
    x = ph.raster().astype(np.float32)
    t_raster = time.perf_counter() - t0
    sim = O.Simulation(ph, x, w["angles"], w["paths_per_angle"], w["model"], w["seed"])
    # calibrate on a small sample, then size the timed one to ~target_s
    probe = np.arange(0, n_rows, max(1, n_rows // 2000), dtype=np.int64)
    t0 = time.perf_counter()
    sim.rows(probe, threads=cores)
    rate = len(probe) / max(time.perf_counter() - t0, 1e-6)
    n_s = int(min(n_rows, max(len(probe), rate * target_s)))
    rows = np.linspace(0, n_rows - 1, n_s).astype(np.int64)
    t0 = time.perf_counter()
    rp, _, _, _, _ = sim.rows(rows, threads=cores)
    t_rows = time.perf_counter() - t0
    frac = n_s / n_rows
    t_total = t_rows + t_raster * frac  # raster prorated to the sample
    return {"value": n_s / t_total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_s} of {n_rows} rows (even stride) + full raster prorated; "
                      f"{int(rp[-1])} nonzeros in {t_total:.1f} s",
            "nnz_per_s": float(rp[-1]) / t_total}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload, args.angles, args.paths_per_angle)
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    n_rows = W.n_rows(w)
    ph = O.Phantom(w["phantom"])
    per_step = max(1000, int(args.reference_rows))
    times = []
    nnz = 0
    for s in range(args.warmup + args.steps):
        rows = (np.arange(per_step, dtype=np.int64) * (n_rows // per_step) + s) % n_rows
        t0 = time.perf_counter()
        x = ph.raster().astype(np.float32)
        t_r = time.perf_counter() - t0
        sim = O.Simulation(ph, x, w["angles"], w["paths_per_angle"], w["model"], w["seed"])
        t0 = time.perf_counter()
        rp, _, _, _, _ = sim.rows(rows, threads=cores)
        t = time.perf_counter() - t0 + t_r * per_step / n_rows
        if s >= args.warmup:
            times.append(t)
            nnz += int(rp[-1])
    total = sum(times)
    value = per_step * args.steps / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w["name"], "rows": n_rows, "grid": list(w["phantom"]["n"][:w["phantom"]["dim"]]),
                       "sample_rows_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} of {n_rows} rows per step (even stride), raster prorated"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "nnz_per_s": nnz / total}
    print(json.dumps(line), flush=True)


def accuracy(w, rows, rp_dev, col_dev, val_dev, b_dev, x_max, threads):
    """Max / RMS error of A's values and of b against the oracle on the given
    global rows (the comparison rule of the parity tests): indices must match
    exactly, value errors relative to the row sum, b errors relative to
    max(|b|, row sum x max RSP).  rp_dev etc. hold the rows first_row + i."""
    import torch
    from oracle import oracle as O
    first = int(w.get("first_row", 0))
    loc = torch.as_tensor(rows - first, dtype=torch.int64, device=rp_dev.device)
    r0, r1 = rp_dev[loc], rp_dev[loc + 1]
    lens = (r1 - r0).cpu().numpy()
    idx = torch.repeat_interleave(r0, r1 - r0) + (
        torch.arange(int(lens.sum()), device=rp_dev.device) -
        torch.repeat_interleave(torch.cumsum(r1 - r0, 0) - (r1 - r0), r1 - r0))
    col_g = col_dev[idx].cpu().numpy()
    val_g = val_dev[idx].cpu().numpy().astype(np.float64)
    b_g = b_dev[loc].cpu().numpy().astype(np.float64)
    ph = O.Phantom(w["phantom"])
    x = ph.raster().astype(np.float32)
    full_angles = w.get("all_angles", w["angles"])
    sim = O.Simulation(ph, x, full_angles, w["paths_per_angle"], w["model"], w["seed"])
    rp_o, col_o, val_o, _, b_o = sim.rows(rows, threads=threads)
    ok_idx = bool(np.array_equal(np.diff(rp_o), lens) and np.array_equal(col_o, col_g))
    out = {"rows": int(len(rows)), "nnz": int(len(col_o)), "indices_exact": ok_idx}
    if ok_idx and len(col_o):
        rid = np.repeat(np.arange(len(rows)), np.diff(rp_o))
        rowsum = np.bincount(rid, weights=val_o, minlength=len(rows))
        aerr = np.abs(val_g - val_o)
        berr = np.abs(b_g - b_o)
        scale = np.maximum(np.abs(b_o), rowsum * float(x_max))
        out.update(val_max_rel=float((aerr / np.maximum(rowsum[rid], 1e-30)).max()),
                   val_rms_abs=float(np.sqrt(np.mean(aerr ** 2))), val_max_abs=float(aerr.max()),
                   b_max_rel=float((berr / np.maximum(scale, 1e-30)).max()),
                   b_rms_abs=float(np.sqrt(np.mean(berr ** 2))))
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2108_12369_gb300 import build as B, pct, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    prec = {"mixed": pct.PREC_MIXED, "f64": pct.PREC_F64}[args.precision]
    w_all = workload(args.workload, args.angles, args.paths_per_angle)
    # one acquisition split into contiguous angle blocks, one per rank (Sec. IV)
    w = shard.shard_workload(w_all, rank, world)
    w["all_angles"] = w_all["angles"]
    ph = pct.Phantom(w["phantom"])
    geo = pct.GeometryArgs(w)
    n_rows = geo.n_rows
    total_rows = W.n_rows(w_all)
    ws = torch.empty(pct.simulate_workspace_size(ph, geo, prec), dtype=torch.uint8, device=dev)
    x = torch.empty(ph.nvox, dtype=torch.float32, device=dev)
    rp = torch.empty(n_rows + 1, dtype=torch.int64, device=dev)
    b = torch.empty(max(n_rows, 1), dtype=torch.float32, device=dev)
    pct.phantom_rasterize(ph, x)
    pct.simulate_count(ph, geo, prec, ws, rp)
    nnz = int(rp[-1].item())
    col = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    val = torch.empty(max(nnz, 1), dtype=torch.float32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def make_step(p, wsp):
        def step(ev=None):
            if ev:
                ev[0].record(stream)
            pct.phantom_rasterize(ph, x)
            pct.simulate_count(ph, geo, p, wsp, rp)
            n = int(rp[-1].item())  # nnz read-back sizes the fill, as a caller must
            if n != nnz:
                raise RuntimeError("nnz changed between steps")
            if ev:
                ev[1].record(stream)
            pct.simulate_fill(ph, geo, p, wsp, rp, x, col, val, b)
            if ev:
                ev[2].record(stream)
        return step

    step = make_step(prec, ws)
    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for s in range(args.steps):
        step(evs[s])
        flush.zero_()  # L2 flush between steps, outside the step's events
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    fill_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_s = sum(step_ms) / 1e3
    nz_off, nnz_total = 0, nnz
    if world > 1:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
        nz_off, nnz_total = shard.nnz_offsets(nnz)  # the blocks' places in the global CSR
    value = total_rows * args.steps / total_s

    # accuracy of this form against the oracle on an even stride sample of
    # this rank's rows (after the timed loop)
    x_max = float(x.max().item())
    sample = None
    acc = {}
    if rank == 0 and args.accuracy_rows > 0 and n_rows > 0:
        first = int(w["first_row"])
        sample = first + np.unique(np.linspace(0, n_rows - 1, min(args.accuracy_rows, n_rows)).astype(np.int64))
        acc[args.precision] = accuracy(w, sample, rp, col, val, b, x_max, os.cpu_count() or 1)

    # the other arithmetic form on the same workload, same buffers: the mixed
    # form's speedup over the all-FP64 form at the accuracy reported
    other = None
    if rank == 0 and world == 1 and args.fp64_steps > 0 and args.precision == "mixed":
        ws64 = torch.empty(pct.simulate_workspace_size(ph, geo, pct.PREC_F64), dtype=torch.uint8, device=dev)
        step64 = make_step(pct.PREC_F64, ws64)
        step64()
        flush.zero_()
        torch.cuda.synchronize()
        ev64 = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.fp64_steps)]
        for s in range(args.fp64_steps):
            step64(ev64[s])
            flush.zero_()
        torch.cuda.synchronize()
        ms64 = statistics.mean(e[0].elapsed_time(e[2]) for e in ev64)
        other = {"fp64_ms_per_step": ms64, "mixed_ms_per_step": 1e3 * total_s / args.steps,
                 "mixed_speedup": ms64 / (1e3 * total_s / args.steps), "fp64_steps": args.fp64_steps,
                 "fp64_fill_ms": statistics.mean(e[1].elapsed_time(e[2]) for e in ev64)}
        if sample is not None:
            acc["f64"] = accuracy(w, sample, rp, col, val, b, x_max, os.cpu_count() or 1)
        del ws64

    # end to end through the C ABI with host buffers: angle / basis tables go
    # up from host memory inside every call; pct_simulate_host counts and
    # fills the acquisition in blocks of E2E_ANGLES_PER_BLOCK angles and
    # writes the row pointers, the CSR and b to pinned host memory every step
    # (through a 1 GB device staging buffer; a block's copies overlap the
    # next block's count and fill)
    small = args.no_e2e
    del col, val  # the host path needs no device CSR
    h_rp = torch.empty(1 if small else n_rows + 1, dtype=torch.int64, pin_memory=True)
    h_col = torch.empty(1 if small else max(nnz, 1), dtype=torch.int32, pin_memory=True)
    h_val = torch.empty(1 if small else max(nnz, 1), dtype=torch.float32, pin_memory=True)
    h_b = torch.empty(1 if small else max(n_rows, 1), dtype=torch.float32, pin_memory=True)
    staging = torch.empty(256 if small else 1 << 30, dtype=torch.uint8, device=dev)
    e2e_steps = 0 if small else max(1, min(args.steps, 5))

    def step_host():
        pct.phantom_rasterize(ph, x)
        got = pct.simulate_host(ph, geo, prec, E2E_ANGLES_PER_BLOCK, ws, x, staging, h_rp, h_col, h_val, h_b)
        if got != nnz:
            raise RuntimeError("nnz changed between steps")

    for _ in range(args.warmup if e2e_steps else 0):
        step_host()  # warm-up (first launches, first writes to the pinned pages), untimed
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(e2e_steps + 1)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ee[0].record(stream)
    for k in range(e2e_steps):
        step_host()
        ee[k + 1].record(stream)
    torch.cuda.synchronize()
    e2e_step_ms = [ee[k].elapsed_time(ee[k + 1]) for k in range(e2e_steps)]
    e2e_s = sum(e2e_step_ms) / 1e3
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = total_rows * e2e_steps / e2e_s if e2e_steps else None
    K = w["model"].get("spline_segments", 1) if w["model"]["model"] == W.SPLINE else 1
    n_blocks = -(-len(w["angles"]) // E2E_ANGLES_PER_BLOCK)
    # per block: its angles' cos / sin, the spline basis in FP64 and double-float
    h2d = len(w["angles"]) * 16 + n_blocks * (K + 1) * 64
    # per block: its row pointers (one more than its rows); all entries and b
    d2h = (n_rows + n_blocks) * 8 + nnz * 8 + n_rows * 4

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = peaks()
    alg_bytes = 8.0 * nnz + 12.0 * n_rows  # col + val per nonzero; row_ptr read + b write per row
    fill_avg_s = statistics.mean(fill_ms) / 1e3
    achieved = alg_bytes / fill_avg_s / 1e9
    traffic = recorded_traffic(args.precision, w["name"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "mixed" else "f64", "precision": args.precision,
        "data": "synthetic",
        "config": {"workload": w["name"], "grid": list(w["phantom"]["n"][:w["phantom"]["dim"]]),
                   "voxel_mm": w["phantom"]["h"][0], "angles": len(w_all["angles"]),
                   "paths_per_angle": w["paths_per_angle"], "rows": total_rows, "rows_rank0": n_rows,
                   "nnz": nnz_total, "nnz_rank0": nnz,
                   "path_model": "spline" if w["model"]["model"] == W.SPLINE else "straight",
                   "spline_segments": K, "noise_rel": w["model"].get("noise_rel", 0.0),
                   "l2": "512 MB write between steps (untimed); outputs per step >> L2",
                   "parallelism": (f"angle blocks of one acquisition over {world} GPUs (global row bases)"
                                   if world > 1 else "one GPU")},
        "csr_gbs": (8.0 * nnz_total + 12.0 * total_rows) * args.steps / total_s / 1e9,
        "nnz_per_s": nnz_total * args.steps / total_s,
        "roofline": {"bound": "hbm", "kernel": FILL_KERNEL[args.precision], "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} hbm_gbs (copy, burst)",
                     "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
                     "fill_ms": statistics.mean(fill_ms)},
        "phase_ms": {"raster_count_scan_readback": statistics.mean(
            [e[0].elapsed_time(e[1]) for e in evs]), "fill": statistics.mean(fill_ms)},
        "wall_s_timed_loop": t_wall,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "api": "pct_phantom_rasterize + pct_simulate_host", "angles_per_block": E2E_ANGLES_PER_BLOCK,
                "steps": e2e_steps, "step_ms": [round(v, 2) for v in e2e_step_ms]},
        "gpu_launches": LAUNCHES_PER_STEP[args.precision] * args.steps,
    }
    if other is not None:
        line["mixed_vs_f64"] = other
    if acc:
        line["accuracy_vs_oracle"] = acc
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w_all, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _timed(fn, reps):
    """Mean device ms of fn() over reps calls (events on the current stream)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_project(args):
    """Projectors (Sec. II, A x = b): matrix-free y = A x and g += A^T r over
    10M-row chunks of the 256x256x160 head workload (100M spline paths),
    and the explicit-CSR forward / adjoint on the NEO-2 CSR."""
    import torch

    from paper_2108_12369_gb300 import build as B, pct
    torch.cuda.set_device(0)
    B.build()
    prec = {"mixed": pct.PREC_MIXED, "f64": pct.PREC_F64}[args.precision]
    peak, peak_kind = peaks()
    out = {"metric": "projector rows/s", "unit": "rows/s", "n_gpus": 1, "precision": args.precision,
           "data": "synthetic", "higher_is_better": True}
    # matrix-free on the large 3D workload
    w = W.head_3d_large()
    ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
    chunk = 10_000_000
    ws = torch.empty(pct.projector_workspace_size(ph, geo, chunk, prec), dtype=torch.uint8, device="cuda")
    x = torch.empty(ph.nvox, dtype=torch.float32, device="cuda")
    pct.phantom_rasterize(ph, x)
    y = torch.empty(chunk, dtype=torch.float32, device="cuda")
    r = torch.ones(chunk, dtype=torch.float32, device="cuda")
    g = torch.zeros(ph.nvox, dtype=torch.float32, device="cuda")
    k = geo.n_rows // chunk  # every chunk: one pass over the whole acquisition
    fwd = lambda: [pct.forward(ph, geo, None, c * chunk, chunk, x, y, ws, precision=prec) for c in range(k)]
    adj = lambda: [pct.adjoint(ph, geo, None, c * chunk, chunk, r, g, ws, precision=prec) for c in range(k)]
    fwd()
    adj()
    f_ms = _timed(fwd, 1) / k
    a_ms = _timed(adj, 1) / k
    out["matrix_free"] = {"workload": "head_3d_large (256x256x160 voxels of 1 mm, 500 angles x 200k spline paths)",
                          "chunk_rows": chunk, "chunks_timed": k, "rows_timed": k * chunk,
                          "forward_ms_per_chunk": f_ms, "adjoint_ms_per_chunk": a_ms,
                          "forward_rows_per_s": chunk / (f_ms / 1e3), "adjoint_rows_per_s": chunk / (a_ms / 1e3)}
    del ws, y, r, g
    # explicit CSR on NEO-2
    w2 = W.neo2_2d_spline()
    ph2, geo2 = pct.Phantom(w2["phantom"]), pct.GeometryArgs(w2)
    sim = pct.simulate(ph2, geo2, prec)
    n, nnz = geo2.n_rows, sim["nnz"]
    x2 = sim["x_true"]
    y2 = torch.empty(n, dtype=torch.float32, device="cuda")
    g2 = torch.zeros(ph2.nvox, dtype=torch.float32, device="cuda")
    r2 = torch.ones(n, dtype=torch.float32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    pct.forward(None, None, sim, 0, n, x2, y2)
    cf, ca = [], []
    for _ in range(k):
        flush.zero_()
        cf.append(_timed(lambda: pct.forward(None, None, sim, 0, n, x2, y2), 1))
        flush.zero_()
        ca.append(_timed(lambda: pct.adjoint(None, None, sim, 0, n, r2, g2), 1))
    alg = 8.0 * nnz + 8.0 * (n + 1) + 4.0 * n  # col + val, row_ptr, y (x / g gathers hit L2)
    fm, am = statistics.mean(cf), statistics.mean(ca)
    out["csr"] = {"workload": "neo2_2d_spline CSR (3.6M rows, %d nonzeros), L2 flushed before each call" % nnz,
                  "forward_ms": fm, "adjoint_ms": am,
                  "roofline_forward": {"bound": "hbm", "achieved": alg / (fm / 1e3) / 1e9, "peak": peak,
                                       "unit": "GB/s", "frac": alg / (fm / 1e3) / 1e9 / peak,
                                       "peak_kind": peak_kind},
                  "roofline_adjoint": {"bound": "hbm", "achieved": alg / (am / 1e3) / 1e9, "peak": peak,
                                       "unit": "GB/s", "frac": alg / (am / 1e3) / 1e9 / peak,
                                       "peak_kind": peak_kind}}
    out["value"] = out["matrix_free"]["forward_rows_per_s"]
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Batch scheduler: the heterogeneous instance set (2D 128^2-512^2, 3D
    64^3-160^3, 10k-2M paths, straight and spline) in one persistent launch
    per phase, replayed from CUDA graphs, with the autotuner.  The lean form
    (no per-segment records) is allowed when the full form's workspace would
    not leave room for the CSR; the memory beside the CSR then keeps the full
    form for the largest instances."""
    import torch

    from paper_2108_12369_gb300 import build as B, pct
    torch.cuda.set_device(0)
    B.build()
    insts = W.batch_instances(args.batch_count, max_paths=args.batch_max_paths)
    rows = sum(len(w["angles"]) * w["paths_per_angle"] for w in insts)
    free, total_mem = torch.cuda.mem_get_info()
    full_ws = pct.batch_workspace_size(insts)
    csr_guess = 8.0 * 250 * rows  # ~250 nonzeros per row
    lean = args.batch_form == "lean" or (args.batch_form == "auto" and full_ws + csr_guess > 0.8 * free)
    # with the lean form allowed, the memory left beside the CSR holds the
    # largest instances' segment records (those keep the faster full-form fill)
    spare = int(min(full_ws, 0.8 * free - csr_guess)) if lean and args.batch_form == "auto" else 0
    bt = pct.Batch(insts, autotune=True, lean=lean, workspace_bytes=spare)
    for bx, ph in zip(bt.x_true, bt.phantoms):
        pct.phantom_rasterize(ph, bx)
    bt.count()
    nnz = bt.nnz()
    bt.fill(nnz)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        bt.count()
        bt.fill(nnz)
    tc, tf = [], []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        bt.count()
        nz = bt.nnz()  # synchronises: the read-back sizes the fill, as a caller must
        e[1].record()
        bt.fill(nz)
        e[2].record()
        torch.cuda.synchronize()
        tc.append(e[0].elapsed_time(e[1]))
        tf.append(e[1].elapsed_time(e[2]))
    ms = statistics.mean(tc) + statistics.mean(tf)
    tuning = bt.params()
    print(json.dumps({"metric": "batched proton paths/s", "value": rows / (ms / 1e3), "unit": "paths/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "data": "synthetic",
                      "phase_ms": {"count_and_nnz": statistics.mean(tc), "fill": statistics.mean(tf)},
                      "config": {"workload": "batch of heterogeneous instances", "instances": len(insts),
                                 "rows": rows, "nnz": int(sum(nnz)),
                                 "max_paths_per_instance": args.batch_max_paths,
                                 "form": ("lean, full for the largest instances" if spare > 0 else "lean")
                                 if lean else "mixed",
                                 "workspace_gb": bt.workspace.numel() / 1e9,
                                 "lean_minimum_gb": pct.batch_workspace_size(insts, lean=lean) / 1e9,
                                 "autotuned": tuning,
                                 "step": "count + nnz read-back + fill of every instance (graph replays)"}}),
          flush=True)


def run_sap(args):
    """Reconstruction (Sec. II-D, III): SAP with the paper's settings -- M =
    100 strings, lambda = 0.1, 20 iterations from x = 0 -- on simulated NEO 1
    (constant 1 mm chords, as the paper's examples) and NEO 2 (exact chords,
    spline paths) systems.  Reports the time per iteration and the relative
    image error and residual."""
    import torch

    from paper_2108_12369_gb300 import build as B, pct
    torch.cuda.set_device(0)
    B.build()
    out = {"metric": "SAP iterations/s", "unit": "iterations/s", "n_gpus": 1, "higher_is_better": True,
           "data": "synthetic", "cases": {}}
    cases = {"neo1_2d_straight_constant_chord": W.neo1_2d_straight(n_angles=180, paths_per_angle=1000),
             "neo2_2d_spline": W.neo2_2d_spline(n_angles=360, paths_per_angle=2000, n=200, h=1.0)}
    cases["neo1_2d_straight_constant_chord"]["model"] = dict(
        cases["neo1_2d_straight_constant_chord"]["model"], chord=W.CHORD_CONSTANT)
    for name, w in cases.items():
        ph, geo = pct.Phantom(w["phantom"]), pct.GeometryArgs(w)
        sim = pct.simulate(ph, geo, pct.PREC_MIXED)
        n = ph.nvox
        ws = torch.empty(pct.sap_workspace_size(n, 100), dtype=torch.uint8, device="cuda")
        x = torch.zeros(n, dtype=torch.float32, device="cuda")
        pct.sap(sim, sim["b"], n, 100, 0.1, 1, x, workspace=ws)  # warm-up
        x.zero_()
        ms = _timed(lambda: pct.sap(sim, sim["b"], n, 100, 0.1, 20, x, workspace=ws), 1)
        A = torch.sparse_csr_tensor(sim["row_ptr"], sim["col"].long(), sim["val"], size=(geo.n_rows, n))
        xt = sim["x_true"]
        out["cases"][name] = {"rows": geo.n_rows, "nnz": sim["nnz"], "strings": 100, "lambda": 0.1, "iterations": 20,
                              "ms_per_iteration": ms / 20,
                              "rel_image_error": (torch.linalg.norm(x - xt) / torch.linalg.norm(xt)).item(),
                              "rel_residual": (torch.linalg.norm(A @ x - sim["b"]) /
                                               torch.linalg.norm(sim["b"])).item()}
        del sim, ws, A
    out["value"] = 1e3 / out["cases"]["neo2_2d_spline"]["ms_per_iteration"]
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "f64"], default="mixed")
    ap.add_argument("--workload", default="head_3d_spline")
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the all-FP64 form (0: skip)")
    ap.add_argument("--accuracy-rows", type=int, default=2000,
                    help="rows sampled for the error statistics against the oracle (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--reference-rows", type=int, default=60000)
    ap.add_argument("--angles", type=int, default=0, help="override the angle count (profiling)")
    ap.add_argument("--paths-per-angle", type=int, default=0, help="override protons per angle (profiling)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host round trip (CSR larger than host RAM)")
    ap.add_argument("--mode", choices=["csr", "project", "batch", "sap"], default="csr",
                    help="csr: the headline CSR generation; project / batch / sap: the projector, batch and "
                         "reconstruction rows")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-max-paths", type=int, default=2_000_000)
    ap.add_argument("--batch-form", choices=["auto", "mixed", "lean"], default="auto")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "project":
        run_project(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "sap":
        run_sap(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
