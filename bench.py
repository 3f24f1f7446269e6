#!/usr/bin/env python
"""Throughput of the coupled LB/FD step on GB300.

One bench step = one coupled time step (pull-stream, FD scalar update,
cumulant collision: the whole hot path, one fused kernel launch) over the
whole batch.  Default workload: 16 2-D D2Q9 channels of widths 16..196 and
length 1024 with isothermal walls, packed into one masked domain, mixed
precision (FP32, FP64 Arrhenius above 1000 K).

Timing: W warm-up steps, then K timed steps; before every timed step a
256 MiB buffer is written to flush the L2 (the state is 104 MiB per
buffer), and each step is bracketed by CUDA events on the launch stream.
Under torchrun each rank runs its own replica (the channels are independent
problems: weak scaling, no collective on the data path).

--impl reference times the FP64 oracle (the plain CPU restatement of the
method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_05657_gb300 import inputs  # noqa: E402

METRIC = "coupled MLUPS & HBM GB/s (% roofline); adjoint grad-steps/s vs plain FP64 GPU"
FLUSH_BYTES = 256 << 20


def workload(name: str, precision: str):
    """(cfg, solid, T, Y, description) of a named workload."""
    if name == "batched16x1024":
        cfg, solid, T, Y, seg = inputs.batched_channels()
        desc = ("16 D2Q9 channels, widths 16..196 (step 12), length 1024, isothermal 300 K walls, 1 solid row "
                "between, closed adiabatic ignition end, constant-pressure open end")
    elif name == "channel256x32":
        cfg, solid, T, Y = inputs.channel(nx=256, ny=32)
        T, Y = inputs.ignition_fields(cfg, solid, 0, 20, burnt=False)
        desc = "D2Q9 channel 256x32, adiabatic walls"
    elif name == "burner2048x512":
        cfg, solid, T, Y = inputs.cylinder_burner()
        desc = "D2Q9 2048x512 staggered cylinders d=40 pitch 64, 373 K"
    elif name == "porous512x256x256":
        cfg, solid, T, Y = inputs.sphere_packing()
        desc = "D3Q27 512x256x256 overlapping spheres r in [8,16], porosity 0.80"
    elif name == "porous128x64x64":
        cfg, solid, T, Y = inputs.sphere_packing(nx=128, ny=64, nz=64, x_range=(16, 112))
        desc = "D3Q27 128x64x64 overlapping spheres r in [8,16], porosity 0.80 (profiling size)"
    elif name == "porous256x128x128":
        cfg, solid, T, Y = inputs.sphere_packing(nx=256, ny=128, nz=128, x_range=(32, 224))
        desc = "D3Q27 256x128x128 overlapping spheres r in [8,16], porosity 0.80 (profiling size)"
    else:
        raise SystemExit(f"unknown workload {name}")
    cfg["precision"] = precision
    return cfg, solid, T, Y, desc


def sample_workload(name: str, precision: str, length: int = 96):
    """A bounded slice of the workload for the CPU oracle (same physics and
    geometry rules, fewer cells)."""
    if name == "batched16x1024":
        cfg, solid, T, Y, seg = inputs.batched_channels(length=length)
        return cfg, solid, T, Y, f"the 16 channels cut to length {length} ({1711 * length} cells)"
    if name == "channel256x32":
        cfg, solid, T, Y = inputs.channel(nx=256, ny=32)
        T, Y = inputs.ignition_fields(cfg, solid, 0, 20, burnt=False)
        return cfg, solid, T, Y, "the full 256x32 channel"
    if name == "burner2048x512":
        cfg, solid, T, Y = inputs.cylinder_burner(nx=256, ny=128, x_range=(64, 192))
        return cfg, solid, T, Y, "a 256x128 crop of the burner geometry"
    if name == "porous128x64x64":
        cfg, solid, T, Y = inputs.sphere_packing(nx=32, ny=16, nz=16, x_range=(4, 28), r_range=(2.0, 4.0))
        return cfg, solid, T, Y, "a 32x16x16 sphere packing"
    if name == "porous256x128x128":
        cfg, solid, T, Y = inputs.sphere_packing(nx=32, ny=16, nz=16, x_range=(4, 28), r_range=(2.0, 4.0))
        return cfg, solid, T, Y, "a 32x16x16 sphere packing"
    cfg, solid, T, Y = inputs.sphere_packing(nx=32, ny=16, nz=16, x_range=(4, 28), r_range=(2.0, 4.0))
    return cfg, solid, T, Y, "a 32x16x16 sphere packing"


def bytes_per_cell(cfg) -> int:
    Q = 9 if cfg["dim"] == 2 else 27
    e = 8 if cfg["precision"] == "fp64" else 4
    return (Q + 1 + 5) * e * 2 + 1  # read + write every state value, read the mask byte


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """sha256 over the CUDA sources and the C header, in name order."""
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2304_05657_gb300", "csrc", "*")))
    files.append(os.path.join(ROOT, "include", "lbfd.h"))
    for path in files:
        if path.endswith((".cu", ".cuh", ".h")):
            h.update(os.path.basename(path).encode())
            with open(path, "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def measured_traffic(workload: str, variant: int, precision: str):
    """DRAM bytes per step (ncu dram__bytes_read.sum + dram__bytes_write.sum
    over the kernels of one step) recorded in profiles/traffic.json, or None
    when the record is for other kernel sources, variant or precision."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[workload]
    except Exception:
        return None, None
    per_variant = rec.get("dram_bytes_per_step", {})
    if (rec.get("csrc_sha256") != kernel_source_hash() or rec.get("precision") != precision
            or str(variant) not in per_variant):
        return None, rec.get("csrc_sha256")
    return float(per_variant[str(variant)]) * float(rec.get("scale_to_workload", 1.0)), rec.get("csrc_sha256")


def measured_instructions(workload: str, variant: int, precision: str):
    """Warp instructions per step (ncu smsp__inst_executed.sum over the
    kernels of one step) from profiles/traffic.json, under the same rules
    as measured_traffic."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[workload]
    except Exception:
        return None
    per_variant = rec.get("warp_instructions_per_step", {})
    if (rec.get("csrc_sha256") != kernel_source_hash() or rec.get("precision") != precision
            or str(variant) not in per_variant):
        return None
    return float(per_variant[str(variant)]) * float(rec.get("scale_to_workload", 1.0))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str, path: str):
        self.path = path
        self.proc = None
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "20",
                 "-i", gpu_index], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle (FP64, single thread, plain C) on a bounded sample."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle

    oracle.build()
    # about 60 s of oracle work in total: cells per step scale as 1/(K+W)
    length = int(max(4, min(1024, 60 * 4.0e5 / ((args.steps + args.warmup) * 1711))))
    cfg, solid, T, Y, sdesc = sample_workload(args.workload, "fp64", length)
    fluid = int((solid == 0).sum())
    sim = oracle.Sim(cfg, solid)
    sim.set_state(T, Y)
    for _ in range(args.warmup):
        sim.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        sim.step(1)
        times.append(time.perf_counter() - t0)
    sec = float(np.sum(times))
    value = fluid * args.steps / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "sample": sdesc, "fluid_cells": fluid},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sdesc},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(args, precision):
    """Oracle timing on a bounded sample (rank 0, N = 1 only), plus the
    accuracy of the CUDA path on the same sample."""
    import oracle

    from paper_2304_05657_gb300 import lbfd

    oracle.build()
    cfg, solid, T, Y, sdesc = sample_workload(args.workload, "fp64")
    fluid = int((solid == 0).sum())
    sim = oracle.Sim(cfg, solid)
    sim.set_state(T, Y)
    steps = args.baseline_steps
    t0 = time.perf_counter()
    sim.step(steps)
    sec = time.perf_counter() - t0
    To, Yo, go = sim.get_state()
    gpu = lbfd.Solver(dict(cfg, precision=precision), solid)
    gpu.set_state(T, Y)
    gpu.step(steps)
    Tg, Yg, gg = gpu.get_state()
    gpu.close()
    err_T = float(np.linalg.norm(Tg - To) / np.linalg.norm(To))
    errs = [float(np.linalg.norm(Yg[k] - Yo[k]) / np.linalg.norm(Yo[k])) for k in range(5)
            if np.linalg.norm(Yo[k]) > 0]
    err_Y = max(errs) if errs else float("nan")
    return {"value": fluid * steps / sec / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": f"{sdesc}, {steps} steps from the workload's initial state",
            "gpu_rel_l2_vs_oracle": {"T": err_T, "Y_max": err_Y, "steps": steps}}


def gradient_rate(args):
    """Gradient steps per second of flame position w.r.t. (ln A, Ta, T_wall,
    u_in) on the 512x64 cold-wall channel: the mixed tangent form (FP32
    forward, FP64 Arrhenius above T_fp64, FP64 accumulation of the
    gradient) and the FP64 tangent form, next to plain FP64 (and mixed)
    steps per second on the same case; CUDA events on the handle's stream."""
    import torch

    from paper_2304_05657_gb300 import lbfd

    cfg, solid, T, Y = inputs.channel(nx=512, ny=64, walls="isothermal", T_wall=300.0)
    out = {"workload": "D2Q9 channel 512x64, isothermal 300 K walls, objective: flame position",
           "mode": "tangent-linear (forward), 4 directions; grad_steps_per_s: FP32 forward with FP64 "
                   "Arrhenius above 1000 K and FP64 gradient accumulation",
           "steps": args.grad_steps}
    stream = torch.cuda.current_stream()
    grads = {}
    key = {"tangent_mixed": "grad_steps_per_s", "tangent": "grad_steps_per_s_fp64_tangent",
           "fp64": "fp64_steps_per_s", "mixed": "mixed_steps_per_s"}
    for prec in ("tangent_mixed", "tangent", "fp64", "mixed"):
        s = lbfd.Solver(dict(cfg, precision=prec), solid, stream=stream)
        s.init_fields(T, Y)
        if prec in ("fp64", "mixed"):
            s.autotune(reps=5)
        s.step(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(args.grad_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        out[key[prec]] = args.grad_steps / (e0.elapsed_time(e1) * 1e-3)
        if prec.startswith("tangent"):
            J, g = s.gradient(lbfd.OBJ_FLAME_POSITION)
            grads[prec] = np.asarray(g, dtype=np.float64)
        s.close()
    # the discrete adjoint (reverse mode, FP64): forward with checkpoints
    # every K steps, then the backward sweep with recomputation per segment
    # (the tangent runs above also started from this initial state and ran
    # 5 + grad_steps steps: the same map)
    K = max(1, args.grad_steps // 4)
    s = lbfd.Solver(dict(cfg, precision="fp64"), solid, stream=stream)
    s.init_fields(T, Y)
    s.autotune(reps=5)
    s.init_fields(T, Y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, ga = s.adjoint_gradient(5 + args.grad_steps, K)
    torch.cuda.synchronize()
    out["adjoint_grad_steps_per_s"] = (5 + args.grad_steps) / (time.perf_counter() - t0)
    out["adjoint_checkpoint_every"] = K
    s.close()
    gt = grads["tangent"]
    out["adjoint_vs_tangent_max_rel"] = float(np.max(np.abs(np.asarray(ga) - gt) / np.abs(gt)))
    out["dJ_dtheta"] = dict(zip(lbfd.THETA, [float(x) for x in grads["tangent_mixed"]]))
    out["dJ_dtheta_fp64_tangent"] = dict(zip(lbfd.THETA, [float(x) for x in grads["tangent"]]))
    out["mixed_vs_fp64_tangent_max_rel"] = float(np.max(np.abs(grads["tangent_mixed"] - grads["tangent"])
                                                       / np.abs(grads["tangent"])))
    out["grad_vs_fp64_step_time"] = out["fp64_steps_per_s"] / out["grad_steps_per_s"]
    return out


def fp64_form(args, flush):
    """The plain FP64 form on the same workload and state recipe, timed the
    same way (flush + events per step) over fewer steps."""
    import torch

    from paper_2304_05657_gb300 import lbfd

    cfg, solid, T, Y, _ = workload(args.workload, "fp64")
    stream = torch.cuda.current_stream()
    s = lbfd.Solver(cfg, solid, stream=stream)
    s.init_fields(T, Y)
    done = 0
    while done < args.prerun:
        n = min(1000, args.prerun - done)
        s.step_graph(n)
        done += n
    s.step(3)
    best, _ = s.autotune(reps=3)
    ms = []
    for _ in range(args.fp64_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(1)
        e1.record(stream)
        ms.append((e0, e1))
    torch.cuda.synchronize()
    t = sum(a.elapsed_time(b) for a, b in ms) / len(ms)
    fluid = int((solid == 0).sum())
    s.close()
    return {"value": fluid / (t * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": t, "steps": args.fp64_steps,
            "kernel_variant": best, "dtype": "f64", "roofline_frac": fluid * 241 / (t * 1e-3) / 1e9 / peaks()[0]}


def run_ours(args):
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2304_05657_gb300 import build as libbuild
    from paper_2304_05657_gb300 import lbfd

    if rank == 0:
        libbuild.build()
    if world > 1:
        torch.distributed.barrier()
    precision = args.precision
    cfg, solid, T, Y, desc = workload(args.workload, precision)
    stream = torch.cuda.current_stream()
    s = lbfd.Solver(cfg, solid, stream=stream)
    s.init_fields(T, Y)
    # advance the physical state to mid-run (flames burning) before timing
    done = 0
    while done < args.prerun:
        n = min(1000, args.prerun - done)
        s.step_graph(n)
        done += n
    torch.cuda.synchronize()
    T_now = s.read_field(lbfd.FIELD_T)
    hot_fraction = float(((T_now > cfg["T_fp64"]) & (solid.ravel() == 0)).sum() / max(1, (solid == 0).sum()))
    fluid = int((solid == 0).sum())
    ncell = solid.size
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def one_step(ev0=None, ev1=None):
        flush.zero_()
        if ev0 is not None:
            ev0.record(stream)
        s.step(1)
        if ev1 is not None:
            ev1.record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if args.variant is None:
        best, tune_ms = s.autotune(reps=10)
    else:
        s.variant = args.variant
        best, tune_ms = args.variant, []
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    sampler = ClockSampler(gpu_index, os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv")
                           if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else f"/tmp/lbfd_clocks_{rank}.csv")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        one_step(ev0[i], ev1[i])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    total_ms = float(step_ms.sum())
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    diag = s.diagnostics()

    # end to end through the C ABI with pinned host buffers
    nbytes = s.state_bytes()
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    s.get_state_raw(host.data_ptr(), nbytes)
    e2e_steps = min(args.steps, args.e2e_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s.set_state_raw(host.data_ptr(), nbytes)
        s.step(1)
        s.get_state_raw(host.data_ptr(), nbytes)
    torch.cuda.synchronize()
    e2e_sec = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_sec], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_sec = float(t.item())

    value = fluid * world * args.steps / (total_ms * 1e-3) / 1e6
    e2e_value = fluid * world * e2e_steps / e2e_sec / 1e6
    bpc = bytes_per_cell(cfg)
    alg_bytes = fluid * bpc + (ncell - fluid) * 1
    mean_s = float(step_ms.mean()) * 1e-3
    peak, peak_kind = peaks()
    achieved = alg_bytes / mean_s / 1e9
    traffic, _ = measured_traffic(args.workload, s.variant, precision)
    # the bound that the counters show: instruction issue.  Peak = one warp
    # instruction per cycle per SM sub-partition (4 per SM) at the SM clock
    # sampled during the timed region.
    insts = measured_instructions(args.workload, s.variant, precision)
    issue = None
    if insts is not None:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        peak_ips = sms * 4 * mhz * 1e6
        issue = {"warp_instructions_per_step": insts, "achieved_warp_inst_per_s": insts / mean_s,
                 "peak_warp_inst_per_s": peak_ips, "frac": insts / mean_s / peak_ips,
                 "note": "instructions of every kernel of the step (ncu), over the event-timed step"}
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "cells": ncell, "fluid_cells": fluid,
                   "precision": precision, "l2": "flushed before every timed step (256 MiB write)",
                   "state_bytes_per_buffer": nbytes, "parallelism": f"replicas x{world}",
                   "kernel_variant": s.variant, "launches_per_step": s.launches_per_step,
                   "autotune_ms_per_variant": [round(float(t), 4) for t in tune_ms]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "traffic_unit": "DRAM bytes per step (ncu, all kernels of one step)",
                     "algorithmic_bytes_per_step": alg_bytes, "algorithmic_bytes_per_cell": bpc,
                     "kernel": "one lbfd_step (the tile kernel with its boundary and wall kernels)",
                     "mean_launch_ms": mean_s * 1e3, "issue": issue},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "steps": e2e_steps, "api": "lbfd_set_state_raw + lbfd_step + lbfd_get_state_raw (pinned)"},
        "gpu_launches": args.steps * s.launches_per_step,
        "clocks": clocks,
        "wall_ms_per_step_with_flush": 1e3 * t_wall / args.steps,
        "diagnostics_after": {k: diag[k] for k in ("x_f", "T_max", "n_nonfinite")},
        "prerun_steps": args.prerun,
        "fluid_fraction_above_T_fp64": hot_fraction,
    }
    if rank == 0 and world == 1 and not args.no_baseline:
        line["cpu_baseline"] = cpu_baseline(args, precision)
    if rank == 0 and world == 1 and args.grad_steps > 0:
        line["gradient"] = gradient_rate(args)
    if rank == 0 and world == 1 and args.fp64_steps > 0 and precision == "mixed":
        line["fp64_form"] = fp64_form(args, flush)
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="batched16x1024",
                    choices=["batched16x1024", "channel256x32", "burner2048x512", "porous512x256x256",
                             "porous128x64x64", "porous256x128x128"])
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--baseline-steps", type=int, default=40)
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--grad-steps", type=int, default=200, help="gradient-rate steps (0: skip)")
    ap.add_argument("--fp64-steps", type=int, default=100, help="steps of the FP64 comparison (0: skip)")
    ap.add_argument("--prerun", type=int, default=None,
                    help="untimed physical steps before warm-up (default: 10000 for the batched channels)")
    ap.add_argument("--variant", type=int, default=None, help="kernel variant (default: autotune)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.prerun is None:
        args.prerun = 10000 if args.workload == "batched16x1024" else 0
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
