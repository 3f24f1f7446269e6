#!/usr/bin/env python
"""Throughput of the coupled LB/FD step on GB300.

One bench step = one coupled time step (pull-stream, FD scalar update,
cumulant collision: the whole hot path) over the whole grid, one
`lbfd_step` call: the interior tile kernel plus the kernels of the
boundary-cell lists (`launches_per_step` in the JSON line).  Default
workload: the D3Q27 512x256x256 random sphere packing (33.5 M cells, 4.4 GB
of FP32 state per buffer, far beyond the 129 MB L2), mixed precision (FP32,
FP64 Arrhenius above 1000 K).  `secondary` repeats the measurement on the
16 packed 2-D channels.

Timing: W warm-up steps, then K timed steps; before every timed step a
256 MiB buffer is written to flush the L2, and each step is bracketed by
CUDA events on the launch stream.  Under torchrun each rank runs its own
replica (weak scaling, no collective on the data path).

--impl reference times the FP64 oracle (the plain CPU restatement of the
method) on all host cores on a bounded crop of the same workload.
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


def crop(cfg, solid, T, Y, x0, x1, y1, z1=None):
    """The box x0 <= x < x1, y < y1 (z < z1) of a workload: same geometry,
    fields and face types, fewer cells."""
    c = dict(cfg)
    c["nx"], c["ny"] = x1 - x0, y1
    if cfg["dim"] == 3:
        c["nz"] = z1
        sol = np.ascontiguousarray(solid[:z1, :y1, x0:x1])
        shp = (cfg["nz"], cfg["ny"], cfg["nx"])
        sl = (slice(0, z1), slice(0, y1), slice(x0, x1))
    else:
        sol = np.ascontiguousarray(solid[:y1, x0:x1])
        shp = (cfg["ny"], cfg["nx"])
        sl = (slice(0, y1), slice(x0, x1))
    Tc = np.ascontiguousarray(T.reshape(shp)[sl]).ravel()
    Yc = np.ascontiguousarray(Y.reshape((5,) + shp)[(slice(None),) + sl]).reshape(5, -1)
    return c, sol, Tc, Yc


def porous_crop(cfg, solid, T, Y, length: int):
    """A 32x32 cross-section of the sphere packing, `length` columns from
    x = 416 (the end of the packing and the hot band behind it)."""
    x0 = min(416, cfg["nx"] - length)
    return crop(cfg, solid, T, Y, x0, x0 + length, min(32, cfg["ny"]), min(32, cfg["nz"]))


def sample_workload(name: str, precision: str, length: int = 96, full=None):
    """A bounded slice of the workload for the CPU oracle (same physics and
    geometry rules, fewer cells).  `full` = (cfg, solid, T, Y) of the
    workload when it has been built already."""
    if name == "porous512x256x256":
        if full is None:
            full = workload(name, precision)[:4]
        cfg, solid, T, Y = porous_crop(*full, length)
        return cfg, solid, T, Y, (f"a {length}x32x32 crop of the 512x256x256 packing (x from "
                                  f"{min(416, 512 - length)}, y and z from 0: packing end and hot band)")
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
    cfg, solid, T, Y = inputs.sphere_packing(nx=32, ny=16, nz=16, x_range=(4, 28), r_range=(2.0, 4.0))
    return cfg, solid, T, Y, "a 32x16x16 sphere packing"


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if not model.isdigit():
                    break
    except Exception:
        pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


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


def measured_fp64_flops(workload: str, variant: int):
    """FP64 flops per step of the FP64 form (ncu: 2 x DFMA + DADD + DMUL
    thread instructions over the kernels of one step) from
    profiles/traffic.json, under the same rules as measured_traffic."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[workload + ":fp64"]
    except Exception:
        return None
    per_variant = rec.get("fp64_flops_per_step", {})
    if rec.get("csrc_sha256") != kernel_source_hash() or str(variant) not in per_variant:
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


def oracle_rate(cfg, solid, T, Y, steps: int, threads: int, warmup: int = 0):
    """Oracle MLUPS over `steps` steps from (T, Y, g = 0) with `threads`
    OpenMP threads; returns (MLUPS, threads used, seconds, oracle Sim)."""
    import oracle

    used = oracle.set_threads(threads)
    sim = oracle.Sim(cfg, solid)
    sim.set_state(T, Y)
    if warmup:
        sim.step(warmup)
    t0 = time.perf_counter()
    sim.step(steps)
    sec = time.perf_counter() - t0
    oracle.set_threads(1)
    fluid = int((solid == 0).sum())
    return fluid * steps / sec / 1e6, used, sec, sim


def run_reference(args):
    """The oracle (FP64, plain C, OpenMP over grid rows on every host core)
    on a bounded crop of the workload; rank 0 only."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle

    oracle.build()
    cores, model = host_cpu()
    # about 60 s of oracle work: cells per step scale as 1/(K + W)
    if args.workload == "porous512x256x256":
        rate = 0.05e6 * cores  # cell updates per second, D3Q27 (about 0.07 M per core measured)
        length = int(max(4, min(96, 60 * rate / ((args.steps + args.warmup) * 1024))))
    else:
        length = int(max(4, min(1024, 60 * 4.0e5 * cores / ((args.steps + args.warmup) * 1711))))
    cfg, solid, T, Y, sdesc = sample_workload(args.workload, "fp64", length)
    fluid = int((solid == 0).sum())
    value, used, sec, _ = oracle_rate(cfg, solid, T, Y, args.steps, cores, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "sample": sdesc, "fluid_cells": fluid},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": used, "kind": "oracle", "sample": sdesc,
                         "cpu_model": model, "nproc": cores},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(args, precision, full):
    """Oracle timing on a bounded sample (rank 0, N = 1 only): one thread,
    then OpenMP over every host core; plus the accuracy of the CUDA path
    on the same sample."""
    import oracle

    from paper_2304_05657_gb300 import lbfd

    oracle.build()
    cores, model = host_cpu()
    cfg, solid, T, Y, sdesc = sample_workload(args.workload, "fp64", 64, full=full)
    three = cfg["dim"] == 3
    steps1 = 4 if three else args.baseline_steps
    stepsN = args.baseline_steps
    v1, _, _, _ = oracle_rate(cfg, solid, T, Y, steps1, 1)
    vN, used, _, sim = oracle_rate(cfg, solid, T, Y, stepsN, cores)
    To, Yo, go = sim.get_state()
    gpu = lbfd.Solver(dict(cfg, precision=precision), solid)
    gpu.init_fields(T, Y)
    gpu.step(stepsN)
    Tg, Yg, gg = gpu.get_state()
    gpu.close()
    fl = solid.ravel() == 0
    err_T = float(np.linalg.norm(Tg[fl] - To[fl]) / np.linalg.norm(To[fl]))
    errs = [float(np.linalg.norm(Yg[k][fl] - Yo[k][fl]) / np.linalg.norm(Yo[k][fl])) for k in range(5)
            if np.linalg.norm(Yo[k][fl]) > 0]
    err_Y = max(errs) if errs else float("nan")
    err_g = float(np.max(np.abs(gg[:, fl] - go[:, fl])) / max(1e-300, np.max(np.abs(go[:, fl]))))
    return {"value": vN, "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"{sdesc}, {stepsN} steps from the workload's initial state",
            "nproc": cores, "cpu_model": model,
            "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1, "steps": steps1},
            "gpu_rel_l2_vs_oracle": {"T": err_T, "Y_max": err_Y, "g_max_abs_over_max": err_g,
                                     "steps": stepsN, "gpu_precision": precision}}


def gradient_rate(args):
    """Gradient steps per second of the flame position after S steps with
    respect to (ln A, Ta, T_wall, u_in) on the 512x64 cold-wall channel
    (S = --grad-steps, 4000 by default, checkpoints every --grad-checkpoint
    = 200 steps for the adjoint): the discrete adjoint (reverse mode), the
    mixed tangent (FP32 forward, FP64 Arrhenius above T_fp64 and FP64
    accumulation) and the FP64 tangent, next to plain FP64 (and mixed)
    steps per second on the same case; the adjoint checked against central
    differences of the FP64 step (relative step 1e-4, absolute in ln A).
    CUDA events on the handle's stream; the adjoint is timed on the host
    around its synchronous call."""
    import torch

    from paper_2304_05657_gb300 import grad, lbfd

    cfg, solid, T, Y = inputs.channel(nx=512, ny=64, walls="isothermal", T_wall=300.0)
    S, K = args.grad_steps, args.grad_checkpoint
    out = {"workload": "D2Q9 channel 512x64, isothermal 300 K walls, objective: flame position after "
                       f"{S} steps", "steps": S, "adjoint_checkpoint_every": K}
    stream = torch.cuda.current_stream()
    grads = {}
    key = {"tangent_mixed": "tangent_mixed_grad_steps_per_s", "tangent": "tangent_fp64_grad_steps_per_s",
           "fp64": "fp64_steps_per_s", "mixed": "mixed_steps_per_s"}
    for prec in ("tangent_mixed", "tangent", "fp64", "mixed"):
        s = lbfd.Solver(dict(cfg, precision=prec), solid, stream=stream)
        if prec in ("fp64", "mixed"):
            s.init_fields(T, Y)
            s.autotune(reps=5)
        s.init_fields(T, Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(S)
        e1.record(stream)
        torch.cuda.synchronize()
        out[key[prec]] = S / (e0.elapsed_time(e1) * 1e-3)
        if prec.startswith("tangent"):
            J, g = s.gradient(lbfd.OBJ_FLAME_POSITION)
            grads[prec] = np.asarray(g, dtype=np.float64)
        s.close()
    # the discrete adjoint: forward with checkpoints every K steps, then the
    # backward sweep with recomputation per segment
    s = lbfd.Solver(dict(cfg, precision="fp64"), solid, stream=stream)
    s.init_fields(T, Y)
    s.autotune(reps=5)
    s.init_fields(T, Y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ja, ga = s.adjoint_gradient(S, K)
    torch.cuda.synchronize()
    out["adjoint_grad_steps_per_s"] = S / (time.perf_counter() - t0)
    s.close()
    out["adjoint_vs_fp64_step_time"] = out["fp64_steps_per_s"] / out["adjoint_grad_steps_per_s"]
    # the same with the FP32 forward pass (mixed kernels; its steps recorded
    # in FP32), the adjoints accumulated in FP64
    s = lbfd.Solver(dict(cfg, precision="mixed"), solid, stream=stream)
    s.init_fields(T, Y)
    s.autotune(reps=5)
    s.init_fields(T, Y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Jm, gm = s.adjoint_gradient(S, K)
    torch.cuda.synchronize()
    out["adjoint_mixed_grad_steps_per_s"] = S / (time.perf_counter() - t0)
    s.close()
    # against the FP64 CPU adjoint of the oracle on a bounded sample: the
    # first 10 steps of the same case
    from oracle import adjoint as cpu_adjoint

    ns = 10
    s = lbfd.Solver(dict(cfg, precision="fp64"), solid, stream=stream)
    s.init_fields(T, Y)
    _, g10 = s.adjoint_gradient(ns, 5)
    s.close()
    t0 = time.perf_counter()
    _, c10 = cpu_adjoint.adjoint_gradient(cfg, solid, T, Y, ns, checkpoint_every=5)
    out["cpu_adjoint"] = {"steps": ns, "seconds": time.perf_counter() - t0,
                          "gpu_adjoint_vs_cpu_adjoint_max_rel": float(np.max(np.abs(g10 - c10) / np.abs(c10))),
                          "sample": "the first 10 steps of the same case (torch autograd through the FP64 "
                                    "restatement of the step, CPU)"}

    def J_fp64(theta):
        c = grad.apply_theta(cfg, theta)
        c["precision"] = "fp64"
        r = lbfd.Solver(c, solid, stream=stream)
        r.init_fields(T, Y)
        r.step(S)
        x = r.diagnostics()["x_f"] * cfg["dx"]
        r.close()
        return x

    theta = grad.theta_of(cfg)
    fd = np.zeros(4)
    for k in range(4):
        h = 1e-4 if k == 0 else 1e-4 * abs(theta[k])
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd[k] = (J_fp64(tp) - J_fp64(tm)) / (2 * h)
    ga = np.asarray(ga)
    gt = grads["tangent"]
    out["dJ_dtheta_adjoint"] = dict(zip(lbfd.THETA, [float(x) for x in ga]))
    out["dJ_dtheta_central_fd"] = dict(zip(lbfd.THETA, [float(x) for x in fd]))
    out["adjoint_vs_fd_max_rel"] = float(np.max(np.abs(ga - fd) / np.abs(fd)))
    out["adjoint_vs_tangent_max_rel"] = float(np.max(np.abs(ga - gt) / np.abs(gt)))
    out["tangent_mixed_vs_fp64_max_rel"] = float(np.max(np.abs(grads["tangent_mixed"] - gt) / np.abs(gt)))
    out["adjoint_mixed_vs_fp64_adjoint_max_rel"] = float(np.max(np.abs(np.asarray(gm) - ga) / np.abs(ga)))
    out["J_m"] = Ja
    return out


def flame_speed_accuracy():
    """Flame speed S_F = u_in - dx_f/dt (x_f sampled every 50 steps over
    steps 1000-2000, least-squares slope) of the 256x32 adiabatic channel
    ignited at the inlet: the mixed and FP64 GPU forms against the FP64
    oracle (all host cores)."""
    import oracle

    from paper_2304_05657_gb300 import lbfd

    cfg, solid, T, Y = inputs.channel(nx=256, ny=32)
    T, Y = inputs.ignition_fields(cfg, solid, 0, 20, burnt=False)

    def history(sim, step, diag):
        step(sim, 1000)
        ts, xs = [], []
        for i in range(21):
            ts.append(50 * i)
            xs.append(diag(sim))
            if i < 20:
                step(sim, 50)
        return cfg["u_in"] - np.polyfit(ts, xs, 1)[0]

    oracle.build()
    used = oracle.set_threads(os.cpu_count() or 1)
    o = oracle.Sim(cfg, solid)
    o.set_state(T, Y)
    So = history(o, lambda m, n: m.step(n), lambda m: m.diagnostics()["x_f"])
    oracle.set_threads(1)
    out = {"workload": "D2Q9 channel 256x32, adiabatic walls, unburnt mixture at 2000 K in columns 0-19",
           "S_F_oracle": So, "oracle_threads": used}
    for prec in ("mixed", "fp64"):
        s = lbfd.Solver(dict(cfg, precision=prec), solid)
        s.init_fields(T, Y)
        Sg = history(s, lambda m, n: m.step_graph(n), lambda m: m.diagnostics()["x_f"])
        s.close()
        out[f"S_F_{prec}"] = Sg
        out[f"{prec}_rel_err"] = abs(Sg - So) / abs(So)
    return out


def fp64_form(args, flush, full):
    """The plain FP64 form on the same workload and state recipe, timed the
    same way (flush + events per step) over fewer steps."""
    import torch

    from paper_2304_05657_gb300 import lbfd

    cfg, solid, T, Y = full
    cfg = dict(cfg, precision="fp64")
    three = cfg["dim"] == 3
    stream = torch.cuda.current_stream()
    s = lbfd.Solver(cfg, solid, stream=stream)
    s.init_fields(T, Y)
    prerun = 0 if three else args.prerun
    done = 0
    while done < prerun:
        n = min(1000, prerun - done)
        s.step_graph(n)
        done += n
    s.step(3)
    best, _ = s.autotune(reps=1 if three else 3)
    steps = args.fp64_steps if args.fp64_steps is not None else (10 if three else 100)
    ms = []
    for _ in range(steps):
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
    out = {"value": fluid / (t * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": t, "steps": steps,
           "kernel_variant": best, "dtype": "f64",
           "roofline_frac": fluid * bytes_per_cell(cfg) / (t * 1e-3) / 1e9 / peaks()[0],
           "prerun_steps": prerun}
    flops = measured_fp64_flops(args.workload, best)
    if flops is not None:
        rate = flops / (t * 1e-3) / 1e12
        out["fp64_tflops"] = {"achieved": rate, "peak_nominal": 1.25, "frac": rate / 1.25,
                              "flops_per_step": flops,
                              "note": "2 x DFMA + DADD + DMUL thread instructions of one step (ncu), over the "
                                      "event-timed step; GB300's FP64 rate is 1.25 TFLOP/s nominal"}
    return out


def prerun_graph(s, steps: int):
    done = 0
    while done < steps:
        n = min(1000, steps - done)
        s.step_graph(n)
        done += n


def timed_steps(s, flush, stream, steps: int):
    """Per-step CUDA-event times [ms] of `steps` single steps, each after
    an L2 flush; the events are recorded on the launch stream."""
    import torch

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev0[i].record(stream)
        s.step(1)
        ev1[i].record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])


def secondary(args, flush):
    """The same measurement on the 16 packed 2-D channels (105 MB of state
    per buffer, close to the L2 size): pre-run 10 000 steps so that the
    flames burn, autotune, then --secondary-steps flushed steps."""
    import torch

    from paper_2304_05657_gb300 import lbfd

    cfg, solid, T, Y, desc = workload("batched16x1024", args.precision)
    stream = torch.cuda.current_stream()
    s = lbfd.Solver(cfg, solid, stream=stream)
    s.init_fields(T, Y)
    prerun_graph(s, 10000)
    for _ in range(3):
        s.step(1)
    best, _ = s.autotune(reps=10)
    ms = timed_steps(s, flush, stream, args.secondary_steps)
    # the channel study itself (Sec. IV.A): flame speed of every channel from
    # the slope of its flame position over 2000 more steps, burning flags,
    # quenching width and the dead-zone thickness
    from paper_2304_05657_gb300 import channels

    seg = inputs.batched_channels()[4]
    tr = channels.FlameSpeedTracker(segments=seg)
    for n in range(0, 2001, 200):
        if n:
            s.step_graph(200)
        tr.record(s, n)
    widths = [y1 - y0 for y0, y1 in seg]
    burning = tr.burning()
    study = {"widths": widths, "S_F": [float(v) for v in tr.flame_speed(window=11)],
             "burning": [bool(b) for b in burning],
             "quenching_width": channels.quenching_width(widths, burning),
             "delta_dead": [d if b else None for d, b in zip(channels.channel_dead_zones(s, seg), burning)],
             "note": "lattice units (cells, cells per step), after 10 000 + warm-up + timed steps; S_F = u_in - "
                     "dx_f/dt fitted over 2000 steps; delta_dead: smallest wall distance of the per-column "
                     "peak heat release over the columns within 10 % of the channel's peak (null where the "
                     "channel does not burn)"}
    fluid = int((solid == 0).sum())
    mean_s = float(ms.mean()) * 1e-3
    alg = fluid * bytes_per_cell(cfg) + (solid.size - fluid)
    traffic, _ = measured_traffic("batched16x1024", best, args.precision)
    out = {"workload": "batched16x1024", "description": desc, "value": fluid / mean_s / 1e6, "unit": "MLUPS",
           "ms_per_step": mean_s * 1e3, "steps": args.secondary_steps, "kernel_variant": best,
           "launches_per_step": s.launches_per_step, "prerun_steps": 10000,
           "roofline": {"bound": "hbm", "achieved": alg / mean_s / 1e9, "peak": peaks()[0], "unit": "GB/s",
                        "frac": alg / mean_s / 1e9 / peaks()[0], "traffic": traffic,
                        "algorithmic_bytes_per_step": alg},
           "channel_study": study}
    # the same steps in one persistent launch (grid-wide barriers between steps)
    for _ in range(3):
        s.step(1)
    s.step_persistent(10)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step_persistent(args.secondary_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    tp = e0.elapsed_time(e1) / args.secondary_steps
    out["persistent"] = {"ms_per_step": tp, "value": fluid / (tp * 1e-3) / 1e6, "unit": "MLUPS",
                         "launches": 1, "steps": args.secondary_steps, "l2": "not flushed between steps"}
    s.close()
    return out


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
    # advance the physical state (flow developed, flames burning) before timing
    prerun_graph(s, args.prerun)
    torch.cuda.synchronize()
    T_now = s.read_field(lbfd.FIELD_T)
    hot_fraction = float(((T_now > cfg["T_fp64"]) & (solid.ravel() == 0)).sum() / max(1, (solid == 0).sum()))
    del T_now
    fluid = int((solid == 0).sum())
    ncell = solid.size
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    if args.variant is not None:
        s.variant = args.variant
    timed_steps(s, flush, stream, args.warmup)
    if args.variant is None:
        best, tune_ms = s.autotune(reps=10)
    else:
        best, tune_ms = args.variant, []
    torch.cuda.synchronize()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local if world > 1 else 0]
    import tempfile

    clock_csv = os.path.join(tempfile.gettempdir(), f"lbfd_clocks_{os.getpid()}_{rank}.csv")
    sampler = ClockSampler(gpu_index, clock_csv)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    step_ms = timed_steps(s, flush, stream, args.steps)
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
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
    del host
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
                   "precision": precision, "l2": "flushed before every timed step (256 MiB write); the state "
                   f"({nbytes / 1e9:.2f} GB per buffer) is also far larger than the L2",
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
    s.close()
    extra = rank == 0 and world == 1
    if extra and not args.no_baseline:
        line["cpu_baseline"] = cpu_baseline(args, precision, (cfg, solid, T, Y))
    if extra and args.fp64_steps != 0 and precision == "mixed":
        line["fp64_form"] = fp64_form(args, flush, (cfg, solid, T, Y))
    if extra and args.secondary_steps > 0 and args.workload != "batched16x1024":
        line["secondary"] = secondary(args, flush)
    if extra and not args.no_baseline:
        line["flame_speed_accuracy"] = flame_speed_accuracy()
    if extra and args.grad_steps > 0:
        line["gradient"] = gradient_rate(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="porous512x256x256",
                    choices=["porous512x256x256", "batched16x1024", "channel256x32", "burner2048x512",
                             "porous128x64x64", "porous256x128x128"])
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--baseline-steps", type=int, default=40)
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--grad-steps", type=int, default=4000, help="gradient-rate steps (0: skip)")
    ap.add_argument("--grad-checkpoint", type=int, default=200, help="adjoint checkpoint interval")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="steps of the FP64 comparison (0: skip; default 10 in 3-D, 100 in 2-D)")
    ap.add_argument("--secondary-steps", type=int, default=300,
                    help="timed steps of the 2-D batched record (0: skip)")
    ap.add_argument("--prerun", type=int, default=None,
                    help="untimed physical steps before warm-up (default: 10000 for the batched channels, "
                         "1000 for the 512x256x256 packing)")
    ap.add_argument("--variant", type=int, default=None, help="kernel variant (default: autotune)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.prerun is None:
        args.prerun = {"batched16x1024": 10000, "porous512x256x256": 1000}.get(args.workload, 0)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
