#!/usr/bin/env python3
"""Benchmark of the semi-implicit Fourier pseudo-spectral PFC step on GB300.

Workload (one bench step = one pfc_step call advancing the state by INNER time steps):
  2D one-mode PFC, 4096 x 4096 periodic grid, dx = pi/4, dt = 0.5, r = -0.25, psi0 = -0.25 plus a
  periodic-Voronoi polycrystal of 64 triangular one-mode grains (amplitude 0.2, lattice
  wavenumber 1, SplitMix64 seed 2) and U[-0.01, 0.01] noise; FP32-mixed path (FP32 data and
  butterflies, FP64-generated twiddles, FP64 mean and reductions).
Metric: grid-point-steps/s = (grid points) x (time steps) / time, whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference implementation: the paper
ships no code) on the host cores, one time step of the same workload per bench step.
Multi-GPU runs are independent replicas (the single-domain step has no data-parallel split).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
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

METRIC = "PFC grid-point-steps/s and FFT HBM GB/s (% peak) vs plain FP64 step, 1 GB300"
UNIT = "grid-point-steps/s"
NY = NX = 4096
DX, DT, R_OP, MEAN = math.pi / 4, 0.5, -0.25, -0.25
INNER = 100
WORKLOAD = ("2D one-mode PFC 4096x4096, dx=pi/4, dt=0.5, r=-0.25, psi0=-0.25 + 64-grain "
            "triangular polycrystal (amp 0.2, q=1, seed 2) + U[-0.01,0.01] noise; "
            f"{INNER} semi-implicit time steps per bench step; FP32-mixed")
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 / cuFFT context timings")
    ap.add_argument("--no-autotune", action="store_true",
                    help="--config 4a/4b: keep the planner's tiles instead of autotuning them")
    ap.add_argument("--autotune", action="store_true",
                    help="autotune the plan's tiles before timing (--config 1/3, and the headline)")
    ap.add_argument("--config", choices=sorted(CONFIGS), default=None,
                    help="time one of the other workloads instead of the 4096^2 headline (1 GPU)")
    return ap.parse_args()


# The other workloads of the method, each timed with the same discipline (warm-up, CUDA events,
# a 512 MiB L2 flush between timed steps) and reported against the HBM roofline at its modelled
# bytes per grid point per step. Sweeps count full reads or writes of a half spectrum (or of the
# real field): single-field step 5 (row 2, line 3); coupled pair 10 (row 2 x 2 fields, line
# reads X0, X1, C0, C1 and writes X0, X1); adjoint step 17 (entry of psi_n 2, psi^3 row pass 2,
# entry of lambda 2, adjoint line pass 3 reads + 2 writes, exit 2, 3 psi_n^2 mix 4).
CONFIGS = {
    "1": dict(desc="2D one-mode 128x128 FP64, dx=pi/4, dt=0.5, r=-0.25, psi0=-0.25+U[-0.01,0.01] "
                   "(seed 1); 100 time steps per bench step (launch-bound, L2-resident)",
              kind="plan", dims=(128, 128), prec="fp64", op=(0, -0.25, 0.0, 0.0), dt=0.5, inner=100,
              sweeps=5),
    "3": dict(desc="3D two-mode 512^3 FP32-mixed, dx=pi/4, dt=0.1, r=-0.3, R1=0.05, q2=sqrt(4/3), "
                   "psi0=-0.35+U[-0.02,0.02] (seed 3); 10 time steps per bench step",
              kind="plan", dims=(512, 512, 512), prec="fp32", op=(1, -0.3, 0.05, math.sqrt(4.0 / 3.0)),
              dt=0.1, inner=10, sweeps=5),
    "4a": dict(desc="1024 batched 2D one-mode domains, nx, ny from {64,128,256,512}, r~U[-0.4,-0.1], "
                    "mean~U[-0.4,-0.2] (seed 4), noise 0.01, dt=0.5, FP32-mixed; 20 time steps per bench "
                    "step, tiles and schedule autotuned",
               kind="batch", prec="fp32", dt=0.5, inner=20, sweeps=5, autotune=True),
    "4p": dict(desc="1024 batched 2D one-mode domains as config 4a, FP32-mixed; 20 time steps per bench step "
                    "in one persistent cooperative launch (replayed as a one-node CUDA graph)",
               kind="batch", prec="fp32", dt=0.5, inner=20, sweeps=5, schedule="persistent"),
    "4": dict(desc="config 4 in one persistent launch: the 1024 domains of config 4a and the coupled pair of "
                   "config 4b (256^3, alpha=0.1) stepped together, FP32-mixed, dt=0.5; 20 time steps per bench step; "
                   "rate in grid points of the domains plus grid points of the pair (both fields of a pair point "
                   "counted once) per second; block size autotuned",
              kind="batch", prec="fp32", dt=0.5, inner=20, sweeps=5, pair=(256, 256, 256), autotune=True),
    "4b": dict(desc="coupled density/composition pair 256^3 FP32-mixed, alpha=0.1, one-mode r=-0.25 "
                    "for both, means -0.25/-0.2, noise 0.01 (seeds 5, 6), dt=0.5; 10 time steps per "
                    "bench step", kind="pair", dims=(256, 256, 256), prec="fp32", dt=0.5, inner=10,
               sweeps=10, autotune=True),
    "5": dict(desc="adjoint step, 3D one-mode 256^3 FP32-mixed, dx=pi/4, dt=0.5, r=-0.25, "
                   "psi0=-0.25+U[-0.01,0.01] (seed 6); 10 adjoint steps per bench step",
              kind="adjoint", dims=(256, 256, 256), prec="fp32", op=(0, -0.25, 0.0, 0.0), dt=0.5,
              inner=10, sweeps=17),
    "5d": dict(desc="adjoint step, 3D one-mode 256^3 FP64, as config 5; 5 adjoint steps per bench step",
               kind="adjoint", dims=(256, 256, 256), prec="fp64", op=(0, -0.25, 0.0, 0.0), dt=0.5,
               inner=5, sweeps=17),
    "5s": dict(desc="adjoint over recorded segments, 3D one-mode 256^3 FP32-mixed, as config 5: per bench step "
                    "the forward recompute of a 20-step segment with its record (pfc_step_record) and the "
                    "fused adjoint over it (pfc_adjoint_segment); rate in rollout steps (forward + adjoint) x points",
               kind="segment", dims=(256, 256, 256), prec="fp32", op=(0, -0.25, 0.0, 0.0), dt=0.5,
               inner=20, sweeps=14),
    "h": dict(desc="hydrodynamic PFC 256^3 FP32-mixed (density and three velocity components), one-mode "
                   "r=-0.25, dx=pi/4, dt=0.5, rho=1, Gamma=1, a0=2, psi0=-0.25+U[-0.1,0.1] (seed 91), "
                   "v0=0.05 U[-1,1] (seeds 92-94); 2 steps per bench step (20 transforms of the grid a step)",
              kind="hydro", dims=(256, 256, 256), prec="fp32", op=(0, -0.25, 0.0, 0.0), dt=0.5, inner=2,
              sweeps=110),
    "af": dict(desc="amplitude-expansion PFC, 3D BCC set of six complex amplitudes at 256^3 FP32-mixed, "
                    "one-mode r=-0.25, psibar=-0.2, dx=1.1, dt=0.4, eta=0.1+0.02(U[-1,1]+iU[-1,1]) (torch "
                    "generator, seed 9); 10 steps per bench step; rate in grid points x amplitudes per second, "
                    "11 sweeps of 8 B a step", kind="apfc", dims=(256, 256, 256), prec="fp32",
               op=(0, -0.25, 0.0, 0.0), dt=0.4, inner=10, sweeps=22),
    "3d64": dict(desc="3D two-mode 512^3 FP64 (three-pass schedule), as config 3; 4 time steps per bench step",
                 kind="plan", dims=(512, 512, 512), prec="fp64", op=(1, -0.3, 0.05, math.sqrt(4.0 / 3.0)),
                 dt=0.1, inner=4, sweeps=9),
    "750": dict(desc="3D one-mode 750^3 FP32-mixed (the paper's best single-GPU size; mixed-radix schedule, "
                     "radices 2, 3, 5), dx=pi/4, dt=0.5, r=-0.25, psi0=-0.25+U[-0.01,0.01] (seed 6); "
                     "4 time steps per bench step",
                kind="plan", dims=(750, 750, 750), prec="fp32", op=(0, -0.25, 0.0, 0.0), dt=0.5, inner=4,
                sweeps=11),
    "1400": dict(desc="3D one-mode 1400^3 FP32-mixed (the paper's largest grid, 4 H100 there; mixed-radix "
                      "schedule, radices 8, 7, 5), dx=pi/4, dt=0.5, r=-0.25, psi0=-0.25+U[-0.01,0.01] "
                      "(torch generator, seed 8); 2 time steps per bench step",
                 kind="plan", dims=(1400, 1400, 1400), prec="fp32", op=(0, -0.25, 0.0, 0.0), dt=0.5,
                 inner=2, sweeps=11, device_draw=True),
    "L": dict(desc="the largest power-of-two 3D one-mode grid whose FP32-mixed plan and state fit the GPU's "
                   "free memory (2048^3 on a GB300), dx=pi/4, dt=0.5, r=-0.25, psi0=-0.25+U[-0.01,0.01] "
                   "(torch generator, seed 8), three-pass schedule; 3 time steps per bench step",
              kind="largest", prec="fp32", op=(0, -0.25, 0.0, 0.0), dt=0.5, inner=3, sweeps=9),
}

# Bytes of a plan's real state, its scratch (3 half spectra for a three-pass plan) and slack, per
# grid point, FP32-mixed: the largest cube is chosen from the free memory with this.
BYTES_PER_POINT_FP32_THREE_PASS = 4 + 3 * 4 + 1


def largest_cube(free_bytes):
    n = 256
    while (2 * n) ** 3 * BYTES_PER_POINT_FP32_THREE_PASS <= free_bytes and 2 * n <= 4096:
        n *= 2
    return n


def run_config(args):
    """Time one of CONFIGS on GPU 0 and print one JSON line."""
    import numpy as np
    import torch
    from paper_2603_26818_gb300 import binding, inputs

    c = CONFIGS[args.config]
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    prec = c["prec"]
    dtype = torch.float64 if prec == "fp64" else torch.float32
    vb = 8 if prec == "fp64" else 4
    extra = {}
    if c["kind"] == "batch":
        draws = inputs.batch_draws(1024, seed=4)
        obj = binding.Batch([(d[0], d[1]) for d in draws], [d[2] for d in draws], DX, c["dt"], precision=prec)
        parts = [inputs.uniform_state((ny, nx), m, 0.01, seed=1000 + i).ravel() for i, (ny, nx, r, m) in enumerate(draws)]
        state = torch.from_numpy(np.concatenate(parts)).to(device=dev, dtype=dtype)
        npts = state.numel()
        run = lambda: obj.step(state, c["inner"])
        if c.get("pair"):
            # the coupled pair of config 4b in the same persistent launch
            shape = c["pair"]
            p0 = inputs.uniform_state(shape, -0.25, 0.01, seed=5)
            c0 = inputs.uniform_state(shape, -0.2, 0.01, seed=6)
            obj.attach_pair(shape, [binding.make_op(0, -0.25), binding.make_op(0, -0.25)], 0.1)
            pair_state = torch.from_numpy(np.stack([p0, c0])).to(device=dev, dtype=dtype)
            extra["pair_points"] = int(p0.size)
            extra["pair_grid"] = list(shape)
            run = lambda: obj.step_with_pair(state, pair_state, c["inner"])
        if c.get("schedule") == "persistent":
            obj.set_schedule("persistent", threads=int(os.environ.get("PFC_BENCH_PB_THREADS", "256")),
                             onchip_smem_max=int(os.environ.get("PFC_BENCH_PB_ONCHIP", "0")),
                             onchip_block_share=float(os.environ.get("PFC_BENCH_PB_SHARE", "-1")))
            extra["schedule"] = obj.schedule_info()
        if c.get("autotune") and not args.no_autotune:
            # tiles of every size class chosen by measurement (untimed)
            extra["autotune"] = {"candidates": 6, "trial_steps": 8,
                                 "ms_per_step_sum_of_classes": obj.autotune(6, 8)}
            extra["schedule"] = obj.schedule_info()
        extra["classes"] = [[k[f] for f in ("ny", "nx", "members", "Py", "W", "gpc", "threads_line")]
                            for k in obj.info()]
        extra["classes_fields"] = ["ny", "nx", "members", "Py", "W", "gpc", "threads_line"]
    elif c["kind"] == "pair":
        shape = c["dims"]
        p0 = inputs.uniform_state(shape, -0.25, 0.01, seed=5)
        c0 = inputs.uniform_state(shape, -0.2, 0.01, seed=6)
        ops = [binding.make_op(0, -0.25), binding.make_op(0, -0.25)]
        obj = binding.Plan(shape, DX, c["dt"], ops, precision=prec, coupling=0.1)
        state = torch.from_numpy(np.stack([p0, c0])).to(device=dev, dtype=dtype)
        npts = p0.size
        run = lambda: obj.step(state, c["inner"])
        if c.get("autotune") and not args.no_autotune:
            extra["autotune"] = {"candidates": 6, "trial_steps": 8, "ms_per_step": obj.autotune(6, 8)}
        extra["plan"] = obj.info()
    elif c["kind"] == "hydro":
        shape = c["dims"]
        obj = binding.Hydro(shape, DX, c["dt"], c["op"], rho=1.0, gamma=1.0, a0=2.0, precision=prec)
        state = torch.from_numpy(inputs.uniform_state(shape, -0.25, 0.1, seed=91)).to(device=dev, dtype=dtype)
        vel = torch.from_numpy(0.05 * np.stack([inputs.uniform_state(shape, 0.0, 1.0, seed=92 + j)
                                                 for j in range(3)])).to(device=dev, dtype=dtype)
        npts = state.numel()
        run = lambda: obj.step(state, vel, c["inner"])
    elif c["kind"] == "apfc":
        shape = c["dims"]
        kv = inputs.apfc_bcc(1.0)
        obj = binding.Apfc(shape, 1.1, c["dt"], c["op"], kv, -0.2, precision=prec)
        g = torch.Generator(device=dev)
        g.manual_seed(9)
        re = 0.1 + 0.02 * (2 * torch.rand((len(kv),) + tuple(shape), generator=g, device=dev) - 1)
        im = 0.02 * (2 * torch.rand((len(kv),) + tuple(shape), generator=g, device=dev) - 1)
        state = torch.complex(re, im).to(torch.complex64 if prec == "fp32" else torch.complex128)
        del re, im
        npts = state.numel()
        extra["amplitudes"] = len(kv)
        extra["resonance_terms"] = obj.resonances()
        run = lambda: obj.step(state, c["inner"])
    elif c["kind"] == "largest":
        torch.cuda.empty_cache()
        n = largest_cube(torch.cuda.mem_get_info()[0])
        shape = (n, n, n)
        obj = binding.Plan(shape, DX, c["dt"], [binding.make_op(*c["op"])], precision=prec)
        state = seeded_uniform_state(shape, -0.25, 0.01, 8, dtype, dev)
        npts = state.numel()
        extra["plan"] = obj.info()
        extra["grid"] = list(shape)
        extra["chosen_from_free_bytes"] = True
        run = lambda: obj.step(state, c["inner"])
    else:
        shape = c["dims"]
        seed = {"1": 1, "3": 3, "3d64": 3}.get(args.config, 6)
        mean, amp = {"1": (-0.25, 0.01), "3": (-0.35, 0.02), "3d64": (-0.35, 0.02)}.get(args.config, (-0.25, 0.01))
        obj = binding.Plan(shape, DX, c["dt"], [binding.make_op(*c["op"])], precision=prec)
        if c.get("device_draw"):
            state = seeded_uniform_state(shape, mean, amp, 8, dtype, dev)
        else:
            state = torch.from_numpy(inputs.uniform_state(shape, mean, amp, seed=seed)).to(device=dev, dtype=dtype)
        npts = state.numel()
        if args.autotune and c["kind"] == "plan":
            extra["autotune"] = {"candidates": 8, "trial_steps": c["inner"],
                                 "ms_per_step": obj.autotune(8, c["inner"])}
        extra["plan"] = obj.info()
        if c["kind"] == "plan":
            run = lambda: obj.step(state, c["inner"])
        elif c["kind"] == "segment":
            nb = obj.record_bytes(c["inner"])
            rec = torch.empty(nb, dtype=torch.uint8, device=dev)
            lam = torch.ones_like(state) * 1e-3
            dr = torch.zeros(1, dtype=torch.float64, device=dev)
            x = state.clone()
            extra["record_bytes"] = nb

            def run():
                x.copy_(state)
                obj.step_record(x, c["inner"], rec)
                obj.adjoint_segment(rec, c["inner"], lam, dr)
        else:
            lam = state.clone()
            lam_out = torch.empty_like(state)
            dr = torch.zeros(1, dtype=torch.float64, device=dev)

            def run():
                for _ in range(c["inner"]):
                    obj.step_adjoint(state, lam, lam_out, dr)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
    steps = args.steps * c["inner"]
    value = npts * steps / (total * 1e-3)
    bpp = c["sweeps"] * vb       # bytes per grid point per step (a half spectrum ~ N/2 complex)
    step_bytes = bpp * npts
    if "pair_points" in extra:
        # the pair: 10 sweeps a step (row pass 2 x 2 fields, line pass reads 4 arrays, writes 2)
        step_bytes += 10 * vb * extra["pair_points"]
        npts += extra["pair_points"]
        bpp = step_bytes / npts
    peak, peak_kind = hbm_peak()
    gbs = step_bytes * steps / (total * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
            "data": "synthetic", "config": {"workload": c["desc"], "id": args.config, "points": npts,
                                            "time_steps_per_step": c["inner"],
                                            "l2": "512 MiB buffer written between timed steps", **extra},
            "roofline": {"bound": "hbm", "model_bytes_per_point_step": bpp, "achieved": gbs, "peak": peak,
                         "unit": "GB/s", "frac": gbs / peak, "peak_kind": peak_kind, "traffic": None},
            "clocks": clk.summary()}
    if c["kind"] in ("plan", "largest"):
        prof, _ = obj.profile_steps(state, c["inner"])
        line["roofline"]["per_kernel_ms_per_step"] = {k: prof[k] / c["inner"] for k in ("row", "line", "mid")}
    print(json.dumps(line), flush=True)


def seeded_uniform_state(shape, mean, amp, seed, dtype, dev):
    """mean + U[-amp, amp] drawn on the device by a seeded torch generator (for grids too large to
    draw on the host)."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x = torch.empty(shape, dtype=dtype, device=dev)
    x.uniform_(mean - amp, mean + amp, generator=g)
    return x


def time_plan(torch, plan, state, inner, steps, warmup, flush):
    """ms per time step of plan.step(state, inner), L2 flushed between timed calls, CUDA events."""
    for _ in range(warmup):
        plan.step(state, inner)
    torch.cuda.synchronize()
    total = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        flush.fill_(1.0)
        e0.record()
        plan.step(state, inner)
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    return total / (steps * inner)


def other_grids(torch, dev, flush):
    """Rates of the 512^3 two-mode grid (FP32-mixed, two-pass) and of the largest FP32 cube that
    fits the free memory (three-pass), with per-kernel times and HBM fractions."""
    from paper_2603_26818_gb300 import binding, inputs
    peak, _ = hbm_peak()
    out = {}
    two = binding.make_op(1, -0.3, 0.05, math.sqrt(4.0 / 3.0))
    psi0 = inputs.uniform_state((512, 512, 512), -0.35, 0.02, seed=3)
    p = binding.Plan((512, 512, 512), DX, 0.1, [two], precision="fp32")
    x = torch.from_numpy(psi0).to(device=dev, dtype=torch.float32)
    ms = time_plan(torch, p, x, 10, 5, 3, flush)
    prof, _ = p.profile_steps(x, 10)
    npts = 512 ** 3
    half = 512 * 512 * 257 * 8
    out["512cube_two_mode_fp32"] = {
        "grid_point_steps_per_s": npts / (ms * 1e-3), "ms_per_time_step": ms, "plan": p.info(),
        "hbm_frac_at_20_B_per_pt": 20 * npts / (ms * 1e-3) / 1e9 / peak,
        "per_kernel_ms_per_step": {k: prof[k] / 10 for k in ("row", "line")},
        "per_kernel_frac": {"row": 2 * half / (prof["row"] / 10 * 1e-3) / 1e9 / peak,
                            "line": 3 * half / (prof["line"] / 10 * 1e-3) / 1e9 / peak}}
    p.close()
    del x
    torch.cuda.empty_cache()
    n = largest_cube(torch.cuda.mem_get_info()[0])
    shape = (n, n, n)
    p = binding.Plan(shape, DX, 0.5, [binding.make_op(0, -0.25)], precision="fp32")
    x = seeded_uniform_state(shape, -0.25, 0.01, 8, torch.float32, dev)
    ms = time_plan(torch, p, x, 3, 3, 2, flush)
    prof, _ = p.profile_steps(x, 3)
    info = p.info()
    npts = n ** 3
    sweeps = 9 if info["Ry"] * info["Rz"] > 1 else 5
    half = n * n * (n // 2 + 1) * 8
    out["largest_cube_fp32"] = {
        "grid": [n, n, n], "grid_point_steps_per_s": npts / (ms * 1e-3), "ms_per_time_step": ms,
        "plan": info, "sweeps_per_step": sweeps,
        "hbm_frac_at_model_bytes": sweeps * 4 * npts / (ms * 1e-3) / 1e9 / peak,
        "per_kernel_ms_per_step": {k: prof[k] / 3 for k in ("row", "line", "mid")},
        "per_kernel_frac": {"row": 2 * half / (prof["row"] / 3 * 1e-3) / 1e9 / peak,
                            "line": 3 * half / (prof["line"] / 3 * 1e-3) / 1e9 / peak,
                            "mid": 4 * half / max(prof["mid"] / 3 * 1e-3, 1e-12) / 1e9 / peak},
        "state": "psi0 = -0.25 + U[-0.01, 0.01] from a seeded torch generator (seed 8)"}
    p.close()
    del x
    torch.cuda.empty_cache()
    return out


def other_workloads(torch, dev, flush):
    """Rates of the other rows at their bench sizes, short timings (same discipline): the
    1024-domain ensemble on the graph and the persistent schedule, the paper's 750^3 grid
    (mixed radix) and the amplitude-expansion BCC set at 256^3."""
    import numpy as np
    from paper_2603_26818_gb300 import binding, inputs
    peak, _ = hbm_peak()
    out = {}
    draws = inputs.batch_draws(1024, seed=4)
    parts = [inputs.uniform_state((ny, nx), m, 0.01, seed=1000 + i).ravel() for i, (ny, nx, r, m) in enumerate(draws)]
    x0 = torch.from_numpy(np.concatenate(parts)).to(device=dev, dtype=torch.float32)
    for sched in ("graph", "persistent"):
        b = binding.Batch([(d[0], d[1]) for d in draws], [d[2] for d in draws], DX, 0.5, precision="fp32")
        if sched == "persistent":
            b.set_schedule("persistent", threads=256)
        x = x0.clone()
        ms = time_plan(torch, b, x, 20, 3, 2, flush)
        out[f"batch_1024_domains_{sched}"] = {
            "grid_point_steps_per_s": x.numel() / (ms * 1e-3), "ms_per_time_step": ms,
            "hbm_frac_at_20_B_per_pt": 20 * x.numel() / (ms * 1e-3) / 1e9 / peak,
            "tiles": "planner" if sched == "graph" else b.schedule_info()}
        b.close()
        del x
    del x0
    torch.cuda.empty_cache()
    shape = (750, 750, 750)
    p = binding.Plan(shape, DX, 0.5, [binding.make_op(0, -0.25)], precision="fp32")
    x = seeded_uniform_state(shape, -0.25, 0.01, 8, torch.float32, dev)
    ms = time_plan(torch, p, x, 4, 2, 2, flush)
    npts = 750 ** 3
    out["mixed_radix_750cube_fp32"] = {"grid_point_steps_per_s": npts / (ms * 1e-3), "ms_per_time_step": ms,
                                       "hbm_frac_at_44_B_per_pt": 44 * npts / (ms * 1e-3) / 1e9 / peak}
    p.close()
    del x
    torch.cuda.empty_cache()
    shape = (256, 256, 256)
    kv = inputs.apfc_bcc(1.0)
    a = binding.Apfc(shape, 1.1, 0.4, (0, -0.25, 0.0, 0.0), kv, -0.2, precision="fp32")
    g = torch.Generator(device=dev)
    g.manual_seed(9)
    re = 0.1 + 0.02 * (2 * torch.rand((6,) + shape, generator=g, device=dev) - 1)
    im = 0.02 * (2 * torch.rand((6,) + shape, generator=g, device=dev) - 1)
    eta = torch.complex(re, im)
    del re, im
    ms = time_plan(torch, a, eta, 10, 3, 2, flush)
    npts = eta.numel()
    out["apfc_bcc6_256cube_fp32"] = {"amplitude_point_steps_per_s": npts / (ms * 1e-3), "ms_per_time_step": ms,
                                     "hbm_frac_at_88_B_per_amplitude_point": 88 * npts / (ms * 1e-3) / 1e9 / peak}
    a.close()
    del eta
    torch.cuda.empty_cache()
    return out


def precision_report(torch, dev):
    """FP32-mixed against the FP64 path, per workload: relative L2 errors after each workload's
    full length (the FP64 paths are pinned to the oracle by the test suite). Both runs start from
    the same FP32-representable state, so the figure is the FP32 path's arithmetic; where the
    workload's own FP64 draws differ visibly from their FP32 rounding (small fluctuations about a
    large mean, linearly unstable), the error against the FP64 draws is reported beside it."""
    import numpy as np
    from paper_2603_26818_gb300 import binding, inputs
    from paper_2603_26818_gb300.autograd import rollout
    out = {}

    def relerr(a, b):
        return float((a.double() - b.double()).norm() / b.double().norm())

    # 512^3 two-mode, 500 steps (the FP64 plan is three-pass)
    two = binding.make_op(1, -0.3, 0.05, math.sqrt(4.0 / 3.0))
    psi0 = inputs.uniform_state((512, 512, 512), -0.35, 0.02, seed=3)
    res = {}
    x0 = torch.from_numpy(psi0).to(device=dev, dtype=torch.float32)
    for prec in ("fp64", "fp32"):
        p = binding.Plan((512, 512, 512), DX, 0.1, [two], precision=prec)
        x = x0.double() if prec == "fp64" else x0.clone()
        p.step(x, 500)
        res[prec] = (x, p.mass(x)[0])
        p.close()
    a, b = res["fp32"][0], res["fp64"][0]
    m0 = float(psi0.astype(np.float32).astype(np.float64).mean())
    out["3_512cube_two_mode_500_steps"] = {
        "rel_l2_fp32_vs_fp64": relerr(a, b),
        "rel_l2_of_fluctuation": float((a.double() - b).norm() / (b - b.mean()).norm()),
        "mass_drift_rel_fp32": abs(res["fp32"][1] - m0) / abs(m0)}
    del res, a, b
    torch.cuda.empty_cache()
    # 1024-domain ensemble, 200 steps, every domain; coupled pair 256^3, 200 steps
    draws = inputs.batch_draws(1024, seed=4)
    parts = np.concatenate([inputs.uniform_state((ny, nx), m, 0.01, seed=1000 + i).ravel()
                            for i, (ny, nx, r, m) in enumerate(draws)])
    b32 = binding.Batch([(d[0], d[1]) for d in draws], [d[2] for d in draws], DX, 0.5, precision="fp32")
    b64 = binding.Batch([(d[0], d[1]) for d in draws], [d[2] for d in draws], DX, 0.5, precision="fp64")
    x = torch.from_numpy(parts).to(device=dev, dtype=torch.float32)
    y = x.double()
    yin = torch.from_numpy(parts).to(device=dev)
    for bt, z in ((b32, x), (b64, y), (b64, yin)):
        bt.step(z, 200)
    errs = np.array([relerr(b32.view(x, d), b64.view(y, d)) for d in range(len(draws))])
    errs_in = np.array([relerr(b32.view(x, d), b64.view(yin, d)) for d in range(len(draws))])
    b32.close()
    b64.close()
    out["4a_ensemble_1024_domains_200_steps"] = {
        "rel_l2_max_over_domains": float(errs.max()), "rel_l2_median": float(np.median(errs)),
        "domains_above_1e-5": int((errs > 1e-5).sum()),
        "against_fp64_draws": {"rel_l2_max_over_domains": float(errs_in.max()),
                               "domains_above_1e-5": int((errs_in > 1e-5).sum())}}
    p0 = inputs.uniform_state((256, 256, 256), -0.25, 0.01, seed=5)
    c0 = inputs.uniform_state((256, 256, 256), -0.2, 0.01, seed=6)
    ops = [binding.make_op(0, -0.25), binding.make_op(0, -0.25)]
    xs = {}
    x0 = torch.from_numpy(np.stack([p0, c0])).to(device=dev, dtype=torch.float32)
    for prec in ("fp64", "fp32"):
        p = binding.Plan((256, 256, 256), DX, 0.5, ops, precision=prec, coupling=0.1)
        x = x0.double() if prec == "fp64" else x0.clone()
        p.step(x, 200)
        xs[prec] = x
        p.close()
    out["4b_coupled_pair_256cube_200_steps"] = {
        "rel_l2_psi": relerr(xs["fp32"][0], xs["fp64"][0]), "rel_l2_c": relerr(xs["fp32"][1], xs["fp64"][1])}
    del xs
    # adjoint: 256^3 one-mode, 200 steps, checkpoints every 20, gradients FP32 vs FP64
    shape = (256, 256, 256)
    psi0 = inputs.uniform_state(shape, -0.25, 0.01, seed=6).astype(np.float32).astype(np.float64)
    p = binding.Plan(shape, DX, 0.5, [binding.make_op(0, -0.25)], precision="fp64")
    p.set_r(-0.2)
    tg64 = torch.from_numpy(psi0).to(device=dev)
    p.step(tg64, 200)
    p.close()
    tg64 = tg64.float().double()   # one target for both precisions
    grads = {}
    for prec, dt_ in (("fp64", torch.float64), ("fp32", torch.float32)):
        p = binding.Plan(shape, DX, 0.5, [binding.make_op(0, -0.25)], precision=prec)
        tg = tg64.to(dt_)
        x0 = torch.from_numpy(psi0).to(device=dev, dtype=dt_).requires_grad_(True)
        rt = torch.tensor(-0.25, dtype=torch.float64, requires_grad=True)
        loss = 0.5 * ((rollout(x0, rt, p, 200, 20) - tg) ** 2).sum()
        loss.backward()
        grads[prec] = (x0.grad.detach(), float(rt.grad))
        p.close()
    out["5_adjoint_256cube_200_steps"] = {
        "rel_l2_grad_psi0": relerr(grads["fp32"][0], grads["fp64"][0]),
        "rel_err_grad_r": abs(grads["fp32"][1] - grads["fp64"][1]) / abs(grads["fp64"][1])}
    return out


def make_input():
    from paper_2603_26818_gb300 import inputs
    return inputs.polycrystal_2d(NY, NX, DX, MEAN, 64, 0.2, 1.0, 0.01, seed=2)


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            # start the timed region only once sampling runs (nvidia-smi takes a moment to start)
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.f.name) == 0 and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------- peaks
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# device code of the two kernels whose counters the roofline quotes (k_row_cube_cl and
# k_line_v2): the headers they are compiled from. Other kernels, the host code that launches
# them and the instantiation units do not enter; the tiling a counter was taken on is checked
# separately (ncu_traffic).
KERNEL_HEADERS = ("pfc_fft.cuh", "pfc_pass.cuh", "pfc_row_cluster.cuh", "pfc_line_v2.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2603_26818_gb300", "csrc")
    for n in KERNEL_HEADERS:
        h.update(open(os.path.join(csrc, n), "rb").read())
    return h.hexdigest()[:16]


def kernel_names(info):
    """Names (as ncu prints them, without arguments) of the row and line kernels a FP32 plan runs."""
    row = "k_row_cube_cl<float, 2, 11>" if info.get("row_cluster") == 2 else "k_row<float, ROW_CUBE>"
    ly = info["Qy"].bit_length() - 1
    if info["W"] >= 2 and info["threads_line"] >= 64:   # the two-column update pass
        line = f"k_line_v2<512, {ly}, 0>" if info["Qz"] == 1 and ly in (8, 9, 10) else "k_line_v2<512>"
    else:
        fixed = info["Qz"] == 1 and info["threads_line"] <= 512 and 6 <= ly <= 10
        line = f"k_line<float, LINE_STEP, 512, {ly}, 0>" if fixed else "k_line<float, LINE_STEP>"
    return {"row": row, "line": line}


def ncu_traffic(kernel_key, plan_info=None):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel
    source and (when the summary records it) on the same tiling as plan_info."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        t = json.load(f)
    if t.get("source_hash") != kernel_source_hash():
        return None
    k = t.get("kernels", {}).get(kernel_key)
    if k is None:
        return None
    if plan_info is not None and "plan" in k:
        if any(plan_info.get(f) != v for f, v in k["plan"].items()):
            return None
    return k.get("dram_bytes_per_launch_full_size")


# ------------------------------------------------------------------------------- oracle
def cpu_baseline(psi0, nsteps):
    import oracle
    t0 = time.perf_counter()
    oracle.step(psi0, DX, DT, (0, R_OP, 0.0, 0.0), nsteps)
    dt = time.perf_counter() - t0
    return {"value": NY * NX * nsteps / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{nsteps} time steps of the 4096x4096 workload, FP64 C oracle (own FFT, "
                      f"OpenMP over lines), {dt:.1f} s"}


def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return
    import oracle
    oracle.build()
    psi = make_input()
    for _ in range(args.warmup):
        psi = oracle.step(psi, DX, DT, (0, R_OP, 0.0, 0.0), 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi = oracle.step(psi, DX, DT, (0, R_OP, 0.0, 0.0), 1)
    el = time.perf_counter() - t0
    v = NY * NX * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD.replace(f"{INNER} semi-implicit time steps per bench step; FP32-mixed",
                                                    "1 time step per bench step; FP64 CPU oracle"),
                       "grid": [NY, NX], "time_steps_per_step": 1},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} timed time steps of the 4096x4096 workload"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------- ours
def replica_throughput(dist, local_ms, world, work_per_rank, device):
    """Max over ranks of the timed milliseconds, and the whole-job rate: the work of all ranks
    (independent replicas) divided by that slowest time. dist is torch.distributed or None."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * work_per_rank / (ms_max * 1e-3)


def fma_peaks():
    """Measured plain-FMA rates of this GPU (libpfc_probe.so), TFLOP/s, or None."""
    try:
        lib = ctypes.CDLL(os.path.join(ROOT, "paper_2603_26818_gb300", "libpfc_probe.so"))
    except OSError:
        return None
    out = {}
    for name, fp64 in (("fp32_tflops", 0), ("fp64_tflops", 1)):
        v = ctypes.c_double()
        if lib.pfcp_fma_peak(fp64, ctypes.byref(v)) != 0:
            return None
        out[name] = v.value / 1e12
    return out


def time_cufft(torch, dev, psi0, precision, nsteps):
    """Vendor cuFFT plain step (baseline library), grid-point-steps/s."""
    import ctypes
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2603_26818_gb300", "libpfc_cufft_baseline.so"))
    lib.pfcb_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    lib.pfcb_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    lib.pfcb_destroy.argtypes = [ctypes.c_void_p]
    dt = torch.float64 if precision == 0 else torch.float32
    x = torch.from_numpy(psi0).to(device=dev, dtype=dt)
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 2)(NY, NX)
    st = torch.cuda.current_stream().cuda_stream
    if lib.pfcb_create(ctypes.byref(h), 2, dims, DX, DT, 0, R_OP, 0.0, 0.0, precision, ctypes.c_void_p(st)) != 0:
        return None, None
    lib.pfcb_step(h, ctypes.c_void_p(x.data_ptr()), 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lib.pfcb_step(h, ctypes.c_void_p(x.data_ptr()), nsteps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lib.pfcb_destroy(h)
    return NY * NX * nsteps / (ms * 1e-3), x


def run_ours(args):
    import numpy as np
    import torch
    from paper_2603_26818_gb300 import binding

    rank, local, world = env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    psi0 = make_input()
    op = binding.make_op(0, R_OP)
    plan = binding.Plan((NY, NX), DX, DT, [op], precision="fp32")
    tuned_ms = plan.autotune(8, INNER) if args.autotune else None
    state = torch.from_numpy(psi0).to(device=dev, dtype=torch.float32)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    npts = NY * NX

    for _ in range(args.warmup):
        plan.step(state, INNER)
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM, L2 flushed between timed steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(1.0)
            evs[k][0].record()
            plan.step(state, INNER)
            evs[k][1].record()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        # ---- end to end through the public API with host buffers (pinned), copies timed
        # (inside the clock sampling window too)
        h_in = torch.from_numpy(psi0.astype(np.float32)).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        d = torch.empty_like(state)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record()
        for k in range(args.steps):
            d.copy_(h_in, non_blocking=True)
            plan.step(d, INNER)
            h_out.copy_(d, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    ms_max, value = replica_throughput(dist, ms, world, npts * INNER * args.steps, dev)
    launches_per_call = 2 * 1 + 1 + 2 * INNER + 1
    _, e2e_value = replica_throughput(dist, e0.elapsed_time(e1), world, npts * INNER * args.steps, dev)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": h_in.numel() * 4, "d2h_bytes_per_step": h_out.numel() * 4}

    # ---- per-kernel timing with events between launches on the plan's stream
    prof, nl = plan.profile_steps(state, INNER)
    H = NY * (NX // 2 + 1)
    alg = {"row": 2 * 8 * H, "line": 3 * 8 * H}          # bytes per launch: 2 and 3 sweeps
    dom = max(("row", "line"), key=lambda k: prof[k])
    dur = prof[dom] * 1e-3 / INNER
    peak, peak_kind = hbm_peak()
    achieved = alg[dom] / dur / 1e9
    key = kernel_names(plan.info())[dom]
    roof = {"bound": "hbm", "kernel": key, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": ncu_traffic(key, plan.info()),
            "algorithmic_bytes_per_launch": alg[dom], "avg_launch_ms": dur * 1e3,
            "per_kernel_ms_per_step": {k: prof[k] / INNER for k in ("row", "line")},
            "per_kernel_gbs": {k: alg[k] / (prof[k] * 1e-3 / INNER) / 1e9 for k in ("row", "line")},
            "step_gbs_at_20_B_per_pt": 20 * npts * INNER / (ms_max * 1e-3 / args.steps) / 1e9}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [NY, NX], "time_steps_per_step": INNER,
                       "precision": "fp32-mixed", "parallelism": f"replicas{world}",
                       "l2": "512 MiB buffer written between timed steps",
                       "plan": plan.info(),
                       "tiles": ({"autotuned": True, "ms_per_step": tuned_ms} if args.autotune
                                 else "planner")},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches_per_call * args.steps,
            "clocks": clk.summary()}

    if not args.no_extras and rank == 0:
        extras = {}
        # our FP64 path and the vendor plain steps, for context (same workload, fewer steps)
        p64 = binding.Plan((NY, NX), DX, DT, [op], precision="fp64")
        x64 = torch.from_numpy(psi0).to(device=dev)
        p64.step(x64, 2)
        torch.cuda.synchronize()
        e0.record()
        p64.step(x64, 20)
        e1.record()
        torch.cuda.synchronize()
        extras["ours_fp64"] = npts * 20 / (e0.elapsed_time(e1) * 1e-3)
        v, _ = time_cufft(torch, dev, psi0, 0, 20)
        extras["cufft_plain_fp64"] = v
        v, _ = time_cufft(torch, dev, psi0, 1, 100)
        extras["cufft_plain_fp32"] = v
        extras["speedup_vs_plain_fp64"] = value / world / extras["cufft_plain_fp64"] if extras["cufft_plain_fp64"] else None
        # precision report: FP32-mixed vs our FP64 path after 1000 steps from psi0
        a = torch.from_numpy(psi0).to(device=dev, dtype=torch.float32)
        b = a.double()                      # the same FP32-representable start
        bin_ = torch.from_numpy(psi0).to(device=dev)   # the FP64 draws
        m0 = float(b.mean())
        plan.step(a, 1000)
        p64.step(b, 1000)
        p64.step(bin_, 1000)
        torch.cuda.synchronize()
        diff = (a.double() - b).norm() / b.norm()
        fl = (b - b.mean()).norm()
        extras["precision_1000_steps"] = {
            "rel_l2_fp32_vs_fp64": float(diff),
            "rel_l2_of_fluctuation": float((a.double() - b).norm() / fl),
            "rel_l2_against_fp64_draws": float((a.double() - bin_).norm() / bin_.norm()),
            "mass_drift_rel_fp32": abs(plan.mass(a)[0] - m0) / abs(m0),
            "mass_drift_rel_fp64": abs(p64.mass(b)[0] - m0) / abs(m0)}
        del a, b, bin_, x64
        p64.close()
        torch.cuda.empty_cache()
        # the other grids' rates (512^3, the largest cube that fits) and the other workloads'
        # FP32-mixed precision
        extras["other_grids"] = other_grids(torch, dev, flush)
        extras["other_workloads"] = other_workloads(torch, dev, flush)
        extras["precision_per_config"] = {"2_4096sq_polycrystal_1000_steps": extras["precision_1000_steps"],
                                          **precision_report(torch, dev)}
        # ALU view: the transform flops of a step (5 log2 N per point for one r2c and one c2r,
        # plus ~20 pointwise) against the measured plain-FMA rates; the FP64 path is bound there
        peaks = fma_peaks()
        if peaks:
            fpp = 5 * math.log2(npts) + 20
            extras["alu"] = {
                "flops_per_point_step": fpp,
                "fp32_path_tflops": value / world * fpp / 1e12, "fp32_fma_peak_tflops": peaks["fp32_tflops"],
                "fp32_frac": value / world * fpp / 1e12 / peaks["fp32_tflops"],
                "fp64_path_tflops": extras["ours_fp64"] * fpp / 1e12, "fp64_fma_peak_tflops": peaks["fp64_tflops"],
                "fp64_frac": extras["ours_fp64"] * fpp / 1e12 / peaks["fp64_tflops"],
                "peak_kind": "measured (libpfc_probe.so: 8 independent FMA chains per thread)"}
        line["context"] = extras

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(psi0, 32)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.config is not None:
        return run_config(args)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
