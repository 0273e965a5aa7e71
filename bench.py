"""Benchmark: explicit 2D UGKS steps on the mesh-sweep channel workload (800x400 cells,
28^2 velocities on [-4,4]^2, Kn 0.05), in velocity-cell updates per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--prec fp32f|fp64]

Prints one JSON line (rank 0).  One step = one UGKS step (ghost fill, velocity sums,
interface scalars, W update, f update) over the whole workload.  `value` is timed with
CUDA events on the library's stream with the state resident in HBM (f is 4 GB FP64 /
2 GB FP32, far larger than L2, so no flush is needed); `e2e` goes through the C ABI with
host buffers (pinned): every step copies f and W in, steps, and reads W back.
The plain FP64 path and the FP32-f form (FP32 f, FP64 moments / W / interface scalars)
are both timed; `value` is the form named by --prec and the other is reported beside it.
Multi-GPU: one independent replica per rank (the step does not shard here), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1810_08137_gb300 import inputs as I  # noqa: E402

METRIC = "velocity-cell updates/s per UGKS step"
UNIT = "vc/s"
KERNELS = ("ghost_x", "ghost_y", "sums", "faces", "cells", "update")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 form: FP64 flops per velocity-cell as executed (FMA = 2 flops), from the ncu
# instruction counts of its kernels (DFMA, DMUL, DADD per velocity-cell; the capture in
# profiles/fp64_step_kernels_channel_200x100_v28.md): the update's two passes
# 2 x 58.8 + 25.6 + 12.5, the sums kernel 2 x 43.4 + 13.3 + 18.4.  The peak is measured
# in the run (ugks_fp64_rate: chains of FP64 FMAs on every SM).
FP64_UPDATE_FLOPS_PER_VC = 2 * 58.8 + 25.6 + 12.5
FP64_SUMS_FLOPS_PER_VC = 2 * 43.4 + 13.3 + 18.4
# DRAM traffic of the FP32-f update kernel per velocity-cell (read + write), from the ncu
# capture of the current kernel summarised in profiles/fp32f_step_kernels_channel_400x200_v28.md
# (dram__bytes_read.sum + dram__bytes_write.sum of one kb_strip launch at 400x200x28^2);
# set to None when the kernel changes until it is captured again.
UPDATE_TRAFFIC_PER_VC = (601.562112e6 + 465.784064e6) / 62.72e6
# FP32 lane operations of the FP32-f update kernel per velocity-cell on the FMA pipe (a packed
# pair instruction = 2), from the same capture's instruction mix: FFMA2 43.4, FMUL2 15.0,
# FADD2 6.6, FFMA 5.0, FADD 3.4, FMUL 1.4 per velocity-cell; the peak is the FMA pipe's
# 128 FP32 lanes per SM per clock on 152 SMs at the 2070 MHz maximum clock.
UPDATE_FP32_OPS_PER_VC = 2 * (43.4 + 15.0 + 6.6) + 5.0 + 3.4 + 1.4
FP32_LANE_OPS_PEAK = 152 * 128 * 2.07e9


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 3 + k and r[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "samples": len(sm), "reasons": reasons}


def max_over_ranks(x: float, device) -> float:
    """Maximum of x over the ranks of the default process group (x itself on one rank)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(world_size: int, vc_per_step: int, steps: int, ms: float) -> float:
    """Whole-job throughput: every rank runs its own replica of the workload (weak scaling),
    timed by the slowest rank."""
    return world_size * vc_per_step * steps / (ms * 1e-3)


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_form(ugks, torch, cfg, prec, steps, warmup, stream, prim):
    """Time `steps` device-resident UGKS steps as the library runs them (one CUDA graph
    replay per step), then the same number of steps again with the library's per-kernel
    events (direct launches, one event between kernels) for the kernel breakdown."""
    s = ugks.Solver(cfg, prec, stream=stream.cuda_stream)
    s.init_maxwellian(*prim)
    s.step(warmup)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    s.profile(True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms_prof = e0.elapsed_time(e1)
    kt = s.kernel_times()
    s.profile(False)
    s.sync()
    return s, ms, ms_prof, kt


def e2e_form(ugks, torch, cfg, prec, steps, stream, f_host, W_host):
    """Through the C ABI with host buffers: per step, copy f and W in, step, read W back."""
    s = ugks.Solver(cfg, prec, stream=stream.cuda_stream)
    W_out = np.empty((4, cfg.nc))
    s.set_state(f_host, W_host)  # warm-up of the path
    s.step(1)
    s.moments()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        s.set_state(f_host, W_host)
        s.step(1)
        W_out[:] = s.moments()
    t = time.perf_counter() - t0
    s.close()
    return t


def pinned(torch, shape):
    t = torch.empty(shape, dtype=torch.float64, pin_memory=True)
    return t, t.numpy()


def cpu_baseline(cfg, prim, budget_s=20.0):
    """The FP64 oracle as it stands, all host cores, on whole steps of the same workload."""
    from oracle import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    f, W = oracle.init_maxwellian(cfg, *prim)
    t0 = time.perf_counter()
    n = 0
    while True:
        f, W = oracle.step(cfg, f, W, 1)
        n += 1
        if time.perf_counter() - t0 > budget_s / 2 or n >= 3:
            break
    t = time.perf_counter() - t0
    value = cfg.vc * n / t
    # the same oracle on one thread: one step of a band of rows of the same channel (same
    # velocity grid, Kn, boundaries) sized to about budget_s / 4 of single-thread work
    oracle.set_threads(1)
    per_thread = value / cores
    ny_s = max(2, min(cfg.ny, int(cfg.ny * (budget_s / 4) * per_thread / cfg.vc)))
    sub = cfg.replace(ny=ny_s, ly=cfg.ly * ny_s / cfg.ny)
    sp = [x.reshape(cfg.ny, cfg.nx)[:ny_s].reshape(-1) for x in prim]
    fs, Ws = oracle.init_maxwellian(sub, *sp)
    t0 = time.perf_counter()
    oracle.step(sub, fs, Ws, 1)
    t1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} full step(s) of {cfg.name} ({cfg.vc} vc/step), FP64 C oracle, "
                      f"OpenMP over faces and cells",
            "single_thread": {"value": sub.vc / t1, "unit": UNIT, "cores": 1,
                              "sample": f"1 step of a {sub.nx}x{sub.ny} band of {cfg.name} "
                                        f"({sub.vc} vc)"}}


def large_velocity_bench(ugks, torch, stream, warmup, grids=(51, 101, 151, 201)):
    """Large velocity space (200x100 mesh, N^2 velocities on [-20,20]^2, Kn 0.01): both
    forms per velocity grid, graph-replayed steps timed with CUDA events."""
    out = []
    for n in grids:
        cfg = I.workload_large_velocity(n)
        prim = I.initial_prim(cfg, I.seed_for(3, n))
        row = {"workload": cfg.name, "vc_per_step": cfg.vc}
        for prec, name, steps in ((ugks.FP32F, "fp32f", 10), (ugks.FP64, "fp64", 2)):
            s = ugks.Solver(cfg, prec, stream=stream.cuda_stream)
            s.init_maxwellian(*prim)
            s.step(warmup)
            s.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(steps)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            # per-kernel breakdown from the library's events (direct launches)
            s.profile(True)
            s.step(max(1, steps // 2))
            kt = s.kernel_times()
            s.profile(False)
            s.close()
            torch.cuda.empty_cache()
            row[name] = {"ms_per_step": ms, "value": cfg.vc / (ms * 1e-3), "steps": steps,
                         "kernel_ms_per_step": {k: kt[k][1] / max(kt[k][0], 1) for k in KERNELS}}
        row["fp32f_vs_fp64"] = row["fp32f"]["value"] / row["fp64"]["value"]
        out.append(row)
    return {"unit": UNIT, "grids": out}


def split_bench(ugks, torch, stream, warmup, grids=(101, 201)):
    """Velocity-space split of the FP32-f sums on a small mesh with a large velocity grid
    (the large-velocity channel's grid, [-20,20]^2 and Kn 0.01, on the 40x20 mesh of the
    small channel): the automatic split against one warp per cell, graph-replayed steps."""
    out = []
    for n in grids:
        base = I.workload_large_velocity(n)
        cfg = base.replace(nx=40, ny=20, name=f"channel_40x20_v{n}_r20")
        prim = I.initial_prim(cfg, I.seed_for(3, 1000 + n))
        row = {"workload": cfg.name, "vc_per_step": cfg.vc}
        s = ugks.Solver(cfg, ugks.FP32F, stream=stream.cuda_stream)
        s.init_maxwellian(*prim)
        auto = s.sums_split
        for split in sorted({1, auto}):
            s.set_sums_split(split)
            s.step(warmup)
            s.sync()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            steps = 20
            e0.record(stream)
            s.step(steps)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            s.profile(True)
            s.step(10)
            kt = s.kernel_times()
            s.profile(False)
            row[f"split{split}"] = {"ms_per_step": ms, "value": cfg.vc / (ms * 1e-3),
                                    "sums_ms": kt["sums"][1] / max(kt["sums"][0], 1)}
        s.close()
        row["auto_split"] = auto
        row["speedup"] = row["split1"]["ms_per_step"] / row[f"split{auto}"]["ms_per_step"]
        out.append(row)
    return {"unit": UNIT, "grids": out}


def shakhov_bench(ugks, torch, stream, cfg, prim, warmup, steps=10):
    """The Shakhov model (Pr = 2/3) on the bench workload: FP32-f and FP64 step times."""
    shk = cfg.replace(pr=2.0 / 3.0, name=cfg.name + "_pr0.667")
    out = {"workload": shk.name, "pr": shk.pr, "vc_per_step": shk.vc}
    for prec, name, n in ((ugks.FP32F, "fp32f", steps), (ugks.FP64, "fp64", 2)):
        s = ugks.Solver(shk, prec, stream=stream.cuda_stream)
        s.init_maxwellian(*prim)
        s.step(warmup)
        s.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(n)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        s.profile(True)
        s.step(max(1, n // 2))
        kt = s.kernel_times()
        s.profile(False)
        s.close()
        torch.cuda.empty_cache()
        out[name] = {"ms_per_step": ms, "value": shk.vc / (ms * 1e-3), "steps": n,
                     "kernel_ms_per_step": {k: kt[k][1] / max(kt[k][0], 1) for k in KERNELS}}
    return out


def batch_bench(ugks, torch, stream, steps, warmup):
    """Uneven batch: 64 channel instances drawn log-uniform (meshes 50x25..400x200,
    16^2..64^2 velocities, Kn 1e-3..1, inlet rho 1.05..1.5), FP32-f, stepped together;
    tile shapes from the autotuner; throughput over all instances."""
    cfgs = I.workload_batch(64)
    B = ugks.Batch(64, 150 * 2**30, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    slots = []
    for k, c in enumerate(cfgs):
        s = B.admit(c)
        B.instance(s).init_maxwellian(*I.initial_prim(c, I.seed_for(4, k)))
        slots.append(s)
    B.sync()
    t_admit = time.perf_counter() - t0
    tuned_ms = B.tune(2)
    # both step modes, same tiles: one persistent launch vs seven phase launches per step
    mode_ms = {}
    tuned_mode = B.persistent
    for mode in (True, False):
        B.set_persistent(mode)
        B.step(2)
        B.sync()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        B.step(5)
        a1.record(stream)
        a1.synchronize()
        mode_ms["persistent" if mode else "phases"] = a0.elapsed_time(a1) / 5
    B.set_persistent(tuned_mode)
    B.step(warmup)
    B.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    B.sync()
    vc = sum(c.vc for c in cfgs)
    rows = sorted({B.walk_rows(s) for s in slots})
    out = {"workload": "batch64: meshes 50x25..400x200, 16^2..64^2 velocities, Kn 1e-3..1, "
                       "inlet rho 1.05..1.5 (log-uniform draws, seeded)",
           "instances": len(cfgs), "vc_per_step": vc, "value": vc * steps / (ms * 1e-3),
           "unit": UNIT, "ms_per_step": ms / steps, "steps": steps, "precision": "fp32f",
           "tuned_walk_rows": rows, "tuned_ms_per_step": tuned_ms,
           "admit_s": t_admit, "device_bytes": B.bytes_used,
           "persistent": B.persistent, "launches_per_step": 1 if B.persistent else 7,
           "ms_per_step_by_mode": mode_ms,
           "tuned_walk_vtile": sorted({B.walk_vtile(s) for s in slots})}
    B.close()
    return out


def serve_bench(ugks, stream, n_req=24, scale="small"):
    """Poisson arrivals (20 req/s) of channel solves drawn as in the batch, each run to a
    residual of 1e-6 or 20000 steps, 150 GB HBM budget, continuous batching.  scale="full":
    the batch's ranges (meshes 50x25..400x200, 16^2..64^2 velocities); scale="small" scales
    meshes and velocity grids down (nx 20..50, 16^2..32^2) so each request reaches steady
    state in seconds and the default bench run stays short."""
    from paper_1810_08137_gb300 import serve
    cfgs, arr, prims = I.workload_serving(n_req, scale=scale)
    reqs = serve.make_requests(cfgs, arr, prims)
    srv = serve.gpu_server(150 * 2**30, 64, stream=stream.cuda_stream, tol=1e-6,
                           max_steps=20000, check_every=50)
    st = srv.run(reqs)
    srv.batch_handle.close()
    s = st.summary()
    ranges = "nx 50..400, 16^2..64^2" if scale == "full" else "nx 20..50, 16^2..32^2"
    s.update({"workload": f"{n_req} requests, Poisson 20/s, {ranges} velocities, "
                          "Kn 1e-3..1, residual 1e-6 or 20000 steps, 150 GB budget",
              "unit": "s (time to steady state)", "vc_unit": UNIT,
              "steps_per_request": [r.steps for r in st.requests],
              "vc_per_request_step": [r.cfg.vc for r in st.requests]})
    return s


def reference_arm(args, cfg, prim):
    ws, rank, _ = dist()
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    # bounded sample per step: a band of rows of the same channel (same velocity grid,
    # Kn, boundaries), sized so warmup + steps stay within ~2-3 minutes
    f, W = oracle.init_maxwellian(cfg, *prim)
    t0 = time.perf_counter()
    oracle.step(cfg, f, W, 1)
    t_full = time.perf_counter() - t0
    total = max(1, args.steps + args.warmup)
    frac = min(1.0, 150.0 / (total * t_full))
    ny_s = max(2, int(cfg.ny * frac))
    sub = cfg.replace(ny=ny_s, ly=cfg.ly * ny_s / cfg.ny)
    sp = [x.reshape(cfg.ny, cfg.nx)[:ny_s].reshape(-1) for x in prim]
    fs, Ws = oracle.init_maxwellian(sub, *sp)
    fs, Ws = oracle.step(sub, fs, Ws, args.warmup)
    t0 = time.perf_counter()
    fs, Ws = oracle.step(sub, fs, Ws, args.steps)
    t = time.perf_counter() - t0
    value = sub.vc * args.steps / t
    sample = (f"{sub.nx}x{sub.ny} band of {cfg.name} (same velocity grid, Kn, boundaries; "
              f"{sub.vc} vc/step), {args.steps} timed steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": cfg.name},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--prec", default="fp32f", choices=["fp32f", "fp64"])
    ap.add_argument("--mesh", type=int, default=800, help="nx of the mesh sweep (ny = nx/2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-large-velocity", action="store_true")
    ap.add_argument("--serve-full", action="store_true",
                    help="only the request-serving workload at full request sizes (64 requests "
                         "drawn as in the uneven batch); prints its own JSON line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    cfg = I.workload_mesh_sweep(args.mesh)
    prim = I.initial_prim(cfg, I.seed_for(2, args.mesh))
    if args.impl == "reference":
        reference_arm(args, cfg, prim)
        return

    import torch
    from paper_1810_08137_gb300 import build, ugks
    ws, rank, local = dist()
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.Stream()
    hbm, hbm_src = peaks()
    main_prec = ugks.FP32F if args.prec == "fp32f" else ugks.FP64
    other_prec = ugks.FP64 if main_prec == ugks.FP32F else ugks.FP32F

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()


    if args.serve_full:
        with torch.cuda.stream(stream):
            with Clocks(local) as clk:
                sv = serve_bench(ugks, stream, n_req=64, scale="full")
        print(json.dumps({"metric": "time to steady state (serving, continuous batching)",
                          "value": sv["p50_s"], "unit": "s", "p99_s": sv["p99_s"],
                          "higher_is_better": False, "n_gpus": 1, "dtype": "f32 (f) + f64",
                          "data": "synthetic", "config": {"workload": sv["workload"]},
                          "serving": sv, "clocks": clk.summary()}), flush=True)
        return

    results = {}
    with torch.cuda.stream(stream):
        fp64_peak = ugks.fp64_rate(stream.cuda_stream)
        for prec in (other_prec, ugks.DF64, main_prec):
            # the FP64-accurate forms are slower per step: time fewer of their steps
            n = args.steps if prec == main_prec else max(3, min(args.steps, 10))
            barrier()
            with Clocks(local) as clk:
                s, ms, ms_prof, kt = run_form(ugks, torch, cfg, prec, n, args.warmup, stream, prim)
            barrier()
            ms = max_over_ranks(ms, "cuda")
            results[prec] = (ms, ms_prof, kt, clk.summary(), n)
            if prec == main_prec:
                f_host_t, f_host = pinned(torch, (cfg.nc, cfg.nq, 2))
                W_host_t, W_host = pinned(torch, (4, cfg.nc))
                fd = torch.empty((cfg.nc, cfg.nq, 2), dtype=torch.float64, device="cuda")
                Wd = torch.empty((4, cfg.nc), dtype=torch.float64, device="cuda")
                s.get_state_device(fd, Wd)
                s.sync()
                f_host_t.copy_(fd)
                W_host_t.copy_(Wd)
                del fd, Wd
            s.close()
            torch.cuda.empty_cache()
        barrier()
        t_e2e = e2e_form(ugks, torch, cfg, main_prec, args.e2e_steps, stream, f_host, W_host)
        t_e2e = max_over_ranks(t_e2e, "cuda")
        del f_host_t, W_host_t, f_host, W_host
        batch = None if args.no_batch else batch_bench(ugks, torch, stream, args.steps, args.warmup)
        large = None if args.no_large_velocity else large_velocity_bench(ugks, torch, stream, args.warmup)
        split = None if args.no_large_velocity else split_bench(ugks, torch, stream, args.warmup)
        shakhov = None if args.no_large_velocity else shakhov_bench(ugks, torch, stream, cfg, prim,
                                                                     args.warmup)
        serving = None if (args.no_serve or ws > 1) else serve_bench(ugks, stream)

    def form_json(prec):
        ms, ms_prof, kt, clk, n = results[prec]
        bpv = 8 if prec == ugks.FP32F else 16  # bytes per velocity-cell of f (h, b)
        if prec == ugks.DF64:
            n_up, t_up = kt["update"]
            n_sm, t_sm = kt["sums"]
            ach_up = 2 * bpv * cfg.vc / (t_up / n_up * 1e-3) / 1e9
            return {"value": job_value(ws, cfg.vc, n, ms), "ms_per_step": ms / n, "steps": n,
                    "kernel_ms_per_step": {k: kt[k][1] / max(kt[k][0], 1) for k in KERNELS},
                    "roofline": {"bound": "hbm", "kernel": "update", "achieved": ach_up, "peak": hbm,
                                 "unit": "GB/s", "frac": ach_up / hbm, "traffic": None,
                                 "peak_source": hbm_src, "algorithmic_bytes_per_vc": 2 * bpv},
                    "step_hbm_frac": 2 * bpv * cfg.vc / (ms / n * 1e-3) / 1e9 / hbm,
                    "clocks": clk}
        n_up, t_up = kt["update"]
        n_sm, t_sm = kt["sums"]
        t_launch = t_up / n_up * 1e-3  # seconds per update (FP64 form: its two passes together)
        # algorithmic bytes: update reads f once and writes it once, sums reads f once
        ach_up = 2 * bpv * cfg.vc / t_launch / 1e9
        ach_sm = bpv * cfg.vc / (t_sm / n_sm * 1e-3) / 1e9
        step_bytes = 3 * bpv * cfg.vc
        if prec == ugks.FP32F:
            traffic = None if UPDATE_TRAFFIC_PER_VC is None else UPDATE_TRAFFIC_PER_VC * cfg.vc
            roof = {"bound": "hbm", "kernel": "update", "achieved": ach_up, "peak": hbm,
                    "unit": "GB/s", "frac": ach_up / hbm, "traffic": traffic,
                    "peak_source": hbm_src, "algorithmic_bytes_per_vc": 2 * bpv}
            ops = UPDATE_FP32_OPS_PER_VC * cfg.vc / t_launch
            roof["alu"] = {"bound": "alu (FP32 FMA pipe)", "achieved": ops / 1e12,
                           "peak": FP32_LANE_OPS_PEAK / 1e12, "unit": "T FP32 lane-ops/s",
                           "frac": ops / FP32_LANE_OPS_PEAK, "ops_per_vc": UPDATE_FP32_OPS_PER_VC}
            roof_sums = {"achieved": ach_sm, "frac": ach_sm / hbm, "unit": "GB/s",
                         "algorithmic_bytes_per_vc": bpv}
        else:
            ach = FP64_UPDATE_FLOPS_PER_VC * cfg.vc / t_launch / 1e9
            roof = {"bound": "alu", "kernel": "update", "achieved": ach, "peak": fp64_peak,
                    "unit": "GFLOP/s (FP64)", "frac": ach / fp64_peak, "traffic": None,
                    "peak_source": "measured in this run (ugks_fp64_rate)",
                    "flops_per_vc": FP64_UPDATE_FLOPS_PER_VC, "hbm_frac": ach_up / hbm}
            ach_s = FP64_SUMS_FLOPS_PER_VC * cfg.vc / (t_sm / n_sm * 1e-3) / 1e9
            roof_sums = {"bound": "alu", "achieved": ach_s, "peak": fp64_peak,
                         "unit": "GFLOP/s (FP64)", "frac": ach_s / fp64_peak,
                         "flops_per_vc": FP64_SUMS_FLOPS_PER_VC, "hbm_frac": ach_sm / hbm}
        return {
            "value": job_value(ws, cfg.vc, n, ms),
            "ms_per_step": ms / n,
            "steps": n,
            "ms_per_step_profiled": ms_prof / n,
            "kernel_ms_per_step": {k: kt[k][1] / max(kt[k][0], 1) for k in KERNELS},
            "roofline": roof,
            "roofline_sums": roof_sums,
            "step_hbm_frac": step_bytes / (ms / n * 1e-3) / 1e9 / hbm,
            "clocks": clk,
        }
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    main = form_json(main_prec)
    other = form_json(other_prec)
    dff = form_json(ugks.DF64)
    cpu = None if (args.no_cpu_baseline or ws > 1) else cpu_baseline(cfg, prim)
    h2d = cfg.nc * cfg.nq * 2 * 8 + 4 * cfg.nc * 8
    d2h = 4 * cfg.nc * 8
    line = {
        "metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (f) + f64 (velocity sums across f32 chunks, W, cell scalars) + f64/double-f32 (interface scalars)" if main_prec == ugks.FP32F else "f64",
        "data": "synthetic",
        "config": {"workload": cfg.name, "cells": cfg.nc, "velocities": cfg.nq,
                   "vc_per_step": cfg.vc, "kn": cfg.kn, "precision": args.prec,
                   "l2": "inputs larger than L2 (f >= 2 GB), no flush",
                   "parallelism": f"replicas x{ws}"},
        "roofline": main["roofline"],
        "kernel_ms_per_step": main["kernel_ms_per_step"],
        "roofline_sums": main["roofline_sums"],
        "step_hbm_frac": main["step_hbm_frac"],
        "ms_per_step_profiled": main["ms_per_step_profiled"],
        "other_form": {"precision": "fp64" if other_prec == ugks.FP64 else "fp32f",
                       "value": other["value"], "ms_per_step": other["ms_per_step"],
                       "steps": other["steps"],
                       "kernel_ms_per_step": other["kernel_ms_per_step"],
                       "roofline": other["roofline"], "roofline_sums": other["roofline_sums"],
                       "step_hbm_frac": other["step_hbm_frac"],
                       "clocks": other["clocks"]},
        "df64_form": dict(dff, precision="df64: FP64-accurate, double-FP32 f and per-velocity "
                                          "arithmetic on the FP32 pipe, interface in FP64 / "
                                          "double-FP32, FP64 cell scalars",
                          vs_fp64=dff["value"] / (other["value"] if other_prec == ugks.FP64 else main["value"])),
        "vs_fp64": (main["value"] / other["value"]) if main_prec == ugks.FP32F else 1.0,
        "clocks": main["clocks"],
        "e2e": {"value": ws * cfg.vc * args.e2e_steps / t_e2e, "unit": UNIT,
                "steps": args.e2e_steps, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": 7 * args.steps,  # 6 phase kernels + the buffer flip per step
        "cpu_baseline": cpu,
        "batch": batch,
        "serving": serving,
        "large_velocity": large,
        "sums_split": split,
        "shakhov": shakhov,
    }
    if batch:
        batch["vs_fp64_single"] = batch["value"] / (other["value"] if other_prec == ugks.FP64 else main["value"])
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
