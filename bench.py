"""Throughput benchmark of the T2S2-FDLBM D2Q9 step on GB300.

Workload: Taylor-vortex throughput case on a 4096 x 4096 periodic uniform grid
of [0, 2pi)^2, random-phase sinusoidal initial velocity of amplitude 0.01
(seeded), nu = 0.001, CFL = 0.5, blend 0.1, FP32-deviation storage.  One bench
step = one time step of the whole grid (one launch of the fused kernel).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is the whole-job cell-update rate (MLUPS)
measured with CUDA events on the stream the kernels are launched on, with the
state already resident in HBM.  ``e2e`` is the same metric through the C ABI
with pinned host buffers: initial fields in, K steps, mass/residual and
moments out, all inside the timed region.  With N > 1 (torchrun) every rank
runs an independent replica (the step has no exchange across replicas).
``--impl reference`` times the CPU FP64 oracle on a bounded sample of the same
workload (a 512 x 512 grid) on the host cores.
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
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "D2Q9 T2S2-FDLBM MLUPS & % HBM roofline, FP32 vs FP64; adjoint/forward cost"
N_GRID = 4096
# nu = 0.001 (the Taylor-vortex viscosity of Sec. 3A): with nu = 0.01 the scheme is
# unstable at the 4096^2 spacing (dt/tau = 0.026, nearly collisionless transport).
NU, CFL, BLEND, U0, SEED = 0.001, 0.5, 0.1, 0.01, 2026
BYTES_PER_CELL = {"fp32": 72, "fp64": 144}   # 9 populations read once + written once
# FP64 is bound by the FP64 units, not HBM.  The FP64 fused step executes
# 80.0 M DADD + 60.3 M DMUL + 212.5 M DFMA thread instructions per 1,474,560
# thread-rows (ncu, 1024^2, 9 x 32 CTAs of 128 threads x 40 rows): 383 flop
# per node of sweep work, the algorithmic figure per cell update (the halo
# recompute of a given tiling comes on top).
FP64_FLOP_PER_CELL = 383
FP64_NOMINAL_TFLOPS = 1.25   # GB300 nominal FP64 rate (non-tensor), context only
SAMPLE_N = 512                                # oracle sample grid


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=50)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_GRID)
    p.add_argument("--fp64-steps", type=int, default=100)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--variant", default="auto", choices=["auto", "scalar", "warp"],
                   help="FP32 fused kernel variant for the headline timing")
    p.add_argument("--no-variants", action="store_true", help="skip timing the other variant")
    p.add_argument("--no-batched", action="store_true", help="skip the 64-case batched sweep")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurements")
    p.add_argument("--no-cavity", action="store_true", help="skip the 257^2 cavity march")
    p.add_argument("--no-sweep", action="store_true", help="skip the 512^2..4096^2 size sweep")
    p.add_argument("--rows", type=int, default=0, help="tile height of the fused kernel (0: automatic)")
    p.add_argument("--cavity-steps", type=int, default=0, metavar="K",
                   help="only time K steps of the 257^2 cavity (FP32, fused walls) and print that")
    p.add_argument("--adjoint-cost", type=int, default=0, metavar="N",
                   help="only time adjoint against forward steps on an N^2 grid and print that")
    p.add_argument("--no-walled", action="store_true", help="skip the walled-grid throughput cases")
    p.add_argument("--fdlbm2", action="store_true", help="only time the T2S2-FDLBM2 cases at --n and print that")
    p.add_argument("--walled", type=int, default=0, metavar="N",
                   help="only time the walled-grid cases (cavity (N+1)^2, channel N x (N+1)) and print that")
    return p.parse_args()


def workload_fields(n):
    import inputs as I
    import numpy as np
    rng = np.random.default_rng(SEED)
    phase = tuple(float(v) for v in rng.uniform(0.0, 2 * math.pi, size=2))
    ax = I.periodic_axis(n, 0.0, 2 * math.pi)
    f = I.taylor_green(ax, ax, u0=U0, phase=phase)
    return ax, f, phase


def config(n, precision, steps):
    return {"workload": f"taylor-green throughput {n}x{n} periodic uniform, {precision} "
                        f"(random-phase u0={U0}, nu={NU}, CFL={CFL}, blend={BLEND})",
            "nx": n, "ny": n, "precision": precision, "bench_steps": steps,
            "l2": "inputs larger than L2 (state 2 x %.0f MB)" % (9 * n * n * (4 if precision == 'fp32' else 8) / 1e6)}


# ----------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.bracket = 0

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", f"--id={self.uuid}", f"--query-gpu={self.Q}",
                   "--format=csv,noheader,nounits", "-lms", "200"]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def snapshot(self):
        """One sample now (used right before and right after a short timed
        region, which the 200 ms sampler may miss)."""
        try:
            r = subprocess.run(["nvidia-smi", f"--id={self.uuid}", f"--query-gpu={self.Q}",
                                "--format=csv,noheader,nounits"], capture_output=True, text=True,
                               timeout=10)
            if r.returncode == 0 and r.stdout.strip():
                self.lines.append(r.stdout.strip().splitlines()[0])
                self.bracket += 1
        except (OSError, subprocess.TimeoutExpired):
            pass

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "bracketing_samples": self.bracket, "reasons": sorted(reasons),
                "window": "200 ms sampler over the whole GPU part of the run, plus one sample "
                          "right before and one right after the timed region"}


# ----------------------------------------------------------------------- helpers
# committed ncu DRAM-traffic record and the sources it was taken from, per kernel
TRAFFIC = {
    "fused-warp": ("warp_fp32_traffic.json",
                   ["step_fused_warp.cu", "packed.cuh", "tma.cuh", "lattice.cuh"]),
    "fused": ("fused_fp32_traffic.json", ["step_fused.cu", "lattice.cuh"]),
}


def sources_sha256(names):
    h = hashlib.sha256()
    for nm in names:
        h.update((ROOT / "paper_1911_12913_gb300" / "csrc" / nm).read_bytes())
    return h.hexdigest()


def kernel_traffic(kernel_desc):
    """Per-launch DRAM bytes of the timed kernel from the committed ncu record,
    valid only while the kernel's sources are unchanged."""
    rec = TRAFFIC.get(kernel_desc.split()[0])
    if rec is None:
        return None
    f = ROOT / "profiles" / rec[0]
    if not f.exists():
        return None
    d = json.loads(f.read_text())
    if d.get("kernel_sha256") != sources_sha256(rec[1]):
        return None
    return d.get("dram_bytes_per_launch_full")


def peaks():
    try:
        return json.loads((ROOT / "MEASURED_PEAKS.json").read_text())
    except (OSError, ValueError):
        return {}


def fp64_peak(stream):
    """Measured FP64 FMA rate (TFLOP/s) of this GPU: independent FMA chains
    (libfdlbm's fdlbm_probe_fp64_fma), best of 3 launches of about 0.1 s,
    timed with CUDA events on the launching stream."""
    import ctypes
    import torch
    from paper_1911_12913_gb300 import binding as B
    L = B.load()
    blocks = 152 * 8
    out = torch.zeros(blocks, dtype=torch.float64, device="cuda")
    flop = ctypes.c_double()
    best = None
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = L.fdlbm_probe_fp64_fma(blocks, 20000, out.data_ptr(), ctypes.c_void_p(stream.cuda_stream),
                                    ctypes.byref(flop))
        e1.record(stream)
        torch.cuda.synchronize()
        assert rc == 0
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    return flop.value / best / 1e12


def cpu_oracle_rate(n, target_s=12.0, nthreads=None, steps=None):
    """Time the FP64 oracle (as it stands) on an n x n sample of the workload."""
    import oracle as O
    ax, f, phase = workload_fields(n)
    nthreads = nthreads or (os.cpu_count() or 1)
    o = O.Oracle(ax, ax, nu=NU, dt=O.time_step(CFL, ax, ax), beta=BLEND, nthreads=nthreads)
    o.init_fields(f["rho"], f["ux"], f["uy"], [f["dudx"], f["dudy"], f["dvdx"], f["dvdy"]])
    if steps is None:
        t0 = time.perf_counter()
        o.step(2)
        per = (time.perf_counter() - t0) / 2
        steps = max(2, int(target_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    return n * n * steps / el / 1e6, steps, el, nthreads


# ----------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    ax, f, phase = workload_fields(SAMPLE_N)
    nthreads = os.cpu_count() or 1
    o = O.Oracle(ax, ax, nu=NU, dt=O.time_step(CFL, ax, ax), beta=BLEND, nthreads=nthreads)
    o.init_fields(f["rho"], f["ux"], f["uy"], [f["dudx"], f["dudy"], f["dvdx"], f["dvdy"]])
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    el = time.perf_counter() - t0
    mlups = SAMPLE_N * SAMPLE_N * args.steps / el / 1e6
    sample = (f"{SAMPLE_N}x{SAMPLE_N} sample of the {N_GRID}x{N_GRID} workload (same nu, CFL, "
              f"blend, phase), FP64 oracle, {args.steps} steps")
    out = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": config(N_GRID, "fp32", args.steps),
           "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": nthreads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------------- batched sweep
def run_batched(stream_dev, ncases=64, seed=2024, steps=200, graph_steps=50):
    """64 independent cases (cavity and channel, 33..513 cells per axis, half
    tanh-stretched, Re log-uniform in [10, 2000]) in one batch: CUDA-graph
    replay of the batched staged kernels with an autotuned block shape."""
    import numpy as np
    import torch
    import inputs as I
    from paper_1911_12913_gb300.solver import FDLBMBatch

    specs = I.batched_cases(ncases, seed=seed)
    probs = [I.batched_problem(cs) for cs in specs]
    cases = [dict(xa=p["xa"], ya=p["ya"], nu=p["nu"], cfl=CFL, blend=BLEND, wall_u=p["wall_u"],
                  has_force=p["force"] is not None) for p in probs]
    b = FDLBMBatch(cases, precision="fp32", graph_steps=graph_steps, autotune=True,
                   device=stream_dev)
    for c, p in enumerate(probs):
        v = b.case(c)
        if p["force"] is not None:
            v.set_force(p["force"])
        one = np.ones((p["ya"].n, p["xa"].n))
        v.init_fields(one, 0 * one, 0 * one)
    b.step(2 * graph_steps)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    b.sync()
    t = e0.elapsed_time(e1) / 1e3
    kernel = b.describe
    # the same steps in the other two modes (per-stage staged launches, and
    # one persistent cooperative launch per graph replay)
    other = {}
    for name, mode in (("staged", 1), ("persistent", 2)):
        b._L.fdlbm_batch_set_mode(b._h, mode)
        b.step(2 * graph_steps)
        b.sync()
        e0.record(b.stream)
        b.step(steps)
        e1.record(b.stream)
        b.sync()
        other[name] = b.cells * steps / (e0.elapsed_time(e1) / 1e3) / 1e6
    finite = all(np.isfinite(b.case(c).reduce()[0]) for c in range(len(probs)))
    out = {"cases": len(probs), "cells": b.cells, "steps": steps,
           "MLUPS": b.cells * steps / t / 1e6, "ms_per_step": t / steps * 1e3,
           "bytes_per_cell": 72, "hbm_frac": 72 * b.cells * steps / t / 1e9 / (peaks().get("hbm_gbs") or 6800.0),
           "kernel": kernel, "all_finite": bool(finite),
           "staged_MLUPS": other["staged"], "persistent_MLUPS": other["persistent"],
           "workload": f"{ncases} cases seed {seed}: cavity/channel, 33..513 cells, half stretched, "
                       f"Re log-uniform [10, 2000], CFL {CFL}, blend {BLEND}, FP32"}
    b.close()
    return out


# ----------------------------------------------------------------------- size sweep
def run_sweep(dev, stream, sizes=(512, 1024, 2048, 4096)):
    """The throughput sweep of the configs: MLUPS and HBM fraction per size, FP32
    (automatic kernel) and FP64, on the random-phase Taylor-vortex field."""
    import torch
    from paper_1911_12913_gb300.solver import FDLBM

    hbm = peaks().get("hbm_gbs") or 6800.0
    out = []
    for n in sizes:
        ax, f, _ = workload_fields(n)
        grad = [f["dudx"], f["dudy"], f["dvdx"], f["dvdy"]]
        for prec, k in (("fp32", 400), ("fp64", 20)):
            s = FDLBM(ax, ax, nu=NU, cfl=CFL, blend=BLEND, precision=prec, stream=stream)
            s.init_fields(f["rho"], f["ux"], f["uy"], grad)
            s.step(5)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            s.step(k)
            e1.record(stream)
            torch.cuda.synchronize()
            s.sync()
            t = e0.elapsed_time(e1) / 1e3 / k
            out.append({"n": n, "precision": prec, "kernel": s.describe, "MLUPS": n * n / t / 1e6,
                        "GBs": BYTES_PER_CELL[prec] * n * n / t / 1e9,
                        "hbm_frac": BYTES_PER_CELL[prec] * n * n / t / 1e9 / hbm, "steps": k})
            del s
            torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------- T2S2-FDLBM2
def run_fdlbm2(dev, stream, n=N_GRID):
    """T2S2-FDLBM2 (Eq. 5.23) on the throughput workload: the fused sweeps in FP32
    (the automatic kernel, the warp tile, and the scalar sweep) and FP64 against
    the staged kernels in FP32 (extra line, not the headline)."""
    import torch
    from paper_1911_12913_gb300.solver import FDLBM

    hbm = peaks().get("hbm_gbs") or 6800.0
    ax, f, _ = workload_fields(n)
    grad = [f["dudx"], f["dudy"], f["dvdx"], f["dvdy"]]
    out = {}
    for name, prec, path, k, var in (("fused_fp32", "fp32", "fused", 200, "auto"),
                                     ("fused_scalar_fp32", "fp32", "fused", 200, "scalar"),
                                     ("staged_fp32", "fp32", "staged", 20, "auto"),
                                     ("fused_fp64", "fp64", "fused", 10, "auto")):
        s = FDLBM(ax, ax, nu=NU, cfl=CFL, blend=BLEND, precision=prec, scheme=2, path=path,
                  stream=stream, variant=var)
        s.init_fields(f["rho"], f["ux"], f["uy"], grad)
        s.step(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        s.sync()
        t = e0.elapsed_time(e1) / 1e3 / k
        out[name] = {"kernel": s.describe, "MLUPS": n * n / t / 1e6, "ms_per_step": t * 1e3,
                     "hbm_frac": BYTES_PER_CELL[prec] * n * n / t / 1e9 / hbm, "steps": k}
        del s
        torch.cuda.empty_cache()
    out["workload"] = f"{n}x{n} random-phase Taylor vortex, T2S2-FDLBM2 (h = dt)"
    return out


# ----------------------------------------------------------------------- lid-driven cavity
def run_cavity(dev, n_cells=256, c=1.5, U=0.1, Re=1000.0, cfl=0.9, eta=0.1, tol=1e-8):
    """Sec. 3C cavity on the (n_cells + 1)^2 tanh grid: FP64 march to E(u) < tol
    (checked every 100 steps, CUDA-graph replay of 100 steps), then the same
    number of steps with FP32-deviation storage.  Wall-clock timing of the whole
    march, residual checks included."""
    import numpy as np
    import torch
    import inputs as I
    from paper_1911_12913_gb300.analysis import march_to_steady, stream_function, vortex_centre
    from paper_1911_12913_gb300.solver import FDLBM

    ax = I.tanh_axis(n_cells, c)
    lid = [(0, 0), (0, 0), (0, 0), (U, 0.0)]
    res = {}
    u = {}
    steps_cap = 1_000_000
    for prec in ("fp64", "fp32"):
        s = FDLBM(ax, ax, nu=U / Re, cfl=cfl, blend=eta, precision=prec, wall_u=lid,
                  graph_steps=100, device=dev)
        one = np.ones((ax.n, ax.n))
        s.init_fields(one, 0 * one, 0 * one)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, r, _ = march_to_steady(s, tol, max_steps=steps_cap)
        el = time.perf_counter() - t0
        _, ux, uy = s.moments()
        psi = stream_function(ax.coords, ux)
        xc, yc, _ = vortex_centre(ax.coords, ax.coords, psi, (0.3, 0.7, 0.3, 0.8), -1)
        u[prec] = (ux, uy)
        res[prec] = {"steps": steps, "E_u": r, "converged": bool(r < tol), "t": steps * s.dt,
                     "wall_s": el, "MLUPS": ax.n * ax.n * steps / el / 1e6,
                     "primary_vortex": [round(xc, 4), round(yc, 4)], "kernel": s.describe,
                     "launches_per_step": s.kernels_per_step}
        steps_cap = steps   # FP32 runs as many steps as FP64 needed
        del s
    du = [np.linalg.norm(u["fp32"][k] - u["fp64"][k]) / np.linalg.norm(u["fp64"][k]) for k in (0, 1)]
    res["fp32"]["rel_L2_u_vs_fp64"] = float(np.hypot(*du))
    res["workload"] = (f"lid-driven cavity {ax.n}x{ax.n} tanh c={c}, lid U={U}, Re={Re:g}, CFL {cfl}, "
                       f"eta {eta}, walls Eq. 3.10, march to E(u) < {tol:g}")
    res["paper_primary_vortex"] = [0.5330, 0.5670]
    return res


def cavity_steps(k, n_cells=256, c=1.5, U=0.1, Re=1000.0, cfl=0.9, eta=0.1):
    """K steps of the 257^2 cavity from rest in FP32 (the automatic kernel: the
    fused sweep with walls), timed with CUDA events."""
    import numpy as np
    import torch
    import inputs as I
    from paper_1911_12913_gb300.solver import FDLBM

    ax = I.tanh_axis(n_cells, c)
    s = FDLBM(ax, ax, nu=U / Re, cfl=cfl, blend=eta, precision="fp32",
              wall_u=[(0, 0), (0, 0), (0, 0), (U, 0.0)])
    one = np.ones((ax.n, ax.n))
    s.init_fields(one, 0 * one, 0 * one)
    s.step(5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s.stream)
    s.step(k)
    e1.record(s.stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / k
    return {"steps": k, "us_per_step": t * 1e6, "MLUPS": ax.n * ax.n / t / 1e6, "kernel": s.describe}


# ----------------------------------------------------------------------- reverse mode
def adjoint_cost(dev, m, k=200, seed=11):
    """Time k adjoint steps against k forward steps on an m^2 periodic FP32 grid
    with a force field (the configuration of the inverse problem)."""
    import numpy as np
    import torch
    import inputs as I
    from paper_1911_12913_gb300.solver import FDLBM

    ax = I.periodic_axis(m, 0.0, 2 * math.pi)
    s = FDLBM(ax, ax, nu=0.01, cfl=CFL, blend=BLEND, precision="fp32", has_force=True,
              adjoint=True, device=dev)
    v = I.spectral_vorticity_velocity(m, seed, kmax=8, umax=0.01)
    one = np.ones((m, m))
    s.init_fields(one, v["ux"], v["uy"], [v["dudx"], v["dudy"], v["dvdx"], v["dvdy"]])
    g = s.save_state(s.new_buffer())
    lam, lam2 = s.new_buffer(), s.new_buffer()
    dF = torch.zeros((2, m, m), dtype=torch.float64, device=s.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    s.step(5)
    s.adjoint_step(g, lam, lam2, dF)
    torch.cuda.synchronize()
    ev[0].record(s.stream)
    s.step(k)
    ev[1].record(s.stream)
    for _ in range(k):
        s.adjoint_step(g, lam, lam2, dF)
        lam, lam2 = lam2, lam
    ev[2].record(s.stream)
    torch.cuda.synchronize()
    fwd = ev[0].elapsed_time(ev[1]) / k
    adj = ev[1].elapsed_time(ev[2]) / k
    return {"n": m, "forward_ms": fwd, "adjoint_ms": adj, "ratio": adj / fwd,
            "forward_kernel": s.describe, "adjoint_kernels_per_step": 1}


def run_walled(stream, n=N_GRID, steps=100, hbm=None):
    """Walled grids at the throughput size, FP32, the automatic kernel (at this
    size: the warp-tile interior plus the walls-sweep frame): the lid-driven
    cavity on (n+1)^2 uniform nodes (lid U = 0.1, Re = 1000, CFL 0.9), and the
    channel on n x (n+1) nodes (periodic x, walls y), without and with a
    uniform body force, and the cavity in T2S2-FDLBM2.  Bytes per cell: 72,
    or 80 with the force field."""
    import numpy as np
    import torch
    import inputs as I
    from paper_1911_12913_gb300.solver import FDLBM

    hbm = hbm or (peaks().get("hbm_gbs") or 6800.0)
    pa = I.periodic_axis(n, 0.0, 1.0)
    wa = I.wall_axis(n, 0.0, 1.0)
    lid = [(0.0, 0.0), (0.0, 0.0), (0.0, 0.0), (0.1, 0.0)]
    out = {}
    for name, xa, force, scheme in (("cavity", wa, None, 1), ("channel", pa, None, 1),
                                    ("channel_forced", pa, 1e-6, 1), ("cavity_fdlbm2", wa, None, 2)):
        s = FDLBM(xa, wa, nu=1e-4, cfl=0.9, blend=BLEND, precision="fp32", stream=stream,
                  wall_u=lid, has_force=force is not None, scheme=scheme)
        if force is not None:
            F = np.zeros((2, wa.n, xa.n))
            F[0] = force
            s.set_force(F)
        one = np.ones((wa.n, xa.n))
        s.init_fields(one, 0 * one, 0 * one)
        s.step(10)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        s.sync()
        t = e0.elapsed_time(e1) / 1e3 / steps
        cells = xa.n * wa.n
        bpc = 80 if force is not None else 72
        out[name] = {"nodes": [xa.n, wa.n], "kernel": s.describe, "MLUPS": cells / t / 1e6,
                     "ms_per_step": t * 1e3, "bytes_per_cell": bpc,
                     "hbm_frac": bpc * cells / t / 1e9 / hbm, "steps": steps,
                     "launches_per_step": s.kernels_per_step}
        del s
        torch.cuda.empty_cache()
    out["workload"] = (f"walls Eq. 3.10: cavity {n + 1}^2 uniform, lid U=0.1, Re=1000 (T2S2-FDLBM1 "
                       f"and T2S2-FDLBM2); channel {n}x{n + 1} periodic x, walls y, unforced and with "
                       f"F=1e-6; CFL 0.9, blend {BLEND}, FP32, from rest")
    return out


def run_adjoint(dev, n=256, nsteps=2000, iters=6, seed=11):
    """Adjoint cost against the forward step (256^2 and 4096^2, FP32), and the
    inverse problem: recover a hidden smooth body force on a 256^2 periodic grid
    from the final-velocity misfit of a 2000-step rollout (initial vorticity with
    a k^-3 spectrum up to k = 8), by gradient descent with the adjoint."""
    import numpy as np
    import torch
    import inputs as I
    from paper_1911_12913_gb300.adjoint import rollout_velocity
    from paper_1911_12913_gb300.solver import FDLBM

    ratios = [adjoint_cost(dev, 256), adjoint_cost(dev, 4096)]
    torch.cuda.empty_cache()

    # inverse problem
    ax = I.periodic_axis(n, 0.0, 2 * math.pi)
    s = FDLBM(ax, ax, nu=0.01, cfl=CFL, blend=BLEND, precision="fp32", has_force=True,
              adjoint=True, device=dev)
    v = I.spectral_vorticity_velocity(n, seed, kmax=8, umax=0.01)
    one = np.ones((n, n))
    s.init_fields(one, v["ux"], v["uy"], [v["dudx"], v["dudy"], v["dvdx"], v["dvdy"]])
    f0 = s.save_state(s.new_buffer())
    h = I.spectral_vorticity_velocity(n, seed + 1, kmax=8, umax=1e-5)
    hidden = torch.tensor(np.stack([h["ux"], h["uy"]]), dtype=torch.float64, device=s.device)
    with torch.no_grad():
        target = rollout_velocity(s, hidden, f0, nsteps).clone()
    F = torch.zeros_like(hidden)
    losses, t_grad = [], []
    for it in range(iters):
        Fv = F.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u = rollout_velocity(s, Fv, f0, nsteps)
        J = 0.5 * ((u - target) ** 2).sum()
        J.backward()
        torch.cuda.synchronize()
        t_grad.append(time.perf_counter() - t0)
        g = Fv.grad.detach()
        losses.append(float(J.detach()))
        # step along -g with the Gauss-Newton length 2 J / |g|^2, halved until J falls
        alpha = 2.0 * losses[-1] / float((g * g).sum())
        for _ in range(8):
            trial = F - alpha * g
            with torch.no_grad():
                ut = rollout_velocity(s, trial, f0, nsteps)
            if float(0.5 * ((ut - target) ** 2).sum()) < losses[-1]:
                break
            alpha *= 0.5
        F = trial
    with torch.no_grad():
        uf = rollout_velocity(s, F, f0, nsteps)
    final = float(0.5 * ((uf - target) ** 2).sum())
    err = float(torch.linalg.norm(F - hidden) / torch.linalg.norm(hidden))
    return {"cost": ratios,
            "inverse": {"grid": f"{n}x{n} periodic FP32", "steps": nsteps,
                        "checkpoints": int(math.ceil(math.sqrt(nsteps))),
                        "loss": losses + [final], "force_rel_error": err,
                        "gradient_s": statistics.median(t_grad),
                        "setup": "initial vorticity E(k)~k^-3 up to k=8, max|u|=0.01; hidden force same "
                                 "spectral form, max 1e-5; nu=0.01, CFL 0.5; gradient descent with the "
                                 "hand-written adjoint and sqrt(N) checkpointing"}}


# ----------------------------------------------------------------------- our arm
class Ranks:
    """The ranks of a run, from RANK / WORLD_SIZE / LOCAL_RANK.  Every rank runs
    an independent replica of the workload (the step has no data-path
    collective); the only collectives are the barriers around the timed region
    and the maximum of the ranks' times."""

    def __init__(self, backend="nccl", device=None):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        if device is None:
            torch.cuda.set_device(self.local)
            device = torch.device("cuda", self.local)
        self.device = device
        if self.world > 1 and not dist.is_initialized():
            kw = {"device_id": device} if backend == "nccl" else {}
            dist.init_process_group(backend, **kw)

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max(self, v):
        if self.world == 1:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def aggregate(self, units_per_rank, seconds_max):
        """Whole-job throughput: the units of all ranks over the slowest rank's time."""
        return self.world * units_per_rank / seconds_max

    def close(self):
        if self.world > 1 and self.dist.is_initialized():
            self.dist.destroy_process_group()


def run_ours(args):
    import numpy as np
    import torch

    ranks = Ranks("nccl")
    world, rank, dev = ranks.world, ranks.rank, ranks.device
    barrier, max_over_ranks = ranks.barrier, ranks.max

    from paper_1911_12913_gb300.solver import FDLBM

    n = args.n
    N = n * n
    ax, f, phase = workload_fields(n)
    grad = [f["dudx"], f["dudy"], f["dvdx"], f["dvdy"]]
    stream = torch.cuda.current_stream(dev)

    # the clock sampler runs over the whole GPU part of the run (it starts before
    # the warm-up); one sample is also taken right before and right after the
    # timed region, which at a few steps is shorter than the sampling period
    uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    clk = Clocks(uuid).__enter__()

    # ---------------- device-resident timing (FP32 deviation, the headline)
    s = FDLBM(ax, ax, nu=NU, cfl=CFL, blend=BLEND, precision="fp32", stream=stream,
              variant=args.variant, rows_per_cta=args.rows)
    kernel_desc = s.describe
    s.init_fields(f["rho"], f["ux"], f["uy"], grad)
    m0, _ = s.reduce()
    s.step(args.warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    clk.snapshot()
    torch.cuda.synchronize()
    ev0.record(stream)
    s.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk.snapshot()
    barrier()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms)
    m1, _ = s.reduce()
    mass_drift = abs(m1 - m0) / abs(m0)
    launches = args.steps * s.kernels_per_step
    per_launch_s = ms / 1e3 / args.steps
    value = ranks.aggregate(N * args.steps, ms_max / 1e3) / 1e6

    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = BYTES_PER_CELL["fp32"] * N / per_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": kernel_traffic(kernel_desc),
                "peak_source": peak_note + " (MEASURED_PEAKS.json hbm_gbs, burst copy)",
                "bytes_per_cell": BYTES_PER_CELL["fp32"], "kernel": kernel_desc}
    del s
    torch.cuda.empty_cache()

    # ---------------- both FP32 fused variants, same workload, shorter runs
    variants = {}
    if not args.no_variants:
        for var in ("scalar", "warp"):
            try:
                sv = FDLBM(ax, ax, nu=NU, cfl=CFL, blend=BLEND, precision="fp32", stream=stream,
                           variant=var)
            except Exception as exc:  # variant not applicable to this grid
                variants[var] = {"unavailable": str(exc)}
                continue
            sv.init_fields(f["rho"], f["ux"], f["uy"], grad)
            sv.step(5)
            kv = max(100, args.steps // 4)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sv.step(kv)
            e1.record(stream)
            torch.cuda.synchronize()
            sv.sync()
            tv = e0.elapsed_time(e1) / 1e3 / kv
            variants[var] = {"kernel": sv.describe, "MLUPS": N / tv / 1e6,
                             "ms_per_step": tv * 1e3, "hbm_frac": BYTES_PER_CELL["fp32"] * N / tv / 1e9 / hbm,
                             "steps": kv}
            del sv
            torch.cuda.empty_cache()

    # ---------------- FP64 beside it (same workload, shorter run)
    # ---------------- the same workload with a body-force field (warp-tile kernel
    # with Eqs. 3.3 and 3.12; 80 B per cell: the force field is read once more)
    forced = None
    if not args.no_variants:
        import inputs as I
        hF = I.spectral_vorticity_velocity(n, 12, kmax=8, umax=1e-5)
        sf = FDLBM(ax, ax, nu=NU, cfl=CFL, blend=BLEND, precision="fp32", stream=stream,
                   has_force=True)
        sf.set_force(np.stack([hF["ux"], hF["uy"]]))
        sf.init_fields(f["rho"], f["ux"], f["uy"], grad)
        sf.step(5)
        kv = max(100, args.steps // 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sf.step(kv)
        e1.record(stream)
        torch.cuda.synchronize()
        sf.sync()
        tv = e0.elapsed_time(e1) / 1e3 / kv
        forced = {"kernel": sf.describe, "MLUPS": N / tv / 1e6, "ms_per_step": tv * 1e3,
                  "bytes_per_cell": 80, "hbm_frac": 80 * N / tv / 1e9 / hbm, "steps": kv,
                  "force": "smooth field, k^-3 spectrum up to k = 8, max 1e-5"}
        del sf
        torch.cuda.empty_cache()

    fp64 = None
    if args.fp64_steps > 0:
        s64 = FDLBM(ax, ax, nu=NU, cfl=CFL, blend=BLEND, precision="fp64", stream=stream)
        s64.init_fields(f["rho"], f["ux"], f["uy"], grad)
        s64.step(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64.step(args.fp64_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        t64 = ms64 / 1e3 / args.fp64_steps
        peak64 = fp64_peak(stream)
        fp64 = {"value": N / t64 / 1e6, "unit": "MLUPS", "ms_per_step": ms64 / args.fp64_steps,
                "steps": args.fp64_steps,
                "hbm_achieved_gbs": BYTES_PER_CELL["fp64"] * N / t64 / 1e9,
                "hbm_frac": BYTES_PER_CELL["fp64"] * N / t64 / 1e9 / hbm,
                "roofline": {"bound": "alu", "achieved": FP64_FLOP_PER_CELL * N / t64 / 1e12,
                             "peak": peak64, "unit": "TFLOP/s",
                             "frac": FP64_FLOP_PER_CELL * N / t64 / 1e12 / peak64,
                             "flop_per_cell": FP64_FLOP_PER_CELL,
                             "peak_source": "measured in this run: independent FP64 FMA chains "
                                            "(fdlbm_probe_fp64_fma), best of 4 launches",
                             "nominal_tflops": FP64_NOMINAL_TFLOPS}}
        del s64
        torch.cuda.empty_cache()

    # ---------------- walled grids at the throughput size (cavity, channel)
    walled = None
    if not args.no_walled:
        walled = run_walled(stream, n, hbm=hbm)

    # ---------------- 64-case batched sweep (cavity / channel mixes, FP32)
    batched = None
    if not args.no_batched:
        batched = run_batched(stream_dev=dev)
        torch.cuda.empty_cache()

    # ---------------- reverse mode: adjoint cost and the 256^2 inverse problem
    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(dev)
        torch.cuda.empty_cache()

    # ---------------- the throughput sweep over sizes
    sweep = None
    if not args.no_sweep:
        sweep = run_sweep(dev, stream)

    # ---------------- T2S2-FDLBM2: fused sweep against the staged kernels
    fdlbm2 = None
    if not args.no_sweep and rank == 0:
        fdlbm2 = run_fdlbm2(dev, stream, n)

    # ---------------- 257^2 lid-driven cavity at Re = 1000 to steady state
    cavity = None
    if not args.no_cavity and rank == 0:
        cavity = run_cavity(dev)
        torch.cuda.empty_cache()

    # ---------------- end to end through the C ABI with pinned host buffers
    # The job a user runs: upload the initial fields, K steps, the mass /
    # residual reduction, read the moments back.  Headline: FP32 fields (the
    # density as rho - rho0), the storage precision of the solver; beside it
    # the same job with FP64 fields.
    import ctypes
    s = FDLBM(ax, ax, nu=NU, cfl=CFL, blend=BLEND, precision="fp32", stream=stream)
    L, h = s._L, s._h
    mass, resid = ctypes.c_double(), ctypes.c_double()
    gkeys = ("dudx", "dudy", "dvdx", "dvdy")

    def pinned(a, dt):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()

    io = {}
    for dt, tag in ((np.float32, "f32"), (np.float64, "f64")):
        r0 = f["rho"] - 1.0 if tag == "f32" else f["rho"]
        fin = [pinned(r0, dt), pinned(f["ux"], dt), pinned(f["uy"], dt)]
        gin = pinned(np.stack([f[k] for k in gkeys]), dt)
        outs = [torch.empty((n, n), dtype=torch.float32 if tag == "f32" else torch.float64).pin_memory()
                for _ in range(3)]
        init = L.fdlbm_init_fields_f32 if tag == "f32" else L.fdlbm_init_fields
        mom = L.fdlbm_moments_f32 if tag == "f32" else L.fdlbm_moments
        io[tag] = (fin, gin, outs, init, mom, np.dtype(dt).itemsize)

    def e2e_job(tag, k, ev=None):
        fin, gin, outs, init, mom, _ = io[tag]
        if ev: ev[0].record(stream)
        rc = init(h, *(t.data_ptr() for t in fin), gin.data_ptr(), 0)
        if ev: ev[1].record(stream)
        rc |= L.fdlbm_step(h, k)
        if ev: ev[2].record(stream)
        rc |= L.fdlbm_reduce(h, ctypes.byref(mass), ctypes.byref(resid))
        if ev: ev[3].record(stream)
        rc |= mom(h, *(o.data_ptr() for o in outs), 0)
        if ev: ev[4].record(stream)
        assert rc == 0, L.fdlbm_last_error(h)

    e2e = None
    for tag in ("f32", "f64"):
        e2e_job(tag, args.warmup)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_job(tag, args.steps)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        barrier()
        e2e_s = max_over_ranks(e2e_s)
        # the same job once more with CUDA events between its phases
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        e2e_job(tag, args.steps, ev)
        torch.cuda.synchronize()
        names = ("init_fields", "steps", "reduce", "moments")
        brk = {nm: ev[i].elapsed_time(ev[i + 1]) for i, nm in enumerate(names)}
        b = io[tag][5]
        rec = {"value": ranks.aggregate(N * args.steps, e2e_s) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 7 * N * b / args.steps,
               "d2h_bytes_per_step": (3 * N * b + 3 * 8) / args.steps,
               "job_ms": e2e_s * 1e3, "breakdown_ms": brk,
               "job": f"init_fields{'_f32' if tag == 'f32' else ''}(pinned host drho|rho, u, grad u; "
                      f"{'FP32' if tag == 'f32' else 'FP64'}) + K steps + reduce + "
                      f"moments{'_f32' if tag == 'f32' else ''}(pinned host), per rank"}
        if tag == "f32":
            e2e = rec
        else:
            e2e["fp64_fields"] = rec
    del s

    clk.__exit__(None, None, None)
    clocks = clk.summary()
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            rate, st, el, th = cpu_oracle_rate(SAMPLE_N)
            cpu = {"value": rate, "unit": "MLUPS", "cores": th, "kind": "oracle",
                   "sample": f"{SAMPLE_N}x{SAMPLE_N} sample of the workload, FP64 oracle, "
                             f"{st} steps in {el:.1f} s"}
        out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f32", "data": "synthetic",
               "config": config(n, "fp32", args.steps), "clocks": clocks,
               "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
               "cpu_baseline": cpu, "fp64": fp64, "fp32_variants": variants, "fp32_forced": forced,
               "walled": walled, "batched": batched, "adjoint": adjoint,
               "cavity": cavity, "sweep": sweep, "fdlbm2": fdlbm2,
               "mass_drift_rel": mass_drift,
               "parallelism": "replicas" if world > 1 else "single"}
        print(json.dumps(out), flush=True)
    ranks.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.cavity_steps:
        print(json.dumps(cavity_steps(args.cavity_steps)), flush=True)
        return 0
    if args.fdlbm2:
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        print(json.dumps(run_fdlbm2(dev, torch.cuda.current_stream(dev), args.n)), flush=True)
        return 0
    if args.walled:
        import torch
        stream = torch.cuda.current_stream(torch.device("cuda", torch.cuda.current_device()))
        print(json.dumps(run_walled(stream, args.walled, steps=max(1, args.steps))), flush=True)
        return 0
    if args.adjoint_cost:
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        print(json.dumps(adjoint_cost(dev, args.adjoint_cost, k=max(1, args.steps))), flush=True)
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
