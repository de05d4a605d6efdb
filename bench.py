"""Benchmark of the fused CDI phase-field step on GB300.

Workload (one "step" = one explicit Euler CDI step of the whole box):
  256^3 periodic unit box, sphere R = 0.15 at (0.35, 0.35, 0.35) with the
  tanh profile, 3D deformation face velocity (discrete curl of a staggered
  vector potential) scaled by cos(pi t / 3), eps = dx, gamma = U (on the
  crossover line of Eq. 17), dt = 0.1 dx / U.  FP32 stencil with FP64-summed
  mass; FP64 and the adjoint step are measured on the same box.

Metric: Gcell-updates/s of the FP32 step (whole job, all ranks).  Inputs
(phi 64 MiB + three face velocities 192 MiB) exceed the 129 MB L2, so no
flush is done between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the plain reference
implementation of the same discretisation) on the host cores, on a bounded
sample of the same workload per step.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 256
BYTES_F32 = 20   # phi read 4 + u, v, w 12 + phi write 4 per cell-update
BYTES_F64 = 40
BYTES_ADJ_F32 = 24  # phi, lam', u, v, w read + lam write
FLOPS_PER_CELL = 51  # 17 per mesh point per direction (Section 3.3.3) x 3
METRIC = "Gcell-updates/s per phi step (FP32 CDI step, 256^3 deformation)"
PROFILE_F32 = os.path.join(ROOT, "profiles", "fwd_f32_deformation256.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N, help="box edge (default 256)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batch and 512^3 lines")
    ap.add_argument("--launch", default="",
                    help="TILE,NCHUNKS: fixed FP32 forward launch instead of the autotuner "
                         "(FP64 then keeps its default launch); for profiler captures")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("csrc/cdi_fwd.cu", "csrc/cdi_fwd_common.cuh", "csrc/cdi_reduce.cuh", "csrc/cdi_async.cuh",
              "csrc/cdi_internal.cuh", "build.py"):
        h.update(open(os.path.join(ROOT, "paper_1803_01262_gb300", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, if it is current."""
    if not os.path.exists(PROFILE_F32):
        return None
    kv = {}
    for line in open(PROFILE_F32):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if (kv.get("kernel_source_sha") or "").split()[:1] != [kernel_source_hash()]:
        return None
    try:
        return float(kv["dram_bytes_per_launch"].split()[0])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index),
                                      f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.1)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (every rank gets it); x itself on one process.
    The timings of a multi-rank run are the slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(fields, dt, eps, gamma, planes, steps):
    """Gcell-updates/s of the oracle on `planes` z-planes of the box (periodic wrap)."""
    import oracle
    sub = [np.ascontiguousarray(x[:planes]) for x in (fields.phi, fields.u, fields.v, fields.w)]
    oracle.step(*sub, fields.h, dt, eps, gamma)  # warm (build, page-in)
    t = time.perf_counter()
    p = sub[0]
    for i in range(steps):
        p = oracle.step(p, *sub[1:], fields.h, dt, eps, gamma, math.cos(math.pi * i * dt / 3.0))
    el = time.perf_counter() - t
    return p.size * steps / el / 1e9, el


def _oracle_slab(task):
    """One process of the all-cores baseline: `steps` oracle steps of its own z-slab of the
    box, taken as an independent periodic box (the same per-cell work)."""
    import oracle
    phi, u, v, w, h, dt, eps, gamma, steps = task
    p = phi
    for i in range(steps):
        p = oracle.step(p, u, v, w, h, dt, eps, gamma, math.cos(math.pi * i * dt / 3.0))
    return p.size * steps


def cpu_oracle_rate_all_cores(fields, dt, eps, gamma, steps):
    """Gcell-updates/s of the oracle run as one process per host core, each on a z-slab of
    the box (spawned processes: none inherits CUDA state); returns (rate, processes, s)."""
    import multiprocessing
    import oracle
    oracle.build()
    nproc = max(1, min(os.cpu_count() or 1, fields.phi.shape[0] // 4))
    nz = fields.phi.shape[0]
    bounds = [nz * k // nproc for k in range(nproc + 1)]
    tasks = [tuple(np.ascontiguousarray(x[bounds[k]:bounds[k + 1]])
                   for x in (fields.phi, fields.u, fields.v, fields.w)) + (fields.h, dt, eps, gamma, steps)
             for k in range(nproc)]
    with multiprocessing.get_context("spawn").Pool(nproc) as pool:
        pool.map(_oracle_slab, [t[:8] + (1,) for t in tasks])   # warm: import, load, page in
        t0 = time.perf_counter()
        cells = sum(pool.map(_oracle_slab, tasks))
        el = time.perf_counter() - t0
    return cells / el / 1e9, nproc, el


def run_reference(args):
    """--impl reference: the FP64 CPU oracle timed on the host (rank 0 only)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1803_01262_gb300 import inputs as I
    import oracle
    oracle.build()
    f = I.deformation_3d(args.n)
    dt, eps, gamma = 0.1 * f.h / f.U, f.h, f.U
    # Bounded per-step sample so K + W steps take about two minutes at ~6 Mcell/s.
    budget_cells = 6e6 * 120.0 / max(1, args.steps + args.warmup)
    planes = int(max(1, min(args.n, budget_cells // (args.n * args.n))))
    sub = [np.ascontiguousarray(x[:planes]) for x in (f.phi, f.u, f.v, f.w)]
    p = sub[0]
    for i in range(args.warmup):
        p = oracle.step(p, *sub[1:], f.h, dt, eps, gamma)
    t = time.perf_counter()
    for i in range(args.steps):
        p = oracle.step(p, *sub[1:], f.h, dt, eps, gamma, math.cos(math.pi * i * dt / 3.0))
    el = time.perf_counter() - t
    cells = p.size
    val = cells * args.steps / el / 1e9
    sample = (f"{planes} of {args.n} z-planes ({args.n}x{args.n}x{planes} = {cells} cells, periodic "
              f"wrap) of the {args.n}^3 deformation box per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Gcell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / max(1, args.steps) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"cdi_step_deformation_{args.n}^3", "sample_per_step": sample},
        "cpu_baseline": {"value": val, "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def inverse_512(dev, iters=3):
    """Sphere-parameter inverse problem at 512^3, FP32: 200 steps, checkpoint every 16.

    Velocity: 32-mode random divergence-free field (kmax 4, seed 7), eps = dx,
    gamma = U, dt = 0.1 dx / U.  Target: the rollout of the sphere (0.5, 0.5,
    0.5, R 0.2); start: (0.52, 0.485, 0.51, R 0.18).  One untimed gradient, then
    ``iters`` timed Adam iterations (each: 200 forward steps, the checkpoint
    recompute, 200 adjoint steps).  dL/dR is checked against a central
    difference of the FP32 rollout.
    """
    import torch
    from paper_1803_01262_gb300 import autograd as AG
    from paper_1803_01262_gb300 import cdi
    from paper_1803_01262_gb300 import inputs as I
    n, nst, ck = 512, 200, 16
    h = 1.0 / n
    vel = [x.to(torch.float32).contiguous() for x in I.random_velocity_torch((n, n, n), h, 32, 4, 7, device=dev)]
    g = cdi.Grid(n, n, n, h, torch.float32)
    g.set_velocity(*vel)
    eps, gamma = h, g.U
    dt = 0.1 * h / g.U
    true = torch.tensor([0.5, 0.5, 0.5, 0.2], dtype=torch.float64, device=dev)
    init = torch.tensor([0.52, 0.485, 0.51, 0.18], dtype=torch.float64, device=dev)

    def roll(th):
        return AG.rollout(AG.sphere_phi(th, g.shape, h, eps).float().contiguous(), *vel, g, nst, dt, eps,
                          gamma, ckpt_every=ck)
    with torch.no_grad():
        target = roll(true).detach()

    def loss(th):
        return ((roll(th).double() - target.double()) ** 2).sum() * h ** 3
    th = init.clone().requires_grad_(True)
    loss(th).backward()
    grad = th.grad.detach().cpu().tolist()
    with torch.no_grad():
        dR = 2e-3
        e = torch.tensor([0, 0, 0, dR], dtype=torch.float64, device=dev)
        fd = (float(loss(init + e)) - float(loss(init - e))) / (2 * dR)
    # untimed: one Adam iteration (the caching allocator settles on the first ones)
    AG.inverse_problem(target, *vel, g, nst, dt, eps, gamma, init, iters=1, lr=5e-3, ckpt_every=ck)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    theta, losses = AG.inverse_problem(target, *vel, g, nst, dt, eps, gamma, init, iters=iters, lr=5e-3,
                                       ckpt_every=ck)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out = {"workload": "sphere inverse problem 512^3 FP32, 32-mode random velocity, 200 steps, "
                       "checkpoint every 16, Adam on (cx, cy, cz, R)",
           "ms_per_gradient": el / iters * 1e3, "iters": iters,
           "steps_per_gradient": {"forward": nst, "adjoint": nst,
                                  "recompute": sum(min(s + ck, nst) - s - 1 for s in range(0, nst, ck))},
           "losses": losses, "theta": theta.cpu().tolist(),
           "grad_at_start": grad, "fd_dL_dR": fd, "grad_rel_err_R": abs(grad[3] - fd) / abs(fd)}
    del g, vel, target
    return out


def size_1024(dev, peak, nst=500, ck=32, inner=8):
    """1024^3 FP32: 64-mode random velocity (kmax 4, seed 11, U = 1), four spheres, eps = dx,
    gamma = U, dt = 0.1 dx / U.  500 timed forward steps (one native run, CUDA events):
    Gcell-updates/s, HBM fraction, FP64-reduced mass drift and tolerant bound violations over
    the run.  Then one gradient of L = sum(w phi_500) dV (w = phi_0) through the 500 steps,
    checkpoint every 32 (recomputed in sub-segments of 8), timed, and its directional
    derivative along phi_0 (1 - phi_0) against a central difference of two FP32 rollouts."""
    import torch
    from paper_1803_01262_gb300 import autograd as AG
    from paper_1803_01262_gb300 import cdi
    from paper_1803_01262_gb300 import inputs as I
    n = 1024
    h = 1.0 / n
    shape = (n, n, n)
    sph = [((0.3, 0.3, 0.3), 0.12), ((0.7, 0.35, 0.6), 0.15), ((0.45, 0.75, 0.25), 0.1),
           ((0.8, 0.8, 0.8), 0.13)]
    vel = [t.float() for t in I.random_velocity_torch(shape, h, 64, 4, 11, device=dev)]
    phi0 = I.spheres_phi_torch(shape, h, sph, h, device=dev).float()
    g = cdi.Grid(n, n, n, h, torch.float32)
    g.set_velocity(*vel)
    eps, gamma = h, g.U
    dt = 0.1 * h / g.U
    s1, s2 = phi0.clone(), torch.empty_like(phi0)
    g.autotune(s1, s2, dt, eps, gamma, reps=2)
    del s1, s2
    launch = g.get_launch()
    a, b = phi0.clone(), torch.empty_like(phi0)
    g.run(a, b, 3, dt, eps, gamma)      # warm-up
    a.copy_(phi0)
    g.reset_run_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = g.run(a, b, nst, dt, eps, gamma)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st = g.stats()
    m0 = phi0.double().sum().item()
    del a, b, out
    gbs = BYTES_F32 * n ** 3 / (ms / nst * 1e-3) / 1e9
    res = {"workload": "cdi_step_random64_4spheres_1024^3", "steps": nst,
           "value": n ** 3 * nst / (ms * 1e-3) / 1e9, "unit": "Gcell-updates/s",
           "ms_per_step": ms / nst, "achieved_gbs": gbs, "frac": gbs / peak, "launch": launch,
           "mass_drift_rel": abs(st["sum"] - m0) / m0, "n_tol_run": int(st["n_tol_run"]),
           "n_strict_run": int(st["n_strict_run"]), "steps_run": int(st["steps_run"]),
           "min_run": st["min_run"], "max_run": st["max_run"]}

    w64 = phi0.double()

    def lossval(pT):
        return float(torch.sum(pT.double() * w64)) * h ** 3

    def roll(p0):
        x, y = p0.clone(), torch.empty_like(p0)
        return g.run(x, y, nst, dt, eps, gamma)
    x = phi0.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outT = AG.rollout(x, *vel, g, nst, dt, eps, gamma, ckpt_every=ck, inner_every=inner)
    outT.backward((phi0 * h ** 3).contiguous())
    torch.cuda.synchronize()
    tg = time.perf_counter() - t0
    delta = phi0 * (1 - phi0)
    dd = float(torch.sum(x.grad.double() * delta.double()))
    del x, outT
    alpha = 1e-2
    with torch.no_grad():
        fd = (lossval(roll(phi0 + alpha * delta)) - lossval(roll(phi0 - alpha * delta))) / (2 * alpha)
    res["gradient"] = {"ms_per_gradient": tg * 1e3, "checkpoint_every": ck, "inner_every": inner,
                       "loss": "sum(phi_0 phi_500) dV", "direction": "phi_0 (1 - phi_0)",
                       "adjoint_dir_deriv": dd, "fd_dir_deriv": fd, "rel_err": abs(dd - fd) / abs(fd)}
    del g, vel, phi0, w64, delta
    torch.cuda.empty_cache()
    return res


def slab_line(dev, f, dt, eps, gamma, K, W, dist, barrier, maxrank):
    """The box split into z slabs, one per rank (one slab with its own periodic halo at
    N = 1): every step exchanges two halo planes with each neighbour (NCCL point-to-point
    between ranks; device copies at N = 1) and updates the rank's owned planes with
    cdi_step_planes.  Strong scaling of the one box."""
    import torch
    from paper_1803_01262_gb300 import slab as S
    ws = dist.get_world_size() if dist is not None else 1
    rank = dist.get_rank() if dist is not None else 0
    T = [torch.from_numpy(x).to(dev, torch.float32) for x in (f.phi, f.u, f.v, f.w)]
    d = S.SlabDomain(rank, ws, *T, f.h)
    del T
    run = S.SlabRun([d], S.DistTransport() if dist is not None else S.LocalTransport())
    for i in range(W):
        run.step(dt, eps, gamma, 1.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record()
    for i in range(K):
        run.step(dt, eps, gamma, math.cos(math.pi * i * dt / 3.0))
    e1.record()
    barrier()
    ms = maxrank(e0.elapsed_time(e1))
    st = run.stats()
    cells = f.phi.size
    return {"workload": f"cdi_step_deformation_{f.phi.shape[0]}^3 split into {ws} z slab(s), halo 2 planes",
            "parallelism": f"slab{ws}", "scaling": "strong", "steps": K,
            "value": cells * K / (ms * 1e-3) / 1e9, "unit": "Gcell-updates/s", "ms_per_step": ms / K,
            "planes_per_rank": [b - a for a, b in d.slabs], "n_tol_last_step": st["n_tol"],
            "exchange": "NCCL send/recv" if ws > 1 else "device copies (own periodic halo)"}


def phase_line(dev):
    """Phase diagram of the (eps/dx, gamma/|u|) plane: 16 x 16 Table 2 drop boxes (50 x 50,
    FP64) advanced by one batched launch per step for at least one advection period each,
    with Section 2.2's centre-product sharpening and, as a second sweep, the face-product
    form; the bounded points of both side by side."""
    import numpy as np
    import torch
    from paper_1803_01262_gb300 import phase as P
    pts = [(float(a), float(b)) for a in np.linspace(0.55, 2.0, 16) for b in np.linspace(0.3, 3.0, 16)]
    P.phase_diagram(pts[:4], nsteps=10, autotune=False)       # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rows, info = P.phase_diagram(pts)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out = {"workload": "phase diagram: 256 periodic 50x50 drop boxes (Table 2 setup), eps/dx 0.55..2,"
                       " gamma/|u| 0.3..3, FP64 Euler, one batched launch per step",
           "boxes": len(rows), "cells": info["cells"], "steps": info["nsteps"],
           "run_ms": info["run_ms"], "value": info["cells"] * info["nsteps"] / (info["run_ms"] * 1e-3) / 1e9,
           "unit": "Gcell-updates/s", "seconds_total_incl_setup_and_autotune": el,
           "bounded": sum(r["bounded"] for r in rows), "sufficient": sum(r["sufficient"] for r in rows),
           "sufficient_and_unbounded": sum(r["sufficient"] and not r["bounded"] for r in rows),
           "launch": info["launch"]}
    del info
    rows_f, info_f = P.phase_diagram(pts, sharpen="face")
    out["face_product"] = {
        "bounded": sum(r["bounded"] for r in rows_f),
        "sufficient_and_unbounded": sum(r["sufficient"] and not r["bounded"] for r in rows_f),
        "bounded_centre_not_face": sum(a["bounded"] and not b["bounded"] for a, b in zip(rows, rows_f)),
        "bounded_face_not_centre": sum(b["bounded"] and not a["bounded"] for a, b in zip(rows, rows_f)),
        "value": info_f["cells"] * info_f["nsteps"] / (info_f["run_ms"] * 1e-3) / 1e9,
        "launch": info_f["launch"]}
    grid = {}
    for a, b in zip(rows, rows_f):
        grid.setdefault(f"{a['eps_over_dx']:.3f}", []).append(
            ("S" if a["sufficient"] else "-") + ("C" if a["bounded"] else ".") + ("F" if b["bounded"] else "."))
    out["grid_by_eps_over_dx"] = {k: " ".join(v) for k, v in grid.items()}
    out["grid_legend"] = ("per eps/dx row, gamma/|u| 0.3..3 left to right: S sufficient condition holds, "
                          "C bounded with the centre form, F bounded with the face-product form")
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_1803_01262_gb300 import build as B
    from paper_1803_01262_gb300 import cdi
    from paper_1803_01262_gb300 import inputs as I

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())

    f = I.deformation_3d(args.n)   # every rank advances its own box (weak scaling)
    dt, eps, gamma = 0.1 * f.h / f.U, f.h, f.U
    T = 3.0
    n = args.n
    cells = n ** 3

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def maxrank(x):
        return max_over_ranks(x, dist, dev)

    def setup(dtype):
        g = cdi.Grid(n, n, n, f.h, dtype)
        vel = [torch.from_numpy(x).to(dev, dtype) for x in (f.u, f.v, f.w)]
        g.set_velocity(*vel)
        a = torch.from_numpy(f.phi).to(dev, dtype)
        b = torch.empty_like(a)
        if args.launch:
            if dtype == torch.float32:
                tile, nch = (int(x) for x in args.launch.split(","))
                g.set_launch(cdi.CDI_KERNEL_FORWARD, tile, 0, nch)
            return g, vel, a, b
        # untimed set-up: the library's autotuner picks the tile and z chunking
        # on scratch copies of the field
        s1, s2 = a.clone(), torch.empty_like(a)
        g.autotune(s1, s2, dt, eps, gamma, reps=3)
        del s1, s2
        return g, vel, a, b

    def time_steps(step, K, W):
        """W untimed calls of step(i), then two timed passes of K calls on the launching stream:
        the first between one pair of CUDA events (the throughput, and the average duration of
        a launch over the timed region: the launches run back to back, each overlapping the end
        of the previous one through programmatic dependent launch, so total / K is the launch
        duration the roofline uses), the second with an event pair around every launch (each
        launch's isolated duration: an event between two launches cuts that overlap, so these
        read a few microseconds longer)."""
        s = torch.cuda.current_stream()
        for i in range(W):
            step(i)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        start.record(s)
        for i in range(K):
            step(W + i)
        stop.record(s)
        barrier()
        total_ms = start.elapsed_time(stop)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for i in range(K):
            ev0[i].record(s)
            step(W + K + i)
            ev1[i].record(s)
        barrier()
        kern_ms = [e0.elapsed_time(e1) for e0, e1 in zip(ev0, ev1)]
        return total_ms, kern_ms

    def fwd_stepper(g, a, b):
        buf = [a, b]

        def step(i):
            g.step(buf[i & 1], buf[(i + 1) & 1], dt, eps, gamma, math.cos(math.pi * i * dt / T))
        return step

    def time_run(g, a, b, K, W):
        """The forward steps as a user runs them: W untimed steps, then K steps as ONE
        cdi_run between one pair of CUDA events (each step's statistics are finished inside
        the next step's launch: the throughput and the launch duration the roofline uses);
        then K single cdi_step calls with an event pair around each (isolated durations)."""
        s = torch.cuda.current_stream()
        step = fwd_stepper(g, a, b)
        for i in range(W):
            step(i)
        x, y = (a, b) if W % 2 == 0 else (b, a)
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        start.record(s)
        out = g.run(x, y, K, dt, eps, gamma, period=T, t0=W * dt)
        stop.record(s)
        barrier()
        total_ms = start.elapsed_time(stop)
        z = W + K
        if out is not a:  # keep the ping-pong order of fwd_stepper for the per-launch pass
            a.copy_(out)
            z = z + (z & 1)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for i in range(K):
            ev0[i].record(s)
            step(z + i)
            ev1[i].record(s)
        barrier()
        kern_ms = [e0.elapsed_time(e1) for e0, e1 in zip(ev0, ev1)]
        return total_ms, kern_ms

    def adj_stepper(g, phi_k, la, lb):
        buf = [la, lb]

        def step(i):
            g.step_adjoint(phi_k, buf[i & 1], buf[(i + 1) & 1], dt, eps, gamma,
                           math.cos(math.pi * i * dt / T))
        return step

    K, W = args.steps, max(3, args.warmup)

    # ---- FP32 fused step (the headline) ----
    g32, vel32, a32, b32 = setup(torch.float32)
    launch32 = g32.get_launch()
    with ClockSampler(local) as clk:
        total_ms, kern_ms = time_run(g32, a32, b32, K, W)
    total_ms = maxrank(total_ms)
    st = g32.stats()
    iso_kernel_ms = sum(kern_ms) / len(kern_ms)
    ms_per_step = total_ms / K
    avg_kernel_ms = ms_per_step
    value = ws * cells * K / (total_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    achieved = BYTES_F32 * cells / (avg_kernel_ms * 1e-3) / 1e9
    traffic = profiled_traffic()

    # ---- FP64 fused step on the same box (bound by the FP64 pipe: its roof is measured) ----
    fp64_fma_per_s = cdi.probe_fp64_rate()
    K64 = max(10, min(K // 4, 500))
    g64, vel64, a64, b64 = setup(torch.float64)
    t64, k64 = time_steps(fwd_stepper(g64, a64, b64), K64, W)
    t64 = maxrank(t64)
    v64 = ws * cells * K64 / (t64 * 1e-3) / 1e9
    iso64 = sum(k64) / len(k64)
    avg64 = t64 / K64
    del g64, vel64, a64, b64

    # ---- FP32 adjoint step ----
    Ka = max(10, K // 4)
    lam_a = torch.from_numpy(np.random.default_rng(0).standard_normal((n, n, n))).to(dev, torch.float32)
    lam_b = torch.empty_like(lam_a)
    ta, ka = time_steps(adj_stepper(g32, a32, lam_a, lam_b), Ka, W)
    ta = maxrank(ta)
    iso_adj = sum(ka) / len(ka)
    avg_adj = ta / Ka
    del lam_a, lam_b

    # ---- end to end through the C ABI with host buffers ----
    Ke = max(3, min(K, 50))
    pin_in = torch.from_numpy(f.phi.astype(np.float32)).pin_memory()
    pin_out = torch.empty_like(pin_in).pin_memory()
    hin, hout = pin_in.numpy(), pin_out.numpy()
    for i in range(3):
        g32.step_host(hin, hout, dt, eps, gamma, 1.0)
    barrier()
    t0 = time.perf_counter()
    for i in range(Ke):
        g32.step_host(hin, hout, dt, eps, gamma, math.cos(math.pi * i * dt / T))
        hin, hout = hout, hin
    barrier()
    te = maxrank(time.perf_counter() - t0)
    e2e_val = ws * cells * Ke / te / 1e9
    del g32, vel32, a32, b32

    # ---- the same box as z slabs with halo exchange (one slab per rank) ----
    slab = None
    if not args.no_extra:
        slab = slab_line(dev, f, dt, eps, gamma, max(10, min(K, 400)), W, dist, barrier, maxrank)

    # ---- batched boxes: 64 independent periodic boxes, edges ~U{32..160} ----
    batch = None
    if not args.no_extra:
        raw = I.random_boxes(64, 32, 160, seed=0)
        boxes = []
        for r in raw:
            fb = r["fields"]
            Df = sum(1 for q in fb.phi.shape if q > 1)
            bdt = 0.9 * fb.h * fb.h / (2 * Df * r["gamma"] * r["eps"])   # 0.9 x Eq. 25 limit
            boxes.append(dict(dx=fb.h, dt=bdt, eps=r["eps"], gamma=r["gamma"],
                              u=torch.from_numpy(fb.u).to(dev, torch.float32),
                              v=torch.from_numpy(fb.v).to(dev, torch.float32),
                              w=torch.from_numpy(fb.w).to(dev, torch.float32),
                              phi_a=torch.from_numpy(fb.phi).to(dev, torch.float32),
                              phi_b=torch.empty(fb.phi.shape, dtype=torch.float32, device=dev)))
        del raw
        bt = cdi.Batch(boxes)
        bt.autotune(reps=3)   # untimed set-up: work-unit tile and z depth
        binfo = bt.info()
        blaunch = bt.get_launch()
        Kb = max(4, min(K, 400)) // 2 * 2
        bt.run(Kb)      # capture + warm-up
        barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        bt.run(Kb)
        s1.record()
        barrier()
        tb = maxrank(s0.elapsed_time(s1))
        bst = bt.stats()
        batch = {"workload": "64 periodic boxes, edges U{32..160}, 1-3 ellipsoids, 32-mode "
                             "random velocity, eps/dx in {1, 1.5}, gamma on the crossover line, FP32",
                 "cells": binfo["cells"], "units": binfo["units"], "blocks": binfo["nblocks"],
                 "value": ws * binfo["cells"] * Kb / (tb * 1e-3) / 1e9, "unit": "Gcell-updates/s",
                 "ms_per_step": tb / Kb, "steps": Kb, "launch": "one kernel per step, CUDA graph",
                 "tile": ["32x8", "32x16", "64x8", "32x4", "whole plane", "row bands", "padded row bands"][blaunch["tile"]],
                 "zdepth": blaunch["zdepth"],
                 "achieved_gbs": BYTES_F32 * binfo["cells"] / (tb / Kb * 1e-3) / 1e9,
                 "n_tol_run_total": int(sum(x["n_tol_run"] for x in bst))}
        del bt, boxes

    # ---- 512^3 FP32 (same deformation workload) ----
    big = None
    if not args.no_extra:
        fbig = I.deformation_3d(512)
        gb = cdi.Grid(512, 512, 512, fbig.h, torch.float32)
        vb = [torch.from_numpy(x).to(dev, torch.float32) for x in (fbig.u, fbig.v, fbig.w)]
        gb.set_velocity(*vb)
        ab = torch.from_numpy(fbig.phi).to(dev, torch.float32)
        bb = torch.empty_like(ab)
        dtb = 0.1 * fbig.h / fbig.U
        s1, s2 = ab.clone(), torch.empty_like(ab)
        gb.autotune(s1, s2, dtb, 1.0 / 512, gb.U, reps=2)
        del s1, s2
        del fbig
        buf = [ab, bb]

        def big_step(i):
            gb.step(buf[i & 1], buf[(i + 1) & 1], dtb, 1.0 / 512, gb.U, math.cos(math.pi * i * dtb / T))
        Kbig = max(4, min(K, 300))
        tbig, kbig = time_steps(big_step, Kbig, W)
        tbig = maxrank(tbig)
        avg_big = tbig / Kbig
        big = {"workload": "cdi_step_deformation_512^3", "value": ws * 512 ** 3 * Kbig / (tbig * 1e-3) / 1e9,
               "unit": "Gcell-updates/s", "kernel_ms": avg_big, "steps": Kbig,
               "achieved_gbs": BYTES_F32 * 512 ** 3 / (avg_big * 1e-3) / 1e9,
               "frac": BYTES_F32 * 512 ** 3 / (avg_big * 1e-3) / 1e9 / peak,
               "run_depth_autotuned": gb.get_run_depth()["depth"]}
        # temporal blocking: cdi_run at depth 1 and at depth 2 (two steps per launch, which
        # reads phi, u, v, w and writes phi once per two steps: 20 B per launch and cell)
        depth_cmp = {}
        for depth in (1, 2):
            gb.set_run_depth(depth, 0)
            gb.run(ab, bb, 4, dtb, 1.0 / 512, gb.U, period=T)
            barrier()
            r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            Kd = max(4, min(K, 200)) // 2 * 2
            r0.record()
            gb.run(ab, bb, Kd, dtb, 1.0 / 512, gb.U, period=T)
            r1.record()
            barrier()
            msd = maxrank(r0.elapsed_time(r1)) / Kd
            launch_ms = msd * depth
            depth_cmp[f"depth{depth}"] = {
                "ms_per_step": msd, "value": ws * 512 ** 3 / (msd * 1e-3) / 1e9, "steps": Kd,
                "bytes_per_cell_step_algorithmic": BYTES_F32 / depth,
                "achieved_gbs": BYTES_F32 * 512 ** 3 / (launch_ms * 1e-3) / 1e9,
                "frac": BYTES_F32 * 512 ** 3 / (launch_ms * 1e-3) / 1e9 / peak}
        big["temporal_blocking"] = depth_cmp
        del gb, vb, ab, bb, buf

    # ---- inverse problem through the adjoint, 512^3 ----
    inverse = None
    if not args.no_extra:
        inverse = inverse_512(dev)
        torch.cuda.empty_cache()

    # ---- phase diagram as one batched workload ----
    phase = None
    if not args.no_extra:
        phase = phase_line(dev)

    # ---- 1024^3: 500 forward steps and a gradient through them ----
    big1024 = None
    if not args.no_extra:
        big1024 = size_1024(dev, peak)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            planes = max(1, int(round(4 * 6e6 * 3 / (n * n))))  # the whole box up to 256^3
            planes = min(planes, n)
            rate, el = cpu_oracle_rate(f, dt, eps, gamma, planes, 12)   # ~10 s of CPU work
            cpu = {"value": rate, "unit": "Gcell-updates/s", "cores": 1, "kind": "oracle",
                   "sample": f"12 FP64 oracle steps on {planes} of {n} z-planes of the {n}^3 box "
                             f"({n}x{n}x{planes} cells, periodic wrap), {el:.1f} s, single thread"}
            prate, nproc, pel = cpu_oracle_rate_all_cores(f, dt, eps, gamma, 12)
            cpu["all_cores"] = {"value": prate, "unit": "Gcell-updates/s", "cores": nproc,
                                "sample": f"12 FP64 oracle steps of the {n}^3 box as {nproc} processes, "
                                          f"each on its own z-slab taken as a periodic box, {pel:.1f} s"}
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": "Gcell-updates/s", "n_gpus": ws, "steps": K,
            "warmup": W, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"cdi_step_deformation_{n}^3", "grid": [n, n, n],
                       "eps_over_dx": 1.0, "gamma_over_U": 1.0, "cfl": 0.1,
                       "reduction": "fp64 mass/min/max/violations fused per step",
                       "l2": "inputs 268 MB > 129 MB L2, no flush",
                       "timing": "throughput over K steps between two CUDA events; the roofline's "
                                 "launch duration is that pass's total / K (launches overlap through "
                                 "programmatic dependent launch); isolated per-launch durations from "
                                 "a second K-step pass with events between launches",
                       "parallelism": f"replicas{ws}" if ws > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "bytes_per_cell": BYTES_F32,
                         "kernel_ms": avg_kernel_ms, "isolated_launch_ms": iso_kernel_ms,
                         "launch": launch32},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "Gcell-updates/s",
                    "h2d_bytes_per_step": cells * 4, "d2h_bytes_per_step": cells * 4 + 88,
                    "api": "cdi_step_host (pinned host phi in, phi + stats out)"},
            "gpu_launches": K,
            "fp64": {"value": v64, "unit": "Gcell-updates/s", "ms_per_step": t64 / K64,
                     "kernel_ms": avg64, "isolated_launch_ms": iso64, "steps": K64,
                     "achieved_gbs": BYTES_F64 * cells / (avg64 * 1e-3) / 1e9,
                     "gflops_fp64": FLOPS_PER_CELL * cells / (avg64 * 1e-3) / 1e9,
                     "fp32_speedup": value / v64,
                     "roofline": {"bound": "fp64",
                                  "achieved": FLOPS_PER_CELL * cells / (avg64 * 1e-3) / 1e9,
                                  "peak": 2.0 * fp64_fma_per_s / 1e9, "unit": "GFLOP/s",
                                  "frac": FLOPS_PER_CELL * cells / (avg64 * 1e-3) / (2.0 * fp64_fma_per_s),
                                  "flops_per_cell": FLOPS_PER_CELL,
                                  "peak_kind": "measured: cdi_probe_fp64_rate (independent FP64 FMA chains "
                                               "on every SM, 2 flops each), this run",
                                  "traffic": None}},
            "adjoint": {"kernel_ms": avg_adj, "isolated_launch_ms": iso_adj, "ms_per_step": ta / Ka, "steps": Ka,
                        "adj_over_fwd": avg_adj / avg_kernel_ms,
                        "achieved_gbs": BYTES_ADJ_F32 * cells / (avg_adj * 1e-3) / 1e9},
            "batch": batch,
            "slab": slab,
            "size_512": big,
            "inverse_512": inverse,
            "size_1024": big1024,
            "phase_diagram": phase,
            "stats_last_step": {"mass": st["mass"], "min": st["min"], "max": st["max"],
                                "n_tol": st["n_tol"]},
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
