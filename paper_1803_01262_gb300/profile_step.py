"""Run a fixed number of CDI steps in one launch configuration (for profilers).

The deformation workload of the benchmark (sphere R = 0.15 at (0.35, 0.35,
0.35) in an n^3 periodic box, deformation face velocity, eps = dx,
gamma = U, dt = 0.1 dx / U), with the forward (or adjoint) kernel's launch
configuration set explicitly so that a profiler capture is deterministic:

    python -m paper_1803_01262_gb300.profile_step --n 256 --dtype f32 --tile 4 --nchunks 9 --steps 3

``--depth 2`` runs the forward steps as ``cdi_run`` at run depth 2 (two steps per launch,
``--nchunks`` its work split).  ``--kernel batch`` runs the 64-box batch workload of the benchmark instead
(edges U{32..160}, seed 0), with ``--tile`` / ``--zdepth`` as its work-unit
tile and planes per unit (``--tile -1``: the autotuner's choice);
``--kernel phase`` the benchmark's phase-diagram sweep (256 FP64 boxes of
50 x 50 cells, the Table 2 drop at a 16 x 16 grid of (eps/dx, gamma/|u|)
points) with ``--tile`` as its batch tile (4: one unit per whole box).
"""
from __future__ import annotations

import argparse
import math

import torch

from . import cdi
from . import inputs as I


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--kernel", choices=["forward", "adjoint", "batch", "phase"], default="forward")
    ap.add_argument("--zdepth", type=int, default=64)
    ap.add_argument("--tile", type=int, default=-1)
    ap.add_argument("--nchunks", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--depth", type=int, default=1, help="forward: steps per launch (cdi_run)")
    ap.add_argument("--run", action="store_true",
                    help="forward, batch: the steps as one run (cdi_run / graph), as the bench times them")
    args = ap.parse_args()
    dtype = torch.float32 if args.dtype == "f32" else torch.float64
    if args.kernel == "batch":
        return run_batch(args, dtype)
    if args.kernel == "phase":
        return run_phase(args)
    n = args.n
    f = I.deformation_3d(n)
    g = cdi.Grid(n, n, n, f.h, dtype)
    vel = [torch.from_numpy(x).cuda().to(dtype) for x in (f.u, f.v, f.w)]
    g.set_velocity(*vel)
    which = cdi.CDI_KERNEL_FORWARD if args.kernel == "forward" else cdi.CDI_KERNEL_ADJOINT
    g.set_launch(which, args.tile, 0, args.nchunks)
    a = torch.from_numpy(f.phi).cuda().to(dtype)
    b = torch.empty_like(a)
    dt, eps, gamma = 0.1 * f.h / f.U, f.h, f.U
    lam = torch.ones_like(a) if args.kernel == "adjoint" else None
    if args.kernel == "forward" and args.depth == 2:
        g.set_run_depth(2, args.nchunks)
        g.run(a, b, 2 * args.steps, dt, eps, gamma, period=3.0)
        torch.cuda.synchronize()
        print("run depth", g.get_run_depth())
        return
    if args.kernel == "forward" and args.run:
        g.run(a, b, args.steps, dt, eps, gamma, period=3.0)
        torch.cuda.synchronize()
        print("launch", g.get_launch(which))
        return
    for i in range(args.steps):
        vs = math.cos(math.pi * i * dt / 3.0)
        if args.kernel == "forward":
            g.step(a, b, dt, eps, gamma, vs)
            a, b = b, a
        else:
            g.step_adjoint(a, lam, b, dt, eps, gamma, vs)
    torch.cuda.synchronize()
    print("launch", g.get_launch(which))


def run_batch(args, dtype):
    import numpy as np
    boxes = []
    for r in I.random_boxes(64, 32, 160, seed=0):
        f = r["fields"]
        Df = sum(1 for q in f.phi.shape if q > 1)
        dt = 0.9 * f.h * f.h / (2 * Df * r["gamma"] * r["eps"])
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)
        boxes.append(dict(dx=f.h, dt=dt, eps=r["eps"], gamma=r["gamma"], u=d(f.u), v=d(f.v), w=d(f.w),
                          phi_a=d(f.phi), phi_b=torch.empty(f.phi.shape, dtype=dtype, device="cuda")))
    b = cdi.Batch(boxes)
    if args.tile < 0:
        b.autotune(reps=2)
    else:
        b.set_launch(args.tile, args.zdepth)
    if args.run:
        b.run(args.steps)
    else:
        for _ in range(args.steps):
            b.step(1.0)
    torch.cuda.synchronize()
    print("launch", b.get_launch(), b.info())


def run_phase(args):
    import numpy as np
    from . import phase as P
    pts = [(float(a), float(b)) for a in np.linspace(0.55, 2.0, 16) for b in np.linspace(0.3, 3.0, 16)]
    b = cdi.Batch(P.phase_boxes(pts, 50, torch.float64))
    if args.tile < 0:
        b.autotune(reps=2)
    else:
        b.set_launch(args.tile, 0)
    for _ in range(args.steps):
        b.step(1.0)
    torch.cuda.synchronize()
    print("launch", b.get_launch(), b.info())


if __name__ == "__main__":
    main()
