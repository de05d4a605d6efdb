"""Phase-diagram sweeps of the (eps/dx, gamma/|u|) plane as one batched workload.

Section 2.2 maps where the explicit CDI step keeps phi in [0, 1]: above the
crossover line of Eq. 17 (Eq. 23/24 for several dimensions) boundedness is
guaranteed, below it the step can leave [0, 1] (Table 2, Fig. 5).  Here every
point of a grid of (eps/dx, gamma/|u|) values is one small periodic 2D box --
the drop of Table 2 (diameter 1 in a 2 x 2 box, n x n cells, uniform velocity
(sqrt2/2, sqrt2/2)) -- and all boxes advance together, one batched launch per
step (``cdi.Batch``).

Each box takes its own explicit Euler step by the rule the Table 2 check uses,
dt = min(dx^2 / (4 gamma eps), dx / (u + v + 2 gamma)), and all boxes run the
same number of steps: at least one advection period T = 2 sqrt2 for every box
(the box with the smallest step sets the count).  Boxes with larger steps run
longer than a period; above the line that cannot produce a violation, below it
violations appear within the first steps of the transition, so the
classification is that of a one-period run.
"""
from __future__ import annotations

import math

import torch

from . import cdi
from . import inputs as I

PERIOD = 2.0 * math.sqrt(2.0)


def euler_dt(eps_over_dx: float, gamma_over_u: float, n: int = 50, L: float = 2.0) -> float:
    """Euler step of a Table 2 box: min(dx^2/(4 gamma eps), dx/(u + v + 2 gamma)), |u| = 1."""
    h = L / n
    eps, gamma = eps_over_dx * h, gamma_over_u
    c = math.sqrt(2.0) / 2.0
    return cdi.max_dt_mixed(h, eps, gamma, (c, c), cdi.CDI_EULER)


def phase_boxes(points, n=50, dtype=torch.float64, device="cuda"):
    """Batch box descriptions (cdi.Batch dicts) of the drop of Table 2 for each
    (eps/dx, gamma/|u|) point."""
    boxes = []
    for eoh, gu in points:
        f, _ = I.drop_2d_uniform(eoh, n=n)
        d = lambda a: torch.from_numpy(a).to(device, dtype).contiguous()
        boxes.append(dict(dx=f.h, dt=euler_dt(eoh, gu, n), eps=eoh * f.h, gamma=gu,
                          u=d(f.u), v=d(f.v), w=d(f.w), phi_a=d(f.phi),
                          phi_b=torch.empty(f.phi.shape, dtype=dtype, device=device)))
    return boxes


def phase_diagram(points, n=50, nsteps=None, dtype=torch.float64, device="cuda", autotune=True,
                  sharpen="centre"):
    """Advance the Table 2 drop at every (eps/dx, gamma/|u|) point together and
    classify it.

    Returns (rows, info): one dict per point with the step dt, the minimum and
    maximum of phi over the run, the tolerant violation count (phi outside
    [-eps_mach, 1 + eps_mach], summed over steps and cells), ``bounded`` (no
    tolerant violation) and ``sufficient`` (the point satisfies the paper's
    sufficient condition as ``cdi.check_condition`` reads it: Eq. 17 with U
    the largest face-velocity component, and A <= 1/(2 D_f)); and the run's
    step count, cells, batch launch configuration, the batch itself and the
    run's device time (run_ms, CUDA events around the graph replay).
    ``sharpen="face"`` runs every box with the face-product sharpening instead of
    Section 2.2's centre form (the boundedness proof covers the centre form only).
    """
    boxes = phase_boxes(points, n, dtype, device)
    if nsteps is None:
        nsteps = max(int(math.ceil(PERIOD / b["dt"])) for b in boxes)
    bt = cdi.Batch(boxes)
    if sharpen != "centre":
        bt.set_sharpening(sharpen)
    if autotune:
        bt.autotune(reps=2)
    bt.reset_run_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    bt.run(nsteps)
    e1.record()
    st = bt.stats()
    U = math.sqrt(2.0) / 2.0                 # largest face-velocity component
    rows = []
    for (eoh, gu), b, s in zip(points, boxes, st):
        A = b["dt"] * b["gamma"] * b["eps"] / b["dx"] ** 2
        rows.append(dict(eps_over_dx=eoh, gamma_over_u=gu, dt=b["dt"], min_run=s["min_run"],
                         max_run=s["max_run"], n_tol_run=int(s["n_tol_run"]),
                         n_strict_run=int(s["n_strict_run"]), bounded=int(s["n_tol_run"]) == 0,
                         sufficient=cdi.check_condition(eoh, gu / U, A, 2)))
    info = dict(nsteps=nsteps, cells=bt.info()["cells"], launch=bt.get_launch(), batch=bt,
                run_ms=e0.elapsed_time(e1))
    return rows, info
