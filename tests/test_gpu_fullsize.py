"""Full-size workloads in the launch configuration the bench times.

A cell's update reads the cells within distance 2 and their normals one cell
further, so the oracle run on the periodic 7^3 sub-cube around a cell gives
that cell's step exactly; sampled cells (random, interface, periodic seams)
are checked that way, the whole box through properties that hold at any size
(discrete mass conservation for a divergence-free velocity, no tolerant bound
violation on the crossover line).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R = 3  # sub-cube radius


def subcube(t, c):
    idx = [torch.arange(c[d] - R, c[d] + R + 1, device=t.device) % t.shape[d] for d in range(3)]
    return t[idx[0][:, None, None], idx[1][None, :, None], idx[2][None, None, :]].double().cpu().numpy()


def sampled_cells(phi, n_random, n_interface, seed):
    nz, ny, nx = phi.shape
    rng = np.random.default_rng(seed)
    cells = [tuple(int(rng.integers(0, n)) for n in phi.shape) for _ in range(n_random)]
    cells += [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny - 1, nx // 2), (nz // 2, 0, nx - 1),
              (nz - 1, ny // 3, 0)]
    band = torch.nonzero((phi > 0.05) & (phi < 0.95))
    pick = torch.randint(0, band.shape[0], (n_interface,), generator=torch.Generator().manual_seed(seed))
    cells += [tuple(int(x) for x in band[int(p)].tolist()) for p in pick]
    return cells


def check_cells(cells, phi, u, v, w, out, h, dt, eps, gamma, vs, tol):
    worst = 0.0
    for c in cells:
        sub = [subcube(t, c) for t in (phi, u, v, w)]
        ref = oracle.step(*sub, h, dt, eps, gamma, vs)[R, R, R]
        worst = max(worst, abs(float(out[c]) - ref))
    assert worst <= tol, worst


def run_full(shape, spheres, nmodes, seed, eps_over_h=1.0, cfl=0.1, vs=0.8):
    nz, ny, nx = shape
    h = 1.0 / nx
    eps = eps_over_h * h
    u64, v64, w64 = I.random_velocity_torch(shape, h, nmodes, 4, seed)
    vel = [t.float() for t in (u64, v64, w64)]
    del u64, v64, w64
    phi = I.spheres_phi_torch(shape, h, spheres, eps).float()
    U, gamma = 1.0, 1.0           # velocity rescaled to U = 1; gamma = U (crossover line)
    dt = cfl * h / U
    g = cdi.Grid(nx, ny, nz, h, torch.float32)
    g.set_velocity(*vel)
    s1, s2 = phi.clone(), torch.empty_like(phi)
    g.autotune(s1, s2, dt, eps, gamma, reps=2)     # as the bench does (untimed set-up)
    del s1, s2
    out = torch.empty_like(phi)
    g.step(phi, out, dt, eps, gamma, vs, check=True)
    st = g.stats()
    return g, phi, vel, out, st, h, dt, eps, gamma, vs


def test_random_velocity_512_one_sphere_sampled():
    """512^3, 32-mode random divergence-free velocity, one sphere (the inverse-problem case)."""
    g, phi, vel, out, st, h, dt, eps, gamma, vs = run_full(
        (512, 512, 512), [((0.42, 0.55, 0.47), 0.2)], 32, 7)
    cells = sampled_cells(phi, 48, 48, 1)
    check_cells(cells, phi, *vel, out, h, dt, eps, gamma, vs, 1e-6)
    assert st["n_tol"] == 0
    m0 = phi.double().sum().item()
    assert abs(st["sum"] - m0) / m0 <= 1e-6
    # compensated per-thread FP32 sums, groups of four added uncompensated (~1e-9 relative)
    assert st["sum"] == pytest.approx(out.double().sum().item(), rel=1e-8)


def test_random_velocity_1024_four_spheres_sampled():
    """1024^3 (the largest configuration), 64-mode velocity, four spheres, two steps."""
    sph = [((0.3, 0.3, 0.3), 0.12), ((0.7, 0.35, 0.6), 0.15), ((0.45, 0.75, 0.25), 0.1),
           ((0.8, 0.8, 0.8), 0.13)]
    g, phi, vel, out, st, h, dt, eps, gamma, vs = run_full((1024, 1024, 1024), sph, 64, 11)
    cells = sampled_cells(phi, 32, 32, 2)
    check_cells(cells, phi, *vel, out, h, dt, eps, gamma, vs, 1e-6)
    assert st["n_tol"] == 0
    m0 = phi.double().sum().item()
    assert abs(st["sum"] - m0) / m0 <= 1e-6
    # a second step reads the first step's output (ping-pong buffers of the bench)
    out2 = torch.empty_like(phi)
    g.step(out, out2, dt, eps, gamma, vs)
    st2 = g.stats()
    del phi
    check_cells(cells[:16], out, *vel, out2, h, dt, eps, gamma, vs, 1e-6)
    assert st2["n_tol"] == 0 and abs(st2["sum"] - m0) / m0 <= 2e-6


def test_batch_64_boxes_full_workload():
    """The bench's 64-box batch (edges U{32..160}), autotuned launch, 4 steps: the three
    smallest boxes against the oracle cell by cell, every box through its mass and bounds."""
    raw = I.random_boxes(64, 32, 160, seed=0)
    boxes = []
    for r in raw:
        fb = r["fields"]
        Df = sum(1 for q in fb.phi.shape if q > 1)
        bdt = 0.9 * fb.h * fb.h / (2 * Df * r["gamma"] * r["eps"])
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)
        boxes.append(dict(dx=fb.h, dt=bdt, eps=r["eps"], gamma=r["gamma"], u=d(fb.u), v=d(fb.v),
                          w=d(fb.w), phi_a=d(fb.phi), phi_b=torch.empty(fb.phi.shape, device="cuda"),
                          fields=fb))
    b = cdi.Batch(boxes)
    b.autotune(reps=2)
    nsteps = 4
    b.run(nsteps)
    st = b.stats()
    for i, x in enumerate(boxes):
        cur = b.current(i)
        assert st[i]["steps_run"] == nsteps and st[i]["n_tol_run"] == 0
        # the fused sum: compensated FP32 per thread, FP64 across threads (a few units of
        # FP32 rounding in the worst case, ~1e-9 typically; the tile decides how many cells
        # each thread's compensated partial holds)
        assert abs(st[i]["sum"] - cur.double().sum().item()) <= 1e-7 * abs(st[i]["sum"])
    order = sorted(range(len(boxes)), key=lambda i: boxes[i]["fields"].phi.size)[:3]
    for i in order:
        x = boxes[i]
        f = x["fields"]
        rin = [np.asarray(a, np.float32).astype(np.float64) for a in (f.phi, f.u, f.v, f.w)]
        ref = oracle.run(*rin, f.h, x["dt"], x["eps"], x["gamma"], nsteps)
        assert np.abs(b.current(i).double().cpu().numpy() - ref).max() <= 5e-6, i
        m0 = rin[0].sum()
        assert abs(st[i]["sum"] - m0) / m0 <= 1e-6
