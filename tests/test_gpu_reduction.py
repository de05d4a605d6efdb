"""The fused FP32 reductions against exact sums.  FP32 kernels reduce their statistics in FP32
arithmetic, the sum carried as an unevaluated pair of floats.  On a field of dyadic values
k / 2^12 every per-thread partial and every combination of partials is exact (the field's sum
needs at most 34 significant bits, the pair holds about 48), so the reported sum must equal the
exact sum of the field, whichever kernel, tile and work split produced it.  An Euler step with
dt = 0 returns its input bit for bit (phi + 0 * div), so the fused statistics of such a step
are those of the dyadic input."""
import numpy as np
import pytest
import torch

from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def dyadic(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 4097, size=shape).astype(np.float64) / 4096.0


def grid_with_velocity(shape, seed):
    nz, ny, nx = shape
    h = 1.0 / max(shape)
    g = cdi.Grid(nx, ny, nz, h, torch.float32)
    vel = [torch.from_numpy(x).to("cuda", torch.float32) for x in I.random_velocity(shape, h, 8, 3, seed)]
    g.set_velocity(*vel)
    return g, vel, h


def check_exact(st, p):
    # numpy's float64 sum of the dyadic values is exact: every partial sum fits 53 bits
    assert st["sum"] == p.sum()
    assert st["min"] == p.min() and st["max"] == p.max()
    assert st["n_strict"] == 0 and st["n_tol"] == 0


@pytest.mark.parametrize("shape", [(64, 256, 256), (7, 33, 40), (1, 1, 1)])
def test_stats_kernel_sum_is_exact(shape):
    p = dyadic(shape, 1)
    g = cdi.Grid(shape[2], shape[1], shape[0], 0.1, torch.float32)
    check_exact(g.mass_and_bounds(torch.from_numpy(p).to("cuda", torch.float32)), p)


@pytest.mark.parametrize("tile", range(cdi.FWD_TILES))
@pytest.mark.parametrize("nchunks", [cdi.CDI_NCHUNKS_BALANCED, cdi.CDI_NCHUNKS_ROTATED, 0, 3])
def test_step_fused_sum_is_exact(tile, nchunks):
    shape = (33, 64, 128)
    p = dyadic(shape, 2)
    g, vel, h = grid_with_velocity(shape, 3)
    g.set_launch(cdi.CDI_KERNEL_FORWARD, tile, 0, nchunks)
    a = torch.from_numpy(p).to("cuda", torch.float32)
    b = torch.empty_like(a)
    g.step(a, b, 0.0, h, 1.0)
    assert torch.equal(a, b)
    check_exact(g.stats(), p)


@pytest.mark.parametrize("nchunks", [cdi.CDI_NCHUNKS_ROTATED, 0, 4])
def test_two_steps_per_pass_sums_are_exact(nchunks):
    """The temporally blocked pass reduces two steps' partials in one launch."""
    shape = (40, 48, 128)
    p = dyadic(shape, 4)
    g, vel, h = grid_with_velocity(shape, 5)
    g.set_run_depth(2, nchunks)
    g.reset_run_stats()
    a = torch.from_numpy(p).to("cuda", torch.float32)
    b = torch.empty_like(a)
    out = g.run(a, b, 4, 0.0, h, 1.0)
    assert torch.equal(out, torch.from_numpy(p).to("cuda", torch.float32))
    st = g.stats()
    check_exact(st, p)
    assert st["steps_run"] == 4 and st["min_run"] == p.min() and st["max_run"] == p.max()


def test_batch_box_sums_are_exact():
    """Every box's statistics, folded by the block that completes the box."""
    shapes = [(9, 40, 64), (1, 50, 50), (17, 23, 31), (30, 64, 128)]
    boxes, ps = [], []
    for i, s in enumerate(shapes):
        p = dyadic(s, 10 + i)
        h = 1.0 / max(s)
        vel = [torch.from_numpy(x).to("cuda", torch.float32) for x in I.random_velocity(s, h, 8, 3, 20 + i)]
        boxes.append(dict(dx=h, dt=0.0, eps=h, gamma=1.0, u=vel[0], v=vel[1], w=vel[2],
                          phi_a=torch.from_numpy(p).to("cuda", torch.float32),
                          phi_b=torch.empty(s, dtype=torch.float32, device="cuda")))
        ps.append(p)
    b = cdi.Batch(boxes)
    for tile in range(cdi.BATCH_TILES):
        try:
            b.set_launch(tile, 0)
        except cdi.CDIError:
            continue
        b.step(1.0)
        st = b.stats()
        for i, p in enumerate(ps):
            assert torch.equal(b.current(i).cpu(), torch.from_numpy(p).float()), (tile, i)
            check_exact(st[i], p)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("tile,nchunks", [(4, cdi.CDI_NCHUNKS_ROTATED), (4, 3), (0, 1), (6, 0)])
@pytest.mark.parametrize("nsteps", [1, 2, 3, 6])
def test_run_statistics_equal_stepwise(dtype, tile, nchunks, nsteps):
    """cdi_run finishes each step's statistics in the next step's launch (the last step its
    own); the record and the run accumulators equal those of the same steps taken one
    cdi_step at a time, bit for bit.  Planted values outside [0, 1] make the violation
    counts take part."""
    shape = (24, 32, 128)
    nz, ny, nx = shape
    h = 1.0 / max(shape)
    p0 = I.random_phi(shape, 8, smooth=True)
    p0[2:7, 4:9, 6:11], p0[17:22, 26:31, 97:102] = -0.3, 1.4   # blocks outlive a few steps
    phi = torch.from_numpy(p0).to("cuda", dtype)
    vel = [torch.from_numpy(x).to("cuda", dtype) for x in I.random_velocity(shape, h, 8, 3, 9)]
    g = cdi.Grid(nx, ny, nz, h, dtype)
    g.set_velocity(*vel)
    g.set_launch(cdi.CDI_KERNEL_FORWARD, tile, 0, nchunks)
    eps, gamma = h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    g.reset_run_stats()
    out_run = g.run(phi.clone(), torch.empty_like(phi), nsteps, dt, eps, gamma, period=0.7, t0=0.05).clone()
    s_run = g.stats()
    g.reset_run_stats()
    p, q = phi.clone(), torch.empty_like(phi)
    for i in range(nsteps):
        g.step(p, q, dt, eps, gamma, float(np.cos(np.pi * (0.05 + i * dt) / 0.7)))
        p, q = q, p
    s_steps = g.stats()
    assert torch.equal(out_run, p)
    assert s_steps["n_strict_run"] > 0
    for k in ("mass", "sum", "min", "max", "n_strict", "n_tol", "min_run", "max_run", "n_strict_run",
              "n_tol_run", "steps_run"):
        assert s_run[k] == s_steps[k], (k, s_run[k], s_steps[k])
