"""Every launch configuration of the Euler step computes the same bits.  The kernels evaluate
the fluxes of Section 2.2 in one written order (the fused multiply-adds are the ones the
sources call; the compiler contracts nothing else), so the result of a step depends neither on
the tile shape, nor on how the tile columns are cut into work units (a unit's first z face is
evaluated in its prologue, the others are carried from the plane below), nor on whether a box
is stepped alone, in a batch, or two steps per pass."""
import numpy as np
import pytest
import torch

from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SPLITS = [1, 3, cdi.CDI_NCHUNKS_BALANCED, cdi.CDI_NCHUNKS_ROTATED, 0]


def setup(shape, dtype, seed):
    nz, ny, nx = shape
    h = 1.0 / max(shape)
    phi = torch.from_numpy(I.random_phi(shape, seed, smooth=True)).to("cuda", dtype)
    vel = [torch.from_numpy(x).to("cuda", dtype) for x in I.random_velocity(shape, h, 8, 3, seed + 1)]
    g = cdi.Grid(nx, ny, nz, h, dtype)
    g.set_velocity(*vel)
    eps, gamma = 1.1 * h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    return g, phi, vel, (dt, eps, gamma)


def run(g, phi, nsteps, prm):
    a, b = phi.clone(), torch.empty_like(phi)
    return g.run(a, b, nsteps, *prm).clone()


def eligible(tile, shape, dtype):
    nz, ny, nx = shape
    vx = 4 if dtype == torch.float32 else 2
    if tile in (4, 5) and nx % vx:
        return False
    if tile == 6 and (nx % (16 * vx) or ny % 16):
        return False
    return True


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", [(20, 48, 128), (9, 21, 68), (33, 64, 64), (1, 40, 128), (5, 7, 8)])
def test_every_tile_and_split_same_bits(dtype, shape):
    g, phi, vel, prm = setup(shape, dtype, 3 + shape[0])
    g.set_launch(cdi.CDI_KERNEL_FORWARD, 0, 0, 1)
    ref = run(g, phi, 4, prm)
    checked = 0
    for tile in range(cdi.FWD_TILES):
        if not eligible(tile, shape, dtype):
            continue
        for nch in SPLITS:
            g.set_launch(cdi.CDI_KERNEL_FORWARD, tile, 0, nch)
            out = run(g, phi, 4, prm)
            assert torch.equal(out, ref), (tile, nch, (out - ref).abs().max().item())
            checked += 1
    assert checked >= 10


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", [(20, 48, 128), (9, 24, 64)])
@pytest.mark.parametrize("nsteps", [4, 5])
def test_two_steps_per_pass_same_bits(dtype, shape, nsteps):
    g, phi, vel, prm = setup(shape, dtype, 11)
    g.set_launch(cdi.CDI_KERNEL_FORWARD, 4, 0, 1)
    ref = run(g, phi, nsteps, prm)
    for nch in [cdi.CDI_NCHUNKS_BALANCED, cdi.CDI_NCHUNKS_ROTATED, 0, 2]:
        g.set_run_depth(2, nch)
        out = run(g, phi, nsteps, prm)
        assert torch.equal(out, ref), (nch, (out - ref).abs().max().item())
    g.set_run_depth(1)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch_same_bits_as_single_grid(dtype):
    shapes = [(20, 48, 128), (9, 21, 68), (1, 40, 128), (5, 7, 8), (12, 33, 35)]
    singles, boxes = [], []
    for i, s in enumerate(shapes):
        g, phi, vel, (dt, eps, gamma) = setup(s, dtype, 40 + i)
        g.set_launch(cdi.CDI_KERNEL_FORWARD, 0, 0, 1)
        singles.append(run(g, phi, 3, (dt, eps, gamma)))
        boxes.append(dict(dx=1.0 / max(s), dt=dt, eps=eps, gamma=gamma, u=vel[0], v=vel[1], w=vel[2],
                          phi_a=phi.clone(), phi_b=torch.empty_like(phi)))
    checked = 0
    for tile in range(cdi.BATCH_TILES):
        fresh = [dict(x, phi_a=x["phi_a"].clone(), phi_b=torch.empty_like(x["phi_b"])) for x in boxes]
        b = cdi.Batch(fresh)
        try:
            b.set_launch(tile, 0)
        except cdi.CDIError:
            continue
        for _ in range(3):
            b.step(1.0)
        for i, ref in enumerate(singles):
            out = b.current(i)
            assert torch.equal(out, ref), (tile, i, (out - ref).abs().max().item())
        checked += 1
    assert checked >= 4
