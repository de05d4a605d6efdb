"""GPU parity of the discrete-adjoint step against the FP64 oracle adjoint."""
import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def case(shape, seed, smooth):
    h = 1.0 / max(shape)
    phi = 0.02 + 0.96 * I.random_phi(shape, seed, smooth=smooth)
    u, v, w = I.random_velocity(shape, h, 8, 3, seed + 1)
    lam = np.random.default_rng(seed + 2).standard_normal(shape)
    return phi, u, v, w, lam, h


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", [(1, 1, 29), (1, 23, 17), (5, 6, 7), (17, 21, 66), (2, 3, 40)])
@pytest.mark.parametrize("with_vel", [False, True])
def test_adjoint_parity(dtype, shape, with_vel):
    smooth = dtype == torch.float32
    phi, u, v, w, lam, h = case(shape, 7 + sum(shape), smooth)
    t = np.float64 if dtype == torch.float64 else np.float32
    phi, u, v, w, lam = (np.asarray(x, t).astype(np.float64) for x in (phi, u, v, w, lam))
    dt, eps, gamma, vs = 0.15 * h * h / (1.3 * 1.1 * h), 1.1 * h, 1.3, 0.7
    nz, ny, nx = shape
    g = cdi.Grid(nx, ny, nz, h, dtype)
    vel = [dev(x, dtype) for x in (u, v, w)]
    g.set_velocity(*vel)
    out = torch.empty(shape, dtype=dtype, device="cuda")
    grads = None
    if with_vel:
        g0 = np.random.default_rng(1).standard_normal((3,) + shape)
        grads = [dev(x, dtype) for x in g0]
    g.step_adjoint(dev(phi, dtype), dev(lam, dtype), out, dt, eps, gamma, vs, grads=grads)
    ref = oracle.adjoint(phi, u, v, w, lam, h, dt, eps, gamma, vs, want_vel=with_vel,
                         tiny=oracle.adjoint_floor_of(t))
    if with_vel:
        ref, rgu, rgv, rgw = ref
    scale = max(1.0, np.abs(ref).max())
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert np.abs(out.double().cpu().numpy() - ref).max() <= tol * scale
    if with_vel:
        for gd, rg, base in zip(grads, (rgu, rgv, rgw), g0):
            base = np.asarray(base, t).astype(np.float64)
            s2 = max(1.0, np.abs(rg).max())
            assert np.abs(gd.double().cpu().numpy() - (base + rg)).max() <= tol * s2 * 4


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("tile", range(cdi.ADJ_TILES))
@pytest.mark.parametrize("shape,nchunks", [((9, 21, 68), 0), ((1, 40, 128), 1), ((3, 10, 8), 2),
                                           ((6, 13, 96), 3), ((20, 9, 64), 7), ((2, 17, 132), 0)])
@pytest.mark.parametrize("with_vel", [False, True])
def test_adjoint_every_tile(dtype, tile, shape, nchunks, with_vel):
    """Each adjoint kernel (one cell per thread, and the vector kernel where nx allows)
    and z chunking gives the oracle's adjoint step, ragged tiles and chunks included."""
    phi, u, v, w, lam, h = case(shape, 11 + shape[2], dtype == torch.float32)
    t = np.float64 if dtype == torch.float64 else np.float32
    phi, u, v, w, lam = (np.asarray(x, t).astype(np.float64) for x in (phi, u, v, w, lam))
    dt, eps, gamma, vs = 0.15 * h * h / (1.3 * 1.1 * h), 1.1 * h, 1.3, 0.7
    nz, ny, nx = shape
    g = cdi.Grid(nx, ny, nz, h, dtype)
    g.set_velocity(*[dev(x, dtype) for x in (u, v, w)])
    g.set_launch(cdi.CDI_KERNEL_ADJOINT, tile, 0, nchunks)
    assert g.get_launch(cdi.CDI_KERNEL_ADJOINT)["tile"] == tile
    out = torch.empty(shape, dtype=dtype, device="cuda")
    grads = None
    if with_vel:
        g0 = np.random.default_rng(5).standard_normal((3,) + shape)
        grads = [dev(x, dtype) for x in g0]
    g.step_adjoint(dev(phi, dtype), dev(lam, dtype), out, dt, eps, gamma, vs, grads=grads)
    ref = oracle.adjoint(phi, u, v, w, lam, h, dt, eps, gamma, vs, want_vel=with_vel,
                         tiny=oracle.adjoint_floor_of(t))
    if with_vel:
        ref, rgu, rgv, rgw = ref
    scale = max(1.0, np.abs(ref).max())
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert np.abs(out.double().cpu().numpy() - ref).max() <= tol * scale
    if with_vel:
        for gd, rg, base in zip(grads, (rgu, rgv, rgw), g0):
            base = np.asarray(base, t).astype(np.float64)
            s2 = max(1.0, np.abs(rg).max())
            assert np.abs(gd.double().cpu().numpy() - (base + rg)).max() <= tol * s2 * 4


def tail_case(shape, eps_cells, seed):
    """A tanh sphere whose far tails fall through 1e-19 (|g|^2 ~ FLT_MIN) to ~1e-26."""
    nz, ny, nx = shape
    h = 1.0 / nx
    c = (0.5 * nx * h, 0.45 * ny * h, 0.55 * nz * h)
    d = I.sphere_distance(shape, h, c, 6 * h)
    phi = 1.0 / (1.0 + np.exp(-d / (eps_cells * h)))  # = (1 + tanh(d / 2 eps)) / 2, no cancellation
    u, v, w = I.random_velocity(shape, h, 8, 3, seed)
    lam = np.random.default_rng(seed + 1).standard_normal(shape)
    return phi, u, v, w, lam, h


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("tile", range(cdi.ADJ_TILES))
def test_adjoint_floor_regime(dtype, tile):
    """Where |g| falls to the adjoint's floor delta (the tails of a sharp sphere, and its
    bulk next to phi = 1 where FP32 neighbours differ by units in the last place) the
    adjoint differentiates n = g / sqrt(|g|^2 + delta^2): it matches the oracle adjoint with
    that floor on every kernel, and (so that the case means something) in FP32 not the
    oracle's unit-normal adjoint."""
    shape = (24, 20, 64)
    t = np.float32 if dtype == torch.float32 else np.float64
    phi, u, v, w, lam, h = tail_case(shape, 0.5, 3)
    phi, u, v, w, lam = (np.asarray(x, t).astype(np.float64) for x in (phi, u, v, w, lam))
    g2 = sum((np.roll(phi, -1, a) - np.roll(phi, 1, a)) ** 2 for a in (0, 1, 2))
    fl = oracle.adjoint_floor_of(t)
    assert ((g2 > 0) & (g2 < fl)).sum() > 100   # the regime is present
    dt, eps, gamma, vs = 0.1 * h, 0.5 * h, 1.0, 1.0
    g = cdi.Grid(shape[2], shape[1], shape[0], h, dtype)
    g.set_velocity(*[dev(x, dtype) for x in (u, v, w)])
    g.set_launch(cdi.CDI_KERNEL_ADJOINT, tile, 0, 0)
    out = torch.empty(shape, dtype=dtype, device="cuda")
    g.step_adjoint(dev(phi, dtype), dev(lam, dtype), out, dt, eps, gamma, vs)
    ref = oracle.adjoint(phi, u, v, w, lam, h, dt, eps, gamma, vs, tiny=fl)
    unit = oracle.adjoint(phi, u, v, w, lam, h, dt, eps, gamma, vs)
    tol = 2e-6 if dtype == torch.float32 else 1e-12
    scale = max(1.0, np.abs(ref).max())
    got = out.double().cpu().numpy()
    assert np.abs(got - ref).max() <= tol * scale
    if dtype == torch.float32:
        assert np.abs(unit - ref).max() > 1e-4 * scale


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", [(64, 64, 256), (9, 21, 68), (2, 17, 132), (20, 9, 64)])
@pytest.mark.parametrize("with_vel", [False, True])
@pytest.mark.parametrize("split", [cdi.CDI_NCHUNKS_BALANCED, cdi.CDI_NCHUNKS_ROTATED])
def test_adjoint_balanced_split(dtype, shape, with_vel, split):
    """The vector adjoint with equal contiguous tile-plane shares per block (shares cut
    inside a column and one-plane shares) gives the oracle's adjoint step."""
    phi, u, v, w, lam, h = case(shape, 13 + shape[0], dtype == torch.float32)
    t = np.float64 if dtype == torch.float64 else np.float32
    phi, u, v, w, lam = (np.asarray(x, t).astype(np.float64) for x in (phi, u, v, w, lam))
    dt, eps, gamma, vs = 0.15 * h * h / (1.3 * 1.1 * h), 1.1 * h, 1.3, 0.7
    nz, ny, nx = shape
    g = cdi.Grid(nx, ny, nz, h, dtype)
    g.set_velocity(*[dev(x, dtype) for x in (u, v, w)])
    g.set_launch(cdi.CDI_KERNEL_ADJOINT, 3, 0, split)
    assert g.get_launch(cdi.CDI_KERNEL_ADJOINT)["nchunks"] == split
    out = torch.empty(shape, dtype=dtype, device="cuda")
    grads = None
    if with_vel:
        g0 = np.random.default_rng(6).standard_normal((3,) + shape)
        grads = [dev(x, dtype) for x in g0]
    g.step_adjoint(dev(phi, dtype), dev(lam, dtype), out, dt, eps, gamma, vs, grads=grads)
    ref = oracle.adjoint(phi, u, v, w, lam, h, dt, eps, gamma, vs, want_vel=with_vel,
                         tiny=oracle.adjoint_floor_of(t))
    if with_vel:
        ref, rgu, rgv, rgw = ref
    scale = max(1.0, np.abs(ref).max())
    tol = 1e-12 if dtype == torch.float64 else 2e-6
    assert np.abs(out.double().cpu().numpy() - ref).max() <= tol * scale
    if with_vel:
        for gd, rg, base in zip(grads, (rgu, rgv, rgw), g0):
            base = np.asarray(base, t).astype(np.float64)
            s2 = max(1.0, np.abs(rg).max())
            assert np.abs(gd.double().cpu().numpy() - (base + rg)).max() <= tol * s2 * 4
    with pytest.raises(cdi.CDIError):
        g.set_launch(cdi.CDI_KERNEL_ADJOINT, 0, 0, split)


def test_adjoint_constant_lambda_gpu():
    """lam' = const gives lam = lam' exactly (J^T 1 = 1 from conservation)."""
    shape = (6, 10, 40)
    phi, u, v, w, lam, h = case(shape, 3, False)
    g = cdi.Grid(40, 10, 6, h, torch.float64)
    vel = [dev(x, torch.float64) for x in (u, v, w)]
    g.set_velocity(*vel)
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    l1 = torch.full(shape, 2.5, dtype=torch.float64, device="cuda")
    g.step_adjoint(dev(phi, torch.float64), l1, out, 0.1 * h * h, h, 1.0, 1.0)
    assert torch.all(out == 2.5)


def test_adjoint_dot_product_gpu():
    """<J dphi, lam> with J dphi from GPU forward FD == <dphi, J^T lam> from the GPU adjoint."""
    shape = (12, 16, 40)
    phi, u, v, w, lam, h = case(shape, 11, True)
    dt, eps, gamma = 0.1 * h * h / (1.2 * h), 1.2 * h, 1.0
    g = cdi.Grid(40, 16, 12, h, torch.float64)
    vel = [dev(x, torch.float64) for x in (u, v, w)]
    g.set_velocity(*vel)
    dphi = np.random.default_rng(5).standard_normal(shape)
    hh = 1e-6
    a = torch.empty(shape, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    g.step(dev(phi + hh * dphi, torch.float64), a, dt, eps, gamma)
    g.step(dev(phi - hh * dphi, torch.float64), b, dt, eps, gamma)
    jv = ((a - b) / (2 * hh)).cpu().numpy()
    out = torch.empty_like(a)
    g.step_adjoint(dev(phi, torch.float64), dev(lam, torch.float64), out, dt, eps, gamma)
    lhs, rhs = (jv * lam).sum(), (dphi * out.cpu().numpy()).sum()
    assert abs(lhs - rhs) <= 1e-7 * (abs(lhs) + abs(rhs))
