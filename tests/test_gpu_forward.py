"""GPU parity of the fused forward CDI step against the FP64 oracle.

Every test goes through the C ABI (libcdi.so via the ctypes binding) on
seeded synthetic inputs.  Tolerances: FP64 1e-12 absolute per step; FP32
1e-6 absolute per step against the oracle evaluated in FP64 on the same
FP32-rounded inputs.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-6}
NPT = {torch.float64: np.float64, torch.float32: np.float32}


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rounded(f, dtype):
    """The inputs as the GPU sees them, back in float64 for the oracle."""
    t = NPT[dtype]
    return [np.asarray(x, dtype=t).astype(np.float64) for x in (f.phi, f.u, f.v, f.w)]


def make_grid(f, dtype):
    nz, ny, nx = f.phi.shape
    g = cdi.Grid(nx, ny, nz, f.h, dtype)
    vel = [dev(x, dtype) for x in (f.u, f.v, f.w)]
    g.set_velocity(*vel)
    return g, vel


def gpu_step(f, dtype, dt, eps, gamma, vs=1.0):
    g, _ = make_grid(f, dtype)
    a = dev(f.phi, dtype)
    b = torch.empty_like(a)
    g.step(a, b, dt, eps, gamma, vs)
    st = g.stats()
    return b.double().cpu().numpy(), st, g


def random_fields(shape, seed, solenoidal=True, smooth=False):
    h = 1.0 / max(shape)
    phi = I.random_phi(shape, seed, smooth=smooth)
    if solenoidal:
        u, v, w = I.random_velocity(shape, h, 8, 3, seed + 7)
    else:
        rng = np.random.default_rng(seed + 3)
        u, v, w = (rng.uniform(-1, 1, shape) for _ in range(3))
    return I.Fields(phi, u, v, w, h, I.face_umax(u, v, w))


SHAPES = [(1, 1, 1), (1, 1, 37), (1, 5, 3), (3, 1, 8), (2, 3, 4), (7, 19, 45), (33, 20, 70),
          (1, 130, 67), (19, 17, 40)]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("solenoidal", [True, False])
def test_step_parity(dtype, shape, solenoidal):
    f = random_fields(shape, 100 + sum(shape), solenoidal)
    eps, gamma = 1.2 * f.h, 1.1
    dt = 0.1 * f.h * f.h / (gamma * eps)
    ours, st, _ = gpu_step(f, dtype, dt, eps, gamma, 0.9)
    phi, u, v, w = rounded(f, dtype)
    ref = oracle.step(phi, u, v, w, f.h, dt, eps, gamma, 0.9)
    assert np.abs(ours - ref).max() <= TOL[dtype]
    # fused reductions of phi' against the oracle's plain sums of the reference
    rs = oracle.stats(ref, f.h ** sum(1 for s in shape if s > 1), 0.0)
    n = ref.size
    assert abs(st["sum"] - rs["sum"]) <= TOL[dtype] * n
    assert abs(st["min"] - rs["min"]) <= TOL[dtype] and abs(st["max"] - rs["max"]) <= TOL[dtype]
    # FP64 sums directly; FP32 keeps compensated float partials (Kahan bound ~1e-7 relative)
    assert abs(st["sum"] - ours.sum()) <= (1e-12 * n if dtype == torch.float64 else 1e-7 * abs(ours.sum()))
    assert st["min"] == ours.min() and st["max"] == ours.max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_single_vortex_128_parity_and_invariants(dtype):
    """128 x 128 drop in the single vortex (Section 3.3.1, Eq. 33), eps = dx, gamma = U."""
    f = I.single_vortex_2d(128)
    eps, gamma = f.h, f.U
    dt = 0.1 * f.h / f.U
    g, vel = make_grid(f, dtype)
    a = dev(f.phi, dtype)
    b = torch.empty_like(a)
    g.reset_run_stats()
    out = g.run(a, b, 200, dt, eps, gamma, period=4.0, check=True)
    st = g.stats()
    phi, u, v, w = rounded(f, dtype)
    ref = oracle.run(phi, u, v, w, f.h, dt, eps, gamma, 200, period=4.0)
    err = np.abs(out.double().cpu().numpy() - ref).max()
    assert err <= (1e-11 if dtype == torch.float64 else 2e-5), err
    assert st["steps_run"] == 200 and st["n_tol_run"] == 0
    m0 = phi.sum()
    assert abs(st["sum"] - m0) / m0 <= (1e-13 if dtype == torch.float64 else 1e-6)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_deformation_256_full_size(dtype):
    """The 256^3 deformation workload, one step in the bench's launch configuration."""
    f = I.deformation_3d(256)
    eps, gamma = f.h, f.U
    dt = 0.1 * f.h / f.U
    ours, st, _ = gpu_step(f, dtype, dt, eps, gamma, 1.0)
    phi, u, v, w = rounded(f, dtype)
    ref = oracle.step(phi, u, v, w, f.h, dt, eps, gamma, 1.0)
    assert np.abs(ours - ref).max() <= TOL[dtype]
    assert st["n_tol"] == 0
    assert abs(st["sum"] - phi.sum()) / phi.sum() <= (1e-13 if dtype == torch.float64 else 1e-6)


def test_run_equals_steps_and_host_step():
    f = random_fields((9, 14, 33), 5, smooth=True)
    dt, eps, gamma = 0.1 * f.h, f.h, 1.0
    dt = 0.1 * f.h * f.h / (gamma * eps)
    g, vel = make_grid(f, torch.float64)
    a, b = dev(f.phi, torch.float64), torch.empty(f.phi.shape, dtype=torch.float64, device="cuda")
    x = g.run(a.clone(), b, 7, dt, eps, gamma, period=0.5, t0=0.1)
    p = a.clone()
    q = torch.empty_like(p)
    for i in range(7):
        g.step(p, q, dt, eps, gamma, math.cos(math.pi * (0.1 + i * dt) / 0.5))
        p, q = q, p
    assert torch.equal(x, p)
    hin = np.ascontiguousarray(f.phi)
    hout = np.empty_like(hin)
    st = g.step_host(hin, hout, dt, eps, gamma, 0.3)
    g.step(a, q, dt, eps, gamma, 0.3)
    assert np.array_equal(hout, q.cpu().numpy())
    assert st["sum"] == pytest.approx(hout.sum(), rel=1e-14)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", [(40, 24, 64), (17, 10, 20), (16, 8, 8), (64, 33, 36)])
def test_host_step_slab_pipeline(dtype, shape):
    """cdi_step_host for nz >= 16 runs 8 z slabs through two copy streams and the kernel
    (slabs of two planes included): the result equals the device step to the kernels'
    parity tolerance (the slabs run the vector kernel where nx allows, the full step the
    grid's tuned tile), the statistics likewise, one run step per call."""
    f = random_fields(shape, 21 + shape[0], True, smooth=True)
    dt, eps, gamma = 0.1 * f.h * f.h / (1.1 * f.h), 1.1 * f.h, 1.0
    g, vel = make_grid(f, dtype)
    t = NPT[dtype]
    hin = torch.from_numpy(np.asarray(f.phi, t)).pin_memory().numpy()
    hout = torch.empty(shape, dtype=dtype).pin_memory().numpy()
    g.reset_run_stats()
    st = g.step_host(hin, hout, dt, eps, gamma, 0.7)
    st = g.step_host(hin, hout, dt, eps, gamma, 0.7)
    assert st["steps_run"] == 2
    d = torch.empty(shape, dtype=dtype, device="cuda")
    g.step(dev(f.phi, dtype), d, dt, eps, gamma, 0.7)
    sd = g.stats()
    assert np.abs(hout - d.cpu().numpy()).max() <= TOL[dtype]
    assert st["min"] == hout.min() and st["max"] == hout.max()
    assert st["n_strict"] == sd["n_strict"] and st["n_tol"] == sd["n_tol"]
    assert st["sum"] == pytest.approx(hout.astype(np.float64).sum(), rel=1e-13 if dtype == torch.float64 else 1e-7)
    assert st["mass"] == pytest.approx(sd["mass"], rel=1e-12 if dtype == torch.float64 else 1e-6)
    # non-pinned host arrays take the same path
    out2 = np.empty_like(hout)
    g.step_host(np.ascontiguousarray(hin), out2, dt, eps, gamma, 0.7)
    assert np.array_equal(out2, hout)


def test_bounded_wait_timeout_is_reported():
    """A bounded device wait that runs out (an mbarrier nothing completes) ends its kernel
    after the limit and is reported as CDI_ERR_TIMEOUT; the context and the grid stay
    usable: the next step's statistics are clean."""
    import time
    f = random_fields((8, 12, 16), 4, True, smooth=True)
    g, vel = make_grid(f, torch.float32)
    t0 = time.perf_counter()
    with pytest.raises(cdi.CDIError) as e:
        g.probe_bounded_wait(0.05)
    assert e.value.code == cdi.CDI_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    a = dev(f.phi, torch.float32)
    b = torch.empty_like(a)
    dt = 0.1 * f.h * f.h / f.h
    g.step(a, b, dt, f.h, 1.0)
    st = g.stats()                      # raises if the status word were still set
    assert st["n_tol"] == 0
    with pytest.raises(cdi.CDIError):
        g.probe_bounded_wait(5.0)       # limit out of range


def test_condition_flag():
    f = I.single_vortex_2d(32)
    g, vel = make_grid(f, torch.float64)
    a = dev(f.phi, torch.float64)
    b = torch.empty_like(a)
    U = g.U
    assert U == pytest.approx(f.U, rel=1e-15)
    dt = 0.1 * f.h / U
    g.step(a, b, dt, f.h, U, 1.0, check=True)                # on the crossover line
    with pytest.raises(cdi.CDIError) as e:
        g.step(a, b, dt, 0.8 * f.h, 0.8 * U, 1.0, check=True)  # below it
    assert e.value.code == cdi.CDI_ERR_CONDITION
    with pytest.raises(cdi.CDIError) as e:
        g.step(a, b, 0.3 * f.h / U, f.h, U, 1.0, check=True)   # A > 1/4
    assert e.value.code == cdi.CDI_ERR_CONDITION
    g.step(a, b, 0.3 * f.h / U, f.h, U, 1.0, check=False)      # allowed when unchecked


def test_argument_errors():
    f = random_fields((4, 5, 6), 1)
    g, vel = make_grid(f, torch.float32)
    a = dev(f.phi, torch.float32)
    with pytest.raises(cdi.CDIError) as e:
        g.step(a, a, 1e-3, f.h, 1.0)
    assert e.value.code == cdi.CDI_ERR_ARG
    with pytest.raises(ValueError):
        g.step(a, torch.empty(3, 3, 3, device="cuda"), 1e-3, f.h, 1.0)
    with pytest.raises(cdi.CDIError):
        cdi.Grid(0, 4, 4, 0.1)
    h = cdi.Grid(6, 5, 4, 0.1)
    with pytest.raises(cdi.CDIError) as e:
        h.step(a, torch.empty_like(a), 1e-3, 0.1, 1.0)
    assert e.value.code == cdi.CDI_ERR_STATE


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_mass_and_bounds_planted(dtype):
    shape = (13, 27, 41)
    p = I.random_phi(shape, 3)
    p[0, 0, 0], p[5, 6, 7], p[12, 26, 40] = -0.25, 1.5, -1e-30
    t = NPT[dtype]
    tol = float(np.finfo(t).eps)
    p[1, 1, 1] = 1.0 + tol            # inside the tolerant bound, outside [0, 1]
    p[3, 3, 3] = -0.0                 # not below 0 (the FP64 range tests run on integer keys)
    g = cdi.Grid(shape[2], shape[1], shape[0], 0.1, dtype)
    s = g.mass_and_bounds(dev(p, dtype))
    pr = p.astype(t).astype(np.float64)
    rs = oracle.stats(pr, 0.1 ** 3, tol)
    assert s["n_strict"] == rs["n_strict"] == 4
    assert s["n_tol"] == rs["n_tol"] == 2
    assert s["min"] == rs["min"] and s["max"] == rs["max"]
    assert abs(s["sum"] - rs["sum"]) <= 1e-12 * p.size
    assert abs(s["mass"] - rs["mass"]) <= 1e-12 * p.size


def test_nan_detected():
    f = random_fields((4, 8, 32), 2)
    f.phi[2, 3, 4] = np.nan
    g, vel = make_grid(f, torch.float32)
    a = dev(f.phi, torch.float32)
    b = torch.empty_like(a)
    g.step(a, b, 1e-4, f.h, 1.0)
    with pytest.raises(cdi.CDIError) as e:
        g.stats()
    assert e.value.code == cdi.CDI_ERR_NAN


def test_reproducible_reduction():
    f = I.deformation_3d(64)
    g, vel = make_grid(f, torch.float32)
    a = dev(f.phi, torch.float32)
    b = torch.empty_like(a)
    sums = []
    for _ in range(3):
        g.step(a, b, 0.1 * f.h / f.U, f.h, f.U)
        sums.append(g.stats()["sum"])
    assert sums[0] == sums[1] == sums[2]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("tile", range(cdi.FWD_TILES))
@pytest.mark.parametrize("shape,nchunks", [((9, 21, 68), 0), ((11, 18, 136), 3), ((1, 40, 128), 1),
                                           ((5, 7, 4), 2), ((20, 33, 72), 7), ((7, 32, 128), 2),
                                           ((1, 16, 64), 1), ((3, 48, 192), 0)])
def test_every_launch_configuration(dtype, tile, shape, nchunks):
    """Each kernel variant and z chunking gives the oracle's step (ragged tiles included)."""
    W = 64 if dtype == torch.float32 else 32
    if tile == 6 and (shape[2] % W or shape[1] % 16):
        pytest.skip("tile 6 needs nx % W == 0 and ny % 16 == 0")
    f = random_fields(shape, 31 + shape[2], True, smooth=(tile % 2 == 0))
    eps, gamma = 1.1 * f.h, 0.9
    dt = 0.12 * f.h * f.h / (gamma * eps)
    g, vel = make_grid(f, dtype)
    g.set_launch(cdi.CDI_KERNEL_FORWARD, tile, 0, nchunks)
    a = dev(f.phi, dtype)
    b = torch.empty_like(a)
    g.step(a, b, dt, eps, gamma, 0.8)
    st = g.stats()
    phi, u, v, w = rounded(f, dtype)
    ref = oracle.step(phi, u, v, w, f.h, dt, eps, gamma, 0.8)
    ours = b.double().cpu().numpy()
    assert np.abs(ours - ref).max() <= TOL[dtype]
    assert st["min"] == ours.min() and st["max"] == ours.max()
    assert abs(st["sum"] - ours.sum()) <= 1e-7 * abs(ours.sum())  # compensated FP32 partials


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape,tile,bps", [((64, 64, 256), 4, 1), ((64, 64, 256), 0, 1),
                                            ((2, 512, 512), 4, 1), ((2, 512, 512), 1, 1),
                                            ((9, 21, 68), 4, 0), ((9, 21, 68), 3, 0),
                                            ((5, 7, 4), 0, 0), ((16, 32, 128), 6, 1)])
@pytest.mark.parametrize("split", [cdi.CDI_NCHUNKS_BALANCED, cdi.CDI_NCHUNKS_ROTATED])
def test_balanced_split(dtype, shape, tile, bps, split):
    """Equal contiguous shares of the tile-planes per block (CDI_NCHUNKS_BALANCED, and rotated
    columns, CDI_NCHUNKS_ROTATED): shares cut inside a tile column, shares spanning many short
    columns, one-plane shares."""
    f = random_fields(shape, 17 + shape[0], True, smooth=True)
    eps, gamma = 1.1 * f.h, 0.9
    dt = 0.12 * f.h * f.h / (gamma * eps)
    g, vel = make_grid(f, dtype)
    g.set_launch(cdi.CDI_KERNEL_FORWARD, tile, bps, split)
    assert g.get_launch()["nchunks"] == split
    a = dev(f.phi, dtype)
    b = torch.empty_like(a)
    g.step(a, b, dt, eps, gamma, 0.8)
    st = g.stats()
    phi, u, v, w = rounded(f, dtype)
    ref = oracle.step(phi, u, v, w, f.h, dt, eps, gamma, 0.8)
    ours = b.double().cpu().numpy()
    assert np.abs(ours - ref).max() <= TOL[dtype]
    assert st["min"] == ours.min() and st["max"] == ours.max()
    assert abs(st["sum"] - ours.sum()) <= (1e-12 * ours.size if dtype == torch.float64 else 1e-7 * abs(ours.sum()))


def test_autotune_keeps_result():
    f = I.deformation_3d(64)
    g, vel = make_grid(f, torch.float32)
    a = dev(f.phi, torch.float32)
    b = torch.empty_like(a)
    dt = 0.1 * f.h / f.U
    g.step(a, b, dt, f.h, f.U)
    ref = b.clone()
    s1, s2 = torch.empty_like(a), torch.empty_like(a)
    ms = g.autotune(s1, s2, dt, f.h, f.U, reps=2)
    assert ms > 0
    cfg = g.get_launch()
    assert 0 <= cfg["tile"] < cdi.FWD_TILES and cfg["nblocks"] > 0
    g.step(a, b, dt, f.h, f.U)
    assert torch.allclose(b, ref, atol=1e-6, rtol=0)
