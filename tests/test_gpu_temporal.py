"""Two Euler steps per pass (cdi_run at depth 2, temporal blocking) against one step per
launch on forward tile 4 and against the FP64 oracle; the statistics of both steps of a pass
in the run accumulators.  The two paths evaluate the same expressions in the same order (no
fused multiply-add beyond those the sources write), so although they split the planes into
different work units, and a unit's first z face is evaluated in its prologue rather than
carried from the plane below, they agree bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-6}
NPT = {torch.float64: np.float64, torch.float32: np.float32}


def _setup(shape, dtype, seed):
    h = 1.0 / max(shape)
    phi = I.random_phi(shape, seed, smooth=True)
    u, v, w = I.random_velocity(shape, h, 8, 3, seed + 1)
    nz, ny, nx = shape
    g = cdi.Grid(nx, ny, nz, h, dtype)
    vel = [torch.from_numpy(x).to("cuda", dtype) for x in (u, v, w)]
    g.set_velocity(*vel)
    return g, vel, (phi, u, v, w), h


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", [(20, 24, 64), (9, 21, 68), (33, 20, 72), (5, 7, 8), (1, 40, 128),
                                   (40, 16, 128), (2, 33, 36), (64, 32, 64)])
@pytest.mark.parametrize("nchunks", [-1, -2, 0, 3])
def test_two_steps_per_pass_bit_for_bit(dtype, shape, nchunks):
    g, vel, f, h = _setup(shape, dtype, 7 + shape[0])
    eps, gamma = 1.2 * h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    phi0 = torch.from_numpy(f[0]).to("cuda", dtype)
    nsteps = 5
    g.set_launch(cdi.CDI_KERNEL_FORWARD, 4, 0, nchunks)
    g.set_run_depth(1)
    g.reset_run_stats()
    a, b = phi0.clone(), torch.empty_like(phi0)
    r1 = g.run(a, b, nsteps, dt, eps, gamma, period=0.7, t0=0.05).clone()
    s1 = g.stats()
    g.set_run_depth(2, nchunks)
    assert g.get_run_depth()["depth"] == 2
    g.reset_run_stats()
    a, b = phi0.clone(), torch.empty_like(phi0)
    r2 = g.run(a, b, nsteps, dt, eps, gamma, period=0.7, t0=0.05)
    s2 = g.stats()
    assert torch.equal(r1, r2)
    for k in ("min", "max", "min_run", "max_run"):
        assert s1[k] == s2[k], k
    for k in ("n_strict", "n_tol", "n_strict_run", "n_tol_run", "steps_run"):
        assert s1[k] == s2[k], k
    assert s2["steps_run"] == nsteps
    assert s2["sum"] == pytest.approx(s1["sum"], rel=1e-13 if dtype == torch.float64 else 1e-6)
    # an even count ends on a two-step pass: its second step's record
    g.reset_run_stats()
    a, b = phi0.clone(), torch.empty_like(phi0)
    r4 = g.run(a, b, 4, dt, eps, gamma, period=0.7, t0=0.05)
    s4 = g.stats()
    rin = [np.asarray(x, NPT[dtype]).astype(np.float64) for x in f]
    ref = oracle.run(*rin, h, dt, eps, gamma, 4, period=0.7, t0=0.05, tiny=oracle.floor_of(NPT[dtype]))
    got = r4.double().cpu().numpy()
    assert np.abs(got - ref).max() <= 4 * TOL[dtype]
    assert s4["steps_run"] == 4 and s4["min"] == got.min() and s4["max"] == got.max()
    assert s4["sum"] == pytest.approx(got.sum(), rel=1e-12 if dtype == torch.float64 else 1e-6)


def test_run_depth_refusals_and_autotune():
    g, vel, f, h = _setup((6, 8, 30), torch.float32, 3)   # nx % 4 != 0
    with pytest.raises(cdi.CDIError):
        g.set_run_depth(2)
    with pytest.raises(cdi.CDIError):
        g.set_run_depth(3)
    g2, vel2, f2, h2 = _setup((24, 32, 64), torch.float32, 4)
    g2.set_sharpening("face")
    with pytest.raises(cdi.CDIError):
        g2.set_run_depth(2)
    g2.set_sharpening("centre")
    a = torch.from_numpy(f2[0]).to("cuda", torch.float32)
    b = torch.empty_like(a)
    ms = g2.autotune(a.clone(), b, 0.01 * h2, h2, 1.0, reps=2)
    assert ms > 0 and g2.get_run_depth()["depth"] in (1, 2)
