"""GPU Runge-Kutta steps (Section 2.3, Eq. 26-28) against the oracle's schemes."""
import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("scheme", ["euler", "rk2", "rk3", "rk4"])
@pytest.mark.parametrize("shape", [(6, 20, 64), (5, 9, 37), (1, 40, 96)])
def test_rk_step_parity(dtype, scheme, shape):
    h = 1.0 / max(shape)
    phi = I.random_phi(shape, 7, smooth=True)
    u, v, w = I.random_velocity(shape, h, 8, 3, 11)
    U = I.face_umax(u, v, w)
    eps, gamma = h, U
    lim = {"euler": 1.0, "rk2": 1.0, "rk3": 2.51 / 2, "rk4": 2.79 / 2}[scheme]
    Df = sum(1 for s in shape if s > 1)
    dt = 0.9 * lim * h * h / (2 * Df * gamma * eps)
    t = np.float64 if dtype == torch.float64 else np.float32
    rin = [np.asarray(x, t).astype(np.float64) for x in (phi, u, v, w)]
    nz, ny, nx = shape
    g = cdi.Grid(nx, ny, nz, h, dtype)
    vel = [dev(x, dtype) for x in (u, v, w)]
    g.set_velocity(*vel)
    a = dev(phi, dtype)
    b = torch.empty_like(a)
    w1, w2 = torch.empty_like(a), torch.empty_like(a)
    g.reset_run_stats()
    out = g.run_rk(a, b, w1, w2, 3, dt, eps, gamma, scheme, period=0.7, t0=0.05, check=True)
    st = g.stats()
    ref = oracle.rk_run(*rin, h, dt, eps, gamma, 3, scheme, period=0.7, t0=0.05)
    tol = 1e-12 if dtype == torch.float64 else 4e-6
    ours = out.double().cpu().numpy()
    assert np.abs(ours - ref).max() <= tol
    assert st["steps_run"] == 3 and st["n_tol_run"] == 0
    assert st["min"] == ours.min() and st["max"] == ours.max()
    assert abs(st["sum"] - rin[0].sum()) <= (1e-12 if dtype == torch.float64 else 1e-6) * rin[0].sum()


def test_rk_input_preserved_and_checked():
    shape = (8, 16, 64)
    h = 1.0 / 64
    phi = I.random_phi(shape, 2, smooth=True)
    u, v, w = I.random_velocity(shape, h, 8, 3, 5)
    g = cdi.Grid(64, 16, 8, h, torch.float64)
    vel = [dev(x, torch.float64) for x in (u, v, w)]
    g.set_velocity(*vel)
    a = dev(phi, torch.float64)
    a0 = a.clone()
    b, w1, w2 = torch.empty_like(a), torch.empty_like(a), torch.empty_like(a)
    U = g.U
    big = 2.79 / 4 / 3 * h * h / (U * h)  # RK4 limit in 3D, fine for rk4
    g.step_rk(a, b, w1, w2, 0.99 * big, h, U, "rk4", check=True)
    assert torch.equal(a, a0)
    with pytest.raises(cdi.CDIError) as e:
        g.step_rk(a, b, w1, w2, 0.99 * big, h, U, "rk2", check=True)  # beyond Eq. 26
    assert e.value.code == cdi.CDI_ERR_CONDITION
    with pytest.raises(cdi.CDIError):
        g.step_rk(a, b, a, w2, 0.5 * big, h, U, "rk4")  # work array aliases the input
