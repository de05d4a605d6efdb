"""The non-default face-product sharpening (CDI_SHARPEN_FACE) against the oracle's face form."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I
from paper_1803_01262_gb300 import phase as P

pytestmark = pytest.mark.gpu
TOL = {torch.float64: 1e-12, torch.float32: 1e-6}
NPT = {torch.float64: np.float64, torch.float32: np.float32}


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def case(shape, seed, dtype):
    h = 1.0 / max(shape)
    phi = 0.02 + 0.96 * I.random_phi(shape, seed, smooth=True)
    u, v, w = I.random_velocity(shape, h, 8, 3, seed + 1)
    t = NPT[dtype]
    return [np.asarray(x, t).astype(np.float64) for x in (phi, u, v, w)] + [h]


def face_grid(shape, h, dtype, vel):
    nz, ny, nx = shape
    g = cdi.Grid(nx, ny, nz, h, dtype)
    g.set_velocity(*[dev(x, dtype) for x in vel])
    g.set_sharpening("face")
    assert g.get_sharpening() == "face" and g.get_launch()["tile"] == 0
    return g


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", [(1, 1, 29), (1, 23, 17), (5, 6, 7), (9, 21, 68), (20, 33, 40)])
@pytest.mark.parametrize("nchunks", [0, 3, cdi.CDI_NCHUNKS_BALANCED])
def test_face_step_parity(dtype, shape, nchunks):
    phi, u, v, w, h = case(shape, 5 + sum(shape), dtype)
    g = face_grid(shape, h, dtype, (u, v, w))
    g.set_launch(cdi.CDI_KERNEL_FORWARD, 0, 0, nchunks)
    dt, eps, gamma = 0.12 * h * h / (1.1 * h), 1.1 * h, 1.0
    a = dev(phi, dtype)
    b = torch.empty_like(a)
    g.step(a, b, dt, eps, gamma, 0.8)
    st = g.stats()
    ref = oracle.step(phi, u, v, w, h, dt, eps, gamma, 0.8, tiny=oracle.floor_of(NPT[dtype]), sharpen="face")
    ours = b.double().cpu().numpy()
    assert np.abs(ours - ref).max() <= TOL[dtype]
    assert st["min"] == ours.min() and st["max"] == ours.max()
    # and it is a different scheme from the default one
    cen = oracle.step(phi, u, v, w, h, dt, eps, gamma, 0.8)
    assert np.abs(cen - ref).max() > 1e-6


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_face_run_parity_and_modes(dtype):
    shape = (12, 20, 36)
    phi, u, v, w, h = case(shape, 41, dtype)
    g = face_grid(shape, h, dtype, (u, v, w))
    dt, eps, gamma = 0.1 * h, h, 1.2
    a, b = dev(phi, dtype), torch.empty(shape, dtype=dtype, device="cuda")
    out = g.run(a, b, 25, dt, eps, gamma, period=0.9)
    ref = oracle.run(phi, u, v, w, h, dt, eps, gamma, 25, period=0.9, sharpen="face",
                     tiny=oracle.floor_of(NPT[dtype]))
    assert np.abs(out.double().cpu().numpy() - ref).max() <= 50 * TOL[dtype]
    # the centre-only paths refuse the face form
    lam = torch.zeros_like(a)
    with pytest.raises(cdi.CDIError):
        g.step_adjoint(a, lam, torch.empty_like(a), dt, eps, gamma)
    with pytest.raises(cdi.CDIError):
        g.step_rk(a, b, torch.empty_like(a), torch.empty_like(a), dt, eps, gamma, "rk2")
    with pytest.raises(cdi.CDIError):
        g.set_launch(cdi.CDI_KERNEL_FORWARD, 4, 0, 0)
    # back to the default form and launch
    g.set_sharpening("centre")
    g.step(dev(phi, dtype), b, dt, eps, gamma)
    cen = oracle.step(phi, u, v, w, h, dt, eps, gamma, tiny=oracle.floor_of(NPT[dtype]))
    assert np.abs(b.double().cpu().numpy() - cen).max() <= TOL[dtype]


def test_face_host_step():
    """cdi_step_host in the face form (nz >= 16: unpipelined) equals the device step."""
    shape = (20, 12, 16)
    phi, u, v, w, h = case(shape, 3, torch.float64)
    g = face_grid(shape, h, torch.float64, (u, v, w))
    dt, eps, gamma = 0.1 * h, h, 1.0
    hout = np.empty(shape)
    g.step_host(np.ascontiguousarray(phi), hout, dt, eps, gamma)
    d = torch.empty(shape, dtype=torch.float64, device="cuda")
    g.step(dev(phi, torch.float64), d, dt, eps, gamma)
    assert np.array_equal(hout, d.cpu().numpy())


def test_face_form_boundedness_on_table2_points():
    """Empirical boundedness of the face form (not covered by the proof) on Table 2's seven
    points, one period each with the Table 2 step: the GPU classification equals the oracle's, and
    the face form loses point 5, which the centre form keeps."""
    outcome = []
    tol = np.finfo(np.float64).eps
    for eoh, gu in ((1.5, 0.5), (1.0, 1.0), (5 / 6, 1.5), (1.5, 1.5), (0.9, 0.9), (0.8, 0.8), (0.7, 0.7)):
        f, _ = I.drop_2d_uniform(eoh)
        dt = P.euler_dt(eoh, gu)
        nst = int(math.ceil(P.PERIOD / dt))
        g = face_grid(f.phi.shape, f.h, torch.float64, (f.u, f.v, f.w))
        a, b = dev(f.phi, torch.float64), torch.empty(f.phi.shape, dtype=torch.float64, device="cuda")
        g.reset_run_stats()
        g.run(a, b, nst, dt, eoh * f.h, gu)
        gpu_bad = g.stats()["n_tol_run"]
        p, bad = f.phi, 0
        for _ in range(nst):
            p = oracle.step(p, f.u, f.v, f.w, f.h, dt, eoh * f.h, gu, sharpen="face")
            bad += int(((p < -tol) | (p > 1 + tol)).sum())
        assert (gpu_bad == 0) == (bad == 0), (eoh, gu, gpu_bad, bad)
        outcome.append(bad == 0)
    # point 5 meets the sufficient condition and stays bounded with the centre form
    # (Table 2), but not with the face form
    assert outcome == [True] * 4 + [False] * 3, outcome
