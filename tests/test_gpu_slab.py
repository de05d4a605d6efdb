"""The z-slab decomposition on one GPU: cdi_step_planes against the oracle, and two or three
slabs of one box in one process, exchanging halos by device copies through the same plan as
the multi-rank path, stepped by the CUDA library and compared with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I
from paper_1803_01262_gb300 import slab as S

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-6}
NPT = {torch.float64: np.float64, torch.float32: np.float32}


def _fields(shape, seed):
    h = 1.0 / max(shape)
    phi = I.random_phi(shape, seed, smooth=True)
    u, v, w = I.random_velocity(shape, h, 8, 3, seed + 1)
    return phi, u, v, w, h


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape,zr", [((20, 24, 64), (3, 17)), ((9, 17, 45), (0, 9)), ((12, 16, 32), (2, 10)),
                                      ((6, 5, 7), (5, 6))])
def test_step_planes(dtype, shape, zr):
    phi, u, v, w, h = _fields(shape, 3 + shape[0])
    nz, ny, nx = shape
    eps, gamma = 1.2 * h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    g = cdi.Grid(nx, ny, nz, h, dtype)
    vel = [torch.from_numpy(x).to("cuda", dtype) for x in (u, v, w)]
    g.set_velocity(*vel)
    a = torch.from_numpy(phi).to("cuda", dtype)
    b = torch.full_like(a, 7.0)
    g.step_planes(a, b, zr[0], zr[1], dt, eps, gamma, 0.8)
    st = g.stats()
    r = [np.asarray(x, NPT[dtype]).astype(np.float64) for x in (phi, u, v, w)]
    ref = oracle.step(*r, h, dt, eps, gamma, 0.8, tiny=oracle.floor_of(NPT[dtype]))
    got = b.double().cpu().numpy()
    assert np.abs(got[zr[0]:zr[1]] - ref[zr[0]:zr[1]]).max() <= TOL[dtype]
    outside = np.ones(nz, bool)
    outside[zr[0]:zr[1]] = False
    assert (got[outside] == 7.0).all()
    rs = oracle.stats(ref[zr[0]:zr[1]], h ** 3, 0.0)
    assert st["sum"] == pytest.approx(rs["sum"], rel=1e-12 if dtype == torch.float64 else 1e-6)
    assert st["steps_run"] == 1


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape,world", [((32, 24, 64), 2), ((19, 17, 45), 3), ((40, 16, 128), 2), ((8, 8, 8), 1)])
def test_slabs_on_one_gpu_match_oracle(dtype, shape, world):
    phi, u, v, w, h = _fields(shape, 21 + world)
    eps, gamma = 1.2 * h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    T = [torch.from_numpy(x).to("cuda", dtype) for x in (phi, u, v, w)]
    doms = [S.SlabDomain(r, world, *T, h) for r in range(world)]
    run = S.SlabRun(doms, S.LocalTransport())
    r = [np.asarray(x, NPT[dtype]).astype(np.float64) for x in (phi, u, v, w)]
    tiny = oracle.floor_of(NPT[dtype])
    nsteps = 3 if dtype == torch.float64 else 1
    ref = r[0]
    for i in range(nsteps):
        vs = 1.0 - 0.4 * i
        run.step(dt, eps, gamma, vs)
        ref = oracle.step(ref, *r[1:], h, dt, eps, gamma, vs, tiny=tiny)
    got = run.gather_local().double().cpu().numpy()
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= TOL[dtype] * nsteps
    st = run.stats()
    rs = oracle.stats(ref, h ** 3, float(np.finfo(NPT[dtype]).eps))
    assert st["sum"] == pytest.approx(rs["sum"], rel=1e-12 if dtype == torch.float64 else 1e-6)
    assert st["n_tol"] == rs["n_tol"] == 0
    # a slab's velocity arrays are its planes and halos of the full arrays
    for d in doms:
        idx = [(z % shape[0]) for z in range(d.z_begin - S.HALO, d.z_end + S.HALO)]
        assert torch.equal(d.w, T[3][idx])
