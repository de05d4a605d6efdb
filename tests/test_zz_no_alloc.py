"""cdi_step_noalloc against cdi_step and the FP64 oracle, through the C ABI, on two
calls in a row; and that calls after the first allocate no device memory.

cdi_step_noalloc serves callers that may not allocate device memory when
they step (code inside callbacks or allocator hooks, fixed-pool frameworks,
latency-critical loops): it takes no grid object and keeps its reduction
scratch in a fixed array inside the library.  This file is collected last
so that a run stopping at the first failure has run every other test first;
it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import build as B
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-6}


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", [(24, 40, 64), (9, 17, 45), (1, 128, 128)])
def test_noalloc_matches_grid_step_twice(dtype, shape):
    B.build()
    from paper_1803_01262_gb300 import cdi

    h = 1.0 / max(shape)
    phi = I.random_phi(shape, 4, smooth=True)
    u, v, w = I.random_velocity(shape, h, 8, 3, 9)
    du, dv_, dw = (dev(x, dtype) for x in (u, v, w))
    eps, gamma = 1.2 * h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    nz, ny, nx = shape

    g = cdi.Grid(nx, ny, nz, h, dtype)
    g.set_velocity(du, dv_, dw)
    stats_dev = torch.zeros(ctypes.sizeof(cdi.Stats), dtype=torch.uint8, device="cuda")

    a = dev(phi, dtype)
    ref_in = a.clone()
    for call in range(2):  # two calls in a row share the fixed scratch
        vs = 0.9 if call == 0 else -0.4
        out = torch.empty_like(a)
        cdi.step_noalloc(a, out, du, dv_, dw, h, dt, eps, gamma, vs, stats_dev)
        ref = torch.empty_like(a)
        g.step(ref_in, ref, dt, eps, gamma, vs)
        st_ref = g.stats()
        st = cdi.stats_from_device(stats_dev)
        assert (out - ref).abs().max().item() <= TOL[dtype]
        assert st["min"] == pytest.approx(st_ref["min"], abs=TOL[dtype])
        assert st["max"] == pytest.approx(st_ref["max"], abs=TOL[dtype])
        assert st["n_strict"] == st_ref["n_strict"] and st["n_tol"] == st_ref["n_tol"]
        assert st["sum"] == pytest.approx(st_ref["sum"], rel=1e-12 if dtype == torch.float64 else 1e-7)
        assert st["mass"] == pytest.approx(st["sum"] * h ** sum(1 for s in shape if s > 1), rel=1e-14)
        # and against the FP64 oracle on the same input
        npt = np.float64 if dtype == torch.float64 else np.float32
        want = oracle.step(a.double().cpu().numpy(), *(x.double().cpu().numpy() for x in (du, dv_, dw)),
                           h, dt, eps, gamma, vs, tiny=oracle.floor_of(npt))
        assert np.abs(out.double().cpu().numpy() - want).max() <= TOL[dtype]
        a, ref_in = out, ref


def test_noalloc_allocates_nothing_after_the_first_call():
    """After a warm-up call, 100 calls leave the device's free memory unchanged."""
    B.build()
    from paper_1803_01262_gb300 import cdi

    shape = (32, 48, 64)
    h = 1.0 / 64
    phi = torch.from_numpy(I.random_phi(shape, 5, smooth=True)).to("cuda", torch.float32)
    u, v, w = (torch.from_numpy(x).to("cuda", torch.float32) for x in I.random_velocity(shape, h, 8, 3, 2))
    out = torch.empty_like(phi)
    st = torch.zeros(ctypes.sizeof(cdi.Stats), dtype=torch.uint8, device="cuda")
    args = (h, 0.05 * h, 1.2 * h, 1.0, 1.0, st)
    cdi.step_noalloc(phi, out, u, v, w, *args)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for i in range(100):
        cdi.step_noalloc(phi if i % 2 == 0 else out, out if i % 2 == 0 else phi, u, v, w, *args)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_bad_arguments():
    B.build()
    from paper_1803_01262_gb300 import cdi

    a = torch.zeros((4, 4, 8), device="cuda")
    b = torch.zeros((4, 4, 8), device="cuda")
    st = torch.zeros(ctypes.sizeof(cdi.Stats), dtype=torch.uint8, device="cuda")
    with pytest.raises(cdi.CDIError) as e:
        cdi.step_noalloc(a, a, a, a, a, 0.1, 1e-3, 0.1, 1.0, 1.0, st)  # in == out
    assert e.value.code == cdi.CDI_ERR_ARG
    vel = torch.zeros((4, 4, 8), device="cuda")
    with pytest.raises(cdi.CDIError) as e:
        cdi.step_noalloc(a, b, b, vel, vel, 0.1, 1e-3, 0.1, 1.0, 1.0, st)  # out == u
    assert e.value.code == cdi.CDI_ERR_ARG
    with pytest.raises(cdi.CDIError) as e:  # the record inside phi_out
        cdi.step_noalloc(a, b, vel, vel, vel, 0.1, 1e-3, 0.1, 1.0, 1.0, b.view(torch.uint8))
    assert e.value.code == cdi.CDI_ERR_ARG
