"""Argument checks of the C ABI that return before any CUDA call, exercised on the host:
each bad argument gets its documented error code and a message, and nothing is touched."""
import ctypes

import pytest
import torch

from paper_1803_01262_gb300 import build as B
from paper_1803_01262_gb300 import cdi


@pytest.fixture(scope="module")
def L():
    B.build()
    return cdi.lib()


def msg(L):
    return L.cdi_last_error_string().decode()


def test_create_grid_arguments(L):
    g = ctypes.c_void_p()
    assert L.cdi_create_grid(None, 4, 4, 4, 0.1, cdi.CDI_F32) == cdi.CDI_ERR_ARG
    for ext in ((0, 4, 4), (4, -1, 4), (4, 4, 0)):
        assert L.cdi_create_grid(ctypes.byref(g), *ext, 0.1, cdi.CDI_F32) == cdi.CDI_ERR_DIM
        assert "extents" in msg(L) and not g.value
    assert L.cdi_create_grid(ctypes.byref(g), 1 << 16, 1 << 15, 1, 0.1, cdi.CDI_F32) == cdi.CDI_ERR_DIM
    assert L.cdi_create_grid(ctypes.byref(g), 1 << 12, 1 << 12, 1 << 12, 0.1, cdi.CDI_F32) == cdi.CDI_ERR_DIM
    for dx in (0.0, -1.0, float("nan"), float("inf")):
        assert L.cdi_create_grid(ctypes.byref(g), 4, 4, 4, dx, cdi.CDI_F32) == cdi.CDI_ERR_ARG
    assert L.cdi_create_grid(ctypes.byref(g), 4, 4, 4, 0.1, 7) == cdi.CDI_ERR_ARG
    assert "dtype" in msg(L)


def test_valid_grid_needs_a_device(L):
    """Valid arguments reach the CUDA runtime: without a GPU the call fails with CDI_ERR_CUDA
    (no CPU fallback), with one it creates and frees a grid."""
    g = ctypes.c_void_p()
    rc = L.cdi_create_grid(ctypes.byref(g), 8, 8, 8, 0.1, cdi.CDI_F32)
    if torch.cuda.is_available():
        assert rc == cdi.CDI_OK and g.value
        assert L.cdi_destroy_grid(g) == cdi.CDI_OK
    else:
        assert rc == cdi.CDI_ERR_CUDA and not g.value and msg(L)


def test_null_grid_everywhere(L):
    assert L.cdi_destroy_grid(None) == cdi.CDI_OK
    nx = ctypes.c_int()
    assert L.cdi_grid_info(None, ctypes.byref(nx), None, None, None, None) == cdi.CDI_ERR_ARG
    assert L.cdi_set_velocity(None, None, None, None, -1.0, None) == cdi.CDI_ERR_ARG
    assert L.cdi_step(None, None, None, 1e-3, 0.1, 1.0, 1.0, 0, None) == cdi.CDI_ERR_ARG
    assert L.cdi_mass_and_bounds(None, None, None, None) == cdi.CDI_ERR_ARG
    assert "NULL" in msg(L)


def test_batch_create_arguments(L):
    b = ctypes.c_void_p()
    assert L.cdi_batch_create(None, None, 1, cdi.CDI_F32) == cdi.CDI_ERR_ARG
    assert L.cdi_batch_create(ctypes.byref(b), None, 0, cdi.CDI_F32) == cdi.CDI_ERR_ARG
    assert not b.value


def test_null_batch_everywhere(L):
    """A NULL batch is refused before any CUDA call, the run and its wait probe included."""
    assert L.cdi_batch_step(None, 1.0, None) == cdi.CDI_ERR_ARG
    assert L.cdi_batch_run(None, 4, None) == cdi.CDI_ERR_ARG
    assert L.cdi_batch_probe_box_wait(None, 0.05, None) == cdi.CDI_ERR_ARG
    assert L.cdi_batch_reset_run_stats(None, None) == cdi.CDI_ERR_ARG
    assert "NULL" in msg(L)


def test_step_noalloc_arguments(L):
    """Every rejection below happens before the first CUDA call, so the fake (never
    dereferenced) addresses are safe on any machine."""
    A, B2, U = 0x10000, 0x20000, 0x30000   # 16-byte aligned, disjoint for 8x8x8 FP32
    S = 0x40000

    def call(nx=8, ny=8, nz=8, dx=0.1, dtype=cdi.CDI_F32, pi=A, po=B2, u=U, v=U, w=U, dt=1e-3,
             eps=0.1, gamma=1.0, vs=1.0, st=S):
        return L.cdi_step_noalloc(nx, ny, nz, dx, dtype, pi, po, u, v, w, dt, eps, gamma, vs, st, None)

    assert call(nx=0) == cdi.CDI_ERR_DIM
    assert call(nx=1 << 16, ny=1 << 15) == cdi.CDI_ERR_DIM
    for bad in (dict(dx=0.0), dict(eps=-1.0), dict(gamma=-1.0), dict(dt=-1.0), dict(vs=float("nan"))):
        assert call(**bad) == cdi.CDI_ERR_ARG, bad
    assert call(dtype=5) == cdi.CDI_ERR_ARG
    for bad in (dict(pi=None), dict(po=None), dict(u=None), dict(st=None), dict(v=None), dict(w=None)):
        assert call(**bad) == cdi.CDI_ERR_ARG, bad
    assert call(pi=A + 4) == cdi.CDI_ERR_ARG and "aligned" in msg(L)
    assert call(st=S + 4) == cdi.CDI_ERR_ARG
    assert call(po=A + 16) == cdi.CDI_ERR_ARG and "overlap" in msg(L)
