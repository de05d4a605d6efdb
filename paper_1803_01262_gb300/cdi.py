"""Thin Python binding of the CDI C ABI (include/cdi.h).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_lib/libcdi.so``.  Device arrays are torch CUDA tensors shaped
``(nz, ny, nx)``, contiguous, of the grid's dtype; streams are torch streams
(default: the current stream).  There is no fallback: if the library is
missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
# CDI_LIBRARY=checked selects the bounds-checked build (build.build(checked=True)).
LIB_PATH = os.path.join(_PKG, "_lib", "libcdi_checked.so" if os.environ.get("CDI_LIBRARY") == "checked"
                        else "libcdi.so")

CDI_OK, CDI_ERR_ARG, CDI_ERR_DIM, CDI_ERR_CUDA = 0, -1, -2, -3
CDI_ERR_CONDITION, CDI_ERR_NAN, CDI_ERR_TIMEOUT, CDI_ERR_STATE = -4, -5, -6, -7
CDI_ERR_BOUNDS = -8
CDI_F32, CDI_F64 = 0, 1
CDI_EULER, CDI_RK2, CDI_RK3, CDI_RK4 = 0, 1, 2, 3
CDI_CHECK_CONDITION = 1
CDI_KERNEL_FORWARD, CDI_KERNEL_ADJOINT = 0, 1
CDI_NCHUNKS_BALANCED = -1   # forward work split: equal contiguous shares per block
CDI_NCHUNKS_ROTATED = -2    # near-equal shares (column starts weighted), columns rotated so
                            # neighbouring tiles share their halo rows in L2
CDI_SHARPEN_CENTRE, CDI_SHARPEN_FACE = 0, 1
SHARPEN = {"centre": CDI_SHARPEN_CENTRE, "face": CDI_SHARPEN_FACE}
FWD_TILES = 7
ADJ_TILES = 4
BATCH_TILES = 7

_ERRNAMES = {-1: "CDI_ERR_ARG", -2: "CDI_ERR_DIM", -3: "CDI_ERR_CUDA", -4: "CDI_ERR_CONDITION",
             -5: "CDI_ERR_NAN", -6: "CDI_ERR_TIMEOUT", -7: "CDI_ERR_STATE", -8: "CDI_ERR_BOUNDS"}


class CDIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("sum", ctypes.c_double), ("min", ctypes.c_double),
                ("max", ctypes.c_double), ("n_strict", ctypes.c_longlong),
                ("n_tol", ctypes.c_longlong), ("min_run", ctypes.c_double),
                ("max_run", ctypes.c_double), ("n_strict_run", ctypes.c_longlong),
                ("n_tol_run", ctypes.c_longlong), ("steps_run", ctypes.c_longlong)]

    def as_dict(self):
        """The record as a dict keyed by its field names."""
        return {k: getattr(self, k) for k, _ in self._fields_}


_V = ctypes.c_void_p
_I = ctypes.c_int
_Dbl = ctypes.c_double
_P = ctypes.POINTER

# name -> argtypes (all return int unless listed in _RESTYPE)
SIGNATURES = {
    "cdi_version": [],
    "cdi_last_error_string": [],
    "cdi_create_grid": [_P(_V), _I, _I, _I, _Dbl, _I],
    "cdi_destroy_grid": [_V],
    "cdi_grid_info": [_V, _P(_I), _P(_I), _P(_I), _P(_Dbl), _P(_I)],
    "cdi_set_velocity": [_V, _V, _V, _V, _Dbl, _V],
    "cdi_get_umax": [_V, _P(_Dbl)],
    "cdi_step": [_V, _V, _V, _Dbl, _Dbl, _Dbl, _Dbl, _I, _V],
    "cdi_run": [_V, _V, _V, _I, _Dbl, _Dbl, _Dbl, _Dbl, _Dbl, _I, _P(_I), _V],
    "cdi_step_planes": [_V, _V, _V, _I, _I, _Dbl, _Dbl, _Dbl, _Dbl, _I, _V],
    "cdi_step_stats": [_V, _P(Stats), _V],
    "cdi_reset_run_stats": [_V, _V],
    "cdi_mass_and_bounds": [_V, _V, _P(Stats), _V],
    "cdi_step_host": [_V, _V, _V, _Dbl, _Dbl, _Dbl, _Dbl, _I, _P(Stats), _V],
    "cdi_step_adjoint": [_V, _V, _V, _V, _V, _V, _V, _Dbl, _Dbl, _Dbl, _Dbl, _V],
    "cdi_check_condition": [_Dbl, _Dbl, _Dbl, _I],
    "cdi_max_dt": [_Dbl, _Dbl, _Dbl, _I, _I, _P(_Dbl)],
    "cdi_max_dt_mixed": [_Dbl, _Dbl, _Dbl, _P(_Dbl), _I, _I, _P(_Dbl)],
    "cdi_set_sharpening": [_V, _I],
    "cdi_probe_bounded_wait": [_V, _Dbl, _V],
    "cdi_is_checked_build": [],
    "cdi_probe_fp64_rate": [_P(_Dbl), _V],
    "cdi_host_slab_plan": [_I, _P(_I), _P(_I), _P(_I)],
    "cdi_probe_bounds_check": [_V, _V],
    "cdi_get_sharpening": [_V, _P(_I)],
    "cdi_set_launch": [_V, _I, _I, _I, _I],
    "cdi_set_run_depth": [_V, _I, _I],
    "cdi_get_run_depth": [_V, _P(_I), _P(_I), _P(_I)],
    "cdi_get_launch": [_V, _I, _P(_I), _P(_I), _P(_I)],
    "cdi_autotune": [_V, _V, _V, _Dbl, _Dbl, _Dbl, _I, _P(_Dbl), _V],
    "cdi_step_noalloc": [_I, _I, _I, _Dbl, _I, _V, _V, _V, _V, _V, _Dbl, _Dbl, _Dbl, _Dbl, _V, _V],
    "cdi_batch_create": [_P(_V), _V, _I, _I],
    "cdi_batch_destroy": [_V],
    "cdi_batch_info": [_V, _P(_I), _P(_I), _P(_I), _P(ctypes.c_longlong)],
    "cdi_batch_step": [_V, _Dbl, _V],
    "cdi_batch_run": [_V, _I, _V],
    "cdi_batch_stats": [_V, _V, _V],
    "cdi_batch_reset_run_stats": [_V, _V],
    "cdi_batch_probe_box_wait": [_V, _Dbl, _V],
    "cdi_batch_set_launch": [_V, _I, _I],
    "cdi_batch_set_sharpening": [_V, _I],
    "cdi_batch_get_sharpening": [_V, _P(_I)],
    "cdi_batch_get_launch": [_V, _P(_I), _P(_I), _P(_I), _P(_I)],
    "cdi_batch_autotune": [_V, _I, _P(ctypes.c_float), _V],
    "cdi_step_rk": [_V, _V, _V, _V, _V, _Dbl, _Dbl, _Dbl, _Dbl, _Dbl, _I, _I, _V],
    "cdi_run_rk": [_V, _V, _V, _V, _V, _I, _Dbl, _Dbl, _Dbl, _Dbl, _Dbl, _I, _I, _P(_I), _V],
}
SCHEMES = {"euler": CDI_EULER, "rk2": CDI_RK2, "rk3": CDI_RK3, "rk4": CDI_RK4}
_RESTYPE = {"cdi_last_error_string": ctypes.c_char_p}

_lib = None
_lock = threading.Lock()


def lib():
    """Load libcdi.so (built by ``paper_1803_01262_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise CDIError(CDI_ERR_STATE, f"CUDA library not built: {LIB_PATH} is missing "
                                              "(run paper_1803_01262_gb300.build.build())")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = _RESTYPE.get(name, ctypes.c_int)
            _lib = L
    return _lib


def _err():
    return lib().cdi_last_error_string().decode(errors="replace")


def _ck(rc):
    if rc < 0:
        raise CDIError(rc, _err())
    return rc


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(dtype):
    if dtype == torch.float32:
        return CDI_F32
    if dtype == torch.float64:
        return CDI_F64
    raise ValueError("dtype must be torch.float32 or torch.float64")


def host_slab_plan(nz):
    """The slab plan of the host-buffer step (cdi_host_slab_plan): (bounds[9], copy_lo[8],
    copy_hi[8]) as lists."""
    b, lo, hi = (ctypes.c_int * 9)(), (ctypes.c_int * 8)(), (ctypes.c_int * 8)()
    _ck(lib().cdi_host_slab_plan(int(nz), b, lo, hi))
    return list(b), list(lo), list(hi)


def probe_fp64_rate(stream=None):
    """Measured FP64 FMA instructions per second of the current device."""
    out = ctypes.c_double()
    _ck(lib().cdi_probe_fp64_rate(ctypes.byref(out), _stream(stream)))
    return out.value


def is_checked_build():
    """True if the loaded library is the bounds-checked build."""
    return bool(lib().cdi_is_checked_build())


def check_condition(eps_over_dx, gamma_over_U, A, Df):
    """Eq. 17/24 and A <= 1/(2 D_f): True if both hold."""
    return bool(_ck(lib().cdi_check_condition(eps_over_dx, gamma_over_U, A, Df)))


def max_dt(dx, eps, gamma, Df, scheme=CDI_EULER):
    """Largest bounded step of Eq. 25-28 for the given scheme."""
    out = ctypes.c_double()
    _ck(lib().cdi_max_dt(dx, eps, gamma, Df, scheme, ctypes.byref(out)))
    return out.value


def max_dt_mixed(dx, eps, gamma, umax, scheme=CDI_EULER):
    """min(diffusive limit of the scheme, mixed advective-diffusive limit): Eq. 31/32 for
    RK4, the Eq. 10 analogue for Euler; ``umax`` lists the largest |velocity component| of
    each non-degenerate axis."""
    um = (ctypes.c_double * len(umax))(*[float(x) for x in umax])
    out = ctypes.c_double()
    _ck(lib().cdi_max_dt_mixed(dx, eps, gamma, um, len(umax), scheme, ctypes.byref(out)))
    return out.value


def step_noalloc(phi_in, phi_out, u, v, w, dx, dt, eps, gamma, vel_scale, stats_dev, stream=None):
    """One forward step through cdi_step_noalloc (no device allocation by the library).

    For callers that cannot allocate device memory at step time.  All
    arguments are preallocated CUDA tensors; ``stats_dev`` is a device tensor
    of at least ``ctypes.sizeof(Stats)`` bytes that receives the statistics.
    Returns nothing; read ``stats_dev`` with :func:`stats_from_device`.
    """
    nz, ny, nx = phi_in.shape
    code = _dtype_code(phi_in.dtype)
    for t in (phi_in, phi_out, u, v, w):
        if t is not None and (not t.is_cuda or not t.is_contiguous() or t.dtype != phi_in.dtype
                              or tuple(t.shape) != (nz, ny, nx)):
            raise ValueError("arrays must be contiguous CUDA tensors of one dtype and shape")
    if stats_dev.numel() * stats_dev.element_size() < ctypes.sizeof(Stats):
        raise ValueError("stats_dev is too small")
    p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    _ck(lib().cdi_step_noalloc(nx, ny, nz, float(dx), code, p(phi_in), p(phi_out), p(u), p(v), p(w),
                               dt, eps, gamma, vel_scale, p(stats_dev), _stream(stream)))


def stats_from_device(stats_dev):
    """Decode a cdi_stats record held in a device tensor (synchronises)."""
    raw = bytes(stats_dev.view(torch.uint8)[:ctypes.sizeof(Stats)].cpu().numpy())
    return Stats.from_buffer_copy(raw).as_dict()


class Grid:
    """A periodic nx x ny x nz grid of spacing dx on the current CUDA device."""

    def __init__(self, nx, ny, nz, dx, dtype=torch.float32):
        self.shape = (nz, ny, nx)
        self.dx = float(dx)
        self.dtype = dtype
        self._h = ctypes.c_void_p()
        _ck(lib().cdi_create_grid(ctypes.byref(self._h), nx, ny, nz, self.dx, _dtype_code(dtype)))
        self._vel = None

    @property
    def Df(self):
        """Number of axes with extent > 1 (D_f of Eq. 19 and Eq. 25)."""
        return sum(1 for s in self.shape if s > 1)

    def close(self):
        """Free the grid and its device scratch (cdi_destroy_grid); idempotent."""
        if self._h:
            lib().cdi_destroy_grid(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arr(self, t, name):
        if t is None:
            return None
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype or tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous {self.dtype} of shape {self.shape}")
        return ctypes.c_void_p(t.data_ptr())

    def set_velocity(self, u, v, w=None, umax=None, stream=None):
        """Borrow face velocities; U computed on the device unless umax is given."""
        _ck(lib().cdi_set_velocity(self._h, self._arr(u, "u"), self._arr(v, "v"),
                                   self._arr(w, "w"), -1.0 if umax is None else float(umax),
                                   _stream(stream)))
        self._vel = (u, v, w)  # keep the borrowed storage alive

    @property
    def U(self):
        """U of the velocity set: the largest face |component| (Eq. 24 reading)."""
        out = ctypes.c_double()
        _ck(lib().cdi_get_umax(self._h, ctypes.byref(out)))
        return out.value

    def step(self, phi_in, phi_out, dt, eps, gamma, vel_scale=1.0, check=False, stream=None):
        """phi_out = one Euler CDI step of phi_in (fused statistics in the record)."""
        _ck(lib().cdi_step(self._h, self._arr(phi_in, "phi_in"), self._arr(phi_out, "phi_out"),
                           dt, eps, gamma, vel_scale, CDI_CHECK_CONDITION if check else 0,
                           _stream(stream)))
        return phi_out

    def step_planes(self, phi_in, phi_out, z_lo, z_hi, dt, eps, gamma, vel_scale=1.0, check=False,
                    stream=None):
        """The Euler step on planes [z_lo, z_hi) of phi_out only (cdi_step_planes); the
        statistics record covers those planes."""
        _ck(lib().cdi_step_planes(self._h, self._arr(phi_in, "phi_in"), self._arr(phi_out, "phi_out"),
                                  int(z_lo), int(z_hi), dt, eps, gamma, vel_scale,
                                  CDI_CHECK_CONDITION if check else 0, _stream(stream)))
        return phi_out

    def run(self, a, b, nsteps, dt, eps, gamma, period=0.0, t0=0.0, check=False, stream=None):
        """nsteps steps ping-ponging a <-> b (native loop); returns the result tensor."""
        fb = ctypes.c_int()
        _ck(lib().cdi_run(self._h, self._arr(a, "a"), self._arr(b, "b"), nsteps, t0, dt, eps,
                          gamma, period, CDI_CHECK_CONDITION if check else 0, ctypes.byref(fb),
                          _stream(stream)))
        return b if fb.value else a

    def step_rk(self, phi_in, phi_out, work1, work2, dt, eps, gamma, scheme="rk4", t=0.0,
                period=0.0, check=False, stream=None):
        """One Runge-Kutta step (Section 2.3); work1/work2 are scratch tensors of the grid's shape."""
        _ck(lib().cdi_step_rk(self._h, self._arr(phi_in, "phi_in"), self._arr(phi_out, "phi_out"),
                              self._arr(work1, "work1"), self._arr(work2, "work2"), dt, eps, gamma,
                              t, period, SCHEMES[scheme], CDI_CHECK_CONDITION if check else 0,
                              _stream(stream)))
        return phi_out

    def run_rk(self, a, b, work1, work2, nsteps, dt, eps, gamma, scheme="rk4", period=0.0, t0=0.0,
               check=False, stream=None):
        """nsteps RK steps ping-ponging a <-> b; returns the tensor holding the result."""
        fb = ctypes.c_int()
        _ck(lib().cdi_run_rk(self._h, self._arr(a, "a"), self._arr(b, "b"), self._arr(work1, "work1"),
                             self._arr(work2, "work2"), nsteps, t0, dt, eps, gamma, period,
                             SCHEMES[scheme], CDI_CHECK_CONDITION if check else 0, ctypes.byref(fb),
                             _stream(stream)))
        return b if fb.value else a

    def stats(self, stream=None):
        """Statistics of the last fused step (synchronises)."""
        s = Stats()
        _ck(lib().cdi_step_stats(self._h, ctypes.byref(s), _stream(stream)))
        return s.as_dict()

    def reset_run_stats(self, stream=None):
        """Zero the run accumulators (*_run, steps_run) of the statistics record."""
        _ck(lib().cdi_reset_run_stats(self._h, _stream(stream)))

    def mass_and_bounds(self, phi, stream=None):
        """Mass, sum, min, max and violation counts of any field phi (synchronises)."""
        s = Stats()
        _ck(lib().cdi_mass_and_bounds(self._h, self._arr(phi, "phi"), ctypes.byref(s),
                                      _stream(stream)))
        return s.as_dict()

    def step_host(self, phi_in, phi_out, dt, eps, gamma, vel_scale=1.0, check=False,
                  stream=None):
        """Host-buffer step (numpy arrays, ideally pinned); returns the statistics."""
        for a in (phi_in, phi_out):
            if not isinstance(a, np.ndarray) or a.shape != self.shape or not a.flags.c_contiguous:
                raise ValueError("host arrays must be C-contiguous numpy arrays of the grid shape")
        s = Stats()
        _ck(lib().cdi_step_host(self._h, ctypes.c_void_p(phi_in.ctypes.data),
                                ctypes.c_void_p(phi_out.ctypes.data), dt, eps, gamma, vel_scale,
                                CDI_CHECK_CONDITION if check else 0, ctypes.byref(s),
                                _stream(stream)))
        return s.as_dict()

    def probe_bounded_wait(self, limit_s=0.05, stream=None):
        """Make a bounded device wait run out (see cdi_probe_bounded_wait); raises CDIError
        with CDI_ERR_TIMEOUT when the time-out is reported, as it should be."""
        _ck(lib().cdi_probe_bounded_wait(self._h, limit_s, _stream(stream)))

    def probe_bounds_check(self, stream=None):
        """Checked builds: make the index check record one bad index (cdi_probe_bounds_check);
        raises CDIError with CDI_ERR_BOUNDS when it is reported, as it should be."""
        _ck(lib().cdi_probe_bounds_check(self._h, _stream(stream)))

    def set_sharpening(self, mode):
        """"centre" (Section 2.2, the default) or "face" (face-product sharpening, forward
        tile 0 with Euler steps only)."""
        _ck(lib().cdi_set_sharpening(self._h, SHARPEN[mode]))

    def get_sharpening(self):
        """The sharpening form of the forward step: "centre" (default) or "face"."""
        m = ctypes.c_int()
        _ck(lib().cdi_get_sharpening(self._h, ctypes.byref(m)))
        return {v: k for k, v in SHARPEN.items()}[m.value]

    def set_launch(self, which=CDI_KERNEL_FORWARD, tile=-1, blocks_per_sm=0, nchunks=0):
        """Force a launch configuration (tile < 0: the default)."""
        _ck(lib().cdi_set_launch(self._h, which, tile, blocks_per_sm, nchunks))

    def get_launch(self, which=CDI_KERNEL_FORWARD):
        """The launch configuration in use: tile, blocks per launch, z chunks (-1: balanced)."""
        t, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _ck(lib().cdi_get_launch(self._h, which, ctypes.byref(t), ctypes.byref(b), ctypes.byref(c)))
        return dict(tile=t.value, nblocks=b.value, nchunks=c.value)

    def set_run_depth(self, depth, nchunks=0):
        """Steps per pass of run(): 1, or 2 (two Euler steps per launch, temporal blocking)."""
        _ck(lib().cdi_set_run_depth(self._h, int(depth), int(nchunks)))

    def get_run_depth(self):
        """The run depth and the two-steps-per-pass launch: depth, blocks, z chunks."""
        d, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _ck(lib().cdi_get_run_depth(self._h, ctypes.byref(d), ctypes.byref(b), ctypes.byref(c)))
        return dict(depth=d.value, nblocks=b.value, nchunks=c.value)

    def autotune(self, a, b, dt, eps, gamma, reps=5, stream=None):
        """Time all forward configurations on scratch buffers a, b; keep the fastest."""
        ms = ctypes.c_double()
        _ck(lib().cdi_autotune(self._h, self._arr(a, "a"), self._arr(b, "b"), dt, eps, gamma, reps,
                               ctypes.byref(ms), _stream(stream)))
        return ms.value

    def step_adjoint(self, phi_k, lam_next, lam_k, dt, eps, gamma, vel_scale=1.0, grads=None,
                     stream=None):
        """lam_k = J^T lam_next; if grads=(gu, gv, gw) the velocity gradient is added to them."""
        g = grads if grads is not None else (None, None, None)
        _ck(lib().cdi_step_adjoint(self._h, self._arr(phi_k, "phi_k"),
                                   self._arr(lam_next, "lam_next"), self._arr(lam_k, "lam_k"),
                                   self._arr(g[0], "gu"), self._arr(g[1], "gv"),
                                   self._arr(g[2], "gw"), dt, eps, gamma, vel_scale,
                                   _stream(stream)))
        return lam_k


class BoxDesc(ctypes.Structure):
    """Mirror of cdi_box_desc."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("eps", ctypes.c_double),
                ("gamma", ctypes.c_double), ("u", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("phi_a", ctypes.c_void_p), ("phi_b", ctypes.c_void_p)]


class Batch:
    """Independent periodic boxes advanced by one launch per step (cdi_batch_*).

    ``boxes`` is a list of dicts with keys dx, dt, eps, gamma, u, v, w, phi_a,
    phi_b (CUDA tensors shaped (nz, ny, nx), one dtype for all boxes).  The
    state starts in phi_a; :meth:`current` returns the tensor holding it.
    """

    def __init__(self, boxes):
        if not boxes:
            raise ValueError("empty batch")
        self.dtype = boxes[0]["phi_a"].dtype
        descs = (BoxDesc * len(boxes))()
        keep = []
        for i, b in enumerate(boxes):
            nz, ny, nx = b["phi_a"].shape
            for k in ("u", "v", "w", "phi_a", "phi_b"):
                t = b[k]
                if (not t.is_cuda or t.dtype != self.dtype or not t.is_contiguous()
                        or tuple(t.shape) != (nz, ny, nx)):
                    raise ValueError(f"box {i}: {k} must be a contiguous CUDA tensor of the box shape")
                keep.append(t)
            descs[i] = BoxDesc(nx, ny, nz, float(b["dx"]), float(b["dt"]), float(b["eps"]),
                               float(b["gamma"]), b["u"].data_ptr(), b["v"].data_ptr(),
                               b["w"].data_ptr(), b["phi_a"].data_ptr(), b["phi_b"].data_ptr())
        self._keep = keep
        self.boxes = boxes
        self._h = ctypes.c_void_p()
        _ck(lib().cdi_batch_create(ctypes.byref(self._h), ctypes.cast(descs, ctypes.c_void_p),
                                   len(boxes), _dtype_code(self.dtype)))

    def close(self):
        """Free the batch's device tables and captured graphs; idempotent."""
        if self._h:
            lib().cdi_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        """Parity (which buffer holds the state), work units, blocks per launch, cells."""
        p, u, n, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        _ck(lib().cdi_batch_info(self._h, ctypes.byref(p), ctypes.byref(u), ctypes.byref(n),
                                 ctypes.byref(c)))
        return dict(parity=p.value, units=u.value, nblocks=n.value, cells=c.value)

    def current(self, i):
        """The tensor holding box i's current state."""
        return self.boxes[i]["phi_b" if self.info()["parity"] else "phi_a"]

    def step(self, vel_scale=1.0, stream=None):
        """One Euler step of every box with face velocity vel_scale * (u, v, w)."""
        _ck(lib().cdi_batch_step(self._h, vel_scale, _stream(stream)))

    def run(self, nsteps, stream=None):
        """nsteps steps as one replay of a captured CUDA graph."""
        _ck(lib().cdi_batch_run(self._h, nsteps, _stream(stream)))

    def set_launch(self, tile=-1, zdepth=-1):
        """Work-unit tile (0..3: 32x8, 32x16, 64x8, 32x4; 4: one unit per whole 2D box, for
        batches of 2D boxes whose planes fit in shared memory; 5: bands of whole rows, for
        batches with 3D boxes of nx <= 1024; 6: bands of whole rows of the batch's padded
        copies, 16-byte vectors of cells per thread) and planes per unit (0: whole box)."""
        _ck(lib().cdi_batch_set_launch(self._h, tile, zdepth))

    def set_sharpening(self, mode):
        """"centre" (Section 2.2, the default) or "face" (face-product sharpening; batch tiles 0
        and 4 only)."""
        _ck(lib().cdi_batch_set_sharpening(self._h, SHARPEN[mode]))

    def get_sharpening(self):
        """The sharpening form of the batch: "centre" or "face"."""
        m = ctypes.c_int()
        _ck(lib().cdi_batch_get_sharpening(self._h, ctypes.byref(m)))
        return {v: k for k, v in SHARPEN.items()}[m.value]

    def get_launch(self):
        """The batch launch configuration: tile, z depth, blocks per launch, work units."""
        t, z, n, u = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _ck(lib().cdi_batch_get_launch(self._h, ctypes.byref(t), ctypes.byref(z), ctypes.byref(n),
                                       ctypes.byref(u)))
        return dict(tile=t.value, zdepth=z.value, nblocks=n.value, units=u.value)

    def autotune(self, reps=3, stream=None):
        """Time every tile x z depth and keep the fastest; returns its ms per launch."""
        ms = ctypes.c_float()
        _ck(lib().cdi_batch_autotune(self._h, reps, ctypes.byref(ms), _stream(stream)))
        return ms.value

    def stats(self, stream=None):
        """Per-box statistics records, last step and run accumulators (synchronises)."""
        out = (Stats * len(self.boxes))()
        _ck(lib().cdi_batch_stats(self._h, ctypes.cast(out, ctypes.c_void_p), _stream(stream)))
        return [s.as_dict() for s in out]

    def reset_run_stats(self, stream=None):
        """Zero every box's run accumulators."""
        _ck(lib().cdi_batch_reset_run_stats(self._h, _stream(stream)))

    def probe_box_wait(self, limit_s=0.05, stream=None):
        """Make the run's per-box wait run out (see cdi_batch_probe_box_wait); raises CDIError
        with code CDI_ERR_TIMEOUT, the expected result.  No box is stepped."""
        _ck(lib().cdi_batch_probe_box_wait(self._h, limit_s, _stream(stream)))
