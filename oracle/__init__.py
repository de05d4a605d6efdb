"""FP64 CPU oracle for the CDI phase-field step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and nothing here imports the product.

The arithmetic lives in ``cdi_oracle.c`` (plain C, nested loops, float64),
compiled with gcc into ``oracle/_lib/libcdi_oracle.so`` by :func:`build`.
Functions take numpy arrays shaped ``(nz, ny, nx)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdi_oracle.c")
_OUT = os.path.join(_HERE, "_lib", "libcdi_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, -O2) if needed."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d = ctypes.c_int, ctypes.c_double
            lib.oracle_rhs.argtypes = [i, i, i, d, _D, _D, _D, _D, d, d, d, d, _D]
            lib.oracle_step.argtypes = [i, i, i, d, _D, _D, _D, _D, d, d, d, d, d, _D]
            lib.oracle_rhs_face.argtypes = lib.oracle_rhs.argtypes
            lib.oracle_step_face.argtypes = lib.oracle_step.argtypes
            lib.oracle_stats.argtypes = [ctypes.c_long, _D, d, d, _D,
                                         ctypes.POINTER(ctypes.c_longlong)]
            lib.oracle_adjoint.argtypes = [i, i, i, d, _D, _D, _D, _D, _D, d, d, d, d, d,
                                           _D, _D, _D, _D]
            for f in (lib.oracle_rhs, lib.oracle_step, lib.oracle_stats, lib.oracle_adjoint,
                      lib.oracle_rhs_face, lib.oracle_step_face):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(phi, u, v, w):
    phi, u, v, w = (_f64(x) for x in (phi, u, v, w))
    if phi.ndim != 3 or any(x.shape != phi.shape for x in (u, v, w)):
        raise ValueError("phi, u, v, w must share one (nz, ny, nx) shape")
    return phi, u, v, w


def floor_of(dtype) -> float:
    """The floor under |g|^2 of a step computed in ``dtype``: its smallest
    normal number (FLT_MIN, DBL_MIN).  0 gives the paper's unit normal."""
    return float(np.finfo(dtype).tiny)


def adjoint_floor_of(dtype) -> float:
    """The floor under |g|^2 that the backward pass of a ``dtype`` step takes:
    (8 machine epsilons)^2, i.e. delta = 16 units in the last place of values
    just below 1.  The forward step divides by |g| (its floor, ``floor_of``,
    is invisible); the adjoint differentiates n = g / sqrt(|g|^2 + delta^2),
    which is the same wherever |g| >> delta and caps the normal's derivative
    phi (1 - phi)/|g| where g is at the rounding level of phi.  (The paper
    has no adjoint; this is the reading taken for it.)"""
    return float((8.0 * np.finfo(dtype).eps) ** 2)


SHARPEN = ("centre", "face")


def rhs(phi, u, v, w, dx, eps, gamma, vel_scale=1.0, tiny=0.0, sharpen="centre"):
    """d phi/dt of Eq. 1 discretised by the five steps of Section 2.2; the
    normal is g / sqrt(|g|^2 + tiny) (0 where g = 0).  ``sharpen="face"``
    takes the non-default face-product sharpening phi_f (1 - phi_f) n_f."""
    phi, u, v, w = _check(phi, u, v, w)
    nz, ny, nx = phi.shape
    out = np.empty_like(phi)
    f = {"centre": _load().oracle_rhs, "face": _load().oracle_rhs_face}[sharpen]
    rc = f(nx, ny, nz, dx, _p(phi), _p(u), _p(v), _p(w), eps, gamma, vel_scale, tiny, _p(out))
    if rc:
        raise ValueError("oracle_rhs: bad arguments")
    return out


def step(phi, u, v, w, dx, dt, eps, gamma, vel_scale=1.0, tiny=0.0, sharpen="centre"):
    """One explicit Euler step of the CDI equation (Eq. 11 generalised to 3D);
    ``sharpen`` as in :func:`rhs`."""
    phi, u, v, w = _check(phi, u, v, w)
    nz, ny, nx = phi.shape
    out = np.empty_like(phi)
    f = {"centre": _load().oracle_step, "face": _load().oracle_step_face}[sharpen]
    rc = f(nx, ny, nz, dx, _p(phi), _p(u), _p(v), _p(w), dt, eps, gamma, vel_scale, tiny, _p(out))
    if rc:
        raise ValueError("oracle_step: bad arguments")
    return out


def run(phi, u, v, w, dx, dt, eps, gamma, nsteps, period=0.0, t0=0.0, tiny=0.0, sharpen="centre"):
    """nsteps Euler steps; velocity scaled by cos(pi t / period) when period > 0."""
    p = _f64(phi)
    t = t0
    for _ in range(nsteps):
        s = np.cos(np.pi * t / period) if period > 0 else 1.0
        p = step(p, u, v, w, dx, dt, eps, gamma, s, tiny, sharpen)
        t += dt
    return p


# Explicit Runge-Kutta schemes of Section 2.3 (Eq. 26-28), written from their
# published definitions; each takes a right-hand side f(phi, t).
RK_SCHEMES = ("euler", "rk2", "rk3", "rk4")


def rk_advance(f, phi, t, dt, scheme):
    """One step of: explicit Euler; the explicit midpoint rule (RK2); Wray's
    low-storage third-order scheme (RK3: gamma = 8/15, 5/12, 3/4, zeta = 0,
    -17/60, -5/12, stage times t, t + 8/15 dt, t + 2/3 dt); classic RK4."""
    if scheme == "euler":
        return phi + dt * f(phi, t)
    if scheme == "rk2":
        half = phi + 0.5 * dt * f(phi, t)
        return phi + dt * f(half, t + 0.5 * dt)
    if scheme == "rk3":
        g = (8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0)
        z = (0.0, -17.0 / 60.0, -5.0 / 12.0)
        c = (0.0, 8.0 / 15.0, 2.0 / 3.0)
        p, prev = phi, None
        for s in range(3):
            r = f(p, t + c[s] * dt)
            p = p + dt * (g[s] * r + (z[s] * prev if prev is not None else 0.0))
            prev = r
        return p
    if scheme == "rk4":
        k1 = f(phi, t)
        k2 = f(phi + 0.5 * dt * k1, t + 0.5 * dt)
        k3 = f(phi + 0.5 * dt * k2, t + 0.5 * dt)
        k4 = f(phi + dt * k3, t + dt)
        return phi + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    raise ValueError(scheme)


def rk_step(phi, u, v, w, dx, dt, eps, gamma, scheme, t=0.0, period=0.0, tiny=0.0):
    """One RK step of the CDI equation; velocity scaled by cos(pi t/period) at each stage time."""
    phi, u, v, w = _check(phi, u, v, w)

    def f(p, tt):
        s = np.cos(np.pi * tt / period) if period > 0 else 1.0
        return rhs(p, u, v, w, dx, eps, gamma, s, tiny)
    return rk_advance(f, phi, t, dt, scheme)


def rk_run(phi, u, v, w, dx, dt, eps, gamma, nsteps, scheme, period=0.0, t0=0.0, tiny=0.0):
    p = _f64(phi)
    for i in range(nsteps):
        p = rk_step(p, u, v, w, dx, dt, eps, gamma, scheme, t0 + i * dt, period, tiny)
    return p


def stats(phi, dV, tol):
    """{mass, sum, min, max, n_strict, n_tol} of a field (plain sequential sum)."""
    phi = _f64(phi).ravel()
    o = np.empty(4)
    c = np.empty(2, dtype=np.int64)
    _load().oracle_stats(phi.size, _p(phi), dV, tol, _p(o),
                         c.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return dict(mass=o[0], sum=o[1], min=o[2], max=o[3], n_strict=int(c[0]), n_tol=int(c[1]))


def adjoint(phi, u, v, w, lam_next, dx, dt, eps, gamma, vel_scale=1.0, want_vel=False,
            tiny=0.0):
    """Discrete adjoint of one Euler step (of :func:`step` with the same
    ``tiny``): returns lam (and velocity gradients)."""
    phi, u, v, w = _check(phi, u, v, w)
    lam_next = _f64(lam_next)
    nz, ny, nx = phi.shape
    lam = np.empty_like(phi)
    g = [np.zeros_like(phi) for _ in range(3)] if want_vel else [None] * 3
    rc = _load().oracle_adjoint(nx, ny, nz, dx, _p(phi), _p(u), _p(v), _p(w), _p(lam_next),
                                dt, eps, gamma, vel_scale, tiny, _p(lam), _p(g[0]), _p(g[1]),
                                _p(g[2]))
    if rc:
        raise ValueError("oracle_adjoint: bad arguments")
    return (lam, *g) if want_vel else lam
