"""Seeded synthetic inputs for the CDI phase-field step.

This module is shared by the CUDA path, its tests, the bench and the FP64
oracle.  It holds none of the method's arithmetic (no normals, fluxes or
updates): only initial phase fields, face velocities and their parameters.
Everything is generated on the host in float64 with numpy; callers cast to
float32 where the FP32 path is exercised.  For boxes too large for host
generation (512^3 and up) the ``*_torch`` variants evaluate the same
definitions on a CUDA device in float64 (mode table from the same seeded
PCG64 stream), chunked along z.

Grid conventions (Section 2.2 of the paper: phi at cell centres, velocity
components on faces, uniform isotropic spacing h):

* arrays are indexed ``[k, j, i]`` (z, y, x) with ``i`` fastest;
* cell ``(i, j, k)`` has its centre at ``((i+1/2)h, (j+1/2)h, (k+1/2)h)``;
* ``u[k, j, i]`` is the x-velocity on the right face ``i+1/2`` of that cell,
  ``v`` on face ``j+1/2``, ``w`` on face ``k+1/2`` (periodic);
* box edge lengths are ``L_d = N_d h``.

Divergence-free velocities are built as the discrete staggered curl of an
edge-centred vector potential, so the discrete divergence
``(u_{i+1/2}-u_{i-1/2} + v_{j+1/2}-v_{j-1/2} + w_{k+1/2}-w_{k-1/2})/h``
vanishes up to round-off for any potential.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Fields", "centres", "tanh_profile", "periodic_delta", "sphere_distance",
    "ellipsoid_distance", "staggered_curl", "single_vortex_2d",
    "deformation_3d", "fourier_potential", "random_velocity", "face_umax",
    "drop_2d_uniform", "random_boxes", "random_phi",
    "spheres_phi_torch", "random_velocity_torch",
]


@dataclass
class Fields:
    """One periodic box: phase field, face velocities and spacing."""
    phi: np.ndarray          # (nz, ny, nx) float64
    u: np.ndarray            # (nz, ny, nx) float64, x-faces i+1/2
    v: np.ndarray            # y-faces j+1/2
    w: np.ndarray            # z-faces k+1/2
    h: float                 # grid spacing (isotropic)
    U: float                 # max over faces of |velocity component|

    @property
    def shape(self):
        return self.phi.shape


def centres(n: int, h: float, offset: float = 0.5) -> np.ndarray:
    """Coordinates ``(i + offset) h`` for ``i = 0..n-1``."""
    return (np.arange(n, dtype=np.float64) + offset) * h


def tanh_profile(s: np.ndarray, eps: float) -> np.ndarray:
    """Olsson-Kreiss profile 0.5(1 + tanh(s / 2 eps)), s > 0 inside (Section 1)."""
    return 0.5 * (1.0 + np.tanh(s / (2.0 * eps)))


def periodic_delta(x: np.ndarray, c: float, L: float) -> np.ndarray:
    """Minimum-image displacement x - c in a periodic interval of length L."""
    d = x - c
    return d - L * np.round(d / L)


def sphere_distance(shape, h, centre, radius):
    """Signed distance R - |x - c| (periodic minimum image), positive inside.

    ``shape`` is (nz, ny, nx); ``centre`` is given as (x, y, z).  Axes of
    extent 1 are ignored (a 2D/1D problem embedded in the 3D layout).
    """
    nz, ny, nx = shape
    r2 = np.zeros(shape, dtype=np.float64)
    for n, c, ax in ((nx, centre[0], 2), (ny, centre[1], 1), (nz, centre[2], 0)):
        if n == 1:
            continue
        d = periodic_delta(centres(n, h), c, n * h)
        sh = [1, 1, 1]
        sh[ax] = n
        r2 = r2 + (d * d).reshape(sh)
    return radius - np.sqrt(r2)


def ellipsoid_distance(shape, h, centre, semi_axes):
    """Approximate signed distance of an axis-aligned ellipsoid, positive inside.

    Uses s = (1 - rho) * min(a) with rho = |(x - c) / a| (periodic minimum
    image), which equals the exact distance for a sphere.
    """
    nz, ny, nx = shape
    rho2 = np.zeros(shape, dtype=np.float64)
    for n, c, a, ax in ((nx, centre[0], semi_axes[0], 2),
                        (ny, centre[1], semi_axes[1], 1),
                        (nz, centre[2], semi_axes[2], 0)):
        if n == 1:
            continue
        d = periodic_delta(centres(n, h), c, n * h) / a
        sh = [1, 1, 1]
        sh[ax] = n
        rho2 = rho2 + (d * d).reshape(sh)
    return (1.0 - np.sqrt(rho2)) * min(semi_axes)


def staggered_curl(Ax, Ay, Az, h):
    """Discrete curl of an edge-centred vector potential on the staggered grid.

    ``Ax[k,j,i]`` lives on the x-edge (i, j+1/2, k+1/2), ``Ay[k,j,i]`` on the
    y-edge (i+1/2, j, k+1/2), ``Az[k,j,i]`` on the z-edge (i+1/2, j+1/2, k).
    Returns face velocities (u, v, w) whose discrete divergence is zero up to
    round-off.  ``None`` components are treated as zero.
    """
    shape = next(a.shape for a in (Ax, Ay, Az) if a is not None)
    z = np.zeros(shape, dtype=np.float64)
    Ax = z if Ax is None else Ax
    Ay = z if Ay is None else Ay
    Az = z if Az is None else Az

    def dm(a, axis):  # backward difference a[..] - a[..-1] along axis (periodic)
        return a - np.roll(a, 1, axis=axis)

    u = (dm(Az, 1) - dm(Ay, 0)) / h
    v = (dm(Ax, 0) - dm(Az, 2)) / h
    w = (dm(Ay, 2) - dm(Ax, 1)) / h
    return u, v, w


def face_umax(u, v, w) -> float:
    """U = max over all faces of |velocity component| (Eq. 24 reading)."""
    return float(max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max()))


def _edge_coords(n, h, shape_axis, stagger):
    """Coordinate of index along one axis: centres (stagger 0) or faces (1)."""
    return centres(n, h, 0.5 if stagger == 0 else 1.0)


def single_vortex_2d(n: int, radius=0.15, centre=(0.5, 0.75), eps_over_h=1.0):
    """Drop in a single vortex (Section 3.3.1, Eq. 33) on an n x n x 1 grid.

    The streamfunction Psi = sin^2(pi x) sin^2(pi y) / pi is sampled at cell
    corners; u = -dPsi/dy, v = dPsi/dx through the staggered curl with
    A_z = -Psi.  The time factor cos(pi t / T) is applied by the stepper.
    """
    h = 1.0 / n
    xc = centres(n, h, 1.0)  # corner coordinates (i+1) h
    Psi = (np.sin(np.pi * xc)[None, :] ** 2) * (np.sin(np.pi * xc)[:, None] ** 2) / np.pi
    Az = -Psi.reshape(1, n, n)
    u, v, w = staggered_curl(None, None, Az, h)
    eps = eps_over_h * h
    phi = tanh_profile(sphere_distance((1, n, n), h, (centre[0], centre[1], 0.0), radius), eps)
    return Fields(phi, u, v, w, h, face_umax(u, v, w))


def deformation_3d(n: int, radius=0.15, centre=(0.35, 0.35, 0.35), eps_over_h=1.0):
    """Sphere in the 3D deformation field on an n^3 periodic unit box.

    u = 2 sin^2(pi x) sin(2 pi y) sin(2 pi z), v = -sin(2 pi x) sin^2(pi y) sin(2 pi z),
    w = -sin(2 pi x) sin(2 pi y) sin^2(pi z) are the curl of
    A = (0, cos2pix sin2piy sin^2piz / 2pi, -(cos2pix sin^2piy + cos2piy) sin2piz / 2pi),
    sampled on the edges and differenced with the staggered curl.
    """
    h = 1.0 / n
    xc = centres(n, h, 0.5)   # cell-centre coordinate
    xf = centres(n, h, 1.0)   # face / edge coordinate
    tp = 2.0 * np.pi
    # A_y on y-edges (i+1/2, j, k+1/2): x face, y centre, z face
    Ay = (np.cos(tp * xf)[None, None, :] * np.sin(tp * xc)[None, :, None]
          * (np.sin(np.pi * xf)[:, None, None] ** 2)) / tp
    # A_z on z-edges (i+1/2, j+1/2, k): x face, y face, z centre
    Az = -((np.cos(tp * xf)[None, None, :] * (np.sin(np.pi * xf)[None, :, None] ** 2)
            + np.cos(tp * xf)[None, :, None]) * np.sin(tp * xc)[:, None, None]) / tp
    Ay = np.broadcast_to(Ay, (n, n, n)).copy()
    Az = np.broadcast_to(Az, (n, n, n)).copy()
    u, v, w = staggered_curl(None, Ay, Az, h)
    eps = eps_over_h * h
    phi = tanh_profile(sphere_distance((n, n, n), h, centre, radius), eps)
    return Fields(phi, u, v, w, h, face_umax(u, v, w))


def _mode_table(rng, nmodes, kmax, ndim):
    """Wave vectors k (nonzero integers, |k| <= kmax), amplitudes a ~ N(0,1)/|k|^2, phases."""
    r = np.arange(-kmax, kmax + 1)
    if ndim == 3:
        K = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    else:
        K = np.stack(np.meshgrid(r, r, indexing="ij"), -1).reshape(-1, 2)
        K = np.concatenate([K, np.zeros((K.shape[0], 1), dtype=K.dtype)], 1)
    n2 = (K * K).sum(1)
    K = K[(n2 > 0) & (n2 <= kmax * kmax)]
    pick = rng.integers(0, K.shape[0], size=nmodes)
    k = K[pick].astype(np.int64)
    kn2 = (k * k).sum(1).astype(np.float64)
    amp = rng.standard_normal((nmodes, 3)) / kn2[:, None]
    theta = rng.uniform(0.0, 2.0 * np.pi, size=nmodes)
    return k, amp, theta


def _eval_modes(shape, offsets, k, coef, theta):
    """sum_m coef_m cos(2 pi sum_d k_md (idx_d + off_d) / N_d + theta_m) on a grid.

    Evaluated separably: exp(i 2 pi k_x x / L_x) etc. per axis, combined with
    one complex matrix product over modes (a library primitive).  The phase
    argument uses (k * idx mod N) / N so it is exact before the cosine.
    """
    nz, ny, nx = shape

    def axis_exp(n, kd, off):
        idx = np.arange(n, dtype=np.int64)
        # exact reduction of the integer part, then add the offset term
        ph = ((kd[:, None] * idx[None, :]) % n).astype(np.float64) / n + (kd[:, None] * off) / n
        return np.exp(2j * np.pi * ph)  # (M, n)

    ex = axis_exp(nx, k[:, 0], offsets[0])
    ey = axis_exp(ny, k[:, 1], offsets[1])
    ez = axis_exp(nz, k[:, 2], offsets[2])
    c = coef * np.exp(1j * theta)                       # (M,)
    yz = (c[:, None, None] * ez[:, :, None] * ey[:, None, :])  # (M, nz, ny)
    out = yz.reshape(len(c), nz * ny).T @ ex          # (nz*ny, nx)
    return np.ascontiguousarray(out.real.reshape(nz, ny, nx))


def fourier_potential(shape, nmodes=32, kmax=4, seed=0):
    """Edge-centred vector potential A = sum_m a_m cos(2 pi k_m . x / L + theta_m).

    k_m uniform over nonzero integer vectors with |k| <= kmax (k_z = 0 when
    nz == 1), a_m in R^3 iid N(0,1)/|k_m|^2, theta_m ~ U[0, 2 pi).  Seeded
    with numpy's PCG64 ``default_rng(seed)``.
    """
    rng = np.random.default_rng(seed)
    ndim = 3 if shape[0] > 1 else 2
    k, amp, theta = _mode_table(rng, nmodes, kmax, ndim)
    # (x, y, z) offsets of each edge family in units of h
    Ax = _eval_modes(shape, (0.5, 1.0, 1.0), k, amp[:, 0], theta)
    Ay = _eval_modes(shape, (1.0, 0.5, 1.0), k, amp[:, 1], theta)
    Az = _eval_modes(shape, (1.0, 1.0, 0.5), k, amp[:, 2], theta)
    return Ax, Ay, Az


def random_velocity(shape, h, nmodes=32, kmax=4, seed=0, umax=1.0):
    """Random divergence-free face velocity, rescaled so U = umax."""
    Ax, Ay, Az = fourier_potential(shape, nmodes, kmax, seed)
    if shape[0] == 1:  # 2D: only the streamfunction component acts in-plane
        Ax = None
        Ay = None
    u, v, w = staggered_curl(Ax, Ay, Az, h)
    U = face_umax(u, v, w)
    if U == 0.0:  # e.g. a 1x1x1 box: the discrete curl vanishes identically
        return u, v, w
    s = umax / U
    return u * s, v * s, w * s


def drop_2d_uniform(eps_over_h, n=50, L=2.0, D=1.0):
    """2D drop of diameter D centred in an L x L periodic box (Section 3.2.1).

    Uniform velocity (sqrt2/2, sqrt2/2).  Returns Fields with the tanh
    initial condition and also the sharp top-hat on the same grid.
    """
    h = L / n
    eps = eps_over_h * h
    s = sphere_distance((1, n, n), h, (L / 2, L / 2, 0.0), D / 2)
    phi = tanh_profile(s, eps)
    c = math.sqrt(2.0) / 2.0
    u = np.full((1, n, n), c)
    v = np.full((1, n, n), c)
    w = np.zeros((1, n, n))
    f = Fields(phi, u, v, w, h, c)
    tophat = (s > 0).astype(np.float64)
    return f, tophat


def random_phi(shape, seed=0, smooth=False):
    """Random phase field in [0, 1]: iid uniform, or a smoothed version."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.0, 1.0, size=shape)
    if smooth:
        for ax in range(3):
            if shape[ax] > 2:
                p = 0.25 * np.roll(p, 1, ax) + 0.5 * p + 0.25 * np.roll(p, -1, ax)
    return p


def random_boxes(nbox=64, nmin=32, nmax=160, seed=0, nmodes=32, kmax=4,
                 eps_choices=(1.0, 1.5), cubic=False):
    """Batch of independent periodic boxes with uneven sizes (batched workload).

    Edge lengths N_d ~ U{nmin..nmax}; h = 1 / min_d N_d (shortest edge has
    length 1); 1-3 ellipsoids with semi-axes in [0.08, 0.2] combined by the
    max of their signed distances; own seeded divergence-free velocity with
    U = 1; eps/h drawn from ``eps_choices``; gamma = U * r with
    r = 1 / (2 eps/h - 1), i.e. exactly on the crossover line of Eq. 17.
    Returns a list of dicts with keys fields, eps, gamma.
    """
    rng = np.random.default_rng(seed)
    boxes = []
    for b in range(nbox):
        if cubic:
            n = int(rng.integers(nmin, nmax + 1))
            dims = (n, n, n)
        else:
            dims = tuple(int(x) for x in rng.integers(nmin, nmax + 1, size=3))
        nz, ny, nx = dims[2], dims[1], dims[0]
        shape = (nz, ny, nx)
        h = 1.0 / min(dims)
        L = (nx * h, ny * h, nz * h)
        s = np.full(shape, -np.inf)
        for _ in range(int(rng.integers(1, 4))):
            ax = tuple(float(a) for a in rng.uniform(0.08, 0.2, size=3))
            c = tuple(float(rng.uniform(0, L[d])) for d in range(3))
            s = np.maximum(s, ellipsoid_distance(shape, h, c, ax))
        eoh = float(eps_choices[int(rng.integers(0, len(eps_choices)))])
        eps = eoh * h
        phi = tanh_profile(s, eps)
        vseed = int(rng.integers(0, 2**31 - 1))
        u, v, w = random_velocity(shape, h, nmodes, kmax, vseed, 1.0)
        U = face_umax(u, v, w)
        gamma = U / (2.0 * eoh - 1.0)
        boxes.append(dict(fields=Fields(phi, u, v, w, h, U), eps=eps, gamma=gamma,
                          eps_over_h=eoh))
    return boxes


# ---------------------------------------------------------------------------
# Device-side variants for large boxes (float64 on a CUDA device via torch).

def spheres_phi_torch(shape, h, spheres, eps, device="cuda", zchunk=64):
    """tanh profile of the union of spheres (max of the periodic signed
    distances R - |x - c|), as ``sphere_distance`` + ``tanh_profile``.
    ``spheres`` is a list of ((x, y, z), R); returns a float64 tensor."""
    import torch
    nz, ny, nx = shape
    out = torch.empty(shape, dtype=torch.float64, device=device)
    ax = [((torch.arange(n, dtype=torch.float64, device=device) + 0.5) * h) for n in (nx, ny, nz)]

    def pd(x, c, L):
        d = x - c
        return d - L * torch.round(d / L)
    for z0 in range(0, nz, zchunk):
        z1 = min(nz, z0 + zchunk)
        s = None
        for (c, R) in spheres:
            dx = pd(ax[0], c[0], nx * h).view(1, 1, nx)
            dy = pd(ax[1], c[1], ny * h).view(1, ny, 1)
            dz = pd(ax[2][z0:z1], c[2], nz * h).view(z1 - z0, 1, 1)
            d = R - torch.sqrt(dx * dx + dy * dy + dz * dz)
            s = d if s is None else torch.maximum(s, d)
        out[z0:z1] = 0.5 * (1.0 + torch.tanh(s / (2.0 * eps)))
    return out


def _eval_modes_torch(shape, offsets, k, coef, theta, device, zchunk=32):
    """``_eval_modes`` on the device: sum_m coef_m cos(2 pi k_m.(idx + off)/N + theta_m)."""
    import torch
    nz, ny, nx = shape

    def axis_exp(n, kd, off):
        idx = torch.arange(n, dtype=torch.int64, device=device)
        kt = torch.as_tensor(kd, dtype=torch.int64, device=device)
        ph = ((kt[:, None] * idx[None, :]) % n).to(torch.float64) / n + (kt[:, None].to(torch.float64) * off) / n
        return torch.polar(torch.ones_like(ph), 2.0 * math.pi * ph)  # (M, n) complex128
    ex = axis_exp(nx, k[:, 0], offsets[0])
    ey = axis_exp(ny, k[:, 1], offsets[1])
    ez = axis_exp(nz, k[:, 2], offsets[2])
    c = torch.polar(torch.as_tensor(coef, dtype=torch.float64, device=device),
                    torch.as_tensor(theta, dtype=torch.float64, device=device))
    out = torch.empty(shape, dtype=torch.float64, device=device)
    for z0 in range(0, nz, zchunk):
        z1 = min(nz, z0 + zchunk)
        yz = c[:, None, None] * ez[:, z0:z1, None] * ey[:, None, :]          # (M, zc, ny)
        out[z0:z1] = (yz.reshape(len(coef), -1).T @ ex).real.reshape(z1 - z0, ny, nx)
    return out


def random_velocity_torch(shape, h, nmodes=32, kmax=4, seed=0, umax=1.0, device="cuda"):
    """``random_velocity`` on the device (same seeded mode table): the discrete
    staggered curl of the Fourier vector potential, rescaled so U = umax.
    Returns float64 tensors (u, v, w)."""
    import torch
    rng = np.random.default_rng(seed)
    ndim = 3 if shape[0] > 1 else 2
    k, amp, theta = _mode_table(rng, nmodes, kmax, ndim)
    Az = _eval_modes_torch(shape, (1.0, 1.0, 0.5), k, amp[:, 2], theta, device)
    if shape[0] == 1:  # 2D: only the streamfunction component acts in-plane
        Ax = torch.zeros_like(Az)
        Ay = torch.zeros_like(Az)
    else:
        Ax = _eval_modes_torch(shape, (0.5, 1.0, 1.0), k, amp[:, 0], theta, device)
        Ay = _eval_modes_torch(shape, (1.0, 0.5, 1.0), k, amp[:, 1], theta, device)

    def dm(a, axis):
        return a - torch.roll(a, 1, dims=axis)
    u = (dm(Az, 1) - dm(Ay, 0)) / h
    v = (dm(Ax, 0) - dm(Az, 2)) / h
    del Az
    w = (dm(Ay, 2) - dm(Ax, 1)) / h
    del Ax, Ay
    U = float(max(u.abs().max(), v.abs().max(), w.abs().max()))
    if U > 0.0:
        sc = umax / U
        u.mul_(sc)
        v.mul_(sc)
        w.mul_(sc)
    return u, v, w
