"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/cdi_oracle.c) against something other
than itself: the paper's coefficient form (Eq. 13, Eq. 18-22), the printed
1D scheme (Eq. 11), the phi -> 1 - phi symmetry (Eq. 16), discrete
conservation, the boundedness theorem (Eq. 17/24 with A <= 1/(2 D_f)), the
below-line classification of Table 2, a constructed exact discrete
equilibrium, Table 1's E_eps, equivariances, and (for the adjoint) finite
differences and a brute-force Jacobian transpose.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1803_01262_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
AX = (2, 1, 0)  # array axis of x, y, z


def coefficient_form_step(phi, u, v, w, dx, dt, eps, gamma, sharpen=True):
    """Eq. 18-22 (and Eq. 13 in 1D), written for 3D: phi' = sum C phi.

    C_c = 1 - 2 D A - (B A / gamma) sum_d (u^d_{c+1/2} - u^d_{c-1/2})   (Eq. 19, D = 3
          terms of the 3D stencil; degenerate axes contribute their A too)
    C_{c-e_d} = A [1 + B (n^d_{c-e_d} (1 - phi_{c-e_d}) + u^d_{c-1/2} / gamma)]   (Eq. 21)
    C_{c+e_d} = A [1 + B (-n^d_{c+e_d} (1 - phi_{c+e_d}) - u^d_{c+1/2} / gamma)]  (Eq. 22)
    """
    A = dt * gamma * eps / dx ** 2
    B = dx / (2 * eps)
    g = [np.roll(phi, -1, a) - np.roll(phi, 1, a) for a in AX]
    m = np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
    safe = np.where(m > 0, m, 1.0)
    n = [np.where((m > 0) & sharpen, gd / safe, 0.0) for gd in g]
    vel = (u, v, w)
    Cc = 1 - 6 * A - (B * A / gamma) * sum(vel[d] - np.roll(vel[d], 1, AX[d]) for d in range(3))
    out = Cc * phi
    for d in range(3):
        a = AX[d]
        pm, nm, um = np.roll(phi, 1, a), np.roll(n[d], 1, a), np.roll(vel[d], 1, a)
        pp, npp, up = np.roll(phi, -1, a), np.roll(n[d], -1, a), vel[d]
        out = out + A * (1 + B * (nm * (1 - pm) + um / gamma)) * pm
        out = out + A * (1 + B * (-npp * (1 - pp) - up / gamma)) * pp
    return out


def eq11_1d(phi, u, dx, dt, eps, gamma):
    """The printed 1D update, Eq. 11, with the sharpening sign read as in Eq. 13."""
    pp, pm = np.roll(phi, -1), np.roll(phi, 1)
    n = np.sign(pp - pm)
    npp, nm = np.roll(n, -1), np.roll(n, 1)
    adv = -u * (pp - pm) / (2 * dx)
    dif = gamma * eps * (pp - 2 * phi + pm) / dx ** 2
    shp = gamma * ((pp ** 2 - pp) * npp - (pm ** 2 - pm) * nm) / (2 * dx)
    return phi + dt * (adv + dif + shp)


def rand_case(shape, seed, solenoidal=True, h=0.05):
    rng = np.random.default_rng(seed)
    phi = I.random_phi(shape, seed)
    if solenoidal:
        u, v, w = I.random_velocity(shape, h, nmodes=8, kmax=3, seed=seed + 1)
    else:
        u, v, w = (rng.standard_normal(shape) for _ in range(3))
    return phi, u, v, w, h


@pytest.mark.parametrize("shape", [(1, 1, 17), (1, 9, 11), (5, 6, 7), (4, 4, 4), (3, 1, 8)])
@pytest.mark.parametrize("solenoidal", [True, False])
def test_coefficient_form(shape, solenoidal):
    """Flux form == Eq. 13 / Eq. 18-22 coefficient form (any periodic u)."""
    phi, u, v, w, h = rand_case(shape, 11, solenoidal)
    dt, eps, gamma = 0.3 * h * h, 1.2 * h, 0.8
    a = oracle.step(phi, u, v, w, h, dt, eps, gamma)
    b = coefficient_form_step(phi, u, v, w, h, dt, eps, gamma)
    assert np.abs(a - b).max() < 2e-15


F32_TINY, F64_TINY = 1.17549435e-38, 2.2250738585072014e-308


@pytest.mark.parametrize("shape", [(1, 9, 11), (5, 6, 7)])
def test_floor_invisible_at_working_scale(shape):
    """The floor under |g|^2 is invisible wherever |g|^2 is far above it: DBL_MIN
    changes no bit of a step or an adjoint on O(1) fields, FLT_MIN changes no
    value by more than a few ulps."""
    phi, u, v, w, h = rand_case(shape, 12)
    lam = np.random.default_rng(2).standard_normal(shape)
    args = dict(dx=h, dt=0.2 * h * h, eps=h, gamma=1.1, vel_scale=0.9)
    base = oracle.step(phi, u, v, w, **args)
    assert np.array_equal(oracle.step(phi, u, v, w, tiny=F64_TINY, **args), base)
    assert np.abs(oracle.step(phi, u, v, w, tiny=F32_TINY, **args) - base).max() < 1e-15
    abase = oracle.adjoint(phi, u, v, w, lam, **args)
    assert np.array_equal(oracle.adjoint(phi, u, v, w, lam, tiny=F64_TINY, **args), abase)
    assert np.abs(oracle.adjoint(phi, u, v, w, lam, tiny=F32_TINY, **args) - abase).max() < 1e-14


@pytest.mark.parametrize("solenoidal", [True, False])
def test_floor_above_gradient_removes_sharpening(solenoidal):
    """A floor far above |g|^2 shrinks the normal to ~g/sqrt(tiny) -> 0: the step becomes
    the sharpening-free advection-diffusion step of Eq. 18-22 (all n = 0); a floor
    placed anywhere but under the root (e.g. on the numerator) fails this."""
    phi, u, v, w, h = rand_case((4, 5, 6), 13, solenoidal)
    dt, eps, gamma = 0.3 * h * h, 1.2 * h, 0.8
    a = oracle.step(phi, u, v, w, h, dt, eps, gamma, tiny=1e40)
    b = coefficient_form_step(phi, u, v, w, h, dt, eps, gamma, sharpen=False)
    assert np.abs(a - b).max() < 2e-15
    assert np.abs(a - coefficient_form_step(phi, u, v, w, h, dt, eps, gamma)).max() > 1e-4


def test_eq11_1d():
    """ny = nz = 1 reduces exactly to the printed 1D scheme (Eq. 11)."""
    n, h = 40, 1.0 / 40
    x = I.centres(n, h)
    phi = I.tanh_profile(0.25 - np.abs(x - 0.5), h)
    rng = np.random.default_rng(3)
    phi = np.clip(phi + 0.05 * rng.standard_normal(n), 0, 1)
    u = 0.7
    dt, eps, gamma = 0.2 * h, 1.1 * h, 1.3
    ours = oracle.step(phi.reshape(1, 1, n), np.full((1, 1, n), u), np.zeros((1, 1, n)),
                       np.zeros((1, 1, n)), h, dt, eps, gamma)[0, 0]
    ref = eq11_1d(phi, u, h, dt, eps, gamma)
    assert np.abs(ours - ref).max() < 1e-15


def test_sign_reading_matters():
    """A plausible mistake (the '+' printed in Eq. 11) is caught by Eq. 13."""
    n, h = 32, 1.0 / 32
    phi = I.tanh_profile(0.2 - np.abs(I.centres(n, h) - 0.5), h)
    pp, pm = np.roll(phi, -1), np.roll(phi, 1)
    nn = np.sign(pp - pm)
    wrong = ((pp ** 2 - pp) * np.roll(nn, -1) - (pm ** 2 + pm) * np.roll(nn, 1))
    right = ((pp ** 2 - pp) * np.roll(nn, -1) - (pm ** 2 - pm) * np.roll(nn, 1))
    assert np.abs(wrong - right).max() > 0.1


@pytest.mark.parametrize("shape", [(1, 12, 10), (6, 5, 7), (2, 3, 4)])
def test_symmetry_eq16(shape):
    """step(1 - phi) = 1 - step(phi) for discretely solenoidal u (Eq. 16)."""
    phi, u, v, w, h = rand_case(shape, 5)
    args = (u, v, w, h, 0.2 * h * h, h, 1.0)
    a = oracle.step(1 - phi, *args)
    b = 1 - oracle.step(phi, *args)
    assert np.abs(a - b).max() < 1e-15
    # the floor keeps the symmetry (|g| is even under phi -> 1 - phi)
    a = oracle.step(1 - phi, *args, tiny=1e-3)
    b = 1 - oracle.step(phi, *args, tiny=1e-3)
    assert np.abs(a - b).max() < 1e-15


def test_symmetry_defect_is_divergence():
    """For non-solenoidal u the Eq. 16 defect is exactly -dt * div(u) (derived)."""
    phi, u, v, w, h = rand_case((4, 5, 6), 8, solenoidal=False)
    dt = 0.1 * h * h
    a = oracle.step(1 - phi, u, v, w, h, dt, h, 1.0)
    b = 1 - oracle.step(phi, u, v, w, h, dt, h, 1.0)
    div = sum(vel - np.roll(vel, 1, AX[d]) for d, vel in enumerate((u, v, w))) / h
    assert np.abs((a - b) + dt * div).max() < 1e-13


@pytest.mark.parametrize("solenoidal", [True, False])
def test_conservation(solenoidal):
    """sum phi^{k+1} = sum phi^k to round-off for any periodic u (telescoping fluxes)."""
    phi, u, v, w, h = rand_case((7, 8, 9), 2, solenoidal)
    p = phi
    for _ in range(10):
        p = oracle.step(p, u, v, w, h, 0.2 * h * h, 1.5 * h, 1.0)
    assert abs(p.sum() - phi.sum()) / phi.sum() < 1e-14


def test_constant_field():
    """phi = c with discretely solenoidal u stays c to round-off."""
    shape = (6, 7, 8)
    _, u, v, w, h = rand_case(shape, 4)
    for c in (0.0, 0.3, 1.0):
        p = oracle.step(np.full(shape, c), u, v, w, h, 0.2 * h * h, h, 1.0)
        assert np.abs(p - c).max() < 1e-14


def stencil_rhs_at(phi, u, v, w, dx, eps, gamma, c):
    """d phi/dt at cell c = (k, j, i) evaluated on its own from the five steps of
    Section 2.2: every normal, sharpening value and face flux it needs is formed
    from explicit neighbour indices (no whole-array passes), a third formulation
    next to the oracle's passes and the coefficient form."""
    nz, ny, nx = phi.shape
    ext = (nx, ny, nz)
    vel = (u, v, w)

    def at(a, q):
        return a[q[2] % nz, q[1] % ny, q[0] % nx]

    def shift(q, d, s):
        r = list(q)
        r[d] += s
        return tuple(r)

    def sharp(q):
        g = [at(phi, shift(q, d, 1)) - at(phi, shift(q, d, -1)) for d in range(3)]
        m = math.sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2])
        p = at(phi, q)
        return [0.0 if m == 0 else p * (1 - p) * gd / m for gd in g]

    q0 = (c[2], c[1], c[0])  # (i, j, k)
    div = 0.0
    for d in range(3):
        if ext[d] == 1:
            continue   # a degenerate axis: its faces carry equal fluxes
        for lo, hi, sign in ((q0, shift(q0, d, 1), 1.0), (shift(q0, d, -1), q0, -1.0)):
            uf = at(vel[d], lo)   # u[k][j][i] is the face at i + 1/2
            pl, pr = at(phi, lo), at(phi, hi)
            F = uf * (pl + pr) / 2 - gamma * eps * (pr - pl) / dx + gamma * (sharp(lo)[d] + sharp(hi)[d]) / 2
            div += sign * F
    return -div / dx


@pytest.mark.parametrize("shape", [(1, 1, 6), (1, 5, 6), (3, 4, 5), (6, 6, 6), (2, 3, 1)])
@pytest.mark.parametrize("solenoidal", [True, False])
def test_brute_force_stencil(shape, solenoidal):
    """The oracle's right-hand side equals a cell-by-cell evaluation from the stencil."""
    phi, u, v, w, h = rand_case(shape, 17 + sum(shape), solenoidal)
    eps, gamma = 1.3 * h, 0.8
    ref = oracle.rhs(phi, u, v, w, h, eps, gamma)
    nz, ny, nx = shape
    brute = np.array([[[stencil_rhs_at(phi, u, v, w, h, eps, gamma, (k, j, i)) for i in range(nx)]
                       for j in range(ny)] for k in range(nz)])
    assert np.abs(brute - ref).max() <= 1e-12 * np.abs(ref).max()


def test_stencil_footprint_is_25_points():
    """d phi/dt at a cell depends on exactly 25 cells: itself, +-1 and +-2 along each axis
    and the 12 edge diagonals (normals of the face neighbours reach one cell beyond)."""
    n = 7
    phi, u, v, w, h = rand_case((n, n, n), 5)
    eps, gamma = h, 1.0
    c = (3, 3, 3)
    base = oracle.rhs(phi, u, v, w, h, eps, gamma)[c]
    found = set()
    for k in range(n):
        for j in range(n):
            for i in range(n):
                q = phi.copy()
                q[k, j, i] += 1e-6
                if abs(oracle.rhs(q, u, v, w, h, eps, gamma)[c] - base) > 1e-12:
                    found.add((k - 3, j - 3, i - 3))
    axes = {t for d in range(3) for s in (-2, -1, 1, 2) for t in [tuple(s if e == d else 0 for e in range(3))]}
    diag = {t for a in range(3) for b in range(a + 1, 3) for sa in (-1, 1) for sb in (-1, 1)
            for t in [tuple(sa if e == a else sb if e == b else 0 for e in range(3))]}
    assert found == {(0, 0, 0)} | axes | diag and len(found) == 25


def discrete_equilibrium_1d(n, e):
    """Exact zero-flux profile of the scheme at u = 0, eps/dx = e (derived).

    With n = +1 on a rising profile, a zero face flux means
    e (phi_{i+1} - phi_i) = (phi_i (1 - phi_i) + phi_{i+1} (1 - phi_{i+1})) / 2,
    a quadratic in either neighbour.  March it up and down from 0.5, then
    mirror it so the periodic box holds a drop.
    """
    half = n // 2
    up = np.empty(half)
    c0 = half // 2
    up[c0] = 0.5
    for i in range(c0, half - 1):
        p = up[i]
        c = e * p + 0.5 * p * (1 - p)
        up[i + 1] = -(e - 0.5) + math.sqrt((e - 0.5) ** 2 + 2 * c)
    for i in range(c0, 0, -1):
        x = up[i]
        q = e * x - 0.5 * x * (1 - x)
        up[i - 1] = (e + 0.5) - math.sqrt((e + 0.5) ** 2 - 2 * q)
    return np.concatenate([up, up[::-1]])


@pytest.mark.parametrize("e", [0.7, 1.0, 1.5])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_discrete_equilibrium_is_stationary(e, axis):
    """A constructed exact discrete equilibrium is left unchanged by a step.

    This fixes the sharpening sign, the centre-product-then-average
    interpolation (Section 2.2, second step), the diffusion coefficient and
    the dx scaling: a face-product sharpening term or a wrong sign moves it.
    """
    n, h = 240, 1.0 / 240
    prof = discrete_equilibrium_1d(n, e)
    shape = [4, 3, 5]
    shape[AX[axis]] = n
    sh = [1, 1, 1]
    sh[AX[axis]] = n
    phi = np.broadcast_to(prof.reshape(sh), shape).copy()
    z = np.zeros(shape)
    dt = 0.16 * h * h / (1.0 * e * h)  # A = 0.16
    p = oracle.step(phi, z, z, z, h, dt, e * h, 1.0)
    assert np.abs(p - phi).max() < 1e-15
    # the analytic tanh profile is only near-stationary: it does move
    x = I.centres(n, h)
    tanh = I.tanh_profile(0.25 - np.abs(x - 0.5), e * h)
    t = np.broadcast_to(tanh.reshape(sh), shape).copy()
    assert np.abs(oracle.step(t, z, z, z, h, dt, e * h, 1.0) - t).max() > 1e-6


def test_tanh_relaxes_to_the_discrete_equilibrium():
    """The analytic tanh drop at u = 0 is only near-stationary (a ~4% face-flux residual at
    eps = dx); stepping it, the per-step change decays by more than ten orders of magnitude
    within 1000 steps, the 0.5-contour stays where it was (the drop is symmetric and mass is
    conserved), and the profile it settles to has zero flux through every face:
    e (phi_R - phi_L) = (s_L + s_R) / 2 with s = phi (1 - phi) n (derived)."""
    n, e = 200, 1.0
    h = 1.0 / n
    x = I.centres(n, h)
    phi = I.tanh_profile(0.25 - np.abs(x - 0.5), e * h).reshape(1, 1, n)
    z = np.zeros_like(phi)
    dt = 0.16 * h * h / (e * h)  # A = 0.16

    def change(p):
        return np.abs(oracle.step(p, z, z, z, h, dt, e * h, 1.0) - p).max()

    def contour(p):
        p = p.ravel()
        i = int(np.argmax((p[:-1] < 0.5) & (p[1:] >= 0.5)))
        return x[i] + (0.5 - p[i]) / (p[i + 1] - p[i]) * h

    def face_flux(p):  # gamma = 1, dx = 1 units
        p = p.ravel()
        sgn = np.sign(np.roll(p, -1) - np.roll(p, 1))
        s = p * (1 - p) * sgn
        return -e * (np.roll(p, -1) - p) + 0.5 * (s + np.roll(s, -1)), 0.5 * (s + np.roll(s, -1))

    F0, S0 = face_flux(phi)
    assert 0.01 < np.abs(F0).max() / np.abs(S0).max() < 0.06
    relaxed = oracle.run(phi, z, z, z, h, dt, e * h, 1.0, 1000)
    assert change(relaxed) < 1e-10 * change(phi)
    assert abs(contour(relaxed) - contour(phi)) < 1e-9 * h
    assert abs(relaxed.sum() - phi.sum()) < 1e-12 * phi.sum()
    F, S = face_flux(relaxed)
    assert np.abs(F).max() < 1e-12 * np.abs(S).max()


def test_face_product_variant_is_not_stationary():
    """The face-product reading of the sharpening term breaks the equilibrium."""
    n, h, e = 240, 1.0 / 240, 1.0
    p = discrete_equilibrium_1d(n, e)
    pr = np.roll(p, -1)
    pf = 0.5 * (p + pr)
    nn = np.sign(np.roll(p, -1) - np.roll(p, 1))
    nf = 0.5 * (nn + np.roll(nn, -1))
    F = -e * (pr - p) + pf * (1 - pf) * nf  # gamma = dx = 1 units
    assert np.abs(F - np.roll(F, 1)).max() > 1e-4


def test_face_form_not_stationary_in_the_oracle():
    """The oracle's face-product form moves the discrete equilibrium that its default
    (centre-product) form leaves unchanged."""
    n, h = 240, 1.0 / 240
    p = discrete_equilibrium_1d(n, 1.0).reshape(1, 1, n)
    z = np.zeros_like(p)
    args = (z, z, z, h, 0.2 * h * h, h, 1.0)
    assert np.abs(oracle.step(p, *args) - p).max() < 1e-15
    assert np.abs(oracle.step(p, *args, sharpen="face") - p).max() > 1e-6


def test_face_form_1d_closed_form():
    """Where a face's two cells have equal normals n, the face-product flux exceeds the
    centre-product flux by gamma n (phi_R - phi_L)^2 / 4 (phi_f (1 - phi_f) against the
    mean of phi (1 - phi)), so on cells whose four neighbouring normals agree the two steps
    differ by -(dt/dx) of the difference of that term across the cell."""
    n = 64
    h = 1.0 / n
    x = I.centres(n, h)
    phi = 0.5 * (1 + np.tanh((0.3 - np.abs(x - 0.5)) / (2 * 1.3 * h)))
    phi = (phi + 0.02 * np.sin(6 * np.pi * x)).reshape(1, 1, n)
    u = np.full((1, 1, n), 0.4)
    z = np.zeros_like(phi)
    dt, eps, gamma = 0.1 * h, 1.1 * h, 0.9
    c = oracle.step(phi, u, z, z, h, dt, eps, gamma)[0, 0]
    f = oracle.step(phi, u, z, z, h, dt, eps, gamma, sharpen="face")[0, 0]
    p = phi[0, 0]
    nn = np.sign(np.roll(p, -1) - np.roll(p, 1))
    D = gamma * nn * (np.roll(p, -1) - p) ** 2 / 4          # on face i+1/2 (cells i, i+1)
    expect = c - dt / h * (D - np.roll(D, 1))
    ok = (np.roll(nn, 1) == nn) & (np.roll(nn, -1) == nn) & (nn != 0)
    assert ok.sum() > n // 2
    assert np.abs(f - expect)[ok].max() < 1e-15
    assert np.abs(f - c)[ok].max() > 1e-5


@pytest.mark.parametrize("solenoidal", [True, False])
def test_face_form_conserves_and_is_symmetric(solenoidal):
    """The face form telescopes like the centre form (conservation for any periodic u) and
    keeps Eq. 16's phi -> 1 - phi symmetry for discretely solenoidal u."""
    phi, u, v, w, h = rand_case((5, 6, 7), 23, solenoidal)
    args = dict(dx=h, dt=0.2 * h * h, eps=h, gamma=1.2, sharpen="face")
    out = oracle.step(phi, u, v, w, **args)
    assert abs(out.sum() - phi.sum()) < 1e-12 * phi.size
    if solenoidal:
        assert np.abs(oracle.step(1 - phi, u, v, w, **args) - (1 - out)).max() < 1e-15


def test_boundedness_theorem_random_boxes():
    """0 <= phi <= 1 (within machine eps) under Eq. 24 and A <= 1/(2 D_f).

    1000 seeded small periodic boxes with random solenoidal velocity, eps/dx
    on or above the crossover line (every fifth box exactly on it), A up to
    1/(2 D_f) (every seventh box exactly at it), U = max face |component|.
    """
    rng = np.random.default_rng(2024)
    tol = np.finfo(np.float64).eps
    worst = 0
    for b in range(1000):
        dims = rng.integers(3, 10, size=3)
        if b % 4 == 0:
            dims[0] = 1
        shape = tuple(int(x) for x in dims)
        h = 1.0 / max(shape)
        phi = I.random_phi(shape, int(rng.integers(1 << 30)), smooth=bool(b % 2))
        u, v, w = I.random_velocity(shape, h, 8, 3, int(rng.integers(1 << 30)))
        U = I.face_umax(u, v, w)
        eoh = float(rng.uniform(0.55, 2.0))
        gmin = 1.0 / (2 * eoh - 1) if eoh > 0.5 else np.inf
        gamma = U * gmin * (1.0 if b % 5 == 0 else float(rng.uniform(1.0, 2.0)))
        Df = sum(1 for s in shape if s > 1)
        eps = eoh * h
        dt = (1.0 if b % 7 == 0 else float(rng.uniform(0.5, 1.0))) * h * h / (2 * Df * gamma * eps)
        p = phi
        for _ in range(25):
            p = oracle.step(p, u, v, w, h, dt, eps, gamma)
            worst = max(worst, int(((p < -tol) | (p > 1 + tol)).sum()))
    assert worst == 0


def _table2_run(eoh, gu):
    f, _ = I.drop_2d_uniform(eoh)
    h, eps, gamma = f.h, eoh * f.h, gu
    dt = min(h * h / (4 * gamma * eps), h / (f.u.max() + f.v.max() + 2 * gamma))
    T = 2 * math.sqrt(2)
    n = int(math.ceil(T / dt))
    dt = T / n
    p, tol, bad = f.phi, np.finfo(float).eps, 0
    for _ in range(n):
        p = oracle.step(p, f.u, f.v, f.w, h, dt, eps, gamma)
        bad += int(((p < -tol) | (p > 1 + tol)).sum())
    return bad


@pytest.mark.parametrize("point,eoh,gu,bounded", [
    (1, 1.5, 0.5, True), (2, 1.0, 1.0, True), (3, 5 / 6, 1.5, True), (4, 1.5, 1.5, True),
    (5, 0.9, 0.9, True), (6, 0.8, 0.8, False), (7, 0.7, 0.7, False)])
def test_table2_uniform_classification(point, eoh, gu, bounded):
    """Table 2 (uniform velocity): points 1-5 bounded, 6-7 not.

    The paper ran RK4; here explicit Euler with A <= 1/4.  Points 1-5 satisfy
    Eq. 23 (component maxima), 6-7 violate it, as the paper explains.
    """
    assert (_table2_run(eoh, gu) == 0) == bounded


def test_table1_e_eps():
    """E_eps of the 2D drop initial condition reproduces Table 1 within 3%."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_e_eps.txt"))
    for _, eoh, _, ref in rows:
        f, th = I.drop_2d_uniform(eoh)
        E = np.abs(f.phi - th).sum() * f.h ** 2 / 4.0
        assert abs(E / ref - 1) < 0.03, (eoh, E, ref)


@pytest.mark.parametrize("sharpen", ["centre", "face"])
def test_equivariance(sharpen):
    """Periodic shift, x<->y swap (with u<->v) and x-reflection (u -> -u); for the face form
    the reflection also pins the normal's two-sided interpolation to the face."""
    phi, u, v, w, h = rand_case((5, 6, 6), 9)
    args = dict(dx=h, dt=0.2 * h * h, eps=h, gamma=1.1, sharpen=sharpen)
    base = oracle.step(phi, u, v, w, **args)
    r = lambda a: np.roll(np.roll(a, 2, 2), -1, 0)
    assert np.abs(oracle.step(r(phi), r(u), r(v), r(w), **args) - r(base)).max() == 0.0
    s = lambda a: np.swapaxes(a, 1, 2)
    sw = oracle.step(s(phi), s(v), s(u), s(w), **args)
    assert np.abs(sw - s(base)).max() < 1e-15
    fl = lambda a: a[:, :, ::-1]
    ur = -np.roll(fl(u), -1, 2)  # face i+1/2 of the mirror is face N-2-i+1/2
    rf = oracle.step(fl(phi), ur, fl(v), fl(w), **args)
    assert np.abs(rf - fl(base)).max() < 1e-15


def test_degenerate_z_is_2d():
    """nz = 1: any w is inert and the 2D coefficient form (Eq. 18) holds."""
    phi, u, v, w, h = rand_case((1, 8, 9), 12)
    a = oracle.step(phi, u, v, w, h, 0.2 * h * h, h, 1.0)
    b = oracle.step(phi, u, v, np.zeros_like(w) + 3.0, h, 0.2 * h * h, h, 1.0)
    assert np.array_equal(a, b)


def test_velocity_generators():
    """Staggered curl is discretely solenoidal; analytic fields are reproduced."""
    for f in (I.single_vortex_2d(32), I.deformation_3d(24)):
        div = sum(vel - np.roll(vel, 1, AX[d]) for d, vel in enumerate((f.u, f.v, f.w)))
        assert np.abs(div).max() / f.h < 1e-11
    n = 64
    f = I.single_vortex_2d(n)
    xf, yc = I.centres(n, f.h, 1.0), I.centres(n, f.h, 0.5)
    ua = -np.sin(np.pi * xf)[None, :] ** 2 * np.sin(2 * np.pi * yc)[:, None]
    assert np.abs(f.u[0] - ua).max() < 5e-3
    n = 32
    f = I.deformation_3d(n)
    xf, xc = I.centres(n, f.h, 1.0), I.centres(n, f.h, 0.5)
    ua = (2 * np.sin(np.pi * xf)[None, None, :] ** 2 * np.sin(2 * np.pi * xc)[None, :, None]
          * np.sin(2 * np.pi * xc)[:, None, None])
    assert np.abs(f.u - ua).max() < 2e-2
    u, v, w = I.random_velocity((6, 7, 8), 0.1, 16, 4, 3)
    div = sum(vel - np.roll(vel, 1, AX[d]) for d, vel in enumerate((u, v, w)))
    assert np.abs(div).max() < 1e-10 and abs(I.face_umax(u, v, w) - 1.0) < 1e-15


def test_stats():
    """Oracle reductions against plain numpy on a field with planted violations."""
    p = I.random_phi((4, 5, 6), 1)
    p[0, 0, 0], p[1, 2, 3], p[3, 4, 5] = -1e-20, 1 + 1e-10, -0.3
    s = oracle.stats(p, 0.5, 1e-15)
    assert s["n_strict"] == 3 and s["n_tol"] == 2
    assert s["min"] == -0.3 and s["max"] == 1 + 1e-10
    assert abs(s["sum"] - p.sum()) < 1e-12 and abs(s["mass"] - 0.5 * p.sum()) < 1e-12


# ---------------------------------------------------------------- adjoint pins

def _fd_jvp(phi, u, v, w, dphi, args, hfd=1e-6):
    a = oracle.step(phi + hfd * dphi, u, v, w, **args)
    b = oracle.step(phi - hfd * dphi, u, v, w, **args)
    return (a - b) / (2 * hfd)


@pytest.mark.parametrize("shape", [(1, 1, 12), (1, 7, 8), (4, 5, 6), (32, 32, 32)])
def test_adjoint_dot_product(shape):
    """<J dphi, lam> (central FD) == <dphi, J^T lam> (adjoint) to 1e-7 relative."""
    rng = np.random.default_rng(7)
    phi, u, v, w, h = rand_case(shape, 21)
    phi = 0.1 + 0.8 * I.random_phi(shape, 3, smooth=True)
    args = dict(dx=h, dt=0.2 * h * h, eps=1.2 * h, gamma=1.3, vel_scale=0.8)
    lam = rng.standard_normal(shape)
    dphi = rng.standard_normal(shape)
    jv = _fd_jvp(phi, u, v, w, dphi, args)
    jt = oracle.adjoint(phi, u, v, w, lam, **args)
    lhs, rhs = (jv * lam).sum(), (dphi * jt).sum()
    assert abs(lhs - rhs) <= 1e-7 * (abs(lhs) + abs(rhs))


def test_adjoint_sampled_entries_32():
    """On a 32^3 box with a tanh sphere, entries of the adjoint J^T lam at sampled cells of
    the interface band (|g|^2 > 1e-4, where a small perturbation keeps the normal in its
    linear range; in the tails |g| ~ 1e-5 and it does not) equal Richardson-extrapolated
    central differences of <lam, step(phi)> in phi at that cell to 1e-9 relative (they agree
    to ~3e-11; leaving the sharpening out of the adjoint moves entries by ~14%)."""
    shape = (32, 32, 32)
    rng = np.random.default_rng(11)
    _, u, v, w, h = rand_case(shape, 31)
    phi = I.tanh_profile(I.sphere_distance(shape, h, (0.45 * 32 * h, 0.5 * 32 * h, 0.55 * 32 * h), 8 * h), 1.2 * h)
    args = dict(dx=h, dt=0.2 * h * h, eps=1.2 * h, gamma=1.3, vel_scale=0.8)
    lam = rng.standard_normal(shape)
    jt = oracle.adjoint(phi, u, v, w, lam, **args)
    g2 = sum((np.roll(phi, -1, a) - np.roll(phi, 1, a)) ** 2 for a in AX)
    band = np.argwhere(g2 > 1e-4)
    cells = [tuple(int(i) for i in band[j]) for j in rng.choice(len(band), 8, replace=False)]
    cells.append(tuple(int(i) for i in np.unravel_index(np.argmax(g2), shape)))

    def dl(c, e):
        pp, pm = phi.copy(), phi.copy()
        pp[c] += e
        pm[c] -= e
        return ((oracle.step(pp, u, v, w, **args) - oracle.step(pm, u, v, w, **args)) * lam).sum() / (2 * e)

    for c in cells:
        fd = (4 * dl(c, 5e-6) - dl(c, 1e-5)) / 3
        assert abs(fd - jt[c]) <= 1e-9 * abs(jt[c]), (c, fd, jt[c])


@pytest.mark.parametrize("shape", [(1, 1, 12), (4, 5, 6)])
def test_adjoint_dot_product_with_floor(shape):
    """With the floor of the same size as |g|^2 (so that n = g/sqrt(|g|^2 + tiny) is far
    from a unit vector) the adjoint is still the transpose of the step's Jacobian."""
    rng = np.random.default_rng(17)
    phi, u, v, w, h = rand_case(shape, 22)
    phi = 0.1 + 0.8 * I.random_phi(shape, 5, smooth=True)
    g2 = sum((np.roll(phi, -1, a) - np.roll(phi, 1, a)) ** 2 for a in AX)
    tiny = float(np.median(g2))
    args = dict(dx=h, dt=0.2 * h * h, eps=1.2 * h, gamma=1.3, vel_scale=0.8, tiny=tiny)
    lam = rng.standard_normal(shape)
    dphi = rng.standard_normal(shape)
    jv = _fd_jvp(phi, u, v, w, dphi, args)
    jt = oracle.adjoint(phi, u, v, w, lam, **args)
    lhs, rhs = (jv * lam).sum(), (dphi * jt).sum()
    assert abs(lhs - rhs) <= 1e-7 * (abs(lhs) + abs(rhs))
    # and the floor matters here: the unit-normal adjoint differs
    jt0 = oracle.adjoint(phi, u, v, w, lam, **{**args, "tiny": 0.0})
    assert abs((dphi * jt0).sum() - rhs) > 1e-4 * abs(rhs)


def test_adjoint_brute_force_transpose():
    """Adjoint columns == rows of the FD Jacobian on a tiny box (every entry)."""
    shape = (3, 4, 5)
    phi, u, v, w, h = rand_case(shape, 31)
    phi = 0.05 + 0.9 * I.random_phi(shape, 4, smooth=True)
    args = dict(dx=h, dt=0.2 * h * h, eps=h, gamma=1.0, vel_scale=1.0)
    n = phi.size
    J = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        J[:, c] = _fd_jvp(phi, u, v, w, e.reshape(shape), args).ravel()
    for r in range(0, n, 7):
        e = np.zeros(n)
        e[r] = 1.0
        col = oracle.adjoint(phi, u, v, w, e.reshape(shape), **args).ravel()
        assert np.abs(col - J[r]).max() < 1e-7


def test_adjoint_velocity_gradient():
    """Velocity gradient of <lam, phi'> against central FD in each component."""
    rng = np.random.default_rng(3)
    shape = (4, 4, 5)
    phi, u, v, w, h = rand_case(shape, 41)
    args = dict(dx=h, dt=0.2 * h * h, eps=h, gamma=1.0, vel_scale=0.7)
    lam = rng.standard_normal(shape)
    _, gu, gv, gw = oracle.adjoint(phi, u, v, w, lam, want_vel=True, **args)
    vel = [u, v, w]
    for d, g in enumerate((gu, gv, gw)):
        dv = rng.standard_normal(shape)
        vp = [x.copy() for x in vel]
        vm = [x.copy() for x in vel]
        vp[d] += 1e-6 * dv
        vm[d] -= 1e-6 * dv
        fd = ((oracle.step(phi, *vp, **args) - oracle.step(phi, *vm, **args)) / 2e-6 * lam).sum()
        assert abs(fd - (g * dv).sum()) <= 1e-7 * abs(fd) + 1e-12


def test_adjoint_constant_lambda():
    """lam' = const gives lam = lam' exactly: J^T 1 = 1 follows from conservation."""
    phi, u, v, w, h = rand_case((4, 5, 6), 51, solenoidal=False)
    lam = oracle.adjoint(phi, u, v, w, np.full(phi.shape, 2.5), h, 0.2 * h * h, h, 1.0)
    assert np.abs(lam - 2.5).max() == 0.0


# ------------------------------------------------------------ RK pins (Section 2.3)

@pytest.mark.parametrize("scheme,poly", [
    ("euler", [1, 1]), ("rk2", [1, 1, 1 / 2]), ("rk3", [1, 1, 1 / 2, 1 / 6]),
    ("rk4", [1, 1, 1 / 2, 1 / 6, 1 / 24])])
def test_rk_amplification_polynomials(scheme, poly):
    """On y' = lam y each scheme multiplies y by its stability polynomial R(z), z = lam dt
    (explicit midpoint and Wray's RK3 and classic RK4 are all order-p, p-stage schemes)."""
    for z in (-0.7, -0.1, 0.3, -1.9):
        got = oracle.rk_advance(lambda y, t: z * y, np.array([1.0]), 0.0, 1.0, scheme)[0]
        assert abs(got - sum(c * z ** k for k, c in enumerate(poly))) < 1e-14


def test_rk_time_dependent_stage_times():
    """Stage times: y' = cos(t) integrated over one step matches sin to the scheme's order."""
    for scheme, p in (("rk2", 2), ("rk3", 3), ("rk4", 4)):
        errs = []
        for dt in (0.2, 0.1):
            y = np.array([0.0])
            for i in range(int(round(1.0 / dt))):
                y = oracle.rk_advance(lambda yy, t: np.cos(t) + 0 * yy, y, i * dt, dt, scheme)
            errs.append(abs(y[0] - np.sin(1.0)))
        assert errs[1] < errs[0] and np.log2(errs[0] / errs[1]) > p - 0.3


@pytest.mark.parametrize("scheme,order", [("euler", 1), ("rk2", 2), ("rk3", 3), ("rk4", 4)])
def test_rk_convergence_order_on_cdi(scheme, order):
    """Temporal order of each scheme on the CDI right-hand side (smooth 2D field)."""
    shape = (1, 16, 16)
    h = 1.0 / 16
    phi = 0.2 + 0.6 * I.random_phi(shape, 3, smooth=True)
    u, v, w = I.random_velocity(shape, h, 6, 2, 4)
    eps, gamma, T = h, 1.0, 0.004
    ref = oracle.rk_run(phi, u, v, w, h, T / 256, eps, gamma, 256, "rk4", period=0.5)
    errs = []
    for n in (16, 32):
        out = oracle.rk_run(phi, u, v, w, h, T / n, eps, gamma, n, scheme, period=0.5)
        errs.append(np.abs(out - ref).max())
    rate = np.log2(errs[0] / errs[1])
    assert rate > order - 0.15, (scheme, errs, rate)


@pytest.mark.parametrize("scheme", ["rk2", "rk3", "rk4"])
def test_rk_conservation_and_boundedness(scheme):
    """Every stage conserves mass; with dt = Eq. 26-28 and parameters on the crossover line
    the solution stays in [0, 1] (the paper's observation for RK, Section 2.3)."""
    rng = np.random.default_rng(9)
    tol = np.finfo(float).eps
    lim = {"rk2": 1.0 / 2, "rk3": 2.51 / 4, "rk4": 2.79 / 4}[scheme]
    for b in range(6):
        shape = (int(rng.integers(3, 8)), int(rng.integers(3, 8)), int(rng.integers(3, 8)))
        h = 1.0 / max(shape)
        phi = I.random_phi(shape, b, smooth=True)
        u, v, w = I.random_velocity(shape, h, 8, 2, 100 + b)
        U = I.face_umax(u, v, w)
        eps, gamma = h, U
        dt = 0.95 * lim * h * h / (3 * gamma * eps)
        p = phi
        for _ in range(20):
            p = oracle.rk_step(p, u, v, w, h, dt, eps, gamma, scheme)
            assert ((p < -tol) | (p > 1 + tol)).sum() == 0
        assert abs(p.sum() - phi.sum()) <= 1e-13 * phi.sum()


def test_adjoint_floor_values():
    """delta = 8 machine epsilons = 16 units in the last place just below 1."""
    assert oracle.adjoint_floor_of(np.float32) == 2.0 ** -40
    assert oracle.adjoint_floor_of(np.float64) == 2.0 ** -98
    assert np.sqrt(oracle.adjoint_floor_of(np.float32)) == 16 * (1.0 - float(np.nextafter(np.float32(1), 0)))
