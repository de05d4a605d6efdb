"""Checkpoint-recompute autograd over the adjoint kernel; inverse problem."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1803_01262_gb300 import autograd as AG
from paper_1803_01262_gb300 import cdi
from paper_1803_01262_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def fd_richardson(f, h):
    """Central difference extrapolated over h and h/2 (error O(h^4)).

    The plain central difference of these rollouts converges as h^2 (about
    3e-6 relative at h = 1e-6), so the 1e-6 check needs the extrapolation.
    """
    d1 = (f(h) - f(-h)) / (2 * h)
    d2 = (f(h / 2) - f(-h / 2)) / h
    return (4 * d2 - d1) / 3


def setup(n=32, dtype=torch.float64, seed=5):
    shape = (n, n, n)
    h = 1.0 / n
    u, v, w = I.random_velocity(shape, h, 16, 3, seed)
    eps, gamma = h, 1.0
    dt = 0.1 * h
    g = cdi.Grid(n, n, n, h, dtype)
    vel = [dev(x, dtype) for x in (u, v, w)]
    return g, vel, (u, v, w), h, eps, gamma, dt


def test_rollout_grad_vs_oracle_fd():
    """d/dphi0 of <lam, phi_T> through 12 steps: adjoint (GPU) vs central FD of the oracle.

    phi0 is a smooth field in [0.1, 0.9]: where |grad phi| is tiny (the flat
    far field of a tanh profile) n = g/|g| is not linear on the scale of a
    finite-difference step, so FD in phi0 is not a valid reference there.
    """
    g, vel, npvel, h, eps, gamma, dt = setup()
    p0 = 0.1 + 0.8 * I.random_phi(g.shape, 2, smooth=True)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(g.shape)
    x = dev(p0).requires_grad_(True)
    out = AG.rollout(x, *vel, g, 12, dt, eps, gamma, period=2.0, ckpt_every=5)
    (out * dev(lam)).sum().backward()
    d = rng.standard_normal(g.shape)

    def J(t):
        return (oracle.run(p0 + t * d, *npvel, h, dt, eps, gamma, 12, period=2.0) * lam).sum()
    fd = fd_richardson(J, 1e-6)
    an = (x.grad.cpu().numpy() * d).sum()
    assert abs(fd - an) <= 1e-6 * abs(fd)


def test_sphere_parameter_grad_vs_oracle_fd():
    """d/dtheta of <lam, phi_T(theta)> for the inverse problem's (centre, radius).

    The perturbation of phi0 induced by theta scales with phi itself, so the
    finite differences stay in the linear regime on the tanh profile.
    """
    g, vel, npvel, h, eps, gamma, dt = setup()
    theta0 = np.array([0.45, 0.5, 0.55, 0.2])
    lam = np.random.default_rng(4).standard_normal(g.shape)
    th = torch.tensor(theta0, dtype=torch.float64, device="cuda", requires_grad=True)
    out = AG.rollout(AG.sphere_phi(th, g.shape, h, eps).contiguous(), *vel, g, 10, dt, eps, gamma,
                     ckpt_every=4)
    (out * dev(lam)).sum().backward()
    an = th.grad.cpu().numpy()

    def J(t):
        p = I.tanh_profile(I.sphere_distance(g.shape, h, tuple(t[:3]), t[3]), eps)
        return (oracle.run(p, *npvel, h, dt, eps, gamma, 10) * lam).sum()
    for i in range(4):
        e = np.zeros(4)
        e[i] = 1.0
        fd = fd_richardson(lambda t: J(theta0 + t * e), 1e-6)
        assert abs(fd - an[i]) <= 1e-6 * abs(fd), (i, fd, an[i])


@pytest.mark.parametrize("k", [1, 3, 7, 20])
def test_checkpoint_interval_invariance(k):
    g, vel, _, h, eps, gamma, dt = setup(n=24)
    theta = torch.tensor([0.5, 0.5, 0.5, 0.25], dtype=torch.float64, device="cuda")
    phi0 = AG.sphere_phi(theta, g.shape, h, eps).contiguous()
    lam = torch.randn(g.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    grads = []
    for kk in (k, 20):
        x = phi0.clone().requires_grad_(True)
        out = AG.rollout(x, *vel, g, 20, dt, eps, gamma, ckpt_every=kk)
        (out * lam).sum().backward()
        grads.append(x.grad)
    assert torch.equal(grads[0], grads[1])


def test_velocity_gradient_vs_fd():
    g, vel, npvel, h, eps, gamma, dt = setup(n=16)
    p0 = 0.1 + 0.8 * I.random_phi(g.shape, 6, smooth=True)
    uu = [t.clone().requires_grad_(True) for t in vel]
    out = AG.rollout(dev(p0), *uu, g, 6, dt, eps, gamma, ckpt_every=4)
    rng = np.random.default_rng(3)
    lam = rng.standard_normal(g.shape)
    (out * dev(lam)).sum().backward()
    for c in range(3):
        d = rng.standard_normal(g.shape)

        def J(t):
            vv = [x.copy() for x in npvel]
            vv[c] += t * d
            return (oracle.run(p0, *vv, h, dt, eps, gamma, 6) * lam).sum()
        fd = fd_richardson(J, 1e-6)
        an = (uu[c].grad.cpu().numpy() * d).sum()
        assert abs(fd - an) <= 1e-6 * abs(fd), (c, fd, an)


def test_inverse_problem_recovers_sphere():
    """Gradient descent on (centre, radius) through 40 steps of the FP32 rollout."""
    n = 32
    g, vel, _, h, eps, gamma, dt = setup(n=n, dtype=torch.float32, seed=8)
    true = torch.tensor([0.52, 0.47, 0.5, 0.22], dtype=torch.float64, device="cuda")
    target = AG.rollout(AG.sphere_phi(true, g.shape, h, eps).float().contiguous(), *vel, g, 40, dt, eps,
                        gamma, ckpt_every=16).detach()
    init = torch.tensor([0.47, 0.51, 0.46, 0.18], dtype=torch.float64, device="cuda")
    theta, losses = AG.inverse_problem(target, *vel, g, 40, dt, eps, gamma, init, iters=60, lr=4e-3)
    assert losses[-1] < 0.05 * losses[0]
    assert (theta - true).abs().max().item() < 0.5 * (init - true).abs().max().item()


@pytest.mark.parametrize("n", [128, 512])
def test_long_fp32_rollout_gradient(n):
    """The inverse problem's configuration (512^3; 128^3 as the small case): 200 FP32 steps,
    checkpoint every 16, 32-mode random velocity.  dL/dtheta of the sphere parameters from
    the adjoint matches central differences of the FP32 rollout.  The far tails of phi reach
    |g|^2 ~ FLT_MIN here; an adjoint of the unit normal instead of the step's regularised
    normal grows there without bound over the 200 steps."""
    h = 1.0 / n
    vel = [x.to(torch.float32).contiguous() for x in I.random_velocity_torch((n, n, n), h, 32, 4, 7)]
    g = cdi.Grid(n, n, n, h, torch.float32)
    g.set_velocity(*vel)
    eps, gamma, dt = h, g.U, 0.1 * h / g.U
    true = torch.tensor([0.5, 0.5, 0.5, 0.2], dtype=torch.float64, device="cuda")
    init = torch.tensor([0.52, 0.485, 0.51, 0.18], dtype=torch.float64, device="cuda")

    def roll(th):
        return AG.rollout(AG.sphere_phi(th, g.shape, h, eps).float().contiguous(), *vel, g, 200, dt, eps,
                          gamma, ckpt_every=16)
    with torch.no_grad():
        target = roll(true)

    def loss(th):
        return ((roll(th).double() - target.double()) ** 2).sum() * h ** 3
    th = init.clone().requires_grad_(True)
    loss(th).backward()
    grad = th.grad.cpu().numpy()
    fd = np.empty(4)
    with torch.no_grad():
        for c in range(4):
            e = torch.zeros(4, dtype=torch.float64, device="cuda")
            e[c] = 2e-3
            fd[c] = (float(loss(init + e)) - float(loss(init - e))) / 4e-3
    assert np.all(np.isfinite(grad))
    assert np.abs(grad - fd).max() <= 0.02 * np.abs(fd).max(), (grad, fd)
    assert abs(grad[3] - fd[3]) <= 0.01 * abs(fd[3]), (grad, fd)
