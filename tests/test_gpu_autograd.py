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
    """d/dphi0 of <lam, phi_T> through 12 steps: adjoint (GPU) vs central FD of the oracle."""
    g, vel, npvel, h, eps, gamma, dt = setup()
    theta = torch.tensor([0.45, 0.5, 0.55, 0.2], dtype=torch.float64, device="cuda")
    phi0 = AG.sphere_phi(theta, g.shape, h, eps).contiguous()
    rng = np.random.default_rng(1)
    lam = dev(rng.standard_normal(g.shape))
    x = phi0.clone().requires_grad_(True)
    out = AG.rollout(x, *vel, g, 12, dt, eps, gamma, period=2.0, ckpt_every=5)
    (out * lam).sum().backward()
    grad = x.grad.cpu().numpy()
    d = rng.standard_normal(g.shape)
    p0 = phi0.cpu().numpy()
    hfd = 1e-6

    def J(p):
        return (oracle.run(p, *npvel, h, dt, eps, gamma, 12, period=2.0) * lam.cpu().numpy()).sum()
    fd = (J(p0 + hfd * d) - J(p0 - hfd * d)) / (2 * hfd)
    an = (grad * d).sum()
    assert abs(fd - an) <= 1e-6 * abs(fd)


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
    theta = torch.tensor([0.5, 0.4, 0.5, 0.25], dtype=torch.float64, device="cuda")
    phi0 = AG.sphere_phi(theta, g.shape, h, eps).contiguous()
    uu = [t.clone().requires_grad_(True) for t in vel]
    out = AG.rollout(phi0, *uu, g, 6, dt, eps, gamma, ckpt_every=4)
    w = torch.linspace(0, 1, out.numel(), dtype=torch.float64, device="cuda").reshape(out.shape)
    (out * w).sum().backward()
    rng = np.random.default_rng(3)
    p0 = phi0.cpu().numpy()
    for c in range(3):
        d = rng.standard_normal(g.shape)
        vp = [x.copy() for x in npvel]
        vm = [x.copy() for x in npvel]
        vp[c] += 1e-6 * d
        vm[c] -= 1e-6 * d
        wn = w.cpu().numpy()
        fd = ((oracle.run(p0, *vp, h, dt, eps, gamma, 6) - oracle.run(p0, *vm, h, dt, eps, gamma, 6)) * wn).sum() / 2e-6
        an = (uu[c].grad.cpu().numpy() * d).sum()
        assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-12


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
