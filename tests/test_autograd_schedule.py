"""Host logic of the checkpoint-recompute rollout and the inverse problem, on the CPU.

A stand-in grid whose step is an elementwise nonlinear map (and whose adjoint
is that map's exact transpose) checks that the backward applies the adjoint
at the right recomputed state, in the right order, for every checkpoint and
sub-segment layout: the gradient must equal torch autograd through the same
map, and must not depend on the layout.
"""
import math

import pytest
import torch

from paper_1803_01262_gb300 import autograd as AG


class FakeGrid:
    """phi' = phi + dt vs (sin(phi) + u phi); its adjoint lam = lam' (1 + dt vs (cos(phi) + u)),
    and the velocity gradient it accumulates, d phi'/du = dt vs phi (v and w do not enter)."""

    def __init__(self):
        self.steps = 0
        self.adjoints = 0

    def set_velocity(self, u, v, w, umax=-1.0):
        self.u = u

    def step(self, a, b, dt, eps, gamma, vs=1.0):
        self.steps += 1
        b.copy_(a + dt * vs * (torch.sin(a) + self.u * a))

    def step_adjoint(self, phi, lam, out, dt, eps, gamma, vs=1.0, grads=None):
        self.adjoints += 1
        if grads is not None:
            grads[0].add_(lam * dt * vs * phi)
        out.copy_(lam * (1 + dt * vs * (torch.cos(phi) + self.u)))


def reference(phi0, u, nsteps, dt, period):
    p = phi0
    for i in range(nsteps):
        vs = math.cos(math.pi * i * dt / period) if period > 0 else 1.0
        p = p + dt * vs * (torch.sin(p) + u * p)
    return p


@pytest.mark.parametrize("nsteps,ckpt,inner", [(1, 16, None), (7, 16, None), (16, 16, None),
                                               (37, 16, None), (37, 16, 4), (37, 16, 5), (37, 16, 1),
                                               (50, 8, 3), (33, 32, 8), (200, 16, 16), (41, 1, None)])
@pytest.mark.parametrize("period", [0.0, 0.37])
def test_gradient_matches_autograd_for_every_layout(nsteps, ckpt, inner, period):
    g = torch.Generator().manual_seed(nsteps)
    phi0 = torch.rand(5, 4, 6, dtype=torch.float64, generator=g)
    u = torch.rand(5, 4, 6, dtype=torch.float64, generator=g) - 0.5
    w = torch.randn(5, 4, 6, dtype=torch.float64, generator=g)
    dt = 0.05
    x = phi0.clone().requires_grad_(True)
    (reference(x, u, nsteps, dt, period) * w).sum().backward()
    want = x.grad.clone()

    grid = FakeGrid()
    y = phi0.clone().requires_grad_(True)
    out = AG.rollout(y, u, u, u, grid, nsteps, dt, 1.0, 1.0, period=period, ckpt_every=ckpt,
                     inner_every=inner)
    assert torch.allclose(out, reference(phi0, u, nsteps, dt, period), rtol=0, atol=1e-14)
    fwd_steps = grid.steps
    (out * w).sum().backward()
    assert torch.allclose(y.grad, want, rtol=1e-13, atol=1e-14)
    assert grid.adjoints == nsteps
    # recompute count: each segment [s, e) reaches its last sub-start, then each sub-segment
    # recomputes its own states
    inn = min(inner or ckpt, ckpt)
    expect = 0
    for s in range(0, nsteps, ckpt):
        e = min(s + ckpt, nsteps)
        last = s + ((e - 1 - s) // inn) * inn
        expect += last - s + sum(min(ss + inn, e) - ss - 1 for ss in range(s, e, inn))
    assert grid.steps - fwd_steps == expect


@pytest.mark.parametrize("nsteps,ckpt,inner", [(1, 16, None), (37, 16, 5), (50, 8, 3)])
@pytest.mark.parametrize("period", [0.0, 0.37])
def test_velocity_gradient_matches_autograd(nsteps, ckpt, inner, period):
    """The velocity gradient summed over the recomputed states (each step with its own
    velocity scale) equals torch autograd through the same map; phi0's gradient too."""
    g = torch.Generator().manual_seed(100 + nsteps)
    phi0 = torch.rand(4, 5, 3, dtype=torch.float64, generator=g)
    u0 = torch.rand(4, 5, 3, dtype=torch.float64, generator=g) - 0.5
    v = torch.zeros_like(u0)
    w = torch.randn(4, 5, 3, dtype=torch.float64, generator=g)
    dt = 0.05
    x, ur = phi0.clone().requires_grad_(True), u0.clone().requires_grad_(True)
    (reference(x, ur, nsteps, dt, period) * w).sum().backward()

    y, uy = phi0.clone().requires_grad_(True), u0.clone().requires_grad_(True)
    out = AG.rollout(y, uy, v, v, FakeGrid(), nsteps, dt, 1.0, 1.0, period=period, ckpt_every=ckpt,
                     inner_every=inner)
    (out * w).sum().backward()
    assert torch.allclose(uy.grad, ur.grad, rtol=1e-13, atol=1e-14)
    assert torch.allclose(y.grad, x.grad, rtol=1e-13, atol=1e-14)


def test_rejects_bad_intervals():
    grid = FakeGrid()
    p = torch.zeros(2, 2, 2, dtype=torch.float64)
    with pytest.raises(ValueError):
        AG.rollout(p, p, p, p, grid, 3, 0.1, 1.0, 1.0, ckpt_every=0)
    with pytest.raises(ValueError):
        AG.rollout(p, p, p, p, grid, 3, 0.1, 1.0, 1.0, ckpt_every=4, inner_every=0)


def test_sphere_phi_matches_the_host_generator():
    """The differentiable torch sphere equals the numpy generator's tanh sphere (periodic
    minimum image) to rounding."""
    import numpy as np

    from paper_1803_01262_gb300 import inputs as I
    shape, h = (12, 10, 14), 1.0 / 14
    p = torch.tensor([0.45, 0.62, 0.05, 0.25], dtype=torch.float64)   # wraps in z
    a = AG.sphere_phi(p, shape, h, h).numpy()
    b = I.tanh_profile(I.sphere_distance(shape, h, (0.45, 0.62, 0.05), 0.25), h)
    assert np.abs(a - b).max() < 1e-14


def test_inverse_problem_loop_descends():
    """The inverse-problem loop (sphere -> rollout -> loss -> adjoint -> Adam) on the stand-in
    grid: the loss falls by two orders and the parameters approach the target's."""
    shape, h = (12, 12, 12), 1.0 / 12

    class Grid(FakeGrid):
        dx, Df, dtype = h, 3, torch.float64

    Grid.shape = shape
    g = Grid()
    u = torch.full(shape, 0.3, dtype=torch.float64)
    z = torch.zeros(shape, dtype=torch.float64)
    true = torch.tensor([0.5, 0.5, 0.5, 0.3], dtype=torch.float64)
    with torch.no_grad():
        target = AG.rollout(AG.sphere_phi(true, shape, h, h), u, z, z, g, 20, 0.02, h, 1.0)
    init = torch.tensor([0.47, 0.52, 0.5, 0.27], dtype=torch.float64)
    theta, losses = AG.inverse_problem(target, u, z, z, g, 20, 0.02, h, 1.0, init, iters=40, lr=5e-3,
                                       ckpt_every=8)
    assert losses[-1] < 0.02 * losses[0]
    assert float((theta - true).abs().max()) < 0.5 * float((init - true).abs().max())
