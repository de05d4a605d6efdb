"""Differentiable CDI rollouts: torch.autograd over the hand-written adjoint kernel.

``rollout(phi0, grid, nsteps, dt, eps, gamma, ...)`` advances phi0 by nsteps
explicit CDI steps (``cdi_step``) and, on backward, applies the discrete
adjoint step (``cdi_step_adjoint``) in reverse with recompute from
checkpoints: the forward keeps phi every ``ckpt_every`` steps; the backward
recomputes one segment at a time (ckpt_every - 1 extra forward steps per
segment) and walks it backwards.  With ``inner_every`` < ``ckpt_every`` a
segment is itself recomputed in sub-segments of ``inner_every`` steps: one
pass over the segment keeps only the sub-segment starts, then each
sub-segment (last first) is recomputed in full and walked backwards, so the
backward holds ckpt_every / inner_every + inner_every states instead of
ckpt_every (at 1024^3 FP32, 32 steps per checkpoint: 48 GB instead of
124 GB) for about ckpt_every more forward steps per segment.  If the face
velocities require grad, their gradients are accumulated by the adjoint
kernel on the same pass.

The velocity of step i is vel_scale_i * (u, v, w) with
vel_scale_i = cos(pi t_i / period) (1 when period <= 0), t_i = t0 + i dt.
"""
from __future__ import annotations

import math

import torch

from .cdi import Grid


def _scale(i, t0, dt, period):
    return math.cos(math.pi * (t0 + i * dt) / period) if period > 0 else 1.0


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, u, v, w, grid, nsteps, dt, eps, gamma, period, t0, ckpt_every, inner_every):
        grid.set_velocity(u, v, w, umax=0.0)
        ckpts = {0: phi0.detach().clone()}
        a = phi0.detach().clone()
        b = torch.empty_like(a)
        for i in range(nsteps):
            grid.step(a, b, dt, eps, gamma, _scale(i, t0, dt, period))
            a, b = b, a
            if (i + 1) % ckpt_every == 0 and i + 1 < nsteps:
                ckpts[i + 1] = a.clone()
        ctx.grid = grid
        ctx.args = (nsteps, dt, eps, gamma, period, t0, ckpt_every, inner_every)
        ctx.ckpts = ckpts
        ctx.save_for_backward(u, v, w)
        return a

    @staticmethod
    def backward(ctx, grad_out):
        u, v, w = ctx.saved_tensors
        grid = ctx.grid
        nsteps, dt, eps, gamma, period, t0, k, inner = ctx.args
        grid.set_velocity(u, v, w, umax=0.0)
        want_vel = any(ctx.needs_input_grad[1:4])
        grads = [torch.zeros_like(u), torch.zeros_like(v), torch.zeros_like(w)] if want_vel else None
        lam = grad_out.contiguous().clone()
        lam_b = torch.empty_like(lam)

        def fwd(p, i):
            nxt = torch.empty_like(p)
            grid.step(p, nxt, dt, eps, gamma, _scale(i, t0, dt, period))
            return nxt

        for s in reversed(sorted(ctx.ckpts)):
            e = min(s + k, nsteps)
            # sub-segment starts s, s + inner, ... (< e), recomputed from the checkpoint
            subs = {s: ctx.ckpts[s]}
            p = ctx.ckpts[s]
            last = s + ((e - 1 - s) // inner) * inner
            for i in range(s, last):
                p = fwd(p, i)
                if (i + 1 - s) % inner == 0:
                    subs[i + 1] = p
            del p
            for ss in reversed(sorted(subs)):
                ee = min(ss + inner, e)
                states = [subs.pop(ss)]     # states ss .. ee-1
                for i in range(ss, ee - 1):
                    states.append(fwd(states[-1], i))
                for i in range(ee - 1, ss - 1, -1):
                    grid.step_adjoint(states[i - ss], lam, lam_b, dt, eps, gamma,
                                      _scale(i, t0, dt, period), grads=grads)
                    lam, lam_b = lam_b, lam
                del states
        ctx.ckpts = None
        gu = gv = gw = None
        if want_vel:
            gu, gv, gw = grads
        return lam, gu, gv, gw, None, None, None, None, None, None, None, None, None


def rollout(phi0, u, v, w, grid: Grid, nsteps, dt, eps, gamma, period=0.0, t0=0.0, ckpt_every=16,
            inner_every=None):
    """Differentiable nsteps-step CDI rollout (see module docstring)."""
    if ckpt_every < 1:
        raise ValueError("ckpt_every must be >= 1")
    inner = ckpt_every if inner_every is None else int(inner_every)
    if inner < 1:
        raise ValueError("inner_every must be >= 1")
    return _Rollout.apply(phi0, u, v, w, grid, int(nsteps), float(dt), float(eps), float(gamma),
                          float(period), float(t0), int(ckpt_every), min(inner, int(ckpt_every)))


def sphere_phi(params, shape, h, eps):
    """Differentiable tanh sphere 0.5(1 + tanh((R - |x - c|)/(2 eps))) on the grid.

    params = (cx, cy, cz, R) as a torch tensor; periodic minimum image in a box
    of edge lengths N_d h.  Used by the inverse problem (input side, in torch).
    """
    nz, ny, nx = shape
    dev, dt = params.device, params.dtype
    r2 = 0
    for n, c, ax in ((nx, params[0], 2), (ny, params[1], 1), (nz, params[2], 0)):
        x = (torch.arange(n, device=dev, dtype=dt) + 0.5) * h
        L = n * h
        d = x - c
        d = d - L * torch.round(d / L)
        sh = [1, 1, 1]
        sh[ax] = n
        r2 = r2 + (d * d).reshape(sh)
    s = params[3] - torch.sqrt(r2)
    return 0.5 * (1.0 + torch.tanh(s / (2.0 * eps)))


def inverse_problem(target, u, v, w, grid: Grid, nsteps, dt, eps, gamma, init, iters=30, lr=5e-3,
                    ckpt_every=16, period=0.0):
    """Recover sphere parameters (cx, cy, cz, R) whose rollout matches ``target``.

    Plain Adam on L = sum (phi_T(theta) - target)^2 dV; gradients flow through
    the adjoint kernel (phi) and torch (sphere_phi).  Returns (params, losses).
    """
    theta = init.detach().clone().to(torch.float64).requires_grad_(True)
    opt = torch.optim.Adam([theta], lr=lr)
    dV = grid.dx ** grid.Df
    losses = []
    for _ in range(iters):
        opt.zero_grad()
        phi0 = sphere_phi(theta, grid.shape, grid.dx, eps).to(grid.dtype).contiguous()
        out = rollout(phi0, u, v, w, grid, nsteps, dt, eps, gamma, period, 0.0, ckpt_every)
        loss = ((out.double() - target.double()) ** 2).sum() * dV
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    return theta.detach(), losses
