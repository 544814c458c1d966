"""Reverse-mode differentiation of the evolution through the library's VJP
entry points (gh_rk4_step_vjp, gh_constraint_energy_vjp, gh_perturbation_vjp).

Argument marshalling and control flow only: every forward and reverse step
runs in libgh's CUDA kernels.

* ``RK4Step`` / ``ConstraintEnergy``: torch.autograd.Function wrappers, so a
  loss built from steps and constraint energies can call ``.backward()``.
* ``constraint_energy_gradient``: the time-integrated constraint energy
  E = sum_{n=1..N} dt * sum_shells norm2(u_n) of an N-step evolution and its
  gradient with respect to u_0, with checkpoints every ``ckpt`` steps: the
  forward pass keeps only every ckpt-th state; the reverse pass recomputes each
  segment's states from its checkpoint and runs the step VJPs backwards.
"""
import torch

from . import gh


class RK4Step(torch.autograd.Function):
    """u_{n+1} = gh_rk4_step(dom, dt, u_n) (with the domain's filters)."""

    @staticmethod
    def forward(ctx, u, dom, dt):
        out = u.detach().clone()
        gh.gh_rk4_step(dom, dt, out, dom.new_work())
        ctx.dom, ctx.dt = dom, dt
        ctx.save_for_backward(u.detach())
        return out

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        ub = torch.zeros_like(u)
        gh.gh_rk4_step_vjp(ctx.dom, ctx.dt, u, g.contiguous(), ub, gh.new_vjp_work(ctx.dom))
        return ub, None, None


class ConstraintEnergy(torch.autograd.Function):
    """Scalar sum over shells of the quadrature constraint norms of u."""

    @staticmethod
    def forward(ctx, u, dom):
        n2 = torch.zeros(len(dom.shells), dtype=torch.float64, device=u.device)
        gh.gh_constraints(dom, u.detach(), None, n2)
        ctx.dom = dom
        ctx.save_for_backward(u.detach())
        return n2.sum()

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        ub = torch.zeros_like(u)
        gh.gh_constraint_energy_vjp(ctx.dom, u, float(g), ub)
        return ub, None


def constraint_energy(dom, u):
    n2 = torch.zeros(len(dom.shells), dtype=torch.float64, device=u.device)
    gh.gh_constraints(dom, u, None, n2)
    return float(n2.sum())


def evolve_energy(dom, u0, dt, n_steps):
    """E = sum_{n=1..N} dt * sum_shells norm2(u_n) (forward only)."""
    u = u0.clone()
    work = dom.new_work()
    n2 = torch.zeros(len(dom.shells), dtype=torch.float64, device=u.device)
    acc = torch.zeros((), dtype=torch.float64, device=u.device)
    for _ in range(n_steps):
        gh.gh_rk4_step(dom, dt, u, work)
        gh.gh_constraints(dom, u, None, n2)
        acc += dt * n2.sum()
    return float(acc)


def constraint_energy_gradient(dom, u0, dt, n_steps, ckpt=20):
    """(E, dE/du_0) for E = sum_{n=1..N} dt C(u_n), u_n = S(u_{n-1}), with
    checkpoints every ckpt steps.

    Adjoint recursion: lam_N = dt grad C(u_N); lam_n = dt grad C(u_n) +
    S'(u_n)^T lam_{n+1}; dE/du_0 = S'(u_0)^T lam_1.  The reverse pass walks the
    segments (a, b] backwards, recomputing u_a..u_b from the checkpoint u_a.
    """
    work = dom.new_work()
    vwork = gh.new_vjp_work(dom)
    n2 = torch.zeros(len(dom.shells), dtype=torch.float64, device=u0.device)
    checkpoints = {0: u0.clone()}
    u = u0.clone()
    E = torch.zeros((), dtype=torch.float64, device=u0.device)
    for n in range(1, n_steps + 1):
        gh.gh_rk4_step(dom, dt, u, work)
        gh.gh_constraints(dom, u, None, n2)
        E += dt * n2.sum()
        if n % ckpt == 0 and n < n_steps:
            checkpoints[n] = u.clone()
    lam = torch.zeros_like(u0)
    nxt = torch.zeros_like(u0)
    for a in sorted(checkpoints, reverse=True):
        b = min(a + ckpt, n_steps)
        states = [checkpoints[a]]
        s = checkpoints[a].clone()
        for _ in range(a, b):
            gh.gh_rk4_step(dom, dt, s, work)
            states.append(s.clone())
        for n in range(b, a, -1):
            gh.gh_constraint_energy_vjp(dom, states[n - a], dt, lam)
            gh.gh_rk4_step_vjp(dom, dt, states[n - 1 - a], lam, nxt, vwork)
            lam, nxt = nxt, lam
    return float(E), lam
