"""Reverse-mode differentiation of the evolution through the library's VJP
entry points (gh_rk4_step_vjp, gh_constraint_energy_vjp, gh_perturbation_vjp).

Argument marshalling and control flow only: every forward and reverse step
runs in libgh's CUDA kernels.

* ``RK4Step`` (alias ``GHStep``) / ``ConstraintEnergy``: torch.autograd.Function
  wrappers, so a loss built from steps and constraint energies can call
  ``.backward()``.
* ``evolve``: N steps as one differentiable call with checkpoints every
  ``ckpt`` steps (the backward pass recomputes each segment from its
  checkpoint and runs the step VJPs backwards).
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


GHStep = RK4Step


class Evolve(torch.autograd.Function):
    """u_N after n_steps gh_rk4_step calls from u_0 (with the domain's filters).

    Forward keeps u_0, u_ckpt, u_2ckpt, ...; backward walks the segments
    (a, b] from the last, recomputes the segment's states and RK4 stage states
    from its checkpoint (gh_rk4_step_save) and applies the saved-stage step
    VJPs from step b down to a + 1: ubar_{n-1} = S'(u_{n-1})^T ubar_n.  With a
    rotating frame each recomputed or reversed step runs with the clock at
    t_0 + n dt, and backward leaves the clock where it found it.
    """

    @staticmethod
    def forward(ctx, u0, dom, dt, n_steps, ckpt):
        rot = getattr(dom, "rotating", False)
        ctx.t0 = gh.gh_get_time(dom) if rot else 0.0
        u = u0.detach().clone()
        work = dom.new_work()
        ctx.checkpoints = {0: u.clone()}
        for n in range(1, n_steps + 1):
            gh.gh_rk4_step(dom, dt, u, work)
            if n % ckpt == 0 and n < n_steps:
                ctx.checkpoints[n] = u.clone()
        ctx.dom, ctx.dt, ctx.n_steps, ctx.ckpt, ctx.rot = dom, dt, n_steps, ckpt, rot
        return u

    @staticmethod
    def backward(ctx, g):
        dom, dt, n_steps, ckpt, rot = ctx.dom, ctx.dt, ctx.n_steps, ctx.ckpt, ctx.rot
        t_end = gh.gh_get_time(dom) if rot else 0.0

        def clock(n):
            if rot:
                gh.gh_set_time(dom, ctx.t0 + n * dt)

        work = dom.new_work()
        vwork = gh.new_vjp_work(dom)
        N = dom.state_size
        lam = g.detach().contiguous().clone()
        nxt = torch.zeros_like(lam)
        for a in sorted(ctx.checkpoints, reverse=True):
            b = min(a + ckpt, n_steps)
            states = [ctx.checkpoints[a]]
            stages = torch.empty((b - a, 3 * N), dtype=torch.float64, device=lam.device)
            s = ctx.checkpoints[a].clone()
            for i in range(a, b):
                clock(i)
                gh.gh_rk4_step_save(dom, dt, s, work, stages[i - a])
                states.append(s.clone())
            for n in range(b, a, -1):
                clock(n - 1)
                gh.gh_rk4_step_vjp_saved(dom, dt, states[n - 1 - a], stages[n - 1 - a], lam, nxt, vwork, 0.0)
                lam, nxt = nxt, lam
        if rot:
            gh.gh_set_time(dom, t_end)
        ctx.checkpoints = None
        return lam, None, None, None, None


def evolve(dom, u0, dt, n_steps, ckpt=20):
    """u_N = S^N(u_0), differentiable with respect to u_0 (checkpointed; see Evolve)."""
    if n_steps < 1 or ckpt < 1:
        raise ValueError("need n_steps >= 1 and ckpt >= 1")
    return Evolve.apply(u0, dom, dt, n_steps, ckpt)


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
    """E = sum_{n=1..N} dt * sum_shells norm2(u_n) (forward only).  The norm of
    u_n (n < N) comes out of the first stage of step n+1 (gh_rk4_step's
    norm2_pre); u_N takes one gh_constraints call."""
    u = u0.clone()
    work = dom.new_work()
    ns = len(dom.shells)
    norms = torch.zeros((n_steps + 1, ns), dtype=torch.float64, device=u.device)
    for n in range(n_steps):
        gh.gh_rk4_step(dom, dt, u, work, norms[n])          # norms[n] = C(u_n)
    gh.gh_constraints(dom, u, None, norms[n_steps])
    return float(dt * norms[1:].sum())


def constraint_energy_gradient(dom, u0, dt, n_steps, ckpt=20):
    """(E, dE/du_0) for E = sum_{n=1..N} dt C(u_n), u_n = S(u_{n-1}), with
    checkpoints every ckpt steps.

    Adjoint recursion: lam_N = dt grad C(u_N); lam_n = dt grad C(u_n) +
    S'(u_n)^T lam_{n+1}; dE/du_0 = S'(u_0)^T lam_1.  The forward pass keeps the
    checkpoints u_0, u_ckpt, ... and, for the last segment, every state and its
    RK4 stage states; the reverse pass walks the segments (a, b] backwards,
    recomputing the other segments' states and stages from their checkpoints.

    With a rotating frame every evaluation runs at the domain clock, so the
    clock is set to t_0 + n dt before each step that is saved, recomputed or
    reversed (gh_rk4_step_save leaves it alone); on return it reads t_0 + N dt.
    """
    rot = getattr(dom, "rotating", False)
    t0 = gh.gh_get_time(dom) if rot else 0.0

    def clock(n):
        if rot:
            gh.gh_set_time(dom, t0 + n * dt)

    work = dom.new_work()
    vwork = gh.new_vjp_work(dom)
    N = dom.state_size
    ns = len(dom.shells)
    norms = torch.zeros((n_steps + 1, ns), dtype=torch.float64, device=u0.device)
    last = ((n_steps - 1) // ckpt) * ckpt          # start of the last segment
    checkpoints = {0: u0.clone()}
    u = u0.clone()
    saved_states, saved_stages = None, None
    for n in range(1, n_steps + 1):
        if n - 1 == last:
            saved_states = [u.clone()]
            saved_stages = torch.empty((n_steps - last, 3 * N), dtype=torch.float64, device=u0.device)
        if n - 1 >= last:
            clock(n - 1)
            gh.gh_rk4_step_save(dom, dt, u, work, saved_stages[n - 1 - last], norms[n - 1])
            saved_states.append(u.clone())
        else:
            gh.gh_rk4_step(dom, dt, u, work, norms[n - 1])
        if n % ckpt == 0 and n < n_steps:
            checkpoints[n] = u.clone()
    clock(n_steps)
    gh.gh_constraints(dom, u, None, norms[n_steps])
    E = float(dt * norms[1:].sum())
    lam = torch.zeros_like(u0)
    nxt = torch.zeros_like(u0)
    for a in sorted(checkpoints, reverse=True):
        b = min(a + ckpt, n_steps)
        if a == last:
            states, stages = saved_states, saved_stages
        else:
            states = [checkpoints[a]]
            stages = torch.empty((b - a, 3 * N), dtype=torch.float64, device=u0.device)
            s = checkpoints[a].clone()
            for i in range(a, b):
                clock(i)
                gh.gh_rk4_step_save(dom, dt, s, work, stages[i - a])
                states.append(s.clone())
        if b == n_steps:
            clock(n_steps)
            gh.gh_constraint_energy_vjp(dom, states[b - a], dt, lam)      # lam_N = dt grad C(u_N)
        for n in range(b, a, -1):
            # lam_{n-1} = S'(u_{n-1})^T lam_n + dt grad C(u_{n-1}) (no C term for u_0)
            cw = dt if n - 1 >= 1 else 0.0
            clock(n - 1)
            gh.gh_rk4_step_vjp_saved(dom, dt, states[n - 1 - a], stages[n - 1 - a], lam, nxt, vwork, cw)
            lam, nxt = nxt, lam
    clock(n_steps)
    return E, lam
