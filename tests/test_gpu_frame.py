"""Parity of the rotating dual frame (Sec. 3.1 dual frame, Sec. 3.3
SpatialCoordJac) with the oracle through the C ABI: right-hand sides at a
given time and RK4 steps that advance the domain's clock, on a Schwarzschild
shell rotating about a tilted axis and on two Kerr shells rotating about the
spin axis; captured RK4 graphs that replay with the live clock; the reverse
mode in the moving frame against finite differences; a static frame after a
rotating one; the refusals."""
import numpy as np
import pytest
import torch

from oracle import dp5 as odp5
from oracle import frame
from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, assert_output_parity, flat, to_dev, to_host, oracle_domain, oracle_initial_state, gpu_domain

pytestmark = pytest.mark.gpu


def _gh():
    from paper_1804_09101_gb300 import gh
    return gh


def _schw():
    w = workloads.schwarzschild_single_shell()
    w.noise_amp = 1e-6
    return w, (0.3, -0.5, 0.8), 0.4


def _kerr2():
    w = workloads.Workload(name="kerr2_rot", shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0, chi=0.7,
                           radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=7, noise_amp=1e-6)
    return w, (0.0, 0.0, 1.0), 0.25


CASES = {"schw_tilted_axis": _schw, "kerr2_spin_axis": _kerr2}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w, axis, omega = CASES[request.param]()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    return w, axis, omega, odom, u0


def _dom(w, odom, axis, omega):
    gh = _gh()
    dom = gpu_domain(w, odom)
    gh.gh_set_rotating_frame(dom, axis, omega)
    return dom


def test_rhs_matches_oracle_at_a_given_time(case):
    gh = _gh()
    w, axis, omega, odom, u0 = case
    dom = _dom(w, odom, axis, omega)
    gh.gh_set_time(dom, 1.7)
    u = to_dev(flat(u0))
    k = dom.new_state()
    gh.gh_rhs(dom, u, k)
    ref = flat(frame.rhs(odom, u0, 1.7, axis, omega))
    scale = np.abs(flat(u0)).max()
    assert_output_parity(to_host(k), ref, scale, "rhs")
    # and it is not the static right-hand side
    from oracle import evolve
    assert np.abs(flat(evolve.rhs(odom, u0)) - ref).max() > 1e3 * REL_TOL * scale


def test_rk4_steps_match_oracle_and_advance_the_clock(case):
    gh = _gh()
    w, axis, omega, odom, u0 = case
    dom = _dom(w, odom, axis, omega)
    gh.gh_set_time(dom, 0.3)
    u = to_dev(flat(u0))
    work = dom.new_work()
    ou, t = u0, 0.3
    for _ in range(2):
        gh.gh_rk4_step(dom, w.dt, u, work)
        ou = frame.rk4_step(odom, ou, t, w.dt, axis, omega)
        t += w.dt
    assert abs(gh.gh_get_time(dom) - t) < 1e-15
    assert np.abs(to_host(u) - flat(ou)).max() <= REL_TOL * np.abs(flat(u0)).max()


def test_dormand_prince_attempt_uses_the_stage_times():
    gh = _gh()
    w, axis, omega = _schw()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    dom = _dom(w, odom, axis, omega)
    gh.gh_set_time(dom, 0.5)
    u = to_dev(flat(u0))
    dt = 0.02
    err, ok, _ = gh.gh_dp5_step(dom, dt, 1e-9, 1e-9, u, gh.new_dp5_work(dom))
    # oracle: the same tableau with f(u) evaluated at the stage times
    A, c, b, bh = odp5.tableau()
    k = []
    for s in range(7):
        us = u0 if s == 0 else [a + dt * sum(A[s][j] * k[j][i] for j in range(s)) for i, a in enumerate(u0)]
        k.append(frame.rhs(odom, us, 0.5 + c[s] * dt, axis, omega))
    unew = [a + dt * sum(b[j] * k[j][i] for j in range(7)) for i, a in enumerate(u0)]
    e = [dt * sum((b[j] - bh[j]) * k[j][i] for j in range(7)) for i in range(len(u0))]
    oerr = odp5.error_norm(u0, unew, e, 1e-9, 1e-9)
    assert abs(err - oerr) <= 1e-6 * max(oerr, 1e-3)
    assert ok == (oerr <= 1.0)
    if ok:
        assert np.abs(to_host(u) - flat(unew)).max() <= REL_TOL * np.abs(flat(u0)).max()
        assert abs(gh.gh_get_time(dom) - 0.52) < 1e-15


def test_static_again_and_refusals():
    gh = _gh()
    w, axis, omega = _schw()
    dom = gh.Domain.from_workload(w)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    k0, k1 = dom.new_state(), dom.new_state()
    gh.gh_rhs(dom, u, k0)
    gh.gh_set_rotating_frame(dom, axis, omega)
    gh.gh_set_time(dom, 2.0)
    with pytest.raises(RuntimeError):
        gh.gh_set_rotating_frame(dom, (0.0, 0.0, 0.0), 1.0)
    # one clock per domain: a hole with its own dt scale cannot rotate
    gh.gh_set_dt_scale(dom, 0, 0.5)
    with pytest.raises(RuntimeError):
        gh.gh_rk4_step(dom, w.dt, u.clone(), dom.new_work())
    with pytest.raises(RuntimeError):
        gh.gh_rhs_vjp(dom, u, u.clone(), torch.zeros_like(u))
    gh.gh_set_dt_scale(dom, 0, 1.0)
    gh.gh_set_rotating_frame(dom, axis, 0.0)
    gh.gh_rhs(dom, u, k1)
    torch.cuda.synchronize()
    assert torch.equal(k0, k1)


def test_captured_graph_replays_with_the_live_clock(case):
    """The stage frames come from the device clock, so a captured RK4 step
    replayed n times equals n direct steps bit for bit (each replay sees its
    own time) and advances the domain's clock by n dt; and both equal the
    oracle's moving-frame steps."""
    gh = _gh()
    w, axis, omega, odom, u0 = case
    dom = _dom(w, odom, axis, omega)
    gh.gh_set_time(dom, 0.1)
    a = to_dev(flat(u0))
    work = dom.new_work()
    for _ in range(3):
        gh.gh_rk4_step(dom, w.dt, a, work)
    gh.gh_set_time(dom, 0.1)
    b = to_dev(flat(u0))
    work2 = dom.new_work()
    gh.gh_rk4_graph_capture(dom, w.dt, b, work2)
    assert abs(gh.gh_get_time(dom) - 0.1) < 1e-15
    gh.gh_rk4_graph_launch(dom, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert abs(gh.gh_get_time(dom) - (0.1 + 3 * w.dt)) < 1e-15
    ou, t = u0, 0.1
    for _ in range(3):
        ou = frame.rk4_step(odom, ou, t, w.dt, axis, omega)
        t += w.dt
    assert np.abs(to_host(b) - flat(ou)).max() <= REL_TOL * np.abs(flat(u0)).max()
    # after the replays, a direct step continues from the advanced clock
    gh.gh_rk4_step(dom, w.dt, b, work2)
    ou = frame.rk4_step(odom, ou, t, w.dt, axis, omega)
    assert np.abs(to_host(b) - flat(ou)).max() <= REL_TOL * np.abs(flat(u0)).max()


def test_noalloc_rhs_and_constraints_follow_the_clock():
    """gh_rhs_noalloc takes its frame from the device clock like gh_rhs (bit for
    bit), and the constraint norm of the rotating exact solution stays at its
    truncation level at any time."""
    gh = _gh()
    w, axis, omega = _schw()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    dom = _dom(w, odom, axis, omega)
    u = to_dev(flat(u0))
    for t in (0.0, 0.9, 2.3):
        gh.gh_set_time(dom, t)
        k1, k2 = dom.new_state(), dom.new_state()
        gh.gh_rhs(dom, u, k1)
        gh.gh_rhs_noalloc(dom, u, k2)
        torch.cuda.synchronize()
        assert torch.equal(k1, k2), t
    gh.gh_set_time(dom, 0.0)
    n0 = torch.zeros(len(w.shells), dtype=torch.float64, device="cuda")
    gh.gh_constraints(dom, u, None, n0)
    ue = to_dev(flat(frame.exact_state(odom, 1.7, axis, omega)))
    gh.gh_set_time(dom, 1.7)
    n1 = torch.zeros(len(w.shells), dtype=torch.float64, device="cuda")
    gh.gh_constraints(dom, ue, None, n1)
    torch.cuda.synchronize()
    assert float(n1.sum()) <= 10 * float(n0.sum()) + 1e-20


def _fd_dot(gh, dom, fwd, u0, v, dw, h=1e-6):
    up, um = fwd(to_dev(u0 + h * dw)), fwd(to_dev(u0 - h * dw))
    return float(v @ ((up - um) / (2 * h)))


def test_reverse_mode_in_the_moving_frame(case):
    """<v, J w> by central differences equals <J^T v, w> for the RHS and the
    RK4 step at a nonzero time: the reverse passes use the rotated DiffJac,
    gauge and boundary background of each stage time and transpose the
    grid-velocity term."""
    gh = _gh()
    w, axis, omega, odom, u0 = case
    dom = _dom(w, odom, axis, omega)
    x = flat(u0)
    rng = np.random.default_rng(51)
    v = rng.standard_normal(x.shape)
    dw = rng.standard_normal(x.shape)

    def rhs(u):
        gh.gh_set_time(dom, 0.7)
        k = dom.new_state()
        gh.gh_rhs(dom, u, k)
        return to_host(k)

    def step(u):
        gh.gh_set_time(dom, 0.7)
        gh.gh_rk4_step(dom, w.dt, u, dom.new_work())
        return to_host(u)

    lhs = _fd_dot(gh, dom, rhs, x, v, dw)
    gh.gh_set_time(dom, 0.7)
    ub = dom.new_state()
    gh.gh_rhs_vjp(dom, to_dev(x), to_dev(v), ub)
    assert abs(lhs - float(to_host(ub) @ dw)) <= 1e-6 * abs(lhs)
    lhs = _fd_dot(gh, dom, step, x, v, dw)
    gh.gh_set_time(dom, 0.7)
    ub = dom.new_state()
    gh.gh_rk4_step_vjp(dom, w.dt, to_dev(x), to_dev(v), ub, gh.new_vjp_work(dom))
    assert abs(lhs - float(to_host(ub) @ dw)) <= 1e-6 * abs(lhs)
    # without the frame terms the identity fails
    gh.gh_set_rotating_frame(dom, axis, 0.0)
    ub0 = dom.new_state()
    gh.gh_rk4_step_vjp(dom, w.dt, to_dev(x), to_dev(v), ub0, gh.new_vjp_work(dom))
    assert abs(lhs - float(to_host(ub0) @ dw)) > 1e-3 * abs(lhs)


def test_checkpointed_energy_gradient_in_the_moving_frame():
    """The checkpointed gradient of the time-integrated constraint energy
    (the clock set for every saved, recomputed and reversed step) against a
    central difference of the forward evolution."""
    from paper_1804_09101_gb300.adjoint import constraint_energy_gradient, evolve_energy
    gh = _gh()
    w, axis, omega = _schw()
    odom = oracle_domain(w)
    u0 = to_dev(flat(oracle_initial_state(w, odom)))
    dom = _dom(w, odom, axis, omega)
    steps, dt = 7, 0.01
    gh.gh_set_time(dom, 0.4)
    E, lam = constraint_energy_gradient(dom, u0, dt, steps, ckpt=3)
    assert abs(gh.gh_get_time(dom) - (0.4 + steps * dt)) < 1e-14
    g = torch.Generator(device="cuda").manual_seed(52)
    dw = 1e-3 * torch.randn(dom.state_size, dtype=torch.float64, device="cuda", generator=g)
    h = 1e-4
    gh.gh_set_time(dom, 0.4)
    Ep = evolve_energy(dom, u0 + h * dw, dt, steps)
    gh.gh_set_time(dom, 0.4)
    Em = evolve_energy(dom, u0 - h * dw, dt, steps)
    fd = (Ep - Em) / (2 * h)
    an = float((lam * dw).sum())
    assert abs(fd - an) <= 1e-5 * abs(fd), (fd, an)
