"""Parity of the full constraint-preserving outer condition
(GH_BC_CONSTRAINT_PRESERVING_FULL: Bjorhus form for u^psi and u^0, and the
constraint part of u^- with its gauge and physical parts frozen; Sec. 5) with
the oracle's "cp_full" through the C ABI: right-hand sides and RK4 steps on
one- and two-shell domains with gamma1 = -1 and 0.5; the no-allocation RHS
and the captured RK4 graph agree with the plain calls; the static-grid
refusals; the reverse mode through the condition (nonlinear in u through the
inverse metric, the lapse and the 5x5 solve) against central differences of
the forward path."""
import numpy as np
import pytest
import torch

from oracle import evolve
from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, assert_output_parity, flat, to_dev, to_host, oracle_domain, oracle_initial_state, gpu_domain

pytestmark = pytest.mark.gpu


def _gh():
    from paper_1804_09101_gb300 import gh
    return gh


def _kerr2(gamma1=-1.0):
    return workloads.Workload(name="kerr2_g1_%g" % gamma1, shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0,
                              chi=0.9, gamma1=gamma1, radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=7,
                              noise_amp=1e-6,
                              pulse=workloads.Pulse("psi_pulse", 1e-3, 5.0, 0.7, 2, workloads.random_coeffs(7, 2)))


def _schw(gamma1=-1.0):
    w = workloads.schwarzschild_single_shell()
    w.gamma1 = gamma1
    w.noise_amp = 1e-4
    w.name = "schwarzschild_g1_%g" % gamma1
    return w


CASES = {"schw": _schw, "schw_g05": lambda: _schw(0.5), "kerr2": _kerr2, "kerr2_g05": lambda: _kerr2(0.5)}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w = CASES[request.param]()
    odom = oracle_domain(w)
    odom.outer_bc = "cp_full"
    u0 = oracle_initial_state(w, odom)
    return w, odom, u0


def _dom(w, odom):
    gh = _gh()
    dom = gpu_domain(w, odom)
    gh.gh_set_outer_bc(dom, gh.GH_BC_CONSTRAINT_PRESERVING_FULL)
    return dom


def test_rhs_matches_oracle(case):
    gh = _gh()
    w, odom, u0 = case
    dom = _dom(w, odom)
    u = to_dev(flat(u0))
    k = dom.new_state()
    gh.gh_rhs(dom, u, k)
    ref = flat(evolve.rhs(odom, u0))
    assert_output_parity(to_host(k), ref, np.abs(flat(u0)).max(), "rhs")
    # the u^- part changes the outer boundary's right-hand side
    odom.outer_bc = "cp"
    cp = flat(evolve.rhs(odom, u0))
    odom.outer_bc = "cp_full"
    assert np.abs(cp - ref).max() > 1e3 * REL_TOL * np.abs(ref).max()


def test_rk4_steps_match_oracle(case):
    gh = _gh()
    w, odom, u0 = case
    dom = _dom(w, odom)
    u = to_dev(flat(u0))
    work = dom.new_work()
    ou = u0
    for _ in range(2):
        gh.gh_rk4_step(dom, w.dt, u, work)
        ou = evolve.rk4_step(odom, ou, w.dt)
    assert np.abs(to_host(u) - flat(ou)).max() <= REL_TOL * np.abs(flat(u0)).max()


def test_noalloc_and_graph_agree_with_plain_calls():
    gh = _gh()
    w = _kerr2(0.5)
    dom = gh.Domain.from_workload(w)
    gh.gh_set_outer_bc(dom, gh.GH_BC_CONSTRAINT_PRESERVING_FULL)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    u += 1e-6 * torch.randn(dom.state_size, dtype=torch.float64, device=u.device)
    k1, k2 = dom.new_state(), dom.new_state()
    gh.gh_rhs(dom, u, k1)
    gh.gh_rhs_noalloc(dom, u, k2)
    torch.cuda.synchronize()
    assert torch.equal(k1, k2)
    a, b = u.clone(), u.clone()
    wa, wb = dom.new_work(), dom.new_work()
    for _ in range(3):
        gh.gh_rk4_step(dom, w.dt, a, wa)
    gh.gh_rk4_graph_capture(dom, w.dt, b, wb)
    gh.gh_rk4_graph_launch(dom, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_static_grid_refusals():
    gh = _gh()
    w = _schw()
    dom = gh.Domain.from_workload(w)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    gh.gh_set_outer_bc(dom, gh.GH_BC_CONSTRAINT_PRESERVING_FULL)
    with pytest.raises(gh.GHError) as e:
        gh.gh_set_rotating_frame(dom, (0.0, 0.0, 1.0), 0.2)
    assert e.value.status == gh.GH_ENOTSUP
    with pytest.raises(gh.GHError) as e:
        gh.gh_set_frame_map(dom, (0.0, 0.0, 1.0), 0.2, 0.0, (0.0, 0.0, 0.0))
    assert e.value.status == gh.GH_ENOTSUP
    # the other order: a moving grid first
    d2 = gh.Domain.from_workload(w)
    gh.gh_set_analytic_kerr_schild(d2, -1, w.M, w.chi, d2.new_state())
    gh.gh_set_rotating_frame(d2, (0.0, 0.0, 1.0), 0.2)
    with pytest.raises(gh.GHError) as e:
        gh.gh_set_outer_bc(d2, gh.GH_BC_CONSTRAINT_PRESERVING_FULL)
    assert e.value.status == gh.GH_ENOTSUP
    # and the domain still steps with the u^psi and u^0 conditions
    gh.gh_set_outer_bc(d2, gh.GH_BC_CONSTRAINT_PRESERVING)
    k = d2.new_state()
    gh.gh_rhs(d2, u, k)
    gh.gh_sync(d2)


@pytest.mark.parametrize("make", [_schw, lambda: _schw(0.5), _kerr2, lambda: _kerr2(0.5)])
def test_rhs_vjp_dot_product_against_finite_differences(make):
    """<v, J w> by central differences of gh_rhs equals <J^T v, w> from
    gh_rhs_vjp; restricted to the outer sphere's cotangent it differs from the
    transpose of the u^psi and u^0 condition alone."""
    gh = _gh()
    w = make()
    odom = oracle_domain(w)
    u0 = flat(oracle_initial_state(w, odom))
    dom = _dom(w, odom)
    rng = np.random.default_rng(25)
    v = rng.standard_normal(u0.shape)
    dw = rng.standard_normal(u0.shape)
    h = 1e-6
    kp, km = dom.new_state(), dom.new_state()
    gh.gh_rhs(dom, to_dev(u0 + h * dw), kp)
    gh.gh_rhs(dom, to_dev(u0 - h * dw), km)
    jw = (to_host(kp) - to_host(km)) / (2 * h)
    ub = dom.new_state()
    gh.gh_rhs_vjp(dom, to_dev(u0), to_dev(v), ub)
    lhs, rhs = float(v @ jw), float(to_host(ub) @ dw)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs), (lhs, rhs)
    # the outer sphere's cotangent alone: the same identity, and not mode 1's transpose
    vb = np.zeros_like(v)
    slab = 50 * 2 * (w.shells[-1][3] + 1) ** 2      # the last radial slice of the last shell
    vb[-slab:] = v[-slab:]
    ub_full = dom.new_state()
    gh.gh_rhs_vjp(dom, to_dev(u0), to_dev(vb), ub_full)
    lhs_b, rhs_b = float(vb @ jw), float(to_host(ub_full) @ dw)
    assert abs(lhs_b - rhs_b) <= 1e-6 * abs(lhs_b), (lhs_b, rhs_b)
    gh.gh_set_outer_bc(dom, gh.GH_BC_CONSTRAINT_PRESERVING)
    ub_cp = dom.new_state()
    gh.gh_rhs_vjp(dom, to_dev(u0), to_dev(vb), ub_cp)
    assert float((ub_full - ub_cp).abs().max()) > 1e-6 * float(ub_full.abs().max())


def test_rk4_step_vjp_dot_product():
    gh = _gh()
    w = _kerr2(0.5)
    odom = oracle_domain(w)
    u0 = flat(oracle_initial_state(w, odom))
    dom = _dom(w, odom)
    rng = np.random.default_rng(26)
    v = rng.standard_normal(u0.shape)
    dw = rng.standard_normal(u0.shape)
    h = 1e-6
    work = dom.new_work()
    up, um = to_dev(u0 + h * dw), to_dev(u0 - h * dw)
    gh.gh_rk4_step(dom, w.dt, up, work)
    gh.gh_rk4_step(dom, w.dt, um, work)
    jw = (to_host(up) - to_host(um)) / (2 * h)
    ub = dom.new_state()
    gh.gh_rk4_step_vjp(dom, w.dt, to_dev(u0), to_dev(v), ub, gh.new_vjp_work(dom))
    lhs, rhs = float(v @ jw), float(to_host(ub) @ dw)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs), (lhs, rhs)
