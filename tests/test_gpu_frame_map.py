"""The general dual-frame map on the GPU (gh_set_frame_map: expansion,
rotation about any axis, translation; Sec. 3.1 dual frame, Sec. 3.3
SpatialCoordJac) against the oracle's moving-frame right-hand side and RK4
steps, with the hole's gauge source and boundary background evaluated at the
moving points by both sides (the oracle from its sympy Kerr-Schild metric, the
library from its device jets).  Bars: output parity for the RHS, 1e-11 of
max|u| for states."""
import numpy as np
import pytest
import torch

from oracle import frame
from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, assert_output_parity, flat, to_dev, to_host, oracle_domain, oracle_initial_state

pytestmark = pytest.mark.gpu


def _gh():
    from paper_1804_09101_gb300 import gh
    return gh


def _schw():
    w = workloads.schwarzschild_single_shell()
    w.noise_amp = 1e-6
    return w, dict(axis=(0.3, -0.5, 0.8), omega=0.3, adot=0.05, V=(0.02, -0.03, 0.04))


def _kerr2():
    # a Kerr hole (spin along z) under a rotation about a tilted axis: not
    # symmetric under the map, so the gauge source must be re-evaluated
    w = workloads.Workload(name="kerr2_map", shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0, chi=0.7,
                           radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=7, noise_amp=1e-6)
    return w, dict(axis=(0.6, 0.0, 0.8), omega=0.25, adot=-0.03, V=(-0.04, 0.05, 0.0))


CASES = {"schw_expand_translate_tilted": _schw, "kerr2_contract_translate_tilted": _kerr2}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w, m = CASES[request.param]()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    return w, m, odom, u0


def _dom(w, m):
    gh = _gh()
    dom = gh.Domain.from_workload(w)
    scratch = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, scratch)   # the hole the map evaluates
    gh.gh_set_frame_map(dom, m["axis"], m["omega"], m["adot"], m["V"])
    return dom


def test_map_rhs_matches_oracle_at_a_given_time(case):
    gh = _gh()
    w, m, odom, u0 = case
    dom = _dom(w, m)
    gh.gh_set_time(dom, 1.7)
    u = to_dev(flat(u0))
    k = dom.new_state()
    gh.gh_rhs(dom, u, k)
    ref = flat(frame.rhs_map(odom, u0, 1.7, frame.AffineMap(**m)))
    scale = np.abs(flat(u0)).max()
    assert_output_parity(to_host(k), ref, scale, "rhs")
    # and it is not the rotating frame's right-hand side
    rot = flat(frame.rhs(odom, u0, 1.7, m["axis"], m["omega"]))
    assert np.abs(rot - ref).max() > 1e3 * REL_TOL * scale


def test_map_rk4_steps_match_oracle_and_advance_the_clock(case):
    gh = _gh()
    w, m, odom, u0 = case
    dom = _dom(w, m)
    gh.gh_set_time(dom, 0.3)
    u = to_dev(flat(u0))
    work = dom.new_work()
    mp = frame.AffineMap(**m)
    ou, t = u0, 0.3
    for _ in range(2):
        gh.gh_rk4_step(dom, w.dt, u, work)
        ou = frame.rk4_step_map(odom, ou, t, w.dt, mp)
        t += w.dt
    assert abs(gh.gh_get_time(dom) - t) < 1e-15
    assert np.abs(to_host(u) - flat(ou)).max() <= REL_TOL * np.abs(flat(u0)).max()


def test_map_graph_replays_equal_direct_steps(case):
    gh = _gh()
    w, m, odom, u0 = case
    dom = _dom(w, m)
    gh.gh_set_time(dom, 0.1)
    a = to_dev(flat(u0))
    wa = dom.new_work()
    for _ in range(3):
        gh.gh_rk4_step(dom, w.dt, a, wa)
    gh.gh_set_time(dom, 0.1)
    b = to_dev(flat(u0))
    wb = dom.new_work()
    gh.gh_rk4_graph_capture(dom, w.dt, b, wb)
    gh.gh_rk4_graph_launch(dom, 3)
    gh.gh_sync(dom)
    assert torch.equal(a, b)
    assert abs(gh.gh_get_time(dom) - (0.1 + 3 * w.dt)) < 1e-14


def test_map_rotation_alone_is_the_rotating_frame():
    """A Kerr hole rotated about its spin axis: the general map (the hole
    evaluated at the rotated points) and the rotating frame (the stored gauge
    source rotated) agree to rounding."""
    gh = _gh()
    w = workloads.Workload(name="kerr2_rot", shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0, chi=0.7,
                           radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=7, noise_amp=1e-6)
    odom = oracle_domain(w)
    u0 = to_dev(flat(oracle_initial_state(w, odom)))
    d1 = _dom(w, dict(axis=(0.0, 0.0, 1.0), omega=0.25, adot=0.0, V=(0.0, 0.0, 0.0)))
    d2 = gh.Domain.from_workload(w)
    gh.gh_set_analytic_kerr_schild(d2, -1, w.M, w.chi, d2.new_state())
    gh.gh_set_rotating_frame(d2, (0.0, 0.0, 1.0), 0.25)
    out = []
    for d in (d1, d2):
        gh.gh_set_time(d, 1.3)
        k = d.new_state()
        gh.gh_rhs(d, u0, k)
        out.append(to_host(k))
    assert np.abs(out[0] - out[1]).max() <= 1e-11 * np.abs(to_host(u0)).max()


def test_map_refusals():
    gh = _gh()
    w, m = _schw()
    dom = gh.Domain.from_workload(w)
    with pytest.raises(RuntimeError):           # no hole set: nothing to evaluate at the moving points
        gh.gh_set_frame_map(dom, m["axis"], m["omega"], m["adot"], m["V"])
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    with pytest.raises(RuntimeError):
        gh.gh_set_frame_map(dom, (0.0, 0.0, 0.0), 0.1, 0.0, (0.0, 0.0, 0.0))
    gh.gh_set_frame_map(dom, m["axis"], m["omega"], m["adot"], m["V"])
    with pytest.raises(gh.GHError) as e:
        gh.gh_rhs_vjp(dom, u, u.clone(), torch.zeros_like(u))
    assert e.value.status == gh.GH_ENOTSUP


def _kerr_tilted():
    return workloads.Workload(name="kerr2_tilted", shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0, chi=0.7,
                              radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=7, noise_amp=1e-6)


def test_map_identity_is_the_static_frame():
    """With no rotation, expansion or translation the map's gauge source (the
    Kerr-Schild closed form H_a = -2 d_i (H l_a l_i), evaluated every stage)
    and boundary data equal the stored ones (from the Christoffel symbols of
    the full metric) to rounding: a tilted spin, so no component vanishes."""
    gh = _gh()
    w = _kerr_tilted()
    spin = (0.7 * 0.6, 0.0, 0.7 * 0.8)
    odom = oracle_domain(w)
    u0 = to_dev(flat(oracle_initial_state(w, odom)))
    out = []
    for use_map in (True, False):
        d = gh.Domain.from_workload(w)
        gh.gh_set_analytic_kerr_schild(d, -1, w.M, spin, d.new_state())
        if use_map:
            gh.gh_set_frame_map(d, (0.0, 0.0, 1.0), 0.0, 0.0, (0.0, 0.0, 0.0))
        gh.gh_set_time(d, 0.9)
        k = d.new_state()
        gh.gh_rhs(d, u0, k)
        out.append(to_host(k))
    assert np.abs(out[0] - out[1]).max() <= 1e-12 * np.abs(out[1]).max()


def test_map_reevaluates_when_the_time_or_the_hole_changes():
    """The moving-point buffers are reused only at the frame they were
    evaluated at: going back to an earlier time reproduces it bit for bit, and
    a new hole mass gives the right-hand side of a domain made with it."""
    gh = _gh()
    w = _kerr_tilted()
    m = dict(axis=(0.6, 0.0, 0.8), omega=0.25, adot=-0.03, V=(-0.04, 0.05, 0.0))
    odom = oracle_domain(w)
    u0 = to_dev(flat(oracle_initial_state(w, odom)))
    dom = _dom(w, m)

    def rhs(d, t):
        gh.gh_set_time(d, t)
        k = d.new_state()
        gh.gh_rhs(d, u0, k)
        gh.gh_sync(d)
        return k

    k1 = rhs(dom, 1.7)
    k2 = rhs(dom, 0.4)
    assert not torch.equal(k1, k2)
    assert torch.equal(rhs(dom, 1.7), k1)
    gh.gh_set_analytic_kerr_schild(dom, -1, 1.1, w.chi, dom.new_state())
    k4 = rhs(dom, 1.7)
    fresh = gh.Domain.from_workload(w)
    gh.gh_set_analytic_kerr_schild(fresh, -1, 1.1, w.chi, fresh.new_state())
    gh.gh_set_frame_map(fresh, m["axis"], m["omega"], m["adot"], m["V"])
    assert not torch.equal(k4, k1)
    assert torch.equal(k4, rhs(fresh, 1.7))
