"""Parity of the tensor spherical-harmonic S2 filter (spin-weighted harmonics in
the complex frame r_hat, m, conj(m); Secs. 3.1 and 3.4) with the oracle
through the C ABI: the filter alone on seeded, non-band-limited states (one
and two shells, a given keep and floor(2L/3), keep = 0 and keep = L), RK4 steps with the filter; at full size the properties that hold at
any resolution (constant Cartesian tensors are kept when keep >= 3, the
filter is a projection); the captured RK4 graph agrees with the plain calls,
switching back restores the per-component filter; the reverse mode (the
filter's transpose exactly, and the RK4 step's VJP against finite
differences)."""
import numpy as np
import pytest
import torch

from oracle import evolve
from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, flat, unflat, to_dev, to_host, oracle_domain, oracle_initial_state, gpu_domain

pytestmark = pytest.mark.gpu


def _gh():
    from paper_1804_09101_gb300 import gh
    return gh


def _wl(name, shells, keep, radial=True):
    return workloads.Workload(name=name, shells=shells, M=1.0, chi=0.7, gamma1=-1.0, radial_filter_on=radial,
                              sh_keep_l=keep, dt=0.005, seed=11, noise_amp=1e-6,
                              pulse=workloads.Pulse("psi_pulse", 1e-3, 4.0, 0.7, 2, workloads.random_coeffs(11, 2)))


CASES = {
    "one_shell_keep4": lambda: _wl("tf1", [(1.5, 5.0, 7, 7)], 4, radial=False),
    "two_shells_keep4": lambda: _wl("tf2", [(1.3, 3.0, 7, 7), (3.0, 6.0, 7, 7)], 4),
    "two_thirds_L9": lambda: _wl("tf3", [(1.5, 5.0, 5, 9)], -2, radial=False),
    "keep0": lambda: _wl("tf4", [(1.5, 5.0, 5, 5)], 0, radial=False),
    "keepL": lambda: _wl("tf5", [(1.5, 5.0, 5, 6)], 6, radial=False),
}


def _tensor_domain(w, odom=None):
    gh = _gh()
    dom = gpu_domain(w, odom)
    gh.gh_set_sh_filter(dom, "tensor")
    return dom


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w = CASES[request.param]()
    odom = oracle_domain(w)
    odom.sh_filter = "tensor"
    return w, odom


def test_filter_matches_oracle(case):
    gh = _gh()
    w, odom = case
    dom = _tensor_domain(w, odom)
    # O(1) seeded noise on every field: every frame component and spin is exercised
    rng = np.random.default_rng(2024)
    x = rng.standard_normal(dom.state_size)
    u = to_dev(x)
    gh.gh_apply_filters(dom, u, dom.new_work())
    ref = flat(evolve.apply_filters(odom, unflat(x, odom)))
    assert np.abs(to_host(u) - ref).max() <= REL_TOL * np.abs(x).max()
    # and it is not the per-component filter
    odom.sh_filter = "component"
    comp = flat(evolve.apply_filters(odom, unflat(x, odom)))
    odom.sh_filter = "tensor"
    assert np.abs(comp - ref).max() > 1e-3


def test_rk4_steps_match_oracle():
    gh = _gh()
    w = CASES["two_shells_keep4"]()
    odom = oracle_domain(w)
    odom.sh_filter = "tensor"
    u0 = oracle_initial_state(w, odom)
    dom = _tensor_domain(w, odom)
    u = to_dev(flat(u0))
    work = dom.new_work()
    ou = u0
    for _ in range(2):
        gh.gh_rk4_step(dom, w.dt, u, work)
        ou = evolve.rk4_step(odom, ou, w.dt)
    assert np.abs(to_host(u) - flat(ou)).max() <= REL_TOL * np.abs(flat(u0)).max()


def _constant_tensors(w, seed):
    """Every field constant in space (random values): Cartesian tensors of rank
    <= 3 whose frame components have l <= rank."""
    rng = np.random.default_rng(seed)
    vals = rng.standard_normal(50)
    out = []
    for (_, _, n_r, L) in w.shells:                # [n_r, 50, n_theta, n_phi]
        a = np.empty((n_r, 50, L + 1, 2 * (L + 1)))
        a[...] = vals[None, :, None, None]
        out.append(a)
    return flat(out)


@pytest.mark.parametrize("make", [workloads.kerr_four_shells, workloads.kerr_eight_shells_large])
def test_full_size_properties(make):
    gh = _gh()
    w = make()
    w.radial_filter_on = False
    dom = gh.Domain.from_workload(w)
    gh.gh_set_sh_filter(dom, "tensor")
    work = dom.new_work()
    # constant Cartesian tensors survive any keep >= 3
    c = to_dev(_constant_tensors(w, 5))
    c0 = c.clone()
    gh.gh_apply_filters(dom, c, work)
    torch.cuda.synchronize()
    assert float((c - c0).abs().max()) <= REL_TOL * float(c0.abs().max())
    # a projection: filtering twice is filtering once
    g = torch.Generator(device="cuda").manual_seed(9)
    x = torch.randn(dom.state_size, dtype=torch.float64, device="cuda", generator=g)
    gh.gh_apply_filters(dom, x, work)
    y = x.clone()
    gh.gh_apply_filters(dom, y, work)
    torch.cuda.synchronize()
    assert float((y - x).abs().max()) <= REL_TOL * float(x.abs().max())
    # and it removes something from non-band-limited data
    z = torch.randn(dom.state_size, dtype=torch.float64, device="cuda", generator=g)
    z0 = z.clone()
    gh.gh_apply_filters(dom, z, work)
    torch.cuda.synchronize()
    assert float((z - z0).abs().max()) > 1e-2


def test_keep_below_rank_changes_constant_tensors():
    """keep = 1 removes the l = 2, 3 parts of constant rank-2 and rank-3
    tensors while the per-component filter keeps every constant."""
    gh = _gh()
    w = _wl("tf6", [(1.5, 5.0, 5, 5)], 1, radial=False)
    dom = gh.Domain.from_workload(w)
    work = dom.new_work()
    c0 = to_dev(_constant_tensors(w, 6))
    a = c0.clone()
    gh.gh_apply_filters(dom, a, work)
    gh.gh_set_sh_filter(dom, "tensor")
    b = c0.clone()
    gh.gh_apply_filters(dom, b, work)
    torch.cuda.synchronize()
    assert float((a - c0).abs().max()) <= REL_TOL * float(c0.abs().max())
    assert float((b - c0).abs().max()) > 1e-2


def test_graph_and_mode_switch():
    gh = _gh()
    w = CASES["two_shells_keep4"]()
    dom = gh.Domain.from_workload(w)
    with pytest.raises(RuntimeError):
        gh.gh_set_sh_filter(dom, 5)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    g = torch.Generator(device="cuda").manual_seed(3)
    u += 1e-6 * torch.randn(dom.state_size, dtype=torch.float64, device="cuda", generator=g)
    comp = u.clone()
    gh.gh_apply_filters(dom, comp, dom.new_work())
    gh.gh_set_sh_filter(dom, "tensor")
    a, b = u.clone(), u.clone()
    wa, wb = dom.new_work(), dom.new_work()
    for _ in range(3):
        gh.gh_rk4_step(dom, w.dt, a, wa)
    gh.gh_rk4_graph_capture(dom, w.dt, b, wb)
    gh.gh_rk4_graph_launch(dom, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    gh.gh_set_sh_filter(dom, "component")
    back = u.clone()
    gh.gh_apply_filters(dom, back, dom.new_work())
    torch.cuda.synchronize()
    assert torch.equal(back, comp)


def test_dp5_attempt_matches_oracle():
    """One Dormand-Prince 5(4) attempt with the tensor filter after it."""
    from oracle import dp5 as odp5
    gh = _gh()
    w = CASES["two_shells_keep4"]()
    odom = oracle_domain(w)
    odom.sh_filter = "tensor"
    u0 = oracle_initial_state(w, odom)
    dom = _tensor_domain(w, odom)
    u = to_dev(flat(u0))
    work = torch.zeros(dom.dp5_work_size, dtype=torch.float64, device="cuda")
    err, ok, dtn = gh.gh_dp5_step(dom, w.dt, 1e-8, 1e-8, u, work)
    ou, oerr, ook, odtn = odp5.dp5_step(odom, u0, w.dt, 1e-8, 1e-8)
    assert ok == ook and ok
    assert abs(err - oerr) <= 1e-9 * max(1.0, abs(oerr))
    assert np.abs(to_host(u) - flat(ou)).max() <= REL_TOL * np.abs(flat(u0)).max()


def test_holes_of_different_resolution_in_one_domain():
    """Three holes of L = 7, 11 and 5 (plans with different K, shared memory
    and items in one launch): each hole's part equals the oracle's tensor
    filter (floor(2L/3) per hole, radial filter on) of that hole alone."""
    gh = _gh()
    holes = _three_holes()
    shells = [s + (b,) for b, h in enumerate(holes) for s in h["shells"]]
    dom = gh.Domain(shells, radial_filter_on=True, sh_keep_l=-2)
    gh.gh_set_sh_filter(dom, "tensor")
    x = np.random.default_rng(77).standard_normal(dom.state_size)
    u = to_dev(x)
    gh.gh_apply_filters(dom, u, dom.new_work())
    got = to_host(u)
    off = 0
    for h in holes:
        odom = evolve.Domain(h["shells"], h["M"], h["chi"], radial_filter_on=True, sh_keep_l=-2,
                             sh_filter="tensor")
        n = 50 * sum(nr * 2 * (L + 1) ** 2 for (_, _, nr, L) in h["shells"])
        ref = flat(evolve.apply_filters(odom, unflat(x[off:off + n], odom)))
        assert np.abs(got[off:off + n] - ref).max() <= REL_TOL * np.abs(x[off:off + n]).max(), h
        off += n


def _three_holes():
    return [dict(M=1.0, chi=0.3, shells=[(1.6, 8.0, 9, 7)]),
            dict(M=0.7, chi=0.8, shells=[(0.9, 3.0, 7, 11), (3.0, 9.0, 7, 11)]),
            dict(M=1.5, chi=0.0, shells=[(2.5, 20.0, 11, 5)])]


@pytest.mark.parametrize("which", ["one_shell_keep4", "two_shells_keep4", "three_holes"])
def test_filter_transpose_exact(which):
    """A step with dt = 0 is the filters alone, u -> S u, and its VJP is S^T ybar:
    <ybar, S x> = <S^T ybar, x> to rounding (the transpose of the spin
    projection is D P D^-1 with the quadrature weights D)."""
    gh = _gh()
    u = None
    if which == "three_holes":
        holes = _three_holes()
        shells = [s + (b,) for b, h in enumerate(holes) for s in h["shells"]]
        dom = gh.Domain(shells, radial_filter_on=True, sh_keep_l=-2)
        u = dom.new_state()
        for b, h in enumerate(holes):
            gh.gh_set_analytic_kerr_schild(dom, b, h["M"], h["chi"], u)
    else:
        w = CASES[which]()
        dom = gh.Domain.from_workload(w)
        u = dom.new_state()
        gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    gh.gh_set_sh_filter(dom, "tensor")
    # a valid metric plus noise: the right-hand side is finite, so the dt = 0
    # step is exactly the filters
    rng = np.random.default_rng(31)
    x = to_host(u) + 1e-2 * rng.standard_normal(dom.state_size)
    yb = rng.standard_normal(dom.state_size)
    u = to_dev(x)
    gh.gh_rk4_step(dom, 0.0, u, dom.new_work())
    sx = to_host(u)
    g = dom.new_state()
    gh.gh_rk4_step_vjp(dom, 0.0, to_dev(x), to_dev(yb), g, gh.new_vjp_work(dom))
    lhs, rhs = float(yb @ sx), float(to_host(g) @ x)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(yb), (lhs, rhs)
    # and it is not the per-component transpose
    gh.gh_set_sh_filter(dom, "component")
    g2 = dom.new_state()
    gh.gh_rk4_step_vjp(dom, 0.0, to_dev(x), to_dev(yb), g2, gh.new_vjp_work(dom))
    assert float((g2 - g).abs().max()) > 1e-3


def test_step_vjp_dot_product_against_finite_differences():
    gh = _gh()
    w = CASES["two_shells_keep4"]()
    odom = oracle_domain(w)
    u0 = flat(oracle_initial_state(w, odom))
    dom = _tensor_domain(w, odom)
    rng = np.random.default_rng(32)
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
