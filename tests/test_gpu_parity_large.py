"""Parity at the full size of the large workload (Kerr a = 0.95, 8 shells
r in [1.2, 100], N_r = 41, L = 31; 671,744 points) and on the largest legal
shell (N_r = 64, L = 47), in the launch configuration the benchmark times
(folded angular maps, autotuned schedule).

The input is the workload's initial data plus seeded noise (1e-4 on every
value).  The oracle's whole-shell right-hand side is minutes of work at this size, so
it is evaluated one point at a time at sampled points: the radial derivative
along the point's radial line, the angular derivatives by the harmonic
analysis of the point's (r, field) slices and the synthesis of the
derivative harmonics at the point, the DiffJac contraction, the pointwise GH
algebra, and at boundary points the oracle's characteristic conditions
(interface upwinding from both shells' interior values, outer freezing).
The RK4 step at this size is checked by a property that holds at any size
(it equals u + dt/6 (k1 + 2 k2 + 2 k3 + k4) built from gh_rhs calls, followed
by the filters) and against the oracle's own RK4 step at every point, with
the oracle's per-shell work spread over worker processes (one shell per
task)."""
import numpy as np
import pytest
import torch

from oracle import gh as ogh
from oracle import spectral
from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, OUT_TOL, flat, to_dev, to_host, oracle_domain, oracle_initial_state, gpu_domain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    w = workloads.kerr_eight_shells_large()
    # seeded N(0,1) * 1e-4 on every value, so that the right-hand side is far
    # from the stationary background's truncation error at every point
    w.noise_amp = 1e-4
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    return w, odom, u0


def _interior_rhs_at(odom, u, s, ir, j, k, jac):
    """The oracle's GH right-hand side (before boundary conditions) at point
    (ir, j, k) of shell s, from that point's radial line and angular slice."""
    g = odom.grids[s]
    us = u[s]
    dr = spectral.radial_derivative(us[:, :, j, k], g)[ir]                     # [50]
    c = spectral.sh_analysis(us[ir], g)                                         # [50, modes]
    th, ph = g["theta"][j:j + 1], g["phi"][k:k + 1]
    dth = spectral.sh_synthesis(c, spectral.real_ylm_dtheta(g["L"], th, ph))[:, 0, 0]
    dph = spectral.sh_synthesis(c, spectral.real_ylm_dphi(g["L"], th, ph))[:, 0, 0]
    J = jac[s][:, :, ir, j, k]                                                  # [3 (x^i), 3 (r, th, ph)]
    du = J[:, 0:1] * dr[None] + J[:, 1:2] * dth[None] + J[:, 2:3] * dph[None]   # [3, 50]
    U = us[ir, :, j, k]
    H = odom.H[s][ir, :, j, k]
    dH = odom.dH[s][ir, :, j, k].reshape(3, 4)
    return ogh.gh_rhs_pointwise(U[None], du[None], H[None], dH[None], odom.gamma0, odom.gamma1, odom.gamma2)[0]


def _bg_at(odom, s, ir, j, k):
    bg = odom.boundary_bg(s, ir)
    return {key: np.asarray(v)[j:j + 1, k:k + 1] for key, v in bg.items()}


def _check_sampled_rhs(w, odom, u0, n_interior=6, n_boundary=2, seed=2025):
    """gh_rhs (autotuned schedule) against the oracle at sampled interior and
    boundary points of every shell; returns the number of points compared."""
    from paper_1804_09101_gb300 import gh
    dom = gpu_domain(w, odom)
    gh.gh_autotune(dom, 3)
    k = dom.new_state()
    gh.gh_rhs(dom, to_dev(flat(u0)), k)
    got = to_host(k)
    del k
    scale = np.abs(flat(u0)).max()
    offs = np.cumsum([0] + [int(np.prod(sh)) for sh in odom.shapes()])
    jac = [spectral.spherical_jacobian(g) for g in odom.grids]
    rng = np.random.default_rng(seed)

    def gpu_at(s, ir, j, kk):
        n_r, _, nth, nph = odom.shapes()[s]
        idx = offs[s] + ((ir * 50 + np.arange(50)) * nth + j) * nph + kk
        return got[idx]

    n_cmp, worst, d_max, ref_max = 0, 0.0, 0.0, 0.0
    ns = len(odom.grids)
    for s in range(ns):
        n_r, _, nth, nph = odom.shapes()[s]
        # interior points
        for _ in range(n_interior):
            ir, j, kk = int(rng.integers(1, n_r - 1)), int(rng.integers(0, nth)), int(rng.integers(0, nph))
            ref = _interior_rhs_at(odom, u0, s, ir, j, kk, jac)
            err = np.abs(gpu_at(s, ir, j, kk) - ref).max() / scale
            worst = max(worst, err)
            ref_max = max(ref_max, float(np.abs(ref).max()))
            n_cmp += 1
        # the boundary slice at r_out: an interface with shell s + 1, or the outer boundary
        for _ in range(n_boundary):
            j, kk = int(rng.integers(0, nth)), int(rng.integers(0, nph))
            a = _interior_rhs_at(odom, u0, s, n_r - 1, j, kk, jac)
            bg = _bg_at(odom, s, n_r - 1, j, kk)
            if s + 1 < ns:
                b = _interior_rhs_at(odom, u0, s + 1, 0, j, kk, jac)
                na, nb = ogh.apply_interface_bc(a[None, None], b[None, None], bg, odom.gamma1, odom.gamma2)
                err = max(np.abs(gpu_at(s, n_r - 1, j, kk) - na[0, 0]).max(),
                          np.abs(gpu_at(s + 1, 0, j, kk) - nb[0, 0]).max()) / scale
                ref_max = max(ref_max, float(np.abs(na).max()), float(np.abs(nb).max()))
            else:
                new = ogh.apply_outer_bc(a[None, None], bg, odom.gamma1, odom.gamma2)
                err = np.abs(gpu_at(s, n_r - 1, j, kk) - new[0, 0]).max() / scale
                ref_max = max(ref_max, float(np.abs(new).max()))
            worst = max(worst, err)
            n_cmp += 1
    assert worst < REL_TOL, worst
    # and relative to the right-hand side's own size at the sampled points
    assert worst * scale <= OUT_TOL * ref_max, (worst * scale, ref_max)
    return n_cmp


def test_rhs_at_sampled_points_full_size(large):
    w, odom, u0 = large
    assert _check_sampled_rhs(w, odom, u0) == 8 * len(odom.grids)


def test_rhs_at_sampled_points_largest_legal_shell():
    """The largest shell gh_create_domain accepts (n_r = 64, L = 47: 294,912
    points), r in [1.5, 20] around a Kerr hole a = 0.7 (inner boundary inside
    the horizon r_+ = 1.71), with the radial filter and keep l <= 31."""
    w = workloads.Workload(name="max_shell", shells=[(1.5, 20.0, 64, 47)], M=1.0, chi=0.7,
                           radial_filter_on=True, sh_keep_l=31, dt=0.002, seed=31, noise_amp=1e-4)
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    assert _check_sampled_rhs(w, odom, u0, n_interior=10, n_boundary=4, seed=47) == 14


def test_rk4_step_is_the_composition_of_its_parts_full_size(large):
    """u1 = F(u0 + dt/6 (k1 + 2 k2 + 2 k3 + k4)) with k from gh_rhs at the
    stage states and F = gh_apply_filters, against gh_rk4_step."""
    from paper_1804_09101_gb300 import gh
    w, odom, u0 = large
    dom = gpu_domain(w, odom)
    gh.gh_autotune(dom, 3)
    dt = w.dt
    u = to_dev(flat(u0))
    ks = []
    x = u
    for c in (0.5, 0.5, 1.0, None):
        kk = dom.new_state()
        gh.gh_rhs(dom, x, kk)
        ks.append(kk)
        if c is not None:
            x = u + c * dt * kk
    ref = u + (dt / 6.0) * (ks[0] + 2.0 * ks[1] + 2.0 * ks[2] + ks[3])
    del ks, x
    work = dom.new_work()
    gh.gh_apply_filters(dom, ref, work)
    step = u.clone()
    gh.gh_rk4_step(dom, dt, step, work)
    torch.cuda.synchronize()
    err = float((step - ref).abs().max()) / float(u.abs().max())
    assert err < REL_TOL, err


def test_rk4_step_full_size_matches_the_oracle_step(large, monkeypatch):
    """One gh_rk4_step of the large workload (8 shells, N_r = 41, L = 31, with
    its radial and SH filters), in the launch configuration the benchmark
    times, against the oracle's rk4_step at every one of the 33.6 M values.
    The oracle's interior right-hand sides and filters run one shell per
    worker process; its rk4_step and apply_boundaries are the oracle's own."""
    from oracle import evolve
    from oracle_pool import ShellPool
    from paper_1804_09101_gb300 import gh
    w, odom, u0 = large
    dom = gpu_domain(w, odom)
    gh.gh_autotune(dom, 3)
    u = to_dev(flat(u0))
    gh.gh_rk4_step(dom, w.dt, u, dom.new_work())
    got = to_host(u)
    del u
    pool = ShellPool(len(odom.grids))
    try:
        pool.install(monkeypatch)
        ref = flat(evolve.rk4_step(odom, u0, w.dt))
    finally:
        pool.close()
    err = float(np.abs(got - ref).max()) / float(np.abs(flat(u0)).max())
    assert err < REL_TOL, err
    # the step moved the state by far more than the tolerance
    assert float(np.abs(ref - flat(u0)).max()) > 1e4 * REL_TOL * float(np.abs(flat(u0)).max())
