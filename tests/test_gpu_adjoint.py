"""The library's vector-Jacobian products against finite differences of its
own forward path and of the oracle, and the gradient of the time-integrated
constraint energy with respect to the Pi-mode coefficients against central
finite differences (the adjoint workload)."""
import numpy as np
import pytest
import torch

from oracle import evolve
from paper_1804_09101_gb300 import workloads
from parity_helpers import flat, unflat, to_dev, to_host, oracle_domain, oracle_initial_state, gpu_domain

pytestmark = pytest.mark.gpu


def _kerr2():
    return workloads.Workload(name="kerr2", shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0, chi=0.9,
                              radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=7, noise_amp=1e-6,
                              pulse=workloads.Pulse("psi_pulse", 1e-3, 4.0, 1.0, 2, workloads.random_coeffs(7, 2)))


def _setup(w):
    odom = oracle_domain(w)
    u0 = flat(oracle_initial_state(w, odom))
    dom = gpu_domain(w, odom)
    return odom, u0, dom


@pytest.mark.parametrize("wname", ["schwarzschild", "kerr2"])
def test_rhs_vjp_dot_product_against_finite_differences(wname):
    """<v, J w> by central differences of gh_rhs equals <J^T v, w> from gh_rhs_vjp."""
    from paper_1804_09101_gb300 import gh
    w = workloads.schwarzschild_single_shell() if wname == "schwarzschild" else _kerr2()
    odom, u0, dom = _setup(w)
    rng = np.random.default_rng(5)
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
    assert abs(lhs - rhs) <= 1e-6 * max(abs(lhs), 1e-30), (lhs, rhs)


def test_rhs_vjp_against_the_oracle_directional_derivative():
    """The same identity with J w from central differences of the oracle's RHS."""
    from paper_1804_09101_gb300 import gh
    w = _kerr2()
    odom, u0, dom = _setup(w)
    rng = np.random.default_rng(6)
    v = rng.standard_normal(u0.shape)
    dw = rng.standard_normal(u0.shape)
    h = 1e-6
    jw = (flat(evolve.rhs(odom, unflat(u0 + h * dw, odom))) - flat(evolve.rhs(odom, unflat(u0 - h * dw, odom)))) / (2 * h)
    ub = dom.new_state()
    gh.gh_rhs_vjp(dom, to_dev(u0), to_dev(v), ub)
    lhs, rhs = float(v @ jw), float(to_host(ub) @ dw)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("wname", ["schwarzschild", "kerr2"])
def test_rk4_step_vjp_dot_product(wname):
    from paper_1804_09101_gb300 import gh
    w = workloads.schwarzschild_single_shell() if wname == "schwarzschild" else _kerr2()
    odom, u0, dom = _setup(w)
    rng = np.random.default_rng(7)
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


def test_constraint_energy_vjp():
    from paper_1804_09101_gb300 import gh
    from paper_1804_09101_gb300.adjoint import constraint_energy
    w = _kerr2()
    odom, u0, dom = _setup(w)
    rng = np.random.default_rng(8)
    dw = rng.standard_normal(u0.shape) * 1e-3
    h = 1e-4
    fd = (constraint_energy(dom, to_dev(u0 + h * dw)) - constraint_energy(dom, to_dev(u0 - h * dw))) / (2 * h)
    ub = dom.new_state()
    gh.gh_constraint_energy_vjp(dom, to_dev(u0), 1.0, ub)
    an = float(to_host(ub) @ dw)
    assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


def _adjoint_setup(n_r=11, L=7, steps=200):
    from paper_1804_09101_gb300 import gh
    w = workloads.adjoint_single_shell()
    dom = gh.Domain([(1.8, 10.0, n_r, L)])
    base = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, base)
    p = w.pulse

    def state(c):
        u = base.clone()
        gh.gh_add_perturbation(dom, 1, 1.0, p.center, p.width, p.lmax, c, u)
        return u
    return w, dom, state, p


@pytest.mark.parametrize("steps", [20, 200])
def test_energy_gradient_wrt_pi_mode_coefficients_matches_central_fd(steps):
    """The adjoint workload: 16 l <= 3 coefficients on Pi, E = sum over the
    steps of dt * constraint energy, checkpoints every 20 steps; every
    gradient entry against central differences with h = 1e-6."""
    from paper_1804_09101_gb300 import gh
    from paper_1804_09101_gb300.adjoint import constraint_energy_gradient, evolve_energy
    w, dom, state, p = _adjoint_setup()
    c0 = np.asarray(p.coeffs, float)
    E, lam = constraint_energy_gradient(dom, state(c0), w.dt, steps, ckpt=20)
    g = gh.gh_perturbation_vjp(dom, 1, p.center, p.width, p.lmax, lam)
    h = 1e-6
    gfd = np.zeros(16)
    for k in range(16):
        e = np.zeros(16)
        e[k] = h
        gfd[k] = (evolve_energy(dom, state(c0 + e), w.dt, steps) - evolve_energy(dom, state(c0 - e), w.dt, steps)) / (2 * h)
    scale = np.abs(gfd).max()
    assert np.abs(g - gfd).max() <= 1e-6 * scale, (g, gfd)


def test_energy_gradient_matches_oracle_fd_on_a_tiny_grid():
    """Tiny grid (N_r = 5, L = 3), 3 steps: the library's adjoint gradient
    against central differences of the oracle's own evolution."""
    from paper_1804_09101_gb300 import gh
    from paper_1804_09101_gb300.adjoint import constraint_energy_gradient
    from oracle import perturb
    w, dom, state, p = _adjoint_setup(n_r=5, L=3)
    c0 = np.asarray(p.coeffs, float)
    steps = 3
    E, lam = constraint_energy_gradient(dom, state(c0), w.dt, steps, ckpt=2)
    g = gh.gh_perturbation_vjp(dom, 1, p.center, p.width, p.lmax, lam)
    odom = evolve.Domain([(1.8, 10.0, 5, 3)], w.M, w.chi)

    def oracle_E(c):
        u = [odom.u_exact[0] + perturb.pi_modes(odom.grids[0], p.center, p.width, p.lmax, c)]
        return evolve.constraint_energy(odom, u, w.dt, steps)
    h = 1e-6
    gfd = np.zeros(16)
    for k in range(16):
        e = np.zeros(16)
        e[k] = h
        gfd[k] = (oracle_E(c0 + e) - oracle_E(c0 - e)) / (2 * h)
    assert np.abs(g - gfd).max() <= 1e-6 * np.abs(gfd).max(), (g, gfd)


def test_autograd_functions_chain():
    """RK4Step and ConstraintEnergy compose under torch.autograd."""
    from paper_1804_09101_gb300 import gh
    from paper_1804_09101_gb300.adjoint import RK4Step, ConstraintEnergy, constraint_energy
    w = _kerr2()
    odom, u0, dom = _setup(w)
    x = to_dev(u0).requires_grad_(True)
    y = RK4Step.apply(RK4Step.apply(x, dom, w.dt), dom, w.dt)
    loss = ConstraintEnergy.apply(y, dom)
    loss.backward()
    dw = np.random.default_rng(9).standard_normal(u0.shape) * 1e-3
    h = 1e-4

    def f(u):
        t = to_dev(u)
        work = dom.new_work()
        gh.gh_rk4_step(dom, w.dt, t, work)
        gh.gh_rk4_step(dom, w.dt, t, work)
        return constraint_energy(dom, t)
    fd = (f(u0 + h * dw) - f(u0 - h * dw)) / (2 * h)
    an = float(to_host(x.grad) @ dw)
    assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


@pytest.mark.parametrize("ckpt", [3, 20])
def test_checkpointed_evolve_backward_matches_step_chain_and_fd(ckpt):
    """adjoint.evolve: its gradient equals the chain of RK4Step gradients
    (the same VJPs, recomputed from checkpoints) and central differences of
    <w, u_N> along a random direction; the forward result equals N plain steps."""
    from paper_1804_09101_gb300 import gh
    from paper_1804_09101_gb300.adjoint import GHStep, evolve
    w = _kerr2()
    odom, u0, dom = _setup(w)
    n = 7
    wt = to_dev(np.random.default_rng(21).standard_normal(u0.shape))
    x = to_dev(u0).requires_grad_(True)
    y = evolve(dom, x, w.dt, n, ckpt)
    (y * wt).sum().backward()
    plain = to_dev(u0)
    work = dom.new_work()
    for _ in range(n):
        gh.gh_rk4_step(dom, w.dt, plain, work)
    assert np.array_equal(to_host(y.detach()), to_host(plain))
    x2 = to_dev(u0).requires_grad_(True)
    y2 = x2
    for _ in range(n):
        y2 = GHStep.apply(y2, dom, w.dt)
    (y2 * wt).sum().backward()
    g1, g2 = to_host(x.grad), to_host(x2.grad)
    assert np.abs(g1 - g2).max() <= 1e-12 * np.abs(g2).max()
    dw = np.random.default_rng(22).standard_normal(u0.shape) * 1e-3
    h = 1e-4

    def f(u):
        t = to_dev(u)
        for _ in range(n):
            gh.gh_rk4_step(dom, w.dt, t, work)
        return float((t * wt).sum())
    fd = (f(u0 + h * dw) - f(u0 - h * dw)) / (2 * h)
    an = float(g1 @ dw)
    assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


def test_saved_stage_step_and_vjp_agree_with_the_plain_ones():
    from paper_1804_09101_gb300 import gh
    w = _kerr2()
    odom, u0, dom = _setup(w)
    a, b = to_dev(u0), to_dev(u0)
    stages = torch.zeros(3 * dom.state_size, dtype=torch.float64, device="cuda")
    gh.gh_rk4_step(dom, w.dt, a, dom.new_work())
    gh.gh_rk4_step_save(dom, w.dt, b, dom.new_work(), stages)
    assert np.array_equal(to_host(a), to_host(b))
    v = to_dev(np.random.default_rng(10).standard_normal(u0.shape))
    r1, r2 = dom.new_state(), dom.new_state()
    gh.gh_rk4_step_vjp(dom, w.dt, to_dev(u0), v, r1, gh.new_vjp_work(dom))
    gh.gh_rk4_step_vjp_saved(dom, w.dt, to_dev(u0), stages, v, r2, gh.new_vjp_work(dom), 0.0)
    assert np.abs(to_host(r1) - to_host(r2)).max() <= 1e-13 * np.abs(to_host(r1)).max()
    # the fused constraint term equals a separate constraint-energy VJP
    r3 = dom.new_state()
    gh.gh_rk4_step_vjp_saved(dom, w.dt, to_dev(u0), stages, v, r3, gh.new_vjp_work(dom), 0.37)
    gh.gh_constraint_energy_vjp(dom, to_dev(u0), 0.37, r2)
    assert np.abs(to_host(r3) - to_host(r2)).max() <= 1e-12 * np.abs(to_host(r2)).max()


def _fold_case(name):
    if name == "schwarzschild":
        return workloads.schwarzschild_single_shell()
    if name == "kerr2":
        return _kerr2()
    if name == "even_L":
        # even L: odd N_theta (an equator ring) and N_phi % 4 == 2 (no quarter point)
        return workloads.Workload(name="even_L", shells=[(1.6, 3.0, 7, 6), (3.0, 5.0, 7, 6)], M=1.0, chi=0.4,
                                  radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=21, noise_amp=1e-7)
    if name == "fft_rings_32":
        # N_phi = 32: the transposed maps' ring FFTs of 16 complex values
        return workloads.Workload(name="fft_rings_32", shells=[(1.5, 2.5, 3, 15), (2.5, 4.0, 5, 15)], M=1.0,
                                  chi=0.6, radial_filter_on=True, sh_keep_l=10, dt=0.002, seed=13, noise_amp=1e-6)
    if name == "fft_rings_64":
        # N_phi = 64: ring FFTs of 32 complex values
        return workloads.Workload(name="fft_rings_64", shells=[(1.5, 2.5, 3, 31), (2.5, 4.0, 3, 31)], M=1.0,
                                  chi=0.6, radial_filter_on=True, sh_keep_l=20, dt=0.002, seed=14, noise_amp=1e-6)
    # three shells of 288 angular points and a filter keeping l <= 7
    return workloads.Workload(name="ragged", shells=[(1.5, 2.5, 5, 11), (2.5, 4.0, 5, 11), (4.0, 7.0, 5, 11)],
                              M=1.0, chi=0.5, radial_filter_on=True, sh_keep_l=7, dt=0.005, seed=9, noise_amp=1e-7)


@pytest.mark.parametrize("wname", ["schwarzschild", "kerr2", "even_L", "ragged", "fft_rings_32", "fft_rings_64"])
def test_folded_transposes_equal_the_separable_ones(wname):
    """The reverse mode with the folded angular maps (the default) and with the
    plain separable transposes applies the same linear maps, so gh_rhs_vjp and
    the RK4 step's VJP (filters included) agree to rounding."""
    from paper_1804_09101_gb300 import gh
    w = _fold_case(wname)
    odom = oracle_domain(w)
    u0 = flat(oracle_initial_state(w, odom))
    dom_f = gpu_domain(w, odom, "folded")
    dom_s = gpu_domain(w, odom, "separable")
    rng = np.random.default_rng(71)
    v = to_dev(rng.standard_normal(u0.shape))
    u = to_dev(u0)
    out = []
    for dom in (dom_f, dom_s):
        ub = dom.new_state()
        gh.gh_rhs_vjp(dom, u, v, ub)
        ub2 = dom.new_state()
        gh.gh_rk4_step_vjp(dom, w.dt, u, v, ub2, torch.zeros(dom.vjp_work_size, dtype=torch.float64, device="cuda"))
        out.append((to_host(ub), to_host(ub2)))
    for a, b in zip(*out):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("wname", ["kerr2", "even_L", "ragged", "fft_rings_32", "fft_rings_64"])
def test_folded_filter_transpose_is_exact(wname):
    """A step with dt = 0 is the filters alone, so its VJP is F^T:
    <ybar, F x> = <F^T ybar, x> to rounding, with the folded maps.  The step
    VJP is taken at a physical state (it re-evaluates the right-hand side
    there, with weight dt = 0); x and ybar are random."""
    from paper_1804_09101_gb300 import gh
    w = _fold_case(wname)
    odom = oracle_domain(w)
    u0 = flat(oracle_initial_state(w, odom))
    dom = gpu_domain(w, odom, "folded")
    rng = np.random.default_rng(72)
    x = rng.standard_normal(dom.state_size)
    y = rng.standard_normal(dom.state_size)
    fx = to_dev(x)
    gh.gh_apply_filters(dom, fx, dom.new_work())
    fty = dom.new_state()
    gh.gh_rk4_step_vjp(dom, 0.0, to_dev(u0), to_dev(y), fty,
                       torch.zeros(dom.vjp_work_size, dtype=torch.float64, device="cuda"))
    lhs, rhs = float(y @ to_host(fx)), float(to_host(fty) @ x)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(y), (lhs, rhs)


def test_folded_transposes_with_both_paths_in_one_domain():
    """Independent holes of L = 7 (ring FFTs: three launches per map) and
    L = 11, 5 (the quarter-folded DFT: one fused launch) in one domain: the
    folded reverse mode equals the separable one on every hole."""
    from paper_1804_09101_gb300 import gh
    holes = [dict(M=1.0, chi=0.3, shells=[(1.6, 8.0, 9, 7)], dt=0.004, seed=11),
             dict(M=0.7, chi=0.8, shells=[(0.9, 3.0, 7, 11), (3.0, 9.0, 7, 11)], dt=0.003, seed=12),
             dict(M=1.5, chi=0.0, shells=[(2.5, 20.0, 11, 5)], dt=0.006, seed=13)]
    shells = [sh + (b,) for b, h in enumerate(holes) for sh in h["shells"]]
    doms = []
    for alg in (gh.GH_ALG_SEPARABLE_FOLDED, gh.GH_ALG_SEPARABLE):
        dom = gh.Domain(shells, radial_filter_on=True, sh_keep_l=-2)
        gh.gh_set_algorithm(dom, alg)
        doms.append(dom)
    u = doms[0].new_state()
    for dom in doms:                     # each domain's holes (background, gauge) and time-step scales
        ud = dom.new_state()
        for b, h in enumerate(holes):
            gh.gh_set_analytic_kerr_schild(dom, b, h["M"], h["chi"], ud)
            gh.gh_set_dt_scale(dom, b, h["dt"])
        u.copy_(ud)
    rng = np.random.default_rng(73)
    u += to_dev(rng.standard_normal(u.numel()) * 1e-7)
    v = to_dev(rng.standard_normal(u.numel()))
    out = []
    for dom in doms:
        ub = dom.new_state()
        gh.gh_rhs_vjp(dom, u, v, ub)
        ub2 = dom.new_state()
        gh.gh_rk4_step_vjp(dom, 1.0, u, v, ub2, torch.zeros(dom.vjp_work_size, dtype=torch.float64, device="cuda"))
        out.append((to_host(ub), to_host(ub2)))
    for a, b in zip(*out):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), np.abs(a - b).max() / np.abs(b).max()
