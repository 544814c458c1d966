"""Element-by-element parity of the CUDA path (through the C ABI) with the CPU
oracle, on the same seeded inputs.  Bar: max|gpu - oracle| <= 1e-11 max|u|,
and for right-hand sides, derivatives and constraints also <= 1e-10 of the
oracle output's own maximum.

Cases span several GEMM tiles with ragged tails (n_r * 50 rows and
N_theta N_phi columns that are not multiples of 64), the smallest legal
shell (n_r = 3, L = 1), multi-shell interfaces, the outer boundary and the
excision boundary, and the full 4-shell Kerr workload.
"""
import numpy as np
import pytest
import torch

from oracle import evolve, spectral, perturb
from paper_1804_09101_gb300 import workloads
from parity_helpers import (REL_TOL, flat, unflat, to_dev, to_host, oracle_domain, oracle_initial_state,
                            gpu_domain, max_rel, assert_output_parity)

pytestmark = pytest.mark.gpu


def _gh():
    from paper_1804_09101_gb300 import gh
    return gh


def w_schwarzschild():
    return workloads.schwarzschild_single_shell()


def w_kerr_two_shells():
    w = workloads.Workload(name="kerr2", shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0, chi=0.9,
                           radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=7, noise_amp=1e-8,
                           pulse=workloads.Pulse("psi_pulse", 1e-3, 4.0, 1.0, 2, workloads.random_coeffs(7, 2)))
    return w


def w_ragged():
    # N_theta N_phi = 288 (4.5 tiles), n_r * 50 = 250 rows (3.9 tiles), three shells
    return workloads.Workload(name="ragged", shells=[(1.5, 2.5, 5, 11), (2.5, 4.0, 5, 11), (4.0, 7.0, 5, 11)],
                              M=1.0, chi=0.5, radial_filter_on=True, sh_keep_l=7, dt=0.005, seed=9,
                              noise_amp=1e-7)


def w_minimal():
    return workloads.Workload(name="minimal", shells=[(1.8, 4.0, 3, 1)], M=1.0, chi=0.0, dt=0.01, seed=3,
                              noise_amp=1e-6)


def w_pi_modes():
    w = workloads.adjoint_single_shell()
    w.steps = 2
    return w


def w_even_L():
    # even L: odd N_theta (an equator ring) and N_phi % 4 == 2 (no quarter point)
    return workloads.Workload(name="even_L", shells=[(1.6, 3.0, 7, 6), (3.0, 5.0, 7, 6)], M=1.0, chi=0.4,
                              radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=21, noise_amp=1e-7)


def w_singlebh_k1():
    # the paper's SingleBH grid family, member k = 1 (N_r = 13, N_theta = 8), two shells
    w = workloads.grid_family_workload("singlebh", 1)
    w.shells = w.shells[:2]
    w.name = "singlebh_k1_2shells"
    return w


def w_bbh_k1():
    # the paper's BBH grid family, member k = 1 (N_r = 5, N_theta = 9: even L), two shells
    w = workloads.grid_family_workload("bbh", 1)
    w.shells = w.shells[:2]
    w.name = "bbh_k1_2shells"
    return w


def w_fft_rings_32():
    # N_phi = 32: the folded maps' register FFT of 16 complex values, with the
    # SH filter (keep l <= 10)
    return workloads.Workload(name="fft_rings_32", shells=[(1.5, 2.5, 3, 15), (2.5, 4.0, 5, 15)], M=1.0,
                              chi=0.6, radial_filter_on=True, sh_keep_l=10, dt=0.002, seed=13, noise_amp=1e-6)


def w_fft_rings_64():
    # N_phi = 64: the register FFT of 32 complex values (keep l <= 20)
    return workloads.Workload(name="fft_rings_64", shells=[(1.5, 2.5, 3, 31), (2.5, 4.0, 3, 31)], M=1.0,
                              chi=0.6, radial_filter_on=True, sh_keep_l=20, dt=0.002, seed=14, noise_amp=1e-6)


def w_paper_singlebh():
    # the paper's own test problem: tilted spin (0.2, 0.3, 0.4), two 10 x 19 x 38 shells
    return workloads.paper_single_bh()


CASES = {"schwarzschild": w_schwarzschild, "kerr2": w_kerr_two_shells, "ragged": w_ragged,
         "minimal": w_minimal, "even_L": w_even_L, "singlebh_k1": w_singlebh_k1, "bbh_k1": w_bbh_k1,
         "paper_singlebh": w_paper_singlebh, "fft_rings_32": w_fft_rings_32,
         "fft_rings_64": w_fft_rings_64}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w = CASES[request.param]()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    return w, odom, u0


def test_kerr_schild_initial_data_and_gauge(case):
    gh = _gh()
    w, odom, _ = case
    dom = gh.Domain.from_workload(w)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    ref = flat(odom.u_exact)
    assert max_rel(to_host(u), ref, np.abs(ref).max()) < REL_TOL
    H = torch.zeros(4 * dom.num_points, dtype=torch.float64, device="cuda")
    dH = torch.zeros(12 * dom.num_points, dtype=torch.float64, device="cuda")
    gh.gh_get_gauge(dom, H, dH)
    assert max_rel(to_host(H), flat(odom.H), np.abs(ref).max()) < REL_TOL
    assert max_rel(to_host(dH), flat(odom.dH), np.abs(ref).max()) < REL_TOL


def test_perturbations():
    gh = _gh()
    for w in [w_kerr_two_shells(), w_pi_modes()]:
        odom = oracle_domain(w)
        ref = flat(oracle_initial_state(w, odom)) - w.noise()
        dom = gh.Domain.from_workload(w)
        u = to_dev(flat(odom.u_exact))
        p = w.pulse
        gh.gh_add_perturbation(dom, 0 if p.kind == "psi_pulse" else 1, p.amplitude, p.center, p.width,
                               p.lmax, p.coeffs, u)
        assert max_rel(to_host(u), ref, np.abs(ref).max()) < REL_TOL


ALGS = ["separable", "dense", "folded"]


@pytest.mark.parametrize("alg", ALGS)
def test_cartesian_derivatives(case, alg):
    gh = _gh()
    w, odom, u0 = case
    dom = gpu_domain(w, odom, alg)
    u = to_dev(flat(u0))
    du = torch.zeros(3 * dom.state_size, dtype=torch.float64, device="cuda")
    gh.gh_derivatives(dom, u, du)
    # oracle: per shell [3, n_r, 50, th, ph]; library: [3][state]
    ref3 = np.stack([flat([spectral.cartesian_gradient(us, g)[i] for us, g in zip(u0, odom.grids)])
                     for i in range(3)])
    got = to_host(du).reshape(3, -1)
    assert_output_parity(got, ref3, np.abs(flat(u0)).max(), "derivatives")


@pytest.mark.parametrize("alg", ALGS)
def test_rhs(case, alg):
    gh = _gh()
    w, odom, u0 = case
    dom = gpu_domain(w, odom, alg)
    u = to_dev(flat(u0))
    k = dom.new_state()
    gh.gh_rhs(dom, u, k)
    ref = flat(evolve.rhs(odom, u0))
    assert_output_parity(to_host(k), ref, np.abs(flat(u0)).max(), "rhs")


def test_constraints(case):
    gh = _gh()
    w, odom, u0 = case
    dom = gpu_domain(w, odom)
    u = to_dev(flat(u0))
    c = torch.zeros(64 * dom.num_points, dtype=torch.float64, device="cuda")
    n2 = torch.zeros(len(w.shells), dtype=torch.float64, device="cuda")
    gh.gh_constraints(dom, u, c, n2)
    cref, nref = evolve.constraints(odom, u0)
    assert_output_parity(to_host(c), flat(cref), np.abs(flat(u0)).max(), "constraints")
    assert np.abs(to_host(n2) - np.array(nref)).max() <= 1e-10 * max(max(nref), 1e-30) + 1e-28


@pytest.mark.parametrize("alg", ALGS)
def test_filters(case, alg):
    gh = _gh()
    w, odom, u0 = case
    if not (w.radial_filter_on or w.sh_keep_l >= 0):
        pytest.skip("workload has no filter")
    dom = gpu_domain(w, odom, alg)
    u = to_dev(flat(u0))
    gh.gh_apply_filters(dom, u, dom.new_work())
    ref = flat(evolve.apply_filters(odom, u0))
    assert max_rel(to_host(u), ref, np.abs(flat(u0)).max()) < REL_TOL


@pytest.mark.parametrize("name,steps,alg", [("schwarzschild", 20, "separable"), ("kerr2", 3, "separable"),
                                            ("ragged", 2, "separable"), ("minimal", 5, "separable"),
                                            ("kerr2", 2, "dense"), ("kerr2", 3, "folded"),
                                            ("schwarzschild", 5, "folded"), ("paper_singlebh", 2, "separable"),
                                            ("paper_singlebh", 2, "folded"), ("even_L", 3, "folded"),
                                            ("bbh_k1", 2, "folded")])
def test_rk4_steps(name, steps, alg):
    gh = _gh()
    w = CASES[name]()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    dom = gpu_domain(w, odom, alg)
    u = to_dev(flat(u0))
    work = dom.new_work()
    n2 = torch.zeros(len(w.shells), dtype=torch.float64, device="cuda")
    ref = u0
    for _ in range(steps):
        gh.gh_rk4_step(dom, w.dt, u, work, n2)
        _, nref = evolve.constraints(odom, ref)
        assert np.abs(to_host(n2) - np.array(nref)).max() <= 1e-9 * max(max(nref), 1e-30) + 1e-28
        ref = evolve.rk4_step(odom, ref, w.dt)
    gh.gh_sync(dom)
    err = max_rel(to_host(u), flat(ref), np.abs(flat(u0)).max())
    assert err < REL_TOL, err


def test_rhs_full_size_four_shell_kerr():
    """The full 4-shell Kerr workload (N_r = 21, L = 15, 43,008 points), all
    points, both angular algorithms, plus one full RK4 step with filters."""
    gh = _gh()
    w = workloads.kerr_four_shells()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    ref = flat(evolve.rhs(odom, u0))
    for alg in ALGS:
        dom = gpu_domain(w, odom, alg)
        u = to_dev(flat(u0))
        k = dom.new_state()
        gh.gh_rhs(dom, u, k)
        assert_output_parity(to_host(k), ref, np.abs(flat(u0)).max(), alg)
    dom = gpu_domain(w, odom)
    u = to_dev(flat(u0))
    gh.gh_rk4_step(dom, w.dt, u, dom.new_work())
    ref1 = flat(evolve.rk4_step(odom, u0, w.dt))
    assert max_rel(to_host(u), ref1, np.abs(flat(u0)).max()) < REL_TOL


def test_exact_solution_is_stationary_to_truncation_on_the_gpu():
    """With its own Kerr-Schild data and gauge, the library's RHS is pure
    truncation error, falling exponentially with resolution."""
    gh = _gh()
    errs = []
    for (n_r, L) in [(11, 7), (17, 13), (23, 19)]:
        dom = gh.Domain([(3.0, 6.0, n_r, L)])
        u = dom.new_state()
        gh.gh_set_analytic_kerr_schild(dom, -1, 1.0, 0.9, u)
        k = dom.new_state()
        gh.gh_rhs(dom, u, k)
        errs.append(float(to_host(k.abs().max().reshape(1))[0]))
    assert errs[1] < 0.05 * errs[0] and errs[2] < 0.05 * errs[1], errs
