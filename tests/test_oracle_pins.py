"""Pins of the CPU oracle against what the mathematics and the paper fix.

Each test checks the oracle against something other than itself: closed
forms, textbook formulas, a library routine (scipy), exact quadrature
identities, the exact Kerr-Schild solution (the paper's stationary test
problem, Sec. 3.1), or brute-force finite differences.  None of these tests
needs a GPU.
"""
import numpy as np
import pytest
from scipy.special import sph_harm_y

from oracle import grid, spectral, gh, kerr_schild, evolve
import exact_solutions


# ------------------------------------------------------------------ grids
@pytest.mark.parametrize("n", [5, 8, 11, 21])
def test_clenshaw_curtis_exact_on_polynomials(n):
    x = grid.cgl_nodes(n)
    w = grid.clenshaw_curtis_weights(n)
    for k in range(n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("L", [3, 7, 15])
def test_gauss_legendre_exact_to_degree_2L_plus_1(L):
    g = grid.shell_grid(1.0, 2.0, 5, L)
    for k in range(2 * L + 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(g["wth"], g["cth"] ** k) - exact) < 1e-14
    assert np.all(np.diff(g["theta"]) > 0)


def test_volume_weights_sum_to_shell_volume():
    for (a, b, n, L) in [(1.8, 10.0, 11, 7), (1.3, 3.0, 21, 15)]:
        g = grid.shell_grid(a, b, n, L)
        vol = 4.0 * np.pi * (b ** 3 - a ** 3) / 3.0
        assert abs(grid.volume_weights(g).sum() - vol) < 1e-13 * vol


# ----------------------------------------------------------- radial part
def test_radial_derivative_exact_below_degree_n_r():
    g = grid.shell_grid(1.8, 10.0, 11, 3)
    x = g["x"]
    rng = np.random.default_rng(0)
    c = rng.standard_normal(11)
    u = np.polynomial.polynomial.polyval(x, c)
    du = np.polynomial.polynomial.polyval(x, np.polynomial.polynomial.polyder(c))
    got = spectral.radial_derivative(u[:, None, None] * np.ones((1, 4, 8)), g)
    assert np.abs(got[:, 0, 0] - du * 2.0 / 8.2).max() < 1e-12 * np.abs(du).max()


def _textbook_cgl_matrix(x):
    """Closed-form Chebyshev collocation derivative matrix (Gottlieb-Hussaini form)."""
    n = len(x)
    c = np.ones(n)
    c[0] = c[-1] = 2.0
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (c[i] / c[j]) * (-1.0) ** (i + j) / (x[i] - x[j])
    D -= np.diag(D.sum(axis=1))
    return D


@pytest.mark.parametrize("n", [5, 11, 21])
def test_radial_derivative_delta_probe_is_textbook_matrix(n):
    """Trace the oracle's operator with delta inputs (the paper's tracing idea,
    Sec. 3.4) and compare with the closed-form collocation matrix."""
    g = grid.shell_grid(-1.0, 1.0, n, 1)
    probe = np.eye(n)[:, :, None, None] * np.ones((1, 1, 2, 4))
    Dtraced = spectral.radial_derivative(probe, g)[:, :, 0, 0]
    assert np.abs(Dtraced - _textbook_cgl_matrix(g["x"])).max() < 1e-11 * n * n


def test_expcheb_filter_scales_each_chebyshev_mode():
    g = grid.shell_grid(-1.0, 1.0, 11, 1)
    s = spectral.expcheb_sigma(11, 36.0, 32)
    assert s[0] == 1.0 and abs(s[-1] - np.exp(-36.0)) < 1e-30
    for k in [0, 3, 7, 10]:
        Tk = spectral.cheb_T(k, g["x"])[:, None, None] * np.ones((1, 2, 4))
        out = spectral.radial_filter(Tk, g, 36.0, 32)
        assert np.abs(out - s[k] * Tk).max() < 1e-13
    # strength and order measured from the filter's action on T_k: the gain is
    # exp(-36 (k/(N-1))^p) with p = 32 (the ExpCheb filter of order 32, Sec. 3.4)
    gain = {}
    for k in [7, 9]:
        Tk = spectral.cheb_T(k, g["x"])
        out = spectral.radial_filter(Tk[:, None, None], g, 36.0, 32)[:, 0, 0]
        gain[k] = float(out @ Tk / (Tk @ Tk))
    order = np.log(np.log(gain[7]) / np.log(gain[9])) / np.log(7.0 / 9.0)
    strength = -np.log(gain[9]) / 0.9 ** order
    assert abs(order - 32.0) < 1e-6 and abs(strength - 36.0) < 1e-6, (order, strength)


# ---------------------------------------------------------- angular part
def _real_from_scipy(l, m, th, ph, diff):
    """Real Y_lm (up to the per-mode sign convention) from scipy's complex one."""
    mm = abs(m)
    if diff:
        y, dy = sph_harm_y(l, mm, th, ph, diff_n=1)
        y = dy[..., 0]
    else:
        y = sph_harm_y(l, mm, th, ph)
    if m == 0:
        return np.real(y)
    return np.sqrt(2.0) * (np.real(y) if m > 0 else np.imag(y))


@pytest.mark.parametrize("L", [2, 7])
def test_real_ylm_and_dtheta_match_scipy(L):
    g = grid.shell_grid(1.0, 2.0, 3, L)
    TH, PH = np.meshgrid(g["theta"], g["phi"], indexing="ij")
    Y = spectral.real_ylm(L, g["theta"], g["phi"])
    dY = spectral.real_ylm_dtheta(L, g["theta"], g["phi"])
    for i, (l, m) in enumerate(spectral.sh_modes(L)):
        ref = _real_from_scipy(l, m, TH, PH, False)
        dref = _real_from_scipy(l, m, TH, PH, True)
        k = np.argmax(np.abs(ref))
        sgn = np.sign(Y[i].flat[k] / ref.flat[k])
        assert np.abs(Y[i] - sgn * ref).max() < 1e-13
        assert np.abs(dY[i] - sgn * dref).max() < 1e-12 * max(1.0, l)


def test_dtheta_closed_forms_low_l():
    th = np.linspace(0.1, 3.0, 7)
    dY = spectral.real_ylm_dtheta(2, th, np.zeros(1))[:, :, 0]
    modes = spectral.sh_modes(2)
    i10 = modes.index((1, 0))
    i20 = modes.index((2, 0))
    assert np.abs(dY[i10] + np.sqrt(3 / (4 * np.pi)) * np.sin(th)).max() < 1e-14
    ref20 = np.sqrt(5 / (16 * np.pi)) * (-6.0 * np.cos(th) * np.sin(th))
    assert np.abs(dY[i20] - ref20).max() < 1e-14


def test_real_ylm_orthonormal_on_grid():
    g = grid.shell_grid(1.0, 2.0, 3, 7)
    Y = spectral.real_ylm(7, g["theta"], g["phi"])
    w = g["wth"][:, None] * g["wphi"]
    G = np.einsum("ajk,bjk,jk->ab", Y, Y, w)
    assert np.abs(G - np.eye(len(Y))).max() < 1e-13


def test_sh_truncation_filter_keeps_low_l_and_drops_high_l():
    L, keep = 7, 4
    g = grid.shell_grid(1.0, 2.0, 3, L)
    Y = spectral.real_ylm(L, g["theta"], g["phi"])
    for i, (l, m) in enumerate(spectral.sh_modes(L)):
        out = spectral.sh_truncation_filter(Y[i][None], g, keep)[0]
        ref = Y[i] if l <= keep else 0.0 * Y[i]
        assert np.abs(out - ref).max() < 1e-13


@pytest.mark.parametrize("n_r,L,deg", [(11, 7, 5), (9, 5, 5)])
def test_cartesian_gradient_exact_on_polynomials(n_r, L, deg):
    """Radial + angular derivatives + DiffJac: exact on polynomials in (x,y,z)
    of total degree <= min(n_r - 1, L)."""
    g = grid.shell_grid(1.8, 10.0, n_r, L)
    X, Y, Z = grid.cartesian_coords(g)
    rng = np.random.default_rng(3)
    terms = [(a, b, c) for a in range(deg + 1) for b in range(deg + 1 - a)
             for c in range(deg + 1 - a - b)]
    coef = rng.standard_normal(len(terms))
    f = sum(k * X ** a * Y ** b * Z ** c for k, (a, b, c) in zip(coef, terms))
    fx = sum(k * a * X ** max(a - 1, 0) * Y ** b * Z ** c for k, (a, b, c) in zip(coef, terms))
    fy = sum(k * b * X ** a * Y ** max(b - 1, 0) * Z ** c for k, (a, b, c) in zip(coef, terms))
    fz = sum(k * c * X ** a * Y ** b * Z ** max(c - 1, 0) for k, (a, b, c) in zip(coef, terms))
    d = spectral.cartesian_gradient(f[:, None], g)[:, :, 0]
    scale = np.abs(f).max()
    for i, ref in enumerate([fx, fy, fz]):
        assert np.abs(d[i] - ref).max() < 1e-11 * scale


# ----------------------------------------------------------- Kerr-Schild
def _sample_points():
    rng = np.random.default_rng(5)
    P = rng.uniform(-6, 6, size=(40, 3))
    P = P[np.linalg.norm(P, axis=1) > 2.0]
    return P[:, 0], P[:, 1], P[:, 2]


TILTED = (0.2, 0.3, 0.4)     # the paper's test-problem spin vector (Sec. 3.1)


@pytest.mark.parametrize("chi", [0.0, 0.9, TILTED])
def test_kerr_schild_null_vector_and_determinant(chi):
    X, Y, Z = _sample_points()
    g, dg, ddg = kerr_schild.metric_and_derivatives(X, Y, Z, 1.0, chi)
    assert np.abs(np.linalg.det(g) + 1.0).max() < 1e-12
    eta = np.diag([-1.0, 1, 1, 1])
    # l_a l_b = (g - eta)/(2H) has rank one; l is null: eta^ab (g-eta)_ab = 0
    assert np.abs(np.einsum("ab,...ab->...", eta, g - eta)).max() < 1e-13


def test_kerr_schild_reduces_to_schwarzschild():
    X, Y, Z = _sample_points()
    g, _, _ = kerr_schild.metric_and_derivatives(X, Y, Z, 1.3, 0.0)
    R = np.sqrt(X * X + Y * Y + Z * Z)
    l = np.stack([np.ones_like(R), X / R, Y / R, Z / R], axis=-1)
    ref = np.diag([-1.0, 1, 1, 1]) + 2 * (1.3 / R)[:, None, None] * l[:, :, None] * l[:, None, :]
    assert np.abs(g - ref).max() < 1e-14


def _rotation_taking_z_to(n):
    """Rodrigues rotation matrix R with R e_z = n (unit vector)."""
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(z, n)
    c = float(np.dot(z, n))
    K = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    return np.eye(3) + K + K @ K / (1.0 + c)


def test_spin_vector_form_is_the_rotated_z_axis_metric():
    """Kerr-Schild with spin vector a equals the z-axis metric of the same |a|
    evaluated at R^T x and transformed as a tensor (R e_z = a/|a|): the vector
    formula is pinned by rotation covariance, not by itself."""
    X, Y, Z = _sample_points()
    a = np.array(TILTED) * 1.3
    amag = float(np.linalg.norm(a))
    R = _rotation_taking_z_to(a / amag)
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-15
    x = np.stack([X, Y, Z], axis=-1)
    xr = x @ R                                      # R^T x for row vectors
    gz, dgz, _ = kerr_schild.metric_and_derivatives(xr[:, 0], xr[:, 1], xr[:, 2], 1.3, amag)
    L = np.eye(4)
    L[1:, 1:] = R
    ref = np.einsum("ac,...cd,bd->...ab", L, gz, L)
    # d_i g(x) = R_ij (d_j g^z)(R^T x), transformed on ab as above
    dref = np.einsum("ij,ac,...jcd,bd->...iab", R, L, dgz, L)
    g, dg, _ = kerr_schild.metric_and_derivatives(X, Y, Z, 1.3, tuple(a))
    assert np.abs(g - ref).max() < 1e-13
    assert np.abs(dg - dref).max() < 1e-12


def test_spin_vector_along_z_matches_the_scalar_form():
    X, Y, Z = _sample_points()
    g1, dg1, ddg1 = kerr_schild.metric_and_derivatives(X, Y, Z, 1.0, 0.9)
    g2, dg2, ddg2 = kerr_schild.metric_and_derivatives(X, Y, Z, 1.0, (0.0, 0.0, 0.9))
    assert np.abs(g1 - g2).max() < 1e-14
    assert np.abs(dg1 - dg2).max() < 1e-13
    assert np.abs(ddg1 - ddg2).max() < 1e-12


@pytest.mark.parametrize("chi", [0.0, 0.9, TILTED])
def test_kerr_schild_derivatives_match_finite_differences(chi):
    X, Y, Z = _sample_points()
    g, dg, ddg = kerr_schild.metric_and_derivatives(X, Y, Z, 1.0, chi)
    h = 1e-5
    for i in range(3):
        e = [0.0, 0.0, 0.0]
        e[i] = h
        gp, dgp, _ = kerr_schild.metric_and_derivatives(X + e[0], Y + e[1], Z + e[2], 1.0, chi)
        gm, dgm, _ = kerr_schild.metric_and_derivatives(X - e[0], Y - e[1], Z - e[2], 1.0, chi)
        assert np.abs((gp - gm) / (2 * h) - dg[:, i]).max() < 1e-8
        assert np.abs((dgp - dgm) / (2 * h) - ddg[:, :, i]).max() < 1e-7


@pytest.mark.parametrize("chi", [0.0, 0.9, TILTED])
def test_gauge_source_zeroes_gauge_constraint_and_dH_matches_fd(chi):
    """H_a = -Gamma_a computed from d g (kerr_schild) makes C_a = H_a + Gamma_a,
    computed through the t/Pi/Phi identity (gh), vanish; d_i H by FD."""
    X, Y, Z = _sample_points()
    g, dg, ddg = kerr_schild.metric_and_derivatives(X, Y, Z, 1.0, chi)
    H, dH = kerr_schild.gauge_source(g, dg, ddg)
    psi, Pi, Phi = kerr_schild.gh_fields(g, dg)
    s = gh.spacetime_split(psi)
    _, Gam = gh.christoffel_first_kind(s, Pi, Phi)
    assert np.abs(gh.gauge_constraint(s, Gam, H)).max() < 1e-13
    h = 1e-5
    for i in range(3):
        e = [0.0, 0.0, 0.0]
        e[i] = h
        Hp, _ = kerr_schild.gauge_source(*kerr_schild.metric_and_derivatives(
            X + e[0], Y + e[1], Z + e[2], 1.0, chi))
        Hm, _ = kerr_schild.gauge_source(*kerr_schild.metric_and_derivatives(
            X - e[0], Y - e[1], Z - e[2], 1.0, chi))
        assert np.abs((Hp - Hm) / (2 * h) - dH[:, i]).max() < 1e-7


def test_inverse_spacetime_metric():
    X, Y, Z = _sample_points()
    g, _, _ = kerr_schild.metric_and_derivatives(X, Y, Z, 1.0, 0.7)
    s = gh.spacetime_split(g)
    assert np.abs(np.einsum("...ab,...bc->...ac", s["psi_inv"], g) - np.eye(4)).max() < 1e-13


# ------------------------------------------------------- GH right-hand side
@pytest.mark.slow
@pytest.mark.parametrize("chi,shell", [(0.0, (1.8, 10.0)), (0.9, (3.0, 6.0))])
def test_rhs_of_exact_kerr_schild_converges_exponentially(chi, shell):
    """The stationary exact solution has d_t u = 0: the discrete RHS is pure
    truncation error and must fall exponentially with resolution (this pins
    every term of the RHS that does not multiply a constraint)."""
    errs = []
    for (n_r, L) in [(11, 7), (17, 13), (23, 19)]:
        dom = evolve.Domain([(shell[0], shell[1], n_r, L)], 1.0, chi)
        errs.append(np.abs(evolve.rhs_interior(dom, dom.u_exact)[0]).max())
    assert errs[1] < 0.05 * errs[0] and errs[2] < 0.05 * errs[1], errs
    assert errs[2] < 1e-6


def test_rhs_equals_the_time_derivative_of_flat_space_in_moving_coordinates():
    """The pointwise GH right-hand side at exact data of a solution equals its
    exact time derivative, except for the d_t H_b part of -2 alpha nabla_(a H_b),
    which the right-hand side leaves out (gauge source held fixed in time):
    RHS(Pi_ab) = d_t Pi_ab + alpha (delta^0_a d_t H_b + delta^0_b d_t H_a).
    The solution is flat space in time-dependent, non-linear coordinates
    (tests/exact_solutions.py), where every constraint vanishes.  Pins every
    term that does not multiply a constraint, including the Pi-Pi,
    Gamma-Gamma and t t Pi Pi terms that vanish on stationary Kerr-Schild
    data.  Any damping parameters: the constraints vanish."""
    f_g, f_dg = exact_solutions.moving_minkowski_metric()
    rng = np.random.default_rng(15)
    t = rng.uniform(0.0, 1.0, 4)
    x, y, z = rng.uniform(-0.5, 0.5, (3, 4))
    u, du, H, dH, want = exact_solutions.expected_rhs(f_g, f_dg, t, x, y, z)
    for g0, g1, g2 in [(1.0, -1.0, 1.0), (0.3, 0.7, 2.0)]:
        got = gh.gh_rhs_pointwise(u, du, H, dH, g0, g1, g2)
        assert np.abs(got - want).max() < 1e-8, np.abs(got - want).max()
    # the data are not trivial: the Pi-Pi contraction is of order 1e-2
    psi, Pi, _ = gh.unpack_fields(u)
    assert np.abs(np.einsum("...cd,...ca,...db->...ab", np.linalg.inv(psi), Pi, Pi)).max() > 1e-3


def test_constraint_components_of_fields_with_a_known_violation():
    """psi_ab a quadratic polynomial in (x, y, z) (differentiated exactly on the
    grid), Phi_iab = d_i psi_ab + delta_iab with delta linear in (x, y, z):
    then C_iab = -delta_iab and C_ijab = d_i delta_jab - d_j delta_iab (a
    constant), stored at 4 + 10 i + p and 34 + 10 q + p with
    q = 0, 1, 2 for (ij) = (xy), (xz), (yz).  The quadrature norm is checked
    against the same values summed with the volume weights."""
    g = grid.shell_grid(2.0, 3.5, 7, 5)
    X, Y, Z = grid.cartesian_coords(g)                     # [n_r, th, ph]
    rng = np.random.default_rng(16)
    a0, A, B = rng.standard_normal(10), rng.standard_normal((10, 3)), rng.standard_normal((10, 3, 3))
    D0, D1 = rng.standard_normal((3, 10)), rng.standard_normal((3, 10, 3))
    P = np.stack([X, Y, Z])                                # [3, n_r, th, ph]
    psi = 1e-2 * (a0[:, None, None, None] + np.einsum("pk,k...->p...", A, P)
                  + np.einsum("pkl,k...,l...->p...", B, P, P))
    for q, (a, b) in enumerate(gh.PAIRS):
        psi[q] += {(0, 0): -1.0, (1, 1): 1.0, (2, 2): 1.0, (3, 3): 1.0}.get((a, b), 0.0)
    dpsi = 1e-2 * (A.T[:, :, None, None, None] + np.einsum("pkl,l...->kp...", B + np.swapaxes(B, 1, 2), P))
    delta = D0[:, :, None, None, None] + np.einsum("ipk,k...->ip...", D1, P)     # [3 (i), 10, ...]
    Phi = dpsi + delta
    u = np.zeros((g["n_r"], 50) + X.shape[1:])
    u[:, 0:10] = np.moveaxis(psi, 0, 1)
    u[:, 10:20] = 0.01 * rng.standard_normal((g["n_r"], 10) + X.shape[1:])
    for i in range(3):
        u[:, 20 + 10 * i:30 + 10 * i] = np.moveaxis(Phi[i], 0, 1)
    dom = evolve.Domain([(2.0, 3.5, 7, 5)], 1.0, 0.0)
    cs, norms = evolve.constraints(dom, [u])
    c = cs[0]                                               # [n_r, 64, th, ph]
    scale = np.abs(delta).max()
    for i in range(3):
        assert np.abs(c[:, 4 + 10 * i:14 + 10 * i] + np.moveaxis(delta[i], 0, 1)).max() < 1e-10 * scale
    for q, (i, j) in enumerate([(0, 1), (0, 2), (1, 2)]):
        want = D1[j, :, i] - D1[i, :, j]                   # d_i delta_j - d_j delta_i, per pair
        assert np.abs(c[:, 34 + 10 * q:44 + 10 * q] - want[None, :, None, None]).max() < 1e-9 * scale
    w = grid.volume_weights(g)
    assert abs(norms[0] - float(np.sum(w * np.sum(c * c, axis=1)))) < 1e-12 * norms[0]


def _minkowski_point_state(rng, n=6):
    psi = np.broadcast_to(np.diag([-1.0, 1, 1, 1]), (n, 4, 4)).copy()
    Pi = np.zeros((n, 4, 4))
    Phi = rng.standard_normal((n, 3, 4, 4))
    Phi = 0.5 * (Phi + np.swapaxes(Phi, -1, -2))
    Phi[:, :, 0, :] = 0.0
    Phi[:, :, :, 0] = 0.0
    return psi, Pi, Phi


def test_three_index_constraint_decays_at_rate_gamma2_on_minkowski():
    """alpha=1, beta=0, Pi=0, Phi_i0b=0 and d psi = 0: C_iab = -Phi_iab and the
    RHS gives d_t C_iab = -gamma2 C_iab exactly (linear damping)."""
    rng = np.random.default_rng(11)
    psi, Pi, Phi = _minkowski_point_state(rng)
    u = gh.pack_fields(psi, Pi, Phi)
    du = np.zeros(u.shape[:-1] + (3, 50))
    du[..., 20:] = rng.standard_normal(du[..., 20:].shape)   # d_k Phi arbitrary
    for g2 in [0.5, 1.0, 2.0]:
        r = gh.gh_rhs_pointwise(u, du, np.zeros((len(u), 4)), np.zeros((len(u), 3, 4)), 1.0, -1.0, g2)
        _, dPi, dPhi = gh.unpack_fields(r)
        dpsi_dt, _, _ = gh.unpack_fields(r)
        # d_t C_iab = d_i (d_t psi_ab) - d_t Phi_iab; d_t psi is spatially constant (0) here
        assert np.abs(dpsi_dt).max() < 1e-15
        assert np.abs(-dPhi - (-g2) * (-Phi)).max() < 1e-14


def test_gauge_constraint_damping_rates_on_minkowski():
    """psi = eta, Pi = Phi = 0, d H = 0 and H = h: C_a = h_a.  The gamma0 term
    gives d_t C_0 = -2 gamma0 C_0 and d_t C_i = -gamma0 C_i; checked by a
    directional derivative of the oracle's own C_a along its own RHS."""
    rng = np.random.default_rng(12)
    n = 5
    psi = np.broadcast_to(np.diag([-1.0, 1, 1, 1]), (n, 4, 4)).copy()
    u = gh.pack_fields(psi, np.zeros((n, 4, 4)), np.zeros((n, 3, 4, 4)))
    h = rng.standard_normal((n, 4))
    du = np.zeros((n, 3, 50))
    zero_dH = np.zeros((n, 3, 4))
    for g0 in [0.5, 1.0]:
        r = gh.gh_rhs_pointwise(u, du, h, zero_dH, g0, -1.0, 1.0)
        eps = 1e-6

        def C(v):
            p, P, F = gh.unpack_fields(v)
            s = gh.spacetime_split(p)
            _, Gam = gh.christoffel_first_kind(s, P, F)
            return gh.gauge_constraint(s, Gam, h)
        dC = (C(u + eps * r) - C(u - eps * r)) / (2 * eps)
        assert np.abs(dC[:, 0] - (-2 * g0) * h[:, 0]).max() < 1e-8
        assert np.abs(dC[:, 1:] - (-g0) * h[:, 1:]).max() < 1e-8


def test_gamma1_gamma2_terms_vanish_when_three_index_constraint_vanishes():
    """Every gamma1 and gamma2 term multiplies C_iab = d_i psi_ab - Phi_iab; with
    d psi = Phi the RHS does not depend on gamma1, gamma2."""
    X, Y, Z = _sample_points()
    g, dg, ddg = kerr_schild.metric_and_derivatives(X, Y, Z, 1.0, 0.6)
    psi, Pi, Phi = kerr_schild.gh_fields(g, dg)
    rng = np.random.default_rng(13)
    Pi = Pi + 0.01 * rng.standard_normal(Pi.shape)
    u = gh.pack_fields(psi, 0.5 * (Pi + np.swapaxes(Pi, -1, -2)), Phi)
    du = rng.standard_normal(u.shape[:-1] + (3, 50))
    du[..., 0:10] = u[..., None, 20:50].reshape(u.shape[:-1] + (3, 10))   # d_i psi = Phi_i
    H = rng.standard_normal((len(X), 4))
    dH = rng.standard_normal((len(X), 3, 4))
    r1 = gh.gh_rhs_pointwise(u, du, H, dH, 1.0, -1.0, 1.0)
    r2 = gh.gh_rhs_pointwise(u, du, H, dH, 1.0, 0.7, 3.0)
    assert np.abs(r1 - r2).max() < 1e-12 * np.abs(r1).max()


# ------------------------------------------------------ characteristic BCs
def test_characteristic_round_trip():
    X, Y, Z = _sample_points()
    g, dg, _ = kerr_schild.metric_and_derivatives(X, Y, Z, 1.0, 0.8)
    bg = gh.boundary_background(g, X, Y, Z)
    v = np.random.default_rng(4).standard_normal((len(X), 50))
    w = gh.to_char(v, bg, 1.0)
    back = gh.from_char(*w, bg, 1.0)
    psi, Pi, Phi = gh.unpack_fields(v)
    assert np.abs(back - v).max() < 1e-13
    assert abs(np.einsum("...i,...i->...", bg["n_dn"], bg["n_up"]) - 1.0).max() < 1e-14


@pytest.mark.parametrize("r_in,chi", [(1.8, 0.0), (1.3, 0.9)])
def test_all_speeds_point_into_the_hole_at_excision(r_in, chi):
    """Inside the horizon every characteristic speed along +R is <= 0, so the
    excision boundary needs no condition (the paper's no-op case, Sec. 5)."""
    g = grid.shell_grid(r_in, 10.0, 5, 7)
    X, Y, Z = grid.cartesian_coords(g)
    gm, _, _ = kerr_schild.metric_and_derivatives(X[0], Y[0], Z[0], 1.0, chi)
    bg = gh.boundary_background(gm, X[0], Y[0], Z[0])
    for v in gh.char_speeds(bg, -1.0):
        assert np.all(v <= 1e-15)


def test_outer_bc_zeroes_only_incoming_fields():
    g = grid.shell_grid(1.8, 10.0, 5, 3)
    X, Y, Z = grid.cartesian_coords(g)
    gm, _, _ = kerr_schild.metric_and_derivatives(X[-1], Y[-1], Z[-1], 1.0, 0.0)
    bg = gh.boundary_background(gm, X[-1], Y[-1], Z[-1])
    v = np.random.default_rng(8).standard_normal(X[-1].shape + (50,))
    out = gh.apply_outer_bc(v, bg, -1.0, 1.0)
    w_in = gh.to_char(v, bg, 1.0)
    w_out = gh.to_char(out, bg, 1.0)
    vpsi, v0, vp, vm = gh.char_speeds(bg, -1.0)
    assert np.all(vp > 0) and np.all(vm < 0) and np.all(v0 < 0) and np.all(vpsi == 0)
    assert np.abs(w_out[0] - w_in[0]).max() < 1e-13      # zero speed: untouched
    assert np.abs(w_out[2] - w_in[2]).max() < 1e-13      # outgoing: untouched
    assert np.abs(w_out[1]).max() < 1e-13 and np.abs(w_out[3]).max() < 1e-13


@pytest.mark.parametrize("gamma1", [-1.0, 0.5])
def test_interface_exchange_is_upwind_per_characteristic_family(gamma1):
    """At a shared radius outside the horizon (speeds of both signs), each
    characteristic family of the new time derivatives is, on both sides, the
    value of the side it comes from: the outer shell's where it moves inward
    (v < 0), the inner shell's where it moves outward (v > 0); a zero-speed
    family keeps each side's own value.  gamma1 = -1 gives v_psi = 0, gamma1 =
    0.5 an inward v_psi."""
    g = grid.shell_grid(3.0, 6.0, 5, 5)
    X, Y, Z = grid.cartesian_coords(g)
    gm, _, _ = kerr_schild.metric_and_derivatives(X[-1], Y[-1], Z[-1], 1.0, 0.7)
    bg = gh.boundary_background(gm, X[-1], Y[-1], Z[-1])
    rng = np.random.default_rng(14)
    a = rng.standard_normal(X[-1].shape + (50,))
    b = rng.standard_normal(X[-1].shape + (50,))
    na, nb = gh.apply_interface_bc(a, b, bg, gamma1, 1.0)
    wa, wb = gh.to_char(a, bg, 1.0), gh.to_char(b, bg, 1.0)
    wna, wnb = gh.to_char(na, bg, 1.0), gh.to_char(nb, bg, 1.0)
    speeds = gh.char_speeds(bg, gamma1)
    assert np.all(speeds[1] < 0) and np.all(speeds[2] > 0) and np.all(speeds[3] < 0)
    for q, v in enumerate(speeds):
        ext = v.reshape(v.shape + (1,) * (wa[q].ndim - v.ndim))
        want_a = np.where(ext < 0, wb[q], wa[q])        # inward: the outer side's value
        want_b = np.where(ext > 0, wa[q], wb[q])        # outward: the inner side's value
        assert np.abs(wna[q] - want_a).max() < 1e-12, q
        assert np.abs(wnb[q] - want_b).max() < 1e-12, q
    if gamma1 == -1.0:
        assert np.all(speeds[0] == 0)
        assert np.abs(wna[0] - wa[0]).max() < 1e-13 and np.abs(wnb[0] - wb[0]).max() < 1e-13
    else:
        assert np.all(speeds[0] < 0)
        assert np.abs(wna[0] - wb[0]).max() < 1e-13


def test_domain_boundaries_touch_only_boundary_slices_and_upwind_by_side():
    """ApplyBCs on a two-shell domain with random time derivatives: interior
    slices and the excision slice are untouched; at the shared radius the
    inner shell's outer slice and the outer shell's inner slice carry, per
    characteristic family, the outer shell's value where it moves inward and
    the inner shell's where it moves outward; at the outer boundary every
    incoming family is zero."""
    dom = evolve.Domain([(1.8, 4.0, 5, 5), (4.0, 8.0, 5, 5)], 1.0, 0.6)
    rng = np.random.default_rng(17)
    d = [rng.standard_normal((5, 50) + g["theta"].shape + g["phi"].shape) for g in dom.grids]
    out = evolve.apply_boundaries(dom, d)
    assert np.array_equal(out[0][:4], d[0][:4]) and np.array_equal(out[1][1:4], d[1][1:4])
    bg = dom.boundary_bg(0, 4)
    last = lambda a: np.moveaxis(a, 0, -1)
    wi, wo = gh.to_char(last(d[0][4]), bg, dom.gamma2), gh.to_char(last(d[1][0]), bg, dom.gamma2)
    ni, no = gh.to_char(last(out[0][4]), bg, dom.gamma2), gh.to_char(last(out[1][0]), bg, dom.gamma2)
    for q, v in enumerate(gh.char_speeds(bg, dom.gamma1)):
        ext = v.reshape(v.shape + (1,) * (wi[q].ndim - v.ndim))
        assert np.abs(ni[q] - np.where(ext < 0, wo[q], wi[q])).max() < 1e-12, q
        assert np.abs(no[q] - np.where(ext > 0, wi[q], wo[q])).max() < 1e-12, q
    bgo = dom.boundary_bg(1, 4)
    wout = gh.to_char(last(out[1][4]), bgo, dom.gamma2)
    for q, v in enumerate(gh.char_speeds(bgo, dom.gamma1)):
        ext = v.reshape(v.shape + (1,) * (wout[q].ndim - v.ndim))
        assert np.abs(np.where(ext < 0, wout[q], 0.0)).max() < 1e-12, q


# ------------------------------------------------- constraint energy (R13)
def test_constraint_energy_sums_the_rk4_decay_of_a_violation_on_flat_space():
    """E = sum_{n=1..N} dt sum_shells int sum_c C_c^2 dV on a closed form.

    Flat space (M = 0: alpha = 1, beta = 0, H = 0) with a small violation
    Phi_x,yz = delta exp(-((R - 6)/w)^2) and nothing else.  The linear GH
    system gives, already at the semi-discrete level, d_t C_iab = -gamma2
    C_iab and d_t C_ijab = -gamma2 C_ijab: both are linear in the state and
    the derivative maps cancel (C_iab exactly, C_ijab up to the commutator of
    the discrete derivatives, small on a resolved bump).  The gauge
    constraint starts at zero (the violation has no trace part and no time
    component) and grows only like t^2 (d_t Pi_yz = -d_x Phi_x,yz feeds
    Phi_y,yz and Phi_z,yz, whose trace enters Gamma_z), so its share of E is
    of order t^4: about 1e-8 over this run of t = 0.02.  The bump is four
    widths inside both boundaries, so no boundary condition acts.  Classic
    RK4 multiplies each decaying mode by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24
    per step, z = -gamma2 dt, so with E_0 the integrated squared constraints
    of the initial state, E = dt E_0 sum_{n=1..N} R(z)^(2n).  Summing from
    n = 0 instead misses by 0.4 %, dropping dt by a factor 500."""
    dom = evolve.Domain([(2.0, 10.0, 33, 3)], 0.0, 0.0, 1.0, -1.0, 1.0)
    g = dom.grids[0]
    X, Y, Z = grid.cartesian_coords(g)
    R = np.sqrt(X * X + Y * Y + Z * Z)
    u = dom.u_exact[0].copy()
    assert np.abs(u[:, 10:]).max() == 0.0                     # flat: Pi = Phi = 0
    u[:, 20 + gh.PAIRS.index((2, 3))] += 1e-8 * np.exp(-((R - 6.0) / 1.0) ** 2)
    cs, n0 = evolve.constraints(dom, [u])
    assert np.abs(cs[0][:, 0:4]).max() == 0.0 and n0[0] > 0.0
    dt, N = 0.002, 10
    z = -dom.gamma2 * dt
    Rz = 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0
    want = dt * n0[0] * sum(Rz ** (2 * n) for n in range(1, N + 1))
    E = evolve.constraint_energy(dom, [u], dt, N)
    assert abs(E - want) <= 1e-7 * want, (E, want)


# ------------------------------------------------------------------ RK4
def test_rk4_matches_stability_polynomial(monkeypatch):
    lam = -0.7 + 0.3j
    dt = 0.1

    def fake_rhs(dom, u):
        return [lam * a for a in u]

    class D:
        radial_filter_on = False
        sh_keep_l = -1
        grids = [None]
    monkeypatch.setattr(evolve, "rhs", fake_rhs)
    u = [np.ones(3, dtype=complex)]
    out = evolve.rk4_step(D(), u, dt)
    z = lam * dt
    assert abs(out[0][0] - (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)) < 1e-15


# ------------------------------------------------------------- perturbations
def _pulse_setup(M):
    from oracle import perturb
    g = grid.shell_grid(3.0, 8.0, 31, 11)
    u_bg, _, _ = kerr_schild.kerr_schild_shell(g, M, 0.0)
    coeffs = np.random.default_rng(41).standard_normal(len(spectral.sh_modes(2)))
    du = perturb.psi_pulse(g, u_bg, 1e-3, 5.5, 1.2, 2, coeffs)
    return g, u_bg, du, coeffs


def test_psi_pulse_phi_is_the_gradient_of_psi():
    """dPhi_iab = d_i dpsi_ab: against the oracle's spectral Cartesian gradient
    of dpsi on a grid that resolves the pulse (an independent route: radial
    Chebyshev and Y_lm derivatives instead of the chain rule on G(r) S)."""
    g, _, du, _ = _pulse_setup(1.0)
    grad = spectral.cartesian_gradient(du[:, 0:10], g)            # [3, n_r, 10, th, ph]
    for i in range(3):
        phi = du[:, 20 + 10 * i:30 + 10 * i]
        assert np.abs(grad[i] - phi).max() <= 1e-7 * np.abs(phi).max()
    # the same pulse on all ten components
    assert np.array_equal(du[:, 0], du[:, 7]) and np.array_equal(du[:, 20], du[:, 29])


def test_psi_pulse_is_ingoing_on_flat_space():
    """With M = 0 (alpha = 1, beta = 0) Pi_ab = -d_t psi_ab and an ingoing
    wave f(t + R) has d_t f = d_R f, so dPi must equal -d_R dpsi."""
    g, _, du, _ = _pulse_setup(0.0)
    dR = spectral.radial_derivative(du[:, 0:10], g)
    assert np.abs(du[:, 10:20] + dR).max() <= 1e-7 * np.abs(dR).max()


def test_pi_modes_recover_their_coefficients():
    """Y_lm analysis of each radial slice of the Pi mode perturbation returns
    exp(-((R - Rc)/w)^2) c_lm (l <= 3 < L, exact quadrature); psi and Phi
    are untouched."""
    from oracle import perturb
    g = grid.shell_grid(2.0, 9.0, 9, 7)
    coeffs = np.random.default_rng(42).standard_normal(len(spectral.sh_modes(3)))
    du = perturb.pi_modes(g, 4.0, 2.0, 3, coeffs)
    c = spectral.sh_analysis(du[:, 12], g)                            # [n_r, modes of L = 7]
    G = np.exp(-((g["r"] - 4.0) / 2.0) ** 2)
    ref = np.zeros_like(c)
    ref[:, :len(coeffs)] = G[:, None] * coeffs[None, :]
    assert np.abs(c - ref).max() <= 1e-12 * np.abs(ref).max()
    assert not du[:, 0:10].any() and not du[:, 20:].any()
