"""Pins of the u^- part of the oracle's constraint-preserving outer condition
(outer_bc = "cp_full"; Sec. 5 names a constraint-preserving outer boundary,
the reading is in ``oracle.gh.uminus_constraint_part``) against what fixes it:

1. The derivative of the gauge constraint C_a that the condition uses is the
   derivative of the oracle's own C_a: central differences of
   ``constraints_pointwise`` along random directions.
2. The defining property of the Bjorhus form: the boundary u^- derivative does
   not hold u^-'s own normal derivative.  On exact Kerr-Schild data plus a
   perturbation of u^- alone that vanishes on the outer sphere but not its
   normal derivative, the interior D_t u^- at the boundary changes and the
   condition's u^- derivative does not (and with the condition written along
   the incoming null direction, or with its shift terms or its Bjorhus weight
   wrong, it would).
3. The u^- time derivative lies in the constraint subspace: S_ab l^b = 0 and
   its transverse traceless part vanishes (the gauge and physical parts stay
   frozen), with the null tetrad built here from the background's lapse,
   shift, spatial metric and normal.
4. The u^psi, u^0 and u^+ time derivatives are those of the "cp" condition.
"""
import numpy as np

from oracle import evolve, gh, grid


def _moveto(a):           # [50, th, ph] -> [th, ph, 50]
    return np.moveaxis(a, 0, -1)


def _perturbed_domain(outer_bc, chi=0.5, seed=3, amp=1e-3):
    dom = evolve.Domain([(2.5, 6.0, 9, 5)], M=1.0, chi=chi, gamma1=0.5, outer_bc=outer_bc)
    rng = np.random.default_rng(seed)
    u = dom.u_exact[0].copy()
    # smooth perturbation: low-order functions of the Cartesian coordinates with seeded weights
    X, Y, Z = grid.cartesian_coords(dom.grids[0])          # [n_r, th, ph]
    for f in range(50):
        c = rng.normal(size=4)
        u[:, f] += amp * (c[0] + c[1] * X / 6.0 + c[2] * Y * Z / 36.0 + c[3] * np.sin(0.7 * X + 0.3 * Z))
    return dom, [u]


def _outer_data(dom, u):
    s = len(dom.grids) - 1
    nr = dom.u_exact[s].shape[0]
    bg = dom.boundary_bg(s, nr - 1)
    ub = _moveto(u[s][nr - 1])
    dub = np.moveaxis(evolve.cartesian_derivatives(dom, u)[s][:, nr - 1], (0, 1), (-2, -1))
    Hb = _moveto(dom.H[s][nr - 1])
    dHb = _moveto(dom.dH[s][nr - 1]).reshape(Hb.shape[:-1] + (3, 4))
    return bg, ub, dub, Hb, dHb


def _C(u, H):
    return gh.constraints_pointwise(u, np.zeros(u.shape[:-1] + (3, 50)), H)[..., 0:4]


def _tetrad(bg):
    """The null tetrad and projector, built independently of the oracle."""
    N, beta, g = bg["alpha"], bg["beta_up"], bg["g_dn"]
    n_dn, n_up = bg["n_dn"], bg["n_up"]
    shp = N.shape
    psi4 = np.zeros(shp + (4, 4))
    bd = np.einsum("...ij,...j->...i", g, beta)
    psi4[..., 1:, 1:] = g
    psi4[..., 0, 1:] = psi4[..., 1:, 0] = bd
    psi4[..., 0, 0] = -N ** 2 + (beta * bd).sum(-1)
    psi4inv = np.linalg.inv(psi4)
    t_up = np.concatenate([1.0 / N[..., None], -beta / N[..., None]], axis=-1)
    n4_up = np.concatenate([np.zeros(shp + (1,)), n_up], axis=-1)
    l_up = (t_up + n4_up) / np.sqrt(2.0)
    k_up = (t_up - n4_up) / np.sqrt(2.0)
    l_dn = np.einsum("...ab,...b->...a", psi4, l_up)
    k_dn = np.einsum("...ab,...b->...a", psi4, k_up)
    # projector onto the 2-surface orthogonal to l and k (l.k = -1)
    P_mixed = np.eye(4) + np.einsum("...a,...b->...ab", l_up, k_dn) + np.einsum("...a,...b->...ab", k_up, l_dn)
    P_up = np.einsum("...ac,...cb->...ab", P_mixed, psi4inv)
    return l_up, k_up, l_dn, P_up, n_dn


def test_gauge_constraint_derivative_matches_central_differences():
    dom, u = _perturbed_domain("cp")
    rng = np.random.default_rng(11)
    U = _moveto(u[0][3])[1:3, 2:5]                         # a few interior points
    H = _moveto(dom.H[0][3])[1:3, 2:5]
    for trial in range(3):
        v = rng.normal(size=U.shape)
        w = rng.normal(size=H.shape)
        d = gh.gauge_constraint_derivative(U, v, H, w)
        h = 1e-6
        fd = (_C(U + h * v, H + h * w) - _C(U - h * v, H - h * w)) / (2 * h)
        assert np.abs(d - fd).max() <= 1e-7 * np.abs(d).max(), (trial, np.abs(d - fd).max())


def _uminus_only_perturbation(dom, eps=1e-3, seed=8):
    """d u with d Pi = d w / 2, d Phi_i = -n_i d w / 2 (d psi = 0) and
    d w_ab = eps (r_out - r) g_ab(theta, phi), with n the outer sphere's
    background normal carried along each radial line: on the outer sphere d u
    vanishes and its normal derivative is a pure u^- one (d u^psi, d u^+ and
    d u^0 have zero normal derivative there), and every factor is a low
    polynomial in r or a function of angle alone, so the spectral radial
    derivative is exact."""
    g = dom.grids[0]
    X, Y, Z = grid.cartesian_coords(g)
    R = np.sqrt(X * X + Y * Y + Z * Z)
    rng = np.random.default_rng(seed)
    nr = dom.u_exact[0].shape[0]
    du = np.zeros_like(dom.u_exact[0])
    r_out = R[-1].max()
    n = dom.boundary_bg(0, nr - 1)["n_dn"]                             # [th, ph, 3]
    for ir in range(nr):
        for p in range(10):
            c = rng.normal(size=3)
            dw = eps * (r_out - R[ir]) * (c[0] + c[1] * X[ir] / R[ir] + c[2] * Y[ir] * Z[ir] / R[ir] ** 2)
            du[ir, 10 + p] = 0.5 * dw
            for i in range(3):
                du[ir, 20 + 10 * i + p] = -0.5 * n[..., i] * dw
    return du


def test_uminus_condition_ignores_the_normal_derivative_of_uminus():
    dom = evolve.Domain([(2.5, 6.0, 9, 5)], M=1.0, chi=0.5, gamma1=0.5, outer_bc="cp_full")
    u = dom.u_exact[0]
    du = _uminus_only_perturbation(dom)
    bg = _outer_data(dom, [u])[0]
    out = {}
    for name, state in (("exact", u), ("perturbed", u + du)):
        dom.outer_bc = "freeze"
        interior = gh.to_char(_moveto(evolve.rhs_interior(dom, [state])[0][-1]), bg, dom.gamma2)
        dom.outer_bc = "cp_full"
        full = gh.to_char(_moveto(evolve.rhs(dom, [state])[0][-1]), bg, dom.gamma2)
        out[name] = interior, full
    d_int = [np.abs(a - b).max() for a, b in zip(out["exact"][0], out["perturbed"][0])]
    d_full = [np.abs(a - b).max() for a, b in zip(out["exact"][1], out["perturbed"][1])]
    assert d_int[3] > 1e-4                           # the interior D_t u^- sees the normal derivative
    assert max(d_int[:3]) <= 1e-10 * d_int[3]        # the other families do not (it vanishes on the sphere)
    assert max(d_full) <= 1e-10 * d_int[3], d_full   # the condition's u^- derivative does not either


def test_uminus_derivative_lies_in_the_constraint_subspace():
    dom, u = _perturbed_domain("cp_full", chi=0.7, seed=5)
    dudt = evolve.rhs(dom, u)
    bg = _outer_data(dom, u)[0]
    _, _, _, wm = gh.to_char(_moveto(dudt[-1][-1]), bg, dom.gamma2)
    l_up, k_up, l_dn, P_up, _ = _tetrad(bg)
    scale = np.abs(wm).max()
    assert scale > 1e-6                                      # not frozen
    assert np.abs(np.einsum("...ab,...b->...a", wm, l_up)).max() <= 1e-12 * scale
    PSP = np.einsum("...ac,...bd,...cd->...ab", P_up, P_up, wm)
    # the transverse traceless part: P^ac P^bd S_cd - (1/2) P^ab (P^cd S_cd)
    trace = np.einsum("...cd,...cd->...", P_up, wm)
    TT = PSP - 0.5 * P_up * trace[..., None, None]
    assert np.abs(TT).max() <= 1e-12 * scale
    # and it has a component along the transverse trace and along l l
    assert np.abs(trace).max() > 1e-3 * scale
    assert np.abs(np.einsum("...a,...b,...ab->...", k_up, k_up, wm)).max() > 1e-3 * scale


def test_other_families_keep_their_constraint_preserving_values():
    res = {}
    for mode in ("cp", "cp_full"):
        dom, u = _perturbed_domain(mode)
        dudt = evolve.rhs(dom, u)
        bg = _outer_data(dom, u)[0]
        res[mode] = gh.to_char(_moveto(dudt[-1][-1]), bg, dom.gamma2)
        interior = dudt[-1][:-1]
        res[mode + "_int"] = interior
    for q in range(3):                      # equal up to the rounding of the round trip through (Pi, Phi)
        assert np.abs(res["cp"][q] - res["cp_full"][q]).max() <= 1e-13 * np.abs(res["cp"][q]).max()
    assert np.array_equal(res["cp_int"], res["cp_full_int"])
    # "cp" freezes u^- (zero up to the round trip's rounding); "cp_full" does not
    assert np.abs(res["cp"][3]).max() <= 1e-12 * np.abs(res["cp_full"][3]).max()
