"""Pins of the oracle's constraint-preserving outer boundary condition
(Bjorhus form for the u^psi and u^0 families; Sec. 5 names the condition, the
GH literature gives it) against two properties that fix its form:

1. The correction is a multiple of the constraints: on data that satisfy
   C_iab = 0 and C_ijab = 0 exactly, the incoming u^psi and u^0 time
   derivatives keep their interior values (freezing would zero them).
2. It removes the incoming normal derivative: a perturbation that vanishes on
   the boundary sphere but has a normal derivative there changes the interior
   D_t u^0 (and D_t u^psi) at the boundary, but not the constraint-preserving
   values.
"""
import numpy as np

from oracle import evolve, gh, grid, spectral


def _moveto(a):           # [50, th, ph] -> [th, ph, 50]
    return np.moveaxis(a, 0, -1)


def _outer(dom, u, dudt_int, mode):
    dom.outer_bc = mode
    out = evolve.apply_boundaries(dom, dudt_int, u)
    return _moveto(out[-1][-1])


def _nr(dom):
    return dom.u_exact[-1].shape[0]


def _bg(dom):
    return dom.boundary_bg(len(dom.grids) - 1, _nr(dom) - 1)


def test_correction_vanishes_on_constraint_satisfying_data():
    dom = evolve.Domain([(2.0, 6.0, 9, 5)], M=1.0, chi=0.0, gamma1=0.5)
    g = dom.grids[0]
    X, Y, Z = grid.cartesian_coords(g)             # [n_r, th, ph]
    eps = 1e-2
    # psi = Minkowski + eps * quadratic polynomial; Phi = d psi exactly; Pi smooth
    P = [X * Y, Y + Z * Z, X * Z, 1.0 + X * X, Y * Z, X - Y, Z, X * Y * 0.5, Y * Y, X * Z - Y]
    dP = [[Y, X, 0 * X], [0 * X, 1 + 0 * X, 2 * Z], [Z, 0 * X, X], [2 * X, 0 * X, 0 * X], [0 * X, Z, Y],
          [1 + 0 * X, -1 + 0 * X, 0 * X], [0 * X, 0 * X, 1 + 0 * X], [0.5 * Y, 0.5 * X, 0 * X],
          [0 * X, 2 * Y, 0 * X], [Z, -1 + 0 * X, X]]
    eta = np.zeros(10)
    eta[0], eta[4], eta[7], eta[9] = -1.0, 1.0, 1.0, 1.0
    shape = dom.u_exact[0].shape
    u = np.zeros(shape)
    for p in range(10):
        u[:, p] = eta[p] + eps * P[p]
        u[:, 10 + p] = 0.3 * eps * np.sin(X + 0.5 * p) * np.cos(Y)
        for i in range(3):
            u[:, 20 + 10 * i + p] = eps * dP[p][i]
    # constraints of this state vanish to rounding
    du = spectral.cartesian_gradient(u, g)
    assert np.abs(du[:, :, 0:10] - np.stack([u[:, 20:30], u[:, 30:40], u[:, 40:50]])).max() < 1e-12
    dudt = evolve.rhs_interior(dom, [u])
    cp = _outer(dom, [u], dudt, "cp")
    fr = _outer(dom, [u], dudt, "freeze")
    bg = _bg(dom)
    D = gh.to_char(_moveto(dudt[0][-1]), bg, dom.gamma2)
    W = gh.to_char(cp, bg, dom.gamma2)
    F = gh.to_char(fr, bg, dom.gamma2)
    v_psi, v_0, v_p, v_m = gh.char_speeds(bg, dom.gamma1)
    assert (v_0 < 0).any()
    scale = np.abs(D[1]).max()
    assert scale > 1e-6
    # incoming u^0 and u^psi keep their interior values; u^- is frozen in both
    assert np.abs(W[1] - D[1]).max() < 1e-11 * max(1.0, scale)
    inc = (v_psi < 0)
    assert np.abs((W[0] - D[0])[inc]).max() < 1e-11
    assert np.abs(F[1][(v_0 < 0)]).max() < 1e-14 * scale
    assert np.abs(W[3][(v_m < 0)]).max() < 1e-14 * scale


def _normal_derivative_case(field):
    dom = evolve.Domain([(1.8, 10.0, 11, 7)], M=1.0, chi=0.0, gamma1=0.5)
    g = dom.grids[0]
    X, Y, Z = grid.cartesian_coords(g)
    R = np.sqrt(X * X + Y * Y + Z * Z)
    Rout = 10.0
    h = 1e-3 * (R - Rout)                  # vanishes on the outer sphere, dh/dR = 1e-3
    u0 = dom.u_exact[0].copy()
    u1 = u0.copy()
    E = np.linspace(0.3, 1.2, 10)
    if field == "Phi":
        # delta Phi_iab = h (delta_ik - x_i x_k / R^2) E_ab
        x = [X / R, Y / R, Z / R]
        for i in range(3):
            for k in range(3):
                Pik = (1.0 if i == k else 0.0) - x[i] * x[k]
                for p in range(10):
                    u1[:, 20 + 10 * i + p] += h * Pik * E[p] * (1.0 + 0.1 * k)
    else:
        for p in range(10):
            u1[:, p] += h * E[p]
    return dom, u0, u1


def test_constraint_preserving_u0_removes_the_normal_derivative():
    dom, u0, u1 = _normal_derivative_case("Phi")
    bg = _bg(dom)
    d0, d1 = evolve.rhs_interior(dom, [u0]), evolve.rhs_interior(dom, [u1])
    D0 = gh.to_char(_moveto(d0[0][-1]), bg, dom.gamma2)[1]
    D1 = gh.to_char(_moveto(d1[0][-1]), bg, dom.gamma2)[1]
    W0 = gh.to_char(_outer(dom, [u0], d0, "cp"), bg, dom.gamma2)[1]
    W1 = gh.to_char(_outer(dom, [u1], d1, "cp"), bg, dom.gamma2)[1]
    change = np.abs(D1 - D0).max()
    assert change > 1e-5                      # the interior equation sees the normal derivative
    assert np.abs(W1 - W0).max() < 1e-9 * change * 1e3


def test_constraint_preserving_upsi_removes_the_normal_derivative():
    dom, u0, u1 = _normal_derivative_case("psi")
    bg = _bg(dom)
    v_psi = gh.char_speeds(bg, dom.gamma1)[0]
    assert (v_psi < 0).all()                  # gamma1 = 0.5: u^psi is incoming at the outer boundary
    d0, d1 = evolve.rhs_interior(dom, [u0]), evolve.rhs_interior(dom, [u1])
    D0 = gh.to_char(_moveto(d0[0][-1]), bg, dom.gamma2)[0]
    D1 = gh.to_char(_moveto(d1[0][-1]), bg, dom.gamma2)[0]
    W0 = gh.to_char(_outer(dom, [u0], d0, "cp"), bg, dom.gamma2)[0]
    W1 = gh.to_char(_outer(dom, [u1], d1, "cp"), bg, dom.gamma2)[0]
    change = np.abs(D1 - D0).max()
    assert change > 1e-5
    assert np.abs(W1 - W0).max() < 1e-9 * change * 1e3
