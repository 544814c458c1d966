"""Rotating dual frame (oracle): SpatialCoordJac and the time-dependent map.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's code evolves the fields at collocation points fixed in grid
coordinates while the equations are written in inertial coordinates, the two
related by a time-dependent map (Sec. 3.1, dual frame; Sec. 3.3 models the
SpatialCoordJac operation that applies the map's Jacobian to tensor
indices).  The map here is a rigid rotation about a unit axis e at rate
Omega: x = R(t) x_g with R(t) the rotation by the angle Omega t.  The evolved
variables are the inertial-frame components of the fields at the grid
points, so

    d/dt u(t, x_g) = F(u, d^I u) + xdot^k d^I_k u,
    d^I_k = R_kj d^g_j   (the map's Jacobian applied to the derivative index),
    xdot  = Omega e x x  (the grid velocity at the inertial position x),

with F the GH right-hand side of the inertial frame (``gh.gh_rhs_pointwise``)
and d^g the derivative in grid Cartesian coordinates (the static DiffJac).

The boundary conditions act on the inertial-frame time derivative F (the
freezing and upwind conditions are statements about the physical time
derivative at the boundary), and the grid-velocity term is added after
them: d/dt u = ApplyBCs(F) + xdot^k d^I_k u.  For the stationary hole this
gives exactly the rotation of its components.

Reading (the paper fixes no map): the background hole must be invariant
under rotations about e (Schwarzschild about any axis, Kerr about its spin
axis).  Then its gauge source and the boundary background at a moving grid
point are the t = 0 values with their tensor components rotated,
H_a(R x_g) = Lambda_a^b H_b(x_g), Lambda = diag(1, R), and the
characteristic speeds do not change (the grid velocity is tangential to the
spheres: n . xdot = 0).
"""
import numpy as np

from . import evolve, gh, grid, spectral


def rotation(axis, angle):
    """Rodrigues rotation matrix about the unit vector axis by angle."""
    e = np.asarray(axis, dtype=float)
    e = e / np.linalg.norm(e)
    K = np.array([[0.0, -e[2], e[1]], [e[2], 0.0, -e[0]], [-e[1], e[0], 0.0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def _lam(R):
    L = np.eye(4)
    L[1:, 1:] = R
    return L


def rotate_fields(u, R):
    """Rotate the tensor components of u[..., 50]: psi'_ab = L_ac L_bd psi_cd,
    Pi' likewise, Phi'_iab = R_ij L_ac L_bd Phi_jcd."""
    L = _lam(R)
    psi, Pi, Phi = gh.unpack_fields(u)
    psi2 = np.einsum("ac,bd,...cd->...ab", L, L, psi)
    Pi2 = np.einsum("ac,bd,...cd->...ab", L, L, Pi)
    Phi2 = np.einsum("ij,ac,bd,...jcd->...iab", R, L, L, Phi)
    return gh.pack_fields(psi2, Pi2, Phi2)


def rotate_gauge(H, dH, R):
    """H'_a = L_ab H_b, dH'_ia = R_ij L_ab dH_jb (H[..., 4], dH[..., 3, 4])."""
    L = _lam(R)
    return np.einsum("ab,...b->...a", L, H), np.einsum("ij,ab,...jb->...ia", R, L, dH)


def rotate_bg(bg, R):
    return dict(n_dn=np.einsum("ij,...j->...i", R, bg["n_dn"]), n_up=np.einsum("ij,...j->...i", R, bg["n_up"]),
                alpha=bg["alpha"], beta_up=np.einsum("ij,...j->...i", R, bg["beta_up"]))


def rhs(dom, u, t, axis, omega):
    """Moving-frame right-hand side at time t: ApplyBCs on the inertial-frame
    right-hand side, then the grid-velocity term at every point."""
    R = rotation(axis, omega * t)
    e = np.asarray(axis, dtype=float)
    e = e / np.linalg.norm(e)
    F, adv = [], []
    for s, us in enumerate(u):
        g = dom.grids[s]
        dug = spectral.cartesian_gradient(us, g)                  # [3, n_r, 50, th, ph], grid frame
        U = evolve._points_last(us)
        dUg = np.moveaxis(dug, (0, 2), (-2, -1))                  # [n_r, th, ph, 3, 50]
        dUi = np.einsum("kj,...jf->...kf", R, dUg)                 # inertial derivative index
        H = evolve._points_last(dom.H[s])
        dH = evolve._points_last(dom.dH[s]).reshape(U.shape[:-1] + (3, 4))
        Ht, dHt = rotate_gauge(H, dH, R)
        F.append(evolve._fields_axis1(gh.gh_rhs_pointwise(U, dUi, Ht, dHt, dom.gamma0, dom.gamma1, dom.gamma2)))
        X, Y, Z = grid.cartesian_coords(g)
        xg = np.stack([X, Y, Z], axis=-1)
        xi = np.einsum("kj,...j->...k", R, xg)
        xdot = omega * np.cross(np.broadcast_to(e, xi.shape), xi)
        adv.append(evolve._fields_axis1(np.einsum("...k,...kf->...f", xdot, dUi)))
    Fb = evolve.apply_boundaries(dom, F, u, bg_map=lambda bg: rotate_bg(bg, R))
    return [a + b for a, b in zip(Fb, adv)]


def rk4_step(dom, u, t, dt, axis, omega):
    """Classic RK4 in the moving frame (stage times t, t+dt/2, t+dt/2, t+dt);
    filters after the step."""
    k1 = rhs(dom, u, t, axis, omega)
    k2 = rhs(dom, [a + 0.5 * dt * k for a, k in zip(u, k1)], t + 0.5 * dt, axis, omega)
    k3 = rhs(dom, [a + 0.5 * dt * k for a, k in zip(u, k2)], t + 0.5 * dt, axis, omega)
    k4 = rhs(dom, [a + dt * k for a, k in zip(u, k3)], t + dt, axis, omega)
    new = [a + dt / 6.0 * (p + 2.0 * q + 2.0 * r + s) for a, p, q, r, s in zip(u, k1, k2, k3, k4)]
    return evolve.apply_filters(dom, new)


def exact_state(dom, t, axis, omega):
    """The stationary hole seen at the grid points at time t: its t = 0 values
    with rotated tensor components (the hole is invariant under the rotation)."""
    R = rotation(axis, omega * t)
    return [evolve._fields_axis1(rotate_fields(evolve._points_last(u0), R)) for u0 in dom.u_exact]


def exact_rate(dom, t, axis, omega, h=1e-4):
    """d/dt exact_state by a fourth-order central difference in t (the state
    is a trigonometric polynomial of degree 4 in Omega t)."""
    f = lambda tt: exact_state(dom, tt, axis, omega)
    a, b, c, d = f(t - 2 * h), f(t - h), f(t + h), f(t + 2 * h)
    return [(aa - 8 * bb + 8 * cc - dd) / (12 * h) for aa, bb, cc, dd in zip(a, b, c, d)]


# ------------------------------------------------------------ general maps
# The dual frame with a general affine map (Sec. 3.1: grid and inertial
# coordinates share the time and are related by a time-dependent map):
#
#     x = a(t) R(t) x_g + T(t),  a(t) = 1 + adot t,  R(t) = rotation(axis, Omega t),
#     T(t) = V t,
#
# an expansion, a rotation about any axis and a translation.  The evolved
# variables are again the inertial components at the grid points, so
#
#     d/dt u(t, x_g) = ApplyBCs(F(u, d^I u)) + xdot^k d^I_k u,
#     d^I_k = (1/a) R_kj d^g_j,   xdot = adot R x_g + a Omega e x (R x_g) + V.
#
# Reading (the paper fixes no map): the hole is not assumed symmetric under
# the map, so its gauge source and the boundary background are evaluated at
# the moving inertial points x (the analytic Kerr-Schild solution, as at
# t = 0); the boundary is the moving sphere |x - T| = a r, with its unit
# normal from x - T, and the characteristic speeds relative to it are the
# inertial ones minus n . xdot; the boundary conditions act on the inertial
# rate F as for the rotation (which this map reduces to when adot = 0, V = 0).

class AffineMap:
    """x = (1 + adot t) R(axis, Omega t) x_g + V t."""

    def __init__(self, axis=(0.0, 0.0, 1.0), omega=0.0, adot=0.0, V=(0.0, 0.0, 0.0)):
        e = np.asarray(axis, dtype=float)
        self.e = e / np.linalg.norm(e)
        self.omega, self.adot = float(omega), float(adot)
        self.V = np.asarray(V, dtype=float)

    def at(self, t):
        """(a, R, T) at time t."""
        return 1.0 + self.adot * t, rotation(self.e, self.omega * t), self.V * t

    def points(self, g, t):
        """Inertial positions x[n_r, th, ph, 3] of the grid points, and the
        grid velocity xdot there."""
        a, R, T = self.at(t)
        X, Y, Z = grid.cartesian_coords(g)
        xg = np.stack([X, Y, Z], axis=-1)
        Rx = np.einsum("kj,...j->...k", R, xg)
        x = a * Rx + T
        xdot = self.adot * Rx + a * self.omega * np.cross(np.broadcast_to(self.e, Rx.shape), Rx) + self.V
        return x, xdot


def _spin(dom):
    return dom.chi * dom.M if np.ndim(dom.chi) == 0 else tuple(float(c) * dom.M for c in dom.chi)


def _hole_at(dom, x):
    """The hole's metric, first and second derivatives at the points x[..., 3]."""
    from . import kerr_schild
    return kerr_schild.metric_and_derivatives(x[..., 0], x[..., 1], x[..., 2], dom.M, _spin(dom))


def map_gauge(dom, x):
    """H_a, d_i H_a of the hole at the inertial points x[..., 3]."""
    from . import kerr_schild
    return kerr_schild.gauge_source(*_hole_at(dom, x))


def map_bg(dom, s, ir, mp, t):
    """Boundary background of radial slice ir of shell s at time t: the hole's
    metric at the moving points, the unit normal of the moving sphere (from
    x - T), and n . xdot."""
    g = dom.grids[s]
    x, _ = mp.points(g, t)
    a, _, T = mp.at(t)
    gm, _, _ = _hole_at(dom, x[ir])
    xc = x[ir] - T
    bg = gh.boundary_background(gm, xc[..., 0], xc[..., 1], xc[..., 2])
    # the rotation moves the sphere within itself (its velocity is orthogonal
    # to x - T), so only the expansion and the translation move it along n
    radial = (mp.adot / a) * xc + mp.V
    bg["n_xdot"] = np.einsum("...i,...i->...", bg["n_dn"], radial)
    return bg


def rhs_map(dom, u, t, mp):
    """Right-hand side in the frame of the affine map mp at time t."""
    a, R, T = mp.at(t)
    F, adv = [], []
    for s, us in enumerate(u):
        g = dom.grids[s]
        dug = spectral.cartesian_gradient(us, g)                  # [3, n_r, 50, th, ph], grid frame
        U = evolve._points_last(us)
        dUg = np.moveaxis(dug, (0, 2), (-2, -1))                  # [n_r, th, ph, 3, 50]
        dUi = np.einsum("kj,...jf->...kf", R, dUg) / a             # inertial derivative index
        x, xdot = mp.points(g, t)
        H, dH = map_gauge(dom, x)
        F.append(evolve._fields_axis1(gh.gh_rhs_pointwise(U, dUi, H, dH, dom.gamma0, dom.gamma1, dom.gamma2)))
        adv.append(evolve._fields_axis1(np.einsum("...k,...kf->...f", xdot, dUi)))
    Fb = evolve.apply_boundaries(dom, F, u, bg_fn=lambda s, ir: map_bg(dom, s, ir, mp, t))
    return [p + q for p, q in zip(Fb, adv)]


def rk4_step_map(dom, u, t, dt, mp):
    """Classic RK4 in the frame of mp (stage times t, t+dt/2, t+dt/2, t+dt);
    filters after the step."""
    k1 = rhs_map(dom, u, t, mp)
    k2 = rhs_map(dom, [p + 0.5 * dt * k for p, k in zip(u, k1)], t + 0.5 * dt, mp)
    k3 = rhs_map(dom, [p + 0.5 * dt * k for p, k in zip(u, k2)], t + 0.5 * dt, mp)
    k4 = rhs_map(dom, [p + dt * k for p, k in zip(u, k3)], t + dt, mp)
    new = [p + dt / 6.0 * (q + 2.0 * r + 2.0 * w + z) for p, q, r, w, z in zip(u, k1, k2, k3, k4)]
    return evolve.apply_filters(dom, new)


def exact_state_map(dom, t, mp):
    """The stationary hole at the moving points: its fields at x(t, x_g)."""
    from . import kerr_schild
    out = []
    for g in dom.grids:
        x, _ = mp.points(g, t)
        gm, dg, _ = _hole_at(dom, x)
        psi, Pi, Phi = kerr_schild.gh_fields(gm, dg)
        out.append(evolve._fields_axis1(gh.pack_fields(psi, Pi, Phi)))
    return out


def exact_rate_map(dom, t, mp, h=1e-3):
    """d/dt exact_state_map by a sixth-order central difference in t."""
    f = lambda tt: exact_state_map(dom, tt, mp)
    m3, m2, m1, p1, p2, p3 = (f(t + c * h) for c in (-3, -2, -1, 1, 2, 3))
    return [(-a + 9 * b - 45 * c + 45 * d - 9 * e + q) / (60 * h) for a, b, c, d, e, q in zip(m3, m2, m1, p1, p2, p3)]
