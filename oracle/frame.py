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
