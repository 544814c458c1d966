"""Exact solution for tests: flat spacetime in time-dependent, non-linear
coordinates, x^mu = F^mu(t, x, y, z) close to the identity.

Its metric is g_ab = J^m_a eta_mn J^n_b with J = dF/dx.  With the gauge source
H_a = -Gamma_a of that metric every constraint of the first-order GH system
vanishes, so the exact time derivative of the fields is what the GH equations
must give.  Unlike stationary Kerr-Schild data it has d_t H_a != 0 and
psi^cd Pi_ca Pi_db != 0.  Test code only (the oracle pins and a GPU check use
it); nothing here is shared with the oracle or the library.
"""
import numpy as np

PAIRS = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def moving_minkowski_metric():
    """Lambdified (g, dg): g(t, x, y, z) -> 16 entries g_ab (row-major),
    dg(t, x, y, z) -> 64 entries d_c g_ab ([c][a][b])."""
    import sympy as sp
    t, x, y, z = c = sp.symbols("t x y z", real=True)
    F = [t + sp.Rational(1, 5) * sp.sin(t) * (1 + sp.Rational(3, 10) * x) + sp.Rational(1, 10) * x * y,
         x + sp.Rational(3, 20) * sp.sin(sp.Rational(7, 10) * t + y / 2),
         y + z * t / 10,
         z + t ** 2 / 20]
    J = sp.Matrix(4, 4, lambda m, a: sp.diff(F[m], c[a]))
    g = J.T * sp.diag(-1, 1, 1, 1) * J
    f_g = sp.lambdify(c, [g[a, b] for a in range(4) for b in range(4)], "numpy")
    f_dg = sp.lambdify(c, [sp.diff(g[a, b], v) for v in c for a in range(4) for b in range(4)], "numpy")
    return f_g, f_dg


def moving_minkowski_fields(f_g, f_dg, t, x, y, z):
    """(u[..., 50], H[..., 4], alpha[...]) at events (t, x, y, z) (scalars or
    arrays of one shape), from the exact metric and its exact first
    derivatives: Phi_iab = d_i g_ab, Pi_ab = -(d_t g_ab - beta^k Phi_kab)/alpha,
    H_a = -g^bc Gamma_abc with Gamma_abc = (d_b g_ac + d_c g_ab - d_a g_bc)/2."""
    shape = np.broadcast(t, x, y, z).shape

    def arr(vals, tail):
        return np.stack([np.broadcast_to(np.asarray(v, dtype=float), shape) for v in vals], -1).reshape(shape + tail)

    g = arr(f_g(t, x, y, z), (4, 4))
    dg = arr(f_dg(t, x, y, z), (4, 4, 4))                      # [..., c, a, b] = d_c g_ab
    gi3 = np.linalg.inv(g[..., 1:, 1:])
    b_up = np.einsum("...ij,...j->...i", gi3, g[..., 0, 1:])
    alpha = np.sqrt(np.einsum("...i,...i->...", b_up, g[..., 0, 1:]) - g[..., 0, 0])
    Phi = dg[..., 1:, :, :]
    Pi = -(dg[..., 0, :, :] - np.einsum("...k,...kab->...ab", b_up, Phi)) / alpha[..., None, None]
    Gam = 0.5 * (np.einsum("...bac->...abc", dg) + np.einsum("...cab->...abc", dg) - dg)
    H = -np.einsum("...bc,...abc->...a", np.linalg.inv(g), Gam)
    u = np.zeros(shape + (50,))
    for q, (a, b) in enumerate(PAIRS):
        u[..., q] = g[..., a, b]
        u[..., 10 + q] = Pi[..., a, b]
        for i in range(3):
            u[..., 20 + 10 * i + q] = Phi[..., i, a, b]
    return u, H, alpha


def central_diff(f, p, axis, h=2e-3):
    """8th-order central difference of f(p) along coordinate `axis` of p = [t, x, y, z]."""
    w = [1 / 280, -4 / 105, 1 / 5, -4 / 5, 0.0, 4 / 5, -1 / 5, 4 / 105, -1 / 280]
    acc = 0.0
    for j, c in enumerate(w):
        if c:
            q = list(p)
            q[axis] = q[axis] + (j - 4) * h
            acc = acc + c * np.asarray(f(q))
    return acc / h


def expected_rhs(f_g, f_dg, t, x, y, z):
    """(u, du[..., 3, 50], H, dH[..., 3, 4], want[..., 50]) at the events:
    want = d_t u plus, for Pi_ab, alpha (delta^0_a d_t H_b + delta^0_b d_t H_a),
    the part of -2 alpha nabla_(a H_b) that a right-hand side holding H fixed
    in time leaves out."""
    fields = lambda q: moving_minkowski_fields(f_g, f_dg, *q)[0]
    gauge = lambda q: moving_minkowski_fields(f_g, f_dg, *q)[1]
    p = [t, x, y, z]
    u, H, alpha = moving_minkowski_fields(f_g, f_dg, t, x, y, z)
    du = np.stack([central_diff(fields, p, 1 + k) for k in range(3)], axis=-2)
    dH = np.stack([central_diff(gauge, p, 1 + k) for k in range(3)], axis=-2)
    want = central_diff(fields, p, 0)
    dt_H = central_diff(gauge, p, 0)
    for q, (a, b) in enumerate(PAIRS):
        if a == 0:
            want[..., 10 + q] += alpha * dt_H[..., b]
        if b == 0:
            want[..., 10 + q] += alpha * dt_H[..., a]
    return u, du, H, dH, want
