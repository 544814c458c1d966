"""Analytic Kerr-Schild data for one spinning black hole (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper evolves analytic Kerr-Schild data for an isolated hole of mass m
and dimensionless spin chi (Sec. 3.1, Eq. dimensionlessspin) but does not
print the metric.  This module writes out the standard Kerr-Schild form,
with the spin along +z and a = chi * M:

    g_ab = eta_ab + 2 H l_a l_b,
    H    = M r^3 / (r^4 + a^2 z^2),
    l_a  = (1, (r x + a y)/(r^2 + a^2), (r y - a x)/(r^2 + a^2), z / r),
    r^2  = (R^2 - a^2)/2 + sqrt((R^2 - a^2)^2 / 4 + a^2 z^2),  R^2 = x^2+y^2+z^2.

First and second spatial derivatives come from sympy's symbolic
differentiation of exactly these expressions, evaluated with numpy
(lambdify): the definition written out, no hand-derived derivative.

For a spin vector a = chi M (any direction; the paper's own test uses
chi = (0.2, 0.3, 0.4), Sec. 3.1) the same form reads, with a.x the Euclidean
dot product and a x x the cross product,

    H    = M r^3 / (r^4 + (a.x)^2),
    l_i  = (r x_i - (a x x)_i + (a.x) a_i / r) / (r^2 + a^2),
    r^2  = (R^2 - a^2)/2 + sqrt((R^2 - a^2)^2 / 4 + (a.x)^2),

which reduces to the expressions above for a along +z.

From the metric the GH evolved fields and the gauge source follow:
    psi_ab   = g_ab,
    Phi_iab  = d_i g_ab,
    Pi_ab    = (1/alpha) beta^i Phi_iab           (stationary: d_t g_ab = 0),
    H_a      = -Gamma_a  (so the gauge constraint C_a = H_a + Gamma_a is 0),
    d_i H_a  = -d_i Gamma_a,  d_t H_a = 0.
"""
import functools

import numpy as np
import sympy as sp

from . import gh


@functools.lru_cache(maxsize=1)
def _lambdified():
    x, y, z, M, a = sp.symbols("x y z M a", real=True)
    R2 = x * x + y * y + z * z
    r2 = (R2 - a * a) / 2 + sp.sqrt((R2 - a * a) ** 2 / 4 + a * a * z * z)
    r = sp.sqrt(r2)
    H = M * r ** 3 / (r ** 4 + a * a * z * z)
    l = [sp.Integer(1), (r * x + a * y) / (r2 + a * a), (r * y - a * x) / (r2 + a * a), z / r]
    eta = sp.diag(-1, 1, 1, 1)
    X = [x, y, z]
    g, dg, ddg = [], [], []
    for A in range(4):
        for B in range(A, 4):
            gab = eta[A, B] + 2 * H * l[A] * l[B]
            g.append(gab)
            row = []
            for i in range(3):
                d = sp.diff(gab, X[i])
                dg.append(d)
                for j in range(i, 3):
                    row.append(sp.diff(d, X[j]))
            ddg.append(row)
    # ddg flattened: for each (A<=B): pairs (i<=j) -> 6 entries
    ddg_flat = [e for row in ddg for e in row]
    f_g = sp.lambdify((x, y, z, M, a), g, modules="numpy", cse=True)
    f_dg = sp.lambdify((x, y, z, M, a), dg, modules="numpy", cse=True)
    f_ddg = sp.lambdify((x, y, z, M, a), ddg_flat, modules="numpy", cse=True)
    return f_g, f_dg, f_ddg


@functools.lru_cache(maxsize=1)
def _lambdified_vector():
    x, y, z, M, ax, ay, az = sp.symbols("x y z M ax ay az", real=True)
    R2 = x * x + y * y + z * z
    a2 = ax * ax + ay * ay + az * az
    ad = ax * x + ay * y + az * z
    r2 = (R2 - a2) / 2 + sp.sqrt((R2 - a2) ** 2 / 4 + ad * ad)
    r = sp.sqrt(r2)
    H = M * r ** 3 / (r ** 4 + ad * ad)
    X = [x, y, z]
    A = [ax, ay, az]
    cross = [ay * z - az * y, az * x - ax * z, ax * y - ay * x]
    l = [sp.Integer(1)] + [(r * X[i] - cross[i] + ad * A[i] / r) / (r2 + a2) for i in range(3)]
    eta = sp.diag(-1, 1, 1, 1)
    g, dg, ddg = [], [], []
    for P in range(4):
        for Q in range(P, 4):
            gab = eta[P, Q] + 2 * H * l[P] * l[Q]
            g.append(gab)
            for i in range(3):
                d = sp.diff(gab, X[i])
                dg.append(d)
                for j in range(i, 3):
                    ddg.append(sp.diff(d, X[j]))
    args = (x, y, z, M, ax, ay, az)
    return (sp.lambdify(args, g, modules="numpy", cse=True), sp.lambdify(args, dg, modules="numpy", cse=True),
            sp.lambdify(args, ddg, modules="numpy", cse=True))


_PAIRS = [(A, B) for A in range(4) for B in range(A, 4)]


def metric_and_derivatives(X, Y, Z, M, a):
    """g[..., 4, 4], dg[..., 3, 4, 4] (d_i g_ab), ddg[..., 3, 3, 4, 4] (d_i d_j g_ab).

    a: the spin parameter along +z (a scalar), or a spin vector (3 numbers)."""
    if np.ndim(a) == 0:
        f_g, f_dg, f_ddg = _lambdified()
        args = (X, Y, Z, M, a)
    else:
        f_g, f_dg, f_ddg = _lambdified_vector()
        args = (X, Y, Z, M) + tuple(float(c) for c in a)
    shp = np.shape(X)
    one = np.ones(shp)
    gv = [np.asarray(v) * one for v in f_g(*args)]
    dgv = [np.asarray(v) * one for v in f_dg(*args)]
    ddgv = [np.asarray(v) * one for v in f_ddg(*args)]
    g = np.zeros(shp + (4, 4))
    dg = np.zeros(shp + (3, 4, 4))
    ddg = np.zeros(shp + (3, 3, 4, 4))
    ij = [(i, j) for i in range(3) for j in range(i, 3)]
    for p, (A, B) in enumerate(_PAIRS):
        g[..., A, B] = g[..., B, A] = gv[p]
        for i in range(3):
            dg[..., i, A, B] = dg[..., i, B, A] = dgv[3 * p + i]
        for q, (i, j) in enumerate(ij):
            v = ddgv[6 * p + q]
            ddg[..., i, j, A, B] = ddg[..., i, j, B, A] = v
            ddg[..., j, i, A, B] = ddg[..., j, i, B, A] = v
    return g, dg, ddg


def gauge_source(g, dg, ddg):
    """H_a = -Gamma_a and d_i H_a = -d_i Gamma_a of a stationary metric.

    Gamma_abc = (d_b g_ac + d_c g_ab - d_a g_bc)/2 with d_0 = 0, and
    Gamma_a = g^{bc} Gamma_abc.  Its spatial derivative is
    d_i Gamma_a = (d_i g^{bc}) Gamma_abc + g^{bc} d_i Gamma_abc, where
    d_i g^{bc} = -g^{bd} (d_i g_de) g^{ec}.
    Returns H[..., 4] and dH[..., 3, 4] (d_i H_a).
    """
    shp = g.shape[:-2]
    D = np.zeros(shp + (4, 4, 4))          # D[c, a, b] = d_c g_ab, c spacetime
    D[..., 1:, :, :] = dg
    DD = np.zeros(shp + (3, 4, 4, 4))      # DD[i, c, a, b] = d_i d_c g_ab
    DD[..., :, 1:, :, :] = ddg
    ginv = np.linalg.inv(g)
    Gam = 0.5 * (np.einsum("...bac->...abc", D) + np.einsum("...cab->...abc", D)
                 - np.einsum("...abc->...abc", D))
    Gam_a = np.einsum("...bc,...abc->...a", ginv, Gam)
    dGam = 0.5 * (np.einsum("...ibac->...iabc", DD) + np.einsum("...icab->...iabc", DD)
                  - np.einsum("...iabc->...iabc", DD))
    dginv = -np.einsum("...bd,...ide,...ec->...ibc", ginv, dg, ginv)
    dGam_a = (np.einsum("...ibc,...abc->...ia", dginv, Gam)
              + np.einsum("...bc,...iabc->...ia", ginv, dGam))
    return -Gam_a, -dGam_a


def gh_fields(g, dg):
    """(psi[...,4,4], Pi[...,4,4], Phi[...,3,4,4]) of a stationary metric."""
    split = gh.spacetime_split(g)
    alpha, beta_up = split["alpha"], split["beta_up"]
    Pi = np.einsum("...i,...iab->...ab", beta_up, dg) / alpha[..., None, None]
    return g.copy(), Pi, dg.copy()


def kerr_schild_shell(g_shell, M, chi):
    """Exact KS data on one shell grid (a = chi M; chi a number: spin along +z,
    or a dimensionless spin vector of 3 numbers).

    Returns (u[n_r, 50, n_th, n_ph], H[n_r, 4, n_th, n_ph], dH[n_r, 12, n_th, n_ph]);
    dH is ordered dH[4*i + a] = d_i H_a.
    """
    from . import grid
    X, Y, Z = grid.cartesian_coords(g_shell)
    a = chi * M if np.ndim(chi) == 0 else tuple(float(c) * M for c in chi)
    g, dg, ddg = metric_and_derivatives(X, Y, Z, M, a)
    psi, Pi, Phi = gh_fields(g, dg)
    H, dH = gauge_source(g, dg, ddg)
    u = gh.pack_fields(psi, Pi, Phi)                    # [n_r, n_th, n_ph, 50]
    u = np.moveaxis(u, -1, 1)
    Hs = np.moveaxis(H, -1, 1)
    dHs = np.moveaxis(dH.reshape(dH.shape[:-2] + (12,)), -1, 1)
    return u, Hs, dHs
