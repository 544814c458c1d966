"""Naive spectral transforms on one shell (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper's description of spectral operations (Sec. 3.4):
collocation values are mapped to spectral coefficients (Eq. PhysToSpec),
an operation is applied to the coefficients (Eq. Deriv for derivatives, a
filter function for filtering), and the result is mapped back (Eq.
SpecToPhys).  On a shell the expansion is in T_k(r) Y_lm(theta, phi)
(Sec. 3.4, the I1 x S2 expansion), and the differentiator has one radial and
two angular parts (Eq. DifferentiatorI1S2).

Every operation here is computed as an explicit analysis sum followed by an
explicit synthesis sum: the oracle never folds them into one matrix.

Array convention: a shell function has shape [n_r, ..., n_th, n_ph]; the
radial axis is axis 0 and the two angular axes are the last two.
"""
import numpy as np


# ---------------------------------------------------------------- Chebyshev
def cheb_T(k, x):
    """Chebyshev polynomial T_k(x) = cos(k arccos x) for |x| <= 1."""
    return np.cos(k * np.arccos(np.clip(x, -1.0, 1.0)))


def cheb_analysis(u, x):
    """Coefficients a_k of u on the CGL points x (Eq. PhysToSpec).

    a_k = 2 / ((N-1) cbar_k) * sum_j u_j T_k(x_j) / cbar_j,
    cbar_0 = cbar_{N-1} = 2, cbar_j = 1 otherwise.  Axis 0 of u is radial.
    """
    n = len(x)
    cbar = np.ones(n)
    cbar[0] = cbar[-1] = 2.0
    a = np.zeros_like(u, dtype=float)
    for k in range(n):
        acc = np.zeros(u.shape[1:])
        for j in range(n):
            acc = acc + u[j] * cheb_T(k, x[j]) / cbar[j]
        a[k] = 2.0 / ((n - 1) * cbar[k]) * acc
    return a


def cheb_synthesis(a, x):
    """Values sum_k a_k T_k(x_j) at the points x (Eq. SpecToPhys)."""
    n = a.shape[0]
    out = np.zeros((len(x),) + a.shape[1:])
    for j in range(len(x)):
        acc = np.zeros(a.shape[1:])
        for k in range(n):
            acc = acc + a[k] * cheb_T(k, x[j])
        out[j] = acc
    return out


def cheb_derivative_coeffs(a):
    """Coefficients b of du/dx from the coefficients a of u (Eq. Deriv).

    Uses T'_{k+1}/(k+1) - T'_{k-1}/(k-1) = 2 T_k, which gives the backward
    recurrence cbar_k b_k = b_{k+2} + 2 (k+1) a_{k+1}, with b_{N-1} = b_N = 0
    and cbar_0 = 2, cbar_k = 1 for k > 0.
    """
    n = a.shape[0]
    b = np.zeros((n + 2,) + a.shape[1:])
    for k in range(n - 2, -1, -1):
        cb = 2.0 if k == 0 else 1.0
        b[k] = (b[k + 2] + 2.0 * (k + 1) * a[k + 1]) / cb
    return b[:n]


def radial_derivative(u, g):
    """d u / d r on the shell g (axis 0 of u is radial).

    d/dr = (2 / (r_out - r_in)) d/dx for the affine map r(x).
    """
    a = cheb_analysis(u, g["x"])
    b = cheb_derivative_coeffs(a)
    return cheb_synthesis(b, g["x"]) * (2.0 / (g["r_out"] - g["r_in"]))


def expcheb_sigma(n, alpha, order):
    """Exponential Chebyshev filter factors sigma_k = exp(-alpha (k/(n-1))^order)."""
    k = np.arange(n)
    return np.exp(-alpha * (k / (n - 1.0)) ** order)


def radial_filter(u, g, alpha, order):
    """Exponential Chebyshev filter along r: T_k -> sigma_k T_k (Sec. 3.4, ExpCheb)."""
    a = cheb_analysis(u, g["x"])
    s = expcheb_sigma(len(g["x"]), alpha, order)
    a = a * s.reshape((-1,) + (1,) * (a.ndim - 1))
    return cheb_synthesis(a, g["x"])


# ------------------------------------------------------ spherical harmonics
def assoc_legendre_normalized(L, theta):
    """Normalised associated Legendre functions Pbar_l^m(cos theta), 0<=m<=l<=L.

    Pbar is normalised so that Y_l0 = Pbar_l^0 and the real harmonics below
    are orthonormal on the unit sphere; no Condon-Shortley phase.  Built by
    the standard three-term recurrence in l at fixed m, seeded by the
    diagonal Pbar_m^m.  theta may be complex (used for complex-step
    differentiation), so only analytic operations are used.
    Returns an array P[l, m, ...theta shape].
    """
    theta = np.asarray(theta)
    ct = np.cos(theta)
    st = np.sin(theta)
    P = np.zeros((L + 1, L + 1) + theta.shape, dtype=np.result_type(theta, float))
    P[0, 0] = np.sqrt(1.0 / (4.0 * np.pi))
    for m in range(1, L + 1):
        P[m, m] = np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * P[m - 1, m - 1]
    for m in range(0, L):
        P[m + 1, m] = np.sqrt(2.0 * m + 3.0) * ct * P[m, m]
    for m in range(0, L + 1):
        for l in range(m + 2, L + 1):
            a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            P[l, m] = a * (ct * P[l - 1, m] - b * P[l - 2, m])
    return P


def sh_modes(L):
    """The (l, m) list of real harmonics with l <= L, m = -l..l."""
    return [(l, m) for l in range(L + 1) for m in range(-l, l + 1)]


def _phi_factor(m, phi):
    if m == 0:
        return np.ones_like(phi)
    if m > 0:
        return np.sqrt(2.0) * np.cos(m * phi)
    return np.sqrt(2.0) * np.sin(-m * phi)


def _dphi_factor(m, phi):
    if m == 0:
        return np.zeros_like(phi)
    if m > 0:
        return -np.sqrt(2.0) * m * np.sin(m * phi)
    return np.sqrt(2.0) * (-m) * np.cos(-m * phi)


def real_ylm(L, theta, phi):
    """Real orthonormal Y_lm on the grid: Y[mode, j, k] for modes sh_modes(L).

    Y_l0 = Pbar_l^0, Y_lm = sqrt(2) Pbar_l^m cos(m phi) (m > 0),
    Y_l,-m = sqrt(2) Pbar_l^m sin(m phi).
    """
    P = assoc_legendre_normalized(L, theta)
    modes = sh_modes(L)
    Y = np.zeros((len(modes), len(theta), len(phi)))
    for i, (l, m) in enumerate(modes):
        Y[i] = P[l, abs(m)][:, None] * _phi_factor(m, phi)[None, :]
    return Y


def real_ylm_dtheta(L, theta, phi, h=1e-30):
    """d Y_lm / d theta by complex-step differentiation of Pbar (exact to rounding).

    dP/dtheta = Im(P(theta + i h)) / h; no subtraction, so no cancellation.
    """
    P = assoc_legendre_normalized(L, np.asarray(theta) + 1j * h)
    dP = P.imag / h
    modes = sh_modes(L)
    Y = np.zeros((len(modes), len(theta), len(phi)))
    for i, (l, m) in enumerate(modes):
        Y[i] = dP[l, abs(m)][:, None] * _phi_factor(m, phi)[None, :]
    return Y


def real_ylm_dphi(L, theta, phi):
    """d Y_lm / d phi, from the analytic derivative of the phi factor."""
    P = assoc_legendre_normalized(L, theta)
    modes = sh_modes(L)
    Y = np.zeros((len(modes), len(theta), len(phi)))
    for i, (l, m) in enumerate(modes):
        Y[i] = P[l, abs(m)][:, None] * _dphi_factor(m, phi)[None, :]
    return Y


def sh_analysis(u, g):
    """Coefficients c_lm = sum_jk w_j (2 pi / N_phi) Y_lm(theta_j, phi_k) u_jk.

    The last two axes of u are (theta, phi); returns [..., mode].
    """
    Y = real_ylm(g["L"], g["theta"], g["phi"])
    w = g["wth"][:, None] * g["wphi"]
    return np.einsum("...jk,ijk->...i", u, Y * w[None])


def sh_synthesis(c, B):
    """sum_mode c[..., mode] B[mode, j, k] for a basis table B (Y or a derivative)."""
    return np.einsum("...i,ijk->...jk", c, B)


def angular_derivatives(u, g):
    """(d u/d theta, d u/d phi) of the projection of u onto Y_lm, l <= L.

    The paper's angular parts of Eq. DifferentiatorI1S2: analysis onto the
    harmonics, then synthesis of the derivative of each harmonic.
    """
    c = sh_analysis(u, g)
    dth = sh_synthesis(c, real_ylm_dtheta(g["L"], g["theta"], g["phi"]))
    dph = sh_synthesis(c, real_ylm_dphi(g["L"], g["theta"], g["phi"]))
    return dth, dph


def sh_truncation_filter(u, g, keep_l):
    """Heaviside filter in l: drop every Y_lm with l > keep_l, then synthesise."""
    c = sh_analysis(u, g)
    modes = sh_modes(g["L"])
    mask = np.array([1.0 if l <= keep_l else 0.0 for (l, m) in modes])
    return sh_synthesis(c * mask, real_ylm(g["L"], g["theta"], g["phi"]))


# ------------------------------------------------------------- DiffJac
def spherical_jacobian(g):
    """J[i, d] = d(r, theta, phi)_d / d x^i on the grid, shape [3, 3, n_r, n_th, n_ph].

    Standard spherical coordinates x = r sin th cos ph, y = r sin th sin ph,
    z = r cos th.  This is the paper's DiffJac contraction (Sec. 3.3, Eq.
    DiffJac) for the map from (r, theta, phi) to Cartesian coordinates.
    """
    r = g["r"][:, None, None]
    st = g["sth"][None, :, None]
    ct = g["cth"][None, :, None]
    cp = np.cos(g["phi"])[None, None, :]
    sp = np.sin(g["phi"])[None, None, :]
    one = np.ones((g["n_r"], g["n_th"], g["n_ph"]))
    J = np.zeros((3, 3) + one.shape)
    J[0, 0] = st * cp * one
    J[1, 0] = st * sp * one
    J[2, 0] = ct * one
    J[0, 1] = ct * cp / r * one
    J[1, 1] = ct * sp / r * one
    J[2, 1] = -st / r * one
    J[0, 2] = -sp / (r * st) * one
    J[1, 2] = cp / (r * st) * one
    J[2, 2] = 0.0 * one
    return J


def cartesian_gradient(u, g):
    """d_i u (i = x, y, z) of a shell function u[n_r, ..., n_th, n_ph].

    Radial and angular derivatives (Eq. DifferentiatorI1S2), then the DiffJac
    contraction d_i u = J[i, d] d_d u (Eq. DiffJac).  Returns [3, *u.shape].
    """
    dr = radial_derivative(u, g)
    dth, dph = angular_derivatives(u, g)
    J = spherical_jacobian(g)
    extra = u.ndim - 3

    def bc(a):
        return a.reshape(a.shape[:1] + (1,) * extra + a.shape[1:])

    out = np.zeros((3,) + u.shape)
    for i in range(3):
        out[i] = bc(J[i, 0]) * dr + bc(J[i, 1]) * dth + bc(J[i, 2]) * dph
    return out
