"""Collocation grids and quadrature weights of one spherical shell (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A shell is the product topology I1 x S2 of the paper (Sec. 3.4, the
paragraph introducing spherical shells with the spectral expansion in
T_k(r) Y_lm(theta, phi)).  The paper does not fix the collocation points;
this oracle uses the standard choices for that expansion:

* radial: N_r Chebyshev-Gauss-Lobatto (CGL) points x_j = -cos(pi j/(N_r-1)),
  mapped affinely to [r_in, r_out]; Clenshaw-Curtis weights;
* polar: N_theta = L+1 Gauss-Legendre points in cos(theta), theta ascending;
* azimuthal: N_phi = 2(L+1) uniform points phi_k = 2 pi k / N_phi.

Grid functions are stored as arrays indexed [r][theta][phi] (phi fastest).
"""
import numpy as np


def cgl_nodes(n):
    """CGL points on [-1, 1], ascending: x_j = -cos(pi j / (n-1))."""
    j = np.arange(n)
    return -np.cos(np.pi * j / (n - 1))


def clenshaw_curtis_weights(n):
    """Clenshaw-Curtis weights for the n CGL points (exact for degree <= n-1).

    w_j = (c_j / N) * (1 - sum_{k=1}^{floor(N/2)} b_k cos(2 pi j k / N) / (4k^2 - 1))
    with N = n-1, c_0 = c_N = 1 and c_j = 2 otherwise, b_k = 1 for k = N/2 and
    2 otherwise.  The formula is symmetric in j -> N-j, so it holds for the
    ascending ordering as well.
    """
    N = n - 1
    w = np.zeros(n)
    for j in range(n):
        s = 0.0
        for k in range(1, N // 2 + 1):
            b = 1.0 if 2 * k == N else 2.0
            s += b * np.cos(2.0 * np.pi * j * k / N) / (4.0 * k * k - 1.0)
        c = 1.0 if j in (0, N) else 2.0
        w[j] = c / N * (1.0 - s)
    return w


def gauss_legendre(n):
    """Gauss-Legendre nodes/weights on [-1, 1] (library routine), ascending in x."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def shell_grid(r_in, r_out, n_r, L):
    """Return a dict with the 1-D coordinates and weights of one shell.

    Keys: x (CGL), r, wr (Clenshaw-Curtis, in x), theta (ascending), cth, sth,
    wth (Gauss-Legendre weight of each theta point), phi, wphi (scalar).
    The end points of r are set to r_in / r_out exactly so that shells that
    share a radius share bit-identical boundary coordinates.
    """
    x = cgl_nodes(n_r)
    r = 0.5 * (r_in + r_out) + 0.5 * (r_out - r_in) * x
    r[0] = r_in
    r[-1] = r_out
    wr = clenshaw_curtis_weights(n_r)
    nth = L + 1
    mu, wmu = gauss_legendre(nth)
    # theta ascending  <=>  cos(theta) descending
    cth = mu[::-1].copy()
    wth = wmu[::-1].copy()
    theta = np.arccos(cth)
    sth = np.sqrt(1.0 - cth * cth)
    nph = 2 * (L + 1)
    phi = 2.0 * np.pi * np.arange(nph) / nph
    return dict(r_in=r_in, r_out=r_out, n_r=n_r, L=L, n_th=nth, n_ph=nph,
                x=x, r=r, wr=wr, theta=theta, cth=cth, sth=sth, wth=wth,
                phi=phi, wphi=2.0 * np.pi / nph)


def cartesian_coords(g):
    """Cartesian (x, y, z) of every point, each shaped [n_r, n_th, n_ph]."""
    r = g["r"][:, None, None]
    st = g["sth"][None, :, None]
    ct = g["cth"][None, :, None]
    cp = np.cos(g["phi"])[None, None, :]
    sp = np.sin(g["phi"])[None, None, :]
    X = r * st * cp
    Y = r * st * sp
    Z = r * ct * np.ones_like(cp)
    return X, Y, Z


def volume_weights(g):
    """Quadrature weight of each point for integrals over the shell volume.

    dV = r^2 dr dOmega, dr = (r_out - r_in)/2 dx, dOmega = d(cos theta) dphi.
    """
    wr = g["wr"] * 0.5 * (g["r_out"] - g["r_in"]) * g["r"] ** 2
    return wr[:, None, None] * g["wth"][None, :, None] * g["wphi"] * np.ones(
        (1, 1, g["n_ph"]))
