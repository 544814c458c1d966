"""Tensor spherical-harmonic truncation filter on S2 shells (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's S2 filter acts on tensors through tensor spherical harmonics, so
that all components of a tensor are truncated consistently in angular
resolution; in its implementation the filter couples the tensor components
(Sec. 3.1, and the CSR filter matrix of Sec. 3.4).  The paper does not write
the harmonics out.  Reading used here: express every Cartesian index of a
rank-n spatial tensor in the local complex frame

    E_0 = r_hat,  E_+ = m = (theta_hat + i phi_hat)/sqrt(2),  E_- = conj(m),

so that each frame component c_A = T_{i1..in} E_{A1}^{i1} .. E_{An}^{in} has
spin weight s = (number of m) - (number of conj(m)); expand c_A in
spin-weighted harmonics sY_lm (l >= |s|), keep l <= L_f, and rebuild
T' = sum_A c'_A conj(E_{A1}) x .. x conj(E_{An}) (conj(E) is the dual basis).
A rank-0 tensor gets the scalar Y_lm truncation.  sY_lm follow the explicit
formula of Goldberg et al. (1967); for s = 0 they are the complex Y_lm with
the Condon-Shortley phase, and eth raises s (both pinned in the tests).
Analysis is by quadrature on the Gauss-Legendre x uniform grid, which is
exact for l, l' <= L.

The GH fields split into tensors of the spatial rotation group:
psi_00, Pi_00 (rank 0), psi_0i, Pi_0i, Phi_i00 (rank 1), psi_ij, Pi_ij
(rank 2, symmetric), Phi_i0j (rank 2), Phi_ijk (rank 3, symmetric in jk).
"""
import itertools
from math import comb, factorial, pi, sqrt

import numpy as np

from . import gh

PAIR = {(a, b): p for p, (a, b) in enumerate(gh.PAIRS)}


def swsh(s, l, m, theta, phi):
    """Spin-weighted spherical harmonic sY_lm(theta, phi) (Goldberg et al. 1967)."""
    theta = np.asarray(theta, dtype=float)
    if abs(s) > l or abs(m) > l:
        return np.zeros(np.broadcast(theta, phi).shape, dtype=complex)
    pref = (-1) ** m * sqrt(factorial(l + m) * factorial(l - m) * (2 * l + 1)
                            / (4 * pi * factorial(l + s) * factorial(l - s)))
    cot = 1.0 / np.tan(theta / 2)
    acc = 0.0
    for r in range(0, l - s + 1):
        k = r + s - m
        if 0 <= k <= l + s:
            acc = acc + comb(l - s, r) * comb(l + s, k) * (-1) ** (l - r - s) * cot ** (2 * r + s - m)
    return pref * np.sin(theta / 2) ** (2 * l) * acc * np.exp(1j * m * np.asarray(phi))


def frame(g):
    """E[A][i] on the (theta, phi) grid of shell grid g: A = 0 (r_hat), 1 (m), 2 (conj m)."""
    th = g["theta"][:, None]
    ph = g["phi"][None, :]
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    rhat = np.stack([st * cp, st * sp, ct * np.ones_like(cp)])
    that = np.stack([ct * cp, ct * sp, -st * np.ones_like(cp)])
    phat = np.stack([-sp * np.ones_like(th), cp * np.ones_like(th), 0 * th * cp])
    m = (that + 1j * phat) / sqrt(2.0)
    return np.stack([rhat.astype(complex), m, np.conj(m)]), [0, 1, -1]


def spin_project(f, s, Lf, g):
    """Projection of the spin-s function f[th, ph] onto sY_lm, |s| <= l <= Lf."""
    th = g["theta"][:, None]
    ph = g["phi"][None, :]
    w = g["wth"][:, None] * (2 * pi / len(g["phi"]))
    out = np.zeros(f.shape, dtype=complex)
    for l in range(abs(s), Lf + 1):
        for m in range(-l, l + 1):
            Y = swsh(s, l, m, th, ph)
            a = np.sum(w * np.conj(Y) * f)
            out = out + a * Y
    return out


def tensor_filter(T, rank, g, Lf):
    """Filter a rank-n Cartesian tensor field T[3, .., 3, th, ph] (real)."""
    if rank == 0:
        return spin_project(T.astype(complex), 0, Lf, g).real
    E, spin = frame(g)
    out = np.zeros(T.shape, dtype=complex)
    for A in itertools.product(range(3), repeat=rank):
        c = np.zeros(T.shape[rank:], dtype=complex)
        for I in itertools.product(range(3), repeat=rank):
            w = T[I].astype(complex)
            for k in range(rank):
                w = w * E[A[k]][I[k]]
            c = c + w
        s = sum(spin[a] for a in A)
        c2 = spin_project(c, s, Lf, g)
        for I in itertools.product(range(3), repeat=rank):
            w = c2
            for k in range(rank):
                w = w * np.conj(E[A[k]][I[k]])
            out[I] = out[I] + w
    return out.real


def filter_fields(u, g, Lf):
    """Tensor filter of one radial slice u[50, th, ph] of the GH fields."""
    out = np.zeros_like(u)
    for base in (0, 10):                                     # psi, Pi
        out[base + PAIR[(0, 0)]] = tensor_filter(u[base + PAIR[(0, 0)]], 0, g, Lf)
        V = np.stack([u[base + PAIR[(0, 1 + i)]] for i in range(3)])
        V2 = tensor_filter(V, 1, g, Lf)
        for i in range(3):
            out[base + PAIR[(0, 1 + i)]] = V2[i]
        T = np.stack([np.stack([u[base + PAIR[(min(i, j) + 1, max(i, j) + 1)]] for j in range(3)])
                      for i in range(3)])
        T2 = tensor_filter(T, 2, g, Lf)
        for i in range(3):
            for j in range(i, 3):
                out[base + PAIR[(i + 1, j + 1)]] = T2[i, j]
    phi = lambda i, p: u[20 + 10 * i + p]
    V = np.stack([phi(i, PAIR[(0, 0)]) for i in range(3)])
    V2 = tensor_filter(V, 1, g, Lf)
    T = np.stack([np.stack([phi(i, PAIR[(0, 1 + j)]) for j in range(3)]) for i in range(3)])
    T2 = tensor_filter(T, 2, g, Lf)
    R3 = np.stack([np.stack([np.stack([phi(i, PAIR[(min(j, k) + 1, max(j, k) + 1)]) for k in range(3)])
                             for j in range(3)]) for i in range(3)])
    R32 = tensor_filter(R3, 3, g, Lf)
    for i in range(3):
        out[20 + 10 * i + PAIR[(0, 0)]] = V2[i]
        for j in range(3):
            out[20 + 10 * i + PAIR[(0, 1 + j)]] = T2[i, j]
            for k in range(j, 3):
                out[20 + 10 * i + PAIR[(j + 1, k + 1)]] = R32[i, j, k]
    return out


def filter_state(dom, u, Lf):
    """Tensor filter of every radial slice of every shell (u[s][n_r, 50, th, ph])."""
    return [np.stack([filter_fields(us[r], g, Lf) for r in range(us.shape[0])]) for us, g in zip(u, dom.grids)]
