"""Seeded-coefficient perturbations added to the exact Kerr-Schild data (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's test problem is the stationary hole itself (Sec. 3.1); it adds
no perturbation.  The perturbations here make the synthetic workloads
non-trivial while keeping their structure (a smooth shell of radiation, or
angular modes on Pi).  Their coefficients are drawn by the seeded input
generator and passed in; this module only evaluates them.

Pulse on psi (ingoing Gaussian shell):
    dpsi_ab = A exp(-(R-Rc)^2/w^2) S(theta, phi),  S = sum_{l<=lmax} c_lm Y_lm,
    dPhi_iab = d_i dpsi_ab,
    dPi_ab = -(1/alpha)(d_R dpsi_ab - beta^k d_k dpsi_ab)   (background alpha, beta),
applied identically to all 10 components.
Mode perturbation on Pi:
    dPi_ab = exp(-((R-Rc)/w)^2) sum_{l<=lmax} c_lm Y_lm, all 10 components.
"""
import numpy as np

from . import grid, spectral, gh


def _angular_sum(g, coeffs, lmax):
    modes = spectral.sh_modes(lmax)
    assert len(coeffs) == len(modes)
    Y = spectral.real_ylm(lmax, g["theta"], g["phi"])
    dYt = spectral.real_ylm_dtheta(lmax, g["theta"], g["phi"])
    dYp = spectral.real_ylm_dphi(lmax, g["theta"], g["phi"])
    S = np.einsum("i,ijk->jk", coeffs, Y)
    St = np.einsum("i,ijk->jk", coeffs, dYt)
    Sp = np.einsum("i,ijk->jk", coeffs, dYp)
    return S, St, Sp


def psi_pulse(g, u_bg, A, Rc, w, lmax, coeffs):
    """Return the perturbation du[n_r, 50, n_th, n_ph] of the ingoing psi pulse."""
    S, St, Sp = _angular_sum(g, np.asarray(coeffs, float), lmax)
    r = g["r"][:, None, None]
    G = np.exp(-((r - Rc) / w) ** 2)
    dG = -2.0 * (r - Rc) / (w * w) * G
    f = A * G * S[None]                                   # [n_r, th, ph]
    fr = A * dG * S[None]
    fth = A * G * St[None]
    fph = A * G * Sp[None]
    J = spectral.spherical_jacobian(g)                    # [3, 3, n_r, th, ph]
    df = np.stack([J[i, 0] * fr + J[i, 1] * fth + J[i, 2] * fph for i in range(3)], axis=-1)
    psi_bg, _, _ = gh.unpack_fields(np.moveaxis(u_bg, 1, -1))
    s = gh.spacetime_split(psi_bg)
    bdf = np.einsum("...k,...k->...", s["beta_up"], df)
    pi = -(fr - bdf) / s["alpha"]
    du = np.zeros_like(u_bg)
    for p in range(10):
        du[:, p] = f
        du[:, 10 + p] = pi
        for i in range(3):
            du[:, 20 + 10 * i + p] = df[..., i]
    return du


def pi_modes(g, Rc, w, lmax, coeffs):
    """Return du[n_r, 50, n_th, n_ph] for the Pi mode perturbation."""
    S, _, _ = _angular_sum(g, np.asarray(coeffs, float), lmax)
    r = g["r"][:, None, None]
    G = np.exp(-((r - Rc) / w) ** 2)
    du = np.zeros((g["n_r"], 50, g["n_th"], g["n_ph"]))
    for p in range(10):
        du[:, 10 + p] = G * S[None]
    return du
