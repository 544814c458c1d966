"""Pins of the oracle's tensor spherical-harmonic filter (Sec. 3.1: filtering
in a shell through tensor spherical harmonics; Sec. 3.4: the filter couples
the tensor components), independent of its own formulas: the spin-weighted
harmonics reduce to scipy's Y_lm at s = 0 and obey the eth ladder; they are
orthonormal under the grid quadrature; rank 0 is the scalar truncation; vector
fields built from scalar harmonics with the oracle's own derivatives (radial
Y r_hat, gradient, curl) pass unchanged below the cut and vanish above it,
where the per-component scalar filter does neither; the filter is idempotent
and real."""
import numpy as np
import pytest
from scipy.special import sph_harm_y

from oracle import grid, spectral, tensor_filter as tf


def test_spin_zero_is_scipy_ylm_and_eth_raises_spin():
    th = np.array([0.3, 1.1, 2.5])
    ph = np.array([0.4, 2.0, 5.5])
    for l in range(5):
        for m in range(-l, l + 1):
            assert np.abs(tf.swsh(0, l, m, th, ph) - sph_harm_y(l, m, th, ph)).max() < 1e-12
    e = 1e-6
    for s in range(3):
        for l in range(s + 1, 6):
            for m in range(-l, l + 1):
                d = (tf.swsh(s, l, m, th + e, ph) - tf.swsh(s, l, m, th - e, ph)) / (2 * e)
                v = tf.swsh(s, l, m, th, ph)
                eth = -(d - s / np.tan(th) * v + 1j / np.sin(th) * (1j * m) * v)
                ref = np.sqrt((l - s) * (l + s + 1)) * tf.swsh(s + 1, l, m, th, ph)
                assert np.abs(eth - ref).max() < 1e-6


def test_orthonormal_under_grid_quadrature():
    g = grid.shell_grid(2.0, 3.0, 3, 7)
    th, ph = g["theta"][:, None], g["phi"][None, :]
    w = g["wth"][:, None] * 2 * np.pi / len(g["phi"])
    for s in (0, 1, -2, 3):
        modes = [(l, m) for l in range(abs(s), 8) for m in range(-l, l + 1)]
        Y = [tf.swsh(s, l, m, th, ph) for l, m in modes]
        G = np.array([[np.sum(w * np.conj(a) * b) for b in Y] for a in Y])
        assert np.abs(G - np.eye(len(modes))).max() < 1e-12


def test_rank_zero_is_the_scalar_truncation():
    g = grid.shell_grid(2.0, 3.0, 3, 7)
    rng = np.random.default_rng(1)
    f = rng.standard_normal((1, 1, len(g["theta"]), len(g["phi"])))
    a = tf.tensor_filter(f[0, 0], 0, g, 4)
    b = spectral.sh_truncation_filter(f, g, 4)[0, 0]
    assert np.abs(a - b).max() < 1e-12


def _vector_fields(g, l, m):
    """Radial Y r_hat, gradient r grad Y and curl r_hat x r grad Y of the real Y_lm."""
    L = g["L"]
    th, ph = g["theta"], g["phi"]
    modes = spectral.sh_modes(L)
    i = modes.index((l, m))
    Y = spectral.real_ylm(L, th, ph)[i]
    dY = spectral.real_ylm_dtheta(L, th, ph)[i]
    dP = spectral.real_ylm_dphi(L, th, ph)[i]
    E, _ = tf.frame(g)
    rhat = E[0].real
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    cp, sp = np.cos(ph)[None, :], np.sin(ph)[None, :]
    that = np.stack([ct * cp, ct * sp, -st * np.ones_like(cp)])
    phat = np.stack([-sp * np.ones_like(st), cp * np.ones_like(st), 0 * st * cp])
    grad = that * dY + phat * dP / st
    curl = np.cross(rhat, grad, axis=0)
    return rhat * Y, grad, curl


@pytest.mark.parametrize("l,m", [(2, 1), (3, -2), (4, 0)])
def test_vector_harmonics_pass_below_and_vanish_above_the_cut(l, m):
    g = grid.shell_grid(2.0, 3.0, 3, 9)
    for kind, V in zip(("radial", "gradient", "curl"), _vector_fields(g, l, m)):
        assert np.abs(tf.tensor_filter(V, 1, g, l) - V).max() < 1e-12
        assert np.abs(tf.tensor_filter(V, 1, g, l - 1)).max() < 1e-12
        comp = np.stack([spectral.sh_truncation_filter(V[i][None, None], g, l)[0, 0] for i in range(3)])
        if kind == "curl":
            # x x grad Y_lm = i L Y_lm: Cartesian components of degree l, kept by both filters
            assert np.abs(comp - V).max() < 1e-12
        else:
            # components of degree l + 1: the per-component scalar filter changes the field
            assert np.abs(comp - V).max() > 1e-3


def test_rank_two_and_three_products_of_harmonics():
    g = grid.shell_grid(2.0, 3.0, 3, 9)
    _, g1, c1 = _vector_fields(g, 2, 1)
    r2, g2, _ = _vector_fields(g, 1, -1)
    T = np.einsum("i...,j...->ij...", g1, c1)              # spin 0, +-2 parts, degree <= 4
    assert np.abs(tf.tensor_filter(T, 2, g, 4) - T).max() < 1e-12
    R = np.einsum("i...,j...,k...->ijk...", g2, g1, r2)    # degree <= 1 + 2 + 1
    assert np.abs(tf.tensor_filter(R, 3, g, 4) - R).max() < 1e-12


def test_idempotent_and_real_on_random_fields():
    g = grid.shell_grid(2.0, 3.0, 3, 7)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((50, len(g["theta"]), len(g["phi"])))
    a = tf.filter_fields(u, g, 4)
    b = tf.filter_fields(a, g, 4)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()
    assert np.abs(a - u).max() > 0.1
