"""The library's right-hand side on an exact solution of the GH system,
checked against the mathematics instead of the oracle: flat spacetime in
time-dependent, non-linear coordinates (tests/exact_solutions.py).  With the
gauge source H_a = -Gamma_a of that metric every constraint vanishes, so the
right-hand side must be the exact time derivative of the data, plus the d_t H
part of nabla_(a H_b) that a right-hand side holding H fixed in time leaves out
(exact_solutions.expected_rhs).  Unlike the stationary Kerr-Schild data, these
data have psi^cd Pi_ca Pi_db != 0 and a time-dependent lapse and shift.

Two shells share an interface, where the upwind exchange must leave the exact
values alone (both sides agree); the outermost slice carries the freezing
condition and is left out of the comparison."""
import numpy as np
import pytest

import exact_solutions
from oracle import grid
from parity_helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("alg", ["folded", "separable"])
def test_rhs_is_the_exact_time_derivative_of_flat_space_in_moving_coordinates(alg):
    from paper_1804_09101_gb300 import gh
    shells = [(2.0, 3.0, 15, 19), (3.0, 4.5, 15, 19)]     # truncation error about 2e-9 here
    t0 = 0.4
    f_g, f_dg = exact_solutions.moving_minkowski_metric()
    dom = gh.Domain(shells, 1.0, -1.0, 1.0)
    gh.gh_set_algorithm(dom, {"separable": gh.GH_ALG_SEPARABLE, "folded": gh.GH_ALG_SEPARABLE_FOLDED}[alg])
    state, Hs, dHs, wants = [], [], [], []
    for (r_in, r_out, n_r, L) in shells:
        g = grid.shell_grid(r_in, r_out, n_r, L)
        X, Y, Z = grid.cartesian_coords(g)                                   # [n_r, th, ph]
        u, du, H, dH, want = exact_solutions.expected_rhs(f_g, f_dg, np.full(X.shape, t0), X, Y, Z)
        state.append(np.moveaxis(u, -1, 1).ravel())                          # [r][field][th][ph]
        Hs.append(np.moveaxis(H, -1, 1).ravel())                             # [r][a][th][ph]
        dHs.append(np.moveaxis(dH.reshape(dH.shape[:-2] + (12,)), -1, 1).ravel())   # [r][4i+a][th][ph]
        wants.append(np.moveaxis(want, -1, 1))
    u = to_dev(np.concatenate(state))
    gh.gh_set_gauge(dom, to_dev(np.concatenate(Hs)), to_dev(np.concatenate(dHs)))
    gh.gh_set_background(dom, u)
    k = dom.new_state()
    gh.gh_rhs(dom, u, k)
    got = to_host(k)
    off = 0
    worst = 0.0
    for s, (r_in, r_out, n_r, L) in enumerate(shells):
        n = n_r * 50 * (L + 1) * 2 * (L + 1)
        gs = got[off:off + n].reshape(wants[s].shape)
        keep = slice(0, n_r - 1) if s == len(shells) - 1 else slice(0, n_r)   # all but the outer boundary
        worst = max(worst, float(np.abs(gs[keep] - wants[s][keep]).max()))
        off += n
    scale = max(float(np.abs(w).max()) for w in wants)
    assert scale > 0.05 and worst < 1e-8 * max(1.0, scale), (worst, scale)
