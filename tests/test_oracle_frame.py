"""Pins of the oracle's rotating dual frame (Sec. 3.1 dual frame, Sec. 3.3
SpatialCoordJac): with no rotation it is the static right-hand side; the
stationary hole seen from the rotating grid (its components rotating in
time) has a moving-frame right-hand side equal to its exact time derivative,
to truncation error that falls with resolution, and dropping the grid-velocity
term or the Jacobian breaks that; rotations compose."""
import numpy as np
import pytest

from oracle import evolve, frame


def _err(dom, t, axis, omega):
    u = frame.exact_state(dom, t, axis, omega)
    r = frame.rhs(dom, u, t, axis, omega)
    ref = frame.exact_rate(dom, t, axis, omega)
    scale = max(np.abs(x).max() for x in ref)
    return max(np.abs(a - b).max() for a, b in zip(r, ref)) / scale, scale


def test_no_rotation_is_the_static_rhs():
    dom = evolve.Domain([(1.8, 6.0, 9, 5)], M=1.0, chi=0.6)
    u = [x + 1e-6 for x in dom.u_exact]
    a = frame.rhs(dom, u, 0.37, (0.0, 0.0, 1.0), 0.0)
    b = evolve.rhs(dom, u)
    assert max(np.abs(x - y).max() for x, y in zip(a, b)) < 1e-14


def test_rotations_compose_and_preserve_the_metric_determinant():
    dom = evolve.Domain([(1.8, 6.0, 5, 3)], M=1.0, chi=0.0)
    u = evolve._points_last(dom.u_exact[0])
    R1 = frame.rotation((0.2, 0.3, 0.9), 0.7)
    R2 = frame.rotation((1.0, -0.4, 0.1), -1.3)
    a = frame.rotate_fields(frame.rotate_fields(u, R1), R2)
    b = frame.rotate_fields(u, R2 @ R1)
    assert np.abs(a - b).max() < 1e-13
    from oracle import gh
    psi, _, _ = gh.unpack_fields(a)
    assert np.abs(np.linalg.det(psi) + 1.0).max() < 1e-12


@pytest.mark.parametrize("M,chi,axis", [(1.0, 0.0, (0.3, -0.5, 0.8)), (1.0, 0.7, (0.0, 0.0, 1.0))])
def test_rotating_exact_solution_matches_its_time_derivative(M, chi, axis):
    omega, t = 0.3, 0.8
    errs = []
    for n_r, L in [(7, 5), (13, 11)]:
        dom = evolve.Domain([(2.0, 5.0, n_r, L)], M=M, chi=chi)
        e, scale = _err(dom, t, axis, omega)
        errs.append(e)
    assert scale > 1e-2                         # the components really rotate
    assert errs[1] < 3e-3 and errs[1] < 0.05 * errs[0]   # truncation error, falling with resolution
    # without the grid-velocity term (or with the static Jacobian) the residual is O(1)
    dom = evolve.Domain([(2.0, 5.0, 13, 11)], M=M, chi=chi)
    u = frame.exact_state(dom, t, axis, omega)
    ref = frame.exact_rate(dom, t, axis, omega)
    scale = max(np.abs(x).max() for x in ref)
    static = evolve.rhs(dom, u)
    assert max(np.abs(a - b).max() for a, b in zip(static, ref)) / scale > 0.1


# ------------------------------------------------------------ general maps
MAPS = {"expand+translate+tilted rotation": dict(axis=(0.3, -0.5, 0.8), omega=0.3, adot=0.05, V=(0.02, -0.03, 0.04)),
        "contraction+translation": dict(axis=(0.0, 0.0, 1.0), omega=0.0, adot=-0.04, V=(-0.05, 0.0, 0.03))}


def _map_err(dom, t, mp):
    u = frame.exact_state_map(dom, t, mp)
    r = frame.rhs_map(dom, u, t, mp)
    ref = frame.exact_rate_map(dom, t, mp)
    scale = max(np.abs(x).max() for x in ref)
    return max(np.abs(a - b).max() for a, b in zip(r, ref)) / scale, scale


@pytest.mark.parametrize("name", sorted(MAPS))
def test_moving_exact_solution_matches_its_time_derivative_under_a_general_map(name):
    """A spinning hole (spin 0.6 along z, not symmetric under the map) seen
    from a grid that expands or contracts, translates and rotates about a
    tilted axis: the moving-frame right-hand side equals the exact time
    derivative of its values at the moving points, to truncation error that
    falls with resolution; the static Jacobian or no grid velocity leaves an
    O(1) residual."""
    mp = frame.AffineMap(**MAPS[name])
    t = 0.8
    errs = []
    for n_r, L in [(7, 5), (13, 11)]:
        dom = evolve.Domain([(2.0, 5.0, n_r, L)], M=1.0, chi=0.6)
        e, scale = _map_err(dom, t, mp)
        errs.append(e)
    assert scale > 1e-2
    assert errs[1] < 2e-3 and errs[1] < 0.05 * errs[0], errs
    dom = evolve.Domain([(2.0, 5.0, 13, 11)], M=1.0, chi=0.6)
    u = frame.exact_state_map(dom, t, mp)
    ref = frame.exact_rate_map(dom, t, mp)
    scale = max(np.abs(x).max() for x in ref)
    static = frame.rhs_map(dom, u, t, frame.AffineMap())          # the identity map at the moved state
    assert max(np.abs(a - b).max() for a, b in zip(static, ref)) / scale > 0.1


def test_general_map_without_expansion_or_translation_is_the_rotating_frame():
    """adot = 0 and V = 0 about the spin axis of a Kerr hole: the gauge source
    and background evaluated at the rotated points equal the rotated stored
    ones, so the general map's right-hand side is the rotating frame's."""
    dom = evolve.Domain([(2.0, 5.0, 9, 7), (5.0, 8.0, 9, 7)], M=1.0, chi=0.7)
    rng = np.random.default_rng(41)
    u = [x + 1e-5 * rng.standard_normal(x.shape) for x in dom.u_exact]
    a = frame.rhs_map(dom, u, 0.9, frame.AffineMap(axis=(0.0, 0.0, 1.0), omega=0.4))
    b = frame.rhs(dom, u, 0.9, (0.0, 0.0, 1.0), 0.4)
    scale = max(np.abs(x).max() for x in b)
    assert max(np.abs(x - y).max() for x, y in zip(a, b)) <= 1e-11 * scale


def test_identity_map_is_the_static_rhs():
    dom = evolve.Domain([(2.0, 5.0, 9, 7), (5.0, 8.0, 9, 7)], M=1.0, chi=0.5)
    rng = np.random.default_rng(42)
    u = [x + 1e-5 * rng.standard_normal(x.shape) for x in dom.u_exact]
    a = frame.rhs_map(dom, u, 0.6, frame.AffineMap())
    b = evolve.rhs(dom, u)
    scale = max(np.abs(x).max() for x in b)
    assert max(np.abs(x - y).max() for x, y in zip(a, b)) <= 1e-11 * scale


def test_a_boundary_outrunning_every_family_freezes_them_all():
    """An outer sphere expanding faster than the fastest outgoing speed has
    every characteristic family incoming relative to it, so ApplyBCs sets the
    whole inertial rate there to zero; with no expansion only the incoming
    families are set to zero."""
    from oracle import gh
    dom = evolve.Domain([(2.0, 5.0, 7, 5)], M=1.0, chi=0.3)
    rng = np.random.default_rng(43)
    F = [rng.standard_normal(x.shape) for x in dom.u_exact]
    t = 0.0
    fast = frame.AffineMap(adot=1.0)                 # n . xdot = r_out = 5 at t = 0
    bg = frame.map_bg(dom, 0, 6, fast, t)
    assert min(np.min(v) for v in gh.char_speeds(bg, dom.gamma1)) < 0
    assert max(np.max(v) for v in gh.char_speeds(bg, dom.gamma1)) < 0
    out = evolve.apply_boundaries(dom, F, None, bg_fn=lambda s, ir: frame.map_bg(dom, s, ir, fast, t))
    assert np.abs(out[0][6]).max() == 0.0 and np.abs(out[0][5] - F[0][5]).max() == 0.0
    still = evolve.apply_boundaries(dom, F, None, bg_fn=lambda s, ir: frame.map_bg(dom, s, ir, frame.AffineMap(), t))
    assert np.abs(still[0][6]).max() > 0.1


def test_translated_boundary_normal_points_from_the_moving_centre():
    """Under a pure translation the boundary sphere is |x - T| = r: its normal
    at the grid point x_g is along x_g (normalised with the metric at x), and
    n . xdot = n . V."""
    dom = evolve.Domain([(2.0, 5.0, 5, 3)], M=1.0, chi=0.5)
    mp = frame.AffineMap(V=(0.3, -0.2, 0.25))
    t = 1.7
    bg = frame.map_bg(dom, 0, 4, mp, t)
    from oracle import grid
    X, Y, Z = grid.cartesian_coords(dom.grids[0])
    xg = np.stack([X[4], Y[4], Z[4]], axis=-1)
    cross = np.cross(bg["n_dn"], xg)
    assert np.abs(cross).max() < 1e-13 * np.abs(xg).max()
    assert np.abs(bg["n_xdot"] - bg["n_dn"] @ mp.V).max() < 1e-14
