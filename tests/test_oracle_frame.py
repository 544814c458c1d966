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
