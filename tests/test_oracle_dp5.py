"""Pins of the oracle's Dormand-Prince 5(4) step (Sec. 2.1 names the method;
the pair is Dormand & Prince 1980) against what Runge-Kutta theory fixes
independently of the tableau: the order conditions (rooted trees up to order
5 for b, order 4 for b_hat), the published stability function of the pair,
observed convergence orders, and the controller's behaviour."""
from fractions import Fraction

import numpy as np

from oracle import dp5


def _order_conditions(A, c, b, order):
    """Residuals of the Butcher order conditions of all rooted trees up to order."""
    n = len(b)
    mv = lambda v: [sum(A[i][j] * v[j] for j in range(n)) for i in range(n)]
    dot = lambda x, y: sum(p * q for p, q in zip(x, y))
    mul = lambda x, y: [p * q for p, q in zip(x, y)]
    one = [Fraction(1)] * n
    c2, c3, c4 = mul(c, c), mul(mul(c, c), c), mul(mul(c, c), mul(c, c))
    Ac, Ac2, Ac3 = mv(c), mv(c2), mv(c3)
    AAc = mv(Ac)
    conds = [(dot(b, one), Fraction(1)),
             (dot(b, c), Fraction(1, 2)),
             (dot(b, c2), Fraction(1, 3)), (dot(b, Ac), Fraction(1, 6)),
             (dot(b, c3), Fraction(1, 4)), (dot(b, mul(c, Ac)), Fraction(1, 8)),
             (dot(b, Ac2), Fraction(1, 12)), (dot(b, AAc), Fraction(1, 24))]
    if order >= 5:
        conds += [(dot(b, c4), Fraction(1, 5)), (dot(b, mul(c2, Ac)), Fraction(1, 10)),
                  (dot(b, mul(c, Ac2)), Fraction(1, 15)), (dot(b, mul(c, AAc)), Fraction(1, 30)),
                  (dot(b, mul(Ac, Ac)), Fraction(1, 20)), (dot(b, Ac3), Fraction(1, 20)),
                  (dot(b, mv(mul(c, Ac))), Fraction(1, 40)), (dot(b, mv(Ac2)), Fraction(1, 60)),
                  (dot(b, mv(AAc)), Fraction(1, 120))]
    return [got - want for got, want in conds]


def test_fifth_order_weights_satisfy_all_order_conditions_exactly():
    A, c, b, _ = dp5.tableau(exact=True)
    assert all(r == 0 for r in _order_conditions(A, c, b, 5))
    for i in range(7):                       # c_i = sum_j a_ij
        assert c[i] == sum(A[i])


def test_fourth_order_companion_is_order_four_not_five():
    A, c, _, bh = dp5.tableau(exact=True)
    assert all(r == 0 for r in _order_conditions(A, c, bh, 4))
    assert any(r != 0 for r in _order_conditions(A, c, bh, 5))


def test_stability_function_is_the_published_one():
    # R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 + z^5/120 + z^6/600 (Hairer, Norsett & Wanner)
    for z in [-0.3, -1.7, 0.4 + 0.9j, -2.5 + 1.0j]:
        u_new, _, _, _ = dp5.attempt(lambda v: [z * v[0]], [np.array([1.0 + 0j])], 1.0, 1.0, 1.0)
        R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24 + z ** 5 / 120 + z ** 6 / 600
        assert abs(u_new[0][0] - R) < 1e-14 * max(1.0, abs(R))


def test_observed_orders_of_solution_and_error_estimate():
    # u' = -u^2 + sin(t) as an autonomous system (t, u): global error O(dt^5),
    # local error estimate O(dt^5)
    f = lambda v: [np.ones(1), -v[1] ** 2 + np.sin(v[0])]

    def solve(n):
        v = [np.zeros(1), np.ones(1)]
        for _ in range(n):
            v, _, _, _ = dp5.attempt(f, v, 1.0 / n, 1e-30, 1.0)
        return v[1][0]

    ref = solve(2048)
    e1, e2 = abs(solve(32) - ref), abs(solve(64) - ref)   # asymptotic range, above rounding
    assert 4.7 < np.log2(e1 / e2) < 5.4
    ests = []
    for h in (0.1, 0.05):
        _, err, _, _ = dp5.attempt(f, [np.zeros(1), np.ones(1)], h, 0.0, 1.0)   # err = |e| (atol = 1)
        ests.append(err)
    assert 4.5 < np.log2(ests[0] / ests[1]) < 5.6


def test_controller_rejects_large_steps_and_clamps_growth():
    f = lambda v: [-50.0 * v[0]]
    u = [np.ones(4)]
    _, err, ok, dt_next = dp5.attempt(f, u, 0.5, 1e-8, 1e-8)
    assert not ok and err > 1 and np.isclose(dt_next, 0.5 * dp5.FAC_MIN)
    _, err, ok, dt_next = dp5.attempt(lambda v: [0.0 * v[0]], u, 0.5, 1e-8, 1e-8)
    assert ok and err == 0.0 and np.isclose(dt_next, 0.5 * dp5.FAC_MAX)
    _, err, ok, dt_next = dp5.attempt(f, u, 1e-3, 1e-6, 1e-6)
    assert ok and np.isclose(dt_next, 1e-3 * min(5.0, max(0.2, 0.9 * err ** -0.2)))
    # the exponent 1/5 matches the embedded pair's dt^5 local error: from an
    # unclamped error estimate, one controller step lands near err = 0.9^5
    g = lambda v: [-1.0 * v[0]]
    for dt in (0.2, 0.1):
        _, err, _, dt_next = dp5.attempt(g, u, dt, 1e-8, 1e-8)
        assert 0.2 < dt_next / dt < 5.0
        _, err2, _, _ = dp5.attempt(g, u, dt_next, 1e-8, 1e-8)
        assert abs(err2 - 0.9 ** 5) < 0.05, (dt, err, err2)
