"""Dormand-Prince 5(4) adaptive time step (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's evolution code advances the method of lines with a Dormand-Prince
stepper (Sec. 2.1).  This is the standard embedded pair of Dormand & Prince
(1980): seven stages, a fifth-order solution b that is also the last row of
the stage matrix, and a fourth-order companion b_hat whose difference gives
the local error estimate.  The paper does not print the controller; the
reading used here is the common one (Hairer, Norsett & Wanner, Solving ODEs I,
Sec. II.4):

  err = sqrt( mean over every value of (e / (atol + rtol max(|u_n|, |u_n+1|)))^2 ),
  e = dt sum_i (b_i - b_hat_i) k_i,
  accepted when err <= 1,
  dt_next = dt min(5, max(0.2, 0.9 err^(-1/5)))   (5 when err = 0).

The filters act once per accepted step, after it (as for RK4).  No stage is
reused from the previous step (no first-same-as-last shortcut): with filters
the last stage's right-hand side is not that of the filtered new state.
"""
from fractions import Fraction as _F

import numpy as np

from . import evolve

# stage matrix A (strictly lower triangular), nodes c, weights b (order 5)
# and b_hat (order 4) of the Dormand-Prince pair
_A = [
    [],
    [_F(1, 5)],
    [_F(3, 40), _F(9, 40)],
    [_F(44, 45), _F(-56, 15), _F(32, 9)],
    [_F(19372, 6561), _F(-25360, 2187), _F(64448, 6561), _F(-212, 729)],
    [_F(9017, 3168), _F(-355, 33), _F(46732, 5247), _F(49, 176), _F(-5103, 18656)],
    [_F(35, 384), _F(0), _F(500, 1113), _F(125, 192), _F(-2187, 6784), _F(11, 84)],
]
_B = [_F(35, 384), _F(0), _F(500, 1113), _F(125, 192), _F(-2187, 6784), _F(11, 84), _F(0)]
_BHAT = [_F(5179, 57600), _F(0), _F(7571, 16695), _F(393, 640), _F(-92097, 339200), _F(187, 2100),
         _F(1, 40)]

SAFETY, FAC_MIN, FAC_MAX = 0.9, 0.2, 5.0


def tableau(exact=False):
    """(A, c, b, b_hat): A as a 7 x 7 list, c the row sums.  Fractions if exact."""
    conv = (lambda x: x) if exact else float
    A = [[conv(_A[i][j]) if j < len(_A[i]) else conv(_F(0)) for j in range(7)] for i in range(7)]
    c = [conv(sum(_A[i], _F(0))) for i in range(7)]
    return A, c, [conv(x) for x in _B], [conv(x) for x in _BHAT]


def error_norm(u, u_new, e, rtol, atol):
    """Scaled RMS norm of the error estimate over every value of every array."""
    tot, n = 0.0, 0
    for a, b, x in zip(u, u_new, e):
        sc = atol + rtol * np.maximum(np.abs(a), np.abs(b))
        tot += float(np.sum((x / sc) ** 2))
        n += x.size
    return float(np.sqrt(tot / n))


def next_dt(dt, err):
    if err == 0.0:
        return dt * FAC_MAX
    return dt * min(FAC_MAX, max(FAC_MIN, SAFETY * err ** (-0.2)))


def attempt(f, u, dt, rtol, atol):
    """One Dormand-Prince attempt for u' = f(u), u a list of arrays.

    Returns (u_new, err, accepted, dt_next); u_new is the fifth-order
    solution whether or not the step is accepted."""
    A, _, b, bh = tableau()
    k = []
    for s in range(7):
        if s == 0:
            us = u
        else:
            us = [a + dt * sum(A[s][j] * k[j][i] for j in range(s)) for i, a in enumerate(u)]
        k.append(f(us))
    u_new = [a + dt * sum(b[j] * k[j][i] for j in range(7)) for i, a in enumerate(u)]
    e = [dt * sum((b[j] - bh[j]) * k[j][i] for j in range(7)) for i in range(len(u))]
    err = error_norm(u, u_new, e, rtol, atol)
    return u_new, err, err <= 1.0, next_dt(dt, err)


def dp5_step(dom, u, dt, rtol, atol):
    """One attempt on the shell domain: the GH right-hand side with its
    boundary conditions, then the filters if the step is accepted.
    Returns (u_next, err, accepted, dt_next) with u_next = u when rejected."""
    u_new, err, ok, dt_next = attempt(lambda v: evolve.rhs(dom, v), u, dt, rtol, atol)
    if ok:
        return evolve.apply_filters(dom, u_new), err, ok, dt_next
    return u, err, ok, dt_next
