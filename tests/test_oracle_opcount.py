"""The oracle's operation-counting build (oracle/opcount.py), pinned against
counts with closed forms, and the algorithmic flop count of the fused
pointwise stage that the benchmark's roofline divides by.

The counter is pinned by: a dot product of length n (2n - 1), a general
3 x 3 matrix product (45), the product of a symmetric matrix with itself (its
six distinct entries only), the adjugate inverse (42), constant folding and
reachability; the symbolic run of gh_rhs_pointwise is pinned to the float
oracle by evaluating its graph at random inputs."""
import json
import os

import numpy as np
import pytest

from oracle import gh, opcount
from paper_1804_09101_gb300 import costmodel

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pointwise_flops.json")


def _vars(g, prefix, shape):
    out = np.empty(shape, dtype=object)
    for idx in np.ndindex(shape):
        out[idx] = g.var(prefix + "_".join(map(str, idx)))
    return out


@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_dot_product_costs_2n_minus_1(n):
    g = opcount.Graph()
    a, b = _vars(g, "a", (n,)), _vars(g, "b", (n,))
    assert opcount.count([opcount._Numpy.einsum("i,i->", a, b)])["total"] == 2 * n - 1


def test_general_matrix_product_costs_45():
    g = opcount.Graph()
    A, B = _vars(g, "a", (3, 3)), _vars(g, "b", (3, 3))
    c = opcount.count(opcount._Numpy.einsum("ij,jk->ik", A, B))
    assert c["mul"] == 27 and c["add"] == 18 and c["total"] == 45


def test_symmetric_entries_are_counted_once():
    """A A for symmetric A (one variable per pair): the (i,k) and (k,i)
    entries are the same sums of the same products, so only the six
    distinct entries count (12 sums); their 18 products include each
    off-diagonal square twice (in two diagonal entries), so 15 distinct."""
    g = opcount.Graph()
    A = np.empty((3, 3), dtype=object)
    for i in range(3):
        for j in range(i, 3):
            A[i, j] = A[j, i] = g.var("a%d%d" % (i, j))
    c = opcount.count(opcount._Numpy.einsum("ij,jk->ik", A, A))
    assert c["mul"] == 15 and c["add"] == 12


def test_adjugate_inverse_costs_42_and_inverts():
    g = opcount.Graph()
    A = _vars(g, "a", (1, 3, 3))
    inv = opcount._Numpy.linalg.inv(A)
    c = opcount.count(inv)
    assert c["total"] == 42 and c["div"] == 1          # 9 cofactors x 3, det 5, 1/det, 9 products
    rng = np.random.default_rng(3)
    vals = {A[0, i, j].name: float(x) for (i, j), x in np.ndenumerate(rng.standard_normal((3, 3)) + 3 * np.eye(3))}
    M = np.array([[vals[A[0, i, j].name] for j in range(3)] for i in range(3)])
    assert np.abs(opcount.evaluate(inv[0], vals) - np.linalg.inv(M)).max() < 1e-13


def test_constants_fold_and_identities_are_free():
    g = opcount.Graph()
    x = g.var("x")
    assert opcount.count([x * 0.0 + 1.0 * x - 0.0])["total"] == 0
    assert opcount.count([(2.0 * 3.0) * x])["total"] == 1
    assert opcount.count([x * g.var("y"), g.var("y") * x])["total"] == 1      # commutative: one node
    assert opcount.count([-x, 0.0 - x, -(-x), (-1.0) * x])["total"] == 0       # negation is free
    _ = x * x * x                                                             # built but not an output
    assert opcount.count([x + 1.0])["total"] == 1


def test_symbolic_rhs_computes_the_float_oracle():
    """The counted graph is the oracle's function: evaluated at random inputs
    it equals gh_rhs_pointwise in floats (near-Minkowski metric, so that the
    lapse is real)."""
    out, names = opcount.symbolic_rhs()
    rng = np.random.default_rng(11)
    u = np.zeros(50)
    for p, (a, b) in enumerate(gh.PAIRS):
        u[p] = (-1.0 if a == b == 0 else 1.0 if a == b else 0.0)
    u = u + 0.1 * rng.standard_normal(50)
    du = rng.standard_normal((3, 50))
    H, dH = rng.standard_normal(4), rng.standard_normal((3, 4))
    flat = np.concatenate([u, du.ravel(), H, dH.ravel()])
    got = opcount.evaluate(out[0], dict(zip(names, map(float, flat))))
    ref = gh.gh_rhs_pointwise(u[None], du[None], H[None], dH[None], *opcount.GENERIC_GAMMA)[0]
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_diffjac_has_eight_jacobian_entries():
    d = opcount.diffjac_count()
    assert d["nonzero"] == 8 and d["per_field"] == 13 and d["total"] == 650


def test_rk4_combinations_per_value():
    # three stage states (2 each) and u + dt/6 (k1 + 2 k2 + 2 k3 + k4) (3 adds, 2 doublings,
    # the dt/6 product and the final add)
    assert opcount.rk4_combine_count() == 13


def test_stored_count_is_the_counting_builds_and_the_benchmarks():
    doc = json.load(open(GOLDEN))
    res = opcount.pointwise_kernel_count()
    assert doc["gh_rhs"] == res["gh_rhs"] and doc["total"] == res["total"]
    assert costmodel.POINTWISE_FLOPS_PER_POINT == res["total"]
    assert costmodel.POINTWISE_GH_RHS_FLOPS_PER_POINT == res["gh_rhs"]["total"]
