"""Operation-counting build of the oracle's pointwise GH algebra.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The algorithmic flop count of the GH right-hand side at one point (Sec. 3.5,
GHEqns), taken from the equations as the oracle writes them rather than from
any kernel: ``gh_rhs_pointwise`` (oracle/gh.py) runs unchanged on symbolic
scalars that record every arithmetic operation in an expression graph.

Conventions of the count:

* every +, -, x, / and sqrt is one flop (a fused multiply-add is two); a
  negation is free (it folds into the operation that uses it);
* an operation whose operands are all known numbers is folded (a constant);
  x + 0, x - 0, x * 1 and x * 0 cost nothing;
* identical operations on identical operands are counted once (common
  subexpressions shared); + and x are commutative, so a*b and b*a are the
  same node.  This shares the work of symmetric index pairs, which the
  oracle stores twice (psi_ab and psi_ba are the same input);
* only operations that an output actually depends on are counted, and only
  the packed outputs (a <= b of every symmetric pair) are outputs;
* each einsum is contracted pairwise in the order numpy's ``optimal`` path
  picks (the oracle's default einsum would sum the full product of all its
  operands, term by term, and count several times the work);
* the 3 x 3 spatial inverse is the adjugate over the determinant (the
  oracle's float path calls LAPACK, which no count can see into).

The damping parameters are generic numbers (not 0 or +-1), so products with
them are counted; products of parameters alone fold into constants, as a
kernel computes them once per launch.

``python -m oracle.opcount`` writes ``tests/golden/pointwise_flops.json``.
"""
import importlib.util
import json
import os

import numpy as np

ADD, SUB, MUL, DIV, SQRT, NEG, VAR = "add", "sub", "mul", "div", "sqrt", "neg", "var"
FREE = (VAR, NEG)               # a negation folds into the operation that uses it


class Graph:
    """Hash-consed expression graph: one node per distinct operation."""

    def __init__(self):
        self.nodes = {}

    def node(self, op, args, name=None):
        key = (op, tuple(("c", a) if isinstance(a, float) else ("n", id(a)) for a in args), name)
        n = self.nodes.get(key)
        if n is None:
            n = Sym(self, op, args, name)
            self.nodes[key] = n
        return n

    def var(self, name):
        return self.node(VAR, (), name)


def _num(x):
    if isinstance(x, np.ndarray):
        if x.ndim != 0:
            return None
        x = x.item()
    if isinstance(x, (int, float, np.floating, np.integer)) and not isinstance(x, bool):
        return float(x)
    return x if isinstance(x, Sym) else None


def _order(a, b):
    """Canonical operand order of a commutative operation."""
    ka = (0, a, 0) if isinstance(a, float) else (1, 0.0, id(a))
    kb = (0, b, 0) if isinstance(b, float) else (1, 0.0, id(b))
    return (a, b) if ka <= kb else (b, a)


class Sym:
    """A symbolic scalar: a node of the graph."""
    __slots__ = ("g", "op", "args", "name")
    __array_priority__ = 1000

    def __init__(self, g, op, args, name):
        self.g, self.op, self.args, self.name = g, op, args, name

    # -- arithmetic with folding of constants and identities
    def _bin(self, other, fn, swap=False):
        o = _num(other)
        if o is None:
            return NotImplemented
        return fn(o, self) if swap else fn(self, o)

    def __add__(self, o): return self._bin(o, _add)
    def __radd__(self, o): return self._bin(o, _add, True)
    def __sub__(self, o): return self._bin(o, _sub)
    def __rsub__(self, o): return self._bin(o, _sub, True)
    def __mul__(self, o): return self._bin(o, _mul)
    def __rmul__(self, o): return self._bin(o, _mul, True)
    def __truediv__(self, o): return self._bin(o, _div)
    def __rtruediv__(self, o): return self._bin(o, _div, True)
    def __neg__(self): return _neg(self)
    def __pos__(self): return self

    def sqrt(self):
        return self.g.node(SQRT, (self,))


def _graph(a, b):
    return a.g if isinstance(a, Sym) else b.g


def _add(a, b):
    if isinstance(a, float) and isinstance(b, float):
        return a + b
    if isinstance(a, float) and a == 0.0:
        return b
    if isinstance(b, float) and b == 0.0:
        return a
    return _graph(a, b).node(ADD, _order(a, b))


def _sub(a, b):
    if isinstance(a, float) and isinstance(b, float):
        return a - b
    if isinstance(b, float) and b == 0.0:
        return a
    if a is b:
        return 0.0
    if isinstance(a, float) and a == 0.0:
        return _neg(b)
    return _graph(a, b).node(SUB, (a, b))


def _neg(a):
    if isinstance(a, float):
        return -a
    if a.op == NEG:
        return a.args[0]
    return a.g.node(NEG, (a,))


def _mul(a, b):
    if isinstance(a, float) and isinstance(b, float):
        return a * b
    for x, y in ((a, b), (b, a)):
        if isinstance(x, float):
            if x == 0.0:
                return 0.0
            if x == 1.0:
                return y
            if x == -1.0:
                return _neg(y)
    return _graph(a, b).node(MUL, _order(a, b))


def _div(a, b):
    if isinstance(a, float) and isinstance(b, float):
        return a / b
    if isinstance(a, float) and a == 0.0:
        return 0.0
    if isinstance(b, float) and b == 1.0:
        return a
    return _graph(a, b).node(DIV, (a, b))


def _leaves(outputs):
    """The scalars of a (possibly nested) list or array of outputs."""
    out = []
    for o in np.asarray(outputs, dtype=object).ravel():
        if isinstance(o, np.ndarray):
            out.extend(_leaves(o))
        else:
            out.append(o)
    return out


def count(outputs):
    """Operations by kind that the outputs depend on: {op: n, "total": n}."""
    seen, by_op = set(), {}
    stack = [o for o in _leaves(outputs) if isinstance(o, Sym)]
    while stack:
        n = stack.pop()
        if id(n) in seen:
            continue
        seen.add(id(n))
        if n.op not in FREE:
            by_op[n.op] = by_op.get(n.op, 0) + 1
        stack.extend(a for a in n.args if isinstance(a, Sym))
    by_op["total"] = sum(v for k, v in by_op.items())
    return by_op


def evaluate(outputs, values):
    """Numerical value of each output with the variables set from
    ``values`` (name -> float): checks that a graph computes what the
    float code computes."""
    import math
    memo = {}

    def ev(x):
        if isinstance(x, float):
            return x
        k = id(x)
        if k in memo:
            return memo[k]
        stack = [x]
        while stack:
            n = stack[-1]
            pend = [a for a in n.args if isinstance(a, Sym) and id(a) not in memo]
            if pend:
                stack.extend(pend)
                continue
            stack.pop()
            if id(n) in memo:
                continue
            a = [memo[id(v)] if isinstance(v, Sym) else v for v in n.args]
            memo[id(n)] = {VAR: lambda: values[n.name], NEG: lambda: -a[0], ADD: lambda: a[0] + a[1],
                           SUB: lambda: a[0] - a[1],
                           MUL: lambda: a[0] * a[1], DIV: lambda: a[0] / a[1],
                           SQRT: lambda: math.sqrt(a[0])}[n.op]()
        return memo[k]

    arr = np.asarray(outputs, dtype=object)
    return np.vectorize(ev, otypes=[float])(arr)


class _Numpy:
    """numpy as the oracle module sees it in the counting build: object arrays,
    pairwise einsum contractions in numpy's optimal order, the adjugate inverse."""

    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def zeros(shape, dtype=None):
        out = np.empty(shape, dtype=object)
        out.fill(0.0)
        return out

    @staticmethod
    def einsum(*operands, **kw):
        kw.setdefault("optimize", "optimal")
        return np.einsum(*operands, **kw)

    @staticmethod
    def sqrt(x):
        return np.vectorize(lambda v: v.sqrt() if isinstance(v, Sym) else float(np.sqrt(v)), otypes=[object])(x)

    class linalg:
        @staticmethod
        def inv(a):
            """Inverse of [..., 3, 3] object matrices: adjugate / determinant."""
            out = np.empty(a.shape, dtype=object)
            for idx in np.ndindex(a.shape[:-2]):
                m = a[idx]
                cof = np.empty((3, 3), dtype=object)
                for i in range(3):
                    for j in range(3):
                        r = [x for x in range(3) if x != i]
                        c = [x for x in range(3) if x != j]
                        minor = m[r[0], c[0]] * m[r[1], c[1]] - m[r[0], c[1]] * m[r[1], c[0]]
                        cof[i, j] = minor if (i + j) % 2 == 0 else -minor
                det = m[0, 0] * cof[0, 0] + m[0, 1] * cof[0, 1] + m[0, 2] * cof[0, 2]
                rdet = 1.0 / det
                for i in range(3):
                    for j in range(3):
                        out[idx + (i, j)] = cof[j, i] * rdet
            return out


def counting_module(name="gh"):
    """A fresh copy of oracle/<name>.py whose numpy is the counting shim."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".py")
    spec = importlib.util.spec_from_file_location("oracle_counting_" + name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.np = _Numpy()
    return mod


# generic damping parameters: no 0 or +-1, so every product with them counts
GENERIC_GAMMA = (0.731, -0.617, 1.379)


def symbolic_rhs():
    """The oracle's gh_rhs_pointwise at one symbolic point: (outputs [1, 50],
    input names in the order u (50), d_k u (3 x 50), H_a (4), d_i H_a (3 x 4))."""
    ghc = counting_module("gh")
    g = Graph()
    names = (["u%d" % f for f in range(50)] + ["d%du%d" % (k, f) for k in range(3) for f in range(50)]
             + ["H%d" % a for a in range(4)] + ["d%dH%d" % (i, a) for i in range(3) for a in range(4)])
    v = [g.var(n) for n in names]
    u = np.array([v[:50]], dtype=object)
    du = np.array([[v[50 + 50 * k:100 + 50 * k] for k in range(3)]], dtype=object)
    H = np.array([v[200:204]], dtype=object)
    dH = np.array([[v[204 + 4 * i:208 + 4 * i] for i in range(3)]], dtype=object)
    return ghc.gh_rhs_pointwise(u, du, H, dH, *GENERIC_GAMMA), names


def pointwise_rhs_count():
    """Flops of the GH right-hand side at one point (Sec. 3.5, GHEqns):
    inputs u (50), Cartesian derivatives d_k u (150), H_a (4), d_i H_a (12)."""
    out, _ = symbolic_rhs()
    return count(out)


def diffjac_count():
    """Flops of DiffJac at one point (Sec. 3.3, Eq. DiffJac) for 50 fields:
    d_i u = sum_d J[i, d] d_d u over the Jacobian entries the oracle's
    spherical map leaves nonzero (d phi / d z vanishes identically)."""
    from . import grid, spectral
    J = spectral.spherical_jacobian(grid.shell_grid(1.5, 3.0, 5, 3))
    nz = [[bool(np.any(J[i, d] != 0.0)) for d in range(3)] for i in range(3)]
    per_field = sum(2 * sum(row) - 1 for row in nz)     # products plus the adds between them
    return dict(per_field=per_field, total=50 * per_field, nonzero=sum(map(sum, nz)))


def rk4_combine_count():
    """Flops per value of one RK4 step's combinations (Sec. 2.1, method of
    lines; the oracle's rk4_step): three stage states u + c dt k (a product
    and a sum each; c dt is a per-step constant) and the update
    u + dt/6 (k1 + 2 k2 + 2 k3 + k4), counted on one symbolic value."""
    g = Graph()
    u, k1, k2, k3, k4 = (g.var(n) for n in ("u", "k1", "k2", "k3", "k4"))
    dt = 0.0173                                        # a generic step
    stages = [u + 0.5 * dt * k1, u + 0.5 * dt * k2, u + dt * k3]
    new = u + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return count(stages + [new])["total"]


def pointwise_kernel_count():
    """Algorithmic flops per point of one launch of the fused pointwise stage
    (DiffJac + GH right-hand side + a quarter of the RK4 combinations)."""
    rhs = pointwise_rhs_count()
    dj = diffjac_count()
    comb = rk4_combine_count()
    return dict(gh_rhs=rhs, diffjac=dj["total"], rk4_combine_per_value_per_step=comb,
                rk4_combine_per_stage=50 * comb / 4.0,
                total=rhs["total"] + dj["total"] + 50 * comb / 4.0)


def main():
    res = pointwise_kernel_count()
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                        "pointwise_flops.json")
    doc = dict(source="python -m oracle.opcount (oracle/opcount.py: the oracle's gh_rhs_pointwise on "
                      "operation-counting scalars)", **res)
    with open(path, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(doc, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
