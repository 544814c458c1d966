"""Helpers shared by the GPU parity tests: build the same seeded inputs for the
oracle and for the library, and compare element by element.

Tolerance: the library must match the oracle to
    max |gpu - oracle| <= 1e-11 * max |u|
where u is the state the operation was applied to (the bound is set by
summation order: both sides evaluate the same sums in FP64, in different
orders and through different factorisations of the operators).  Outputs that
are not states (right-hand sides, derivatives, constraints) must also match
relative to their own size:
    max |gpu - oracle| <= 1e-10 * max |oracle output|
which the test inputs keep meaningful: their outputs are within a few orders
of magnitude of the input (the smallest, the Schwarzschild shell's
right-hand side, is 3.6e-3 of it), while rounding leaves about 1e-14 of it.
"""
import numpy as np
import torch

from oracle import evolve, perturb
from paper_1804_09101_gb300 import gh, workloads

REL_TOL = 1e-11
OUT_TOL = 1e-10


def flat(lst):
    return np.concatenate([a.ravel() for a in lst])


def unflat(vec, dom):
    out, o = [], 0
    for shp in dom.shapes():
        n = int(np.prod(shp))
        out.append(vec[o:o + n].reshape(shp))
        o += n
    return out


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def to_host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def oracle_domain(w):
    return evolve.Domain(w.shells, w.M, w.chi, w.gamma0, w.gamma1, w.gamma2, w.filt_alpha,
                         w.filt_order, w.radial_filter_on, w.sh_keep_l)


def oracle_initial_state(w, odom):
    """Exact data + perturbation + seeded noise, as the oracle builds it."""
    u = [a.copy() for a in odom.u_exact]
    if w.pulse is not None:
        p = w.pulse
        for s, g in enumerate(odom.grids):
            if p.kind == "psi_pulse":
                u[s] = u[s] + perturb.psi_pulse(g, odom.u_exact[s], p.amplitude, p.center, p.width,
                                                p.lmax, p.coeffs)
            else:
                u[s] = u[s] + perturb.pi_modes(g, p.center, p.width, p.lmax, p.coeffs)
    return unflat(flat(u) + w.noise(), odom)


def gpu_domain(w, odom=None, algorithm="default"):
    """Library domain with the oracle's gauge source and background (when given)."""
    dom = gh.Domain.from_workload(w)
    if algorithm != "default":
        gh.gh_set_algorithm(dom, {"dense": gh.GH_ALG_DENSE, "separable": gh.GH_ALG_SEPARABLE,
                                  "folded": gh.GH_ALG_SEPARABLE_FOLDED}[algorithm])
    if odom is not None:
        gh.gh_set_gauge(dom, to_dev(flat(odom.H)), to_dev(flat(odom.dH)))
        gh.gh_set_background(dom, to_dev(flat(odom.u_exact)))
    return dom


def max_rel(got, ref, scale):
    return float(np.abs(got - ref).max() / scale)


def assert_output_parity(got, ref, u_scale, what=""):
    """Both bars for an output that is not a state: 1e-11 of the input's
    size and 1e-10 of the output's own."""
    d = float(np.abs(got - ref).max())
    r = float(np.abs(ref).max())
    assert d <= REL_TOL * u_scale, (what, "state-relative", d / u_scale)
    assert d <= OUT_TOL * r, (what, "output-relative", d / r if r else d)
