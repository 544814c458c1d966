"""The library's per-point GH algebra (csrc/gh_point.cuh), compiled for the
host: its forward pass against the oracle's GH right-hand side and
constraints, and its hand-derived reverse pass against central finite
differences of its own forward pass.  No GPU needed."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import gh as ogh, kerr_schild

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("harness") / "point_harness.so")
    src = os.path.join(HERE, "point_harness.cpp")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", src, "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(out)
    P = ctypes.c_void_p
    D = ctypes.c_double
    L.h_point_rhs.argtypes = [P, P, P, P, P, D, D, D, P]
    L.h_point_rhs_vjp.argtypes = [P, P, P, P, P, D, D, D, P, P, P]
    L.h_point_constraint_energy.argtypes = [P, P, P, P, P, D, P, P]
    L.h_point_constraint_energy.restype = D
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _point(seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(2.0, 4.0, 3) * rng.choice([-1, 1], 3)
    g, dg, _ = kerr_schild.metric_and_derivatives(x[0], x[1], x[2], 1.0, 0.7)
    psi = g + 0.05 * (lambda m: 0.5 * (m + m.T))(rng.standard_normal((4, 4)))
    Pi = rng.standard_normal((4, 4)) * 0.3
    Pi = 0.5 * (Pi + Pi.T)
    Phi = dg + 0.1 * rng.standard_normal((3, 4, 4))
    Phi = 0.5 * (Phi + np.swapaxes(Phi, -1, -2))
    u = ogh.pack_fields(psi, Pi, Phi)
    ds = rng.standard_normal((50, 3)) * 0.5
    th, ph, r = rng.uniform(0.3, 2.8), rng.uniform(0, 6.28), rng.uniform(2, 5)
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    rs = rng.uniform(0.2, 1.0)
    J = np.array([[st * cp * rs, ct * cp / r, -sp / (r * st)],
                  [st * sp * rs, ct * sp / r, cp / (r * st)],
                  [ct * rs, -st / r, 0.0]])
    H = rng.standard_normal(4) * 0.3
    dH = rng.standard_normal(12) * 0.3
    return u, np.ascontiguousarray(ds), np.ascontiguousarray(J), H, dH


G = (1.0, -1.0, 1.0)
G2 = (0.7, 0.4, 1.3)


def _fwd(lib, u, ds, J, H, dH, g):
    out = np.zeros(50)
    lib.h_point_rhs(_p(u), _p(ds), _p(J), _p(H), _p(dH), *g, _p(out))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("g", [G, G2])
def test_forward_matches_oracle(lib, seed, g):
    u, ds, J, H, dH = _point(seed)
    du = np.einsum("id,fd->if", J, ds)                 # Cartesian d_i of every field
    ref = ogh.gh_rhs_pointwise(u, du, H, dH.reshape(3, 4), *g)
    got = _fwd(lib, u, ds, J, H, dH, g)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("g", [G, G2])
def test_reverse_pass_matches_finite_differences(lib, seed, g):
    u, ds, J, H, dH = _point(seed)
    rng = np.random.default_rng(100 + seed)
    kb = rng.standard_normal(50)
    ub = np.zeros(50)
    dsb = np.zeros(150)
    lib.h_point_rhs_vjp(_p(u), _p(ds), _p(J), _p(H), _p(dH), *g, _p(kb), _p(ub), _p(dsb))
    h = 1e-6
    # every input component separately (central differences)
    for k in range(50):
        e = np.zeros(50)
        e[k] = h
        fd = (kb @ _fwd(lib, u + e, ds, J, H, dH, g) - kb @ _fwd(lib, u - e, ds, J, H, dH, g)) / (2 * h)
        assert abs(fd - ub[k]) < 1e-6 * max(1.0, abs(fd)), (k, fd, ub[k])
    for k in range(150):
        e = np.zeros(150)
        e[k] = h
        e = e.reshape(50, 3)
        fd = (kb @ _fwd(lib, u, ds + e, J, H, dH, g) - kb @ _fwd(lib, u, ds - e, J, H, dH, g)) / (2 * h)
        assert abs(fd - dsb[k]) < 1e-6 * max(1.0, abs(fd)), (k, fd, dsb[k])


@pytest.mark.parametrize("seed", [1, 2])
def test_constraint_energy_and_gradient(lib, seed):
    u, ds, J, H, dH = _point(seed)
    du = np.einsum("id,fd->if", J, ds)
    ref = ogh.constraints_pointwise(u, du, H)
    ub = np.zeros(50)
    dsb = np.zeros(150)
    e = lib.h_point_constraint_energy(_p(u), _p(ds), _p(J), _p(H), _p(dH), 0.0, _p(ub), _p(dsb))
    assert abs(e - np.sum(ref * ref)) < 1e-12 * np.sum(ref * ref)
    w = 0.37
    lib.h_point_constraint_energy(_p(u), _p(ds), _p(J), _p(H), _p(dH), w, _p(ub), _p(dsb))
    h = 1e-6

    def E(uu, dd):
        z1, z2 = np.zeros(50), np.zeros(150)
        return lib.h_point_constraint_energy(_p(uu), _p(dd), _p(J), _p(H), _p(dH), 0.0, _p(z1), _p(z2))
    for k in range(50):
        ee = np.zeros(50)
        ee[k] = h
        fd = w * (E(u + ee, ds) - E(u - ee, ds)) / (2 * h)
        assert abs(fd - ub[k]) < 1e-6 * max(1.0, abs(fd)), (k, fd, ub[k])
    for k in range(150):
        ee = np.zeros(150)
        ee[k] = h
        ee = ee.reshape(50, 3)
        fd = w * (E(u, ds + ee) - E(u, ds - ee)) / (2 * h)
        assert abs(fd - dsb[k]) < 1e-6 * max(1.0, abs(fd)), (k, fd, dsb[k])


def test_fused_rhs_and_constraint_reverse_pass_is_the_sum(lib):
    u, ds, J, H, dH = _point(4)
    P = ctypes.c_void_p
    lib.h_point_rhs_vjp_and_constraint.argtypes = [P, P, P, P, P, ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_double, P, ctypes.c_double, P, P]
    kb = np.random.default_rng(3).standard_normal(50)
    ub1, dsb1 = np.zeros(50), np.zeros(150)
    lib.h_point_rhs_vjp(_p(u), _p(ds), _p(J), _p(H), _p(dH), *G, _p(kb), _p(ub1), _p(dsb1))
    lib.h_point_constraint_energy(_p(u), _p(ds), _p(J), _p(H), _p(dH), 0.37, _p(ub1), _p(dsb1))
    ub2, dsb2 = np.zeros(50), np.zeros(150)
    lib.h_point_rhs_vjp_and_constraint(_p(u), _p(ds), _p(J), _p(H), _p(dH), *G, _p(kb), 0.37, _p(ub2), _p(dsb2))
    assert np.allclose(ub1, ub2, rtol=1e-14, atol=1e-14) and np.allclose(dsb1, dsb2, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("seed", [3, 8])
@pytest.mark.parametrize("w", [0.0, 0.37])
def test_pair_restricted_reverse_passes_sum_to_the_full_one(lib, seed, w):
    u, ds, J, H, dH = _point(seed)
    G = (1.0, -1.0, 1.0)
    P = ctypes.c_void_p
    D = ctypes.c_double
    lib.h_point_vjp_pairsum.argtypes = [P, P, P, P, P, D, D, D, P, D, P, P]
    lib.h_point_rhs_vjp_and_constraint.argtypes = [P, P, P, P, P, D, D, D, P, D, P, P]
    kb = np.random.default_rng(seed + 100).standard_normal(50)
    ub1, dsb1 = np.zeros(50), np.zeros(150)
    lib.h_point_rhs_vjp_and_constraint(_p(u), _p(ds), _p(J), _p(H), _p(dH), *G, _p(kb), w, _p(ub1), _p(dsb1))
    if w == 0.0:
        ub1, dsb1 = np.zeros(50), np.zeros(150)
        lib.h_point_rhs_vjp(_p(u), _p(ds), _p(J), _p(H), _p(dH), *G, _p(kb), _p(ub1), _p(dsb1))
    ub2, dsb2 = np.zeros(50), np.zeros(150)
    lib.h_point_vjp_pairsum(_p(u), _p(ds), _p(J), _p(H), _p(dH), *G, _p(kb), w, _p(ub2), _p(dsb2))
    assert np.abs(ub2 - ub1).max() <= 1e-12 * max(1.0, np.abs(ub1).max())
    assert np.abs(dsb2 - dsb1).max() <= 1e-12 * max(1.0, np.abs(dsb1).max())
