"""Multi-shell domain, full right-hand side with boundaries, RK4, filters, energy (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The domain is a set of concentric spherical shells around one hole (Sec. 3.1:
nested I1 x S2 shells centred on the hole).  One right-hand side evaluation
is the paper's module sequence Deriv -> Jacobian -> GHEqns -> ApplyBCs
(Sec. 3.1 module list).  The time stepper is the classic four-stage RK4 (the
paper's code uses a Dormand-Prince stepper, Sec. 2.1; RK4 is the method the
library implements), followed once per step by the filters (Sec. 3.4,
spectral filter; ExpCheb along r and a Heaviside cut in l on the sphere).

State layout: a list with one array per shell, u[s] shaped
[n_r, 50, n_th, n_ph].
"""
import numpy as np

from . import grid, spectral, gh, kerr_schild


class Domain:
    """Shells, exact background and gauge source for one Kerr-Schild hole."""

    def __init__(self, shells, M, chi, gamma0=1.0, gamma1=-1.0, gamma2=1.0,
                 filt_alpha=36.0, filt_order=32, radial_filter_on=False, sh_keep_l=-1, outer_bc="freeze",
                 sh_filter="component"):
        self.specs = list(shells)                 # (r_in, r_out, n_r, L)
        self.M, self.chi = M, chi
        self.gamma0, self.gamma1, self.gamma2 = gamma0, gamma1, gamma2
        self.filt_alpha, self.filt_order = filt_alpha, filt_order
        self.radial_filter_on, self.sh_keep_l = radial_filter_on, sh_keep_l
        # "freeze", "cp" (constraint preserving, Bjorhus form for u^psi and u^0, u^- frozen) or
        # "cp_full" (also the constraint part of u^-)
        self.outer_bc = outer_bc
        self.sh_filter = sh_filter                # "component" (each Cartesian component) or "tensor"
        self.grids = [grid.shell_grid(*s) for s in self.specs]
        self.u_exact, self.H, self.dH = [], [], []
        for g in self.grids:
            u, H, dH = kerr_schild.kerr_schild_shell(g, M, chi)
            self.u_exact.append(u)
            self.H.append(H)
            self.dH.append(dH)
        self._bg = {}

    def shapes(self):
        return [(g["n_r"], 50, g["n_th"], g["n_ph"]) for g in self.grids]

    def boundary_bg(self, s, ir):
        """Background characteristic data on radial slice ir of shell s."""
        key = (s, ir)
        if key not in self._bg:
            g = self.grids[s]
            X, Y, Z = grid.cartesian_coords(g)
            psi_bg, _, _ = gh.unpack_fields(np.moveaxis(self.u_exact[s][ir], 0, -1))
            self._bg[key] = gh.boundary_background(psi_bg, X[ir], Y[ir], Z[ir])
        return self._bg[key]


def _points_last(a):
    """[n_r, F, n_th, n_ph] -> [n_r, n_th, n_ph, F]."""
    return np.moveaxis(a, 1, -1)


def _fields_axis1(a):
    return np.moveaxis(a, -1, 1)


def cartesian_derivatives(dom, u):
    """d_i u for every shell: list of [3, n_r, 50, n_th, n_ph] (Deriv + Jacobian)."""
    return [spectral.cartesian_gradient(us, g) for us, g in zip(u, dom.grids)]


def rhs_interior(dom, u):
    """Pointwise GH right-hand side on every shell, before boundary conditions."""
    out = []
    for s, us in enumerate(u):
        du = spectral.cartesian_gradient(us, dom.grids[s])       # [3, n_r, 50, th, ph]
        U = _points_last(us)
        dU = np.moveaxis(du, (0, 2), (-2, -1))                   # [n_r, th, ph, 3, 50]
        H = _points_last(dom.H[s])
        dH = _points_last(dom.dH[s]).reshape(U.shape[:-1] + (3, 4))
        r = gh.gh_rhs_pointwise(U, dU, H, dH, dom.gamma0, dom.gamma1, dom.gamma2)
        out.append(_fields_axis1(r))
    return out


def apply_boundaries(dom, dudt, u=None, bg_map=None, bg_fn=None):
    """ApplyBCs: outer freezing (or constraint-preserving) condition, upwind
    interface exchange, no-op at excision.  u is needed for the
    constraint-preserving outer condition; bg_map transforms the boundary
    background (the rotating frame rotates its vectors); bg_fn(s, ir), when
    given, supplies the background of radial slice ir of shell s instead (a
    general time-dependent map evaluates it at the moving points).

    Shells are ordered by radius; shell s's outer slice and shell s+1's inner
    slice are the same physical points.
    """
    out = [d.copy() for d in dudt]
    ns = len(out)
    bgf = (lambda b: b) if bg_map is None else bg_map
    if bg_fn is not None:
        dom = _BgOverride(dom, bg_fn)
    for s in range(ns - 1):
        nr = out[s].shape[0]
        bg = bgf(dom.boundary_bg(s, nr - 1))
        a = np.moveaxis(out[s][nr - 1], 0, -1)
        b = np.moveaxis(out[s + 1][0], 0, -1)
        na, nb = gh.apply_interface_bc(a, b, bg, dom.gamma1, dom.gamma2)
        out[s][nr - 1] = np.moveaxis(na, -1, 0)
        out[s + 1][0] = np.moveaxis(nb, -1, 0)
    s = ns - 1
    nr = out[s].shape[0]
    bg = bgf(dom.boundary_bg(s, nr - 1))
    a = np.moveaxis(out[s][nr - 1], 0, -1)
    if dom.outer_bc in ("cp", "cp_full"):
        ub = np.moveaxis(u[s][nr - 1], 0, -1)                                    # [th, ph, 50]
        dub = np.moveaxis(spectral.cartesian_gradient(u[s], dom.grids[s])[:, nr - 1], (0, 1), (-2, -1))
        Hb = dHb = None
        if dom.outer_bc == "cp_full":
            if bg_map is not None or bg_fn is not None:
                raise NotImplementedError("the u^- constraint part is defined on a static grid")
            Hb = np.moveaxis(dom.H[s][nr - 1], 0, -1)                            # [th, ph, 4]
            dHb = np.moveaxis(dom.dH[s][nr - 1], 0, -1).reshape(Hb.shape[:-1] + (3, 4))
        new = gh.apply_outer_bc_cp(a, ub, dub, bg, dom.gamma1, dom.gamma2, Hb, dHb)
    else:
        new = gh.apply_outer_bc(a, bg, dom.gamma1, dom.gamma2)
    out[s][nr - 1] = np.moveaxis(new, -1, 0)
    return out


class _BgOverride:
    """The domain with boundary_bg(s, ir) taken from a function."""

    def __init__(self, dom, fn):
        self._dom, self._fn = dom, fn

    def __getattr__(self, k):
        return getattr(self._dom, k)

    def boundary_bg(self, s, ir):
        return self._fn(s, ir)


def rhs(dom, u):
    """One full right-hand side evaluation: interior GH RHS, then ApplyBCs."""
    return apply_boundaries(dom, rhs_interior(dom, u), u)


def apply_filters(dom, u):
    """Radial ExpCheb filter (if on), then the SH truncation filter (if on):
    per Cartesian component, or through tensor harmonics (sh_filter =
    "tensor", oracle/tensor_filter.py).  sh_keep_l = -2 keeps l <= floor(2L/3)."""
    from . import tensor_filter
    out = []
    for us, g in zip(u, dom.grids):
        v = us
        if dom.radial_filter_on:
            v = spectral.radial_filter(v, g, dom.filt_alpha, dom.filt_order)
        keep = (2 * g["L"]) // 3 if dom.sh_keep_l == -2 else dom.sh_keep_l
        if keep >= 0:
            if dom.sh_filter == "tensor":
                v = np.stack([tensor_filter.filter_fields(v[r], g, keep) for r in range(v.shape[0])])
            else:
                v = spectral.sh_truncation_filter(v, g, keep)
        out.append(v)
    return out


def rk4_step(dom, u, dt):
    """Classic RK4: c = (0, 1/2, 1/2, 1), b = (1, 2, 2, 1)/6; filters after the step."""
    k1 = rhs(dom, u)
    k2 = rhs(dom, [a + 0.5 * dt * k for a, k in zip(u, k1)])
    k3 = rhs(dom, [a + 0.5 * dt * k for a, k in zip(u, k2)])
    k4 = rhs(dom, [a + dt * k for a, k in zip(u, k3)])
    new = [a + dt / 6.0 * (p + 2.0 * q + 2.0 * r + s)
           for a, p, q, r, s in zip(u, k1, k2, k3, k4)]
    return apply_filters(dom, new)


def constraints(dom, u):
    """Per shell: the 64 constraint components [n_r, 64, th, ph] and the
    quadrature norm sum_points w_p sum_c C_c^2."""
    cs, norms = [], []
    for s, us in enumerate(u):
        g = dom.grids[s]
        du = spectral.cartesian_gradient(us, g)
        U = _points_last(us)
        dU = np.moveaxis(du, (0, 2), (-2, -1))
        H = _points_last(dom.H[s])
        c = gh.constraints_pointwise(U, dU, H)
        w = grid.volume_weights(g)
        norms.append(float(np.sum(w * np.sum(c * c, axis=-1))))
        cs.append(_fields_axis1(c))
    return cs, norms


def constraint_energy(dom, u0, dt, n_steps):
    """E = sum_{n=1..N} dt * sum_shells int sum_c C_c^2 dV, evaluated after each step."""
    u = [a.copy() for a in u0]
    E = 0.0
    for _ in range(n_steps):
        u = rk4_step(dom, u, dt)
        _, norms = constraints(dom, u)
        E += dt * sum(norms)
    return E
