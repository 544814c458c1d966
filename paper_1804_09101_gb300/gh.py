"""Thin Python binding of libgh (include/gh.h): argument marshalling only.

Every function has the name of the C entry point it wraps and takes torch
tensors that must be contiguous float64 CUDA tensors; all arithmetic runs in
the library's CUDA kernels.  Calls are enqueued on torch's current CUDA
stream.  There is no CPU fallback: if libgh.so cannot be loaded, importing
this module raises.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgh.so")

GH_OK, GH_EINVAL, GH_ENOMEM, GH_ECUDA, GH_ETIMEOUT, GH_ENONFINITE, GH_ENOTSUP = range(7)
_NAMES = ["GH_OK", "GH_EINVAL", "GH_ENOMEM", "GH_ECUDA", "GH_ETIMEOUT", "GH_ENONFINITE", "GH_ENOTSUP"]

NF = 50


class GHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_NAMES[status] if 0 <= status < len(_NAMES) else status, msg))
        self.status = status


class gh_shell(ctypes.Structure):
    _fields_ = [("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
                ("n_r", ctypes.c_int), ("L", ctypes.c_int), ("bh", ctypes.c_int)]


class gh_params(ctypes.Structure):
    _fields_ = [("gamma0", ctypes.c_double), ("gamma1", ctypes.c_double), ("gamma2", ctypes.c_double),
                ("filt_alpha", ctypes.c_double), ("filt_order", ctypes.c_int),
                ("radial_filter_on", ctypes.c_int), ("sh_keep_l", ctypes.c_int)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libgh.so not built at %s (run __graft_entry__.build())" % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    sigs = {
        "gh_create_domain": ([ctypes.POINTER(gh_shell), I, ctypes.POINTER(gh_params), P, ctypes.POINTER(P)], I),
        "gh_destroy_domain": ([P], I),
        "gh_set_stream": ([P, P], I),
        "gh_set_overlap": ([P, I], I),
        "gh_state_size": ([P], ctypes.c_longlong),
        "gh_num_points": ([P], ctypes.c_longlong),
        "gh_rk4_work_size": ([P], ctypes.c_longlong),
        "gh_num_shells": ([P], I),
        "gh_launch_count": ([P], ctypes.c_longlong),
        "gh_last_error": ([P], ctypes.c_char_p),
        "gh_set_analytic_kerr_schild": ([P, I, D, D, P], I),
        "gh_set_analytic_kerr_schild_spin": ([P, I, D, ctypes.POINTER(D), P], I),
        "gh_set_dt_scale": ([P, I, D], I),
        "gh_rk4_graph_capture": ([P, D, P, P, P], I),
        "gh_rk4_step_host": ([P, D, I, P, P, P], I),
        "gh_rk4_graph_launch": ([P, I], I),
        "gh_set_gauge": ([P, P, P], I),
        "gh_set_background": ([P, P], I),
        "gh_get_gauge": ([P, P, P], I),
        "gh_add_perturbation": ([P, I, D, D, D, I, P, P], I),
        "gh_derivatives": ([P, P, P], I),
        "gh_rhs": ([P, P, P], I),
        "gh_rhs_noalloc": ([P, P, P], I),
        "gh_rk4_step": ([P, D, P, P, P], I),
        "gh_apply_filters": ([P, P, P], I),
        "gh_constraints": ([P, P, P, P], I),
        "gh_sync": ([P], I),
        "gh_set_algorithm": ([P, I], I),
        "gh_autotune": ([P, I], I),
        "gh_set_outer_bc": ([P, I], I),
        "gh_set_sh_filter": ([P, I], I),
        "gh_set_rotating_frame": ([P, ctypes.POINTER(D), D], I),
        "gh_set_time": ([P, D], I),
        "gh_set_frame_map": ([P, ctypes.POINTER(D), D, D, ctypes.POINTER(D)], I),
        "gh_get_time": ([P, ctypes.POINTER(D)], I),
        "gh_dp5_work_size": ([P], ctypes.c_longlong),
        "gh_dp5_step": ([P, D, D, D, P, P, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(D)], I),
        "gh_get_schedule": ([P, ctypes.POINTER(I), I], I),
        "gh_set_schedule": ([P, ctypes.POINTER(I), I], I),
        "gh_rhs_vjp": ([P, P, P, P], I),
        "gh_rk4_vjp_work_size": ([P], ctypes.c_longlong),
        "gh_rk4_step_vjp": ([P, D, P, P, P, P], I),
        "gh_rk4_step_save": ([P, D, P, P, P, P], I),
        "gh_rk4_step_vjp_saved": ([P, D, P, P, P, P, P, D], I),
        "gh_constraint_energy_vjp": ([P, P, D, P], I),
        "gh_perturbation_vjp": ([P, I, D, D, I, P, P], I),
        "gh_profile_enable": ([P, I], I),
        "gh_profile_read": ([P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)], I),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = _load()


def library():
    """The loaded libgh.so (ctypes.CDLL)."""
    return _lib


def _ptr(t, name, numel=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    if numel is not None and t.numel() < numel:
        raise ValueError("%s has %d elements, needs %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


class Domain:
    """Owns a gh_domain handle (shells, cached matrices, scratch)."""

    def __init__(self, shells, gamma0=1.0, gamma1=-1.0, gamma2=1.0, filt_alpha=36.0, filt_order=32,
                 radial_filter_on=False, sh_keep_l=-1):
        shells = [tuple(s) + (0,) if len(s) == 4 else tuple(s) for s in shells]
        arr = (gh_shell * len(shells))(*[gh_shell(float(a), float(b), int(n), int(L), int(h))
                                         for (a, b, n, L, h) in shells])
        self.params = gh_params(gamma0, gamma1, gamma2, filt_alpha, int(filt_order),
                                int(bool(radial_filter_on)), int(sh_keep_l))
        h = ctypes.c_void_p()
        st = _lib.gh_create_domain(arr, len(shells), ctypes.byref(self.params),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(h))
        if st != GH_OK:
            raise GHError(st, _lib.gh_last_error(None).decode())
        self.handle = h
        self.shells = [tuple(s) for s in shells]
        self.state_size = _lib.gh_state_size(h)
        self.rotating = False
        self.num_points = _lib.gh_num_points(h)
        self.work_size = _lib.gh_rk4_work_size(h)
        self.vjp_work_size = _lib.gh_rk4_vjp_work_size(h)
        self.dp5_work_size = _lib.gh_dp5_work_size(h)

    @classmethod
    def from_workload(cls, w):
        return cls(w.shells, w.gamma0, w.gamma1, w.gamma2, w.filt_alpha, w.filt_order,
                   w.radial_filter_on, w.sh_keep_l)

    def _check(self, st):
        if st != GH_OK:
            raise GHError(st, _lib.gh_last_error(self.handle).decode())

    def _stream(self):
        _lib.gh_set_stream(self.handle, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    def close(self):
        if getattr(self, "handle", None):
            _lib.gh_destroy_domain(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self):
        return _lib.gh_launch_count(self.handle)

    # -- allocation helpers (torch owns the memory)
    def new_state(self):
        return torch.zeros(self.state_size, dtype=torch.float64, device="cuda")

    def new_work(self):
        return torch.zeros(self.work_size, dtype=torch.float64, device="cuda")


def gh_set_analytic_kerr_schild(dom, bh, M, chi, u):
    """Exact Kerr-Schild data; chi a number (spin along +z) or a 3-vector."""
    dom._stream()
    if hasattr(chi, "__len__"):
        v = (ctypes.c_double * 3)(*[float(c) for c in chi])
        dom._check(_lib.gh_set_analytic_kerr_schild_spin(dom.handle, int(bh), float(M), v,
                                                         _ptr(u, "u", dom.state_size)))
    else:
        dom._check(_lib.gh_set_analytic_kerr_schild(dom.handle, int(bh), float(M), float(chi),
                                                    _ptr(u, "u", dom.state_size)))


def gh_set_dt_scale(dom, bh, scale):
    """gh_set_dt_scale: hole bh advances by dt * scale in every RK4 step."""
    dom._stream()
    dom._check(_lib.gh_set_dt_scale(dom.handle, int(bh), float(scale)))


def _host_ptr(t, name, numel):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float64 CPU tensor" % name)
    if t.numel() < numel:
        raise ValueError("%s has %d elements, needs %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def gh_rk4_step_host(dom, dt, n_steps, u_in, u_out, norm2=None):
    """gh_rk4_step_host: n_steps RK4 steps of a HOST state (CPU float64 tensors,
    pinned for full-speed copies); copies in, steps on the device, copies out.
    One step with pinned buffers: the step's own kernels read u_in and write
    u_out, overlapping the link transfers with the step's work."""
    dom._stream()
    dom._check(_lib.gh_rk4_step_host(dom.handle, float(dt), int(n_steps),
                                     _host_ptr(u_in, "u_in", dom.state_size),
                                     _host_ptr(u_out, "u_out", dom.state_size),
                                     _host_ptr(norm2, "norm2", len(dom.shells))))


def gh_rk4_graph_capture(dom, dt, u, work, norm2_pre=None):
    """gh_rk4_graph_capture: record one gh_rk4_step with these buffers as a CUDA graph (nothing runs)."""
    dom._stream()
    dom._check(_lib.gh_rk4_graph_capture(dom.handle, float(dt), _ptr(u, "u", dom.state_size),
                                         _ptr(work, "work", dom.work_size), _ptr(norm2_pre, "norm2_pre")))


def gh_rk4_graph_launch(dom, n_steps):
    """gh_rk4_graph_launch: replay the captured step n_steps times on the current stream."""
    dom._stream()
    dom._check(_lib.gh_rk4_graph_launch(dom.handle, int(n_steps)))


def gh_set_gauge(dom, H, dH):
    """gh_set_gauge: H [r][4][th][ph] and dH [r][12][th][ph] (entry 4i+a = d_i H_a) per shell."""
    dom._stream()
    dom._check(_lib.gh_set_gauge(dom.handle, _ptr(H, "H", 4 * dom.num_points), _ptr(dH, "dH", 12 * dom.num_points)))


def gh_get_gauge(dom, H, dH):
    """gh_get_gauge: copy the gauge source out, in the layout gh_set_gauge takes."""
    dom._stream()
    dom._check(_lib.gh_get_gauge(dom.handle, _ptr(H, "H", 4 * dom.num_points), _ptr(dH, "dH", 12 * dom.num_points)))


def gh_set_background(dom, u_bg):
    """gh_set_background: boundary background (lapse, shift, normal) from the metric part of u_bg."""
    dom._stream()
    dom._check(_lib.gh_set_background(dom.handle, _ptr(u_bg, "u_bg", dom.state_size)))


def gh_add_perturbation(dom, kind, A, Rc, w, lmax, coeffs, u):
    """gh_add_perturbation: add the psi pulse (kind 0) or the Pi modes (kind 1)
    to u; coeffs holds (lmax+1)^2 values."""
    import numpy as np
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    if c.size != (lmax + 1) ** 2:
        raise ValueError("need (lmax+1)^2 coefficients")
    dom._stream()
    dom._check(_lib.gh_add_perturbation(dom.handle, int(kind), float(A), float(Rc), float(w), int(lmax),
                                        c.ctypes.data_as(ctypes.c_void_p), _ptr(u, "u", dom.state_size)))


def gh_derivatives(dom, u, du):
    """gh_derivatives: Cartesian derivatives of all 50 fields into du (3 states)."""
    dom._stream()
    dom._check(_lib.gh_derivatives(dom.handle, _ptr(u, "u", dom.state_size), _ptr(du, "du", 3 * dom.state_size)))


def gh_rhs(dom, u, dudt):
    """gh_rhs: dudt = F(u), the GH right-hand side with its boundary conditions."""
    dom._stream()
    dom._check(_lib.gh_rhs(dom.handle, _ptr(u, "u", dom.state_size), _ptr(dudt, "dudt", dom.state_size)))


def gh_rhs_noalloc(dom, u, dudt):
    """gh_rhs with the library's fixed work area: no device allocation at call time."""
    dom._stream()
    dom._check(_lib.gh_rhs_noalloc(dom.handle, _ptr(u, "u", dom.state_size), _ptr(dudt, "dudt", dom.state_size)))


def gh_rk4_step(dom, dt, u, work, norm2_pre=None):
    """gh_rk4_step: one RK4 step of u in place, then the filters; norm2_pre
    (optional) receives the constraint norms of the incoming u."""
    dom._stream()
    dom._check(_lib.gh_rk4_step(dom.handle, float(dt), _ptr(u, "u", dom.state_size),
                                _ptr(work, "work", dom.work_size), _ptr(norm2_pre, "norm2_pre")))


def gh_apply_filters(dom, u, work):
    """gh_apply_filters: the domain's radial and angular filters on u in place."""
    dom._stream()
    dom._check(_lib.gh_apply_filters(dom.handle, _ptr(u, "u", dom.state_size), _ptr(work, "work", dom.work_size)))


def gh_constraints(dom, u, c_out, norm2):
    """gh_constraints: the 64 constraint components (c_out, optional) and the per-shell quadrature norms."""
    dom._stream()
    dom._check(_lib.gh_constraints(dom.handle, _ptr(u, "u", dom.state_size),
                                   _ptr(c_out, "c_out", 64 * dom.num_points), _ptr(norm2, "norm2", len(dom.shells))))


KERNEL_FAMILIES = ["radial", "angular", "pointwise", "bc", "radial_filter", "angular_filter", "reduce", "combine"]


def gh_set_overlap(dom, on=True):
    """gh_set_overlap: radial map on the domain's second stream beside the angular maps (default on)."""
    dom._check(_lib.gh_set_overlap(dom.handle, int(bool(on))))


def gh_profile_enable(dom, on=True):
    """gh_profile_enable: per-family CUDA-event timing of the library's launches (gh_profile_read)."""
    dom._stream()
    dom._check(_lib.gh_profile_enable(dom.handle, int(bool(on))))


def gh_profile_read(dom, family):
    """(total_ms, launches) of one kernel family since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    dom._check(_lib.gh_profile_read(dom.handle, int(family), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


GH_ALG_DENSE, GH_ALG_SEPARABLE, GH_ALG_SEPARABLE_FOLDED = 0, 1, 2


def gh_set_algorithm(dom, algorithm):
    """gh_set_algorithm: angular maps by GH_ALG_SEPARABLE_FOLDED (default), GH_ALG_SEPARABLE or GH_ALG_DENSE."""
    dom._stream()
    dom._check(_lib.gh_set_algorithm(dom.handle, int(algorithm)))


GH_BC_FREEZE, GH_BC_CONSTRAINT_PRESERVING, GH_BC_CONSTRAINT_PRESERVING_FULL = 0, 1, 2
GH_SH_FILTER_COMPONENT, GH_SH_FILTER_TENSOR = 0, 1


def gh_set_rotating_frame(dom, axis, omega):
    """Rigid rotation of the grid about axis at rate omega (0: static)."""
    v = (ctypes.c_double * 3)(*[float(c) for c in axis])
    dom._stream()
    dom._check(_lib.gh_set_rotating_frame(dom.handle, v, float(omega)))
    dom.rotating = float(omega) != 0.0


def gh_set_frame_map(dom, axis, omega, adot, V):
    """General map of the grid: x = (1 + adot t) R(axis, omega t) x_grid + V t;
    the hole's gauge source and boundary data are evaluated at the moving
    points every stage (set the holes with gh_set_analytic_kerr_schild first)."""
    a = (ctypes.c_double * 3)(*[float(c) for c in axis])
    v = (ctypes.c_double * 3)(*[float(c) for c in V])
    dom._stream()
    dom._check(_lib.gh_set_frame_map(dom.handle, a, float(omega), float(adot), v))
    dom.rotating = True


def gh_set_time(dom, t):
    """gh_set_time: set the domain clock (the rotating frame's angle follows it)."""
    dom._check(_lib.gh_set_time(dom.handle, float(t)))


def gh_get_time(dom):
    """gh_get_time: the domain clock."""
    t = ctypes.c_double()
    dom._check(_lib.gh_get_time(dom.handle, ctypes.byref(t)))
    return t.value


def gh_set_outer_bc(dom, mode):
    """gh_set_outer_bc: outer condition code: freezing (0), constraint preserving for u^psi and u^0 (1),
    and also the constraint part of u^- (2)."""
    dom._stream()
    dom._check(_lib.gh_set_outer_bc(dom.handle, int(mode)))


def gh_set_sh_filter(dom, mode):
    """0 / "component": each field truncated as a scalar; 1 / "tensor": the
    tensor spherical-harmonic filter (spin-weighted harmonics in the complex
    frame)."""
    mode = {"component": 0, "tensor": 1}.get(mode, mode)
    dom._stream()
    dom._check(_lib.gh_set_sh_filter(dom.handle, int(mode)))


def gh_dp5_step(dom, dt, rtol, atol, u, work):
    """One Dormand-Prince 5(4) attempt; returns (err, accepted, dt_next).  On
    acceptance u holds the new (filtered) state, else it is unchanged."""
    err, acc, dtn = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
    dom._stream()
    dom._check(_lib.gh_dp5_step(dom.handle, float(dt), float(rtol), float(atol), _ptr(u, "u", dom.state_size),
                                _ptr(work, "work", dom.dp5_work_size), ctypes.byref(err), ctypes.byref(acc),
                                ctypes.byref(dtn)))
    return err.value, bool(acc.value), dtn.value


def new_dp5_work(dom):
    """A zeroed device work area for gh_dp5_step."""
    return torch.zeros(dom.dp5_work_size, dtype=torch.float64, device="cuda")


SCHEDULE_LEN = 9
SCHEDULE_KEYS = ("radial_chains", "radial_groups", "radial_filter_chains", "radial_filter_groups",
                 "fold_deriv_threads", "fold_deriv_budget", "fold_filter_threads", "fold_filter_budget",
                 "adjoint_pair_split")


def gh_autotune(dom, reps=5):
    """Time the work-schedule candidates of the radial and folded angular maps
    on this domain and keep the fastest (results are bitwise unchanged)."""
    dom._stream()
    dom._check(_lib.gh_autotune(dom.handle, int(reps)))


def gh_get_schedule(dom):
    """gh_get_schedule: the work schedule as a dict keyed by SCHEDULE_KEYS."""
    v = (ctypes.c_int * SCHEDULE_LEN)()
    dom._check(_lib.gh_get_schedule(dom.handle, v, SCHEDULE_LEN))
    return dict(zip(SCHEDULE_KEYS, list(v)))


def gh_set_schedule(dom, sched):
    """Install a schedule; keys left out keep their current values."""
    cur = gh_get_schedule(dom)
    cur.update(sched)
    v = (ctypes.c_int * SCHEDULE_LEN)(*[int(cur[k]) for k in SCHEDULE_KEYS])
    dom._stream()
    dom._check(_lib.gh_set_schedule(dom.handle, v, SCHEDULE_LEN))


def gh_rhs_vjp(dom, u, kbar, ubar):
    """ubar += (dF/du)^T kbar for F = gh_rhs."""
    dom._stream()
    dom._check(_lib.gh_rhs_vjp(dom.handle, _ptr(u, "u", dom.state_size), _ptr(kbar, "kbar", dom.state_size),
                               _ptr(ubar, "ubar", dom.state_size)))


def gh_rk4_step_vjp(dom, dt, u_n, ubar_np1, ubar_n, work):
    """ubar_n = (d step/d u_n)^T ubar_np1."""
    dom._stream()
    dom._check(_lib.gh_rk4_step_vjp(dom.handle, float(dt), _ptr(u_n, "u_n", dom.state_size),
                                    _ptr(ubar_np1, "ubar_np1", dom.state_size), _ptr(ubar_n, "ubar_n", dom.state_size),
                                    _ptr(work, "work", dom.vjp_work_size)))


def gh_rk4_step_save(dom, dt, u, work, stages, norm2_pre=None):
    """gh_rk4_step that also writes its three intermediate stage states to stages."""
    dom._stream()
    dom._check(_lib.gh_rk4_step_save(dom.handle, float(dt), _ptr(u, "u", dom.state_size),
                                     _ptr(work, "work", dom.work_size), _ptr(norm2_pre, "norm2_pre"),
                                     _ptr(stages, "stages", 3 * dom.state_size)))


def gh_rk4_step_vjp_saved(dom, dt, u_n, stages, ubar_np1, ubar_n, work, cweight=0.0):
    """Step VJP reusing saved stage states; adds cweight * grad(constraint energy)(u_n)."""
    dom._stream()
    dom._check(_lib.gh_rk4_step_vjp_saved(dom.handle, float(dt), _ptr(u_n, "u_n", dom.state_size),
                                          _ptr(stages, "stages", 3 * dom.state_size),
                                          _ptr(ubar_np1, "ubar_np1", dom.state_size),
                                          _ptr(ubar_n, "ubar_n", dom.state_size),
                                          _ptr(work, "work", dom.vjp_work_size), float(cweight)))


def gh_constraint_energy_vjp(dom, u, weight, ubar):
    """ubar += weight * d(sum of the shells' constraint norms)/du."""
    dom._stream()
    dom._check(_lib.gh_constraint_energy_vjp(dom.handle, _ptr(u, "u", dom.state_size), float(weight),
                                             _ptr(ubar, "ubar", dom.state_size)))


def gh_perturbation_vjp(dom, kind, Rc, w, lmax, ubar):
    """Gradient of <ubar, u> with respect to the perturbation coefficients (numpy array)."""
    import numpy as np
    g = np.zeros((lmax + 1) ** 2)
    dom._stream()
    dom._check(_lib.gh_perturbation_vjp(dom.handle, int(kind), float(Rc), float(w), int(lmax),
                                        _ptr(ubar, "ubar", dom.state_size), g.ctypes.data_as(ctypes.c_void_p)))
    return g


def new_vjp_work(dom):
    """A zeroed device work area for the step VJPs."""
    return torch.zeros(dom.vjp_work_size, dtype=torch.float64, device="cuda")


def gh_sync(dom):
    """gh_sync: wait until the domain's stream is idle; raises on an error
    latched on the device (and clears it)."""
    dom._check(_lib.gh_sync(dom.handle))
