"""gh_rk4_step_host replays its own captured step: it must follow every setter
that changes the step's launches (here the outer condition, the angular
algorithm and a rotating frame) and advance the domain clock like direct
steps, bit for bit against the same steps on a device state."""
import numpy as np
import pytest
import torch

from paper_1804_09101_gb300 import workloads

pytestmark = pytest.mark.gpu


def _gh():
    from paper_1804_09101_gb300 import gh
    return gh


def _kerr2():
    return workloads.Workload(name="kerr2_host", shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0, chi=0.7,
                              gamma1=0.5, radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=9, noise_amp=1e-6)


def _setup():
    gh = _gh()
    w = _kerr2()
    dom = gh.Domain.from_workload(w)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    u += torch.from_numpy(w.noise()).to(u.device)
    return gh, w, dom, u


def _device_steps(gh, dom, dt, u0, n):
    u = u0.clone()
    work = dom.new_work()
    for _ in range(n):
        gh.gh_rk4_step(dom, dt, u, work)
    gh.gh_sync(dom)
    return u.cpu().numpy()


def _host_steps(gh, dom, dt, u0, n):
    src = u0.cpu().pin_memory()
    out = torch.empty_like(src).pin_memory()
    gh.gh_rk4_step_host(dom, dt, n, src, out)
    return out.numpy()


def test_host_path_follows_setter_changes():
    gh, w, dom, u0 = _setup()
    first = _host_steps(gh, dom, w.dt, u0, 2)
    assert np.array_equal(first, _device_steps(gh, dom, w.dt, u0, 2))
    gh.gh_set_outer_bc(dom, gh.GH_BC_CONSTRAINT_PRESERVING)
    cp = _host_steps(gh, dom, w.dt, u0, 2)
    assert np.array_equal(cp, _device_steps(gh, dom, w.dt, u0, 2))
    assert not np.array_equal(cp, first)
    gh.gh_set_algorithm(dom, gh.GH_ALG_SEPARABLE)
    sep = _host_steps(gh, dom, w.dt, u0, 2)
    assert np.array_equal(sep, _device_steps(gh, dom, w.dt, u0, 2))
    # a new dt is a new capture
    half = _host_steps(gh, dom, 0.5 * w.dt, u0, 2)
    assert np.array_equal(half, _device_steps(gh, dom, 0.5 * w.dt, u0, 2))


def test_host_path_rotating_frame_advances_the_clock():
    gh, w, dom, u0 = _setup()
    gh.gh_set_rotating_frame(dom, (0.0, 0.0, 1.0), 0.3)
    gh.gh_set_time(dom, 0.2)
    host = _host_steps(gh, dom, w.dt, u0, 3)
    t_host = gh.gh_get_time(dom)
    gh.gh_set_time(dom, 0.2)
    dev = _device_steps(gh, dom, w.dt, u0, 3)
    assert np.array_equal(host, dev)
    assert abs(t_host - gh.gh_get_time(dom)) == 0.0
    assert abs(t_host - (0.2 + 3 * w.dt)) < 1e-14


def _one_step_calls(gh, dom, dt, u0, n, pinned=True, in_place=False):
    src = u0.cpu()
    if pinned:
        src = src.pin_memory()
    out = src if in_place else (torch.empty_like(src).pin_memory() if pinned else torch.empty_like(src))
    for _ in range(n):
        gh.gh_rk4_step_host(dom, dt, 1, src, out)
        if not in_place:
            src.copy_(out)
    return out.numpy().copy()


def test_one_step_calls_move_the_state_from_the_step_kernels():
    """With one step per call and pinned buffers the step's first radial map
    reads u_in and its last filter writes u_out; the results equal device
    steps bit for bit, also in place (u_in == u_out), after a setter change,
    with a rotating frame, and from pageable buffers (plain copies)."""
    gh, w, dom, u0 = _setup()
    dev = _device_steps(gh, dom, w.dt, u0, 3)
    assert np.array_equal(_one_step_calls(gh, dom, w.dt, u0, 3), dev)
    assert np.array_equal(_one_step_calls(gh, dom, w.dt, u0, 3, in_place=True), dev)
    assert np.array_equal(_one_step_calls(gh, dom, w.dt, u0, 3, pinned=False), dev)
    gh.gh_set_outer_bc(dom, gh.GH_BC_CONSTRAINT_PRESERVING)
    cp = _one_step_calls(gh, dom, w.dt, u0, 2)
    assert np.array_equal(cp, _device_steps(gh, dom, w.dt, u0, 2))
    gh.gh_set_rotating_frame(dom, (0.0, 0.0, 1.0), 0.3)
    gh.gh_set_time(dom, 0.1)
    host = _one_step_calls(gh, dom, w.dt, u0, 2)
    t_host = gh.gh_get_time(dom)
    gh.gh_set_time(dom, 0.1)
    assert np.array_equal(host, _device_steps(gh, dom, w.dt, u0, 2))
    assert t_host == gh.gh_get_time(dom)


def test_one_step_call_norms_match_the_device_step():
    gh, w, dom, u0 = _setup()
    src = u0.cpu().pin_memory()
    out = torch.empty_like(src).pin_memory()
    n_host = torch.zeros(len(w.shells), dtype=torch.float64)
    gh.gh_rk4_step_host(dom, w.dt, 1, src, out, n_host)
    u = u0.clone()
    n_dev = torch.zeros(len(w.shells), dtype=torch.float64, device="cuda")
    gh.gh_rk4_step(dom, w.dt, u, dom.new_work(), n_dev)
    gh.gh_sync(dom)
    assert np.array_equal(out.numpy(), u.cpu().numpy())
    assert np.array_equal(n_host.numpy(), n_dev.cpu().numpy())
