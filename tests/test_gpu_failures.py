"""Failure detection on the GPU without faulting it: host-side fault injection
(GH_FAULT) and the device's non-finite latch, driven by ordinary data.

* GH_FAULT=launch: every compute entry point returns GH_ECUDA before it
  launches anything, and the domain works again once the variable is unset.
* GH_FAULT=host_alloc: gh_rk4_step_host's second device allocation fails; the
  call reports GH_ENOMEM, and the next call allocates all of its buffers again
  instead of stepping on a missing one.
* A NaN written into one value of the state (a host-made input, nothing
  faults) makes the constraint norm non-finite; gh_sync reports GH_ENONFINITE
  once and clears the latch.
"""
import os

import numpy as np
import pytest
import torch

from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture
def fault_env():
    old = os.environ.get("GH_FAULT")
    yield os.environ
    if old is None:
        os.environ.pop("GH_FAULT", None)
    else:
        os.environ["GH_FAULT"] = old


def _domain():
    from paper_1804_09101_gb300 import gh
    w = workloads.schwarzschild_single_shell()
    dom = gh.Domain.from_workload(w)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    u += torch.from_numpy(w.noise()).cuda()
    return w, dom, u


def test_injected_launch_failure_stops_every_compute_call_before_it_launches(fault_env):
    from paper_1804_09101_gb300 import gh
    w, dom, u = _domain()
    k = dom.new_state()
    kb = dom.new_state()
    work = dom.new_work()
    norm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    gh.gh_sync(dom)
    n0 = dom.launch_count()
    fault_env["GH_FAULT"] = "launch"
    calls = {
        "gh_rhs": lambda: gh.gh_rhs(dom, u, k),
        "gh_rhs_noalloc": lambda: gh.gh_rhs_noalloc(dom, u, k),
        "gh_rk4_step": lambda: gh.gh_rk4_step(dom, w.dt, u, work, norm2),
        "gh_constraints": lambda: gh.gh_constraints(dom, u, None, norm2),
        "gh_apply_filters": lambda: gh.gh_apply_filters(dom, u, work),
        "gh_rhs_vjp": lambda: gh.gh_rhs_vjp(dom, u, k, kb),
    }
    before = to_host(u).copy()
    for name, call in calls.items():
        with pytest.raises(gh.GHError) as e:
            call()
        assert e.value.status == gh.GH_ECUDA and "GH_FAULT=launch" in str(e.value), name
    assert dom.launch_count() == n0                       # nothing was launched
    assert np.array_equal(to_host(u), before)             # the state is untouched
    del fault_env["GH_FAULT"]
    gh.gh_rhs(dom, u, k)
    gh.gh_rhs_noalloc(dom, u, k)
    gh.gh_sync(dom)
    assert dom.launch_count() > n0


def test_failed_host_step_allocation_reports_enomem_and_the_next_call_recovers(fault_env):
    from paper_1804_09101_gb300 import gh
    w, dom, u = _domain()
    u_host = u.detach().cpu().pin_memory()
    out1 = torch.empty_like(u_host).pin_memory()
    out2 = torch.empty_like(u_host).pin_memory()
    n0 = dom.launch_count()
    fault_env["GH_FAULT"] = "host_alloc"
    with pytest.raises(gh.GHError) as e:
        gh.gh_rk4_step_host(dom, w.dt, 1, u_host, out1)
    assert e.value.status == gh.GH_ENOMEM and "host_alloc" in str(e.value)
    assert dom.launch_count() == n0
    del fault_env["GH_FAULT"]
    gh.gh_rk4_step_host(dom, w.dt, 1, u_host, out1)       # allocates all three buffers
    gh.gh_rk4_step_host(dom, w.dt, 1, u_host, out2)       # reuses them
    work = dom.new_work()
    ref = u.clone()
    gh.gh_rk4_step(dom, w.dt, ref, work)
    ref = to_host(ref)
    scale = np.abs(u_host.numpy()).max()
    for out in (out1, out2):
        assert np.abs(out.numpy() - ref).max() <= REL_TOL * scale


def test_nonfinite_input_latches_enonfinite_once(fault_env):
    from paper_1804_09101_gb300 import gh
    w, dom, u = _domain()
    work = dom.new_work()
    norm2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    gh.gh_rk4_step(dom, w.dt, u, work, norm2)
    gh.gh_sync(dom)                                      # finite: no error
    u[12345] = float("nan")                              # one value, written from the host side
    gh.gh_rk4_step(dom, w.dt, u, work, norm2)
    with pytest.raises(gh.GHError) as e:
        gh.gh_sync(dom)
    assert e.value.status == gh.GH_ENONFINITE
    assert not torch.isfinite(norm2).all()
    gh.gh_sync(dom)                                      # the latch was cleared
    fresh = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, fresh)
    gh.gh_rk4_step(dom, w.dt, fresh, work, norm2)
    gh.gh_sync(dom)                                      # finite again, no stale error
    assert torch.isfinite(norm2).all()
