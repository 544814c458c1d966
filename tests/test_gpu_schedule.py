"""The work-schedule autotuner and explicit schedules: every schedule of the
radial and folded angular maps gives bitwise identical derivatives, filters
and RK4 steps; invalid schedules are rejected."""
import numpy as np
import pytest
import torch

from paper_1804_09101_gb300 import gh, workloads

pytestmark = pytest.mark.gpu


def _domain():
    w = workloads.kerr_four_shells(n_r=9, L=7)
    dom = gh.Domain.from_workload(w)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    g = torch.Generator().manual_seed(7)
    u += 1e-6 * torch.randn(dom.state_size, generator=g, dtype=torch.float64).to(u.device)
    return w, dom, u


def _outputs(w, dom, u):
    d = torch.empty((3, dom.state_size), dtype=torch.float64, device=u.device)
    gh.gh_derivatives(dom, u, d)
    f = u.clone()
    gh.gh_apply_filters(dom, f, dom.new_work())
    s = u.clone()
    gh.gh_rk4_step(dom, w.dt, s, dom.new_work())
    torch.cuda.synchronize()
    return d.cpu().numpy(), f.cpu().numpy(), s.cpu().numpy()


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_autotune_keeps_results_bitwise():
    w, dom, u = _domain()
    ref = _outputs(w, dom, u)
    gh.gh_autotune(dom, reps=2)
    sched = gh.gh_get_schedule(dom)
    assert 2 <= sched["radial_chains"] <= 4 and 1 <= sched["radial_groups"] <= 4
    assert sched["fold_deriv_threads"] % 32 == 0
    _same(ref, _outputs(w, dom, u))


@pytest.mark.parametrize("sched", [
    (2, 1, 2, 1, 128, 49152, 128, 49152, 1),
    (3, 2, 4, 3, 32, 8192, 64, 8192, 0),
    (4, 4, 3, 2, 512, 200 * 1024, 256, 112 * 1024, 1),
    (2, 3, 2, 4, 96, 24576, 480, 65536, 0),
])
def test_every_schedule_gives_identical_results(sched):
    w, dom, u = _domain()
    ref = _outputs(w, dom, u)
    gh.gh_set_schedule(dom, dict(zip(gh.SCHEDULE_KEYS, sched)))
    assert tuple(gh.gh_get_schedule(dom).values()) == sched
    _same(ref, _outputs(w, dom, u))


@pytest.mark.parametrize("bad", [
    (1, 1, 2, 1, 128, 49152, 128, 49152, 0),     # chains < 2
    (2, 5, 2, 1, 128, 49152, 128, 49152, 0),     # groups > 4
    (2, 1, 2, 1, 100, 49152, 128, 49152, 0),     # threads not a multiple of 32
    (2, 1, 2, 1, 128, 1024, 128, 49152, 0),      # budget below 8 KiB
    (2, 1, 2, 1, 128, 49152, 1024, 49152, 0),    # threads above 512
    (2, 1, 2, 1, 128, 49152, 128, 49152, 2),     # pair split not 0 or 1
])
def test_invalid_schedules_are_rejected(bad):
    w, dom, u = _domain()
    with pytest.raises(RuntimeError):
        gh.gh_set_schedule(dom, dict(zip(gh.SCHEDULE_KEYS, bad)))


def test_schedules_of_two_domains_do_not_interfere():
    # the shared-memory limit of a kernel is process-wide: a second domain with
    # a small schedule must not break the launches of a first one with a large
    # schedule
    w1 = workloads.kerr_four_shells(n_r=9, L=15)
    d1 = gh.Domain.from_workload(w1)
    u1 = d1.new_state()
    gh.gh_set_analytic_kerr_schild(d1, -1, w1.M, w1.chi, u1)
    s = gh.gh_get_schedule(d1)
    s.update(fold_deriv_budget=200 * 1024, fold_filter_budget=200 * 1024)
    gh.gh_set_schedule(d1, s)
    ref = _outputs(w1, d1, u1)
    w2, d2, u2 = _domain()
    s2 = gh.gh_get_schedule(d2)
    s2.update(fold_deriv_budget=8192, fold_filter_budget=8192)
    gh.gh_set_schedule(d2, s2)
    _outputs(w2, d2, u2)
    _same(ref, _outputs(w1, d1, u1))


@pytest.mark.parametrize("cweight", [0.0, 0.01])
def test_pair_split_and_per_point_reverse_passes_agree(cweight):
    w, dom, u = _domain()
    N = dom.state_size
    g = torch.Generator().manual_seed(11)
    kb = torch.randn(N, generator=g, dtype=torch.float64).to(u.device)
    work = gh.new_vjp_work(dom)
    stages = torch.empty(3 * N, dtype=torch.float64, device=u.device)
    s0 = u.clone()
    gh.gh_rk4_step_save(dom, w.dt, s0.clone(), dom.new_work(), stages)
    out = {}
    for split in (0, 1):
        sch = gh.gh_get_schedule(dom)
        sch["adjoint_pair_split"] = split
        gh.gh_set_schedule(dom, sch)
        ub = torch.zeros_like(u)
        gh.gh_rhs_vjp(dom, u, kb, ub)
        nx = torch.zeros_like(u)
        gh.gh_rk4_step_vjp_saved(dom, w.dt, s0, stages, kb, nx, work, cweight)
        torch.cuda.synchronize()
        out[split] = (ub.cpu().numpy(), nx.cpu().numpy())
    for a, b in zip(out[0], out[1]):
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())
