"""Parity of the library's Dormand-Prince 5(4) step (Sec. 2.1's stepper) with
the oracle's, through the C ABI: the error norm, the accept/reject decision,
the next step size and the new state, for an accepted and a rejected attempt
and for a short adaptive evolution; plus argument checks."""
import numpy as np
import pytest

from oracle import dp5 as odp5
from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, flat, unflat, to_dev, to_host, oracle_domain, oracle_initial_state, gpu_domain

pytestmark = pytest.mark.gpu


def _gh():
    from paper_1804_09101_gb300 import gh
    return gh


def _kerr2():
    return workloads.Workload(name="kerr2", shells=[(1.3, 3.0, 9, 7), (3.0, 6.0, 9, 7)], M=1.0, chi=0.9,
                              radial_filter_on=True, sh_keep_l=4, dt=0.005, seed=7, noise_amp=1e-6)


CASES = {"schwarzschild": workloads.schwarzschild_single_shell, "kerr2": _kerr2}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    w = CASES[request.param]()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    return w, odom, u0


def _err_tol(err):
    # the error estimate is a small difference of stage derivatives, so its
    # rounding is relative to the stages, not to err itself
    return 1e-6 * max(err, 1e-3)


@pytest.mark.parametrize("dt,rtol", [(0.02, 1e-9), (0.4, 1e-12)])
def test_single_attempt_matches_oracle(case, dt, rtol):
    gh = _gh()
    w, odom, u0 = case
    dom = gpu_domain(w, odom)
    u = to_dev(flat(u0))
    work = gh.new_dp5_work(dom)
    err, ok, dtn = gh.gh_dp5_step(dom, dt, rtol, rtol, u, work)
    ou, oerr, ook, odtn = odp5.dp5_step(odom, u0, dt, rtol, rtol)
    assert abs(err - oerr) <= _err_tol(oerr), (err, oerr)
    assert ok == ook
    assert abs(dtn - odtn) <= 0.2 * _err_tol(oerr) / max(oerr, 1e-3) * odtn + 1e-15
    scale = np.abs(flat(u0)).max()
    assert np.abs(to_host(u) - flat(ou)).max() <= REL_TOL * scale
    if not ok:
        assert np.array_equal(to_host(u), flat(u0))


def test_short_adaptive_evolution_matches_oracle():
    gh = _gh()
    w = _kerr2()
    odom = oracle_domain(w)
    u0 = oracle_initial_state(w, odom)
    dom = gpu_domain(w, odom)
    u = to_dev(flat(u0))
    work = gh.new_dp5_work(dom)
    dt_g = dt_o = 0.3
    ou = u0
    seq_g, seq_o = [], []
    for _ in range(5):
        err, ok, dt_g = gh.gh_dp5_step(dom, dt_g, 1e-8, 1e-8, u, work)
        ou, oerr, ook, dt_o = odp5.dp5_step(odom, ou, dt_o, 1e-8, 1e-8)
        seq_g.append(ok)
        seq_o.append(ook)
        assert abs(dt_g - dt_o) <= 1e-6 * dt_o
    assert seq_g == seq_o and not all(seq_g) and any(seq_g)
    assert np.abs(to_host(u) - flat(ou)).max() <= REL_TOL * np.abs(flat(u0)).max()


def test_arguments_are_checked():
    gh = _gh()
    w = workloads.schwarzschild_single_shell()
    dom = gh.Domain.from_workload(w)
    u = dom.new_state()
    work = gh.new_dp5_work(dom)
    for dt, rtol, atol in [(0.0, 1e-8, 1e-8), (-1.0, 1e-8, 1e-8), (0.1, -1.0, 1e-8), (0.1, 0.0, 0.0)]:
        with pytest.raises(RuntimeError):
            gh.gh_dp5_step(dom, dt, rtol, atol, u, work)
    gh.gh_set_dt_scale(dom, 0, 0.5)
    with pytest.raises(RuntimeError):
        gh.gh_dp5_step(dom, 0.1, 1e-8, 1e-8, u, work)
