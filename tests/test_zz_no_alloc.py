"""gh_rhs_noalloc (no device allocation at call time) against gh_rhs.

Callers that cannot allocate GPU memory while they run (a host whose memory
pool owns the device, a time-critical loop) use gh_rhs_noalloc; it must give
the same right-hand side as gh_rhs, call after call, even though every call
reuses the same fixed work area inside the library.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, flat, to_dev, to_host, oracle_domain, oracle_initial_state, gpu_domain

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algorithm", ["default", "folded", "separable", "dense"])
def test_noalloc_rhs_matches_gh_rhs_on_two_calls_in_a_row(algorithm):
    """Every angular algorithm writes its outputs into the shared array, which
    still holds the previous call's values: the results must equal gh_rhs bit
    for bit (same kernels, same order), on two calls in a row with different
    inputs, and within the parity tolerance of each other's scale."""
    from paper_1804_09101_gb300 import gh
    w = workloads.schwarzschild_single_shell()
    odom = oracle_domain(w)
    u0 = flat(oracle_initial_state(w, odom))
    dom = gpu_domain(w, odom, algorithm=algorithm)
    scale = np.abs(u0).max()
    inputs = [u0, u0 + 1e-6 * np.random.default_rng(1).standard_normal(u0.shape)]
    for x in inputs:                       # two calls in a row, different inputs
        u = to_dev(x)
        ref = dom.new_state()
        gh.gh_rhs(dom, u, ref)
        got = dom.new_state()
        gh.gh_rhs_noalloc(dom, u, got)
        got, ref = to_host(got), to_host(ref)
        assert np.array_equal(got, ref), np.abs(got - ref).max() / scale
        assert np.abs(got - ref).max() / scale < REL_TOL


def test_noalloc_rejects_a_domain_larger_than_its_work_area():
    from paper_1804_09101_gb300 import gh
    w = workloads.kerr_four_shells()          # 2,150,400 doubles > 2^20
    dom = gh.Domain.from_workload(w)
    u = dom.new_state()
    k = dom.new_state()
    with pytest.raises(gh.GHError) as e:
        gh.gh_rhs_noalloc(dom, u, k)
    assert e.value.status == gh.GH_EINVAL and "work area" in str(e.value)
