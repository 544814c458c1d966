"""Batched evolution of independent holes in one domain: parity with the
oracle (one oracle domain per hole), bitwise agreement with the plain
per-hole launch loop, per-hole time steps, and CUDA-graph replay."""
import numpy as np
import pytest
import torch

from oracle import evolve
from paper_1804_09101_gb300 import workloads
from parity_helpers import REL_TOL, assert_output_parity, flat, to_dev, to_host

pytestmark = pytest.mark.gpu


def _small_batch():
    # three holes: two single-shell holes of different (n_r, L) and one two-shell hole
    holes = [dict(M=1.0, chi=0.3, shells=[(1.6, 8.0, 9, 7)], dt=0.004, seed=11),
             dict(M=0.7, chi=0.8, shells=[(0.9, 3.0, 7, 11), (3.0, 9.0, 7, 11)], dt=0.003, seed=12),
             dict(M=1.5, chi=0.0, shells=[(2.5, 20.0, 11, 5)], dt=0.006, seed=13)]
    return holes


def _build(holes, gh, keep=-2):
    shells = [s + (b,) for b, h in enumerate(holes) for s in h["shells"]]
    dom = gh.Domain(shells, radial_filter_on=True, sh_keep_l=keep)
    u = dom.new_state()
    for b, h in enumerate(holes):
        gh.gh_set_analytic_kerr_schild(dom, b, h["M"], h["chi"], u)
        gh.gh_set_dt_scale(dom, b, h["dt"])
    noise = np.concatenate([np.random.default_rng(h["seed"]).standard_normal(
        50 * sum(n * 2 * (L + 1) ** 2 for (_, _, n, L) in h["shells"])) * 1e-8 for h in holes])
    u += to_dev(noise)
    return dom, u, noise


def test_batched_rk4_matches_oracle_per_hole():
    from paper_1804_09101_gb300 import gh
    holes = _small_batch()
    dom, u, noise = _build(holes, gh)
    u_start = to_host(u).copy()
    work = dom.new_work()
    for _ in range(2):
        gh.gh_rk4_step(dom, 1.0, u, work)
    got = to_host(u)
    off = 0
    for h in holes:
        keep = -2
        odom = evolve.Domain(h["shells"], h["M"], h["chi"], radial_filter_on=True, sh_keep_l=0)
        n = 50 * sum(nr * 2 * (L + 1) ** 2 for (_, _, nr, L) in h["shells"])
        # per-shell floor(2L/3) truncation: one hole has one L
        odom.sh_keep_l = (2 * h["shells"][0][3]) // 3
        ref = []
        o = off
        for shp in odom.shapes():
            m = int(np.prod(shp))
            ref.append(u_start[o:o + m].reshape(shp))
            o += m
        for _ in range(2):
            ref = evolve.rk4_step(odom, ref, h["dt"])
        err = np.abs(got[off:off + n] - flat(ref)).max() / np.abs(u_start[off:off + n]).max()
        assert err < REL_TOL, (h, err)
        off += n


def test_batched_equals_plain_per_hole_loop_bitwise():
    from paper_1804_09101_gb300 import gh
    holes = _small_batch()
    dom, u, _ = _build(holes, gh)
    work = dom.new_work()
    gh.gh_rk4_step(dom, 1.0, u, work)
    got = to_host(u)
    off = 0
    for h in holes:
        d1, u1, _ = _build([h], gh)
        gh.gh_rk4_step(d1, 1.0, u1, d1.new_work())
        n = d1.state_size
        assert np.array_equal(got[off:off + n], to_host(u1)), h
        off += n


def test_graph_replay_equals_direct_steps():
    from paper_1804_09101_gb300 import gh
    holes = _small_batch()
    dom, u, _ = _build(holes, gh)
    u2 = u.clone()
    work = dom.new_work()
    work2 = dom.new_work()
    for _ in range(3):
        gh.gh_rk4_step(dom, 1.0, u, work)
    gh.gh_rk4_graph_capture(dom, 1.0, u2, work2)
    gh.gh_rk4_graph_launch(dom, 3)
    gh.gh_sync(dom)
    assert np.array_equal(to_host(u), to_host(u2))


def test_radial_map_on_the_side_stream_changes_no_bit():
    """gh_set_overlap: the radial map on the domain's second stream, beside the
    angular maps, against both on one stream: direct steps, a graph replay and
    a right-hand side issued on a user stream are bitwise the same."""
    from paper_1804_09101_gb300 import gh
    holes = _small_batch()
    runs = []
    for on in (0, 1):
        dom, u, _ = _build(holes, gh)
        gh.gh_set_overlap(dom, on)
        work = dom.new_work()
        for _ in range(2):
            gh.gh_rk4_step(dom, 1.0, u, work)
        u2 = u.clone()
        work2 = dom.new_work()
        gh.gh_rk4_graph_capture(dom, 1.0, u2, work2)
        gh.gh_rk4_graph_launch(dom, 2)
        user = torch.cuda.Stream()
        user.wait_stream(torch.cuda.current_stream())   # after the replays
        with torch.cuda.stream(user):
            k = dom.new_state()
            gh.gh_rhs(dom, u2, k)
            kh = k.cpu()
        torch.cuda.synchronize()
        runs.append((to_host(u), to_host(u2), kh.numpy()))
    for name, a, b in zip(("steps", "replays", "rhs on a user stream"), runs[0], runs[1]):
        assert np.array_equal(a, b), (name, np.abs(a - b).max())
    assert gh._lib.gh_set_overlap(dom.handle, 2) != 0      # GH_EINVAL


def test_host_buffer_steps_equal_device_steps_bitwise():
    """gh_rk4_step_host (host state in and out, pinned or pageable) against the
    same steps on a device state, with the constraint norms of the last step."""
    from paper_1804_09101_gb300 import gh
    holes = _small_batch()
    dom, u, _ = _build(holes, gh)
    u0 = to_host(u).copy()
    work = dom.new_work()
    n2 = torch.zeros(len(dom.shells), dtype=torch.float64, device="cuda")
    for _ in range(3):
        gh.gh_rk4_step(dom, 1.0, u, work, n2)
    want, want_n2 = to_host(u), n2.cpu().numpy()
    for pinned in (True, False):
        src = torch.from_numpy(u0.copy())
        out = torch.empty_like(src)
        norms = torch.zeros(len(dom.shells), dtype=torch.float64)
        if pinned:
            src, out, norms = src.pin_memory(), out.pin_memory(), norms.pin_memory()
        gh.gh_rk4_step_host(dom, 1.0, 3, src, out, norms)
        assert np.array_equal(out.numpy(), want), pinned
        assert np.array_equal(norms.numpy(), want_n2), pinned
    inplace = torch.from_numpy(u0.copy()).pin_memory()
    gh.gh_rk4_step_host(dom, 1.0, 3, inplace, inplace)
    assert np.array_equal(inplace.numpy(), want)


def test_batched_workload_builds_and_steps():
    from paper_1804_09101_gb300 import gh
    w = workloads.batched_workload(n_bh=8)
    dom = gh.Domain(w.shells, radial_filter_on=True, sh_keep_l=-2)
    u = dom.new_state()
    for b, h in enumerate(w.holes):
        gh.gh_set_analytic_kerr_schild(dom, b, h["M"], h["chi"], u)
        gh.gh_set_dt_scale(dom, b, h["dt"])
    u0 = u.clone()
    work = dom.new_work()
    n2 = torch.zeros(len(w.holes), dtype=torch.float64, device="cuda")
    for _ in range(5):
        gh.gh_rk4_step(dom, 1.0, u, work, n2)
    gh.gh_sync(dom)
    # every hole stays finite over a few steps; under-resolved rapidly spinning
    # holes at L = 7 drift by their (large) truncation error, so only a loose
    # bound is meaningful here
    assert torch.isfinite(u).all()
    assert float((u - u0).abs().max()) < float(u0.abs().max())


def test_full_size_batched_workload_sampled_holes_match_oracle():
    """The full 64-hole workload (613,888 points, one domain, autotuned, one
    captured CUDA graph per RK4 step, as the benchmark runs it) on the
    oracle's exact data plus seeded noise: the right-hand side of every point
    of the largest hole and of three seeded sample holes, and their state
    after one graph-launched RK4 step (each hole with its own dt), against the
    oracle run on each of those holes alone."""
    from paper_1804_09101_gb300 import gh
    w = workloads.batched_workload(64)
    # noise of 1e-4 keeps every hole's right-hand side far above rounding
    # (the best-resolved holes' exact-data right-hand side is below 1e-6), so
    # the output-relative bar means something
    w.noise_amp = 1e-4
    odoms = [evolve.Domain([(h["r_in"], h["r_out"], h["n_r"], h["L"])], h["M"], h["chi"], w.gamma0, w.gamma1,
                           w.gamma2, w.filt_alpha, w.filt_order, True, (2 * h["L"]) // 3) for h in w.holes]
    u_host = np.concatenate([flat(od.u_exact) for od in odoms]) + w.noise()
    dom = gh.Domain(w.shells, w.gamma0, w.gamma1, w.gamma2, w.filt_alpha, w.filt_order, True, -2)
    gh.gh_set_gauge(dom, to_dev(np.concatenate([flat(od.H) for od in odoms])),
                    to_dev(np.concatenate([flat(od.dH) for od in odoms])))
    gh.gh_set_background(dom, to_dev(np.concatenate([flat(od.u_exact) for od in odoms])))
    for b, h in enumerate(w.holes):
        gh.gh_set_dt_scale(dom, b, h["dt"])
    gh.gh_autotune(dom, 3)
    u = to_dev(u_host)
    k = dom.new_state()
    gh.gh_rhs(dom, u, k)
    k_host = to_host(k)
    del k
    work = dom.new_work()
    gh.gh_rk4_graph_capture(dom, 1.0, u, work)     # the capture does not step u
    gh.gh_rk4_graph_launch(dom, 1)
    u1 = to_host(u)
    offs = np.cumsum([0] + [50 * h["n_r"] * 2 * (h["L"] + 1) ** 2 for h in w.holes])
    largest = int(np.argmax(np.diff(offs)))
    picks = sorted({largest} | set(int(b) for b in np.random.default_rng(9).choice(len(w.holes), 3, replace=False)))
    for b in picks:
        od, h = odoms[b], w.holes[b]
        sl = slice(offs[b], offs[b + 1])
        ub = [u_host[sl].reshape(od.shapes()[0])]
        scale = np.abs(u_host[sl]).max()
        assert_output_parity(k_host[sl], flat(evolve.rhs(od, ub)), scale, (b, h))
        assert np.abs(u1[sl] - flat(evolve.rk4_step(od, ub, h["dt"]))).max() <= REL_TOL * scale, (b, h)
