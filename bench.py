"""Benchmark: GH right-hand-side grid-point evaluations per second on one GB300.

One step = one full pass of the hot path on the 4-shell Kerr workload
(a = 0.9, M = 1, shells [1.3, 3, 6, 12, 30], N_r = 21, L = 15; 43,008 points):
an RK4 step (4 right-hand sides with derivatives, the fused GH kernel,
characteristic boundary conditions and stage combines), the exponential
Chebyshev and SH 2/3 filters, and the quadrature constraint norms (computed
inside the first stage).  Throughput = points x 4 RHS evaluations per step / time.

Each timed step replays the step captured once as a CUDA graph
(gh_rk4_graph_capture / gh_rk4_graph_launch; --no-graph times direct
gh_rk4_step calls).  The per-kernel times behind the roofline come from a second
timed region of the same steps called directly with the library's CUDA-event
brackets, which would otherwise add gaps to the headline region.  The state
(17 MB) fits in L2, so L2 is flushed (a 256 MB write) before every timed step,
outside the step's events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (torchrun, one rank per GPU) every rank evolves its own replica:
the workload is one coupled black hole and does not shard (replicas only).
"--impl reference" times the CPU oracle (the only reference this method has).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel
# from the ncu captures of the current kernels (None once a kernel changes).
TRAFFIC_PER_LAUNCH = {
    # pointwise_kernel<1,0,0>, 4-shell L=15: 122.1 MB read + 110.1 MB written
    ("kerr_a0.9_4shells_nr21_L15", "folded", "pointwise"): 232.2e6,
    # fold_angular_kernel<1>, 8-shell L=31: 269.1 MB read + 482.5 MB written
    ("kerr_a0.95_8shells_nr41_L31", "folded", "angular"): 751.6e6,
    # fold_angular_kernel<1>, 4-shell L=15: 17.3 MB read + 8.7 MB written
    ("kerr_a0.9_4shells_nr21_L15", "folded", "angular"): 26.0e6,
    # fold_angular_kernel<1>, the paper's 2-shell L=18 grid: 5.9 MB read, 0 written (L2-resident)
    ("paper_singlebh_chi0.2_0.3_0.4_2shells_nr10_L18", "folded", "angular"): 5.9e6,
}

METRIC = "GH RHS grid-point evals/s (FP64, 1 GB300) + % roofline; batched vs plain; adjoint/fwd"
UNIT = "grid-point RHS evals/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true",
                   help="keep the default work schedule instead of running gh_autotune before timing")
    p.add_argument("--stepper", default="rk4", choices=["rk4", "dp5"],
                   help="rk4 (fixed step, the headline) or dp5 (Dormand-Prince 5(4), adaptive)")
    p.add_argument("--schedule", default=None,
                   help="explicit work schedule as JSON (keys of gh.SCHEDULE_KEYS) instead of gh_autotune")
    p.add_argument("--workload", default="kerr4",
                   choices=["kerr4", "large", "schwarzschild", "batched", "adjoint", "families", "paper"],
                   help="kerr4: 4-shell Kerr a=0.9 (default, the headline); large: 8-shell Kerr a=0.95, "
                        "N_r=41, L=31; schwarzschild: 1 shell N_r=11, L=7; batched: 64 independent "
                        "single-shell holes of uneven resolution, one CUDA graph per RK4 step, "
                        "compared with the plain per-hole launch loop")
    p.add_argument("--no-graph", action="store_true",
                   help="time direct gh_rk4_step calls instead of replays of the captured step graph")
    p.add_argument("--no-overlap", action="store_true",
                   help="run the radial and angular derivative maps one after the other on one stream "
                        "(default: the radial map on the domain's second stream, beside the angular maps)")
    p.add_argument("--sh-filter", default="component", choices=["component", "tensor"],
                   help="angular filter: per Cartesian component (default) or tensor spherical harmonics "
                        "(spin-weighted harmonics in the complex frame)")
    p.add_argument("--algorithm", default="auto", choices=["auto", "folded", "separable", "dense"],
                   help="angular maps: folded separable (default), plain separable, or dense traced matrices")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


# ------------------------------------------------------------- oracle timing
def oracle_setup(w):
    import numpy as np
    from oracle import evolve, perturb
    dom = evolve.Domain(w.shells, w.M, w.chi, w.gamma0, w.gamma1, w.gamma2, w.filt_alpha,
                        w.filt_order, w.radial_filter_on, w.sh_keep_l)
    u = []
    for s, g in enumerate(dom.grids):
        p = w.pulse
        u.append(dom.u_exact[s] + perturb.psi_pulse(g, dom.u_exact[s], p.amplitude, p.center, p.width,
                                                      p.lmax, p.coeffs))
    return dom, u


def cpu_baseline(w, min_seconds=10.0):
    """Time the oracle's full right-hand side (all shells) until >= min_seconds."""
    from oracle import evolve
    dom, u = oracle_setup(w)
    evals = 0
    t0 = time.perf_counter()
    while True:
        evolve.rhs(dom, u)
        evals += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return dict(value=w.points() * evals / el, unit=UNIT, cores=blas_threads(), kind="oracle",
                sample="%d full right-hand-side evaluation(s) of the 4-shell workload (%d points), "
                       "%.1f s, numpy FP64 on the host" % (evals, w.points(), el))


REFERENCE_BUDGET_S = 150.0     # the whole --impl reference run, warm-up included


def run_reference(args, w):
    """The oracle on the host cores, timed per step.  A step is one full oracle
    right-hand side of the workload when the run fits the time budget at that
    size; otherwise a bounded sample of it: the interior right-hand side of one
    shell, taking the shells in turn (about a quarter of the work, no
    boundary exchange).  The value counts the points each step evaluated."""
    import types
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import evolve
    dom, u = oracle_setup(w)
    t0 = time.perf_counter()
    evolve.rhs(dom, u)                       # first warm-up step, also sizes the sample
    t_full = time.perf_counter() - t0
    full = t_full * (args.steps + args.warmup) <= REFERENCE_BUDGET_S
    shells_pts = [g["n_r"] * g["n_th"] * g["n_ph"] for g in dom.grids]

    def step(i):
        if full:
            evolve.rhs(dom, u)
            return w.points()
        s = i % len(dom.grids)
        one = types.SimpleNamespace(grids=[dom.grids[s]], H=[dom.H[s]], dH=[dom.dH[s]],
                                    gamma0=dom.gamma0, gamma1=dom.gamma1, gamma2=dom.gamma2)
        evolve.rhs_interior(one, [u[s]])
        return shells_pts[s]

    for i in range(args.warmup - 1):
        step(i)
    pts = 0
    t0 = time.perf_counter()
    for i in range(args.steps):
        pts += step(i)
    el = time.perf_counter() - t0
    value = pts / el
    what = ("one full oracle right-hand-side evaluation (all %d shells)" % len(dom.grids) if full else
            "the oracle's interior right-hand side of one shell, the shells in turn (a bounded sample: "
            "a full right-hand side takes %.2f s here)" % t_full)
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000.0 * el / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=w.name, points=w.points(), step=what),
                cpu_baseline=dict(value=value, unit=UNIT, cores=blas_threads(), kind="oracle",
                                  sample="%d steps of %s; %d points evaluated" % (args.steps, what, pts)),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.skip = 0
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def _rows(self):
        self.f.flush()
        rows = []
        for ln in open(self.f.name):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        return rows

    def start(self):
        """Start sampling every 50 ms and wait for the first sample, so that the
        samples taken from here on fall inside the region timed next."""
        self.skip = 0
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and not self._rows():
            time.sleep(0.02)
        self.skip = len(self._rows())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        allrows = self._rows()
        os.unlink(self.f.name)
        rows = allrows[self.skip:] or allrows[-1:]     # the samples inside the timed region
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(smax) if smax else None,
                    reasons=reasons, samples=len(allrows) - self.skip, interval_ms=50)


# ------------------------------------------------------------- our arm
def run_ours(args, w):
    import torch
    from paper_1804_09101_gb300 import build
    build.build()
    from paper_1804_09101_gb300 import costmodel, gh, replicas

    rank, world, local = dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    dom = gh.Domain.from_workload(w)
    gh.gh_set_overlap(dom, not args.no_overlap)
    if args.algorithm == "auto":
        args.algorithm = "folded"          # the library's default
    else:
        gh.gh_set_algorithm(dom, {"dense": gh.GH_ALG_DENSE, "separable": gh.GH_ALG_SEPARABLE,
                                  "folded": gh.GH_ALG_SEPARABLE_FOLDED}[args.algorithm])
    if args.schedule:
        gh.gh_set_schedule(dom, json.loads(args.schedule))
    elif not args.no_autotune:
        gh.gh_autotune(dom, 5)
    if args.sh_filter == "tensor":
        gh.gh_set_sh_filter(dom, "tensor")
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    p = w.pulse
    if p is not None:
        gh.gh_add_perturbation(dom, 0, p.amplitude, p.center, p.width, p.lmax, p.coeffs, u)
    if w.noise_amp:
        u += torch.from_numpy(w.noise()).to(dev)
    work = dom.new_work()
    norm2 = torch.zeros(len(w.shells), dtype=torch.float64, device=dev)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()

    for _ in range(args.warmup):
        flush.zero_()
        gh.gh_rk4_step(dom, w.dt, u, work, norm2)
    gh.gh_sync(dom)
    use_graph = not args.no_graph
    if use_graph:
        # the step as one captured CUDA graph (the library's API for repeated
        # steps); warm-up replays
        gh.gh_rk4_graph_capture(dom, w.dt, u, work, norm2)
        for _ in range(args.warmup):
            flush.zero_()
            gh.gh_rk4_graph_launch(dom, 1)
        gh.gh_sync(dom)

    def one_step():
        if use_graph:
            gh.gh_rk4_graph_launch(dom, 1)
        else:
            gh.gh_rk4_step(dom, w.dt, u, work, norm2)

    # ---- device-resident timed region (the headline value)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    n0 = dom.launch_count()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        one_step()
        ev[i][1].record(stream)
    barrier()
    launches = dom.launch_count() - n0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    gh.gh_sync(dom)
    total_ms = replicas.max_over_ranks(total_ms, pg)

    # ---- second timed region: the same steps, called directly with the
    # library's per-family CUDA-event brackets (on the domain's stream), for
    # the kernel times and the roofline (the brackets' event records would
    # add gaps to the headline region)
    gh.gh_profile_enable(dom, True)
    for fam in range(len(gh.KERNEL_FAMILIES)):
        gh.gh_profile_read(dom, fam)
    barrier()
    for i in range(args.steps):
        flush.zero_()
        gh.gh_rk4_step(dom, w.dt, u, work, norm2)
    barrier()
    fam_ms = {}
    for fam, name in enumerate(gh.KERNEL_FAMILIES):
        fam_ms[name] = gh.gh_profile_read(dom, fam)
    gh.gh_profile_enable(dom, False)
    gh.gh_sync(dom)

    pts = w.points()
    value = replicas.job_throughput(pts * 4 * args.steps, world, total_ms)

    # ---- end to end through the C ABI with host buffers: gh_rk4_step_host copies
    # the state in from pinned host memory, steps, and copies the state and the
    # constraint norms out, every step
    u_host = u.detach().cpu().pin_memory()
    out_host = torch.empty_like(u_host).pin_memory()
    n_host = torch.empty(len(w.shells), dtype=torch.float64).pin_memory()
    gh.gh_rk4_step_host(dom, w.dt, 1, u_host, out_host, n_host)     # allocates its device buffers
    e2e_ms = 0.0
    barrier()
    for i in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gh.gh_rk4_step_host(dom, w.dt, 1, u_host, out_host, n_host)
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    barrier()
    e2e_ms = replicas.max_over_ranks(e2e_ms, pg)
    e2e_value = replicas.job_throughput(pts * 4 * args.steps, world, e2e_ms)
    state_bytes = dom.state_size * 8

    # ---- roofline of the dominant kernel (the family with the largest time)
    dom_name = max(fam_ms, key=lambda n: fam_ms[n][0])
    d_ms, d_n = fam_ms[dom_name]
    d_flops = costmodel.family_flops(dom_name, w.shells, args.algorithm, w.sh_keep_l)
    achieved = d_flops / (d_ms / d_n / 1000.0) / 1e12 if (d_n and d_flops) else None
    peak = costmodel.GB300_FP64_PEAK_TFLOPS
    kernel_names = {"angular": {"folded": "fold_angular_kernel<true> (d/dtheta, d/dphi: folded phi DFT, "
                                          "parity-split Legendre maps, folded inverse DFT)",
                                "separable": "sep_angular_kernel<true> (d/dtheta, d/dphi: phi DFT, "
                                             "Legendre maps, inverse DFT)",
                                "dense": "gemm_batched_kernel (dense angular maps)"}[args.algorithm],
                    "pointwise": "pointwise_kernel (DiffJac + GH RHS + RK4 combine)",
                    "radial": "radial_kernel<false> (Chebyshev d/dx)"}
    traffic = TRAFFIC_PER_LAUNCH.get((w.name, args.algorithm, dom_name))
    roofline = dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s",
                    frac=(achieved / peak) if achieved else None, traffic=traffic,
                    kernel=kernel_names.get(dom_name, dom_name), family=dom_name,
                    flops_per_launch=d_flops, launch_ms=d_ms / d_n if d_n else None,
                    peak_source="derived FP64 FFMA peak: 152 SMs x 4 flop/clk x 2.07 GHz "
                                "(recipe nominal 1.25 TFLOP/s; own FFMA loop measured 1.20)")
    kernels = {name: dict(ms_per_step=v[0] / args.steps, launches_per_step=v[1] / args.steps)
               for name, v in fam_ms.items() if v[1]}

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=w.name, points=pts, shells=[list(s) for s in w.shells], chi=w.chi,
                            dt=w.dt, rhs_evals_per_step=4,
                            step="RK4 step + ExpCheb(36,32) + SH keep l<=%d + constraint norms" % w.sh_keep_l,
                            sh_filter={"component": "per Cartesian component (scalar Y_lm truncation)",
                                       "tensor": "tensor spherical harmonics (spin-weighted sY_lm of the "
                                                 "31 independent complex frame components)"}[args.sh_filter],
                            l2="flushed before every timed step (256 MB write, outside the step events)",
                            timed_step=("one replay of the captured RK4 graph (gh_rk4_graph_launch)" if use_graph
                                        else "one gh_rk4_step call"),
                            kernel_times="per-family CUDA events on the domain's stream, from a second "
                                         "timed region of the same steps called directly (the maps one "
                                         "after the other)",
                            overlap=not args.no_overlap,
                            parallelism="replicas" if world > 1 else "single GPU", algorithm=args.algorithm,
                            schedule=gh.gh_get_schedule(dom),
                            autotuned=not (args.no_autotune or args.schedule)),
                e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=state_bytes,
                         d2h_bytes_per_step=state_bytes + 8 * len(w.shells),
                         call="gh_rk4_step_host, pinned host buffers, one step per call"),
                gpu_launches=launches, roofline=roofline, kernels=kernels)
    if args.sh_filter == "tensor":
        tf = costmodel.tensor_filter_flops(w.shells, w.sh_keep_l)
        f_ms, f_n = fam_ms["angular_filter"]
        tf_ach = tf["total"] / (f_ms / f_n / 1000.0) / 1e12 if f_n else None
        line["tensor_filter"] = dict(
            kernels="tf_frame_kernel + tf_spin_kernel + tf_unframe_kernel", ms_per_step=f_ms / args.steps,
            flops_per_launch=tf["total"], flops_split={k: tf[k] for k in ("frame", "spin", "unframe")},
            achieved=tf_ach, peak=peak, unit="TFLOP/s", frac=(tf_ach / peak) if tf_ach else None, bound="alu")
    if clk is not None:
        line["clocks"] = clk
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "kerr4":
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def run_batched(args):
    """64 independent holes: batched (one domain, CUDA graph per step) vs plain loop."""
    import torch
    from paper_1804_09101_gb300 import build
    build.build()
    from paper_1804_09101_gb300 import costmodel, gh, workloads
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workloads.batched_workload()
    noise = torch.from_numpy(w.noise()).to(dev)
    stream = torch.cuda.current_stream()

    # ---- batched: every hole in one domain
    dom = gh.Domain(w.shells, w.gamma0, w.gamma1, w.gamma2, w.filt_alpha, w.filt_order,
                    w.radial_filter_on, w.sh_keep_l)
    u = dom.new_state()
    for b_, h in enumerate(w.holes):
        gh.gh_set_analytic_kerr_schild(dom, b_, h["M"], h["chi"], u)
        gh.gh_set_dt_scale(dom, b_, h["dt"])
    u += noise
    if not args.no_autotune:
        gh.gh_autotune(dom, 5)
    work = dom.new_work()
    norm2 = torch.zeros(len(w.holes), dtype=torch.float64, device=dev)
    # per-family profile from direct (non-graph) steps
    for _ in range(2):
        gh.gh_rk4_step(dom, 1.0, u, work, norm2)
    gh.gh_profile_enable(dom, True)
    for fam in range(len(gh.KERNEL_FAMILIES)):
        gh.gh_profile_read(dom, fam)
    for _ in range(3):
        gh.gh_rk4_step(dom, 1.0, u, work, norm2)
    fam_ms = {name: gh.gh_profile_read(dom, fam) for fam, name in enumerate(gh.KERNEL_FAMILIES)}
    gh.gh_profile_enable(dom, False)
    gh.gh_rk4_graph_capture(dom, 1.0, u, work, norm2)
    gh.gh_rk4_graph_launch(dom, args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    n0 = dom.launch_count()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    gh.gh_rk4_graph_launch(dom, args.steps)
    e.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = dom.launch_count() - n0
    batched_ms = a.elapsed_time(e)
    # Holes with high spin at L = 7 are under-resolved near the ring singularity
    # and can blow up within tens of steps; that is reported, not hidden.
    try:
        gh.gh_sync(dom)
    except gh.GHError as err:
        if err.status != gh.GH_ENONFINITE:
            raise
    nonfinite_holes = int((~torch.isfinite(norm2)).sum())

    # ---- plain: one domain per hole, launched hole after hole
    doms = []
    off = 0
    for b_, h in enumerate(w.holes):
        d1 = gh.Domain([w.shells[b_][:4]], w.gamma0, w.gamma1, w.gamma2, w.filt_alpha, w.filt_order,
                       w.radial_filter_on, w.sh_keep_l)
        u1 = d1.new_state()
        gh.gh_set_analytic_kerr_schild(d1, 0, h["M"], h["chi"], u1)
        gh.gh_set_dt_scale(d1, 0, h["dt"])
        u1 += noise[off:off + d1.state_size]
        off += d1.state_size
        if not args.no_autotune:
            gh.gh_autotune(d1, 3)
        doms.append((d1, u1, d1.new_work(), torch.zeros(1, dtype=torch.float64, device=dev)))
    for _ in range(args.warmup):
        for d1, u1, w1, n1 in doms:
            gh.gh_rk4_step(d1, 1.0, u1, w1, n1)
    torch.cuda.synchronize()
    psteps = max(1, min(args.steps, 20))
    a.record(stream)
    for _ in range(psteps):
        for d1, u1, w1, n1 in doms:
            gh.gh_rk4_step(d1, 1.0, u1, w1, n1)
    e.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(e)

    pts = w.points()
    value = pts * 4 * args.steps / (batched_ms / 1000.0)
    plain_value = pts * 4 * psteps / (plain_ms / 1000.0)
    dom_name = max(fam_ms, key=lambda n: fam_ms[n][0])
    d_ms, d_n = fam_ms[dom_name]
    d_flops = costmodel.family_flops(dom_name, [s[:4] for s in w.shells], "folded", None)
    if dom_name == "angular_filter":
        d_flops = sum(costmodel.fold_angular_flops([s[:4]], K=(2 * s[3]) // 3, two=False) for s in w.shells)
    achieved = d_flops / (d_ms / d_n / 1000.0) / 1e12 if (d_n and d_flops) else None
    peak = costmodel.GB300_FP64_PEAK_TFLOPS
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=1, steps=args.steps, warmup=args.warmup,
                ms_per_step=batched_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=w.name, points=pts, holes=len(w.holes),
                            step="batched: one CUDA-graph replay of an RK4 step over all holes "
                                 "(per-hole dt, ExpCheb + per-shell 2/3 SH truncation, constraint norms)",
                            l2="state %.0f MB > L2" % (dom.state_size * 8 / 1e6),
                            plain_value=plain_value, plain_ms_per_step=plain_ms / psteps,
                            plain_steps=psteps, batched_over_plain=value / plain_value,
                            plain="one domain per hole, gh_rk4_step hole after hole (18 launches each)",
                            nonfinite_holes_at_end=nonfinite_holes),
                gpu_launches=launches,
                roofline=dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s",
                              frac=(achieved / peak) if achieved else None, traffic=None, family=dom_name,
                              flops_per_launch=d_flops, launch_ms=d_ms / d_n if d_n else None),
                kernels={name: dict(ms_per_step=v[0] / 3, launches_per_step=v[1] / 3)
                         for name, v in fam_ms.items() if v[1]})
    if clk is not None:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Adjoint workload: gradient of the 200-step time-integrated constraint
    energy with respect to 16 Pi-mode coefficients (checkpoints every 20 steps),
    timed against the forward evolution that defines it."""
    import numpy as np
    import torch
    from paper_1804_09101_gb300 import build
    build.build()
    from paper_1804_09101_gb300 import gh, workloads
    from paper_1804_09101_gb300.adjoint import constraint_energy_gradient, evolve_energy
    w = workloads.adjoint_single_shell()
    dom = gh.Domain.from_workload(w)
    if not args.no_autotune:
        gh.gh_autotune(dom, 5)
    u0 = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u0)
    p = w.pulse
    gh.gh_add_perturbation(dom, 1, 1.0, p.center, p.width, p.lmax, p.coeffs, u0)
    steps = w.steps
    for _ in range(max(1, args.warmup // 3)):
        evolve_energy(dom, u0, w.dt, steps)
        constraint_energy_gradient(dom, u0, w.dt, steps, ckpt=20)
    reps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        E = evolve_energy(dom, u0, w.dt, steps)
    torch.cuda.synchronize()
    fwd = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        E2, lam = constraint_energy_gradient(dom, u0, w.dt, steps, ckpt=20)
        g = gh.gh_perturbation_vjp(dom, 1, p.center, p.width, p.lmax, lam)
    torch.cuda.synchronize()
    bwd = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        E3, lam3 = constraint_energy_gradient(dom, u0, w.dt, steps, ckpt=steps)
    torch.cuda.synchronize()
    bwd_all = (time.perf_counter() - t0) / reps
    pts = w.points()
    line = dict(metric=METRIC, value=pts * 4 * steps / fwd, unit=UNIT, n_gpus=1, steps=reps, warmup=args.warmup,
                ms_per_step=1000.0 * fwd / steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=w.name, points=pts, evolution_steps=steps, checkpoint_every=20,
                            parameters=16, forward_s=fwd, gradient_s=bwd, adjoint_over_forward=bwd / fwd,
                            backward_over_forward=(bwd - fwd) / fwd,
                            keep_all_states_gradient_s=bwd_all,
                            keep_all_states_backward_over_forward=(bwd_all - fwd) / fwd,
                            energy=E, grad_norm=float(np.linalg.norm(g)),
                            timing="wall clock around whole evolutions (host-driven launches), "
                                   "mean of %d repetitions; gradient_s includes its own forward pass, "
                                   "backward_over_forward excludes it (backward incl. checkpoint "
                                   "recomputation)" % reps))
    print(json.dumps(line), flush=True)


def run_dp5(args, w):
    """Dormand-Prince 5(4) adaptive evolution of the workload: each timed
    attempt is 7 right-hand sides, 6 stage combinations and the error norm
    (device time between CUDA events around the call, which ends with the
    error norm read back to the host controller); rejected attempts count as
    work done.  rtol = atol = 1e-8, starting from the workload's dt."""
    import torch
    from paper_1804_09101_gb300 import build
    build.build()
    from paper_1804_09101_gb300 import gh
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    dom = gh.Domain.from_workload(w)
    if not args.no_autotune:
        gh.gh_autotune(dom, 5)
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    p = w.pulse
    if p is not None:
        gh.gh_add_perturbation(dom, 0, p.amplitude, p.center, p.width, p.lmax, p.coeffs, u)
    if w.noise_amp:
        u += torch.from_numpy(w.noise()).to(u.device)
    work = gh.new_dp5_work(dom)
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    dt = w.dt
    for _ in range(args.warmup):
        _, _, dt = gh.gh_dp5_step(dom, dt, 1e-8, 1e-8, u, work)
    clocks = ClockSampler(0)
    clocks.start()
    n0 = dom.launch_count()
    tot_ms, acc, t_sim = 0.0, 0, 0.0
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dt0 = dt
        _, ok, dt = gh.gh_dp5_step(dom, dt, 1e-8, 1e-8, u, work)
        b.record(stream)
        b.synchronize()
        tot_ms += a.elapsed_time(b)
        acc += int(ok)
        t_sim += dt0 if ok else 0.0
    clk = clocks.stop()
    launches = dom.launch_count() - n0
    pts = w.points()
    line = dict(metric=METRIC, value=pts * 7 * args.steps / (tot_ms / 1e3), unit=UNIT, n_gpus=1,
                steps=args.steps, warmup=args.warmup, ms_per_step=tot_ms / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=w.name, points=pts, stepper="Dormand-Prince 5(4), rtol = atol = 1e-8",
                            rhs_evals_per_step=7, accepted=acc, attempts=args.steps, simulated_time=t_sim,
                            final_dt=dt, l2="flushed before every timed attempt",
                            schedule=gh.gh_get_schedule(dom)),
                gpu_launches=launches)
    if clk is not None:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def run_families(args):
    """The paper's benchmark grid families (Sec. 3.4) on four Kerr shells:
    SingleBH k = 0..8 (odd L) and BBH k = 0..8 (even L), all with the folded
    angular maps.  Per member: the derivative step (radial + angular maps,
    the paper's Differentiator), the full RHS and the RK4 step, timed with CUDA
    events after warm-up; the paper's dense-matrix Differentiator flop count
    beside the library's own count."""
    import torch
    from paper_1804_09101_gb300 import build
    build.build()
    from paper_1804_09101_gb300 import costmodel, gh, workloads
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device="cuda")
    reps = max(3, args.steps // 10)

    def timed(fn):
        for _ in range(3):
            fn()
        tot = 0.0
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / reps

    members = []
    tot_units, tot_ms, launches = 0.0, 0.0, 0
    for family in ("singlebh", "bbh"):
        for k in range(9):
            w = workloads.grid_family_workload(family, k)
            dom = gh.Domain.from_workload(w)
            if not args.no_autotune:
                gh.gh_autotune(dom, 3)
            u = dom.new_state()
            gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
            u += torch.from_numpy(w.noise()).to(u.device)
            du = torch.empty(3 * dom.state_size, dtype=torch.float64, device="cuda")
            kk = dom.new_state()
            work = dom.new_work()
            d_ms = timed(lambda: gh.gh_derivatives(dom, u, du))
            r_ms = timed(lambda: gh.gh_rhs(dom, u, kk))
            us = u.clone()
            n0 = dom.launch_count()
            s_ms = timed(lambda: gh.gh_rk4_step(dom, w.dt, us, work))
            launches += (dom.launch_count() - n0) // (reps + 3)
            pts = w.points()
            n_r, L = workloads.grid_family_resolution(family, k)
            nth, nph = L + 1, 2 * (L + 1)
            _, F_dense = costmodel.i1s2_differentiator(50, n_r, nth, nph)
            alg = "folded"
            F_lib = (costmodel.radial_flops(w.shells) + costmodel.family_flops("angular", w.shells, alg)) / 4
            members.append(dict(family=family, k=k, n_r=n_r, n_theta=nth, n_phi=nph, points=pts,
                                algorithm=alg, deriv_ms=d_ms, rhs_ms=r_ms, rk4_step_ms=s_ms,
                                rhs_evals_per_s=pts / (r_ms / 1e3),
                                step_evals_per_s=4 * pts / (s_ms / 1e3),
                                paper_dense_deriv_flops_per_shell=F_dense,
                                library_deriv_flops_per_shell=F_lib,
                                deriv_tflops=4 * F_lib / (d_ms / 1e3) / 1e12))
            tot_units += 4 * pts
            tot_ms += s_ms
            del dom
    line = dict(metric=METRIC, value=tot_units / (tot_ms / 1e3), unit=UNIT, n_gpus=1, steps=reps,
                warmup=3, ms_per_step=tot_ms / len(members), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload="paper grid families (SingleBH, BBH k=0..8) on 4 Kerr a=0.9 shells",
                            value="all members' RK4 grid-point RHS evaluations / sum of their step times",
                            l2="flushed before every timed call", members=members),
                gpu_launches=launches)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    from paper_1804_09101_gb300 import workloads
    w = {"kerr4": workloads.kerr_four_shells, "large": workloads.kerr_eight_shells_large,
         "schwarzschild": workloads.schwarzschild_single_shell,
         "batched": workloads.kerr_four_shells, "adjoint": workloads.kerr_four_shells,
         "families": workloads.kerr_four_shells, "paper": workloads.paper_single_bh}[args.workload]()
    if args.workload == "adjoint":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the adjoint workload has no oracle arm"}))
            return
        run_adjoint(args)
        return
    if args.workload == "families":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the grid-family sweep has no oracle arm"}))
            return
        run_families(args)
        return
    if args.workload == "batched":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no oracle arm"}))
            return
        run_batched(args)
        return
    if args.impl == "reference":
        run_reference(args, w)
    elif args.stepper == "dp5":
        run_dp5(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
