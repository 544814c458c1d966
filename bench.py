"""Benchmark: GH right-hand-side grid-point evaluations per second on one GB300.

One step = one full pass of the hot path on the 8-shell Kerr workload (the
largest configuration: a = 0.95, M = 1, eight geometric shells spanning
r in [1.2, 100], N_r = 41, L = 31 (32 x 64 angular points); 671,744 points,
a 269 MB state): an RK4 step (4 right-hand sides with derivatives, the fused
GH kernel, characteristic boundary conditions and stage combines), the
exponential Chebyshev and SH 2/3 filters, and the quadrature constraint norms
(computed inside the first stage).  Throughput = points x 4 RHS evaluations
per step / time.

Each timed step replays the step captured once as a CUDA graph
(gh_rk4_graph_capture / gh_rk4_graph_launch; --no-graph times direct
gh_rk4_step calls).  The per-kernel times behind the roofline come from a second
timed region of the same steps called directly with the library's CUDA-event
brackets, which would otherwise add gaps to the headline region.  The large
state is bigger than L2, so the K steps are timed back to back; a workload
whose state fits in L2 (--workload kerr4) gets a 256 MB L2 flush before every
timed step, outside the step's events.

The same line carries the other two parts of the metric, measured after the
headline region: batched_over_plain (64 independent holes of uneven
resolution as one domain replayed as a CUDA graph, against the per-hole loop
of step calls) and adjoint_over_forward (gradient of the 200-step constraint
energy with checkpoints every 20 steps, against the forward evolution), plus
the 4-shell workload's throughput as a secondary figure (--no-extras skips
them).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload ...]

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
    # the three launches of the ring-FFT angular map, 8-shell L=31: analysis 268.8 + 210.3 MB,
    # Legendre 264.7 + 469.5 MB, synthesis 529.1 + 482.6 MB (read + written)
    ("kerr_a0.95_8shells_nr41_L31", "folded", "angular"): 2225.0e6,
    # the same, 4-shell L=15: 17.3 + 0, 16.7 + 16.9, 33.4 + 17.9 MB (the scratch mostly L2-resident)
    ("kerr_a0.9_4shells_nr21_L15", "folded", "angular"): 102.2e6,
    # the paper's 2-shell L=18 grid: not captured since the kernel changed
    ("paper_singlebh_chi0.2_0.3_0.4_2shells_nr10_L18", "folded", "angular"): None,
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
    p.add_argument("--workload", default="large",
                   choices=["kerr4", "large", "schwarzschild", "batched", "adjoint", "families", "paper"],
                   help="large: 8-shell Kerr a=0.95, N_r=41, L=31 (default, the headline); kerr4: 4-shell "
                        "Kerr a=0.9, N_r=21, L=15; schwarzschild: 1 shell N_r=11, L=7; batched: 64 "
                        "independent single-shell holes of uneven resolution, one CUDA graph per RK4 step, "
                        "compared with the plain per-hole launch loop")
    p.add_argument("--frame", default="static", choices=["static", "rotating", "map"],
                   help="grid motion: static (default); rotating about the hole's spin axis at 0.25; map: the "
                        "general map (expansion 0.01, translation (0.01, 0, 0), rotation 0.25 about a tilted "
                        "axis), with the hole's gauge source and boundary data evaluated at the moving points "
                        "every stage")
    p.add_argument("--outer-bc", default="freeze", choices=["freeze", "cp", "cp_full"],
                   help="outer boundary condition: freeze (default); cp: constraint preserving for u^psi and "
                        "u^0; cp_full: also the constraint part of u^- (static grid only)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the batched, adjoint and 4-shell figures added to the large workload's line")
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
FULL_RHS_POINTS = 50_000       # above this, one full oracle right-hand side takes minutes
L2_BYTES = 129e6               # GB300 L2


def oracle_setup(w, shells=None):
    """The oracle's domain for the workload (or for the listed shells of it:
    each shell's exact data and gauge source depend on that shell alone) and
    the workload's initial state on it."""
    import numpy as np
    from oracle import evolve, perturb
    idx = list(range(len(w.shells))) if shells is None else list(shells)
    dom = evolve.Domain([w.shells[i] for i in idx], w.M, w.chi, w.gamma0, w.gamma1, w.gamma2, w.filt_alpha,
                        w.filt_order, w.radial_filter_on, w.sh_keep_l)
    sizes = [n_r * 50 * (L + 1) * 2 * (L + 1) for (_, _, n_r, L) in w.shells]
    offs = np.cumsum([0] + sizes)
    noise = w.noise() if w.noise_amp else None
    u = []
    for j, (i, g) in enumerate(zip(idx, dom.grids)):
        a = dom.u_exact[j].copy()
        p = w.pulse
        if p is not None:
            if p.kind == "psi_pulse":
                a = a + perturb.psi_pulse(g, dom.u_exact[j], p.amplitude, p.center, p.width, p.lmax, p.coeffs)
            else:
                a = a + perturb.pi_modes(g, p.center, p.width, p.lmax, p.coeffs)
        if noise is not None:
            a = a + noise[offs[i]:offs[i + 1]].reshape(a.shape)
        u.append(a)
    return dom, u


def oracle_interior_rhs_slice(dom, u, s, ir):
    """The oracle's GH right-hand side (before boundary conditions) on radial
    slice ir of shell s: the radial derivative of the shell's lines, the
    harmonic analysis and derivative synthesis of the slice, DiffJac and the
    pointwise GH algebra -- the steps of the oracle's rhs_interior restricted
    to one slice."""
    import numpy as np
    from oracle import gh as ogh
    from oracle import spectral
    g = dom.grids[s]
    us = u[s]
    dr = spectral.radial_derivative(us, g)[ir]                       # [50, th, ph]
    dth, dph = spectral.angular_derivatives(us[ir], g)               # [50, th, ph]
    J = spectral.spherical_jacobian(g)[:, :, ir]                     # [3, 3, th, ph]
    du = J[:, 0, None] * dr[None] + J[:, 1, None] * dth[None] + J[:, 2, None] * dph[None]
    U = np.moveaxis(us[ir], 0, -1)                                   # [th, ph, 50]
    dU = np.moveaxis(du, (0, 1), (-2, -1))                           # [th, ph, 3, 50]
    H = np.moveaxis(dom.H[s][ir], 0, -1)
    dH = np.moveaxis(dom.dH[s][ir], 0, -1).reshape(U.shape[:-1] + (3, 4))
    return ogh.gh_rhs_pointwise(U, dU, H, dH, dom.gamma0, dom.gamma1, dom.gamma2)


def cpu_baseline(w, min_seconds=10.0):
    """The oracle on the host cores: full right-hand sides (all shells) until
    >= min_seconds when one fits in a few seconds, else one interior
    right-hand side of the first shell (a bounded sample of the workload)."""
    from oracle import evolve
    if w.points() <= FULL_RHS_POINTS:
        dom, u = oracle_setup(w)
        evals = 0
        t0 = time.perf_counter()
        while True:
            evolve.rhs(dom, u)
            evals += 1
            el = time.perf_counter() - t0
            if el >= min_seconds:
                break
        pts = w.points() * evals
        sample = ("%d full right-hand-side evaluation(s) of %s (%d points), %.1f s, numpy FP64 on the host"
                  % (evals, w.name, w.points(), el))
    else:
        dom, u = oracle_setup(w, shells=[0])
        t0 = time.perf_counter()
        evolve.rhs_interior(dom, u)
        el = time.perf_counter() - t0
        g = dom.grids[0]
        pts = g["n_r"] * g["n_th"] * g["n_ph"]
        sample = ("one interior right-hand side of the first of %d shells of %s (%d of %d points, no "
                  "boundary exchange: a bounded sample), %.1f s, numpy FP64 on the host"
                  % (len(w.shells), w.name, pts, w.points(), el))
    return dict(value=pts / el, unit=UNIT, cores=blas_threads(), kind="oracle", sample=sample)


REFERENCE_BUDGET_S = 150.0     # the whole --impl reference run, warm-up included


def run_reference(args, w):
    """The oracle on the host cores, timed per step.  A step is one full oracle
    right-hand side of the workload when the run fits the time budget at that
    size; otherwise a bounded sample of it: the interior right-hand side of one
    shell, taking the shells in turn, or, where one shell alone is too slow
    for the budget (the large workload), of one radial slice, taking the
    shells and slices in turn.  The value counts the points each step
    evaluated."""
    import types
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import evolve
    dom, u = oracle_setup(w)
    shells_pts = [g["n_r"] * g["n_th"] * g["n_ph"] for g in dom.grids]
    n_steps = args.steps + args.warmup
    ns = len(dom.grids)

    def one_shell(s):
        return types.SimpleNamespace(grids=[dom.grids[s]], H=[dom.H[s]], dH=[dom.dH[s]],
                                     gamma0=dom.gamma0, gamma1=dom.gamma1, gamma2=dom.gamma2)

    mode = "slice"
    t_full = None
    if w.points() <= FULL_RHS_POINTS:
        t0 = time.perf_counter()
        evolve.rhs(dom, u)                   # sizes the sample (and warms up)
        t_full = time.perf_counter() - t0
        mode = "full" if t_full * n_steps <= REFERENCE_BUDGET_S else "shell"

    def step(i):
        if mode == "full":
            evolve.rhs(dom, u)
            return w.points()
        if mode == "shell":
            s = i % ns
            evolve.rhs_interior(one_shell(s), [u[s]])
            return shells_pts[s]
        s = i % ns
        ir = (i // ns) % dom.grids[s]["n_r"]
        oracle_interior_rhs_slice(dom, u, s, ir)
        return dom.grids[s]["n_th"] * dom.grids[s]["n_ph"]

    for i in range(args.warmup - (1 if t_full is not None else 0)):
        step(i)
    pts = 0
    t0 = time.perf_counter()
    for i in range(args.steps):
        pts += step(i)
    el = time.perf_counter() - t0
    value = pts / el
    what = {"full": "one full oracle right-hand-side evaluation (all %d shells)" % ns,
            "shell": "the oracle's interior right-hand side of one shell, the shells in turn (a bounded "
                     "sample: a full right-hand side takes %.2f s here)" % (t_full or 0.0),
            "slice": "the oracle's interior right-hand side on one radial slice of one shell (the radial "
                     "derivative of the shell's lines, the slice's harmonic analysis and derivative "
                     "synthesis, DiffJac, the pointwise GH algebra), the shells and slices in turn (a "
                     "bounded sample of the workload)"}[mode]
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
KERNEL_NAMES = {"pointwise": "pointwise_kernel (DiffJac + GH RHS + RK4 combine)",
                "radial": "radial_kernel<false> (Chebyshev d/dx)"}
ANGULAR_NAMES = {"folded": "fold_fft_analysis_kernel + fold_legendre_kernel + fold_fft_synthesis_kernel (d/dtheta, "
                           "d/dphi: per-ring real FFTs, parity-split Legendre maps factorised for high m, inverse "
                           "ring FFTs; three launches per map)",
                 "separable": "sep_angular_kernel<true> (d/dtheta, d/dphi: phi DFT, Legendre maps, inverse DFT)",
                 "dense": "gemm_batched_kernel (dense angular maps)"}
PEAK_SOURCE = ("derived FP64 peak: 152 SMs x 4 SMSPs x one 32-lane DFMA every 64 cycles = 4 flop/clk/SM, at "
               "2.07 GHz (the recipe's nominal 1.25 TFLOP/s; an FFMA loop measured 1.20)")


def make_state(dom, w, dev):
    import torch
    from paper_1804_09101_gb300 import gh
    u = dom.new_state()
    gh.gh_set_analytic_kerr_schild(dom, -1, w.M, w.chi, u)
    p = w.pulse
    if p is not None:
        gh.gh_add_perturbation(dom, 0 if p.kind == "psi_pulse" else 1, p.amplitude, p.center, p.width, p.lmax,
                               p.coeffs, u)
    if w.noise_amp:
        u += torch.from_numpy(w.noise()).to(dev)
    return u


def roofline_of(fam_ms, w, algorithm, sh_keep_l):
    """Roofline object of the kernel family with the largest measured time:
    its algorithmic flops per launch over its CUDA-event duration."""
    from paper_1804_09101_gb300 import costmodel
    dom_name = max(fam_ms, key=lambda n: fam_ms[n][0])
    d_ms, d_n = fam_ms[dom_name]
    d_flops = costmodel.family_flops(dom_name, w.shells, algorithm, sh_keep_l)
    achieved = d_flops / (d_ms / d_n / 1000.0) / 1e12 if (d_n and d_flops) else None
    peak = costmodel.GB300_FP64_PEAK_TFLOPS
    names = dict(KERNEL_NAMES, angular=ANGULAR_NAMES[algorithm])
    r = dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s", frac=(achieved / peak) if achieved else None,
             traffic=TRAFFIC_PER_LAUNCH.get((w.name, algorithm, dom_name)), kernel=names.get(dom_name, dom_name),
             family=dom_name, flops_per_launch=d_flops, launch_ms=d_ms / d_n if d_n else None, peak_source=PEAK_SOURCE)
    if dom_name == "pointwise":
        r["flops_per_point"] = costmodel.POINTWISE_FLOPS_PER_POINT
        r["flops_source"] = costmodel.POINTWISE_FLOPS_SOURCE
        r["executed_flops_per_point"] = costmodel.POINTWISE_EXECUTED_FLOPS_PER_POINT
    return r


def measure_rk4(args, w, pg=None, host_e2e=True, clock_index=0):
    """Time K RK4 steps of workload w (graph replays unless --no-graph): the
    headline region, then the same steps called directly with the library's
    per-family event brackets (kernel times), then end to end through
    gh_rk4_step_host with pinned host buffers.  Returns the fields of the
    bench line."""
    import torch
    from paper_1804_09101_gb300 import gh, replicas
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    dom = gh.Domain.from_workload(w)
    gh.gh_set_overlap(dom, not args.no_overlap)
    algorithm = "folded" if args.algorithm == "auto" else args.algorithm
    if args.algorithm != "auto":
        gh.gh_set_algorithm(dom, {"dense": gh.GH_ALG_DENSE, "separable": gh.GH_ALG_SEPARABLE,
                                  "folded": gh.GH_ALG_SEPARABLE_FOLDED}[algorithm])
    if args.schedule:
        gh.gh_set_schedule(dom, json.loads(args.schedule))
    elif not args.no_autotune:
        gh.gh_autotune(dom, 5)
    if args.sh_filter == "tensor":
        gh.gh_set_sh_filter(dom, "tensor")
    u = make_state(dom, w, dev)
    frame = getattr(args, "frame", "static")
    if frame == "rotating":
        gh.gh_set_rotating_frame(dom, (0.0, 0.0, 1.0), 0.25)
    elif frame == "map":
        gh.gh_set_frame_map(dom, (0.6, 0.0, 0.8), 0.25, 0.01, (0.01, 0.0, 0.0))
    outer_bc = getattr(args, "outer_bc", "freeze")
    gh.gh_set_outer_bc(dom, {"freeze": gh.GH_BC_FREEZE, "cp": gh.GH_BC_CONSTRAINT_PRESERVING,
                             "cp_full": gh.GH_BC_CONSTRAINT_PRESERVING_FULL}[outer_bc])
    work = dom.new_work()
    norm2 = torch.zeros(len(w.shells), dtype=torch.float64, device=dev)
    state_bytes = dom.state_size * 8
    big = state_bytes > L2_BYTES
    flush = None if big else torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()

    def pre():
        if flush is not None:
            flush.zero_()

    for _ in range(args.warmup):
        pre()
        gh.gh_rk4_step(dom, w.dt, u, work, norm2)
    gh.gh_sync(dom)
    use_graph = not args.no_graph
    if use_graph:
        # the step as one captured CUDA graph (the library's API for repeated
        # steps); warm-up replays
        gh.gh_rk4_graph_capture(dom, w.dt, u, work, norm2)
        for _ in range(args.warmup):
            pre()
            gh.gh_rk4_graph_launch(dom, 1)
        gh.gh_sync(dom)

    def one_step():
        if use_graph:
            gh.gh_rk4_graph_launch(dom, 1)
        else:
            gh.gh_rk4_step(dom, w.dt, u, work, norm2)

    # ---- device-resident timed region (the headline value): the state is
    # larger than L2, so the K steps run back to back between one pair of
    # events; otherwise L2 is flushed before each step, outside its events
    clocks = ClockSampler(clock_index) if clock_index is not None else None
    if clocks:
        clocks.start()
    barrier()
    n0 = dom.launch_count()
    if big:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(args.steps):
            one_step()
        b.record(stream)
        barrier()
        total_ms = a.elapsed_time(b)
    else:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for i in range(args.steps):
            pre()
            ev[i][0].record(stream)
            one_step()
            ev[i][1].record(stream)
        barrier()
        total_ms = sum(x.elapsed_time(y) for x, y in ev)
    launches = dom.launch_count() - n0
    clk = clocks.stop() if clocks else None
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
        pre()
        gh.gh_rk4_step(dom, w.dt, u, work, norm2)
    barrier()
    fam_ms = {name: gh.gh_profile_read(dom, fam) for fam, name in enumerate(gh.KERNEL_FAMILIES)}
    gh.gh_profile_enable(dom, False)
    gh.gh_sync(dom)

    pts = w.points()
    out = dict(value=replicas.job_throughput(pts * 4 * args.steps, world, total_ms),
               ms_per_step=total_ms / args.steps, launches=launches, clocks=clk, fam_ms=fam_ms,
               roofline=roofline_of(fam_ms, w, algorithm, w.sh_keep_l), algorithm=algorithm,
               schedule=gh.gh_get_schedule(dom), use_graph=use_graph, big=big, state_bytes=state_bytes,
               kernels={name: dict(ms_per_step=v[0] / args.steps, launches_per_step=v[1] / args.steps)
                        for name, v in fam_ms.items() if v[1]})
    if host_e2e:
        # ---- end to end through the C ABI with host buffers: gh_rk4_step_host
        # copies the state in from pinned host memory, steps, and copies the
        # state and the constraint norms out, every step
        u_host = u.detach().cpu().pin_memory()
        out_host = torch.empty_like(u_host).pin_memory()
        n_host = torch.empty(len(w.shells), dtype=torch.float64).pin_memory()
        gh.gh_rk4_step_host(dom, w.dt, 1, u_host, out_host, n_host)     # allocates its device buffers
        e2e_ms = 0.0
        barrier()
        for i in range(args.steps):
            pre()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gh.gh_rk4_step_host(dom, w.dt, 1, u_host, out_host, n_host)
            b.record(stream)
            b.synchronize()
            e2e_ms += a.elapsed_time(b)
        barrier()
        e2e_ms = replicas.max_over_ranks(e2e_ms, pg)
        out["e2e"] = dict(value=replicas.job_throughput(pts * 4 * args.steps, world, e2e_ms), unit=UNIT,
                          h2d_bytes_per_step=state_bytes, d2h_bytes_per_step=state_bytes + 8 * len(w.shells),
                          call="gh_rk4_step_host, pinned host buffers, one step per call")
    if args.sh_filter == "tensor":
        from paper_1804_09101_gb300 import costmodel
        tf = costmodel.tensor_filter_flops(w.shells, w.sh_keep_l)
        f_ms, f_n = fam_ms["angular_filter"]
        tf_ach = tf["total"] / (f_ms / f_n / 1000.0) / 1e12 if f_n else None
        peak = costmodel.GB300_FP64_PEAK_TFLOPS
        out["tensor_filter"] = dict(
            kernels="tf_frame_kernel + tf_spin_kernel + tf_unframe_kernel", ms_per_step=f_ms / args.steps,
            flops_per_launch=tf["total"], flops_split={k: tf[k] for k in ("frame", "spin", "unframe")},
            achieved=tf_ach, peak=peak, unit="TFLOP/s", frac=(tf_ach / peak) if tf_ach else None, bound="alu")
    del dom
    return out


def run_ours(args, w):
    import torch
    from paper_1804_09101_gb300 import build
    build.build()
    rank, world, local = dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    torch.cuda.set_device(local)
    m = measure_rk4(args, w, pg, clock_index=local)
    big = m["big"]
    line = dict(metric=METRIC, value=m["value"], unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=m["ms_per_step"], higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=w.name, points=w.points(), shells=[list(s) for s in w.shells], chi=w.chi,
                            dt=w.dt, rhs_evals_per_step=4,
                            step="RK4 step + ExpCheb(36,32) + SH keep l<=%s + constraint norms"
                                 % ("floor(2L/3)" if w.sh_keep_l == -2 else w.sh_keep_l),
                            sh_filter={"component": "per Cartesian component (scalar Y_lm truncation)",
                                       "tensor": "tensor spherical harmonics (spin-weighted sY_lm of the "
                                                 "31 independent complex frame components)"}[args.sh_filter],
                            l2=("inputs larger than L2: a %.0f MB state (7 states live: state, 3 derivative "
                                "scratch, 3 RK4 work), K steps back to back between one pair of events"
                                % (m["state_bytes"] / 1e6)) if big else
                               "flushed before every timed step (256 MB write, outside the step events)",
                            timed_step=("one replay of the captured RK4 graph (gh_rk4_graph_launch)"
                                        if m["use_graph"] else "one gh_rk4_step call"),
                            kernel_times="per-family CUDA events on the domain's stream, from a second "
                                         "timed region of the same steps called directly",
                            overlap=not args.no_overlap, frame=args.frame, outer_bc=args.outer_bc,
                            parallelism="replicas" if world > 1 else "single GPU", algorithm=m["algorithm"],
                            schedule=m["schedule"], autotuned=not (args.no_autotune or args.schedule)),
                e2e=m["e2e"], gpu_launches=m["launches"], roofline=m["roofline"], kernels=m["kernels"])
    if "tensor_filter" in m:
        line["tensor_filter"] = m["tensor_filter"]
    if m["clocks"] is not None:
        line["clocks"] = m["clocks"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0 and world == 1 and args.workload == "large" and not args.no_extras:
        line.update(extras(args))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def extras(args):
    """The metric's other parts, measured after the headline region: the
    batched/plain ratio, the adjoint/forward ratio and the 4-shell workload's
    throughput.  A part that fails is reported with its error instead of
    losing the line."""
    import traceback
    from paper_1804_09101_gb300 import workloads
    out = dict(batched_over_plain=None, adjoint_over_forward=None, secondary={})
    try:
        b = measure_batched(args)
        out["batched_over_plain"] = b["batched_over_plain"]
        out["secondary"]["batched"] = dict(
            workload=b["workload"], points=b["points"], holes=b["holes"], value=b["value"],
            plain_value=b["plain_value"], batched_over_plain=b["batched_over_plain"],
            steps=b["steps"], plain_steps=b["plain_steps"], nonfinite_holes_at_end=b["nonfinite_holes_at_end"],
            plain_nonfinite_holes_at_end=b["plain_nonfinite_holes_at_end"],
            chunk=b["chunk"],
            timed_from="chunks of %d steps, each from the initial data (exact + seeded noise; the reset "
                       "outside the timed events), so the timed steps see finite values only" % b["chunk"],
            how="one domain over all holes, one CUDA-graph replay per RK4 step, against one "
                "domain per hole stepped by gh_rk4_step hole after hole")
    except Exception:
        out["secondary"]["batched"] = dict(error=traceback.format_exc(limit=3)[-600:])
    try:
        a = measure_adjoint(args)
        # the backward pass with its checkpoint recomputation over the forward
        # evolution; the whole gradient (its own forward included) is
        # gradient_over_forward
        out["adjoint_over_forward"] = a["backward_over_forward"]
        out["secondary"]["adjoint"] = dict(
            workload=a["workload"], points=a["points"], evolution_steps=a["evolution_steps"],
            checkpoint_every=a["checkpoint_every"], forward_s=a["forward_s"], gradient_s=a["gradient_s"],
            gradient_over_forward=a["adjoint_over_forward"], backward_over_forward=a["backward_over_forward"],
            keep_all_states_backward_over_forward=a["keep_all_states_backward_over_forward"],
            timing=a["timing"])
    except Exception:
        out["secondary"]["adjoint"] = dict(error=traceback.format_exc(limit=3)[-600:])
    try:
        out["secondary"]["kerr4_step_vjp"] = measure_step_vjp(args, workloads.kerr_four_shells())
    except Exception:
        out["secondary"]["kerr4_step_vjp"] = dict(error=traceback.format_exc(limit=3)[-600:])
    try:
        wk = workloads.kerr_four_shells()
        k4 = measure_rk4(args, wk, None, host_e2e=False, clock_index=None)
        out["secondary"]["kerr4"] = dict(
            workload=wk.name, points=wk.points(), value=k4["value"], ms_per_step=k4["ms_per_step"],
            roofline=k4["roofline"], l2="flushed before every timed step (256 MB write, outside the step events)")
    except Exception:
        out["secondary"]["kerr4"] = dict(error=traceback.format_exc(limit=3)[-600:])
    return out


BATCH_CHUNK = 20   # batched steps timed per chunk from the initial data (the coarsest holes last longer)


def measure_batched(args):
    """64 independent holes: batched (one domain, CUDA graph per step) vs the
    plain loop (one domain per hole, gh_rk4_step hole after hole)."""
    import torch
    from paper_1804_09101_gb300 import gh, workloads
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
    u_init = u.clone()
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
    # The coarsest holes (L = 7 or N_r <= 13 around the ring singularity of the
    # high spins) leave the exact solution by O(1) and go non-finite after
    # 30-1000 steps.  The timed steps therefore run in chunks of BATCH_CHUNK
    # steps, each from the initial data (the reset outside the timed events),
    # so that every timed step runs on finite values; the count of holes with
    # a non-finite norm or state after any chunk is reported.
    clocks = ClockSampler(local)
    clocks.start()
    n0 = dom.launch_count()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    batched_ms = 0.0
    nonfinite_holes = 0
    done = 0
    while done < args.steps:
        k = min(BATCH_CHUNK, args.steps - done)
        u.copy_(u_init)
        a.record(stream)
        gh.gh_rk4_graph_launch(dom, k)
        e.record(stream)
        e.synchronize()
        batched_ms += a.elapsed_time(e)
        bad = int((~torch.isfinite(norm2)).sum())
        if not bool(torch.isfinite(u).all()):
            bad = max(bad, 1)
        nonfinite_holes = max(nonfinite_holes, bad)
        done += k
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = dom.launch_count() - n0
    try:
        gh.gh_sync(dom)
    except gh.GHError as err:          # reported below (nonfinite_holes_at_end), not hidden
        if err.status != gh.GH_ENONFINITE:
            raise

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
        doms.append((d1, u1, d1.new_work(), torch.zeros(1, dtype=torch.float64, device=dev), u1.clone()))
    for _ in range(args.warmup):
        for d1, u1, w1, n1, _ in doms:
            gh.gh_rk4_step(d1, 1.0, u1, w1, n1)
    for d1, u1, w1, n1, i1 in doms:          # timed from the initial data, as the batched steps
        u1.copy_(i1)
    torch.cuda.synchronize()
    psteps = max(1, min(args.steps, 20))
    a.record(stream)
    for _ in range(psteps):
        for d1, u1, w1, n1, _ in doms:
            gh.gh_rk4_step(d1, 1.0, u1, w1, n1)
    e.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(e)
    plain_nonfinite = sum(int((~torch.isfinite(n1)).sum()) for _, _, _, n1, _ in doms)
    for d1, *_ in doms:
        try:
            gh.gh_sync(d1)
        except gh.GHError as err:
            if err.status != gh.GH_ENONFINITE:
                raise

    pts = w.points()
    value = pts * 4 * args.steps / (batched_ms / 1000.0)
    plain_value = pts * 4 * psteps / (plain_ms / 1000.0)
    return dict(workload=w.name, points=pts, holes=len(w.holes), value=value, plain_value=plain_value,
                batched_over_plain=value / plain_value, batched_ms=batched_ms, plain_ms=plain_ms,
                steps=args.steps, chunk=BATCH_CHUNK, plain_steps=psteps, nonfinite_holes_at_end=nonfinite_holes,
                plain_nonfinite_holes_at_end=plain_nonfinite,
                launches=launches, clocks=clk, fam_ms=fam_ms, state_bytes=dom.state_size * 8, w=w)


def run_batched(args):
    from paper_1804_09101_gb300 import build
    build.build()
    from paper_1804_09101_gb300 import costmodel
    b = measure_batched(args)
    w, fam_ms = b["w"], b["fam_ms"]
    dom_name = max(fam_ms, key=lambda n: fam_ms[n][0])
    d_ms, d_n = fam_ms[dom_name]
    d_flops = costmodel.family_flops(dom_name, [s[:4] for s in w.shells], "folded", None)
    if dom_name == "angular_filter":
        d_flops = sum(costmodel.fold_angular_flops([s[:4]], K=(2 * s[3]) // 3, two=False) for s in w.shells)
    achieved = d_flops / (d_ms / d_n / 1000.0) / 1e12 if (d_n and d_flops) else None
    peak = costmodel.GB300_FP64_PEAK_TFLOPS
    line = dict(metric=METRIC, value=b["value"], unit=UNIT, n_gpus=1, steps=args.steps, warmup=args.warmup,
                ms_per_step=b["batched_ms"] / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=w.name, points=b["points"], holes=b["holes"],
                            step="batched: one CUDA-graph replay of an RK4 step over all holes "
                                 "(per-hole dt, ExpCheb + per-shell 2/3 SH truncation, constraint norms)",
                            l2="state %.0f MB > L2" % (b["state_bytes"] / 1e6),
                            plain_value=b["plain_value"], plain_ms_per_step=b["plain_ms"] / b["plain_steps"],
                            plain_steps=b["plain_steps"], batched_over_plain=b["batched_over_plain"],
                            plain="one domain per hole, gh_rk4_step hole after hole",
                            nonfinite_holes_at_end=b["nonfinite_holes_at_end"],
                            plain_nonfinite_holes_at_end=b["plain_nonfinite_holes_at_end"],
                            timed_from="chunks of %d steps, each from the initial data (the reset outside the "
                                       "timed events), so the timed steps see finite values only" % b["chunk"]),
                batched_over_plain=b["batched_over_plain"], gpu_launches=b["launches"],
                roofline=dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s",
                              frac=(achieved / peak) if achieved else None, traffic=None, family=dom_name,
                              flops_per_launch=d_flops, launch_ms=d_ms / d_n if d_n else None),
                kernels={name: dict(ms_per_step=v[0] / 3, launches_per_step=v[1] / 3)
                         for name, v in fam_ms.items() if v[1]})
    if b["clocks"] is not None:
        line["clocks"] = b["clocks"]
    print(json.dumps(line), flush=True)


def measure_adjoint(args):
    """Adjoint workload: gradient of the 200-step time-integrated constraint
    energy with respect to 16 Pi-mode coefficients (checkpoints every 20 steps),
    timed against the forward evolution that defines it."""
    import numpy as np
    import torch
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
    return dict(workload=w.name, points=w.points(), evolution_steps=steps, checkpoint_every=20, parameters=16,
                forward_s=fwd, gradient_s=bwd, adjoint_over_forward=bwd / fwd,
                backward_over_forward=(bwd - fwd) / fwd, keep_all_states_gradient_s=bwd_all,
                keep_all_states_backward_over_forward=(bwd_all - fwd) / fwd, energy=E,
                grad_norm=float(np.linalg.norm(g)), reps=reps, w=w,
                timing="wall clock around whole evolutions (host-driven launches), mean of %d repetitions; "
                       "gradient_s includes its own forward pass, backward_over_forward excludes it (backward "
                       "incl. checkpoint recomputation)" % reps)


def measure_step_vjp(args, w):
    """One RK4 step's vector-Jacobian product (stage states recomputed, filters
    transposed) against the step itself: direct calls, CUDA events, L2
    flushed before each call."""
    import torch
    from paper_1804_09101_gb300 import gh
    dom = gh.Domain.from_workload(w)
    if not args.no_autotune:
        gh.gh_autotune(dom, 5)
    dev = torch.device("cuda", torch.cuda.current_device())
    u = make_state(dom, w, dev)
    work = dom.new_work()
    vwork = torch.zeros(dom.vjp_work_size, dtype=torch.float64, device=dev)
    ybar = torch.ones_like(u)
    ubar = dom.new_state()
    flush = torch.empty(32 * 1024 * 1024, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    steps = max(3, args.steps)

    def timed(fn):
        for _ in range(3):
            fn()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    us = u.clone()
    step_ms = timed(lambda: gh.gh_rk4_step(dom, w.dt, us, work))
    vjp_ms = timed(lambda: gh.gh_rk4_step_vjp(dom, w.dt, u, ybar, ubar, vwork))
    # the same VJP from stage states kept by the forward step (gh_rk4_step_save),
    # as a checkpointed adjoint that stores stages would run it
    stages = torch.zeros(3 * dom.state_size, dtype=torch.float64, device=dev)
    uf = u.clone()
    save_ms = timed(lambda: gh.gh_rk4_step_save(dom, w.dt, uf, work, stages))
    gh.gh_rk4_step_save(dom, w.dt, u.clone(), work, stages)        # the stage states of u itself
    saved_ms = timed(lambda: gh.gh_rk4_step_vjp_saved(dom, w.dt, u, stages, ybar, ubar, vwork))
    gh.gh_sync(dom)
    return dict(workload=w.name, points=w.points(), step_ms=step_ms, step_vjp_ms=vjp_ms,
                step_vjp_over_step=vjp_ms / step_ms, save_step_ms=save_ms, step_vjp_saved_ms=saved_ms,
                step_vjp_saved_over_step=saved_ms / step_ms,
                how="gh_rk4_step_vjp (recomputes the stage states) and gh_rk4_step_vjp_saved (stage states "
                    "kept by gh_rk4_step_save) against gh_rk4_step, direct calls, CUDA events, L2 flushed "
                    "before each call")


def run_adjoint(args):
    from paper_1804_09101_gb300 import build
    build.build()
    a = measure_adjoint(args)
    steps = a["evolution_steps"]
    line = dict(metric=METRIC, value=a["points"] * 4 * steps / a["forward_s"], unit=UNIT, n_gpus=1,
                steps=a["reps"], warmup=args.warmup, ms_per_step=1000.0 * a["forward_s"] / steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                adjoint_over_forward=a["adjoint_over_forward"],
                config={k: v for k, v in a.items() if k not in ("w", "reps")})
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
