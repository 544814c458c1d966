"""Operation-count models: the paper's (Secs. 3.3 and 3.4) and this library's.

The paper models each operation by its minimum memory transactions M
(doubles moved) and floating-point operations F, with arithmetic intensity
I = F / M (Sec. 2.3).  Its printed values pin these functions in the tests.
The library's own counts (what its kernels compute per launch) are used for
the roofline fractions the benchmark reports.
"""

# GB300 FP64 pipe: 152 SMs x 4 FP64 flop/clk/SM (2 DFMA) x 2.07 GHz maximum SM clock.
GB300_SMS = 152
GB300_FP64_FLOP_PER_CLK_PER_SM = 4
GB300_MAX_SM_GHZ = 2.07
GB300_FP64_PEAK_TFLOPS = GB300_SMS * GB300_FP64_FLOP_PER_CLK_PER_SM * GB300_MAX_SM_GHZ / 1000.0


# ------------------------------------------------------------ paper, Sec. 3.3
def diffjac_intensity(n_e, d=3):
    """DiffJac: M = N_x (2 N_e + d) d, F = N_x N_e (2d - 1) d, so I = 5 N_e / (2 N_e + 3) for d = 3."""
    M = (2 * n_e + d) * d
    F = n_e * (2 * d - 1) * d
    return F / M


SPATIAL_COORD_JAC = {
    # structure: (M per point, F per point), Sec. 3.3
    "a": (15, 15), "aa": (30, 75), "ab": (48, 120), "abb": (120, 495),
}


def spatial_coord_jac_intensity(structure):
    M, F = SPATIAL_COORD_JAC[structure]
    return F / M


# ------------------------------------------------------------ paper, Sec. 3.4
def i1s2_differentiator(n_e, n_r, n_th, n_ph):
    """Dense-matrix differentiator on an I1 x S2 shell: (M, F)."""
    na = n_th * n_ph
    M = n_e * (n_r ** 2 + 2 * na ** 2 + 6 * n_r * na)
    F = n_e * n_r * na * (2 * n_r + 4 * na - 3)
    return M, F


def singlebh_grid(k):
    """SingleBH benchmark shells: N_r = 9 + 4k, N_theta = 6 + 2k, N_phi = 4k + 12."""
    return 9 + 4 * k, 6 + 2 * k, 4 * k + 12


def bbh_grid(k):
    """BBH benchmark shells: N_r = 4 + k, N_theta = 7 + 2k, N_phi = 4k + 14."""
    return 4 + k, 7 + 2 * k, 4 * k + 14


# ------------------------------------------------------------ this library
def angular_deriv_flops(shells):
    """FP64 flops of one angular-derivative launch: two dense maps per shell,
    each a (50 n_r) x N_a x N_a product (N_a = N_theta N_phi), 2 flops per FMA."""
    f = 0
    for (_, _, n_r, L) in shells:
        na = (L + 1) * 2 * (L + 1)
        f += 2 * (2 * 50 * n_r * na * na)
    return f


def angular_filter_flops(shells):
    f = 0
    for (_, _, n_r, L) in shells:
        na = (L + 1) * 2 * (L + 1)
        f += 2 * 50 * n_r * na * na
    return f


def radial_flops(shells):
    """FP64 flops of one folded radial launch (radial_kernel), per column of
    n_r values: the fold 2 h, the ceil(n_r/2) folded rows of n_r FMAs each,
    and the outputs 2 h + (n_r mod 2), with h = floor(n_r/2)."""
    f = 0
    for sh in shells:
        n_r, L = sh[2], sh[3]
        na = (L + 1) * 2 * (L + 1)
        h = n_r // 2
        f += 50 * na * (2 * h + 2 * (n_r - h) * n_r + 2 * h + n_r % 2)
    return f


def _shell_dims(shell):
    _, _, n_r, L = shell[:4]
    nth, nph = L + 1, 2 * (L + 1)
    return n_r, nth, nph, nth * nph


def _keep(shell, K):
    """The kept degree of a shell: its L when K is None, floor(2L/3) for -2."""
    L = shell[3]
    if K is None:
        return L
    return (2 * L) // 3 if K == -2 else K


def sep_angular_flops(shells, K=None, two=True):
    """FP64 flops of one separable angular launch (sep_angular_kernel):
    per (r, field) row, 2 nth nph M (phi DFT) + n_out 2 nth^2 M (Legendre maps)
    + n_out 2 na M (inverse DFT), M = 2K + 1, n_out = 2 (derivatives) or 1 (filter)."""
    f = 0
    n_out = 2 if two else 1
    for sh in shells:
        n_r, nth, nph, na = _shell_dims(sh)
        M = 2 * _keep(sh, K) + 1
        f += 50 * n_r * (2 * nth * nph * M + n_out * 2 * nth * nth * M + n_out * 2 * na * M)
    return f


# FP64 flops per point of the fused pointwise kernel (DiffJac + GH right-hand
# side + RK4 stage combine) in its FMA-chain formulation: ncu's executed
# DFMA/DADD/DMUL counts of one launch on the 4-shell Kerr workload
# (2 x 2,398,144 + 53,760 + 587,328 warp instructions x 32 lanes / 43,008
# points).
POINTWISE_EXECUTED_FLOPS_PER_POINT = 4046

# Algorithmic FP64 flops per point of one launch of the fused pointwise stage,
# independent of the kernel: the GH right-hand side as the equations define it
# (Sec. 3.5, GHEqns), counted by running the oracle's pointwise algebra on
# operation-counting scalars (common subexpressions and symmetric pairs
# shared, each einsum contracted in numpy's optimal pairwise order, negation
# free), plus DiffJac (Eq. DiffJac: 8 nonzero Jacobian entries, 13 flops per
# field) and a quarter of the RK4 step's 13 combination flops per value.
# Written by the counting build into the test suite's golden file, which a
# CPU test compares with these constants.
POINTWISE_GH_RHS_FLOPS_PER_POINT = 3694
POINTWISE_FLOPS_PER_POINT = POINTWISE_GH_RHS_FLOPS_PER_POINT + 650 + 50 * 13 / 4.0     # 4506.5
POINTWISE_FLOPS_SOURCE = ("algorithmic: the GH equations counted on the oracle's pointwise algebra (3,694 per "
                          "point) + DiffJac (650) + RK4 stage combinations (162.5); the kernel executes 4,046")


# A mode's half-size Legendre map is applied as analysis then synthesis when
# (1 + n_out)(K + 1 - m) is below this percentage of 2 n_out hs (the fused
# map's FMAs per output ring); the library's fold plans use the same rule.
FOLD_RANK_PERCENT = 75


def fold_rank_m0(K, hs, n_out):
    """First mode m whose Legendre map the folded kernel factorises (K + 1: none)."""
    for m in range(K + 1):
        if (1 + n_out) * (K + 1 - m) * 100 < FOLD_RANK_PERCENT * 2 * n_out * hs:
            return m
    return K + 1


FOLD_FFT_NPHI = (16, 32, 64)   # rings transformed by register FFTs (fold_fft_analysis/synthesis_kernel)


def ring_fft_flops(nph, forward=True):
    """FP64 flops of one ring's phi transform on the FFT path (an FMA is 2):
    the radix-2 DIT FFT of n = nph/2 complex values, per stage of span S
    4 flops for each butterfly with twiddle 1 or +-i, 10 for (+-1 +- i)/sqrt 2
    (two adds, four FMAs) and 12 for a general twiddle (six FMAs); plus the
    real split (forward) or fold (inverse), 18 per pair of modes (m, n - m)
    and, forward, 1 for the mean.  N_phi = 64: 835 forward, 834 inverse."""
    n = nph // 2
    f, S = 0, 1
    while S < n:
        per_group = 4 if S == 1 else (8 if S == 2 else 2 * 4 + 2 * 10 + (S - 4) * 12)
        f += (n // (2 * S)) * per_group
        S *= 2
    return f + 18 * (n // 2 - 1) + (1 if forward else 0)


def fold_angular_flops(shells, K=None, two=True):
    """FP64 flops of one folded separable map, per (r, field) row.  For
    N_phi = 16, 32, 64 (three launches: fold_fft_analysis_kernel,
    fold_legendre_kernel, fold_fft_synthesis_kernel) the phi transforms are
    register FFTs (ring_fft_flops per ring and transform, N_theta M for the
    s/t split); otherwise (fold_angular_kernel) the quarter-folded DFT: fold
    8 (W - 1) N_theta; phase A half M (4 W + 2) plus
    (hs - half) M 2 W for an odd N_theta's equator ring; phase B per mode
    (cos m, and sin m for m >= 1): fused, n_out hs 4 hs (two dot products of
    length hs per output, each a multiply and hs - 1 FMAs, and the two
    mirror combinations); factorised (m >= m0, rank r = K + 1 - m), the
    analysis (2 hs - 1) r plus n_out hs (2 r + 2); phase C n_out N_theta W
    (2 M + 8), with W = N_phi/4 + 1 (N_phi % 4 == 0) or (N_phi + 2)/4,
    half = floor(N_theta/2), hs = ceil(N_theta/2), M = 2K+1.  An ncu count of
    the executed DFMA/DADD/DMUL is 1.1 % (8 shells, L = 31) and 2.3 % (4
    shells, L = 15) below this."""
    f = 0
    n_out = 2 if two else 1
    for sh in shells:
        n_r, nth, nph, na = _shell_dims(sh)
        Kk = _keep(sh, K)
        M = 2 * Kk + 1
        W = nph // 4 + 1 if nph % 4 == 0 else (nph + 2) // 4
        half, hs = nth // 2, (nth + 1) // 2
        m0 = fold_rank_m0(Kk, hs, n_out)
        phase_b = 0
        for m in range(Kk + 1):
            modes = 1 if m == 0 else 2
            r = Kk + 1 - m
            if m < m0:
                phase_b += modes * n_out * hs * 4 * hs
            else:
                phase_b += modes * ((2 * hs - 1) * r + n_out * hs * (2 * r + 2))
        if nph in FOLD_FFT_NPHI and nth % 2 == 0:
            # one forward FFT per ring, the s/t split of every coefficient,
            # one inverse FFT per ring and output
            per_row = (nth * ring_fft_flops(nph) + nth * M + phase_b
                       + n_out * nth * ring_fft_flops(nph, forward=False))
        else:
            per_row = (8 * (W - 1) * nth + half * M * (4 * W + 2) + (hs - half) * M * 2 * W
                       + phase_b + n_out * nth * W * (2 * M + 8))
        f += 50 * n_r * per_row
    return f


def family_flops(family, shells, algorithm="folded", keep_l=-1):
    """Algorithmic FP64 flops of one launch of a kernel family."""
    pts = sum(n_r * 2 * (L + 1) ** 2 for (_, _, n_r, L) in shells)
    if family == "angular":
        return {"separable": sep_angular_flops, "dense": angular_deriv_flops,
                "folded": fold_angular_flops}[algorithm](shells)
    if family == "angular_filter":
        if algorithm == "separable":
            return sep_angular_flops(shells, K=keep_l, two=False)
        if algorithm == "folded":
            return fold_angular_flops(shells, K=keep_l, two=False)
        return angular_filter_flops(shells)
    if family in ("radial", "radial_filter"):
        return radial_flops(shells)
    if family == "pointwise":
        return POINTWISE_FLOPS_PER_POINT * pts
    return None


# The nine tensor groups of the GH fields (psi_00, psi_0i, psi_ij, Pi_00, Pi_0i,
# Pi_ij, Phi_i00, Phi_i0j, Phi_ijk): rank, and whether the last two indices are
# symmetric.
TENSOR_GROUPS = [(0, False), (1, False), (2, True), (0, False), (1, False), (2, True), (1, False), (2, False),
                 (3, True)]


def tensor_filter_row_spins():
    """Spin weights of the independent complex frame components (one per class
    under conjugation m <-> conj(m) and the symmetric index pair)."""
    import itertools
    spins = []
    for rank, sym in TENSOR_GROUPS:
        tuples = list(itertools.product(range(3), repeat=rank))
        for t in tuples:
            variants = []
            for c in (0, 1):
                for sw in ((0, 1) if sym else (0,)):
                    e = list(t)
                    if sw:
                        e[-2], e[-1] = e[-1], e[-2]
                    if c:
                        e = [0 if a == 0 else 3 - a for a in e]
                    variants.append(tuple(e))
            if min(variants) == t:
                spins.append(sum({0: 0, 1: 1, 2: -1}[a] for a in t))
    return spins


def tensor_filter_flops(shells, keep_l):
    """FP64 flops (FMA = 2) of one tensor-harmonic filter application
    (tf_frame_kernel, tf_spin_kernel, tf_unframe_kernel).  Per point, the frame
    kernels contract each rank-n group index by index in the real frame
    (8 * 3^(n-1) FMAs per index, the zero phi_hat_z term skipped) and form the
    complex combinations with additions; per (r, independent component) row of
    spin s the spin kernel does the quarter fold (16 adds per slot pair), the
    folded forward DFT (4 W FMAs per ring and m >= 0), the analysis and
    synthesis (2 N_theta FMAs per coefficient each, sum_m n_b(s, m)
    coefficients, n_b = K - max(|m|, |s|) + 1) and the folded inverse DFT
    (4 (K+1) FMAs per ring and slot), W = N_phi/4 + 1."""
    spins = tensor_filter_row_spins()
    frame = unframe = spin = 0
    per_pt_f = per_pt_u = 0
    for rank, _ in TENSOR_GROUPS:
        n = 3 ** rank
        fma = rank * 8 * 3 ** (rank - 1) if rank else 0
        nz = 2 * 3 ** (rank - 1) if rank else 0          # outputs with a nonzero frame index, per pass
        per_pt_f += 2 * fma + (rank - 1 if rank else 0) * nz * 2
        per_pt_u += 2 * fma + rank * nz * 2 + (n - 1)
    per_pt_f += 2 * len(spins)                            # the 1/sqrt(2) scaling of the stored components
    for sh in shells:
        n_r, nth, nph, na = _shell_dims(sh)
        L = sh[3]
        K = (2 * L) // 3 if keep_l == -2 else keep_l
        if K < 0:
            continue
        h, W, K1 = nph // 2, nph // 4 + 1, K + 1
        frame += per_pt_f * n_r * na
        unframe += per_pt_u * n_r * na
        fold = nth * (4 + (4 if h % 2 == 0 else 0) + 16 * (W - 1 - (1 if h % 2 == 0 else 0)))
        fwd = nth * K1 * (8 * W + 8)
        inv = nth * W * (8 * K1 + 16)
        for s in spins:
            ncoef = sum(max(0, K - max(abs(m), abs(s)) + 1) for m in range(-K, K + 1))
            theta = ncoef * nth * 4 * 2 + nth * K1 * 4
            spin += n_r * (fold + fwd + theta + inv)
    return dict(frame=frame, spin=spin, unframe=unframe, total=frame + spin + unframe)
