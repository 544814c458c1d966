"""Synthetic workloads and seeded input generators.

This module holds no arithmetic of the method: it only names the workload
shapes and draws seeded random numbers (numpy PCG64).  Both the library's
tests and benchmark and the CPU oracle take their random inputs from here, so
the two sides see identical inputs.

The workloads stand in for the paper's private SpEC single-black-hole runs
(Sec. 3.1: a spinning Kerr-Schild hole surrounded by concentric I1 x S2
shells with N_r of order 10-40 and N_phi = 2 N_theta); no public dataset
exists for them.
"""
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class Pulse:
    """Coefficients of a perturbation; evaluated by the library or the oracle."""
    kind: str               # "psi_pulse" (ingoing Gaussian shell on psi) or "pi_modes"
    amplitude: float
    center: float
    width: float
    lmax: int
    coeffs: np.ndarray      # (lmax+1)^2 real Y_lm coefficients


@dataclass
class Workload:
    name: str
    shells: List[Tuple[float, float, int, int]]   # (r_in, r_out, n_r, L)
    M: float
    chi: float
    gamma0: float = 1.0
    gamma1: float = -1.0
    gamma2: float = 1.0
    filt_alpha: float = 36.0
    filt_order: int = 32
    radial_filter_on: bool = False
    sh_keep_l: int = -1                 # -1: angular filter off
    dt: float = 0.01
    steps: int = 20
    seed: int = 0
    noise_amp: float = 0.0
    pulse: Optional[Pulse] = None

    def points(self):
        return sum(n_r * 2 * (L + 1) ** 2 for (_, _, n_r, L) in self.shells)

    def state_len(self):
        return 50 * self.points()

    def noise(self):
        """Seeded N(0,1) * noise_amp on every field value (concatenated state)."""
        if self.noise_amp == 0.0:
            return np.zeros(self.state_len())
        rng = np.random.default_rng(self.seed)
        return rng.standard_normal(self.state_len()) * self.noise_amp


def n_modes(lmax):
    return (lmax + 1) ** 2


def random_coeffs(seed, lmax):
    """c_lm ~ N(0,1)/sqrt(n_modes), drawn after a fixed offset of the stream."""
    rng = np.random.default_rng(seed + 7919)
    n = n_modes(lmax)
    return rng.standard_normal(n) / np.sqrt(n)


def schwarzschild_single_shell(n_r=11, L=7, seed=101):
    """M=1 Schwarzschild in Kerr-Schild coordinates, one shell r in [1.8, 10]."""
    return Workload(name="schwarzschild_1shell_nr%d_L%d" % (n_r, L),
                    shells=[(1.8, 10.0, n_r, L)], M=1.0, chi=0.0,
                    dt=0.01, steps=20, seed=seed, noise_amp=1e-8)


def kerr_four_shells(n_r=21, L=15, seed=102):
    """Kerr a=0.9 M=1, shells [1.3,3,6,12,30], ingoing pulse, both filters on.
    gamma2 = 4: with 1 a three-index constraint mode near the excision sphere
    grows until the run goes non-finite near t = 7.5; with 4 it runs to t = 50."""
    b = [1.3, 3.0, 6.0, 12.0, 30.0]
    keep = (2 * L) // 3
    return Workload(name="kerr_a0.9_4shells_nr%d_L%d" % (n_r, L),
                    shells=[(b[i], b[i + 1], n_r, L) for i in range(4)], M=1.0, chi=0.9,
                    gamma2=4.0, radial_filter_on=True, sh_keep_l=keep, dt=0.005, steps=10000,
                    seed=seed,
                    pulse=Pulse("psi_pulse", 1e-4, 20.0, 2.0, 4, random_coeffs(seed, 4)))


def kerr_eight_shells_large(n_r=41, L=31, seed=105):
    """Kerr a=0.95 M=1, 8 geometric shells spanning [1.2, 100], pulse at R=50;
    gamma2 = 4 as for the 4-shell workload."""
    b = [1.2 * (100.0 / 1.2) ** (k / 8.0) for k in range(9)]
    b[-1] = 100.0
    keep = (2 * L) // 3
    return Workload(name="kerr_a0.95_8shells_nr%d_L%d" % (n_r, L),
                    shells=[(b[i], b[i + 1], n_r, L) for i in range(8)], M=1.0, chi=0.95,
                    gamma2=4.0, radial_filter_on=True, sh_keep_l=keep, dt=0.002, steps=500,
                    seed=seed,
                    pulse=Pulse("psi_pulse", 1e-5, 50.0, 4.0, 8, random_coeffs(seed, 8)))


def paper_single_bh(seed=107):
    """The paper's own test problem (Sec. 3.1): M = 1, spin vector
    chi = (0.2, 0.3, 0.4), two shells [1.62, 6] and [6, 12] with 10 x 19 x 38
    points each (N_r = 10, L = 18: 7,220 points per shell).  No radial filter
    (as in the paper's production runs, Sec. 3.4); SH filter keep l <= 12;
    dt = 0.25 x the smallest grid spacing; seeded 1e-8 noise."""
    shells = [(1.62, 6.0, 10, 18), (6.0, 12.0, 10, 18)]
    return Workload(name="paper_singlebh_chi0.2_0.3_0.4_2shells_nr10_L18", shells=shells, M=1.0,
                    chi=(0.2, 0.3, 0.4), radial_filter_on=False, sh_keep_l=12,
                    dt=_stable_dt(1.62, 6.0, 10, 18), steps=100, seed=seed, noise_amp=1e-8)


def grid_family_resolution(family, k):
    """(N_r, L) of member k of the paper's benchmark grid families (Sec. 3.4):
    SingleBH N_r = 9 + 4k, N_theta = 6 + 2k; BBH N_r = 4 + k, N_theta = 7 + 2k;
    both with N_phi = 2 N_theta, i.e. L = N_theta - 1 on this grid."""
    if family == "singlebh":
        return 9 + 4 * k, 5 + 2 * k
    if family == "bbh":
        return 4 + k, 6 + 2 * k
    raise ValueError(family)


def grid_family_workload(family, k, seed=106):
    """Four Kerr a=0.9 shells [1.3, 3, 6, 12, 30] at the resolution of family
    member k, both filters on, seeded N(0,1) 1e-8 noise."""
    n_r, L = grid_family_resolution(family, k)
    b = [1.3, 3.0, 6.0, 12.0, 30.0]
    return Workload(name="%s_k%d_4shells_nr%d_L%d" % (family, k, n_r, L),
                    shells=[(b[i], b[i + 1], n_r, L) for i in range(4)], M=1.0, chi=0.9,
                    radial_filter_on=True, sh_keep_l=(2 * L) // 3, dt=0.001, steps=20,
                    seed=seed + 17 * k + (0 if family == "singlebh" else 1000), noise_amp=1e-8)


def adjoint_single_shell(seed=104):
    """The single Schwarzschild shell with 16 l<=3 mode coefficients on Pi."""
    w = schwarzschild_single_shell(seed=seed)
    w.name = "adjoint_schwarzschild_1shell"
    w.noise_amp = 0.0
    w.steps = 200
    rng = np.random.default_rng(seed)
    c0 = 1e-3 * rng.standard_normal(16)
    w.pulse = Pulse("pi_modes", 1.0, 5.9, 1.5, 3, c0)
    return w


@dataclass
class BatchedWorkload:
    """Independent single-shell holes evolved together (one shell per hole)."""
    name: str
    holes: list                      # dicts: M, chi, r_in, r_out, n_r, L, dt, seed
    gamma0: float = 1.0
    gamma1: float = -1.0
    gamma2: float = 4.0              # as the Kerr shell workloads (1 left 20 of 64 holes non-finite in 1,000 steps, 4 leaves 8)
    filt_alpha: float = 36.0
    filt_order: int = 32
    radial_filter_on: bool = True
    sh_keep_l: int = -2              # floor(2L/3) on each shell
    noise_amp: float = 1e-8

    @property
    def shells(self):
        return [(h["r_in"], h["r_out"], h["n_r"], h["L"], b) for b, h in enumerate(self.holes)]

    def points(self):
        return sum(h["n_r"] * 2 * (h["L"] + 1) ** 2 for h in self.holes)

    def state_len(self):
        return 50 * self.points()

    def noise(self):
        """Seeded N(0,1) * noise_amp per hole, concatenated in shell order."""
        parts = []
        for h in self.holes:
            n = 50 * h["n_r"] * 2 * (h["L"] + 1) ** 2
            parts.append(np.random.default_rng(h["seed"]).standard_normal(n) * self.noise_amp)
        return np.concatenate(parts)


def _stable_dt(r_in, r_out, n_r, L):
    """0.25 x the smallest grid spacing: the CGL gap or r_in sin(theta_1) 2 pi / N_phi."""
    cgl_gap = 0.5 * (r_out - r_in) * (1.0 - np.cos(np.pi / (n_r - 1)))
    mu = np.polynomial.legendre.leggauss(L + 1)[0]
    s1 = np.sqrt(1.0 - mu.max() ** 2)
    ang_gap = r_in * s1 * 2.0 * np.pi / (2 * (L + 1))
    return 0.25 * min(cgl_gap, ang_gap)


def batched_workload(n_bh=64, seed=103):
    """The batched many-hole workload: seeded spins, masses and resolutions,
    inner radius 0.9 x the polar horizon radius M + sqrt(M^2 - a^2), outer 20 M."""
    holes = []
    for d in batched_black_holes(n_bh, seed):
        M, chi = d["M"], d["chi"]
        a = chi * M
        r_in = 0.9 * (M + np.sqrt(M * M - a * a))
        r_out = 20.0 * M
        holes.append(dict(M=M, chi=chi, r_in=r_in, r_out=r_out, n_r=d["n_r"], L=d["L"], seed=d["seed"],
                          dt=_stable_dt(r_in, r_out, d["n_r"], d["L"])))
    return BatchedWorkload(name="batched_%dbh" % n_bh, holes=holes)


def batched_black_holes(n_bh=64, seed=103):
    """Independent single-shell holes of uneven resolution (seeded draws).

    Returns a list of (M, chi, r_in_factor, r_out_factor, n_r, L, seed_i):
    the inner radius is 0.9 times the polar horizon radius M + sqrt(M^2 - a^2)
    and the outer radius is 20 M.
    """
    rng = np.random.default_rng(seed)
    out = []
    nrs = [9, 13, 17, 21, 25, 33]
    Ls = [7, 11, 15, 23]
    for b in range(n_bh):
        chi = float(rng.uniform(0.0, 0.95))
        M = float(rng.uniform(0.5, 2.0))
        n_r = int(nrs[rng.integers(0, len(nrs))])
        L = int(Ls[rng.integers(0, len(Ls))])
        out.append(dict(M=M, chi=chi, n_r=n_r, L=L, seed=seed * 1000 + b))
    return out
