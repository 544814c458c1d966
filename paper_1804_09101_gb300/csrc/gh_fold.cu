// Symmetry-folded separable angular maps (d/dtheta, d/dphi and the SH
// truncation filter).  The same linear maps as sep_angular_kernel -- the
// projection onto the real Y_lm, l <= K, followed by synthesis of values or
// derivatives (the angular parts of Eq. DifferentiatorI1S2) -- evaluated with
// fewer FP64 operations, since FP64 throughput bounds this kernel on GB300:
//  * phi DFT: cos(m phi_k) and sin(m phi_k) are even/odd under k <-> N - k and
//    (-1)^m even/odd under k <-> N/2 - k, so each ring is folded into four
//    quarter-length vectors and every coefficient is a dot product of length
//    W = floor(N/4) + 1 (a quarter of the dense DFT; for N % 4 == 2 no point is
//    its own quarter mirror and W = (N + 2)/4);
//  * Legendre maps: on symmetric Gauss-Legendre nodes Pbar_lm has parity
//    (-1)^{l+m} about the equator (d/dtheta flips it), so each map acts on the
//    symmetric and antisymmetric halves with half-size matrices (odd N_theta:
//    the equator ring belongs to the symmetric half and is its own mirror);
//  * inverse DFT: the same foldings produce four output points per quarter-ring
//    sum.
// Per (r, field) row: about 2 (N_theta M (N/4+1) + n_out M N_theta N_theta/2 +
// n_out N_theta (N/4+1) M) flops, M = 2K+1, instead of 2 M (N_theta N_phi +
// n_out N_theta^2 + n_out N_theta N_phi).
#include <cuda_runtime.h>

#include "gh_geom.cuh"
#include "gh_internal.h"

namespace gh {

constexpr int FOLD_MAX_THREADS = 512;

__device__ __forceinline__ double flip_sign(double v, unsigned long long mask) {
  // v or -v without an FP64 instruction (mask is 0 or the sign bit)
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)mask);
}

// One block takes RB consecutive (r, field) rows of one shell.  Shared memory
// per row: the input ring values and their quarter folds, later reused for the
// synthesis coefficients, plus the Fourier coefficients of both half-rings.
// The thread count is a launch parameter (a multiple of 32, at most 512).
template <bool TWO>
__global__ void __launch_bounds__(FOLD_MAX_THREADS)
fold_angular_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                    const double* __restrict__ in, double* __restrict__ out0, double* __restrict__ out1) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const FoldPlan& P = TWO ? sh.fd : sh.ff;
  const int nth = sh.nth, nph = sh.nph, na = sh.na;
  const int K = P.K, M = P.M, N4 = P.N4, half = P.half, W = P.W, hs = P.hs, N2 = nph / 2;
  const bool qself = P.qself != 0;
  constexpr int NO = TWO ? 2 : 1;
  const int T = blockDim.x;
  const int rows = NF * sh.n_r;
  const int RB = P.rows_per_cta;
  const int row0 = (blockIdx.x - begin[s]) * RB;
  const int nr = min(RB, rows - row0);
  const int r1 = max(na + 4 * nth * W, NO * nth * M);
  double* U = sm;                                   // [RB][na]
  double* F = U + (size_t)RB * na;                  // [RB][nth][4][W]
  double* OUT = sm;                                 // [NO][RB][nth][M] (after U, F are dead)
  double* AB = sm + (size_t)RB * r1;                // [RB][M][2 hs]: s (hs) then t (hs)
  const int ncoef = P.ncoef;
  double* COEF = AB + (size_t)RB * M * 2 * hs;      // [RB][2][ncoef]: a_l of the cos, then the sin modes m >= m0
  const long long gbase = sh.off + (long long)row0 * na;
  for (int i = threadIdx.x; i < nr * na; i += T) U[i] = in[gbase + i];
  __syncthreads();
  // fold every ring: Cp, Cm (cos, even / odd m), Sp, Sm (sin, odd / even m)
  for (int o = threadIdx.x; o < nr * nth * W; o += T) {
    const int k = o % W;
    const int rj = o / W;
    const double* ring = U + (size_t)rj * nph;
    double* f = F + (size_t)rj * 4 * W;
    auto ev = [&](int kk) { return (kk == 0 || kk == N2) ? ring[kk] : ring[kk] + ring[nph - kk]; };
    auto od = [&](int kk) { return (kk == 0 || kk == N2) ? 0.0 : ring[kk] - ring[nph - kk]; };
    if (!(qself && k == N4)) {
      const double e1 = ev(k), e2 = ev(N2 - k), o1 = od(k), o2 = od(N2 - k);
      f[k] = e1 + e2;
      f[W + k] = e1 - e2;
      f[2 * W + k] = o1 + o2;
      f[3 * W + k] = o1 - o2;
    } else {
      f[k] = ev(N4);
      f[W + k] = 0.0;
      f[2 * W + k] = od(N4);
      f[3 * W + k] = 0.0;
    }
  }
  __syncthreads();
  // phase A: Fourier coefficient of mode for rings j and N_theta-1-j, stored as
  // their sum (symmetric part s) and difference (antisymmetric part t); the
  // equator ring of an odd N_theta is symmetric (s = its coefficient, t = 0)
  for (int o = threadIdx.x; o < nr * hs * M; o += T) {
    const int mode = o % M;
    const int t = o / M;
    const int jh = t % hs;
    const int rr = t / hs;
    const bool cosm = mode <= K;
    const int m = cosm ? mode : mode - K;
    const int q = cosm ? (m % 2 == 0 ? 0 : 1) : (m % 2 == 1 ? 2 : 3);
    const double* tab = (cosm ? P.Tc : P.Ts) + (size_t)m * W;
    const double* f1 = F + ((size_t)(rr * nth + jh) * 4 + q) * W;
    double* ab = AB + ((size_t)rr * M + mode) * 2 * hs;
    if (jh < half) {
      const double* f2 = F + ((size_t)(rr * nth + nth - 1 - jh) * 4 + q) * W;
      double c1 = f1[0] * __ldg(tab), c2 = f2[0] * __ldg(tab);
      for (int k = 1; k < W; ++k) {
        const double tv = __ldg(tab + k);
        c1 = fma(f1[k], tv, c1);
        c2 = fma(f2[k], tv, c2);
      }
      ab[jh] = c1 + c2;
      ab[hs + jh] = c1 - c2;
    } else {
      double c1 = f1[0] * __ldg(tab);
      for (int k = 1; k < W; ++k) c1 = fma(f1[k], __ldg(tab + k), c1);
      ab[jh] = c1;
      ab[hs + jh] = 0.0;
    }
  }
  __syncthreads();
  // phase B1: for modes m >= m0, the Legendre analysis a_l = sum_j A_l(j) (s or
  // t)_j for l = m .. K (s part for l + m even, t part for l + m odd)
  if (ncoef > 0) {
    for (int o = threadIdx.x; o < nr * 2 * ncoef; o += T) {
      const int slot = o % ncoef;
      const int t = o / ncoef;
      const int sinp = t & 1;
      const int rr = t >> 1;
      const int m = __ldg(P.slot_m + slot);
      if (sinp && m == 0) continue;               // no sin mode 0
      const int idx = slot - __ldg(P.coef_off + m);
      const int mode = sinp ? K + m : m;
      const double* v = AB + ((size_t)rr * M + mode) * 2 * hs + ((idx & 1) ? hs : 0);
      const double* a = P.A + (size_t)slot * hs;
      double acc = v[0] * __ldg(a);
      for (int jj = 1; jj < hs; ++jj) acc = fma(v[jj], __ldg(a + jj), acc);
      COEF[((size_t)rr * 2 + sinp) * ncoef + slot] = acc;
    }
    __syncthreads();
  }
  // phase B: half-size Legendre maps (tables carry the synthesis factors);
  // modes m >= m0 synthesise from their coefficients instead
  const unsigned long long sbit = 0x8000000000000000ULL;
  for (int o = threadIdx.x; o < nr * M * hs; o += T) {
    const int j = o % hs;
    const int t = o / hs;
    const int mode = t % M;
    const int rr = t / M;
    const bool cosm = mode <= K;
    const int m = cosm ? mode : mode - K;
    const double* ab = AB + ((size_t)rr * M + mode) * 2 * hs;
    double Sv[2], Tv[2];
    if (m >= P.m0) {
      const int off = __ldg(P.coef_off + m), nl = K + 1 - m;
      const double* a = COEF + ((size_t)rr * 2 + (cosm ? 0 : 1)) * ncoef + off;
      const double* y0 = P.Y0 + (size_t)off * hs + j;
      const double* y1 = TWO ? P.Y1 + (size_t)off * hs + j : nullptr;
      Sv[0] = Tv[0] = 0.0;
      if (TWO) Sv[1] = Tv[1] = 0.0;
      for (int idx = 0; idx < nl; idx += 2) {         // l + m even: the s part
        const double av = a[idx];
        Sv[0] = fma(__ldg(y0 + (size_t)idx * hs), av, Sv[0]);
        if (TWO) Sv[1] = fma(__ldg(y1 + (size_t)idx * hs), av, Sv[1]);
      }
      for (int idx = 1; idx < nl; idx += 2) {         // l + m odd: the t part
        const double av = a[idx];
        Tv[0] = fma(__ldg(y0 + (size_t)idx * hs), av, Tv[0]);
        if (TWO) Tv[1] = fma(__ldg(y1 + (size_t)idx * hs), av, Tv[1]);
      }
    } else {
      const size_t mo = (size_t)m * hs * hs + j;
      const double* Q0s = P.Q0s + mo;
      const double* Q0t = P.Q0t + mo;
      const double* Q1s = TWO ? P.Q1s + mo : nullptr;
      const double* Q1t = TWO ? P.Q1t + mo : nullptr;
      const double sv0 = ab[0], tv0 = ab[hs];
      Sv[0] = __ldg(Q0s) * sv0;
      Tv[0] = __ldg(Q0t) * tv0;
      if (TWO) {
        Sv[1] = __ldg(Q1s) * sv0;
        Tv[1] = __ldg(Q1t) * tv0;
      }
      for (int jp = 1; jp < hs; ++jp) {
        const double sv = ab[jp], tv = ab[hs + jp];
        Sv[0] = fma(__ldg(Q0s + jp * hs), sv, Sv[0]);
        Tv[0] = fma(__ldg(Q0t + jp * hs), tv, Tv[0]);
        if (TWO) {
          Sv[1] = fma(__ldg(Q1s + jp * hs), sv, Sv[1]);
          Tv[1] = fma(__ldg(Q1t + jp * hs), tv, Tv[1]);
        }
      }
    }
    const bool eq = (j >= half);            // the equator ring of an odd N_theta
#pragma unroll
    for (int o2 = 0; o2 < NO; ++o2) {
      // parity of the output about the equator
      const unsigned long long par = ((o2 == 0 ? P.sigma0 : P.sigma1) < 0.0) ? sbit : 0ULL;
      unsigned long long flip = 0ULL;
      int slot = mode;
      if (TWO && o2 == 1) {
        // d/dphi: the value projection of cos mode m feeds sin slot m with
        // factor -m, that of sin mode m feeds cos slot m with +m
        if (cosm) {
          if (m == 0) {
            double* c = OUT + (size_t)RB * nth * M + (size_t)rr * nth * M;
            c[(size_t)j * M] = 0.0;
            if (!eq) c[(size_t)(nth - 1 - j) * M] = 0.0;
            continue;
          }
          slot = K + m;
          flip = sbit;
        } else {
          slot = m;
        }
      }
      const double y1 = Sv[o2] + Tv[o2];
      double* c = OUT + (size_t)o2 * RB * nth * M + (size_t)rr * nth * M;
      c[(size_t)j * M + slot] = flip_sign(y1, flip);
      if (!eq) c[(size_t)(nth - 1 - j) * M + slot] = flip_sign(Sv[o2] - Tv[o2], flip ^ par);
    }
  }
  __syncthreads();
  // phase C: quarter-ring sums give four output points each; one item per
  // (output, ring, k)
  for (int o = threadIdx.x; o < NO * nr * nth * W; o += T) {
    const int k = o % W;
    const int t = o / W;
    const int o2 = TWO ? t % NO : 0;
    const int rj = TWO ? t / NO : t;
    const int rr = rj / nth;
    const int j = rj - rr * nth;
    const double* c = OUT + (size_t)o2 * RB * nth * M + (size_t)rj * M;
    double Ee = c[0] * __ldg(P.Tc + k), Eo = 0.0, Oe = 0.0, Oo = 0.0;
    for (int m = 1; m <= K; m += 2) {
      const double tc1 = __ldg(P.Tc + (size_t)m * W + k);
      const double ts1 = __ldg(P.Ts + (size_t)m * W + k);
      Eo = fma(c[m], tc1, Eo);
      Oo = fma(c[K + m], ts1, Oo);
      if (m + 1 <= K) {
        const double tc2 = __ldg(P.Tc + (size_t)(m + 1) * W + k);
        const double ts2 = __ldg(P.Ts + (size_t)(m + 1) * W + k);
        Ee = fma(c[m + 1], tc2, Ee);
        Oe = fma(c[K + m + 1], ts2, Oe);
      }
    }
    const double Ek = Ee + Eo, Eh = Ee - Eo, Ok = Oe + Oo, Oh = Oo - Oe;
    double* dst = (o2 == 0 ? out0 : out1) + gbase + (long long)rr * na + (long long)j * nph;
    if (k == 0) {
      dst[0] = Ek + Ok;
      dst[N2] = Eh + Oh;
    } else if (qself && k == N4) {
      dst[N4] = Ek + Ok;
      dst[nph - N4] = Ek - Ok;
    } else {
      dst[k] = Ek + Ok;
      dst[N2 - k] = Eh + Oh;
      dst[N2 + k] = Eh - Oh;
      dst[nph - k] = Ek - Ok;
    }
  }
}

// ---------------------------------------------------------------------------
// Exact transpose of fold_angular_kernel (reverse mode).  TWO: out +=
// Theta^T in0 + Phi^T in1 (the cotangents of d/dtheta and d/dphi); one:
// out = S^T in0 (the filter).  The forward map of a row is C_o B_o A (analysis
// A with its ring folding, half-size Legendre maps B_o, synthesis C_o of
// output o), so the transpose is A^T sum_o B_o^T C_o^T, evaluated in three
// phases with the same tables and foldings:
//  * C_o^T is the forward's fold and phase A on each cotangent ring (the
//    quarter-ring combinations are the transposed four-point outputs);
//  * B_o^T reads the Legendre tables with input and output swapped, the
//    output parity (and the d/dphi slot map) now combining the mirrored rings
//    of the cotangent before the map, the symmetric/antisymmetric split after;
//  * A^T is the forward's phase C on the per-ring coefficient cotangents.
// Shared memory per row: region 1 (the cotangent ring and its folds, later the
// parity-combined coefficients) and CB (the analysed coefficients of both
// outputs, later the per-ring coefficient cotangents).
__host__ __device__ inline size_t fold_adj_row_doubles(int na, int nth, int W, int M, int n_out) {
  const size_t hs2 = 2 * (size_t)((nth + 1) / 2);
  size_t r1 = (size_t)na + 4 * (size_t)nth * W;
  if ((size_t)n_out * M * hs2 > r1) r1 = (size_t)n_out * M * hs2;
  return r1 + (size_t)n_out * nth * M;
}

template <bool TWO>
__global__ void __launch_bounds__(FOLD_MAX_THREADS)
fold_adjoint_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                    const double* __restrict__ in0, const double* __restrict__ in1, double* __restrict__ out) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const FoldPlan& P = TWO ? sh.fd : sh.ff;
  const int nth = sh.nth, nph = sh.nph, na = sh.na;
  const int K = P.K, M = P.M, N4 = P.N4, half = P.half, W = P.W, hs = P.hs, N2 = nph / 2;
  const bool qself = P.qself != 0;
  constexpr int NO = TWO ? 2 : 1;
  const int T = blockDim.x;
  const int rows = NF * sh.n_r;
  const int RB = P.adj_rows_per_cta;
  const int row0 = (blockIdx.x - begin[s]) * RB;
  const int nr = min(RB, rows - row0);
  size_t r1 = (size_t)na + 4 * (size_t)nth * W;
  if ((size_t)NO * M * 2 * hs > r1) r1 = (size_t)NO * M * 2 * hs;
  double* Y = sm;                                   // [RB][na] one output's cotangent rings
  double* F = Y + (size_t)RB * na;                  // [RB][nth][4][W] their folds
  double* SV = sm;                                  // [NO][RB][M][2 hs] parity-combined (after Y, F)
  double* CB = sm + (size_t)RB * r1;                // [NO][RB][nth][M] analysed coefficients
  double* AB = CB;                                  // [RB][nth][M] coefficient cotangents (after CB)
  const long long gbase = sh.off + (long long)row0 * na;
  const unsigned long long sbit = 0x8000000000000000ULL;
  // phase 1 (C_o^T): fold and analyse every cotangent ring of each output
#pragma unroll
  for (int o2 = 0; o2 < NO; ++o2) {
    const double* in = o2 == 0 ? in0 : in1;
    if (o2 > 0) __syncthreads();                    // Y and F are reused
    for (int i = threadIdx.x; i < nr * na; i += T) Y[i] = in[gbase + i];
    __syncthreads();
    for (int o = threadIdx.x; o < nr * nth * W; o += T) {
      const int k = o % W;
      const int rj = o / W;
      const double* ring = Y + (size_t)rj * nph;
      double* f = F + (size_t)rj * 4 * W;
      auto ev = [&](int kk) { return (kk == 0 || kk == N2) ? ring[kk] : ring[kk] + ring[nph - kk]; };
      auto od = [&](int kk) { return (kk == 0 || kk == N2) ? 0.0 : ring[kk] - ring[nph - kk]; };
      if (!(qself && k == N4)) {
        const double e1 = ev(k), e2 = ev(N2 - k), o1 = od(k), o2v = od(N2 - k);
        f[k] = e1 + e2;
        f[W + k] = e1 - e2;
        f[2 * W + k] = o1 + o2v;
        f[3 * W + k] = o1 - o2v;
      } else {
        f[k] = ev(N4);
        f[W + k] = 0.0;
        f[2 * W + k] = od(N4);
        f[3 * W + k] = 0.0;
      }
    }
    __syncthreads();
    // one item per (row, ring pair, mode): the coefficients of ring j and of
    // its mirror share the table loads
    for (int o = threadIdx.x; o < nr * hs * M; o += T) {
      const int mode = o % M;
      const int t = o / M;
      const int jh = t % hs;
      const int rr = t / hs;
      const bool cosm = mode <= K;
      const int m = cosm ? mode : mode - K;
      const int q = cosm ? (m % 2 == 0 ? 0 : 1) : (m % 2 == 1 ? 2 : 3);
      const double* tab = (cosm ? P.Tc : P.Ts) + (size_t)m * W;
      const double* f1 = F + ((size_t)(rr * nth + jh) * 4 + q) * W;
      double* cb = CB + ((size_t)o2 * RB + rr) * nth * M + mode;
      if (jh < half) {
        const double* f2 = F + ((size_t)(rr * nth + nth - 1 - jh) * 4 + q) * W;
        double c1 = f1[0] * __ldg(tab), c2 = f2[0] * __ldg(tab);
        for (int k = 1; k < W; ++k) {
          const double tv = __ldg(tab + k);
          c1 = fma(f1[k], tv, c1);
          c2 = fma(f2[k], tv, c2);
        }
        cb[(size_t)jh * M] = c1;
        cb[(size_t)(nth - 1 - jh) * M] = c2;
      } else {
        double c1 = f1[0] * __ldg(tab);
        for (int k = 1; k < W; ++k) c1 = fma(f1[k], __ldg(tab + k), c1);
        cb[(size_t)jh * M] = c1;
      }
    }
  }
  __syncthreads();
  // phase 2a: per (output, row, mode, j < hs) the cotangents of the forward's
  // symmetric and antisymmetric map outputs Sv, Tv (the forward wrote
  // c[j] = f (Sv + Tv) and c[nth-1-j] = f p (Sv - Tv), f the d/dphi sign, p
  // the output parity; the equator ring of an odd N_theta only Sv + Tv)
  for (int o = threadIdx.x; o < NO * nr * M * hs; o += T) {
    const int j = o % hs;
    int t = o / hs;
    const int mode = t % M;
    t /= M;
    const int rr = t % nr;
    const int o2 = TWO ? t / nr : 0;
    const bool cosm = mode <= K;
    const int m = cosm ? mode : mode - K;
    double* sv = SV + (((size_t)o2 * RB + rr) * M + mode) * 2 * hs;
    int slot = mode;
    unsigned long long flip = 0ULL;
    if (TWO && o2 == 1) {
      if (cosm) {
        if (m == 0) {                  // the forward wrote a constant zero
          sv[j] = 0.0;
          sv[hs + j] = 0.0;
          continue;
        }
        slot = K + m;
        flip = sbit;
      } else {
        slot = m;
      }
    }
    const unsigned long long par = ((o2 == 0 ? P.sigma0 : P.sigma1) < 0.0) ? sbit : 0ULL;
    const double* cb = CB + ((size_t)o2 * RB + rr) * nth * M + slot;
    const double y1 = flip_sign(cb[(size_t)j * M], flip);
    if (j < half) {
      const double y2 = flip_sign(cb[(size_t)(nth - 1 - j) * M], flip ^ par);
      sv[j] = y1 + y2;
      sv[hs + j] = y1 - y2;
    } else {
      sv[j] = y1;
      sv[hs + j] = y1;
    }
  }
  __syncthreads();
  // phase 2b (B_o^T, summed over outputs, then the transposed split into the
  // rings j and N_theta-1-j): one item per (row, mode, jp)
  for (int o = threadIdx.x; o < nr * M * hs; o += T) {
    const int jp = o % hs;
    const int t = o / hs;
    const int mode = t % M;
    const int rr = t / M;
    const bool cosm = mode <= K;
    const int m = cosm ? mode : mode - K;
    const size_t mo = (size_t)m * hs * hs + (size_t)jp * hs;
    double sb = 0.0, tb = 0.0;
#pragma unroll
    for (int o2 = 0; o2 < NO; ++o2) {
      const double* Qs = (o2 == 0 ? P.Q0s : P.Q1s) + mo;
      const double* Qt = (o2 == 0 ? P.Q0t : P.Q1t) + mo;
      const double* sv = SV + (((size_t)o2 * RB + rr) * M + mode) * 2 * hs;
      for (int j = 0; j < hs; ++j) {
        sb = fma(__ldg(Qs + j), sv[j], sb);
        tb = fma(__ldg(Qt + j), sv[hs + j], tb);
      }
    }
    double* ab = AB + (size_t)rr * nth * M + mode;
    if (jp < half) {
      ab[(size_t)jp * M] = sb + tb;
      ab[(size_t)(nth - 1 - jp) * M] = sb - tb;
    } else {
      ab[(size_t)jp * M] = sb;           // the equator's t entry was a constant zero
    }
  }
  __syncthreads();
  // phase 3 (A^T): the forward's synthesis of four ring points per
  // quarter-ring sum, from the coefficient cotangents
  for (int o = threadIdx.x; o < nr * nth * W; o += T) {
    const int k = o % W;
    const int rj = o / W;
    const int rr = rj / nth;
    const int j = rj - rr * nth;
    const double* c = AB + (size_t)rj * M;
    double Ee = c[0] * __ldg(P.Tc + k), Eo = 0.0, Oe = 0.0, Oo = 0.0;
    for (int m = 1; m <= K; m += 2) {
      const double tc1 = __ldg(P.Tc + (size_t)m * W + k);
      const double ts1 = __ldg(P.Ts + (size_t)m * W + k);
      Eo = fma(c[m], tc1, Eo);
      Oo = fma(c[K + m], ts1, Oo);
      if (m + 1 <= K) {
        const double tc2 = __ldg(P.Tc + (size_t)(m + 1) * W + k);
        const double ts2 = __ldg(P.Ts + (size_t)(m + 1) * W + k);
        Ee = fma(c[m + 1], tc2, Ee);
        Oe = fma(c[K + m + 1], ts2, Oe);
      }
    }
    const double Ek = Ee + Eo, Eh = Ee - Eo, Ok = Oe + Oo, Oh = Oo - Oe;
    double* dst = out + gbase + (long long)rr * na + (long long)j * nph;
    auto put = [&](int idx, double v) { dst[idx] = TWO ? dst[idx] + v : v; };
    if (k == 0) {
      put(0, Ek + Ok);
      put(N2, Eh + Oh);
    } else if (qself && k == N4) {
      put(N4, Ek + Ok);
      put(nph - N4, Ek - Ok);
    } else {
      put(k, Ek + Ok);
      put(N2 - k, Eh + Oh);
      put(N2 + k, Eh - Oh);
      put(nph - k, Ek - Ok);
    }
  }
}

size_t fold_adjoint_row_doubles(int na, int nth, int W, int M, int n_out) {
  return fold_adj_row_doubles(na, nth, W, M, n_out);
}

cudaError_t launch_fold_adjoint(gh_domain* d, bool two, const double* in0, const double* in1, double* out) {
  if (two)
    fold_adjoint_kernel<true><<<d->fda_blocks, FOLD_ADJ_THREADS, d->fda_smem, d->stream>>>(
        d->shells_d, d->n_shells, d->fda_block_begin_d, in0, in1, out);
  else
    fold_adjoint_kernel<false><<<d->ffa_blocks, FOLD_ADJ_THREADS, d->ffa_smem, d->stream>>>(
        d->shells_d, d->n_shells, d->ffa_block_begin_d, in0, nullptr, out);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t fold_set_smem_limits(size_t bytes) {
  cudaError_t e = raise_smem_limit((const void*)fold_angular_kernel<true>, bytes);
  if (e != cudaSuccess) return e;
  return raise_smem_limit((const void*)fold_angular_kernel<false>, bytes);
}

cudaError_t fold_adjoint_set_smem_limits(size_t bytes) {
  cudaError_t e = raise_smem_limit((const void*)fold_adjoint_kernel<true>, bytes);
  if (e != cudaSuccess) return e;
  return raise_smem_limit((const void*)fold_adjoint_kernel<false>, bytes);
}

cudaError_t launch_fold_deriv(gh_domain* d, const double* in, double* dth, double* dph) {
  fold_angular_kernel<true><<<d->fd_blocks, d->fd_threads, d->fd_smem, d->stream>>>(
      d->shells_d, d->n_shells, d->fd_block_begin_d, in, dth, dph);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_fold_filter(gh_domain* d, const double* in, double* out) {
  fold_angular_kernel<false><<<d->ff_blocks, d->ff_threads, d->ff_smem, d->stream>>>(
      d->shells_d, d->n_shells, d->ff_block_begin_d, in, out, nullptr);
  d->launches++;
  return cudaGetLastError();
}

}  // namespace gh
