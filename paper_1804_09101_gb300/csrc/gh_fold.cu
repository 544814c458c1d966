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
// For N_phi = 16, 32, 64 the phi transforms are real FFTs of each ring in
// registers instead (about 570 FP64 instructions per 64-point ring and
// transform, against about 1,200 for the folded DFT), and a map runs as three
// launches (ring FFTs, Legendre stage, inverse ring FFTs) through state-sized
// scratch; fold_angular_kernel serves the other N_phi in one launch.
#include <cuda_runtime.h>

#include <cmath>

#include "gh_geom.cuh"
#include "gh_internal.h"

namespace gh {

constexpr int FOLD_MAX_THREADS = 512;
// The ring-FFT kernels run FOLD_FFT_WARPS warps of 32 rings per block, three
// blocks per SM (the transforms hold a ring of N_phi <= 64 values in registers,
// up to 168 registers a thread under that bound).

__device__ __forceinline__ double flip_sign(double v, unsigned long long mask) {
  // v or -v without an FP64 instruction (mask is 0 or the sign bit)
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)mask);
}

// ---------------------------------------------------------------------------
// Real FFT of one ring held in registers, for N_phi = 2n = 16, 32, 64.  The
// folded DFT below costs about N_theta M W FMAs per ring each way (1,200 FP64
// instructions at N_phi = 64); the FFT takes about 570.  A ring of N real
// values is packed as n complex values z_j = x_{2j} + i x_{2j+1}, transformed
// by a radix-2 decimation-in-time FFT of size n (input in bit-reversed order,
// output in natural order), and split into the cos/sin coefficients
//   c_m = sum_k x_k cos(2 pi m k / N),  s_m = sum_k x_k sin(2 pi m k / N)
// with X_m = c_m - i s_m = (E_m + w^m O_m), E and O the transforms of the even
// and odd samples, E_m = (Z_m + conj Z_{n-m}) / 2, O_m = (Z_m - conj Z_{n-m}) / 2i,
// w = exp(-2 pi i / N).  The synthesis x_k = sum_m c_m cos(m phi_k) + s_m
// sin(m phi_k) runs the same steps backwards: the Hermitian spectrum is folded
// into n complex values Zc_m = (S_m + i w^-m D_m) / 2 (S, D the sum and
// difference of X_m and conj X_{n-m}) and one FFT with the opposite sign gives
// x_{2j} + i x_{2j+1}.  Butterflies with twiddle 1, +-i or (+-1 +- i)/sqrt 2 are
// special-cased; a general one forms a + w b with two FMA chains and a - w b as
// 2a - (a + w b).  Twiddles e^{2 pi i k / 64} come from constant memory.
__constant__ double c_fft_cos[64], c_fft_sin[64], c_fft_hcos[64], c_fft_hsin[64];

template <int LOG>
__host__ __device__ constexpr int bit_reverse(int j) {
  int r = 0;
  for (int b = 0; b < LOG; ++b)
    if ((j >> b) & 1) r |= 1 << (LOG - 1 - b);
  return r;
}

// One radix-2 stage of span S = 2^LS, then the next.  Twiddle of butterfly j
// in a group: w = exp(SIGN 2 pi i j / (2 S)) = table entry j * 32 / S.
template <int LOG, int SIGN, int LS>
__device__ __forceinline__ void fft_stages(double (&re)[1 << LOG], double (&im)[1 << LOG]) {
  constexpr int n = 1 << LOG, S = 1 << LS;
#pragma unroll
  for (int bf = 0; bf < n / 2; ++bf) {
    const int j = bf % S;
    const int a = (bf / S) * 2 * S + j, b = a + S;
    const double ar = re[a], ai = im[a], br = re[b], bi = im[b];
    if (j == 0) {
      re[a] = ar + br;
      im[a] = ai + bi;
      re[b] = ar - br;
      im[b] = ai - bi;
    } else if (4 * j == 2 * S) {           // w = SIGN i: w b = SIGN (-b_im + i b_re)
      const double tr = SIGN > 0 ? -bi : bi, ti = SIGN > 0 ? br : -br;
      re[a] = ar + tr;
      im[a] = ai + ti;
      re[b] = ar - tr;
      im[b] = ai - ti;
    } else if (8 * j == 2 * S || 8 * j == 6 * S) {
      // w = (sr + i si) / sqrt 2 with sr = +-1 (j = S/4 or 3S/4), si = SIGN
      const double c = c_fft_cos[8];
      const double u = (8 * j == 2 * S) ? (SIGN > 0 ? br - bi : br + bi) : (SIGN > 0 ? -br - bi : bi - br);
      const double v = (8 * j == 2 * S) ? (SIGN > 0 ? bi + br : bi - br) : (SIGN > 0 ? br - bi : -bi - br);
      re[a] = fma(c, u, ar);
      im[a] = fma(c, v, ai);
      re[b] = fma(-c, u, ar);
      im[b] = fma(-c, v, ai);
    } else {
      const int idx = j * (32 / S);
      const double wr = c_fft_cos[idx];
      const double wi = SIGN > 0 ? c_fft_sin[idx] : -c_fft_sin[idx];
      const double pr = fma(wr, br, fma(-wi, bi, ar));
      const double pi = fma(wr, bi, fma(wi, br, ai));
      re[a] = pr;
      im[a] = pi;
      re[b] = fma(2.0, ar, -pr);
      im[b] = fma(2.0, ai, -pi);
    }
  }
  if constexpr (LS + 1 < LOG) fft_stages<LOG, SIGN, LS + 1>(re, im);
}

// Forward transform of the ring x[0 .. 2n) (stride 1, shared memory): on
// return re[m] = c_m and im[m] = s_m for m = 0 .. n - 1.
template <int LOG>
__device__ __forceinline__ void ring_rfft(const double* __restrict__ x, double (&re)[1 << LOG], double (&im)[1 << LOG]) {
  constexpr int n = 1 << LOG, st = 32 >> LOG;    // table stride of w = exp(-2 pi i / 2n)
#pragma unroll
  for (int t = 0; t < n; ++t) {
    re[bit_reverse<LOG>(t)] = x[2 * t];
    im[bit_reverse<LOG>(t)] = x[2 * t + 1];
  }
  fft_stages<LOG, -1, 0>(re, im);
  {
    const double z0r = re[0], z0i = im[0];
    re[0] = z0r + z0i;
    im[0] = 0.0;
  }
  // m = n/2: c = Re Z, s = Im Z (unchanged)
#pragma unroll
  for (int k = 1; k < n / 2; ++k) {
    const double ar = re[k], ai = im[k], br = re[n - k], bi = im[n - k];
    const double er = ar + br, ei = ai - bi, dr = ar - br, di = ai + bi;
    const double hc = c_fft_hcos[k * st], hsn = c_fft_hsin[k * st];
    const double tr = fma(hc, di, -hsn * dr);
    const double ti = fma(hc, dr, hsn * di);
    re[k] = fma(0.5, er, tr);
    im[k] = fma(-0.5, ei, ti);
    re[n - k] = fma(0.5, er, -tr);
    im[n - k] = fma(0.5, ei, ti);
  }
}

// Inverse of ring_rfft's map: from c_m = cf[m] (m <= K) and s_m = cf[K + m]
// (1 <= m <= K), zero above K, the values x_{2j} = re[j], x_{2j+1} = im[j].
template <int LOG>
__device__ __forceinline__ void ring_irfft(const double* __restrict__ cf, int K, double (&re)[1 << LOG],
                                           double (&im)[1 << LOG]) {
  constexpr int n = 1 << LOG, st = 32 >> LOG;
  auto cm = [&](int m) { return m <= K ? cf[m] : 0.0; };
  auto sm = [&](int m) { return m <= K ? cf[K + m] : 0.0; };
  {
    const double c0 = cf[0];
    re[0] = c0;
    im[0] = c0;
    re[bit_reverse<LOG>(n / 2)] = cm(n / 2);
    im[bit_reverse<LOG>(n / 2)] = sm(n / 2);
  }
#pragma unroll
  for (int m = 1; m < n / 2; ++m) {
    const double c1 = cm(m), s1 = sm(m), c2 = cm(n - m), s2 = sm(n - m);
    const double Sr = c1 + c2, Si = s2 - s1, Dr = c1 - c2, Di = -s1 - s2;
    const double hc = c_fft_hcos[m * st], hsn = c_fft_hsin[m * st];
    const double Tr = fma(hc, Dr, -hsn * Di);
    const double Ti = fma(hc, Di, hsn * Dr);
    re[bit_reverse<LOG>(m)] = fma(0.5, Sr, -Ti);
    im[bit_reverse<LOG>(m)] = fma(0.5, Si, Tr);
    re[bit_reverse<LOG>(n - m)] = fma(0.5, Sr, Ti);
    im[bit_reverse<LOG>(n - m)] = fma(-0.5, Si, Tr);
  }
  fft_stages<LOG, 1, 0>(re, im);
}

// Writes (ACC: adds) one synthesised ring, x_{2t} = re[t], x_{2t+1} = im[t].
template <int LOG, bool ACC>
__device__ __forceinline__ void store_ring(double* __restrict__ dst, const double (&re)[1 << LOG],
                                           const double (&im)[1 << LOG]) {
  constexpr int n = 1 << LOG;
  if ((reinterpret_cast<unsigned long long>(dst) & 15ULL) == 0) {
    double2* d2 = reinterpret_cast<double2*>(dst);
#pragma unroll
    for (int t = 0; t < n; ++t) {
      double2 v = make_double2(re[t], im[t]);
      if (ACC) {
        const double2 o = d2[t];
        v.x += o.x;
        v.y += o.y;
      }
      d2[t] = v;
    }
  } else {
#pragma unroll
    for (int t = 0; t < n; ++t) {
      dst[2 * t] = ACC ? dst[2 * t] + re[t] : re[t];
      dst[2 * t + 1] = ACC ? dst[2 * t + 1] + im[t] : im[t];
    }
  }
}

// Phases B1 and B of the folded maps (fold_angular_kernel, fold_legendre_kernel):
// from the symmetric/antisymmetric Fourier coefficients AB [RB][M][2 hs] of nr
// rows, the synthesis coefficients OUT [NO][RB][nth][M] of every output ring
// (COEF [RB][2][ncoef] holds the analysed a_l of the factorised modes).  The
// caller synchronises before reading OUT.
template <bool TWO>
__device__ __forceinline__ void fold_legendre_phase(const FoldPlan& P, const double* __restrict__ AB,
                                                    double* __restrict__ COEF, double* __restrict__ OUT, int RB,
                                                    int nr, int nth) {
  const int K = P.K, M = P.M, half = P.half, hs = P.hs, ncoef = P.ncoef, T = blockDim.x;
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
    auto emit = [&](int o2, double sv, double tv) {
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
            return;
          }
          slot = K + m;
          flip = sbit;
        } else {
          slot = m;
        }
      }
      double* c = OUT + (size_t)o2 * RB * nth * M + (size_t)rr * nth * M;
      c[(size_t)j * M + slot] = flip_sign(sv + tv, flip);
      if (!eq) c[(size_t)(nth - 1 - j) * M + slot] = flip_sign(sv - tv, flip ^ par);
    };
    emit(0, Sv[0], Tv[0]);
    if (TWO) emit(1, Sv[1], Tv[1]);
  }
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
  fold_legendre_phase<TWO>(P, AB, COEF, OUT, RB, nr, nth);
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
// The folded maps of shells with N_phi = 16, 32, 64 run as three launches:
// fold_fft_analysis_kernel (the phi analysis of every ring by register FFT),
// fold_legendre_kernel (phases B1 and B above) and fold_fft_synthesis_kernel
// (the inverse FFT of every output ring).  Split this way each part runs at
// the occupancy it needs: the FFTs hold a ring in registers (168 a thread), the
// Legendre maps want many warps to hide their shared and L2 loads.  Between the
// launches the coefficients go through state-sized scratch buffers with the
// state's own row stride na: AB [row][M][2 hs] and, per output, OUT
// [row][N_theta][M] (both smaller than a row of values).

// One warp per 32 consecutive rings of a shell (whole rows: N_theta divides
// 32).  The rings are staged in shared memory with stride 2n + 1; ring j and its
// mirror N_theta-1-j sit on adjacent lanes and form s = c(j) + c(mirror),
// t = c(j) - c(mirror) by shuffle.
template <int LOG>
__device__ __forceinline__ void warp_ring_analysis(const double* __restrict__ st, double* __restrict__ abg,
                                                   long long row0, int nw, int nth, int na, int hs, int K) {
  constexpr int n = 1 << LOG;
  const unsigned long long sbit = 0x8000000000000000ULL;
  const int lane = threadIdx.x & 31;
  const bool act = lane < nw;              // nw is a multiple of N_theta: lane pairs are all in or all out
  const int q = act ? lane : nw - 1;
  const int rw = q / nth, qq = q - rw * nth, p = qq >> 1, mir = qq & 1;
  const int j = mir ? nth - 1 - p : p;
  double re[n], im[n];
  ring_rfft<LOG>(st + (size_t)(rw * nth + j) * (2 * n + 1), re, im);
  double* ab = abg + (row0 + rw) * na + (mir ? hs : 0) + p;
  const unsigned long long neg = mir ? sbit : 0ULL;
#pragma unroll
  for (int m = 0; m < n; ++m) {
    if (m <= K) {
      const double cv = re[m], cp = __shfl_xor_sync(0xffffffffu, cv, 1);
      if (act) ab[(size_t)m * 2 * hs] = cp + flip_sign(cv, neg);
      if (m > 0) {
        const double sv = im[m], sp = __shfl_xor_sync(0xffffffffu, sv, 1);
        if (act) ab[(size_t)(K + m) * 2 * hs] = sp + flip_sign(sv, neg);
      }
    }
  }
}

template <bool TWO>
__global__ void __launch_bounds__(FOLD_FFT_WARPS * 32, 3)
fold_fft_analysis_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                         const double* __restrict__ in, double* __restrict__ ab_g) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const FoldPlan& P = TWO ? sh.fd : sh.ff;
  const int fl = P.fft_log, nth = sh.nth, nph = sh.nph, na = sh.na;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n_rings = (long long)NF * sh.n_r * nth;
  const long long ring0 = ((long long)(blockIdx.x - begin[s]) * FOLD_FFT_WARPS + warp) * 32;
  if (ring0 >= n_rings) return;
  const int nw = (int)min(32LL, n_rings - ring0);
  double* st = sm + (size_t)warp * 32 * (nph + 1);
  const double* src = in + sh.off + ring0 * nph;
  for (int i = lane; i < nw * nph; i += 32) st[i + (i >> (fl + 1))] = src[i];
  __syncwarp();
  double* abg = ab_g + sh.off;
  const long long row0 = ring0 / nth;
  if (fl == 5) warp_ring_analysis<5>(st, abg, row0, nw, nth, na, P.hs, P.K);
  else if (fl == 4) warp_ring_analysis<4>(st, abg, row0, nw, nth, na, P.hs, P.K);
  else warp_ring_analysis<3>(st, abg, row0, nw, nth, na, P.hs, P.K);
}

// RB rows of one shell per block: AB in, phases B1 and B, OUT out.
template <bool TWO>
__global__ void __launch_bounds__(FOLD_MAX_THREADS)
fold_legendre_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                     const double* __restrict__ ab_g, double* __restrict__ c0_g, double* __restrict__ c1_g) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const FoldPlan& P = TWO ? sh.fd : sh.ff;
  constexpr int NO = TWO ? 2 : 1;
  const int nth = sh.nth, na = sh.na, M = P.M, hs = P.hs, T = blockDim.x;
  const int rows = NF * sh.n_r;
  const int RB = P.rows_per_cta;
  const int row0 = (blockIdx.x - begin[s]) * RB;
  const int nr = min(RB, rows - row0);
  const int abn = M * 2 * hs, outn = nth * M;
  double* AB = sm;                                  // [RB][M][2 hs]
  double* COEF = AB + (size_t)RB * abn;             // [RB][2][ncoef]
  double* OUT = COEF + (size_t)RB * 2 * P.ncoef;    // [NO][RB][nth][M]
  const long long gbase = sh.off + (long long)row0 * na;
  for (int i = threadIdx.x; i < nr * abn; i += T) {
    const int rr = i / abn;
    AB[i] = ab_g[gbase + (long long)rr * na + (i - rr * abn)];
  }
  __syncthreads();
  fold_legendre_phase<TWO>(P, AB, COEF, OUT, RB, nr, nth);
  __syncthreads();
#pragma unroll
  for (int o2 = 0; o2 < NO; ++o2) {
    double* cg = o2 == 0 ? c0_g : c1_g;
    const double* src = OUT + (size_t)o2 * RB * outn;
    for (int i = threadIdx.x; i < nr * outn; i += T) {
      const int rr = i / outn;
      cg[gbase + (long long)rr * na + (i - rr * outn)] = src[i];
    }
  }
}

// One warp per 32 consecutive rings of one output: the rings' coefficients
// (M each) are staged in shared memory, one lane synthesises a ring.
template <bool TWO>
__global__ void __launch_bounds__(FOLD_FFT_WARPS * 32, 3)
fold_fft_synthesis_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                          const double* __restrict__ c0_g, const double* __restrict__ c1_g,
                          double* __restrict__ out0, double* __restrict__ out1) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const FoldPlan& P = TWO ? sh.fd : sh.ff;
  constexpr int NO = TWO ? 2 : 1;
  const int fl = P.fft_log, nth = sh.nth, nph = sh.nph, na = sh.na, M = P.M, K = P.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n_rings = (long long)NF * sh.n_r * nth;
  const long long wpo = (n_rings + 31) / 32;       // warps per output
  const long long w = (long long)(blockIdx.x - begin[s]) * FOLD_FFT_WARPS + warp;
  const int o2 = (int)(w / wpo);
  if (o2 >= NO) return;
  const long long ring0 = (w - o2 * wpo) * 32;
  const int nw = (int)min(32LL, n_rings - ring0);
  const long long row0 = ring0 / nth;
  const double* cg = (o2 == 0 ? c0_g : c1_g) + sh.off + row0 * na;
  double* st = sm + (size_t)warp * 32 * M;
  const int rown = nth * M;
  for (int i = lane; i < nw * M; i += 32) {
    const int rw = i / rown;
    st[i] = cg[(long long)rw * na + (i - rw * rown)];
  }
  __syncwarp();
  if (lane >= nw) return;
  const int rw = lane / nth, j = lane - rw * nth;
  double* dst = (o2 == 0 ? out0 : out1) + sh.off + (row0 + rw) * na + (long long)j * nph;
  const double* cf = st + (size_t)lane * M;
  if (fl == 5) {
    double re[32], im[32];
    ring_irfft<5>(cf, K, re, im);
    store_ring<5, false>(dst, re, im);
  } else if (fl == 4) {
    double re[16], im[16];
    ring_irfft<4>(cf, K, re, im);
    store_ring<4, false>(dst, re, im);
  } else {
    double re[8], im[8];
    ring_irfft<3>(cf, K, re, im);
    store_ring<3, false>(dst, re, im);
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

// Phase 2b of the transposed maps (fold_adjoint_kernel, fold_adj_legendre_kernel):
// B_o^T summed over the outputs, then the transposed split into the rings j and
// N_theta-1-j.  SV [NO][RB][M][2 hs] in (the parity-combined cotangents of the
// forward's symmetric and antisymmetric map outputs), AB [RB][N_theta][M] out
// (the cotangents of every ring's Fourier coefficients).  One item per
// (row, mode, jp); the caller synchronises before reading AB.
template <bool TWO>
__device__ __forceinline__ void fold_adj_legendre_phase(const FoldPlan& P, const double* __restrict__ SV,
                                                        double* __restrict__ AB, int RB, int nr, int nth) {
  constexpr int NO = TWO ? 2 : 1;
  const int K = P.K, M = P.M, half = P.half, hs = P.hs, T = blockDim.x;
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
  fold_adj_legendre_phase<TWO>(P, SV, AB, RB, nr, nth);
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

// ---------------------------------------------------------------------------
// Transposed maps of the shells with ring FFTs, as three launches like the
// forward: fold_fft_adj_analysis_kernel (C_o^T: the analysis of every
// cotangent ring and the parity combination of phase 2a), fold_adj_legendre_kernel
// (phase 2b) and fold_fft_adj_synthesis_kernel (A^T: the synthesis of every
// ring from its coefficient cotangents, added to the output for the
// derivative maps).  Scratch as in the forward (row stride na): SV of output o
// [row][M][2 hs], AB [row][N_theta][M].

// The cotangent rings of output o2 analysed as in warp_ring_analysis; the
// parity-combined cotangents are SV[mode][j] = f (c_j[slot] + p c_mirror[slot])
// and SV[mode][hs + j] = f (c_j[slot] - p c_mirror[slot]), p the output's
// parity about the equator, slot and f the d/dphi slot map and sign (cos mode m
// from sin slot m with -1, sin mode m from cos slot m; cos mode 0 of d/dphi is
// a constant zero in the forward, so its cotangent entries are zero).
template <int LOG>
__device__ __forceinline__ void warp_ring_adj_analysis(const double* __restrict__ st, double* __restrict__ svg,
                                                       long long row0, int nw, int nth, int na, int hs, int K,
                                                       bool dphi, bool odd_parity) {
  constexpr int n = 1 << LOG;
  const unsigned long long sbit = 0x8000000000000000ULL;
  const int lane = threadIdx.x & 31;
  const bool act = lane < nw;
  const int q = act ? lane : nw - 1;
  const int rw = q / nth, qq = q - rw * nth, p = qq >> 1, mir = qq & 1;
  const int j = mir ? nth - 1 - p : p;
  double re[n], im[n];
  ring_rfft<LOG>(st + (size_t)(rw * nth + j) * (2 * n + 1), re, im);
  double* sv = svg + (row0 + rw) * na + (mir ? hs : 0) + p;
  const unsigned long long par = odd_parity ? sbit : 0ULL, sgn = mir ? sbit : 0ULL;
  // lane j: f own + f p other; its mirror lane: f other - f p own
  auto put = [&](int mode, double own, unsigned long long f) {
    const double other = __shfl_xor_sync(0xffffffffu, own, 1);
    const double a = mir ? other : own, b = mir ? own : other;
    if (act) sv[(size_t)mode * 2 * hs] = flip_sign(a, f) + flip_sign(b, f ^ par ^ sgn);
  };
#pragma unroll
  for (int m = 0; m < n; ++m) {
    if (m <= K) {
      if (!dphi) {
        put(m, re[m], 0ULL);
        if (m > 0) put(K + m, im[m], 0ULL);
      } else if (m == 0) {
        if (act) sv[0] = 0.0;
      } else {
        put(m, im[m], sbit);
        put(K + m, re[m], 0ULL);
      }
    }
  }
}

template <bool TWO>
__global__ void __launch_bounds__(FOLD_FFT_WARPS * 32, 3)
fold_fft_adj_analysis_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                             const double* __restrict__ in0, const double* __restrict__ in1,
                             double* __restrict__ sv0_g, double* __restrict__ sv1_g) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const FoldPlan& P = TWO ? sh.fd : sh.ff;
  constexpr int NO = TWO ? 2 : 1;
  const int fl = P.fft_log, nth = sh.nth, nph = sh.nph, na = sh.na;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n_rings = (long long)NF * sh.n_r * nth;
  const long long wpo = (n_rings + 31) / 32;
  const long long w = (long long)(blockIdx.x - begin[s]) * FOLD_FFT_WARPS + warp;
  const int o2 = (int)(w / wpo);
  if (o2 >= NO) return;
  const long long ring0 = (w - o2 * wpo) * 32;
  const int nw = (int)min(32LL, n_rings - ring0);
  double* st = sm + (size_t)warp * 32 * (nph + 1);
  const double* src = (o2 == 0 ? in0 : in1) + sh.off + ring0 * nph;
  for (int i = lane; i < nw * nph; i += 32) st[i + (i >> (fl + 1))] = src[i];
  __syncwarp();
  double* svg = (o2 == 0 ? sv0_g : sv1_g) + sh.off;
  const long long row0 = ring0 / nth;
  const bool dphi = TWO && o2 == 1;
  const bool odd = (o2 == 0 ? P.sigma0 : P.sigma1) < 0.0;
  if (fl == 5) warp_ring_adj_analysis<5>(st, svg, row0, nw, nth, na, P.hs, P.K, dphi, odd);
  else if (fl == 4) warp_ring_adj_analysis<4>(st, svg, row0, nw, nth, na, P.hs, P.K, dphi, odd);
  else warp_ring_adj_analysis<3>(st, svg, row0, nw, nth, na, P.hs, P.K, dphi, odd);
}

template <bool TWO>
__global__ void __launch_bounds__(FOLD_ADJ_THREADS)
fold_adj_legendre_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                         const double* __restrict__ sv0_g, const double* __restrict__ sv1_g,
                         double* __restrict__ ab_g) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const FoldPlan& P = TWO ? sh.fd : sh.ff;
  constexpr int NO = TWO ? 2 : 1;
  const int nth = sh.nth, na = sh.na, M = P.M, hs = P.hs, T = blockDim.x;
  const int rows = NF * sh.n_r;
  const int RB = P.adj_rows_per_cta;
  const int row0 = (blockIdx.x - begin[s]) * RB;
  const int nr = min(RB, rows - row0);
  const int svn = M * 2 * hs, abn = nth * M;
  double* SV = sm;                                  // [NO][RB][M][2 hs]
  double* AB = SV + (size_t)NO * RB * svn;          // [RB][N_theta][M]
  const long long gbase = sh.off + (long long)row0 * na;
#pragma unroll
  for (int o2 = 0; o2 < NO; ++o2) {
    const double* src = o2 == 0 ? sv0_g : sv1_g;
    double* dst = SV + (size_t)o2 * RB * svn;
    for (int i = threadIdx.x; i < nr * svn; i += T) {
      const int rr = i / svn;
      dst[i] = src[gbase + (long long)rr * na + (i - rr * svn)];
    }
  }
  __syncthreads();
  fold_adj_legendre_phase<TWO>(P, SV, AB, RB, nr, nth);
  __syncthreads();
  for (int i = threadIdx.x; i < nr * abn; i += T) {
    const int rr = i / abn;
    ab_g[gbase + (long long)rr * na + (i - rr * abn)] = AB[i];
  }
}

// One warp per 32 consecutive rings: A^T of each ring (its synthesis from the
// coefficient cotangents), added to out for the derivative maps, written for
// the filter.
template <bool TWO>
__global__ void __launch_bounds__(FOLD_FFT_WARPS * 32, 3)
fold_fft_adj_synthesis_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                              const double* __restrict__ ab_g, double* __restrict__ out) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const FoldPlan& P = TWO ? sh.fd : sh.ff;
  const int fl = P.fft_log, nth = sh.nth, nph = sh.nph, na = sh.na, M = P.M, K = P.K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n_rings = (long long)NF * sh.n_r * nth;
  const long long ring0 = ((long long)(blockIdx.x - begin[s]) * FOLD_FFT_WARPS + warp) * 32;
  if (ring0 >= n_rings) return;
  const int nw = (int)min(32LL, n_rings - ring0);
  const long long row0 = ring0 / nth;
  const double* ag = ab_g + sh.off + row0 * na;
  double* st = sm + (size_t)warp * 32 * M;
  const int rown = nth * M;
  for (int i = lane; i < nw * M; i += 32) {
    const int rw = i / rown;
    st[i] = ag[(long long)rw * na + (i - rw * rown)];
  }
  __syncwarp();
  if (lane >= nw) return;
  const int rw = lane / nth, j = lane - rw * nth;
  double* dst = out + sh.off + (row0 + rw) * na + (long long)j * nph;
  const double* cf = st + (size_t)lane * M;
  if (fl == 5) {
    double re[32], im[32];
    ring_irfft<5>(cf, K, re, im);
    store_ring<5, TWO>(dst, re, im);
  } else if (fl == 4) {
    double re[16], im[16];
    ring_irfft<4>(cf, K, re, im);
    store_ring<4, TWO>(dst, re, im);
  } else {
    double re[8], im[8];
    ring_irfft<3>(cf, K, re, im);
    store_ring<3, TWO>(dst, re, im);
  }
}

size_t fold_adjoint_row_doubles(int na, int nth, int W, int M, int n_out, bool fft) {
  // FFT path: fold_adj_legendre_kernel's SV [NO][M][2 hs] and AB [N_theta][M]
  if (fft) return (size_t)n_out * M * 2 * (size_t)((nth + 1) / 2) + (size_t)nth * M;
  return fold_adj_row_doubles(na, nth, W, M, n_out);
}

template <bool TWO>
cudaError_t launch_fold_adjoint_fft(gh_domain* d, const double* in0, const double* in1, double* out) {
  const gh_domain::FoldFftMap& m = d->fxa[TWO ? 0 : 1];
  if (m.an_blocks == 0) return cudaSuccess;
  fold_fft_adj_analysis_kernel<TWO><<<m.an_blocks, FOLD_FFT_WARPS * 32, m.an_smem, d->stream>>>(
      d->shells_d, d->n_shells, m.an_begin_d, in0, in1, d->fft_c0, d->fft_c1);
  fold_adj_legendre_kernel<TWO><<<m.leg_blocks, FOLD_ADJ_THREADS, m.leg_smem, d->stream>>>(
      d->shells_d, d->n_shells, m.leg_begin_d, d->fft_c0, d->fft_c1, d->fft_ab);
  fold_fft_adj_synthesis_kernel<TWO><<<m.sy_blocks, FOLD_FFT_WARPS * 32, m.sy_smem, d->stream>>>(
      d->shells_d, d->n_shells, m.sy_begin_d, d->fft_ab, out);
  d->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_fold_adjoint(gh_domain* d, bool two, const double* in0, const double* in1, double* out) {
  const int blocks = two ? d->fda_blocks : d->ffa_blocks;
  if (blocks > 0) {
    if (two)
      fold_adjoint_kernel<true><<<d->fda_blocks, FOLD_ADJ_THREADS, d->fda_smem, d->stream>>>(
          d->shells_d, d->n_shells, d->fda_block_begin_d, in0, in1, out);
    else
      fold_adjoint_kernel<false><<<d->ffa_blocks, FOLD_ADJ_THREADS, d->ffa_smem, d->stream>>>(
          d->shells_d, d->n_shells, d->ffa_block_begin_d, in0, nullptr, out);
    d->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return two ? launch_fold_adjoint_fft<true>(d, in0, in1, out) : launch_fold_adjoint_fft<false>(d, in0, nullptr, out);
}

cudaError_t fold_fft_tables() {
  double c[64], sn[64], hc[64], hsn[64];
  for (int k = 0; k < 64; ++k) {
    const double ang = 2.0 * 3.14159265358979323846 * (double)k / 64.0;
    c[k] = std::cos(ang);
    sn[k] = std::sin(ang);
    hc[k] = 0.5 * c[k];
    hsn[k] = 0.5 * sn[k];
  }
  cudaError_t e = cudaMemcpyToSymbol(c_fft_cos, c, sizeof(c));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_fft_sin, sn, sizeof(sn));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_fft_hcos, hc, sizeof(hc));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_fft_hsin, hsn, sizeof(hsn));
  return e;
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

cudaError_t fold_fft_adj_set_smem_limits(size_t an_bytes, size_t leg_bytes, size_t sy_bytes) {
  cudaError_t e = raise_smem_limit((const void*)fold_fft_adj_analysis_kernel<true>, an_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_fft_adj_analysis_kernel<false>, an_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_adj_legendre_kernel<true>, leg_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_adj_legendre_kernel<false>, leg_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_fft_adj_synthesis_kernel<true>, sy_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_fft_adj_synthesis_kernel<false>, sy_bytes);
  return e;
}

cudaError_t fold_fft_set_smem_limits(size_t an_bytes, size_t leg_bytes, size_t sy_bytes) {
  cudaError_t e = raise_smem_limit((const void*)fold_fft_analysis_kernel<true>, an_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_fft_analysis_kernel<false>, an_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_legendre_kernel<true>, leg_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_legendre_kernel<false>, leg_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_fft_synthesis_kernel<true>, sy_bytes);
  if (e == cudaSuccess) e = raise_smem_limit((const void*)fold_fft_synthesis_kernel<false>, sy_bytes);
  return e;
}

// The FFT-path launches of one map (TWO: derivatives, else the filter).
template <bool TWO>
cudaError_t launch_fold_fft(gh_domain* d, const double* in, double* out0, double* out1) {
  const gh_domain::FoldFftMap& m = d->fxm[TWO ? 0 : 1];
  if (m.an_blocks == 0) return cudaSuccess;
  fold_fft_analysis_kernel<TWO><<<m.an_blocks, FOLD_FFT_WARPS * 32, m.an_smem, d->stream>>>(
      d->shells_d, d->n_shells, m.an_begin_d, in, d->fft_ab);
  fold_legendre_kernel<TWO><<<m.leg_blocks, TWO ? d->fd_threads : d->ff_threads, m.leg_smem, d->stream>>>(
      d->shells_d, d->n_shells, m.leg_begin_d, d->fft_ab, d->fft_c0, d->fft_c1);
  fold_fft_synthesis_kernel<TWO><<<m.sy_blocks, FOLD_FFT_WARPS * 32, m.sy_smem, d->stream>>>(
      d->shells_d, d->n_shells, m.sy_begin_d, d->fft_c0, d->fft_c1, out0, out1);
  d->launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_fold_deriv(gh_domain* d, const double* in, double* dth, double* dph) {
  if (d->fd_blocks > 0) {
    fold_angular_kernel<true><<<d->fd_blocks, d->fd_threads, d->fd_smem, d->stream>>>(
        d->shells_d, d->n_shells, d->fd_block_begin_d, in, dth, dph);
    d->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_fold_fft<true>(d, in, dth, dph);
}

cudaError_t launch_fold_filter(gh_domain* d, const double* in, double* out) {
  if (d->ff_blocks > 0) {
    fold_angular_kernel<false><<<d->ff_blocks, d->ff_threads, d->ff_smem, d->stream>>>(
        d->shells_d, d->n_shells, d->ff_block_begin_d, in, out, nullptr);
    d->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_fold_fft<false>(d, in, out, nullptr);
}

}  // namespace gh
