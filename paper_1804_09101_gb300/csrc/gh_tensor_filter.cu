// Tensor spherical-harmonic truncation filter on S2 shells (the tensor-coupled
// S2 filter of Secs. 3.1 and 3.4).  Every Cartesian index of the GH tensors
// is expressed in the local complex frame E_0 = r_hat, E_1 = m = (theta_hat +
// i phi_hat)/sqrt(2), E_2 = conj(m); a frame component c_A = T_I E_A1^I1 ..
// has spin weight s = #m - #conj(m) and is projected onto the spin-weighted
// harmonics sY_lm, |s| <= l <= K; the filtered tensor is
// Re sum_A c'_A conj(E_A1) x .. (conj(E) is the dual basis).  Three kernels:
//   tf_frame_kernel   per point: the complex components of the 9 tensor groups
//                     (psi_00, psi_0i, psi_ij, the same for Pi, Phi_i00,
//                     Phi_i0j, Phi_ijk), one index contracted at a time; the
//                     31 independent ones of the 65 are stored;
//   tf_spin_kernel    per (r, independent component) row: complex phi DFT
//                     (m = -K..K), the real N_theta x N_theta map of (s, m),
//                     inverse DFT;
//   tf_unframe_kernel per point: all 65 from the 31, back to the Cartesian
//                     components.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "gh_geom.cuh"
#include "gh_internal.h"
#include "gh_tensor.cuh"

namespace gh {

// The 9 tensor groups (psi_00, psi_0i, psi_ij, Pi_00, Pi_0i, Pi_ij, Phi_i00,
// Phi_i0j, Phi_ijk): rank, and the field of each Cartesian index tuple o
// (row-major, first index slowest).  Everything here is constexpr so that the
// unrolled contractions keep only what is stored.
__host__ __device__ constexpr int tf_rank(int g) {
  return (g == 0 || g == 3) ? 0 : (g == 1 || g == 4 || g == 6) ? 1 : (g == 8 ? 3 : 2);
}
__host__ __device__ constexpr int tf_size(int g) {
  return tf_rank(g) == 0 ? 1 : tf_rank(g) == 1 ? 3 : tf_rank(g) == 2 ? 9 : 27;
}
__host__ __device__ constexpr bool tf_sym(int g) { return g == 2 || g == 5 || g == 8; }  // last two indices
__host__ __device__ constexpr int tf_digit(int g, int o, int k) {
  int div = 1;
  for (int q = k + 1; q < tf_rank(g); ++q) div *= 3;
  return (o / div) % 3;
}
__host__ __device__ constexpr int tf_field(int g, int o) {
  return g < 6 ? (g % 3 == 0 ? 10 * (g / 3) + sym_index(0, 0)
                  : g % 3 == 1 ? 10 * (g / 3) + sym_index(0, 1 + o)
                               : 10 * (g / 3) + sym_index(1 + o / 3, 1 + o % 3))
       : g == 6 ? 20 + 10 * o + sym_index(0, 0)
       : g == 7 ? 20 + 10 * (o / 3) + sym_index(0, 1 + o % 3)
                : 20 + 10 * (o / 9) + sym_index(1 + (o / 3) % 3, 1 + o % 3);
}
__host__ __device__ constexpr bool tf_written(int g, int o) {  // the stored tuple of a symmetric pair
  return !tf_sym(g) || tf_digit(g, o, tf_rank(g) - 2) <= tf_digit(g, o, tf_rank(g) - 1);
}
// The frame components of a real tensor obey c_conj(A) = conj(c_A) (conj
// swaps m and conj(m)), and a symmetric pair gives equal components: each
// class {A, swap(A), conj(A), conj(swap(A))} is represented by its first tuple.
__host__ __device__ constexpr int tf_variant(int g, int o, int c, int sw) {
  const int r = tf_rank(g);
  int e[3] = {0, 0, 0};
  for (int k = 0; k < r; ++k) e[k] = tf_digit(g, o, k);
  if (sw) {
    const int x = e[r - 2];
    e[r - 2] = e[r - 1];
    e[r - 1] = x;
  }
  if (c)
    for (int k = 0; k < r; ++k) e[k] = e[k] == 0 ? 0 : 3 - e[k];
  int v = 0;
  for (int k = 0; k < r; ++k) v = 3 * v + e[k];
  return v;
}
__host__ __device__ constexpr int tf_best(int g, int o) {
  int best = o;
  for (int c = 0; c < 2; ++c)
    for (int sw = 0; sw < (tf_sym(g) ? 2 : 1); ++sw)
      if (tf_variant(g, o, c, sw) < best) best = tf_variant(g, o, c, sw);
  return best;
}
__host__ __device__ constexpr bool tf_best_conj(int g, int o) {  // c_o = conj(c_best)
  int best = o;
  bool cj = false;
  for (int c = 0; c < 2; ++c)
    for (int sw = 0; sw < (tf_sym(g) ? 2 : 1); ++sw)
      if (tf_variant(g, o, c, sw) < best) {
        best = tf_variant(g, o, c, sw);
        cj = c != 0;
      }
  return cj;
}
__host__ __device__ constexpr int tf_row(int g, int o) {  // independent row of tuple o, -1 if not canonical
  if (tf_best(g, o) != o) return -1;
  int row = 0;
  for (int gg = 0; gg < g; ++gg)
    for (int oo = 0; oo < tf_size(gg); ++oo) row += tf_best(gg, oo) == oo;
  for (int oo = 0; oo < o; ++oo) row += tf_best(g, oo) == oo;
  return row;
}
__host__ __device__ constexpr int tf_spin(int g, int o) {  // #m - #conj(m)
  int s = 0;
  for (int k = 0; k < tf_rank(g); ++k) s += tf_digit(g, o, k) == 1 ? 1 : (tf_digit(g, o, k) == 2 ? -1 : 0);
  return s;
}
static_assert(tf_row(8, 26) < 0 && tf_row(8, 9 * 1 + 3 * 2 + 2) == TF_ROWS - 1, "31 independent components");

__constant__ signed char c_tf_spin[TF_ROWS];   // spin of each independent row

constexpr int TF_THREADS = 128;

struct Cx {
  double re, im;
};

__device__ __forceinline__ void frame_vectors(const ShellDev& sh, int q, Cx E[3][3]) {
  const int j = q / sh.nph, k = q - j * sh.nph;
  const double st = sh.sth[j], ct = sh.cth[j], sp = sh.sph[k], cp = sh.cph[k];
  const double rh[3] = {st * cp, st * sp, ct};
  const double th[3] = {ct * cp, ct * sp, -st};
  const double ph[3] = {-sp, cp, 0.0};
  const double h = 0.70710678118654752440;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    E[0][i] = {rh[i], 0.0};
    E[1][i] = {h * th[i], h * ph[i]};
    E[2][i] = {h * th[i], -h * ph[i]};
  }
}

// Contract every index of a rank-n tensor (3^n values, row-major, first index
// slowest) with the frame.  Forward (INV = false): Cartesian -> frame,
// c_..A.. = sum_i E_A^i T_..i.. (T real); inverse: frame -> Cartesian with the
// dual basis, T_..i.. = sum_A conj(E_A^i) c_..A...  Fully unrolled (t stays
// in registers); products with a real factor (the input tensor, r_hat, the z
// component of m) skip the zero imaginary part.
template <int RANK, bool INV>
__device__ __forceinline__ void contract(Cx* t, const Cx E[3][3]) {
  constexpr int n = RANK == 0 ? 1 : RANK == 1 ? 3 : RANK == 2 ? 9 : 27;
#pragma unroll
  for (int k = 0; k < RANK; ++k) {
    const int stride = k == RANK - 1 ? 1 : (k == RANK - 2 ? 3 : 9);
    Cx w[n];
#pragma unroll
    for (int o = 0; o < n; ++o) {
      const int Ak = (o / stride) % 3;          // output index
      const int base = o - Ak * stride;
      Cx acc = {0.0, 0.0};
#pragma unroll
      for (int i = 0; i < 3; ++i) {             // summed index
        const int a = INV ? i : Ak, x = INV ? Ak : i;
        const Cx e = INV ? Cx{E[a][x].re, -E[a][x].im} : E[a][x];
        const bool e_real = a == 0 || x == 2;
        const bool v_real = !INV && k == 0;
        const Cx v = t[base + i * stride];
        if (e_real && v_real) {
          acc.re = fma(e.re, v.re, acc.re);
        } else if (e_real) {
          acc.re = fma(e.re, v.re, acc.re);
          acc.im = fma(e.re, v.im, acc.im);
        } else if (v_real) {
          acc.re = fma(e.re, v.re, acc.re);
          acc.im = fma(e.im, v.re, acc.im);
        } else {
          acc.re = fma(e.re, v.re, fma(-e.im, v.im, acc.re));
          acc.im = fma(e.re, v.im, fma(e.im, v.re, acc.im));
        }
      }
      w[o] = acc;
    }
#pragma unroll
    for (int o = 0; o < n; ++o) t[o] = w[o];
  }
}

// component buffer: per radial slice, TF_ROWS rows of na complex values
__device__ __forceinline__ long long tf_index(const ShellDev& sh, int ir, int row, int q) {
  return 2LL * ((sh.pt_off + (long long)ir * sh.na) * TF_ROWS + (long long)row * sh.na + q);
}

template <int G, int O>
__device__ __forceinline__ void tf_load_u(Cx* t, const double* __restrict__ u, long long ubase, int na) {
  t[O] = {u[ubase + (long long)tf_field(G, O) * na], 0.0};
}
template <int G, int O>
__device__ __forceinline__ void tf_store_c(const Cx* t, const ShellDev& sh, int ir, int q, double* __restrict__ cb) {
  constexpr int row = tf_row(G, O);
  if constexpr (row >= 0) {
    const long long c = tf_index(sh, ir, row, q);
    cb[c] = t[O].re;
    cb[c + 1] = t[O].im;
  }
}
template <int G, int O>
__device__ __forceinline__ void tf_load_c(Cx* t, const ShellDev& sh, int ir, int q, const double* __restrict__ cb) {
  constexpr int row = tf_row(G, tf_best(G, O));
  const long long c = tf_index(sh, ir, row, q);
  t[O] = {cb[c], tf_best_conj(G, O) ? -cb[c + 1] : cb[c + 1]};
}
template <int G, int O>
__device__ __forceinline__ void tf_store_u(const Cx* t, double* __restrict__ out, long long ubase, int na) {
  if constexpr (tf_written(G, O)) out[ubase + (long long)tf_field(G, O) * na] = t[O].re;
}

template <int G, int... O>
__device__ __forceinline__ void frame_group(std::integer_sequence<int, O...>, const ShellDev& sh, int ir, int q,
                                            const Cx E[3][3], const double* __restrict__ u, long long ubase,
                                            double* __restrict__ cb) {
  Cx t[sizeof...(O)];
  (tf_load_u<G, O>(t, u, ubase, sh.na), ...);
  contract<tf_rank(G), false>(t, E);
  (tf_store_c<G, O>(t, sh, ir, q, cb), ...);
}

template <int G, int... O>
__device__ __forceinline__ void unframe_group(std::integer_sequence<int, O...>, const ShellDev& sh, int ir, int q,
                                              const Cx E[3][3], const double* __restrict__ cb, long long ubase,
                                              double* __restrict__ out) {
  Cx t[sizeof...(O)];
  (tf_load_c<G, O>(t, sh, ir, q, cb), ...);
  contract<tf_rank(G), true>(t, E);
  (tf_store_u<G, O>(t, out, ubase, sh.na), ...);
}

template <int... G>
__device__ __forceinline__ void frame_all(std::integer_sequence<int, G...>, const ShellDev& sh, int ir, int q,
                                          const Cx E[3][3], const double* __restrict__ u, long long ub,
                                          double* __restrict__ cb) {
  (frame_group<G>(std::make_integer_sequence<int, tf_size(G)>{}, sh, ir, q, E, u, ub, cb), ...);
}
template <int... G>
__device__ __forceinline__ void unframe_all(std::integer_sequence<int, G...>, const ShellDev& sh, int ir, int q,
                                            const Cx E[3][3], const double* __restrict__ cb, long long ub,
                                            double* __restrict__ out) {
  (unframe_group<G>(std::make_integer_sequence<int, tf_size(G)>{}, sh, ir, q, E, cb, ub, out), ...);
}

__global__ void __launch_bounds__(TF_THREADS)
tf_frame_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                const double* __restrict__ u, double* __restrict__ cb) {
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + TF_THREADS - 1) / TF_THREADS;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * TF_THREADS + threadIdx.x;
  if (q >= na) return;
  Cx E[3][3];
  frame_vectors(sh, q, E);
  const long long ub = sh.off + (long long)ir * NF * na + q;
  frame_all(std::make_integer_sequence<int, 9>{}, sh, ir, q, E, u, ub, cb);
}

__global__ void __launch_bounds__(TF_THREADS)
tf_unframe_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                  const double* __restrict__ cb, double* __restrict__ out) {
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + TF_THREADS - 1) / TF_THREADS;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * TF_THREADS + threadIdx.x;
  if (q >= na) return;
  Cx E[3][3];
  frame_vectors(sh, q, E);
  const long long ub = sh.off + (long long)ir * NF * na + q;
  unframe_all(std::make_integer_sequence<int, 9>{}, sh, ir, q, E, cb, ub, out);
}

// One independent component row of one radial slice: the projection onto
// sY_lm, |s| <= l <= K, of a complex function on the (theta, phi) grid:
//   F_m(theta_i) = (1/N_phi) sum_k f(theta_i, phi_k) e^{-i m phi_k},  |m| <= K
//   G_m(theta_j) = sum_i Q^{s,m}[j][i] F_m(theta_i)
//   f'(theta_j, phi_k) = sum_m G_m(theta_j) e^{i m phi_k}.
// phi_{k+N/2} = phi_k + pi multiplies e^{i m phi} by (-1)^m (half-period fold
// of both transforms), and +m, -m share their cos / sin products.
__global__ void __launch_bounds__(TF_THREADS)
tf_spin_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
               double* __restrict__ cb) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const TensorFilterPlan& P = sh.tf;
  const int na = sh.na, nth = sh.nth, nph = sh.nph, h = nph / 2, K = P.K, M2 = 2 * K + 1, K1 = K + 1;
  const int rr = blockIdx.x - begin[s];           // (ir, row)
  const int row = rr % TF_ROWS;
  const int ir = rr / TF_ROWS;
  const int sp = c_tf_spin[row];
  double* f = sm;                                 // [na][2]
  double* F = f + 2 * na;                         // [nth][M2][2], m = -K..K
  double* PM = F + 2 * nth * M2;                  // [nth][K1][4]: G_m + G_-m, G_m - G_-m
  double* gp = cb + tf_index(sh, ir, row, 0);
  for (int i = threadIdx.x; i < 2 * na; i += blockDim.x) f[i] = gp[i];
  __syncthreads();
  const double inv = 1.0 / nph;
  for (int o = threadIdx.x; o < nth * K1; o += blockDim.x) {
    const int m = o % K1, j = o / K1;
    const double sg = (m & 1) ? -1.0 : 1.0;
    const double* c = P.tc + (size_t)m * nph;
    const double* sn = P.ts + (size_t)m * nph;
    const double* fr = f + 2 * j * nph;
    double ac = 0.0, bs = 0.0, bc = 0.0, as = 0.0;
    for (int k = 0; k < h; ++k) {
      const double a = fma(sg, fr[2 * (k + h)], fr[2 * k]);
      const double b = fma(sg, fr[2 * (k + h) + 1], fr[2 * k + 1]);
      const double cs = __ldg(c + k), ss = __ldg(sn + k);
      ac = fma(a, cs, ac);
      bs = fma(b, ss, bs);
      bc = fma(b, cs, bc);
      as = fma(a, ss, as);
    }
    double* Fj = F + 2 * (j * M2 + K);
    Fj[2 * m] = (ac + bs) * inv;                  // (a + ib) e^{-i m phi}
    Fj[2 * m + 1] = (bc - as) * inv;
    Fj[-2 * m] = (ac - bs) * inv;                 // (a + ib) e^{+i m phi}
    Fj[-2 * m + 1] = (bc + as) * inv;
  }
  __syncthreads();
  const double* Qs = P.Q + (size_t)(sp + 3) * M2 * nth * nth;
  for (int o = threadIdx.x; o < nth * K1; o += blockDim.x) {
    const int m = o % K1, j = o / K1;
    const double* Qp = Qs + ((size_t)(K + m) * nth + j) * nth;
    const double* Qn = Qs + ((size_t)(K - m) * nth + j) * nth;
    double pr = 0.0, pi = 0.0, nr = 0.0, ni = 0.0;
    for (int i = 0; i < nth; ++i) {
      const double qp = __ldg(Qp + i), qn = __ldg(Qn + i);
      const double* Fi = F + 2 * (i * M2 + K);
      pr = fma(qp, Fi[2 * m], pr);
      pi = fma(qp, Fi[2 * m + 1], pi);
      nr = fma(qn, Fi[-2 * m], nr);
      ni = fma(qn, Fi[-2 * m + 1], ni);
    }
    double* q4 = PM + 4 * (j * K1 + m);
    if (m == 0) {
      q4[0] = pr;
      q4[1] = pi;
      q4[2] = 0.0;
      q4[3] = 0.0;
    } else {
      q4[0] = pr + nr;
      q4[1] = pi + ni;
      q4[2] = pr - nr;
      q4[3] = pi - ni;
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nth * h; o += blockDim.x) {
    const int k = o % h, j = o / h;
    // sum_m G_m e^{i m phi} = sum_{m>=0} (G_m + G_-m) cos m phi + i (G_m - G_-m) sin m phi
    double er = 0.0, ei = 0.0, orr = 0.0, oi = 0.0;
    const double* q4 = PM + 4 * j * K1;
    for (int m = 0; m < K1; m += 2) {
      const double cs = __ldg(P.tc + (size_t)m * nph + k), ss = __ldg(P.ts + (size_t)m * nph + k);
      er = fma(q4[4 * m], cs, fma(-q4[4 * m + 3], ss, er));
      ei = fma(q4[4 * m + 1], cs, fma(q4[4 * m + 2], ss, ei));
    }
    for (int m = 1; m < K1; m += 2) {
      const double cs = __ldg(P.tc + (size_t)m * nph + k), ss = __ldg(P.ts + (size_t)m * nph + k);
      orr = fma(q4[4 * m], cs, fma(-q4[4 * m + 3], ss, orr));
      oi = fma(q4[4 * m + 1], cs, fma(q4[4 * m + 2], ss, oi));
    }
    double* g0 = gp + 2 * (j * nph + k);
    g0[0] = er + orr;
    g0[1] = ei + oi;
    g0[2 * h] = er - orr;
    g0[2 * h + 1] = ei - oi;
  }
}

namespace {

// Orthonormal basis of the spin-s, azimuthal-m harmonics sY_lm, l0 <= l <= K
// (l0 = max(|m|, |s|)), in theta: with x = cos(theta) they span
// sin(theta/2)^|s+m| cos(theta/2)^|m-s| p(x), deg p <= K - l0, and the p are
// the Jacobi polynomials P_n^(|s+m|, |m-s|) (their weight is the square of the
// prefactor).  Built by the Jacobi three-term recurrence and normalised under
// the Gauss-Legendre quadrature, which integrates these products exactly.  The
// projection kernel sum_l y_l(j) y_l(i) does not depend on the phase convention
// of the harmonics.
void spin_theta_map(int s, int m, int K, const std::vector<double>& x, const std::vector<double>& w,
                    double* Q) {
  const int nth = (int)x.size();
  const int am = m < 0 ? -m : m, as = s < 0 ? -s : s;
  const int l0 = am > as ? am : as;
  for (int q = 0; q < nth * nth; ++q) Q[q] = 0.0;
  if (l0 > K) return;
  const int nb = K - l0 + 1;
  const long double a = std::abs(s + m), b = std::abs(m - s);
  const long double two_pi = 6.283185307179586476925286766559L;
  std::vector<long double> B((size_t)nb * nth);
  for (int j = 0; j < nth; ++j) {
    const long double xj = x[j];
    const long double pre = std::pow((1.0L - xj) / 2.0L, a / 2.0L) * std::pow((1.0L + xj) / 2.0L, b / 2.0L);
    long double p0 = 1.0L, p1 = (a + 1.0L) + (a + b + 2.0L) * (xj - 1.0L) / 2.0L;
    B[j] = pre * p0;
    if (nb > 1) B[(size_t)nth + j] = pre * p1;
    for (int n = 2; n < nb; ++n) {
      const long double c = 2.0L * n + a + b;
      const long double p2 = ((c - 1.0L) * (c * (c - 2.0L) * xj + a * a - b * b) * p1 -
                              2.0L * (n + a - 1.0L) * (n + b - 1.0L) * c * p0) /
                             (2.0L * n * (n + a + b) * (c - 2.0L));
      p0 = p1;
      p1 = p2;
      B[(size_t)n * nth + j] = pre * p2;
    }
  }
  // modified Gram-Schmidt under <f, g> = 2 pi sum_i w_i f_i g_i (the basis is
  // orthogonal already; this normalises it and removes rounding)
  for (int n = 0; n < nb; ++n) {
    long double* bn = &B[(size_t)n * nth];
    for (int k = 0; k < n; ++k) {
      const long double* bk = &B[(size_t)k * nth];
      long double dot = 0.0L;
      for (int i = 0; i < nth; ++i) dot += two_pi * w[i] * bk[i] * bn[i];
      for (int i = 0; i < nth; ++i) bn[i] -= dot * bk[i];
    }
    long double nn = 0.0L;
    for (int i = 0; i < nth; ++i) nn += two_pi * w[i] * bn[i] * bn[i];
    const long double inv = 1.0L / std::sqrt(nn);
    for (int i = 0; i < nth; ++i) bn[i] *= inv;
  }
  for (int j = 0; j < nth; ++j)
    for (int i = 0; i < nth; ++i) {
      long double acc = 0.0L;
      for (int n = 0; n < nb; ++n) acc += B[(size_t)n * nth + j] * B[(size_t)n * nth + i];
      Q[(size_t)j * nth + i] = (double)(two_pi * w[i] * acc);
    }
}

template <typename T>
cudaError_t tf_upload(gh_domain* d, const std::vector<T>& h, T** out) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(T) * (h.empty() ? 1 : h.size()));
  if (e != cudaSuccess) return e;
  d->owned.push_back(p);
  *out = (T*)p;
  return h.empty() ? cudaSuccess : cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

}  // namespace

cudaError_t tensor_filter_prepare(gh_domain* d, const std::vector<std::vector<double>>& gl_x,
                                  const std::vector<std::vector<double>>& gl_w) {
  if (d->tf_buf) return cudaSuccess;
  cudaError_t e;
  signed char spin[TF_ROWS];
  for (int g = 0; g < 9; ++g)
    for (int o = 0; o < tf_size(g); ++o)
      if (tf_row(g, o) >= 0) spin[tf_row(g, o)] = (signed char)tf_spin(g, o);
  if ((e = cudaMemcpyToSymbol(c_tf_spin, spin, sizeof(spin))) != cudaSuccess) return e;
  // per-shell tables, shared between shells of the same (L, keep)
  std::map<std::pair<int, int>, TensorFilterPlan> cache;
  std::vector<int> pb(d->n_shells + 1), rb(d->n_shells + 1);
  int np = 0, nr = 0;
  size_t smem = 0;
  for (int s = 0; s < d->n_shells; ++s) {
    ShellDev& sh = d->shells_h[s];
    pb[s] = np;
    rb[s] = nr;
    np += sh.n_r * ((sh.na + TF_THREADS - 1) / TF_THREADS);
    sh.tf.K = sh.keep;
    if (sh.keep < 0) continue;
    nr += sh.n_r * TF_ROWS;
    const int K = sh.keep, M2 = 2 * K + 1, nth = sh.nth, nph = sh.nph;
    smem = std::max(smem, sizeof(double) * (size_t)(2 * sh.na + 2 * nth * M2 + 4 * nth * (K + 1)));
    const auto key = std::make_pair(sh.L, K);
    if (!cache.count(key)) {
      TensorFilterPlan P{};
      P.K = K;
      std::vector<double> Q((size_t)7 * M2 * nth * nth);
      for (int sp = -3; sp <= 3; ++sp)
        for (int m = -K; m <= K; ++m)
          spin_theta_map(sp, m, K, gl_x[s], gl_w[s], &Q[((size_t)(sp + 3) * M2 + (m + K)) * nth * nth]);
      std::vector<double> tc((size_t)(K + 1) * nph), ts((size_t)(K + 1) * nph);
      for (int m = 0; m <= K; ++m)
        for (int k = 0; k < nph; ++k) {
          const double ang = 2.0 * 3.14159265358979323846 * (double)((m * k) % nph) / nph;
          tc[(size_t)m * nph + k] = std::cos(ang);
          ts[(size_t)m * nph + k] = std::sin(ang);
        }
      double* p = nullptr;
      if ((e = tf_upload(d, Q, &p)) != cudaSuccess) return e;
      P.Q = p;
      if ((e = tf_upload(d, tc, &p)) != cudaSuccess) return e;
      P.tc = p;
      if ((e = tf_upload(d, ts, &p)) != cudaSuccess) return e;
      P.ts = p;
      cache[key] = P;
    }
    sh.tf = cache[key];
  }
  pb[d->n_shells] = np;
  rb[d->n_shells] = nr;
  std::vector<int> both(pb);
  both.insert(both.end(), rb.begin(), rb.end());
  if ((e = tf_upload(d, both, &d->tf_pb_d)) != cudaSuccess) return e;
  d->tf_point_blocks = np;
  d->tf_rows = nr;
  d->tf_smem = smem;
  static size_t spin_smem = 0;
  if ((e = raise_smem_limit((const void*)tf_spin_kernel, smem, &spin_smem)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(d->shells_d, d->shells_h.data(), sizeof(ShellDev) * d->shells_h.size(),
                      cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  void* p = nullptr;
  if ((e = cudaMalloc(&p, sizeof(double) * 2 * TF_ROWS * (size_t)d->points)) != cudaSuccess) return e;
  d->owned.push_back(p);
  d->tf_buf = (double*)p;
  return cudaSuccess;
}

cudaError_t launch_tensor_filter(gh_domain* d, const double* in, double* out) {
  cudaError_t e;
  if (!d->tf_buf) return cudaErrorNotReady;
  const int n = d->n_shells;
  tf_frame_kernel<<<d->tf_point_blocks, TF_THREADS, 0, d->stream>>>(d->shells_d, n, d->tf_pb_d, in, d->tf_buf);
  d->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (d->tf_rows > 0) {
    tf_spin_kernel<<<d->tf_rows, TF_THREADS, d->tf_smem, d->stream>>>(d->shells_d, n, d->tf_pb_d + n + 1, d->tf_buf);
    d->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  tf_unframe_kernel<<<d->tf_point_blocks, TF_THREADS, 0, d->stream>>>(d->shells_d, n, d->tf_pb_d, d->tf_buf, out);
  d->launches++;
  return cudaGetLastError();
}

}  // namespace gh
