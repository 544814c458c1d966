// Tensor spherical-harmonic truncation filter on S2 shells (the tensor-coupled
// S2 filter of Secs. 3.1 and 3.4).  Every Cartesian index of the GH tensors
// is expressed in the local complex frame E_0 = r_hat, E_1 = m = (theta_hat +
// i phi_hat)/sqrt(2), E_2 = conj(m); a frame component c_A = T_I E_A1^I1 ..
// has spin weight s = #m - #conj(m) and is projected onto the spin-weighted
// harmonics sY_lm, |s| <= l <= K; the filtered tensor is
// sum_A c'_A conj(E_A1) x .. (conj(E) is the dual basis).  Three kernels:
//   tf_frame_kernel   per point: the components of the 9 tensor groups
//                     (psi_00, psi_0i, psi_ij, the same for Pi, Phi_i00,
//                     Phi_i0j, Phi_ijk) in the real frame (r_hat, theta_hat,
//                     phi_hat), then the complex combinations; the 31
//                     independent ones of the 65 are stored;
//   tf_spin_kernel    per (r, independent component) row: quarter-folded phi
//                     DFT (m = -K..K), analysis onto and synthesis from the
//                     spin-weighted theta functions of each (s, m), folded
//                     inverse DFT;
//   tf_unframe_kernel per point: all 65 from the 31, back to the real frame
//                     and to the Cartesian components.
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

constexpr int TF_THREADS = 128;        // per-point kernels
constexpr int TF_SPIN_MAX_THREADS = 128;

struct Cx {
  double re, im;
};

// Real orthonormal frame e[a][i]: a = 0 r_hat, 1 theta_hat, 2 phi_hat (phi_hat_z = 0).
__device__ __forceinline__ void real_frame(const ShellDev& sh, int q, double e[3][3]) {
  const int j = q / sh.nph, k = q - j * sh.nph;
  const double st = sh.sth[j], ct = sh.cth[j], sp = sh.sph[k], cp = sh.cph[k];
  e[0][0] = st * cp; e[0][1] = st * sp; e[0][2] = ct;
  e[1][0] = ct * cp; e[1][1] = ct * sp; e[1][2] = -st;
  e[2][0] = -sp;     e[2][1] = cp;      e[2][2] = 0.0;
}

// Contract every index of a rank-n real tensor (3^n values, row-major, first
// index slowest) with the real frame: forward R_..a.. = sum_i e_a^i T_..i..,
// inverse T_..i.. = sum_a e_a^i R_..a...  Fully unrolled (t stays in
// registers); the zero phi_hat_z term is skipped.
template <int RANK, bool INV>
__device__ __forceinline__ void contract_real(double* t, const double e[3][3]) {
  constexpr int n = RANK == 0 ? 1 : RANK == 1 ? 3 : RANK == 2 ? 9 : 27;
#pragma unroll
  for (int k = 0; k < RANK; ++k) {
    const int stride = k == RANK - 1 ? 1 : (k == RANK - 2 ? 3 : 9);
    double w[n];
#pragma unroll
    for (int o = 0; o < n; ++o) {
      const int out = (o / stride) % 3;
      const int base = o - out * stride;
      double acc = 0.0;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const int a = INV ? x : out, i = INV ? out : x;
        if (a == 2 && i == 2) continue;
        acc = fma(e[a][i], t[base + x * stride], acc);
      }
      w[o] = acc;
    }
#pragma unroll
    for (int o = 0; o < n; ++o) t[o] = w[o];
  }
}

// Real frame -> complex frame, index by index: A = 0 keeps R_0, A = 1 takes
// R_1 + i R_2, A = 2 takes R_1 - i R_2 (the 1/sqrt(2) of each m is applied at
// the store).  Additions only.
template <int RANK>
__device__ __forceinline__ void complexify(const double* R, Cx* c) {
  constexpr int n = RANK == 0 ? 1 : RANK == 1 ? 3 : RANK == 2 ? 9 : 27;
#pragma unroll
  for (int o = 0; o < n; ++o) c[o] = {R[o], 0.0};
#pragma unroll
  for (int k = 0; k < RANK; ++k) {
    const int stride = k == RANK - 1 ? 1 : (k == RANK - 2 ? 3 : 9);
    Cx w[n];
#pragma unroll
    for (int o = 0; o < n; ++o) {
      const int A = (o / stride) % 3;
      const int base = o - A * stride;
      const Cx v1 = c[base + stride], v2 = c[base + 2 * stride];
      if (A == 0) {
        w[o] = c[base];
      } else if (k == 0) {                       // inputs still real
        w[o] = {v1.re, A == 1 ? v2.re : -v2.re};
      } else if (A == 1) {
        w[o] = {v1.re - v2.im, v1.im + v2.re};
      } else {
        w[o] = {v1.re + v2.im, v1.im - v2.re};
      }
    }
#pragma unroll
    for (int o = 0; o < n; ++o) c[o] = w[o];
  }
}

// Complex frame -> real frame (the dual basis conj(E)), index by index:
// R_0 = c_0, R_1 = c_1 + c_2, R_2 = i (c_2 - c_1) (1/sqrt(2) at the end); the
// result is real, only its real part is kept.
template <int RANK>
__device__ __forceinline__ void decomplexify(Cx* c, double* R) {
  constexpr int n = RANK == 0 ? 1 : RANK == 1 ? 3 : RANK == 2 ? 9 : 27;
#pragma unroll
  for (int k = 0; k < RANK; ++k) {
    const int stride = k == RANK - 1 ? 1 : (k == RANK - 2 ? 3 : 9);
    Cx w[n];
#pragma unroll
    for (int o = 0; o < n; ++o) {
      const int a = (o / stride) % 3;
      const int base = o - a * stride;
      const Cx v1 = c[base + stride], v2 = c[base + 2 * stride];
      if (a == 0)
        w[o] = c[base];
      else if (a == 1)
        w[o] = {v1.re + v2.re, v1.im + v2.im};
      else
        w[o] = {v1.im - v2.im, v2.re - v1.re};
    }
#pragma unroll
    for (int o = 0; o < n; ++o) c[o] = w[o];
  }
#pragma unroll
  for (int o = 0; o < n; ++o) R[o] = c[o].re;
}

// (1/sqrt(2))^(number of m and conj(m) indices of tuple o)
__host__ __device__ constexpr double tf_scale(int g, int o) {
  int n = 0;
  for (int k = 0; k < tf_rank(g); ++k) n += tf_digit(g, o, k) != 0;
  return n == 0 ? 1.0 : n == 1 ? 0.70710678118654752440 : n == 2 ? 0.5 : 0.35355339059327376220;
}

// component buffer: per radial slice, TF_ROWS rows of na complex values
__device__ __forceinline__ long long tf_index(const ShellDev& sh, int ir, int row, int q) {
  return 2LL * ((sh.pt_off + (long long)ir * sh.na) * TF_ROWS + (long long)row * sh.na + q);
}

template <int G, int O>
__device__ __forceinline__ void tf_load_u(double* t, const double* __restrict__ u, long long ubase, int na) {
  t[O] = u[ubase + (long long)tf_field(G, O) * na];
}
template <int G, int O>
__device__ __forceinline__ void tf_store_c(const Cx* c, const ShellDev& sh, int ir, int q, double* __restrict__ cb) {
  constexpr int row = tf_row(G, O);
  if constexpr (row >= 0) {
    constexpr double f = tf_scale(G, O);
    const long long i = tf_index(sh, ir, row, q);
    cb[i] = f * c[O].re;
    cb[i + 1] = f * c[O].im;
  }
}
template <int G, int O>
__device__ __forceinline__ void tf_load_c(Cx* c, const ShellDev& sh, int ir, int q, const double* __restrict__ cb) {
  constexpr int row = tf_row(G, tf_best(G, O));
  const long long i = tf_index(sh, ir, row, q);
  c[O] = {cb[i], tf_best_conj(G, O) ? -cb[i + 1] : cb[i + 1]};
}
template <int G, int O>
__device__ __forceinline__ void tf_scale_r(double* R) {
  if constexpr (tf_scale(G, O) != 1.0) R[O] *= tf_scale(G, O);
}
template <int G, int O>
__device__ __forceinline__ void tf_store_u(const double* t, double* __restrict__ out, long long ubase, int na) {
  if constexpr (tf_written(G, O)) out[ubase + (long long)tf_field(G, O) * na] = t[O];
}

template <int G, int... O>
__device__ __forceinline__ void frame_group(std::integer_sequence<int, O...>, const ShellDev& sh, int ir, int q,
                                            const double e[3][3], const double* __restrict__ u, long long ubase,
                                            double* __restrict__ cb) {
  double t[sizeof...(O)];
  Cx c[sizeof...(O)];
  (tf_load_u<G, O>(t, u, ubase, sh.na), ...);
  contract_real<tf_rank(G), false>(t, e);
  complexify<tf_rank(G)>(t, c);
  (tf_store_c<G, O>(c, sh, ir, q, cb), ...);
}

template <int G, int... O>
__device__ __forceinline__ void unframe_group(std::integer_sequence<int, O...>, const ShellDev& sh, int ir, int q,
                                              const double e[3][3], const double* __restrict__ cb, long long ubase,
                                              double* __restrict__ out) {
  Cx c[sizeof...(O)];
  double t[sizeof...(O)];
  (tf_load_c<G, O>(c, sh, ir, q, cb), ...);
  decomplexify<tf_rank(G)>(c, t);
  (tf_scale_r<G, O>(t), ...);
  contract_real<tf_rank(G), true>(t, e);
  (tf_store_u<G, O>(t, out, ubase, sh.na), ...);
}

template <int... G>
__device__ __forceinline__ void frame_all(std::integer_sequence<int, G...>, const ShellDev& sh, int ir, int q,
                                          const double e[3][3], const double* __restrict__ u, long long ub,
                                          double* __restrict__ cb) {
  (frame_group<G>(std::make_integer_sequence<int, tf_size(G)>{}, sh, ir, q, e, u, ub, cb), ...);
}
template <int... G>
__device__ __forceinline__ void unframe_all(std::integer_sequence<int, G...>, const ShellDev& sh, int ir, int q,
                                            const double e[3][3], const double* __restrict__ cb, long long ub,
                                            double* __restrict__ out) {
  (unframe_group<G>(std::make_integer_sequence<int, tf_size(G)>{}, sh, ir, q, e, cb, ub, out), ...);
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
  double e[3][3];
  real_frame(sh, q, e);
  const long long ub = sh.off + (long long)ir * NF * na + q;
  frame_all(std::make_integer_sequence<int, 9>{}, sh, ir, q, e, u, ub, cb);
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
  double e[3][3];
  real_frame(sh, q, e);
  const long long ub = sh.off + (long long)ir * NF * na + q;
  unframe_all(std::make_integer_sequence<int, 9>{}, sh, ir, q, e, cb, ub, out);
}

// ---- transpose of the filter (reverse mode).  The spin projection P is
// self-adjoint under the quadrature inner product sum_j w_j conj(f) g, so its
// transpose is D P D^-1 with D = diag(w_j) per theta ring: the transposed
// frame kernels divide by and multiply with w_j around the unchanged spin
// kernel.  The transposes of the per-point steps: complexify <-> decomplexify,
// forward <-> inverse real contraction, the conjugate/symmetric expansion of
// the stored rows -> accumulation into them.
__host__ __device__ constexpr int tf_first_row(int g) { return tf_row(g, 0); }   // tuple 0 is canonical
__host__ __device__ constexpr int tf_group_rows(int g) {
  int n = 0;
  for (int o = 0; o < tf_size(g); ++o) n += tf_best(g, o) == o;
  return n;
}

template <int G, int O>
__device__ __forceinline__ void tf_load_ubar(double* t, const double* __restrict__ ub, long long ubase, int na) {
  if constexpr (tf_written(G, O)) t[O] = ub[ubase + (long long)tf_field(G, O) * na];
  else t[O] = 0.0;
}
template <int G, int O>
__device__ __forceinline__ void tf_accum_row(const Cx* c, Cx* acc) {
  constexpr int r = tf_row(G, tf_best(G, O)) - tf_first_row(G);
  if constexpr (tf_best_conj(G, O)) {
    acc[r].re += c[O].re;
    acc[r].im -= c[O].im;
  } else {
    acc[r].re += c[O].re;
    acc[r].im += c[O].im;
  }
}
template <int G, int O>
__device__ __forceinline__ void tf_load_cbar(Cx* c, const ShellDev& sh, int ir, int q, const double* __restrict__ cb,
                                             double w) {
  constexpr int row = tf_row(G, O);
  if constexpr (row >= 0) {
    constexpr double f = tf_scale(G, O);
    const long long i = tf_index(sh, ir, row, q);
    c[O] = {f * w * cb[i], f * w * cb[i + 1]};
  } else {
    c[O] = {0.0, 0.0};
  }
}
template <int G, int O>
__device__ __forceinline__ void tf_add_u(const double* t, double* uacc) {
  uacc[tf_field(G, O)] += t[O];
}

// U^T, then D^-1: Cartesian cotangent -> row cotangents / w_j
template <int G, int... O>
__device__ __forceinline__ void unframe_t_group(std::integer_sequence<int, O...>, const ShellDev& sh, int ir, int q,
                                                const double e[3][3], double iw, const double* __restrict__ ub,
                                                long long ubase, double* __restrict__ cb) {
  double t[sizeof...(O)];
  Cx c[sizeof...(O)];
  (tf_load_ubar<G, O>(t, ub, ubase, sh.na), ...);
  contract_real<tf_rank(G), false>(t, e);
  (tf_scale_r<G, O>(t), ...);
  complexify<tf_rank(G)>(t, c);
  Cx acc[tf_group_rows(G)];
#pragma unroll
  for (int r = 0; r < tf_group_rows(G); ++r) acc[r] = {0.0, 0.0};
  (tf_accum_row<G, O>(c, acc), ...);
#pragma unroll
  for (int r = 0; r < tf_group_rows(G); ++r) {
    const long long i = tf_index(sh, ir, tf_first_row(G) + r, q);
    cb[i] = iw * acc[r].re;
    cb[i + 1] = iw * acc[r].im;
  }
}

// D, then F^T: row cotangents -> Cartesian cotangent (accumulated per field)
template <int G, int... O>
__device__ __forceinline__ void frame_t_group(std::integer_sequence<int, O...>, const ShellDev& sh, int ir, int q,
                                              const double e[3][3], double w, const double* __restrict__ cb,
                                              double* uacc) {
  Cx c[sizeof...(O)];
  double t[sizeof...(O)];
  (tf_load_cbar<G, O>(c, sh, ir, q, cb, w), ...);
  decomplexify<tf_rank(G)>(c, t);
  contract_real<tf_rank(G), true>(t, e);
  (tf_add_u<G, O>(t, uacc), ...);
}

template <int... G>
__device__ __forceinline__ void unframe_t_all(std::integer_sequence<int, G...>, const ShellDev& sh, int ir, int q,
                                              const double e[3][3], double iw, const double* __restrict__ ub,
                                              long long ubase, double* __restrict__ cb) {
  (unframe_t_group<G>(std::make_integer_sequence<int, tf_size(G)>{}, sh, ir, q, e, iw, ub, ubase, cb), ...);
}
template <int... G>
__device__ __forceinline__ void frame_t_all(std::integer_sequence<int, G...>, const ShellDev& sh, int ir, int q,
                                            const double e[3][3], double w, const double* __restrict__ cb,
                                            double* uacc) {
  (frame_t_group<G>(std::make_integer_sequence<int, tf_size(G)>{}, sh, ir, q, e, w, cb, uacc), ...);
}

__global__ void __launch_bounds__(TF_THREADS)
tf_unframe_t_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                    const double* __restrict__ ub, double* __restrict__ cb) {
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + TF_THREADS - 1) / TF_THREADS;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * TF_THREADS + threadIdx.x;
  if (q >= na) return;
  double e[3][3];
  real_frame(sh, q, e);
  const double iw = 1.0 / sh.wth[q / sh.nph];
  const long long base = sh.off + (long long)ir * NF * na + q;
  unframe_t_all(std::make_integer_sequence<int, 9>{}, sh, ir, q, e, iw, ub, base, cb);
}

__global__ void __launch_bounds__(TF_THREADS)
tf_frame_t_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                  const double* __restrict__ cb, double* __restrict__ out) {
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + TF_THREADS - 1) / TF_THREADS;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * TF_THREADS + threadIdx.x;
  if (q >= na) return;
  double e[3][3];
  real_frame(sh, q, e);
  const double w = sh.wth[q / sh.nph];
  double uacc[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) uacc[f] = 0.0;
  frame_t_all(std::make_integer_sequence<int, 9>{}, sh, ir, q, e, w, cb, uacc);
  const long long base = sh.off + (long long)ir * NF * na + q;
#pragma unroll
  for (int f = 0; f < NF; ++f) out[base + (long long)f * na] = uacc[f];
}

__device__ __forceinline__ int tf_nb(int K, int s, int m) {
  const int am = m < 0 ? -m : m, as = s < 0 ? -s : s;
  const int n = K - (am > as ? am : as) + 1;
  return n > 0 ? n : 0;
}

// Shared-memory doubles of the spin kernel for one shell.
__host__ __device__ inline int tf_spin_smem_doubles(int nth, int K, int W) {
  const int K1 = K + 1, M2 = 2 * K + 1, nthp = nth | 1;
  const int ab = 8 * W * nthp, pm = 4 * nth * K1;
  return 2 * K1 * W + (ab > pm ? ab : pm) + 2 * nth * M2 + 2 * K1 * K1;
}

// One independent component row of one radial slice: the projection onto
// sY_lm, |s| <= l <= K, of a complex function f on the (theta, phi) grid.
//   F_m(theta_i) = (1/N_phi) sum_k f(theta_i, phi_k) e^{-i m phi_k},  |m| <= K,
//   a_n = sum_i 2 pi w_i b_n(theta_i) F_m(theta_i),  G_m(theta_j) = sum_n b_n(theta_j) a_n
//   (b_n the orthonormal theta functions of (s, m)),
//   f'(theta_j, phi_k) = sum_m G_m(theta_j) e^{i m phi_k}.
// Both phi transforms are quarter-folded: phi + pi multiplies e^{i m phi} by
// (-1)^m and pi - phi maps it to (-1)^m e^{-i m phi}, so slots k and h - k
// (h = N_phi/2) share one cos/sin pair, and +m, -m share their products.
// Items are laid out so that the lanes of a warp have equal trip counts.
__global__ void __launch_bounds__(TF_SPIN_MAX_THREADS)
tf_spin_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
               double* __restrict__ cb) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const TensorFilterPlan& P = sh.tf;
  const int nth = sh.nth, nph = sh.nph, h = nph / 2, K = P.K, M2 = 2 * K + 1, K1 = K + 1, W = P.W;
  const int nthp = nth | 1;
  const int rr = blockIdx.x - begin[s];           // (ir, row)
  const int row = rr % TF_ROWS;
  const int ir = rr / TF_ROWS;
  const int sp = c_tf_spin[row];
  const int sb = (sp + 3) * M2;
  double* TC = sm;                                // [K1][W]
  double* TS = TC + K1 * W;                       // [K1][W]
  double* AB = TS + K1 * W;                       // [p][A.re A.im B.re B.im][W][nthp]
  double* PM = AB;                                // later [m][P.re P.im M.re M.im][nth]
  const int r1 = 8 * W * nthp > 4 * nth * K1 ? 8 * W * nthp : 4 * nth * K1;
  double* F = AB + r1;                            // [M2][re, im][nth], m = -K..K
  double* AC = F + 2 * nth * M2;                  // [packed item][2]
  double* gp = cb + tf_index(sh, ir, row, 0);
  for (int i = threadIdx.x; i < K1 * W; i += blockDim.x) {
    TC[i] = __ldg(P.twc + i);
    TS[i] = __ldg(P.tws + i);
  }
  // fold: g^p_k = f_k + (-1)^p f_{k+h};  A^p_k = g^p_k + (-1)^p g^p_{h-k},
  // B^p_k = g^p_k - (-1)^p g^p_{h-k} (k = 0: A = g, B = 0; 2k = h: A = B = g)
  for (int o = threadIdx.x; o < nth * W; o += blockDim.x) {
    const int k = o % W, j = o / W;
    const double* fj = gp + 2 * j * nph;
    const double ar = fj[2 * k], ai = fj[2 * k + 1], br = fj[2 * (k + h)], bi = fj[2 * (k + h) + 1];
    double A0r = ar + br, A0i = ai + bi, A1r = ar - br, A1i = ai - bi;
    double B0r = 0.0, B0i = 0.0, B1r = 0.0, B1i = 0.0;
    if (2 * k == h) {
      B0r = A0r; B0i = A0i; B1r = A1r; B1i = A1i;
    } else if (k > 0) {
      const int k2 = h - k;
      const double cr = fj[2 * k2], ci = fj[2 * k2 + 1], dr = fj[2 * (k2 + h)], di = fj[2 * (k2 + h) + 1];
      const double g0r = cr + dr, g0i = ci + di, g1r = cr - dr, g1i = ci - di;
      B0r = A0r - g0r; B0i = A0i - g0i; A0r += g0r; A0i += g0i;
      B1r = A1r + g1r; B1i = A1i + g1i; A1r -= g1r; A1i -= g1i;
    }
    double* a0 = AB + (size_t)k * nthp + j;
    const int cs = W * nthp;                      // stride between the 8 arrays
    a0[0 * cs] = A0r; a0[1 * cs] = A0i; a0[2 * cs] = B0r; a0[3 * cs] = B0i;
    a0[4 * cs] = A1r; a0[5 * cs] = A1i; a0[6 * cs] = B1r; a0[7 * cs] = B1i;
  }
  __syncthreads();
  // forward: F_{+-m} = (1/N) (sum_k A^p_k c_mk -+ i sum_k B^p_k s_mk), p = m mod 2
  const double inv = 1.0 / nph;
  for (int o = threadIdx.x; o < nth * K1; o += blockDim.x) {
    const int j = o % nth, m = o / nth;
    const int cs = W * nthp;
    const double* ab = AB + (size_t)(m & 1) * 4 * cs + j;
    const double* tc = TC + m * W;
    const double* ts = TS + m * W;
    double acr = 0.0, aci = 0.0, bsr = 0.0, bsi = 0.0;
    for (int k = 0; k < W; ++k) {
      const double c = tc[k], sn = ts[k];
      const double* a = ab + (size_t)k * nthp;
      acr = fma(a[0], c, acr);
      aci = fma(a[cs], c, aci);
      bsr = fma(a[2 * cs], sn, bsr);
      bsi = fma(a[3 * cs], sn, bsi);
    }
    double* Fp = F + (size_t)(K + m) * 2 * nth + j;
    double* Fn = F + (size_t)(K - m) * 2 * nth + j;
    Fp[0] = (acr + bsi) * inv;
    Fp[nth] = (aci - bsr) * inv;
    if (m > 0) {
      Fn[0] = (acr - bsi) * inv;
      Fn[nth] = (aci + bsr) * inv;
    }
  }
  __syncthreads();
  // analysis: one packed item (m, n) per thread, N_theta terms each
  {
    const int i0 = __ldg(P.ist + sp + 3), n_it = __ldg(P.ist + sp + 4) - i0;
    for (int o = threadIdx.x; o < n_it; o += blockDim.x) {
      const int v = __ldg(P.items + i0 + o), mi = v >> 8, n = v & 255;
      const int nb = tf_nb(K, sp, mi - K);
      const double* an = P.An + __ldg(P.coff + sb + mi) + n;
      const double* Fm = F + (size_t)mi * 2 * nth;
      double re = 0.0, im = 0.0;
      for (int i = 0; i < nth; ++i) {
        const double a = __ldg(an + (size_t)i * nb);
        re = fma(a, Fm[i], re);
        im = fma(a, Fm[nth + i], im);
      }
      AC[2 * o] = re;
      AC[2 * o + 1] = im;
    }
  }
  __syncthreads();
  // synthesis of G_{+m}, G_{-m} on every ring, stored as P = G_m + G_-m, M = G_m - G_-m
  for (int o = threadIdx.x; o < nth * K1; o += blockDim.x) {
    const int j = o % nth, m = o / nth;
    const int nb = tf_nb(K, sp, m);
    double pr = 0.0, pi = 0.0, nr = 0.0, ni = 0.0;
    {
      const double* sy = P.Sy + __ldg(P.coff + sb + K + m) + j;
      const double* ac = AC + 2 * __ldg(P.cidx + sb + K + m);
      for (int n = 0; n < nb; ++n) {
        const double b = __ldg(sy + (size_t)n * nth);
        pr = fma(b, ac[2 * n], pr);
        pi = fma(b, ac[2 * n + 1], pi);
      }
    }
    if (m > 0) {
      const double* sy = P.Sy + __ldg(P.coff + sb + K - m) + j;
      const double* ac = AC + 2 * __ldg(P.cidx + sb + K - m);
      for (int n = 0; n < nb; ++n) {
        const double b = __ldg(sy + (size_t)n * nth);
        nr = fma(b, ac[2 * n], nr);
        ni = fma(b, ac[2 * n + 1], ni);
      }
    }
    double* pm = PM + (size_t)m * 4 * nth + j;
    pm[0] = pr + nr;
    pm[nth] = pi + ni;
    pm[2 * nth] = pr - nr;
    pm[3 * nth] = pi - ni;
  }
  __syncthreads();
  // inverse: sum_m G_m e^{i m phi} = sum_{m>=0} P_m cos m phi + i M_m sin m phi,
  // split into even / odd m and cos / sin parts for the four slots k, k + h,
  // h - k, 2h - k
  for (int o = threadIdx.x; o < nth * W; o += blockDim.x) {
    const int k = o % W, j = o / W;
    double cer = 0.0, cei = 0.0, ser = 0.0, sei = 0.0, cor = 0.0, coi = 0.0, sor = 0.0, soi = 0.0;
    for (int m = 0; m < K1; m += 2) {
      const double c = TC[m * W + k], sn = TS[m * W + k];
      const double* pm = PM + (size_t)m * 4 * nth + j;
      cer = fma(pm[0], c, cer);
      cei = fma(pm[nth], c, cei);
      ser = fma(-pm[3 * nth], sn, ser);
      sei = fma(pm[2 * nth], sn, sei);
    }
    for (int m = 1; m < K1; m += 2) {
      const double c = TC[m * W + k], sn = TS[m * W + k];
      const double* pm = PM + (size_t)m * 4 * nth + j;
      cor = fma(pm[0], c, cor);
      coi = fma(pm[nth], c, coi);
      sor = fma(-pm[3 * nth], sn, sor);
      soi = fma(pm[2 * nth], sn, soi);
    }
    double* g = gp + 2 * j * nph;
    const double er = cer + ser, ei = cei + sei, fr = cer - ser, fi = cei - sei;   // even: C + S, C - S
    const double orr = cor + sor, oi = coi + soi, qr = cor - sor, qi = coi - soi;  // odd
    g[2 * k] = er + orr;
    g[2 * k + 1] = ei + oi;
    g[2 * (k + h)] = er - orr;
    g[2 * (k + h) + 1] = ei - oi;
    if (k > 0 && 2 * k != h) {
      g[2 * (h - k)] = fr - qr;
      g[2 * (h - k) + 1] = fi - qi;
      g[2 * (nph - k)] = fr + qr;
      g[2 * (nph - k) + 1] = fi + qi;
    }
  }
}

namespace {

// Orthonormal basis b_n(theta), n < n_b = K - l0 + 1 (l0 = max(|m|, |s|)), of
// the theta parts of the spin-s, azimuthal-m harmonics sY_lm, l0 <= l <= K:
// with x = cos(theta) they span sin(theta/2)^|s+m| cos(theta/2)^|m-s| p(x),
// deg p <= K - l0, and the p are the Jacobi polynomials P_n^(|s+m|, |m-s|)
// (their weight is the square of the prefactor).  Built by the Jacobi
// three-term recurrence and normalised under <f, g> = 2 pi sum_i w_i f_i g_i
// (Gauss-Legendre, exact for these products).  The projection sum_n b_n b_n
// does not depend on the phase convention of the harmonics.  B: [n_b][N_theta].
int spin_theta_basis(int s, int m, int K, const std::vector<double>& x, const std::vector<double>& w,
                     std::vector<long double>& B) {
  const int nth = (int)x.size();
  const int am = m < 0 ? -m : m, as = s < 0 ? -s : s;
  const int l0 = am > as ? am : as;
  B.clear();
  if (l0 > K) return 0;
  const int nb = K - l0 + 1;
  const long double a = std::abs(s + m), b = std::abs(m - s);
  const long double two_pi = 6.283185307179586476925286766559L;
  B.assign((size_t)nb * nth, 0.0L);
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
  // modified Gram-Schmidt (the basis is orthogonal already; this normalises
  // it and removes rounding)
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
  return nb;
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
  int np = 0, nr = 0, max_items = 0;
  size_t smem = 0;
  for (int s = 0; s < d->n_shells; ++s) {
    ShellDev& sh = d->shells_h[s];
    pb[s] = np;
    rb[s] = nr;
    np += sh.n_r * ((sh.na + TF_THREADS - 1) / TF_THREADS);
    sh.tf.K = sh.keep;
    if (sh.keep < 0) continue;
    nr += sh.n_r * TF_ROWS;
    const int K = sh.keep, M2 = 2 * K + 1, K1 = K + 1, nth = sh.nth, nph = sh.nph, W = nph / 4 + 1;
    smem = std::max(smem, sizeof(double) * (size_t)tf_spin_smem_doubles(nth, K, W));
    max_items = std::max(max_items, nth * K1);
    const auto key = std::make_pair(sh.L, K);
    if (!cache.count(key)) {
      TensorFilterPlan P{};
      P.K = K;
      P.W = W;
      std::vector<double> twc((size_t)K1 * W), tws((size_t)K1 * W);
      for (int m = 0; m <= K; ++m)
        for (int k = 0; k < W; ++k) {
          const double ang = 2.0 * 3.14159265358979323846 * (double)((m * k) % nph) / nph;
          twc[(size_t)m * W + k] = std::cos(ang);
          tws[(size_t)m * W + k] = std::sin(ang);
        }
      std::vector<double> An, Sy;
      std::vector<int> coff(7 * M2), cidx(7 * M2), ist(8), items;
      std::vector<long double> B;
      const long double two_pi = 6.283185307179586476925286766559L;
      for (int sp = -3; sp <= 3; ++sp) {
        ist[sp + 3] = (int)items.size();
        int c = 0;
        for (int m = -K; m <= K; ++m) {
          const int nb = spin_theta_basis(sp, m, K, gl_x[s], gl_w[s], B);
          coff[(sp + 3) * M2 + m + K] = (int)An.size();
          cidx[(sp + 3) * M2 + m + K] = c;
          for (int i = 0; i < nth; ++i)
            for (int n = 0; n < nb; ++n) An.push_back((double)(two_pi * gl_w[s][i] * B[(size_t)n * nth + i]));
          for (int n = 0; n < nb; ++n)
            for (int j = 0; j < nth; ++j) Sy.push_back((double)B[(size_t)n * nth + j]);
          for (int n = 0; n < nb; ++n) items.push_back(((m + K) << 8) | n);
          c += nb;
        }
      }
      ist[7] = (int)items.size();
      std::vector<int> ints(coff);
      ints.insert(ints.end(), cidx.begin(), cidx.end());
      ints.insert(ints.end(), ist.begin(), ist.end());
      ints.insert(ints.end(), items.begin(), items.end());
      double* p = nullptr;
      int* q = nullptr;
      if ((e = tf_upload(d, twc, &p)) != cudaSuccess) return e;
      P.twc = p;
      if ((e = tf_upload(d, tws, &p)) != cudaSuccess) return e;
      P.tws = p;
      if ((e = tf_upload(d, An, &p)) != cudaSuccess) return e;
      P.An = p;
      if ((e = tf_upload(d, Sy, &p)) != cudaSuccess) return e;
      P.Sy = p;
      if ((e = tf_upload(d, ints, &q)) != cudaSuccess) return e;
      P.coff = q;
      P.cidx = q + 7 * M2;
      P.ist = q + 14 * M2;
      P.items = q + 14 * M2 + 8;
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
  d->tf_spin_threads = max_items >= 4 * TF_SPIN_MAX_THREADS ? TF_SPIN_MAX_THREADS : TF_SPIN_MAX_THREADS / 2;
  if ((e = raise_smem_limit((const void*)tf_spin_kernel, smem)) != cudaSuccess) return e;
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
    tf_spin_kernel<<<d->tf_rows, d->tf_spin_threads, d->tf_smem, d->stream>>>(d->shells_d, n, d->tf_pb_d + n + 1,
                                                                             d->tf_buf);
    d->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  tf_unframe_kernel<<<d->tf_point_blocks, TF_THREADS, 0, d->stream>>>(d->shells_d, n, d->tf_pb_d, d->tf_buf, out);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_tensor_filter_transpose(gh_domain* d, const double* in, double* out) {
  cudaError_t e;
  if (!d->tf_buf) return cudaErrorNotReady;
  const int n = d->n_shells;
  tf_unframe_t_kernel<<<d->tf_point_blocks, TF_THREADS, 0, d->stream>>>(d->shells_d, n, d->tf_pb_d, in, d->tf_buf);
  d->launches++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (d->tf_rows > 0) {
    tf_spin_kernel<<<d->tf_rows, d->tf_spin_threads, d->tf_smem, d->stream>>>(d->shells_d, n, d->tf_pb_d + n + 1,
                                                                             d->tf_buf);
    d->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  tf_frame_t_kernel<<<d->tf_point_blocks, TF_THREADS, 0, d->stream>>>(d->shells_d, n, d->tf_pb_d, d->tf_buf, out);
  d->launches++;
  return cudaGetLastError();
}

}  // namespace gh
