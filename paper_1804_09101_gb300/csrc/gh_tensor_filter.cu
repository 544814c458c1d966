// Tensor spherical-harmonic truncation filter on S2 shells (the tensor-coupled
// S2 filter of Secs. 3.1 and 3.4).  Every Cartesian index of the GH tensors
// is expressed in the local complex frame E_0 = r_hat, E_1 = m = (theta_hat +
// i phi_hat)/sqrt(2), E_2 = conj(m); a frame component c_A = T_I E_A1^I1 ..
// has spin weight s = #m - #conj(m) and is projected onto the spin-weighted
// harmonics sY_lm, |s| <= l <= K; the filtered tensor is
// Re sum_A c'_A conj(E_A1) x .. (conj(E) is the dual basis).  Three kernels:
//   tf_frame_kernel   per point: the 65 complex components of the 9 tensor
//                     groups (psi_00, psi_0i, psi_ij, the same for Pi, Phi_i00,
//                     Phi_i0j, Phi_ijk), one index contracted at a time;
//   tf_spin_kernel    per (r, component) row: complex phi DFT (m = -K..K), the
//                     real N_theta x N_theta map of (s, m), inverse DFT;
//   tf_unframe_kernel per point: back to the Cartesian components.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "gh_geom.cuh"
#include "gh_internal.h"
#include "gh_tensor.cuh"

namespace gh {

// 9 tensor groups: rank, first component slot, field of each Cartesian index tuple
__constant__ int c_tf_rank[9] = {0, 1, 2, 0, 1, 2, 1, 2, 3};
__constant__ int c_tf_slot[9] = {0, 1, 4, 13, 14, 17, 26, 29, 38};
__constant__ int c_tf_field[9][27];
__constant__ unsigned char c_tf_write[9][27];  // 1 for the stored (canonical) index tuple

constexpr int TF_THREADS = 128;

struct Cx {
  double re, im;
};
__device__ __forceinline__ Cx cmul(Cx a, Cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

__device__ __forceinline__ void frame_vectors(const ShellDev& sh, int q, Cx E[3][3]) {
  const int j = q / sh.nph, k = q - j * sh.nph;
  const double st = sh.sth[j], ct = sh.cth[j], sp = sh.sph[k], cp = sh.cph[k];
  const double rh[3] = {st * cp, st * sp, ct};
  const double th[3] = {ct * cp, ct * sp, -st};
  const double ph[3] = {-sp, cp, 0.0};
  const double h = 0.70710678118654752440;
  for (int i = 0; i < 3; ++i) {
    E[0][i] = {rh[i], 0.0};
    E[1][i] = {h * th[i], h * ph[i]};
    E[2][i] = {h * th[i], -h * ph[i]};
  }
}

// Contract every index of a rank-n tensor (3^n values, row-major, first index
// slowest) with the frame.  Forward (inverse = false): Cartesian -> frame,
// c_..A.. = sum_i E_A^i T_..i..; inverse: frame -> Cartesian with the dual
// basis, T_..i.. = sum_A conj(E_A^i) c_..A...
__device__ __forceinline__ void contract(int rank, Cx* t, Cx* w, const Cx E[3][3], bool inverse) {
  int n = 1;
  for (int k = 0; k < rank; ++k) n *= 3;
  for (int k = 0; k < rank; ++k) {
    // contract index k: output index Ak of w from summed index i of t
    int stride = 1;
    for (int q = k + 1; q < rank; ++q) stride *= 3;
    for (int o = 0; o < n; ++o) {
      const int Ak = (o / stride) % 3;
      const int base = o - Ak * stride;
      Cx acc = {0.0, 0.0};
      for (int i = 0; i < 3; ++i) {
        Cx e = inverse ? E[i][Ak] : E[Ak][i];
        if (inverse) e.im = -e.im;
        const Cx v = t[base + i * stride];
        acc.re += e.re * v.re - e.im * v.im;
        acc.im += e.re * v.im + e.im * v.re;
      }
      w[o] = acc;
    }
    for (int o = 0; o < n; ++o) t[o] = w[o];
  }
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
  const long long ubase = sh.off + (long long)ir * NF * na + q;
  const long long cbase = 2LL * TF_SLOTS * (sh.pt_off + (long long)ir * na);
  for (int g = 0; g < 9; ++g) {
    const int rank = c_tf_rank[g];
    const int n = rank == 0 ? 1 : (rank == 1 ? 3 : (rank == 2 ? 9 : 27));
    Cx t[27], w[27];
    for (int o = 0; o < n; ++o) t[o] = {u[ubase + (long long)c_tf_field[g][o] * na], 0.0};
    contract(rank, t, w, E, false);
    for (int o = 0; o < n; ++o) {
      const long long c = cbase + 2LL * ((long long)(c_tf_slot[g] + o) * na + q);
      cb[c] = t[o].re;
      cb[c + 1] = t[o].im;
    }
  }
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
  const long long ubase = sh.off + (long long)ir * NF * na + q;
  const long long cbase = 2LL * TF_SLOTS * (sh.pt_off + (long long)ir * na);
  for (int g = 0; g < 9; ++g) {
    const int rank = c_tf_rank[g];
    const int n = rank == 0 ? 1 : (rank == 1 ? 3 : (rank == 2 ? 9 : 27));
    Cx t[27], w[27];
    for (int o = 0; o < n; ++o) {
      const long long c = cbase + 2LL * ((long long)(c_tf_slot[g] + o) * na + q);
      t[o] = {cb[c], cb[c + 1]};
    }
    contract(rank, t, w, E, true);
    for (int o = 0; o < n; ++o)
      if (c_tf_write[g][o]) out[ubase + (long long)c_tf_field[g][o] * na] = t[o].re;
  }
}

// spin of component o of group g: #m - #conj(m) over its frame indices
__device__ __forceinline__ int slot_spin(int rank, int o) {
  int sp = 0;
  for (int k = 0; k < rank; ++k) {
    const int a = o % 3;
    o /= 3;
    sp += (a == 1) ? 1 : (a == 2 ? -1 : 0);
  }
  return sp;
}

__global__ void __launch_bounds__(TF_THREADS)
tf_spin_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
               double* __restrict__ cb) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const TensorFilterPlan& P = sh.tf;
  const int na = sh.na, nth = sh.nth, nph = sh.nph, K = P.K, M2 = 2 * K + 1;
  const int row = blockIdx.x - begin[s];          // (ir, slot)
  const int slot = row % TF_SLOTS;
  const int ir = row / TF_SLOTS;
  int g = 0;
  while (g + 1 < 9 && c_tf_slot[g + 1] <= slot) ++g;
  const int sp = slot_spin(c_tf_rank[g], slot - c_tf_slot[g]);
  double* f = sm;                                 // [na][2]
  double* F = f + 2 * na;                         // [nth][M2][2]
  double* G = F + 2 * nth * M2;                   // [nth][M2][2]
  double* row_ptr = cb + 2LL * TF_SLOTS * (sh.pt_off + (long long)ir * na) + 2LL * slot * na;
  for (int i = threadIdx.x; i < 2 * na; i += blockDim.x) f[i] = row_ptr[i];
  __syncthreads();
  const double inv = 1.0 / nph;
  for (int o = threadIdx.x; o < nth * M2; o += blockDim.x) {
    const int mi = o % M2, j = o / M2, m = mi - K, am = m < 0 ? -m : m;
    const double sg = m < 0 ? -1.0 : 1.0;
    const double* c = P.tc + (size_t)am * nph;
    const double* sn = P.ts + (size_t)am * nph;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < nph; ++k) {
      // f e^{-i m phi}: (a + i b)(cos - i sg sin)
      const double a = f[2 * (j * nph + k)], b = f[2 * (j * nph + k) + 1];
      const double cs = __ldg(c + k), ss = sg * __ldg(sn + k);
      re = fma(a, cs, fma(b, ss, re));
      im = fma(b, cs, fma(-a, ss, im));
    }
    F[2 * o] = re * inv;
    F[2 * o + 1] = im * inv;
  }
  __syncthreads();
  const double* Qs = P.Q + (size_t)(sp + 3) * M2 * nth * nth;
  for (int o = threadIdx.x; o < nth * M2; o += blockDim.x) {
    const int mi = o % M2, j = o / M2;
    const double* Qm = Qs + ((size_t)mi * nth + j) * nth;
    double re = 0.0, im = 0.0;
    for (int i = 0; i < nth; ++i) {
      const double qv = __ldg(Qm + i);
      re = fma(qv, F[2 * (i * M2 + mi)], re);
      im = fma(qv, F[2 * (i * M2 + mi) + 1], im);
    }
    G[2 * o] = re;
    G[2 * o + 1] = im;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < na; o += blockDim.x) {
    const int k = o % nph, j = o / nph;
    double re = 0.0, im = 0.0;
    for (int mi = 0; mi < M2; ++mi) {
      const int m = mi - K, am = m < 0 ? -m : m;
      const double cs = __ldg(P.tc + (size_t)am * nph + k), ss = (m < 0 ? -1.0 : 1.0) * __ldg(P.ts + (size_t)am * nph + k);
      const double a = G[2 * (j * M2 + mi)], b = G[2 * (j * M2 + mi) + 1];
      re = fma(a, cs, fma(-b, ss, re));
      im = fma(b, cs, fma(a, ss, im));
    }
    row_ptr[2 * o] = re;
    row_ptr[2 * o + 1] = im;
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
  // index tuple -> field, and which tuples are the stored ones
  int map[9][27];
  unsigned char wr[9][27];
  std::memset(map, 0, sizeof(map));
  std::memset(wr, 0, sizeof(wr));
  for (int base = 0, g0 = 0; base <= 10; base += 10, g0 += 3) {
    map[g0][0] = base + sym_index(0, 0);
    wr[g0][0] = 1;
    for (int i = 0; i < 3; ++i) {
      map[g0 + 1][i] = base + sym_index(0, 1 + i);
      wr[g0 + 1][i] = 1;
      for (int j = 0; j < 3; ++j) {
        map[g0 + 2][3 * i + j] = base + sym_index(1 + i, 1 + j);
        wr[g0 + 2][3 * i + j] = i <= j;
      }
    }
  }
  for (int i = 0; i < 3; ++i) {
    map[6][i] = 20 + 10 * i + sym_index(0, 0);
    wr[6][i] = 1;
    for (int j = 0; j < 3; ++j) {
      map[7][3 * i + j] = 20 + 10 * i + sym_index(0, 1 + j);
      wr[7][3 * i + j] = 1;
      for (int k = 0; k < 3; ++k) {
        map[8][9 * i + 3 * j + k] = 20 + 10 * i + sym_index(1 + j, 1 + k);
        wr[8][9 * i + 3 * j + k] = j <= k;
      }
    }
  }
  if ((e = cudaMemcpyToSymbol(c_tf_field, map, sizeof(map))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(c_tf_write, wr, sizeof(wr))) != cudaSuccess) return e;
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
    nr += sh.n_r * TF_SLOTS;
    const int K = sh.keep, M2 = 2 * K + 1, nth = sh.nth, nph = sh.nph;
    smem = std::max(smem, sizeof(double) * (size_t)(2 * sh.na + 4 * nth * M2));
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
  if ((e = cudaMalloc(&p, sizeof(double) * 2 * TF_SLOTS * (size_t)d->points)) != cudaSuccess) return e;
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
