// libgh host side: grids, the cached operator matrices (the paper's matrix
// dictionary, Sec. 3.4), domain setup and the C ABI entry points of gh.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "gh_internal.h"

namespace {

thread_local std::string g_create_error;
constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------ grids
// Chebyshev-Gauss-Lobatto points x_j = -cos(pi j / N), ascending.
std::vector<double> cgl_points(int n) {
  std::vector<double> x(n);
  const int N = n - 1;
  for (int j = 0; j < n; ++j) x[j] = -std::cos(kPi * j / N);
  x[0] = -1.0;
  x[N] = 1.0;
  return x;
}

// Clenshaw-Curtis weights on the CGL points (symmetric, so the ascending
// order needs no change).
std::vector<double> clenshaw_curtis(int n) {
  const int N = n - 1;
  std::vector<double> w(n);
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int k = 1; 2 * k <= N; ++k) {
      const double b = (2 * k == N) ? 1.0 : 2.0;
      s += b * std::cos(2.0 * kPi * j * k / N) / (4.0 * k * k - 1.0);
    }
    const double c = (j == 0 || j == N) ? 1.0 : 2.0;
    w[j] = c / N * (1.0 - s);
  }
  return w;
}

// Gauss-Legendre nodes (descending in x, i.e. theta ascending) and weights,
// by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  // make the node set exactly symmetric about the equator (the folded angular
  // maps rely on x_{n-1-i} = -x_i and w_{n-1-i} = w_i)
  for (int i = 0; i < n / 2; ++i) {
    x[n - 1 - i] = -x[i];
    w[n - 1 - i] = w[i];
  }
  if (n % 2) x[n / 2] = 0.0;
}

// Normalised associated Legendre functions Pbar_l^m(theta_j) and their theta
// derivatives, tables [l][m][j] of (L+1)^2 x nth.
void legendre_tables(int L, const std::vector<double>& ct, const std::vector<double>& st,
                     std::vector<double>& P, std::vector<double>& dP) {
  const int nth = (int)ct.size();
  const int W = L + 1;
  P.assign((size_t)W * W * nth, 0.0);
  dP.assign((size_t)W * W * nth, 0.0);
  auto at = [&](std::vector<double>& T, int l, int m, int j) -> double& {
    return T[((size_t)l * W + m) * nth + j];
  };
  for (int j = 0; j < nth; ++j) {
    at(P, 0, 0, j) = std::sqrt(0.25 / kPi);
    for (int m = 1; m <= L; ++m)
      at(P, m, m, j) = std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * st[j] * at(P, m - 1, m - 1, j);
    for (int m = 0; m < L; ++m) at(P, m + 1, m, j) = std::sqrt(2.0 * m + 3.0) * ct[j] * at(P, m, m, j);
    for (int m = 0; m <= L; ++m)
      for (int l = m + 2; l <= L; ++l) {
        const double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
        const double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
        at(P, l, m, j) = a * (ct[j] * at(P, l - 1, m, j) - b * at(P, l - 2, m, j));
      }
    // sin(th) dP_l^m/dth = l cos(th) P_l^m - sqrt((2l+1)(l^2-m^2)/(2l-1)) P_{l-1}^m
    for (int l = 0; l <= L; ++l)
      for (int m = 0; m <= l; ++m) {
        const double prev = (l > m) ? at(P, l - 1, m, j) : 0.0;
        const double c = (l > m) ? std::sqrt((2.0 * l + 1.0) * ((double)l * l - (double)m * m) / (2.0 * l - 1.0)) : 0.0;
        at(dP, l, m, j) = (l * ct[j] * at(P, l, m, j) - c * prev) / st[j];
      }
  }
}

// ------------------------------------------------------------ matrices
// d/dx on the CGL points, closed form with the negative-sum diagonal.
std::vector<double> cgl_derivative_matrix(int n) {
  const int N = n - 1;
  std::vector<double> D((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double rowsum = 0.0;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      const double ci = (i == 0 || i == N) ? 2.0 : 1.0;
      const double cj = (j == 0 || j == N) ? 2.0 : 1.0;
      // x_i - x_j = 2 sin(pi (i+j) / 2N) sin(pi (i-j) / 2N)
      const double dx = 2.0 * std::sin(kPi * (i + j) / (2.0 * N)) * std::sin(kPi * (i - j) / (2.0 * N));
      const double v = (ci / cj) * (((i + j) % 2) ? -1.0 : 1.0) / dx;
      D[(size_t)i * n + j] = v;
      rowsum += v;
    }
    D[(size_t)i * n + i] = -rowsum;
  }
  return D;
}

// Exponential Chebyshev filter C^-1 diag(sigma) C on the CGL points.
std::vector<double> cgl_filter_matrix(int n, double alpha, int order) {
  const int N = n - 1;
  std::vector<double> F((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double cj = (j == 0 || j == N) ? 2.0 : 1.0;
      double acc = 0.0;
      for (int k = 0; k <= N; ++k) {
        const double ck = (k == 0 || k == N) ? 2.0 : 1.0;
        const double sigma = std::exp(-alpha * std::pow((double)k / N, order));
        const double Ti = std::cos(kPi * k * (N - i) / N);
        const double Tj = std::cos(kPi * k * (N - j) / N);
        acc += Ti * sigma * 2.0 / (N * ck * cj) * Tj;
      }
      F[(size_t)i * n + j] = acc;
    }
  return F;
}

// Folded rows of a centro-symmetric (sigma = +1) or centro-antisymmetric
// (sigma = -1) n x n matrix for radial_kernel: rows i < ceil(n/2), each
// [A_i0 .. A_i,h-1, (M_im for odd n), B_i,h-1 .. B_i0] with
// A_ij = (M_ij + M_i,n-1-j)/2, B_ij = (M_ij - M_i,n-1-j)/2, h = n/2.
std::vector<double> fold_radial_matrix(const std::vector<double>& M, int n) {
  const int h = n / 2, ne = n - h;
  std::vector<double> F((size_t)ne * n, 0.0);
  for (int i = 0; i < ne; ++i) {
    for (int j = 0; j < h; ++j) {
      const double a = M[(size_t)i * n + j], b = M[(size_t)i * n + (n - 1 - j)];
      F[(size_t)i * n + j] = 0.5 * (a + b);
      F[(size_t)i * n + (n - 1 - j)] = 0.5 * (a - b);
    }
    if (n % 2) F[(size_t)i * n + h] = M[(size_t)i * n + h];
  }
  return F;
}

struct AngularGrid {
  int L, nth, nph, na;
  std::vector<double> ct, st, wgl;
};

AngularGrid angular_grid(int L) {
  AngularGrid g;
  g.L = L;
  g.nth = L + 1;
  g.nph = 2 * (L + 1);
  g.na = g.nth * g.nph;
  gauss_legendre(g.nth, g.ct, g.wgl);
  g.st.resize(g.nth);
  for (int j = 0; j < g.nth; ++j) g.st[j] = std::sqrt((1.0 - g.ct[j]) * (1.0 + g.ct[j]));
  return g;
}

// Transposed angular maps B[q][p] = M[p][q] for
//   kind 0: d/dtheta of the projection onto Y_lm, l <= L
//   kind 1: d/dphi   of the projection onto Y_lm, l <= L
//   kind 2: projection onto Y_lm with l <= keep (Heaviside filter in l)
// using M[(j,k)][(j',k')] = W_j' sum_m c_m phi_m(k-k') sum_l A_lm(j) P_lm(j'),
// c_0 = 1, c_m = 2, phi_m = cos(m dphi) or -m sin(m dphi).
std::vector<double> angular_matrix(const AngularGrid& g, int kind, int keep) {
  std::vector<double> P, dP;
  legendre_tables(g.L, g.ct, g.st, P, dP);
  const int W = g.L + 1, nth = g.nth, nph = g.nph, na = g.na;
  const int lmax = (kind == 2) ? keep : g.L;
  // Q[m][j][j'] = sum_{l=m}^{lmax} A_lm(j) P_lm(j')
  std::vector<double> Q((size_t)W * nth * nth, 0.0);
  for (int m = 0; m <= lmax; ++m)
    for (int j = 0; j < nth; ++j)
      for (int jp = 0; jp < nth; ++jp) {
        double acc = 0.0;
        for (int l = m; l <= lmax; ++l) {
          const double a = (kind == 0) ? dP[((size_t)l * W + m) * nth + j] : P[((size_t)l * W + m) * nth + j];
          acc += a * P[((size_t)l * W + m) * nth + jp];
        }
        Q[((size_t)m * nth + j) * nth + jp] = acc;
      }
  // phi factor table F[m][dk]
  std::vector<double> F((size_t)W * nph);
  for (int m = 0; m <= lmax; ++m)
    for (int dk = 0; dk < nph; ++dk) {
      const double ang = 2.0 * kPi * m * dk / nph;
      const double c = (m == 0) ? 1.0 : 2.0;
      F[(size_t)m * nph + dk] = (kind == 1) ? -c * m * std::sin(ang) : c * std::cos(ang);
    }
  const double wphi = 2.0 * kPi / nph;
  std::vector<double> B((size_t)na * na);
  for (int j = 0; j < nth; ++j)
    for (int k = 0; k < nph; ++k) {
      const int p = j * nph + k;
      for (int jp = 0; jp < nth; ++jp)
        for (int kp = 0; kp < nph; ++kp) {
          const int q = jp * nph + kp;
          const int dk = ((k - kp) % nph + nph) % nph;
          double acc = 0.0;
          for (int m = 0; m <= lmax; ++m)
            acc += F[(size_t)m * nph + dk] * Q[((size_t)m * nth + j) * nth + jp];
          B[(size_t)q * na + p] = acc * g.wgl[jp] * wphi;
        }
    }
  return B;
}

// Separable plan (see sep_angular_kernel): modes cos m = 0..K then sin m = 1..K.
//   F[k][mode]          forward DFT
//   G0[mode][k]         c_m (2 pi / N_phi) x (cos m phi_k | sin m phi_k)
//   G1[mode][k]         the phi derivative of G0 (derivative plan only)
//   Q0[m][j_in][j_out]  sum_{l=m..K} A_lm(j_out) Pbar_lm(j_in) w_GL(j_in),
//                       A = dPbar/dtheta (derivative plan) or Pbar (filter)
//   Q1[m][j_in][j_out]  the same with A = Pbar (derivative plan only)
struct SepHost {
  int K, M;
  std::vector<double> F, G0, G1, Q0, Q1;
  std::vector<double> F0T, F1T, Q0T, Q1T, GT;   // transposed map (adjoint)
};

void sep_transpose(SepHost& h, int nth, int nph, bool deriv) {
  const int M = h.M, K = h.K;
  h.F0T.assign((size_t)nph * M, 0.0);
  h.GT.assign((size_t)M * nph, 0.0);
  if (deriv) h.F1T.assign((size_t)nph * M, 0.0);
  for (int mode = 0; mode < M; ++mode)
    for (int k = 0; k < nph; ++k) {
      h.F0T[(size_t)k * M + mode] = h.G0[(size_t)mode * nph + k];
      if (deriv) h.F1T[(size_t)k * M + mode] = h.G1[(size_t)mode * nph + k];
      h.GT[(size_t)mode * nph + k] = h.F[(size_t)k * M + mode];
    }
  h.Q0T.assign((size_t)(K + 1) * nth * nth, 0.0);
  if (deriv) h.Q1T.assign((size_t)(K + 1) * nth * nth, 0.0);
  for (int m = 0; m <= K; ++m)
    for (int a = 0; a < nth; ++a)
      for (int b = 0; b < nth; ++b) {
        h.Q0T[((size_t)m * nth + a) * nth + b] = h.Q0[((size_t)m * nth + b) * nth + a];
        if (deriv) h.Q1T[((size_t)m * nth + a) * nth + b] = h.Q1[((size_t)m * nth + b) * nth + a];
      }
}

SepHost sep_plan(const AngularGrid& g, int K, bool deriv) {
  SepHost h;
  h.K = K;
  h.M = 2 * K + 1;
  const int M = h.M, nph = g.nph, nth = g.nth, W = g.L + 1;
  std::vector<double> P, dP;
  legendre_tables(g.L, g.ct, g.st, P, dP);
  h.F.assign((size_t)nph * M, 0.0);
  h.G0.assign((size_t)M * nph, 0.0);
  if (deriv) h.G1.assign((size_t)M * nph, 0.0);
  const double wphi = 2.0 * kPi / nph;
  for (int mode = 0; mode < M; ++mode) {
    const bool cosm = mode <= K;
    const int m = cosm ? mode : mode - K;
    const double c = (m == 0) ? 1.0 : 2.0;
    for (int k = 0; k < nph; ++k) {
      const double ang = 2.0 * kPi * (double)m * k / nph;
      const double cs = std::cos(ang), sn = std::sin(ang);
      h.F[(size_t)k * M + mode] = cosm ? cs : sn;
      h.G0[(size_t)mode * nph + k] = c * wphi * (cosm ? cs : sn);
      if (deriv) h.G1[(size_t)mode * nph + k] = c * wphi * m * (cosm ? -sn : cs);
    }
  }
  h.Q0.assign((size_t)(K + 1) * nth * nth, 0.0);
  if (deriv) h.Q1.assign((size_t)(K + 1) * nth * nth, 0.0);
  for (int m = 0; m <= K; ++m)
    for (int ji = 0; ji < nth; ++ji)
      for (int jo = 0; jo < nth; ++jo) {
        double a0 = 0.0, a1 = 0.0;
        for (int l = m; l <= K; ++l) {
          const double pin = P[((size_t)l * W + m) * nth + ji];
          const double po = P[((size_t)l * W + m) * nth + jo];
          const double dpo = dP[((size_t)l * W + m) * nth + jo];
          a0 += (deriv ? dpo : po) * pin;
          a1 += po * pin;
        }
        h.Q0[((size_t)m * nth + ji) * nth + jo] = a0 * g.wgl[ji];
        if (deriv) h.Q1[((size_t)m * nth + ji) * nth + jo] = a1 * g.wgl[ji];
      }
  sep_transpose(h, nth, nph, deriv);
  return h;
}

// Rows per block of the transposed separable kernel: inputs (2 or 1 rows of
// Na), their analyses (2 or 1 of nth x M) and one Legendre output.
int sep_adj_rows_per_block(int na, int nth, int M, bool two, int n_rows) {
  const size_t per_row = (two ? 2 : 1) * (size_t)na + (two ? 3 : 2) * (size_t)nth * M;
  const size_t budget = 64 * 1024 / sizeof(double);
  int rb = (int)(budget / per_row);
  if (rb < 1) rb = 1;
  if (rb > 64) rb = 64;
  if (rb > n_rows) rb = n_rows;
  return rb;
}

// Rows of one shell that a separable block holds in shared memory.
int sep_rows_per_block(int na, int nth, int M, bool two, int n_rows) {
  const size_t per_row = (size_t)na + (two ? 3 : 2) * (size_t)nth * M;
  const size_t budget = 64 * 1024 / sizeof(double);
  int rb = (int)(budget / per_row);
  if (rb < 1) rb = 1;
  if (rb > 64) rb = 64;
  if (rb > n_rows) rb = n_rows;
  return rb;
}

// Folded plan (see fold_angular_kernel).  A mode's Legendre map is factorised
// when (1 + n_out)(K + 1 - m) is below GH_FOLD_RANK_PERCENT % of the fused
// 2 n_out hs^2 / hs (the FMA count per output ring; the factorised form adds a
// shared-memory pass and a barrier, so the break-even is below 100 %).
#ifndef GH_FOLD_RANK_PERCENT
#define GH_FOLD_RANK_PERCENT 75
#endif
struct FoldHost {
  int K, M, N4, half, W, hs, qself;
  std::vector<double> Tc, Ts, Q0s, Q0t, Q1s, Q1t;
  double s0, s1;
  int m0;                               // first mode taken as analysis then synthesis
  std::vector<int> coef_off, slot_m;    // [K + 2], [coef_off[K + 1]]
  std::vector<double> A, Y0, Y1;        // [slots][hs]
};

// The phi grid has N_phi = 2(L+1) points (always even) and the Gauss-Legendre
// theta nodes are symmetric, so every shell can be folded.
bool fold_applicable(const AngularGrid& g) { return g.nph % 2 == 0; }

FoldHost fold_plan(const AngularGrid& g, int K, bool deriv) {
  FoldHost h;
  h.K = K;
  h.M = 2 * K + 1;
  h.N4 = g.nph / 4;
  h.qself = (g.nph % 4 == 0) ? 1 : 0;
  h.W = h.qself ? h.N4 + 1 : (g.nph + 2) / 4;
  h.half = g.nth / 2;
  h.hs = (g.nth + 1) / 2;
  const int W = h.W, nth = g.nth, half = h.half, hs = h.hs, Wl = g.L + 1;
  h.Tc.assign((size_t)(K + 1) * W, 0.0);
  h.Ts.assign((size_t)(K + 1) * W, 0.0);
  for (int m = 0; m <= K; ++m)
    for (int k = 0; k < W; ++k) {
      const double ang = 2.0 * kPi * (double)m * k / g.nph;
      h.Tc[(size_t)m * W + k] = std::cos(ang);
      h.Ts[(size_t)m * W + k] = std::sin(ang);
    }
  std::vector<double> P, dP;
  legendre_tables(g.L, g.ct, g.st, P, dP);
  // synthesis factor of mode m: c_m for the first output, m c_m for the value
  // map that feeds d/dphi
  auto cfac = [&](int m) { return (m == 0 ? 1.0 : 2.0) * 2.0 * kPi / g.nph; };
  auto build = [&](bool dtheta, bool mscale, std::vector<double>& Qs, std::vector<double>& Qt) {
    Qs.assign((size_t)(K + 1) * hs * hs, 0.0);
    Qt.assign((size_t)(K + 1) * hs * hs, 0.0);
    std::vector<double> Q((size_t)nth * nth);
    for (int m = 0; m <= K; ++m) {
      for (int jo = 0; jo < nth; ++jo)
        for (int ji = 0; ji < nth; ++ji) {
          double acc = 0.0;
          for (int l = m; l <= K; ++l) {
            const double a = dtheta ? dP[((size_t)l * Wl + m) * nth + jo] : P[((size_t)l * Wl + m) * nth + jo];
            acc += a * P[((size_t)l * Wl + m) * nth + ji];
          }
          Q[(size_t)jo * nth + ji] = acc * g.wgl[ji];
        }
      const double f = (mscale ? (double)m : 1.0) * cfac(m);
      // inputs: s_ji = in_ji + in_{nth-1-ji}, t_ji = in_ji - in_{nth-1-ji} (ji < half);
      // an odd N_theta's equator ring is s_eq = in_eq, t_eq = 0.  Outputs jo < hs
      // (jo = half: the equator).
      for (int ji = 0; ji < hs; ++ji)
        for (int jo = 0; jo < hs; ++jo) {
          double qs, qt;
          if (ji < half) {
            const double q1 = Q[(size_t)jo * nth + ji], q2 = Q[(size_t)jo * nth + (nth - 1 - ji)];
            qs = 0.5 * (q1 + q2);
            qt = 0.5 * (q1 - q2);
          } else {
            qs = Q[(size_t)jo * nth + ji];
            qt = 0.0;
          }
          Qs[((size_t)m * hs + ji) * hs + jo] = f * qs;
          Qt[((size_t)m * hs + ji) * hs + jo] = f * qt;
        }
    }
  };
  build(deriv, false, h.Q0s, h.Q0t);
  if (deriv) build(false, true, h.Q1s, h.Q1t);
  h.s0 = deriv ? -1.0 : 1.0;
  h.s1 = 1.0;
  // Factorised Legendre maps.  The half-size map of mode m has rank K + 1 - m
  // (the degrees l = m .. K, split by the parity of l + m between the s and t
  // parts): projecting onto a_l = sum_j Pbar_lm(theta_j) w_j (s or t)_j and
  // synthesising sum_l Y_o(l, j) a_l costs (1 + n_out)(K + 1 - m) hs FMAs per
  // mode instead of the fused 2 n_out hs^2, so it is taken where cheaper.
  const int n_out = deriv ? 2 : 1;
  h.m0 = K + 1;
  for (int m = 0; m <= K; ++m)
    if ((1 + n_out) * (K + 1 - m) * 100 < GH_FOLD_RANK_PERCENT * 2 * n_out * hs) {
      h.m0 = m;
      break;
    }
  h.coef_off.assign((size_t)K + 2, 0);
  for (int m = 0; m <= K; ++m) h.coef_off[m + 1] = h.coef_off[m] + (m >= h.m0 ? K + 1 - m : 0);
  const int ns = h.coef_off[K + 1];
  h.slot_m.assign((size_t)std::max(ns, 1), 0);
  h.A.assign((size_t)std::max(ns, 1) * hs, 0.0);
  h.Y0.assign((size_t)std::max(ns, 1) * hs, 0.0);
  h.Y1.assign((size_t)std::max(ns, 1) * hs, 0.0);
  for (int m = h.m0; m <= K; ++m)
    for (int l = m; l <= K; ++l) {
      const int slot = h.coef_off[m] + (l - m);
      h.slot_m[slot] = m;
      const size_t pl = ((size_t)l * Wl + m) * nth;
      for (int j = 0; j < hs; ++j) {
        h.A[(size_t)slot * hs + j] = P[pl + j] * g.wgl[j];
        h.Y0[(size_t)slot * hs + j] = cfac(m) * (deriv ? dP[pl + j] : P[pl + j]);
        h.Y1[(size_t)slot * hs + j] = deriv ? (double)m * cfac(m) * P[pl + j] : 0.0;
      }
    }
  return h;
}

// Rings whose phi transforms run as a register FFT in fold_angular_kernel:
// N_phi = 16, 32 or 64 (log2 of the complex size N_phi / 2), else 0.
#ifndef GH_FOLD_FFT_MAX_NPHI
#define GH_FOLD_FFT_MAX_NPHI 64
#endif
int fold_fft_log(const AngularGrid& g) {
  // the ring-FFT kernels take whole rows per warp of 32 rings and pair ring j
  // with its mirror on adjacent lanes: N_theta must divide 32 (and be even)
  if (g.nph > GH_FOLD_FFT_MAX_NPHI || g.nth % 2 != 0 || 32 % g.nth != 0) return 0;
  if (g.nph == 16) return 3;
  if (g.nph == 32) return 4;
  if (g.nph == 64) return 5;
  return 0;
}

// Shared memory (doubles) per row of the fused folded kernel: ring values and
// their quarter folds (reused for the synthesis coefficients) plus the Fourier
// coefficients of the half-rings; of fold_legendre_kernel (legendre_only): the
// half-ring coefficients, the factorised modes' a_l and the synthesis
// coefficients.
size_t fold_row_doubles(int na, int nth, int W, int M, int n_out, int ncoef, bool legendre_only) {
  const size_t ab = (size_t)M * 2 * (size_t)((nth + 1) / 2);
  if (legendre_only) return ab + 2 * (size_t)ncoef + (size_t)n_out * nth * M;
  return std::max((size_t)na + 4 * (size_t)nth * W, (size_t)n_out * nth * M) + ab + 2 * (size_t)ncoef;
}

int fold_rows_per_block(int na, int nth, int W, int M, int n_out, int ncoef, bool legendre_only, int n_rows,
                        int budget_bytes) {
  int rb = (int)((size_t)budget_bytes /
                 (sizeof(double) * fold_row_doubles(na, nth, W, M, n_out, ncoef, legendre_only)));
  if (rb < 1) rb = 1;
  if (rb > 64) rb = 64;
  if (rb > n_rows) rb = n_rows;
  return rb;
}

// ------------------------------------------------------------ helpers
gh_status fail(gh_domain* d, gh_status s, const std::string& msg) {
  if (d) d->err = msg;
  else g_create_error = msg;
  return s;
}

#define GH_CUDA(d, call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail((d), e_ == cudaErrorMemoryAllocation ? GH_ENOMEM : GH_ECUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

template <typename T>
cudaError_t upload(gh_domain* d, const std::vector<T>& h, T** out) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sizeof(T) * (h.empty() ? 1 : h.size()));
  if (e != cudaSuccess) return e;
  d->owned.push_back(p);
  if (!h.empty()) e = cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
  *out = (T*)p;
  return e;
}

cudaError_t alloc_zero(gh_domain* d, size_t bytes, void** out) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 8);
  if (e != cudaSuccess) return e;
  d->owned.push_back(p);
  e = cudaMemset(p, 0, bytes ? bytes : 8);
  *out = p;
  return e;
}

// Rows per block, block maps and shared memory of the folded kernels from the
// domain's current schedule (fd/ff threads and budgets); re-run by gh_autotune.
cudaError_t fold_build_maps(gh_domain* d) {
  const int n_shells = d->n_shells;
  // fused kernel: the shells without ring FFTs; the FFT path: the others
  std::vector<int> fb2(n_shells + 1), ffb(n_shells + 1);
  std::vector<int> an[2], leg[2], sy[2];
  for (int k = 0; k < 2; ++k) {
    an[k].assign(n_shells + 1, 0);
    leg[k].assign(n_shells + 1, 0);
    sy[k].assign(n_shells + 1, 0);
  }
  int nfd = 0, nff = 0, nan[2] = {0, 0}, nleg[2] = {0, 0}, nsy[2] = {0, 0};
  size_t smfd = 0, smff = 0, sman[2] = {0, 0}, smleg[2] = {0, 0}, smsy[2] = {0, 0};
  bool any_fft = false;
  for (int s = 0; s < n_shells; ++s) {
    gh::ShellDev& sh = d->shells_h[s];
    const int rows = gh::NF * sh.n_r;
    const int W = sh.fd.W;
    const bool fft = sh.fd.fft_log != 0;
    any_fft = any_fft || fft;
    const long long rings = (long long)rows * sh.nth;
    const int ring_warps = (int)((rings + 31) / 32);
    for (int k = 0; k < 2; ++k) {
      gh::FoldPlan& P = k == 0 ? sh.fd : sh.ff;
      const int n_out = k == 0 ? 2 : 1;
      const bool on = k == 0 || sh.ff.M > 0;
      int& nb = k == 0 ? nfd : nff;
      size_t& sm = k == 0 ? smfd : smff;
      (k == 0 ? fb2 : ffb)[s] = nb;
      an[k][s] = nan[k];
      leg[k][s] = nleg[k];
      sy[k][s] = nsy[k];
      if (!on) continue;
      P.rows_per_cta = fold_rows_per_block(sh.na, sh.nth, W, P.M, n_out, P.ncoef, fft, rows,
                                           k == 0 ? d->fd_budget : d->ff_budget);
      const size_t row_bytes = sizeof(double) * (size_t)P.rows_per_cta *
                               fold_row_doubles(sh.na, sh.nth, W, P.M, n_out, P.ncoef, fft);
      if (!fft) {
        nb += (rows + P.rows_per_cta - 1) / P.rows_per_cta;
        sm = std::max(sm, row_bytes);
        continue;
      }
      nan[k] += (ring_warps + gh::FOLD_FFT_WARPS - 1) / gh::FOLD_FFT_WARPS;
      nleg[k] += (rows + P.rows_per_cta - 1) / P.rows_per_cta;
      nsy[k] += (n_out * ring_warps + gh::FOLD_FFT_WARPS - 1) / gh::FOLD_FFT_WARPS;
      sman[k] = std::max(sman[k], sizeof(double) * gh::FOLD_FFT_WARPS * 32 * (size_t)(sh.nph + 1));
      smleg[k] = std::max(smleg[k], row_bytes);
      smsy[k] = std::max(smsy[k], sizeof(double) * gh::FOLD_FFT_WARPS * 32 * (size_t)P.M);
    }
  }
  fb2[n_shells] = nfd;
  ffb[n_shells] = nff;
  d->fd_blocks = nfd;
  d->ff_blocks = nff;
  d->fd_smem = smfd;
  d->ff_smem = smff;
  for (int k = 0; k < 2; ++k) {
    an[k][n_shells] = nan[k];
    leg[k][n_shells] = nleg[k];
    sy[k][n_shells] = nsy[k];
    gh_domain::FoldFftMap& m = d->fxm[k];
    m.an_blocks = nan[k];
    m.leg_blocks = nleg[k];
    m.sy_blocks = nsy[k];
    m.an_smem = sman[k];
    m.leg_smem = smleg[k];
    m.sy_smem = smsy[k];
  }
  // transposed maps (reverse mode): a fixed thread count and budget; the
  // shells with ring FFTs take the three-launch form as in the forward
  std::vector<int> fa2(n_shells + 1), ffa(n_shells + 1);
  std::vector<int> aan[2], aleg[2], asy[2];
  for (int k = 0; k < 2; ++k) {
    aan[k].assign(n_shells + 1, 0);
    aleg[k].assign(n_shells + 1, 0);
    asy[k].assign(n_shells + 1, 0);
  }
  int nfa = 0, nffa = 0, naan[2] = {0, 0}, naleg[2] = {0, 0}, nasy[2] = {0, 0};
  size_t smfa = 0, smffa = 0, smaan[2] = {0, 0}, smaleg[2] = {0, 0}, smasy[2] = {0, 0};
  auto adj_rows = [](size_t row_doubles, int n_rows) {
    int rb = (int)((size_t)gh::FOLD_ADJ_BUDGET / (sizeof(double) * row_doubles));
    return std::max(1, std::min(std::min(rb, 64), n_rows));
  };
  for (int s = 0; s < n_shells; ++s) {
    gh::ShellDev& sh = d->shells_h[s];
    const int rows = gh::NF * sh.n_r;
    const int W = sh.fd.W;
    const bool fft = sh.fd.fft_log != 0;
    const int ring_warps = (int)(((long long)rows * sh.nth + 31) / 32);
    for (int k = 0; k < 2; ++k) {
      gh::FoldPlan& P = k == 0 ? sh.fd : sh.ff;
      const int n_out = k == 0 ? 2 : 1;
      int& nb = k == 0 ? nfa : nffa;
      size_t& sm = k == 0 ? smfa : smffa;
      (k == 0 ? fa2 : ffa)[s] = nb;
      aan[k][s] = naan[k];
      aleg[k][s] = naleg[k];
      asy[k][s] = nasy[k];
      if (k == 1 && sh.ff.M <= 0) continue;
      const size_t rd = gh::fold_adjoint_row_doubles(sh.na, sh.nth, W, P.M, n_out, fft);
      P.adj_rows_per_cta = adj_rows(rd, rows);
      const size_t bytes = sizeof(double) * (size_t)P.adj_rows_per_cta * rd;
      if (!fft) {
        nb += (rows + P.adj_rows_per_cta - 1) / P.adj_rows_per_cta;
        sm = std::max(sm, bytes);
        continue;
      }
      naan[k] += (n_out * ring_warps + gh::FOLD_FFT_WARPS - 1) / gh::FOLD_FFT_WARPS;
      naleg[k] += (rows + P.adj_rows_per_cta - 1) / P.adj_rows_per_cta;
      nasy[k] += (ring_warps + gh::FOLD_FFT_WARPS - 1) / gh::FOLD_FFT_WARPS;
      smaan[k] = std::max(smaan[k], sizeof(double) * gh::FOLD_FFT_WARPS * 32 * (size_t)(sh.nph + 1));
      smaleg[k] = std::max(smaleg[k], bytes);
      smasy[k] = std::max(smasy[k], sizeof(double) * gh::FOLD_FFT_WARPS * 32 * (size_t)P.M);
    }
  }
  for (int k = 0; k < 2; ++k) {
    aan[k][n_shells] = naan[k];
    aleg[k][n_shells] = naleg[k];
    asy[k][n_shells] = nasy[k];
    gh_domain::FoldFftMap& m = d->fxa[k];
    m.an_blocks = naan[k];
    m.leg_blocks = naleg[k];
    m.sy_blocks = nasy[k];
    m.an_smem = smaan[k];
    m.leg_smem = smaleg[k];
    m.sy_smem = smasy[k];
  }
  fa2[n_shells] = nfa;
  ffa[n_shells] = nffa;
  d->fda_blocks = nfa;
  d->ffa_blocks = nffa;
  d->fda_smem = smfa;
  d->ffa_smem = smffa;
  cudaError_t e;
  if (!d->fd_block_begin_d) {
    if ((e = upload(d, fb2, &d->fd_block_begin_d)) != cudaSuccess) return e;
    if ((e = upload(d, ffb, &d->ff_block_begin_d)) != cudaSuccess) return e;
    if ((e = upload(d, fa2, &d->fda_block_begin_d)) != cudaSuccess) return e;
    if ((e = upload(d, ffa, &d->ffa_block_begin_d)) != cudaSuccess) return e;
  } else {
    if ((e = cudaMemcpy(d->fd_block_begin_d, fb2.data(), sizeof(int) * fb2.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(d->ff_block_begin_d, ffb.data(), sizeof(int) * ffb.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  }
  auto put = [&](const std::vector<int>& h, int*& dev) -> cudaError_t {
    if (!dev) return upload(d, h, &dev);
    return cudaMemcpy(dev, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice);
  };
  for (int k = 0; k < 2; ++k) {
    if ((e = put(an[k], d->fxm[k].an_begin_d)) != cudaSuccess) return e;
    if ((e = put(leg[k], d->fxm[k].leg_begin_d)) != cudaSuccess) return e;
    if ((e = put(sy[k], d->fxm[k].sy_begin_d)) != cudaSuccess) return e;
    if ((e = put(aan[k], d->fxa[k].an_begin_d)) != cudaSuccess) return e;
    if ((e = put(aleg[k], d->fxa[k].leg_begin_d)) != cudaSuccess) return e;
    if ((e = put(asy[k], d->fxa[k].sy_begin_d)) != cudaSuccess) return e;
  }
  if (any_fft && !d->fft_ab) {
    void* p = nullptr;
    if ((e = alloc_zero(d, sizeof(double) * d->state, &p)) != cudaSuccess) return e;
    d->fft_ab = (double*)p;
    if ((e = alloc_zero(d, sizeof(double) * d->state, &p)) != cudaSuccess) return e;
    d->fft_c0 = (double*)p;
    if ((e = alloc_zero(d, sizeof(double) * d->state, &p)) != cudaSuccess) return e;
    d->fft_c1 = (double*)p;
  }
  if ((e = gh::fold_fft_set_smem_limits(std::max(sman[0], sman[1]), std::max(smleg[0], smleg[1]),
                                        std::max(smsy[0], smsy[1]))) != cudaSuccess)
    return e;
  if ((e = gh::fold_fft_adj_set_smem_limits(std::max(smaan[0], smaan[1]), std::max(smaleg[0], smaleg[1]),
                                            std::max(smasy[0], smasy[1]))) != cudaSuccess)
    return e;
  if (d->shells_d &&
      (e = cudaMemcpy(d->shells_d, d->shells_h.data(), sizeof(gh::ShellDev) * d->shells_h.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  if ((e = gh::fold_adjoint_set_smem_limits(std::max(smfa, smffa))) != cudaSuccess) return e;
  return gh::fold_set_smem_limits(std::max(smfd, smff));
}

bool fault_injected(const char* what) {
  const char* f = std::getenv("GH_FAULT");
  return f && std::strcmp(f, what) == 0;
}

gh_status check_latched(gh_domain* d) {
  if (fault_injected("launch")) return fail(d, GH_ECUDA, "GH_FAULT=launch: injected launch failure");
  return GH_OK;
}

// Profiler brackets (no-ops unless gh_profile_enable(dom, 1)).
cudaEvent_t take_event(gh_domain* d) {
  if (!d->event_pool.empty()) {
    cudaEvent_t e = d->event_pool.back();
    d->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  gh_domain* d;
  int fam;
  cudaEvent_t a = nullptr;
  ProfScope(gh_domain* dd, int f) : d(dd), fam(f) {
    if (d->prof) {
      a = take_event(d);
      cudaEventRecord(a, d->stream);
    }
  }
  ~ProfScope() {
    if (d->prof && a) {
      cudaEvent_t b = take_event(d);
      cudaEventRecord(b, d->stream);
      d->pending.push_back({fam, a, b});
    }
  }
};

gh_status derivatives(gh_domain* d, const double* u) {
  if (d->overlap && !d->prof) {
    GH_CUDA(d, gh::launch_derivatives(d, u));
    return GH_OK;
  }
  {
    ProfScope p(d, GH_K_RADIAL);
    GH_CUDA(d, gh::launch_radial(d, u, d->d_r, false));
  }
  {
    ProfScope p(d, GH_K_ANGULAR);
    GH_CUDA(d, gh::launch_angular_deriv(d, u));
  }
  return GH_OK;
}

gh_status filters(gh_domain* d, double* src, double* u, double* tmp, double* dest_host = nullptr) {
  // src -> (angular) -> (radial) -> u, or -> dest_host (pinned host memory, as
  // seen from the device) when given; tmp must not alias src or u.  The two
  // filters act on different axes (the angular maps on the rows, the radial on
  // the columns of the [row][angle] layout), so they commute; the radial one
  // runs last because its column-wise stores are coalesced, also into host memory.
  const bool rad = d->params.radial_filter_on != 0;
  const bool ang = d->params.sh_keep_l != -1;
  double* dest = dest_host ? dest_host : u;
  double* cur = src;
  if (ang) {
    ProfScope p(d, GH_K_ANGULAR_FILTER);
    double* dst = rad ? d->d_r : ((cur == dest) ? tmp : dest);
    if (d->sh_filter_mode == GH_SH_FILTER_TENSOR)
      GH_CUDA(d, gh::launch_tensor_filter(d, cur, dst));
    else
      GH_CUDA(d, gh::launch_angular_filter(d, cur, dst));
    cur = dst;
  }
  if (rad) {
    ProfScope p(d, GH_K_RADIAL_FILTER);
    double* dst = (cur == dest) ? tmp : dest;
    GH_CUDA(d, gh::launch_radial(d, cur, dst, true));
    cur = dst;
  }
  if (cur != dest)
    GH_CUDA(d, cudaMemcpyAsync(dest, cur, sizeof(double) * d->state, cudaMemcpyDefault, d->stream));
  return GH_OK;
}

}  // namespace

// Dense traced matrices (the paper's Eq. DifferentiatorI1S2 maps) and their
// batched GEMM plans, built on first use.
gh_status build_dense(gh_domain* d) {
  if (d->ang_deriv_d) return GH_OK;
  std::map<int, std::pair<double*, double*>> ang_cache;   // L -> (Bth, Bph)
  std::map<std::pair<int, int>, double*> filt_cache;      // (L, keep) -> S
  std::vector<gh::GemmProb> pd, pf;
  int tiles = 0, ftiles = 0;
  for (int s = 0; s < d->n_shells; ++s) {
    gh::ShellDev& sh = d->shells_h[s];
    AngularGrid ag = angular_grid(sh.L);
    if (!ang_cache.count(sh.L)) {
      double *Bt = nullptr, *Bp = nullptr;
      GH_CUDA(d, upload(d, angular_matrix(ag, 0, 0), &Bt));
      GH_CUDA(d, upload(d, angular_matrix(ag, 1, 0), &Bp));
      ang_cache[sh.L] = {Bt, Bp};
    }
    sh.Bth = ang_cache[sh.L].first;
    sh.Bph = ang_cache[sh.L].second;
    if (sh.keep >= 0) {
      const auto key = std::make_pair(sh.L, sh.keep);
      if (!filt_cache.count(key)) {
        double* Sd = nullptr;
        GH_CUDA(d, upload(d, angular_matrix(ag, 2, sh.keep), &Sd));
        filt_cache[key] = Sd;
      }
      sh.Sf = filt_cache[key];
    }
    for (int c = 0; c < 2; ++c) {
      gh::GemmProb P;
      std::memset(&P, 0, sizeof(P));
      P.a_off = sh.off;
      P.c_off = sh.off;
      P.B = c == 0 ? sh.Bth : sh.Bph;
      P.M = sh.n_r * gh::NF;
      P.N = sh.na;
      P.K = sh.na;
      P.lda = P.ldb = P.ldc = sh.na;
      P.tiles_n = (P.N + 63) / 64;
      P.tile_begin = tiles;
      P.c_sel = c;
      tiles += ((P.M + 63) / 64) * P.tiles_n;
      pd.push_back(P);
    }
    if (sh.Sf) {
      gh::GemmProb P;
      std::memset(&P, 0, sizeof(P));
      P.a_off = sh.off;
      P.c_off = sh.off;
      P.B = sh.Sf;
      P.M = sh.n_r * gh::NF;
      P.N = sh.na;
      P.K = sh.na;
      P.lda = P.ldb = P.ldc = sh.na;
      P.tiles_n = (P.N + 63) / 64;
      P.tile_begin = ftiles;
      ftiles += ((P.M + 63) / 64) * P.tiles_n;
      pf.push_back(P);
    }
  }
  d->ang_filt_np = (int)pf.size();
  d->ang_filt_tiles = ftiles;
  if (!pf.empty()) GH_CUDA(d, upload(d, pf, &d->ang_filt_d));
  d->ang_deriv_np = (int)pd.size();
  d->ang_deriv_tiles = tiles;
  GH_CUDA(d, upload(d, pd, &d->ang_deriv_d));
  return GH_OK;
}

// =================================================================== C ABI
// ------------------------------------------------------------ autotuner
namespace {
// Average time of one call of f over reps calls (after one warm-up call),
// measured with CUDA events on the domain's stream.
template <typename F>
cudaError_t time_calls(gh_domain* d, int reps, F f, float* ms) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
  e = f();
  if (e == cudaSuccess) e = cudaEventRecord(a, d->stream);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = f();
  if (e == cudaSuccess) e = cudaEventRecord(b, d->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  *ms = t / reps;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

bool schedule_ok(const int* v) {
  auto in = [](int x, int lo, int hi) { return x >= lo && x <= hi; };
  return in(v[0], 2, 4) && in(v[1], 1, 4) && in(v[2], 2, 4) && in(v[3], 1, 4) &&
         in(v[4], 32, 512) && v[4] % 32 == 0 && in(v[5], 8 * 1024, 200 * 1024) &&
         in(v[6], 32, 512) && v[6] % 32 == 0 && in(v[7], 8 * 1024, 200 * 1024) && in(v[8], 0, 1);
}

// The host path's captured step is rebuilt after any change to the step's
// launches (algorithm, schedule, overlap, frame, outer condition, S2 filter).
void invalidate_host_graph(gh_domain* d) {
  if (d->host_graph) {
    cudaGraphExecDestroy(d->host_graph);
    d->host_graph = nullptr;
  }
  if (d->host_graph_io) {
    cudaGraphExecDestroy(d->host_graph_io);
    d->host_graph_io = nullptr;
  }
}

// The device address of a pinned (page-locked, mapped) host buffer, or NULL
// for any other pointer (pageable host memory, device memory).
const double* device_view(const double* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();                  // clear the sticky-free error of an unknown pointer
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return (const double*)a.devicePointer;
}
double* device_view(double* p) { return const_cast<double*>(device_view((const double*)p)); }

void invalidate_graph(gh_domain* d) {
  if (d->graph_exec) {
    cudaGraphExecDestroy(d->graph_exec);
    d->graph_exec = nullptr;
  }
  invalidate_host_graph(d);
}
}  // namespace

namespace gh {
Frame frame_at(const gh_domain* d, double t) {
  Frame f;
  f.on = frame_moving(d) ? 1 : 0;
  f.gen = d->map_gen ? 1 : 0;
  f.a = d->map_gen ? 1.0 + d->map_adot * t : 1.0;
  f.adot = d->map_gen ? d->map_adot : 0.0;
  for (int i = 0; i < 3; ++i) {
    f.V[i] = d->map_gen ? d->map_V[i] : 0.0;
    f.T[i] = f.V[i] * t;
  }
  const double n = std::sqrt(d->rot_axis[0] * d->rot_axis[0] + d->rot_axis[1] * d->rot_axis[1] +
                             d->rot_axis[2] * d->rot_axis[2]);
  const double e[3] = {d->rot_axis[0] / n, d->rot_axis[1] / n, d->rot_axis[2] / n};
  const double th = d->rot_omega * t, c = std::cos(th), sn = std::sin(th);
  // Rodrigues: R = I + sin K + (1 - cos) K^2, K the cross-product matrix of e
  const double K[9] = {0.0, -e[2], e[1], e[2], 0.0, -e[0], -e[1], e[0], 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double k2 = 0.0;
      for (int m = 0; m < 3; ++m) k2 += K[3 * i + m] * K[3 * m + j];
      f.R[3 * i + j] = (i == j ? 1.0 : 0.0) + sn * K[3 * i + j] + (1.0 - c) * k2;
    }
  for (int i = 0; i < 3; ++i) f.w[i] = d->rot_omega * e[i];
  if (!f.on)
    for (int i = 0; i < 9; ++i) f.R[i] = (i % 4 == 0) ? 1.0 : 0.0;
  return f;
}
gh_status check_latched(gh_domain* d) { return ::check_latched(d); }
}  // namespace gh

extern "C" {

gh_status gh_create_domain(const gh_shell* shells, int n_shells, const gh_params* params,
                           void* stream, gh_domain** out) {
  if (!out) return fail(nullptr, GH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!shells || n_shells < 1 || n_shells > 1024) return fail(nullptr, GH_EINVAL, "need 1..1024 shells");
  if (!params) return fail(nullptr, GH_EINVAL, "params is NULL");
  for (int s = 0; s < n_shells; ++s) {
    const gh_shell& sh = shells[s];
    if (!(sh.r_in > 0.0) || !(sh.r_out > sh.r_in) || sh.n_r < 3 || sh.n_r > 64 || sh.L < 1 || sh.L > 47)
      return fail(nullptr, GH_EINVAL, "shell " + std::to_string(s) + ": need 0 < r_in < r_out, 3 <= n_r <= 64, 1 <= L <= 47");
    if (sh.bh < 0) return fail(nullptr, GH_EINVAL, "shell " + std::to_string(s) + ": bh must be >= 0");
    if (s > 0 && shells[s].bh == shells[s - 1].bh) {
      if (shells[s].r_in != shells[s - 1].r_out)
        return fail(nullptr, GH_EINVAL, "shell " + std::to_string(s) + " does not start where shell " +
                                            std::to_string(s - 1) + " ends");
      if (shells[s].L != shells[s - 1].L)
        return fail(nullptr, GH_EINVAL, "adjacent shells of one hole must have the same L (shared boundary points)");
    }
    for (int t = 0; t + 1 < s; ++t)
      if (shells[t].bh == sh.bh && shells[s - 1].bh != sh.bh)
        return fail(nullptr, GH_EINVAL, "the shells of hole " + std::to_string(sh.bh) + " are not consecutive");
  }
  if (params->sh_keep_l < -2) return fail(nullptr, GH_EINVAL, "sh_keep_l must be >= -2");
  if (params->sh_keep_l >= 0)
    for (int s = 0; s < n_shells; ++s)
      if (params->sh_keep_l > shells[s].L) return fail(nullptr, GH_EINVAL, "sh_keep_l exceeds a shell's L");
  if (params->radial_filter_on && !(params->filt_order > 0)) return fail(nullptr, GH_EINVAL, "filt_order must be > 0");
  if (fault_injected("alloc")) return fail(nullptr, GH_ENOMEM, "GH_FAULT=alloc: injected allocation failure");

  gh_domain* d = new gh_domain();
  d->n_shells = n_shells;
  d->params = *params;
  d->stream = (cudaStream_t)stream;
  cudaGetDevice(&d->device);
  auto bail = [&](gh_status st) {
    g_create_error = d->err;
    gh_destroy_domain(d);
    return st;
  };
#define CREATE_CUDA(call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      d->err = std::string(#call) + ": " + cudaGetErrorString(e_);                         \
      return bail(e_ == cudaErrorMemoryAllocation ? GH_ENOMEM : GH_ECUDA);                 \
    }                                                                                      \
  } while (0)

  // matrix dictionary keyed by the parameters that make a map new (Sec. 3.4)
  std::map<int, std::pair<double*, double*>> radial_cache;              // n_r -> (D, F)
  std::map<int, std::pair<double*, double*>> radial_t_cache;            // n_r -> (D^T, F^T)
  std::map<std::tuple<int, int, int>, gh::SepPlan> sep_cache;           // (L, K, kind) -> plan
  std::map<std::tuple<int, int, int>, gh::SepAdjPlan> sep_adj_cache;    // its transpose
  std::map<std::tuple<int, int, int>, gh::FoldPlan> fold_cache;         // folded plans
  bool all_fold = true;
  std::map<int, AngularGrid> grids;

  long long off = 0, pts = 0;
  d->shells_h.resize(n_shells);
  for (int s = 0; s < n_shells; ++s) {
    const gh_shell& in = shells[s];
    gh::ShellDev& sh = d->shells_h[s];
    std::memset(&sh, 0, sizeof(sh));
    sh.n_r = in.n_r;
    sh.L = in.L;
    sh.nth = in.L + 1;
    sh.nph = 2 * (in.L + 1);
    sh.na = sh.nth * sh.nph;
    sh.off = off;
    sh.pt_off = pts;
    sh.r_in = in.r_in;
    sh.r_out = in.r_out;
    sh.rscale = 2.0 / (in.r_out - in.r_in);
    sh.bh = in.bh;
    sh.dt_scale = 1.0;
    sh.keep = params->sh_keep_l == -2 ? (2 * in.L) / 3 : params->sh_keep_l;
    off += (long long)sh.n_r * gh::NF * sh.na;
    pts += (long long)sh.n_r * sh.na;
    if (!radial_cache.count(sh.n_r)) {
      double *Dd = nullptr, *Fd = nullptr;
      CREATE_CUDA(upload(d, fold_radial_matrix(cgl_derivative_matrix(sh.n_r), sh.n_r), &Dd));
      CREATE_CUDA(upload(d, fold_radial_matrix(cgl_filter_matrix(sh.n_r, params->filt_alpha,
                                                                  params->filt_order > 0 ? params->filt_order : 1),
                                               sh.n_r),
                         &Fd));
      radial_cache[sh.n_r] = {Dd, Fd};
    }
    sh.Dr = radial_cache[sh.n_r].first;
    sh.Fr = radial_cache[sh.n_r].second;
    if (!radial_t_cache.count(sh.n_r)) {
      auto tr = [](std::vector<double> m, int n) {
        std::vector<double> t(m.size());
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) t[(size_t)j * n + i] = m[(size_t)i * n + j];
        return t;
      };
      double *DT = nullptr, *FT = nullptr;
      CREATE_CUDA(upload(d, fold_radial_matrix(tr(cgl_derivative_matrix(sh.n_r), sh.n_r), sh.n_r), &DT));
      CREATE_CUDA(upload(d, fold_radial_matrix(tr(cgl_filter_matrix(sh.n_r, params->filt_alpha,
                                                                      params->filt_order > 0 ? params->filt_order : 1),
                                                   sh.n_r),
                                                sh.n_r),
                         &FT));
      radial_t_cache[sh.n_r] = {DT, FT};
    }
    sh.DrT = radial_t_cache[sh.n_r].first;
    sh.FrT = radial_t_cache[sh.n_r].second;
    if (!grids.count(sh.L)) grids[sh.L] = angular_grid(sh.L);
    const AngularGrid& ag = grids[sh.L];
    // separable angular plans, cached by (L, K, kind)
    auto get_plan = [&](int K, bool deriv, gh::SepPlan& out, gh::SepAdjPlan& adj) -> cudaError_t {
      auto key = std::make_tuple(sh.L, K, deriv ? 1 : 0);
      if (!sep_cache.count(key)) {
        SepHost h = sep_plan(ag, K, deriv);
        gh::SepPlan P;
        gh::SepAdjPlan T;
        std::memset(&P, 0, sizeof(P));
        std::memset(&T, 0, sizeof(T));
        P.K = T.K = h.K;
        P.M = T.M = h.M;
        double* q = nullptr;
        cudaError_t e;
        if ((e = upload(d, h.F, &q)) != cudaSuccess) return e; P.F = q;
        if ((e = upload(d, h.G0, &q)) != cudaSuccess) return e; P.G0 = q;
        if ((e = upload(d, h.Q0, &q)) != cudaSuccess) return e; P.Q0 = q;
        if ((e = upload(d, h.F0T, &q)) != cudaSuccess) return e; T.F0T = q;
        if ((e = upload(d, h.Q0T, &q)) != cudaSuccess) return e; T.Q0T = q;
        if ((e = upload(d, h.GT, &q)) != cudaSuccess) return e; T.GT = q;
        if (deriv) {
          if ((e = upload(d, h.G1, &q)) != cudaSuccess) return e; P.G1 = q;
          if ((e = upload(d, h.Q1, &q)) != cudaSuccess) return e; P.Q1 = q;
          if ((e = upload(d, h.F1T, &q)) != cudaSuccess) return e; T.F1T = q;
          if ((e = upload(d, h.Q1T, &q)) != cudaSuccess) return e; T.Q1T = q;
        }
        sep_cache[key] = P;
        sep_adj_cache[key] = T;
      }
      out = sep_cache[key];
      adj = sep_adj_cache[key];
      return cudaSuccess;
    };
    CREATE_CUDA(get_plan(sh.L, true, sh.sd, sh.sda));
    sh.sd.rows_per_cta = sep_rows_per_block(sh.na, sh.nth, sh.sd.M, true, gh::NF * sh.n_r);
    sh.sda.rows_per_cta = sep_adj_rows_per_block(sh.na, sh.nth, sh.sda.M, true, gh::NF * sh.n_r);
    if (fold_applicable(ag)) {
      auto get_fold = [&](int K, bool deriv, gh::FoldPlan& out) -> cudaError_t {
        auto key = std::make_tuple(sh.L, K, deriv ? 1 : 0);
        if (!fold_cache.count(key)) {
          FoldHost f = fold_plan(ag, K, deriv);
          gh::FoldPlan P;
          std::memset(&P, 0, sizeof(P));
          P.K = f.K;
          P.M = f.M;
          P.N4 = f.N4;
          P.half = f.half;
          P.W = f.W;
          P.hs = f.hs;
          P.qself = f.qself;
          P.two = deriv ? 1 : 0;
          P.sigma0 = f.s0;
          P.sigma1 = f.s1;
          double* q = nullptr;
          cudaError_t e;
          if ((e = upload(d, f.Tc, &q)) != cudaSuccess) return e; P.Tc = q;
          if ((e = upload(d, f.Ts, &q)) != cudaSuccess) return e; P.Ts = q;
          if ((e = upload(d, f.Q0s, &q)) != cudaSuccess) return e; P.Q0s = q;
          if ((e = upload(d, f.Q0t, &q)) != cudaSuccess) return e; P.Q0t = q;
          if (deriv) {
            if ((e = upload(d, f.Q1s, &q)) != cudaSuccess) return e; P.Q1s = q;
            if ((e = upload(d, f.Q1t, &q)) != cudaSuccess) return e; P.Q1t = q;
          }
          P.m0 = f.m0;
          P.ncoef = f.coef_off[f.K + 1];
          P.fft_log = fold_fft_log(ag);
          if ((e = upload(d, f.A, &q)) != cudaSuccess) return e; P.A = q;
          if ((e = upload(d, f.Y0, &q)) != cudaSuccess) return e; P.Y0 = q;
          if ((e = upload(d, f.Y1, &q)) != cudaSuccess) return e; P.Y1 = q;
          int* qi = nullptr;
          if ((e = upload(d, f.coef_off, &qi)) != cudaSuccess) return e; P.coef_off = qi;
          if ((e = upload(d, f.slot_m, &qi)) != cudaSuccess) return e; P.slot_m = qi;
          fold_cache[key] = P;
        }
        out = fold_cache[key];
        return cudaSuccess;
      };
      CREATE_CUDA(get_fold(sh.L, true, sh.fd));
      if (sh.keep >= 0) CREATE_CUDA(get_fold(sh.keep, false, sh.ff));
    } else {
      all_fold = false;
    }
    if (sh.keep >= 0) {
      CREATE_CUDA(get_plan(sh.keep, false, sh.sf, sh.sfa));
      sh.sf.rows_per_cta = sep_rows_per_block(sh.na, sh.nth, sh.sf.M, false, gh::NF * sh.n_r);
      sh.sfa.rows_per_cta = sep_adj_rows_per_block(sh.na, sh.nth, sh.sfa.M, false, gh::NF * sh.n_r);
    }
    // grid tables
    std::vector<double> x = cgl_points(sh.n_r), wcc = clenshaw_curtis(sh.n_r);
    std::vector<double> r(sh.n_r), wr(sh.n_r);
    for (int i = 0; i < sh.n_r; ++i) {
      r[i] = 0.5 * (in.r_in + in.r_out) + 0.5 * (in.r_out - in.r_in) * x[i];
      if (i == 0) r[i] = in.r_in;
      if (i == sh.n_r - 1) r[i] = in.r_out;
      wr[i] = wcc[i] * 0.5 * (in.r_out - in.r_in) * r[i] * r[i];
    }
    std::vector<double> wth(sh.nth), cph(sh.nph), sph(sh.nph);
    for (int j = 0; j < sh.nth; ++j) wth[j] = ag.wgl[j] * 2.0 * kPi / sh.nph;
    for (int k = 0; k < sh.nph; ++k) {
      cph[k] = std::cos(2.0 * kPi * k / sh.nph);
      sph[k] = std::sin(2.0 * kPi * k / sh.nph);
    }
    double* p = nullptr;
    CREATE_CUDA(upload(d, r, &p)); sh.r = p;
    CREATE_CUDA(upload(d, wr, &p)); sh.wr = p;
    CREATE_CUDA(upload(d, ag.ct, &p)); sh.cth = p;
    CREATE_CUDA(upload(d, ag.st, &p)); sh.sth = p;
    CREATE_CUDA(upload(d, wth, &p)); sh.wth = p;
    CREATE_CUDA(upload(d, cph, &p)); sh.cph = p;
    CREATE_CUDA(upload(d, sph, &p)); sh.sph = p;
    void* gz = nullptr;
    CREATE_CUDA(alloc_zero(d, sizeof(double) * (size_t)sh.n_r * gh::NGAUGE * sh.na, &gz));
    sh.gauge = (double*)gz;
    sh.bc_inner = -1;
    sh.bc_outer = -1;
  }
  d->state = off;
  d->points = pts;

  // boundary slices: internal boundaries, then the outer boundary
  std::vector<int> bc_begin;
  int bpts = 0;
  for (int s = 0; s < n_shells; ++s) {
    gh::BcSliceDev b;
    std::memset(&b, 0, sizeof(b));
    gh::ShellDev& sa = d->shells_h[s];
    b.bh = sa.bh;
    b.dt_scale = 1.0;
    if (s + 1 < n_shells && d->shells_h[s + 1].bh == sa.bh) {
      gh::ShellDev& sb = d->shells_h[s + 1];
      b.kind = 1;
      b.shell_b = s + 1;
      b.off_b = sb.off;
      sb.bc_inner = (int)d->bc_h.size();
    } else {
      b.kind = 0;
      b.shell_b = -1;
      b.off_b = 0;
    }
    b.shell_a = s;
    b.na = sa.na;
    b.off_a = sa.off + (long long)(sa.n_r - 1) * gh::NF * sa.na;
    sa.bc_outer = (int)d->bc_h.size();
    // flat background: n = R-hat, alpha = 1, beta = 0
    std::vector<double> bg((size_t)gh::NBG * sa.na, 0.0);
    const AngularGrid& ag = grids[sa.L];
    for (int j = 0; j < sa.nth; ++j)
      for (int k = 0; k < sa.nph; ++k) {
        const int q = j * sa.nph + k;
        const double ph = 2.0 * kPi * k / sa.nph;
        const double nh[3] = {ag.st[j] * std::cos(ph), ag.st[j] * std::sin(ph), ag.ct[j]};
        for (int i = 0; i < 3; ++i) {
          bg[(size_t)i * sa.na + q] = nh[i];
          bg[(size_t)(3 + i) * sa.na + q] = nh[i];
        }
        bg[(size_t)6 * sa.na + q] = 1.0;
        for (int m : {10, 13, 15}) bg[(size_t)m * sa.na + q] = 1.0;   // g_ij = delta_ij
      }
    double* bgd = nullptr;
    CREATE_CUDA(upload(d, bg, &bgd));
    b.bg = bgd;
    bc_begin.push_back(bpts);
    bpts += sa.na;
    d->bc_h.push_back(b);
  }
  bc_begin.push_back(bpts);
  d->bc_points = bpts;
  CREATE_CUDA(upload(d, d->bc_h, &d->bc_d));
  CREATE_CUDA(upload(d, bc_begin, &d->bc_pt_begin_d));
  CREATE_CUDA(upload(d, d->shells_h, &d->shells_d));

  // launch maps
  std::vector<int> rb(n_shells + 1), pb(n_shells + 1);
  int nrb = 0, npb = 0;
  for (int s = 0; s < n_shells; ++s) {
    const gh::ShellDev& sh = d->shells_h[s];
    rb[s] = nrb;
    pb[s] = npb;
    nrb += (int)((gh::NF * (long long)sh.na + 127) / 128);
    d->max_n_r = std::max(d->max_n_r, sh.n_r);
    npb += sh.n_r * ((sh.na + gh::PT_THREADS - 1) / gh::PT_THREADS);
  }
  rb[n_shells] = nrb;
  pb[n_shells] = npb;
  d->rad_blocks = nrb;
  d->pt_blocks = npb;
  // the pair-split reverse kernel wins while ten threads per point still leave
  // FP64 units idle or lightly loaded (measured crossover near 10^4 points)
  d->adj_pair_split = (long long)npb * gh::PT_THREADS <= 8192;
  {
    // default radial row groups: about 12 warps per FP64 unit (4 per SM)
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const double warps = nrb * (double)gh::RAD_THREADS_HOST / 32.0;
    const int g = (int)std::ceil(12.0 * 4.0 * sms / std::max(1.0, warps));
    d->rad_groups = d->radf_groups = std::min(4, std::max(1, g));
  }
  {
    std::vector<int> ab(n_shells + 1);
    int nab = 0;
    for (int s = 0; s < n_shells; ++s) {
      ab[s] = nab;
      nab += d->shells_h[s].n_r * ((d->shells_h[s].na + gh::ADJ_PT_THREADS - 1) / gh::ADJ_PT_THREADS);
    }
    ab[n_shells] = nab;
    d->adj_pt_blocks = nab;
    CREATE_CUDA(upload(d, ab, &d->adj_pt_block_begin_d));
  }
  CREATE_CUDA(upload(d, rb, &d->rad_block_begin_d));
  CREATE_CUDA(upload(d, pb, &d->pt_block_begin_d));

  // separable angular launch maps (blocks of RB rows per shell)
  {
    std::vector<int> sb(n_shells + 1), fb(n_shells + 1);
    int nsb = 0, nfb = 0;
    size_t smd = 0, smf = 0;
    for (int s = 0; s < n_shells; ++s) {
      const gh::ShellDev& sh = d->shells_h[s];
      const int rows = gh::NF * sh.n_r;
      sb[s] = nsb;
      nsb += (rows + sh.sd.rows_per_cta - 1) / sh.sd.rows_per_cta;
      smd = std::max(smd, sizeof(double) * (size_t)sh.sd.rows_per_cta * (sh.na + 3 * (size_t)sh.nth * sh.sd.M));
      fb[s] = nfb;
      if (sh.sf.M > 0) {
        nfb += (rows + sh.sf.rows_per_cta - 1) / sh.sf.rows_per_cta;
        smf = std::max(smf, sizeof(double) * (size_t)sh.sf.rows_per_cta * (sh.na + 2 * (size_t)sh.nth * sh.sf.M));
      }
    }
    sb[n_shells] = nsb;
    fb[n_shells] = nfb;
    d->sd_blocks = nsb;
    d->sf_blocks = nfb;
    d->sd_smem = smd;
    d->sf_smem = smf;
    CREATE_CUDA(upload(d, sb, &d->sd_block_begin_d));
    CREATE_CUDA(upload(d, fb, &d->sf_block_begin_d));
    CREATE_CUDA(gh::sep_set_smem_limits(std::max(smd, smf)));
    CREATE_CUDA(gh::radial_set_smem_limits());
    // transposed maps
    std::vector<int> ab(n_shells + 1), afb(n_shells + 1);
    int nab = 0, nafb = 0;
    size_t sma = 0, smfa = 0;
    for (int s = 0; s < n_shells; ++s) {
      const gh::ShellDev& sh = d->shells_h[s];
      const int rows = gh::NF * sh.n_r;
      ab[s] = nab;
      nab += (rows + sh.sda.rows_per_cta - 1) / sh.sda.rows_per_cta;
      sma = std::max(sma, sizeof(double) * (size_t)sh.sda.rows_per_cta *
                              (2 * (size_t)sh.na + 3 * (size_t)sh.nth * sh.sda.M));
      afb[s] = nafb;
      if (sh.sfa.M > 0) {
        nafb += (rows + sh.sfa.rows_per_cta - 1) / sh.sfa.rows_per_cta;
        smfa = std::max(smfa, sizeof(double) * (size_t)sh.sfa.rows_per_cta *
                                  ((size_t)sh.na + 2 * (size_t)sh.nth * sh.sfa.M));
      }
    }
    ab[n_shells] = nab;
    afb[n_shells] = nafb;
    d->sda_blocks = nab;
    d->sfa_blocks = nafb;
    d->sda_smem = sma;
    d->sfa_smem = smfa;
    CREATE_CUDA(upload(d, ab, &d->sda_block_begin_d));
    CREATE_CUDA(upload(d, afb, &d->sfa_block_begin_d));
    CREATE_CUDA(gh::sep_adj_set_smem_limits(std::max(sma, smfa)));
    // folded maps
    d->fold_ok = all_fold;
    if (all_fold) CREATE_CUDA(gh::fold_fft_tables());
    if (all_fold) CREATE_CUDA(fold_build_maps(d));
    d->algorithm = all_fold ? 2 : 1;
  }

  // scratch
  void* p = nullptr;
  CREATE_CUDA(alloc_zero(d, sizeof(double) * d->state, &p)); d->d_r = (double*)p;
  CREATE_CUDA(alloc_zero(d, sizeof(double) * d->state, &p)); d->d_th = (double*)p;
  CREATE_CUDA(alloc_zero(d, sizeof(double) * d->state, &p)); d->d_ph = (double*)p;
  CREATE_CUDA(alloc_zero(d, sizeof(double) * (size_t)d->pt_blocks, &p)); d->partial = (double*)p;
  CREATE_CUDA(alloc_zero(d, sizeof(int), &p)); d->err_flag = (int*)p;
  CREATE_CUDA(alloc_zero(d, sizeof(double) * gh::DP_MAX_BLOCKS, &p)); d->dp_partial = (double*)p;
  CREATE_CUDA(alloc_zero(d, sizeof(double), &p)); d->dp_err = (double*)p;
  CREATE_CUDA(cudaStreamCreateWithFlags(&d->side, cudaStreamNonBlocking));
  CREATE_CUDA(cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming));
  CREATE_CUDA(cudaEventCreateWithFlags(&d->ev_join, cudaEventDisableTiming));
  CREATE_CUDA(cudaDeviceSynchronize());
#undef CREATE_CUDA
  *out = d;
  return GH_OK;
}

gh_status gh_destroy_domain(gh_domain* d) {
  if (!d) return GH_EINVAL;
  cudaStreamSynchronize(d->stream);
  for (auto& b : d->pending) {
    cudaEventDestroy(b.a);
    cudaEventDestroy(b.b);
  }
  for (cudaEvent_t e : d->event_pool) cudaEventDestroy(e);
  if (d->side) {
    cudaStreamSynchronize(d->side);
    cudaStreamDestroy(d->side);
  }
  if (d->ev_fork) cudaEventDestroy(d->ev_fork);
  if (d->ev_join) cudaEventDestroy(d->ev_join);
  if (d->graph_exec) cudaGraphExecDestroy(d->graph_exec);
  if (d->host_graph) cudaGraphExecDestroy(d->host_graph);
  if (d->host_graph_io) cudaGraphExecDestroy(d->host_graph_io);
  for (void* p : d->owned) cudaFree(p);
  delete d;
  return GH_OK;
}

gh_status gh_set_stream(gh_domain* d, void* stream) {
  if (!d) return GH_EINVAL;
  d->stream = (cudaStream_t)stream;
  return GH_OK;
}

gh_status gh_set_overlap(gh_domain* d, int on) {
  if (!d || (on != 0 && on != 1)) return fail(d, GH_EINVAL, "on must be 0 or 1");
  d->overlap = on != 0;
  invalidate_host_graph(d);
  return GH_OK;
}

long long gh_state_size(const gh_domain* d) { return d ? d->state : -1; }
long long gh_num_points(const gh_domain* d) { return d ? d->points : -1; }
long long gh_rk4_work_size(const gh_domain* d) { return d ? 3 * d->state : -1; }
int gh_num_shells(const gh_domain* d) { return d ? d->n_shells : -1; }
long long gh_launch_count(const gh_domain* d) { return d ? d->launches : -1; }

const char* gh_last_error(const gh_domain* d) { return d ? d->err.c_str() : g_create_error.c_str(); }

gh_status gh_set_analytic_kerr_schild_spin(gh_domain* d, int bh, double M, const double chi[3], double* u) {
  if (!d || !u || !chi) return fail(d, GH_EINVAL, "null argument");
  const double c2 = chi[0] * chi[0] + chi[1] * chi[1] + chi[2] * chi[2];
  if (!(M > 0.0) || !(c2 < 1.0)) return fail(d, GH_EINVAL, "need M > 0 and |chi| < 1");
  if (bh < -1) return fail(d, GH_EINVAL, "bh must be -1 (all) or a hole index");
  if (gh_status s = check_latched(d)) return s;
  GH_CUDA(d, gh::launch_kerr_schild(d, bh, M, chi, u));
  GH_CUDA(d, gh::launch_bc_background(d, u, bh));
  // the hole's parameters, for a general map's evaluations at moving points
  int nbh = 0;
  for (const auto& sh : d->shells_h) nbh = std::max(nbh, sh.bh + 1);
  if ((int)d->holes.size() < 4 * nbh) d->holes.resize(4 * (size_t)nbh, 0.0);
  for (int b = 0; b < nbh; ++b)
    if (bh == -1 || bh == b) {
      d->holes[4 * b] = M;
      for (int i = 0; i < 3; ++i) d->holes[4 * b + 1 + i] = chi[i] * M;
    }
  if (d->holes_d && d->map_gen) {
    GH_CUDA(d, cudaMemcpyAsync(d->holes_d, d->holes.data(), sizeof(double) * d->holes.size(), cudaMemcpyHostToDevice,
                               d->stream));
    GH_CUDA(d, cudaMemsetAsync(d->map_gate_d, 0, sizeof(gh::MapGate), d->stream));   // new holes: re-evaluate
  }
  return GH_OK;
}

gh_status gh_set_analytic_kerr_schild(gh_domain* d, int bh, double M, double chi, double* u) {
  const double v[3] = {0.0, 0.0, chi};
  return gh_set_analytic_kerr_schild_spin(d, bh, M, v, u);
}

gh_status gh_set_dt_scale(gh_domain* d, int bh, double scale) {
  if (!d) return GH_EINVAL;
  if (!(scale > 0.0)) return fail(d, GH_EINVAL, "scale must be > 0");
  int hit = 0;
  for (auto& sh : d->shells_h)
    if (sh.bh == bh) { sh.dt_scale = scale; ++hit; }
  for (auto& b : d->bc_h)
    if (b.bh == bh) b.dt_scale = scale;
  if (!hit) return fail(d, GH_EINVAL, "no shell belongs to hole " + std::to_string(bh));
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  GH_CUDA(d, cudaMemcpy(d->shells_d, d->shells_h.data(), sizeof(gh::ShellDev) * d->shells_h.size(),
                        cudaMemcpyHostToDevice));
  GH_CUDA(d, cudaMemcpy(d->bc_d, d->bc_h.data(), sizeof(gh::BcSliceDev) * d->bc_h.size(), cudaMemcpyHostToDevice));
  return GH_OK;
}

}  // extern "C"

extern "C" gh_status rk4_step_impl(gh_domain* d, double dt, double* u, double* work, double* norm2_pre,
                                   double* stages, const double* host_in = nullptr, double* host_out = nullptr);

namespace {
// One gh_rk4_step captured on a private stream and instantiated into *exec
// (replacing what it held); nothing executes and the clock stays.
gh_status capture_step(gh_domain* d, double dt, double* u, double* work, double* norm2_pre, cudaGraphExec_t* exec,
                       long long* n_launches, const double* host_in = nullptr, double* host_out = nullptr) {
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  cudaStream_t saved = d->stream;
  cudaStream_t cap = nullptr;
  GH_CUDA(d, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  const bool prof = d->prof;
  d->prof = false;
  d->stream = cap;
  const long long n0 = d->launches;
  const double t0 = d->time;      // capturing executes nothing: the clock stays
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  gh_status st = GH_OK;
  if (e == cudaSuccess) {
    st = check_latched(d);
    if (st == GH_OK) st = rk4_step_impl(d, dt, u, work, norm2_pre, nullptr, host_in, host_out);
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (e2 != cudaSuccess && st == GH_OK) e = e2;
  }
  d->time = t0;
  d->stream = saved;
  d->prof = prof;
  cudaStreamDestroy(cap);
  const long long n = d->launches - n0;
  d->launches = n0;
  if (st != GH_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(d, GH_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  }
  if (*exec) {
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(d, GH_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  *n_launches = n;
  return GH_OK;
}
}  // namespace

extern "C" {

gh_status gh_rk4_graph_capture(gh_domain* d, double dt, double* u, double* work, double* norm2_pre) {
  if (!d || !u || !work) return fail(d, GH_EINVAL, "null argument");
  if (gh_status s = capture_step(d, dt, u, work, norm2_pre, &d->graph_exec, &d->graph_step_launches)) return s;
  d->graph_dt = dt;
  return GH_OK;
}

gh_status gh_rk4_graph_launch(gh_domain* d, int n_steps) {
  if (!d || n_steps < 0) return fail(d, GH_EINVAL, "bad arguments");
  if (!d->graph_exec) return fail(d, GH_EINVAL, "no graph captured (call gh_rk4_graph_capture first)");
  if (gh_status s = check_latched(d)) return s;
  for (int i = 0; i < n_steps; ++i) GH_CUDA(d, cudaGraphLaunch(d->graph_exec, d->stream));
  d->launches += (long long)n_steps * d->graph_step_launches;
  d->time += n_steps * d->graph_dt;     // each replay advances the device clock by the captured dt
  return GH_OK;
}

gh_status gh_set_gauge(gh_domain* d, const double* H, const double* dH) {
  if (!d || !H || !dH) return fail(d, GH_EINVAL, "null argument");
  // user layout per shell: H [r][4][na], dH [r][12][na]; internal [r][16][na]
  long long hoff = 0, dhoff = 0;
  for (int s = 0; s < d->n_shells; ++s) {
    const gh::ShellDev& sh = d->shells_h[s];
    const size_t na = sh.na;
    for (int ir = 0; ir < sh.n_r; ++ir) {
      GH_CUDA(d, cudaMemcpyAsync(sh.gauge + (size_t)ir * gh::NGAUGE * na, H + hoff + (size_t)ir * 4 * na,
                                 sizeof(double) * 4 * na, cudaMemcpyDeviceToDevice, d->stream));
      GH_CUDA(d, cudaMemcpyAsync(sh.gauge + (size_t)ir * gh::NGAUGE * na + 4 * na,
                                 dH + dhoff + (size_t)ir * 12 * na, sizeof(double) * 12 * na,
                                 cudaMemcpyDeviceToDevice, d->stream));
    }
    hoff += (long long)sh.n_r * 4 * na;
    dhoff += (long long)sh.n_r * 12 * na;
  }
  return GH_OK;
}

gh_status gh_get_gauge(const gh_domain* dc, double* H, double* dH) {
  gh_domain* d = const_cast<gh_domain*>(dc);
  if (!d || !H || !dH) return fail(d, GH_EINVAL, "null argument");
  long long hoff = 0, dhoff = 0;
  for (int s = 0; s < d->n_shells; ++s) {
    const gh::ShellDev& sh = d->shells_h[s];
    const size_t na = sh.na;
    for (int ir = 0; ir < sh.n_r; ++ir) {
      GH_CUDA(d, cudaMemcpyAsync(H + hoff + (size_t)ir * 4 * na, sh.gauge + (size_t)ir * gh::NGAUGE * na,
                                 sizeof(double) * 4 * na, cudaMemcpyDeviceToDevice, d->stream));
      GH_CUDA(d, cudaMemcpyAsync(dH + dhoff + (size_t)ir * 12 * na, sh.gauge + (size_t)ir * gh::NGAUGE * na + 4 * na,
                                 sizeof(double) * 12 * na, cudaMemcpyDeviceToDevice, d->stream));
    }
    hoff += (long long)sh.n_r * 4 * na;
    dhoff += (long long)sh.n_r * 12 * na;
  }
  return GH_OK;
}

gh_status gh_set_background(gh_domain* d, const double* u_bg) {
  if (!d || !u_bg) return fail(d, GH_EINVAL, "null argument");
  GH_CUDA(d, gh::launch_bc_background(d, u_bg, -1));
  return GH_OK;
}

gh_status gh_add_perturbation(gh_domain* d, int kind, double A, double Rc, double w, int lmax,
                              const double* coeffs, double* u) {
  if (!d || !u || !coeffs) return fail(d, GH_EINVAL, "null argument");
  if (kind != 0 && kind != 1) return fail(d, GH_EINVAL, "kind must be 0 or 1");
  if (lmax < 0 || lmax > 16 || !(w > 0.0)) return fail(d, GH_EINVAL, "need 0 <= lmax <= 16 and w > 0");
  const size_t n = (size_t)(lmax + 1) * (lmax + 1);
  double* cd = nullptr;
  GH_CUDA(d, cudaMallocAsync(&cd, sizeof(double) * n, d->stream));
  GH_CUDA(d, cudaMemcpyAsync(cd, coeffs, sizeof(double) * n, cudaMemcpyHostToDevice, d->stream));
  GH_CUDA(d, gh::launch_perturbation(d, kind, A, Rc, w, lmax, cd, u));
  GH_CUDA(d, cudaFreeAsync(cd, d->stream));
  return GH_OK;
}

// The moving frame at the domain clock for one evaluation (no-op when static);
// a general map's gauge source and boundary background for it.
gh_status frame_now(gh_domain* d) {
  if (!gh::frame_moving(d)) return GH_OK;
  const double off = 0.0;
  GH_CUDA(d, gh::launch_frames(d, &off, 1, 0.0));
  d->frd = d->frames_d;
  GH_CUDA(d, gh::launch_map_stage(d));
  return GH_OK;
}

gh_status gh_derivatives(gh_domain* d, const double* u, double* du) {
  if (!d || !u || !du) return fail(d, GH_EINVAL, "null argument");
  if (gh_status s = check_latched(d)) return s;
  if (gh_status s = derivatives(d, u)) return s;
  if (gh_status s = frame_now(d)) return s;
  GH_CUDA(d, gh::launch_cartesian(d, u, du));
  return GH_OK;
}

gh_status gh_rhs(gh_domain* d, const double* u, double* dudt) {
  if (!d || !u || !dudt) return fail(d, GH_EINVAL, "null argument");
  if (u == dudt) return fail(d, GH_EINVAL, "u and dudt must not overlap");
  if (gh_status s = check_latched(d)) return s;
  if (gh_status s = frame_now(d)) return s;
  if (gh_status s = derivatives(d, u)) return s;
  {
    ProfScope p(d, GH_K_POINTWISE);
    GH_CUDA(d, gh::launch_pointwise(d, u, dudt, 0, 0.0, nullptr, nullptr, nullptr, false));
  }
  {
    ProfScope p(d, GH_K_BC);
    GH_CUDA(d, gh::launch_bc(d, dudt, 0, 0.0, nullptr, nullptr, nullptr, u));
  }
  return GH_OK;
}

// One RK4 step; with stages != NULL the three intermediate stage states
// u_n + dt/2 k1, u_n + dt/2 k2, u_n + dt k3 are written there (and used as the
// stage buffers) instead of the work area.
gh_status rotation_guard(gh_domain* d) {
  if (!gh::frame_moving(d)) return GH_OK;
  for (const auto& sh : d->shells_h)
    if (sh.dt_scale != 1.0) return fail(d, GH_ENOTSUP, "the rotating frame needs dt_scale = 1 on every shell");
  return GH_OK;
}

// host_in / host_out (host-memory step, device-visible pinned buffers): the
// stage-1 radial map reads u_n from host_in and writes its device image to u,
// the angular maps then read u; the last filter writes u_{n+1} to host_out
// (u keeps u_n).  Both NULL: the device step.
gh_status rk4_step_impl(gh_domain* d, double dt, double* u, double* work, double* norm2_pre, double* stages,
                        const double* host_in, double* host_out) {
  if (gh_status s = rotation_guard(d)) return s;
  static const int fidx[4] = {0, 1, 1, 2};     // stage times t, t + dt/2, t + dt/2, t + dt
  double* us = work;
  double* k = work + d->state;
  double* acc = work + 2 * d->state;
  const bool filt = d->params.radial_filter_on || d->params.sh_keep_l != -1;
  if (gh::frame_moving(d)) {
    // the step's frames from the device clock, which then advances by dt
    // (gh_rk4_step only: the adjoint's recomputation leaves the clock alone)
    const double off[3] = {0.0, 0.5 * dt, dt};
    GH_CUDA(d, gh::launch_frames(d, off, 3, stages ? 0.0 : dt));
  }
  for (int stage = 1; stage <= 4; ++stage) {
    const double* in = (stage == 1) ? u : (stages ? stages + (stage - 2) * d->state : us);
    d->frd = d->frames_d ? d->frames_d + fidx[stage - 1] : nullptr;
    if (d->map_gen && (stage != 3)) GH_CUDA(d, gh::launch_map_stage(d));   // stage 3 shares stage 2's time
    if (stage == 1 && host_in) {
      {
        ProfScope p(d, GH_K_RADIAL);
        GH_CUDA(d, gh::launch_radial_on(d, host_in, d->d_r, false, d->stream, u));
      }
      ProfScope p(d, GH_K_ANGULAR);
      GH_CUDA(d, gh::launch_angular_deriv(d, u));
    } else if (gh_status s = derivatives(d, in)) {
      return s;
    }
    double* target = (stage == 4) ? (filt ? us : u) : (stages ? stages + (stage - 1) * d->state : us);
    {
      ProfScope p(d, GH_K_POINTWISE);
      GH_CUDA(d, gh::launch_pointwise(d, in, k, stage, dt, u, acc, target, stage == 1 && norm2_pre));
    }
    if (stage == 1 && norm2_pre) {
      ProfScope p(d, GH_K_REDUCE);
      GH_CUDA(d, gh::launch_norm_reduce(d, norm2_pre));
    }
    {
      ProfScope p(d, GH_K_BC);
      GH_CUDA(d, gh::launch_bc(d, k, stage, dt, u, acc, target, in));
    }
  }
  if (filt) {
    if (gh_status s = filters(d, us, u, k, host_out)) return s;
  } else if (host_out) {
    GH_CUDA(d, cudaMemcpyAsync(host_out, u, sizeof(double) * d->state, cudaMemcpyDefault, d->stream));
  }
  if (!stages) d->time += dt;   // gh_rk4_step advances the clock; the adjoint's recomputation does not
  return GH_OK;
}

gh_status gh_rk4_step(gh_domain* d, double dt, double* u, double* work, double* norm2_pre) {
  if (!d || !u || !work) return fail(d, GH_EINVAL, "null argument");
  if (gh_status s = check_latched(d)) return s;
  return rk4_step_impl(d, dt, u, work, norm2_pre, nullptr);
}

gh_status gh_rk4_step_host(gh_domain* d, double dt, int n_steps, const double* u_in, double* u_out,
                           double* norm2_out) {
  if (!d || !u_in || !u_out) return fail(d, GH_EINVAL, "null argument");
  if (n_steps < 1) return fail(d, GH_EINVAL, "need n_steps >= 1");
  if (gh_status s = check_latched(d)) return s;
  const size_t bytes = sizeof(double) * (size_t)d->state;
  if (!d->host_u || !d->host_work || !d->host_norm) {
    // All three buffers or none: a failed allocation leaves the domain without
    // any, so the next call allocates again instead of launching on a null
    // buffer (what did get allocated is freed with the domain).
    void* pu = nullptr;
    void* pw = nullptr;
    void* pn = nullptr;
    GH_CUDA(d, alloc_zero(d, bytes, &pu));
    if (fault_injected("host_alloc")) return fail(d, GH_ENOMEM, "GH_FAULT=host_alloc: injected allocation failure");
    GH_CUDA(d, alloc_zero(d, 3 * bytes, &pw));
    GH_CUDA(d, alloc_zero(d, sizeof(double) * (size_t)d->n_shells, &pn));
    d->host_u = (double*)pu;
    d->host_work = (double*)pw;
    d->host_norm = (double*)pn;
  }
  const int want_norm = norm2_out ? 1 : 0;
  // One step with both buffers in pinned (device-visible) host memory and a
  // filter at the end of the step: the step's own kernels move the state, the
  // stage-1 radial map reading u_n from u_in and the last filter writing
  // u_{n+1} to u_out, so the link transfers overlap the FP64 work of those
  // kernels instead of preceding and following the step.
  const bool filt = d->params.radial_filter_on || d->params.sh_keep_l != -1;
  const double* hin = nullptr;
  double* hout = nullptr;
  if (n_steps == 1 && filt) {
    hin = device_view(u_in);
    hout = device_view(u_out);
    if (!hin || !hout) hin = hout = nullptr;
  }
  if (hin) {
    if (!d->host_graph_io || d->host_graph_io_dt != dt || d->host_graph_io_norm != want_norm ||
        d->host_graph_io_in != hin || d->host_graph_io_out != hout) {
      if (d->host_graph_io) {
        cudaGraphExecDestroy(d->host_graph_io);
        d->host_graph_io = nullptr;
      }
      if (gh_status s = capture_step(d, dt, d->host_u, d->host_work, want_norm ? d->host_norm : nullptr,
                                     &d->host_graph_io, &d->host_graph_io_launches, hin, hout))
        return s;
      d->host_graph_io_dt = dt;
      d->host_graph_io_norm = want_norm;
      d->host_graph_io_in = hin;
      d->host_graph_io_out = hout;
    }
    GH_CUDA(d, cudaGraphLaunch(d->host_graph_io, d->stream));
    d->launches += d->host_graph_io_launches;
    d->time += dt;
    if (norm2_out)
      GH_CUDA(d, cudaMemcpyAsync(norm2_out, d->host_norm, sizeof(double) * (size_t)d->n_shells,
                                 cudaMemcpyDeviceToHost, d->stream));
    GH_CUDA(d, cudaStreamSynchronize(d->stream));
    return GH_OK;
  }
  // otherwise copies around the step as a captured graph on the domain's own
  // buffers (captured once per dt and norm choice, and again after a setter
  // changes the step's launches)
  if (!d->host_graph || d->host_graph_dt != dt || d->host_graph_norm != want_norm) {
    if (gh_status s = capture_step(d, dt, d->host_u, d->host_work, want_norm ? d->host_norm : nullptr,
                                   &d->host_graph, &d->host_graph_launches))
      return s;
    d->host_graph_dt = dt;
    d->host_graph_norm = want_norm;
  }
  GH_CUDA(d, cudaMemcpyAsync(d->host_u, u_in, bytes, cudaMemcpyHostToDevice, d->stream));
  for (int i = 0; i < n_steps; ++i) {
    GH_CUDA(d, cudaGraphLaunch(d->host_graph, d->stream));
    d->launches += d->host_graph_launches;
    d->time += dt;                       // each replay advances the device clock by dt
  }
  GH_CUDA(d, cudaMemcpyAsync(u_out, d->host_u, bytes, cudaMemcpyDeviceToHost, d->stream));
  if (norm2_out)
    GH_CUDA(d, cudaMemcpyAsync(norm2_out, d->host_norm, sizeof(double) * (size_t)d->n_shells,
                               cudaMemcpyDeviceToHost, d->stream));
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  return GH_OK;
}

gh_status gh_rk4_step_save(gh_domain* d, double dt, double* u, double* work, double* norm2_pre, double* stages) {
  if (!d || !u || !work || !stages) return fail(d, GH_EINVAL, "null argument");
  if (gh_status s = check_latched(d)) return s;
  return rk4_step_impl(d, dt, u, work, norm2_pre, stages);
}

long long gh_dp5_work_size(const gh_domain* d) { return d ? 9LL * (long long)d->state : 0; }

gh_status gh_dp5_step(gh_domain* d, double dt, double rtol, double atol, double* u, double* work,
                      double* err_out, int* accepted, double* dt_next) {
  if (!d || !u || !work || !err_out || !accepted || !dt_next) return fail(d, GH_EINVAL, "null argument");
  if (!(dt > 0.0) || !(rtol >= 0.0) || !(atol >= 0.0) || (rtol == 0.0 && atol == 0.0))
    return fail(d, GH_EINVAL, "need dt > 0, rtol >= 0, atol >= 0, not both tolerances zero");
  for (const auto& sh : d->shells_h)
    if (sh.dt_scale != 1.0) return fail(d, GH_ENOTSUP, "the Dormand-Prince step needs dt_scale = 1 on every shell");
  if (gh_status s = check_latched(d)) return s;
  if (gh_status s = rotation_guard(d)) return s;
  static const double cdp[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
  // Dormand & Prince (1980) pair: stage matrix rows 2..7 (row 7 = b) and b - b_hat
  static const double A[7][6] = {
      {0, 0, 0, 0, 0, 0},
      {1.0 / 5, 0, 0, 0, 0, 0},
      {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
      {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
      {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
      {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
      {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
  static const double bh[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640, -92097.0 / 339200, 187.0 / 2100,
                               1.0 / 40};
  const long long N = d->state;
  double* k[7];
  for (int j = 0; j < 7; ++j) k[j] = work + j * N;
  double* ustage = work + 7 * N;
  double* unew = work + 8 * N;
  if (gh::frame_moving(d)) {
    double off[7];
    for (int s = 0; s < 7; ++s) off[s] = cdp[s] * dt;
    GH_CUDA(d, gh::launch_frames(d, off, 7, 0.0));
  }
  for (int s = 0; s < 7; ++s) {
    const double* in = (s == 0) ? u : (s == 6 ? unew : ustage);
    d->frd = d->frames_d ? d->frames_d + s : nullptr;
    GH_CUDA(d, gh::launch_map_stage(d));
    if (gh_status st = derivatives(d, in)) return st;
    {
      ProfScope p(d, GH_K_POINTWISE);
      GH_CUDA(d, gh::launch_pointwise(d, in, k[s], 0, 0.0, nullptr, nullptr, nullptr, false));
    }
    {
      ProfScope p(d, GH_K_BC);
      GH_CUDA(d, gh::launch_bc(d, k[s], 0, 0.0, nullptr, nullptr, nullptr, in));
    }
    if (s < 6) {
      // next stage state (s = 5 gives the fifth-order solution, row 7 = b)
      gh::LinComb lc;
      lc.nk = s + 1;
      for (int j = 0; j <= s; ++j) {
        lc.k[j] = k[j];
        lc.c[j] = dt * A[s + 1][j];
      }
      ProfScope p(d, GH_K_COMBINE);
      GH_CUDA(d, gh::launch_dp5_lincomb(d, u, lc, s == 5 ? unew : ustage));
    }
  }
  {
    gh::LinComb lc;
    lc.nk = 7;
    for (int j = 0; j < 7; ++j) {
      lc.k[j] = k[j];
      lc.c[j] = dt * ((j < 6 ? A[6][j] : 0.0) - bh[j]);
    }
    ProfScope p(d, GH_K_COMBINE);
    GH_CUDA(d, gh::launch_dp5_error(d, u, unew, lc, rtol, atol, d->dp_err));
  }
  double err = 0.0;
  GH_CUDA(d, cudaMemcpyAsync(&err, d->dp_err, sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  const bool ok = err <= 1.0;
  // controller: dt min(5, max(0.2, 0.9 err^(-1/5))), 5 when err = 0
  const double fac = (err == 0.0) ? 5.0 : std::min(5.0, std::max(0.2, 0.9 * std::pow(err, -0.2)));
  *err_out = err;
  *accepted = ok ? 1 : 0;
  *dt_next = dt * fac;
  if (ok) {
    d->time += dt;
    GH_CUDA(d, gh::launch_frames(d, nullptr, 0, dt));     // the device clock follows
    const bool filt = d->params.radial_filter_on || d->params.sh_keep_l != -1;
    if (filt) {
      if (gh_status st = filters(d, unew, u, ustage)) return st;
    } else {
      GH_CUDA(d, cudaMemcpyAsync(u, unew, sizeof(double) * N, cudaMemcpyDeviceToDevice, d->stream));
    }
  }
  return GH_OK;
}

gh_status gh_apply_filters(gh_domain* d, double* u, double* work) {
  if (!d || !u || !work) return fail(d, GH_EINVAL, "null argument");
  if (gh_status s = check_latched(d)) return s;
  return filters(d, u, u, work);
}

gh_status gh_constraints(gh_domain* d, const double* u, double* c_out, double* norm2) {
  if (!d || !u || !norm2) return fail(d, GH_EINVAL, "null argument");
  if (gh_status s = check_latched(d)) return s;
  if (gh_status s = frame_now(d)) return s;
  if (gh_status s = derivatives(d, u)) return s;
  GH_CUDA(d, gh::launch_constraints(d, u, c_out));
  GH_CUDA(d, gh::launch_norm_reduce(d, norm2));
  return GH_OK;
}

gh_status gh_set_algorithm(gh_domain* d, int algorithm) {
  if (!d || (algorithm != GH_ALG_DENSE && algorithm != GH_ALG_SEPARABLE && algorithm != GH_ALG_SEPARABLE_FOLDED))
    return fail(d, GH_EINVAL, "algorithm must be GH_ALG_DENSE, GH_ALG_SEPARABLE or GH_ALG_SEPARABLE_FOLDED");
  if (algorithm == GH_ALG_SEPARABLE_FOLDED && !d->fold_ok)
    return fail(d, GH_EINVAL, "the folded maps are not available on this domain");
  if (algorithm == GH_ALG_DENSE) {
    GH_CUDA(d, cudaStreamSynchronize(d->stream));
    if (gh_status st = build_dense(d)) return st;
  }
  d->algorithm = algorithm;
  invalidate_host_graph(d);
  return GH_OK;
}


gh_status gh_get_schedule(const gh_domain* d, int* v, int n) {
  if (!d || !v || n < GH_SCHEDULE_LEN) return GH_EINVAL;
  v[0] = d->rad_chains; v[1] = d->rad_groups; v[2] = d->radf_chains; v[3] = d->radf_groups;
  v[4] = d->fd_threads; v[5] = d->fd_budget; v[6] = d->ff_threads; v[7] = d->ff_budget;
  v[8] = d->adj_pair_split ? 1 : 0;
  return GH_OK;
}

gh_status gh_set_schedule(gh_domain* d, const int* v, int n) {
  if (!d) return GH_EINVAL;
  if (!v || n < GH_SCHEDULE_LEN || !schedule_ok(v)) return fail(d, GH_EINVAL, "invalid schedule");
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  d->rad_chains = v[0]; d->rad_groups = v[1]; d->radf_chains = v[2]; d->radf_groups = v[3];
  d->fd_threads = v[4]; d->fd_budget = v[5]; d->ff_threads = v[6]; d->ff_budget = v[7];
  d->adj_pair_split = v[8] != 0;
  if (d->fold_ok) GH_CUDA(d, fold_build_maps(d));
  invalidate_graph(d);
  return GH_OK;
}

gh_status gh_autotune(gh_domain* d, int reps) {
  if (!d) return GH_EINVAL;
  if (reps < 1) return fail(d, GH_EINVAL, "reps must be >= 1");
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  const double* in = d->d_r;
  double* o1 = d->d_th;
  double* o2 = d->d_ph;
  float ms = 0.f;
  // radial derivative and radial filter: FMA chains per pass x row groups
  for (int filter = 0; filter < 2; ++filter) {
    int& ch = filter ? d->radf_chains : d->rad_chains;
    int& gr = filter ? d->radf_groups : d->rad_groups;
    float best = 1e30f;
    int bc = ch, bg = gr;
    for (int c = 2; c <= 4; ++c)
      for (int g = 1; g <= 4; ++g) {
        ch = c;
        gr = g;
        GH_CUDA(d, time_calls(d, reps, [&] { return gh::launch_radial(d, in, o1, filter != 0); }, &ms));
        if (ms < best) { best = ms; bc = c; bg = g; }
      }
    ch = bc;
    gr = bg;
  }
  // folded angular maps: threads per block x shared-memory budget per block
  if (d->fold_ok) {
    const int threads[] = {128, 256, 384, 512};
    const int budgets[] = {16 * 1024,  24 * 1024,  32 * 1024,  48 * 1024, 64 * 1024,
                           96 * 1024, 112 * 1024, 160 * 1024, 200 * 1024};
    bool any_filter = false;
    for (const auto& sh : d->shells_h) any_filter = any_filter || sh.ff.M > 0;
    for (int filter = 0; filter < (any_filter ? 2 : 1); ++filter) {
      int& th = filter ? d->ff_threads : d->fd_threads;
      int& bu = filter ? d->ff_budget : d->fd_budget;
      float best = 1e30f;
      int bt = th, bb = bu;
      for (int t : threads)
        for (int b : budgets) {
          th = t;
          bu = b;
          GH_CUDA(d, fold_build_maps(d));
          if (filter)
            GH_CUDA(d, time_calls(d, reps, [&] { return gh::launch_fold_filter(d, in, o1); }, &ms));
          else
            GH_CUDA(d, time_calls(d, reps, [&] { return gh::launch_fold_deriv(d, in, o1, o2); }, &ms));
          if (ms < best) { best = ms; bt = t; bb = b; }
        }
      th = bt;
      bu = bb;
    }
    GH_CUDA(d, fold_build_maps(d));
  }
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  invalidate_graph(d);
  return GH_OK;
}

gh_status gh_set_rotating_frame(gh_domain* d, const double axis[3], double omega) {
  if (!d || !axis) return GH_EINVAL;
  const double n = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
  if (!(n > 0.0) || !std::isfinite(omega)) return fail(d, GH_EINVAL, "need a nonzero axis and a finite rate");
  if (omega != 0.0 && d->outer_bc == GH_BC_CONSTRAINT_PRESERVING_FULL)
    return fail(d, GH_ENOTSUP, "the u^- constraint part of the outer condition is defined on a static grid");
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  for (int i = 0; i < 3; ++i) d->rot_axis[i] = axis[i];
  d->rot_omega = omega;
  d->map_gen = false;                   // a rotation alone (stored background rotated)
  d->map_adot = 0.0;
  for (int i = 0; i < 3; ++i) d->map_V[i] = 0.0;
  d->fr = gh::frame_at(d, d->time);
  d->frd = nullptr;
  if (omega != 0.0 && !d->clock_d) {
    void* p = nullptr;
    GH_CUDA(d, cudaMalloc(&p, sizeof(double)));
    d->owned.push_back(p);
    d->clock_d = (double*)p;
    GH_CUDA(d, cudaMalloc(&p, sizeof(gh::Frame) * 8));
    d->owned.push_back(p);
    d->frames_d = (gh::Frame*)p;
  }
  if (d->clock_d) GH_CUDA(d, cudaMemcpy(d->clock_d, &d->time, sizeof(double), cudaMemcpyHostToDevice));
  invalidate_graph(d);
  return GH_OK;
}

gh_status gh_set_frame_map(gh_domain* d, const double axis[3], double omega, double adot, const double V[3]) {
  if (!d || !axis || !V) return GH_EINVAL;
  const double n = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
  if (!(n > 0.0) || !std::isfinite(omega) || !std::isfinite(adot) || !std::isfinite(V[0]) || !std::isfinite(V[1]) ||
      !std::isfinite(V[2]))
    return fail(d, GH_EINVAL, "need a nonzero axis and finite rates");
  if (d->outer_bc == GH_BC_CONSTRAINT_PRESERVING_FULL)
    return fail(d, GH_ENOTSUP, "the u^- constraint part of the outer condition is defined on a static grid");
  for (const auto& sh : d->shells_h)
    if (4 * (size_t)sh.bh + 3 >= d->holes.size() || !(d->holes[4 * sh.bh] > 0.0))
      return fail(d, GH_EINVAL, "the map evaluates each hole at the moving points: set every hole with "
                                "gh_set_analytic_kerr_schild first");
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  if (!d->map_buf) {
    long long nd = 0;
    for (const auto& sh : d->shells_h) nd += (long long)sh.n_r * gh::NGAUGE * sh.na;
    for (const auto& sl : d->bc_h) nd += 11LL * sl.na;
    void* p = nullptr;
    GH_CUDA(d, alloc_zero(d, sizeof(double) * (size_t)nd, &p));
    d->map_buf = (double*)p;
    double* q = d->map_buf;
    for (auto& sh : d->shells_h) {
      sh.gauge_t = q;
      q += (long long)sh.n_r * gh::NGAUGE * sh.na;
    }
    for (auto& sl : d->bc_h) {
      sl.bg_t = q;
      q += 11LL * sl.na;
    }
    GH_CUDA(d, cudaMemcpy(d->shells_d, d->shells_h.data(), sizeof(gh::ShellDev) * d->shells_h.size(),
                          cudaMemcpyHostToDevice));
    if (!d->bc_h.empty())
      GH_CUDA(d, cudaMemcpy(d->bc_d, d->bc_h.data(), sizeof(gh::BcSliceDev) * d->bc_h.size(), cudaMemcpyHostToDevice));
    std::vector<int> begin(d->n_shells + 1);
    int blocks = 0;
    for (int s = 0; s < d->n_shells; ++s) {
      begin[s] = blocks;
      blocks += d->shells_h[s].n_r * ((d->shells_h[s].na + 63) / 64);
    }
    begin[d->n_shells] = blocks;
    d->map_blocks = blocks;
    GH_CUDA(d, upload(d, begin, &d->map_pt_begin_d));
    GH_CUDA(d, upload(d, d->holes, &d->holes_d));   // one slot per hole of the domain: its size never changes
    GH_CUDA(d, alloc_zero(d, sizeof(gh::MapGate), &p));
    d->map_gate_d = (gh::MapGate*)p;
  } else {
    GH_CUDA(d, cudaMemcpy(d->holes_d, d->holes.data(), sizeof(double) * d->holes.size(), cudaMemcpyHostToDevice));
  }
  GH_CUDA(d, cudaMemset(d->map_gate_d, 0, sizeof(gh::MapGate)));   // new map: nothing evaluated yet
  if (!d->clock_d) {
    void* p = nullptr;
    GH_CUDA(d, cudaMalloc(&p, sizeof(double)));
    d->owned.push_back(p);
    d->clock_d = (double*)p;
    GH_CUDA(d, cudaMalloc(&p, sizeof(gh::Frame) * 8));
    d->owned.push_back(p);
    d->frames_d = (gh::Frame*)p;
  }
  for (int i = 0; i < 3; ++i) {
    d->rot_axis[i] = axis[i];
    d->map_V[i] = V[i];
  }
  d->rot_omega = omega;
  d->map_adot = adot;
  d->map_gen = true;
  d->fr = gh::frame_at(d, d->time);
  d->frd = nullptr;
  GH_CUDA(d, cudaMemcpy(d->clock_d, &d->time, sizeof(double), cudaMemcpyHostToDevice));
  invalidate_graph(d);
  return GH_OK;
}

gh_status gh_set_time(gh_domain* d, double t) {
  if (!d || !std::isfinite(t)) return GH_EINVAL;
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  d->time = t;
  if (d->clock_d) GH_CUDA(d, cudaMemcpy(d->clock_d, &d->time, sizeof(double), cudaMemcpyHostToDevice));
  return GH_OK;
}

gh_status gh_get_time(const gh_domain* d, double* t) {
  if (!d || !t) return GH_EINVAL;
  *t = d->time;
  return GH_OK;
}

gh_status gh_set_outer_bc(gh_domain* d, int mode) {
  if (!d) return GH_EINVAL;
  if (mode != GH_BC_FREEZE && mode != GH_BC_CONSTRAINT_PRESERVING && mode != GH_BC_CONSTRAINT_PRESERVING_FULL)
    return fail(d, GH_EINVAL,
                "mode must be GH_BC_FREEZE, GH_BC_CONSTRAINT_PRESERVING or GH_BC_CONSTRAINT_PRESERVING_FULL");
  if (mode == GH_BC_CONSTRAINT_PRESERVING_FULL && gh::frame_moving(d))
    return fail(d, GH_ENOTSUP, "the u^- constraint part of the outer condition is defined on a static grid");
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  if (mode == GH_BC_CONSTRAINT_PRESERVING_FULL && !d->cpm_S && d->bc_points) {
    void* p = nullptr;
    GH_CUDA(d, alloc_zero(d, sizeof(double) * 10 * (size_t)d->bc_points, &p));
    d->cpm_S = (double*)p;
  }
  d->outer_bc = mode;
  invalidate_graph(d);
  return GH_OK;
}

gh_status gh_set_sh_filter(gh_domain* d, int mode) {
  if (!d) return GH_EINVAL;
  if (mode != GH_SH_FILTER_COMPONENT && mode != GH_SH_FILTER_TENSOR)
    return fail(d, GH_EINVAL, "mode must be GH_SH_FILTER_COMPONENT or GH_SH_FILTER_TENSOR");
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  if (mode == GH_SH_FILTER_TENSOR && !d->tf_buf && d->params.sh_keep_l != -1) {
    std::vector<std::vector<double>> xs, ws;
    for (const auto& sh : d->shells_h) {
      const AngularGrid ag = angular_grid(sh.L);
      xs.push_back(ag.ct);
      ws.push_back(ag.wgl);
    }
    GH_CUDA(d, gh::tensor_filter_prepare(d, xs, ws));
  }
  d->sh_filter_mode = mode;
  invalidate_graph(d);
  return GH_OK;
}

gh_status gh_profile_enable(gh_domain* d, int on) {
  if (!d) return GH_EINVAL;
  d->prof = on != 0;
  return GH_OK;
}

gh_status gh_profile_read(gh_domain* d, int family, double* total_ms, long long* launches) {
  if (!d || !total_ms || !launches || family < 0 || family >= GH_K_FAMILIES)
    return fail(d, GH_EINVAL, "bad profiler arguments");
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  std::vector<gh_domain::Bracket> keep;
  for (auto& b : d->pending) {
    float ms = 0.f;
    GH_CUDA(d, cudaEventElapsedTime(&ms, b.a, b.b));
    d->prof_ms[b.fam] += ms;
    d->prof_n[b.fam] += 1;
    d->event_pool.push_back(b.a);
    d->event_pool.push_back(b.b);
  }
  d->pending.clear();
  *total_ms = d->prof_ms[family];
  *launches = d->prof_n[family];
  d->prof_ms[family] = 0.0;
  d->prof_n[family] = 0;
  return GH_OK;
}

gh_status gh_sync(gh_domain* d) {
  if (!d) return GH_EINVAL;
  GH_CUDA(d, cudaStreamSynchronize(d->stream));
  int flag = 0;
  GH_CUDA(d, cudaMemcpy(&flag, d->err_flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    GH_CUDA(d, cudaMemset(d->err_flag, 0, sizeof(int)));
    return fail(d, (gh_status)flag, "device reported a non-finite constraint norm");
  }
  return GH_OK;
}

}  // extern "C"
