// The directional derivative of the gauge constraint C_a = H_a + psi^bc Gamma_abc
// that the u^- part of the constraint-preserving outer condition uses, and its
// reverse mode.  A state type ST carries, at one point:
//   u[50]        the fields (psi 0..9, Pi 10..19, Phi_i 20 + 10 i ..),
//   psi_inv[10]  psi^ab packed, N the lapse, t_up[3] = t^i = -N psi^0i,
//   beta[3]      beta^i = N^2 psi^0i,
//   D[40]        d_c psi_ab reconstructed as t_c Pi_ab + g^i_c Phi_iab:
//                D_0ab = -N Pi_ab + beta^i Phi_iab, D_jab = Phi_jab (D[c * 10 + pair]).
#pragma once
#include "gh_tensor.cuh"

namespace gh {

// E_a = X^bc (Y_bac - Y_abc / 2) for a symmetric X^bc and Y[c][pair(a, b)]:
// psi^bc Gamma_abc for Y = D (psi^bc is symmetric, so the two Gamma terms
// that swap b and c contribute equally).  The second sum runs over the ten
// pairs (off-diagonal ones twice).
__device__ __forceinline__ void contract_gamma(const double* X, const double* Y, double out[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) s1 = fma(X[sym_index(b, c)], Y[b * 10 + sym_index(a, c)], s1);
#pragma unroll
    for (int p = 0; p < 10; ++p) s2 = fma(pair_a(p) == pair_b(p) ? X[p] : 2.0 * X[p], Y[a * 10 + p], s2);
    out[a] = fma(-0.5, s2, s1);
  }
}

// Reverse of contract_gamma: Xb += d<ob, E>/dX, Yb += d<ob, E>/dY (either may be null).
__device__ __forceinline__ void contract_gamma_rev(const double* X, const double* Y, const double ob[4], double* Xb,
                                                   double* Yb) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double o = ob[a];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (Xb) Xb[sym_index(b, c)] = fma(o, Y[b * 10 + sym_index(a, c)], Xb[sym_index(b, c)]);
        if (Yb) Yb[b * 10 + sym_index(a, c)] = fma(o, X[sym_index(b, c)], Yb[b * 10 + sym_index(a, c)]);
      }
#pragma unroll
    for (int p = 0; p < 10; ++p) {
      const double w = (pair_a(p) == pair_b(p) ? -0.5 : -1.0) * o;
      if (Xb) Xb[p] = fma(w, Y[a * 10 + p], Xb[p]);
      if (Yb) Yb[a * 10 + p] = fma(w, X[p], Yb[a * 10 + p]);
    }
  }
}

// The parts of C'_a along a field-space direction v (50 fields: psi', Pi',
// Phi') that the reverse mode reuses.
struct CDirParts {
  double Mi[4][4];   // psi^ac psi'_cd
  double dpi[10];    // psi'^ab = -psi^ac psi'_cd psi^db
  double dN;         // N' = N^3 psi'^00 / 2
  double dt[3];      // t'^i = -N' psi^0i - N psi'^0i
  double g0[3];      // g'^i_0 = -N t'^i - N' t^i
  double Dp[40];     // D'_0ab = -N' Pi_ab - N Pi'_ab + g'^i_0 Phi_iab + beta^i Phi'_iab, D'_jab = Phi'_jab
};

template <class ST>
__device__ __forceinline__ void cdir_parts(const ST& s, const double* v, CDirParts& q) {
#pragma unroll
  for (int A = 0; A < 4; ++A)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      double acc = 0.0;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc = fma(s.psi_inv[sym_index(A, c)], v[sym_index(c, e)], acc);
      q.Mi[A][e] = acc;
    }
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < 4; ++e) acc = fma(q.Mi[A][e], s.psi_inv[sym_index(e, B)], acc);
    q.dpi[p] = -acc;
  }
  const double N = s.N;
  q.dN = 0.5 * N * N * N * q.dpi[0];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    q.dt[i] = -q.dN * s.psi_inv[sym_index(0, 1 + i)] - N * q.dpi[sym_index(0, 1 + i)];
    q.g0[i] = -N * q.dt[i] - q.dN * s.t_up[i];
  }
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    double w = -q.dN * s.u[10 + p] - N * v[10 + p];
#pragma unroll
    for (int i = 0; i < 3; ++i) w = fma(q.g0[i], s.u[20 + 10 * i + p], fma(s.beta[i], v[20 + 10 * i + p], w));
    q.Dp[p] = w;
#pragma unroll
    for (int j = 0; j < 3; ++j) q.Dp[(1 + j) * 10 + p] = v[20 + 10 * j + p];
  }
}

// C'_a, the derivative of C_a along (v, dH), by the product rule:
// C'_a = H'_a + psi'^bc (D_bac - D_abc / 2) + psi^bc (D'_bac - D'_abc / 2).
template <class ST>
__device__ __noinline__ void gauge_constraint_dir(const ST& s, const double* v, const double dH[4], double out[4]) {
  CDirParts q;
  cdir_parts(s, v, q);
  double e1[4], e2[4];
  contract_gamma(q.dpi, s.D, e1);
  contract_gamma(s.psi_inv, q.Dp, e2);
#pragma unroll
  for (int a = 0; a < 4; ++a) out[a] = dH[a] + e1[a] + e2[a];
}

// Cotangents of the state's split and of its fields.
struct CStateBar {
  double u[50];
  double psi_inv[10];
  double N;
  double t_up[3];
  double beta[3];
  double D[40];
};

// Reverse of gauge_constraint_dir for a cotangent ob of its output: adds to
// the state's cotangents sb and, when vb is not null, to the direction's.
template <class ST>
__device__ __noinline__ void gauge_constraint_dir_rev(const ST& s, const double* v, const double ob[4],
                                                      CStateBar& sb, double* vb) {
  CDirParts q;
  cdir_parts(s, v, q);
  double dpib[10], Dpb[40];
#pragma unroll
  for (int p = 0; p < 10; ++p) dpib[p] = 0.0;
#pragma unroll
  for (int e = 0; e < 40; ++e) Dpb[e] = 0.0;
  contract_gamma_rev(q.dpi, s.D, ob, dpib, sb.D);
  contract_gamma_rev(s.psi_inv, q.Dp, ob, sb.psi_inv, Dpb);
  const double N = s.N;
  double dNb = 0.0, g0b[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int p = 0; p < 10; ++p) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (vb) vb[20 + 10 * j + p] += Dpb[(1 + j) * 10 + p];
    const double g = Dpb[p];
    dNb = fma(-s.u[10 + p], g, dNb);
    sb.u[10 + p] = fma(-q.dN, g, sb.u[10 + p]);
    sb.N = fma(-v[10 + p], g, sb.N);
    if (vb) vb[10 + p] = fma(-N, g, vb[10 + p]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      g0b[i] = fma(s.u[20 + 10 * i + p], g, g0b[i]);
      sb.u[20 + 10 * i + p] = fma(q.g0[i], g, sb.u[20 + 10 * i + p]);
      sb.beta[i] = fma(v[20 + 10 * i + p], g, sb.beta[i]);
      if (vb) vb[20 + 10 * i + p] = fma(s.beta[i], g, vb[20 + 10 * i + p]);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    // g0_i = -N dt_i - dN t_i
    sb.N = fma(-q.dt[i], g0b[i], sb.N);
    const double dtb = -N * g0b[i];
    dNb = fma(-s.t_up[i], g0b[i], dNb);
    sb.t_up[i] = fma(-q.dN, g0b[i], sb.t_up[i]);
    // dt_i = -dN psi^0i - N psi'^0i
    dNb = fma(-s.psi_inv[sym_index(0, 1 + i)], dtb, dNb);
    sb.psi_inv[sym_index(0, 1 + i)] = fma(-q.dN, dtb, sb.psi_inv[sym_index(0, 1 + i)]);
    sb.N = fma(-q.dpi[sym_index(0, 1 + i)], dtb, sb.N);
    dpib[sym_index(0, 1 + i)] = fma(-N, dtb, dpib[sym_index(0, 1 + i)]);
  }
  // dN = N^3 dpi_00 / 2
  sb.N = fma(1.5 * N * N * q.dpi[0], dNb, sb.N);
  dpib[0] = fma(0.5 * N * N * N, dNb, dpib[0]);
  // dpi_AB = -Mi[A][e] psi^eB;  Mi[A][e] = psi^Ac psi'_ce
  double Mib[4][4];
#pragma unroll
  for (int A = 0; A < 4; ++A)
#pragma unroll
    for (int e = 0; e < 4; ++e) Mib[A][e] = 0.0;
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      Mib[A][e] = fma(-dpib[p], s.psi_inv[sym_index(e, B)], Mib[A][e]);
      sb.psi_inv[sym_index(e, B)] = fma(-dpib[p], q.Mi[A][e], sb.psi_inv[sym_index(e, B)]);
    }
  }
#pragma unroll
  for (int A = 0; A < 4; ++A)
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        sb.psi_inv[sym_index(A, c)] = fma(Mib[A][e], v[sym_index(c, e)], sb.psi_inv[sym_index(A, c)]);
        if (vb) vb[sym_index(c, e)] = fma(Mib[A][e], s.psi_inv[sym_index(A, c)], vb[sym_index(c, e)]);
      }
}

// Reverse of the state's D, t^i, beta^i, N and psi^ab down to the fields:
// D_0ab = -N Pi_ab + beta^i Phi_iab, D_jab = Phi_jab; t^i = -N psi^0i,
// beta^i = N^2 psi^0i, N = (-psi^00)^(-1/2); psi^ab = (psi_ab)^-1 with
// d psi^ab = -psi^ac d psi_cd psi^db (a packed psi_cd, c != d, enters twice).
// Adds to sb.u[0..49]; consumes sb's split cotangents.
template <class ST>
__device__ __noinline__ void state_rev(const ST& s, CStateBar& sb) {
  const double N = s.N;
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    const double g = sb.D[p];
    sb.N = fma(-s.u[10 + p], g, sb.N);
    sb.u[10 + p] = fma(-N, g, sb.u[10 + p]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sb.beta[i] = fma(s.u[20 + 10 * i + p], g, sb.beta[i]);
      sb.u[20 + 10 * i + p] = fma(s.beta[i], g, sb.u[20 + 10 * i + p]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) sb.u[20 + 10 * j + p] += sb.D[(1 + j) * 10 + p];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double p0i = s.psi_inv[sym_index(0, 1 + i)];
    sb.N = fma(-p0i, sb.t_up[i], fma(2.0 * N * p0i, sb.beta[i], sb.N));
    sb.psi_inv[sym_index(0, 1 + i)] += -N * sb.t_up[i] + N * N * sb.beta[i];
  }
  sb.psi_inv[0] = fma(0.5 * N * N * N, sb.N, sb.psi_inv[0]);
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    const int a = pair_a(q), b = pair_b(q);
    const double g = sb.psi_inv[q];
#pragma unroll
    for (int p = 0; p < 10; ++p) {
      const int A = pair_a(p), B = pair_b(p);
      double d = s.psi_inv[sym_index(a, A)] * s.psi_inv[sym_index(B, b)];
      if (A != B) d = fma(s.psi_inv[sym_index(a, B)], s.psi_inv[sym_index(A, b)], d);
      sb.u[p] = fma(-g, d, sb.u[p]);
    }
  }
}

// The state's split (psi^ab, N, t^i, beta^i) and D_cab from s.u.
template <class ST>
__device__ __forceinline__ void cpm_state(ST& s) {
  double psi[10];
#pragma unroll
  for (int p = 0; p < 10; ++p) psi[p] = s.u[p];
  Split sp;
  spacetime_split(psi, sp);
#pragma unroll
  for (int p = 0; p < 10; ++p) s.psi_inv[p] = sp.psi_inv[p];
  s.N = sp.alpha;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    s.t_up[i] = sp.t_up[1 + i];
    s.beta[i] = sp.beta_up[i];
  }
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    double w = -s.N * s.u[10 + p];
#pragma unroll
    for (int i = 0; i < 3; ++i) w = fma(s.beta[i], s.u[20 + 10 * i + p], w);
    s.D[p] = w;
#pragma unroll
    for (int j = 0; j < 3; ++j) s.D[(1 + j) * 10 + p] = s.u[20 + 10 * j + p];
  }
}

// ------------------------------------------------------------ the u^- solve
// Background of an outer point (the freezing condition's fixed background):
// n_i, n^i, beta^i, g_ij packed (xx xy xz yy yz zz), lapse, n.beta.
struct CpmBg {
  double n_dn[3], n_up[3], bb[3], gb[6], Nb, nb;
};

__device__ __forceinline__ void cpm_load_bg(const double* bg, long long na, int q, CpmBg& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    b.n_dn[i] = bg[(long long)i * na + q];
    b.n_up[i] = bg[(long long)(3 + i) * na + q];
    b.bb[i] = bg[(long long)(7 + i) * na + q];
  }
  b.Nb = bg[(long long)6 * na + q];
#pragma unroll
  for (int m = 0; m < 6; ++m) b.gb[m] = bg[(long long)(10 + m) * na + q];
  b.nb = b.n_dn[0] * b.bb[0] + b.n_dn[1] * b.bb[1] + b.n_dn[2] * b.bb[2];
}

// The background's outgoing null vector l = (t + n)/sqrt 2 in both index
// positions (t_a = (-N, 0), t^a = (1, -beta^i)/N, n_a = (n.beta, n_i),
// n^a = (0, n^i)) and the projector P_ab = psi_ab + t_a t_b - n_a n_b.
__device__ __forceinline__ void cpm_tetrad(const CpmBg& b, double l_dn[4], double l_up[4], double P[10]) {
  const double r2 = 0.70710678118654752440;
  double bdn[3];   // beta_i
  bdn[0] = b.gb[0] * b.bb[0] + b.gb[1] * b.bb[1] + b.gb[2] * b.bb[2];
  bdn[1] = b.gb[1] * b.bb[0] + b.gb[3] * b.bb[1] + b.gb[4] * b.bb[2];
  bdn[2] = b.gb[2] * b.bb[0] + b.gb[4] * b.bb[1] + b.gb[5] * b.bb[2];
  const double n4[4] = {b.nb, b.n_dn[0], b.n_dn[1], b.n_dn[2]};
  l_dn[0] = r2 * (-b.Nb + b.nb);
  l_up[0] = r2 / b.Nb;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    l_dn[1 + i] = r2 * b.n_dn[i];
    l_up[1 + i] = r2 * (b.n_up[i] - b.bb[i] / b.Nb);
  }
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
    double psib;
    if (A == 0 && B == 0) psib = -b.Nb * b.Nb + b.bb[0] * bdn[0] + b.bb[1] * bdn[1] + b.bb[2] * bdn[2];
    else if (A == 0) psib = bdn[B - 1];
    else psib = b.gb[s3(A - 1, B - 1)];
    P[p] = psib + ((A == 0 && B == 0) ? b.Nb * b.Nb : 0.0) - n4[A] * n4[B];
  }
}

// Pair p of the time derivative with the u^psi and u^0 conditions (Bjorhus
// form, where incoming), u^+ frozen if incoming and w^- = 0 (into ud), and
// the interior w^- of pair p (into *wm).  kr is the interior right-hand side,
// u the state, du[i] its Cartesian derivatives.
__device__ __forceinline__ void cpm_pair(int p, const double* kr, const double* u, const double (*du)[50],
                                         const CpmBg& b, double gamma1, double gamma2, double* ud, double* wm) {
  const double v_psi = -(1.0 + gamma1) * b.nb, v_0 = -b.nb, v_p = -b.nb + b.Nb;
  const double ps = kr[p], pi = kr[10 + p];
  double ph[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) ph[i] = kr[20 + 10 * i + p];
  const double nphi = b.n_up[0] * ph[0] + b.n_up[1] * ph[1] + b.n_up[2] * ph[2];
  double wpsi = ps, wp = pi + nphi - gamma2 * ps, w0[3];
  *wm = pi - nphi - gamma2 * ps;
#pragma unroll
  for (int i = 0; i < 3; ++i) w0[i] = ph[i] - b.n_dn[i] * nphi;
  if (v_psi < 0.0) {
    double nC3 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) nC3 = fma(b.n_up[i], du[i][p] - u[20 + 10 * i + p], nC3);
    wpsi = fma(v_psi, nC3, wpsi);
  }
  if (v_0 < 0.0) {
    double m[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j) acc = fma(b.n_up[j], du[j][20 + 10 * kk + p] - du[kk][20 + 10 * j + p], acc);
      m[kk] = acc;
    }
    const double nm = b.n_up[0] * m[0] + b.n_up[1] * m[1] + b.n_up[2] * m[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) w0[i] = fma(v_0, m[i] - b.n_dn[i] * nm, w0[i]);
  }
  if (v_p < 0.0) wp = 0.0;
  ud[p] = wpsi;
  ud[10 + p] = 0.5 * wp + gamma2 * wpsi;
#pragma unroll
  for (int i = 0; i < 3; ++i) ud[20 + 10 * i + p] = b.n_dn[i] * (0.5 * wp) + w0[i];
}

// Reverse of cpm_pair: from the cotangents of ud (pair p's five entries) and
// of *wm, adds to krb (the interior right-hand side), ub (the state) and
// dub[i] (its Cartesian derivatives).
__device__ __forceinline__ void cpm_pair_rev(int p, const CpmBg& b, double gamma1, double gamma2, const double* udb,
                                             double wmb, double* krb, double* ub, double (*dub)[50]) {
  const double v_psi = -(1.0 + gamma1) * b.nb, v_0 = -b.nb, v_p = -b.nb + b.Nb;
  const double wpsib = udb[p] + gamma2 * udb[10 + p];
  double wpb = 0.5 * udb[10 + p];
#pragma unroll
  for (int i = 0; i < 3; ++i) wpb = fma(0.5 * b.n_dn[i], udb[20 + 10 * i + p], wpb);
  if (v_p < 0.0) wpb = 0.0;
  double w0b[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) w0b[i] = udb[20 + 10 * i + p];
  double psb = wpsib - gamma2 * (wpb + wmb), pib = wpb + wmb, nphib = wpb - wmb;
  double phb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    phb[i] = w0b[i];
    nphib = fma(-b.n_dn[i], w0b[i], nphib);
  }
  if (v_0 < 0.0) {
    const double nw = b.n_dn[0] * w0b[0] + b.n_dn[1] * w0b[1] + b.n_dn[2] * w0b[2];
    double mb[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) mb[kk] = v_0 * w0b[kk] - v_0 * nw * b.n_up[kk];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dub[j][20 + 10 * kk + p] = fma(b.n_up[j], mb[kk], dub[j][20 + 10 * kk + p]);
        dub[kk][20 + 10 * j + p] = fma(-b.n_up[j], mb[kk], dub[kk][20 + 10 * j + p]);
      }
  }
  if (v_psi < 0.0) {
    const double c = v_psi * wpsib;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dub[i][p] = fma(b.n_up[i], c, dub[i][p]);
      ub[20 + 10 * i + p] = fma(-b.n_up[i], c, ub[20 + 10 * i + p]);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) phb[i] = fma(b.n_up[i], nphib, phb[i]);
  krb[p] += psb;
  krb[10 + p] += pib;
#pragma unroll
  for (int i = 0; i < 3; ++i) krb[20 + 10 * i + p] += phb[i];
}

// Basis tensor e of the u^- subspace (e = 0..3: l_a delta_be + delta_ae l_b;
// 4: P) or, e = 5, the interior w^-; and the field-space direction of a u^-
// time derivative E: Pi' = E/2, Phi_i' = -n_i E/2, psi' = 0.
__device__ __forceinline__ void cpm_basis(int e, const double l_dn[4], const double P[10], const double wm[10],
                                          double E[10]) {
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
    E[p] = (e < 4) ? ((B == e ? l_dn[A] : 0.0) + (A == e ? l_dn[B] : 0.0)) : (e == 4 ? P[p] : wm[p]);
  }
}
__device__ __forceinline__ void cpm_vdir(const double E[10], const double n_dn[3], double* v) {
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    v[p] = 0.0;
    v[10 + p] = 0.5 * E[p];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[20 + 10 * i + p] = -0.5 * n_dn[i] * E[p];
  }
}

// The 5x5 system: res[0] = C' along the corrected time derivative (w^- = 0),
// res[1 + i] = C' along d_i u with d_i H, res[4 + j] = B(E_j) (j = 0..4) and
// res[9] = B(interior w^-), the slopes already divided by N.  Rows 0..3:
// B(S) = -K[0] + (N - n.beta)/(2N) (K[0] + B(D_t u^-)), K[0] = res[0]/N
// + (n^i - beta^i/N) res[1 + i]; row 4: l^b lam_b = 0.  Column 5 is the target.
__device__ __forceinline__ void cpm_system(const double (*res)[4], const CpmBg& b, const double l_up[4],
                                           double M[5][6]) {
  const double f = (b.Nb - b.nb) / (2.0 * b.Nb);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double K = res[0][c] / b.Nb;
#pragma unroll
    for (int i = 0; i < 3; ++i) K = fma(b.n_up[i] - b.bb[i] / b.Nb, res[1 + i][c], K);
#pragma unroll
    for (int j = 0; j < 5; ++j) M[c][j] = res[4 + j][c];
    M[c][5] = fma(f, K + res[9][c], -K);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) M[4][j] = l_up[j];
  M[4][4] = 0.0;
  M[4][5] = 0.0;
}

// Gaussian elimination with partial pivoting on the augmented 5x6 system (M
// is overwritten); false (and x = 0) if a pivot vanishes.
__device__ __forceinline__ bool cpm_solve5(double M[5][6], double x[5]) {
  bool ok = true;
#pragma unroll 1
  for (int c = 0; c < 5 && ok; ++c) {
    int piv = c;
    for (int r = c + 1; r < 5; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (!(fabs(M[piv][c]) > 0.0)) {
      ok = false;
      break;
    }
    if (piv != c)
      for (int e = 0; e < 6; ++e) {
        const double tmp = M[c][e];
        M[c][e] = M[piv][e];
        M[piv][e] = tmp;
      }
    for (int r = c + 1; r < 5; ++r) {
      const double fr = M[r][c] / M[c][c];
      for (int e = c; e < 6; ++e) M[r][e] -= fr * M[c][e];
    }
  }
  for (int e = 0; e < 5; ++e) x[e] = 0.0;
  if (ok) {
    for (int r = 4; r >= 0; --r) {
      double v = M[r][5];
      for (int e = r + 1; e < 5; ++e) v -= M[r][e] * x[e];
      x[r] = v / M[r][r];
    }
  }
  return ok;
}

}  // namespace gh
