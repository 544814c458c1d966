// Per-point GH algebra for the adjoint: the right-hand side of one point
// written out stage by stage with its intermediates kept, and its hand-derived
// reverse pass (vector-Jacobian product).  __host__ __device__ so the same code
// is unit-tested on the CPU against finite differences.
//
// Inputs of one point: u[50] (psi_p, Pi_p, Phi_ip), spherical-basis
// derivatives ds[f*3 + d] of every field (d = 0: d/dx on the CGL coordinate,
// 1: d/dtheta, 2: d/dphi), the DiffJac matrix J[i][d] (Eq. DiffJac; its radial
// column includes dx/dr), and the gauge source H[4], dH[4i + a] = d_i H_a.
// Equations: the first-order GH system (Lindblom et al. 2006), as in the
// forward kernel.
#pragma once

#include "gh_tensor.cuh"

namespace gh {

#ifndef GH_HD
#define GH_HD __host__ __device__
#endif

struct PointIn {
  const double* u;      // [50]
  const double* ds;     // [50 * 3]
  double J[3][3];
  const double* H;      // [4]
  const double* dH;     // [12]
  double g0, g1, g2;
};

// Intermediates of the forward pass that the reverse pass reads.
struct PointFwd {
  Split S;
  double Gam[40];
  double C[4];
  double PH[4];
  double Pm[4][16];
  double Um[3][16];
  double Wm[3][16];
  double tPt, tC;
  double tPi[3], tPig[3];
  double tPhit[3], tPhij[3][3], Mik[3][3];
  double bs[3], Gs[3][3];
};

GH_HD inline int s3h(int i, int j) {
  const int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

GH_HD inline void point_split(const double psi[10], Split& s) {
  const double gxx = psi[4], gxy = psi[5], gxz = psi[6], gyy = psi[7], gyz = psi[8], gzz = psi[9];
  const double cxx = gyy * gzz - gyz * gyz;
  const double cxy = gxz * gyz - gxy * gzz;
  const double cxz = gxy * gyz - gxz * gyy;
  const double cyy = gxx * gzz - gxz * gxz;
  const double cyz = gxy * gxz - gxx * gyz;
  const double czz = gxx * gyy - gxy * gxy;
  const double det = gxx * cxx + gxy * cxy + gxz * cxz;
  const double idet = 1.0 / det;
  s.ginv[0] = cxx * idet; s.ginv[1] = cxy * idet; s.ginv[2] = cxz * idet;
  s.ginv[3] = cyy * idet; s.ginv[4] = cyz * idet; s.ginv[5] = czz * idet;
  const double bx = psi[1], by = psi[2], bz = psi[3];
  s.beta_up[0] = s.ginv[0] * bx + s.ginv[1] * by + s.ginv[2] * bz;
  s.beta_up[1] = s.ginv[1] * bx + s.ginv[3] * by + s.ginv[4] * bz;
  s.beta_up[2] = s.ginv[2] * bx + s.ginv[4] * by + s.ginv[5] * bz;
  const double bb = s.beta_up[0] * bx + s.beta_up[1] * by + s.beta_up[2] * bz;
  s.alpha = sqrt(bb - psi[0]);
  const double ia = 1.0 / s.alpha, ia2 = ia * ia;
  s.t_up[0] = ia;
  for (int i = 0; i < 3; ++i) s.t_up[1 + i] = -s.beta_up[i] * ia;
  s.psi_inv[0] = -ia2;
  for (int i = 0; i < 3; ++i) s.psi_inv[1 + i] = s.beta_up[i] * ia2;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j)
      s.psi_inv[sym_index(1 + i, 1 + j)] = s.ginv[s3h(i, j)] - s.beta_up[i] * s.beta_up[j] * ia2;
}

// Forward intermediates only (what the reverse pass reads).
GH_HD inline void point_intermediates(const PointIn& in, PointFwd& f) {
  const double* psi = in.u;
  const double* Pi = in.u + 10;
  const double* Phi = in.u + 20;
  point_split(psi, f.S);
  const Split& S = f.S;
  const double al = S.alpha;
  // Christoffel symbols: d_c psi_ab = t_c Pi_ab + g^i_c Phi_iab
  double d[40];
  for (int p = 0; p < 10; ++p) {
    d[p] = -al * Pi[p] + S.beta_up[0] * Phi[p] + S.beta_up[1] * Phi[10 + p] + S.beta_up[2] * Phi[20 + p];
    for (int i = 0; i < 3; ++i) d[10 * (1 + i) + p] = Phi[10 * i + p];
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = b; c < 4; ++c)
        f.Gam[a * 10 + sym_index(b, c)] =
            0.5 * (d[b * 10 + sym_index(a, c)] + d[c * 10 + sym_index(a, b)] - d[a * 10 + sym_index(b, c)]);
  for (int a = 0; a < 4; ++a) {
    double acc = 0.0;
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(b, c)] * f.Gam[a * 10 + sym_index(b, c)];
    f.C[a] = in.H[a] + acc;
  }
  for (int dd = 0; dd < 4; ++dd) {
    double acc = 0.0;
    for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(c, dd)] * in.H[c];
    f.PH[dd] = acc;
  }
  for (int a = 0; a < 4; ++a)
    for (int dd = 0; dd < 4; ++dd)
      for (int e = 0; e < 4; ++e) {
        double acc = 0.0;
        for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(dd, c)] * f.Gam[a * 10 + sym_index(c, e)];
        f.Pm[a][dd * 4 + e] = acc;
      }
  for (int i = 0; i < 3; ++i)
    for (int dd = 0; dd < 4; ++dd)
      for (int a = 0; a < 4; ++a) {
        double acc = 0.0;
        for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(dd, c)] * Phi[i * 10 + sym_index(c, a)];
        f.Um[i][dd * 4 + a] = acc;
      }
  for (int j = 0; j < 3; ++j)
    for (int e = 0; e < 16; ++e)
      f.Wm[j][e] = S.ginv[s3h(0, j)] * f.Um[0][e] + S.ginv[s3h(1, j)] * f.Um[1][e] + S.ginv[s3h(2, j)] * f.Um[2][e];
  f.tPt = 0.0;
  f.tC = 0.0;
  for (int i = 0; i < 3; ++i) f.tPi[i] = 0.0;
  for (int c = 0; c < 4; ++c) {
    f.tC += S.t_up[c] * f.C[c];
    for (int dd = 0; dd < 4; ++dd) f.tPt += S.t_up[c] * S.t_up[dd] * Pi[sym_index(c, dd)];
    for (int i = 0; i < 3; ++i) f.tPi[i] += S.t_up[c] * Pi[sym_index(c, 1 + i)];
  }
  for (int j = 0; j < 3; ++j)
    f.tPig[j] = f.tPi[0] * S.ginv[s3h(0, j)] + f.tPi[1] * S.ginv[s3h(1, j)] + f.tPi[2] * S.ginv[s3h(2, j)];
  for (int i = 0; i < 3; ++i) {
    double acc = 0.0;
    for (int c = 0; c < 4; ++c)
      for (int dd = 0; dd < 4; ++dd) acc += S.t_up[c] * S.t_up[dd] * Phi[i * 10 + sym_index(c, dd)];
    f.tPhit[i] = acc;
    for (int j = 0; j < 3; ++j) {
      double t2 = 0.0;
      for (int c = 0; c < 4; ++c) t2 += S.t_up[c] * Phi[i * 10 + sym_index(1 + j, c)];
      f.tPhij[i][j] = t2;
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k)
      f.Mik[i][k] = f.tPhij[i][0] * S.ginv[s3h(0, k)] + f.tPhij[i][1] * S.ginv[s3h(1, k)] +
                    f.tPhij[i][2] * S.ginv[s3h(2, k)];
  for (int dd = 0; dd < 3; ++dd) {
    f.bs[dd] = S.beta_up[0] * in.J[0][dd] + S.beta_up[1] * in.J[1][dd] + S.beta_up[2] * in.J[2][dd];
    for (int i = 0; i < 3; ++i)
      f.Gs[i][dd] = S.ginv[s3h(0, i)] * in.J[0][dd] + S.ginv[s3h(1, i)] * in.J[1][dd] + S.ginv[s3h(2, i)] * in.J[2][dd];
  }
}

// Forward: out[50] = dudt at the point; fills f.
GH_HD inline void point_rhs(const PointIn& in, PointFwd& f, double out[50]) {
  point_intermediates(in, f);
  const double* psi = in.u;
  const double* Pi = in.u + 10;
  const double* Phi = in.u + 20;
  const Split& S = f.S;
  const double al = S.alpha;
  const double g0 = in.g0, g1 = in.g1, g2 = in.g2;
  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
    double T1 = 0.0, T2 = 0.0, T3 = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int dd = 0; dd < 4; ++dd) T1 += f.Wm[j][dd * 4 + A] * Phi[j * 10 + sym_index(dd, B)];
    for (int c = 0; c < 4; ++c) {
      double pc = 0.0;
      for (int dd = 0; dd < 4; ++dd) pc += S.psi_inv[sym_index(c, dd)] * Pi[sym_index(dd, B)];
      T2 += Pi[sym_index(c, A)] * pc;
    }
    for (int dd = 0; dd < 4; ++dd)
      for (int e = 0; e < 4; ++e) T3 += f.Pm[A][dd * 4 + e] * f.Pm[B][e * 4 + dd];
    const double dAHB = (A > 0 ? in.dH[4 * (A - 1) + B] : 0.0);
    const double dBHA = (B > 0 ? in.dH[4 * (B - 1) + A] : 0.0);
    double gh_ = 0.0;
    for (int dd = 0; dd < 4; ++dd) gh_ += f.PH[dd] * f.Gam[dd * 10 + p];
    const double nablaH = 0.5 * (dAHB + dBHA) - gh_;
    const double damp = (B == 0 ? -al * f.C[A] : 0.0) + (A == 0 ? -al * f.C[B] : 0.0) - psi[p] * f.tC;
    double tPiPhi = 0.0, bPhi = 0.0;
    for (int j = 0; j < 3; ++j) {
      tPiPhi += f.tPig[j] * Phi[j * 10 + p];
      bPhi += S.beta_up[j] * Phi[j * 10 + p];
    }
    const double srcPi = 2.0 * al * (T1 - T2 - T3) - 2.0 * al * nablaH - 0.5 * al * f.tPt * Pi[p] - al * tPiPhi +
                         g0 * al * damp - g1 * g2 * bPhi;
    const double* dpsi = in.ds + 3 * p;
    const double* dPi = in.ds + 3 * (10 + p);
    const double bdpsi = f.bs[0] * dpsi[0] + f.bs[1] * dpsi[1] + f.bs[2] * dpsi[2];
    const double bdPi = f.bs[0] * dPi[0] + f.bs[1] * dPi[1] + f.bs[2] * dPi[2];
    double gdPhi = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double* dPhi = in.ds + 3 * (20 + 10 * i + p);
      gdPhi += f.Gs[i][0] * dPhi[0] + f.Gs[i][1] * dPhi[1] + f.Gs[i][2] * dPhi[2];
    }
    out[p] = (1.0 + g1) * bdpsi - al * Pi[p] - g1 * bPhi;
    out[10 + p] = bdPi - al * gdPhi + g1 * g2 * bdpsi + srcPi;
    for (int i = 0; i < 3; ++i) {
      const double* dPhi = in.ds + 3 * (20 + 10 * i + p);
      const double bdPhi = f.bs[0] * dPhi[0] + f.bs[1] * dPhi[1] + f.bs[2] * dPhi[2];
      const double cpsi = in.J[i][0] * dpsi[0] + in.J[i][1] * dpsi[1] + in.J[i][2] * dpsi[2];
      const double cPi = in.J[i][0] * dPi[0] + in.J[i][1] * dPi[1] + in.J[i][2] * dPi[2];
      const double srcPhi = 0.5 * al * f.tPhit[i] * Pi[p] +
                            al * (f.Mik[i][0] * Phi[p] + f.Mik[i][1] * Phi[10 + p] + f.Mik[i][2] * Phi[20 + p]) -
                            al * g2 * Phi[i * 10 + p];
      out[20 + 10 * i + p] = bdPhi - al * cPi + al * g2 * cpsi + srcPhi;
    }
  }
}

// Reverse of C_a = H_a + psi^bc Gam_abc, of the Christoffel symbols and of
// the 3+1 split: adds to psib/Pib/Phib given the accumulated adjoints.
GH_HD inline void gamma_split_reverse(const double psi[10], const double Pi[10], const double Phi[30],
                                      const Split& S, const double Gam[40], const double Cb[4], double Gamb[40],
                                      double& alb, double betab[3], double ginvb[6], double tb[4],
                                      double pinvb[10], double* psib, double* Pib, double* Phib) {
  const double al = S.alpha;
  // ---- C_a = H_a + sum_{b,c} psi_inv(b,c) Gam[a](b,c)
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) {
        pinvb[sym_index(b, c)] += Gam[a * 10 + sym_index(b, c)] * Cb[a];
        Gamb[a * 10 + sym_index(b, c)] += S.psi_inv[sym_index(b, c)] * Cb[a];
      }
  // ---- Gam[a](b<=c) = (d[b](a,c) + d[c](a,b) - d[a](b,c)) / 2
  double db[40];
  for (int e = 0; e < 40; ++e) db[e] = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = b; c < 4; ++c) {
        const double g = 0.5 * Gamb[a * 10 + sym_index(b, c)];
        db[b * 10 + sym_index(a, c)] += g;
        db[c * 10 + sym_index(a, b)] += g;
        db[a * 10 + sym_index(b, c)] -= g;
      }
  // d[0][p] = -al Pi_p + beta^i Phi_ip ; d[1+i][p] = Phi_ip
  for (int p = 0; p < 10; ++p) {
    alb -= Pi[p] * db[p];
    Pib[p] -= al * db[p];
    for (int i = 0; i < 3; ++i) {
      betab[i] += Phi[i * 10 + p] * db[p];
      Phib[i * 10 + p] += S.beta_up[i] * db[p] + db[10 * (1 + i) + p];
    }
  }
  // ---- split: t^a, psi^ab from alpha, beta^i, g^ij
  const double ia = 1.0 / al, ia2 = ia * ia, ia3 = ia2 * ia;
  alb -= tb[0] * ia2;
  for (int i = 0; i < 3; ++i) {
    betab[i] -= tb[1 + i] * ia;
    alb += tb[1 + i] * S.beta_up[i] * ia2;
  }
  alb += pinvb[0] * 2.0 * ia3;
  for (int i = 0; i < 3; ++i) {
    betab[i] += pinvb[1 + i] * ia2;
    alb -= pinvb[1 + i] * 2.0 * S.beta_up[i] * ia3;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      const double pb = pinvb[sym_index(1 + i, 1 + j)];
      ginvb[s3h(i, j)] += pb;
      betab[i] -= pb * S.beta_up[j] * ia2;
      betab[j] -= pb * S.beta_up[i] * ia2;
      alb += pb * 2.0 * S.beta_up[i] * S.beta_up[j] * ia3;
    }
  // alpha = sqrt(beta_i g^ij beta_j - psi_00), beta_i = psi_0i, beta^i = g^ij beta_j
  const double Qb = alb * 0.5 * ia;
  psib[0] -= Qb;
  double blowb[3];
  for (int i = 0; i < 3; ++i) blowb[i] = 2.0 * S.beta_up[i] * Qb;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      const double bi = psi[1 + i], bj = psi[1 + j];
      ginvb[s3h(i, j)] += (i == j ? bi * bj : 2.0 * bi * bj) * Qb;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      blowb[j] += S.ginv[s3h(i, j)] * betab[i];
      ginvb[s3h(i, j)] += betab[i] * psi[1 + j];
    }
  for (int i = 0; i < 3; ++i) psib[1 + i] += blowb[i];
  // g^ij = inverse(g_ij): packed-slot adjoint -> symmetric matrix -> -ginv A ginv -> packed
  double Af[3][3], Gf[3][3], tmp[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Af[i][j] = (i == j) ? ginvb[s3h(i, i)] : 0.5 * ginvb[s3h(i, j)];
      Gf[i][j] = S.ginv[s3h(i, j)];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) tmp[i][j] = Gf[i][0] * Af[0][j] + Gf[i][1] * Af[1][j] + Gf[i][2] * Af[2][j];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      const double bij = -(tmp[i][0] * Gf[0][j] + tmp[i][1] * Gf[1][j] + tmp[i][2] * Gf[2][j]);
      const double bji = -(tmp[j][0] * Gf[0][i] + tmp[j][1] * Gf[1][i] + tmp[j][2] * Gf[2][i]);
      psib[sym_index(1 + i, 1 + j)] += (i == j) ? bij : bij + bji;
    }
}

// Access of the reverse pass to one symmetric pair's entries: the spherical
// derivatives ds15 and the output cotangents kb5 of its five fields (psi_p,
// Pi_p, Phi_xp, Phi_yp, Phi_zp), and the cotangents dsb15 of those
// derivatives.  The pass reads and writes pair p's entries only while it
// handles pair p, so they need not be held for the whole point.
// ArrayPairIO: whole-point arrays ds[150], kb[50], dsb[150] (dsb is added to).
struct ArrayPairIO {
  const double* ds;
  const double* kb;
  double* dsb;
  GH_HD void load(int p, double ds15[15], double kb5[5]) const {
    for (int e = 0; e < 5; ++e) {
      const int fi = e == 0 ? p : 10 * e + p;
      for (int d = 0; d < 3; ++d) ds15[3 * e + d] = ds[3 * fi + d];
      kb5[e] = kb[fi];
    }
  }
  GH_HD void store(int p, const double dsb15[15]) const {
    for (int e = 0; e < 5; ++e) {
      const int fi = e == 0 ? p : 10 * e + p;
      for (int d = 0; d < 3; ++d) dsb[3 * fi + d] += dsb15[3 * e + d];
    }
  }
};

// Reverse pass: given the cotangent kb of dudt (through io), adds the
// cotangents of the point's fields to ub[50] and hands those of its spherical
// derivatives to io.store, pair by pair.  f must hold the intermediates of
// point_rhs for the same inputs.
template <class IO>
GH_HD inline void point_rhs_vjp_io(const PointIn& in, const PointFwd& f, const IO& io, double ub[50]) {
  const double* psi = in.u;
  const double* Pi = in.u + 10;
  const double* Phi = in.u + 20;
  const Split& S = f.S;
  const double al = S.alpha;
  const double g0 = in.g0, g1 = in.g1, g2 = in.g2;
  double* psib = ub;
  double* Pib = ub + 10;
  double* Phib = ub + 20;
  // adjoints of intermediates (packed slots mirror the forward reads)
  double alb = 0.0;
  double betab[3] = {0.0, 0.0, 0.0};
  double ginvb[6] = {0, 0, 0, 0, 0, 0};
  double tb[4] = {0.0, 0.0, 0.0, 0.0};
  double pinvb[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  double Gamb[40];
  for (int e = 0; e < 40; ++e) Gamb[e] = 0.0;
  double Cb[4] = {0.0, 0.0, 0.0, 0.0};
  double PHb[4] = {0.0, 0.0, 0.0, 0.0};
  double Pmb[4][16], Wmb[3][16];
  for (int a = 0; a < 4; ++a)
    for (int e = 0; e < 16; ++e) Pmb[a][e] = 0.0;
  for (int j = 0; j < 3; ++j)
    for (int e = 0; e < 16; ++e) Wmb[j][e] = 0.0;
  double tPtb = 0.0, tCb = 0.0;
  double tPigb[3] = {0.0, 0.0, 0.0};
  double tPhitb[3] = {0.0, 0.0, 0.0};
  double Mikb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double bsb[3] = {0.0, 0.0, 0.0};
  double Gsb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};

  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
    double ds15[15], kb5[5], dsb15[15];
    io.load(p, ds15, kb5);
    for (int e = 0; e < 15; ++e) dsb15[e] = 0.0;
    const double kpsi = kb5[0], kPi = kb5[1];
    const double* dpsi = ds15;
    const double* dPi = ds15 + 3;
    double* dpsib = dsb15;
    double* dPib = dsb15 + 3;
    // ---- recompute the per-pair forward scalars needed below
    double T1 = 0.0, T2 = 0.0, T3 = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int dd = 0; dd < 4; ++dd) T1 += f.Wm[j][dd * 4 + A] * Phi[j * 10 + sym_index(dd, B)];
    double pcv[4];
    for (int c = 0; c < 4; ++c) {
      double pc = 0.0;
      for (int dd = 0; dd < 4; ++dd) pc += S.psi_inv[sym_index(c, dd)] * Pi[sym_index(dd, B)];
      pcv[c] = pc;
      T2 += Pi[sym_index(c, A)] * pc;
    }
    for (int dd = 0; dd < 4; ++dd)
      for (int e = 0; e < 4; ++e) T3 += f.Pm[A][dd * 4 + e] * f.Pm[B][e * 4 + dd];
    const double dAHB = (A > 0 ? in.dH[4 * (A - 1) + B] : 0.0);
    const double dBHA = (B > 0 ? in.dH[4 * (B - 1) + A] : 0.0);
    double gh_ = 0.0;
    for (int dd = 0; dd < 4; ++dd) gh_ += f.PH[dd] * f.Gam[dd * 10 + p];
    const double nablaH = 0.5 * (dAHB + dBHA) - gh_;
    const double damp = (B == 0 ? -al * f.C[A] : 0.0) + (A == 0 ? -al * f.C[B] : 0.0) - psi[p] * f.tC;
    double tPiPhi = 0.0, bPhi = 0.0;
    for (int j = 0; j < 3; ++j) {
      tPiPhi += f.tPig[j] * Phi[j * 10 + p];
      bPhi += S.beta_up[j] * Phi[j * 10 + p];
    }
    double gdPhi = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double* dPhi = ds15 + 3 * (2 + i);
      gdPhi += f.Gs[i][0] * dPhi[0] + f.Gs[i][1] * dPhi[1] + f.Gs[i][2] * dPhi[2];
    }
    // ---- out[p] = (1+g1) bdpsi - al Pi_p - g1 bPhi
    double bdpsib = (1.0 + g1) * kpsi;
    alb -= Pi[p] * kpsi;
    Pib[p] -= al * kpsi;
    double bPhib = -g1 * kpsi;
    // ---- out[10+p] = bdPi - al gdPhi + g1 g2 bdpsi + srcPi
    const double bdPib = kPi;
    alb -= gdPhi * kPi;
    const double gdPhib = -al * kPi;
    bdpsib += g1 * g2 * kPi;
    const double sPb = kPi;
    // ---- out[20+10i+p]
    double cpsib[3], cPib[3];
    for (int i = 0; i < 3; ++i) {
      const double kPhi = kb5[2 + i];
      const double* dPhi = ds15 + 3 * (2 + i);
      double* dPhib = dsb15 + 3 * (2 + i);
      const double cpsi = in.J[i][0] * dpsi[0] + in.J[i][1] * dpsi[1] + in.J[i][2] * dpsi[2];
      const double cPi = in.J[i][0] * dPi[0] + in.J[i][1] * dPi[1] + in.J[i][2] * dPi[2];
      // bdPhi = bs . dPhi
      for (int dd = 0; dd < 3; ++dd) {
        dPhib[dd] += f.bs[dd] * kPhi;
        bsb[dd] += dPhi[dd] * kPhi;
      }
      alb += (-cPi + g2 * cpsi) * kPhi;
      cPib[i] = -al * kPhi;
      cpsib[i] = al * g2 * kPhi;
      // srcPhi = 0.5 al tPhit_i Pi_p + al sum_k Mik Phi_kp - al g2 Phi_ip
      const double mphi = f.Mik[i][0] * Phi[p] + f.Mik[i][1] * Phi[10 + p] + f.Mik[i][2] * Phi[20 + p];
      alb += (0.5 * f.tPhit[i] * Pi[p] + mphi - g2 * Phi[i * 10 + p]) * kPhi;
      tPhitb[i] += 0.5 * al * Pi[p] * kPhi;
      Pib[p] += 0.5 * al * f.tPhit[i] * kPhi;
      for (int k = 0; k < 3; ++k) {
        Mikb[i][k] += al * Phi[k * 10 + p] * kPhi;
        Phib[k * 10 + p] += al * f.Mik[i][k] * kPhi;
      }
      Phib[i * 10 + p] -= al * g2 * kPhi;
    }
    // cpsi_i = J[i] . dpsi ; cPi_i = J[i] . dPi
    for (int dd = 0; dd < 3; ++dd) {
      dpsib[dd] += in.J[0][dd] * cpsib[0] + in.J[1][dd] * cpsib[1] + in.J[2][dd] * cpsib[2];
      dPib[dd] += in.J[0][dd] * cPib[0] + in.J[1][dd] * cPib[1] + in.J[2][dd] * cPib[2];
    }
    // bdpsi = bs . dpsi ; bdPi = bs . dPi
    for (int dd = 0; dd < 3; ++dd) {
      dpsib[dd] += f.bs[dd] * bdpsib;
      bsb[dd] += dpsi[dd] * bdpsib;
      dPib[dd] += f.bs[dd] * bdPib;
      bsb[dd] += dPi[dd] * bdPib;
    }
    // gdPhi = sum_i Gs[i] . dPhi_i
    for (int i = 0; i < 3; ++i) {
      const double* dPhi = ds15 + 3 * (2 + i);
      double* dPhib = dsb15 + 3 * (2 + i);
      for (int dd = 0; dd < 3; ++dd) {
        dPhib[dd] += f.Gs[i][dd] * gdPhib;
        Gsb[i][dd] += dPhi[dd] * gdPhib;
      }
    }
    // ---- srcPi = 2al(T1-T2-T3) - 2al nablaH - 0.5 al tPt Pi_p - al tPiPhi + g0 al damp - g1 g2 bPhi
    alb += sPb * (2.0 * (T1 - T2 - T3) - 2.0 * nablaH - 0.5 * f.tPt * Pi[p] - tPiPhi + g0 * damp);
    const double T1b = 2.0 * al * sPb, T2b = -2.0 * al * sPb, T3b = -2.0 * al * sPb;
    const double nHb = -2.0 * al * sPb;
    tPtb += -0.5 * al * Pi[p] * sPb;
    Pib[p] += -0.5 * al * f.tPt * sPb;
    const double tPiPhib = -al * sPb;
    const double dampb = g0 * al * sPb;
    bPhib += -g1 * g2 * sPb;
    // T1 = sum_j sum_d Wm[j][d][A] Phi_j(d,B)
    for (int j = 0; j < 3; ++j)
      for (int dd = 0; dd < 4; ++dd) {
        Wmb[j][dd * 4 + A] += Phi[j * 10 + sym_index(dd, B)] * T1b;
        Phib[j * 10 + sym_index(dd, B)] += f.Wm[j][dd * 4 + A] * T1b;
      }
    // T2 = sum_c Pi(c,A) pc[c], pc[c] = sum_d psi_inv(c,d) Pi(d,B)
    for (int c = 0; c < 4; ++c) {
      Pib[sym_index(c, A)] += pcv[c] * T2b;
      const double pcb = Pi[sym_index(c, A)] * T2b;
      for (int dd = 0; dd < 4; ++dd) {
        pinvb[sym_index(c, dd)] += Pi[sym_index(dd, B)] * pcb;
        Pib[sym_index(dd, B)] += S.psi_inv[sym_index(c, dd)] * pcb;
      }
    }
    // T3 = sum_{d,e} Pm[A][d][e] Pm[B][e][d]
    for (int dd = 0; dd < 4; ++dd)
      for (int e = 0; e < 4; ++e) {
        Pmb[A][dd * 4 + e] += f.Pm[B][e * 4 + dd] * T3b;
        Pmb[B][e * 4 + dd] += f.Pm[A][dd * 4 + e] * T3b;
      }
    // nablaH = const - sum_d PH[d] Gam[d][p]
    for (int dd = 0; dd < 4; ++dd) {
      PHb[dd] -= f.Gam[dd * 10 + p] * nHb;
      Gamb[dd * 10 + p] -= f.PH[dd] * nHb;
    }
    // damp
    if (B == 0) {
      alb -= f.C[A] * dampb;
      Cb[A] -= al * dampb;
    }
    if (A == 0) {
      alb -= f.C[B] * dampb;
      Cb[B] -= al * dampb;
    }
    psib[p] -= f.tC * dampb;
    tCb -= psi[p] * dampb;
    // tPiPhi = sum_j tPig[j] Phi_jp ; bPhi = sum_j beta^j Phi_jp
    for (int j = 0; j < 3; ++j) {
      tPigb[j] += Phi[j * 10 + p] * tPiPhib;
      Phib[j * 10 + p] += f.tPig[j] * tPiPhib + S.beta_up[j] * bPhib;
      betab[j] += Phi[j * 10 + p] * bPhib;
    }
    io.store(p, dsb15);
  }
  // ---- bs[d] = sum_k beta^k J[k][d] ; Gs[i][d] = sum_k ginv(k,i) J[k][d]
  for (int dd = 0; dd < 3; ++dd) {
    for (int k = 0; k < 3; ++k) betab[k] += in.J[k][dd] * bsb[dd];
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) ginvb[s3h(k, i)] += in.J[k][dd] * Gsb[i][dd];
  }
  // ---- Mik = sum_j tPhij[i][j] ginv(j,k) ; tPhij[i][j] = sum_c t^c Phi_i(1+j,c) ; tPhit
  for (int i = 0; i < 3; ++i) {
    double tPhijb[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) {
        tPhijb[j] += S.ginv[s3h(j, k)] * Mikb[i][k];
        ginvb[s3h(j, k)] += f.tPhij[i][j] * Mikb[i][k];
      }
    for (int j = 0; j < 3; ++j)
      for (int c = 0; c < 4; ++c) {
        tb[c] += Phi[i * 10 + sym_index(1 + j, c)] * tPhijb[j];
        Phib[i * 10 + sym_index(1 + j, c)] += S.t_up[c] * tPhijb[j];
      }
    for (int c = 0; c < 4; ++c)
      for (int dd = 0; dd < 4; ++dd) {
        const double ph = Phi[i * 10 + sym_index(c, dd)];
        tb[c] += S.t_up[dd] * ph * tPhitb[i];
        tb[dd] += S.t_up[c] * ph * tPhitb[i];
        Phib[i * 10 + sym_index(c, dd)] += S.t_up[c] * S.t_up[dd] * tPhitb[i];
      }
  }
  // ---- Wm[j][e] = sum_i ginv(i,j) Um[i][e] ; Um[i][d][a] = sum_c psi_inv(d,c) Phi_i(c,a)
  for (int i = 0; i < 3; ++i) {
    double Umb[16];
    for (int e = 0; e < 16; ++e) {
      Umb[e] = S.ginv[s3h(i, 0)] * Wmb[0][e] + S.ginv[s3h(i, 1)] * Wmb[1][e] + S.ginv[s3h(i, 2)] * Wmb[2][e];
      for (int j = 0; j < 3; ++j) ginvb[s3h(i, j)] += f.Um[i][e] * Wmb[j][e];
    }
    for (int dd = 0; dd < 4; ++dd)
      for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 4; ++c) {
          pinvb[sym_index(dd, c)] += Phi[i * 10 + sym_index(c, a)] * Umb[dd * 4 + a];
          Phib[i * 10 + sym_index(c, a)] += S.psi_inv[sym_index(dd, c)] * Umb[dd * 4 + a];
        }
  }
  // ---- Pm[a][d][e] = sum_c psi_inv(d,c) Gam[a](c,e)
  for (int a = 0; a < 4; ++a)
    for (int dd = 0; dd < 4; ++dd)
      for (int e = 0; e < 4; ++e)
        for (int c = 0; c < 4; ++c) {
          pinvb[sym_index(dd, c)] += f.Gam[a * 10 + sym_index(c, e)] * Pmb[a][dd * 4 + e];
          Gamb[a * 10 + sym_index(c, e)] += S.psi_inv[sym_index(dd, c)] * Pmb[a][dd * 4 + e];
        }
  // ---- PH[d] = sum_c psi_inv(c,d) H_c
  for (int dd = 0; dd < 4; ++dd)
    for (int c = 0; c < 4; ++c) pinvb[sym_index(c, dd)] += in.H[c] * PHb[dd];
  // ---- tPig[j] = sum_i tPi[i] ginv(i,j) ; tPi[i] = sum_c t^c Pi(c,1+i)
  double tPib[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) {
      tPib[i] += S.ginv[s3h(i, j)] * tPigb[j];
      ginvb[s3h(i, j)] += f.tPi[i] * tPigb[j];
    }
  for (int c = 0; c < 4; ++c) {
    for (int i = 0; i < 3; ++i) {
      tb[c] += Pi[sym_index(c, 1 + i)] * tPib[i];
      Pib[sym_index(c, 1 + i)] += S.t_up[c] * tPib[i];
    }
    // tPt = sum_{c,d} t^c t^d Pi(c,d)
    for (int dd = 0; dd < 4; ++dd) {
      const double pv = Pi[sym_index(c, dd)];
      tb[c] += S.t_up[dd] * pv * tPtb;
      tb[dd] += S.t_up[c] * pv * tPtb;
      Pib[sym_index(c, dd)] += S.t_up[c] * S.t_up[dd] * tPtb;
    }
    // tC = sum_c t^c C_c
    tb[c] += f.C[c] * tCb;
    Cb[c] += S.t_up[c] * tCb;
  }
  gamma_split_reverse(psi, Pi, Phi, S, f.Gam, Cb, Gamb, alb, betab, ginvb, tb, pinvb, psib, Pib, Phib);
}

// The reverse pass on whole-point arrays: kb[50], adds to ub[50] and dsb[150].
GH_HD inline void point_rhs_vjp(const PointIn& in, const PointFwd& f, const double kb[50], double ub[50],
                                double dsb[150]) {
  ArrayPairIO io{in.ds, kb, dsb};
  point_rhs_vjp_io(in, f, io, ub);
}

// Constraint energy density at a point, e = sum of the 64 squared stored
// components: C_a = H_a + Gamma_a, C_iab = d_i psi_ab - Phi_iab and
// C_ijab = d_i Phi_jab - d_j Phi_iab (i < j).  Returns e; with w != 0 also adds
// w * de/d(inputs) to ub[50] and dsb[150].
GH_HD inline double point_constraint_energy(const PointIn& in, double w, double ub[50], double dsb[150]) {
  const double* psi = in.u;
  const double* Pi = in.u + 10;
  const double* Phi = in.u + 20;
  Split S;
  point_split(psi, S);
  double d[40], Gam[40];
  for (int p = 0; p < 10; ++p) {
    d[p] = -S.alpha * Pi[p] + S.beta_up[0] * Phi[p] + S.beta_up[1] * Phi[10 + p] + S.beta_up[2] * Phi[20 + p];
    for (int i = 0; i < 3; ++i) d[10 * (1 + i) + p] = Phi[10 * i + p];
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = b; c < 4; ++c)
        Gam[a * 10 + sym_index(b, c)] =
            0.5 * (d[b * 10 + sym_index(a, c)] + d[c * 10 + sym_index(a, b)] - d[a * 10 + sym_index(b, c)]);
  double C[4];
  double e = 0.0;
  for (int a = 0; a < 4; ++a) {
    double acc = 0.0;
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(b, c)] * Gam[a * 10 + sym_index(b, c)];
    C[a] = in.H[a] + acc;
    e += C[a] * C[a];
  }
  double cd[50][3];  // Cartesian derivatives of psi_p and Phi_ip
  for (int f = 0; f < 50; ++f) {
    if (f >= 10 && f < 20) continue;
    const double* ds = in.ds + 3 * f;
    for (int i = 0; i < 3; ++i) cd[f][i] = in.J[i][0] * ds[0] + in.J[i][1] * ds[1] + in.J[i][2] * ds[2];
  }
  const int qi[3] = {0, 0, 1}, qj[3] = {1, 2, 2};
  double cdb[50][3];
  for (int f = 0; f < 50; ++f)
    for (int i = 0; i < 3; ++i) cdb[f][i] = 0.0;
  for (int p = 0; p < 10; ++p) {
    for (int i = 0; i < 3; ++i) {
      const double c3 = cd[p][i] - Phi[i * 10 + p];
      e += c3 * c3;
      if (w != 0.0) {
        cdb[p][i] += 2.0 * w * c3;
        ub[20 + i * 10 + p] -= 2.0 * w * c3;
      }
    }
    for (int q = 0; q < 3; ++q) {
      const int i = qi[q], j = qj[q];
      const double c4 = cd[20 + 10 * j + p][i] - cd[20 + 10 * i + p][j];
      e += c4 * c4;
      if (w != 0.0) {
        cdb[20 + 10 * j + p][i] += 2.0 * w * c4;
        cdb[20 + 10 * i + p][j] -= 2.0 * w * c4;
      }
    }
  }
  if (w == 0.0) return e;
  for (int f = 0; f < 50; ++f)
    for (int dd = 0; dd < 3; ++dd)
      dsb[3 * f + dd] += in.J[0][dd] * cdb[f][0] + in.J[1][dd] * cdb[f][1] + in.J[2][dd] * cdb[f][2];
  double Cb[4];
  for (int a = 0; a < 4; ++a) Cb[a] = 2.0 * w * C[a];
  double Gamb[40];
  for (int q = 0; q < 40; ++q) Gamb[q] = 0.0;
  double alb = 0.0, betab[3] = {0, 0, 0}, ginvb[6] = {0, 0, 0, 0, 0, 0}, tb[4] = {0, 0, 0, 0};
  double pinvb[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  gamma_split_reverse(psi, Pi, Phi, S, Gam, Cb, Gamb, alb, betab, ginvb, tb, pinvb, ub, ub + 10, ub + 20);
  return e;
}

// ---------------------------------------------------------------------------
// Pair-restricted reverse pass.  The vector-Jacobian product is linear in the
// output cotangent, so it is the sum over the symmetric pairs p of the
// products with kb restricted to pair p's five outputs (psi_p, Pi_p, Phi_ip).
// Each restricted product needs only the forward pieces that pair reads
// (Wm[.][.][A], Pm[A], Pm[B] of the full pass) and touches only the matching
// adjoint slices, so ten threads can share one point with short serial paths.
// Inputs: u[50], dsp[15] (spherical derivatives of psi_p, Pi_p, Phi_0p,
// Phi_1p, Phi_2p; d = x, theta, phi), kb5[5] (cotangents of pair p's
// outputs).  Adds to ub[50]; writes the cotangents of dsp to dsb15.
GH_HD inline void point_rhs_vjp_pair(const double* u, const double J[3][3], const double H[4], const double dH[12],
                                     double g0, double g1, double g2, int p, const double dsp[15],
                                     const double kb5[5], double ub[50], double dsb15[15]) {
  const double* psi = u;
  const double* Pi = u + 10;
  const double* Phi = u + 20;
  const int A = pair_a(p), B = pair_b(p);
  Split S;
  point_split(psi, S);
  const double al = S.alpha;
  // ---- forward pieces
  double Gam[40];
  {
    double d[40];
    for (int q = 0; q < 10; ++q) {
      d[q] = -al * Pi[q] + S.beta_up[0] * Phi[q] + S.beta_up[1] * Phi[10 + q] + S.beta_up[2] * Phi[20 + q];
      for (int i = 0; i < 3; ++i) d[10 * (1 + i) + q] = Phi[10 * i + q];
    }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int c = b; c < 4; ++c)
          Gam[a * 10 + sym_index(b, c)] =
              0.5 * (d[b * 10 + sym_index(a, c)] + d[c * 10 + sym_index(a, b)] - d[a * 10 + sym_index(b, c)]);
  }
  double C[4], PH[4];
  for (int a = 0; a < 4; ++a) {
    double acc = 0.0;
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(b, c)] * Gam[a * 10 + sym_index(b, c)];
    C[a] = H[a] + acc;
  }
  for (int dd = 0; dd < 4; ++dd) {
    double acc = 0.0;
    for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(c, dd)] * H[c];
    PH[dd] = acc;
  }
  double PmA[16], PmB[16];
  for (int dd = 0; dd < 4; ++dd)
    for (int e = 0; e < 4; ++e) {
      double a1 = 0.0, a2 = 0.0;
      for (int c = 0; c < 4; ++c) {
        a1 += S.psi_inv[sym_index(dd, c)] * Gam[A * 10 + sym_index(c, e)];
        a2 += S.psi_inv[sym_index(dd, c)] * Gam[B * 10 + sym_index(c, e)];
      }
      PmA[dd * 4 + e] = a1;
      PmB[dd * 4 + e] = a2;
    }
  double UmA[3][4], WmA[3][4];   // Um[i][d][A], Wm[j][d][A]
  for (int i = 0; i < 3; ++i)
    for (int dd = 0; dd < 4; ++dd) {
      double acc = 0.0;
      for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(dd, c)] * Phi[i * 10 + sym_index(c, A)];
      UmA[i][dd] = acc;
    }
  for (int j = 0; j < 3; ++j)
    for (int dd = 0; dd < 4; ++dd)
      WmA[j][dd] = S.ginv[s3h(0, j)] * UmA[0][dd] + S.ginv[s3h(1, j)] * UmA[1][dd] + S.ginv[s3h(2, j)] * UmA[2][dd];
  double tPt = 0.0, tC = 0.0, tPi[3] = {0.0, 0.0, 0.0}, tPig[3];
  for (int c = 0; c < 4; ++c) {
    tC += S.t_up[c] * C[c];
    for (int dd = 0; dd < 4; ++dd) tPt += S.t_up[c] * S.t_up[dd] * Pi[sym_index(c, dd)];
    for (int i = 0; i < 3; ++i) tPi[i] += S.t_up[c] * Pi[sym_index(c, 1 + i)];
  }
  for (int j = 0; j < 3; ++j)
    tPig[j] = tPi[0] * S.ginv[s3h(0, j)] + tPi[1] * S.ginv[s3h(1, j)] + tPi[2] * S.ginv[s3h(2, j)];
  double tPhit[3], tPhij[3][3], Mik[3][3];
  for (int i = 0; i < 3; ++i) {
    double acc = 0.0;
    for (int c = 0; c < 4; ++c)
      for (int dd = 0; dd < 4; ++dd) acc += S.t_up[c] * S.t_up[dd] * Phi[i * 10 + sym_index(c, dd)];
    tPhit[i] = acc;
    for (int j = 0; j < 3; ++j) {
      double t2 = 0.0;
      for (int c = 0; c < 4; ++c) t2 += S.t_up[c] * Phi[i * 10 + sym_index(1 + j, c)];
      tPhij[i][j] = t2;
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k)
      Mik[i][k] = tPhij[i][0] * S.ginv[s3h(0, k)] + tPhij[i][1] * S.ginv[s3h(1, k)] + tPhij[i][2] * S.ginv[s3h(2, k)];
  double bs[3], Gs[3][3];
  for (int dd = 0; dd < 3; ++dd) {
    bs[dd] = S.beta_up[0] * J[0][dd] + S.beta_up[1] * J[1][dd] + S.beta_up[2] * J[2][dd];
    for (int i = 0; i < 3; ++i)
      Gs[i][dd] = S.ginv[s3h(0, i)] * J[0][dd] + S.ginv[s3h(1, i)] * J[1][dd] + S.ginv[s3h(2, i)] * J[2][dd];
  }
  // ---- adjoint accumulators
  double* psib = ub;
  double* Pib = ub + 10;
  double* Phib = ub + 20;
  double alb = 0.0, betab[3] = {0.0, 0.0, 0.0}, ginvb[6] = {0, 0, 0, 0, 0, 0}, tb[4] = {0.0, 0.0, 0.0, 0.0};
  double pinvb[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  double Gamb[40];
  for (int e = 0; e < 40; ++e) Gamb[e] = 0.0;
  double Cb[4] = {0.0, 0.0, 0.0, 0.0}, PHb[4] = {0.0, 0.0, 0.0, 0.0};
  double PmbA[16], PmbB[16], WmbA[3][4];
  for (int e = 0; e < 16; ++e) PmbA[e] = PmbB[e] = 0.0;
  for (int j = 0; j < 3; ++j)
    for (int dd = 0; dd < 4; ++dd) WmbA[j][dd] = 0.0;
  double tPtb = 0.0, tCb = 0.0, tPigb[3] = {0.0, 0.0, 0.0}, tPhitb[3] = {0.0, 0.0, 0.0};
  double Mikb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double bsb[3] = {0.0, 0.0, 0.0}, Gsb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  const double* dpsi = dsp;
  const double* dPi = dsp + 3;
  double* dpsib = dsb15;
  double* dPib = dsb15 + 3;
  for (int e = 0; e < 15; ++e) dsb15[e] = 0.0;
  const double kpsi = kb5[0], kPi = kb5[1];
  // ---- the pair's forward scalars
  double T1 = 0.0, T2 = 0.0, T3 = 0.0;
  for (int j = 0; j < 3; ++j)
    for (int dd = 0; dd < 4; ++dd) T1 += WmA[j][dd] * Phi[j * 10 + sym_index(dd, B)];
  double pcv[4];
  for (int c = 0; c < 4; ++c) {
    double pc = 0.0;
    for (int dd = 0; dd < 4; ++dd) pc += S.psi_inv[sym_index(c, dd)] * Pi[sym_index(dd, B)];
    pcv[c] = pc;
    T2 += Pi[sym_index(c, A)] * pc;
  }
  for (int dd = 0; dd < 4; ++dd)
    for (int e = 0; e < 4; ++e) T3 += PmA[dd * 4 + e] * PmB[e * 4 + dd];
  const double dAHB = (A > 0 ? dH[4 * (A - 1) + B] : 0.0);
  const double dBHA = (B > 0 ? dH[4 * (B - 1) + A] : 0.0);
  double gh_ = 0.0;
  for (int dd = 0; dd < 4; ++dd) gh_ += PH[dd] * Gam[dd * 10 + p];
  const double nablaH = 0.5 * (dAHB + dBHA) - gh_;
  const double damp = (B == 0 ? -al * C[A] : 0.0) + (A == 0 ? -al * C[B] : 0.0) - psi[p] * tC;
  double tPiPhi = 0.0;
  for (int j = 0; j < 3; ++j) tPiPhi += tPig[j] * Phi[j * 10 + p];
  double gdPhi = 0.0;
  for (int i = 0; i < 3; ++i) {
    const double* dPhi = dsp + 6 + 3 * i;
    gdPhi += Gs[i][0] * dPhi[0] + Gs[i][1] * dPhi[1] + Gs[i][2] * dPhi[2];
  }
  // ---- out[p] = (1+g1) bdpsi - al Pi_p - g1 bPhi
  double bdpsib = (1.0 + g1) * kpsi;
  alb -= Pi[p] * kpsi;
  Pib[p] -= al * kpsi;
  double bPhib = -g1 * kpsi;
  // ---- out[10+p] = bdPi - al gdPhi + g1 g2 bdpsi + srcPi
  const double bdPib = kPi;
  alb -= gdPhi * kPi;
  const double gdPhib = -al * kPi;
  bdpsib += g1 * g2 * kPi;
  const double sPb = kPi;
  // ---- out[20+10i+p]
  double cpsib[3], cPib[3];
  for (int i = 0; i < 3; ++i) {
    const double kPhi = kb5[2 + i];
    const double* dPhi = dsp + 6 + 3 * i;
    double* dPhib = dsb15 + 6 + 3 * i;
    const double cpsi = J[i][0] * dpsi[0] + J[i][1] * dpsi[1] + J[i][2] * dpsi[2];
    const double cPi = J[i][0] * dPi[0] + J[i][1] * dPi[1] + J[i][2] * dPi[2];
    for (int dd = 0; dd < 3; ++dd) {
      dPhib[dd] += bs[dd] * kPhi;
      bsb[dd] += dPhi[dd] * kPhi;
    }
    alb += (-cPi + g2 * cpsi) * kPhi;
    cPib[i] = -al * kPhi;
    cpsib[i] = al * g2 * kPhi;
    const double mphi = Mik[i][0] * Phi[p] + Mik[i][1] * Phi[10 + p] + Mik[i][2] * Phi[20 + p];
    alb += (0.5 * tPhit[i] * Pi[p] + mphi - g2 * Phi[i * 10 + p]) * kPhi;
    tPhitb[i] += 0.5 * al * Pi[p] * kPhi;
    Pib[p] += 0.5 * al * tPhit[i] * kPhi;
    for (int k = 0; k < 3; ++k) {
      Mikb[i][k] += al * Phi[k * 10 + p] * kPhi;
      Phib[k * 10 + p] += al * Mik[i][k] * kPhi;
    }
    Phib[i * 10 + p] -= al * g2 * kPhi;
  }
  for (int dd = 0; dd < 3; ++dd) {
    dpsib[dd] += J[0][dd] * cpsib[0] + J[1][dd] * cpsib[1] + J[2][dd] * cpsib[2];
    dPib[dd] += J[0][dd] * cPib[0] + J[1][dd] * cPib[1] + J[2][dd] * cPib[2];
  }
  for (int dd = 0; dd < 3; ++dd) {
    dpsib[dd] += bs[dd] * bdpsib;
    bsb[dd] += dpsi[dd] * bdpsib;
    dPib[dd] += bs[dd] * bdPib;
    bsb[dd] += dPi[dd] * bdPib;
  }
  for (int i = 0; i < 3; ++i) {
    const double* dPhi = dsp + 6 + 3 * i;
    double* dPhib = dsb15 + 6 + 3 * i;
    for (int dd = 0; dd < 3; ++dd) {
      dPhib[dd] += Gs[i][dd] * gdPhib;
      Gsb[i][dd] += dPhi[dd] * gdPhib;
    }
  }
  // ---- srcPi = 2al(T1-T2-T3) - 2al nablaH - 0.5 al tPt Pi_p - al tPiPhi + g0 al damp - g1 g2 bPhi
  alb += sPb * (2.0 * (T1 - T2 - T3) - 2.0 * nablaH - 0.5 * tPt * Pi[p] - tPiPhi + g0 * damp);
  const double T1b = 2.0 * al * sPb, T2b = -2.0 * al * sPb, T3b = -2.0 * al * sPb;
  const double nHb = -2.0 * al * sPb;
  tPtb += -0.5 * al * Pi[p] * sPb;
  Pib[p] += -0.5 * al * tPt * sPb;
  const double tPiPhib = -al * sPb;
  const double dampb = g0 * al * sPb;
  bPhib += -g1 * g2 * sPb;
  for (int j = 0; j < 3; ++j)
    for (int dd = 0; dd < 4; ++dd) {
      WmbA[j][dd] += Phi[j * 10 + sym_index(dd, B)] * T1b;
      Phib[j * 10 + sym_index(dd, B)] += WmA[j][dd] * T1b;
    }
  for (int c = 0; c < 4; ++c) {
    Pib[sym_index(c, A)] += pcv[c] * T2b;
    const double pcb = Pi[sym_index(c, A)] * T2b;
    for (int dd = 0; dd < 4; ++dd) {
      pinvb[sym_index(c, dd)] += Pi[sym_index(dd, B)] * pcb;
      Pib[sym_index(dd, B)] += S.psi_inv[sym_index(c, dd)] * pcb;
    }
  }
  for (int dd = 0; dd < 4; ++dd)
    for (int e = 0; e < 4; ++e) {
      PmbA[dd * 4 + e] += PmB[e * 4 + dd] * T3b;
      PmbB[e * 4 + dd] += PmA[dd * 4 + e] * T3b;
    }
  for (int dd = 0; dd < 4; ++dd) {
    PHb[dd] -= Gam[dd * 10 + p] * nHb;
    Gamb[dd * 10 + p] -= PH[dd] * nHb;
  }
  if (B == 0) {
    alb -= C[A] * dampb;
    Cb[A] -= al * dampb;
  }
  if (A == 0) {
    alb -= C[B] * dampb;
    Cb[B] -= al * dampb;
  }
  psib[p] -= tC * dampb;
  tCb -= psi[p] * dampb;
  for (int j = 0; j < 3; ++j) {
    tPigb[j] += Phi[j * 10 + p] * tPiPhib;
    Phib[j * 10 + p] += tPig[j] * tPiPhib + S.beta_up[j] * bPhib;
    betab[j] += Phi[j * 10 + p] * bPhib;
  }
  // ---- reverse of the pair-independent pieces (restricted where possible)
  for (int dd = 0; dd < 3; ++dd) {
    for (int k = 0; k < 3; ++k) betab[k] += J[k][dd] * bsb[dd];
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) ginvb[s3h(k, i)] += J[k][dd] * Gsb[i][dd];
  }
  for (int i = 0; i < 3; ++i) {
    double tPhijb[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) {
        tPhijb[j] += S.ginv[s3h(j, k)] * Mikb[i][k];
        ginvb[s3h(j, k)] += tPhij[i][j] * Mikb[i][k];
      }
    for (int j = 0; j < 3; ++j)
      for (int c = 0; c < 4; ++c) {
        tb[c] += Phi[i * 10 + sym_index(1 + j, c)] * tPhijb[j];
        Phib[i * 10 + sym_index(1 + j, c)] += S.t_up[c] * tPhijb[j];
      }
    for (int c = 0; c < 4; ++c)
      for (int dd = 0; dd < 4; ++dd) {
        const double ph = Phi[i * 10 + sym_index(c, dd)];
        tb[c] += S.t_up[dd] * ph * tPhitb[i];
        tb[dd] += S.t_up[c] * ph * tPhitb[i];
        Phib[i * 10 + sym_index(c, dd)] += S.t_up[c] * S.t_up[dd] * tPhitb[i];
      }
  }
  // Wm[j][d][A] = sum_i ginv(i,j) Um[i][d][A] ; Um[i][d][A] = sum_c psi_inv(d,c) Phi_i(c,A)
  for (int i = 0; i < 3; ++i) {
    double UmbA[4];
    for (int dd = 0; dd < 4; ++dd) {
      UmbA[dd] = S.ginv[s3h(i, 0)] * WmbA[0][dd] + S.ginv[s3h(i, 1)] * WmbA[1][dd] + S.ginv[s3h(i, 2)] * WmbA[2][dd];
      for (int j = 0; j < 3; ++j) ginvb[s3h(i, j)] += UmA[i][dd] * WmbA[j][dd];
    }
    for (int dd = 0; dd < 4; ++dd)
      for (int c = 0; c < 4; ++c) {
        pinvb[sym_index(dd, c)] += Phi[i * 10 + sym_index(c, A)] * UmbA[dd];
        Phib[i * 10 + sym_index(c, A)] += S.psi_inv[sym_index(dd, c)] * UmbA[dd];
      }
  }
  // Pm[a][d][e] = sum_c psi_inv(d,c) Gam[a](c,e) for a = A and a = B
  for (int w = 0; w < 2; ++w) {
    const int a = (w == 0) ? A : B;
    const double* Pb = (w == 0) ? PmbA : PmbB;
    for (int dd = 0; dd < 4; ++dd)
      for (int e = 0; e < 4; ++e)
        for (int c = 0; c < 4; ++c) {
          pinvb[sym_index(dd, c)] += Gam[a * 10 + sym_index(c, e)] * Pb[dd * 4 + e];
          Gamb[a * 10 + sym_index(c, e)] += S.psi_inv[sym_index(dd, c)] * Pb[dd * 4 + e];
        }
  }
  for (int dd = 0; dd < 4; ++dd)
    for (int c = 0; c < 4; ++c) pinvb[sym_index(c, dd)] += H[c] * PHb[dd];
  double tPib[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) {
      tPib[i] += S.ginv[s3h(i, j)] * tPigb[j];
      ginvb[s3h(i, j)] += tPi[i] * tPigb[j];
    }
  for (int c = 0; c < 4; ++c) {
    for (int i = 0; i < 3; ++i) {
      tb[c] += Pi[sym_index(c, 1 + i)] * tPib[i];
      Pib[sym_index(c, 1 + i)] += S.t_up[c] * tPib[i];
    }
    for (int dd = 0; dd < 4; ++dd) {
      const double pv = Pi[sym_index(c, dd)];
      tb[c] += S.t_up[dd] * pv * tPtb;
      tb[dd] += S.t_up[c] * pv * tPtb;
      Pib[sym_index(c, dd)] += S.t_up[c] * S.t_up[dd] * tPtb;
    }
    tb[c] += C[c] * tCb;
    Cb[c] += S.t_up[c] * tCb;
  }
  gamma_split_reverse(psi, Pi, Phi, S, Gam, Cb, Gamb, alb, betab, ginvb, tb, pinvb, psib, Pib, Phib);
}

// Constraint-energy gradient restricted to pair p: the C_iab and C_ijab terms
// of pair p (which read only pair p's derivatives) and, for p == 0, the C_a
// term.  Adds w * de/d(inputs) to ub[50] and dsb15 (pair p's derivatives).
GH_HD inline void point_constraint_energy_pair(const double* u, const double J[3][3], const double H[4], int p,
                                               const double dsp[15], double w, double ub[50], double dsb15[15]) {
  const double* Phi = u + 20;
  double cpsi[3], cPhi[3][3];   // cPhi[j][i] = d_i Phi_jp
  for (int i = 0; i < 3; ++i) {
    cpsi[i] = J[i][0] * dsp[0] + J[i][1] * dsp[1] + J[i][2] * dsp[2];
    for (int j = 0; j < 3; ++j)
      cPhi[j][i] = J[i][0] * dsp[6 + 3 * j] + J[i][1] * dsp[7 + 3 * j] + J[i][2] * dsp[8 + 3 * j];
  }
  double cpsib[3] = {0.0, 0.0, 0.0}, cPhib[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int i = 0; i < 3; ++i) {
    const double c3 = cpsi[i] - Phi[i * 10 + p];
    cpsib[i] += 2.0 * w * c3;
    ub[20 + i * 10 + p] -= 2.0 * w * c3;
  }
  const int qi[3] = {0, 0, 1}, qj[3] = {1, 2, 2};
  for (int q = 0; q < 3; ++q) {
    const int i = qi[q], j = qj[q];
    const double c4 = cPhi[j][i] - cPhi[i][j];
    cPhib[j][i] += 2.0 * w * c4;
    cPhib[i][j] -= 2.0 * w * c4;
  }
  for (int dd = 0; dd < 3; ++dd) {
    dsb15[dd] += J[0][dd] * cpsib[0] + J[1][dd] * cpsib[1] + J[2][dd] * cpsib[2];
    for (int j = 0; j < 3; ++j)
      dsb15[6 + 3 * j + dd] += J[0][dd] * cPhib[j][0] + J[1][dd] * cPhib[j][1] + J[2][dd] * cPhib[j][2];
  }
  if (p != 0) return;
  const double* psi = u;
  const double* Pi = u + 10;
  Split S;
  point_split(psi, S);
  double d[40], Gam[40];
  for (int q = 0; q < 10; ++q) {
    d[q] = -S.alpha * Pi[q] + S.beta_up[0] * Phi[q] + S.beta_up[1] * Phi[10 + q] + S.beta_up[2] * Phi[20 + q];
    for (int i = 0; i < 3; ++i) d[10 * (1 + i) + q] = Phi[10 * i + q];
  }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = b; c < 4; ++c)
        Gam[a * 10 + sym_index(b, c)] =
            0.5 * (d[b * 10 + sym_index(a, c)] + d[c * 10 + sym_index(a, b)] - d[a * 10 + sym_index(b, c)]);
  double Cb[4];
  for (int a = 0; a < 4; ++a) {
    double acc = 0.0;
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) acc += S.psi_inv[sym_index(b, c)] * Gam[a * 10 + sym_index(b, c)];
    Cb[a] = 2.0 * w * (H[a] + acc);
  }
  double Gamb[40];
  for (int q = 0; q < 40; ++q) Gamb[q] = 0.0;
  double alb = 0.0, betab[3] = {0, 0, 0}, ginvb[6] = {0, 0, 0, 0, 0, 0}, tb[4] = {0, 0, 0, 0};
  double pinvb[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  gamma_split_reverse(psi, Pi, Phi, S, Gam, Cb, Gamb, alb, betab, ginvb, tb, pinvb, ub, ub + 10, ub + 20);
}

}  // namespace gh
