// Shared device helpers: block-to-shell lookup and the per-point DiffJac
// geometry (used by the forward and the adjoint kernels).
#pragma once

#include "gh_internal.h"

namespace gh {

// ---------------------------------------------------------------------------
// Block -> shell lookup: begin[s] is the first block of shell s, begin[n] the
// total.  n is small (tens), so a linear scan is enough.
__device__ __forceinline__ int find_segment(const int* begin, int n, int b) {
  int s = 0;
  while (s + 1 < n && begin[s + 1] <= b) ++s;
  return s;
}

// ---------------------------------------------------------------------------
// Geometry of one point: the DiffJac matrix J[i][d] = d(x_d)/d(x^i) for the
// spherical coordinates (r, theta, phi), with the radial column multiplied by
// dx/dr so that it acts on the CGL-coordinate derivative (Eq. DiffJac).
struct PointGeom {
  double J[3][3];
  double xhat[3];  // x^i / R
  double r;
};

__device__ __forceinline__ void point_geom(const ShellDev& sh, int ir, int q, PointGeom& g) {
  const int j = q / sh.nph, k = q - j * sh.nph;
  const double r = sh.r[ir];
  const double ct = sh.cth[j], st = sh.sth[j], cp = sh.cph[k], sp = sh.sph[k];
  const double ir_ = 1.0 / r;
  const double irs = ir_ / st;
  g.r = r;
  g.xhat[0] = st * cp; g.xhat[1] = st * sp; g.xhat[2] = ct;
  g.J[0][0] = st * cp * sh.rscale; g.J[0][1] = ct * cp * ir_; g.J[0][2] = -sp * irs;
  g.J[1][0] = st * sp * sh.rscale; g.J[1][1] = ct * sp * ir_; g.J[1][2] = cp * irs;
  g.J[2][0] = ct * sh.rscale;      g.J[2][1] = -st * ir_;     g.J[2][2] = 0.0;
}

// ---------------------------------------------------------------------------
constexpr int PERT_LMAX = 16;

// Normalised associated Legendre functions (orthonormal real harmonics, no
// Condon-Shortley phase) and their theta derivatives from
//   sin(th) dP_l^m/dth = l cos(th) P_l^m - sqrt((2l+1)(l^2-m^2)/(2l-1)) P_{l-1}^m.
__device__ inline void legendre_table(int lmax, double ct, double st, double* P, double* dP) {
  const int W = PERT_LMAX + 1;
  for (int i = 0; i < W * W; ++i) { P[i] = 0.0; dP[i] = 0.0; }
  P[0] = sqrt(0.25 / 3.14159265358979323846);
  for (int m = 1; m <= lmax; ++m) P[m * W + m] = sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * P[(m - 1) * W + m - 1];
  for (int m = 0; m < lmax; ++m) P[(m + 1) * W + m] = sqrt(2.0 * m + 3.0) * ct * P[m * W + m];
  for (int m = 0; m <= lmax; ++m)
    for (int l = m + 2; l <= lmax; ++l) {
      const double al = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
      const double bl = sqrt((((double)l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
      P[l * W + m] = al * (ct * P[(l - 1) * W + m] - bl * P[(l - 2) * W + m]);
    }
  for (int l = 0; l <= lmax; ++l)
    for (int m = 0; m <= l; ++m) {
      const double prev = (l > m) ? P[(l - 1) * W + m] : 0.0;
      const double c = (l > m) ? sqrt((2.0 * l + 1.0) * ((double)l * l - (double)m * m) / (2.0 * l - 1.0)) : 0.0;
      dP[l * W + m] = (l * ct * P[l * W + m] - c * prev) / st;
    }
}

// Moving frame: DiffJac followed by the map's Jacobian, J <- R J (the
// SpatialCoordJac of Sec. 3.3 for a rotation; J <- R J / a with the
// expansion of a general map), and the grid velocity w x (x - T) at the point
// (plus (adot / a)(x - T) + V for a general map), x - T = a R x_grid.
__device__ __forceinline__ void frame_geom(const Frame& fr, PointGeom& G, double vel[3]) {
  double J2[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d)
      J2[k][d] = fma(fr.R[3 * k + 2], G.J[2][d], fma(fr.R[3 * k + 1], G.J[1][d], fr.R[3 * k] * G.J[0][d]));
  const double ia = fr.gen ? 1.0 / fr.a : 1.0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int d = 0; d < 3; ++d) G.J[k][d] = fr.gen ? J2[k][d] * ia : J2[k][d];
  const double rr = fr.gen ? fr.a * G.r : G.r;
  double xi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    xi[k] = rr * fma(fr.R[3 * k + 2], G.xhat[2], fma(fr.R[3 * k + 1], G.xhat[1], fr.R[3 * k] * G.xhat[0]));
  vel[0] = fr.w[1] * xi[2] - fr.w[2] * xi[1];
  vel[1] = fr.w[2] * xi[0] - fr.w[0] * xi[2];
  vel[2] = fr.w[0] * xi[1] - fr.w[1] * xi[0];
  if (fr.gen) {
    const double h = fr.adot * ia;
#pragma unroll
    for (int k = 0; k < 3; ++k) vel[k] += fma(h, xi[k], fr.V[k]);
  }
}

// Gauge source of a background invariant under the rotation, at the moving
// point: H_a -> Lambda_a^b H_b, d_i H_a -> R_ij Lambda_a^b d_j H_b.
__device__ __forceinline__ void frame_rotate_h(const Frame& fr, double H[4]) {
  const double h1 = H[1], h2 = H[2], h3 = H[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) H[1 + i] = fma(fr.R[3 * i + 2], h3, fma(fr.R[3 * i + 1], h2, fr.R[3 * i] * h1));
}
__device__ __forceinline__ void frame_rotate_dh(const Frame& fr, double dH[12]) {
  double t[12];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 4; ++a)
      t[4 * i + a] = fma(fr.R[3 * i + 2], dH[8 + a], fma(fr.R[3 * i + 1], dH[4 + a], fr.R[3 * i] * dH[a]));
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dH[4 * i] = t[4 * i];
#pragma unroll
    for (int a = 0; a < 3; ++a)
      dH[4 * i + 1 + a] = fma(fr.R[3 * a + 2], t[4 * i + 3], fma(fr.R[3 * a + 1], t[4 * i + 2], fr.R[3 * a] * t[4 * i + 1]));
  }
}

// The boundary background's vectors at the moving point: n_i, n^i, beta^i
// rotated (lapse and speeds do not change).
__device__ __forceinline__ void frame_rotate_bg(const Frame& fr, double n_dn[3], double n_up[3], double beta[3]) {
  double t1[3], t2[3], t3[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    t1[i] = fma(fr.R[3 * i + 2], n_dn[2], fma(fr.R[3 * i + 1], n_dn[1], fr.R[3 * i] * n_dn[0]));
    t2[i] = fma(fr.R[3 * i + 2], n_up[2], fma(fr.R[3 * i + 1], n_up[1], fr.R[3 * i] * n_up[0]));
    t3[i] = fma(fr.R[3 * i + 2], beta[2], fma(fr.R[3 * i + 1], beta[1], fr.R[3 * i] * beta[0]));
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    n_dn[i] = t1[i];
    n_up[i] = t2[i];
    beta[i] = t3[i];
  }
}

}  // namespace gh
