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

}  // namespace gh
