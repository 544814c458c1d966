// Pointwise GH tensor algebra shared by the RHS, constraint and boundary
// kernels (device code, FP64).  Everything here works on one grid point held
// in registers / local arrays.
//
// Conventions: symmetric pairs packed as p(a,b), a <= b, in the order
// 00,01,02,03,11,12,13,22,23,33; spacetime index 0 is t, 1..3 are x,y,z.
#pragma once

namespace gh {

__host__ __device__ constexpr int sym_index(int a, int b) {
  // packed index of the symmetric pair (a, b)
  return (a <= b) ? (a == 0 ? b : (a == 1 ? 3 + b : (a == 2 ? 5 + b : 9)))
                  : (b == 0 ? a : (b == 1 ? 3 + a : (b == 2 ? 5 + a : 9)));
}

__host__ __device__ constexpr int pair_a(int p) {
  return p < 4 ? 0 : (p < 7 ? 1 : (p < 9 ? 2 : 3));
}
__host__ __device__ constexpr int pair_b(int p) {
  return p < 4 ? p : (p < 7 ? p - 3 : (p < 9 ? p - 5 : 3));
}

// 3+1 quantities of a spacetime metric psi_ab (packed).
struct Split {
  double ginv[6];       // g^ij packed (xx, xy, xz, yy, yz, zz)
  double beta_up[3];    // beta^i
  double alpha;
  double t_up[4];       // t^a
  double psi_inv[10];   // psi^ab packed
};

__device__ __forceinline__ int s3(int i, int j) {
  // packed index of a symmetric 3x3 pair
  int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

__device__ __forceinline__ void spacetime_split(const double psi[10], Split& s) {
  // spatial metric g_ij = psi_ij
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
  const double ia = 1.0 / s.alpha;
  const double ia2 = ia * ia;
  s.t_up[0] = ia;
  s.t_up[1] = -s.beta_up[0] * ia;
  s.t_up[2] = -s.beta_up[1] * ia;
  s.t_up[3] = -s.beta_up[2] * ia;
  s.psi_inv[0] = -ia2;
  s.psi_inv[1] = s.beta_up[0] * ia2;
  s.psi_inv[2] = s.beta_up[1] * ia2;
  s.psi_inv[3] = s.beta_up[2] * ia2;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j)
      s.psi_inv[sym_index(1 + i, 1 + j)] = s.ginv[s3(i, j)] - s.beta_up[i] * s.beta_up[j] * ia2;
}

// d_c psi_ab = t_c Pi_ab + g^i_c Phi_iab with t_c = (-alpha, 0,0,0) and
// g^i_0 = beta^i, g^i_j = delta^i_j.  Returns Gam[a][p(b,c)] =
// (d_b psi_ac + d_c psi_ab - d_a psi_bc)/2.
__device__ __forceinline__ void christoffel(const Split& s, const double Pi[10],
                                            const double Phi[30], double Gam[40]) {
  double d[40];  // d[c*10 + p(a,b)]
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    d[p] = -s.alpha * Pi[p] + s.beta_up[0] * Phi[p] + s.beta_up[1] * Phi[10 + p] +
           s.beta_up[2] * Phi[20 + p];
    d[10 + p] = Phi[p];
    d[20 + p] = Phi[10 + p];
    d[30 + p] = Phi[20 + p];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = b; c < 4; ++c)
        Gam[a * 10 + sym_index(b, c)] =
            0.5 * (d[b * 10 + sym_index(a, c)] + d[c * 10 + sym_index(a, b)] -
                   d[a * 10 + sym_index(b, c)]);
}

// Gamma_a = psi^bc Gamma_abc.
__device__ __forceinline__ void trace_gamma(const Split& s, const double Gam[40], double Ga[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        acc += s.psi_inv[sym_index(b, c)] * Gam[a * 10 + sym_index(b, c)];
    Ga[a] = acc;
  }
}

}  // namespace gh
