// Host build of the library's per-point GH algebra (csrc/gh_point.cuh) for
// unit tests on the CPU: forward right-hand side, its reverse pass, and the
// constraint energy with its gradient.  Test code only; not part of libgh.
#define __host__
#define __device__
#define __forceinline__ inline
#include <cmath>
using std::sqrt;
#include "../paper_1804_09101_gb300/csrc/gh_point.cuh"

static gh::PointIn make_in(const double* u, const double* ds, const double* J, const double* H, const double* dH,
                           double g0, double g1, double g2) {
  gh::PointIn in;
  in.u = u;
  in.ds = ds;
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) in.J[i][d] = J[3 * i + d];
  in.H = H;
  in.dH = dH;
  in.g0 = g0;
  in.g1 = g1;
  in.g2 = g2;
  return in;
}

extern "C" {
void h_point_rhs(const double* u, const double* ds, const double* J, const double* H, const double* dH, double g0,
                 double g1, double g2, double* out) {
  gh::PointIn in = make_in(u, ds, J, H, dH, g0, g1, g2);
  gh::PointFwd f;
  gh::point_rhs(in, f, out);
}

void h_point_rhs_vjp(const double* u, const double* ds, const double* J, const double* H, const double* dH,
                     double g0, double g1, double g2, const double* kb, double* ub, double* dsb) {
  gh::PointIn in = make_in(u, ds, J, H, dH, g0, g1, g2);
  gh::PointFwd f;
  double out[50];
  gh::point_rhs(in, f, out);
  gh::point_rhs_vjp(in, f, kb, ub, dsb);
}

double h_point_constraint_energy(const double* u, const double* ds, const double* J, const double* H,
                                 const double* dH, double w, double* ub, double* dsb) {
  gh::PointIn in = make_in(u, ds, J, H, dH, 1.0, -1.0, 1.0);
  return gh::point_constraint_energy(in, w, ub, dsb);
}
}

extern "C" void h_point_rhs_vjp_and_constraint(const double* u, const double* ds, const double* J, const double* H,
                                               const double* dH, double g0, double g1, double g2, const double* kb,
                                               double w, double* ub, double* dsb) {
  gh::PointIn in = make_in(u, ds, J, H, dH, g0, g1, g2);
  gh::PointFwd f;
  double out[50];
  gh::point_rhs(in, f, out);
  gh::point_rhs_vjp(in, f, kb, ub, dsb);
  gh::point_constraint_energy(in, w, ub, dsb);
}

// Sum over the ten symmetric pairs of the pair-restricted reverse passes (and
// constraint-energy gradients): must equal the full reverse pass.
extern "C" void h_point_vjp_pairsum(const double* u, const double* ds, const double* J, const double* H,
                                    const double* dH, double g0, double g1, double g2, const double* kb, double w,
                                    double* ub, double* dsb) {
  double Jm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) Jm[i][d] = J[3 * i + d];
  for (int p = 0; p < 10; ++p) {
    const int f[5] = {p, 10 + p, 20 + p, 30 + p, 40 + p};
    double dsp[15], kb5[5], dsb15[15];
    for (int e = 0; e < 5; ++e) {
      kb5[e] = kb[f[e]];
      for (int d = 0; d < 3; ++d) dsp[3 * e + d] = ds[3 * f[e] + d];
    }
    gh::point_rhs_vjp_pair(u, Jm, H, dH, g0, g1, g2, p, dsp, kb5, ub, dsb15);
    if (w != 0.0) gh::point_constraint_energy_pair(u, Jm, H, p, dsp, w, ub, dsb15);
    for (int e = 0; e < 5; ++e)
      for (int d = 0; d < 3; ++d) dsb[3 * f[e] + d] += dsb15[3 * e + d];
  }
}
