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
