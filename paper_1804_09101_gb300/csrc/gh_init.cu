// Initial data on the device: the analytic Kerr-Schild solution with its
// gauge source (Sec. 3.1), and seeded-coefficient perturbations.
//
// Derivatives of the metric come from forward-mode second-order jets (value,
// gradient and Hessian in x, y, z carried through every arithmetic
// operation), so d_i g_ab and d_i d_j g_ab are exact to rounding.
#include <cuda_runtime.h>

#include "gh_geom.cuh"
#include "gh_internal.h"
#include "gh_tensor.cuh"

namespace gh {

// ---------------------------------------------------------------- jets
struct Jet {
  double v;
  double g[3];
  double h[6];  // xx xy xz yy yz zz
};

__device__ __forceinline__ int h3(int i, int j) {
  int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

__device__ __forceinline__ Jet jconst(double c) {
  Jet r;
  r.v = c;
  for (int i = 0; i < 3; ++i) r.g[i] = 0.0;
  for (int i = 0; i < 6; ++i) r.h[i] = 0.0;
  return r;
}
__device__ __forceinline__ Jet jvar(double x, int i) {
  Jet r = jconst(x);
  r.g[i] = 1.0;
  return r;
}
__device__ __forceinline__ Jet operator+(const Jet& a, const Jet& b) {
  Jet r;
  r.v = a.v + b.v;
  for (int i = 0; i < 3; ++i) r.g[i] = a.g[i] + b.g[i];
  for (int i = 0; i < 6; ++i) r.h[i] = a.h[i] + b.h[i];
  return r;
}
__device__ __forceinline__ Jet operator-(const Jet& a, const Jet& b) {
  Jet r;
  r.v = a.v - b.v;
  for (int i = 0; i < 3; ++i) r.g[i] = a.g[i] - b.g[i];
  for (int i = 0; i < 6; ++i) r.h[i] = a.h[i] - b.h[i];
  return r;
}
__device__ __forceinline__ Jet operator*(double c, const Jet& a) {
  Jet r;
  r.v = c * a.v;
  for (int i = 0; i < 3; ++i) r.g[i] = c * a.g[i];
  for (int i = 0; i < 6; ++i) r.h[i] = c * a.h[i];
  return r;
}
__device__ __forceinline__ Jet operator*(const Jet& a, const Jet& b) {
  Jet r;
  r.v = a.v * b.v;
  for (int i = 0; i < 3; ++i) r.g[i] = a.v * b.g[i] + a.g[i] * b.v;
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j)
      r.h[h3(i, j)] = a.v * b.h[h3(i, j)] + a.g[i] * b.g[j] + a.g[j] * b.g[i] + a.h[h3(i, j)] * b.v;
  return r;
}
// unary chain rule: f(a) with f' = d1, f'' = d2 at a.v
__device__ __forceinline__ Jet chain(const Jet& a, double f0, double d1, double d2) {
  Jet r;
  r.v = f0;
  for (int i = 0; i < 3; ++i) r.g[i] = d1 * a.g[i];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) r.h[h3(i, j)] = d1 * a.h[h3(i, j)] + d2 * a.g[i] * a.g[j];
  return r;
}
__device__ __forceinline__ Jet jinv(const Jet& a) {
  const double iv = 1.0 / a.v;
  return chain(a, iv, -iv * iv, 2.0 * iv * iv * iv);
}
__device__ __forceinline__ Jet jsqrt(const Jet& a) {
  const double s = sqrt(a.v);
  return chain(a, s, 0.5 / s, -0.25 / (s * a.v));
}
__device__ __forceinline__ Jet operator/(const Jet& a, const Jet& b) { return a * jinv(b); }

// Value-only counterparts of the jet constructors and unary maps, so one
// template gives either the metric's values or its second-order jets.
template <class T> __device__ __forceinline__ T kvar(double x, int i);
template <> __device__ __forceinline__ Jet kvar<Jet>(double x, int i) { return jvar(x, i); }
template <> __device__ __forceinline__ double kvar<double>(double x, int) { return x; }
template <class T> __device__ __forceinline__ T kconst(double c);
template <> __device__ __forceinline__ Jet kconst<Jet>(double c) { return jconst(c); }
template <> __device__ __forceinline__ double kconst<double>(double c) { return c; }
__device__ __forceinline__ double jinv(double a) { return 1.0 / a; }
__device__ __forceinline__ double jsqrt(double a) { return sqrt(a); }

// Kerr-Schild form g_ab = eta_ab + 2 H l_a l_b for the spin vector a = chi M
// (any direction): with a.x the Euclidean dot product and a x x the cross product,
//   r^2 = (R^2 - a^2)/2 + sqrt((R^2 - a^2)^2/4 + (a.x)^2),  H = M r^3 / (r^4 + (a.x)^2),
//   l = (1, (r x_i - (a x x)_i + (a.x) a_i / r) / (r^2 + a^2)).
// Returns H and the spatial l_1..l_3 (l_0 = 1).
template <class T>
__device__ __forceinline__ void kerr_schild_fields(double x, double y, double z, double M, const double av[3], T& H,
                                                   T l[3]) {
  const T X = kvar<T>(x, 0), Y = kvar<T>(y, 1), Z = kvar<T>(z, 2);
  const double ax = av[0], ay = av[1], az = av[2];
  const T a2 = kconst<T>(ax * ax + ay * ay + az * az);
  const T ad = ax * X + ay * Y + az * Z;
  const T R2 = X * X + Y * Y + Z * Z;
  const T hm = 0.5 * (R2 - a2);
  const T ad2 = ad * ad;
  const T r2 = hm + jsqrt(hm * hm + ad2);
  const T r = jsqrt(r2);
  H = M * (r * r2) / (r2 * r2 + ad2);
  const T den = jinv(r2 + a2);
  const T adr = ad / r;
  const T cx = ay * Z - az * Y, cy = az * X - ax * Z, cz = ax * Y - ay * X;
  l[0] = (r * X - cx + ax * adr) * den;
  l[1] = (r * Y - cy + ay * adr) * den;
  l[2] = (r * Z - cz + az * adr) * den;
}

__device__ void kerr_schild_metric(double x, double y, double z, double M, const double av[3], Jet g[10]) {
  Jet H, ls[3];
  kerr_schild_fields(x, y, z, M, av, H, ls);
  const Jet l[4] = {jconst(1.0), ls[0], ls[1], ls[2]};
  const Jet twoH = 2.0 * H;
  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
    const double eta = (A == B) ? (A == 0 ? -1.0 : 1.0) : 0.0;
    g[p] = jconst(eta) + twoH * (l[A] * l[B]);
  }
}

// The metric's values alone (no derivatives).
__device__ void kerr_schild_values(double x, double y, double z, double M, const double av[3], double psi[10]) {
  double H, ls[3];
  kerr_schild_fields(x, y, z, M, av, H, ls);
  const double l[4] = {1.0, ls[0], ls[1], ls[2]};
#pragma unroll
  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
    const double eta = (A == B) ? (A == 0 ? -1.0 : 1.0) : 0.0;
    psi[p] = eta + 2.0 * H * (l[A] * l[B]);
  }
}

// The Kerr-Schild gauge source in closed form. For g = eta + 2 H l l with l
// null under eta, det g = det eta = -1 (matrix determinant lemma), so
// g^bc d_a g_bc = d_a ln|det g| = 0 and Gamma_a = g^bc d_b g_ac; with
// g^bc = eta^bc - 2 H l^b l^c, l^c l_c = 0 and l^c d_b l_c = 0 the l l term
// drops out, leaving Gamma_a = 2 d_i (H l_a l_i) for a stationary metric
// (sum over the spatial i). So H_a = -2 d_i (H l_a l_i) and
// d_j H_a = -2 d_j d_i (H l_a l_i): first and second derivatives of nine
// products of the jets of H and l, instead of the Christoffel symbols of
// the full metric and the derivative of its inverse.
__device__ __forceinline__ void ks_gauge_closed(const Jet& H, const Jet l[3], double Hg[4], double dH[12]) {
  Jet Hl[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Hl[i] = H * l[i];
  // a = 0: P_0i = H l_i
  {
    double acc = Hl[0].g[0] + Hl[1].g[1] + Hl[2].g[2];
    Hg[0] = -2.0 * acc;
#pragma unroll
    for (int j = 0; j < 3; ++j)
      dH[4 * j] = -2.0 * (Hl[0].h[h3(j, 0)] + Hl[1].h[h3(j, 1)] + Hl[2].h[h3(j, 2)]);
  }
  // a = k >= 1: P_ki = H l_k l_i, symmetric in (k, i)
  Jet P[6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = k; i < 3; ++i) P[h3(k, i)] = Hl[k] * l[i];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Hg[1 + k] = -2.0 * (P[h3(k, 0)].g[0] + P[h3(k, 1)].g[1] + P[h3(k, 2)].g[2]);
#pragma unroll
    for (int j = 0; j < 3; ++j)
      dH[4 * j + 1 + k] =
          -2.0 * (P[h3(k, 0)].h[h3(j, 0)] + P[h3(k, 1)].h[h3(j, 1)] + P[h3(k, 2)].h[h3(j, 2)]);
  }
}

// The gauge source of a stationary metric from its jets: H_a = -Gamma_a and
// d_i H_a = -d_i Gamma_a, with Gamma_abc from D[c][ab] = d_c g_ab (d_0 = 0).
__device__ void ks_gauge(const Jet g[10], const Split& S, double H[4], double dH[12]) {
  auto D = [&](int c, int A, int B) -> double { return c == 0 ? 0.0 : g[sym_index(A, B)].g[c - 1]; };
  auto DD = [&](int i, int c, int A, int B) -> double {
    return c == 0 ? 0.0 : g[sym_index(A, B)].h[h3(i, c - 1)];
  };
  for (int A = 0; A < 4; ++A) {
    double acc = 0.0, dacc[3] = {0.0, 0.0, 0.0};
    for (int B = 0; B < 4; ++B)
      for (int C = 0; C < 4; ++C) {
        const double gam = 0.5 * (D(B, A, C) + D(C, A, B) - D(A, B, C));
        const double pinv = S.psi_inv[sym_index(B, C)];
        acc += pinv * gam;
        for (int i = 0; i < 3; ++i) {
          // d_i psi^BC = -psi^BE d_i psi_EF psi^FC
          double dpinv = 0.0;
          for (int E = 0; E < 4; ++E)
            for (int F = 0; F < 4; ++F)
              dpinv -= S.psi_inv[sym_index(B, E)] * D(1 + i, E, F) * S.psi_inv[sym_index(F, C)];
          const double dgam = 0.5 * (DD(i, B, A, C) + DD(i, C, A, B) - DD(i, A, B, C));
          dacc[i] += dpinv * gam + pinv * dgam;
        }
      }
    H[A] = -acc;
    for (int i = 0; i < 3; ++i) dH[4 * i + A] = -dacc[i];
  }
}

// One thread per point: u = (psi, Pi, Phi) of the stationary metric and the
// gauge source H_a = -Gamma_a, d_i H_a = -d_i Gamma_a (d_t H_a = 0).
__global__ void __launch_bounds__(64)
kerr_schild_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                   int bh, double M, double ax, double ay, double az, double* __restrict__ u) {
  const int s = [&] { int t = 0; while (t + 1 < n_shells && begin[t + 1] <= (int)blockIdx.x) ++t; return t; }();
  const ShellDev& sh = shells[s];
  if (bh >= 0 && sh.bh != bh) return;
  const int na = sh.na;
  const int bps = (na + 63) / 64;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * 64 + threadIdx.x;
  if (q >= na) return;
  const int j = q / sh.nph, k = q - j * sh.nph;
  const double r = sh.r[ir];
  const double x = r * sh.sth[j] * sh.cph[k], y = r * sh.sth[j] * sh.sph[k], z = r * sh.cth[j];
  Jet g[10];
  const double av[3] = {ax, ay, az};
  kerr_schild_metric(x, y, z, M, av, g);
  double psi[10], Phi[30], Pi[10];
  for (int p = 0; p < 10; ++p) {
    psi[p] = g[p].v;
    for (int i = 0; i < 3; ++i) Phi[i * 10 + p] = g[p].g[i];
  }
  Split S;
  spacetime_split(psi, S);
  for (int p = 0; p < 10; ++p)
    Pi[p] = (S.beta_up[0] * Phi[p] + S.beta_up[1] * Phi[10 + p] + S.beta_up[2] * Phi[20 + p]) / S.alpha;
  const long long base = sh.off + (long long)ir * NF * na + q;
  for (int p = 0; p < 10; ++p) {
    u[base + (long long)p * na] = psi[p];
    u[base + (long long)(10 + p) * na] = Pi[p];
    for (int i = 0; i < 3; ++i) u[base + (long long)(20 + 10 * i + p) * na] = Phi[i * 10 + p];
  }
  double Hg[4], dHg[12];
  ks_gauge(g, S, Hg, dHg);
  double* gd = sh.gauge + (long long)ir * NGAUGE * na + q;
  for (int c = 0; c < 16; ++c) gd[(long long)c * na] = c < 4 ? Hg[c] : dHg[c - 4];
}

// ------------------------------------------------------- general map
// The inertial position x = a R x_grid + T of grid point (r, q) for frame f,
// and x - T.
__device__ __forceinline__ void map_point(const Frame& f, const ShellDev& sh, double r, int q, double x[3],
                                          double xc[3]) {
  const int j = q / sh.nph, k = q - j * sh.nph;
  const double xg[3] = {r * sh.sth[j] * sh.cph[k], r * sh.sth[j] * sh.sph[k], r * sh.cth[j]};
  for (int i = 0; i < 3; ++i) {
    xc[i] = f.a * fma(f.R[3 * i + 2], xg[2], fma(f.R[3 * i + 1], xg[1], f.R[3 * i] * xg[0]));
    x[i] = xc[i] + f.T[i];
  }
}

// The hole's gauge source at every point's moving position, into gauge_t
// (the reading of a general map: the hole is not assumed symmetric under it).
__global__ void __launch_bounds__(64)
map_gauge_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                 const Frame* __restrict__ frd, const double* __restrict__ holes, const MapGate* __restrict__ gate) {
  if (gate->skip) return;
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + 63) / 64;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * 64 + threadIdx.x;
  if (q >= na) return;
  const Frame f = *frd;
  double x[3], xc[3];
  map_point(f, sh, sh.r[ir], q, x, xc);
  const double* hp = holes + 4 * sh.bh;
  const double av[3] = {hp[1], hp[2], hp[3]};
  Jet H, l[3];
  kerr_schild_fields(x[0], x[1], x[2], hp[0], av, H, l);
  double Hg[4], dHg[12];
  ks_gauge_closed(H, l, Hg, dHg);
  double* gd = sh.gauge_t + (long long)ir * NGAUGE * na + q;
  for (int c = 0; c < 16; ++c) gd[(long long)c * na] = c < 4 ? Hg[c] : dHg[c - 4];
}

// The boundary background at every boundary point's moving position, into
// bg_t: the unit normal of the moving sphere (from x - T), n^i, the lapse, the
// shift and n . xdot from the expansion and the translation (the rotation
// moves the sphere within itself).
__global__ void __launch_bounds__(128)
map_bg_kernel(const BcSliceDev* __restrict__ slices, int n_slices, const int* __restrict__ pt_begin,
              const ShellDev* __restrict__ shells, const Frame* __restrict__ frd, const double* __restrict__ holes,
              const MapGate* __restrict__ gate) {
  if (gate->skip) return;
  const int npts = pt_begin[n_slices];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npts) return;
  const int s = find_segment(pt_begin, n_slices, t);
  const BcSliceDev& sl = slices[s];
  const int q = t - pt_begin[s];
  const ShellDev& sh = shells[sl.shell_a];
  const Frame f = *frd;
  double x[3], xc[3];
  map_point(f, sh, sh.r_out, q, x, xc);
  const double* hp = holes + 4 * sh.bh;
  const double av[3] = {hp[1], hp[2], hp[3]};
  double psi[10];
  kerr_schild_values(x[0], x[1], x[2], hp[0], av, psi);
  Split S;
  spacetime_split(psi, S);
  const double R = sqrt(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
  double n[3] = {xc[0] / R, xc[1] / R, xc[2] / R};
  double nn = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) nn += S.ginv[s3(i, j)] * n[i] * n[j];
  const double inv = 1.0 / sqrt(nn);
  for (int i = 0; i < 3; ++i) n[i] *= inv;
  double nu[3];
  for (int i = 0; i < 3; ++i) nu[i] = S.ginv[s3(i, 0)] * n[0] + S.ginv[s3(i, 1)] * n[1] + S.ginv[s3(i, 2)] * n[2];
  const double h = f.adot / f.a;
  double nx = 0.0;
  for (int i = 0; i < 3; ++i) nx += n[i] * fma(h, xc[i], f.V[i]);
  const int na = sl.na;
  double* b = sl.bg_t;
  for (int i = 0; i < 3; ++i) {
    b[(long long)i * na + q] = n[i];
    b[(long long)(3 + i) * na + q] = nu[i];
    b[(long long)(7 + i) * na + q] = S.beta_up[i];
  }
  b[(long long)6 * na + q] = S.alpha;
  b[(long long)10 * na + q] = nx;
}

// One thread: skip = the buffers hold the frame *frd (compared bit for bit);
// otherwise record *frd as the frame they are about to hold.
__global__ void map_gate_kernel(const Frame* __restrict__ frd, MapGate* __restrict__ gate) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const Frame f = *frd;
  bool same = gate->valid != 0;
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(&f);
  const unsigned long long* b = reinterpret_cast<const unsigned long long*>(&gate->last);
  for (int i = 0; i < (int)(sizeof(Frame) / 8); ++i) same = same && a[i] == b[i];
  gate->skip = same ? 1 : 0;
  if (!same) {
    gate->last = f;
    gate->valid = 1;
  }
}

cudaError_t launch_map_stage(gh_domain* d) {
  if (!d->map_gen) return cudaSuccess;
  map_gate_kernel<<<1, 32, 0, d->stream>>>(d->frd, d->map_gate_d);
  d->launches++;
  map_gauge_kernel<<<d->map_blocks, 64, 0, d->stream>>>(d->shells_d, d->n_shells, d->map_pt_begin_d, d->frd,
                                                        d->holes_d, d->map_gate_d);
  d->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !d->bc_points) return e;
  map_bg_kernel<<<(d->bc_points + 127) / 128, 128, 0, d->stream>>>(d->bc_d, (int)d->bc_h.size(), d->bc_pt_begin_d,
                                                                    d->shells_d, d->frd, d->holes_d, d->map_gate_d);
  d->launches++;
  return cudaGetLastError();
}

// ------------------------------------------------------- perturbations
__global__ void __launch_bounds__(64)
perturbation_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                    int kind, double A, double Rc, double w, int lmax,
                    const double* __restrict__ coeffs, double* __restrict__ u) {
  const int s = [&] { int t = 0; while (t + 1 < n_shells && begin[t + 1] <= (int)blockIdx.x) ++t; return t; }();
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + 63) / 64;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * 64 + threadIdx.x;
  if (q >= na) return;
  const int j = q / sh.nph, k = q - j * sh.nph;
  const double r = sh.r[ir], ct = sh.cth[j], st = sh.sth[j];
  const double phi = 2.0 * 3.14159265358979323846 * k / sh.nph;
  const int W = PERT_LMAX + 1;
  double P[W * W], dP[W * W];
  legendre_table(lmax, ct, st, P, dP);
  double S = 0.0, St = 0.0, Sp = 0.0;
  int idx = 0;
  for (int l = 0; l <= lmax; ++l)
    for (int m = -l; m <= l; ++m, ++idx) {
      const int am = m < 0 ? -m : m;
      double f, fp;
      if (m == 0) { f = 1.0; fp = 0.0; }
      else {
        double sn, cs;
        sincos(am * phi, &sn, &cs);
        const double r2 = 1.41421356237309504880;
        if (m > 0) { f = r2 * cs; fp = -r2 * am * sn; }
        else { f = r2 * sn; fp = r2 * am * cs; }
      }
      const double c = coeffs[idx];
      S += c * P[l * W + am] * f;
      St += c * dP[l * W + am] * f;
      Sp += c * P[l * W + am] * fp;
    }
  const double G = exp(-((r - Rc) / w) * ((r - Rc) / w));
  const long long base = sh.off + (long long)ir * NF * na + q;
  if (kind == 1) {
    for (int p = 0; p < 10; ++p) u[base + (long long)(10 + p) * na] += G * S;
    return;
  }
  const double dG = -2.0 * (r - Rc) / (w * w) * G;
  const double f = A * G * S, fr = A * dG * S, fth = A * G * St, fph = A * G * Sp;
  const double cp = sh.cph[k], sp = sh.sph[k];
  const double df[3] = {st * cp * fr + ct * cp / r * fth - sp / (r * st) * fph,
                        st * sp * fr + ct * sp / r * fth + cp / (r * st) * fph,
                        ct * fr - st / r * fth};
  double psi[10];
  for (int p = 0; p < 10; ++p) psi[p] = u[base + (long long)p * na];
  Split Sp_;
  spacetime_split(psi, Sp_);
  const double bdf = Sp_.beta_up[0] * df[0] + Sp_.beta_up[1] * df[1] + Sp_.beta_up[2] * df[2];
  const double dpi = -(fr - bdf) / Sp_.alpha;
  for (int p = 0; p < 10; ++p) {
    u[base + (long long)p * na] += f;
    u[base + (long long)(10 + p) * na] += dpi;
    for (int i = 0; i < 3; ++i) u[base + (long long)(20 + 10 * i + p) * na] += df[i];
  }
}

cudaError_t launch_kerr_schild(gh_domain* d, int bh, double M, const double chi[3], double* u) {
  // 64-thread blocks: reuse the pointwise block map scaled by 2
  int blocks = 0;
  std::vector<int> begin(d->n_shells + 1);
  for (int s = 0; s < d->n_shells; ++s) {
    begin[s] = blocks;
    blocks += d->shells_h[s].n_r * ((d->shells_h[s].na + 63) / 64);
  }
  begin[d->n_shells] = blocks;
  int* bd = nullptr;
  cudaError_t e = cudaMallocAsync(&bd, sizeof(int) * begin.size(), d->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(bd, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice, d->stream);
  if (e != cudaSuccess) return e;
  kerr_schild_kernel<<<blocks, 64, 0, d->stream>>>(d->shells_d, d->n_shells, bd, bh, M, chi[0] * M, chi[1] * M,
                                                    chi[2] * M, u);
  d->launches++;
  e = cudaGetLastError();
  cudaFreeAsync(bd, d->stream);
  return e;
}

cudaError_t launch_perturbation(gh_domain* d, int kind, double A, double Rc, double w, int lmax,
                                const double* coeffs_dev, double* u) {
  int blocks = 0;
  std::vector<int> begin(d->n_shells + 1);
  for (int s = 0; s < d->n_shells; ++s) {
    begin[s] = blocks;
    blocks += d->shells_h[s].n_r * ((d->shells_h[s].na + 63) / 64);
  }
  begin[d->n_shells] = blocks;
  int* bd = nullptr;
  cudaError_t e = cudaMallocAsync(&bd, sizeof(int) * begin.size(), d->stream);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(bd, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice, d->stream);
  if (e != cudaSuccess) return e;
  perturbation_kernel<<<blocks, 64, 0, d->stream>>>(d->shells_d, d->n_shells, bd, kind, A, Rc, w, lmax,
                                                    coeffs_dev, u);
  d->launches++;
  e = cudaGetLastError();
  cudaFreeAsync(bd, d->stream);
  return e;
}

}  // namespace gh
