// Adjoint (vector-Jacobian products) of the right-hand side, of one RK4 step
// with its filters, and of the constraint energy; and the gradient of a
// Pi-mode perturbation with respect to its coefficients.
//
// Every map of the forward path is linear except the pointwise GH algebra, so
// the adjoint is: the transposed boundary projection (linear in dudt, fixed
// background), the hand-derived reverse pass of the per-point algebra
// (gh_point.cuh), the transposed DiffJac (folded into that pass), and the
// transposed radial and angular maps (Eq. DifferentiatorI1S2 transposed).
#include <cuda_runtime.h>

#include <algorithm>

#include <string>
#include <vector>

#include "gh_geom.cuh"
#include "gh_internal.h"
#include "gh_cpm.cuh"
#include "gh_point.cuh"
#include "gh_tensor.cuh"

namespace gh {

// ---------------------------------------------------------------------------
// Transposed radial map: out[r][col] (+)= sum_q M^T[r][q] in[q][col].  M^T
// keeps the centro-(anti)symmetry of M, so the column is folded as in the
// forward radial kernel and the folded rows of M^T (the exact transposes of
// the folded forward operators) are applied: half the FMAs.
constexpr int ADJ_RAD_THREADS = 128;

size_t radial_adjoint_smem_bytes(int max_n) {
  return sizeof(double) * ((size_t)max_n * ADJ_RAD_THREADS + (size_t)(max_n - max_n / 2) * max_n);
}

template <bool FILTER, bool ACCUM>
__global__ void __launch_bounds__(ADJ_RAD_THREADS)
radial_adjoint_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                      const double* __restrict__ in, double* __restrict__ out, int max_n) {
  extern __shared__ double Vs[];           // [max n_r][ADJ_RAD_THREADS], then the folded rows
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int n = sh.n_r, h = n >> 1, ne = n - h;
  double* Ms = Vs + (size_t)max_n * ADJ_RAD_THREADS;
  const double* M = FILTER ? sh.FrT : sh.DrT;     // folded rows of M^T [ne][n]
  for (int i = threadIdx.x; i < ne * n; i += blockDim.x) Ms[i] = M[i];
  const long long cols = (long long)NF * sh.na;
  const long long col = (long long)(blockIdx.x - begin[s]) * blockDim.x + threadIdx.x;
  const bool valid = col < cols;
  const double* src = in + sh.off + col;
  double* v = Vs + threadIdx.x;
  for (int r = 0; r < n; ++r) v[r * ADJ_RAD_THREADS] = valid ? src[(long long)r * cols] : 0.0;
  for (int j = 0; j < h; ++j) {
    const double a = v[j * ADJ_RAD_THREADS], b = v[(n - 1 - j) * ADJ_RAD_THREADS];
    v[j * ADJ_RAD_THREADS] = a + b;
    v[(n - 1 - j) * ADJ_RAD_THREADS] = a - b;
  }
  __syncthreads();
  if (!valid) return;
  double* dst = out + sh.off + col;
  auto put = [&](int r, double x) {
    const long long o = (long long)r * cols;
    dst[o] = ACCUM ? dst[o] + x : x;
  };
  for (int i = 0; i < ne; ++i) {
    const double* m0 = Ms + i * n;
    double E = m0[0] * v[0];
    for (int q = 1; q < ne; ++q) E = fma(m0[q], v[q * ADJ_RAD_THREADS], E);
    double O = m0[ne] * v[ne * ADJ_RAD_THREADS];
    for (int q = ne + 1; q < n; ++q) O = fma(m0[q], v[q * ADJ_RAD_THREADS], O);
    if (i < h) {
      put(i, E + O);
      put(n - 1 - i, FILTER ? E - O : O - E);
    } else {
      put(i, E + O);
    }
  }
}

// ---------------------------------------------------------------------------
// Transposed separable angular map.  TWO: out += Theta^T in0 + Phi^T in1 (the
// cotangents of d/dtheta and d/dphi); one: out = S^T in0 (the filter).
constexpr int SEPA_THREADS = 256;

template <bool TWO>
__global__ void __launch_bounds__(SEPA_THREADS)
sep_adjoint_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                   const double* __restrict__ in0, const double* __restrict__ in1, double* __restrict__ out) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const SepAdjPlan& P = TWO ? sh.sda : sh.sfa;
  const int nth = sh.nth, nph = sh.nph, na = sh.na, M = P.M, K = P.K;
  const int rows = NF * sh.n_r;
  const int RB = P.rows_per_cta;
  const int row0 = (blockIdx.x - begin[s]) * RB;
  const int nr = min(RB, rows - row0);
  double* Y0 = sm;                                        // [RB][na]
  double* Y1 = Y0 + (size_t)RB * na;                      // [RB][na] (TWO)
  double* A0 = Y1 + (TWO ? (size_t)RB * na : 0);          // [RB][nth][M]
  double* A1 = A0 + (size_t)RB * nth * M;                 // [RB][nth][M] (TWO)
  double* Bm = A1 + (TWO ? (size_t)RB * nth * M : 0);     // [RB][nth][M]
  const long long base = sh.off + (long long)row0 * na;
  for (int i = threadIdx.x; i < nr * na; i += SEPA_THREADS) {
    Y0[i] = in0[base + i];
    if (TWO) Y1[i] = in1[base + i];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nr * nth * M; o += SEPA_THREADS) {
    const int mode = o % M;
    const double* r0 = Y0 + (o / M) * nph;
    double a0 = 0.0, a1 = 0.0;
    if (TWO) {
      const double* r1 = Y1 + (o / M) * nph;
      for (int k = 0; k < nph; ++k) {
        a0 = fma(r0[k], __ldg(P.F0T + k * M + mode), a0);
        a1 = fma(r1[k], __ldg(P.F1T + k * M + mode), a1);
      }
      A1[o] = a1;
    } else {
      for (int k = 0; k < nph; ++k) a0 = fma(r0[k], __ldg(P.F0T + k * M + mode), a0);
    }
    A0[o] = a0;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nr * nth * M; o += SEPA_THREADS) {
    const int j = o % nth;
    const int t = o / nth;
    const int mode = t % M;
    const int rr = t / M;
    const int m = mode <= K ? mode : mode - K;
    const double* a0 = A0 + (size_t)rr * nth * M + mode;
    const double* q0 = P.Q0T + (size_t)m * nth * nth + j;
    double acc = 0.0;
    for (int jp = 0; jp < nth; ++jp) acc = fma(__ldg(q0 + jp * nth), a0[jp * M], acc);
    if (TWO) {
      const double* a1 = A1 + (size_t)rr * nth * M + mode;
      const double* q1 = P.Q1T + (size_t)m * nth * nth + j;
      for (int jp = 0; jp < nth; ++jp) acc = fma(__ldg(q1 + jp * nth), a1[jp * M], acc);
    }
    Bm[((size_t)rr * nth + j) * M + mode] = acc;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nr * na; o += SEPA_THREADS) {
    const int k = o % nph;
    const double* b = Bm + (size_t)(o / nph) * M;
    double acc = 0.0;
    for (int mode = 0; mode < M; ++mode) acc = fma(b[mode], __ldg(P.GT + mode * nph + k), acc);
    out[base + o] = TWO ? out[base + o] + acc : acc;
  }
}

cudaError_t sep_adj_set_smem_limits(size_t bytes) {
  cudaError_t e = raise_smem_limit((const void*)sep_adjoint_kernel<true>, bytes);
  if (e != cudaSuccess) return e;
  return raise_smem_limit((const void*)sep_adjoint_kernel<false>, bytes);
}

// ---------------------------------------------------------------------------
// Transposed boundary conditions, in place on a cotangent of dudt, one thread
// per (boundary point, symmetric pair).  Forward: v' = T^-1 S T v with T the
// characteristic projection and S the zeroing / upwind selection; here
// vbar <- T^T S^T T^-T vbar.
struct CharBar {
  double psi, wp, wm, w0[3];
};

__device__ __forceinline__ void load_pair(const double* k, long long base, int na, int p, double v[5]) {
  v[0] = k[base + (long long)p * na];
  v[1] = k[base + (long long)(10 + p) * na];
  for (int i = 0; i < 3; ++i) v[2 + i] = k[base + (long long)(20 + 10 * i + p) * na];
}

__device__ __forceinline__ void store_pair(double* k, long long base, int na, int p, const double v[5]) {
  k[base + (long long)p * na] = v[0];
  k[base + (long long)(10 + p) * na] = v[1];
  for (int i = 0; i < 3; ++i) k[base + (long long)(20 + 10 * i + p) * na] = v[2 + i];
}

// w_bar = (T^-1)^T v_bar, with T^-1: psi = w_psi, Pi = (w+ + w-)/2 + g2 w_psi,
// Phi_i = n_i (w+ - w-)/2 + w0_i.
__device__ __forceinline__ void inv_t_transpose(const double v[5], const double n_dn[3], double g2, CharBar& w) {
  const double nphib = n_dn[0] * v[2] + n_dn[1] * v[3] + n_dn[2] * v[4];
  w.psi = v[0] + g2 * v[1];
  w.wp = 0.5 * v[1] + 0.5 * nphib;
  w.wm = 0.5 * v[1] - 0.5 * nphib;
  for (int i = 0; i < 3; ++i) w.w0[i] = v[2 + i];
}

// v_bar = T^T w_bar, with T: w_psi = psi, w_pm = Pi +- n^k Phi_k - g2 psi,
// w0_i = Phi_i - n_i n^k Phi_k.
__device__ __forceinline__ void t_transpose(const CharBar& w, const double n_dn[3], const double n_up[3], double g2,
                                            double v[5]) {
  const double nw0 = n_dn[0] * w.w0[0] + n_dn[1] * w.w0[1] + n_dn[2] * w.w0[2];
  v[0] = w.psi - g2 * (w.wp + w.wm);
  v[1] = w.wp + w.wm;
  for (int k = 0; k < 3; ++k) v[2 + k] = n_up[k] * (w.wp - w.wm) + w.w0[k] - n_up[k] * nw0;
}

__device__ __forceinline__ void select_transpose(double& wi, double& wo, double v) {
  if (v < 0.0) {            // forward: both took the outer value
    wo += wi;
    wi = 0.0;
  } else if (v > 0.0) {     // forward: both took the inner value
    wi += wo;
    wo = 0.0;
  }
}

// cp != 0 (constraint-preserving outer condition): at incoming outer points the
// u^psi and u^0 cotangents pass through (the forward adds v_psi n^i C_ip and
// v_0 P_i^k n^j C_jkp instead of freezing), and v_psi w_psi_bar, v_0 w0_bar
// are stashed in cpbar[(p * npts + point) * 4 + {0, 1..3}] for cp_adjoint_kernel.
// cp = 2 also stashes the u^- cotangent in cpm_Sb[p * npts + point].
__global__ void __launch_bounds__(128)
bc_adjoint_kernel(const BcSliceDev* __restrict__ slices, int n_slices, const int* __restrict__ pt_begin,
                  double* __restrict__ kb, double gamma1, double gamma2, int cp, double* __restrict__ cpbar,
                  double* __restrict__ cpm_Sb, const Frame* __restrict__ frd) {
  const int npts = pt_begin[n_slices];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 10 * npts) return;
  const int p = t / npts;
  const int pt = t - p * npts;
  const int s = find_segment(pt_begin, n_slices, pt);
  const BcSliceDev& sl = slices[s];
  const int q = pt - pt_begin[s];
  const int na = sl.na;
  double n_dn[3], n_up[3], beta[3];
  for (int i = 0; i < 3; ++i) {
    n_dn[i] = sl.bg[(long long)i * na + q];
    n_up[i] = sl.bg[(long long)(3 + i) * na + q];
    beta[i] = sl.bg[(long long)(7 + i) * na + q];
  }
  const double alpha = sl.bg[(long long)6 * na + q];
  if (frd) frame_rotate_bg(*frd, n_dn, n_up, beta);   // the background at the moving point
  const double nb = n_dn[0] * beta[0] + n_dn[1] * beta[1] + n_dn[2] * beta[2];
  const double v_psi = -(1.0 + gamma1) * nb, v_0 = -nb, v_p = -nb + alpha, v_m = -nb - alpha;
  if (sl.kind == 0) {
    const long long base = sl.off_a + q;
    double v[5];
    load_pair(kb, base, na, p, v);
    CharBar w;
    inv_t_transpose(v, n_dn, gamma2, w);
    if (cp) {
      double* cb = cpbar + ((long long)p * npts + pt) * 4;
      cb[0] = v_psi < 0.0 ? v_psi * w.psi : 0.0;
      for (int i = 0; i < 3; ++i) cb[1 + i] = v_0 < 0.0 ? v_0 * w.w0[i] : 0.0;
    } else {
      if (v_psi < 0.0) w.psi = 0.0;
      if (v_0 < 0.0) w.w0[0] = w.w0[1] = w.w0[2] = 0.0;
    }
    if (v_p < 0.0) w.wp = 0.0;
    if (v_m < 0.0) {
      // cp = 2: the forward wrote the u^- solve's S; its cotangent goes to cp_minus_adjoint_kernel
      if (cp == 2) cpm_Sb[(long long)p * npts + pt] = w.wm;
      w.wm = 0.0;
    }
    t_transpose(w, n_dn, n_up, gamma2, v);
    store_pair(kb, base, na, p, v);
  } else {
    const long long ba = sl.off_a + q, bb = sl.off_b + q;
    double vi[5], vo[5];
    load_pair(kb, ba, na, p, vi);
    load_pair(kb, bb, na, p, vo);
    CharBar wi, wo;
    inv_t_transpose(vi, n_dn, gamma2, wi);
    inv_t_transpose(vo, n_dn, gamma2, wo);
    select_transpose(wi.psi, wo.psi, v_psi);
    for (int i = 0; i < 3; ++i) select_transpose(wi.w0[i], wo.w0[i], v_0);
    select_transpose(wi.wp, wo.wp, v_p);
    select_transpose(wi.wm, wo.wm, v_m);
    t_transpose(wi, n_dn, n_up, gamma2, vi);
    t_transpose(wo, n_dn, n_up, gamma2, vo);
    store_pair(kb, ba, na, p, vi);
    store_pair(kb, bb, na, p, vo);
  }
}

// Transpose of the constraint-preserving corrections at the outer boundary,
// after the pointwise reverse pass has left the derivative cotangents in
// dr/dth/dph.  Forward, for pair p at an outer point:
//   nC3  = n^i (d_i psi_p - Phi_ip),
//   Pm_i = m_i - n_i (n^k m_k),  m_k = n^j (d_j Phi_kp - d_k Phi_jp),
//   d_i = J_i^d D_d (DiffJac, D = d/dx, d/dtheta, d/dphi).
// Reverse, with c = nC3_bar and Pbar = Pm_bar from bc_adjoint_kernel:
//   D_d psi_p bar += (n^i J_i^d) c,  Phi_ip bar -= n^i c,
//   m_bar_k = Pbar_k - n^k (n_i Pbar_i),
//   (d_j Phi_kp) bar = n^j m_bar_k - n^k m_bar_j,  D_d Phi_kp bar += J_j^d (d_j Phi_kp) bar.
__global__ void __launch_bounds__(128)
cp_adjoint_kernel(const ShellDev* __restrict__ shells, const BcSliceDev* __restrict__ slices, int n_slices,
                  const int* __restrict__ pt_begin, const double* __restrict__ cpbar, double* dr, double* dth,
                  double* dph, double* ubar, const Frame* __restrict__ frd) {
  const int npts = pt_begin[n_slices];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 10 * npts) return;
  const int p = t / npts;
  const int pt = t - p * npts;
  const int s = find_segment(pt_begin, n_slices, pt);
  const BcSliceDev& sl = slices[s];
  if (sl.kind != 0) return;
  const int q = pt - pt_begin[s];
  const int na = sl.na;
  const double* cb = cpbar + ((long long)p * npts + pt) * 4;
  const double c = cb[0], P0 = cb[1], P1 = cb[2], P2 = cb[3];
  if (c == 0.0 && P0 == 0.0 && P1 == 0.0 && P2 == 0.0) return;
  double n_dn[3], n_up[3];
  for (int i = 0; i < 3; ++i) {
    n_dn[i] = sl.bg[(long long)i * na + q];
    n_up[i] = sl.bg[(long long)(3 + i) * na + q];
  }
  const ShellDev& sh = shells[sl.shell_a];
  PointGeom G;
  point_geom(sh, sh.n_r - 1, q, G);
  if (frd) {
    double beta[3] = {0.0, 0.0, 0.0}, vel[3];
    frame_rotate_bg(*frd, n_dn, n_up, beta);
    frame_geom(*frd, G, vel);
  }
  const long long base = sl.off_a + q;
  auto add_d = [&](int f, const double v[3]) {   // D_d bar of field f += sum_i J_i^d v_i
    const long long o = base + (long long)f * na;
    double g[3];
    for (int d = 0; d < 3; ++d) g[d] = G.J[0][d] * v[0] + G.J[1][d] * v[1] + G.J[2][d] * v[2];
    dr[o] += g[0];
    dth[o] += g[1];
    dph[o] += g[2];
  };
  {
    const double v[3] = {n_up[0] * c, n_up[1] * c, n_up[2] * c};
    add_d(p, v);
    for (int i = 0; i < 3; ++i) ubar[base + (long long)(20 + 10 * i + p) * na] -= v[i];
  }
  const double Pb[3] = {P0, P1, P2};
  const double nP = n_dn[0] * P0 + n_dn[1] * P1 + n_dn[2] * P2;
  double mb[3];
  for (int k = 0; k < 3; ++k) mb[k] = Pb[k] - n_up[k] * nP;
  for (int k = 0; k < 3; ++k) {          // field Phi_kp: (d_j Phi_kp) bar for j = 0..2
    double v[3];
    for (int j = 0; j < 3; ++j) v[j] = n_up[j] * mb[k] - n_up[k] * mb[j];
    add_d(20 + 10 * k + p, v);
  }
}

// ---------------------------------------------------------------------------
// Reverse mode of the u^- constraint part of the outer condition (cp = 2).
// Forward at an incoming outer point (cp_minus_kernel): S = l lam + lam l + sig P
// with (lam, sig) = M^-1 T, where the rows of M and the target T are built from
// ten directional derivatives res[e] of C_a (cpm_system), which depend on the
// state u, its Cartesian derivatives du and the interior right-hand side kr
// (through the corrected time derivative ud and the interior w^-).
// Reverse, for the cotangent Sb of S (stashed by bc_adjoint_kernel):
//   xb_b = sum_p Sb_p (l_A [B = b] + [A = b] l_B),  xb_4 = sum_p Sb_p P_p,
//   y = M^-T xb,  Tb = y,  Mb = -y x^T (rows 0..3; row 4 is fixed),
//   resb from cpm_system's linear form, then each res[e] reversed through
//   gauge_constraint_dir_rev (state and direction), the state's split
//   reversed down to the fields (state_rev), and cpm_pair reversed into
//   krb, ub and dub.
// krb is added to the interior right-hand side's cotangent kb at the point
// (before the pointwise reverse pass consumes it); ub and the derivative
// cotangents (dub through the DiffJac transpose) are stashed and added after
// that pass (cp_minus_adjoint_add_kernel), which overwrites the derivative
// scratch and may assign ubar.
struct CpmPoint {
  double u[50], k[50], du[3][50];
  double psi_inv[10], t_up[3], beta[3], N;
  double D[40];
  double ud[50];
  double wm_int[10];
  double l_dn[4], l_up[4], P[10];
  double res[10][4];
};

// The field-space direction of slope evaluation e = 4..9 (w^- = E_e), rebuilt
// where it is needed instead of stored.
__device__ __forceinline__ void cpm_point_vdir(const CpmPoint& S, const CpmBg& b, int e, double* v) {
  double E[10];
  cpm_basis(e - 4, S.l_dn, S.P, S.wm_int, E);
  cpm_vdir(E, b.n_dn, v);
}

struct CpmAdjArgs {
  const BcSliceDev* slices;
  int n_slices;
  const int* pt_begin;
  const ShellDev* shells;
  const double* u;        // the state
  const double* kr;       // its interior right-hand side (before the boundary conditions)
  const double* dr;       // its spherical derivatives
  const double* dth;
  const double* dph;
  const double* Sb;       // [10][npts] cotangent of the condition's u^- derivative
  double* kb;             // cotangent of the interior right-hand side (added to)
  double* stash;          // [200][npts]: ub (50), then the d/dx, d/dtheta, d/dphi cotangents (3 x 50)
  double gamma1, gamma2;
};

__global__ void __launch_bounds__(64) cp_minus_adjoint_kernel(CpmAdjArgs a) {
  const int npts = a.pt_begin[a.n_slices];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npts) return;
  const int sidx = find_segment(a.pt_begin, a.n_slices, t);
  const BcSliceDev& sl = a.slices[sidx];
  if (sl.kind != 0) return;
  const int q = t - a.pt_begin[sidx];
  const int na = sl.na;
  CpmBg b;
  cpm_load_bg(sl.bg, na, q, b);
  if (!((-b.nb - b.Nb) < 0.0)) return;
  double Sb[10];
  bool any = false;
  for (int p = 0; p < 10; ++p) {
    Sb[p] = a.Sb[(long long)p * npts + t];
    any = any || Sb[p] != 0.0;
  }
  // the stash of every incoming outer point is written (zeros where S does not depend on u)
  auto write_zero = [&]() {
    for (int e = 0; e < 200; ++e) a.stash[(long long)e * npts + t] = 0.0;
  };
  if (!any) {
    write_zero();
    return;
  }
  const ShellDev& sh = a.shells[sl.shell_a];
  const long long base = sl.off_a + q;
  PointGeom G;
  point_geom(sh, sh.n_r - 1, q, G);
  const double* gauge = sh.gauge + (long long)(sh.n_r - 1) * NGAUGE * na + q;

  // the primal, as cp_minus_kernel computes it
  CpmPoint S;
  for (int f = 0; f < 50; ++f) {
    const long long o = base + (long long)f * na;
    S.u[f] = a.u[o];
    S.k[f] = a.kr[o];
    for (int i = 0; i < 3; ++i) S.du[i][f] = fma(G.J[i][2], a.dph[o], fma(G.J[i][1], a.dth[o], G.J[i][0] * a.dr[o]));
  }
  cpm_state(S);
  cpm_tetrad(b, S.l_dn, S.l_up, S.P);
  for (int p = 0; p < 10; ++p) cpm_pair(p, S.k, S.u, S.du, b, a.gamma1, a.gamma2, S.ud, &S.wm_int[p]);
  double vtmp[50];
  double dH[3][4];
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 4; ++c) dH[i][c] = gauge[(long long)(4 + 4 * i + c) * na];
  const double zero4[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = 0; e < 10; ++e) {
    if (e >= 4) cpm_point_vdir(S, b, e, vtmp);
    const double* v = (e == 0) ? S.ud : (e <= 3 ? S.du[e - 1] : vtmp);
    double r[4];
    gauge_constraint_dir(S, v, (e >= 1 && e <= 3) ? dH[e - 1] : zero4, r);
    const double sc = (e >= 4) ? 1.0 / b.Nb : 1.0;
    for (int c = 0; c < 4; ++c) S.res[e][c] = r[c] * sc;
  }
  double M0[5][6], W[5][6], x[5];
  cpm_system(S.res, b, S.l_up, M0);
  for (int r = 0; r < 5; ++r)
    for (int c = 0; c < 6; ++c) W[r][c] = M0[r][c];
  if (!cpm_solve5(W, x)) {                    // S = 0 there: no dependence
    write_zero();
    return;
  }

  // reverse: S -> x -> (M, T) -> res
  double xb[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int p = 0; p < 10; ++p) {
    const int A = pair_a(p), B = pair_b(p);
    xb[B] = fma(Sb[p], S.l_dn[A], xb[B]);
    xb[A] = fma(Sb[p], S.l_dn[B], xb[A]);
    xb[4] = fma(Sb[p], S.P[p], xb[4]);
  }
  double y[5];
  for (int r = 0; r < 5; ++r) {
    for (int c = 0; c < 5; ++c) W[r][c] = M0[c][r];
    W[r][5] = xb[r];
  }
  if (!cpm_solve5(W, y)) {
    write_zero();
    return;
  }
  double resb[10][4];
  const double f = (b.Nb - b.nb) / (2.0 * b.Nb);
  for (int c = 0; c < 4; ++c) {
    for (int j = 0; j < 5; ++j) resb[4 + j][c] = -y[c] * x[j];
    const double Kb = (f - 1.0) * y[c];
    resb[9][c] = f * y[c];
    resb[0][c] = Kb / b.Nb;
    for (int i = 0; i < 3; ++i) resb[1 + i][c] = (b.n_up[i] - b.bb[i] / b.Nb) * Kb;
  }
  // res -> state, directions
  CStateBar sb;
  for (int f2 = 0; f2 < 50; ++f2) sb.u[f2] = 0.0;
  for (int p = 0; p < 10; ++p) sb.psi_inv[p] = 0.0;
  sb.N = 0.0;
  for (int i = 0; i < 3; ++i) sb.t_up[i] = sb.beta[i] = 0.0;
  for (int e = 0; e < 40; ++e) sb.D[e] = 0.0;
  double udb[50], dub[3][50], v9b[50];
  for (int f2 = 0; f2 < 50; ++f2) {
    udb[f2] = v9b[f2] = 0.0;
    for (int i = 0; i < 3; ++i) dub[i][f2] = 0.0;
  }
  for (int e = 0; e < 10; ++e) {
    const double sc = (e >= 4) ? 1.0 / b.Nb : 1.0;
    double ob[4];
    for (int c = 0; c < 4; ++c) ob[c] = resb[e][c] * sc;
    if (e >= 4) cpm_point_vdir(S, b, e, vtmp);
    const double* v = (e == 0) ? S.ud : (e <= 3 ? S.du[e - 1] : vtmp);
    double* vb = (e == 0) ? udb : (e <= 3 ? dub[e - 1] : (e == 9 ? v9b : nullptr));
    gauge_constraint_dir_rev(S, v, ob, sb, vb);
  }
  state_rev(S, sb);
  double krb[50];
  for (int f2 = 0; f2 < 50; ++f2) krb[f2] = 0.0;
  for (int p = 0; p < 10; ++p) {
    // the interior w^- enters through e = 9's direction: Pi' = w/2, Phi_i' = -n_i w/2
    double wmb = 0.5 * v9b[10 + p];
    for (int i = 0; i < 3; ++i) wmb = fma(-0.5 * b.n_dn[i], v9b[20 + 10 * i + p], wmb);
    cpm_pair_rev(p, b, a.gamma1, a.gamma2, udb, wmb, krb, sb.u, dub);
  }
  for (int f2 = 0; f2 < 50; ++f2) {
    const long long o = base + (long long)f2 * na;
    a.kb[o] += krb[f2];
    a.stash[(long long)f2 * npts + t] = sb.u[f2];
    for (int dd = 0; dd < 3; ++dd)
      a.stash[(long long)(50 + 50 * dd + f2) * npts + t] =
          G.J[0][dd] * dub[0][f2] + G.J[1][dd] * dub[1][f2] + G.J[2][dd] * dub[2][f2];
  }
}

// After the pointwise reverse pass: ubar and the derivative cotangents
// (overwritten into dr/dth/dph by that pass) take the stashed contributions
// of the u^- condition, one thread per (outer point, field).
__global__ void __launch_bounds__(128)
cp_minus_adjoint_add_kernel(const BcSliceDev* __restrict__ slices, int n_slices, const int* __restrict__ pt_begin,
                            const double* __restrict__ stash, double* ubar, double* dr, double* dth, double* dph) {
  const int npts = pt_begin[n_slices];
  const long long tt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= 50LL * npts) return;
  const int f = (int)(tt / npts);
  const int t = (int)(tt - (long long)f * npts);
  const int sidx = find_segment(pt_begin, n_slices, t);
  const BcSliceDev& sl = slices[sidx];
  if (sl.kind != 0) return;
  const int q = t - pt_begin[sidx];
  CpmBg b;
  cpm_load_bg(sl.bg, sl.na, q, b);
  if (!((-b.nb - b.Nb) < 0.0)) return;
  const long long o = sl.off_a + q + (long long)f * sl.na;
  ubar[o] += stash[(long long)f * npts + t];
  dr[o] += stash[(long long)(50 + f) * npts + t];
  dth[o] += stash[(long long)(100 + f) * npts + t];
  dph[o] += stash[(long long)(150 + f) * npts + t];
}

// ---------------------------------------------------------------------------
// Pointwise reverse pass, one thread per point.  Reads the point's fields and
// the spherical derivatives d/dx, d/dtheta, d/dphi of u from dr/dth/dph,
// adds the field cotangents to ubar, and overwrites dr/dth/dph at the point
// with the derivative cotangents (each thread reads its own values first).
// MODE 0: cotangent kb of dudt (before the boundary conditions).
// MODE 1: gradient of weight * sum_points w_quadrature * (constraint energy).
// MODE 2: both (the RHS cotangent and the constraint-energy gradient at u).

// The constraint-energy gradient as a separate (not inlined) call, so that the
// fused kernel does not hold both reverse passes' locals at once.
__device__ __noinline__ void constraint_part(const PointIn& in, double w, double* ub, double* dsb) {
  point_constraint_energy(in, w, ub, dsb);
}

// The reverse pass's per-pair access on global memory at one point (offset
// base, field stride na): the derivative scratch dr/dth/dph is read and then
// overwritten with the cotangents of those derivatives, pair by pair; kb is the
// cotangent of dudt.  Each thread touches only its own point's entries.
struct GlobalPairIO {
  double* dr;
  double* dth;
  double* dph;
  const double* kb;
  long long base;
  int na;
  __device__ void load(int p, double ds15[15], double kb5[5]) const {
    for (int e = 0; e < 5; ++e) {
      const long long o = base + (long long)(e == 0 ? p : 10 * e + p) * na;
      ds15[3 * e] = dr[o];
      ds15[3 * e + 1] = dth[o];
      ds15[3 * e + 2] = dph[o];
      kb5[e] = kb[o];
    }
  }
  __device__ void store(int p, const double dsb15[15]) const {
    for (int e = 0; e < 5; ++e) {
      const long long o = base + (long long)(e == 0 ? p : 10 * e + p) * na;
      dr[o] = dsb15[3 * e];
      dth[o] = dsb15[3 * e + 1];
      dph[o] = dsb15[3 * e + 2];
    }
  }
};

#ifndef GH_ADJ_MINB
#define GH_ADJ_MINB 12
#endif
template <int MODE>
__global__ void __launch_bounds__(ADJ_PT_THREADS, GH_ADJ_MINB)
pointwise_adjoint_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                         const double* __restrict__ u, double* dr, double* dth, double* dph,
                         const double* __restrict__ kb, double* ubar, double g0, double g1, double g2,
                         double weight, int assign, const Frame* __restrict__ frd = nullptr,
                         const double* __restrict__ kb0 = nullptr) {
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + ADJ_PT_THREADS - 1) / ADJ_PT_THREADS;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * ADJ_PT_THREADS + threadIdx.x;
  if (q >= na) return;
  const long long base = sh.off + (long long)ir * NF * na + q;
  if (MODE == 0) {
    // the plain RHS cotangent: each pair's derivatives, their cotangents and
    // the output cotangents stream from and to global memory, so the thread
    // holds only the point's fields and their cotangents
    double uu[50], ub[50];
    for (int f = 0; f < NF; ++f) {
      uu[f] = u[base + (long long)f * na];
      ub[f] = 0.0;
    }
    const double* gsrc = sh.gauge + (long long)ir * NGAUGE * na + q;
    double H[4], dH[12];
    for (int c = 0; c < 4; ++c) H[c] = gsrc[(long long)c * na];
    for (int c = 0; c < 12; ++c) dH[c] = gsrc[(long long)(4 + c) * na];
    PointGeom G;
    point_geom(sh, ir, q, G);
    double vel[3] = {0.0, 0.0, 0.0};
    if (frd) {
      const Frame fr = *frd;
      frame_geom(fr, G, vel);
      frame_rotate_h(fr, H);
      frame_rotate_dh(fr, dH);
    }
    PointIn in;
    in.u = uu;
    in.ds = nullptr;
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) in.J[i][d] = G.J[i][d];
    in.H = H;
    in.dH = dH;
    in.g0 = g0;
    in.g1 = g1;
    in.g2 = g2;
    PointFwd fw;
    point_intermediates(in, fw);
    const GlobalPairIO io{dr, dth, dph, kb, base, na};
    point_rhs_vjp_io(in, fw, io, ub);
    if (frd && kb0) {
      // transposed grid-velocity term, as below
      double vs[3];
      for (int d = 0; d < 3; ++d) vs[d] = vel[0] * G.J[0][d] + vel[1] * G.J[1][d] + vel[2] * G.J[2][d];
      for (int f = 0; f < NF; ++f) {
        const long long o = base + (long long)f * na;
        const double kv = kb0[o];
        dr[o] = fma(vs[0], kv, dr[o]);
        dth[o] = fma(vs[1], kv, dth[o]);
        dph[o] = fma(vs[2], kv, dph[o]);
      }
    }
    for (int f = 0; f < NF; ++f) {
      const long long o = base + (long long)f * na;
      ubar[o] = assign ? ub[f] : ubar[o] + ub[f];
    }
    return;
  }
  double uu[50], ds[150], ub[50], dsb[150];
  for (int f = 0; f < NF; ++f) {
    const long long o = base + (long long)f * na;
    uu[f] = u[o];
    ds[3 * f] = dr[o];
    ds[3 * f + 1] = dth[o];
    ds[3 * f + 2] = dph[o];
    ub[f] = 0.0;
    dsb[3 * f] = dsb[3 * f + 1] = dsb[3 * f + 2] = 0.0;
  }
  const double* gsrc = sh.gauge + (long long)ir * NGAUGE * na + q;
  double H[4], dH[12];
  for (int c = 0; c < 4; ++c) H[c] = gsrc[(long long)c * na];
  for (int c = 0; c < 12; ++c) dH[c] = gsrc[(long long)(4 + c) * na];
  PointGeom G;
  point_geom(sh, ir, q, G);
  double vel[3] = {0.0, 0.0, 0.0};
  if (frd) {                      // rotating frame: J <- R J, rotated gauge source
    const Frame fr = *frd;
    frame_geom(fr, G, vel);
    frame_rotate_h(fr, H);
    frame_rotate_dh(fr, dH);
  }
  PointIn in;
  in.u = uu;
  in.ds = ds;
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) in.J[i][d] = G.J[i][d];
  in.H = H;
  in.dH = dH;
  in.g0 = g0;
  in.g1 = g1;
  in.g2 = g2;
  if (MODE == 2) {
    double kk[50];
    for (int f = 0; f < NF; ++f) kk[f] = kb[base + (long long)f * na];
    PointFwd fw;
    point_intermediates(in, fw);
    point_rhs_vjp(in, fw, kk, ub, dsb);
  }
  if (MODE == 1) {
    const int j = q / sh.nph;
    point_constraint_energy(in, weight * sh.wr[ir] * sh.wth[j], ub, dsb);
  }
  if (MODE == 2) {
    const int j = q / sh.nph;
    constraint_part(in, weight * sh.wr[ir] * sh.wth[j], ub, dsb);
  }
  if (MODE != 1 && frd && kb0) {
    // the grid-velocity term xdot . (J d u) of every point (added after the
    // boundary conditions), transposed with the cotangent of the final rate
    double vs[3];
    for (int d = 0; d < 3; ++d) vs[d] = vel[0] * G.J[0][d] + vel[1] * G.J[1][d] + vel[2] * G.J[2][d];
    for (int f = 0; f < NF; ++f) {
      const double kv = kb0[base + (long long)f * na];
      for (int d = 0; d < 3; ++d) dsb[3 * f + d] = fma(vs[d], kv, dsb[3 * f + d]);
    }
  }
  for (int f = 0; f < NF; ++f) {
    const long long o = base + (long long)f * na;
    ubar[o] = assign ? ub[f] : ubar[o] + ub[f];
    dr[o] = dsb[3 * f];
    dth[o] = dsb[3 * f + 1];
    dph[o] = dsb[3 * f + 2];
  }
}

// ---------------------------------------------------------------------------
// Element-wise combinations with the per-hole step dts = dt * dt_scale(shell),
// one thread per (field, theta, phi) column of a shell.
//   0: out = x + c * dts * y        1: out = dts * (a x + c y)        2: out += x
//   3: out = dts * (a x + c y) and z += y
__global__ void __launch_bounds__(128)
ew_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin, int mode,
          double* __restrict__ out, const double* __restrict__ x, const double* __restrict__ y, double a,
          double c, double dt, double* __restrict__ z) {
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const long long cols = (long long)NF * sh.na;
  const long long col = (long long)(blockIdx.x - begin[s]) * blockDim.x + threadIdx.x;
  if (col >= cols) return;
  const double dts = dt * sh.dt_scale;
  for (int r = 0; r < sh.n_r; ++r) {
    const long long o = sh.off + (long long)r * cols + col;
    if (mode == 0) out[o] = x[o] + c * dts * y[o];
    else if (mode == 1) out[o] = dts * (a * x[o] + c * y[o]);
    else if (mode == 2) out[o] += x[o];
    else {
      const double yv = y[o];
      out[o] = dts * (a * x[o] + c * yv);
      z[o] += yv;
    }
  }
}

// ---------------------------------------------------------------------------
// Gradient of a Pi-mode perturbation dPi_ab = exp(-((R-Rc)/w)^2) sum c_lm Y_lm
// (all 10 components) with respect to c_lm: per-block partial sums of
// sum_p ubar(Pi_p) G(R) Y_lm over the block's points.
constexpr int PV_THREADS = 64;
constexpr int PV_MAX_MODES = 81;   // lmax <= 8
static_assert(PV_MAX_MODES <= (PERT_LMAX + 1) * (PERT_LMAX + 1), "mode count exceeds the Legendre table");

__global__ void __launch_bounds__(PV_THREADS)
pi_modes_vjp_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                    double Rc, double w, int lmax, const double* __restrict__ ubar, double* __restrict__ partial) {
  __shared__ double red[PV_THREADS];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + PV_THREADS - 1) / PV_THREADS;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * PV_THREADS + threadIdx.x;
  const int nm = (lmax + 1) * (lmax + 1);
  double sG = 0.0, ct = 0.0, st = 1.0, phi = 0.0;
  if (q < na) {
    const int j = q / sh.nph, k = q - j * sh.nph;
    const long long base = sh.off + (long long)ir * NF * na + q;
    double acc = 0.0;
    for (int p = 0; p < 10; ++p) acc += ubar[base + (long long)(10 + p) * na];
    const double r = sh.r[ir];
    sG = acc * exp(-((r - Rc) / w) * ((r - Rc) / w));
    ct = sh.cth[j];
    st = sh.sth[j];
    phi = 2.0 * 3.14159265358979323846 * k / sh.nph;
  }
  const int W = PERT_LMAX + 1;
  double P[W * W], dP[W * W];
  legendre_table(lmax, ct, st, P, dP);
  int idx = 0;
  for (int l = 0; l <= lmax; ++l)
    for (int m = -l; m <= l; ++m, ++idx) {
      const int am = m < 0 ? -m : m;
      double fphi = 1.0;
      if (m != 0) {
        double sn, cs;
        sincos(am * phi, &sn, &cs);
        fphi = 1.41421356237309504880 * (m > 0 ? cs : sn);
      }
      red[threadIdx.x] = (q < na) ? sG * P[l * W + am] * fphi : 0.0;
      __syncthreads();
      for (int stp = PV_THREADS / 2; stp > 0; stp >>= 1) {
        if (threadIdx.x < stp) red[threadIdx.x] += red[threadIdx.x + stp];
        __syncthreads();
      }
      if (threadIdx.x == 0) partial[(long long)blockIdx.x * nm + idx] = red[0];
      __syncthreads();
    }
}

}  // namespace gh

// =================================================================== C ABI
namespace {

gh_status afail(gh_domain* d, gh_status s, const std::string& m) {
  d->err = m;
  return s;
}

#define GH_ACUDA(d, call)                                                                      \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return afail((d), e_ == cudaErrorMemoryAllocation ? GH_ENOMEM : GH_ECUDA,                \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

cudaError_t radial_adjoint_smem_limits() {
  const size_t bytes = gh::radial_adjoint_smem_bytes(64);
  cudaError_t e = gh::raise_smem_limit((const void*)gh::radial_adjoint_kernel<false, true>, bytes);
  if (e == cudaSuccess) e = gh::raise_smem_limit((const void*)gh::radial_adjoint_kernel<true, false>, bytes);
  return e;
}

// Rotating frame: the frames of the domain clock + {0, dt/2, dt} (n of them)
// into the device frame array; the clock does not move (no-op when static).
gh_status frames_at(gh_domain* d, double half, double full, int n) {
  if (d->rot_omega == 0.0) return GH_OK;
  const double off[3] = {0.0, half, full};
  GH_ACUDA(d, gh::launch_frames(d, off, n, 0.0));
  d->frd = d->frames_d;
  return GH_OK;
}

gh_status adj_ready(gh_domain* d) {
  if (gh_status s = gh::check_latched(d)) return s;
  if (d->map_gen)
    return afail(d, GH_ENOTSUP, "the adjoint supports the static grid and the rotating frame, not a general map");
  if (d->algorithm == 0) return afail(d, GH_ENOTSUP, "the adjoint needs a separable angular algorithm");
  if (d->outer_bc == GH_BC_CONSTRAINT_PRESERVING_FULL && d->bc_points && !d->adj_cpm_stash) {
    void* p = nullptr;
    GH_ACUDA(d, cudaMalloc(&p, sizeof(double) * (size_t)d->state));
    d->owned.push_back(p);
    d->adj_kraw = (double*)p;
    GH_ACUDA(d, cudaMalloc(&p, sizeof(double) * 10 * (size_t)d->bc_points));
    d->owned.push_back(p);
    d->adj_cpm_Sb = (double*)p;
    GH_ACUDA(d, cudaMalloc(&p, sizeof(double) * 200 * (size_t)d->bc_points));
    d->owned.push_back(p);
    d->adj_cpm_stash = (double*)p;
  }
  if (d->outer_bc != GH_BC_FREEZE && !d->adj_cpbar && d->bc_points) {
    void* p = nullptr;
    GH_ACUDA(d, cudaMalloc(&p, sizeof(double) * 40 * (size_t)d->bc_points));
    d->owned.push_back(p);
    d->adj_cpbar = (double*)p;
  }
  if (d->rot_omega != 0.0)
    for (const auto& sh : d->shells_h)
      if (sh.dt_scale != 1.0) return afail(d, GH_ENOTSUP, "the rotating frame needs dt_scale = 1 on every shell");
  GH_ACUDA(d, radial_adjoint_smem_limits());
  if (!d->kbt) {
    void* p = nullptr;
    GH_ACUDA(d, cudaMalloc(&p, sizeof(double) * d->state));
    d->owned.push_back(p);
    d->kbt = (double*)p;
  }
  return GH_OK;
}

cudaError_t ew(gh_domain* d, int mode, double* out, const double* x, const double* y, double a, double c,
               double dt, double* z = nullptr) {
  gh::ew_kernel<<<d->rad_blocks, 128, 0, d->stream>>>(d->shells_d, d->n_shells, d->rad_block_begin_d, mode, out,
                                                      x, y, a, c, dt, z);
  d->launches++;
  return cudaGetLastError();
}

// Forward derivatives of u into d_r, d_th, d_ph.
cudaError_t fwd_derivs(gh_domain* d, const double* u) { return gh::launch_derivatives(d, u); }

// ubar += (transposed derivative maps) applied to the derivative cotangents
// in D[0] (d/dx), D[1] (d/dtheta), D[2] (d/dphi).
cudaError_t derivs_transpose_add(gh_domain* d, double* ubar, double* const* D) {
  gh::radial_adjoint_kernel<false, true><<<d->rad_blocks, gh::ADJ_RAD_THREADS,
                                           gh::radial_adjoint_smem_bytes(d->max_n_r), d->stream>>>(
      d->shells_d, d->n_shells, d->rad_block_begin_d, D[0], ubar, d->max_n_r);
  d->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (d->algorithm == 2) return gh::launch_fold_adjoint(d, true, D[1], D[2], ubar);
  gh::sep_adjoint_kernel<true><<<d->sda_blocks, gh::SEPA_THREADS, d->sda_smem, d->stream>>>(
      d->shells_d, d->n_shells, d->sda_block_begin_d, D[1], D[2], ubar);
  d->launches++;
  return cudaGetLastError();
}

// Forward right-hand side k = F(u) with its derivatives written to D[0..2]
// (which the reverse pass at u can then use instead of recomputing them).
cudaError_t rhs_fwd_into(gh_domain* d, const double* u, double* k, double* const* D) {
  cudaError_t e = gh::launch_radial(d, u, D[0], false);
  if (e == cudaSuccess) e = gh::launch_angular_deriv_into(d, u, D[1], D[2]);
  if (e == cudaSuccess) e = gh::launch_pointwise_rhs_from(d, u, D[0], D[1], D[2], k);
  const double* cd[3] = {D[0], D[1], D[2]};
  if (e == cudaSuccess) e = gh::launch_bc(d, k, 0, 0.0, nullptr, nullptr, nullptr, u, cd);
  return e;
}

}  // namespace
namespace gh {

// Pair-split pointwise reverse pass for small grids: one thread per (point,
// symmetric pair): one-warp blocks on a grid of (32-point chunk of the forward
// pointwise kernel) x (pair), so the warps of a chunk spread over the SMs.  Each thread runs the pair-restricted reverse
// pass (and, MODE 2, its share of the constraint-energy gradient), writes the
// cotangents of its pair's derivatives in place and its partial field
// cotangents to ubp[p][state]; adj_pair_reduce_kernel sums the ten partials
// in a fixed order.
constexpr int PAIR_PTS = 32;
template <int MODE>
__global__ void __launch_bounds__(PAIR_PTS)
pointwise_adjoint_pair_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                              const double* __restrict__ u, double* dr, double* dth, double* dph,
                              const double* __restrict__ kb, double* __restrict__ ubp, long long state, double g0,
                              double g1, double g2, double weight) {
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + PAIR_PTS - 1) / PAIR_PTS;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * PAIR_PTS + threadIdx.x;
  const int p = blockIdx.y;
  if (q >= na) return;
  const long long base = sh.off + (long long)ir * NF * na + q;
  double uu[50], ub[50];
  for (int f = 0; f < NF; ++f) {
    uu[f] = u[base + (long long)f * na];
    ub[f] = 0.0;
  }
  const int fid[5] = {p, 10 + p, 20 + p, 30 + p, 40 + p};
  double dsp[15], kb5[5], dsb15[15];
  for (int e = 0; e < 5; ++e) {
    const long long o = base + (long long)fid[e] * na;
    dsp[3 * e] = dr[o];
    dsp[3 * e + 1] = dth[o];
    dsp[3 * e + 2] = dph[o];
    kb5[e] = kb[o];
  }
  const double* gsrc = sh.gauge + (long long)ir * NGAUGE * na + q;
  double H[4], dH[12];
  for (int c = 0; c < 4; ++c) H[c] = gsrc[(long long)c * na];
  for (int c = 0; c < 12; ++c) dH[c] = gsrc[(long long)(4 + c) * na];
  PointGeom G;
  point_geom(sh, ir, q, G);
  point_rhs_vjp_pair(uu, G.J, H, dH, g0, g1, g2, p, dsp, kb5, ub, dsb15);
  if (MODE == 2) {
    const int j = q / sh.nph;
    point_constraint_energy_pair(uu, G.J, H, p, dsp, weight * sh.wr[ir] * sh.wth[j], ub, dsb15);
  }
  for (int e = 0; e < 5; ++e) {
    const long long o = base + (long long)fid[e] * na;
    dr[o] = dsb15[3 * e];
    dth[o] = dsb15[3 * e + 1];
    dph[o] = dsb15[3 * e + 2];
  }
  double* out = ubp + (long long)p * state;
  for (int f = 0; f < NF; ++f) out[base + (long long)f * na] = ub[f];
}

__global__ void __launch_bounds__(256)
adj_pair_reduce_kernel(long long state, const double* __restrict__ ubp, double* __restrict__ ubar, int assign) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < state; i += (long long)gridDim.x * blockDim.x) {
    double acc = ubp[i];
    for (int p = 1; p < 10; ++p) acc += ubp[(long long)p * state + i];
    ubar[i] = assign ? acc : ubar[i] + acc;
  }
}

}  // namespace gh
namespace {

// ubar (+)= J(u)^T kb (+ cweight * grad of the constraint energy at u when
// cweight != 0); assign: overwrite ubar instead of adding; kb is not modified.
// saved: the spherical derivatives of u already computed (three states,
// consumed: overwritten with their cotangents); null: computed here into the
// domain's scratch.
gh_status rhs_vjp(gh_domain* d, const double* u, const double* kb, double* ubar, double cweight = 0.0,
                  bool assign = false, double* const* saved = nullptr) {
  double* const scratch[3] = {d->d_r, d->d_th, d->d_ph};
  double* const* D = saved ? saved : scratch;
  if (!saved) GH_ACUDA(d, fwd_derivs(d, u));
  GH_ACUDA(d, cudaMemcpyAsync(d->kbt, kb, sizeof(double) * d->state, cudaMemcpyDeviceToDevice, d->stream));
  const int cp = d->outer_bc;   // 0 freezing, 1 u^psi and u^0, 2 also the u^- constraint part
  const gh::Frame* frd = d->rot_omega != 0.0 ? d->frd : nullptr;
  if (d->bc_points) {
    gh::bc_adjoint_kernel<<<cdiv(10LL * d->bc_points, 128), 128, 0, d->stream>>>(
        d->bc_d, (int)d->bc_h.size(), d->bc_pt_begin_d, d->kbt, d->params.gamma1, d->params.gamma2, cp,
        d->adj_cpbar, d->adj_cpm_Sb, frd);
    d->launches++;
    GH_ACUDA(d, cudaGetLastError());
  }
  if (cp == 2 && d->bc_points) {
    // the interior right-hand side the forward condition read, then the u^- reverse
    GH_ACUDA(d, gh::launch_pointwise_rhs_from(d, u, D[0], D[1], D[2], d->adj_kraw));
    gh::CpmAdjArgs ca;
    ca.slices = d->bc_d; ca.n_slices = (int)d->bc_h.size(); ca.pt_begin = d->bc_pt_begin_d;
    ca.shells = d->shells_d; ca.u = u; ca.kr = d->adj_kraw; ca.dr = D[0]; ca.dth = D[1]; ca.dph = D[2];
    ca.Sb = d->adj_cpm_Sb; ca.kb = d->kbt; ca.stash = d->adj_cpm_stash;
    ca.gamma1 = d->params.gamma1; ca.gamma2 = d->params.gamma2;
    gh::cp_minus_adjoint_kernel<<<cdiv(d->bc_points, 64), 64, 0, d->stream>>>(ca);
    d->launches++;
    GH_ACUDA(d, cudaGetLastError());
  }
  if (d->adj_pair_split && !frd) {
    // small grid: ten threads per point (one per symmetric pair)
    if (!d->adj_ubp) {
      void* p = nullptr;
      GH_ACUDA(d, cudaMalloc(&p, sizeof(double) * 10 * (size_t)d->state));
      d->owned.push_back(p);
      d->adj_ubp = (double*)p;
    }
    const dim3 grid(d->pt_blocks, 10);
    if (cweight != 0.0)
      gh::pointwise_adjoint_pair_kernel<2><<<grid, gh::PAIR_PTS, 0, d->stream>>>(
          d->shells_d, d->n_shells, d->pt_block_begin_d, u, D[0], D[1], D[2], d->kbt, d->adj_ubp, d->state,
          d->params.gamma0, d->params.gamma1, d->params.gamma2, cweight);
    else
      gh::pointwise_adjoint_pair_kernel<0><<<grid, gh::PAIR_PTS, 0, d->stream>>>(
          d->shells_d, d->n_shells, d->pt_block_begin_d, u, D[0], D[1], D[2], d->kbt, d->adj_ubp, d->state,
          d->params.gamma0, d->params.gamma1, d->params.gamma2, 0.0);
    d->launches++;
    GH_ACUDA(d, cudaGetLastError());
    const long long nb = std::min<long long>((d->state + 255) / 256, 4096);
    gh::adj_pair_reduce_kernel<<<(unsigned)nb, 256, 0, d->stream>>>(d->state, d->adj_ubp, ubar, assign ? 1 : 0);
    d->launches++;
    GH_ACUDA(d, cudaGetLastError());
  } else {
    if (cweight != 0.0)
      gh::pointwise_adjoint_kernel<2><<<d->adj_pt_blocks, gh::ADJ_PT_THREADS, 0, d->stream>>>(
          d->shells_d, d->n_shells, d->adj_pt_block_begin_d, u, D[0], D[1], D[2], d->kbt, ubar,
          d->params.gamma0, d->params.gamma1, d->params.gamma2, cweight, assign ? 1 : 0, frd, kb);
    else
      gh::pointwise_adjoint_kernel<0><<<d->adj_pt_blocks, gh::ADJ_PT_THREADS, 0, d->stream>>>(
          d->shells_d, d->n_shells, d->adj_pt_block_begin_d, u, D[0], D[1], D[2], d->kbt, ubar,
          d->params.gamma0, d->params.gamma1, d->params.gamma2, 0.0, assign ? 1 : 0, frd, kb);
    d->launches++;
    GH_ACUDA(d, cudaGetLastError());
  }
  if (cp && d->bc_points) {
    gh::cp_adjoint_kernel<<<cdiv(10LL * d->bc_points, 128), 128, 0, d->stream>>>(
        d->shells_d, d->bc_d, (int)d->bc_h.size(), d->bc_pt_begin_d, d->adj_cpbar, D[0], D[1], D[2], ubar,
        frd);
    d->launches++;
    GH_ACUDA(d, cudaGetLastError());
  }
  if (cp == 2 && d->bc_points) {
    gh::cp_minus_adjoint_add_kernel<<<cdiv(50LL * d->bc_points, 128), 128, 0, d->stream>>>(
        d->bc_d, (int)d->bc_h.size(), d->bc_pt_begin_d, d->adj_cpm_stash, ubar, D[0], D[1], D[2]);
    d->launches++;
    GH_ACUDA(d, cudaGetLastError());
  }
  GH_ACUDA(d, derivs_transpose_add(d, ubar, D));
  return GH_OK;
}

// Forward RHS k = F(u) (derivatives, pointwise, boundary conditions).
gh_status rhs_fwd(gh_domain* d, const double* u, double* k) {
  GH_ACUDA(d, fwd_derivs(d, u));
  GH_ACUDA(d, gh::launch_pointwise(d, u, k, 0, 0.0, nullptr, nullptr, nullptr, false));
  GH_ACUDA(d, gh::launch_bc(d, k, 0, 0.0, nullptr, nullptr, nullptr, u));
  return GH_OK;
}

}  // namespace

extern "C" {

long long gh_rk4_vjp_work_size(const gh_domain* d) { return d ? 16 * d->state : -1; }

gh_status gh_rhs_vjp(gh_domain* d, const double* u, const double* kbar, double* ubar) {
  if (!d || !u || !kbar || !ubar) return d ? afail(d, GH_EINVAL, "null argument") : GH_EINVAL;
  if (gh_status s = adj_ready(d)) return s;
  if (gh_status s = frames_at(d, 0.0, 0.0, 1)) return s;
  return rhs_vjp(d, u, kbar, ubar);
}

gh_status gh_constraint_energy_vjp(gh_domain* d, const double* u, double weight, double* ubar) {
  if (!d || !u || !ubar) return d ? afail(d, GH_EINVAL, "null argument") : GH_EINVAL;
  if (gh_status s = adj_ready(d)) return s;
  if (gh_status s = frames_at(d, 0.0, 0.0, 1)) return s;
  GH_ACUDA(d, fwd_derivs(d, u));
  gh::pointwise_adjoint_kernel<1><<<d->adj_pt_blocks, gh::ADJ_PT_THREADS, 0, d->stream>>>(
      d->shells_d, d->n_shells, d->adj_pt_block_begin_d, u, d->d_r, d->d_th, d->d_ph, nullptr, ubar,
      d->params.gamma0, d->params.gamma1, d->params.gamma2, weight, 0,
      d->rot_omega != 0.0 ? d->frd : nullptr, nullptr);
  d->launches++;
  GH_ACUDA(d, cudaGetLastError());
  double* const D[3] = {d->d_r, d->d_th, d->d_ph};
  GH_ACUDA(d, derivs_transpose_add(d, ubar, D));
  return GH_OK;
}

}  // extern "C"

namespace {

gh_status step_vjp_impl(gh_domain* d, double dt, const double* u_n, const double* stages, const double* ubar_np1,
                        double* ubar_n, double* work, double cweight) {
  if (gh_status s = adj_ready(d)) return s;
  // stage times t, t + dt/2, t + dt/2, t + dt of the step from the domain clock
  if (gh_status s = frames_at(d, 0.5 * dt, dt, 3)) return s;
  auto at = [&](int i) { if (d->frames_d) d->frd = d->frames_d + i; };
  const long long N = d->state;
  const double *u2, *u3, *u4;
  double* k = work + 3 * N;
  double* kb = work + 4 * N;
  double* g = work + 5 * N;
  double* sb = work + 6 * N;
  // spherical derivatives of u_n, u2 and u3 kept from the recomputation
  double* const D1[3] = {work + 7 * N, work + 8 * N, work + 9 * N};
  double* const D2[3] = {work + 10 * N, work + 11 * N, work + 12 * N};
  double* const D3[3] = {work + 13 * N, work + 14 * N, work + 15 * N};
  const bool keep = stages == nullptr;
  if (stages) {
    u2 = stages;
    u3 = stages + N;
    u4 = stages + 2 * N;
  } else {
    // forward recomputation of the stage states
    double* w2 = work;
    double* w3 = work + N;
    double* w4 = work + 2 * N;
    at(0);
    GH_ACUDA(d, rhs_fwd_into(d, u_n, k, D1));
    GH_ACUDA(d, ew(d, 0, w2, u_n, k, 0.0, 0.5, dt));
    at(1);
    GH_ACUDA(d, rhs_fwd_into(d, w2, k, D2));
    GH_ACUDA(d, ew(d, 0, w3, u_n, k, 0.0, 0.5, dt));
    GH_ACUDA(d, rhs_fwd_into(d, w3, k, D3));
    GH_ACUDA(d, ew(d, 0, w4, u_n, k, 0.0, 1.0, dt));
    u2 = w2;
    u3 = w3;
    u4 = w4;
  }
  // transposed filters: u_new = Fr(Fa(v))  =>  g = Fa^T Fr^T ubar_np1
  const double* gin = ubar_np1;
  const bool ang_f = d->params.sh_keep_l != -1;
  if (d->params.radial_filter_on) {
    double* dst = ang_f ? kb : g;
    gh::radial_adjoint_kernel<true, false><<<d->rad_blocks, gh::ADJ_RAD_THREADS,
                                             gh::radial_adjoint_smem_bytes(d->max_n_r), d->stream>>>(
        d->shells_d, d->n_shells, d->rad_block_begin_d, gin, dst, d->max_n_r);
    d->launches++;
    GH_ACUDA(d, cudaGetLastError());
    gin = dst;
  }
  if (ang_f) {                           // gin is ubar_np1 or kb here, never g
    if (d->sh_filter_mode == GH_SH_FILTER_TENSOR) {
      GH_ACUDA(d, gh::launch_tensor_filter_transpose(d, gin, g));
    } else if (d->algorithm == 2) {
      GH_ACUDA(d, gh::launch_fold_adjoint(d, false, gin, nullptr, g));
    } else {
      gh::sep_adjoint_kernel<false><<<d->sfa_blocks, gh::SEPA_THREADS, d->sfa_smem, d->stream>>>(
          d->shells_d, d->n_shells, d->sfa_block_begin_d, gin, nullptr, g);
      d->launches++;
      GH_ACUDA(d, cudaGetLastError());
    }
    gin = g;
  }
  // ubar_n starts as g (the direct u_n term of u_n + dt/6 (...)); g itself is
  // kept for the stage cotangents
  if (gin != g) GH_ACUDA(d, cudaMemcpyAsync(g, gin, sizeof(double) * N, cudaMemcpyDeviceToDevice, d->stream));
  GH_ACUDA(d, cudaMemcpyAsync(ubar_n, g, sizeof(double) * N, cudaMemcpyDeviceToDevice, d->stream));
  GH_ACUDA(d, ew(d, 1, kb, g, g, 1.0 / 6.0, 0.0, dt));                 // kb4 = dt/6 g
  at(2);
  if (gh_status s = rhs_vjp(d, u4, kb, sb, 0.0, true)) return s;       // sb = J(u4)^T kb4
  GH_ACUDA(d, ew(d, 3, kb, g, sb, 1.0 / 3.0, 1.0, dt, ubar_n));        // kb3 = dt (g/3 + sb); ubar_n += sb
  at(1);
  if (gh_status s = rhs_vjp(d, u3, kb, sb, 0.0, true, keep ? D3 : nullptr)) return s;
  GH_ACUDA(d, ew(d, 3, kb, g, sb, 1.0 / 3.0, 0.5, dt, ubar_n));        // kb2 = dt (g/3 + sb/2)
  if (gh_status s = rhs_vjp(d, u2, kb, sb, 0.0, true, keep ? D2 : nullptr)) return s;
  GH_ACUDA(d, ew(d, 3, kb, g, sb, 1.0 / 6.0, 0.5, dt, ubar_n));        // kb1 = dt (g/6 + sb/2)
  at(0);
  return rhs_vjp(d, u_n, kb, ubar_n, cweight, false, keep ? D1 : nullptr);
}

}  // namespace

extern "C" {

gh_status gh_rk4_step_vjp(gh_domain* d, double dt, const double* u_n, const double* ubar_np1, double* ubar_n,
                          double* work) {
  if (!d || !u_n || !ubar_np1 || !ubar_n || !work) return d ? afail(d, GH_EINVAL, "null argument") : GH_EINVAL;
  return step_vjp_impl(d, dt, u_n, nullptr, ubar_np1, ubar_n, work, 0.0);
}

gh_status gh_rk4_step_vjp_saved(gh_domain* d, double dt, const double* u_n, const double* stages,
                                const double* ubar_np1, double* ubar_n, double* work, double cweight) {
  if (!d || !u_n || !stages || !ubar_np1 || !ubar_n || !work)
    return d ? afail(d, GH_EINVAL, "null argument") : GH_EINVAL;
  return step_vjp_impl(d, dt, u_n, stages, ubar_np1, ubar_n, work, cweight);
}

gh_status gh_perturbation_vjp(gh_domain* d, int kind, double Rc, double w, int lmax, const double* ubar,
                              double* grad) {
  if (!d || !ubar || !grad) return d ? afail(d, GH_EINVAL, "null argument") : GH_EINVAL;
  if (kind != 1) return afail(d, GH_ENOTSUP, "only the Pi-mode perturbation (kind 1) has a gradient entry");
  if (lmax < 0 || (lmax + 1) * (lmax + 1) > gh::PV_MAX_MODES || !(w > 0.0))
    return afail(d, GH_EINVAL, "need 0 <= lmax <= 8 and w > 0");
  const int nm = (lmax + 1) * (lmax + 1);
  std::vector<int> begin(d->n_shells + 1);
  int blocks = 0;
  for (int s = 0; s < d->n_shells; ++s) {
    begin[s] = blocks;
    blocks += d->shells_h[s].n_r * ((d->shells_h[s].na + gh::PV_THREADS - 1) / gh::PV_THREADS);
  }
  begin[d->n_shells] = blocks;
  int* bd = nullptr;
  double* part = nullptr;
  GH_ACUDA(d, cudaMallocAsync(&bd, sizeof(int) * begin.size(), d->stream));
  GH_ACUDA(d, cudaMallocAsync(&part, sizeof(double) * (size_t)blocks * nm, d->stream));
  GH_ACUDA(d, cudaMemcpyAsync(bd, begin.data(), sizeof(int) * begin.size(), cudaMemcpyHostToDevice, d->stream));
  gh::pi_modes_vjp_kernel<<<blocks, gh::PV_THREADS, 0, d->stream>>>(d->shells_d, d->n_shells, bd, Rc, w, lmax,
                                                                     ubar, part);
  d->launches++;
  GH_ACUDA(d, cudaGetLastError());
  std::vector<double> h((size_t)blocks * nm);
  GH_ACUDA(d, cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, d->stream));
  GH_ACUDA(d, cudaFreeAsync(bd, d->stream));
  GH_ACUDA(d, cudaFreeAsync(part, d->stream));
  GH_ACUDA(d, cudaStreamSynchronize(d->stream));
  for (int m = 0; m < nm; ++m) {
    double acc = 0.0;
    for (int b = 0; b < blocks; ++b) acc += h[(size_t)b * nm + m];
    grad[m] = acc;
  }
  return GH_OK;
}

}  // extern "C"
