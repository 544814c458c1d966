// libgh device kernels: spectral contractions, the fused pointwise GH
// right-hand side with the RK4 stage combine, boundary conditions,
// constraints and their quadrature norms.  FP64 throughout.
//
// On GB300 the FP64 FMA pipe (about 1.2 TFLOP/s measured) is faster than the
// FP64 tensor-core path (mma.sync f64, about 1.05 TFLOP/s measured), and every
// kernel here has an arithmetic intensity far above the FP64 ridge point
// (about 0.18 flop per HBM byte), so all of them are FP64-ALU bound.  The
// contractions are therefore register-tiled FFMA kernels, and the design goal
// is to keep the FP64 pipe busy, not to save HBM traffic.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "gh_geom.cuh"
#include "gh_internal.h"
#include "gh_cpm.cuh"
#include "gh_tensor.cuh"

namespace gh {

// ---------------------------------------------------------------------------
// Radial contraction (the R part of Eq. DifferentiatorI1S2, and the radial
// ExpCheb filter): out[r][col] = sum_r' M[r][r'] in[r'][col] for every column
// col = (field, theta, phi) of every shell.  The CGL points are symmetric
// (x_{n-1-j} = -x_j), so d/dx is centro-antisymmetric and the filter
// centro-symmetric: with e_j = v_j + v_{n-1-j}, o_j = v_j - v_{n-1-j} (j < h =
// n/2) and the middle value for odd n,
//   out_i = E_i + O_i,  out_{n-1-i} = sigma (E_i - O_i)  (sigma = -1 for d/dx, +1),
//   E_i = sum_j A_ij e_j (+ M_im v_m),  O_i = sum_j B_ij o_j,
//   A_ij = (M_ij + M_i,n-1-j)/2,  B_ij = (M_ij - M_i,n-1-j)/2,
// for the ceil(n/2) rows i <= n/2 only: half the FMAs of the plain product.
// The host stores each folded row as [A_i0 .. A_i,h-1, (M_im), B_i,h-1 .. B_i0],
// matching the column folded in place (e_j at j, o_j at n-1-j).  One thread per
// column; the block's columns are staged in shared memory (coalesced loads
// along col), the folded rows it needs sit in shared memory too.  blockIdx.y
// splits the folded rows into gridDim.y groups (more, shorter warps per FP64
// unit); within a group CH rows are computed per pass as independent FMA
// chains and the remainder rows one at a time.
constexpr int RAD_THREADS = RAD_THREADS_HOST;
constexpr int MAXR = 64;

template <bool FILTER, int CH>
__global__ void __launch_bounds__(RAD_THREADS)
radial_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
              const double* __restrict__ in, double* __restrict__ out, int max_n,
              double* __restrict__ copy) {
  extern __shared__ double Vs[];           // [max n_r][RAD_THREADS], then the block's folded rows
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int n = sh.n_r, h = n >> 1, ne = n - h;   // ne: even part incl. the middle value
  double* Ms = Vs + (size_t)max_n * RAD_THREADS;
  const double* M = FILTER ? sh.Fr : sh.Dr;       // folded rows [ne][n]
  const int chunk = (ne + gridDim.y - 1) / gridDim.y;
  const int r0 = blockIdx.y * chunk;
  const int r1 = min(ne, r0 + chunk);
  for (int i = threadIdx.x; i < (r1 - r0) * n; i += blockDim.x) Ms[i] = M[r0 * n + i];
  const long long cols = (long long)NF * sh.na;
  const long long col = (long long)(blockIdx.x - begin[s]) * blockDim.x + threadIdx.x;
  const bool valid = col < cols;
  const double* src = in + sh.off + col;
  double* v = Vs + threadIdx.x;
  // copy != NULL: the input (the state in pinned host memory, read once) is
  // also written to copy at the same offsets (row group 0 only)
  double* cp = (copy && blockIdx.y == 0 && valid) ? copy + sh.off + col : nullptr;
  for (int r = 0; r < n; ++r) {
    const double x = valid ? src[(long long)r * cols] : 0.0;
    v[r * RAD_THREADS] = x;
    if (cp) cp[(long long)r * cols] = x;
  }
  for (int j = 0; j < h; ++j) {            // this thread's column, folded in place
    const double a = v[j * RAD_THREADS], b = v[(n - 1 - j) * RAD_THREADS];
    v[j * RAD_THREADS] = a + b;
    v[(n - 1 - j) * RAD_THREADS] = a - b;
  }
  __syncthreads();
  if (r0 >= r1 || !valid) return;
  double* dst = out + sh.off + col;
  auto put = [&](int i, double E, double O) {
    if (i < h) {
      dst[(long long)i * cols] = E + O;
      dst[(long long)(n - 1 - i) * cols] = FILTER ? E - O : O - E;
    } else {
      dst[(long long)i * cols] = E + O;    // middle row (odd n)
    }
  };
  int r = r0;
  for (; r + CH <= r1; r += CH) {
    const double* m0 = Ms + (r - r0) * n;
    double ae[CH], ao[CH];
    const double x0 = v[0], y0 = v[ne * RAD_THREADS];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      ae[c] = m0[c * n] * x0;
      ao[c] = m0[c * n + ne] * y0;
    }
    for (int q = 1; q < ne; ++q) {
      const double x = v[q * RAD_THREADS];
#pragma unroll
      for (int c = 0; c < CH; ++c) ae[c] = fma(m0[c * n + q], x, ae[c]);
    }
    for (int q = ne + 1; q < n; ++q) {
      const double x = v[q * RAD_THREADS];
#pragma unroll
      for (int c = 0; c < CH; ++c) ao[c] = fma(m0[c * n + q], x, ao[c]);
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) put(r + c, ae[c], ao[c]);
  }
  for (; r < r1; ++r) {
    const double* m0 = Ms + (r - r0) * n;
    double E = m0[0] * v[0];
    for (int q = 1; q < ne; ++q) E = fma(m0[q], v[q * RAD_THREADS], E);
    double O = m0[ne] * v[ne * RAD_THREADS];
    for (int q = ne + 1; q < n; ++q) O = fma(m0[q], v[q * RAD_THREADS], O);
    put(r, E, O);
  }
}

cudaError_t raise_smem_limit(const void* f, size_t bytes) {
  // The attribute belongs to the kernel on the current device, so the largest
  // limit set so far is tracked per (kernel, device).
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> current;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = current[std::make_pair(f, dev)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// Dynamic shared memory of radial_kernel: the columns and the folded rows.
size_t radial_smem_bytes(int max_n) {
  return sizeof(double) * ((size_t)max_n * RAD_THREADS + (size_t)(max_n - max_n / 2) * max_n);
}

cudaError_t radial_set_smem_limits() {
  const size_t bytes = radial_smem_bytes(MAXR);
  const void* f[6] = {(const void*)radial_kernel<true, 2>, (const void*)radial_kernel<true, 3>,
                      (const void*)radial_kernel<true, 4>, (const void*)radial_kernel<false, 2>,
                      (const void*)radial_kernel<false, 3>, (const void*)radial_kernel<false, 4>};
  for (int i = 0; i < 6; ++i) {
    cudaError_t e = raise_smem_limit(f[i], bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Batched FP64 GEMM C = A * B (row-major), one flattened tile per block.
// Used for the angular maps of Eq. DifferentiatorI1S2 (A = the state viewed as
// (n_r * 50) x (N_theta N_phi), B = a cached transposed derivative matrix) and
// for the SH truncation filter.  64x64 block tile, 16-deep k slices, 4x4
// outputs per thread, register prefetch of the next slice.
constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
constexpr int GEMM_THREADS = (BM / TM) * (BN / TN);  // 256

__global__ void __launch_bounds__(GEMM_THREADS)
gemm_batched_kernel(const GemmProb* __restrict__ probs, int nprob, const double* __restrict__ in,
                    double* __restrict__ out0, double* __restrict__ out1) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN];
  // locate the problem
  int pi = 0;
  while (pi + 1 < nprob && probs[pi + 1].tile_begin <= (int)blockIdx.x) ++pi;
  const GemmProb P = probs[pi];
  const int t = blockIdx.x - P.tile_begin;
  const int m0 = (t / P.tiles_n) * BM;
  const int n0 = (t % P.tiles_n) * BN;
  const double* A = in + P.a_off;
  const double* B = P.B;
  double* C = (P.c_sel ? out1 : out0) + P.c_off;

  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  constexpr int LA = BM * BK / GEMM_THREADS;  // 4
  constexpr int LB = BK * BN / GEMM_THREADS;  // 4
  double ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + q * GEMM_THREADS;
      const int row = e / BK, kk = e % BK;
      const int gm = m0 + row, gk = k0 + kk;
      ra[q] = (gm < P.M && gk < P.K) ? A[(long long)gm * P.lda + gk] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + q * GEMM_THREADS;
      const int kk = e / BN, col = e % BN;
      const int gk = k0 + kk, gn = n0 + col;
      rb[q] = (gk < P.K && gn < P.N) ? B[(long long)gk * P.ldb + gn] : 0.0;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = tid + q * GEMM_THREADS;
      As[e % BK][e / BK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = tid + q * GEMM_THREADS;
      Bs[e / BN][e % BN] = rb[q];
    }
  };

  load(0);
  for (int k0 = 0; k0 < P.K; k0 += BK) {
    store();
    __syncthreads();
    if (k0 + BK < P.K) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * (BM / TM);
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * (BN / TN);
      if (gn < P.N) C[(long long)gm * P.ldc + gn] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// Separable angular maps.  A row is one (r, field) pair: N_theta x N_phi
// values.  The projection onto Y_lm, l <= K, factorises into
//   A[j][mode]  = sum_k u[j][k] F[k][mode]                      (phi DFT)
//   B[j][mode]  = sum_j' Q_m[j'][j] A[j'][mode]                  (Legendre map of mode m)
//   out[j][k]   = sum_mode B[j][mode] G[mode][k]                 (inverse DFT)
// where Q_m folds the Gauss-Legendre analysis of the Pbar_lm (l = m..K) with
// their synthesis (values, or theta derivatives), and G folds the Fourier
// normalisation (and the phi derivative).  Per value this costs about
// 2 M (N_phi + N_theta + N_phi) flops instead of the 2 N_theta N_phi of a
// dense traced matrix (Eq. DifferentiatorI1S2).  A block loads RB rows into
// shared memory and runs the three phases there.  TWO = true: two outputs
// (d/dtheta and d/dphi) sharing phase A; false: one output (the SH filter).
constexpr int SEP_THREADS = 256;

template <bool TWO>
__global__ void __launch_bounds__(SEP_THREADS)
sep_angular_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                   const double* __restrict__ in, double* __restrict__ out0, double* __restrict__ out1) {
  extern __shared__ double sm[];
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const SepPlan& P = TWO ? sh.sd : sh.sf;
  const int nth = sh.nth, nph = sh.nph, na = sh.na, M = P.M, K = P.K;
  const int rows = NF * sh.n_r;
  const int RB = P.rows_per_cta;
  const int row0 = (blockIdx.x - begin[s]) * RB;
  const int nr = min(RB, rows - row0);
  double* U = sm;                          // [RB][na]
  double* A = U + (size_t)RB * na;         // [RB][nth][M]
  double* B0 = A + (size_t)RB * nth * M;   // [RB][nth][M]
  double* B1 = B0 + (size_t)RB * nth * M;  // [RB][nth][M] (TWO only)
  const double* src = in + sh.off + (long long)row0 * na;
  for (int i = threadIdx.x; i < nr * na; i += SEP_THREADS) U[i] = src[i];
  __syncthreads();
  // phase A: phi DFT of every theta ring
  const double* __restrict__ F = P.F;
  for (int o = threadIdx.x; o < nr * nth * M; o += SEP_THREADS) {
    const int mode = o % M;
    const double* ring = U + (o / M) * nph;
    double acc = 0.0;
    for (int k = 0; k < nph; ++k) acc = fma(ring[k], __ldg(F + k * M + mode), acc);
    A[o] = acc;
  }
  __syncthreads();
  // phase B: Legendre map of each Fourier mode (threads along theta_out)
  const double* __restrict__ Q0 = P.Q0;
  const double* __restrict__ Q1 = P.Q1;
  for (int o = threadIdx.x; o < nr * nth * M; o += SEP_THREADS) {
    const int j = o % nth;
    const int t = o / nth;
    const int mode = t % M;
    const int rr = t / M;
    const int m = mode <= K ? mode : mode - K;
    const double* a = A + (size_t)rr * nth * M + mode;
    const double* q0 = Q0 + (size_t)m * nth * nth + j;
    double acc0 = 0.0, acc1 = 0.0;
    if (TWO) {
      const double* q1 = Q1 + (size_t)m * nth * nth + j;
      for (int jp = 0; jp < nth; ++jp) {
        const double av = a[jp * M];
        acc0 = fma(__ldg(q0 + jp * nth), av, acc0);
        acc1 = fma(__ldg(q1 + jp * nth), av, acc1);
      }
      B1[((size_t)rr * nth + j) * M + mode] = acc1;
    } else {
      for (int jp = 0; jp < nth; ++jp) acc0 = fma(__ldg(q0 + jp * nth), a[jp * M], acc0);
    }
    B0[((size_t)rr * nth + j) * M + mode] = acc0;
  }
  __syncthreads();
  // phase C: inverse DFT into the output rows
  const double* __restrict__ G0 = P.G0;
  const double* __restrict__ G1 = P.G1;
  double* dst0 = out0 + sh.off + (long long)row0 * na;
  double* dst1 = TWO ? out1 + sh.off + (long long)row0 * na : nullptr;
  for (int o = threadIdx.x; o < nr * na; o += SEP_THREADS) {
    const int k = o % nph;
    const int rj = o / nph;
    const double* b0 = B0 + (size_t)rj * M;
    double acc0 = 0.0;
    if (TWO) {
      const double* b1 = B1 + (size_t)rj * M;
      double acc1 = 0.0;
      for (int mode = 0; mode < M; ++mode) {
        acc0 = fma(b0[mode], __ldg(G0 + mode * nph + k), acc0);
        acc1 = fma(b1[mode], __ldg(G1 + mode * nph + k), acc1);
      }
      dst1[o] = acc1;
    } else {
      for (int mode = 0; mode < M; ++mode) acc0 = fma(b0[mode], __ldg(G0 + mode * nph + k), acc0);
    }
    dst0[o] = acc0;
  }
}

cudaError_t sep_set_smem_limits(size_t bytes) {
  cudaError_t e = raise_smem_limit((const void*)sep_angular_kernel<true>, bytes);
  if (e != cudaSuccess) return e;
  return raise_smem_limit((const void*)sep_angular_kernel<false>, bytes);
}

// ---------------------------------------------------------------------------
// Fused pointwise kernel: DiffJac (Eq. DiffJac) + the GH right-hand side
// (GHEqns) for every point of every shell, one thread per point, with the
// RK4 stage combine in the epilogue and, optionally, the constraint energy
// density accumulated into per-block partial sums.
//
// stage 0: write k = dudt everywhere.
// stage 1..4: at points that a boundary condition will still modify, write k
//   and leave the combine to the boundary kernel; elsewhere skip k and write
//   stage 1: acc = k,  us = u0 + dt/2 k;   stage 2: acc += 2k, us = u0 + dt/2 k
//   stage 3: acc += 2k, us = u0 + dt k;    stage 4: us = u0 + dt/6 (acc + k)

struct PointwiseArgs {
  const ShellDev* shells;
  int n_shells;
  const int* begin;
  const double* u;       // state the RHS is evaluated at
  const double* dr;      // d/dx (CGL coordinate) of u
  const double* dth;
  const double* dph;
  double* k;
  const double* u0;
  double* acc;
  double* us;
  double* partial;       // per-block constraint energy (nullable)
  double* c_out;         // constraint components (nullable)
  double gamma0, gamma1, gamma2, dt;
  int stage;
  Frame fr;              // rotating frame of this evaluation (fr.on = 0: static)
  const Frame* frd;      // the same frame in device memory (used when set; from the domain clock)
};

__device__ __forceinline__ double stage_factor(int stage) {
  // u_s = u0 + stage_factor * dt * (k or acc + k)
  return stage == 3 ? 1.0 : (stage == 4 ? 1.0 / 6.0 : 0.5);
}

__device__ __forceinline__ void stage_combine(int stage, double cdt, double kv, long long idx,
                                              const double* u0, double* acc, double* us) {
  // cdt = stage_factor(stage) * dt
  const double u0v = u0[idx];
  if (stage == 1) {
    acc[idx] = kv;
    us[idx] = fma(cdt, kv, u0v);
  } else if (stage == 2 || stage == 3) {
    acc[idx] = fma(2.0, kv, acc[idx]);
    us[idx] = fma(cdt, kv, u0v);
  } else {
    us[idx] = fma(cdt, acc[idx] + kv, u0v);
  }
}

#ifndef GH_PT_MINB
#define GH_PT_MINB 9
#endif
#ifdef GH_PT_MAXNREG
#define GH_PT_BOUNDS __maxnreg__(GH_PT_MAXNREG)
#else
#define GH_PT_BOUNDS __launch_bounds__(PT_THREADS, GH_PT_MINB)
#endif
// The algebra below is arranged so that almost every FP64 operation is an
// FMA (GB300's FP64 pipe issues DADD and DMUL no faster than DFMA): the
// constant factors (alpha, gamma's, 1/2) are folded into per-point
// coefficient arrays, each output is built as one FMA chain, and the
// Christoffel symbols are carried as E = 2 Gamma.
template <bool RHS, bool CONSTRAINTS, bool ROT>
__global__ void GH_PT_BOUNDS
pointwise_kernel(PointwiseArgs a) {
  const int s = find_segment(a.begin, a.n_shells, blockIdx.x);
  const ShellDev& sh = a.shells[s];
  const int na = sh.na;
  const int bps = (na + PT_THREADS - 1) / PT_THREADS;  // blocks per r-slice
  const int lb = blockIdx.x - a.begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * PT_THREADS + threadIdx.x;
  const bool valid = q < na;
  double cdens = 0.0;
  if (valid) {
    const long long base = sh.off + (long long)ir * NF * na + q;
    PointGeom G;
    point_geom(sh, ir, q, G);
    double vel[3] = {0.0, 0.0, 0.0};
    Frame fr;
    if (ROT) {
      fr = a.frd ? *a.frd : a.fr;
      frame_geom(fr, G, vel);
    }
    double psi[10], Pi[10], Phi[30];
#pragma unroll
    for (int p = 0; p < 10; ++p) {
      psi[p] = a.u[base + (long long)p * na];
      Pi[p] = a.u[base + (long long)(10 + p) * na];
    }
#pragma unroll
    for (int p = 0; p < 30; ++p) Phi[p] = a.u[base + (long long)(20 + p) * na];
    // a general map's gauge source was evaluated at this frame's moving point;
    // a rotation's is the stored one with rotated components
    const double* gsrc = ((ROT && fr.gen) ? sh.gauge_t : sh.gauge) + (long long)ir * NGAUGE * na + q;
    double H[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) H[c] = gsrc[(long long)c * na];
    if (ROT && !fr.gen) frame_rotate_h(fr, H);

    Split S;
    spacetime_split(psi, S);
    const double al = S.alpha;
    const double g0 = a.gamma0, g1 = a.gamma1, g2 = a.gamma2;

    // E[a][p(b,c)] = 2 Gamma_abc = d_b psi_ac + d_c psi_ab - d_a psi_bc with
    // d_0 psi = -alpha Pi + beta^k Phi_k, d_i psi = Phi_i.  Entries with a
    // repeated index reduce to one term (a=b: d_c psi_aa) or one FMA.
    double E[40];
    {
      double d0[10];
#pragma unroll
      for (int p = 0; p < 10; ++p)
        d0[p] = fma(S.beta_up[2], Phi[20 + p], fma(S.beta_up[1], Phi[10 + p], fma(S.beta_up[0], Phi[p], -al * Pi[p])));
#define GH_DPSI(c, p) ((c) == 0 ? d0[(p)] : Phi[((c) - 1) * 10 + (p)])
#pragma unroll
      for (int aa = 0; aa < 4; ++aa)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = b; c < 4; ++c) {
            double e;
            if (b == c)
              e = (aa == b) ? GH_DPSI(aa, sym_index(aa, aa))
                            : fma(2.0, GH_DPSI(b, sym_index(aa, b)), -GH_DPSI(aa, sym_index(b, b)));
            else if (aa == b)
              e = GH_DPSI(c, sym_index(aa, aa));
            else if (aa == c)
              e = GH_DPSI(b, sym_index(aa, aa));
            else
              e = (GH_DPSI(b, sym_index(aa, c)) + GH_DPSI(c, sym_index(aa, b))) - GH_DPSI(aa, sym_index(b, c));
            E[aa * 10 + sym_index(b, c)] = e;
          }
#undef GH_DPSI
    }
    // C_a = H_a + psi^bc Gamma_abc: packed sum, diagonal pairs weighted 1/2
    double C[4];
#pragma unroll
    for (int aa = 0; aa < 4; ++aa) {
      double acc = H[aa];
#pragma unroll
      for (int p = 0; p < 10; ++p)
        acc = fma(pair_a(p) == pair_b(p) ? 0.5 * S.psi_inv[p] : S.psi_inv[p], E[aa * 10 + p], acc);
      C[aa] = acc;
    }

    // ---- sources of the Pi equation that need no derivative (10 values)
    double srcPi[10];
    double c1[3], Mp[3][3];   // Phi-equation sources: c1[i] Pi_p + Mp[i][k] Phi_kp
    if (RHS) {
      const double a2 = 2.0 * al;
      // T1: 2 alpha psi^cd g^ij Phi_ica Phi_jdb.  Raise the derivative index
      // first (R^j = 2 alpha g^ij Phi_i), then U_j[d][a] = psi^dc R^j_ca.
      {
        double ga2[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) ga2[m] = a2 * S.ginv[m];
        double R[30];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int p = 0; p < 10; ++p)
            R[j * 10 + p] = fma(ga2[s3(2, j)], Phi[20 + p], fma(ga2[s3(1, j)], Phi[10 + p], ga2[s3(0, j)] * Phi[p]));
        double U[3][16];
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int aa = 0; aa < 4; ++aa) {
              double acc = S.psi_inv[sym_index(d, 0)] * R[j * 10 + sym_index(0, aa)];
#pragma unroll
              for (int c = 1; c < 4; ++c) acc = fma(S.psi_inv[sym_index(d, c)], R[j * 10 + sym_index(c, aa)], acc);
              U[j][d * 4 + aa] = acc;
            }
#pragma unroll
        for (int p = 0; p < 10; ++p) {
          const int A = pair_a(p), B = pair_b(p);
          double acc = U[0][A] * Phi[sym_index(0, B)];
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int d = 0; d < 4; ++d)
              if (j > 0 || d > 0) acc = fma(U[j][d * 4 + A], Phi[j * 10 + sym_index(d, B)], acc);
          srcPi[p] = acc;
        }
      }
      // T2: -2 alpha psi^cd Pi_ca Pi_db  (P[c][b] = -2 alpha psi^cd Pi_db)
      {
        double P[16];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            double acc = S.psi_inv[sym_index(c, 0)] * Pi[sym_index(0, b)];
#pragma unroll
            for (int d = 1; d < 4; ++d) acc = fma(S.psi_inv[sym_index(c, d)], Pi[sym_index(d, b)], acc);
            P[c * 4 + b] = -a2 * acc;
          }
#pragma unroll
        for (int p = 0; p < 10; ++p) {
          const int A = pair_a(p), B = pair_b(p);
#pragma unroll
          for (int c = 0; c < 4; ++c) srcPi[p] = fma(Pi[sym_index(c, A)], P[c * 4 + B], srcPi[p]);
        }
      }
      // T3: -2 alpha psi^cd psi^ef Gamma_ace Gamma_bdf = -(alpha/2) sum_de Q_a[d][e] Q_b[e][d]
      // with Q_a[d][e] = psi^dc E_a[ce]
      {
        double Q[4][16];
#pragma unroll
        for (int aa = 0; aa < 4; ++aa)
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              double acc = S.psi_inv[sym_index(d, 0)] * E[aa * 10 + sym_index(0, e)];
#pragma unroll
              for (int c = 1; c < 4; ++c) acc = fma(S.psi_inv[sym_index(d, c)], E[aa * 10 + sym_index(c, e)], acc);
              Q[aa][d * 4 + e] = acc;
            }
        const double mh = -0.5 * al;
#pragma unroll
        for (int p = 0; p < 10; ++p) {
          const int A = pair_a(p), B = pair_b(p);
          double t3 = Q[A][0] * Q[B][0];
#pragma unroll
          for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (d > 0 || e > 0) t3 = fma(Q[A][d * 4 + e], Q[B][e * 4 + d], t3);
          srcPi[p] = fma(mh, t3, srcPi[p]);
        }
      }
      // remaining Pi sources, one FMA chain per pair:
      //   -2 alpha nabla_(a H_b) = -alpha (d_a H_b + d_b H_a) + alpha psi^cd H_c E_d[ab]
      //   -1/2 alpha t^c t^d Pi_cd Pi_ab
      //   (-alpha t^c Pi_ci g^ij - gamma1 gamma2 beta^j) Phi_jab
      //   + alpha gamma0 (t_b C_a + t_a C_b - psi_ab t^c C_c),  t_a = (-alpha, 0, 0, 0)
      {
        double dH[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) dH[c] = gsrc[(long long)(4 + c) * na];
        if (ROT && !fr.gen) frame_rotate_dh(fr, dH);
        double aH[4], PHa[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) aH[c] = al * H[c];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          double acc = S.psi_inv[sym_index(0, d)] * aH[0];
#pragma unroll
          for (int c = 1; c < 4; ++c) acc = fma(S.psi_inv[sym_index(c, d)], aH[c], acc);
          PHa[d] = acc;
        }
        // tt[p] = t^a t^b, off-diagonal pairs doubled (for t^c t^d X_cd sums)
        double tt[10];
#pragma unroll
        for (int p = 0; p < 10; ++p) {
          const int A = pair_a(p), B = pair_b(p);
          tt[p] = (A == B ? S.t_up[A] : 2.0 * S.t_up[A]) * S.t_up[B];
        }
        double tPt = tt[0] * Pi[0];
#pragma unroll
        for (int p = 1; p < 10; ++p) tPt = fma(tt[p], Pi[p], tPt);
        const double k1 = -0.5 * al * tPt;
        double tPi[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          double acc = S.t_up[0] * Pi[sym_index(0, 1 + i)];
#pragma unroll
          for (int c = 1; c < 4; ++c) acc = fma(S.t_up[c], Pi[sym_index(c, 1 + i)], acc);
          tPi[i] = acc;
        }
        const double g12 = g1 * g2;
        double qv[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const double tg = fma(tPi[2], S.ginv[s3(2, j)], fma(tPi[1], S.ginv[s3(1, j)], tPi[0] * S.ginv[s3(0, j)]));
          qv[j] = fma(-al, tg, -g12 * S.beta_up[j]);
        }
        double tC = S.t_up[0] * C[0];
#pragma unroll
        for (int c = 1; c < 4; ++c) tC = fma(S.t_up[c], C[c], tC);
        const double kd1 = -al * al * g0, kd2 = -al * g0 * tC;
#pragma unroll
        for (int p = 0; p < 10; ++p) {
          const int A = pair_a(p), B = pair_b(p);
          double acc = srcPi[p];
#pragma unroll
          for (int d = 0; d < 4; ++d) acc = fma(PHa[d], E[d * 10 + p], acc);
          if (A > 0 || B > 0) {
            const double dAHB = (A > 0 ? dH[4 * (A - 1) + B] : 0.0);
            const double dBHA = (B > 0 ? dH[4 * (B - 1) + A] : 0.0);
            acc = fma(-al, (A > 0 && B > 0) ? dAHB + dBHA : (A > 0 ? dAHB : dBHA), acc);
          }
          acc = fma(k1, Pi[p], acc);
#pragma unroll
          for (int j = 0; j < 3; ++j) acc = fma(qv[j], Phi[j * 10 + p], acc);
          acc = fma(kd2, psi[p], acc);
          if (p == 0) acc = fma(2.0 * kd1, C[0], acc);
          else if (A == 0) acc = fma(kd1, C[B], acc);
          srcPi[p] = acc;
        }
        // Phi sources: 1/2 alpha t^c t^d Phi_icd Pi_ab + alpha g^jk t^c Phi_ijc Phi_kab
        //              - alpha gamma2 Phi_iab
        const double hal = 0.5 * al, ag2 = al * g2;
        double gal[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) gal[m] = al * S.ginv[m];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          double acc = tt[0] * Phi[i * 10];
#pragma unroll
          for (int p = 1; p < 10; ++p) acc = fma(tt[p], Phi[i * 10 + p], acc);
          c1[i] = hal * acc;
          double tj[3];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            double t2 = S.t_up[0] * Phi[i * 10 + sym_index(1 + j, 0)];
#pragma unroll
            for (int c = 1; c < 4; ++c) t2 = fma(S.t_up[c], Phi[i * 10 + sym_index(1 + j, c)], t2);
            tj[j] = t2;
          }
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const double m = fma(tj[2], gal[s3(2, k)], fma(tj[1], gal[s3(1, k)], tj[0] * gal[s3(0, k)]));
            Mp[i][k] = (i == k) ? m - ag2 : m;
          }
        }
      }
    }

    // loop-invariant coefficients of the derivative terms (spherical basis):
    //   bs[d] = beta^k J_k^d,  Gsa[i][d] = -alpha g^ki J_k^d,
    //   Ja = -alpha J,  Jg = alpha gamma2 J
    double bs[3], Gsa[3][3], Ja[3][3], Jg[3][3];
    {
      const double ag2 = al * g2;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        bs[d] = fma(S.beta_up[2], G.J[2][d], fma(S.beta_up[1], G.J[1][d], S.beta_up[0] * G.J[0][d]));
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const double gj = fma(S.ginv[s3(2, i)], G.J[2][d], fma(S.ginv[s3(1, i)], G.J[1][d], S.ginv[s3(0, i)] * G.J[0][d]));
          Gsa[i][d] = -al * gj;
          Ja[i][d] = -al * G.J[i][d];
          Jg[i][d] = ag2 * G.J[i][d];
        }
      }
    }
    const double g1p = 1.0 + g1, g12 = g1 * g2;
    const double nbg[3] = {-g1 * S.beta_up[0], -g1 * S.beta_up[1], -g1 * S.beta_up[2]};

    // constraint components of this point: c_out[64 pt_off + (ir*64 + comp)*na + q]
    const long long cbase = 64LL * sh.pt_off + (long long)ir * NC * na + q;
    if (CONSTRAINTS) {
      double c2 = C[0] * C[0];
#pragma unroll
      for (int c = 1; c < 4; ++c) c2 = fma(C[c], C[c], c2);
      if (a.c_out) {
#pragma unroll
        for (int c = 0; c < 4; ++c) a.c_out[cbase + (long long)c * na] = C[c];
      }
      cdens = c2;
    }

    const bool on_bc = (ir == 0 && sh.bc_inner >= 0) || (ir == sh.n_r - 1 && sh.bc_outer >= 0);
    const double cdt = stage_factor(a.stage) * a.dt * sh.dt_scale;
    // grid-velocity term xdot^k d_k (spherical basis); at boundary points the
    // boundary kernel adds it after the boundary conditions
    const bool adv = ROT && !on_bc;
    double vs[3] = {0.0, 0.0, 0.0};
    if (adv) {
#pragma unroll
      for (int d = 0; d < 3; ++d) vs[d] = fma(vel[2], G.J[2][d], fma(vel[1], G.J[1][d], vel[0] * G.J[0][d]));
    }
    // ---- derivative terms, one symmetric pair at a time
#pragma unroll 1
    for (int p = 0; p < 10; ++p) {
      double dpsi[3], dPi[3], dPhi[3][3];  // spherical-basis derivatives
      {
        const long long o = base + (long long)p * na;
        dpsi[0] = a.dr[o]; dpsi[1] = a.dth[o]; dpsi[2] = a.dph[o];
        const long long o2 = base + (long long)(10 + p) * na;
        dPi[0] = a.dr[o2]; dPi[1] = a.dth[o2]; dPi[2] = a.dph[o2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const long long o3 = base + (long long)(20 + 10 * i + p) * na;
          dPhi[i][0] = a.dr[o3]; dPhi[i][1] = a.dth[o3]; dPhi[i][2] = a.dph[o3];
        }
      }
      if (CONSTRAINTS) {
        // C_iab = d_i psi_ab - Phi_iab ; C_ijab = d_i Phi_jab - d_j Phi_iab
        double c3[3], c4[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          c3[i] = fma(G.J[i][2], dpsi[2], fma(G.J[i][1], dpsi[1], fma(G.J[i][0], dpsi[0], -Phi[i * 10 + p])));
        // d_k Phi_i = J[k] . dPhi[i]
        auto dk = [&](int k, int i) {
          return fma(G.J[k][2], dPhi[i][2], fma(G.J[k][1], dPhi[i][1], G.J[k][0] * dPhi[i][0]));
        };
        c4[0] = dk(0, 1) - dk(1, 0);
        c4[1] = dk(0, 2) - dk(2, 0);
        c4[2] = dk(1, 2) - dk(2, 1);
#pragma unroll
        for (int i = 0; i < 3; ++i) cdens = fma(c4[i], c4[i], fma(c3[i], c3[i], cdens));
        if (a.c_out) {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            a.c_out[cbase + (long long)(4 + 10 * i + p) * na] = c3[i];
            a.c_out[cbase + (long long)(34 + 10 * i + p) * na] = c4[i];
          }
        }
      }
      if (RHS) {
        const double bdpsi = fma(bs[2], dpsi[2], fma(bs[1], dpsi[1], bs[0] * dpsi[0]));
        double out[5];
        // psi: (1 + gamma1) beta.d psi - alpha Pi - gamma1 beta^k Phi_k
        {
          double acc = fma(-al, Pi[p], g1p * bdpsi);
#pragma unroll
          for (int k = 0; k < 3; ++k) acc = fma(nbg[k], Phi[k * 10 + p], acc);
          out[0] = acc;
        }
        // Pi: src + beta.d Pi - alpha g^ki d_k Phi_i + gamma1 gamma2 beta.d psi
        {
          double acc = fma(g12, bdpsi, srcPi[p]);
#pragma unroll
          for (int d = 0; d < 3; ++d) acc = fma(bs[d], dPi[d], acc);
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) acc = fma(Gsa[i][d], dPhi[i][d], acc);
          out[1] = acc;
        }
        // Phi_i: src + beta.d Phi_i - alpha d_i Pi + alpha gamma2 d_i psi
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          double acc = c1[i] * Pi[p];
#pragma unroll
          for (int k = 0; k < 3; ++k) acc = fma(Mp[i][k], Phi[k * 10 + p], acc);
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            acc = fma(bs[d], dPhi[i][d], acc);
            acc = fma(Ja[i][d], dPi[d], acc);
            acc = fma(Jg[i][d], dpsi[d], acc);
          }
          out[2 + i] = acc;
        }
        if (adv) {
          out[0] = fma(vs[2], dpsi[2], fma(vs[1], dpsi[1], fma(vs[0], dpsi[0], out[0])));
          out[1] = fma(vs[2], dPi[2], fma(vs[1], dPi[1], fma(vs[0], dPi[0], out[1])));
#pragma unroll
          for (int i = 0; i < 3; ++i)
            out[2 + i] = fma(vs[2], dPhi[i][2], fma(vs[1], dPhi[i][1], fma(vs[0], dPhi[i][0], out[2 + i])));
        }
        const int fidx[5] = {p, 10 + p, 20 + p, 30 + p, 40 + p};
#pragma unroll
        for (int e = 0; e < 5; ++e) {
          const long long idx = base + (long long)fidx[e] * na;
          if (a.stage == 0 || on_bc) a.k[idx] = out[e];
          else stage_combine(a.stage, cdt, out[e], idx, a.u0, a.acc, a.us);
        }
      }
    }
  }
  if (CONSTRAINTS) {
    // weighted block sum of the constraint energy density (deterministic order)
    __shared__ double red[PT_THREADS];
    double w = 0.0;
    if (valid) {
      const int j = q / sh.nph;
      w = sh.wr[ir] * sh.wth[j];
    }
    red[threadIdx.x] = valid ? w * cdens : 0.0;
    __syncthreads();
    for (int st = PT_THREADS / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) a.partial[blockIdx.x] = red[0];
  }
}


// ---------------------------------------------------------------------------
// Characteristic boundary conditions (ApplyBCs, Sec. 5), one thread per point
// of every boundary slice.  The projection uses the fixed background (unit
// normal n_i along +R, lapse, shift), so it is linear in dudt:
//   w_psi = psi, w0_iab = Phi_iab - n_i n^k Phi_kab, w_pm = Pi +- n^k Phi_k - g2 psi
//   speeds v_psi = -(1+g1) n.beta, v_0 = -n.beta, v_pm = -n.beta +- alpha.
// Outer boundary: incoming families (v < 0) get zero time derivative.
// Internal boundary: v < 0 families take the outer shell's value on both
// sides, v > 0 families the inner shell's, v = 0 families keep their own.
// After the condition the RK4 stage combine of those points is done here.
struct BcArgs {
  const BcSliceDev* slices;
  int n_slices;
  const int* pt_begin;   // first boundary point of each slice, [n_slices + 1]
  double* k;
  const double* u0;
  double* acc;
  double* us;
  double gamma1, gamma2, dt;
  int stage;
  // constraint-preserving outer condition: the state the RHS was evaluated at,
  // its spherical-basis derivatives and the shells (for the DiffJac matrix)
  int cp_outer;
  const ShellDev* shells;
  const double* u_in;
  const double* dr;
  const double* dth;
  const double* dph;
  Frame fr;              // rotating frame (fr.on = 0: static)
  const Frame* frd;      // the same frame in device memory (used when set)
  const double* cpm_S;   // cp_outer = 2: d_t u^- per (pair, boundary point) from cp_minus_kernel
};

// Bjorhus-form constraint-preserving corrections at an outer-boundary point for
// pair p: nC3 = n^i C_ip (C_iab = d_i psi_ab - Phi_iab) and
// Pm[i] = P_i^k n^j C_jkp (C_jkab = d_j Phi_kab - d_k Phi_jab).
__device__ __forceinline__ void cp_corrections(const BcArgs& a, const Frame& fr, const BcSliceDev& sl, int q, int p,
                                               const double n_dn[3], const double n_up[3], double& nC3,
                                               double Pm[3]) {
  const ShellDev& sh = a.shells[sl.shell_a];
  PointGeom G;
  point_geom(sh, sh.n_r - 1, q, G);
  if (fr.on) {
    double vel[3];
    frame_geom(fr, G, vel);
  }
  const int na = sl.na;
  const long long base = sl.off_a + q;
  auto cart = [&](int f, int i) {
    const long long o = base + (long long)f * na;
    return fma(G.J[i][2], a.dph[o], fma(G.J[i][1], a.dth[o], G.J[i][0] * a.dr[o]));
  };
  nC3 = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) nC3 = fma(n_up[i], cart(p, i) - a.u_in[base + (long long)(20 + 10 * i + p) * na], nC3);
  double dPhi[3][3];   // dPhi[j][k] = d_j Phi_kp
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) dPhi[j][k] = cart(20 + 10 * k + p, j);
  double m[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) acc = fma(n_up[j], dPhi[j][k] - dPhi[k][j], acc);
    m[k] = acc;
  }
  const double nm = n_up[0] * m[0] + n_up[1] * m[1] + n_up[2] * m[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) Pm[i] = m[i] - n_dn[i] * nm;
}

// The characteristic projection couples only the 5 fields of one symmetric
// pair p (psi_p, Pi_p, Phi_xp, Phi_yp, Phi_zp), so each thread handles one
// (boundary point, pair): char fields w_psi, w_plus, w_minus, w0_i.
struct CharPair {
  double psi, wp, wm, w0[3];
};

__device__ __forceinline__ void char_project_pair(const double* k, long long base, int na, int p,
                                                  const double n_dn[3], const double n_up[3], double g2,
                                                  CharPair& c) {
  const double ps = k[base + (long long)p * na];
  const double pi = k[base + (long long)(10 + p) * na];
  double ph[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) ph[i] = k[base + (long long)(20 + 10 * i + p) * na];
  const double nphi = n_up[0] * ph[0] + n_up[1] * ph[1] + n_up[2] * ph[2];
  c.psi = ps;
  c.wp = pi + nphi - g2 * ps;
  c.wm = pi - nphi - g2 * ps;
#pragma unroll
  for (int i = 0; i < 3; ++i) c.w0[i] = ph[i] - n_dn[i] * nphi;
}

// Grid-velocity term xdot^k d_k u of pair p's five fields at a boundary point
// (shell `shell`, radial index ir, slice offset base), from the derivative
// scratch of the state the RHS was evaluated at.
__device__ __forceinline__ void frame_adv(const BcArgs& a, const Frame& fr, int shell, int ir, long long base, int na,
                                          int p, int q, double adv[5]) {
  const ShellDev& sh = a.shells[shell];
  PointGeom G;
  point_geom(sh, ir, q, G);
  double vel[3], vs[3];
  frame_geom(fr, G, vel);
#pragma unroll
  for (int d = 0; d < 3; ++d) vs[d] = fma(vel[2], G.J[2][d], fma(vel[1], G.J[1][d], vel[0] * G.J[0][d]));
  const int f[5] = {p, 10 + p, 20 + p, 30 + p, 40 + p};
#pragma unroll
  for (int e = 0; e < 5; ++e) {
    const long long o = base + (long long)f[e] * na;
    adv[e] = fma(vs[2], a.dph[o], fma(vs[1], a.dth[o], vs[0] * a.dr[o]));
  }
}

__device__ __forceinline__ void char_write_pair(const BcArgs& a, long long base, int na, int p, const CharPair& c,
                                                const double n_dn[3], double g2, double cdt,
                                                const double* adv = nullptr) {
  double v[5];
  v[0] = c.psi;
  v[1] = 0.5 * (c.wp + c.wm) + g2 * c.psi;
  const double h = 0.5 * (c.wp - c.wm);
#pragma unroll
  for (int i = 0; i < 3; ++i) v[2 + i] = n_dn[i] * h + c.w0[i];
  if (adv) {
#pragma unroll
    for (int e = 0; e < 5; ++e) v[e] += adv[e];
  }
  const int f[5] = {p, 10 + p, 20 + p, 30 + p, 40 + p};
#pragma unroll
  for (int e = 0; e < 5; ++e) {
    const long long idx = base + (long long)f[e] * na;
    if (a.stage == 0) a.k[idx] = v[e];
    else stage_combine(a.stage, cdt, v[e], idx, a.u0, a.acc, a.us);
  }
}

__device__ __forceinline__ void select_pair(double& wi, double& wo, double v) {
  // v < 0: both take the outer side's value; v > 0: both take the inner side's.
  if (v < 0.0) wi = wo;
  else if (v > 0.0) wo = wi;
}

__global__ void __launch_bounds__(128) bc_kernel(BcArgs a) {
  const int npts = a.pt_begin[a.n_slices];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 10 * npts) return;
  const int p = t / npts;
  const int pt = t - p * npts;
  const int s = find_segment(a.pt_begin, a.n_slices, pt);
  const BcSliceDev& sl = a.slices[s];
  const int q = pt - a.pt_begin[s];
  const int na = sl.na;
  double n_dn[3], n_up[3], beta[3];
  const Frame fr = (a.fr.on && a.frd) ? *a.frd : a.fr;
  // the background at the moving point: a general map's evaluated there (with
  // the normal velocity of the moving boundary), a rotation's rotated
  const double* bgs = fr.gen ? sl.bg_t : sl.bg;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    n_dn[i] = bgs[(long long)i * na + q];
    n_up[i] = bgs[(long long)(3 + i) * na + q];
    beta[i] = bgs[(long long)(7 + i) * na + q];
  }
  const double alpha = bgs[(long long)6 * na + q];
  if (fr.on && !fr.gen) frame_rotate_bg(fr, n_dn, n_up, beta);
  const double nb = n_dn[0] * beta[0] + n_dn[1] * beta[1] + n_dn[2] * beta[2];
  // speeds relative to the boundary: a moving one shifts them all by -n . xdot
  const double vsh = fr.gen ? bgs[(long long)10 * na + q] : 0.0;
  const double v_psi = -(1.0 + a.gamma1) * nb - vsh, v_0 = -nb - vsh, v_p = -nb + alpha - vsh, v_m = -nb - alpha - vsh;
  const double g2 = a.gamma2;
  if (sl.kind == 0) {
    const long long base = sl.off_a + q;
    CharPair c;
    char_project_pair(a.k, base, na, p, n_dn, n_up, g2, c);
    if (a.cp_outer) {
      // constraint preserving for u^psi and u^0, freezing for u^- (and u^+)
      if (v_psi < 0.0 || v_0 < 0.0) {
        double nC3, Pm[3];
        cp_corrections(a, fr, sl, q, p, n_dn, n_up, nC3, Pm);
        if (v_psi < 0.0) c.psi = fma(v_psi, nC3, c.psi);
        if (v_0 < 0.0) {
#pragma unroll
          for (int i = 0; i < 3; ++i) c.w0[i] = fma(v_0, Pm[i], c.w0[i]);
        }
      }
    } else {
      if (v_psi < 0.0) c.psi = 0.0;
      if (v_0 < 0.0) c.w0[0] = c.w0[1] = c.w0[2] = 0.0;
    }
    if (v_p < 0.0) c.wp = 0.0;
    if (v_m < 0.0) c.wm = (a.cp_outer == 2) ? a.cpm_S[(long long)p * npts + pt] : 0.0;
    double adv[5];
    if (fr.on) frame_adv(a, fr, sl.shell_a, a.shells[sl.shell_a].n_r - 1, base, na, p, q, adv);
    char_write_pair(a, base, na, p, c, n_dn, g2, stage_factor(a.stage) * a.dt * sl.dt_scale,
                    fr.on ? adv : nullptr);
  } else {
    const long long ba = sl.off_a + q, bb = sl.off_b + q;
    CharPair ci, co;
    char_project_pair(a.k, ba, na, p, n_dn, n_up, g2, ci);
    char_project_pair(a.k, bb, na, p, n_dn, n_up, g2, co);
    select_pair(ci.psi, co.psi, v_psi);
#pragma unroll
    for (int i = 0; i < 3; ++i) select_pair(ci.w0[i], co.w0[i], v_0);
    select_pair(ci.wp, co.wp, v_p);
    select_pair(ci.wm, co.wm, v_m);
    double adv_a[5], adv_b[5];
    if (fr.on) {
      frame_adv(a, fr, sl.shell_a, a.shells[sl.shell_a].n_r - 1, ba, na, p, q, adv_a);
      frame_adv(a, fr, sl.shell_b, 0, bb, na, p, q, adv_b);
    }
    char_write_pair(a, ba, na, p, ci, n_dn, g2, stage_factor(a.stage) * a.dt * sl.dt_scale,
                    fr.on ? adv_a : nullptr);
    char_write_pair(a, bb, na, p, co, n_dn, g2, stage_factor(a.stage) * a.dt * sl.dt_scale,
                    fr.on ? adv_b : nullptr);
  }
}

// ---------------------------------------------------------------------------
// The constraint part of u^- in the constraint-preserving outer condition
// (cp_outer = 2).  Reading of Sec. 5's constraint-preserving outer boundary
// for the u^- family: the gauge constraint C_a = H_a + psi^bc Gamma_abc may
// not enter through the boundary.  It propagates like a wave, whose incoming
// characteristic field is its derivative along the outgoing null direction
// (as u^- is -(t + n).d psi for psi),
//   K_a = (d_t C_a - beta^i d_i C_a) / N + n^i d_i C_a
// (background lapse, shift and normal; d_t C_a along a time derivative of the
// state, d_i C_a along its Cartesian derivatives and those of H_a).  With the
// interior equations K_a holds the normal derivative of u^- as 2 B(d_n u^-),
// B the slope of K_a in d_t u^- (a u^- derivative S changes d_t Pi by S/2 and
// d_t Phi_i by -n_i S/2).  In Bjorhus form the condition replaces d_n u^- in
// the u^- equation by the value that makes K_a (interior) vanish, so the
// boundary equation of u^- holds no normal derivative of u^-:
//   B(S) = -K_a[w^- = 0] + (N - n.beta) / (2N) K_a[w^- = D_t u^-].
// S is sought as l_a lam_b + lam_a l_b + sig P_ab with l^b lam_b = 0: the
// l l, l m and transverse-trace parts of a null tetrad of the background
// (l = (t + n)/sqrt 2, P the projector orthogonal to t and n), on which B is
// invertible; its gauge (k k, k m, l k) and physical (transverse traceless)
// parts lie in the kernel of B and stay frozen.  One 5x5 solve per point.

// Three outer-boundary points per warp where u^- is incoming (CPM_WARPS warps
// per block); each point's data lives in shared memory:
//   u, k       the state and its interior right-hand side (50 fields each),
//   du[i]      the Cartesian derivatives d_i u,
//   psi_inv, N, t^i, beta^i and D_cab (the state's split, gh_cpm.cuh),
//   ud         the time derivative with the u^psi, u^0, u^+ conditions and w^- = 0,
//   wm_int     the interior d_t u^- per pair,
//   l_dn, l_up, P  the background null vector and transverse projector,
//   vdir       the field-space directions of the six slope evaluations,
//   res[e]     the ten directional derivatives of C_a (cpm_system).
#ifndef GH_CPM_WARPS
#define GH_CPM_WARPS 2
#endif
constexpr int CPM_WARPS = GH_CPM_WARPS;

struct CpmWarp {
  double u[50], k[50], du[3][50];
  double psi_inv[10], t_up[3], beta[3], N;
  double D[40];
  double ud[50];
  double wm_int[10];
  double l_dn[4], l_up[4], P[10];
  double vdir[6][50];
  double res[10][4];
  double x[5];
};

// Three outer-boundary points per warp, ten lanes each (lanes 30 and 31 idle),
// where u^- is incoming: writes S[pair * npts + point] for bc_kernel (a
// singular system leaves u^- frozen).  The ten lanes of a point evaluate, one
// each, the directional derivatives of C_a that the solve needs: along the
// corrected time derivative with w^- = 0 (e = 0), along d_i u with d_i H
// (e = 1..3), and the slope B along the four l_(a e_b) basis tensors, P and
// the interior w^- (e = 4..9); lane e = 0 solves.  Every lane reaches every
// __syncwarp; a group without a point (or where u^- is not incoming) idles.
__global__ void __launch_bounds__(32 * CPM_WARPS) cp_minus_kernel(BcArgs a, double* __restrict__ Sout) {
  __shared__ CpmWarp smem[3 * CPM_WARPS];
  const int warp = threadIdx.x >> 5, lane0 = threadIdx.x & 31;
  const int sub = lane0 / 10, lane = lane0 - 10 * sub;
  const int npts = a.pt_begin[a.n_slices];
  const int t = (blockIdx.x * CPM_WARPS + warp) * 3 + sub;
  bool active = sub < 3 && t < npts;
  const int sidx = active ? find_segment(a.pt_begin, a.n_slices, t) : 0;
  const BcSliceDev& sl = a.slices[sidx];
  active = active && sl.kind == 0;
  const int q = active ? t - a.pt_begin[sidx] : 0;
  const int na = sl.na;
  CpmBg b;
  if (active) {
    cpm_load_bg(sl.bg, na, q, b);
    active = (-b.nb - b.Nb) < 0.0;          // u^- incoming
  }
  CpmWarp& S = smem[3 * warp + (sub < 3 ? sub : 0)];
  const ShellDev& sh = a.shells[sl.shell_a];
  const long long base = sl.off_a + q;

  // 1. the state, its right-hand side and its Cartesian derivatives
  if (active) {
    PointGeom G;
    point_geom(sh, sh.n_r - 1, q, G);
    for (int f = lane; f < 50; f += 10) {
      S.u[f] = a.u_in[base + (long long)f * na];
      S.k[f] = a.k[base + (long long)f * na];
    }
    for (int e = lane; e < 150; e += 10) {
      const int i = e / 50, f = e - 50 * i;
      const long long o = base + (long long)f * na;
      S.du[i][f] = fma(G.J[i][2], a.dph[o], fma(G.J[i][1], a.dth[o], G.J[i][0] * a.dr[o]));
    }
  }
  __syncwarp();
  // 2. lane 0: the state's split, D and the background tetrad; lane p: pair p
  // of the corrected time derivative (w^- = 0) and of the interior w^-
  if (active && lane == 0) {
    cpm_state(S);
    cpm_tetrad(b, S.l_dn, S.l_up, S.P);
  }
  if (active) cpm_pair(lane, S.k, S.u, S.du, b, a.gamma1, a.gamma2, S.ud, &S.wm_int[lane]);
  __syncwarp();
  // 3. lanes 4..9: the directions of the slopes B(E) = C'(w^- = E) / N for
  // E = l_(a e_b) (b = 0..3), P and the interior w^-
  if (active && lane >= 4) {
    double E[10];
    cpm_basis(lane - 4, S.l_dn, S.P, S.wm_int, E);
    cpm_vdir(E, b.n_dn, S.vdir[lane - 4]);
  }
  __syncwarp();
  // 4. the ten directional derivatives, one per lane and all through one call
  if (active) {
    const double* v = (lane == 0) ? S.ud : (lane <= 3 ? S.du[lane - 1] : S.vdir[lane - 4]);
    double dH[4] = {0.0, 0.0, 0.0, 0.0};
    if (lane >= 1 && lane <= 3) {
      const double* gauge = sh.gauge + (long long)(sh.n_r - 1) * NGAUGE * na + q;
#pragma unroll
      for (int c = 0; c < 4; ++c) dH[c] = gauge[(long long)(4 + 4 * (lane - 1) + c) * na];
    }
    double r[4];
    gauge_constraint_dir(S, v, dH, r);
    const double sc = (lane >= 4) ? 1.0 / b.Nb : 1.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) S.res[lane][c] = r[c] * sc;
  }
  __syncwarp();
  // 5. lane 0: the Bjorhus target and the 5x5 solve
  if (active && lane == 0) {
    double M[5][6], x[5];
    cpm_system(S.res, b, S.l_up, M);
    cpm_solve5(M, x);
#pragma unroll
    for (int e = 0; e < 5; ++e) S.x[e] = x[e];
  }
  __syncwarp();
  // 6. S_ab = l_a lam_b + lam_a l_b + sig P_ab, one pair per lane
  if (active) {
    const int A = pair_a(lane), B = pair_b(lane);
    Sout[(long long)lane * npts + t] = S.l_dn[A] * S.x[B] + S.x[A] * S.l_dn[B] + S.x[4] * S.P[lane];
  }
}

// ---------------------------------------------------------------------------
// Boundary background from the metric part of a state: lapse, shift and the
// unit normal n_i = d_i R / |d R|_g, n^i = g^ij n_j.
__global__ void __launch_bounds__(128)
bc_background_kernel(const ShellDev* __restrict__ shells, BcSliceDev* slices, int n_slices,
                     const int* __restrict__ pt_begin, const double* __restrict__ u, int bh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= pt_begin[n_slices]) return;
  const int s = find_segment(pt_begin, n_slices, t);
  BcSliceDev& sl = slices[s];
  if (bh >= 0 && sl.bh != bh) return;
  const int q = t - pt_begin[s];
  const int na = sl.na;
  const ShellDev& sh = shells[sl.shell_a];
  double psi[10];
#pragma unroll
  for (int p = 0; p < 10; ++p) psi[p] = u[sl.off_a + (long long)p * na + q];
  Split S;
  spacetime_split(psi, S);
  const int j = q / sh.nph, k = q - j * sh.nph;
  const double dR[3] = {sh.sth[j] * sh.cph[k], sh.sth[j] * sh.sph[k], sh.cth[j]};
  double nn = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int m = 0; m < 3; ++m) nn += S.ginv[s3(i, m)] * dR[i] * dR[m];
  const double inv = 1.0 / sqrt(nn);
  double n_dn[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) n_dn[i] = dR[i] * inv;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    sl.bg[(long long)i * na + q] = n_dn[i];
    sl.bg[(long long)(3 + i) * na + q] =
        S.ginv[s3(i, 0)] * n_dn[0] + S.ginv[s3(i, 1)] * n_dn[1] + S.ginv[s3(i, 2)] * n_dn[2];
    sl.bg[(long long)(7 + i) * na + q] = S.beta_up[i];
  }
  sl.bg[(long long)6 * na + q] = S.alpha;
#pragma unroll
  for (int m = 0; m < 6; ++m) sl.bg[(long long)(10 + m) * na + q] = psi[4 + m];   // g_ij, pairs 11 12 13 22 23 33
}

// ---------------------------------------------------------------------------
// Cartesian derivatives d_i u of all 50 fields (Eq. DiffJac applied to the
// output of the radial and angular maps).  One thread per (point, field).
__global__ void __launch_bounds__(PT_THREADS)
cartesian_kernel(const ShellDev* __restrict__ shells, int n_shells, const int* __restrict__ begin,
                 const double* __restrict__ dr, const double* __restrict__ dth,
                 const double* __restrict__ dph, double* __restrict__ du, long long state, Frame fr,
                 const Frame* __restrict__ frd) {
  const int s = find_segment(begin, n_shells, blockIdx.x);
  const ShellDev& sh = shells[s];
  const int na = sh.na;
  const int bps = (na + PT_THREADS - 1) / PT_THREADS;
  const int lb = blockIdx.x - begin[s];
  const int ir = lb / bps;
  const int q = (lb - ir * bps) * PT_THREADS + threadIdx.x;
  if (q >= na) return;
  PointGeom G;
  point_geom(sh, ir, q, G);
  if (fr.on) {
    if (frd) fr = *frd;
    double vel[3];
    frame_geom(fr, G, vel);
  }
  const long long base = sh.off + (long long)ir * NF * na + q;
  for (int f = 0; f < NF; ++f) {
    const long long o = base + (long long)f * na;
    const double a0 = dr[o], a1 = dth[o], a2 = dph[o];
#pragma unroll
    for (int i = 0; i < 3; ++i) du[i * state + o] = G.J[i][0] * a0 + G.J[i][1] * a1 + G.J[i][2] * a2;
  }
}

// ---------------------------------------------------------------------------
// Per-shell sum of the per-block constraint partials, in a fixed order, and
// a latched error if the result is not finite.
__global__ void norm_reduce_kernel(const int* __restrict__ begin, int n_shells,
                                   const double* __restrict__ partial, double* norm2, int* err) {
  const int s = blockIdx.x;
  if (s >= n_shells) return;
  __shared__ double red[256];
  double acc = 0.0;
  for (int b = begin[s] + threadIdx.x; b < begin[s + 1]; b += blockDim.x) acc += partial[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    norm2[s] = red[0];
    if (!isfinite(red[0])) atomicExch(err, (int)GH_ENONFINITE);
  }
}

// ---------------------------------------------------------------------------
// Launchers.
static inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

cudaError_t launch_radial(gh_domain* d, const double* in, double* out, bool filter) {
  return launch_radial_on(d, in, out, filter, d->stream);
}

cudaError_t launch_radial_on(gh_domain* d, const double* in, double* out, bool filter, cudaStream_t st,
                             double* copy) {
  const size_t smem = radial_smem_bytes(d->max_n_r);
  const int ch = filter ? d->radf_chains : d->rad_chains;
  // with a copy-out the input is read by one row group only (it may be host memory)
  const dim3 grid(d->rad_blocks, copy ? 1 : (filter ? d->radf_groups : d->rad_groups));
#define GH_RAD(F, C)                                                                       \
  radial_kernel<F, C><<<grid, RAD_THREADS, smem, st>>>(d->shells_d, d->n_shells,           \
                                                               d->rad_block_begin_d, in, out, d->max_n_r, copy)
  if (filter) {
    if (ch == 4) GH_RAD(true, 4); else if (ch == 3) GH_RAD(true, 3); else GH_RAD(true, 2);
  } else {
    if (ch == 4) GH_RAD(false, 4); else if (ch == 3) GH_RAD(false, 3); else GH_RAD(false, 2);
  }
#undef GH_RAD
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_angular_deriv(gh_domain* d, const double* in) {
  return launch_angular_deriv_into(d, in, d->d_th, d->d_ph);
}

cudaError_t launch_derivatives(gh_domain* d, const double* in) {
  if (!d->overlap) {
    cudaError_t e = launch_radial(d, in, d->d_r, false);
    return e != cudaSuccess ? e : launch_angular_deriv(d, in);
  }
  // radial map on the side stream, angular maps on the domain's stream; the
  // join makes everything enqueued after this call wait for both
  cudaError_t e = cudaEventRecord(d->ev_fork, d->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(d->side, d->ev_fork, 0);
  if (e == cudaSuccess) e = launch_radial_on(d, in, d->d_r, false, d->side);
  if (e == cudaSuccess) e = launch_angular_deriv(d, in);
  if (e == cudaSuccess) e = cudaEventRecord(d->ev_join, d->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(d->stream, d->ev_join, 0);
  return e;
}

cudaError_t launch_angular_deriv_into(gh_domain* d, const double* in, double* dth, double* dph) {
  if (d->algorithm == 2) return launch_fold_deriv(d, in, dth, dph);
  if (d->algorithm == 1)
    sep_angular_kernel<true><<<d->sd_blocks, SEP_THREADS, d->sd_smem, d->stream>>>(
        d->shells_d, d->n_shells, d->sd_block_begin_d, in, dth, dph);
  else
    gemm_batched_kernel<<<d->ang_deriv_tiles, GEMM_THREADS, 0, d->stream>>>(
        d->ang_deriv_d, d->ang_deriv_np, in, dth, dph);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_pointwise_rhs_from(gh_domain* d, const double* u, const double* dr, const double* dth,
                                      const double* dph, double* k) {
  PointwiseArgs a;
  a.shells = d->shells_d; a.n_shells = d->n_shells; a.begin = d->pt_block_begin_d;
  a.u = u; a.dr = dr; a.dth = dth; a.dph = dph;
  a.k = k; a.u0 = nullptr; a.acc = nullptr; a.us = nullptr;
  a.partial = nullptr; a.c_out = nullptr;
  a.gamma0 = d->params.gamma0; a.gamma1 = d->params.gamma1; a.gamma2 = d->params.gamma2;
  a.dt = 0.0; a.stage = 0;
  a.fr = d->fr;
  a.frd = d->fr.on ? d->frd : nullptr;
  if (a.fr.on)
    pointwise_kernel<true, false, true><<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(a);
  else
    pointwise_kernel<true, false, false><<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(a);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_angular_filter(gh_domain* d, const double* in, double* out) {
  if (d->algorithm == 2) return launch_fold_filter(d, in, out);
  if (d->algorithm == 1)
    sep_angular_kernel<false><<<d->sf_blocks, SEP_THREADS, d->sf_smem, d->stream>>>(
        d->shells_d, d->n_shells, d->sf_block_begin_d, in, out, nullptr);
  else
    gemm_batched_kernel<<<d->ang_filt_tiles, GEMM_THREADS, 0, d->stream>>>(
        d->ang_filt_d, d->ang_filt_np, in, out, nullptr);   // filter problems write out0 only
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_pointwise(gh_domain* d, const double* u, double* k, int stage, double dt,
                             const double* u0, double* acc, double* ustage, bool constraints) {
  PointwiseArgs a;
  a.shells = d->shells_d; a.n_shells = d->n_shells; a.begin = d->pt_block_begin_d;
  a.u = u; a.dr = d->d_r; a.dth = d->d_th; a.dph = d->d_ph;
  a.k = k; a.u0 = u0; a.acc = acc; a.us = ustage;
  a.partial = d->partial; a.c_out = nullptr;
  a.gamma0 = d->params.gamma0; a.gamma1 = d->params.gamma1; a.gamma2 = d->params.gamma2;
  a.dt = dt; a.stage = stage;
  a.fr = d->fr;
  a.frd = d->fr.on ? d->frd : nullptr;
  if (a.fr.on) {
    if (constraints)
      pointwise_kernel<true, true, true><<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(a);
    else
      pointwise_kernel<true, false, true><<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(a);
  } else {
    if (constraints)
      pointwise_kernel<true, true, false><<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(a);
    else
      pointwise_kernel<true, false, false><<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(a);
  }
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_constraints(gh_domain* d, const double* u, double* c_out) {
  PointwiseArgs a;
  a.shells = d->shells_d; a.n_shells = d->n_shells; a.begin = d->pt_block_begin_d;
  a.u = u; a.dr = d->d_r; a.dth = d->d_th; a.dph = d->d_ph;
  a.k = nullptr; a.u0 = nullptr; a.acc = nullptr; a.us = nullptr;
  a.partial = d->partial; a.c_out = c_out;
  a.gamma0 = d->params.gamma0; a.gamma1 = d->params.gamma1; a.gamma2 = d->params.gamma2;
  a.dt = 0.0; a.stage = 0;
  a.fr = d->fr;
  a.frd = d->fr.on ? d->frd : nullptr;
  if (a.fr.on)
    pointwise_kernel<false, true, true><<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(a);
  else
    pointwise_kernel<false, true, false><<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(a);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_norm_reduce(gh_domain* d, double* norm2) {
  norm_reduce_kernel<<<d->n_shells, 256, 0, d->stream>>>(d->pt_block_begin_d, d->n_shells,
                                                          d->partial, norm2, d->err_flag);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_bc(gh_domain* d, double* k, int stage, double dt, const double* u0, double* acc,
                      double* ustage, const double* u_in, const double* const* deriv) {
  if (d->bc_points == 0) return cudaSuccess;
  BcArgs a;
  a.slices = d->bc_d; a.n_slices = (int)d->bc_h.size(); a.pt_begin = d->bc_pt_begin_d;
  a.k = k; a.u0 = u0; a.acc = acc; a.us = ustage;
  a.gamma1 = d->params.gamma1; a.gamma2 = d->params.gamma2; a.dt = dt; a.stage = stage;
  a.cp_outer = d->outer_bc;
  a.shells = d->shells_d;
  a.u_in = u_in;
  a.dr = deriv ? deriv[0] : d->d_r;
  a.dth = deriv ? deriv[1] : d->d_th;
  a.dph = deriv ? deriv[2] : d->d_ph;
  a.fr = d->fr;
  a.frd = d->fr.on ? d->frd : nullptr;
  a.cpm_S = d->cpm_S;
  if (a.cp_outer && !u_in) return cudaErrorInvalidValue;
  if (a.cp_outer == 2) {
    if (!d->cpm_S || d->fr.on) return cudaErrorInvalidValue;
    cp_minus_kernel<<<cdiv(d->bc_points, 3 * CPM_WARPS), 32 * CPM_WARPS, 0, d->stream>>>(a, d->cpm_S);
    d->launches++;
  }
  bc_kernel<<<cdiv(10LL * d->bc_points, 128), 128, 0, d->stream>>>(a);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_bc_background(gh_domain* d, const double* u, int bh) {
  if (d->bc_points == 0) return cudaSuccess;
  bc_background_kernel<<<cdiv(d->bc_points, 128), 128, 0, d->stream>>>(
      d->shells_d, d->bc_d, (int)d->bc_h.size(), d->bc_pt_begin_d, u, bh);
  d->launches++;
  return cudaGetLastError();
}

// The rotating frame at n times clock + off[i] (Rodrigues, as on the host),
// then clock += advance; one thread.  Kernels of the same step read the
// frames, never the clock, so captured graphs replay with the live clock.
__global__ void frame_kernel(double* clock, double e0, double e1, double e2, double omega, int gen, double adot,
                             double V0, double V1, double V2, FrameOffsets fo, double advance, Frame* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double t0 = *clock;
  const double K[9] = {0.0, -e2, e1, e2, 0.0, -e0, -e1, e0, 0.0};
  for (int i = 0; i < fo.n; ++i) {
    const double th = omega * (t0 + fo.off[i]);
    double sn, c;
    sincos(th, &sn, &c);
    Frame f;
    f.on = 1;
    for (int r = 0; r < 3; ++r)
      for (int col = 0; col < 3; ++col) {
        double k2 = 0.0;
        for (int m = 0; m < 3; ++m) k2 += K[3 * r + m] * K[3 * m + col];
        f.R[3 * r + col] = (r == col ? 1.0 : 0.0) + sn * K[3 * r + col] + (1.0 - c) * k2;
      }
    f.w[0] = omega * e0;
    f.w[1] = omega * e1;
    f.w[2] = omega * e2;
    const double tt = t0 + fo.off[i];
    f.gen = gen;
    f.a = gen ? fma(adot, tt, 1.0) : 1.0;
    f.adot = gen ? adot : 0.0;
    f.V[0] = gen ? V0 : 0.0;
    f.V[1] = gen ? V1 : 0.0;
    f.V[2] = gen ? V2 : 0.0;
    for (int c = 0; c < 3; ++c) f.T[c] = f.V[c] * tt;
    out[i] = f;
  }
  if (advance != 0.0) *clock = t0 + advance;
}

cudaError_t launch_frames(gh_domain* d, const double* off, int n, double advance) {
  if (!frame_moving(d) || !d->clock_d) return cudaSuccess;
  if (n < 0 || n > 8) return cudaErrorInvalidValue;
  FrameOffsets fo;
  fo.n = n;
  for (int i = 0; i < 8; ++i) fo.off[i] = i < n ? off[i] : 0.0;
  const double nrm = std::sqrt(d->rot_axis[0] * d->rot_axis[0] + d->rot_axis[1] * d->rot_axis[1] +
                               d->rot_axis[2] * d->rot_axis[2]);
  frame_kernel<<<1, 32, 0, d->stream>>>(d->clock_d, d->rot_axis[0] / nrm, d->rot_axis[1] / nrm,
                                        d->rot_axis[2] / nrm, d->rot_omega, d->map_gen ? 1 : 0, d->map_adot,
                                        d->map_V[0], d->map_V[1], d->map_V[2], fo, advance, d->frames_d);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_cartesian(gh_domain* d, const double* u, double* du) {
  (void)u;
  cartesian_kernel<<<d->pt_blocks, PT_THREADS, 0, d->stream>>>(
      d->shells_d, d->n_shells, d->pt_block_begin_d, d->d_r, d->d_th, d->d_ph, du, d->state, d->fr, d->frd);
  d->launches++;
  return cudaGetLastError();
}

}  // namespace gh
