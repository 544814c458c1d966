// Internal declarations shared by the libgh translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/gh.h"

namespace gh {

constexpr int NF = 50;      // evolved fields per point
constexpr int NC = 64;      // stored constraint components per point
constexpr int NGAUGE = 16;  // H_a (4) + d_i H_a (12) per point
constexpr int NBG = 16;     // boundary background per point: n_i, n^i, alpha, beta^i, g_ij (packed xx..zz)
constexpr int DP_MAX_BLOCKS = 1024;  // blocks of the Dormand-Prince elementwise kernels
// Dual frame at one instant (Sec. 3.1 dual frame): inertial position
// x = a R x_grid + T, grid velocity xdot = w x (x - T) + (adot / a)(x - T) + V.
// on = 0: static grid.  gen = 0: the rotation alone (a = 1, T = V = 0), with
// the gauge source and boundary background rotated from their stored values;
// gen = 1: the general map, with both evaluated at the moving points for the
// frame (map_stage kernels) and the speeds taken relative to the moving
// boundary.
struct Frame {
  int on;
  int gen;
  double R[9];
  double w[3];
  double a, adot;
  double T[3], V[3];
};
static_assert(sizeof(Frame) % 8 == 0, "frames are compared as 64-bit words");
// The frame the general map's moving-point buffers (gauge_t, bg_t) were last
// evaluated at (valid = 0: never, or the holes or the map changed since), and
// whether the stage being issued may reuse them (skip).
struct MapGate {
  Frame last;
  int valid;
  int skip;
};
// Stage times of one step relative to the domain clock (frame_kernel).
struct FrameOffsets {
  double off[8];
  int n;
};
// Linear combination of up to seven stage derivatives (passed by value).
struct LinComb {
  const double* k[7];
  double c[7];
  int nk;
};
#ifndef GH_PT_THREADS
#define GH_PT_THREADS 32
#endif
constexpr int PT_THREADS = GH_PT_THREADS;  // threads per block of the per-point kernels
constexpr int RAD_THREADS_HOST = 128;      // threads per block of the radial kernel
#ifndef GH_ADJ_PT_THREADS
#define GH_ADJ_PT_THREADS 32
#endif
constexpr int ADJ_PT_THREADS = GH_ADJ_PT_THREADS;  // threads per block of the pointwise reverse kernel

// Separable spherical-harmonic map of one shell (Y_lm = Pbar_lm(theta) x
// Fourier(phi)): phi-DFT, one N_theta x N_theta Legendre map per Fourier mode,
// inverse DFT.  Modes: cos m = 0..K, then sin m = 1..K (M = 2K + 1).
struct SepPlan {
  int K, M;                     // highest m kept, number of Fourier modes
  int rows_per_cta, pad;
  const double* F;              // [nph][M]  forward DFT  cos(m phi_k) / sin(m phi_k)
  const double* G0;             // [M][nph]  synthesis of output 0
  const double* G1;             // [M][nph]  synthesis of output 1 (derivative plan: d/dphi)
  const double* Q0;             // [K+1][nth_in][nth_out] Legendre map for output 0
  const double* Q1;             // [K+1][nth_in][nth_out] Legendre map for output 1
};

// Transposed separable map (for the adjoint): analysis with the transposed
// synthesis matrices, Legendre maps with theta_in/theta_out swapped, synthesis
// with the transposed DFT.  Two inputs (the d/dtheta and d/dphi cotangents)
// for the derivative plan, one for the filter.
struct SepAdjPlan {
  int K, M;
  int rows_per_cta, pad;
  const double* F0T;            // [nph][M]
  const double* F1T;            // [nph][M]  (derivative plan only)
  const double* Q0T;            // [K+1][nth][nth]
  const double* Q1T;            // [K+1][nth][nth]  (derivative plan only)
  const double* GT;             // [M][nph]
};

// Symmetry-folded separable map (fold_angular_kernel): the phi DFT and its
// inverse use the k <-> N-k and k <-> N/2-k symmetries of cos/sin (a quarter of
// the dense DFT work), the Legendre maps the equatorial parity of Pbar_lm
// (half-size matrices on the symmetric and antisymmetric parts).  Needs
// N_phi % 4 == 0 and N_theta even (odd L).
struct FoldPlan {
  int K, M, N4, half;           // highest m, 2K+1 modes, floor(N_phi/4), floor(N_theta/2)
  int W, hs;                    // quarter-ring points, symmetric half-ring size ceil(N_theta/2)
  int qself;                    // 1 if N_phi % 4 == 0 (the point N_phi/4 is its own mirror)
  int rows_per_cta, two;        // rows per block; 2 outputs (derivatives) or 1 (filter)
  int adj_rows_per_cta;         // rows per block of the transposed map (fold_adjoint_kernel)
  int fft_log;                  // log2(N_phi / 2) where each ring's phi transforms run as a real FFT
                                // in registers (N_phi = 16, 32, 64), else 0 (quarter-folded DFT)
  const double* Tc;             // [K+1][W] cos(m phi_k)
  const double* Ts;             // [K+1][W] sin(m phi_k)
  // [K+1][hs][hs] (transposed: [m][j_in][j_out]) half-size Legendre maps,
  // symmetric (s) and antisymmetric (t) parts, scaled by the synthesis factor
  // of mode m: c_m = (m ? 2 : 1) 2 pi / N_phi for output 0, m c_m for output 1
  const double* Q0s;
  const double* Q0t;
  const double* Q1s;            // output 1 (value map feeding d/dphi; derivative plan only)
  const double* Q1t;
  double sigma0, sigma1;        // parity of output 0 / 1 (-1 for d/dtheta, +1 for values)
  // Modes m >= m0 take the Legendre map as analysis then synthesis (its rank
  // K + 1 - m is below the half-ring size there): per m, slots off[m] ..
  // off[m + 1] - 1 hold l = m .. K (parity of l + m alternating, s part first);
  // A [slots][hs] = Pbar_lm(theta_j) w_j, Y0 / Y1 [slots][hs] the synthesis of
  // output 0 / 1 with the factors of Q0 / Q1; slot_m[slot] = m.
  int m0, ncoef;                // ncoef = off[K + 1] (cos modes; sin modes use a second bank)
  const int* coef_off;          // [K + 2]
  const int* slot_m;            // [ncoef]
  const double* A;
  const double* Y0;
  const double* Y1;
};

// Tensor spherical-harmonic filter of one shell (tensor_filter kernels).  The
// spin-s projection onto sY_lm, |s| <= l <= K, of a complex function: a phi
// DFT per ring, then per (s, m) the analysis onto the n_b = K - max(|m|,|s|) + 1
// orthonormal theta functions and the synthesis back.
struct TensorFilterPlan {
  int K;                        // keep l <= K (-1: off)
  int W;                        // phi slots of the quarter fold: N_phi / 4 + 1 (k = 0 .. W-1)
  const double* twc;            // [K+1][W] cos(m phi_k)
  const double* tws;            // [K+1][W] sin(m phi_k)
  const double* An;             // per (s, m): [N_theta][n_b] analysis, 2 pi w_i b_n(theta_i)
  const double* Sy;             // per (s, m): [n_b][N_theta] synthesis, b_n(theta_j)
  const int* coff;              // [7 spins][2K+1 modes] offset of the (s, m) block in An and Sy
  const int* cidx;              // [7][2K+1] first coefficient of (s, m) in its spin's packed list
  const int* ist;               // [8] start of each spin's packed (m + K) << 8 | n items
  const int* items;
};
constexpr int TF_ROWS = 31;     // independent complex frame components per point (9 tensor groups)

// One shell as the kernels see it (device-resident array of these).
struct ShellDev {
  int n_r, L, nth, nph, na;     // na = nth * nph angular points
  int pad0;
  long long off;                // offset of the shell in a state vector (doubles)
  long long pt_off;             // offset of the shell's first point
  double r_in, r_out, rscale;   // rscale = 2 / (r_out - r_in) = dx/dr
  const double* Dr;             // d/dx on the CGL points, folded rows [ceil(n_r/2)][n_r] (radial_kernel)
  const double* Fr;             // exponential Chebyshev filter, folded rows [ceil(n_r/2)][n_r]
  const double* Bth;            // [na][na] transposed d/dtheta map (out = U * Bth)
  const double* Bph;            // [na][na] transposed d/dphi map
  const double* Sf;             // [na][na] transposed SH truncation filter (or null)
  const double* r;              // [n_r]
  const double* wr;             // [n_r] radial volume weight w_cc * (r_out-r_in)/2 * r^2
  const double* cth;            // [nth] cos(theta)
  const double* sth;            // [nth] sin(theta)
  const double* wth;            // [nth] Gauss-Legendre weight * 2 pi / nph
  const double* cph;            // [nph]
  const double* sph;            // [nph]
  double* gauge;                // [n_r][16][na]
  double* gauge_t;              // [n_r][16][na] at the moving points of the current frame (general map)
  int bc_inner;                 // boundary slice index at r_in, -1 if none (excision)
  int bc_outer;                 // boundary slice index at r_out
  int bh;                       // black hole this shell belongs to
  int keep;                     // SH filter: keep l <= keep (-1: no filter)
  double dt_scale;              // this hole's step = dt * dt_scale
  SepPlan sd;                   // separable d/dtheta, d/dphi
  SepPlan sf;                   // separable SH truncation filter (M = 0 if off)
  SepAdjPlan sda;               // transpose of sd
  SepAdjPlan sfa;               // transpose of sf (M = 0 if off)
  FoldPlan fd;                  // folded d/dtheta, d/dphi (M = 0 if not applicable)
  FoldPlan ff;                  // folded SH filter
  TensorFilterPlan tf;          // tensor-harmonic SH filter (used when selected)
  const double* DrT;            // transpose of d/dx, folded rows [ceil(n_r/2)][n_r] (reverse mode)
  const double* FrT;            // transpose of the filter, folded rows
};

// A boundary slice: the outer boundary of the last shell (kind 0) or an
// internal boundary shared by shell a (its r_out) and shell b (its r_in).
struct BcSliceDev {
  int kind;                     // 0 outer, 1 interface
  int shell_a, shell_b;         // shell_b = -1 for the outer boundary
  int na;
  long long off_a, off_b;       // state offset of the boundary r-slice in a / b
  double* bg;                   // [16][na] n_dn(3) n_up(3) alpha beta_up(3) g_ij(6: xx xy xz yy yz zz)
  double* bg_t;                 // [11][na] the same at the moving points, then n . xdot (general map)
  double dt_scale;              // the hole's step scale (see ShellDev)
  int bh, pad;
};

// One FP64 GEMM problem of a batched launch: C = A * B, row-major.
// A is addressed from one of the input bases, C from one of the output bases.
struct GemmProb {
  long long a_off, c_off;
  const double* B;
  int M, N, K;
  int lda, ldb, ldc;
  int tiles_n;                  // ceil(N / BN)
  int tile_begin;               // first flattened tile index of this problem
  int c_sel;                    // which output base
  int pad;
};

struct MatrixCacheEntry;

}  // namespace gh

struct gh_domain {
  int n_shells = 0;
  gh_params params{};
  cudaStream_t stream = nullptr;
  int device = 0;
  long long state = 0, points = 0;
  std::vector<gh::ShellDev> shells_h;
  gh::ShellDev* shells_d = nullptr;
  std::vector<gh::BcSliceDev> bc_h;
  gh::BcSliceDev* bc_d = nullptr;
  int bc_points = 0;            // total points over all boundary slices
  int* bc_pt_begin_d = nullptr; // first point of each boundary slice, [n + 1]
  // batched GEMM launch plans
  gh::GemmProb* ang_deriv_d = nullptr; int ang_deriv_np = 0, ang_deriv_tiles = 0;
  gh::GemmProb* ang_filt_d = nullptr;  int ang_filt_np = 0, ang_filt_tiles = 0;
  // radial / pointwise launch maps: first block of each shell
  int* rad_block_begin_d = nullptr; int rad_blocks = 0; int max_n_r = 0;
  int* pt_block_begin_d = nullptr;  int pt_blocks = 0;
  // separable angular maps: first block of each shell, dynamic shared memory
  int algorithm = 1;            // 0 dense traced matrices, 1 separable
  int* sd_block_begin_d = nullptr; int sd_blocks = 0; size_t sd_smem = 0;
  int* fd_block_begin_d = nullptr; int fd_blocks = 0; size_t fd_smem = 0;
  int* ff_block_begin_d = nullptr; int ff_blocks = 0; size_t ff_smem = 0;
  // folded maps of the shells with ring FFTs (fft_log != 0), [0] derivatives,
  // [1] filter: block maps and shared memory of the analysis, Legendre and
  // synthesis launches, and the state-sized scratch between them
  struct FoldFftMap {
    int* an_begin_d = nullptr;  int an_blocks = 0;  size_t an_smem = 0;
    int* leg_begin_d = nullptr; int leg_blocks = 0; size_t leg_smem = 0;
    int* sy_begin_d = nullptr;  int sy_blocks = 0;  size_t sy_smem = 0;
  };
  FoldFftMap fxm[2];
  FoldFftMap fxa[2];            // the same for the transposed maps (reverse mode)
  double* fft_ab = nullptr;
  double* fft_c0 = nullptr;
  double* fft_c1 = nullptr;
  // transposed folded maps (reverse mode): launch maps and shared memory
  int* fda_block_begin_d = nullptr; int fda_blocks = 0; size_t fda_smem = 0;
  int* ffa_block_begin_d = nullptr; int ffa_blocks = 0; size_t ffa_smem = 0;
  // folded-map work schedule: threads per block and shared-memory budget per
  // block that sets the rows per block (chosen by gh_autotune, else defaults)
  int fd_threads = 256, ff_threads = 256;
  int fd_budget = 32 * 1024, ff_budget = 32 * 1024;
  // radial-map work schedule: FMA chains per pass (2..4) and row groups (1..4)
  int rad_chains = 2, rad_groups = 1, radf_chains = 2, radf_groups = 1;
  bool fold_ok = false;         // every shell has a folded plan
  int* sf_block_begin_d = nullptr; int sf_blocks = 0; size_t sf_smem = 0;
  // scratch owned by the domain
  double* d_r = nullptr;         // radial derivative  (one state)
  double* d_th = nullptr;        // theta derivative   (one state)
  double* d_ph = nullptr;        // phi derivative     (one state)
  double* partial = nullptr;     // per-block constraint partial sums
  int* err_flag = nullptr;       // latched device error
  std::vector<void*> owned;      // every device allocation, freed on destroy
  std::string err;
  long long launches = 0;
  // adjoint: separable transposed-map launch maps and a cotangent scratch state
  int* sda_block_begin_d = nullptr; int sda_blocks = 0; size_t sda_smem = 0;
  int* sfa_block_begin_d = nullptr; int sfa_blocks = 0; size_t sfa_smem = 0;
  double* kbt = nullptr;        // one state, allocated by the first adjoint call
  int* adj_pt_block_begin_d = nullptr; int adj_pt_blocks = 0;   // ADJ_PT_THREADS-point blocks
  double* pert_partial = nullptr; int pert_partial_len = 0;
  // Dormand-Prince step: per-block partial sums of the error norm and the norm
  double* dp_partial = nullptr;
  // pointwise reverse pass: ten threads per point (one per symmetric pair) on
  // small grids, partial field cotangents in adj_ubp (10 states, lazily)
  bool adj_pair_split = false;
  double* adj_ubp = nullptr;
  double* clock_d = nullptr;    // rotating frame: the domain clock on the device
  gh::Frame* frames_d = nullptr; // [8] frames of the current step's stage times
  const gh::Frame* frd = nullptr; // frame of the launches being issued (device)
  double graph_dt = 0.0;        // dt of the captured RK4 step
  double* adj_cpbar = nullptr;  // reverse mode, constraint-preserving outer condition: [10][bc points][4]
  // reverse mode of the u^- constraint part (outer_bc 2): the interior right-hand
  // side (one state), the cotangent of the condition's u^- derivative [10][bc points]
  // and the stashed field and derivative cotangents [200][bc points]
  double* adj_kraw = nullptr;
  double* adj_cpm_Sb = nullptr;
  double* adj_cpm_stash = nullptr;
  // SH filter mode (gh_set_sh_filter): 0 per Cartesian component, 1 tensor
  // harmonics; complex frame components [shell][r][TF_ROWS][na][2]
  int sh_filter_mode = 0;
  double* tf_buf = nullptr;
  int* tf_pb_d = nullptr;       // tensor-filter launch maps: point blocks, then rows
  int tf_point_blocks = 0, tf_rows = 0, tf_spin_threads = 128;
  size_t tf_smem = 0;
  // rotating dual frame (gh_set_rotating_frame): axis, rate, the domain's
  // time, and the frame of the launches being issued
  double rot_axis[3] = {0.0, 0.0, 1.0};
  double rot_omega = 0.0;
  // general map (gh_set_frame_map): expansion rate, translation velocity, and
  // each hole's mass and spin vector a = chi M (recorded by
  // gh_set_analytic_kerr_schild*), which the map evaluates at moving points
  bool map_gen = false;
  double map_adot = 0.0;
  double map_V[3] = {0.0, 0.0, 0.0};
  std::vector<double> holes;    // [bh][4]: M, a_x, a_y, a_z (M = 0: not set)
  double* holes_d = nullptr;
  double* map_buf = nullptr;    // gauge_t of every shell, then bg_t of every slice
  int* map_pt_begin_d = nullptr; int map_blocks = 0;   // 64-point block map of map_gauge_kernel
  gh::MapGate* map_gate_d = nullptr;   // reuse of the moving-point buffers between stages at one time
  double time = 0.0;
  gh::Frame fr = {0, 0, {1, 0, 0, 0, 1, 0, 0, 0, 1}, {0, 0, 0}, 1.0, 0.0, {0, 0, 0}, {0, 0, 0}};
  // outer boundary condition: 0 freezing, 1 constraint preserving for u^psi and u^0,
  // 2 also the constraint part of u^- (gh_set_outer_bc)
  int outer_bc = 0;
  double* cpm_S = nullptr;      // mode 2: d_t u^- per (pair, boundary point), [10][bc_points]
  double* dp_err = nullptr;
  // CUDA graph of one RK4 step (gh_rk4_graph_capture / _launch)
  cudaGraphExec_t graph_exec = nullptr;
  long long graph_step_launches = 0;
  // gh_rk4_step_host's own captured step on host_u / host_work (dt and whether
  // it writes the norms), rebuilt when a setter changes the step's launches
  cudaGraphExec_t host_graph = nullptr;
  double host_graph_dt = 0.0;
  int host_graph_norm = 0;
  long long host_graph_launches = 0;
  // its one-step form that reads and writes the caller's pinned buffers from
  // the step's kernels (also keyed by those buffers' device addresses)
  cudaGraphExec_t host_graph_io = nullptr;
  double host_graph_io_dt = 0.0;
  int host_graph_io_norm = 0;
  const double* host_graph_io_in = nullptr;
  double* host_graph_io_out = nullptr;
  long long host_graph_io_launches = 0;
  // device state, RK4 work area and norms of gh_rk4_step_host (allocated on first use)
  double* host_u = nullptr;
  double* host_work = nullptr;
  double* host_norm = nullptr;
  // second stream for the radial map, which runs beside the angular maps of
  // the same right-hand side (both read the state, neither reads the other's
  // output); fork and join by events on the domain's stream (gh_set_overlap)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool overlap = true;
  // profiler (gh_profile_enable / gh_profile_read)
  bool prof = false;
  struct Bracket { int fam; cudaEvent_t a, b; };
  std::vector<Bracket> pending;
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[GH_K_FAMILIES] = {0};
  long long prof_n[GH_K_FAMILIES] = {0};
};

namespace gh {

// Kernel launchers (gh_kernels.cu).
cudaError_t launch_radial(gh_domain* d, const double* in, double* out, bool filter);
// copy != NULL: the input is also written to copy (one row group reads it: the
// input may be pinned host memory, the copy its device image).
cudaError_t launch_radial_on(gh_domain* d, const double* in, double* out, bool filter, cudaStream_t st,
                             double* copy = nullptr);
// radial and angular derivative maps of in into d_r, d_th, d_ph: side by side
// on two streams when d->overlap, else one after the other
cudaError_t launch_derivatives(gh_domain* d, const double* in);
cudaError_t launch_angular_deriv(gh_domain* d, const double* in);
cudaError_t launch_angular_filter(gh_domain* d, const double* in, double* out);
cudaError_t launch_angular_deriv_into(gh_domain* d, const double* in, double* dth, double* dph);
cudaError_t sep_set_smem_limits(size_t bytes);
cudaError_t radial_set_smem_limits();
cudaError_t fold_set_smem_limits(size_t bytes);
// Uploads the twiddle table of the folded maps' ring FFTs (constant memory of
// the current device; the same values on every call).
cudaError_t fold_fft_tables();
// Warps (of 32 rings each) per block of the ring-FFT kernels.
constexpr int FOLD_FFT_WARPS = 4;
cudaError_t fold_fft_set_smem_limits(size_t an_bytes, size_t leg_bytes, size_t sy_bytes);
cudaError_t fold_fft_adj_set_smem_limits(size_t an_bytes, size_t leg_bytes, size_t sy_bytes);
// Tensor-harmonic SH filter: tables, launch maps and the component buffer
// (once; gl_x / gl_w are each shell's Gauss-Legendre nodes cos(theta) and
// weights), then in -> out (may alias) using d->tf_buf.
cudaError_t tensor_filter_prepare(gh_domain* d, const std::vector<std::vector<double>>& gl_x,
                                  const std::vector<std::vector<double>>& gl_w);
cudaError_t launch_tensor_filter(gh_domain* d, const double* in, double* out);
// Its transpose (reverse mode): out = S^T in (in and out distinct).
cudaError_t launch_tensor_filter_transpose(gh_domain* d, const double* in, double* out);
// The frame at the device clock + off[i] into frames_d[i], i < n, then the
// clock advances by `advance` (no-op on a static grid).
cudaError_t launch_frames(gh_domain* d, const double* off, int n, double advance);
// True when the grid moves (a rotating frame or a general map).
inline bool frame_moving(const gh_domain* d) { return d->rot_omega != 0.0 || d->map_gen; }
// General map: the gauge source of every point and the boundary background of
// every boundary point at the moving positions of the frame d->frd, unless
// the buffers already hold that frame's (the last stage of one RK4 step and
// the first of the next share a time).
cudaError_t launch_map_stage(gh_domain* d);
// The rotating frame of the domain at time t (identity when not rotating).
Frame frame_at(const gh_domain* d, double t);
// Dormand-Prince step: out = base + sum_j c[j] k[j] (j < nk), and the scaled
// RMS norm of sum_j c[j] k[j] (the embedded error estimate) into err_dev.
cudaError_t launch_dp5_lincomb(gh_domain* d, const double* base, const LinComb& lc, double* out);
cudaError_t launch_dp5_error(gh_domain* d, const double* u, const double* unew, const LinComb& lc, double rtol,
                             double atol, double* err_dev);
// Raise the dynamic shared-memory limit of kernel f on the current device to
// at least `bytes`.  The limit is an attribute of the kernel on that device
// which every domain there shares, so it only ever grows (tracked per kernel
// and device, guarded by a mutex).
cudaError_t raise_smem_limit(const void* f, size_t bytes);
// Host-side fault injection (GH_FAULT=launch): GH_ECUDA before any launch.
gh_status check_latched(gh_domain* d);
cudaError_t launch_fold_deriv(gh_domain* d, const double* in, double* dth, double* dph);
// Transposed folded maps (reverse mode): two: out += Theta^T in0 + Phi^T in1;
// else out = S^T in0 (the SH filter).  Launch maps from fold_build_maps.
#ifndef GH_FOLD_ADJ_THREADS
#define GH_FOLD_ADJ_THREADS 256
#endif
// 256 threads and 48 KiB: the fastest of 128-512 threads and 16-112 KiB on the
// 4-shell (N_r = 21, L = 15) step VJP.
#ifndef GH_FOLD_ADJ_BUDGET
#define GH_FOLD_ADJ_BUDGET (48 * 1024)
#endif
constexpr int FOLD_ADJ_THREADS = GH_FOLD_ADJ_THREADS;
constexpr int FOLD_ADJ_BUDGET = GH_FOLD_ADJ_BUDGET;   // shared-memory budget per block (bytes)
size_t fold_adjoint_row_doubles(int na, int nth, int W, int M, int n_out, bool fft);
cudaError_t fold_adjoint_set_smem_limits(size_t bytes);
cudaError_t launch_fold_adjoint(gh_domain* d, bool two, const double* in0, const double* in1, double* out);
cudaError_t launch_fold_filter(gh_domain* d, const double* in, double* out);
cudaError_t sep_adj_set_smem_limits(size_t bytes);
cudaError_t launch_pointwise_rhs_from(gh_domain* d, const double* u, const double* dr, const double* dth,
                                      const double* dph, double* k);
cudaError_t launch_pointwise(gh_domain* d, const double* u, double* k, int stage, double dt,
                             const double* u0, double* acc, double* ustage, bool constraints);
// Boundary conditions on k = dudt (RK4 combine of boundary points for stage
// >= 1).  u_in: the state the RHS was evaluated at, and deriv[3] its
// spherical-basis derivatives (null: the domain's scratch); both used by the
// constraint-preserving outer condition only.
cudaError_t launch_bc(gh_domain* d, double* k, int stage, double dt, const double* u0, double* acc,
                      double* ustage, const double* u_in = nullptr, const double* const* deriv = nullptr);
cudaError_t launch_constraints(gh_domain* d, const double* u, double* c_out);
cudaError_t launch_norm_reduce(gh_domain* d, double* norm2);
cudaError_t launch_cartesian(gh_domain* d, const double* u, double* du);
cudaError_t launch_bc_background(gh_domain* d, const double* u, int bh);
cudaError_t launch_kerr_schild(gh_domain* d, int bh, double M, const double chi[3], double* u);
cudaError_t launch_perturbation(gh_domain* d, int kind, double A, double Rc, double w,
                                int lmax, const double* coeffs_dev, double* u);

}  // namespace gh
