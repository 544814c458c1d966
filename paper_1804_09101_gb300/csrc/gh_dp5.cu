// Elementwise parts of the Dormand-Prince 5(4) step (the paper's time
// stepper, Sec. 2.1; pair of Dormand & Prince 1980): the stage states as
// linear combinations of the stage derivatives, and the scaled RMS norm of
// the embedded error estimate
//   err^2 = mean_i ( e_i / (atol + rtol max(|u_i|, |unew_i|)) )^2,
//   e = dt sum_j (b_j - bhat_j) k_j,
// reduced in a fixed order (per-block partial sums, then one block).  Both
// kernels stream whole states and are HBM/L2 bound; the right-hand sides
// between them are the usual radial, angular, pointwise and boundary kernels.
#include <cuda_runtime.h>

#include "gh_internal.h"

namespace gh {

constexpr int DP_THREADS = 256;

__global__ void __launch_bounds__(DP_THREADS)
dp5_lincomb_kernel(long long n, const double* __restrict__ base, LinComb lc, double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = base[i];
    for (int j = 0; j < lc.nk; ++j) acc = fma(lc.c[j], lc.k[j][i], acc);
    out[i] = acc;
  }
}

__global__ void __launch_bounds__(DP_THREADS)
dp5_error_kernel(long long n, const double* __restrict__ u, const double* __restrict__ unew, LinComb lc,
                 double rtol, double atol, double* __restrict__ partial) {
  __shared__ double red[DP_THREADS];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double e = 0.0;
    for (int j = 0; j < lc.nk; ++j) e = fma(lc.c[j], lc.k[j][i], e);
    const double sc = atol + rtol * fmax(fabs(u[i]), fabs(unew[i]));
    const double r = e / sc;
    s = fma(r, r, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = DP_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(DP_THREADS)
dp5_norm_kernel(const double* __restrict__ partial, int nparts, long long n, double* __restrict__ err) {
  __shared__ double red[DP_THREADS];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += DP_THREADS) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = DP_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) err[0] = sqrt(red[0] / (double)n);
}

static int dp_blocks(long long n) {
  const long long b = (n + DP_THREADS - 1) / DP_THREADS;
  return (int)(b < DP_MAX_BLOCKS ? b : DP_MAX_BLOCKS);
}

cudaError_t launch_dp5_lincomb(gh_domain* d, const double* base, const LinComb& lc, double* out) {
  dp5_lincomb_kernel<<<dp_blocks(d->state), DP_THREADS, 0, d->stream>>>(d->state, base, lc, out);
  d->launches++;
  return cudaGetLastError();
}

cudaError_t launch_dp5_error(gh_domain* d, const double* u, const double* unew, const LinComb& lc, double rtol,
                             double atol, double* err_dev) {
  const int nb = dp_blocks(d->state);
  dp5_error_kernel<<<nb, DP_THREADS, 0, d->stream>>>(d->state, u, unew, lc, rtol, atol, d->dp_partial);
  d->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dp5_norm_kernel<<<1, DP_THREADS, 0, d->stream>>>(d->dp_partial, nb, d->state, err_dev);
  d->launches++;
  return cudaGetLastError();
}

}  // namespace gh
