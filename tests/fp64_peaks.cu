// Throughput microbenchmarks behind the choice of FP64 pipe for the spectral
// contractions: plain FP64 FMA against the FP64 tensor-core shapes that
// mma.sync offers (m8n8k4, m16n8k4, m16n8k8, m16n8k16) and, for scale, the
// BF16 m16n8k16 shape.  Every warp runs independent accumulator chains in a
// loop; each thread writes one value at the end so that nothing is dead code.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_peaks tests/fp64_peaks.cu
//   ./fp64_peaks            prints one JSON line per kernel
//
// Grid: blocks x 256 threads with blocks = SMs x 8; the output buffer holds one
// double per thread of the grid, the only memory any kernel touches.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#define CK(x)                                                                         \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess) {                                                          \
      std::fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                   \
      std::exit(1);                                                                   \
    }                                                                                 \
  } while (0)

constexpr int THREADS = 256;
constexpr int CHAINS = 8;

__global__ void ffma_kernel(double* out, int iters, double b, double c) {
  double a[CHAINS];
  for (int i = 0; i < CHAINS; ++i) a[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], b, c);
  double s = 0.0;
  for (int i = 0; i < CHAINS; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dmma_m8n8k4_kernel(double* out, int iters, double x) {
  double acc[4][2];
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = 0.0;
  const double a = x + threadIdx.x, b = x - threadIdx.x;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(acc[i][0]), "+d"(acc[i][1])
                   : "d"(a), "d"(b));
  double s = 0.0;
  for (int i = 0; i < 4; ++i) s += acc[i][0] + acc[i][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dmma_m16n8k4_kernel(double* out, int iters, double x) {
  double acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const double a0 = x + threadIdx.x, a1 = x * 0.5, b = x - threadIdx.x;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
                   : "+d"(acc[i][0]), "+d"(acc[i][1]), "+d"(acc[i][2]), "+d"(acc[i][3])
                   : "d"(a0), "d"(a1), "d"(b));
  double s = 0.0;
  for (int i = 0; i < 4; ++i) s += acc[i][0] + acc[i][1] + acc[i][2] + acc[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dmma_m16n8k8_kernel(double* out, int iters, double x) {
  double acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const double a0 = x + threadIdx.x, a1 = x * 0.5, a2 = x * 0.25, a3 = x * 0.125;
  const double b0 = x - threadIdx.x, b1 = x * 2.0;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+d"(acc[i][0]), "+d"(acc[i][1]), "+d"(acc[i][2]), "+d"(acc[i][3])
          : "d"(a0), "d"(a1), "d"(a2), "d"(a3), "d"(b0), "d"(b1));
  double s = 0.0;
  for (int i = 0; i < 4; ++i) s += acc[i][0] + acc[i][1] + acc[i][2] + acc[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dmma_m16n8k16_kernel(double* out, int iters, double x) {
  double acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  double a[8], b[4];
  for (int i = 0; i < 8; ++i) a[i] = x + i + threadIdx.x;
  for (int i = 0; i < 4; ++i) b[i] = x - i;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7,%8,%9,%10,%11}, "
          "{%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
          : "+d"(acc[i][0]), "+d"(acc[i][1]), "+d"(acc[i][2]), "+d"(acc[i][3])
          : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]), "d"(b[0]),
            "d"(b[1]), "d"(b[2]), "d"(b[3]));
  double s = 0.0;
  for (int i = 0; i < 4; ++i) s += acc[i][0] + acc[i][1] + acc[i][2] + acc[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void hmma_bf16_m16n8k16_kernel(double* out, int iters, float x) {
  float acc[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
  unsigned a[4], b[2];
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat162 v = __floats2bfloat162_rn(x + i, x - threadIdx.x);
    a[i] = *reinterpret_cast<unsigned*>(&v);
  }
  for (int i = 0; i < 2; ++i) {
    __nv_bfloat162 v = __floats2bfloat162_rn(x * 0.5f + i, x);
    b[i] = *reinterpret_cast<unsigned*>(&v);
  }
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(acc[i][0]), "+f"(acc[i][1]), "+f"(acc[i][2]), "+f"(acc[i][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  float s = 0.0f;
  for (int i = 0; i < 4; ++i) s += acc[i][0] + acc[i][1] + acc[i][2] + acc[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// DMMA and DFMA in the same warps: 2 m16n8k8 mma.sync (4,096 flops per warp)
// and 32 DFMAs per thread (2,048 flops per warp) per loop iteration.  If the
// two share the FP64 units the combined rate stays near either alone; if
// they are separate pipes it approaches their sum.
__global__ void mixed_dmma_dfma_kernel(double* out, int iters, double x) {
  double acc[2][4];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const double a0 = x + threadIdx.x, a1 = x * 0.5, a2 = x * 0.25, a3 = x * 0.125;
  const double b0 = x - threadIdx.x, b1 = x * 2.0;
  double f[CHAINS];
  for (int i = 0; i < CHAINS; ++i) f[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+d"(acc[i][0]), "+d"(acc[i][1]), "+d"(acc[i][2]), "+d"(acc[i][3])
          : "d"(a0), "d"(a1), "d"(a2), "d"(a3), "d"(b0), "d"(b1));
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < CHAINS; ++i) f[i] = fma(f[i], 0.999999, 1e-7);
  }
  double s = 0.0;
  for (int i = 0; i < 2; ++i) s += acc[i][0] + acc[i][1] + acc[i][2] + acc[i][3];
  for (int i = 0; i < CHAINS; ++i) s += f[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename Launch>
void run(const char* name, double flops_per_warp_iter, int iters, int blocks, double* out, Launch launch) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  launch(iters / 10);                    // warm-up
  CK(cudaDeviceSynchronize());
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    CK(cudaEventRecord(a));
    launch(iters);
    CK(cudaEventRecord(b));
    CK(cudaEventSynchronize(b));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, a, b));
    if (ms < best) best = ms;
  }
  CK(cudaGetLastError());
  const double warps = (double)blocks * THREADS / 32.0;
  const double tflops = flops_per_warp_iter * warps * iters / (best * 1e-3) / 1e12;
  std::printf("{\"kernel\": \"%s\", \"tflops\": %.4f, \"ms\": %.3f, \"iters\": %d, \"blocks\": %d}\n", name, tflops,
              best, iters, blocks);
  CK(cudaEventDestroy(a));
  CK(cudaEventDestroy(b));
}

int main() {
  int dev = 0, sms = 0, clk = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
  const int blocks = sms * 8;
  double* out = nullptr;
  CK(cudaMalloc(&out, sizeof(double) * (size_t)blocks * THREADS));
  std::printf("{\"sms\": %d, \"clock_khz\": %d}\n", sms, clk);
  // flops per warp per loop iteration
  run("ffma_f64", 2.0 * CHAINS * 32, 20000, blocks, out,
      [&](int it) { ffma_kernel<<<blocks, THREADS>>>(out, it, 0.999999, 1e-7); });
  run("dmma_m8n8k4_f64", 4 * 2.0 * 8 * 8 * 4, 20000, blocks, out,
      [&](int it) { dmma_m8n8k4_kernel<<<blocks, THREADS>>>(out, it, 1e-3); });
  run("dmma_m16n8k4_f64", 4 * 2.0 * 16 * 8 * 4, 10000, blocks, out,
      [&](int it) { dmma_m16n8k4_kernel<<<blocks, THREADS>>>(out, it, 1e-3); });
  run("dmma_m16n8k8_f64", 4 * 2.0 * 16 * 8 * 8, 5000, blocks, out,
      [&](int it) { dmma_m16n8k8_kernel<<<blocks, THREADS>>>(out, it, 1e-3); });
  run("dmma_m16n8k16_f64", 4 * 2.0 * 16 * 8 * 16, 2500, blocks, out,
      [&](int it) { dmma_m16n8k16_kernel<<<blocks, THREADS>>>(out, it, 1e-3); });
  run("mixed_dmma_m16n8k8_and_dfma", 2 * 2.0 * 16 * 8 * 8 + 4 * CHAINS * 2.0 * 32, 5000, blocks, out,
      [&](int it) { mixed_dmma_dfma_kernel<<<blocks, THREADS>>>(out, it, 1e-3); });
  run("hmma_bf16_m16n8k16_f32acc", 4 * 2.0 * 16 * 8 * 16, 20000, blocks, out,
      [&](int it) { hmma_bf16_m16n8k16_kernel<<<blocks, THREADS>>>(out, it, 1e-3f); });
  CK(cudaFree(out));
  return 0;
}
