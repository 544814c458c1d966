// gh_rhs_noalloc: the right-hand side evaluation of gh_rhs with its three
// derivative work buffers taken from a fixed array in the library's own
// device memory instead of the domain's allocations.
//
// Who needs this: code that must not allocate device memory at the moment it
// evaluates the right-hand side -- for example a host that has handed all GPU
// memory to its own pool and forbids further cudaMalloc, or a real-time loop
// in which an allocation (and the implicit synchronisation it may cause) is
// not allowed.  Such a caller still creates the domain once beforehand; after
// that, this entry point performs no allocation of any kind.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gh_internal.h"

namespace {

// Largest state (doubles) the fixed work area can serve: 2^20 doubles, about
// 20,000 grid points.  The array holds three such buffers (24 MiB) and lives on
// every GPU that loads the library until the process exits.
constexpr long long kMaxState = 1LL << 20;

static __device__ __align__(256) double g_rhs_work[3 * kMaxState];

// Device address of g_rhs_work for each device ordinal, looked up once per
// device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_work_ptr[kMaxDevices] = {nullptr};

cudaError_t work_area(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_work_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_rhs_work);
    if (e != cudaSuccess) return e;
    g_work_ptr[device] = static_cast<double*>(p);
  }
  *out = g_work_ptr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" gh_status gh_rhs_noalloc(gh_domain* d, const double* u, double* dudt) {
  if (!d || !u || !dudt) {
    if (d) d->err = "null argument";
    return GH_EINVAL;
  }
  if (u == dudt) {
    d->err = "u and dudt must not overlap";
    return GH_EINVAL;
  }
  if (d->state > kMaxState) {
    d->err = "gh_rhs_noalloc: state of " + std::to_string(d->state) + " doubles exceeds the fixed work area (" +
             std::to_string(kMaxState) + " doubles); use gh_rhs";
    return GH_EINVAL;
  }
  if (gh_status s = gh::check_latched(d)) return s;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && dev != d->device) {
    d->err = "gh_rhs_noalloc: the current device is not the domain's device";
    return GH_EINVAL;
  }
  double* w = nullptr;
  if (e == cudaSuccess && gh::frame_moving(d)) {
    const double off = 0.0;            // the frame at the domain clock
    e = gh::launch_frames(d, &off, 1, 0.0);
    d->frd = d->frames_d;
    if (e == cudaSuccess) e = gh::launch_map_stage(d);
  }
  if (e == cudaSuccess) e = work_area(dev, &w);
  if (e == cudaSuccess) e = gh::launch_radial(d, u, w, false);
  if (e == cudaSuccess) e = gh::launch_angular_deriv_into(d, u, w + kMaxState, w + 2 * kMaxState);
  if (e == cudaSuccess) e = gh::launch_pointwise_rhs_from(d, u, w, w + kMaxState, w + 2 * kMaxState, dudt);
  const double* deriv[3] = {w, w + kMaxState, w + 2 * kMaxState};
  if (e == cudaSuccess) e = gh::launch_bc(d, dudt, 0, 0.0, nullptr, nullptr, nullptr, u, deriv);
  if (e != cudaSuccess) {
    d->err = std::string("gh_rhs_noalloc: ") + cudaGetErrorString(e);
    return GH_ECUDA;
  }
  return GH_OK;
}
