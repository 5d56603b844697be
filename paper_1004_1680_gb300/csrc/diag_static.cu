// FP64 diagnostics for callers that cannot allocate device memory.
//
// mhd_diagnostics (mhd_api.cu) keeps its per-block partial sums in scratch
// that mhd_create allocated.  Some callers have no mhd_t and may not call
// cudaMalloc at all: code running inside a framework whose caching allocator
// owns the device memory, latency-critical loops where an allocation (which
// can synchronise the whole device) is not allowed, or plug-in hosts that
// give a component no allocation rights.  mhd_diagnostics_static runs the
// same two kernels on caller-provided fields, with the scratch taken from the
// fixed array below, which every GPU that loads this library holds until the
// process exits.
#include <cstdio>
#include <mutex>

#include "mhd.h"
#include "mhd_launch.h"

namespace {

// The diagnostics grid never has more blocks than this (diag_blocks caps it),
// so the partials of any box fit; the last 16 doubles take the 10 results.
constexpr int kStaticDiagBlocks = 152 * 8;
constexpr int kStaticDiagDoubles = kStaticDiagBlocks * mhd::kDiagSlots + 16;
__device__ __align__(256) double g_diag_scratch[kStaticDiagDoubles];  // 194 KiB per GPU

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_lock;

// Device address of g_diag_scratch on the current device.  In host code the
// name g_diag_scratch is only a host-side stand-in, not a device address; the
// runtime resolves the real address once per device.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "cudaGetDevice", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return mhd::set_error(MHD_E_ARG, "device index", "out of range");
  std::lock_guard<std::mutex> g(g_scratch_lock);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_diag_scratch);
    if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "cudaGetSymbolAddress", cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MHD_OK;
}

}  // namespace

extern "C" int mhd_diagnostics_static(int nx, int ny, int nz, double gamma, const float* const f[8],
                                      double out[10], void* cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !(gamma > 1.0))
    return mhd::set_error(MHD_E_ARG, "mhd_diagnostics_static", "need n >= 1 and gamma > 1");
  const long long N = (long long)nx * ny * nz;
  if (N >= (1LL << 31))
    return mhd::set_error(MHD_E_ARG, "mhd_diagnostics_static",
                          "box too large: at most 2^31 - 1 cells per field");
  if (!f || !out) return mhd::set_error(MHD_E_ARG, "mhd_diagnostics_static", "null argument");
  for (int q = 0; q < 8; q++)
    if (!f[q]) return mhd::set_error(MHD_E_ARG, "mhd_diagnostics_static", "null field pointer");
  mhd::Box box;
  box.n[0] = nx;
  box.n[1] = ny;
  box.n[2] = nz;
  box.stride[0] = 1;
  box.stride[1] = nx;
  box.stride[2] = (long long)nx * ny;
  if (mhd::diag_blocks(box) > kStaticDiagBlocks)
    return mhd::set_error(MHD_E_ARG, "mhd_diagnostics_static", "partials exceed the static scratch");
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  // Every partial slot the final reduction reads is written by this call, so
  // nothing needs clearing; calls that overlap on the GPU share the array and race.
  double* partial = scratch;
  double* result = scratch + (size_t)kStaticDiagBlocks * mhd::kDiagSlots;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = mhd::launch_diagnostics(f, box, gamma, partial, result, s);
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "diagnostics launch", cudaGetErrorString(e));
  e = cudaMemcpyAsync(out, result, sizeof(double) * 10, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "diagnostics copy", cudaGetErrorString(e));
  return MHD_OK;
}
