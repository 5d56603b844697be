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

#include "mhd.h"
#include "mhd_launch.h"

namespace {

// The diagnostics grid never has more blocks than kDiagMaxBlocks (diag_blocks
// caps it), so the partials of any box fit; the last 16 doubles take the 10
// results.
constexpr int kStaticDiagBlocks = mhd::kDiagMaxBlocks;
constexpr int kStaticDiagDoubles = kStaticDiagBlocks * mhd::kDiagSlots + 16;
__device__ __align__(256) double g_diag_scratch[kStaticDiagDoubles];  // 194 KiB per GPU

// Device address of g_diag_scratch in the context current on this thread.
// In host code the name g_diag_scratch is only a host-side stand-in, not a
// device address, so the runtime is asked for the real one.  It is asked on
// every call rather than cached: the address belongs to the context that
// loaded the module, and a cached value would be wrong after a device reset
// (the module is loaded again, possibly elsewhere) or in another context on
// the same device.  The first call in a context loads the module there.
int scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_diag_scratch);
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "cudaGetSymbolAddress", cudaGetErrorString(e));
  *out = static_cast<double*>(p);
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
  const mhd::Box box = mhd::make_box(nx, ny, nz);
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
