// Kernel argument blocks and host-side launchers shared by the library's
// translation units (internal; the public interface is include/mhd.h).
#pragma once
#include <cuda_runtime.h>

#include "mhd_device.cuh"

namespace mhd {

constexpr int kMagWarps = 8;  // interior rows of a magnetic-sweep tile

struct FluidArgs {
  const float* in[8];  // current fields
  float* out[8];       // destinations of fields 0..4 (others unused)
  Box box;
  float gamma;
  const float* tau;    // device scalar: step of this sweep
  unsigned* rate;      // fused CFL rate accumulator (float bits), or nullptr
  int seg;             // pencil segment length along the sweep axis
};

struct MagArgs {
  const float* in[8];
  float* out[3];       // destinations of b_x, b_y, b_z
  Box box;
  const float* tau;
  int seg;
};

struct TransposeArgs {
  const float* in[8];
  float* out[8];
  int n[3];  // input extents, fastest first; the output has n[1] fastest
};

// Record "<where>: <what>" as this thread's last error (mhd_last_error) and
// return code.
int set_error(int code, const char* where, const char* what);

// launchers (return cudaGetLastError of the launch)
cudaError_t launch_transpose01(const TransposeArgs& a, cudaStream_t s);
cudaError_t launch_fluid(int axis, bool rate, const FluidArgs& a, cudaStream_t s);
cudaError_t launch_mag(int axis, const MagArgs& a, cudaStream_t s);
cudaError_t launch_cfl_rate(const float* const f[8], const Box& box, float gamma, unsigned* rate,
                            cudaStream_t s);
// device-side step control: tau = cfl / rate_cur (or the given tau if cfl<0),
// time += 2 tau, rate_next = 0
cudaError_t launch_step_control(const unsigned* rate_cur, unsigned* rate_next, float* tau,
                                double* time, double cfl, double tau_host, cudaStream_t s);
// set the device sweep step to a host value (no time advance)
cudaError_t launch_set_tau(float* tau, double value, cudaStream_t s);
// FP64 diagnostics: per-block partials into `partial` (nblk*kDiagSlots
// doubles), then a fixed-order final reduction into out[10] (device).
constexpr int kDiagSlots = 20;  // 8 (sum, compensation) pairs + max|div b| + min p
int diag_blocks(const Box& box);
cudaError_t launch_diagnostics(const float* const f[8], const Box& box, double gamma, double* partial,
                               double* out, cudaStream_t s);

}  // namespace mhd
