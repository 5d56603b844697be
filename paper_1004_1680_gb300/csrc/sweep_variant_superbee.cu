// Ablation of the paper's scheme: the superbee limiter in the fluid and
// magnetic sweeps (its own translation unit, compiled in parallel).
#include "sweep_fluid.cuh"
#include "sweep_mag.cuh"

namespace mhd {

template cudaError_t launch_fluid_t<2, 0>(int, bool, const FluidArgs&, cudaStream_t);
template cudaError_t launch_mag_t<2>(int, const MagArgs&, cudaStream_t);
template cudaError_t prepare_mag_t<2>();

}  // namespace mhd
