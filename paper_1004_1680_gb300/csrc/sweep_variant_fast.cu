// Ablation of the paper's scheme: the exact fast magnetosonic speed as the
// freezing speed of the fluid sweeps (its own translation unit).
#include "sweep_fluid.cuh"

namespace mhd {

template cudaError_t launch_fluid_t<0, 1>(int, bool, const FluidArgs&, cudaStream_t);

}  // namespace mhd
