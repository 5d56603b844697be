// The fluid sweep of the paper's scheme (van Leer limiter, bound freezing
// speed) and the dispatch to the scheme variants.
#include "sweep_fluid.cuh"

namespace mhd {

template cudaError_t launch_fluid_t<0, 0>(int, bool, const FluidArgs&, cudaStream_t);

cudaError_t launch_fluid(int axis, bool rate, const FluidArgs& a, cudaStream_t s) {
  if (a.fast == 1) return launch_fluid_t<0, 1>(axis, rate, a, s);
  if (a.fast == 2) return launch_fluid_t<0, 2>(axis, rate, a, s);
  switch (a.lim) {
    case 1: return launch_fluid_t<1, 0>(axis, rate, a, s);
    case 2: return launch_fluid_t<2, 0>(axis, rate, a, s);
    default: return launch_fluid_t<0, 0>(axis, rate, a, s);
  }
}

}  // namespace mhd
