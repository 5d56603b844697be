// The fluid sweep of the paper's scheme (van Leer limiter, bound freezing
// speed) and the dispatch to the scheme variants.
#include "sweep_fluid.cuh"

namespace mhd {

template cudaError_t launch_fluid_t<0, false>(int, bool, const FluidArgs&, cudaStream_t);

cudaError_t launch_fluid(int axis, bool rate, const FluidArgs& a, cudaStream_t s) {
  if (a.fast) return launch_fluid_t<0, true>(axis, rate, a, s);
  switch (a.lim) {
    case 1: return launch_fluid_t<1, false>(axis, rate, a, s);
    case 2: return launch_fluid_t<2, false>(axis, rate, a, s);
    default: return launch_fluid_t<0, false>(axis, rate, a, s);
  }
}

}  // namespace mhd
