// The magnetic sweep of the paper's scheme (van Leer limiter) and the
// dispatch to the limiter variants.
#include "sweep_mag.cuh"

namespace mhd {

template cudaError_t launch_mag_t<0>(int, const MagArgs&, cudaStream_t);
template cudaError_t prepare_mag_t<0>();

cudaError_t prepare_mag_kernels() {
  cudaError_t e = prepare_mag_t<0>();
  if (e == cudaSuccess) e = prepare_mag_t<1>();
  if (e == cudaSuccess) e = prepare_mag_t<2>();
  return e;
}

cudaError_t launch_mag(int axis, const MagArgs& a, cudaStream_t s) {
  switch (a.lim) {
    case 1: return launch_mag_t<1>(axis, a, s);
    case 2: return launch_mag_t<2>(axis, a, s);
    default: return launch_mag_t<0>(axis, a, s);
  }
}

}  // namespace mhd
