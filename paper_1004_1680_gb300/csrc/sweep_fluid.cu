// The fluid sweep of the paper's scheme (van Leer limiter, bound freezing
// speed) and the dispatch to the scheme variants.
#include <cstring>

#include "sweep_fluid.cuh"

namespace mhd {

namespace {

// The fields of one sweep and the box: a step cycles through a few such sets
// (the fields alternate between two arrays), so the encoded maps are kept.
struct MapKey {
  const float* f[8];
  int n[3];
  int axis;
  long long stride[3];
};
struct MapEntry {
  MapKey key;
  FluidMaps maps;
  bool used;
};
constexpr int kMapCache = 16;

}  // namespace

bool make_fluid_maps(int axis, const FluidArgs& a, FluidMaps* out) {
  if (axis != 1 && axis != 2) return false;
  const Box& b = a.box;
  const int A = 0, O = (axis == 2) ? 1 : 2, D = axis, T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  if (b.stride[A] != 1 || b.n[D] < 16) return false;
  if ((b.stride[O] * 4) % 16 || (b.stride[D] * 4) % 16) return false;
  for (int q = 0; q < 8; q++)
    if (reinterpret_cast<uintptr_t>(a.in[q]) % 16) return false;
  MapKey key;
  std::memset(&key, 0, sizeof key);
  for (int q = 0; q < 8; q++) key.f[q] = a.in[q];
  for (int k = 0; k < 3; k++) {
    key.n[k] = b.n[k];
    key.stride[k] = b.stride[k];
  }
  key.axis = axis;
  thread_local MapEntry cache[kMapCache];
  thread_local int next = 0;
  for (const MapEntry& e : cache)
    if (e.used && std::memcmp(&e.key, &key, sizeof key) == 0) {
      *out = e.maps;
      return true;
    }
  const cuuint64_t dim[3] = {(cuuint64_t)b.n[A], (cuuint64_t)b.n[O], (cuuint64_t)b.n[D]};
  const cuuint64_t st[2] = {(cuuint64_t)b.stride[O] * 4, (cuuint64_t)b.stride[D] * 4};
  const float* f[7] = {a.in[RHO], a.in[MX + D], a.in[MX + T1], a.in[MX + T2], a.in[EN], a.in[BX + A], a.in[BX + O]};
  FluidMaps m;
  bool ok = true;
  for (int k = 0; k < 7; k++)
    ok = ok && tma_encode_f32(&m.full[k], f[k], dim, st, 32, kFluidWarps, kTmaCh) &&
         tma_encode_f32(&m.row[k], f[k], dim, st, 32, kFluidWarps, 1);
  ok = ok && tma_encode_f32(&m.full[7], a.in[BX + D], dim, st, 32, kFluidWarps, kTmaCh + 1) &&
       tma_encode_f32(&m.row[7], a.in[BX + D], dim, st, 32, kFluidWarps, 1);
  ok = ok && tma_encode_f32(&m.full[8], a.in[BX + A], dim, st, 4, kFluidWarps, kTmaCh) &&
       tma_encode_f32(&m.row[8], a.in[BX + A], dim, st, 4, kFluidWarps, 1);
  ok = ok && tma_encode_f32(&m.full[9], a.in[BX + O], dim, st, 32, 1, kTmaCh) &&
       tma_encode_f32(&m.row[9], a.in[BX + O], dim, st, 32, 1, 1);
  if (!ok) return false;
  MapEntry& e = cache[next];
  next = (next + 1) % kMapCache;
  e.key = key;
  e.maps = m;
  e.used = true;
  *out = m;
  return true;
}

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
