// The magnetic sweep of the paper's scheme (van Leer limiter) and the
// dispatch to the limiter variants.
#include <cstring>

#include "sweep_mag.cuh"

namespace mhd {

namespace {

// The fields and box of one sweep: a step cycles through a few such sets, so
// the encoded maps are kept.
struct MagMapKey {
  const float* f[8];
  int n[3];
  int axis;
  long long stride[3];
};
struct MagMapEntry {
  MagMapKey key;
  MagMaps maps;
  bool used;
};
constexpr int kMagMapCache = 16;

}  // namespace

bool make_mag_maps(int axis, const MagArgs& a, MagMaps* out) {
  if (axis != 1 && axis != 2) return false;
  const Box& b = a.box;
  const int A = 0, O = (axis == 2) ? 1 : 2, D = axis;
  if (b.stride[A] != 1 || b.n[A] % 32 || b.n[O] % kMagWarps || b.n[D] < 16) return false;
  if ((b.stride[O] * 4) % 16 || (b.stride[D] * 4) % 16) return false;
  const float* f[5] = {a.in[RHO], a.in[MX + D], a.in[BX + A], a.in[BX + O], a.in[BX + D]};
  for (const float* p : f)
    if (reinterpret_cast<uintptr_t>(p) % 16) return false;
  MagMapKey key;
  std::memset(&key, 0, sizeof key);
  for (int q = 0; q < 8; q++) key.f[q] = a.in[q];
  for (int k = 0; k < 3; k++) {
    key.n[k] = b.n[k];
    key.stride[k] = b.stride[k];
  }
  key.axis = axis;
  thread_local MagMapEntry cache[kMagMapCache];
  thread_local int next = 0;
  for (const MagMapEntry& e : cache)
    if (e.used && std::memcmp(&e.key, &key, sizeof key) == 0) {
      *out = e.maps;
      return true;
    }
  const cuuint64_t dim[3] = {(cuuint64_t)b.n[A], (cuuint64_t)b.n[O], (cuuint64_t)b.n[D]};
  const cuuint64_t st[2] = {(cuuint64_t)b.stride[O] * 4, (cuuint64_t)b.stride[D] * 4};
  MagMaps m;
  bool ok = true;
  for (int depth = 0; depth < 2; depth++) {  // whole chunks, then single positions
    CUtensorMap* t = depth ? m.row : m.full;
    const cuuint32_t nd = depth ? 1 : kMagCH;
    for (int k = 0; k < 5; k++) ok = ok && tma_encode_f32(&t[k], f[k], dim, st, 32, kMagWarps, nd);
    ok = ok && tma_encode_f32(&t[5], f[0], dim, st, 32, 1, nd) && tma_encode_f32(&t[6], f[1], dim, st, 32, 1, nd) &&
         tma_encode_f32(&t[7], f[3], dim, st, 32, 1, nd);
    ok = ok && tma_encode_f32(&t[8], f[0], dim, st, 4, kMagWarps, nd) &&
         tma_encode_f32(&t[9], f[1], dim, st, 4, kMagWarps, nd) &&
         tma_encode_f32(&t[10], f[2], dim, st, 4, kMagWarps, nd);
  }
  if (!ok) return false;
  MagMapEntry& e = cache[next];
  next = (next + 1) % kMagMapCache;
  e.key = key;
  e.maps = m;
  e.used = true;
  *out = m;
  return true;
}

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
