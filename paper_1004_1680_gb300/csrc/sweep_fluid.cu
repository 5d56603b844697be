// The fluid sweep of the paper's scheme (van Leer limiter, bound freezing
// speed) and the dispatch to the scheme variants.
#include <cstring>

#include "sweep_fluid.cuh"

namespace mhd {

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime.
EncodeTiled encoder() {
  static const EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiled) nullptr;
    }
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// A box of b0 x b1 x b2 FP32 elements of a tensor of extents dim (the first
// contiguous) and byte strides st of dimensions 1 and 2; out-of-range
// elements read as zero.
bool encode(CUtensorMap* m, const float* p, const cuuint64_t dim[3], const cuuint64_t st[2], cuuint32_t b0,
            cuuint32_t b1, cuuint32_t b2) {
  const cuuint32_t box[3] = {b0, b1, b2}, es[3] = {1, 1, 1};
  return encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(p), dim, st, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

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
  if (b.stride[A] != 1 || b.n[A] % 32 || b.n[O] % kFluidWarps || b.n[D] < 16) return false;
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
  if (!encoder()) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)b.n[A], (cuuint64_t)b.n[O], (cuuint64_t)b.n[D]};
  const cuuint64_t st[2] = {(cuuint64_t)b.stride[O] * 4, (cuuint64_t)b.stride[D] * 4};
  const float* f[7] = {a.in[RHO], a.in[MX + D], a.in[MX + T1], a.in[MX + T2], a.in[EN], a.in[BX + A], a.in[BX + O]};
  FluidMaps m;
  bool ok = true;
  for (int k = 0; k < 7; k++)
    ok = ok && encode(&m.full[k], f[k], dim, st, 32, kFluidWarps, kTmaCh) &&
         encode(&m.row[k], f[k], dim, st, 32, kFluidWarps, 1);
  ok = ok && encode(&m.full[7], a.in[BX + D], dim, st, 32, kFluidWarps, kTmaCh + 1) &&
       encode(&m.row[7], a.in[BX + D], dim, st, 32, kFluidWarps, 1);
  ok = ok && encode(&m.full[8], a.in[BX + A], dim, st, 4, kFluidWarps, kTmaCh) &&
       encode(&m.row[8], a.in[BX + A], dim, st, 4, kFluidWarps, 1);
  ok = ok && encode(&m.full[9], a.in[BX + O], dim, st, 32, 1, kTmaCh) &&
       encode(&m.row[9], a.in[BX + O], dim, st, 32, 1, 1);
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
