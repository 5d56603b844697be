// C ABI of the kernels behind the learned coarse-grid correction: the
// tensor-core 3-D convolution (forward and input gradient), its weight
// gradient, weight packing, and the error flag of the bounded waits.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "mhd.h"
#include "mhd_launch.h"

namespace {

__device__ int g_conv_err;  // set by a convolution block whose bounded wait gave up

constexpr int kMaxDevices = 64;
int* g_err_addr[kMaxDevices] = {};
bool g_prepared[kMaxDevices] = {};
std::mutex g_lock;

int device_setup(int** err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "cudaGetDevice", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return mhd::set_error(MHD_E_ARG, "device index", "out of range");
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_prepared[dev]) {
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_conv_err)) != cudaSuccess)
      return mhd::set_error(MHD_E_CUDA, "cudaGetSymbolAddress", cudaGetErrorString(e));
    if ((e = mhd::prepare_conv_kernels()) != cudaSuccess)
      return mhd::set_error(MHD_E_CUDA, "conv kernel attributes", cudaGetErrorString(e));
    g_err_addr[dev] = static_cast<int*>(p);
    g_prepared[dev] = true;
  }
  *err = g_err_addr[dev];
  return MHD_OK;
}

bool valid_channels(int c) { return c == 8 || c == 32; }

}  // namespace

extern "C" {

size_t mhd_conv_pack_bytes(int cin, int cout, int transpose) {
  if (!valid_channels(cin) || !valid_channels(cout)) return 0;
  const int rows = transpose ? cin : cout, cols = transpose ? cout : cin;
  return mhd::conv_image_bytes(rows, cols);
}

int mhd_conv_pack(const float* w, int cin, int cout, int transpose, void* img, void* stream) {
  if (!w || !img || !valid_channels(cin) || !valid_channels(cout))
    return mhd::set_error(MHD_E_ARG, "mhd_conv_pack", "need channels in {8, 32} and non-null buffers");
  cudaError_t e = mhd::launch_conv_pack(w, cin, cout, transpose ? 1 : 0, static_cast<uint16_t*>(img),
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "mhd_conv_pack", cudaGetErrorString(e));
  return MHD_OK;
}

int mhd_conv3d(int nx, int ny, int nz, int cin, int cout, const void* x, const void* img, size_t img_bytes,
               const float* bias, int relu, int flip, const void* mask, void* y_bf16, float* y_f32, void* stream) {
  const long long cells = (long long)nx * ny * nz;
  if (nx < 8 || ny < 16 || nz < 1 || nx % 8 || ny % 16 || cells >= (1LL << 31) || !valid_channels(cin) ||
      !valid_channels(cout) || !x || !img || (!y_bf16 && !y_f32))
    return mhd::set_error(MHD_E_ARG, "mhd_conv3d",
                          "need nx % 8 == 0, ny % 16 == 0, channels in {8, 32}, input, weights and an output");
  // 16-byte copies and stores: activations, mask and outputs 16-byte aligned
  const auto mis = [](const void* p) { return ((uintptr_t)p & 15) != 0; };
  if (mis(x) || mis(img) || mis(mask) || mis(y_bf16) || mis(y_f32))
    return mhd::set_error(MHD_E_ARG, "mhd_conv3d", "buffers must be 16-byte aligned");
  // the blocks copy the 3 npad x kchunks*32 BF16 weights: the image must be exactly that
  if (img_bytes != mhd::conv_image_bytes(cout, cin))
    return mhd::set_error(MHD_E_ARG, "mhd_conv3d", "weight image size does not match cin/cout");
  int* err = nullptr;
  int rc = device_setup(&err);
  if (rc) return rc;
  mhd::ConvArgs a;
  a.x = static_cast<const __nv_bfloat16*>(x);
  a.wpack = static_cast<const uint16_t*>(img);
  a.bias = bias;
  a.y = static_cast<__nv_bfloat16*>(y_bf16);
  a.y32 = y_f32;
  a.mask = static_cast<const __nv_bfloat16*>(mask);
  a.n[0] = nx;
  a.n[1] = ny;
  a.n[2] = nz;
  a.cin = cin;
  a.cout = cout;
  a.npad = mhd::conv_npad(cout);
  a.kchunks = mhd::conv_kchunks(cin);
  a.relu = relu ? 1 : 0;
  a.flip = flip ? 1 : 0;
  a.err = err;
  cudaError_t e = mhd::launch_conv3d(a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "mhd_conv3d", cudaGetErrorString(e));
  return MHD_OK;
}

int mhd_conv3d_wgrad(int nx, int ny, int nz, int cin, int cout, const void* x, const void* gy, float* gw,
                     float* gb, void* stream) {
  const long long cells = (long long)nx * ny * nz;
  if (nx < 1 || ny < 1 || nz < 1 || cells % 64 || cells >= (1LL << 31) || !valid_channels(cin) ||
      !valid_channels(cout) || !x || !gy || !gw)
    return mhd::set_error(MHD_E_ARG, "mhd_conv3d_wgrad", "bad arguments");
  const int n[3] = {nx, ny, nz};
  int* err = nullptr;
  int rc = device_setup(&err);
  if (rc) return rc;
  // the tensor-core path copies 16-byte pieces of whole 8 x 16 x 1 tiles
  const bool tiles = nx % 8 == 0 && ny % 16 == 0 && !(((uintptr_t)x | (uintptr_t)gy) & 15);
  cudaError_t e = mhd::launch_conv_wgrad(static_cast<const __nv_bfloat16*>(x), static_cast<const __nv_bfloat16*>(gy),
                                         n, cin, cout, gw, gb, tiles ? err : nullptr,
                                         static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "mhd_conv3d_wgrad", cudaGetErrorString(e));
  return MHD_OK;
}

namespace {
constexpr int kLayerIn[4] = {8, 32, 32, 32}, kLayerOut[4] = {32, 32, 32, 8};
}  // namespace

int mhd_cnn_forward(int nx, int ny, int nz, const void* x, const void* const img[4], const size_t img_bytes[4],
                    const float* const bias[4], void* const acts[3], float* y, void* stream) {
  if (!x || !img || !img_bytes || !bias || !acts || !y)
    return mhd::set_error(MHD_E_ARG, "mhd_cnn_forward", "null argument");
  for (int l = 0; l < 4; l++)
    if (!img[l] || (l < 3 && !acts[l])) return mhd::set_error(MHD_E_ARG, "mhd_cnn_forward", "null image or buffer");
  const void* h = x;
  for (int l = 0; l < 4; l++) {
    const bool last = l == 3;
    const int rc = mhd_conv3d(nx, ny, nz, kLayerIn[l], kLayerOut[l], h, img[l], img_bytes[l], bias[l], last ? 0 : 1,
                              0, nullptr, last ? nullptr : acts[l], last ? y : nullptr, stream);
    if (rc) return rc;
    if (!last) h = acts[l];
  }
  return MHD_OK;
}

int mhd_cnn_backward(int nx, int ny, int nz, const void* x, const void* const acts[3], const void* gy,
                     const void* const imgT[4], const size_t imgT_bytes[4], float* const gw[4], float* const gb[4],
                     void* const scratch[2], void* stream) {
  if (!x || !acts || !gy || !imgT || !imgT_bytes || !gw || !gb || !scratch || !scratch[0] || !scratch[1])
    return mhd::set_error(MHD_E_ARG, "mhd_cnn_backward", "null argument");
  for (int l = 0; l < 4; l++)
    if (!imgT[l] || !gw[l] || (l < 3 && !acts[l])) return mhd::set_error(MHD_E_ARG, "mhd_cnn_backward", "null buffer");
  const void* g = gy;  // gradient of the loss w.r.t. layer l's output
  for (int l = 3; l >= 0; l--) {
    const void* in = l ? acts[l - 1] : x;  // layer l's input
    int rc = mhd_conv3d_wgrad(nx, ny, nz, kLayerIn[l], kLayerOut[l], in, g, gw[l], gb[l], stream);
    if (rc) return rc;
    if (l == 0) break;
    void* gin = scratch[l & 1];  // gradient w.r.t. layer l's input, through its ReLU mask
    rc = mhd_conv3d(nx, ny, nz, kLayerOut[l], kLayerIn[l], g, imgT[l], imgT_bytes[l], nullptr, 0, 1, acts[l - 1],
                    gin, nullptr, stream);
    if (rc) return rc;
    g = gin;
  }
  return MHD_OK;
}

int mhd_conv_error(int* flag) {
  if (!flag) return mhd::set_error(MHD_E_ARG, "mhd_conv_error", "null argument");
  int* err = nullptr;
  int rc = device_setup(&err);
  if (rc) return rc;
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
  if (e != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "mhd_conv_error", cudaGetErrorString(e));
  *flag = v;
  return v ? mhd::set_error(MHD_E_TIMEOUT, "mhd_conv3d", "a tensor-core wait gave up") : MHD_OK;
}

}  // extern "C"
