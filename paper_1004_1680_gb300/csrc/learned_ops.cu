// Element-wise and stencil kernels of the learned coarse-grid correction
// (everything around the convolutions): restriction of a fine state to a
// coarse grid, input normalisation, projection of the network output onto a
// conservative, divergence-free correction (and its exact adjoint for
// training), the loss, the clipped application of a correction to a state,
// and the Adam update.  Fields are SoA FP32 (8 arrays of nx*ny*nz, as in the
// solver); network tensors are channels-last [cell][8].
#include <cuda_bf16.h>

#include "mhd.h"
#include "mhd_launch.h"

namespace mhd {
namespace {

struct F8 {
  float v[8];
};
struct P8 {
  float* p[8];
};
struct CP8 {
  const float* p[8];
};

__device__ __forceinline__ int cell_of(int i, int j, int k, int nx, int ny, int nz) {
  i = (i + nx) % nx;
  j = (j + ny) % ny;
  k = (k + nz) % nz;
  return i + nx * (j + ny * k);
}

// coarse cell (I, J, K) <- fine r^3 block; face fields: mean of the r^2 fine
// faces tiling the coarse low face (flux preserving, so div b stays 0)
__global__ void restrict_kernel(CP8 f, int nx, int ny, int nz, int r, P8 c) {
  const int NX = nx / r, NY = ny / r, NZ = nz / r;
  const int N = NX * NY * NZ;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x) {
    const int I = idx % NX, J = (idx / NX) % NY, K = idx / (NX * NY);
    double acc[5] = {0, 0, 0, 0, 0};
    for (int kk = 0; kk < r; kk++)
      for (int jj = 0; jj < r; jj++)
        for (int ii = 0; ii < r; ii++) {
          const int fc = (I * r + ii) + nx * ((J * r + jj) + ny * (K * r + kk));
          for (int q = 0; q < 5; q++) acc[q] += f.p[q][fc];
        }
    for (int q = 0; q < 5; q++) c.p[q][idx] = (float)(acc[q] / (r * r * r));
    double bx = 0, by = 0, bz = 0;
    for (int a = 0; a < r; a++)
      for (int b = 0; b < r; b++) {
        bx += f.p[BX][(I * r) + nx * ((J * r + a) + ny * (K * r + b))];
        by += f.p[BY][(I * r + a) + nx * ((J * r) + ny * (K * r + b))];
        bz += f.p[BZ][(I * r + a) + nx * ((J * r + b) + ny * (K * r))];
      }
    c.p[BX][idx] = (float)(bx / (r * r));
    c.p[BY][idx] = (float)(by / (r * r));
    c.p[BZ][idx] = (float)(bz / (r * r));
  }
}

__global__ void normalize_kernel(CP8 s, int N, F8 mu, F8 isig, __nv_bfloat16* x) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
#pragma unroll
    for (int q = 0; q < 8; q++) x[(size_t)c * 8 + q] = __float2bfloat16_rn((s.p[q][c] - mu.v[q]) * isig.v[q]);
}

// Network output y[cell][8] -> correction d: d_q = s_q y_q for q < 5 (cell
// quantities), and b = curl of the edge potential A_c = s_A y_{5+c} (A_x on
// x-edges (i, j-1/2, k-1/2), A_y on (i-1/2, j, k-1/2), A_z on (i-1/2, j-1/2, k)):
// the discrete divergence of d_b vanishes identically.  sums[q] accumulates
// the box totals of d_q (q < 5) for the mean removal.
__global__ void project_kernel(const float* __restrict__ y, int nx, int ny, int nz, F8 sc, P8 d, double* sums) {
  const int N = nx * ny * nz;
  const float sA = sc.v[5];
  double loc[5] = {0, 0, 0, 0, 0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
#pragma unroll
    for (int q = 0; q < 5; q++) {
      const float v = sc.v[q] * y[(size_t)c * 8 + q];
      d.p[q][c] = v;
      loc[q] += v;
    }
    const int jp = cell_of(i, j + 1, k, nx, ny, nz), kp = cell_of(i, j, k + 1, nx, ny, nz);
    const int ip = cell_of(i + 1, j, k, nx, ny, nz);
    const float Ax = y[(size_t)c * 8 + 5], Ay = y[(size_t)c * 8 + 6], Az = y[(size_t)c * 8 + 7];
    d.p[BX][c] = sA * ((y[(size_t)jp * 8 + 7] - Az) * ny - (y[(size_t)kp * 8 + 6] - Ay) * nz);
    d.p[BY][c] = sA * ((y[(size_t)kp * 8 + 5] - Ax) * nz - (y[(size_t)ip * 8 + 7] - Az) * nx);
    d.p[BZ][c] = sA * ((y[(size_t)ip * 8 + 6] - Ay) * nx - (y[(size_t)jp * 8 + 5] - Ax) * ny);
  }
  for (int q = 0; q < 5; q++) {
    double v = loc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sums[q], v);
  }
}

__global__ void subtract_mean_kernel(P8 d, int N, const double* sums) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
#pragma unroll
    for (int q = 0; q < 5; q++) d.p[q][c] -= (float)(sums[q] / N);
}

// loss = sum_q w_q sum_cells (d_q - t_q)^2 ; g_q = 2 w_q (d_q - t_q)
__global__ void loss_kernel(CP8 d, CP8 t, int N, F8 w, double* loss, P8 g) {
  double loc = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const float diff = d.p[q][c] - t.p[q][c];
      loc += (double)w.v[q] * diff * diff;
      if (g.p[0]) g.p[q][c] = 2.f * w.v[q] * diff;
    }
  for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, loc);
}

__global__ void grad_sums_kernel(CP8 g, int N, double* sums) {
  double loc[5] = {0, 0, 0, 0, 0};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
#pragma unroll
    for (int q = 0; q < 5; q++) loc[q] += g.p[q][c];
  for (int q = 0; q < 5; q++) {
    double v = loc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sums[q], v);
  }
}

// adjoint of project + mean removal: gy_q = s_q (g_q - mean g_q) for q < 5;
// gy_{5+c} = s_A (curl^T g_b)_c
__global__ void project_backward_kernel(CP8 g, int nx, int ny, int nz, F8 sc, const double* sums,
                                        __nv_bfloat16* gy) {
  const int N = nx * ny * nz;
  const float sA = sc.v[5];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
#pragma unroll
    for (int q = 0; q < 5; q++)
      gy[(size_t)c * 8 + q] = __float2bfloat16_rn(sc.v[q] * (g.p[q][c] - (float)(sums[q] / N)));
    const int im = cell_of(i - 1, j, k, nx, ny, nz), jm = cell_of(i, j - 1, k, nx, ny, nz),
              km = cell_of(i, j, k - 1, nx, ny, nz);
    const float* gx = g.p[BX];
    const float* gyf = g.p[BY];
    const float* gz = g.p[BZ];
    const float aX = nz * (gyf[km] - gyf[c]) + ny * (gz[c] - gz[jm]);
    const float aY = nz * (gx[c] - gx[km]) + nx * (gz[im] - gz[c]);
    const float aZ = ny * (gx[jm] - gx[c]) + nx * (gyf[c] - gyf[im]);
    gy[(size_t)c * 8 + 5] = __float2bfloat16_rn(sA * aX);
    gy[(size_t)c * 8 + 6] = __float2bfloat16_rn(sA * aY);
    gy[(size_t)c * 8 + 7] = __float2bfloat16_rn(sA * aZ);
  }
}

__device__ __forceinline__ float cell_mag(const float* const* s, int c, int nx, int ny, int nz) {
  const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
  const float bx = 0.5f * (s[BX][c] + s[BX][cell_of(i + 1, j, k, nx, ny, nz)]);
  const float by = 0.5f * (s[BY][c] + s[BY][cell_of(i, j + 1, k, nx, ny, nz)]);
  const float bz = 0.5f * (s[BZ][c] + s[BZ][cell_of(i, j, k + 1, nx, ny, nz)]);
  return 0.5f * (bx * bx + by * by + bz * bz);
}

// pass 1: thermal energy of the uncorrected state
__global__ void thermal_kernel(CP8 s, int nx, int ny, int nz, float* eth) {
  const int N = nx * ny * nz;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const float kin = 0.5f * (s.p[1][c] * s.p[1][c] + s.p[2][c] * s.p[2][c] + s.p[3][c] * s.p[3][c]) / s.p[0][c];
    eth[c] = s.p[4][c] - kin - cell_mag(s.p, c, nx, ny, nz);
  }
}

// pass 2: faces b += d_b (divergence-free, never scaled)
__global__ void add_field_kernel(P8 s, CP8 d, int N) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
    for (int q = 5; q < 8; q++) s.p[q][c] += d.p[q][c];
}

// pass 3: cell quantities with the density clipped at -rho/2 and the whole
// cell correction scaled by the largest of 1, 1/2, 1/4, 0 that keeps the
// thermal energy above half its uncorrected value; if even 0 does not (the
// field correction raised the magnetic energy), e is raised to that bound.
__global__ void add_cells_kernel(P8 s, CP8 d, int nx, int ny, int nz, const float* eth0, int* nclip) {
  const int N = nx * ny * nz;
  int clipped = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const float rho = s.p[0][c];
    float du[5];
    du[0] = fmaxf(d.p[0][c], -0.5f * rho);
    for (int q = 1; q < 5; q++) du[q] = d.p[q][c];
    const float mag = cell_mag(const_cast<const float* const*>(s.p), c, nx, ny, nz);
    const float floor_e = 0.5f * eth0[c];
    float u[5];
    bool done = false;
    for (int t = 0; t < 4 && !done; t++) {
      const float a = t == 0 ? 1.f : (t == 1 ? 0.5f : (t == 2 ? 0.25f : 0.f));
      for (int q = 0; q < 5; q++) u[q] = s.p[q][c] + a * du[q];
      const float kin = 0.5f * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
      if (u[4] - kin - mag >= floor_e) {
        done = true;
        clipped += t > 0;
      }
    }
    if (!done) {  // u holds the uncorrected cell quantities (a = 0)
      const float kin = 0.5f * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) / u[0];
      u[4] = kin + mag + floor_e;
      clipped += 1;
    }
    if (du[0] != d.p[0][c]) clipped += 1;
    for (int q = 0; q < 5; q++) s.p[q][c] = u[q];
  }
  if (nclip && clipped) atomicAdd(nclip, clipped);
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

int blocks(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 152 * 32 ? 152 * 32 : (b < 1 ? 1 : b));
}

CP8 cp8(const float* const f[8]) {
  CP8 r;
  for (int q = 0; q < 8; q++) r.p[q] = f[q];
  return r;
}
P8 p8(float* const f[8]) {
  P8 r;
  for (int q = 0; q < 8; q++) r.p[q] = f ? f[q] : nullptr;
  return r;
}
F8 f8(const float* v, int n) {
  F8 r;
  for (int q = 0; q < 8; q++) r.v[q] = q < n ? v[q] : 0.f;
  return r;
}

int check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MHD_OK : set_error(MHD_E_CUDA, where, cudaGetErrorString(e));
}

bool bad_ptrs(const float* const f[8]) {
  if (!f) return true;
  for (int q = 0; q < 8; q++)
    if (!f[q]) return true;
  return false;
}

}  // namespace
}  // namespace mhd

using namespace mhd;

extern "C" {

int mhd_restrict(int nx, int ny, int nz, int r, const float* const fine[8], float* const coarse[8], void* stream) {
  if (r < 1 || nx % r || ny % r || nz % r || bad_ptrs(fine) || !coarse)
    return set_error(MHD_E_ARG, "mhd_restrict", "dims must be divisible by r; non-null fields");
  const long long N = (long long)(nx / r) * (ny / r) * (nz / r);
  restrict_kernel<<<blocks(N), 256, 0, (cudaStream_t)stream>>>(cp8(fine), nx, ny, nz, r, p8(coarse));
  return check_launch("mhd_restrict");
}

int mhd_cnn_normalize(int nx, int ny, int nz, const float* const s[8], const float mu[8], const float inv_sigma[8],
                      void* x_bf16, void* stream) {
  if (bad_ptrs(s) || !mu || !inv_sigma || !x_bf16) return set_error(MHD_E_ARG, "mhd_cnn_normalize", "null argument");
  const int N = nx * ny * nz;
  normalize_kernel<<<blocks(N), 256, 0, (cudaStream_t)stream>>>(cp8(s), N, f8(mu, 8), f8(inv_sigma, 8),
                                                                static_cast<__nv_bfloat16*>(x_bf16));
  return check_launch("mhd_cnn_normalize");
}

int mhd_cnn_project(int nx, int ny, int nz, const float* y, const float scale[6], float* const d[8], double* sums,
                    void* stream) {
  if (!y || !scale || !d || !sums) return set_error(MHD_E_ARG, "mhd_cnn_project", "null argument");
  const int N = nx * ny * nz;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * 5, s);
  if (e != cudaSuccess) return set_error(MHD_E_CUDA, "mhd_cnn_project", cudaGetErrorString(e));
  project_kernel<<<blocks(N), 256, 0, s>>>(y, nx, ny, nz, f8(scale, 6), p8(d), sums);
  subtract_mean_kernel<<<blocks(N), 256, 0, s>>>(p8(d), N, sums);
  return check_launch("mhd_cnn_project");
}

int mhd_cnn_loss(int nx, int ny, int nz, const float* const d[8], const float* const t[8], const float weight[8],
                 double* loss, float* const g[8], void* stream) {
  if (bad_ptrs(d) || bad_ptrs(t) || !weight || !loss) return set_error(MHD_E_ARG, "mhd_cnn_loss", "null argument");
  const int N = nx * ny * nz;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return set_error(MHD_E_CUDA, "mhd_cnn_loss", cudaGetErrorString(e));
  loss_kernel<<<blocks(N), 256, 0, s>>>(cp8(d), cp8(t), N, f8(weight, 8), loss, p8(g));
  return check_launch("mhd_cnn_loss");
}

int mhd_cnn_project_backward(int nx, int ny, int nz, const float* const g[8], const float scale[6], double* sums,
                             void* gy_bf16, void* stream) {
  if (bad_ptrs(g) || !scale || !sums || !gy_bf16)
    return set_error(MHD_E_ARG, "mhd_cnn_project_backward", "null argument");
  const int N = nx * ny * nz;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * 5, s);
  if (e != cudaSuccess) return set_error(MHD_E_CUDA, "mhd_cnn_project_backward", cudaGetErrorString(e));
  grad_sums_kernel<<<blocks(N), 256, 0, s>>>(cp8(g), N, sums);
  project_backward_kernel<<<blocks(N), 256, 0, s>>>(cp8(g), nx, ny, nz, f8(scale, 6), sums,
                                                    static_cast<__nv_bfloat16*>(gy_bf16));
  return check_launch("mhd_cnn_project_backward");
}

int mhd_correct(int nx, int ny, int nz, float* const s[8], const float* const d[8], float* scratch, int* nclip,
                void* stream) {
  if (!s || bad_ptrs(d) || !scratch) return set_error(MHD_E_ARG, "mhd_correct", "null argument");
  for (int q = 0; q < 8; q++)
    if (!s[q]) return set_error(MHD_E_ARG, "mhd_correct", "null field");
  const int N = nx * ny * nz;
  cudaStream_t st = (cudaStream_t)stream;
  const float* cs[8];
  for (int q = 0; q < 8; q++) cs[q] = s[q];
  thermal_kernel<<<blocks(N), 256, 0, st>>>(cp8(cs), nx, ny, nz, scratch);
  add_field_kernel<<<blocks(N), 256, 0, st>>>(p8(s), cp8(d), N);
  add_cells_kernel<<<blocks(N), 256, 0, st>>>(p8(s), cp8(d), nx, ny, nz, scratch, nclip);
  return check_launch("mhd_correct");
}

int mhd_adam(float* p, const float* g, float* m, float* v, int count, float lr, float beta1, float beta2, float eps,
             int step, void* stream) {
  if (!p || !g || !m || !v || count < 0 || step < 1) return set_error(MHD_E_ARG, "mhd_adam", "bad arguments");
  const float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<blocks(count), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, count, lr, beta1, beta2, eps, bc1, bc2);
  return check_launch("mhd_adam");
}

}  // extern "C"
