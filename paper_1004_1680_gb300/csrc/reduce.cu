// Reductions over the whole box and device-side step control:
//   - CFL signal rate (Section II.B: the fastest wave may cross at most a
//     fraction `cfl` of a cell per sweep): per-cell rate, warp-shuffle max,
//     one atomicMax per warp on the float bits (rates are >= 0, so the
//     unsigned order of the bits is the float order; invalid cells are +inf).
//   - the per-step control kernel that turns the rate into the sweep step
//     on the device, so a run of many steps needs no host round trip;
//   - FP64 diagnostics: compensated (Neumaier) sums of the 8 fields, the
//     max |div b| and the min pressure, reduced in a fixed order (bitwise
//     reproducible).
#include <cfloat>

#include "mhd_device.cuh"
#include "mhd_launch.h"

namespace mhd {

// neighbour index +1 along an axis with periodic wrap
__device__ __forceinline__ long long up1(long long cell, int coord, int n, long long stride) {
  return coord + 1 < n ? cell + stride : cell - (long long)(n - 1) * stride;
}

__global__ void cfl_rate_kernel(const float* __restrict__ rho, const float* __restrict__ mx,
                                const float* __restrict__ my, const float* __restrict__ mz,
                                const float* __restrict__ en, const float* __restrict__ bx,
                                const float* __restrict__ by, const float* __restrict__ bz, Box box,
                                float gamma, unsigned* rate, CellRange r) {
  const long long N = (long long)box.n[0] * box.n[1] * box.n[2];
  float rmax = 0.f;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % box.n[0]);
    const int j = (int)((c / box.n[0]) % box.n[1]);
    const int k = (int)(c / box.stride[2]);
    if (i < r.lo[0] || i >= r.hi[0] || j < r.lo[1] || j >= r.hi[1] || k < r.lo[2] || k >= r.hi[2]) continue;
    float m[3] = {__ldg(mx + c), __ldg(my + c), __ldg(mz + c)};
    float b[3];
    b[0] = 0.5f * (__ldg(bx + c) + __ldg(bx + up1(c, i, box.n[0], box.stride[0])));
    b[1] = 0.5f * (__ldg(by + c) + __ldg(by + up1(c, j, box.n[1], box.stride[1])));
    b[2] = 0.5f * (__ldg(bz + c) + __ldg(bz + up1(c, k, box.n[2], box.stride[2])));
    rmax = fmaxf(rmax, cell_rate(__ldg(rho + c), m, __ldg(en + c), b, gamma, box.n));
  }
  for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(rate, __float_as_uint(rmax));
}

cudaError_t launch_cfl_rate(const float* const f[8], const Box& box, float gamma, unsigned* rate,
                            cudaStream_t s, const CellRange* range) {
  const long long N = (long long)box.n[0] * box.n[1] * box.n[2];
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  CellRange r;
  for (int d = 0; d < 3; d++) {
    r.lo[d] = range ? range->lo[d] : 0;
    r.hi[d] = range ? range->hi[d] : box.n[d];
  }
  cfl_rate_kernel<<<(unsigned)blocks, 256, 0, s>>>(f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7],
                                                   box, gamma, rate, r);
  return cudaGetLastError();
}

__global__ void step_control_kernel(const unsigned* rate_cur, unsigned* rate_next, float* tau,
                                    double* time, double cfl, double tau_host) {
  double t;
  if (cfl > 0.0) {
    const float r = __uint_as_float(*rate_cur);
    t = (r > 0.f && r <= FLT_MAX) ? cfl / (double)r : 0.0;  // invalid state: stand still
  } else {
    t = tau_host;
  }
  const float tf = (float)t;
  *tau = tf;
  *time += 2.0 * (double)tf;
  *rate_next = 0u;
}

cudaError_t launch_step_control(const unsigned* rate_cur, unsigned* rate_next, float* tau,
                                double* time, double cfl, double tau_host, cudaStream_t s) {
  step_control_kernel<<<1, 1, 0, s>>>(rate_cur, rate_next, tau, time, cfl, tau_host);
  return cudaGetLastError();
}

__global__ void ens_control_kernel(const unsigned* rate_cur, unsigned* rate_next, float* tau,
                                   double* time, int nbox, double cfl) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  const float r = __uint_as_float(rate_cur[b]);
  const double t = (r > 0.f && r <= FLT_MAX) ? cfl / (double)r : 0.0;  // invalid state: stand still
  const float tf = (float)t;
  tau[b] = tf;
  time[b] += 2.0 * (double)tf;
  rate_next[b] = 0u;
}

cudaError_t launch_ens_control(const unsigned* rate_cur, unsigned* rate_next, float* tau,
                               double* time, int nbox, double cfl, cudaStream_t s) {
  ens_control_kernel<<<(nbox + 127) / 128, 128, 0, s>>>(rate_cur, rate_next, tau, time, nbox, cfl);
  return cudaGetLastError();
}

__global__ void set_tau_kernel(float* tau, float value) { *tau = value; }

cudaError_t launch_set_tau(float* tau, double value, cudaStream_t s) {
  set_tau_kernel<<<1, 1, 0, s>>>(tau, (float)value);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 compensated sums (Neumaier): a value is the pair (s, c), total s + c.

struct KB {
  double s, c;
};

__device__ __forceinline__ void kb_add(KB& a, double x) {
  const double t = a.s + x;
  a.c += (fabs(a.s) >= fabs(x)) ? (a.s - t) + x : (x - t) + a.s;
  a.s = t;
}

__device__ __forceinline__ KB kb_merge(KB a, KB b) {
  const double t = a.s + b.s;
  const double err = (fabs(a.s) >= fabs(b.s)) ? (a.s - t) + b.s : (b.s - t) + a.s;
  return KB{t, a.c + b.c + err};
}

constexpr int kDiagThreads = 256;

__global__ void __launch_bounds__(kDiagThreads)
diag_partial_kernel(const float* __restrict__ rho, const float* __restrict__ mx,
                    const float* __restrict__ my, const float* __restrict__ mz,
                    const float* __restrict__ en, const float* __restrict__ bx,
                    const float* __restrict__ by, const float* __restrict__ bz, Box box,
                    double gamma, double* __restrict__ partial) {
  const float* f[8] = {rho, mx, my, mz, en, bx, by, bz};
  const long long N = (long long)box.n[0] * box.n[1] * box.n[2];
  KB acc[8];
#pragma unroll
  for (int q = 0; q < 8; q++) acc[q] = KB{0.0, 0.0};
  double divmax = 0.0, pmin = DBL_MAX;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % box.n[0]);
    const int j = (int)((c / box.n[0]) % box.n[1]);
    const int k = (int)(c / box.stride[2]);
    double v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      v[q] = (double)__ldg(f[q] + c);
      kb_add(acc[q], v[q]);
    }
    const double bxh = __ldg(bx + up1(c, i, box.n[0], box.stride[0]));
    const double byh = __ldg(by + up1(c, j, box.n[1], box.stride[1]));
    const double bzh = __ldg(bz + up1(c, k, box.n[2], box.stride[2]));
    const double div = (bxh - v[5]) * box.n[0] + (byh - v[6]) * box.n[1] + (bzh - v[7]) * box.n[2];
    divmax = fmax(divmax, fabs(div));
    const double b0 = 0.5 * (v[5] + bxh), b1 = 0.5 * (v[6] + byh), b2 = 0.5 * (v[7] + bzh);
    const double kin = 0.5 * (v[1] * v[1] + v[2] * v[2] + v[3] * v[3]) / v[0];
    const double p = (gamma - 1.0) * (v[4] - kin - 0.5 * (b0 * b0 + b1 * b1 + b2 * b2));
    pmin = fmin(pmin, p);
  }
  // fixed-order tree: warp shuffles, then warps in order
  __shared__ double sm[kDiagThreads / 32][kDiagSlots];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
      KB other{__shfl_down_sync(0xffffffffu, acc[q].s, o), __shfl_down_sync(0xffffffffu, acc[q].c, o)};
      acc[q] = kb_merge(acc[q], other);
    }
    divmax = fmax(divmax, __shfl_down_sync(0xffffffffu, divmax, o));
    pmin = fmin(pmin, __shfl_down_sync(0xffffffffu, pmin, o));
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
      sm[wid][2 * q] = acc[q].s;
      sm[wid][2 * q + 1] = acc[q].c;
    }
    sm[wid][16] = divmax;
    sm[wid][17] = pmin;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int q = threadIdx.x;
    KB t{sm[0][2 * q], sm[0][2 * q + 1]};
    for (int w = 1; w < kDiagThreads / 32; w++) t = kb_merge(t, KB{sm[w][2 * q], sm[w][2 * q + 1]});
    partial[(long long)blockIdx.x * kDiagSlots + 2 * q] = t.s;
    partial[(long long)blockIdx.x * kDiagSlots + 2 * q + 1] = t.c;
  } else if (threadIdx.x == 8) {
    double m = sm[0][16];
    for (int w = 1; w < kDiagThreads / 32; w++) m = fmax(m, sm[w][16]);
    partial[(long long)blockIdx.x * kDiagSlots + 16] = m;
  } else if (threadIdx.x == 9) {
    double m = sm[0][17];
    for (int w = 1; w < kDiagThreads / 32; w++) m = fmin(m, sm[w][17]);
    partial[(long long)blockIdx.x * kDiagSlots + 17] = m;
  }
}

__global__ void diag_final_kernel(const double* __restrict__ partial, int nblk, double hmin,
                                  double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q < 8) {
    KB t{0.0, 0.0};
    for (int b = 0; b < nblk; b++)
      t = kb_merge(t, KB{partial[(long long)b * kDiagSlots + 2 * q], partial[(long long)b * kDiagSlots + 2 * q + 1]});
    out[q] = t.s + t.c;
  } else if (q == 8) {
    double m = 0.0;
    for (int b = 0; b < nblk; b++) m = fmax(m, partial[(long long)b * kDiagSlots + 16]);
    out[8] = m * hmin;
  } else if (q == 9) {
    double m = DBL_MAX;
    for (int b = 0; b < nblk; b++) m = fmin(m, partial[(long long)b * kDiagSlots + 17]);
    out[9] = m;
  }
}

int diag_blocks(const Box& box) {
  const long long N = (long long)box.n[0] * box.n[1] * box.n[2];
  long long b = (N + 4LL * kDiagThreads - 1) / (4LL * kDiagThreads);
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_diagnostics(const float* const f[8], const Box& box, double gamma, double* partial,
                               double* out, cudaStream_t s) {
  const int nblk = diag_blocks(box);
  diag_partial_kernel<<<nblk, kDiagThreads, 0, s>>>(f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7],
                                                    box, gamma, partial);
  int nmax = box.n[0] > box.n[1] ? box.n[0] : box.n[1];
  nmax = nmax > box.n[2] ? nmax : box.n[2];
  diag_final_kernel<<<1, 32, 0, s>>>(partial, nblk, 1.0 / nmax, out);
  return cudaGetLastError();
}

}  // namespace mhd
