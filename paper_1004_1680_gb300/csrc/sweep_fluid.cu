// Relaxing-TVD fluid sweep along one axis (Section II.B, Eq. 6), FP32.
//
// One thread owns one pencil segment along the sweep axis D and marches along
// it with the FluidPipe of mhd_device.cuh: the 7-point stencil is evaluated
// once per cell, intermediate values live in registers, and each of the 8
// state fields is read once and each of the 5 conserved fields written once
// per cell (the two transverse face fields are also read one pencil over,
// which hits in cache).
//
// No transposes: for the y and z sweeps the 32 lanes of a warp are 32
// neighbouring pencils along x, so every load and store of a plane is a
// coalesced 128-byte row; for the x sweep each thread reads its own pencil in
// aligned 16-byte pieces (4 cells along x per load).
//
// The sweep writes out of place (in -> out): neighbouring threads read the
// transverse faces of this thread's pencil.
//
// With RATE = true the kernel also evaluates the CFL signal rate of every
// cell it writes (Section II.B: the next timestep) and folds the maximum into
// *rate with one atomicMax per warp, saving a separate pass over the state.
#include "mhd_device.cuh"
#include "mhd_launch.h"

namespace mhd {

template <int D>
struct Axes {
  // lane axis A (contiguous pencils across a warp), row axis O, transverse
  // axes of the local frame T1 = (D+1)%3, T2 = (D+2)%3
  static constexpr int A = (D == 0) ? 1 : 0;
  static constexpr int O = (D == 2) ? 1 : 2;
  static constexpr int T1 = (D + 1) % 3;
  static constexpr int T2 = (D + 2) % 3;
};

constexpr int kFluidWarps = 4;

template <int D, bool RATE>
__global__ void __launch_bounds__(32 * kFluidWarps)
fluid_sweep_kernel(FluidArgs a) {
  using X = Axes<D>;
  const int lane = threadIdx.x;
  const int nA = a.box.n[X::A], nO = a.box.n[X::O], nD = a.box.n[D];
  const int pa = blockIdx.x * 32 + lane;
  const int pb = blockIdx.y * kFluidWarps + threadIdx.y;
  const bool active = (pa < nA) && (pb < nO);
  const int ia = min(pa, nA - 1), ib = min(pb, nO - 1);
  const long long sA = a.box.stride[X::A], sO = a.box.stride[X::O], sD = a.box.stride[D];
  const long long base = ia * sA + ib * sO;
  const long long baseA1 = wrapi(ia + 1, nA) * sA + ib * sO;  // pencil +1 along A
  const long long baseO1 = ia * sA + wrapi(ib + 1, nO) * sO;  // pencil +1 along O
  // +1 along the local-frame transverse axes
  const long long baseT1 = (X::T1 == X::A) ? baseA1 : baseO1;
  const long long baseT2 = (X::T2 == X::A) ? baseA1 : baseO1;

  const float* __restrict__ rho = a.in[RHO];
  const float* __restrict__ md = a.in[MX + D];
  const float* __restrict__ m1 = a.in[MX + X::T1];
  const float* __restrict__ m2 = a.in[MX + X::T2];
  const float* __restrict__ en = a.in[EN];
  const float* __restrict__ bd = a.in[BX + D];
  const float* __restrict__ b1 = a.in[BX + X::T1];
  const float* __restrict__ b2 = a.in[BX + X::T2];
  float* __restrict__ o_rho = a.out[RHO];
  float* __restrict__ o_md = a.out[MX + D];
  float* __restrict__ o_m1 = a.out[MX + X::T1];
  float* __restrict__ o_m2 = a.out[MX + X::T2];
  float* __restrict__ o_en = a.out[EN];

  const float gamma = a.gamma;
  const float tau = *a.tau;
  const float c_full = tau * (float)nD;  // tau / h_D
  const float c_half = 0.5f * c_full;    // tau / (2 h_D)
  const int s0 = blockIdx.z * a.seg;
  const int s1 = s0 + a.seg;
  // positions s0-4 .. s1+2 feed outputs s0 .. s1-1 (3 cells of lag, 1 extra
  // warm-up cell so that x chunks start 16-byte aligned)
  const int nchunk = (a.seg + 7 + 3) / 4;

  FluidPipe pipe;
  pipe.init();
  float bc2[3] = {0.f, 0.f, 0.f}, bc3[3] = {0.f, 0.f, 0.f};  // b_c at t-2, t-3 (RATE only)
  float rmax = 0.f;

  for (int c = 0; c < nchunk; c++) {
    const int p0 = s0 - 4 + 4 * c;        // first position of this chunk
    const int pw = wrapi(p0, nD);          // its periodic image (multiple of 4)
    float U[4][5], B[4][3], bdn[5], t1n[4], t2n[4];
    if (D == 0) {
      // 16-byte loads along x: 4 consecutive cells of this pencil
      const long long cx = base + pw;
      float4 v;
#define LD4(dst, ptr, off)                                   \
  v = __ldg(reinterpret_cast<const float4*>((ptr) + (off))); \
  dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
      float t0[4], t1[4], t2[4], t3[4], t4[4], tb1[4], tb2[4];
      LD4(t0, rho, cx) LD4(t1, md, cx) LD4(t2, m1, cx) LD4(t3, m2, cx) LD4(t4, en, cx)
      LD4(bdn, bd, cx) LD4(tb1, b1, cx) LD4(tb2, b2, cx)
      LD4(t1n, b1, baseT1 + pw) LD4(t2n, b2, baseT2 + pw)
#undef LD4
      bdn[4] = __ldg(bd + base + wrapi(p0 + 4, nD));
#pragma unroll
      for (int j = 0; j < 4; j++) {
        U[j][0] = t0[j]; U[j][1] = t1[j]; U[j][2] = t2[j]; U[j][3] = t3[j]; U[j][4] = t4[j];
        B[j][1] = tb1[j]; B[j][2] = tb2[j];
      }
    } else {
      // one coalesced row per plane
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const long long off = (long long)wrapi(p0 + j, nD) * sD;
        U[j][0] = __ldg(rho + base + off);
        U[j][1] = __ldg(md + base + off);
        U[j][2] = __ldg(m1 + base + off);
        U[j][3] = __ldg(m2 + base + off);
        U[j][4] = __ldg(en + base + off);
        bdn[j] = __ldg(bd + base + off);
        B[j][1] = __ldg(b1 + base + off);
        B[j][2] = __ldg(b2 + base + off);
        t1n[j] = __ldg(b1 + baseT1 + off);
        t2n[j] = __ldg(b2 + baseT2 + off);
      }
      bdn[4] = __ldg(bd + base + (long long)wrapi(p0 + 4, nD) * sD);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      // cell-centred field: mean of the low and high face of the cell
      B[j][0] = 0.5f * (bdn[j] + bdn[j + 1]);
      B[j][1] = 0.5f * (B[j][1] + t1n[j]);
      B[j][2] = 0.5f * (B[j][2] + t2n[j]);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float o[5];
      const float bprev0 = pipe.b1[0], bprev1 = pipe.b1[1], bprev2 = pipe.b1[2];  // b_c(t-1)
      pipe.step(U[j], B[j], gamma, c_half, c_full, o);
      const int t = p0 + j;
      const int po = t - 3;  // position of the finished cell
      if (active && po >= s0 && po < s1) {
        const long long cell = base + (long long)wrapi(po, nD) * sD;
        o_rho[cell] = o[0];
        o_md[cell] = o[1];
        o_m1[cell] = o[2];
        o_m2[cell] = o[3];
        o_en[cell] = o[4];
        if (RATE) {
          float m[3], bg[3];
          m[D] = o[1]; m[X::T1] = o[2]; m[X::T2] = o[3];
          bg[D] = bc3[0]; bg[X::T1] = bc3[1]; bg[X::T2] = bc3[2];
          rmax = fmaxf(rmax, cell_rate(o[0], m, o[4], bg, gamma, a.box.n));
        }
      }
      if (RATE) {  // window of b_c: bc2 = b_c(t-1), bc3 = b_c(t-2) for the next step
        bc3[0] = bc2[0]; bc3[1] = bc2[1]; bc3[2] = bc2[2];
        bc2[0] = bprev0; bc2[1] = bprev1; bc2[2] = bprev2;
      }
    }
  }
  if (RATE) {
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if (lane == 0) atomicMax(a.rate, __float_as_uint(rmax));
  }
}

}  // namespace mhd

namespace mhd {

cudaError_t launch_fluid(int axis, bool rate, const FluidArgs& a, cudaStream_t s) {
  const int A = (axis == 0) ? 1 : 0, O = (axis == 2) ? 1 : 2;
  dim3 block(32, kFluidWarps);
  dim3 grid((a.box.n[A] + 31) / 32, (a.box.n[O] + kFluidWarps - 1) / kFluidWarps,
            a.box.n[axis] / a.seg);
  switch (axis * 2 + (rate ? 1 : 0)) {
    case 0: fluid_sweep_kernel<0, false><<<grid, block, 0, s>>>(a); break;
    case 1: fluid_sweep_kernel<0, true><<<grid, block, 0, s>>>(a); break;
    case 2: fluid_sweep_kernel<1, false><<<grid, block, 0, s>>>(a); break;
    case 3: fluid_sweep_kernel<1, true><<<grid, block, 0, s>>>(a); break;
    case 4: fluid_sweep_kernel<2, false><<<grid, block, 0, s>>>(a); break;
    default: fluid_sweep_kernel<2, true><<<grid, block, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace mhd
