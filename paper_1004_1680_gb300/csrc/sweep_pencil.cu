// Ablation of the paper's per-cell freezing speed: one speed per pencil and
// Runge-Kutta stage, the largest bound |v_d| + sqrt((gamma p + |b|^2)/rho)
// along the pencil (the classical global choice of relaxing TVD schemes,
// applied pencil by pencil).  The first stage's speed is the maximum over the
// state U; the second stage's over the stage-1 half-step state built with the
// first.  Both need the whole pencil before its first flux, so a reduction
// kernel (one thread marching one whole pencil, lanes along the coalesced
// axis) runs before the sweep, and the sweep (FRZ = 2) reads the two values.
#include "sweep_fluid.cuh"

namespace mhd {

template cudaError_t launch_fluid_t<0, 2>(int, bool, const FluidArgs&, cudaStream_t);

template <int D>
__global__ void __launch_bounds__(128) pencil_speed_kernel(FluidArgs a, float* __restrict__ c) {
  using X = Axes<D>;
  const Box& box = a.box;
  const int nA = box.n[X::A], nO = box.n[X::O], nD = box.n[D];
  const int pa = blockIdx.x * 32 + threadIdx.x, pb = blockIdx.y * 4 + threadIdx.y;
  if (pa >= nA || pb >= nO) return;
  const long long sA = box.stride[X::A], sO = box.stride[X::O], sD = box.stride[D];
  const long long base = pa * sA + pb * sO;
  const long long baseA1 = wrapi(pa + 1, nA) * sA + pb * sO, baseO1 = pa * sA + wrapi(pb + 1, nO) * sO;
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
  const float gamma = a.gamma;
  const float c_half = 0.5f * (__ldg(a.tau) * a.box.ih[D]);  // tau / (2 h_D), as in the sweep

  // state and cell-centred field of position i of the pencil (periodic), in
  // the sweep's local frame
  auto cell = [&](int i, V5& u, float& bdc, float2& bt) {
    const long long o = wrapi(i, nD) * sD, o1 = wrapi(i + 1, nD) * sD;
    u.p0 = make_float2(__ldg(rho + base + o), __ldg(md + base + o));
    u.p1 = make_float2(__ldg(m1 + base + o), __ldg(m2 + base + o));
    u.e = __ldg(en + base + o);
    bdc = face_mean(__ldg(bd + base + o), __ldg(bd + base + o1));
    bt = make_float2(face_mean(__ldg(b1 + base + o), __ldg(b1 + baseT1 + o)),
                     face_mean(__ldg(b2 + base + o), __ldg(b2 + baseT2 + o)));
  };

  float c1 = 0.f;
  for (int i = 0; i < nD; i++) {
    V5 u;
    float bdc;
    float2 bt;
    cell(i, u, bdc, bt);
    c1 = fmaxf(c1, bound_speed(u, bdc, bt, gamma));
  }
  // stage 1 with c1, as the sweep computes it: at position t the interface
  // flux f(t-1/2) = FR(t-1) - FL(t) and the half-step state
  // Uh(t-1) = U(t-1) - tau/(2h) (f(t-1/2) - f(t-3/2))
  float c2 = 0.f;
  V5 Uprev = v5_zero(), FRprev = v5_zero(), fprev = v5_zero();
  float bdprev = 0.f;
  float2 btprev = make_float2(0.f, 0.f);
  for (int t = -2; t <= nD; t++) {
    V5 u, FR, FL;
    float bdc;
    float2 bt;
    cell(t, u, bdc, bt);
    split_flux<2>(u, bdc, bt, gamma, FR, FL, c1);
    if (t >= -1) {
      const V5 f = v5_sub(FRprev, FL);
      if (t >= 1) c2 = fmaxf(c2, bound_speed(v5_fma(-c_half, v5_sub(f, fprev), Uprev), bdprev, btprev, gamma));
      fprev = f;
    }
    FRprev = FR;
    Uprev = u;
    bdprev = bdc;
    btprev = bt;
  }
  const long long pc = (long long)pb * nA + pa;
  c[pc] = c1;
  c[(long long)nA * nO + pc] = c2;
}

cudaError_t launch_pencil_speeds(int axis, const FluidArgs& a, float* c, cudaStream_t s) {
  const int A = (axis == 0) ? 1 : 0, O = (axis == 2) ? 1 : 2;
  const dim3 block(32, 4), grid((a.box.n[A] + 31) / 32, (a.box.n[O] + 3) / 4);
  if (axis == 0) pencil_speed_kernel<0><<<grid, block, 0, s>>>(a, c);
  if (axis == 1) pencil_speed_kernel<1><<<grid, block, 0, s>>>(a, c);
  if (axis == 2) pencil_speed_kernel<2><<<grid, block, 0, s>>>(a, c);
  return cudaGetLastError();
}

}  // namespace mhd
