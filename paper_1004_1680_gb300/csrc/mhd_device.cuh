// Device-side building blocks of the FP32 sweep kernels: field indexing, the
// projected MHD flux with the relaxation freezing speed, the van Leer limiter,
// and the two marching pipelines (fluid and magnetic) that carry every
// intermediate value of the 2-stage Runge-Kutta update in registers while a
// thread walks along its pencil.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mhd {

enum Field { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BX = 5, BY = 6, BZ = 7 };

// Geometry of a box as the kernels see it.
struct Box {
  int n[3];             // cells along x, y, z
  long long stride[3];  // flat-index stride of a unit step along x, y, z
};

__host__ __device__ inline int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Periodic image of a position within one period of [0, n) (SMALL = false,
// valid for n >= 16) or anywhere (SMALL = true).  Branch-free, so the loads
// of a whole chunk can be issued before the first one is used.
template <bool SMALL>
__device__ __forceinline__ int wrap_near(int i, int n) {
  if constexpr (SMALL) {
    return wrapi(i, n);
  } else {
    i = i < 0 ? i + n : i;
    return i >= n ? i - n : i;
  }
}

// Hardware approximate reciprocal and square root (PTX rcp.approx / sqrt.approx,
// relative error of a few ulp; the FP32 path's tolerance against the FP64
// oracle is four orders of magnitude looser).
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float fast_sqrt(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// x > 0 ? q : 0 as a predicated select (never a branch): q is computed by
// the caller unconditionally, so a limiter costs no control flow.
__device__ __forceinline__ float keep_if_positive(float x, float q) {
  float r;
  asm("{\n\t.reg .pred p;\n\tsetp.gt.f32 p, %1, 0f00000000;\n\tselp.f32 %0, %2, 0f00000000, p;\n\t}"
      : "=f"(r)
      : "f"(x), "f"(q));
  return r;
}

// Half the van Leer limiter of Section II.B: phi(a,b)/2 = ab/(a+b) when a and
// b have the same sign, else 0 (a+b cannot vanish when ab > 0).  The
// second-order correction adds phi/2 to the upwind value.
__device__ __forceinline__ float vanleer_half(float a, float b) {
  const float ab = a * b;
  return keep_if_positive(ab, ab * fast_rcp(a + b));
}

// van Leer limiter of Section II.B: 2ab/(a+b) when a and b have the same
// sign, else 0 (a+b cannot vanish when ab > 0; otherwise the quotient is
// discarded by the select).
__device__ __forceinline__ float vanleer(float a, float b) {
  const float ab = a * b;
  return keep_if_positive(ab, __fdividef(2.f * ab, a + b));
}

// Flux of Eq. 2-3 projected on the sweep axis d, in the sweep's local frame
// (u = (rho, m_d, m_t1, m_t2, e), b = cell-centred (b_d, b_t1, b_t2)), and the
// relaxation freezing speed c = |v_d| + sqrt((gamma p + |b|^2)/rho), which
// bounds the fastest local wave speed (Section II.B, relaxing TVD).
// Returns the right and left movers FR = (cu + F)/2, FL = (cu - F)/2.
__device__ __forceinline__ void split_flux(const float u[5], const float b[3], float gamma,
                                           float FR[5], float FL[5]) {
  float rinv = __fdividef(1.f, u[0]);
  float vd = u[1] * rinv, v1 = u[2] * rinv, v2 = u[3] * rinv;
  float b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  float kin = 0.5f * (u[1] * vd + u[2] * v1 + u[3] * v2);
  float p = (gamma - 1.f) * (u[4] - kin - 0.5f * b2);
  float pstar = p + 0.5f * b2;
  float bv = b[0] * vd + b[1] * v1 + b[2] * v2;
  float F[5];
  F[0] = u[1];
  F[1] = u[1] * vd + pstar - b[0] * b[0];
  F[2] = u[2] * vd - b[0] * b[1];
  F[3] = u[3] * vd - b[0] * b[2];
  F[4] = (u[4] + pstar) * vd - b[0] * bv;
  float c = fabsf(vd) + sqrtf((gamma * p + b2) * rinv);
#pragma unroll
  for (int q = 0; q < 5; q++) {
    float cu = c * u[q];
    FR[q] = 0.5f * (cu + F[q]);
    FL[q] = 0.5f * (cu - F[q]);
  }
}

// Largest signal rate of one cell, max_d (|v_d| + c_f*) * n_d, in the global
// frame (v, b indexed by axis).  Invalid cells (NaN, rho <= 0, p <= 0) report
// +inf so that a max-reduction flags them.
__device__ __forceinline__ float cell_rate(float rho, const float m[3], float e, const float b[3],
                                           float gamma, const int n[3]) {
  float rinv = fast_rcp(rho);
  float v0 = m[0] * rinv, v1 = m[1] * rinv, v2 = m[2] * rinv;
  float b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  float kin = 0.5f * (m[0] * v0 + m[1] * v1 + m[2] * v2);
  float p = (gamma - 1.f) * (e - kin - 0.5f * b2);
  float cf = fast_sqrt((gamma * p + b2) * rinv);
  float r = fmaxf(fmaxf((fabsf(v0) + cf) * n[0], (fabsf(v1) + cf) * n[1]), (fabsf(v2) + cf) * n[2]);
  bool ok = (rho > 0.f) && (p > 0.f) && (r <= 3.0e38f);
  return ok ? r : __int_as_float(0x7f800000);
}

// ---------------------------------------------------------------------------
// Fluid marching pipeline.
//
// A thread walks its periodic pencil one position t at a time, receiving the
// raw state U_t and the frozen cell-centred field b_t.  At step t it forms
//   stage 1:  flux1(t-1/2) = FR(t-1) - FL(t)              (first-order upwind)
//             Uh(t-1)      = U(t-1) - tau/(2h) (flux1(t-1/2) - flux1(t-3/2))
//   stage 2:  FRh, FLh from Uh(t-1)
//             F2(t-5/2)    = [FRh(t-3) + phi(dR)/2] - [FLh(t-2) - phi(dL)/2]
//             Unew(t-3)    = U(t-3) - tau/h (F2(t-5/2) - F2(t-7/2))
// so Unew at position t-3 is produced at step t (the 7-point stencil of
// Section II.B).  Every intermediate value is held in registers.
struct FluidPipe {
  float U1[5], U2[5], U3[5];  // raw U at t-1, t-2, t-3
  float b1[3];                // frozen b at t-1
  float FR1[5];               // stage-1 right mover at t-1
  float f1m[5];               // stage-1 interface flux at t-3/2
  float Rh2[5], Rh3[5], Rh4[5];  // stage-2 right movers at t-2, t-3, t-4
  float Lh2[5], Lh3[5];          // stage-2 left movers at t-2, t-3
  float F2m[5];               // stage-2 interface flux at t-7/2

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int q = 0; q < 5; q++) {
      U1[q] = U2[q] = U3[q] = FR1[q] = f1m[q] = 0.f;
      Rh2[q] = Rh3[q] = Rh4[q] = Lh2[q] = Lh3[q] = F2m[q] = 0.f;
    }
    b1[0] = b1[1] = b1[2] = 0.f;
  }

  // Consume position t; write Unew(t-3) into out.  c_half = tau/(2h),
  // c_full = tau/h.
  __device__ __forceinline__ void step(const float U[5], const float b[3], float gamma,
                                       float c_half, float c_full, float out[5]) {
    float FR[5], FL[5];
    split_flux(U, b, gamma, FR, FL);
    float Uh[5], f1[5];
#pragma unroll
    for (int q = 0; q < 5; q++) {
      f1[q] = FR1[q] - FL[q];
      Uh[q] = U1[q] - c_half * (f1[q] - f1m[q]);
    }
    float Rh[5], Lh[5];
    split_flux(Uh, b1, gamma, Rh, Lh);
#pragma unroll
    for (int q = 0; q < 5; q++) {
      float right = Rh3[q] + 0.5f * vanleer(Rh3[q] - Rh4[q], Rh2[q] - Rh3[q]);
      float left = Lh2[q] - 0.5f * vanleer(Lh2[q] - Lh3[q], Lh[q] - Lh2[q]);
      float F2 = right - left;
      out[q] = U3[q] - c_full * (F2 - F2m[q]);
      F2m[q] = F2;
      // shift the windows
      U3[q] = U2[q];
      U2[q] = U1[q];
      U1[q] = U[q];
      FR1[q] = FR[q];
      f1m[q] = f1[q];
      Rh4[q] = Rh3[q];
      Rh3[q] = Rh2[q];
      Rh2[q] = Rh[q];
      Lh3[q] = Lh2[q];
      Lh2[q] = Lh[q];
    }
    b1[0] = b[0];
    b1[1] = b[1];
    b1[2] = b[2];
  }
};

// ---------------------------------------------------------------------------
// Magnetic advection pipeline for one transverse component q = b_t along the
// sweep axis (Section II.B, advection-constraint step).  Input per position:
// q_t and the face velocity u_t (v_d averaged to the b_t face).  At step t:
//   ubar(t-1/2) = (u(t-1) + u(t))/2                       (edge velocity)
//   g(t-1/2)    = ubar * q_upwind                        (first-order flux)
//   qh(t-1)     = q(t-1) - tau/(2h) (g(t-1/2) - g(t-3/2))
//   f(t-5/2)    = ubar(t-5/2) * (qh_up +- phi(dqh-, dqh+)/2)  (van Leer)
//   qnew(t-3)   = q(t-3) - tau/h (f(t-5/2) - f(t-7/2))
// f(t-5/2) is the edge flux handed to the constraint on b_d.
struct MagPipe {
  float q1, q2, q3;   // q at t-1, t-2, t-3
  float u1;           // face velocity at t-1
  float g1m;          // first-order flux at t-3/2
  float h2, h3;       // qh at t-2, t-3
  float d32, d43;     // qh(t-2) - qh(t-3), qh(t-3) - qh(t-4)
  float ub1, ub2;     // ubar at t-3/2, t-5/2
  float fm;           // edge flux at t-7/2

  __device__ __forceinline__ void init() {
    q1 = q2 = q3 = u1 = g1m = h2 = h3 = d32 = d43 = ub1 = ub2 = fm = 0.f;
  }

  // Returns the edge flux f(t-5/2); writes qnew(t-3) into qnew.
  __device__ __forceinline__ float step(float q, float u, float c_half, float c_full, float &qnew) {
    const float ub = 0.5f * (u1 + u);
    const float g = ub * (ub >= 0.f ? q1 : q);
    const float h = q1 - c_half * (g - g1m);
    const float d21 = h - h2;
    // upwind cell t-3 (ubar >= 0) or t-2, plus half its limited slope
    const bool pos = ub2 >= 0.f;
    const float base = pos ? h3 : h2;
    const float sa = pos ? d43 : d32;
    const float sb = pos ? d32 : d21;
    const float lim = vanleer_half(sa, sb);
    const float f = ub2 * (pos ? base + lim : base - lim);
    qnew = q3 - c_full * (f - fm);
    fm = f;
    q3 = q2;
    q2 = q1;
    q1 = q;
    u1 = u;
    g1m = g;
    d43 = d32;
    d32 = d21;
    h3 = h2;
    h2 = h;
    ub2 = ub1;
    ub1 = ub;
    return f;
  }
};

}  // namespace mhd
