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

// ---------------------------------------------------------------------------
// FP32 arithmetic with every operation rounded explicitly (no multiply-add
// contraction left to the compiler), so that a pencil gives bitwise the same
// result in every kernel that marches it (single box, ensemble work list).
__device__ __forceinline__ float v_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float v_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float v_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float v_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float v_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float v_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ float v_abs(float a) { return fabsf(a); }
__device__ __forceinline__ float v_keep(float x, float q) { return keep_if_positive(x, q); }

template <class T>
__device__ __forceinline__ T v_const(float s);
template <>
__device__ __forceinline__ float v_const<float>(float s) { return s; }

// Half a slope limiter, phi(a,b)/2, of two neighbouring differences; 0
// unless they have the same sign.  LIM 0: van Leer, the limiter of Section
// II.B, phi = 2ab/(a+b) (a+b cannot vanish when ab > 0; otherwise the quotient
// is discarded by the select).  Ablations: LIM 1 minmod, phi = the difference
// of smaller magnitude; LIM 2 superbee, phi = sign(a) max(min(2|a|,|b|),
// min(|a|,2|b|)).
template <int LIM>
__device__ __forceinline__ float half_limited(float a, float b) {
  const float ab = v_mul(a, b);
  if constexpr (LIM == 1) {
    return v_keep(ab, v_mul(0.5f, fabsf(a) < fabsf(b) ? a : b));
  } else if constexpr (LIM == 2) {
    const float A = fabsf(a), B = fabsf(b);
    const float m = fmaxf(fminf(v_add(A, A), B), fminf(A, v_add(B, B)));
    return v_keep(ab, v_mul(0.5f, copysignf(m, a)));
  } else {
    return v_keep(ab, v_div(ab, v_add(a, b)));
  }
}

// Flux of Eq. 2-3 projected on the sweep axis d, in the sweep's local frame
// (u = (rho, m_d, m_t1, m_t2, e), b = cell-centred (b_d, b_t1, b_t2)), and the
// relaxation freezing speed c = |v_d| + sqrt((gamma p + |b|^2)/rho), which
// bounds the fastest local wave speed (Section II.B, relaxing TVD).
// Returns the right and left movers FR = (cu + F)/2, FL = FR - F = (cu - F)/2.
// FAST = true replaces the bound by |v_d| + the fast magnetosonic speed along
// d, c_f^2 = (s + sqrt(s^2 - 4 a^2 v_Ad^2))/2, s = a^2 + v_A^2 (an ablation:
// the smallest freezing speed the relaxation allows).
template <class T, bool FAST = false>
__device__ __forceinline__ void split_flux_t(const T u[5], const T b[3], float gamma, T FR[5], T FL[5]) {
  const T half = v_const<T>(0.5f);
  const T rinv = v_div(v_const<T>(1.f), u[0]);
  const T vd = v_mul(u[1], rinv), v1 = v_mul(u[2], rinv), v2 = v_mul(u[3], rinv);
  const T b2 = v_fma(b[0], b[0], v_fma(b[1], b[1], v_mul(b[2], b[2])));
  const T kin = v_mul(half, v_fma(u[1], vd, v_fma(u[2], v1, v_mul(u[3], v2))));
  const T p = v_mul(v_const<T>(gamma - 1.f), v_fma(v_const<T>(-0.5f), b2, v_sub(u[4], kin)));
  const T pstar = v_fma(half, b2, p);
  const T bv = v_fma(b[0], vd, v_fma(b[1], v1, v_mul(b[2], v2)));
  const T nb0 = -b[0];  // exact; folds into the multiply-adds
  T F[5];
  F[0] = u[1];
  F[1] = v_fma(u[1], vd, v_fma(nb0, b[0], pstar));
  F[2] = v_fma(u[2], vd, v_mul(nb0, b[1]));
  F[3] = v_fma(u[3], vd, v_mul(nb0, b[2]));
  F[4] = v_fma(v_add(u[4], pstar), vd, v_mul(nb0, bv));
  T cs;
  if constexpr (FAST) {
    const T a2 = v_mul(v_mul(v_const<T>(gamma), p), rinv), va2 = v_mul(b2, rinv);
    const T vad2 = v_mul(v_mul(b[0], b[0]), rinv);
    const T sum = v_add(a2, va2);
    const T disc = v_fma(v_mul(v_const<T>(-4.f), a2), vad2, v_mul(sum, sum));
    cs = v_sqrt(v_mul(half, v_add(sum, v_sqrt(fmaxf(disc, 0.f)))));
  } else {
    cs = v_sqrt(v_mul(v_fma(v_const<T>(gamma), p, b2), rinv));
  }
  const T c = v_add(v_abs(vd), cs);
  const T hc = v_mul(half, c);
#pragma unroll
  for (int q = 0; q < 5; q++) {
    FR[q] = v_fma(hc, u[q], v_mul(half, F[q]));
    FL[q] = v_sub(FR[q], F[q]);
  }
}

// Largest signal rate of one cell, max_d (|v_d| + c_f*) * n_d, in the global
// frame (v, b indexed by axis).  Invalid cells (NaN, rho <= 0, p <= 0) report
// +inf so that a max-reduction flags them.  Explicitly rounded (see below).
__device__ __forceinline__ float cell_rate(float rho, const float m[3], float e, const float b[3],
                                           float gamma, const int n[3]) {
  const float rinv = fast_rcp(rho);
  const float v0 = __fmul_rn(m[0], rinv), v1 = __fmul_rn(m[1], rinv), v2 = __fmul_rn(m[2], rinv);
  const float b2 = __fmaf_rn(b[0], b[0], __fmaf_rn(b[1], b[1], __fmul_rn(b[2], b[2])));
  const float kin = __fmul_rn(0.5f, __fmaf_rn(m[0], v0, __fmaf_rn(m[1], v1, __fmul_rn(m[2], v2))));
  const float p = __fmul_rn(gamma - 1.f, __fmaf_rn(-0.5f, b2, __fsub_rn(e, kin)));
  const float cf = fast_sqrt(__fmul_rn(__fmaf_rn(gamma, p, b2), rinv));
  const float r = fmaxf(fmaxf(__fmul_rn(__fadd_rn(fabsf(v0), cf), (float)n[0]),
                              __fmul_rn(__fadd_rn(fabsf(v1), cf), (float)n[1])),
                        __fmul_rn(__fadd_rn(fabsf(v2), cf), (float)n[2]));
  const bool ok = (rho > 0.f) && (p > 0.f) && (r <= 3.0e38f);
  return ok ? r : __int_as_float(0x7f800000);
}

// Optional pressure floor on a finished cell u = (rho, m_d, m_t1, m_t2, e)
// with cell-centred field b: e >= kinetic + magnetic + p_floor / (gamma - 1).
__device__ __forceinline__ float floored_energy(const float u[5], const float b[3], float gamma, float p_floor) {
  const float kin = __fdiv_rn(__fmul_rn(0.5f, __fmaf_rn(u[1], u[1], __fmaf_rn(u[2], u[2], __fmul_rn(u[3], u[3])))),
                              u[0]);
  const float mag = __fmul_rn(0.5f, __fmaf_rn(b[0], b[0], __fmaf_rn(b[1], b[1], __fmul_rn(b[2], b[2]))));
  return fmaxf(u[4], __fadd_rn(__fadd_rn(kin, mag), __fdiv_rn(p_floor, gamma - 1.f)));
}

// cell-centred field component: mean of two faces
__device__ __forceinline__ float face_mean(float lo, float hi) { return __fmul_rn(0.5f, __fadd_rn(lo, hi)); }

// ---------------------------------------------------------------------------
// Fluid marching pipeline (LIM: limiter, FAST: freezing speed; 0 / false is
// the paper's scheme).
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
template <class T, int LIM = 0, bool FAST = false>
struct FluidPipeT {
  T U1[5], U2[5], U3[5];  // raw U at t-1, t-2, t-3
  T b1[3];                // frozen b at t-1
  T FR1[5];               // stage-1 right mover at t-1
  T f1m[5];               // stage-1 interface flux at t-3/2
  T Rh2[5], Rh3[5];       // stage-2 right movers at t-2, t-3
  T dR3[5];                // Rh(t-3) - Rh(t-4), carried from the previous step
  T Lh2[5];                // stage-2 left mover at t-2
  T dL2[5];                // Lh(t-2) - Lh(t-3), carried from the previous step
  T F2m[5];               // stage-2 interface flux at t-7/2

  __device__ __forceinline__ void init() {
    const T z = v_const<T>(0.f);
#pragma unroll
    for (int q = 0; q < 5; q++) {
      U1[q] = U2[q] = U3[q] = FR1[q] = f1m[q] = z;
      Rh2[q] = Rh3[q] = dR3[q] = Lh2[q] = dL2[q] = F2m[q] = z;
    }
    b1[0] = b1[1] = b1[2] = z;
  }

  // Consume position t; write Unew(t-3) into out.  c_half = tau/(2h),
  // c_full = tau/h.
  __device__ __forceinline__ void step(const T U[5], const T b[3], float gamma, float c_half, float c_full,
                                       T out[5]) {
    T FR[5], FL[5];
    split_flux_t<T, FAST>(U, b, gamma, FR, FL);
    const T nch = v_const<T>(-c_half), ncf = v_const<T>(-c_full);
    T Uh[5], f1[5];
#pragma unroll
    for (int q = 0; q < 5; q++) {
      f1[q] = v_sub(FR1[q], FL[q]);
      Uh[q] = v_fma(nch, v_sub(f1[q], f1m[q]), U1[q]);
    }
    T Rh[5], Lh[5];
    split_flux_t<T, FAST>(Uh, b1, gamma, Rh, Lh);
#pragma unroll
    for (int q = 0; q < 5; q++) {
      // the left-hand differences were the right-hand ones one step earlier
      const T dR2 = v_sub(Rh2[q], Rh3[q]), dL1 = v_sub(Lh[q], Lh2[q]);
      const T right = v_add(Rh3[q], half_limited<LIM>(dR3[q], dR2));
      const T left = v_sub(Lh2[q], half_limited<LIM>(dL2[q], dL1));
      const T F2 = v_sub(right, left);
      out[q] = v_fma(ncf, v_sub(F2, F2m[q]), U3[q]);
      F2m[q] = F2;
      // shift the windows
      U3[q] = U2[q];
      U2[q] = U1[q];
      U1[q] = U[q];
      FR1[q] = FR[q];
      f1m[q] = f1[q];
      dR3[q] = dR2;
      Rh3[q] = Rh2[q];
      Rh2[q] = Rh[q];
      dL2[q] = dL1;
      Lh2[q] = Lh[q];
    }
    b1[0] = b[0];
    b1[1] = b[1];
    b1[2] = b[2];
  }
};
template <int LIM, bool FAST>
using FluidPipe = FluidPipeT<float, LIM, FAST>;

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
template <int LIM = 0>
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
    float lim;
    if constexpr (LIM == 0) {
      lim = vanleer_half(sa, sb);
    } else {
      lim = half_limited<LIM>(sa, sb);
    }
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
