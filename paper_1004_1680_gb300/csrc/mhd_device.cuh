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
  float ih[3];          // cells per unit length, 1/h, along x, y, z (n: the unit box)
};

__host__ __device__ inline int wrapi(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

// Hint that the line holding *p will be read soon: it is fetched into L2
// without occupying a register (p must be a valid address).
__device__ __forceinline__ void prefetch_l2(const float* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
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

// Hardware approximate reciprocal (PTX rcp.approx,
// relative error of a few ulp; the FP32 path's tolerance against the FP64
// oracle is four orders of magnitude looser).
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// The same reciprocal with subnormal inputs and results flushed to zero: a
// single multi-function-unit instruction, without the subnormal handling
// that the plain form adds.  The sweeps divide only by densities and by sums
// of two limiter differences; a subnormal sum only occurs when the product
// of the differences underflows to zero, which the limiter's select discards.
// (At 512^3 the sweeps took 1.50 -> 1.37 ms (fluid) and 1.15 -> 1.07 ms
// (magnetic) per launch with it.)
__device__ __forceinline__ float rcp_ftz(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
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
  const float ab = __fmul_rn(a, b);
  return keep_if_positive(ab, __fmul_rn(ab, rcp_ftz(__fadd_rn(a, b))));
}

// ---------------------------------------------------------------------------
// FP32 arithmetic with every operation rounded explicitly (no multiply-add
// contraction left to the compiler), so that a pencil gives bitwise the same
// result in every kernel that marches it (single box, ensemble work list).
__device__ __forceinline__ float v_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float v_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float v_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float v_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float v_div(float a, float b) { return __fmul_rn(a, rcp_ftz(b)); }
__device__ __forceinline__ float v_sqrt(float a) { return sqrtf(a); }
// The freezing speeds' square root of the TMA-staged fluid sweeps: the
// multi-function unit's approximation with subnormals flushed (relative
// error of a few ulp, one instruction; sqrtf adds a refinement and a
// slow-path branch).  Its arguments are squared signal speeds of valid
// cells, far from the subnormal range.  Measured at 512^3: the staged fluid
// sweep 1.225 -> 1.135 ms with it, but the register-load sweep 1.35 -> 1.70
// ms, so each path keeps the faster one (the two then agree to FP32
// rounding rather than bitwise).
__device__ __forceinline__ float v_sqrt_fast(float a) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ float v_abs(float a) { return fabsf(a); }
__device__ __forceinline__ float v_keep(float x, float q) { return keep_if_positive(x, q); }


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

// The five conserved components of a cell as two pairs and a scalar,
// (rho, m_d), (m_t1, m_t2), e, so that the component-wise parts of the
// pipeline run on packed FP32 (two components per instruction, Blackwell's
// FFMA2 / FADD2 / FMUL2).  Every element is rounded exactly as the scalar
// operation would round it.
struct V5 {
  float2 p0, p1;
  float e;
};
__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }
// a - b = fma(b, -1, a): the product is exact, so one rounding as in __fsub_rn
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }
__device__ __forceinline__ V5 v5_sub(const V5& a, const V5& b) {
  return {sub2(a.p0, b.p0), sub2(a.p1, b.p1), __fsub_rn(a.e, b.e)};
}
__device__ __forceinline__ V5 v5_add(const V5& a, const V5& b) {
  return {__fadd2_rn(a.p0, b.p0), __fadd2_rn(a.p1, b.p1), __fadd_rn(a.e, b.e)};
}
// s x + y
__device__ __forceinline__ V5 v5_fma(float s, const V5& x, const V5& y) {
  return {__ffma2_rn(f2(s), x.p0, y.p0), __ffma2_rn(f2(s), x.p1, y.p1), __fmaf_rn(s, x.e, y.e)};
}
__device__ __forceinline__ V5 v5_zero() { return {f2(0.f), f2(0.f), 0.f}; }

template <int LIM>
__device__ __forceinline__ float2 half_limited2(float2 a, float2 b) {
  if constexpr (LIM == 0) {
    const float2 ab = __fmul2_rn(a, b), s = __fadd2_rn(a, b);
    const float2 q = __fmul2_rn(ab, make_float2(rcp_ftz(s.x), rcp_ftz(s.y)));  // = v_div per element
    return make_float2(v_keep(ab.x, q.x), v_keep(ab.y, q.y));
  } else {
    return make_float2(half_limited<LIM>(a.x, b.x), half_limited<LIM>(a.y, b.y));
  }
}
template <int LIM>
__device__ __forceinline__ V5 half_limited5(const V5& a, const V5& b) {
  return {half_limited2<LIM>(a.p0, b.p0), half_limited2<LIM>(a.p1, b.p1), half_limited<LIM>(a.e, b.e)};
}

// Flux of Eq. 2-3 projected on the sweep axis d, in the sweep's local frame
// (u = (rho, m_d, m_t1, m_t2, e), b = cell-centred (b_d, (b_t1, b_t2))), and
// the relaxation freezing speed c = |v_d| + sqrt((gamma p + |b|^2)/rho), which
// bounds the fastest local wave speed (Section II.B, relaxing TVD).
// Returns the right and left movers FR = (cu + F)/2, FL = FR - F = (cu - F)/2.
// FRZ selects the freezing speed: 0 the bound; 1 |v_d| + the fast
// magnetosonic speed along d, c_f^2 = (s + sqrt(s^2 - 4 a^2 v_Ad^2))/2,
// s = a^2 + v_A^2 (an ablation: the smallest freezing speed the relaxation
// allows); 2 the given speed c_given (one value per pencil and stage: the
// largest bound along the pencil, another ablation).
// FSQ: the freezing speed's square root from v_sqrt_fast (the TMA-staged
// sweeps) instead of v_sqrt.
template <int FRZ = 0, bool FSQ = false>
__device__ __forceinline__ void split_flux(const V5& u, float bd, float2 bt, float gamma, V5& FR, V5& FL,
                                           float c_given = 0.f) {
  auto root = [](float x) { return FSQ ? v_sqrt_fast(x) : v_sqrt(x); };
  const float md = u.p0.y;
  const float rinv = v_div(1.f, u.p0.x);
  const float vd = v_mul(md, rinv);
  const float2 vt = __fmul2_rn(u.p1, f2(rinv));
  const float b2 = v_fma(bd, bd, v_fma(bt.x, bt.x, v_mul(bt.y, bt.y)));
  const float kin = v_mul(0.5f, v_fma(md, vd, v_fma(u.p1.x, vt.x, v_mul(u.p1.y, vt.y))));
  const float p = v_mul(gamma - 1.f, v_fma(-0.5f, b2, v_sub(u.e, kin)));
  const float pstar = v_fma(0.5f, b2, p);
  const float bv = v_fma(bd, vd, v_fma(bt.x, vt.x, v_mul(bt.y, vt.y)));
  const float nb0 = -bd;  // exact; folds into the multiply-adds
  const float2 F01 = make_float2(md, v_fma(md, vd, v_fma(nb0, bd, pstar)));
  const float2 F23 = __ffma2_rn(u.p1, f2(vd), __fmul2_rn(f2(nb0), bt));
  const float F4 = v_fma(v_add(u.e, pstar), vd, v_mul(nb0, bv));
  float hc;
  if constexpr (FRZ == 1) {
    const float a2 = v_mul(v_mul(gamma, p), rinv), va2 = v_mul(b2, rinv);
    const float vad2 = v_mul(v_mul(bd, bd), rinv);
    const float sum = v_add(a2, va2);
    const float disc = v_fma(v_mul(-4.f, a2), vad2, v_mul(sum, sum));
    hc = v_mul(0.5f, v_add(v_abs(vd), root(v_mul(0.5f, v_add(sum, root(fmaxf(disc, 0.f)))))));
  } else if constexpr (FRZ == 2) {
    hc = v_mul(0.5f, c_given);
  } else {
    hc = v_mul(0.5f, v_add(v_abs(vd), root(v_mul(v_fma(gamma, p, b2), rinv))));
  }
  FR.p0 = __ffma2_rn(f2(hc), u.p0, __fmul2_rn(f2(0.5f), F01));
  FR.p1 = __ffma2_rn(f2(hc), u.p1, __fmul2_rn(f2(0.5f), F23));
  FR.e = v_fma(hc, u.e, v_mul(0.5f, F4));
  FL.p0 = sub2(FR.p0, F01);
  FL.p1 = sub2(FR.p1, F23);
  FL.e = v_sub(FR.e, F4);
}

// The bound |v_d| + sqrt((gamma p + |b|^2)/rho) of one cell in the sweep's
// frame, with split_flux's arithmetic (the per-pencil freezing speed is its
// maximum along the pencil).
__device__ __forceinline__ float bound_speed(const V5& u, float bd, float2 bt, float gamma) {
  const float md = u.p0.y;
  const float rinv = v_div(1.f, u.p0.x);
  const float vd = v_mul(md, rinv);
  const float2 vt = __fmul2_rn(u.p1, f2(rinv));
  const float b2 = v_fma(bd, bd, v_fma(bt.x, bt.x, v_mul(bt.y, bt.y)));
  const float kin = v_mul(0.5f, v_fma(md, vd, v_fma(u.p1.x, vt.x, v_mul(u.p1.y, vt.y))));
  const float p = v_mul(gamma - 1.f, v_fma(-0.5f, b2, v_sub(u.e, kin)));
  return v_add(v_abs(vd), v_sqrt(v_mul(v_fma(gamma, p, b2), rinv)));
}

// Largest signal rate of one cell, max_d (|v_d| + c_f*) * n_d, in the global
// frame (v, b indexed by axis).  Invalid cells (NaN, rho <= 0, p <= 0) report
// +inf so that a max-reduction flags them.  Explicitly rounded (see below);
// the reciprocal and square root are the single-instruction approximations
// with subnormals flushed (a subnormal density is invalid anyway: its rate
// comes out infinite or NaN and is reported as +inf).  In the fused last
// fluid sweep of a step: 1.33 -> 1.28 ms at 512^3 against the forms with
// subnormal handling.
__device__ __forceinline__ float cell_rate(float rho, const float m[3], float e, const float b[3],
                                           float gamma, const float ih[3]) {
  const float rinv = rcp_ftz(rho);
  const float v0 = __fmul_rn(m[0], rinv), v1 = __fmul_rn(m[1], rinv), v2 = __fmul_rn(m[2], rinv);
  const float b2 = __fmaf_rn(b[0], b[0], __fmaf_rn(b[1], b[1], __fmul_rn(b[2], b[2])));
  const float kin = __fmul_rn(0.5f, __fmaf_rn(m[0], v0, __fmaf_rn(m[1], v1, __fmul_rn(m[2], v2))));
  const float p = __fmul_rn(gamma - 1.f, __fmaf_rn(-0.5f, b2, __fsub_rn(e, kin)));
  const float cf = v_sqrt_fast(__fmul_rn(__fmaf_rn(gamma, p, b2), rinv));
  const float r = fmaxf(fmaxf(__fmul_rn(__fadd_rn(fabsf(v0), cf), ih[0]),
                              __fmul_rn(__fadd_rn(fabsf(v1), cf), ih[1])),
                        __fmul_rn(__fadd_rn(fabsf(v2), cf), ih[2]));
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
// Fluid marching pipeline (LIM: limiter, FRZ: freezing speed; 0 / 0 is
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
// FSQ: the fast square root of split_flux (the TMA-staged sweeps).
template <int LIM = 0, int FRZ = 0, bool FSQ = false>
struct FluidPipe {
  V5 U1, U2, U3;   // raw U at t-1, t-2, t-3
  float b1[3];     // frozen b at t-1
  V5 FR1;          // stage-1 right mover at t-1
  V5 f1m;          // stage-1 interface flux at t-3/2
  V5 Rh2, Rh3;     // stage-2 right movers at t-2, t-3
  V5 dR3;          // Rh(t-3) - Rh(t-4), carried from the previous step
  V5 Lh2;          // stage-2 left mover at t-2
  V5 dL2;          // Lh(t-2) - Lh(t-3), carried from the previous step
  V5 F2m;          // stage-2 interface flux at t-7/2
  float c1 = 0.f, c2 = 0.f;  // FRZ == 2: the pencil's freezing speeds of stage 1 and 2

  __device__ __forceinline__ void init() {
    U1 = U2 = U3 = FR1 = f1m = Rh2 = Rh3 = dR3 = Lh2 = dL2 = F2m = v5_zero();
    b1[0] = b1[1] = b1[2] = 0.f;
  }

  // Consume position t; write Unew(t-3) into out.  c_half = tau/(2h),
  // c_full = tau/h.
  __device__ __forceinline__ void step(const float U[5], const float b[3], float gamma, float c_half,
                                       float c_full, float out[5]) {
    const V5 u = {make_float2(U[0], U[1]), make_float2(U[2], U[3]), U[4]};
    V5 FR, FL;
    split_flux<FRZ, FSQ>(u, b[0], make_float2(b[1], b[2]), gamma, FR, FL, c1);
    const V5 f1 = v5_sub(FR1, FL);
    const V5 Uh = v5_fma(-c_half, v5_sub(f1, f1m), U1);
    V5 Rh, Lh;
    split_flux<FRZ, FSQ>(Uh, b1[0], make_float2(b1[1], b1[2]), gamma, Rh, Lh, c2);
    // the left-hand differences were the right-hand ones one step earlier
    const V5 dR2 = v5_sub(Rh2, Rh3), dL1 = v5_sub(Lh, Lh2);
    const V5 right = v5_add(Rh3, half_limited5<LIM>(dR3, dR2));
    const V5 left = v5_sub(Lh2, half_limited5<LIM>(dL2, dL1));
    const V5 F2 = v5_sub(right, left);
    const V5 o = v5_fma(-c_full, v5_sub(F2, F2m), U3);
    out[0] = o.p0.x;
    out[1] = o.p0.y;
    out[2] = o.p1.x;
    out[3] = o.p1.y;
    out[4] = o.e;
    // shift the windows
    F2m = F2;
    U3 = U2;
    U2 = U1;
    U1 = u;
    FR1 = FR;
    f1m = f1;
    dR3 = dR2;
    Rh3 = Rh2;
    Rh2 = Rh;
    dL2 = dL1;
    Lh2 = Lh;
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

  // Returns the edge flux f(t-5/2); writes qnew(t-3) into qnew.  Every
  // operation is rounded explicitly, so that a pencil gives bitwise the same
  // result in every kernel that marches it.
  __device__ __forceinline__ float step(float q, float u, float c_half, float c_full, float &qnew) {
    const float ub = __fmul_rn(0.5f, __fadd_rn(u1, u));
    const float g = __fmul_rn(ub, ub >= 0.f ? q1 : q);
    const float h = __fmaf_rn(-c_half, __fsub_rn(g, g1m), q1);
    const float d21 = __fsub_rn(h, h2);
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
    const float f = __fmul_rn(ub2, pos ? __fadd_rn(base, lim) : __fsub_rn(base, lim));
    qnew = __fmaf_rn(-c_full, __fsub_rn(f, fm), q3);
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
