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

__global__ void cfl_rate_kernel(const float* __restrict__ rho, const float* __restrict__ mx,
                                const float* __restrict__ my, const float* __restrict__ mz,
                                const float* __restrict__ en, const float* __restrict__ bx,
                                const float* __restrict__ by, const float* __restrict__ bz, Box box,
                                float gamma, unsigned* rate, CellRange r) {
  // a warp walks whole x rows, 32 cells at a time; rows are stepped without
  // a division per row or cell (64-bit integer division is emulated)
  const int nx = box.n[0], ny = box.n[1], nz = box.n[2];
  const int lane = threadIdx.x & 31;
  const long long rows = (long long)ny * nz;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int j = (int)(row % ny);
  long long k = row / ny;
  const int dj = (int)(nwarps % ny);
  const long long dk = nwarps / ny;
  float rmax = 0.f;
  for (; row < rows; row += nwarps) {
    if (j >= r.lo[1] && j < r.hi[1] && k >= r.lo[2] && k < r.hi[2]) {
      const long long rowbase = j * box.stride[1] + k * box.stride[2];
      const long long yoff = (j + 1 < ny) ? box.stride[1] : -(long long)(ny - 1) * box.stride[1];
      const long long zoff = (k + 1 < nz) ? box.stride[2] : -(long long)(nz - 1) * box.stride[2];
      for (int i = r.lo[0] + lane; i < r.hi[0]; i += 32) {
        const long long c = rowbase + i;  // x is the contiguous axis (checked at launch)
        float m[3] = {__ldg(mx + c), __ldg(my + c), __ldg(mz + c)};
        float b[3];
        b[0] = 0.5f * (__ldg(bx + c) + __ldg(bx + (i + 1 < nx ? c + 1 : c - (nx - 1))));
        b[1] = 0.5f * (__ldg(by + c) + __ldg(by + c + yoff));
        b[2] = 0.5f * (__ldg(bz + c) + __ldg(bz + c + zoff));
        rmax = fmaxf(rmax, cell_rate(__ldg(rho + c), m, __ldg(en + c), b, gamma, box.ih));
      }
    }
    j += dj;
    k += dk;
    if (j >= ny) {
      j -= ny;
      k++;
    }
  }
  for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if (lane == 0) atomicMax(rate, __float_as_uint(rmax));
}

cudaError_t launch_cfl_rate(const float* const f[8], const Box& box, float gamma, unsigned* rate,
                            cudaStream_t s, const CellRange* range) {
  if (box.stride[0] != 1) return cudaErrorInvalidValue;
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

__device__ __forceinline__ KB kb_merge(KB a, KB b) {
  const double t = a.s + b.s;
  const double err = (fabs(a.s) >= fabs(b.s)) ? (a.s - t) + b.s : (b.s - t) + a.s;
  return KB{t, a.c + b.c + err};
}

constexpr int kDiagThreads = 256;

// Error-free FP32 transformations (Knuth's TwoSum; the FMA product error):
// s + e == a + b and p + e == a * b exactly (round to nearest, no overflow).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// FP32 window sums without FP64 arithmetic per value (FP64 runs at a small
// fraction of the FP32 rate on this GPU): three FP32 words h + l + t.  Each
// value goes into h by TwoSum; its error goes into l by TwoSum; that error
// into t by a plain add.  With P the largest partial sum of a window of K
// values, |error of h + l| <= K 2^-24 P, so |t's errors| <= K^3 2^-72 P:
// 2^-48 P for K = kWin = 256.  Infinities and NaNs make the sum NaN, as in
// FP64.
constexpr int kWin = 256;
struct FWin {
  float h, l, t;
};

__device__ __forceinline__ void fwin_add(FWin& w, float x) {
  float s, e, s2, e2;
  two_sum(w.h, x, s, e);
  two_sum(w.l, e, s2, e2);
  w.h = s;
  w.l = s2;
  w.t = __fadd_rn(w.t, e2);
}

// A lane's windows add up in a plain FP64 sum (a few windows per lane: their
// roundings stay near 2^-53 of the field's absolute sum); the compensated
// sum starts at the warps' totals.
__device__ __forceinline__ void fwin_flush(FWin& w, double& acc) {
  acc += ((double)w.h + (double)w.l) + (double)w.t;
  w = FWin{0.f, 0.f, 0.f};
}

// The FP64 values of one cell (the formulas the diagnostics define), out of
// line: the filters below reach them for a few cells only.
__device__ __noinline__ double cell_div64(float bxl, float bxh, float byl, float byh, float bzl, float bzh,
                                          int nx, int ny, int nz) {
  return ((double)bxh - bxl) * nx + ((double)byh - byl) * ny + ((double)bzh - bzl) * nz;
}

__device__ __noinline__ double cell_p64(float rho, float m1, float m2, float m3, float e, float bxl,
                                        float bxh, float byl, float byh, float bzl, float bzh, double gamma) {
  const double b0 = 0.5 * ((double)bxl + bxh), b1 = 0.5 * ((double)byl + byh), b2 = 0.5 * ((double)bzl + bzh);
  const double kin = 0.5 * ((double)m1 * m1 + (double)m2 * m2 + (double)m3 * m3) / rho;
  return (gamma - 1.0) * ((double)e - kin - 0.5 * (b0 * b0 + b1 * b1 + b2 * b2));
}

// Float-float tier of the max |div b| filter (inline: out of line it cost
// about 15 % on near-tied states, for no fewer registers).  Each
// difference is exact (TwoSum), times n_d (product error by FMA), summed by
// TwoSum: |D - div| <= 2^-44 dT, dT = sum |(b_high - b_low) n_d|.  True
// unless |div| is certainly below thr.
__device__ __forceinline__ bool div_ff_may_exceed(float bxl, float bxh, float byl, float byh, float bzl,
                                                  float bzh, float nxf, float nyf, float nzf, float thr) {
  float s0, e0, s1, e1, s2, e2, p0, q0, p1, q1, p2, q2;
  two_sum(bxh, -bxl, s0, e0);
  two_sum(byh, -byl, s1, e1);
  two_sum(bzh, -bzl, s2, e2);
  two_prod(s0, nxf, p0, q0);
  two_prod(s1, nyf, p1, q1);
  two_prod(s2, nzf, p2, q2);
  float h01, r01, dh, r2;
  two_sum(p0, p1, h01, r01);
  two_sum(h01, p2, dh, r2);
  const float dl = __fadd_rn(__fadd_rn(__fadd_rn(q0, q1), q2),
                             __fadd_rn(__fadd_rn(__fmaf_rn(e0, nxf, __fmul_rn(e1, nyf)), __fmul_rn(e2, nzf)),
                                       __fadd_rn(r01, r2)));
  const float dT = fabsf(p0) + fabsf(p1) + fabsf(p2);
  const float dabs = fabsf(__fadd_rn(dh, dl));
  return !(dabs + (0x1p-22f * dabs + 0x1p-40f * dT + 1e-37f) < thr);  // NaN: true
}

// Float-float tier of the min p filter:
// |estimate - p| <= 2^-42 (gamma - 1) U.  True unless p certainly exceeds
// the float-float threshold th + tl.
__device__ __forceinline__ bool p_ff_may_undercut(float rho, float m1, float m2, float m3, float e, float bxl,
                                                  float bxh, float byl, float byh, float bzl, float bzh, float rr,
                                                  float g_hi, float g_lo, float U, float th, float tl) {
  float a0, ae0, a1, ae1, a2, ae2, sa, ra, sh, rb;
  two_prod(m1, m1, a0, ae0);
  two_prod(m2, m2, a1, ae1);
  two_prod(m3, m3, a2, ae2);
  two_sum(a0, a1, sa, ra);
  two_sum(sa, a2, sh, rb);
  const float sl = __fadd_rn(__fadd_rn(__fadd_rn(ae0, ae1), ae2), __fadd_rn(ra, rb));
  // an approximate reciprocal rr: k1 within a few ulp of S / rho, the FMA
  // remainder S - k1 rho then corrects it to about 2^-43 S / rho
  const float k1 = __fmul_rn(sh, rr);
  const float k2 = __fmul_rn(__fadd_rn(__fmaf_rn(-k1, rho, sh), sl), rr);  // kin = (k1 + k2) / 2
  float c0h, c0l, c1h, c1l, c2h, c2l;
  two_sum(bxl, bxh, c0h, c0l);
  two_sum(byl, byh, c1h, c1l);
  two_sum(bzl, bzh, c2h, c2l);  // 2 b_c = c_h + c_l exactly
  float w0, we0, w1, we1, w2, we2, sw, rw, mh, rm;
  two_prod(c0h, c0h, w0, we0);
  two_prod(c1h, c1h, w1, we1);
  two_prod(c2h, c2h, w2, we2);
  we0 = __fmaf_rn(2.f * c0h, c0l, we0);
  we1 = __fmaf_rn(2.f * c1h, c1l, we1);
  we2 = __fmaf_rn(2.f * c2h, c2l, we2);
  two_sum(w0, w1, sw, rw);
  two_sum(sw, w2, mh, rm);  // 4 |b_c|^2 = mh + ml
  const float ml = __fadd_rn(__fadd_rn(__fadd_rn(we0, we1), we2), __fadd_rn(rw, rm));
  float d1, de1, d2, de2;
  two_sum(e, -0.5f * k1, d1, de1);
  two_sum(d1, -0.125f * mh, d2, de2);
  const float dlo = __fsub_rn(__fsub_rn(__fadd_rn(de1, de2), 0.5f * k2), 0.125f * ml);
  float ph, phe;
  two_prod(g_hi, d2, ph, phe);
  const float pl = __fadd_rn(phe, __fmaf_rn(g_hi, dlo, __fmul_rn(g_lo, d2)));
  const float dp = 0x1p-38f * g_hi * U + 1e-37f;
  return !(__fadd_rn(__fsub_rn(ph, th), __fsub_rn(__fsub_rn(pl, tl), dp)) > 0.f);  // NaN: true
}

// One pass over the box: the compensated sums of the 8 fields, max |div b|
// (the face differences of each cell) and min p, in FP64 as defined by the
// formulas below.  The extrema are exact FP64 values of those formulas: a
// cell's FP64 value is only evaluated when a float-float estimate (about 44
// bits, error bound with a margin of 16 or more) does not rule it out
// against the warp's running extremum.  Lanes of a warp iterate together
// over whole x rows (lanes past the row's end add zeros); the FP64 values sit
// behind warp votes, and the lanes share their new thresholds right after.
__global__ void __launch_bounds__(kDiagThreads)
diag_partial_kernel(const float* __restrict__ rho, const float* __restrict__ mx,
                    const float* __restrict__ my, const float* __restrict__ mz,
                    const float* __restrict__ en, const float* __restrict__ bx,
                    const float* __restrict__ by, const float* __restrict__ bz, Box box,
                    double gamma, double* __restrict__ partial) {
  const float* f[8] = {rho, mx, my, mz, en, bx, by, bz};
  const int lane = threadIdx.x & 31;
  double acc[8];
  FWin win[8];
#pragma unroll
  for (int q = 0; q < 8; q++) {
    acc[q] = 0.0;
    win[q] = FWin{0.f, 0.f, 0.f};
  }
  double divmax = 0.0, pmin = DBL_MAX;
  float div_thr = 0.f;                        // <= the warp's running max |div b|
  float pt_hi = __int_as_float(0x7f800000), pt_lo = 0.f;  // >= the warp's running min p
  const float nxf = (float)box.n[0], nyf = (float)box.n[1], nzf = (float)box.n[2];
  const float g_hi = (float)(gamma - 1.0), g_lo = (float)((gamma - 1.0) - (double)g_hi);
  // a warp walks whole x rows (no division per cell), 32 cells at a time
  const int nx = box.n[0], ny = box.n[1], nz = box.n[2];
  const long long rows = (long long)ny * nz;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  int it = 0;
  // row r = j + ny k, stepped by nwarps rows without a division per row
  // (64-bit integer division is emulated in software)
  long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int j = (int)(r % ny);
  long long k = r / ny;
  const int dj = (int)(nwarps % ny);
  const long long dk = nwarps / ny;
  for (; r < rows; r += nwarps) {
    const long long rowbase = j * box.stride[1] + k * box.stride[2];
    const long long yoff = (j + 1 < ny) ? box.stride[1] : -(long long)(ny - 1) * box.stride[1];
    const long long zoff = (k + 1 < nz) ? box.stride[2] : -(long long)(nz - 1) * box.stride[2];
    // the 11 values of a lane's cell at x = i0 + lane (x is the contiguous
    // axis, checked at launch); the next chunk's loads go out before this
    // chunk's arithmetic
    float nv[11];
    auto load = [&](int i0, float (&u)[11]) {
      const int ii = min(i0 + lane, nx - 1);
      const long long cc = rowbase + ii;
#pragma unroll
      for (int q = 0; q < 8; q++) u[q] = __ldg(f[q] + cc);
      u[8] = __ldg(bx + (ii + 1 < nx ? cc + 1 : cc - (nx - 1)));
      u[9] = __ldg(by + cc + yoff);
      u[10] = __ldg(bz + cc + zoff);
    };
    load(0, nv);
    for (int i0 = 0; i0 < nx; i0 += 32, it++) {
      const bool valid = i0 + lane < nx;
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; q++) v[q] = valid ? nv[q] : 0.f;
      const float bxh = nv[8], byh = nv[9], bzh = nv[10];
      if (i0 + 32 < nx) load(i0 + 32, nv);
#pragma unroll
      for (int q = 0; q < 8; q++) fwin_add(win[q], v[q]);
      {
        // Three tiers, each behind a warp vote (so that a tier is skipped, not
        // just predicated off, when no lane needs it): an FP32 estimate, a
        // float-float estimate, the FP64 value.  A lane's cell goes on only if
        // the tier's error bound (with a margin of 4 or more) cannot rule it out
        // against the warp's running extremum; a NaN always goes on.
        //
        // div b = sum_d (b_high - b_low) n_d.  FP32: |error| <= 2^-22 dT with
        // dT = sum |(b_high - b_low) n_d|.
        const float t0 = __fmul_rn(__fsub_rn(bxh, v[5]), nxf), t1 = __fmul_rn(__fsub_rn(byh, v[6]), nyf),
                    t2 = __fmul_rn(__fsub_rn(bzh, v[7]), nzf);
        const float d32 = fabsf(t0 + t1 + t2), T32 = fabsf(t0) + fabsf(t1) + fabsf(t2);
        const bool sdiv = valid && !(d32 + (0x1p-20f * T32 + 1e-37f) < div_thr);
        if (__any_sync(0xffffffffu, sdiv)) {
          const bool cand_div = sdiv && div_ff_may_exceed(v[5], bxh, v[6], byh, v[7], bzh, nxf, nyf, nzf, div_thr);
          if (__any_sync(0xffffffffu, cand_div)) {
            if (cand_div) {
              const double div = cell_div64(v[5], bxh, v[6], byh, v[7], bzh, nx, ny, nz);
              divmax = fmax(divmax, fabs(div));
              div_thr = fmaxf(div_thr, __double2float_rd(divmax));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) div_thr = fmaxf(div_thr, __shfl_xor_sync(0xffffffffu, div_thr, o));
          }
        }
        // p = (gamma - 1)(e - |m|^2 / (2 rho) - |b_c|^2 / 2), U = |e| + |kin| +
        // sum ((|b| + |b_high|) / 2)^2 / 2.  FP32: |error| <= 2^-19 (gamma - 1) U.
        const float rr = fast_rcp(v[0]);
        const float kin32 = 0.5f * __fmaf_rn(v[1], v[1], __fmaf_rn(v[2], v[2], __fmul_rn(v[3], v[3]))) * rr;
        const float bc0 = v[5] + bxh, bc1 = v[6] + byh, bc2 = v[7] + bzh;  // 2 b_c
        const float p32 = g_hi * (v[4] - kin32 - 0.125f * __fmaf_rn(bc0, bc0, __fmaf_rn(bc1, bc1, __fmul_rn(bc2, bc2))));
        const float ax = fabsf(v[5]) + fabsf(bxh), ay = fabsf(v[6]) + fabsf(byh), az = fabsf(v[7]) + fabsf(bzh);
        const float U = fabsf(v[4]) + fabsf(kin32) + 0.125f * (ax * ax + ay * ay + az * az);
        // skip while p32 - bound exceeds the threshold pt_hi + pt_lo (>= the
        // warp's min; 2^-22 |pt_hi| covers rounding that sum)
        const bool sp = valid && !(__fsub_rn(p32, 0x1p-17f * g_hi * U + 1e-37f) >
                                   pt_hi + (pt_lo + 0x1p-22f * fabsf(pt_hi)));
        if (__any_sync(0xffffffffu, sp)) {
          const bool cand_p = sp && p_ff_may_undercut(v[0], v[1], v[2], v[3], v[4], v[5], bxh, v[6], byh, v[7], bzh, rr,
                                                      g_hi, g_lo, U, pt_hi, pt_lo);
          if (__any_sync(0xffffffffu, cand_p)) {
            if (cand_p) {
              const double p = cell_p64(v[0], v[1], v[2], v[3], v[4], v[5], bxh, v[6], byh, v[7], bzh, gamma);
              pmin = fmin(pmin, p);
              // float-float upper bound of pmin (pt_hi + pt_lo >= pmin)
              if (fabs(pmin) < 1e38) {
                const float h = __double2float_rn(pmin);
                pt_hi = h;
                pt_lo = __double2float_ru(pmin - (double)h);
              } else {
                pt_hi = pmin > 0.0 ? __int_as_float(0x7f800000) : -FLT_MAX;
                pt_lo = 0.f;
              }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const float oh = __shfl_xor_sync(0xffffffffu, pt_hi, o), ol = __shfl_xor_sync(0xffffffffu, pt_lo, o);
              if (__fadd_rn(__fsub_rn(oh, pt_hi), __fsub_rn(ol, pt_lo)) < 0.f) {
                pt_hi = oh;
                pt_lo = ol;
              }
            }
          }
        }
      }
      if (it % kWin == kWin - 1) {
#pragma unroll
        for (int q = 0; q < 8; q++) fwin_flush(win[q], acc[q]);
      }
    }
    j += dj;
    k += dk;
    if (j >= ny) {
      j -= ny;
      k++;
    }
  }
#pragma unroll
  for (int q = 0; q < 8; q++) fwin_flush(win[q], acc[q]);
  // fixed-order tree: warp shuffles (plain FP64: 5 roundings), then the
  // warps in order and the blocks in order with compensation
  __shared__ double sm[kDiagThreads / 32][kDiagSlots];
  const int wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 8; q++) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], o);
    divmax = fmax(divmax, __shfl_down_sync(0xffffffffu, divmax, o));
    pmin = fmin(pmin, __shfl_down_sync(0xffffffffu, pmin, o));
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
      sm[wid][2 * q] = acc[q];
      sm[wid][2 * q + 1] = 0.0;
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
  if (b > kDiagMaxBlocks) b = kDiagMaxBlocks;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_diagnostics(const float* const f[8], const Box& box, double gamma, double* partial,
                               double* out, cudaStream_t s) {
  if (box.stride[0] != 1) return cudaErrorInvalidValue;
  const int nblk = diag_blocks(box);
  diag_partial_kernel<<<nblk, kDiagThreads, 0, s>>>(f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7],
                                                    box, gamma, partial);
  int nmax = box.n[0] > box.n[1] ? box.n[0] : box.n[1];
  nmax = nmax > box.n[2] ? nmax : box.n[2];
  diag_final_kernel<<<1, 32, 0, s>>>(partial, nblk, 1.0 / nmax, out);
  return cudaGetLastError();
}

}  // namespace mhd
