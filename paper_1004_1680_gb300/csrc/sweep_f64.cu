// FP64 path of the grid update (an ablation: the paper computes in FP32,
// Section III).  The same scheme as the FP32 kernels (Section II.B: relaxing
// TVD fluid sweeps, advection-constraint magnetic sweeps, xyz then zyx),
// written for clarity rather than speed: FP64 runs at a small fraction of
// the FP32 rate on this GPU, so the arithmetic, not memory traffic, bounds
// these kernels.
//  * Every operation is an IEEE double operation rounded once (__dadd_rn,
//    __dmul_rn, __ddiv_rn, __dsqrt_rn; no multiply-add contraction).
//  * Fluid sweep: one thread per whole periodic pencil along any axis, with
//    the marching window of the FP32 pipeline (3 cells of lag).
//  * Magnetic sweep: a flux kernel advects each transverse component (one
//    thread per pencil and component) and stores its edge flux; a
//    constraint kernel then updates b_d of every cell from the stored
//    fluxes of its pencil and the neighbouring pencils.
//  * CFL rate: the largest (|v_d| + c_f*) / h_d over cells, as double bits
//    reduced with an atomic maximum (rates are >= 0).
#include <cstdint>

#include "mhd_launch.h"

namespace mhd {
namespace {

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// half the van Leer limiter, phi(a, b) / 2 = ab / (a + b) for ab > 0, else 0
__device__ __forceinline__ double vl_half(double a, double b) {
  const double ab = dmul(a, b);
  return ab > 0.0 ? ddiv(ab, dadd(a, b)) : 0.0;
}

// Right and left movers FR = (c u + F) / 2, FL = (c u - F) / 2 of Eq. 1-3
// projected on the sweep axis (u = rho, m_d, m_t1, m_t2, e; b = cell-centred
// b_d, b_t1, b_t2), with the freezing speed c = |v_d| + sqrt((gamma p + b^2) / rho).
__device__ __forceinline__ void movers64(const double u[5], const double b[3], double gamma, double FR[5],
                                         double FL[5]) {
  const double vd = ddiv(u[1], u[0]), v1 = ddiv(u[2], u[0]), v2 = ddiv(u[3], u[0]);
  const double bb = dadd(dadd(dmul(b[0], b[0]), dmul(b[1], b[1])), dmul(b[2], b[2]));
  const double kin = dmul(0.5, dadd(dadd(dmul(u[1], vd), dmul(u[2], v1)), dmul(u[3], v2)));
  const double p = dmul(gamma - 1.0, dsub(dsub(u[4], kin), dmul(0.5, bb)));
  const double ps = dadd(p, dmul(0.5, bb));
  const double bv = dadd(dadd(dmul(b[0], vd), dmul(b[1], v1)), dmul(b[2], v2));
  double F[5];
  F[0] = u[1];
  F[1] = dsub(dadd(dmul(u[1], vd), ps), dmul(b[0], b[0]));
  F[2] = dsub(dmul(u[2], vd), dmul(b[0], b[1]));
  F[3] = dsub(dmul(u[3], vd), dmul(b[0], b[2]));
  F[4] = dsub(dmul(dadd(u[4], ps), vd), dmul(b[0], bv));
  const double c = dadd(fabs(vd), __dsqrt_rn(ddiv(dadd(dmul(gamma, p), bb), u[0])));
#pragma unroll
  for (int q = 0; q < 5; q++) {
    FR[q] = dmul(0.5, dadd(dmul(c, u[q]), F[q]));
    FL[q] = dmul(0.5, dsub(dmul(c, u[q]), F[q]));
  }
}

// The fluid marching pipeline (the FP32 FluidPipe's window, in double):
// consuming position t yields Unew at t - 3.
struct FluidPipe64 {
  double U1[5], U2[5], U3[5], b1[3], FR1[5], f1m[5], Rh2[5], Rh3[5], dR3[5], Lh2[5], dL2[5], F2m[5];

  __device__ void init() {
#pragma unroll
    for (int q = 0; q < 5; q++)
      U1[q] = U2[q] = U3[q] = FR1[q] = f1m[q] = Rh2[q] = Rh3[q] = dR3[q] = Lh2[q] = dL2[q] = F2m[q] = 0.0;
    b1[0] = b1[1] = b1[2] = 0.0;
  }

  __device__ void step(const double U[5], const double b[3], double gamma, double c_half, double c_full,
                       double out[5]) {
    double FR[5], FL[5], Uh[5], Rh[5], Lh[5], f1[5];
    movers64(U, b, gamma, FR, FL);
#pragma unroll
    for (int q = 0; q < 5; q++) {
      f1[q] = dsub(FR1[q], FL[q]);                                 // first-order flux at t - 1/2
      Uh[q] = dsub(U1[q], dmul(c_half, dsub(f1[q], f1m[q])));      // half step at t - 1
    }
    movers64(Uh, b1, gamma, Rh, Lh);
#pragma unroll
    for (int q = 0; q < 5; q++) {
      const double dR2 = dsub(Rh2[q], Rh3[q]), dL1 = dsub(Lh[q], Lh2[q]);
      const double right = dadd(Rh3[q], vl_half(dR3[q], dR2));   // upwind cell t - 3
      const double left = dsub(Lh2[q], vl_half(dL2[q], dL1));    // upwind cell t - 2
      const double F2 = dsub(right, left);                       // second-order flux at t - 5/2
      out[q] = dsub(U3[q], dmul(c_full, dsub(F2, F2m[q])));
      F2m[q] = F2;
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

// The magnetic advection pipeline (the FP32 MagPipe in double): consuming
// (q, u) at t yields qnew at t - 3 and the edge flux at t - 5/2.
struct MagPipe64 {
  double q1, q2, q3, u1, g1m, h2, h3, d32, d43, ub1, ub2, fm;

  __device__ void init() { q1 = q2 = q3 = u1 = g1m = h2 = h3 = d32 = d43 = ub1 = ub2 = fm = 0.0; }

  __device__ double step(double q, double u, double c_half, double c_full, double& qnew) {
    const double ub = dmul(0.5, dadd(u1, u));                      // edge velocity at t - 1/2
    const double g = dmul(ub, ub >= 0.0 ? q1 : q);                 // upwind flux
    const double h = dsub(q1, dmul(c_half, dsub(g, g1m)));         // half step at t - 1
    const double d21 = dsub(h, h2);
    const bool pos = ub2 >= 0.0;                                   // edge t - 5/2
    const double base = pos ? h3 : h2;
    const double lim = pos ? vl_half(d43, d32) : vl_half(d32, d21);
    const double f = dmul(ub2, pos ? dadd(base, lim) : dsub(base, lim));
    qnew = dsub(q3, dmul(c_full, dsub(f, fm)));
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

struct Geo {
  int n[3];
  int s[3];
  double ih[3];
};

// one thread per pencil along D (A, O: the other axes)
template <int D>
__global__ void __launch_bounds__(128) fluid64_kernel(Fluid64Args a) {
  constexpr int A = (D == 0) ? 1 : 0, O = (D == 2) ? 1 : 2, T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  const Geo g{{a.n[0], a.n[1], a.n[2]}, {1, a.n[0], a.n[0] * a.n[1]}, {a.ih[0], a.ih[1], a.ih[2]}};
  const int pa = blockIdx.x * 32 + threadIdx.x, pb = blockIdx.y * blockDim.y + threadIdx.y;
  if (pa >= g.n[A] || pb >= g.n[O]) return;
  const int nD = g.n[D];
  const int base = pa * g.s[A] + pb * g.s[O];
  const int eT1 = (T1 == A) ? wrapi(pa + 1, g.n[A]) * g.s[A] + pb * g.s[O] : pa * g.s[A] + wrapi(pb + 1, g.n[O]) * g.s[O];
  const int eT2 = (T2 == A) ? wrapi(pa + 1, g.n[A]) * g.s[A] + pb * g.s[O] : pa * g.s[A] + wrapi(pb + 1, g.n[O]) * g.s[O];
  const double c_full = dmul(a.tau, g.ih[D]), c_half = dmul(0.5, c_full);
  FluidPipe64 pipe;
  pipe.init();
  for (int t = -4; t < nD + 3; t++) {
    const int off = wrapi(t, nD) * g.s[D], off1 = wrapi(t + 1, nD) * g.s[D];
    const int c = base + off;
    const double U[5] = {a.in[RHO][c], a.in[MX + D][c], a.in[MX + T1][c], a.in[MX + T2][c], a.in[EN][c]};
    const double b[3] = {dmul(0.5, dadd(a.in[BX + D][c], a.in[BX + D][base + off1])),
                         dmul(0.5, dadd(a.in[BX + T1][c], a.in[BX + T1][eT1 + off])),
                         dmul(0.5, dadd(a.in[BX + T2][c], a.in[BX + T2][eT2 + off]))};
    double o[5];
    pipe.step(U, b, a.gamma, c_half, c_full, o);
    const int po = t - 3;
    if (po >= 0 && po < nD) {
      const int w = base + po * g.s[D];
      a.out[RHO][w] = o[0];
      a.out[MX + D][w] = o[1];
      a.out[MX + T1][w] = o[2];
      a.out[MX + T2][w] = o[3];
      a.out[EN][w] = o[4];
    }
  }
}

// Advection of b_t along D for one transverse axis t (blockIdx.z: 0 -> T1,
// 1 -> T2): new b_t into out[BX + t], edge fluxes into E[blockIdx.z] (the
// flux of edge i + 1/2 of a pencil stored at its cell i).
template <int D>
__global__ void __launch_bounds__(128) mag64_flux_kernel(Mag64Args a) {
  constexpr int A = (D == 0) ? 1 : 0, O = (D == 2) ? 1 : 2;
  const Geo g{{a.n[0], a.n[1], a.n[2]}, {1, a.n[0], a.n[0] * a.n[1]}, {a.ih[0], a.ih[1], a.ih[2]}};
  const int pa = blockIdx.x * 32 + threadIdx.x, pb = blockIdx.y * blockDim.y + threadIdx.y;
  if (pa >= g.n[A] || pb >= g.n[O]) return;
  const int t = (blockIdx.z == 0) ? (D + 1) % 3 : (D + 2) % 3;
  const int nD = g.n[D];
  const int base = pa * g.s[A] + pb * g.s[O];
  // the pencil one cell down along t (the other side of the b_t face)
  const int baseM = (t == A) ? wrapi(pa - 1, g.n[A]) * g.s[A] + pb * g.s[O]
                             : pa * g.s[A] + wrapi(pb - 1, g.n[O]) * g.s[O];
  const double c_full = dmul(a.tau, g.ih[D]), c_half = dmul(0.5, c_full);
  const double* __restrict__ rho = a.in[RHO];
  const double* __restrict__ md = a.in[MX + D];
  const double* __restrict__ q = a.in[BX + t];
  double* __restrict__ qo = a.out[BX + t];
  double* __restrict__ E = a.E[blockIdx.z];
  MagPipe64 pipe;
  pipe.init();
  for (int s = -4; s < nD + 3; s++) {
    const int off = wrapi(s, nD) * g.s[D];
    const int c = base + off, cm = baseM + off;
    const double u = dmul(0.5, dadd(ddiv(md[c], rho[c]), ddiv(md[cm], rho[cm])));  // v_D on the b_t face
    double qn;
    const double f = pipe.step(q[c], u, c_half, c_full, qn);
    const int po = s - 3;
    if (po >= 0 && po < nD) {
      qo[base + po * g.s[D]] = qn;
      E[base + po * g.s[D]] = f;  // edge po + 1/2
    }
  }
}

// b_D of every cell (low face i along D) takes the edge fluxes of edge
// i - 1/2 of its pencil and of the next pencil along each transverse axis:
// b_D += tau/h_t (E_t(pencil + e_t) - E_t(pencil)), t = T1 then T2.
template <int D>
__global__ void __launch_bounds__(256) mag64_constraint_kernel(Mag64Args a) {
  const int N = a.n[0] * a.n[1] * a.n[2];
  const int s[3] = {1, a.n[0], a.n[0] * a.n[1]};
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    int x[3] = {c % a.n[0], (c / a.n[0]) % a.n[1], c / (a.n[0] * a.n[1])};
    int em[3] = {x[0], x[1], x[2]};
    em[D] = wrapi(x[D] - 1, a.n[D]);  // the cell whose edge flux is edge i - 1/2
    const int ce = em[0] * s[0] + em[1] * s[1] + em[2] * s[2];
    double b = a.in[BX + D][c];
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const int t = (D + 1 + k) % 3;
      int ep[3] = {em[0], em[1], em[2]};
      ep[t] = wrapi(em[t] + 1, a.n[t]);
      const int cp = ep[0] * s[0] + ep[1] * s[1] + ep[2] * s[2];
      b = dadd(b, dmul(dmul(a.tau, a.ih[t]), dsub(a.E[k][cp], a.E[k][ce])));
    }
    a.out[BX + D][c] = b;
  }
}

__global__ void __launch_bounds__(256) cfl64_kernel(const double* __restrict__ rho, const double* __restrict__ mx,
                                                    const double* __restrict__ my, const double* __restrict__ mz,
                                                    const double* __restrict__ en, const double* __restrict__ bx,
                                                    const double* __restrict__ by, const double* __restrict__ bz,
                                                    int nx, int ny, int nz, double ihx, double ihy, double ihz,
                                                    double gamma, unsigned long long* rate) {
  const int N = nx * ny * nz;
  double rmax = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    const int cx = c - i + wrapi(i + 1, nx), cy = c + (wrapi(j + 1, ny) - j) * nx, cz = c + (wrapi(k + 1, nz) - k) * nx * ny;
    const double b[3] = {dmul(0.5, dadd(bx[c], bx[cx])), dmul(0.5, dadd(by[c], by[cy])), dmul(0.5, dadd(bz[c], bz[cz]))};
    const double m[3] = {mx[c], my[c], mz[c]};
    const double r = rho[c];
    double v[3], bb = 0.0, kin = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
      v[d] = ddiv(m[d], r);
      bb = dadd(bb, dmul(b[d], b[d]));
      kin = dadd(kin, dmul(0.5, dmul(m[d], v[d])));
    }
    const double p = dmul(gamma - 1.0, dsub(dsub(en[c], kin), dmul(0.5, bb)));
    const double cf = __dsqrt_rn(ddiv(dadd(dmul(gamma, p), bb), r));
    double rc = fmax(fmax(dmul(dadd(fabs(v[0]), cf), ihx), dmul(dadd(fabs(v[1]), cf), ihy)),
                     dmul(dadd(fabs(v[2]), cf), ihz));
    if (!(r > 0.0) || !(p > 0.0) || !(rc <= 1.0e300)) rc = __longlong_as_double(0x7ff0000000000000LL);
    rmax = fmax(rmax, rc);
  }
  for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(rate, (unsigned long long)__double_as_longlong(rmax));
}

}  // namespace

cudaError_t launch_fluid64(int axis, const Fluid64Args& a, cudaStream_t s) {
  const int A = (axis == 0) ? 1 : 0, O = (axis == 2) ? 1 : 2;
  const dim3 block(32, 4), grid((a.n[A] + 31) / 32, (a.n[O] + 3) / 4);
  if (axis == 0) fluid64_kernel<0><<<grid, block, 0, s>>>(a);
  if (axis == 1) fluid64_kernel<1><<<grid, block, 0, s>>>(a);
  if (axis == 2) fluid64_kernel<2><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mag64(int axis, const Mag64Args& a, cudaStream_t s) {
  const int A = (axis == 0) ? 1 : 0, O = (axis == 2) ? 1 : 2;
  const dim3 block(32, 4), grid((a.n[A] + 31) / 32, (a.n[O] + 3) / 4, 2);
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const int cblocks = (int)((N + 255) / 256 < 152 * 16 ? (N + 255) / 256 : 152 * 16);
  if (axis == 0) {
    mag64_flux_kernel<0><<<grid, block, 0, s>>>(a);
    mag64_constraint_kernel<0><<<cblocks, 256, 0, s>>>(a);
  }
  if (axis == 1) {
    mag64_flux_kernel<1><<<grid, block, 0, s>>>(a);
    mag64_constraint_kernel<1><<<cblocks, 256, 0, s>>>(a);
  }
  if (axis == 2) {
    mag64_flux_kernel<2><<<grid, block, 0, s>>>(a);
    mag64_constraint_kernel<2><<<cblocks, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_cfl64(const double* const f[8], const int n[3], const double ih[3], double gamma,
                         unsigned long long* rate, cudaStream_t s) {
  const long long N = (long long)n[0] * n[1] * n[2];
  const int blocks = (int)((N + 255) / 256 < 152 * 8 ? (N + 255) / 256 : 152 * 8);
  cfl64_kernel<<<blocks, 256, 0, s>>>(f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], n[0], n[1], n[2], ih[0],
                                      ih[1], ih[2], gamma, rate);
  return cudaGetLastError();
}

}  // namespace mhd
