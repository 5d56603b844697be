// Sweeps along the contiguous axis x over whole rows (Section II.B), FP32.
//
// A block holds whole x rows in shared memory: each row's fields arrive by
// one-dimensional bulk copies (one per field row, contiguous 2 KB pieces at
// 512 cells), and each thread owns 4 consecutive cells of the row.  The
// stencil reaches neighbouring threads' cells only at the ends of a thread's
// 4 cells; those values are exchanged through per-thread slots in shared
// memory, around an mbarrier phase, a block barrier or a named barrier of
// the row's own warps.  Every DRAM line is read whole and once, and no
// transposed copy of the state is needed for the x sweeps.
//
// The arithmetic of a cell is that of the marching pipelines of
// mhd_device.cuh (the same operations on the same operands, in the same
// order): the magnetic row sweep gives bitwise the result of the
// register-load x sweep, and the fluid row sweep agrees with it to FP32
// rounding (it takes the freezing speeds' square roots from the hardware
// approximation, as the TMA-staged strided sweeps do).
#pragma once
#include <cmath>

#include "mhd_device.cuh"
#include "mhd_launch.h"
#include "tma.cuh"

namespace mhd {

constexpr int kRowCells = 4;        // consecutive cells per thread
constexpr int kRowMaxThreads = 256; // rows of up to 1024 cells

// One-dimensional bulk copy of `bytes` (a multiple of 16, both addresses
// 16-byte aligned) from global memory into shared memory, completing on the
// mbarrier at `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const float* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(__cvta_generic_to_global(src))), "r"(bytes), "r"(bar)
      : "memory");
}

// ---------------------------------------------------------------------------
// Fluid sweep along x.  A row's copy set is 10 field rows of nx floats: rho,
// m_x, m_y, m_z, e, b_x, b_y, b_y of the row +1 along y, b_z, b_z of the row
// +1 along z (the face fields' high faces of the cell-centred field).  The
// copies of the block's next row are issued at the first exchange of this
// row, once every warp is done with the row before and past this row's
// stage 1: rho, m, e into the other of two buffers (this row's stay
// readable to the end of its computation), the face fields onto the one set
// of face-field rows (read in stage 1 only).
//
// Per row, with thread l owning cells i = 4l .. 4l+3 (periodic along x):
//   stage 1: FR, FL of U; flux1(i+1/2) = FR(i) - FL(i+1);
//            Uh(i) = U(i) - tau/(2h) (flux1(i+1/2) - flux1(i-1/2))
//            exchange: FR(4l+3) to the right, FL(4l) to the left
//   stage 2: Rh, Lh of Uh; F2(i+1/2) = [Rh(i) + phi/2] - [Lh(i+1) - phi/2]
//            exchange: Rh(4l+3) to the right, Rh(4l), Lh(4l), Lh(4l+1) to
//            the left; then F2(4l+7/2) to the right
//   Unew(i) = U(i) - tau/h (F2(i+1/2) - F2(i-1/2))
constexpr int kFRowFields = 10;
constexpr int kFRowBufs = 2;   // buffers of the conserved fields' rows
constexpr int kFRowSlots = 7;  // exchanged V5 values per thread: FR(4l+3), FL(4l); Rh(4l+3), Rh(4l), Lh(4l), Lh(4l+1); F2

// Shared memory: kFRowBufs x 5 rows of rho, m, e, one set of the 5
// face-field rows, the exchange slots.  47.9 KB at 512 cells: 4 blocks per
// SM.
__host__ __device__ constexpr size_t fluid_row_smem(int nx) {
  return (size_t)(kFRowBufs * 5 + 5) * nx * 4 + (size_t)kFRowSlots * (nx / kRowCells) * 20;
}

// The exchange slots of the fluid row sweep: every thread stores its value
// of a slot as one 16-byte and one 4-byte word (conflict-free, two
// instructions) and reads its neighbour's the same way.  Through lane
// shuffles with the warps' end lanes going through shared memory the
// exchange cost about 20 instructions per value: 9.0 against 7.6 warp
// instructions per cell for the strided sweep.
struct RowSlots {
  float4* A;  // [slot][thread]: rho, m_d, m_t1, m_t2 components
  float* E;   // [slot][thread]: e component
  int T;
  __device__ __forceinline__ void put(int slot, int i, const V5& v) const {
    A[slot * T + i] = make_float4(v.p0.x, v.p0.y, v.p1.x, v.p1.y);
    E[slot * T + i] = v.e;
  }
  __device__ __forceinline__ V5 get(int slot, int i) const {
    const float4 a = A[slot * T + i];
    return {make_float2(a.x, a.y), make_float2(a.z, a.w), E[slot * T + i]};
  }
};

__device__ __forceinline__ void fluid_row_issue(const FluidArgs& a, uint32_t dst, uint32_t dstb, uint32_t bar, int r,
                                                int nx, int ny, int nz) {
  const int y = r % ny, z = r / ny;
  const long long sy = nx, sz = (long long)nx * ny;
  const long long o = y * sy + z * sz;
  const long long oy = (y + 1 == ny ? 0 : y + 1) * sy + z * sz;
  const long long oz = y * sy + (z + 1 == nz ? 0 : z + 1) * sz;
  const uint32_t bytes = (uint32_t)nx * 4;
  mbar_expect_tx(bar, kFRowFields * bytes);
  bulk_load(dst + 0 * bytes, a.in[RHO] + o, bytes, bar);
  bulk_load(dst + 1 * bytes, a.in[MX] + o, bytes, bar);
  bulk_load(dst + 2 * bytes, a.in[MY] + o, bytes, bar);
  bulk_load(dst + 3 * bytes, a.in[MZ] + o, bytes, bar);
  bulk_load(dst + 4 * bytes, a.in[EN] + o, bytes, bar);
  bulk_load(dstb + 0 * bytes, a.in[BX] + o, bytes, bar);
  bulk_load(dstb + 1 * bytes, a.in[BY] + o, bytes, bar);
  bulk_load(dstb + 2 * bytes, a.in[BY] + oy, bytes, bar);
  bulk_load(dstb + 3 * bytes, a.in[BZ] + o, bytes, bar);
  bulk_load(dstb + 4 * bytes, a.in[BZ] + oz, bytes, bar);
}

// U of the thread's 4 cells from the staged row
__device__ __forceinline__ void row_state(const float* sb, int nx, int x0, V5 (&U)[kRowCells]) {
  float4 f[5];
#pragma unroll
  for (int q = 0; q < 5; q++) f[q] = *reinterpret_cast<const float4*>(sb + q * nx + x0);
#pragma unroll
  for (int j = 0; j < kRowCells; j++)
    U[j] = {make_float2((&f[0].x)[j], (&f[1].x)[j]), make_float2((&f[2].x)[j], (&f[3].x)[j]), (&f[4].x)[j]};
}
// The cell-centred field of the thread's 4 cells (xn: the first cell of the
// next thread, whose low x face is the last cell's high face): mean of the
// low and high face along each axis.
struct B3 {
  float v[3];
};
// sbb: the staged rows b_x, b_y, b_y(+y), b_z, b_z(+z)
__device__ __forceinline__ void row_fields(const float* sbb, int nx, int x0, int xn, B3 (&B)[kRowCells]) {
  const float4 bx = *reinterpret_cast<const float4*>(sbb + 0 * nx + x0);
  const float4 by0 = *reinterpret_cast<const float4*>(sbb + 1 * nx + x0);
  const float4 by1 = *reinterpret_cast<const float4*>(sbb + 2 * nx + x0);
  const float4 bz0 = *reinterpret_cast<const float4*>(sbb + 3 * nx + x0);
  const float4 bz1 = *reinterpret_cast<const float4*>(sbb + 4 * nx + x0);
  const float bxa[kRowCells + 1] = {bx.x, bx.y, bx.z, bx.w, sbb[xn]};
#pragma unroll
  for (int j = 0; j < kRowCells; j++)
    B[j] = {{face_mean(bxa[j], bxa[j + 1]), face_mean((&by0.x)[j], (&by1.x)[j]), face_mean((&bz0.x)[j], (&bz1.x)[j])}};
}

// 128 registers: 4 blocks of 128 threads (512-cell rows) or 2 of 256
// (1024-cell rows) per SM; no spills since the exchanges go through the
// slots.
template <bool RATE, bool FLOOR, int LIM, int FRZ>
__global__ void __launch_bounds__(kRowMaxThreads, 2) fluid_row_kernel(const __grid_constant__ FluidArgs a) {
  static_assert(FRZ != 2, "the per-pencil freezing speed keeps the pencil sweeps");
  extern __shared__ __align__(128) float rs_dyn[];
  __shared__ alignas(8) unsigned long long rbar[kFRowBufs];
  // split-phase exchanges (stage 1, stage 2, F2; one arrival per warp) and
  // the block's stop flag: a warp whose bounded wait ran out raises it and
  // leaves the row loop; the others see it at their next wait (their waits
  // on the missing warp's arrivals run out too, within the bound)
  __shared__ alignas(8) unsigned long long xbar[3];
  __shared__ int stop;
  const int nx = a.box.n[0], ny = a.box.n[1], nz = a.box.n[2];
  const int T = nx / kRowCells, l = threadIdx.x;
  const int rows = ny * nz;
  const int lane = l & 31, nw = T >> 5;
  const int lm = l == 0 ? T - 1 : l - 1, lp = l + 1 == T ? 0 : l + 1;  // neighbour threads (periodic)
  const float* sbb = rs_dyn + kFRowBufs * 5 * nx;  // the face-field rows
  RowSlots X;
  X.A = reinterpret_cast<float4*>(rs_dyn + (kFRowBufs * 5 + 5) * nx);
  X.E = reinterpret_cast<float*>(X.A + kFRowSlots * T);
  X.T = T;

  const float gamma = a.gamma;
  const float tau = *a.tau;
  const float c_full = tau * a.box.ih[0];
  const float c_half = 0.5f * c_full;
  const int x0 = kRowCells * l;
  const int xn = l + 1 == T ? 0 : x0 + kRowCells;  // the next thread's first cell
  float rmax = 0.f;
  bool gave_up = false;

  if (l == 0) {
    for (int k = 0; k < kFRowBufs; k++) mbar_init(smem_u32(&rbar[k]), 1);
    for (int k = 0; k < 3; k++) mbar_init(smem_u32(&xbar[k]), nw);
    stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // a bounded wait, decided for the whole warp; false: leave the row loop
  auto wait_ok = [&](uint32_t bar, uint32_t parity) {
    const bool ok = sweep_mbar_wait(bar, parity);
    if (__any_sync(~0u, !ok || *reinterpret_cast<volatile int*>(&stop) != 0)) {
      gave_up = true;
      if (lane == 0) *reinterpret_cast<volatile int*>(&stop) = 1;
      return false;
    }
    return true;
  };
  int issued = 0;  // rows issued so far (the same count in every thread)
  for (int k = 0; k < kFRowBufs - 1 && blockIdx.x + k * gridDim.x < rows; k++, issued++)
    if (l == 0)
      fluid_row_issue(a, smem_u32(rs_dyn + k * 5 * nx), smem_u32(sbb), smem_u32(&rbar[k]), blockIdx.x + k * gridDim.x,
                      nx, ny, nz);

  int it = 0, buf = 0, use = 0;  // iteration, its buffer, and the buffer's use count (mbarrier phase)
  for (int r = blockIdx.x; r < rows; r += gridDim.x, it++) {
    const float* sb = rs_dyn + buf * 5 * nx;
    if (!wait_ok(smem_u32(&rbar[buf]), use & 1)) break;
    // stage 1: the interface fluxes inside the thread's cells right away;
    // FR(4l+3) and FL(4l) wait for the neighbours' halves.  The state is read
    // again (16-byte reads: no bank conflicts) wherever it is needed, while
    // the cell-centred field stays in registers through stage 2.
    V5 f1[kRowCells + 1];  // flux1 at 4l-1/2 .. 4l+7/2
    V5 FR3, FL0;
    B3 B[kRowCells];
    row_fields(sbb, nx, x0, xn, B);
    {
      V5 U[kRowCells];
      row_state(sb, nx, x0, U);
      V5 FRp;
#pragma unroll
      for (int j = 0; j < kRowCells; j++) {
        V5 FR, FL;
        split_flux<FRZ, true>(U[j], B[j].v[0], make_float2(B[j].v[1], B[j].v[2]), gamma, FR, FL);
        if (j == 0) FL0 = FL;
        else f1[j] = v5_sub(FRp, FL);
        FRp = FR;
      }
      FR3 = FRp;
    }
    X.put(0, l, FR3);
    X.put(1, l, FL0);
    // split-phase exchange: the interior cells 1 and 2 go on while the
    // neighbours' halves arrive
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&xbar[0]));
    V5 Rh[kRowCells], Lh[kRowCells];
    V5 U[kRowCells];
    row_state(sb, nx, x0, U);
#pragma unroll
    for (int j = 1; j < kRowCells - 1; j++) {
      const V5 Uh = v5_fma(-c_half, v5_sub(f1[j + 1], f1[j]), U[j]);
      // stage 2
      split_flux<FRZ, true>(Uh, B[j].v[0], make_float2(B[j].v[1], B[j].v[2]), gamma, Rh[j], Lh[j]);
    }
    if (!wait_ok(smem_u32(&xbar[0]), it & 1)) break;
    // every warp is done with the previous row and past this row's stage 1:
    // the next row goes into the other buffer and onto the face-field rows
    if (r + (kFRowBufs - 1) * gridDim.x < rows) {
      const int nb = issued % kFRowBufs;
      if (l == 0)
        fluid_row_issue(a, smem_u32(rs_dyn + nb * 5 * nx), smem_u32(sbb), smem_u32(&rbar[nb]),
                        r + (kFRowBufs - 1) * gridDim.x, nx, ny, nz);
      issued++;
    }
    f1[0] = v5_sub(X.get(0, lm), FL0);          // FR(4l-1) - FL(4l)
    f1[kRowCells] = v5_sub(FR3, X.get(1, lp));  // FR(4l+3) - FL(4l+4)
#pragma unroll
    for (int j = 0; j < kRowCells; j += kRowCells - 1) {
      const V5 Uh = v5_fma(-c_half, v5_sub(f1[j + 1], f1[j]), U[j]);
      split_flux<FRZ, true>(Uh, B[j].v[0], make_float2(B[j].v[1], B[j].v[2]), gamma, Rh[j], Lh[j]);
    }
    X.put(2, l, Rh[kRowCells - 1]);
    X.put(3, l, Rh[0]);
    X.put(4, l, Lh[0]);
    X.put(5, l, Lh[1]);
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&xbar[1]));
    // interface i+1/2, i = 4l + j: Rh(i-1..i+1), Lh(i..i+2)
    auto flux2 = [&](int j, const V5& Rl, const V5& Rr, const V5& L1, const V5& L2) {
      const V5 right = v5_add(Rh[j], half_limited5<LIM>(v5_sub(Rh[j], Rl), v5_sub(Rr, Rh[j])));
      const V5 left = v5_sub(L1, half_limited5<LIM>(v5_sub(L1, Lh[j]), v5_sub(L2, L1)));
      return v5_sub(right, left);
    };
    V5 F2[kRowCells];
    F2[1] = flux2(1, Rh[0], Rh[2], Lh[2], Lh[3]);  // inside the thread's cells, while the neighbours' values arrive
    if (!wait_ok(smem_u32(&xbar[1]), it & 1)) break;
    {
      const V5 Rm = X.get(2, lm);                                         // Rh(4l-1)
      const V5 Rp = X.get(3, lp), Lp0 = X.get(4, lp), Lp1 = X.get(5, lp);  // Rh(4l+4), Lh(4l+4), Lh(4l+5)
      F2[0] = flux2(0, Rm, Rh[1], Lh[1], Lh[2]);
      F2[2] = flux2(2, Rh[1], Rh[3], Lh[3], Lp0);
      F2[3] = flux2(3, Rh[2], Rp, Lp0, Lp1);
    }
    X.put(6, l, F2[kRowCells - 1]);
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&xbar[2]));
    // the finished cells: 1 .. 3 while F2(4l-1/2) arrives, then cell 0
    const int y = r % ny, z = r / ny;
    const long long ro = (long long)y * nx + (long long)z * nx * ny + x0;
    const bool rate_row = RATE && y >= a.rate_lo[1] && y < a.rate_hi[1] && z >= a.rate_lo[2] && z < a.rate_hi[2];
    float o[kRowCells][5];
    row_state(sb, nx, x0, U);
    auto finish = [&](int j, const V5& fl) {
      const V5 v = v5_fma(-c_full, v5_sub(F2[j], fl), U[j]);
      o[j][0] = v.p0.x;
      o[j][1] = v.p0.y;
      o[j][2] = v.p1.x;
      o[j][3] = v.p1.y;
      o[j][4] = v.e;
      if (FLOOR) o[j][4] = floored_energy(o[j], B[j].v, gamma, a.p_floor);
      if (RATE && rate_row && x0 + j >= a.rate_lo[0] && x0 + j < a.rate_hi[0])
        rmax = fmaxf(rmax, cell_rate(o[j][0], &o[j][1], o[j][4], B[j].v, gamma, a.box.ih));
    };
#pragma unroll
    for (int j = 1; j < kRowCells; j++) finish(j, F2[j - 1]);
    if (!wait_ok(smem_u32(&xbar[2]), it & 1)) break;
    finish(0, X.get(6, lm));  // F2(4l-1/2)
#pragma unroll
    for (int q = 0; q < 5; q++)
      *reinterpret_cast<float4*>(a.out[q] + ro) = make_float4(o[0][q], o[1][q], o[2][q], o[3][q]);
    if (++buf == kFRowBufs) {
      buf = 0;
      use++;
    }
  }
  if (__syncthreads_or(gave_up)) {
    // record the failure, then let the copies still in flight (the last
    // kFRowBufs issued) land before the block's shared memory is released;
    // row q went into buffer q % kFRowBufs as its use q / kFRowBufs
    if (l == 0) {
      atomicOr(a.err, 1u);
      for (int q = max(0, issued - kFRowBufs); q < issued; q++)
        sweep_mbar_wait(smem_u32(&rbar[q % kFRowBufs]), (q / kFRowBufs) & 1);
    }
    return;
  }
  if (RATE) {
    for (int s = 16; s > 0; s >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, s));
    if ((l & 31) == 0) atomicMax(a.rate, __float_as_uint(rmax));
  }
}

// ---------------------------------------------------------------------------
// Magnetic sweep along x.  A block owns a tile of R rows along y (rows
// j0 .. j0+R-1) and marches it along z over a segment of planes k0 .. k0+L-1,
// one thread group (threadIdx.y) per row plus a halo group for row j0+R.
// For each row the edge fluxes of b_y and b_z along x (MagPipe's arithmetic,
// cell by cell) are
//   E_y(j, k): q = b_y(j, k), face velocity (v(j, k) + v(j-1, k))/2,
//   E_z(j, k): q = b_z(j, k), face velocity (v(j, k) + v(j, k-1))/2,
// and plane k is finished with
//   b_y(j, k) -= tau/h_x (E_y(i+1/2) - E_y(i-1/2)), likewise b_z with E_z,
//   b_x(face i-1/2) += tau/h_y (E_y(j+1, k) - E_y(j, k))
//                    + tau/h_z (E_z(j, k+1) - E_z(j, k))   (at edge i-1/2).
// Step s of the march stages plane p = k0-1+s, forms v(p), E_z(p) and
// E_y(p-1) and finishes plane p-1: E_z(j, p-1) is carried from the step
// before, E_y of row j+1 comes from the neighbouring group through shared
// memory.  Each staged plane holds rho and m_x of rows j0-1 .. j0+R, b_x and
// b_z of the tile's rows and b_y of rows j0 .. j0+R (ten bulk copies, the
// tile's rows in one piece each); two buffers, the copies of plane p+2 going
// into plane p's once every thread has read it (after the step's block
// barrier).  The exchanges along a row wait for the row's own warps only (a
// named barrier per group); a group may run up to a step ahead of the
// others, which the double-buffered v and E_y rows allow.
// Rows per tile: 4 for rows of up to 512 cells (5 groups of nx/4 threads,
// 640 threads), 2 for 1024 cells (3 groups of 256 threads, 768).
__host__ __device__ constexpr int mag_row_tile(int nx) { return nx <= 512 ? 4 : 2; }
// Row slots of a staged plane for a tile of R rows: rho and m_x of rows
// j0-1 .. j0+R, b_x of the tile, b_y of rows j0 .. j0+R, b_z of the tile.
template <int R>
struct MRow {
  static constexpr int Rho = 0, Mx = R + 2, Bx = 2 * (R + 2), By = Bx + R, Bz = By + R + 1, Slots = Bz + R;
};
constexpr int kMRowXch = 12;  // scalar exchange slots per thread: 6 per advection (q, q, qh, qh, qh, f)

template <int R>
__host__ __device__ constexpr size_t mag_row_smem(int nx) {
  return ((size_t)2 * MRow<R>::Slots + 2 * (R + 2) + 2 * (R + 1)) * nx * 4 +
         (size_t)kMRowXch * (R + 1) * (nx / kRowCells) * 4;
}

template <int R>
__device__ __forceinline__ void mag_row_issue(const MagArgs& a, uint32_t dst, uint32_t bar, int j0, int p, int nx,
                                              int ny, int nz) {
  using M = MRow<R>;
  const int k = p < 0 ? p + nz : (p >= nz ? p - nz : p);
  const long long sz = (long long)nx * ny;
  const long long o = (long long)j0 * nx + k * sz;                                // row j0
  const long long om = (long long)(j0 == 0 ? ny - 1 : j0 - 1) * nx + k * sz;      // row j0-1
  const long long op = (long long)(j0 + R == ny ? 0 : j0 + R) * nx + k * sz;      // row j0+R
  const uint32_t row = (uint32_t)nx * 4;
  mbar_expect_tx(bar, M::Slots * row);
  bulk_load(dst + (M::Rho + 0) * row, a.in[RHO] + om, row, bar);
  bulk_load(dst + (M::Rho + 1) * row, a.in[RHO] + o, R * row, bar);
  bulk_load(dst + (M::Rho + R + 1) * row, a.in[RHO] + op, row, bar);
  bulk_load(dst + (M::Mx + 0) * row, a.in[MX] + om, row, bar);
  bulk_load(dst + (M::Mx + 1) * row, a.in[MX] + o, R * row, bar);
  bulk_load(dst + (M::Mx + R + 1) * row, a.in[MX] + op, row, bar);
  bulk_load(dst + M::Bx * row, a.in[BX] + o, R * row, bar);
  bulk_load(dst + M::By * row, a.in[BY] + o, R * row, bar);
  bulk_load(dst + (M::By + R) * row, a.in[BY] + op, row, bar);
  bulk_load(dst + M::Bz * row, a.in[BZ] + o, R * row, bar);
}

// Barrier of thread group g (threadIdx.y) alone: named barrier g + 1 over
// its n threads (a multiple of 32).
__device__ __forceinline__ void group_sync(int g, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(n) : "memory");
}

// Scalar exchange slots of one thread group: every thread stores its value
// of a slot at [slot][thread] and reads its neighbour's (l-1 or l+1,
// periodic over the group's T threads).
struct RowSlots1 {
  float* S;
  int T, l, lm, lp;
  __device__ __forceinline__ void put(int slot, float v) const { S[slot * T + l] = v; }
  __device__ __forceinline__ float left(int slot) const { return S[slot * T + lm]; }
  __device__ __forceinline__ float right(int slot) const { return S[slot * T + lp]; }
};

// One edge-flux row of the thread's 4 cells, in three parts separated by
// the exchange barriers.  u[0..5]: face velocity at cells 4l-1 .. 4l+4.
template <int LIM>
struct RowAdvect {
  float q[kRowCells];          // advected face field at 4l .. 4l+3
  float ub[kRowCells + 1];     // edge velocity at 4l-1/2 .. 4l+7/2
  float qh[kRowCells];         // half-step field
  float f[kRowCells];          // edge flux at 4l+1/2 .. 4l+7/2
  // part 1: edge velocities; q(4l+3) and q(4l) into slots slot, slot+1
  __device__ __forceinline__ void part1(const float (&u)[kRowCells + 2], const RowSlots1& X, int slot) {
#pragma unroll
    for (int e = 0; e <= kRowCells; e++) ub[e] = __fmul_rn(0.5f, __fadd_rn(u[e], u[e + 1]));
    X.put(slot, q[kRowCells - 1]);
    X.put(slot + 1, q[0]);
  }
  // part 2 (after a barrier): first-order fluxes and the half step;
  // qh(4l+3), qh(4l), qh(4l+1) into slots slot+2 .. slot+4
  __device__ __forceinline__ void part2(float c_half, const RowSlots1& X, int slot) {
    const float qL = X.left(slot), qR = X.right(slot + 1);
    float g[kRowCells + 1];  // at 4l-1/2 .. 4l+7/2
#pragma unroll
    for (int e = 0; e <= kRowCells; e++) {
      const float lo = e == 0 ? qL : q[e - 1], hi = e == kRowCells ? qR : q[e];
      g[e] = __fmul_rn(ub[e], ub[e] >= 0.f ? lo : hi);
    }
#pragma unroll
    for (int i = 0; i < kRowCells; i++) qh[i] = __fmaf_rn(-c_half, __fsub_rn(g[i + 1], g[i]), q[i]);
    X.put(slot + 2, qh[kRowCells - 1]);
    X.put(slot + 3, qh[0]);
    X.put(slot + 4, qh[1]);
  }
  // part 3 (after a barrier): the limited edge fluxes f(4l+1/2 .. 4l+7/2)
  __device__ __forceinline__ void part3(const RowSlots1& X, int slot) {
    float h[kRowCells + 3];  // qh at 4l-1 .. 4l+5
    h[0] = X.left(slot + 2);
#pragma unroll
    for (int i = 0; i < kRowCells; i++) h[i + 1] = qh[i];
    h[kRowCells + 1] = X.right(slot + 3);
    h[kRowCells + 2] = X.right(slot + 4);
    float d[kRowCells + 2];  // d(i) = qh(i) - qh(i-1), i = 4l .. 4l+5
#pragma unroll
    for (int i = 0; i < kRowCells + 2; i++) d[i] = __fsub_rn(h[i + 1], h[i]);
#pragma unroll
    for (int e = 0; e < kRowCells; e++) {  // edge 4l+e+1/2
      const float u = ub[e + 1];
      const bool pos = u >= 0.f;
      const float base = pos ? h[e + 1] : h[e + 2];
      const float sa = pos ? d[e] : d[e + 1];
      const float sb = pos ? d[e + 1] : d[e + 2];
      float lim;
      if constexpr (LIM == 0) {
        lim = vanleer_half(sa, sb);
      } else {
        lim = half_limited<LIM>(sa, sb);
      }
      f[e] = __fmul_rn(u, pos ? __fadd_rn(base, lim) : __fsub_rn(base, lim));
    }
  }
};

template <int LIM, int R>
__global__ void __launch_bounds__(R == 4 ? 640 : 768, 1) mag_row_kernel(const __grid_constant__ MagArgs a, int L) {
  using M = MRow<R>;
  extern __shared__ __align__(128) float ms_dyn[];
  __shared__ alignas(8) unsigned long long mbarr[2];
  const int nx = a.box.n[0], ny = a.box.n[1], nz = a.box.n[2];
  const int T = nx / kRowCells, l = threadIdx.x, g = threadIdx.y;
  const bool halo = g == R;
  const int tiles = ny / R;
  const int j0 = (blockIdx.x % tiles) * R, k0 = (blockIdx.x / tiles) * L;
  const int tid = g * T + l;
  float* P = ms_dyn;                                   // [2][slots][nx]
  float* vring = P + 2 * M::Slots * nx;              // [2][R+2][nx]: v of rows j0-1 .. j0+R
  // [2][R+1][nx]: E_y of rows j0 .. j0+R, by step parity (a group may run a
  // step ahead of the one below it, which still reads its E_y row)
  float* ey2 = vring + 2 * (R + 2) * nx;
  RowSlots1 X;
  X.T = T;
  X.l = l;
  X.lm = l == 0 ? T - 1 : l - 1;
  X.lp = l + 1 == T ? 0 : l + 1;
  X.S = ey2 + 2 * (R + 1) * nx + g * kMRowXch * T;

  const float tau = *a.tau;
  const float c_full = tau * a.box.ih[0];
  const float c_half = 0.5f * c_full;
  const float kA = tau * a.box.ih[1];  // tau / h_y
  const float kO = tau * a.box.ih[2];  // tau / h_z
  const int x0 = kRowCells * l;
  const int xm = l == 0 ? nx - 1 : x0 - 1, xp = l + 1 == T ? 0 : x0 + kRowCells;
  const int vs = halo ? R + 1 : g + 1;  // this group's row in the v slots
  const int nsteps = L + 2;

  if (tid == 0) {
    mbar_init(smem_u32(&mbarr[0]), 1);
    mbar_init(smem_u32(&mbarr[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < 2; s++) mag_row_issue<R>(a, smem_u32(P + s * M::Slots * nx), smem_u32(&mbarr[s]), j0, k0 - 1 + s, nx, ny, nz);
  int issued = 2;

  float cbx[kRowCells], cby[kRowCells], cbz[kRowCells];  // raw b at plane p-1
  float ezp[kRowCells + 1] = {0.f, 0.f, 0.f, 0.f, 0.f};  // E_z(p-1) at 4l-1/2 .. 4l+7/2
  bool gave_up = false;
  RowAdvect<LIM> Az, Ay;
  for (int s = 0; s < nsteps; s++) {
    const int p = k0 - 1 + s;
    const float* sb = P + (s & 1) * M::Slots * nx;
    if (!sweep_mbar_wait(smem_u32(&mbarr[s & 1]), (s >> 1) & 1)) gave_up = true;
    float* vcur = vring + (s & 1) * (R + 2) * nx;
    float* ey = ey2 + (s & 1) * (R + 1) * nx;
    const float* vprev = vring + ((s + 1) & 1) * (R + 2) * nx;
    auto ld4 = [&](int slot, float (&d)[kRowCells]) {
      const float4 v = *reinterpret_cast<const float4*>(sb + slot * nx + x0);
      d[0] = v.x;
      d[1] = v.y;
      d[2] = v.z;
      d[3] = v.w;
    };
    // part A: v(p) of this group's rows (the halo group: rows j0-1 and j0+R)
    {
      auto vel = [&](int slot) {
        const float4 r = *reinterpret_cast<const float4*>(sb + (M::Rho + slot) * nx + x0);
        const float4 m = *reinterpret_cast<const float4*>(sb + (M::Mx + slot) * nx + x0);
        *reinterpret_cast<float4*>(vcur + slot * nx + x0) =
            make_float4(v_div(m.x, r.x), v_div(m.y, r.y), v_div(m.z, r.z), v_div(m.w, r.w));
      };
      if (halo) {
        vel(0);
        vel(R + 1);
      } else {
        vel(g + 1);
      }
    }
    // v(p) of a row is read at this step by its own group only; the other
    // groups read it at the next step, after this step's block barrier
    group_sync(g, T);
    const bool doz = !halo && s >= 1, doy = s >= 2;
    // face velocities at cells 4l-1 .. 4l+4 of two v rows: (own + other) / 2
    auto face_u = [&](const float* va, const float* vb, float (&u)[kRowCells + 2]) {
      const float4 a4 = *reinterpret_cast<const float4*>(va + x0), b4 = *reinterpret_cast<const float4*>(vb + x0);
      u[0] = __fmul_rn(0.5f, __fadd_rn(va[xm], vb[xm]));
      u[1] = __fmul_rn(0.5f, __fadd_rn(a4.x, b4.x));
      u[2] = __fmul_rn(0.5f, __fadd_rn(a4.y, b4.y));
      u[3] = __fmul_rn(0.5f, __fadd_rn(a4.z, b4.z));
      u[4] = __fmul_rn(0.5f, __fadd_rn(a4.w, b4.w));
      u[5] = __fmul_rn(0.5f, __fadd_rn(va[xp], vb[xp]));
    };
    if (doz) {  // E_z(p): b_z(p), v of this row at planes p and p-1
      float u[kRowCells + 2];
      face_u(vcur + vs * nx, vprev + vs * nx, u);
      ld4(M::Bz + g, Az.q);  // b_z(p)
      Az.part1(u, X, 0);
    }
    if (doy) {  // E_y(p-1): b_y(p-1), v of rows j and j-1 at plane p-1
      float u[kRowCells + 2];
      face_u(vprev + vs * nx, vprev + (vs - 1) * nx, u);
#pragma unroll
      for (int i = 0; i < kRowCells; i++) Ay.q[i] = cby[i];
      Ay.part1(u, X, 6);
    }
    // the exchanges along a row need only the row's own warps: a named
    // barrier per group (the block-wide ones cost 1.5x the step at 256^3)
    group_sync(g, T);
    if (doz) Az.part2(c_half, X, 0);
    if (doy) Ay.part2(c_half, X, 6);
    group_sync(g, T);
    if (doz) {
      Az.part3(X, 0);
      X.put(5, Az.f[kRowCells - 1]);
    }
    if (doy) {
      Ay.part3(X, 6);
      *reinterpret_cast<float4*>(ey + (vs - 1) * nx + x0) = make_float4(Ay.f[0], Ay.f[1], Ay.f[2], Ay.f[3]);
    }
    // the raw fields of plane p for the next step (read late: fewer live registers)
    float nbx[kRowCells] = {0.f, 0.f, 0.f, 0.f}, nby[kRowCells], nbz[kRowCells] = {0.f, 0.f, 0.f, 0.f};
    if (halo) {
      ld4(M::By + R, nby);
    } else {
      ld4(M::Bx + g, nbx);
      ld4(M::By + g, nby);
      ld4(M::Bz + g, nbz);
    }
    // the step's one block barrier: E_y rows and v(p) published, plane p
    // read by every thread; it also carries a failed wait
    if (__syncthreads_or(gave_up)) {
      gave_up = true;
      break;
    }
    if (s + 2 < nsteps) {  // every thread has read plane p: plane p+2 goes into its buffer
      if (tid == 0) mag_row_issue<R>(a, smem_u32(P + (s & 1) * M::Slots * nx), smem_u32(&mbarr[s & 1]), j0, p + 2, nx, ny, nz);
      issued++;
    }
    float ezc[kRowCells + 1];  // E_z(p) at 4l-1/2 .. 4l+7/2
    if (doz) {
      ezc[0] = X.left(5);
#pragma unroll
      for (int e = 0; e < kRowCells; e++) ezc[e + 1] = Az.f[e];
    }
    if (doy && !halo) {  // finish plane p-1 of row j0+g
      float eyo[kRowCells + 1], eyu[kRowCells];  // E_y of this row at 4l-1/2 .., of row j+1 at 4l-1/2 .. 4l+5/2
      const float* er = ey + g * nx;
      const float* eu = ey + (g + 1) * nx;
      // (reading the cells 4l-1 from shared memory, with 4-way bank conflicts,
      // measured faster than taking them from the neighbour lanes: 1.16
      // against 1.25 ms at 512^3)
      eyo[0] = er[xm];
#pragma unroll
      for (int e = 0; e < kRowCells; e++) eyo[e + 1] = Ay.f[e];
      eyu[0] = eu[xm];
      {
        const float4 t = *reinterpret_cast<const float4*>(eu + x0);
        eyu[1] = t.x;
        eyu[2] = t.y;
        eyu[3] = t.z;
      }
      float obx[kRowCells], oby[kRowCells], obz[kRowCells];
#pragma unroll
      for (int i = 0; i < kRowCells; i++) {
        oby[i] = __fmaf_rn(-c_full, __fsub_rn(eyo[i + 1], eyo[i]), cby[i]);
        obz[i] = __fmaf_rn(-c_full, __fsub_rn(ezp[i + 1], ezp[i]), cbz[i]);
        // b_x on the low face of cell i: the edge fluxes at i-1/2, y first
        float b = __fmaf_rn(kA, __fsub_rn(eyu[i], eyo[i]), cbx[i]);
        obx[i] = __fmaf_rn(kO, __fsub_rn(ezc[i], ezp[i]), b);
      }
      const int kp = p - 1;  // inside [k0, k0 + L)
      const long long ro = (long long)(j0 + g) * nx + (long long)kp * nx * ny + x0;
      *reinterpret_cast<float4*>(a.out[0] + ro) = make_float4(obx[0], obx[1], obx[2], obx[3]);
      *reinterpret_cast<float4*>(a.out[1] + ro) = make_float4(oby[0], oby[1], oby[2], oby[3]);
      *reinterpret_cast<float4*>(a.out[2] + ro) = make_float4(obz[0], obz[1], obz[2], obz[3]);
    }
    // plane p becomes plane p-1 of the next step
#pragma unroll
    for (int i = 0; i < kRowCells; i++) {
      cbx[i] = nbx[i];
      cby[i] = nby[i];
      cbz[i] = nbz[i];
    }
    if (doz)
#pragma unroll
      for (int e = 0; e <= kRowCells; e++) ezp[e] = ezc[e];
  }
  if (__syncthreads_or(gave_up)) {
    if (tid == 0) {
      atomicOr(a.err, 1u);
      for (int q = max(0, issued - 2); q < issued; q++) sweep_mbar_wait(smem_u32(&mbarr[q & 1]), (q >> 1) & 1);
    }
  }
}

// Rows of the box qualify: x contiguous, nx a multiple of 128 (whole warps of
// 4-cell threads) and at most 1024, 16-byte aligned fields, a single box.
inline bool fluid_rows_qualify(const FluidArgs& a) {
  const Box& b = a.box;
  if (a.ens.items || !a.tma || a.fast == 2) return false;
  if (b.stride[0] != 1 || b.stride[1] != b.n[0] || b.stride[2] != (long long)b.n[0] * b.n[1]) return false;
  if (b.n[0] % 128 || b.n[0] > kRowCells * kRowMaxThreads) return false;
  for (int q = 0; q < 8; q++)
    if (reinterpret_cast<uintptr_t>(a.in[q]) % 16 || reinterpret_cast<uintptr_t>(a.out[q]) % 16) return false;
  return true;
}

// Persistent grid: as many blocks as fit on the device at once (at most one
// per row).
template <class K>
inline cudaError_t row_grid(K kernel, int threads, size_t smem, long long rows, int* grid) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  const long long cap = (long long)sms * (per_sm > 0 ? per_sm : 1);
  *grid = (int)(rows < cap ? rows : cap);
  return cudaSuccess;
}

template <int LIM, int FRZ>
cudaError_t launch_fluid_rows(bool rate, const FluidArgs& a, cudaStream_t s) {
  if constexpr (FRZ == 2) {
    return cudaErrorInvalidValue;
  } else {
    const int nx = a.box.n[0];
    const int threads = nx / kRowCells;
    const size_t smem = fluid_row_smem(nx);
    const long long rows = (long long)a.box.n[1] * a.box.n[2];
    const bool floor = a.p_floor > 0.f;
    int grid = 0;
    cudaError_t e;
#define FLUID_ROW_CASE(RR, FF)                                                        \
  if (rate == RR && floor == FF) {                                                    \
    e = row_grid(fluid_row_kernel<RR, FF, LIM, FRZ>, threads, smem, rows, &grid);     \
    if (e != cudaSuccess) return e;                                                   \
    fluid_row_kernel<RR, FF, LIM, FRZ><<<grid, threads, smem, s>>>(a);                \
  }
    FLUID_ROW_CASE(false, false) FLUID_ROW_CASE(true, false) FLUID_ROW_CASE(false, true) FLUID_ROW_CASE(true, true)
#undef FLUID_ROW_CASE
    return cudaGetLastError();
  }
}

}  // namespace mhd

namespace mhd {

// The magnetic row sweep qualifies for single boxes with x contiguous, nx a
// multiple of 128 up to 1024 (a block of (R + 1) x nx/4 threads), ny a
// multiple of the tile's rows and 16-byte aligned fields.
inline bool mag_rows_qualify(const MagArgs& a) {
  const Box& b = a.box;
  if (a.ens.items || !a.tma || a.passes != 1) return false;
  if (b.stride[0] != 1 || b.stride[1] != b.n[0] || b.stride[2] != (long long)b.n[0] * b.n[1]) return false;
  if (b.n[0] % 128 || b.n[0] > 1024 || b.n[1] % mag_row_tile(b.n[0]) || b.n[2] < 2) return false;
  for (int q = 0; q < 8; q++)
    if (reinterpret_cast<uintptr_t>(a.in[q]) % 16) return false;
  for (int q = 0; q < 3; q++)
    if (reinterpret_cast<uintptr_t>(a.out[q]) % 16) return false;
  return true;
}

// Segment length along z: the divisor of nz (at least 8 planes where nz
// allows) that minimises the warm-up planes per segment times the idle share
// of the last wave (one block per SM).
inline int mag_row_segment(int tiles, int nz, int sms) {
  int best = nz;
  double best_cost = 1e30;
  for (int L = nz; L >= 1; L--) {
    if (nz % L || (L < 8 && L != nz)) continue;
    const double items = (double)tiles * (nz / L);
    const double waves = items / sms;
    const double cost = (double)(L + 2) / L * std::ceil(waves) / waves;
    if (cost < best_cost * 0.999) {
      best = L;
      best_cost = cost;
    }
  }
  return best;
}

template <int LIM, int R>
cudaError_t launch_mag_rows_r(const MagArgs& a, cudaStream_t s) {
  const int nx = a.box.n[0], ny = a.box.n[1], nz = a.box.n[2];
  const size_t smem = mag_row_smem<R>(nx);
  cudaError_t e =
      cudaFuncSetAttribute(mag_row_kernel<LIM, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tiles = ny / R;
  const int L = mag_row_segment(tiles, nz, sms > 0 ? sms : 1);
  mag_row_kernel<LIM, R><<<tiles * (nz / L), dim3(nx / kRowCells, R + 1), smem, s>>>(a, L);
  return cudaGetLastError();
}

template <int LIM>
cudaError_t launch_mag_rows(const MagArgs& a, cudaStream_t s) {
  return mag_row_tile(a.box.n[0]) == 4 ? launch_mag_rows_r<LIM, 4>(a, s) : launch_mag_rows_r<LIM, 2>(a, s);
}

}  // namespace mhd
