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
// coalesced 128-byte row; for the x sweep a warp stages 8 cells of its 32
// pencils in shared memory, loading whole 32-byte sectors.
//
// The sweep writes out of place (in -> out): neighbouring threads read the
// transverse faces of this thread's pencil.
//
// With RATE = true the kernel also evaluates the CFL signal rate of every
// cell it writes (Section II.B: the next timestep) and folds the maximum into
// *rate with one atomicMax per warp, saving a separate pass over the state.
//
// LIM selects the slope limiter and FRZ the freezing speed (0 / 0: the
// paper's scheme; the others are ablations).  This header holds the kernel
// template; each scheme variant is instantiated in its own translation unit
// (sweep_fluid.cu: the paper's scheme; sweep_variant_*.cu: the ablations).
#pragma once
#include "mhd_device.cuh"
#include "mhd_launch.h"
#include "sweep_row.cuh"
#include "tma.cuh"

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

// TMA staging of the y and z kernel-axis sweeps.  One thread of the block
// copies each 4-position chunk of the block's 32 x 4 pencils into shared
// memory with 3-D tensor-tile copies, one chunk ahead of the chunk the warps
// compute on (two buffers, one mbarrier each).  A chunk buffer holds, as
// [position][row][lane] floats: rho, m_d, m_t1, m_t2, e, the face field b_A
// of the lane axis and b_O of the row axis (4 positions each), b_d at 5
// positions (the high face of the last cell), and the two neighbour pencils
// one block over: b_A at lanes 32..35 (4 rows x 4 lanes per position, each
// position in its own 128-byte slot: a tile copy lands on a 128-byte
// boundary) and b_O at row 4 (4 x 32).  Chunks that cross the periodic wrap
// along the pencil, and the b_A edge always, are copied one position at a
// time (the row maps).
constexpr int kTmaCh = 4;                                  // positions per chunk
constexpr int kTmaField = kTmaCh * kFluidWarps * 32;       // 512 floats
constexpr int kTmaOffBd = 7 * kTmaField;                   // b_d: 5 positions
constexpr int kTmaOffAe = kTmaOffBd + (kTmaCh + 1) * kFluidWarps * 32;  // b_A, lanes 32..35
constexpr int kTmaAeSlot = 32;                             // floats per position of the b_A edge
constexpr int kTmaOffOe = kTmaOffAe + kTmaCh * kTmaAeSlot; // b_O, row 4
constexpr int kTmaFloats = kTmaOffOe + kTmaCh * 32;        // 4480 floats = 17,920 bytes
constexpr int kTmaBytes = (kTmaFloats - kTmaCh * (kTmaAeSlot - 4 * kFluidWarps)) * 4;  // 17,664 copied
// Copy chunk `p0 .. p0+3` (b_d to p0+4) of the block at lane x0, row y0 into
// the buffer at `dst` and arm its mbarrier with the chunk's bytes.
__device__ __forceinline__ void tma_issue_chunk(const FluidMaps* mp, uint32_t dst, uint32_t bar, int x0, int y0,
                                                int xe, int ye, int p0, int nD) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kTmaBytes) : "memory");
  const bool whole = p0 >= 0 && p0 + kTmaCh < nD;
  if (whole) {
#pragma unroll
    for (int f = 0; f < 7; f++) tma_load3(dst + f * kTmaField * 4, &mp->full[f], x0, y0, p0, bar);
    tma_load3(dst + kTmaOffBd * 4, &mp->full[7], x0, y0, p0, bar);
    tma_load3(dst + kTmaOffOe * 4, &mp->full[9], x0, ye, p0, bar);
  }
#pragma unroll
  for (int j = 0; j < kTmaCh; j++)
    tma_load3(dst + (kTmaOffAe + j * kTmaAeSlot) * 4, &mp->row[8], xe, y0, wrap_near<false>(p0 + j, nD), bar);
  if (!whole) {  // across the periodic wrap: one position at a time
    for (int j = 0; j <= kTmaCh; j++) {
      const int q = wrap_near<false>(p0 + j, nD);
      tma_load3(dst + (kTmaOffBd + j * kFluidWarps * 32) * 4, &mp->row[7], x0, y0, q, bar);
      if (j == kTmaCh) break;
#pragma unroll
      for (int f = 0; f < 7; f++)
        tma_load3(dst + (f * kTmaField + j * kFluidWarps * 32) * 4, &mp->row[f], x0, y0, q, bar);
      tma_load3(dst + (kTmaOffOe + j * 32) * 4, &mp->row[9], x0, ye, q, bar);
    }
  }
}

// x sweeps: each warp stages 8 cells x 32 pencils of every source field in
// shared memory (rows padded to 9 floats: conflict-free column reads), loaded
// as 32-byte row pieces so each DRAM sector is fetched by exactly one load.
constexpr int kXChunk = 8;
constexpr int kXPad = 9;
constexpr int kXTiles = 10;  // rho, m_d, m_t1, m_t2, e, b_d, b_t1, b_t1(+1), b_t2, b_t2(+1)
constexpr int kXTile = 32 * kXPad;

// Stage positions p0 .. p0+7 (periodic along x, p0 a multiple of 4) of the
// pencils whose flat base index lane r holds in `rowbase` into tile[r][0..7].
template <bool SMALL>
__device__ __forceinline__ void stage_rows(float* tile, const float* __restrict__ src,
                                           int rowbase, int p0, int nx, int lane) {
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int r = 16 * k + (lane >> 1), h = lane & 1;
    const int rb = __shfl_sync(0xffffffffu, rowbase, r);
    const float4 v = __ldg(reinterpret_cast<const float4*>(src + rb + wrap_near<SMALL>(p0 + 4 * h, nx)));
    float* t = tile + r * kXPad + 4 * h;
    t[0] = v.x;
    t[1] = v.y;
    t[2] = v.z;
    t[3] = v.w;
  }
}

// The sweep of one block.  TMA = true (kernel axes 1 and 2, single boxes
// whose lane extent is a multiple of 32 and row extent a multiple of 4): the
// chunks come from the shared-memory ring the block's first thread fills with
// tensor-tile copies (`mp`); the arithmetic is the same as with register loads.
template <int D, bool RATE, bool SMALL, bool FLOOR, int LIM, int FRZ, bool TMA>
__device__ __forceinline__ void fluid_sweep_body(const FluidArgs& a, const FluidMaps* mp) {
  using X = Axes<D>;
  static_assert(!TMA || (D != 0 && !SMALL), "TMA staging: kernel axes 1 and 2, long pencils");
  constexpr int CH = (D == 0) ? kXChunk : 4;  // positions per chunk
  static_assert(!TMA || CH == kTmaCh, "chunk of the staged layout");
  __shared__ float xs[(D == 0) ? kFluidWarps * kXTiles * kXTile : 1];
  __shared__ alignas(128) float tb[TMA ? 2 * kTmaFloats : 1];
  __shared__ alignas(8) unsigned long long tbar[2];
  const int lane = threadIdx.x;
  const BlockGeom G = block_geom(a.ens, a.box, a.seg, a.tau, a.rate);
  const int nA = G.box.n[X::A], nO = G.box.n[X::O], nD = G.box.n[D];
  // Pencils of the block: the TMA-staged and x sweeps take a tile of 32
  // lanes x kFluidWarps rows; the register-load y and z sweeps take 32 x
  // kFluidWarps consecutive pencils in row order (lane axis fastest), so a
  // lane extent that is not a multiple of 32 (48 in the ensemble's boxes)
  // leaves no lane idle: a warp then spans at most two rows, each a
  // contiguous piece.
  constexpr bool kLinear = !TMA && D != 0;
  int pa, pb;
  if constexpr (kLinear) {
    const int P = G.bx * (32 * kFluidWarps) + threadIdx.y * 32 + lane;
    pb = P / nA;
    pa = P - pb * nA;
  } else {
    pa = G.bx * 32 + lane;
    pb = G.by * kFluidWarps + threadIdx.y;
  }
  const bool active = (pa < nA) && (pb < nO);
  const int ia = min(pa, nA - 1), ib = min(pb, nO - 1);
  const int sA = (int)G.box.stride[X::A], sO = (int)G.box.stride[X::O], sD = (int)G.box.stride[D];
  const int base = ia * sA + ib * sO;
  const int baseA1 = wrapi(ia + 1, nA) * sA + ib * sO;  // pencil +1 along A
  const int baseO1 = ia * sA + wrapi(ib + 1, nO) * sO;  // pencil +1 along O
  // +1 along the local-frame transverse axes
  const int baseT1 = (X::T1 == X::A) ? baseA1 : baseO1;
  const int baseT2 = (X::T2 == X::A) ? baseA1 : baseO1;

  const float* __restrict__ rho = a.in[RHO] + G.off;
  const float* __restrict__ md = a.in[MX + D] + G.off;
  const float* __restrict__ m1 = a.in[MX + X::T1] + G.off;
  const float* __restrict__ m2 = a.in[MX + X::T2] + G.off;
  const float* __restrict__ en = a.in[EN] + G.off;
  const float* __restrict__ bd = a.in[BX + D] + G.off;
  const float* __restrict__ b1 = a.in[BX + X::T1] + G.off;
  const float* __restrict__ b2 = a.in[BX + X::T2] + G.off;
  float* __restrict__ o_rho = a.out[RHO] + G.off;
  float* __restrict__ o_md = a.out[MX + D] + G.off;
  float* __restrict__ o_m1 = a.out[MX + X::T1] + G.off;
  float* __restrict__ o_m2 = a.out[MX + X::T2] + G.off;
  float* __restrict__ o_en = a.out[EN] + G.off;
  float* xw = xs + (D == 0 ? threadIdx.y * kXTiles * kXTile : 0);  // this warp's tiles
  // 32-bit unsigned indices from the block-uniform field pointers
  const unsigned ub = (unsigned)base, ubT1 = (unsigned)baseT1, ubT2 = (unsigned)baseT2;

  const float gamma = a.gamma;
  const float tau = G.tau;
  const float c_full = tau * G.box.ih[D];  // tau / h_D
  const float c_half = 0.5f * c_full;    // tau / (2 h_D)
  const int s0 = G.bz * G.seg;
  const int s1 = s0 + G.seg;
  // positions s0-4 .. s1+2 feed outputs s0 .. s1-1 (3 cells of lag, 1 extra
  // warm-up cell so that x chunks start 16-byte aligned)
  const int nchunk = (G.seg + 7 + CH - 1) / CH;

  // staged chunks: this thread's element of a field, and the element of its
  // neighbour pencil along A and along O: the next lane / row of the block,
  // or the edge columns / edge row copied from the next block along A / O
  // (from lane / row 0 of the box where the next pencil wraps around; in a
  // tile cut by the box's end the lanes and rows past it read zeros and
  // store nothing); per-position strides of those two
  const int w = threadIdx.y;
  const int t0 = w * 32 + lane;
  const int x0 = G.bx * 32, y0 = G.by * kFluidWarps;
  const bool edgeA = lane == 31 || x0 + lane + 1 >= nA, edgeO = w == kFluidWarps - 1 || y0 + w + 1 >= nO;
  const int nbA = edgeA ? kTmaOffAe + w * 4 : 5 * kTmaField + t0 + 1;
  const int nbA_step = edgeA ? kTmaAeSlot : kFluidWarps * 32;
  const int nbO = edgeO ? kTmaOffOe + lane : 6 * kTmaField + t0 + 32;
  const int nbO_step = edgeO ? 32 : kFluidWarps * 32;
  const int tid = w * 32 + lane;
  // the next block's first lane / row, or lane / row 0 across the box's end
  const int xe = x0 + 32 >= nA ? 0 : x0 + 32, ye = y0 + kFluidWarps >= nO ? 0 : y0 + kFluidWarps;
  const bool full_tile = x0 + 32 <= nA && y0 + kFluidWarps <= nO;
  if constexpr (TMA) {
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tbar[0])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tbar[1])) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) tma_issue_chunk(mp, smem_u32(tb), smem_u32(&tbar[0]), x0, y0, xe, ye, s0 - 4, nD);
  }

  FluidPipe<LIM, FRZ, TMA> pipe;  // the staged sweep takes the fast square root
  pipe.init();
  if constexpr (FRZ == 2) {  // the pencil's freezing speeds (two reduction passes before the sweep)
    const int pc = ib * nA + ia;
    pipe.c1 = __ldg(a.pencil_c + pc);
    pipe.c2 = __ldg(a.pencil_c + (long long)nA * nO + pc);
  }
  float bc2[3] = {0.f, 0.f, 0.f}, bc3[3] = {0.f, 0.f, 0.f};  // b_c at t-1, t-2 (RATE only)
  float rmax = 0.f;
  const bool rate_pencil = RATE && pa >= a.rate_lo[X::A] && pa < a.rate_hi[X::A] && pb >= a.rate_lo[X::O] &&
                           pb < a.rate_hi[X::O];
  bool gave_up = false;  // TMA: a chunk's copies did not arrive within the bound
  int issued = 1;        // TMA: chunks issued so far (the same count in every thread)

  for (int c = 0; c < nchunk; c++) {
    const int p0 = s0 - 4 + CH * c;  // first position of this chunk
    // D != 0: the chunk's planes in registers or staged; D == 0: staged rows
    float U[(D == 0 || TMA) ? 1 : CH][5], B[(D == 0 || TMA) ? 1 : CH][3];
    const float* row = xw + lane * kXPad;
    const float* sb = tb + (TMA ? (c & 1) * kTmaFloats : 0);
    float bd_next = 0.f;
    if constexpr (TMA) {
      // every warp is done with chunk c-1, whose buffer receives chunk c+1
      if (__syncthreads_or(gave_up)) break;
      if (c + 1 < nchunk) {
        if (tid == 0)
          tma_issue_chunk(mp, smem_u32(tb + ((c + 1) & 1) * kTmaFloats), smem_u32(&tbar[(c + 1) & 1]), x0, y0, xe,
                          ye, p0 + CH, nD);
        issued++;
      }
      if (!sweep_mbar_wait(smem_u32(&tbar[c & 1]), (c >> 1) & 1)) gave_up = true;
    } else if constexpr (D == 0) {
      __syncwarp();
      stage_rows<SMALL>(xw + 0 * kXTile, rho, base, p0, nD, lane);
      stage_rows<SMALL>(xw + 1 * kXTile, md, base, p0, nD, lane);
      stage_rows<SMALL>(xw + 2 * kXTile, m1, base, p0, nD, lane);
      stage_rows<SMALL>(xw + 3 * kXTile, m2, base, p0, nD, lane);
      stage_rows<SMALL>(xw + 4 * kXTile, en, base, p0, nD, lane);
      stage_rows<SMALL>(xw + 5 * kXTile, bd, base, p0, nD, lane);
      stage_rows<SMALL>(xw + 6 * kXTile, b1, base, p0, nD, lane);
      stage_rows<SMALL>(xw + 7 * kXTile, b1, baseT1, p0, nD, lane);
      stage_rows<SMALL>(xw + 8 * kXTile, b2, base, p0, nD, lane);
      stage_rows<SMALL>(xw + 9 * kXTile, b2, baseT2, p0, nD, lane);
      bd_next = __ldg(bd + base + wrap_near<SMALL>(p0 + CH, nD));  // high face of the last cell
      __syncwarp();
    } else {
      // one coalesced row per plane (an L2 prefetch of the next chunk's 10
      // rows on top measured slower: 1.50 -> 1.60 ms along y at 512^3).
      // Offsets along the pencil: only a chunk that crosses the periodic
      // wrap needs the wrapped form; the others advance linearly.
      float bdn[CH + 1], t1n[CH], t2n[CH];
      int off[CH + 1];
      if (SMALL || p0 < 0 || p0 + CH >= nD) {
#pragma unroll
        for (int j = 0; j <= CH; j++) off[j] = wrap_near<SMALL>(p0 + j, nD) * sD;
      } else {
        const int o0 = p0 * sD;
#pragma unroll
        for (int j = 0; j <= CH; j++) off[j] = o0 + j * sD;
      }
#pragma unroll
      for (int j = 0; j < CH; j++) {
        U[j][0] = __ldg(rho + (ub + (unsigned)off[j]));
        U[j][1] = __ldg(md + (ub + (unsigned)off[j]));
        U[j][2] = __ldg(m1 + (ub + (unsigned)off[j]));
        U[j][3] = __ldg(m2 + (ub + (unsigned)off[j]));
        U[j][4] = __ldg(en + (ub + (unsigned)off[j]));
        bdn[j] = __ldg(bd + (ub + (unsigned)off[j]));
        B[j][1] = __ldg(b1 + (ub + (unsigned)off[j]));
        B[j][2] = __ldg(b2 + (ub + (unsigned)off[j]));
        t1n[j] = __ldg(b1 + (ubT1 + (unsigned)off[j]));
        t2n[j] = __ldg(b2 + (ubT2 + (unsigned)off[j]));
      }
      bdn[CH] = __ldg(bd + (ub + (unsigned)off[CH]));
#pragma unroll
      for (int j = 0; j < CH; j++) {
        // cell-centred field: mean of the low and high face of the cell
        B[j][0] = face_mean(bdn[j], bdn[j + 1]);
        B[j][1] = face_mean(B[j][1], t1n[j]);
        B[j][2] = face_mean(B[j][2], t2n[j]);
      }
    }
    // The chunk's positions.  `all` (a literal at each call) says that every
    // cell the chunk finishes lies in this segment, so the staged sweep's
    // steady chunks store without a per-position test (1.135 -> 1.108 ms
    // at 512^3).
    auto positions = [&](const bool all) {
#pragma unroll
      for (int j = 0; j < CH; j++) {
        float o[5], Uj[5], Bj[3];
        if constexpr (TMA) {
          const int e = t0 + j * kFluidWarps * 32;  // [position j][row w][lane]
#pragma unroll
          for (int q = 0; q < 5; q++) Uj[q] = sb[q * kTmaField + e];
          const float bA = sb[5 * kTmaField + e], bO = sb[6 * kTmaField + e];
          const float bA1 = sb[nbA + j * nbA_step], bO1 = sb[nbO + j * nbO_step];
          // cell-centred field: mean of the low and high face of the cell
          Bj[0] = face_mean(sb[kTmaOffBd + e], sb[kTmaOffBd + e + kFluidWarps * 32]);
          Bj[1] = (X::T1 == X::A) ? face_mean(bA, bA1) : face_mean(bO, bO1);
          Bj[2] = (X::T2 == X::A) ? face_mean(bA, bA1) : face_mean(bO, bO1);
        } else if constexpr (D == 0) {
#pragma unroll
          for (int q = 0; q < 5; q++) Uj[q] = row[q * kXTile + j];
          const float hi = (j + 1 < CH) ? row[5 * kXTile + j + 1] : bd_next;
          // cell-centred field: mean of the low and high face of the cell
          Bj[0] = face_mean(row[5 * kXTile + j], hi);
          Bj[1] = face_mean(row[6 * kXTile + j], row[7 * kXTile + j]);
          Bj[2] = face_mean(row[8 * kXTile + j], row[9 * kXTile + j]);
        } else {
#pragma unroll
          for (int q = 0; q < 5; q++) Uj[q] = U[j][q];
          Bj[0] = B[j][0];
          Bj[1] = B[j][1];
          Bj[2] = B[j][2];
        }
        const float bprev0 = pipe.b1[0], bprev1 = pipe.b1[1], bprev2 = pipe.b1[2];  // b_c(t-1)
        pipe.step(Uj, Bj, gamma, c_half, c_full, o);
        const int t = p0 + j;
        const int po = t - 3;  // position of the finished cell
        if (all || (active && po >= s0 && po < s1)) {
          const unsigned cell = ub + (unsigned)(po * sD);  // po is inside [s0, s1)
          if (FLOOR) o[4] = floored_energy(o, bc3, gamma, a.p_floor);  // optional (b_c of this cell is bc3)
          o_rho[cell] = o[0];
          o_md[cell] = o[1];
          o_m1[cell] = o[2];
          o_m2[cell] = o[3];
          o_en[cell] = o[4];
          // the rate of interior cells only (ghost layers of non-periodic axes
          // are left out; the whole box otherwise)
          if (RATE && rate_pencil && po >= a.rate_lo[D] && po < a.rate_hi[D]) {
            float m[3], bg[3];
            m[D] = o[1]; m[X::T1] = o[2]; m[X::T2] = o[3];
            bg[D] = bc3[0]; bg[X::T1] = bc3[1]; bg[X::T2] = bc3[2];
            rmax = fmaxf(rmax, cell_rate(o[0], m, o[4], bg, gamma, G.box.ih));
          }
        }
        if (RATE || FLOOR) {  // window of b_c: bc2 = b_c(t-1), bc3 = b_c(t-2) for the next step
          bc3[0] = bc2[0]; bc3[1] = bc2[1]; bc3[2] = bc2[2];
          bc2[0] = bprev0; bc2[1] = bprev1; bc2[2] = bprev2;
        }
      }
  
    };
    if (TMA && full_tile && p0 >= s0 + 3 && p0 < s1)
      positions(true);
    else
      positions(false);
}
  if constexpr (TMA) {
    if (__syncthreads_or(gave_up)) {
      // record the failure, then let the copies still in flight (the last
      // two chunks issued) land before the block's shared memory is released
      if (tid == 0) {
        atomicOr(a.err, 1u);
        for (int q = max(0, issued - 2); q < issued; q++) sweep_mbar_wait(smem_u32(&tbar[q & 1]), (q >> 1) & 1);
      }
      return;
    }
  }
  if (RATE) {
    for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if (lane == 0) atomicMax(G.rate, __float_as_uint(rmax));
  }
}

// 4 blocks of 128 threads per SM, so at most 128 registers per thread: the
// RATE variant spills a few words at that limit (it needs about 160), which
// measured faster than 3 blocks per SM without spills (1.77 against 1.85 ms
// at 512^3).
template <int D, bool RATE, bool SMALL, bool FLOOR, int LIM, int FRZ>
__global__ void __launch_bounds__(32 * kFluidWarps, 4)
fluid_sweep_kernel(FluidArgs a) {
  fluid_sweep_body<D, RATE, SMALL, FLOOR, LIM, FRZ, false>(a, nullptr);
}

// The TMA-staged sweep (kernel axes 1 and 2, scheme (LIM, FRZ)).
template <int D, bool RATE, bool FLOOR, int LIM, int FRZ>
__global__ void __launch_bounds__(32 * kFluidWarps, 4)
fluid_sweep_tma_kernel(const __grid_constant__ FluidArgs a, const __grid_constant__ FluidMaps mp) {
  fluid_sweep_body<D, RATE, false, FLOOR, LIM, FRZ, true>(a, &mp);
}

// Launch of one fluid sweep with scheme (LIM, FRZ): kernel axis, fused CFL
// rate, short axis and pressure floor select the instantiation.
template <int LIM, int FRZ>
cudaError_t launch_fluid_t(int axis, bool rate, const FluidArgs& a, cudaStream_t s) {
  const int A = (axis == 0) ? 1 : 0, O = (axis == 2) ? 1 : 2;
  dim3 block(32, kFluidWarps);
  // tiles of 32 x kFluidWarps pencils (TMA-staged and x sweeps) or runs of
  // 32 kFluidWarps consecutive pencils (register-load y and z sweeps)
  const dim3 tiles((a.box.n[A] + 31) / 32, (a.box.n[O] + kFluidWarps - 1) / kFluidWarps, a.box.n[axis] / a.seg);
  dim3 grid = axis == 0 ? tiles
                        : dim3((unsigned)(((long long)a.box.n[A] * a.box.n[O] + 32 * kFluidWarps - 1) /
                                          (32 * kFluidWarps)),
                               1, a.box.n[axis] / a.seg);
  // ensemble launches: one block per work item; `small` must hold for every
  // box of the launch (the host passes the smallest extent in a.box)
  if (a.ens.items) grid = dim3(a.nblocks, 1, 1);
  const bool small = a.box.n[axis] < 16;
  const bool floor = a.p_floor > 0.f;
  if (axis == 0 && fluid_rows_qualify(a)) {  // x sweeps over whole staged rows
    if (a.tma_used) *a.tma_used = 1;
    return launch_fluid_rows<LIM, FRZ>(rate, a, s);
  }
  {  // TMA-staged y and z kernel-axis sweeps
    FluidMaps mp;
    if (a.tma && !a.ens.items && axis != 0 && !small && make_fluid_maps(axis, a, &mp)) {
      if (a.tma_used) *a.tma_used = 1;
#define FLUID_TMA_CASE(DD, RR, FF) \
  if (axis == DD && rate == RR && floor == FF)                                                       \
    fluid_sweep_tma_kernel<DD, RR, FF, LIM, FRZ><<<tiles, block, 0, s>>>(a, mp);
      FLUID_TMA_CASE(1, false, false) FLUID_TMA_CASE(1, true, false) FLUID_TMA_CASE(2, false, false)
      FLUID_TMA_CASE(2, true, false) FLUID_TMA_CASE(1, false, true) FLUID_TMA_CASE(1, true, true)
      FLUID_TMA_CASE(2, false, true) FLUID_TMA_CASE(2, true, true)
#undef FLUID_TMA_CASE
      return cudaGetLastError();
    }
  }
#define FLUID_CASE(DD, RR)                                                                            \
  if (axis == DD && rate == RR) {                                                                     \
    if (floor) {                                                                                      \
      if (small) fluid_sweep_kernel<DD, RR, true, true, LIM, FRZ><<<grid, block, 0, s>>>(a);         \
      else fluid_sweep_kernel<DD, RR, false, true, LIM, FRZ><<<grid, block, 0, s>>>(a);              \
    } else {                                                                                          \
      if (small) fluid_sweep_kernel<DD, RR, true, false, LIM, FRZ><<<grid, block, 0, s>>>(a);        \
      else fluid_sweep_kernel<DD, RR, false, false, LIM, FRZ><<<grid, block, 0, s>>>(a);             \
    }                                                                                                 \
  }
  FLUID_CASE(0, false) FLUID_CASE(0, true) FLUID_CASE(1, false) FLUID_CASE(1, true)
  FLUID_CASE(2, false) FLUID_CASE(2, true)
#undef FLUID_CASE
  return cudaGetLastError();
}

}  // namespace mhd
