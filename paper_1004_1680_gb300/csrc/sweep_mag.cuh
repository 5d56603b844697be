// Magnetic advection-constraint sweep along one axis D (Section II.B), FP32.
//
// For each transverse axis t the face field b_t is advected along D by the
// upwind + van Leer, 2-stage scheme (MagPipe), and the edge flux f_t it
// produces is applied to b_D:
//   b_t(cell)          -= tau/h_D (f_t(i+1/2) - f_t(i-1/2))
//   b_D(face i+1/2, P) += tau/h_t (f_t(pencil P+e_t) - f_t(pencil P)),
// which keeps the discrete div b of every cell unchanged (Eq. 5).  The edge
// flux lives on the edge (D: i+1/2, t: low face of pencil P); the EMF pieces
// are applied directly and never written to memory.
//
// Velocities v_D = m_D/rho are formed once per loaded value.
//
// A block owns a tile of 32 (lane axis A) x kMagWarps (row axis O) pencils and
// marches all of them together along D.  Two extra warps march the halo
// pencils whose flux the tile needs: row O+kMagWarps (its f along O) and
// column A+32 (its f along A).  Fluxes are exchanged through shared memory
// once per chunk of positions.  Writes are out of place.
//
// mag_sweep_kernel sweeps along x itself (the staged x path: rows of 8 cells
// staged in shared memory); mag_sweep_pipe_kernel sweeps along y and z, and
// along x on the x <-> y exchanged copy.
//
// LIM selects the slope limiter (0: van Leer, the paper's; 1 minmod and 2
// superbee are ablations, instantiated in sweep_variant_*.cu).
#pragma once
#include "mhd_device.cuh"
#include "mhd_launch.h"
#include "sweep_row.cuh"
#include "tma.cuh"

namespace mhd {

// The constraint on b_D from the two transverse edge-flux differences,
// applied in the order of the local frame (first transverse axis first), each
// rounded once: b + k_A (fA1 - fA0) + k_O (fO1 - fO0).
__device__ __forceinline__ float constrain(float b, float kA, float fa0, float fa1, float kO, float fo0,
                                          float fo1, bool a_first) {
  if (a_first) {
    b = __fmaf_rn(kA, __fsub_rn(fa1, fa0), b);
    return __fmaf_rn(kO, __fsub_rn(fo1, fo0), b);
  }
  b = __fmaf_rn(kO, __fsub_rn(fo1, fo0), b);
  return __fmaf_rn(kA, __fsub_rn(fa1, fa0), b);
}

template <int D>
struct MagAxes {
  static constexpr int A = (D == 0) ? 1 : 0;
  static constexpr int O = (D == 2) ? 1 : 2;
  static constexpr int T1 = (D + 1) % 3;
};

// x sweeps stage 8 cells of each warp's 32 pencils in shared memory (rows of
// 9 floats, 32-byte sector loads): v_x = m_x/rho at the pencil and at its -A
// and -O neighbours, and the three face fields.
constexpr int kMXChunk = 8;
constexpr int kMXPad = 9;
constexpr int kMXTiles = 6;
constexpr int kMXTile = 32 * kMXPad;
constexpr size_t kMagXSmem = sizeof(float) * (kMagWarps + 2) * kMXTiles * kMXTile;

template <bool SMALL>
__device__ __forceinline__ void stage_rows_m(float* tile, const float* __restrict__ src,
                                             int rowbase, int p0, int nx, int lane) {
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int r = 16 * k + (lane >> 1), h = lane & 1;
    const int rb = __shfl_sync(0xffffffffu, rowbase, r);
    const float4 v = __ldg(reinterpret_cast<const float4*>(src + rb + wrap_near<SMALL>(p0 + 4 * h, nx)));
    float* t = tile + r * kMXPad + 4 * h;
    t[0] = v.x;
    t[1] = v.y;
    t[2] = v.z;
    t[3] = v.w;
  }
}

// velocity rows: v = m / rho
template <bool SMALL>
__device__ __forceinline__ void stage_vel(float* tile, const float* __restrict__ rho,
                                          const float* __restrict__ m, int rowbase, int p0,
                                          int nx, int lane) {
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int r = 16 * k + (lane >> 1), h = lane & 1;
    const int rb = __shfl_sync(0xffffffffu, rowbase, r);
    const int off = wrap_near<SMALL>(p0 + 4 * h, nx);
    const float4 rr = __ldg(reinterpret_cast<const float4*>(rho + rb + off));
    const float4 mm = __ldg(reinterpret_cast<const float4*>(m + rb + off));
    float* t = tile + r * kMXPad + 4 * h;
    t[0] = v_div(mm.x, rr.x);
    t[1] = v_div(mm.y, rr.y);
    t[2] = v_div(mm.z, rr.z);
    t[3] = v_div(mm.w, rr.w);
  }
}

template <int D, bool SMALL, int LIM>
__global__ void __launch_bounds__(32 * (kMagWarps + 2), 2)
mag_sweep_kernel(MagArgs a) {
  static_assert(D == 0, "y and z sweeps use mag_sweep_pipe_kernel");
  using X = MagAxes<D>;
  constexpr int CH = kMXChunk;
  // double-buffered by chunk parity: a chunk's fluxes are written while the
  // previous chunk's may still be read, so one barrier per chunk suffices
  __shared__ float fA_s[2][CH][kMagWarps][33];       // flux of b_A, column 32 = halo column
  __shared__ float fO_s[2][CH][kMagWarps + 1][32];   // flux of b_O, row kMagWarps = halo row
  extern __shared__ float xs_dyn[];               // staged rows

  const int lane = threadIdx.x, w = threadIdx.y;
  const BlockGeom G = block_geom(a.ens, a.box, a.seg, a.tau, nullptr);
  const int nA = G.box.n[X::A], nO = G.box.n[X::O], nD = G.box.n[D];
  const int a0 = G.bx * 32, b0 = G.by * kMagWarps;
  const int cntA = min(32, nA - a0), cntO = min(kMagWarps, nO - b0);

  // this thread's pencil and role
  int pa, pb;
  bool interior = false;
  int row, col;  // slot in the exchange arrays
  if (w < kMagWarps) {
    pa = a0 + min(lane, cntA - 1);
    pb = b0 + min(w, cntO - 1);
    interior = (lane < cntA) && (w < cntO);
    row = w;
    col = lane;
  } else if (w == kMagWarps) {             // halo row: pencils (a0+lane, b0+cntO)
    pa = a0 + min(lane, cntA - 1);
    pb = wrapi(b0 + cntO, nO);
    row = cntO;
    col = lane;
  } else {                                 // halo column: pencils (a0+cntA, b0+lane)
    pa = wrapi(a0 + cntA, nA);
    pb = b0 + min(lane, cntO - 1);
    row = min(lane, kMagWarps - 1);
    col = cntA;
  }
  const int sA = (int)G.box.stride[X::A], sO = (int)G.box.stride[X::O], sD = (int)G.box.stride[D];
  const int base = pa * sA + pb * sO;
  const int baseAm = wrapi(pa - 1, nA) * sA + pb * sO;  // pencil -1 along A
  const int baseOm = pa * sA + wrapi(pb - 1, nO) * sO;  // pencil -1 along O

  const float* __restrict__ rho = a.in[RHO] + G.off;
  const float* __restrict__ md = a.in[MX + D] + G.off;
  const float* __restrict__ bA = a.in[BX + X::A] + G.off;
  const float* __restrict__ bO = a.in[BX + X::O] + G.off;
  const float* __restrict__ bD = a.in[BX + D] + G.off;
  float* __restrict__ o_bA = a.out[X::A] + G.off;
  float* __restrict__ o_bO = a.out[X::O] + G.off;
  float* __restrict__ o_bD = a.out[D] + G.off;
  float* xw = xs_dyn + w * kMXTiles * kMXTile;

  const float tau = G.tau;
  const float c_full = tau * G.box.ih[D];      // tau / h_D
  const float c_half = 0.5f * c_full;
  const float kA = tau * G.box.ih[X::A];       // tau / h_A
  const float kO = tau * G.box.ih[X::O];       // tau / h_O
  const int s0 = G.bz * G.seg;
  const int s1 = s0 + G.seg;
  // positions s0-4 .. s1+2 feed outputs s0 .. s1-1 (3 cells of lag, 1 extra
  // warm-up cell so that x chunks start 16-byte aligned)
  const int nchunk = (G.seg + 7 + CH - 1) / CH;
  // slots read by the tile: fO rows 0..cntO (row cntO = halo row), fA columns
  // 0..cntA (column cntA = halo column); idle lanes of a partial tile must not
  // overwrite a halo slot
  const bool write_row = (w < kMagWarps) ? (w < cntO) : (w == kMagWarps);
  const bool write_col = (w < kMagWarps) ? (w < cntO && lane < cntA)
                                         : (w == kMagWarps + 1 && lane < cntO);

  MagPipe<LIM> pA, pO;
  pA.init();
  pO.init();
  float bD1 = 0.f, bD2 = 0.f;  // raw b_D at t-1, t-2

  for (int c = 0; c < nchunk; c++) {
    const int p0 = s0 - 4 + CH * c;
    // the chunk's rows staged in shared memory
    const float* rw = xw + lane * kMXPad;
    __syncwarp();
    stage_vel<SMALL>(xw + 0 * kMXTile, rho, md, base, p0, nD, lane);
    stage_vel<SMALL>(xw + 1 * kMXTile, rho, md, baseAm, p0, nD, lane);
    stage_vel<SMALL>(xw + 2 * kMXTile, rho, md, baseOm, p0, nD, lane);
    stage_rows_m<SMALL>(xw + 3 * kMXTile, bA, base, p0, nD, lane);
    stage_rows_m<SMALL>(xw + 4 * kMXTile, bO, base, p0, nD, lane);
    stage_rows_m<SMALL>(xw + 5 * kMXTile, bD, base, p0, nD, lane);
    __syncwarp();
    float bDold[CH];  // raw b_D at the face each position's constraint updates
#pragma unroll
    for (int j = 0; j < CH; j++) {
      const float vj = rw[0 * kMXTile + j];
      const float vAj = rw[1 * kMXTile + j];
      const float vOj = rw[2 * kMXTile + j];
      const float qAj = rw[3 * kMXTile + j];
      const float qOj = rw[4 * kMXTile + j];
      const float qDj = rw[5 * kMXTile + j];
      const float uA = __fmul_rn(0.5f, __fadd_rn(vj, vAj));  // v_D on the b_A face
      const float uO = __fmul_rn(0.5f, __fadd_rn(vj, vOj));  // v_D on the b_O face
      // the halo row needs only the flux along O, the halo column only along A
      float nA_new = 0.f, nO_new = 0.f, fa = 0.f, fo = 0.f;
      if (w != kMagWarps) fa = pA.step(qAj, uA, c_half, c_full, nA_new);
      if (w != kMagWarps + 1) fo = pO.step(qOj, uO, c_half, c_full, nO_new);
      if (write_row) fO_s[c & 1][j][row][col] = fo;
      if (write_col) fA_s[c & 1][j][row][col] = fa;
      bDold[j] = bD2;  // b_D at position t-2, the face of edge t-5/2
      bD2 = bD1;
      bD1 = qDj;
      const int t = p0 + j;
      const int po = t - 3;
      if (interior && po >= s0 && po < s1) {
        const int cell = base + po * sD;  // po is inside [s0, s1)
        o_bA[cell] = nA_new;
        o_bO[cell] = nO_new;
      }
    }
    __syncthreads();
    if (interior) {
#pragma unroll
      for (int j = 0; j < CH; j++) {
        const int t = p0 + j;
        const int pf = t - 2;  // b_D face updated by the edge flux f(t-5/2)
        if (pf >= s0 && pf < s1) {
          const float fa0 = fA_s[c & 1][j][row][col], fa1 = fA_s[c & 1][j][row][col + 1];
          const float fo0 = fO_s[c & 1][j][row][col], fo1 = fO_s[c & 1][j][row + 1][col];
          float b = bDold[j];
          b = constrain(b, kA, fa0, fa1, kO, fo0, fo1, X::T1 == X::A);
          o_bD[base + pf * sD] = b;  // pf is inside [s0, s1)
        }
      }
    }
  }
}

// Sweeps along y and z (D = 1, 2; the x sweeps also run along y, on the
// x <-> y exchanged copy): the same arithmetic as mag_sweep_kernel,
// reorganised for memory-level parallelism and a short instruction stream.
//  * The three warp roles (interior rows, halo row, halo column) run their own
//    specialised loop (mag_pipe_role), chosen once per warp: no role test is
//    left inside the marching loop.  With the tests inside the loop, 124 of
//    246 thread instructions per cell were integer, move and branch overhead
//    (ncu instruction classes at 256^3).
//  * Every thread loads 5 values per position.  An interior pencil loads
//    rho, m_D, b_A, b_O, b_D.  The halo row loads rho, m_D, b_O and rho, m_D
//    of the pencil row below the tile (-O).  The halo column loads rho, m_D,
//    b_A and rho, m_D of the pencil column left of the tile (-A).
//  * v_D = m_D / rho of the -A and -O neighbours comes from shared memory,
//    v_s[row + 1][col + 1] (row 0: the -O pencils, column 0: the -A ones).
//  * The v_D of chunk c + 1 is written to the other half of v_s before
//    chunk c's barrier, which therefore covers both exchanges.  Along y the
//    loads of chunk c + 1 are issued before chunk c is computed; along z,
//    whose positions are a whole plane apart, they are issued after it, and
//    an L2 prefetch of the next chunk's lines goes out before the arithmetic
//    (no registers held): 1.34 -> 1.24 ms at 512^3.  Along y, a prefetch
//    two chunks ahead of the early loads cost 1.15 -> 1.30.
//  * NP = 2 runs two magnetic sweeps along D with the same step in one pass
//    (the two z sweeps in the middle of the schedule, [M_z][M_z], see the same
//    velocity field): each advected component goes through a second MagPipe
//    fed with the first one's output three positions later, with the face
//    velocity delayed to match, and b_D takes the second pass's fluxes on top
//    of the first's.  Every value is rounded as in two separate launches, so
//    the result is bitwise that of two NP = 1 sweeps, for one read and one
//    write of the fields instead of two.
constexpr int kMagCH = 4;  // positions per chunk (one barrier per chunk)

template <int NP>
struct MagShared {
  float fA[NP][2][kMagCH][kMagWarps][33];      // flux of b_A, column 32 = halo column
  float fO[NP][2][kMagCH][kMagWarps + 1][32];  // flux of b_O, row kMagWarps = halo row
  float v[2][kMagCH][kMagWarps + 1][33];       // v_D of the tile's pencils and the -A, -O ones
};

enum { kRoleInterior = 0, kRoleHaloRow = 1, kRoleHaloCol = 2 };

// TMA staging (mag_sweep_tma_kernel): thread 0 copies chunk c+2 into shared
// memory while the block computes chunk c and reads chunk c+1 (two buffers,
// one mbarrier each; a buffer is read only while its chunk's v_D is
// published, before that chunk's barrier).  A chunk buffer holds, as
// [position][row][lane] floats, rho, m_D, b_A, b_O, b_D of the 32 x 8 tile;
// rho and m_D of the row below it and rho, m_D, b_O of the row above it
// (32 lanes); rho, m_D of the four columns left of it and rho, m_D, b_A of
// the four columns right of it (only the nearest column is read).
constexpr int kMRho = 0, kMMd = 1024, kMBA = 2048, kMBO = 3072, kMBD = 4096;  // 4 x 8 x 32
constexpr int kMRhoDn = 5120, kMMdDn = 5248, kMRhoUp = 5376, kMMdUp = 5504, kMBOUp = 5632;  // 4 x 32
constexpr int kMRhoL = 5760, kMMdL = 5888, kMRhoR = 6016, kMMdR = 6144, kMBAR = 6272;      // 4 x 8 x 4
constexpr int kMagTmaFloats = 6400;  // 25,600 bytes per chunk
constexpr size_t kMagTmaSmem = 2 * kMagTmaFloats * 4 + 128;  // dynamic, plus alignment to 128 bytes

// Copy chunk p0 .. p0+3 of the tile at lane x0, row y0 and of its periodic
// neighbour rows and columns into the buffer at `dst`.  The neighbours'
// coordinates are formed here by compare and select (x0, y0 lie inside the
// box) rather than kept in every thread's registers.
__device__ __forceinline__ void mag_issue_chunk(const MagMaps* mp, uint32_t dst, uint32_t bar, int x0, int y0,
                                                int nA, int nO, int p0, int nD) {
  const int ydn = y0 == 0 ? nO - 1 : y0 - 1, yup = y0 + kMagWarps == nO ? 0 : y0 + kMagWarps;
  const int xl = x0 == 0 ? nA - 4 : x0 - 4, xr = x0 + 32 == nA ? 0 : x0 + 32;
  mbar_expect_tx(bar, kMagTmaFloats * 4);
  const bool whole = p0 >= 0 && p0 + kMagCH <= nD;
  const int npos = whole ? 1 : kMagCH;  // across the periodic wrap: one position at a time
  for (int j = 0; j < npos; j++) {
    const CUtensorMap* m = whole ? mp->full : mp->row;
    const int q = whole ? p0 : wrap_near<false>(p0 + j, nD);
    const uint32_t d = dst + 4 * j * 256, r = dst + 4 * j * 32;  // main boxes / row and column boxes
#pragma unroll
    for (int f = 0; f < 5; f++) tma_load3(d + 4 * f * 1024, &m[f], x0, y0, q, bar);
    tma_load3(r + 4 * kMRhoDn, &m[5], x0, ydn, q, bar);
    tma_load3(r + 4 * kMMdDn, &m[6], x0, ydn, q, bar);
    tma_load3(r + 4 * kMRhoUp, &m[5], x0, yup, q, bar);
    tma_load3(r + 4 * kMMdUp, &m[6], x0, yup, q, bar);
    tma_load3(r + 4 * kMBOUp, &m[7], x0, yup, q, bar);
    tma_load3(r + 4 * kMRhoL, &m[8], xl, y0, q, bar);
    tma_load3(r + 4 * kMMdL, &m[9], xl, y0, q, bar);
    tma_load3(r + 4 * kMRhoR, &m[8], xr, y0, q, bar);
    tma_load3(r + 4 * kMMdR, &m[9], xr, y0, q, bar);
    tma_load3(r + 4 * kMBAR, &m[10], xr, y0, q, bar);
  }
}

template <int D, bool SMALL, int LIM, int NP, int ROLE, bool TMA = false>
__device__ __forceinline__ void mag_pipe_role(const MagArgs& a, const BlockGeom& G, MagShared<NP>& sh,
                                              const MagMaps* mp = nullptr, const float* tb = nullptr,
                                              unsigned long long* tfull = nullptr) {
  constexpr bool kEarly = D == 1;  // next chunk's loads before the current chunk's arithmetic
  using X = MagAxes<D>;
  constexpr int CH = kMagCH;
  constexpr bool kA_ = ROLE != kRoleHaloRow;  // advects b_A (flux along A)
  constexpr bool kO_ = ROLE != kRoleHaloCol;  // advects b_O (flux along O)
  const int lane = threadIdx.x, w = threadIdx.y;
  const int nA = G.box.n[X::A], nO = G.box.n[X::O], nD = G.box.n[D];
  const int a0 = G.bx * 32, b0 = G.by * kMagWarps;
  const int cntA = min(32, nA - a0), cntO = min(kMagWarps, nO - b0);

  // this thread's pencil (pa, pb), the extra pencil (ea, eb) of a halo warp,
  // its slots in the exchange arrays and those of the neighbour v_D it reads
  int pa, pb, ea = 0, eb = 0, row, col;
  bool interior = false, wr_row, wr_col, extra = false;
  int vAr, vAc, vOr, vOc;  // v_s slots of the -A and -O neighbours
  if constexpr (ROLE == kRoleInterior) {
    pa = a0 + min(lane, cntA - 1);
    pb = b0 + min(w, cntO - 1);
    interior = (lane < cntA) && (w < cntO);
    row = w;
    col = lane;
    wr_row = w < cntO;
    wr_col = w < cntO && lane < cntA;
    vAr = w + 1; vAc = lane;
    vOr = w;     vOc = lane + 1;
  } else if constexpr (ROLE == kRoleHaloRow) {  // pencils (a0+lane, b0+cntO)
    pa = a0 + min(lane, cntA - 1);
    pb = wrapi(b0 + cntO, nO);
    ea = pa;
    eb = wrapi(b0 - 1, nO);
    extra = true;
    row = cntO;
    col = lane;
    wr_row = true;
    wr_col = false;
    vAr = vAc = 0;
    vOr = cntO; vOc = lane + 1;               // its -O neighbour: tile row cntO - 1
  } else {                                     // halo column: pencils (a0+cntA, b0+lane)
    pa = wrapi(a0 + cntA, nA);
    pb = b0 + min(lane, cntO - 1);
    ea = wrapi(a0 - 1, nA);
    eb = pb;
    extra = lane < kMagWarps;
    row = min(lane, kMagWarps - 1);
    col = cntA;
    wr_row = false;
    wr_col = lane < cntO;
    vAr = min(lane, cntO - 1) + 1; vAc = cntA;  // its -A neighbour: tile column cntA - 1
    vOr = vOc = 0;
  }
  // where this thread's own v_D (interior) or its extra pencil's v_D (halo) goes
  int pr, pc;
  if constexpr (ROLE == kRoleInterior) { pr = w + 1; pc = lane + 1; }
  else if constexpr (ROLE == kRoleHaloRow) { pr = 0; pc = lane + 1; }
  else { pr = lane + 1; pc = 0; }

  const int sA = (int)G.box.stride[X::A], sO = (int)G.box.stride[X::O], sD = (int)G.box.stride[D];
  const int base = pa * sA + pb * sO;
  const int ebase = ea * sA + eb * sO;
  const float* __restrict__ rho = a.in[RHO] + G.off;
  const float* __restrict__ md = a.in[MX + D] + G.off;
  // the role's loads (block-uniform field pointers, 32-bit unsigned
  // indices): own rho and m_D, then interior b_A, b_O, b_D; halo row b_O,
  // rho(-O), m_D(-O); halo column b_A, rho(-A), m_D(-A)
  const float* __restrict__ p2;
  const float* __restrict__ p3;
  const float* __restrict__ p4;
  unsigned i3, i4;
  const unsigned ib = (unsigned)base;
  if constexpr (ROLE == kRoleInterior) {
    p2 = a.in[BX + X::A] + G.off;
    p3 = a.in[BX + X::O] + G.off;
    p4 = a.in[BX + D] + G.off;
    i3 = i4 = ib;
  } else if constexpr (ROLE == kRoleHaloRow) {
    p2 = a.in[BX + X::O] + G.off;
    p3 = rho;
    p4 = md;
    i3 = i4 = (unsigned)ebase;
  } else {
    p2 = a.in[BX + X::A] + G.off;
    p3 = rho;
    p4 = md;
    i3 = i4 = (unsigned)ebase;
  }
  float* __restrict__ o_bA = a.out[X::A] + G.off;
  float* __restrict__ o_bO = a.out[X::O] + G.off;
  float* __restrict__ o_bD = a.out[D] + G.off;

  const float tau = G.tau;
  const float c_full = tau * G.box.ih[D];      // tau / h_D
  const float c_half = 0.5f * c_full;
  const float kA = tau * G.box.ih[X::A];       // tau / h_A
  const float kO = tau * G.box.ih[X::O];       // tau / h_O
  const int s0 = G.bz * G.seg;
  const int s1 = s0 + G.seg;
  // each pass lags its input by 3 positions: positions s0-4NP .. s1+3NP-1
  // feed outputs s0 .. s1-1 (one extra warm-up cell per pass, as in the
  // staged x kernel)
  const int nchunk = (G.seg + 7 * NP + CH - 1) / CH;
  constexpr int kLag = 3 * NP;                 // final b_t at t - kLag, final b_D at face t - kLag + 1

  MagPipe<LIM> pA, pO;      // first pass
  MagPipe<LIM> qA, qO;      // second pass (NP == 2)
  pA.init();
  pO.init();
  qA.init();
  qO.init();
  float uA1 = 0.f, uA2 = 0.f, uA3 = 0.f, uO1 = 0.f, uO2 = 0.f, uO3 = 0.f;  // face velocities at t-1..t-3
  float bD1 = 0.f, bD2 = 0.f;  // raw b_D at t-1, t-2
  float bP1 = 0.f, bP2 = 0.f, bP3 = 0.f;  // b_D after the first pass at faces t-3, t-4, t-5

  float cv[CH], cq2[CH], cq4[CH];  // own v_D; the advected value(s) of the current chunk
  // TMA: the same five values per position from the staged chunk at sb
  auto load_staged = [&](const float* sb, float (&r0)[CH], float (&r1)[CH], float (&r2)[CH], float (&r3)[CH],
                         float (&r4)[CH]) {
#pragma unroll
    for (int j = 0; j < CH; j++) {
      if constexpr (ROLE == kRoleInterior) {
        const int e = j * 256 + w * 32 + lane;
        r0[j] = sb[kMRho + e];
        r1[j] = sb[kMMd + e];
        r2[j] = sb[kMBA + e];
        r3[j] = sb[kMBO + e];
        r4[j] = sb[kMBD + e];
      } else if constexpr (ROLE == kRoleHaloRow) {
        const int e = j * 32 + lane;
        r0[j] = sb[kMRhoUp + e];
        r1[j] = sb[kMMdUp + e];
        r2[j] = sb[kMBOUp + e];
        r3[j] = sb[kMRhoDn + e];
        r4[j] = sb[kMMdDn + e];
      } else {
        const int e = j * 32 + min(lane, kMagWarps - 1) * 4;
        r0[j] = sb[kMRhoR + e];
        r1[j] = sb[kMMdR + e];
        r2[j] = sb[kMBAR + e];
        r3[j] = sb[kMRhoL + e + 3];
        r4[j] = sb[kMMdL + e + 3];
      }
    }
  };
  const int tid = w * 32 + lane;
  bool gave_up = false;  // TMA: a bounded wait ran out (block-uniform after each barrier)
  int issued = 0;        // TMA: chunks issued so far (the same count in every thread)
  if constexpr (TMA) {
    if (tid == 0)
      for (int k = 0; k < 2 && k < nchunk; k++)
        mag_issue_chunk(mp, smem_u32(tb + k * kMagTmaFloats), smem_u32(&tfull[k]), a0, b0, nA, nO,
                        s0 - 4 * NP + CH * k, nD);
    issued = min(2, nchunk);
  }
  auto load_chunk = [&](int p0, float (&r0)[CH], float (&r1)[CH], float (&r2)[CH], float (&r3)[CH],
                        float (&r4)[CH]) {
#pragma unroll
    for (int j = 0; j < CH; j++) {
      const unsigned off = (unsigned)(wrap_near<SMALL>(p0 + j, nD) * sD);
      r0[j] = __ldg(rho + (ib + off));
      r1[j] = __ldg(md + (ib + off));
      r2[j] = __ldg(p2 + (ib + off));
      r3[j] = __ldg(p3 + (i3 + off));
      r4[j] = __ldg(p4 + (i4 + off));
    }
  };
  // v_D of the loaded chunk into registers and v_s[buf]; interior: b_A and
  // b_O (cq2 / r3 kept in cq2, cq4) and b_D; halo warps: their advected field
  // and their extra pencil's v_D
  float cq3[CH];
  auto publish = [&](int buf, const float (&r0)[CH], const float (&r1)[CH], const float (&r2)[CH],
                     const float (&r3)[CH], const float (&r4)[CH]) {
#pragma unroll
    for (int j = 0; j < CH; j++) {
      cv[j] = v_div(r1[j], r0[j]);
      cq2[j] = r2[j];
      if constexpr (ROLE == kRoleInterior) {
        sh.v[buf][j][pr][pc] = cv[j];
        cq3[j] = r3[j];
        cq4[j] = r4[j];
      } else {
        if (extra) sh.v[buf][j][pr][pc] = v_div(r4[j], r3[j]);
      }
    }
  };
  {
    float r0[CH], r1[CH], r2[CH], r3[CH], r4[CH];
    if constexpr (TMA) {
      if (!sweep_mbar_wait(smem_u32(&tfull[0]), 0)) gave_up = true;
      load_staged(tb, r0, r1, r2, r3, r4);
    } else {
      load_chunk(s0 - 4 * NP, r0, r1, r2, r3, r4);
    }
    publish(0, r0, r1, r2, r3, r4);
  }
  if constexpr (TMA) {
    if (__syncthreads_or(gave_up)) gave_up = true;
  } else {
    __syncthreads();
  }

  for (int c = 0; c < nchunk && !gave_up; c++) {
    const int p0 = s0 - 4 * NP + CH * c;
    const bool more = c + 1 < nchunk;
    const int buf = c & 1;
    float n0[CH], n1[CH], n2[CH], n3[CH], n4[CH];
    if constexpr (TMA) {
      // chunk c+2 into the buffer chunk c was read from (before the last barrier)
      if (c + 2 < nchunk) {
        if (tid == 0)
          mag_issue_chunk(mp, smem_u32(tb + buf * kMagTmaFloats), smem_u32(&tfull[buf]), a0, b0, nA, nO,
                          p0 + 2 * CH, nD);
        issued++;
      }
    }
    if (!TMA && kEarly && more) load_chunk(p0 + CH, n0, n1, n2, n3, n4);
    if (!TMA && !kEarly && more) {  // the next chunk's lines into L2 during the arithmetic
#pragma unroll
      for (int j = 0; j < CH; j++) {
        const unsigned off = (unsigned)(wrap_near<SMALL>(p0 + CH + j, nD) * sD);
        prefetch_l2(rho + (ib + off));
        prefetch_l2(md + (ib + off));
        prefetch_l2(p2 + (ib + off));
        prefetch_l2(p3 + (i3 + off));
        prefetch_l2(p4 + (i4 + off));
      }
    }
    float bDold[CH];  // raw b_D at the face each position's constraint updates
    // Every cell and face the chunk finishes lies in this segment: the
    // interior warps of the staged single-pass sweep then store without
    // per-position tests (`all`, a literal at each call; the fused pair
    // would spill with the second copy of its loops).
    const bool steady = TMA && NP == 1 && ROLE == kRoleInterior && p0 - kLag >= s0 && p0 + CH - kLag < s1;
    auto advect = [&](const bool all) {
#pragma unroll
      for (int j = 0; j < CH; j++) {
        const float vj = cv[j];
        float nA_new = 0.f, nO_new = 0.f;
        if constexpr (kA_) {  // flux along A: interior and halo column
          const float uA = __fmul_rn(0.5f, __fadd_rn(vj, sh.v[buf][j][vAr][vAc]));
          const float fa = pA.step(cq2[j], uA, c_half, c_full, nA_new);
          if (wr_col) sh.fA[0][buf][j][row][col] = fa;
          if constexpr (NP == 2) {
            float q2;
            const float fa2 = qA.step(nA_new, uA3, c_half, c_full, q2);
            if (wr_col) sh.fA[1][buf][j][row][col] = fa2;
            nA_new = q2;
            uA3 = uA2;
            uA2 = uA1;
            uA1 = uA;
          }
        }
        if constexpr (kO_) {  // flux along O: interior and halo row
          const float qin = (ROLE == kRoleInterior) ? cq3[j] : cq2[j];
          const float uO = __fmul_rn(0.5f, __fadd_rn(vj, sh.v[buf][j][vOr][vOc]));
          const float fo = pO.step(qin, uO, c_half, c_full, nO_new);
          if (wr_row) sh.fO[0][buf][j][row][col] = fo;
          if constexpr (NP == 2) {
            float q2;
            const float fo2 = qO.step(nO_new, uO3, c_half, c_full, q2);
            if (wr_row) sh.fO[1][buf][j][row][col] = fo2;
            nO_new = q2;
            uO3 = uO2;
            uO2 = uO1;
            uO1 = uO;
          }
        }
        if constexpr (ROLE == kRoleInterior) {
          bDold[j] = bD2;  // b_D at position t-2, the face of edge t-5/2
          bD2 = bD1;
          bD1 = cq4[j];
          const int po = p0 + j - kLag;
          if (all || (interior && po >= s0 && po < s1)) {
            const unsigned cell = ib + (unsigned)(po * sD);  // po is inside [s0, s1)
            o_bA[cell] = nA_new;
            o_bO[cell] = nO_new;
          }
        }
      }
    };
    if (steady)
      advect(true);
    else
      advect(false);
    if constexpr (TMA) {
      if (more) {
        if (!sweep_mbar_wait(smem_u32(&tfull[(c + 1) & 1]), ((c + 1) >> 1) & 1)) gave_up = true;
        load_staged(tb + ((c + 1) & 1) * kMagTmaFloats, n0, n1, n2, n3, n4);
      }
    } else if (!kEarly && more) {
      load_chunk(p0 + CH, n0, n1, n2, n3, n4);
    }
    if (more) publish((c + 1) & 1, n0, n1, n2, n3, n4);
    if constexpr (TMA) {
      if (__syncthreads_or(gave_up)) {
        gave_up = true;
        break;
      }
    } else {
      __syncthreads();
    }
    if constexpr (ROLE == kRoleInterior) {
      auto constraint = [&](const bool all) {
#pragma unroll
        for (int j = 0; j < CH; j++) {
          const int t = p0 + j;
          // first pass: face t-2 takes the edge fluxes f(t-5/2)
          float b = constrain(bDold[j], kA, sh.fA[0][buf][j][row][col], sh.fA[0][buf][j][row][col + 1], kO,
                              sh.fO[0][buf][j][row][col], sh.fO[0][buf][j][row + 1][col], X::T1 == X::A);
          if constexpr (NP == 2) {
            // second pass: face t-5 (first-pass value from three positions ago)
            const float b2 = constrain(bP3, kA, sh.fA[1][buf][j][row][col], sh.fA[1][buf][j][row][col + 1],
                                       kO, sh.fO[1][buf][j][row][col], sh.fO[1][buf][j][row + 1][col],
                                       X::T1 == X::A);
            bP3 = bP2;
            bP2 = bP1;
            bP1 = b;
            b = b2;
          }
          const int pf = t - kLag + 1;
          if (all || (pf >= s0 && pf < s1)) o_bD[ib + (unsigned)(pf * sD)] = b;  // pf is inside [s0, s1)
        }
      };
      if (steady)
        constraint(true);
      else if (interior)
        constraint(false);
    }
  }
  if constexpr (TMA) {
    if (gave_up && tid == 0) {
      // record the failure and let the copies still in flight (at most the
      // last two chunks issued) land before the shared memory is released
      atomicOr(a.err, 1u);
      for (int q = max(0, issued - 2); q < issued; q++) sweep_mbar_wait(smem_u32(&tfull[q & 1]), (q >> 1) & 1);
    }
  }
}

template <int D, bool SMALL, int LIM, int NP>
__global__ void __launch_bounds__(32 * (kMagWarps + 2), 2)
mag_sweep_pipe_kernel(MagArgs a) {
  static_assert(D != 0, "x sweeps use the staged kernel");
  static_assert(NP == 1 || NP == 2, "one or two passes");
  __shared__ MagShared<NP> sh;
  const BlockGeom G = block_geom(a.ens, a.box, a.seg, a.tau, nullptr);
  if (threadIdx.y < kMagWarps) mag_pipe_role<D, SMALL, LIM, NP, kRoleInterior>(a, G, sh);
  else if (threadIdx.y == kMagWarps) mag_pipe_role<D, SMALL, LIM, NP, kRoleHaloRow>(a, G, sh);
  else mag_pipe_role<D, SMALL, LIM, NP, kRoleHaloCol>(a, G, sh);
}

// The TMA-staged sweep along y and z (limiter LIM, long pencils, tiles that
// divide the box): kMagTmaSmem bytes of dynamic shared memory.
template <int D, int NP, int LIM>
__global__ void __launch_bounds__(32 * (kMagWarps + 2), 2)
mag_sweep_tma_kernel(const __grid_constant__ MagArgs a, const __grid_constant__ MagMaps mp) {
  __shared__ MagShared<NP> sh;
  extern __shared__ float mag_dyn[];
  __shared__ alignas(8) unsigned long long tfull[2];
  const BlockGeom G = block_geom(a.ens, a.box, a.seg, a.tau, nullptr);
  // the buffers start at the first 128-byte boundary (a tile copy lands on one)
  const float* tb = mag_dyn + ((128u - (smem_u32(mag_dyn) & 127u)) & 127u) / 4;
  if (threadIdx.y == 0 && threadIdx.x == 0) {
    mbar_init(smem_u32(&tfull[0]), 1);
    mbar_init(smem_u32(&tfull[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.y < kMagWarps) mag_pipe_role<D, false, LIM, NP, kRoleInterior, true>(a, G, sh, &mp, tb, tfull);
  else if (threadIdx.y == kMagWarps) mag_pipe_role<D, false, LIM, NP, kRoleHaloRow, true>(a, G, sh, &mp, tb, tfull);
  else mag_pipe_role<D, false, LIM, NP, kRoleHaloCol, true>(a, G, sh, &mp, tb, tfull);
}

// The x sweep stages rows in more than 48 KB of shared memory; the limit is
// raised once per device before any launch (never during a graph capture).
template <int LIM>
cudaError_t prepare_mag_t() {
  cudaError_t e = cudaFuncSetAttribute(mag_sweep_kernel<0, true, LIM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMagXSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mag_sweep_kernel<0, false, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kMagXSmem);
  {  // the staged sweeps
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mag_sweep_tma_kernel<1, 1, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kMagTmaSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mag_sweep_tma_kernel<2, 1, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kMagTmaSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mag_sweep_tma_kernel<2, 2, LIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kMagTmaSmem);
  }
  return e;
}

template <int LIM>
cudaError_t launch_mag_t(int axis, const MagArgs& a, cudaStream_t s) {
  const int A = (axis == 0) ? 1 : 0, O = (axis == 2) ? 1 : 2;
  dim3 block(32, kMagWarps + 2);
  dim3 grid((a.box.n[A] + 31) / 32, (a.box.n[O] + kMagWarps - 1) / kMagWarps, a.box.n[axis] / a.seg);
  if (a.ens.items) grid = dim3(a.nblocks, 1, 1);  // one block per work item
  const bool small = a.box.n[axis] < 16;
  if (axis == 0 && mag_rows_qualify(a)) {  // x sweeps over whole staged rows
    if (a.tma_used) *a.tma_used = 1;
    return launch_mag_rows<LIM>(a, s);
  }
#define MAG_CASE(DD, SMEM)                                                       \
  if (axis == DD) {                                                              \
    if (small) mag_sweep_kernel<DD, true, LIM><<<grid, block, SMEM, s>>>(a);     \
    else mag_sweep_kernel<DD, false, LIM><<<grid, block, SMEM, s>>>(a);          \
  }
  MAG_CASE(0, kMagXSmem)
#undef MAG_CASE
  if (a.passes == 2 && axis == 0) return cudaErrorInvalidValue;  // the staged x kernel runs one pass
  {
    MagMaps mp;
    if (a.tma && !a.ens.items && !small && axis != 0 && make_mag_maps(axis, a, &mp)) {
      if (a.tma_used) *a.tma_used = 1;
      if (axis == 1) mag_sweep_tma_kernel<1, 1, LIM><<<grid, block, kMagTmaSmem, s>>>(a, mp);
      else if (a.passes == 2) mag_sweep_tma_kernel<2, 2, LIM><<<grid, block, kMagTmaSmem, s>>>(a, mp);
      else mag_sweep_tma_kernel<2, 1, LIM><<<grid, block, kMagTmaSmem, s>>>(a, mp);
      return cudaGetLastError();
    }
  }
  if (axis == 1) {
    if (small) mag_sweep_pipe_kernel<1, true, LIM, 1><<<grid, block, 0, s>>>(a);
    else mag_sweep_pipe_kernel<1, false, LIM, 1><<<grid, block, 0, s>>>(a);
  }
  if (axis == 2) {
    if (a.passes == 2) {
      if (small) mag_sweep_pipe_kernel<2, true, LIM, 2><<<grid, block, 0, s>>>(a);
      else mag_sweep_pipe_kernel<2, false, LIM, 2><<<grid, block, 0, s>>>(a);
    } else {
      if (small) mag_sweep_pipe_kernel<2, true, LIM, 1><<<grid, block, 0, s>>>(a);
      else mag_sweep_pipe_kernel<2, false, LIM, 1><<<grid, block, 0, s>>>(a);
    }
  }
  return cudaGetLastError();
}

}  // namespace mhd
