// Periodic 3x3x3 convolution as an implicit GEMM on the 5th-generation tensor
// cores (tcgen05), for the learned coarse-grid correction network.
//
// GEMM view: D[cell, o] = sum_k A[cell, k] W[o, k], k = (tap, channel) over
// the 27 taps and the cin input channels (channels-last BF16 activations).
// A is never materialised.  A block owns a run of tiles of 8 x TY x 1 cells
// (TY = 32: two 128-row accumulators; 16: one), consecutive along z.  A tile
// needs the halo planes z-1, z, z+1, each (8+2) x (TY+2) cells stored as one
// plane per 8-channel group (16 bytes per cell) in a ring of shared-memory
// slots; consecutive tiles share two of them, so a tile copies one new plane
// (cp.async).  In that layout the canonical K-major core matrix of 8 GEMM
// rows x 8 channels is 8 consecutive halo cells along x, so the operand of
// tap t is its plane's slot addressed from a shifted start: every tap is one
// descriptor offset, with no per-tap gather.  The weights (packed once by
// conv_pack) stay in shared memory for the block's lifetime.  Warps
// specialise: one thread per accumulator issues its 27 x (cin / 16)
// tcgen05.mma (M = 128, N = 32 or 16, K = 16; BF16 in, FP32 in TMEM) into
// one of two TMEM buffers, two warps copy planes, four warps run the
// epilogue of the previous tile (tcgen05.ld, bias, ReLU or the ReLU mask of
// the saved activation, BF16 and/or FP32 16-byte stores); mbarriers pass
// slots and buffers between them.
//
// The input gradient is the same kernel with mirrored taps and the weights
// packed transposed.  The weight gradient (a reduction over the cells) is a
// second tcgen05 kernel with both operands MN-major, described above it.
//
// Every mbarrier wait is bounded: on timeout the block records an error in
// *err, and every role leaves its loop; the MMA threads wait (bounded) for
// their last commit before the tensor memory is freed.
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "mhd_launch.h"

namespace mhd {

namespace {

constexpr int kM = 128;       // GEMM rows per MMA (tile cells per accumulator)
constexpr int kKC = 32;       // k per 32-wide chunk of the packed weight image
constexpr int kTX = 8, kHX = kTX + 2;     // tile: 8 x TY x 1 cells (TY = 16 or 32), halo rows of kHX cells

constexpr long long kSpinLimit = 1LL << 22;  // about 0.5 s of polling

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, canonical layout without swizzle: core
// matrices of 8 x 16 bytes (K-major: 8 rows of M/N, 16 bytes of K; MN-major:
// 8 rows of K, 16 bytes of M/N); `lbo` = byte distance between core matrices
// adjacent along K, `sbo` = between core matrices adjacent along M/N.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;              // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, shape M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One tcgen05.mma (kind::f16, cta_group::1) that accumulates into D.
__device__ __forceinline__ void mma_acc(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(1u)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; i++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 bytes of 8 channels of one cell: the gathered source of one core-matrix row
__device__ __forceinline__ uint4 load16(const __nv_bfloat16* p) {
  return __ldg(reinterpret_cast<const uint4*>(p));
}

}  // namespace

__device__ __forceinline__ int wrap1(int i, int n) {  // i in [-1, n]
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// Shared-memory ring of halo planes for the forward / input-gradient kernel:
// slot = one z plane of a tile's halo, kHX x (TY + 2) cells per channel group
// (plus 4 zero cells read, times zero weights, by the cin = 8 MMAs), one plane
// per 8-channel group.
template <int G, int TY>
struct ConvRing {
  static constexpr int HY = TY + 2;
  static constexpr int PLANE = (kHX * HY + 4) * 16;   // one channel group of one z plane
  static constexpr int SLOT = G * PLANE;              // one z plane of the halo
  static constexpr int NSLOT = 6;
  static constexpr int NACC = TY / 16;                // 128-row accumulators per tile
};

// The block's contiguous run of tiles, z fastest: tile t is column t / nz
// (an 8 x TY patch of the x-y plane) at z = t % nz.  Consecutive tiles of a
// column share two of their three halo planes, so the ring receives one new
// plane per tile, three at the start of a column.
struct TileRun {
  int t0, count, nz, tiles_x;
  __device__ int col(int i) const { return (t0 + i) / nz; }
  __device__ int z(int i) const { return (t0 + i) % nz; }
  __device__ bool fresh(int i) const { return i == 0 || col(i) != col(i - 1); }
};

// Halo plane z (wrapped) of column c into ring slot `slot` by the copying
// threads lt = 0..nl-1; one cp.async group per thread.
template <int G, int TY>
__device__ __forceinline__ void load_plane(uint8_t* slot, const __nv_bfloat16* __restrict__ x, int c, int z,
                                           const TileRun& run, int nx, int ny, int lt, int nl) {
  using R = ConvRing<G, TY>;
  constexpr int P = kHX * G;  // 16-byte pieces per halo row
  const int x0 = (c % run.tiles_x) * kTX, y0 = (c / run.tiles_x) * TY;
  const uint32_t base = smem_addr(slot);
  for (int p = lt; p < R::HY * P; p += nl) {
    const int hy = p / P, l = p - hy * P, hx = l / G, g = l - hx * G;
    const int cell = wrap1(x0 - 1 + hx, nx) + nx * (wrap1(y0 - 1 + hy, ny) + ny * z);
    cp_async16(base + g * R::PLANE + (hy * kHX + hx) * 16, x + (size_t)cell * (8 * G) + g * 8);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// G = cin / 8 channel groups, tiles of 8 x TY x 1 cells (TY / 16 accumulators
// of 128 rows).  Persistent, 256 threads, warp-specialised, z taps packed
// along N:
//  * The block's run of tiles (z fastest) splits into column segments: L
//    consecutive tiles of one 8 x TY column at z = z0 .. z0 + L - 1.  A
//    segment reads its input planes P = z0 - 1 .. z0 + L once each, in
//    order.  Input plane P, shifted in-plane by one of the 9 (ky, kx)
//    offsets, is the A operand of one MMA per 16 input channels whose B
//    holds the weights of the three z taps side by side (N = 3 npad rows:
//    column block j3 = the tap kz = j3 for the forward pass), so one MMA adds
//    the contributions of plane P to the output planes P + 1, P, P - 1.
//  * The accumulators of the output planes live in a ring of kRing slots of
//    npad TMEM columns per 128-row accumulator, in descending order of the
//    output plane, so the three column blocks an input plane writes are
//    adjacent; where they cross the end of the ring the MMA splits in two.
//    The first K step that reaches an output plane (input plane = output
//    plane + 1 - j3 with j3 = 0) writes its block with accumulate off.
//  * Output plane z is complete once input plane z + 1 has been added.
// Roles: warps 0 .. NACC-1, lane 0: the MMAs of accumulator q; warps 2, 3:
// copy input planes into the ring (cp.async); warps 4..7: epilogue of the
// completed output planes (tcgen05.ld, bias, ReLU or the ReLU mask, BF16 /
// FP32 stores).  mbarriers: input slot full (copying threads) / empty (a
// tcgen05.commit after the plane's MMAs); output slot full (a commit after
// the output plane's last MMA) / free (the epilogue warps).  The weights
// (packed once by conv_pack) are copied into shared memory once per block.
// Compared with one N = npad MMA per (tap, 16 channels) and tile, this reads
// each input plane's A operand once for three output planes: about a third
// of the shared-memory operand traffic per MAC.
constexpr int kRing = 8;  // output-plane slots per accumulator

template <int G, int TY>
__global__ void __launch_bounds__(256, 1) conv3d_tc_kernel(ConvArgs a) {
  using R = ConvRing<G, TY>;
  constexpr int NS = R::NSLOT, NACC = R::NACC;
  constexpr int NL = 64;  // copying threads
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npad = a.npad;
  const int Kp = a.kchunks * kKC;
  const int bBytes = 3 * npad * Kp * 2;
  uint8_t* sB = smem;
  uint8_t* ring = smem + ((bBytes + 1023) & ~1023);
  float* sBias = reinterpret_cast<float*>(ring + NS * R::SLOT);
  uint64_t* full = reinterpret_cast<uint64_t*>(sBias + 32);
  uint64_t* empty = full + NS;
  uint64_t* ofull = empty + NS;
  uint64_t* ofree = ofull + kRing;
  uint64_t* wfull = ofree + kRing;  // the weight image has landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wfull + 1);
  const uint32_t tmem_cols = (uint32_t)(NACC * kRing * npad);  // 128 .. 512, a power of two

  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int tiles_x = nx / kTX, tiles_y = ny / TY;
  const int ntiles = tiles_x * tiles_y * nz;
  // The block's run of tiles.  With at least one block per column the runs
  // stay inside one column (a run that crosses into the next column copies
  // two more halo planes, and the slowest block sets the launch's time):
  // column c gets blocks b with b C / B = c and splits its nz tiles evenly.
  // Otherwise blocks take equal contiguous ranges of whole-column order.
  const int ncol = tiles_x * tiles_y, nblk = gridDim.x;
  TileRun run;
  if (ncol <= nblk) {
    const int c = (int)((long long)blockIdx.x * ncol / nblk);
    const int b0 = (int)(((long long)c * nblk + ncol - 1) / ncol);
    const int b1 = (int)(((long long)(c + 1) * nblk + ncol - 1) / ncol);
    const int kc = b1 - b0, r = blockIdx.x - b0;  // kc <= nz: the grid has at most ncol * nz blocks
    const int lo = r * nz / kc, hi = (r + 1) * nz / kc;
    run.t0 = c * nz + lo;
    run.count = hi - lo;
  } else {
    run.t0 = (int)((long long)blockIdx.x * ntiles / nblk);
    run.count = (int)((long long)(blockIdx.x + 1) * ntiles / nblk) - run.t0;
  }
  run.nz = nz;
  run.tiles_x = tiles_x;

  // the weights first: bBytes (a multiple of 16) from a 16-byte aligned
  // image, in flight while the block sets up (the barrier's initialisation
  // is ordered before any wait on it by the block barrier below)
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(wfull)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(wfull)), "r"(bBytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(sB)),
                 "l"(a.wpack), "r"(bBytes), "r"(smem_addr(wfull))
                 : "memory");
  }

  // zero pad cells; the packed weight image (once per block) comes in one
  // bulk asynchronous copy that the MMA threads wait for, while the copying
  // warps start on the input planes
  for (int i = tid; i < NS * G * 4; i += 256)
    *reinterpret_cast<uint4*>(ring + (i / 4) * R::PLANE + (kHX * R::HY + i % 4) * 16) = make_uint4(0u, 0u, 0u, 0u);
  if (tid < 32) sBias[tid] = (a.bias && tid < a.cout) ? __ldg(a.bias + tid) : 0.f;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < NS; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(full + i)), "r"(NL) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(empty + i)), "r"(NACC) : "memory");
    }
    for (int i = 0; i < kRing; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(ofull + i)), "r"(NACC) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_addr(ofree + i)) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // pads, for the tensor core
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  if (warp < NACC) {
    // ---- MMA issue: accumulator q -------------------------------------
    if (lane == 0) {
      const int q = warp;
      const uint32_t sbo_b = (Kp / 8) * 128;
      const uint32_t b_addr = smem_addr(sB);
      const uint32_t dq = tmem + (uint32_t)(q * kRing * npad);
      int k = 0;          // input planes consumed
      int last_out = -1;  // last output plane committed
      ok = mbar_wait(smem_addr(wfull), 0);
      for (int i0 = 0; i0 < run.count && ok;) {
        // the column segment of tiles i0 .. i0 + L - 1 (outputs g = i0 + u)
        int L = 1;
        while (i0 + L < run.count && run.col(i0 + L) == run.col(i0)) L++;
        for (int v = 0; v < L + 2 && ok; v++, k++) {
          const int jlo = v > L - 1 ? v - (L - 1) : 0, jhi = v < 2 ? v : 2;
          const int gtop = i0 + v;  // output plane of block j3 = 0 (started by this input plane if v < L)
          ok = mbar_wait(smem_addr(full + k % NS), (k / NS) & 1);
          if (ok && jlo == 0 && gtop >= kRing)  // its slot's previous output has been read out
            ok = mbar_wait(smem_addr(ofree + gtop % kRing), (gtop / kRing - 1) & 1);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // GEMM row m of accumulator q = tile cell (m % 8, 16 q + m / 8): the
          // rows of a core matrix are 8 consecutive halo cells along x (16
          // bytes apart), 8-row groups one halo row apart (SBO = kHX * 16);
          // the (ky, kx) offset is a shift of the start address.
          const uint64_t a0 = make_desc(smem_addr(ring + (k % NS) * R::SLOT), G == 4 ? R::PLANE : 16, kHX * 16) +
                              (uint64_t)(q * 16 * kHX);
          // The plane's output blocks j0 = jlo .. jhi (output planes gtop - j0
          // in ring slots kRing - 1 - (gtop - j0) % kRing, adjacent except
          // across the end of the ring) as at most three MMA segments, found
          // once per plane: `f` for the plane's first K step, where a block
          // that starts its output plane (j0 = 0) goes alone with accumulate
          // off, `r` for the other K steps.  Per segment: TMEM column (d), N
          // of the instruction descriptor (i), B descriptor offset in 16-byte
          // units (b).
          auto slot_of = [&](int g) { return kRing - 1 - (g % kRing); };
          auto seg_d = [&](int j0) { return dq + (uint32_t)(slot_of(gtop - j0) * npad); };
          auto seg_b = [&](int j0) { return (uint64_t)(((uint32_t)(j0 * npad / 8) * sbo_b) >> 4); };
          const int nall = jhi - jlo + 1;
          // r: [jlo, jlo + rl0) and [jlo + rl0, jhi] (the second if the ring wraps)
          const int rl0 = nall < kRing - slot_of(gtop - jlo) ? nall : kRing - slot_of(gtop - jlo);
          const int nr = rl0 < nall ? 2 : 1;
          const uint32_t rd0 = seg_d(jlo), rd1 = seg_d(jlo + rl0);
          const uint32_t ri0 = make_idesc(kM, rl0 * npad), ri1 = make_idesc(kM, (nall - rl0) * npad);
          const uint64_t rb0 = seg_b(jlo), rb1 = seg_b(jlo + rl0);
          // f: as r, unless jlo = 0: block 0 alone (accumulate off), then
          // [1, 1 + fl1) and [1 + fl1, jhi]
          const bool fresh = jlo == 0;
          const int rest = jhi;  // blocks 1 .. jhi after block 0
          const int fl1 = rest < kRing - slot_of(gtop - 1) ? rest : kRing - slot_of(gtop - 1);
          const int nf = fresh ? 1 + (rest > 0 ? 1 : 0) + (fl1 < rest ? 1 : 0) : nr;
          const uint32_t fd0 = fresh ? seg_d(0) : rd0, fd1 = fresh ? seg_d(1) : rd1, fd2 = seg_d(1 + fl1);
          const uint32_t fi0 = fresh ? make_idesc(kM, npad) : ri0, fi1 = fresh ? make_idesc(kM, fl1 * npad) : ri1;
          const uint32_t fi2 = make_idesc(kM, (rest - fl1) * npad);
          const uint64_t fb0 = fresh ? seg_b(0) : rb0, fb1 = fresh ? seg_b(1) : rb1, fb2 = seg_b(1 + fl1);
          const uint32_t fa0 = fresh ? 0u : 1u;
#pragma unroll
          for (int j = 0; j < 9; j++) {
            const int off = (j / 3) * kHX + j % 3;
#pragma unroll
            for (int h = 0; h < (G == 4 ? 2 : 1); h++) {
              // G = 4: k = 16 channels 16h..16h+15 (planes 2h, 2h+1); G = 1:
              // the 8 channels of offset j, then 8 whose weights are the zero
              // k-group 9
              const uint32_t b_k = (G == 4) ? (uint32_t)((j * 4 + 2 * h) * 128) : (uint32_t)(j * 128);
              const uint32_t lbo_b = (G == 4) ? 128u : (uint32_t)((9 - j) * 128);
              const uint64_t adesc = a0 + (uint64_t)(off + (G == 4 ? h * (2 * R::PLANE / 16) : 0));
              const uint64_t bd = make_desc(b_addr + b_k, lbo_b, sbo_b);
              if (j == 0 && h == 0) {
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(fd0),
                    "l"(adesc), "l"(bd + fb0), "r"(fi0), "r"(fa0)
                    : "memory");
                if (nf > 1)
                  mma_acc(fd1, adesc, bd + fb1, fi1);
                if (nf > 2)
                  mma_acc(fd2, adesc, bd + fb2, fi2);
              } else {
                mma_acc(rd0, adesc, bd + rb0, ri0);
                if (nr > 1)
                  mma_acc(rd1, adesc, bd + rb1, ri1);
              }
            }
          }
          // the input plane is no longer read; output plane gtop - 2 is complete
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_addr(empty + k % NS))
                       : "memory");
          if (jhi == 2) {
            last_out = gtop - 2;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(ofull + last_out % kRing))
                         : "memory");
          }
        }
        i0 += L;
      }
      // nothing of this thread in flight when TMEM is freed
      if (last_out >= 0) {
        const bool done = mbar_wait(smem_addr(ofull + last_out % kRing), (last_out / kRing) & 1);
        ok = ok && done;
      }
    }
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  } else if (warp == 2 || warp == 3) {
    // ---- copies: input plane k goes to slot k % NS ---------------------------
    const int lt = tid - 64;
    int k = 0;
    for (int i0 = 0; i0 < run.count && ok;) {
      int L = 1;
      while (i0 + L < run.count && run.col(i0 + L) == run.col(i0)) L++;
      const int c = run.col(i0), z0 = run.z(i0);
      for (int v = 0; v < L + 2 && ok; v++, k++) {
        if (k >= NS) ok = mbar_wait(smem_addr(empty + k % NS), (k / NS - 1) & 1);
        if (!ok) break;
        load_plane<G, TY>(ring + (k % NS) * R::SLOT, a.x, c, wrap1(z0 - 1 + v, nz), run, nx, ny, lt, NL);
        if (k >= 1) {  // the previous plane's pieces have landed
          asm volatile("cp.async.wait_group 1;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(full + (k - 1) % NS)) : "memory");
        }
      }
      i0 += L;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (ok && k > 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(full + (k - 1) % NS)) : "memory");
    }
  } else if (warp >= 4) {
    // ---- epilogue: TMEM lanes 32 (warp - 4) + lane = GEMM row -------------
    const int ew = warp - 4, row = 32 * ew + lane;
    const int co_n = a.cout;
    for (int g = 0; g < run.count; g++) {
      ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(ofull + g % kRing), (g / kRing) & 1));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int c = run.col(g), z0 = run.z(g);
      const int x0 = (c % tiles_x) * kTX, y0 = (c / tiles_x) * TY;
      const int slot = kRing - 1 - (g % kRing);
#pragma unroll
      for (int q = 0; q < NACC; q++) {
        const int cell = (x0 + (row & 7)) + nx * ((y0 + 16 * q + (row >> 3)) + ny * z0);
        const uint32_t taddr = tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)((q * kRing + slot) * npad);
        float acc[32];
        uint32_t r[16];
#pragma unroll
        for (int half = 0; half < 2; half++) {
          if (half >= npad / 16) break;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(taddr + half * 16));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; j++) acc[half * 16 + j] = __uint_as_float(r[j]);
        }
        // 8 channels (16 bytes of BF16) at a time; cout is 8 or 32
#pragma unroll
        for (int c8 = 0; c8 < 4; c8++) {
          if (c8 >= co_n / 8) break;
          float v[8];
#pragma unroll
          for (int j = 0; j < 8; j++) {
            v[j] = acc[c8 * 8 + j] + sBias[c8 * 8 + j];
            if (a.relu) v[j] = fmaxf(v[j], 0.f);
          }
          if (a.mask) {
            const uint4 mk = load16(a.mask + (size_t)cell * co_n + c8 * 8);
            const uint32_t mw[4] = {mk.x, mk.y, mk.z, mk.w};
#pragma unroll
            for (int j = 0; j < 8; j++) {
              const float m = __bfloat162float(__ushort_as_bfloat16((unsigned short)(mw[j / 2] >> (16 * (j & 1)))));
              v[j] = m > 0.f ? v[j] : 0.f;
            }
          }
          if (a.y)
            *reinterpret_cast<uint4*>(a.y + (size_t)cell * co_n + c8 * 8) =
                make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                           pack_bf16x2(v[6], v[7]));
          if (a.y32) {
            float4* o = reinterpret_cast<float4*>(a.y32 + (size_t)cell * co_n + c8 * 8);
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
          }
        }
      }
      // the slot's TMEM has been read: the output plane kRing later may start in it
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(ofree + g % kRing)) : "memory");
    }
  }
  if (!ok) atomicExch(a.err, 1);
  // the weight copy has landed before the shared memory is released (at once
  // unless a wait above gave up)
  if (tid == 0) mbar_wait(smem_addr(wfull), 0);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// Pack conv weights w[cout][cin][27] (FP32, PyTorch order, tap = (kz*3+ky)*3+kx)
// into the canonical K-major BF16 image of B with the z taps along N:
// row n = j3 * npad + r (column block j3 = 0, 1, 2), k = j * cols + c with j =
// ky * 3 + kx the in-plane offset of the input plane.  Forward (transpose =
// 0): r = output channel, c = input channel, tap (kz, ky, kx) = (j3, j / 3,
// j % 3).  Input gradient (transpose = 1): r = input channel, c = output
// channel, and the taps mirrored, (2 - j3, 2 - j / 3, 2 - j % 3): the kernel
// then runs unchanged.  K is padded to kchunks * 32 with zeros (for 8
// channels the zero k-group 9 pairs with each offset's 8).
__global__ void conv_pack_kernel(const float* __restrict__ w, int cin, int cout, int transpose, int npad,
                                 int kchunks, uint16_t* __restrict__ img) {
  const int Kp = kchunks * kKC;
  const int total = 3 * npad * Kp;
  const int rows = transpose ? cin : cout, cols = transpose ? cout : cin;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int n = e / Kp, k = e % Kp;
    const int j3 = n / npad, r = n % npad;
    const int j = k / cols, c = k % cols;
    float v = 0.f;
    if (r < rows && j < 9) {
      int kz = j3, ky = j / 3, kx = j % 3;
      if (transpose) {
        kz = 2 - kz;
        ky = 2 - ky;
        kx = 2 - kx;
      }
      const int co = transpose ? c : r, ci = transpose ? r : c;
      v = w[((size_t)co * cin + ci) * 27 + (kz * 3 + ky) * 3 + kx];
    }
    const size_t off = (size_t)(n / 8) * (Kp / 8) * 64 + (size_t)(k / 8) * 64 + (n % 8) * 8 + (k % 8);
    img[off] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
}

// Weight gradient on the tensor cores.  gw[o][c][tap] += sum over cells of
// gy[cell][o] x[cell + d(tap)][c] is a GEMM whose reduction runs over the
// cells, computed tile by tile (8 x TY x 1 cells, K = 16 cells per MMA):
// D[row, col] += A[row, cell] B[col, cell], FP32 in TMEM, M = 128.  Both
// operands are MN-major: a cell's 8 channels are the 16 contiguous bytes of
// a core-matrix row, 8 cells along x make a core matrix.
//
// One MMA covers 9 (or 3) taps:
//  * A rows are three copies of the tile's output gradient taken from the
//    planes z0 + 1, z0, z0 - 1 (copy kz = 0, 1, 2; 4 planes of 8 output
//    channels per copy for 32 output channels, one for 8);
//  * B is the tile's x halo in its own z plane, stored row by row as
//    [halo row][channel plane][10 cells], so core matrices adjacent along N
//    are 160 bytes apart both from plane to plane and from the last plane of
//    a row to the first of the next: N = 96 columns = 3 halo rows (ky) x 32
//    input channels (for 8 input channels, 3 rows of 8 plus 8 ignored
//    columns: N = 32);
//  * the start of B, shifted by kx cells, selects the x tap: 3 accumulators.
// Row (kz, o) x column (ky, c) of accumulator kx then sums
// gy[cell'] x[cell' + (kx-1, ky-1, kz-1)] over the tile moved by (0, 0, 1-kz);
// the moved tiles still cover the grid once, so it is one tap of the full
// sum.  Rows and columns beyond the real channels read unused shared memory
// and are never stored.
//
// One block per SM loops over tiles through three operand stages: lane 0 of
// warp 0 issues the MMAs while the copying warps fetch the next tiles'
// operands and a last warp sums copy kz = 1 (the tile's own output gradient)
// for the bias gradient (mbarriers mark a stage full, and empty again once
// tcgen05.commit and the bias warp have both arrived).  At the end warps
// 0..2 read the accumulators (TMEM lane = A row) into shared memory, and the
// block adds its partial gw with coalesced reductions.
struct WgradArgs {
  const __nv_bfloat16* x;
  const __nv_bfloat16* gy;
  int n[3];
  int cin, cout;
  float* gw;
  float* gb;  // may be null
  int* err;
};

template <int TY>
struct WgradTile {
  static constexpr int NT = 8 * TY;                      // cells of a tile
  static constexpr int NTHR = NT + 32;                   // threads: MMA warp, copying warps, bias warp
  static constexpr int NL = NT - 32;                     // copying threads (warps 1 .. NT / 32 - 1)
  static constexpr int APL = NT * 16;                    // one A plane: 8 channels of every tile cell
  static constexpr int A_BYTES = 12 * APL;               // 3 copies x 4 planes; rows 96..127 read B
  static constexpr int HY = TY + 2;                      // halo rows (one z plane)
  static constexpr int SEG = kHX * 16;                   // one halo row of one channel plane
  static constexpr int B_BYTES = (HY + 1) * 4 * SEG;     // 32 input channels, one spare row
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int NSTAGE = 3;
  static constexpr int BASE = 1024;                      // barriers and TMEM address first
  // barriers plus operands of three stages (afterwards: the block's partial
  // gw, 32 x 32 x 27 floats and a pad word per output channel); at least
  // 116 KB so that one block holds an SM (it allocates all 512 TMEM columns)
  static constexpr size_t need = BASE + NSTAGE * (size_t)STAGE;
  static constexpr size_t smem = need > 116 * 1024 ? need : 116 * 1024;
  static_assert(16 * APL <= STAGE, "A rows 96..127 stay inside the stage");
};

template <int TY>
constexpr size_t wgrad_smem_bytes() {
  return WgradTile<TY>::smem;
}

// Copies of one tile's operands into a stage by the copying threads (lt =
// 0..NL-1), one cp.async group per thread.  WIDE: 32 output channels, else 8;
// G4: 32 input channels, else 8.
template <int TY, bool WIDE, bool G4>
__device__ __forceinline__ void wgrad_load(uint8_t* stage, const WgradArgs& a, int x0, int y0, int z0, int lt) {
  using W = WgradTile<TY>;
  constexpr int G = G4 ? 4 : 1, NT = W::NT, NL = W::NL;
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const uint32_t sa = smem_addr(stage), sb = sa + W::A_BYTES;
  // A: copy kz (the plane z0 + 1 - kz), tile cell m, plane g; consecutive
  // threads take consecutive 16-byte pieces of a cell's channels
  constexpr int PA = WIDE ? 3 * 4 * NT : 3 * NT;
#pragma unroll
  for (int i = 0; i < (PA + NL - 1) / NL; i++) {
    const int p = lt + NL * i;
    if (p < PA) {
      if (WIDE) {
        const int kz = p / (4 * NT), r = p % (4 * NT), g = r & 3, m = r >> 2;
        const int cell = (x0 + (m & 7)) + nx * (y0 + (m >> 3) + ny * wrap1(z0 + 1 - kz, nz));
        cp_async16(sa + (4 * kz + g) * W::APL + m * 16, a.gy + (size_t)cell * 32 + g * 8);
      } else {
        const int kz = p / NT, m = p % NT;
        const int cell = (x0 + (m & 7)) + nx * (y0 + (m >> 3) + ny * wrap1(z0 + 1 - kz, nz));
        cp_async16(sa + kz * W::APL + m * 16, a.gy + (size_t)cell * 8);
      }
    }
  }
  // B: halo cell (hx, hy) of plane g = x at (x0 - 1 + hx, y0 - 1 + hy, z0)
  constexpr int P = kHX * G, PB = W::HY * P;
#pragma unroll
  for (int i = 0; i < (PB + NL - 1) / NL; i++) {
    const int p = lt + NL * i;
    if (p < PB) {
      const int hy = p / P, l = p - hy * P, hx = l / G, g = l - hx * G;
      const int cell = wrap1(x0 - 1 + hx, nx) + nx * (wrap1(y0 - 1 + hy, ny) + ny * z0);
      cp_async16(sb + (hy * G + g) * W::SEG + hx * 16, a.x + (size_t)cell * (8 * G) + g * 8);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int TY, bool WIDE, bool G4>
__global__ void __launch_bounds__(8 * TY + 32, 1) conv_wgrad_tc_kernel(WgradArgs a) {
  using W = WgradTile<TY>;
  constexpr uint32_t kCols = 512;
  constexpr int G = G4 ? 4 : 1;
  constexpr int NCOL = G4 ? 96 : 32;  // columns per accumulator
  constexpr int RB = G * W::SEG;      // one halo row of every plane
  constexpr int NS = W::NSTAGE;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // full[s]: the copying threads' pieces of stage s have landed; empty[s]:
  // the MMAs that read stage s are done (tcgen05.commit) and the bias warp
  // has summed it
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + NS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(empty + NS);
  uint8_t* stages = smem + W::BASE;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int st = 0; st < NS; st++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(full + st)), "r"(W::NL) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(smem_addr(empty + st)) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nx = a.n[0], ny = a.n[1];
  const int tiles_x = nx / kTX, tiles_y = ny / TY;
  const int ntiles = tiles_x * tiles_y * a.n[2];
  const int K = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  bool ok = true;
  if (warp == 0) {
    // lane 0 issues every MMA: per tile and x tap kx, TY / 2 K steps
    // (tile rows 2 ks, 2 ks + 1).  A: the next 8 cells 128 B on (lbo), the
    // next 8 rows one plane on (sbo).  B: the next 8 cells one halo row on
    // (lbo), the next 8 columns 160 B on (sbo).  Address fields count 16-byte
    // units, so shifts add to the descriptor.
    if (lane == 0) {
      // M = 128, N = NCOL, BF16 in, FP32 accumulate, both operands MN-major
      constexpr uint32_t idesc = make_idesc(kM, NCOL) | (1u << 15) | (1u << 16);
      int issued = 0;
      for (int k = 0; k < K; k++) {
        const int st = k % NS;
        ok = mbar_wait(smem_addr(full + st), (k / NS) & 1);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_addr = smem_addr(stages + st * W::STAGE);
        const uint64_t ad = make_desc(a_addr, 128, W::APL);
        const uint64_t bd = make_desc(a_addr + W::A_BYTES, RB, W::SEG);
#pragma unroll
        for (int kx = 0; kx < 3; kx++) {
#pragma unroll
          for (int ks = 0; ks < TY / 2; ks++) {
            const uint32_t acc = (k > 0 || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + kx * NCOL),
                "l"(ad + (uint64_t)(16 * ks)), "l"(bd + (uint64_t)(kx + 2 * ks * (RB / 16))), "r"(idesc),
                "r"(acc)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(empty + st))
                     : "memory");
        issued = k + 1;
      }
      // the last issued tile's MMAs, also when a wait gave up, so that
      // nothing is in flight when TMEM is freed
      if (issued > 0) {
        const bool done = mbar_wait(smem_addr(empty + (issued - 1) % NS), ((issued - 1) / NS) & 1);
        ok = ok && done;
      }
    }
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  } else if (warp == W::NT / 32) {
    // bias warp: gb[o] sums the output gradient over the cells, i.e. copy
    // kz = 1 (the tile's own plane) of every tile; lane l keeps channel group
    // l / 8 (one group for 8 output channels), so that the 8 lanes of a
    // quarter warp read 128 contiguous bytes of one plane
    constexpr int GO = WIDE ? 4 : 1;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < K; k++) {
      const int st = k % NS;
      ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(full + st), (k / NS) & 1));  // the warp stays converged
      if (!ok) break;
      if (a.gb) {
        const uint8_t* own = stages + st * W::STAGE + GO * W::APL;
        const int g = WIDE ? lane >> 3 : 0, m0 = WIDE ? lane & 7 : lane;
#pragma unroll 4
        for (int m = m0; m < W::NT; m += 32 / GO) {
          const uint4 v = *reinterpret_cast<const uint4*>(own + g * W::APL + m * 16);
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int q = 0; q < 4; q++) {
            acc[2 * q] += __uint_as_float(w[q] << 16);
            acc[2 * q + 1] += __uint_as_float(w[q] & 0xFFFF0000u);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(empty + st));
    }
    if (a.gb && ok && K > 0) {
#pragma unroll
      for (int q = 0; q < 8; q++) {
        for (int d = 1; d < 32 / GO; d *= 2) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], d);
        if ((lane & (32 / GO - 1)) == 0) atomicAdd(a.gb + 8 * (lane / (32 / GO)) + q, acc[q]);
      }
    }
  } else {
    const int lt = tid - 32;
    for (int k = 0; k < K; k++) {
      const int st = k % NS;
      // stage st was last read by the MMAs of tile k - NS
      if (k >= NS) ok = mbar_wait(smem_addr(empty + st), (k / NS - 1) & 1);
      if (!ok) break;
      const int tile = blockIdx.x + k * gridDim.x;
      wgrad_load<TY, WIDE, G4>(stages + st * W::STAGE, a, (tile % tiles_x) * kTX, ((tile / tiles_x) % tiles_y) * TY,
                               tile / (tiles_x * tiles_y), lt);
      if (k >= 1) {  // the previous tile's pieces
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(smem_addr(full + (k - 1) % NS));
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (ok && K > 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_addr(full + (K - 1) % NS));
    }
  }
  if (!ok) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // The block's partial gw goes through shared memory (the stages are free
  // now) so that the additions to gw are contiguous: gw index
  // i = (o cin + c) 27 + tap sits at word i + o (the pad word per output
  // channel spreads the stores of a warp's lanes over the banks).
  constexpr int CIN = G4 ? 32 : 8, ROW = CIN * 27, TOTAL = (WIDE ? 32 : 8) * ROW;
  float* part = reinterpret_cast<float*>(stages);
  // warps 0..2 hold TMEM lanes 0..95: A row L = 8 q + r of plane q
  if (warp < (WIDE ? 3 : 1) && ok && K > 0) {
    const int L = 32 * warp + lane, q = L >> 3, r = L & 7;
    const int kz = WIDE ? q >> 2 : q, o = WIDE ? 8 * (q & 3) + r : r;
    const bool live = WIDE ? q < 12 : q < 3;
#pragma unroll 1
    for (int kx = 0; kx < 3; kx++) {
#pragma unroll 1
      for (int ch = 0; ch < NCOL / 32; ch++) {  // 32 columns at a time
        uint32_t v[32];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
              "[%16];"
              : "=r"(v[16 * h + 0]), "=r"(v[16 * h + 1]), "=r"(v[16 * h + 2]), "=r"(v[16 * h + 3]),
                "=r"(v[16 * h + 4]), "=r"(v[16 * h + 5]), "=r"(v[16 * h + 6]), "=r"(v[16 * h + 7]),
                "=r"(v[16 * h + 8]), "=r"(v[16 * h + 9]), "=r"(v[16 * h + 10]), "=r"(v[16 * h + 11]),
                "=r"(v[16 * h + 12]), "=r"(v[16 * h + 13]), "=r"(v[16 * h + 14]), "=r"(v[16 * h + 15])
              : "r"(tmem + ((uint32_t)(32 * warp) << 16) + kx * NCOL + ch * 32 + h * 16));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (live) {
          float* dst = part + o * (ROW + 1) + 9 * kz + kx;
          if (G4) {  // columns: ky = ch, c = 0..31
#pragma unroll
            for (int c = 0; c < 32; c++) dst[c * 27 + 3 * ch] = __uint_as_float(v[c]);
          } else {   // columns 8 ky + c, ky < 3
#pragma unroll
            for (int k = 0; k < 24; k++) dst[(k & 7) * 27 + 3 * (k >> 3)] = __uint_as_float(v[k]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (ok && K > 0) {
    // ROW is a multiple of 4, so 4 consecutive indices share o
    const bool vec = ((uintptr_t)a.gw & 15) == 0;
    for (int i = 4 * tid; i < TOTAL; i += 4 * W::NTHR) {
      const float* src = part + i + i / ROW;
      float* dst = a.gw + i;
      if (vec)
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(src[0]), "f"(src[1]),
                     "f"(src[2]), "f"(src[3])
                     : "memory");
      else
        for (int k = 0; k < 4; k++) atomicAdd(dst + k, src[k]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// Weight gradient on the CUDA cores: gw[co][ci][tap] += sum over a chunk of
// cells of gy[cell][co] * x[cell + offset(tap)][ci] (FP32 accumulation,
// atomically added across chunks), and gb[co] += sum gy[cell][co].
constexpr int kWgTile = 64;
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const __nv_bfloat16* __restrict__ x,
                                                         const __nv_bfloat16* __restrict__ gy, int nx, int ny,
                                                         int nz, int cin, int cout, int chunk,
                                                         float* __restrict__ gw, float* __restrict__ gb) {
  __shared__ float sx[kWgTile][33];
  __shared__ float sg[kWgTile][33];
  const int tap = blockIdx.x, tid = threadIdx.x;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int npairs = cin * cout, per = (npairs + 255) / 256;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float bacc = 0.f;
  const int c0 = blockIdx.y * chunk;
  for (int t0 = c0; t0 < c0 + chunk; t0 += kWgTile) {
    __syncthreads();
    for (int e = tid; e < kWgTile * cin; e += 256) {
      const int r = e / cin, ci = e % cin, cell = t0 + r;
      const int x0 = cell % nx, y0 = (cell / nx) % ny, z0 = cell / (nx * ny);
      const int src = (x0 + dx + nx) % nx + nx * ((y0 + dy + ny) % ny + ny * ((z0 + dz + nz) % nz));
      sx[r][ci] = __bfloat162float(x[(size_t)src * cin + ci]);
    }
    for (int e = tid; e < kWgTile * cout; e += 256) {
      const int r = e / cout, co = e % cout;
      sg[r][co] = __bfloat162float(gy[(size_t)(t0 + r) * cout + co]);
    }
    __syncthreads();
    for (int i = 0; i < per; i++) {
      const int pr = tid + 256 * i;
      if (pr < npairs) {
        const int co = pr / cin, ci = pr % cin;
        float a = acc[i];
#pragma unroll 8
        for (int r = 0; r < kWgTile; r++) a += sg[r][co] * sx[r][ci];
        acc[i] = a;
      }
    }
    if (tap == 13 && tid < cout)
      for (int r = 0; r < kWgTile; r++) bacc += sg[r][tid];
  }
  for (int i = 0; i < per; i++) {
    const int pr = tid + 256 * i;
    if (pr < npairs) {
      const int co = pr / cin, ci = pr % cin;
      atomicAdd(&gw[((size_t)co * cin + ci) * 27 + tap], acc[i]);
    }
  }
  if (tap == 13 && tid < cout && gb) atomicAdd(&gb[tid], bacc);
}

namespace {
template <int TY>
cudaError_t launch_wgrad_tc(const __nv_bfloat16* x, const __nv_bfloat16* gy, const int n[3], int cin, int cout,
                            float* gw, float* gb, int* err, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)(n[0] / kTX) * (n[1] / TY) * n[2];
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
  WgradArgs a;
  a.x = x;
  a.gy = gy;
  a.n[0] = n[0];
  a.n[1] = n[1];
  a.n[2] = n[2];
  a.cin = cin;
  a.cout = cout;
  a.gw = gw;
  a.gb = gb;
  a.err = err;
  const size_t smem = wgrad_smem_bytes<TY>();
  constexpr int threads = WgradTile<TY>::NTHR;
  if (cout == 32)
    cin == 32 ? conv_wgrad_tc_kernel<TY, true, true><<<grid, threads, smem, s>>>(a)
              : conv_wgrad_tc_kernel<TY, true, false><<<grid, threads, smem, s>>>(a);
  else
    cin == 32 ? conv_wgrad_tc_kernel<TY, false, true><<<grid, threads, smem, s>>>(a)
              : conv_wgrad_tc_kernel<TY, false, false><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

// Weight and bias gradient: on the tensor cores when err is given (the
// caller has checked that the box tiles into 8 x 16 x 1 cells and that x and
// gy are 16-byte aligned), else on the CUDA cores.
cudaError_t launch_conv_wgrad(const __nv_bfloat16* x, const __nv_bfloat16* gy, const int n[3], int cin, int cout,
                              float* gw, float* gb, int* err, cudaStream_t s) {
  if (err)
    return n[1] % 32 == 0 ? launch_wgrad_tc<32>(x, gy, n, cin, cout, gw, gb, err, s)
                          : launch_wgrad_tc<16>(x, gy, n, cin, cout, gw, gb, err, s);
  return launch_conv_wgrad_cuda_cores(x, gy, n, cin, cout, gw, gb, s);
}

cudaError_t launch_conv_wgrad_cuda_cores(const __nv_bfloat16* x, const __nv_bfloat16* gy, const int n[3], int cin,
                                         int cout, float* gw, float* gb, cudaStream_t s) {
  const long long cells = (long long)n[0] * n[1] * n[2];
  int nchunk = 64;
  while (nchunk > 1 && (cells % ((long long)nchunk * kWgTile))) nchunk >>= 1;
  const int chunk = (int)(cells / nchunk);
  dim3 grid(27, nchunk);
  conv_wgrad_kernel<<<grid, 256, 0, s>>>(x, gy, n[0], n[1], n[2], cin, cout, chunk, gw, gb);
  return cudaGetLastError();
}

int conv_npad(int n) { return n <= 16 ? 16 : 32; }
// K of the packed image: the 9 in-plane offsets x the input channels
int conv_kchunks(int c) { return (9 * c + kKC - 1) / kKC; }
// bytes of the packed weight image (3 npad rows: the z taps along N)
size_t conv_image_bytes(int rows, int cols) { return (size_t)3 * conv_npad(rows) * conv_kchunks(cols) * kKC * 2; }
size_t conv_smem_bytes(int npad, int kchunks, int cin, int ty) {
  const size_t b = (size_t)3 * npad * kchunks * kKC * 2;
  const size_t slot = ty == 32 ? (cin == 32 ? ConvRing<4, 32>::SLOT : ConvRing<1, 32>::SLOT)
                               : (cin == 32 ? ConvRing<4, 16>::SLOT : ConvRing<1, 16>::SLOT);
  // weights, ring, bias, the input and output slot mbarriers, TMEM address
  return ((b + 1023) & ~(size_t)1023) + ConvRing<4, 32>::NSLOT * slot + 32 * sizeof(float) +
         (2 * ConvRing<4, 32>::NSLOT + 2 * kRing + 1) * 8 + 16;
}

namespace {
template <int TY>
cudaError_t prepare_wgrad() {
  const int smem = (int)wgrad_smem_bytes<TY>();
  cudaError_t e = cudaFuncSetAttribute(conv_wgrad_tc_kernel<TY, true, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_wgrad_tc_kernel<TY, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_wgrad_tc_kernel<TY, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv_wgrad_tc_kernel<TY, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  return e;
}

template <int G, int TY>
cudaError_t prepare_one() {
  cudaError_t e = cudaFuncSetAttribute(conv3d_tc_kernel<G, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)conv_smem_bytes(32, conv_kchunks(8 * G), 8 * G, TY));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(conv3d_tc_kernel<G, TY>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

// Resident blocks per device for each kernel variant and shared-memory size,
// found once: a launch then costs no device queries.
constexpr int kCacheDevices = 64, kCacheSizes = 16;
struct GridCache {
  const void* fn[kCacheSizes];
  size_t smem[kCacheSizes];
  int blocks[kCacheSizes];
  int used;
};
GridCache g_grid[kCacheDevices];
std::mutex g_grid_lock;

template <int G, int TY>
cudaError_t launch_variant(const ConvArgs& a, cudaStream_t s) {
  const void* fn = reinterpret_cast<const void*>(conv3d_tc_kernel<G, TY>);
  const size_t smem = conv_smem_bytes(a.npad, a.kchunks, a.cin, TY);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kCacheDevices) return cudaErrorInvalidDevice;
  int cap = 0;
  {
    std::lock_guard<std::mutex> g(g_grid_lock);
    GridCache& c = g_grid[dev];
    for (int i = 0; i < c.used && !cap; i++)
      if (c.fn[i] == fn && c.smem[i] == smem) cap = c.blocks[i];
    if (!cap) {
      int sms = 0, per_sm = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv3d_tc_kernel<G, TY>, 256, smem);
      if (e != cudaSuccess) return e;
      // resident blocks of an SM share its 512 TMEM columns
      const int tmem_cap = 512 / (ConvRing<G, TY>::NACC * kRing * a.npad);
      per_sm = per_sm < tmem_cap ? per_sm : tmem_cap;
      cap = sms * (per_sm > 0 ? per_sm : 1);
      if (c.used < kCacheSizes) {
        c.fn[c.used] = fn;
        c.smem[c.used] = smem;
        c.blocks[c.used] = cap;
        c.used++;
      }
    }
  }
  const long long tiles = (long long)(a.n[0] / kTX) * (a.n[1] / TY) * a.n[2];
  const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
  conv3d_tc_kernel<G, TY><<<grid, 256, smem, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

cudaError_t prepare_conv_kernels() {
  cudaError_t e = prepare_wgrad<32>();
  if (e == cudaSuccess) e = prepare_wgrad<16>();
  if (e == cudaSuccess) e = prepare_one<4, 32>();
  if (e == cudaSuccess) e = prepare_one<4, 16>();
  if (e == cudaSuccess) e = prepare_one<1, 32>();
  if (e == cudaSuccess) e = prepare_one<1, 16>();
  return e;
}

cudaError_t launch_conv_pack(const float* w, int cin, int cout, int transpose, uint16_t* img, cudaStream_t s) {
  const int rows = transpose ? cin : cout, cols = transpose ? cout : cin;
  const int npad = conv_npad(rows), kc = conv_kchunks(cols);
  const int total = 3 * npad * kc * kKC;
  conv_pack_kernel<<<(total + 255) / 256, 256, 0, s>>>(w, cin, cout, transpose, npad, kc, img);
  return cudaGetLastError();
}

// Tiles of 8 x 32 x 1 cells (two accumulators, 8 warps) when ny allows,
// else 8 x 16 x 1.
cudaError_t launch_conv3d(const ConvArgs& a, cudaStream_t s) {
  const bool wide = a.n[1] % 32 == 0;
  if (a.cin == 32) return wide ? launch_variant<4, 32>(a, s) : launch_variant<4, 16>(a, s);
  return wide ? launch_variant<1, 32>(a, s) : launch_variant<1, 16>(a, s);
}

}  // namespace mhd
