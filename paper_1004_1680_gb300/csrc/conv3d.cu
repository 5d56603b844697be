// Periodic 3x3x3 convolution as an implicit GEMM on the 5th-generation tensor
// cores (tcgen05), for the learned coarse-grid correction network.
//
// GEMM view: D[cell, n] = sum_k A[cell, k] B[n, k], k = tap * C + c over the
// 27 taps of the stencil and the C input channels.  A is never materialised:
// for each chunk of 32 k-values a block of 128 threads gathers the shifted
// input rows of its 128 cells (channels-last BF16, periodic wrap) into shared
// memory in the canonical K-major layout (8-row x 16-byte core matrices), one
// elected thread issues two tcgen05.mma (M = 128, K = 16) into an FP32
// accumulator in tensor memory, and a tcgen05.commit arrives on an mbarrier
// once the tensor core has read the chunk (two chunk buffers alternate).  B
// (the weights, packed once per call by conv_pack) sits in shared memory for
// the whole block.  The epilogue reads the accumulator with tcgen05.ld, adds
// the bias, applies ReLU or a gradient mask, and stores BF16 and/or FP32.
//
// The same kernel computes the input gradient (dgrad) with the taps flipped
// and the weights packed transposed.
//
// Every mbarrier wait is bounded: on timeout the block records an error in
// *err, waits (bounded) once more, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "mhd_launch.h"

namespace mhd {

namespace {

constexpr int kM = 128;       // cells per block (GEMM rows)
constexpr int kKC = 32;       // k per staged chunk (two MMAs of K = 16)
constexpr int kChunkBytes = kM * kKC * 2;  // 8 KiB
constexpr uint32_t kTmemCols = 32;
constexpr long long kSpinLimit = 1LL << 22;  // about 0.5 s of polling

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major canonical layout without swizzle:
// core matrices of 8 rows x 16 bytes; `lbo` = byte distance between core
// matrices adjacent along K, `sbo` = between 8-row groups along M/N.
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

__global__ void __launch_bounds__(128, 1) conv3d_tc_kernel(ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int C = a.cin;           // input channels per cell (8 or 32)
  const int Kp = a.kchunks * kKC;
  const int bBytes = a.npad * Kp * 2;
  uint8_t* sB = smem;
  uint8_t* sA = smem + ((bBytes + 1023) & ~1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + 2 * kChunkBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);

  // weights: a straight copy of the packed image
  for (int i = tid; i < bBytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sB)[i] = __ldg(reinterpret_cast<const uint4*>(a.wpack) + i);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // this thread's row: cell of the tile
  const int nx = a.n[0], ny = a.n[1], nz = a.n[2];
  const int cell = blockIdx.x * kM + tid;
  const int x = cell % nx, y = (cell / nx) % ny, z = cell / (nx * ny);
  const int sgn = a.flip ? -1 : 1;
  const uint32_t idesc = make_idesc(kM, a.npad);
  const uint32_t sbo_a = (kKC / 8) * 128, sbo_b = (Kp / 8) * 128;
  bool ok = true;

  for (int c = 0; c < a.kchunks; c++) {
    const int buf = c & 1;
    if (c >= 2 && ok) ok = mbar_wait(smem_addr(&bars[buf]), ((c - 2) >> 1) & 1);
    uint8_t* A = sA + buf * kChunkBytes;
    // gather: 4 core matrices (8 k-values each) of this row
    for (int j = 0; j < kKC / 8; j++) {
      const int k = c * kKC + j * 8;
      const int tap = k / C, ch = k % C;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (tap < 27) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const int sx = (x + sgn * dx + nx) % nx, sy = (y + sgn * dy + ny) % ny, sz = (z + sgn * dz + nz) % nz;
        const int src = sx + nx * (sy + ny * sz);
        v = load16(a.x + (size_t)src * C + ch);
      }
      *reinterpret_cast<uint4*>(A + (tid >> 3) * sbo_a + j * 128 + (tid & 7) * 16) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int s = 0; s < 2; s++) {
        const uint64_t adesc = make_desc(smem_addr(A) + s * 256, 128, sbo_a);
        const uint64_t bdesc = make_desc(smem_addr(sB) + (c * (kKC / 8) + s * 2) * 128, 128, sbo_b);
        const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_addr(&bars[buf]))
                   : "memory");
    }
  }
  const int last = a.kchunks - 1;
  if (ok) ok = mbar_wait(smem_addr(&bars[last & 1]), (last >> 1) & 1);
  if (!ok) {
    if (tid == 0) atomicExch(a.err, 1);
    // give in-flight tensor-core work a bounded chance to finish before freeing
    mbar_wait(smem_addr(&bars[last & 1]), (last >> 1) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __syncthreads_and(ok);  // the epilogue's tcgen05.ld is warp-collective

  if (ok) {
    // epilogue: row `tid` of the accumulator = TMEM lane tid, columns = channels
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    float acc[32];
    uint32_t r[16];
    for (int half = 0; half < a.npad / 16; half++) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + half * 16));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; i++) acc[half * 16 + i] = __uint_as_float(r[i]);
    }
    const int co_n = a.cout;
    for (int co = 0; co < co_n; co++) {
      float v = acc[co] + (a.bias ? __ldg(a.bias + co) : 0.f);
      if (a.relu) v = fmaxf(v, 0.f);
      if (a.mask) v = (__bfloat162float(a.mask[(size_t)cell * co_n + co]) > 0.f) ? v : 0.f;
      if (a.y) a.y[(size_t)cell * co_n + co] = __float2bfloat16_rn(v);
      if (a.y32) a.y32[(size_t)cell * co_n + co] = v;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  (void)lane;
}

// Pack conv weights w[cout][cin][27] (FP32, PyTorch order, tap = (kz*3+ky)*3+kx)
// into the canonical K-major BF16 image of B.  Forward (transpose = 0):
// row n = output channel, k = tap * cin + ci.  Input gradient (transpose = 1):
// row n = input channel, k = tap * cout + co (taps applied flipped).
__global__ void conv_pack_kernel(const float* __restrict__ w, int cin, int cout, int transpose, int npad,
                                 int kchunks, uint16_t* __restrict__ img) {
  const int Kp = kchunks * kKC;
  const int total = npad * Kp;
  const int rows = transpose ? cin : cout, cols = transpose ? cout : cin;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int n = e / Kp, k = e % Kp;
    float v = 0.f;
    const int tap = k / cols, c = k % cols;
    if (n < rows && tap < 27) {
      const int co = transpose ? c : n, ci = transpose ? n : c;
      v = w[((size_t)co * cin + ci) * 27 + tap];
    }
    const size_t off = (size_t)(n / 8) * (Kp / 8) * 64 + (size_t)(k / 8) * 64 + (n % 8) * 8 + (k % 8);
    img[off] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
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

cudaError_t launch_conv_wgrad(const __nv_bfloat16* x, const __nv_bfloat16* gy, const int n[3], int cin, int cout,
                              float* gw, float* gb, cudaStream_t s) {
  const long long cells = (long long)n[0] * n[1] * n[2];
  int nchunk = 64;
  while (nchunk > 1 && (cells % ((long long)nchunk * kWgTile))) nchunk >>= 1;
  const int chunk = (int)(cells / nchunk);
  dim3 grid(27, nchunk);
  conv_wgrad_kernel<<<grid, 256, 0, s>>>(x, gy, n[0], n[1], n[2], cin, cout, chunk, gw, gb);
  return cudaGetLastError();
}

int conv_npad(int n) { return n <= 16 ? 16 : 32; }
int conv_kchunks(int c) { return (27 * c + kKC - 1) / kKC; }
size_t conv_smem_bytes(int npad, int kchunks) {
  const size_t b = (size_t)npad * kchunks * kKC * 2;
  return ((b + 1023) & ~(size_t)1023) + 2 * kChunkBytes + 64;
}

cudaError_t prepare_conv_kernels() {
  return cudaFuncSetAttribute(conv3d_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)conv_smem_bytes(32, conv_kchunks(32)));
}

cudaError_t launch_conv_pack(const float* w, int cin, int cout, int transpose, uint16_t* img, cudaStream_t s) {
  const int rows = transpose ? cin : cout, cols = transpose ? cout : cin;
  const int npad = conv_npad(rows), kc = conv_kchunks(cols);
  const int total = npad * kc * kKC;
  conv_pack_kernel<<<(total + 255) / 256, 256, 0, s>>>(w, cin, cout, transpose, npad, kc, img);
  return cudaGetLastError();
}

cudaError_t launch_conv3d(const ConvArgs& a, cudaStream_t s) {
  const long long cells = (long long)a.n[0] * a.n[1] * a.n[2];
  conv3d_tc_kernel<<<(unsigned)(cells / kM), kM, conv_smem_bytes(a.npad, a.kchunks), s>>>(a);
  return cudaGetLastError();
}

}  // namespace mhd
