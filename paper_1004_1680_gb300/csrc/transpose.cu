// Exchange of the two fastest axes of all 8 state fields.
//
// The x sweeps march along x with one thread per pencil; with x the
// contiguous axis a warp's 32 pencils touch 32 different 128-byte lines per
// position, which HBM serves at a fraction of its bandwidth.  Transposing x
// and y once per group of x sweeps turns them into sweeps along a strided
// axis, where a warp's 32 pencils read one 128-byte row per position.  (The
// paper reorients the grid between every pair of sweeps; here it happens only
// around the x sweeps, which are adjacent across consecutive timesteps.)
//
// in[q] has the fast axis of length n0, then n1, then n2; out[q] gets the
// same values with n1 fastest: out[q][j + n1*(i + n0*k)] = in[q][i + n0*(j + n1*k)].
// A block moves one 32x32 tile of every field through shared memory, so both
// the loads and the stores are coalesced 128-byte rows.
#include "mhd_device.cuh"
#include "mhd_launch.h"

namespace mhd {

constexpr int kTile = 32;
constexpr int kTRows = 8;  // threads along the tile's row index

__global__ void __launch_bounds__(kTile * kTRows)
transpose01_kernel(TransposeArgs a) {
  __shared__ float tile[8][kTile][kTile + 1];
  Box in_box;
  in_box.n[0] = a.n[0];
  in_box.n[1] = a.n[1];
  in_box.n[2] = a.n[2];
  const BlockGeom G = block_geom(a.ens, in_box, 1, nullptr, nullptr);
  const int n0 = G.box.n[0], n1 = G.box.n[1];
  const int i0 = G.bx * kTile, j0 = G.by * kTile, k = G.bz;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long plane = (long long)n0 * n1 * k + G.off;
#pragma unroll
  for (int q = 0; q < 8; q++) {
#pragma unroll
    for (int r = 0; r < kTile / kTRows; r++) {
      const int i = i0 + tx, j = j0 + ty + kTRows * r;
      if (i < n0 && j < n1) tile[q][ty + kTRows * r][tx] = __ldg(a.in[q] + plane + i + (long long)n0 * j);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; q++) {
#pragma unroll
    for (int r = 0; r < kTile / kTRows; r++) {
      const int j = j0 + tx, i = i0 + ty + kTRows * r;
      if (i < n0 && j < n1) a.out[q][plane + j + (long long)n1 * i] = tile[q][tx][ty + kTRows * r];
    }
  }
}

// Exchange of the fastest and the slowest axis (x and z) of all 8 fields of
// one box, for the ablation that sweeps every axis along the contiguous one
// (the paper's data flow): out[q][k + n2*(j + n1*i)] = in[q][i + n0*(j + n1*k)].
// A block moves one 32x32 tile of the (i, k) plane at fixed j.
__global__ void __launch_bounds__(kTile * kTRows)
transpose02_kernel(TransposeArgs a) {
  __shared__ float tile[8][kTile][kTile + 1];
  const int n0 = a.n[0], n1 = a.n[1], n2 = a.n[2];
  const int i0 = blockIdx.x * kTile, k0 = blockIdx.y * kTile, j = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long in_row = (long long)n0 * j, in_plane = (long long)n0 * n1;
  const long long out_row = (long long)n2 * j, out_plane = (long long)n2 * n1;
#pragma unroll
  for (int q = 0; q < 8; q++) {
#pragma unroll
    for (int r = 0; r < kTile / kTRows; r++) {
      const int i = i0 + tx, k = k0 + ty + kTRows * r;
      if (i < n0 && k < n2) tile[q][ty + kTRows * r][tx] = __ldg(a.in[q] + i + in_row + in_plane * k);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; q++) {
#pragma unroll
    for (int r = 0; r < kTile / kTRows; r++) {
      const int k = k0 + tx, i = i0 + ty + kTRows * r;
      if (i < n0 && k < n2) a.out[q][k + out_row + out_plane * i] = tile[q][tx][ty + kTRows * r];
    }
  }
}

cudaError_t launch_transpose02(const TransposeArgs& a, cudaStream_t s) {
  dim3 block(kTile, kTRows);
  dim3 grid((a.n[0] + kTile - 1) / kTile, (a.n[2] + kTile - 1) / kTile, a.n[1]);
  transpose02_kernel<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_transpose01(const TransposeArgs& a, cudaStream_t s) {
  dim3 block(kTile, kTRows);
  dim3 grid((a.n[0] + kTile - 1) / kTile, (a.n[1] + kTile - 1) / kTile, a.n[2]);
  if (a.ens.items) grid = dim3(a.nblocks, 1, 1);  // one block per (box, tile, plane)
  transpose01_kernel<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mhd
