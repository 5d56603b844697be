// Ghost layers of non-periodic axes (an extension: the paper's runs are
// periodic).  A non-periodic axis of n cells keeps kGhost = 4 ghost cells at
// each end inside the box: interior cells kGhost .. n-kGhost-1, wall faces
// kGhost (low) and n-kGhost (the low face of the first high ghost cell).
// The library refills them before every sweep and before every CFL rate; the
// sweeps are the periodic ones (a cell reads at most 3 cells along the sweep
// and 1 pencil across, all inside the ghost layers).
//   outflow (mode 1):    a ghost cell copies the nearest interior cell; ghost
//                        faces of the normal field copy the wall face;
//   reflecting (mode 2): a ghost cell copies its mirror image in the wall with
//                        the normal momentum negated; ghost faces of the
//                        normal field copy their mirror faces, negated.
// Tangential face fields are cell-like along the axis.  Every value written
// comes from an interior cell or a wall face, so one launch fills both ends
// with no ordering between threads; the axes are filled one after another
// (x, y, z), which defines the edge and corner ghosts.
#include "mhd_launch.h"

namespace mhd {

// I: the index type of the element and plane counters (unsigned 32-bit when
// they fit, which avoids emulated 64-bit division per element).
template <typename I>
__global__ void __launch_bounds__(256) ghost_fill_kernel(GhostArgs a) {
  const int k = a.axis;
  const I n1 = (I)a.n1;
  const I plane = (I)a.n1 * (I)a.n2;
  const I total = (I)(2 * kGhost) * plane;
  const int nk = a.nk, wlo = kGhost, whi = nk - kGhost;
  float* const mn = k == 0 ? a.f[1] : (k == 1 ? a.f[2] : a.f[3]);  // normal momentum
  float* const bn = k == 0 ? a.f[5] : (k == 1 ? a.f[6] : a.f[7]);  // normal face field
  for (I id = (I)blockIdx.x * blockDim.x + threadIdx.x; id < total; id += (I)gridDim.x * blockDim.x) {
    // along the contiguous axis the 2 x kGhost ghost cells of a row are
    // neighbouring threads (16 contiguous bytes per side); across it,
    // neighbouring threads take neighbouring rows (contiguous along x)
    I p;
    int layer, side;
    if (k == 0) {
      layer = (int)(id % kGhost);
      side = (int)((id / kGhost) & 1);
      p = id / (2 * kGhost);
    } else {
      const I q = id / plane;
      p = id - q * plane;
      layer = (int)(q % kGhost);
      side = (int)(q / kGhost);
    }
    const I p2 = p / n1;
    const long long base = (long long)(p - p2 * n1) * a.s1 + (long long)p2 * a.s2;
    const int dst = side ? nk - 1 - layer : layer;
    const int src = a.mode == 1 ? (side ? whi - 1 : wlo) : (side ? 2 * whi - 1 - dst : 2 * wlo - 1 - dst);
    const long long di = base + dst * a.sk, si = base + src * a.sk;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      float* const fq = a.f[q];
      if (fq == bn) continue;
      const float v = fq[si];
      fq[di] = (a.mode == 2 && fq == mn) ? -v : v;
    }
    // normal face field: low ghost faces 0..kGhost-1, high ghost faces
    // whi+1 .. nk-1 (the wall faces are interior unknowns)
    if (side == 0 || dst > whi) {
      const int fs = a.mode == 1 ? (side ? whi : wlo) : (side ? 2 * whi - dst : 2 * wlo - dst);
      const float v = bn[base + fs * a.sk];
      bn[di] = a.mode == 2 ? -v : v;
    }
  }
}

cudaError_t launch_ghost_fill(float* const f[8], const Box& box, int axis, int mode, cudaStream_t s) {
  GhostArgs a;
  for (int q = 0; q < 8; q++) a.f[q] = f[q];
  const int t1 = axis == 0 ? 1 : 0, t2 = axis == 2 ? 1 : 2;
  a.axis = axis;
  a.mode = mode;
  a.nk = box.n[axis];
  a.n1 = box.n[t1];
  a.n2 = box.n[t2];
  a.sk = box.stride[axis];
  a.s1 = box.stride[t1];
  a.s2 = box.stride[t2];
  const long long total = 2LL * kGhost * a.n1 * a.n2;
  long long blocks = (total + 255) / 256;
  if (blocks > 65535LL * 16) blocks = 65535LL * 16;
  // 32-bit counters while the element count and the last id + stride fit
  if (total + blocks * 256 < (1LL << 32))
    ghost_fill_kernel<unsigned><<<(unsigned)blocks, 256, 0, s>>>(a);
  else
    ghost_fill_kernel<unsigned long long><<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace mhd
