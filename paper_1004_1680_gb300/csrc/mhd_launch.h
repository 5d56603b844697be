// Kernel argument blocks and host-side launchers shared by the library's
// translation units (internal; the public interface is include/mhd.h).
#pragma once
#include <cuda.h>  // CUtensorMap (the maps are encoded through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mhd_device.cuh"

namespace mhd {

constexpr int kMagWarps = 8;  // interior rows of a magnetic-sweep tile

// One box of an ensemble: physical extents, first cell in the concatenated
// field arrays (a multiple of 32), and pencil segment length per axis.
struct EnsBox {
  int n[3];
  int offset;
  int seg[3];
  int pad;
};

// Ensemble launches (items != nullptr): block b of the grid works on
// items[b] = (box, block x, block y, block z) of that box; the box geometry
// comes from boxes[box] (exchanged x and y when layout == 1), its sweep step
// from tau_arr[box] and its CFL accumulator is rate_arr[box].
struct EnsArgs {
  const int4* items = nullptr;
  const EnsBox* boxes = nullptr;
  const float* tau_arr = nullptr;
  unsigned* rate_arr = nullptr;
  int layout = 0;
  int phys_axis = 0;
};

struct FluidArgs {
  const float* in[8];  // current fields
  float* out[8];       // destinations of fields 0..4 (others unused)
  Box box;
  float gamma;
  float p_floor = 0.f; // optional floor on the gas pressure of the output (0: off)
  const float* tau;    // device scalar: step of this sweep
  unsigned* rate;      // fused CFL rate accumulator (float bits), or nullptr
  int seg;             // pencil segment length along the sweep axis
  EnsArgs ens;         // ensemble launches only
  int nblocks = 0;     // ensemble launches: number of work items
  int lim = 0;         // slope limiter: 0 van Leer (the paper's), 1 minmod, 2 superbee
  int fast = 0;        // freezing speed: 0 the bound, 1 the fast magnetosonic speed, 2 per pencil
  const float* pencil_c = nullptr;  // fast == 2: per-pencil speeds, stage 1 then stage 2 (nA * nO each)
  // cells [rate_lo, rate_hi) per kernel axis enter the fused rate (the
  // interior of a box with ghost layers; every cell by default)
  int rate_lo[3] = {0, 0, 0};
  int rate_hi[3] = {1 << 30, 1 << 30, 1 << 30};
  int tma = 0;              // 1: stage chunks with tensor-tile copies where the sweep qualifies
  unsigned* err = nullptr;  // set to 1 (atomicOr) if a staged chunk did not arrive within the bound
  int* tma_used = nullptr;  // host: set to 1 when the launch was TMA-staged
};

// Tensor maps of a TMA-staged fluid sweep (kernel axes 1 and 2), dimensions
// ordered (lane axis A, row axis O, sweep axis D).  full[]: one chunk of 4
// positions, for rho, m_d, m_t1, m_t2, e, b_A, b_O (32 x 4 x 4), b_d
// (32 x 4 x 5), b_A of the next block's first 4 lanes (4 x 4 x 4; only its
// row form is used) and b_O of its first row (32 x 1 x 4); row[]: the same
// boxes one position long.
// A 3-D tensor map of FP32 elements: tensor extents dim (the first
// contiguous), byte strides st of dimensions 1 and 2, box b0 x b1 x b2;
// out-of-range elements read as zero.  False if the driver's encoder is
// unavailable or rejects the map (tma_maps.cu).
bool tma_encode_f32(CUtensorMap* m, const float* p, const cuuint64_t dim[3], const cuuint64_t st[2], cuuint32_t b0,
                    cuuint32_t b1, cuuint32_t b2);

constexpr int kFluidMaps = 10;
struct FluidMaps {
  CUtensorMap full[kFluidMaps];
  CUtensorMap row[kFluidMaps];
};
// Encode the maps of a sweep along kernel axis 1 or 2; false if the box does
// not qualify (rows not a multiple of 16 bytes, unaligned fields, pencils
// shorter than 16 cells) or the driver's encoder is unavailable.  Lane and
// row extents need not fill the 32 x 4 tiles.
bool make_fluid_maps(int axis, const FluidArgs& a, FluidMaps* m);

struct MagArgs {
  const float* in[8];
  float* out[3];       // destinations of b_x, b_y, b_z
  Box box;
  const float* tau;
  int seg;
  EnsArgs ens;
  int nblocks = 0;
  int lim = 0;         // slope limiter (as FluidArgs::lim)
  int passes = 1;      // 2: two sweeps with the same step in one launch (kernel axis 2 only)
  int tma = 0;              // 1: stage chunks with tensor-tile copies where the sweep qualifies
  unsigned* err = nullptr;  // set to 1 (atomicOr) if a staged chunk did not arrive within the bound
  int* tma_used = nullptr;  // host: set to 1 when the launch was TMA-staged
};

// Ghost layers of a non-periodic axis (boundary.cu): kernel axis `axis` of
// the fields as stored in `box`; the normal momentum and face field of that
// axis are f[1 + axis] and f[5 + axis].
constexpr int kGhost = 4;
struct GhostArgs {
  float* f[8];
  int axis;
  int mode;                  // 1 outflow, 2 reflecting
  int nk, n1, n2;            // extents: the axis, then the other two (n1 the faster)
  long long sk, s1, s2;      // their strides
};
cudaError_t launch_ghost_fill(float* const f[8], const Box& box, int axis, int mode, cudaStream_t s);

struct TransposeArgs {
  const float* in[8];
  float* out[8];
  int n[3];  // input extents, fastest first; the output has n[1] fastest
  EnsArgs ens;   // ensemble: items = (box, tile i, tile j, k); layout = input layout
  int nblocks = 0;
};

// A box of nx x ny x nz cells, x fastest, on the periodic unit cube.
inline Box make_box(int nx, int ny, int nz) {
  Box b;
  b.n[0] = nx;
  b.n[1] = ny;
  b.n[2] = nz;
  b.stride[0] = 1;
  b.stride[1] = nx;
  b.stride[2] = (long long)nx * ny;
  b.ih[0] = (float)nx;
  b.ih[1] = (float)ny;
  b.ih[2] = (float)nz;
  return b;
}

// Resolved geometry of the block a kernel is running: the box as the kernel
// sees it, the block's coordinates, segment, step and CFL accumulator, and
// the offset of the box in the field arrays.
struct BlockGeom {
  Box box;
  int bx, by, bz;
  int seg;
  int off;
  float tau;
  unsigned* rate;
};

__device__ __forceinline__ BlockGeom block_geom(const EnsArgs& e, const Box& box, int seg,
                                                const float* tau, unsigned* rate) {
  BlockGeom g;
  if (e.items) {
    const int4 it = e.items[blockIdx.x];
    const EnsBox eb = e.boxes[it.x];
    const int n0 = e.layout ? eb.n[1] : eb.n[0];
    const int n1 = e.layout ? eb.n[0] : eb.n[1];
    g.box.n[0] = n0;
    g.box.n[1] = n1;
    g.box.n[2] = eb.n[2];
    g.box.stride[0] = 1;
    g.box.stride[1] = n0;
    g.box.stride[2] = (long long)n0 * n1;
    g.box.ih[0] = (float)n0;  // ensemble boxes are periodic unit boxes
    g.box.ih[1] = (float)n1;
    g.box.ih[2] = (float)eb.n[2];
    g.bx = it.y;
    g.by = it.z;
    g.bz = it.w;
    g.seg = eb.seg[e.phys_axis];
    g.off = eb.offset;
    g.tau = tau ? e.tau_arr[it.x] : 0.f;
    g.rate = e.rate_arr ? e.rate_arr + it.x : nullptr;
  } else {
    g.box = box;
    g.bx = blockIdx.x;
    g.by = blockIdx.y;
    g.bz = blockIdx.z;
    g.seg = seg;
    g.off = 0;
    g.tau = tau ? *tau : 0.f;
    g.rate = rate;
  }
  return g;
}

// Record "<where>: <what>" as this thread's last error (mhd_last_error) and
// return code.
int set_error(int code, const char* where, const char* what);

// 3x3x3 periodic convolution on the tensor cores (conv3d.cu).
struct ConvArgs {
  const __nv_bfloat16* x;     // input, channels-last [cell][cin] BF16
  const uint16_t* wpack;      // packed weight image (launch_conv_pack)
  const float* bias;          // [cout] or nullptr
  __nv_bfloat16* y;           // output [cell][cout] BF16, or nullptr
  float* y32;                 // output [cell][cout] FP32, or nullptr
  const __nv_bfloat16* mask;  // zero outputs where mask[cell][co] <= 0 (ReLU backward), or nullptr
  int n[3];
  int cin;                    // input channels per cell (8 or 32)
  int cout;                   // channels written per cell
  int npad, kchunks;          // MMA N and number of 32-wide k chunks
  int relu;
  int flip;                   // 1: input gradient (the mirrored taps come with the transposed pack)
  int* err;                   // set to 1 if a bounded wait gives up
};
int conv_npad(int n);
int conv_kchunks(int c);
size_t conv_image_bytes(int rows, int cols);
size_t conv_smem_bytes(int npad, int kchunks, int cin, int ty);
cudaError_t prepare_conv_kernels();
cudaError_t launch_conv_pack(const float* w, int cin, int cout, int transpose, uint16_t* img, cudaStream_t s);
cudaError_t launch_conv3d(const ConvArgs& a, cudaStream_t s);
cudaError_t launch_conv_wgrad(const __nv_bfloat16* x, const __nv_bfloat16* gy, const int n[3], int cin, int cout,
                              float* gw, float* gb, int* err, cudaStream_t s);
cudaError_t launch_conv_wgrad_cuda_cores(const __nv_bfloat16* x, const __nv_bfloat16* gy, const int n[3], int cin,
                                         int cout, float* gw, float* gb, cudaStream_t s);

// FP64 path (sweep_f64.cu): whole-pencil kernels on the plain layout
struct Fluid64Args {
  const double* in[8];
  double* out[8];  // fields 0..4 written
  int n[3];
  double ih[3];    // cells per unit length
  double gamma;
  double tau;
};
struct Mag64Args {
  const double* in[8];
  double* out[8];  // fields 5..7 written
  double* E[2];    // edge fluxes of the transverse axes (D+1)%3, (D+2)%3 (N each)
  int n[3];
  double ih[3];
  double tau;
};
cudaError_t launch_fluid64(int axis, const Fluid64Args& a, cudaStream_t s);
cudaError_t launch_mag64(int axis, const Mag64Args& a, cudaStream_t s);
cudaError_t launch_cfl64(const double* const f[8], const int n[3], const double ih[3], double gamma,
                         unsigned long long* rate, cudaStream_t s);

// launchers (return cudaGetLastError of the launch)
cudaError_t launch_transpose01(const TransposeArgs& a, cudaStream_t s);
cudaError_t launch_transpose02(const TransposeArgs& a, cudaStream_t s);  // single box only
// ensemble step control: for every box b < nbox, tau[b] = cfl / rate_cur[b]
// (0 for an invalid state), time[b] += 2 tau[b], rate_next[b] = 0
cudaError_t launch_ens_control(const unsigned* rate_cur, unsigned* rate_next, float* tau,
                               double* time, int nbox, double cfl, cudaStream_t s);
cudaError_t launch_fluid(int axis, bool rate, const FluidArgs& a, cudaStream_t s);
cudaError_t launch_mag(int axis, const MagArgs& a, cudaStream_t s);
// one instantiation per scheme variant, each in its own translation unit
template <int LIM, int FRZ>
cudaError_t launch_fluid_t(int axis, bool rate, const FluidArgs& a, cudaStream_t s);
// per-pencil freezing speeds of a fluid sweep along kernel axis `axis`
// (sweep_pencil.cu): c[pencil] = largest bound along the pencil for U, then
// c[nA nO + pencil] for the stage-1 half-step state built with it
cudaError_t launch_pencil_speeds(int axis, const FluidArgs& a, float* c, cudaStream_t s);
template <int LIM>
cudaError_t launch_mag_t(int axis, const MagArgs& a, cudaStream_t s);
template <int LIM>
cudaError_t prepare_mag_t();
extern template cudaError_t launch_fluid_t<0, 0>(int, bool, const FluidArgs&, cudaStream_t);
extern template cudaError_t launch_fluid_t<1, 0>(int, bool, const FluidArgs&, cudaStream_t);
extern template cudaError_t launch_fluid_t<2, 0>(int, bool, const FluidArgs&, cudaStream_t);
extern template cudaError_t launch_fluid_t<0, 1>(int, bool, const FluidArgs&, cudaStream_t);
extern template cudaError_t launch_fluid_t<0, 2>(int, bool, const FluidArgs&, cudaStream_t);
extern template cudaError_t launch_mag_t<0>(int, const MagArgs&, cudaStream_t);
extern template cudaError_t launch_mag_t<1>(int, const MagArgs&, cudaStream_t);
extern template cudaError_t launch_mag_t<2>(int, const MagArgs&, cudaStream_t);
extern template cudaError_t prepare_mag_t<0>();
extern template cudaError_t prepare_mag_t<1>();
extern template cudaError_t prepare_mag_t<2>();
// one-time per-device kernel attributes (call on the current device before launching)
cudaError_t prepare_mag_kernels();
// Tensor maps of a TMA-staged magnetic sweep (kernel axes 1 and 2), dimensions
// ordered (lane axis A, row axis O, sweep axis D): rho, m_D, b_A, b_O, b_D
// over the 32 x 8 tile (32 x 8 x 4), rho, m_D, b_O one row (32 x 1 x 4) and
// rho, m_D, b_A four columns (4 x 8 x 4) of the neighbouring pencils; row[]:
// the same boxes one position long.
constexpr int kMagMaps = 11;
struct MagMaps {
  CUtensorMap full[kMagMaps];
  CUtensorMap row[kMagMaps];
};
// false if the box does not qualify (lane extent not a multiple of 32, row
// extent not a multiple of 8, unaligned fields) or the encoder is unavailable
bool make_mag_maps(int axis, const MagArgs& a, MagMaps* m);
// cells [lo, hi) per kernel axis (the interior of a box with ghost layers)
struct CellRange {
  int lo[3], hi[3];
};
cudaError_t launch_cfl_rate(const float* const f[8], const Box& box, float gamma, unsigned* rate,
                            cudaStream_t s, const CellRange* range = nullptr);
// device-side step control: tau = cfl / rate_cur (or the given tau if cfl<0),
// time += 2 tau, rate_next = 0
cudaError_t launch_step_control(const unsigned* rate_cur, unsigned* rate_next, float* tau,
                                double* time, double cfl, double tau_host, cudaStream_t s);
// set the device sweep step to a host value (no time advance)
cudaError_t launch_set_tau(float* tau, double value, cudaStream_t s);
// FP64 diagnostics: per-block partials into `partial` (nblk*kDiagSlots
// doubles), then a fixed-order final reduction into out[10] (device).
constexpr int kDiagSlots = 20;  // 8 (sum, compensation) pairs + max|div b| + min p
constexpr int kDiagMaxBlocks = 152 * 8;  // cap of the diagnostics grid (diag_blocks)
int diag_blocks(const Box& box);
cudaError_t launch_diagnostics(const float* const f[8], const Box& box, double gamma, double* partial,
                               double* out, cudaStream_t s);

}  // namespace mhd
