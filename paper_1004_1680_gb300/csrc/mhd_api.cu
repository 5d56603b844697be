// Host side of the C ABI declared in include/mhd.h: the box context, its
// device memory, the timestep schedule of Section II.B and error handling.
//
// Memory layout in HBM: one arena of 16 planar FP32 arrays (two copies of the
// 8 fields; every sweep reads one copy and writes the other, field by field),
// plus a few device scalars (sweep step, two CFL-rate accumulators, the
// simulation time) and the FP64 diagnostics scratch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "mhd.h"
#include "mhd_launch.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, const char* what = "") {
  std::snprintf(g_err, sizeof g_err, fmt, what);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  std::snprintf(g_err, sizeof g_err, "%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? MHD_E_OOM : MHD_E_CUDA;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

struct Scalars {  // small device block
  float tau;
  unsigned rate[2];
  unsigned err;  // 1: a staged chunk of a sweep did not arrive within the wait bound
  double time;
  double diag[10];
};

}  // namespace

namespace mhd {
int set_error(int code, const char* where, const char* what) {
  std::snprintf(g_err, sizeof g_err, "%s: %s", where, what);
  return code;
}
}  // namespace mhd

struct mhd_s {
  int n[3];
  double gamma;
  long long N;
  mhd::Box box;
  mhd::Box tbox;       // the same box with x and y exchanged
  mhd::Box zbox;       // the same box with x and z exchanged (x path 3)
  float* arena = nullptr;
  float* cur[8];        // current copy of each field (in the current layout)
  float* spare[8];      // the other copy, written by the next kernel
  int layout = 0;       // 0: x fastest; 1: x and y exchanged (for x sweeps); 2: x and z exchanged
  int xpath = 0;        // x sweeps: 1 direct, 2 through the exchanged layout; 3: every
                        // axis swept along the contiguous one (the paper's data flow)
  int xpath_req = 0;    // requested by mhd_set_xpath (0 = automatic)
  float p_floor = 0.f;  // optional pressure floor after fluid sweeps (0 = off)
  int lim = 0;          // slope limiter (0 = van Leer, the paper's scheme)
  int fast = 0;         // freezing speed (0 = the bound, the paper's scheme)
  int fuse = 1;         // 1: the two z magnetic sweeps of a step run as one launch
  int tma = 1;          // 1: sweeps stage their data with bulk tensor copies where they qualify (y, z: chunks; x: rows)
  long long tma_sweeps = 0;  // sweeps launched TMA-staged
  int bc[3] = {0, 0, 0};  // per physical axis: 0 periodic, 1 outflow, 2 reflecting (ghost layers)
  double cpl[3] = {0.0, 0.0, 0.0};  // cells per unit length per physical axis (0: n, the unit box)
  int own_lo[3] = {0, 0, 0};        // own cells [own_lo, own_hi) per physical axis (the others are
  int own_hi[3] = {1 << 30, 1 << 30, 1 << 30};  // halo copies of another box's cells)
  float* pencil_c = nullptr;  // freezing 2: per-pencil speeds of the sweep being run (2 x N / min n)
  Scalars* sc = nullptr;
  double* diag_partial = nullptr;
  int rcur = 0;
  // FP64 boxes (mhd_create_f64): the state in double, whole-pencil kernels
  bool f64 = false;
  double* arena64 = nullptr;
  double* cur64[8];
  double* spare64[8];
  double* e64 = nullptr;                 // edge fluxes of a magnetic sweep (2 N)
  unsigned long long* rate64 = nullptr;  // CFL rate (double bits)
  double time64 = 0.0;
  cudaStream_t stream = nullptr;
  int seg[3];
  int sms = 0;          // multiprocessors of the device (segment choice)
  // tracing: event pairs around launches (see mhd_profile)
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  // pipelined host runs (mhd_submit / mhd_drain): three staging sets of the 8
  // fields, an input and an output copy stream, and per slot the events
  // "input landed" and "its arrays are no longer read by an output copy"
  float* stage_arena = nullptr;
  float* slot[3][8];
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[3] = {}, ev_free[3] = {}, ev_done = nullptr, ev_out = nullptr;
  bool slot_used[3] = {false, false, false};
  int next_slot = 0;
  bool pipe_pending = false;  // an output copy may still be in flight
};

namespace {

// x sweeps run directly along x when both row sweeps take the box (whole
// x rows staged in shared memory: nx a multiple of 128 up to 1024, ny a
// multiple of the magnetic tile's rows (4, or 2 for rows longer than 512),
// tensor-copy staging on, a freezing speed of its own per cell); otherwise
// they go through the exchanged layout once the state no longer fits in L2
// (the pencil sweeps along x read 32 different lines per warp and position,
// which only L2 can absorb).
int auto_xpath(const mhd_s* m) {
  const bool rows = m->tma && m->fast != 2 && m->n[0] % 128 == 0 && m->n[0] <= 1024 &&
                    m->n[1] % (m->n[0] <= 512 ? 4 : 2) == 0 && m->n[2] >= 2;
  if (rows) return 1;
  return m->N * 32LL > (64LL << 20) ? 2 : 1;
}

// Cells per unit length of each layout's axes (the exchanged layouts permute
// the physical axes).
void set_geometry(mhd_s* m) {
  float ih[3];
  for (int d = 0; d < 3; d++) ih[d] = (float)(m->cpl[d] > 0.0 ? m->cpl[d] : (double)m->n[d]);
  for (int d = 0; d < 3; d++) m->box.ih[d] = ih[d];
  m->tbox.ih[0] = ih[1];
  m->tbox.ih[1] = ih[0];
  m->tbox.ih[2] = ih[2];
  m->zbox.ih[0] = ih[2];
  m->zbox.ih[1] = ih[1];
  m->zbox.ih[2] = ih[0];
}

// Kernel axis of physical axis p in the current layout.
int kernel_axis_of(const mhd_s* m, int p) {
  if (m->layout == 1 && p < 2) return 1 - p;
  if (m->layout == 2 && p != 1) return 2 - p;
  return p;
}

// Cells along physical axis p whose CFL rate counts: the own cells, less
// the ghost layers of a non-periodic axis.
void rate_window(const mhd_s* m, int p, int* lo, int* hi) {
  *lo = std::max(m->bc[p] ? mhd::kGhost : 0, m->own_lo[p]);
  *hi = std::min(m->bc[p] ? m->n[p] - mhd::kGhost : m->n[p], m->own_hi[p]);
}

// Segment length along each axis.  Splitting pencils into segments adds 7
// cells of warm-up per segment but gives the GPU more threads.  First split
// until the pencil segments give about one full wave of threads (152 x 1024:
// enough warps to hide latency); then, since a sweep runs ceil(n_A/32) x
// ceil(n_O/W) blocks per segment of every pencil (W = 4 rows for the fluid
// sweep, 8 for the magnetic one), take among that and further splits (at
// least 32 cells, multiples of 8) the one that minimises (warm-up work) /
// sqrt(last-wave efficiency) summed over the two sweeps, with the resident
// blocks per SM of each kernel (fluid 4, magnetic 2).
int choose_seg(const mhd_s* m, int d) {
  const int nd = m->n[d];
  const long long pencils = m->N / nd;
  const long long want = 152LL * 1024;
  int first = nd;
  while (pencils * (nd / first) < want && first % 8 == 0 && first / 2 >= 32 && nd % (first / 2) == 0)
    first /= 2;
  const int nA = m->n[d == 0 ? 1 : 0], nO = m->n[d == 2 ? 1 : 2];
  const double sms = m->sms > 0 ? m->sms : 152;
  auto cost = [&](int seg) {
    double c = 0.0;
    const int rows[2] = {4, mhd::kMagWarps}, resident[2] = {4, 2};
    for (int k = 0; k < 2; k++) {
      const double blocks = (double)((nA + 31) / 32) * ((nO + rows[k] - 1) / rows[k]) * (nd / seg);
      const double waves = blocks / (sms * resident[k]);
      // a partial last wave costs less than its idle fraction (the SMs that
      // run it go faster alone): its weight enters as a square root, which
      // matches measured sweeps at 256^3, 512^3 and 1024^3
      c += (double)(seg + 7) / seg * std::sqrt(std::ceil(waves) / waves);
    }
    return c;
  };
  int best = first;
  double best_cost = cost(first);
  for (int seg = first; seg % 8 == 0 && seg / 2 >= 32 && nd % (seg / 2) == 0;) {
    seg /= 2;
    const double c = cost(seg);
    if (c < best_cost * 0.999) {
      best = seg;
      best_cost = c;
    }
  }
  return best;
}

// Bracket the launches issued by `body` with an event pair when tracing.
template <class F>
int traced(mhd_s* m, int kind, F body) {
  const bool on = m->ev_used < m->ev_kind.size();
  if (on) CK(cudaEventRecord(m->ev[2 * m->ev_used], m->stream));
  int rc = body();
  if (rc) return rc;
  if (on) {
    CK(cudaEventRecord(m->ev[2 * m->ev_used + 1], m->stream));
    m->ev_kind[m->ev_used++] = kind;
  }
  return MHD_OK;
}

void drop_events(mhd_s* m) {
  for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
  m->ev.clear();
  m->ev_kind.clear();
  m->ev_used = 0;
}

void field_ptrs(const mhd_s* m, const float* out[8]) {
  for (int q = 0; q < 8; q++) out[q] = m->cur[q];
}

// Exchange x and y of all fields (out of place).  In the exchanged layout the
// field slots are relabelled so that slot 1 / 5 hold the momentum / face field
// along the new fast axis (physical y) and slots 2 / 6 those along physical x.
int exchange_xy(mhd_s* m) {
  mhd::TransposeArgs a;
  const mhd::Box& b = m->layout == 0 ? m->box : m->tbox;
  for (int q = 0; q < 8; q++) {
    a.in[q] = m->cur[q];
    a.out[q] = m->spare[q];
  }
  a.n[0] = b.n[0];
  a.n[1] = b.n[1];
  a.n[2] = b.n[2];
  int rc = traced(m, MHD_K_TRANSPOSE, [&] {
    CK(mhd::launch_transpose01(a, m->stream));
    return MHD_OK;
  });
  if (rc) return rc;
  static const int relabel[8] = {0, 2, 1, 3, 4, 6, 5, 7};
  float* nc[8];
  float* ns[8];
  for (int q = 0; q < 8; q++) {
    nc[relabel[q]] = m->spare[q];
    ns[relabel[q]] = m->cur[q];
  }
  for (int q = 0; q < 8; q++) {
    m->cur[q] = nc[q];
    m->spare[q] = ns[q];
  }
  m->layout ^= 1;
  return MHD_OK;
}

// Exchange x and z of all fields (out of place), between layouts 0 and 2;
// slots 1 / 5 and 3 / 7 are relabelled as for exchange_xy.
int exchange_xz(mhd_s* m) {
  mhd::TransposeArgs a;
  const mhd::Box& b = m->layout == 0 ? m->box : m->zbox;
  for (int q = 0; q < 8; q++) {
    a.in[q] = m->cur[q];
    a.out[q] = m->spare[q];
  }
  a.n[0] = b.n[0];
  a.n[1] = b.n[1];
  a.n[2] = b.n[2];
  int rc = traced(m, MHD_K_TRANSPOSE, [&] {
    CK(mhd::launch_transpose02(a, m->stream));
    return MHD_OK;
  });
  if (rc) return rc;
  static const int relabel[8] = {0, 3, 2, 1, 4, 7, 6, 5};
  float* nc[8];
  float* ns[8];
  for (int q = 0; q < 8; q++) {
    nc[relabel[q]] = m->spare[q];
    ns[relabel[q]] = m->cur[q];
  }
  for (int q = 0; q < 8; q++) {
    m->cur[q] = nc[q];
    m->spare[q] = ns[q];
  }
  m->layout = m->layout == 0 ? 2 : 0;
  return MHD_OK;
}

int ensure_layout(mhd_s* m, int layout) {
  if (m->layout == layout) return MHD_OK;
  int rc = MHD_OK;
  if (m->layout == 1) rc = exchange_xy(m);
  if (!rc && m->layout == 2) rc = exchange_xz(m);
  if (!rc && layout == 1) rc = exchange_xy(m);
  if (!rc && layout == 2) rc = exchange_xz(m);
  return rc;
}

// Frame of a sweep along physical axis d: the layout it runs in, the box as
// the kernels see it and the kernel axis.  y sweeps need x fastest; x sweeps
// run in the exchanged layout when xpath == 2 (as kernel axis 1); z sweeps
// run in whichever layout is current.  With xpath == 3 every sweep runs along
// the contiguous axis (kernel axis 0) of the layout that makes d the fastest.
int sweep_frame(mhd_s* m, int d, const mhd::Box** box, int* kaxis) {
  int want = m->layout;
  if (m->xpath == 3) {
    want = d;  // layout 0: x fastest, 1: y fastest, 2: z fastest
  } else {
    if (d == 0) want = (m->xpath == 2) ? 1 : 0;
    if (d == 1) want = 0;
    if (d == 2 && want == 2) want = 0;
  }
  int rc = ensure_layout(m, want);
  if (rc) return rc;
  *box = m->layout == 2 ? &m->zbox : (m->layout ? &m->tbox : &m->box);
  if (m->layout == 2)
    *kaxis = (d == 2) ? 0 : (d == 0 ? 2 : 1);
  else
    *kaxis = (m->layout && d < 2) ? 1 - d : d;
  return MHD_OK;
}

bool any_bc(const mhd_s* m) { return m->bc[0] || m->bc[1] || m->bc[2]; }

// Refill the ghost layers of the non-periodic axes in the current layout:
// physical axis a is kernel axis k there, with its normal momentum and face
// field in slots 1 + k and 5 + k (the exchanges relabel the slots).  Axes in
// physical order x, y, z.
int fill_ghosts(mhd_s* m) {
  if (!any_bc(m)) return MHD_OK;
  const mhd::Box& b = m->layout == 2 ? m->zbox : (m->layout ? m->tbox : m->box);
  for (int a = 0; a < 3; a++) {
    if (!m->bc[a]) continue;
    int k = a;
    if (m->layout == 1 && a < 2) k = 1 - a;
    if (m->layout == 2 && a != 1) k = 2 - a;
    if (int rc = traced(m, MHD_K_CONTROL, [&] {
          CK(mhd::launch_ghost_fill(m->cur, b, k, m->bc[a], m->stream));
          return MHD_OK;
        }))
      return rc;
  }
  return MHD_OK;
}

// CFL rate of the current state into *rate (zeroed first).  With ghost
// layers the rate covers the interior cells only (a ghost cell next to the
// periodic wrap pairs faces from both ends of the axis), after a refill.
int state_rate(mhd_s* m, unsigned* rate) {
  if (int rc = fill_ghosts(m)) return rc;
  const mhd::Box& b = m->layout == 2 ? m->zbox : (m->layout ? m->tbox : m->box);
  mhd::CellRange r;
  for (int a = 0; a < 3; a++) rate_window(m, a, &r.lo[kernel_axis_of(m, a)], &r.hi[kernel_axis_of(m, a)]);
  CK(cudaMemsetAsync(rate, 0, sizeof(unsigned), m->stream));
  const float* cf[8];
  field_ptrs(m, cf);
  return traced(m, MHD_K_CONTROL, [&] {
    CK(mhd::launch_cfl_rate(cf, b, (float)m->gamma, rate, m->stream, &r));
    return MHD_OK;
  });
}

int fluid(mhd_s* m, int d, bool rate) {
  const mhd::Box* box;
  int ka;
  int rc = sweep_frame(m, d, &box, &ka);
  if (rc) return rc;
  if ((rc = fill_ghosts(m))) return rc;
  mhd::FluidArgs a;
  for (int q = 0; q < 8; q++) {
    a.in[q] = m->cur[q];
    a.out[q] = m->spare[q];
  }
  a.box = *box;
  a.gamma = (float)m->gamma;
  a.p_floor = m->p_floor;
  a.tau = &m->sc->tau;
  a.rate = rate ? &m->sc->rate[1 - m->rcur] : nullptr;
  a.seg = m->seg[d];
  a.lim = m->lim;
  a.fast = m->fast;
  for (int p = 0; p < 3; p++)  // the fused rate covers the interior, own cells
    rate_window(m, p, &a.rate_lo[kernel_axis_of(m, p)], &a.rate_hi[kernel_axis_of(m, p)]);
  int staged = 0;
  a.tma = m->tma;
  a.err = &m->sc->err;
  a.tma_used = &staged;
  if (m->fast == 2) {  // per-pencil freezing speeds before the sweep
    a.pencil_c = m->pencil_c;
    if ((rc = traced(m, MHD_K_CONTROL, [&] {
           CK(mhd::launch_pencil_speeds(ka, a, m->pencil_c, m->stream));
           return MHD_OK;
         })))
      return rc;
  }
  rc = traced(m, MHD_K_FLUID_X + d, [&] {
    CK(mhd::launch_fluid(ka, rate, a, m->stream));
    return MHD_OK;
  });
  if (rc) return rc;
  m->tma_sweeps += staged;
  for (int q = 0; q < 5; q++) std::swap(m->cur[q], m->spare[q]);
  return MHD_OK;
}

// passes = 2: two magnetic sweeps along d with the same step in one launch
// (bitwise equal to two launches; kernel axis 2 only, the caller checks).
int magnetic(mhd_s* m, int d, int passes = 1) {
  const mhd::Box* box;
  int ka;
  int rc = sweep_frame(m, d, &box, &ka);
  if (rc) return rc;
  if ((rc = fill_ghosts(m))) return rc;
  mhd::MagArgs a;
  for (int q = 0; q < 8; q++) a.in[q] = m->cur[q];
  for (int q = 0; q < 3; q++) a.out[q] = m->spare[5 + q];
  a.box = *box;
  a.tau = &m->sc->tau;
  a.seg = m->seg[d];
  a.lim = m->lim;
  a.passes = passes;
  int staged = 0;
  a.tma = m->tma;
  a.err = &m->sc->err;
  a.tma_used = &staged;
  rc = traced(m, MHD_K_MAG_X + d, [&] {
    CK(mhd::launch_mag(ka, a, m->stream));
    return MHD_OK;
  });
  if (rc) return rc;
  m->tma_sweeps += staged;
  for (int q = 5; q < 8; q++) std::swap(m->cur[q], m->spare[q]);
  return MHD_OK;
}

// The sweep schedule of one full step (Section II.B): x, y, z forward with
// fluid before magnetic, then z, y, x with magnetic before fluid; the last
// fluid sweep also accumulates the CFL rate of the new state (of its interior
// cells with ghost layers: those cells and the faces their rate reads are
// final once the sweep has written them; a refill changes neither).  The two
// z magnetic sweeps in the middle of the schedule follow each other with the
// same step and run as one launch when fusion is on (bitwise the same
// result), unless the z sweep runs along the contiguous axis (x path 3) or
// ghost layers must be refilled between them.
int full_step(mhd_s* m) {
  int rc;
  for (int d = 0; d < 2; d++) {
    if ((rc = fluid(m, d, false))) return rc;
    if ((rc = magnetic(m, d))) return rc;
  }
  if ((rc = fluid(m, 2, false))) return rc;
  if (m->fuse && m->xpath != 3 && !any_bc(m)) {
    if ((rc = magnetic(m, 2, 2))) return rc;
  } else {
    if ((rc = magnetic(m, 2))) return rc;
    if ((rc = magnetic(m, 2))) return rc;
  }
  if ((rc = fluid(m, 2, false))) return rc;
  for (int d = 1; d >= 0; d--) {
    if ((rc = magnetic(m, d))) return rc;
    if ((rc = fluid(m, d, d == 0))) return rc;
  }
  m->rcur ^= 1;
  return MHD_OK;
}

// Later work on the box's stream waits for the output copies of mhd_submit
// (the box's arrays rotate through the staging sets).
int join_pipeline(mhd_s* m) {
  if (!m->pipe_pending) return MHD_OK;
  CK(cudaEventRecord(m->ev_out, m->s_out));
  CK(cudaStreamWaitEvent(m->stream, m->ev_out, 0));
  return MHD_OK;
}

void free_pipeline(mhd_s* m) {
  if (m->s_in) cudaStreamSynchronize(m->s_in);
  if (m->s_out) cudaStreamSynchronize(m->s_out);
  for (int j = 0; j < 3; j++) {
    if (m->ev_in[j]) cudaEventDestroy(m->ev_in[j]);
    if (m->ev_free[j]) cudaEventDestroy(m->ev_free[j]);
  }
  if (m->ev_done) cudaEventDestroy(m->ev_done);
  if (m->ev_out) cudaEventDestroy(m->ev_out);
  if (m->s_in) cudaStreamDestroy(m->s_in);
  if (m->s_out) cudaStreamDestroy(m->s_out);
  cudaFree(m->stage_arena);
}

int make_pipeline(mhd_s* m) {
  if (m->stage_arena) return MHD_OK;
  cudaError_t e = cudaMalloc(&m->stage_arena, sizeof(float) * (size_t)m->N * 24);
  if (e != cudaSuccess) {
    m->stage_arena = nullptr;
    return cuda_fail(e, "cudaMalloc(staging)");
  }
  for (int j = 0; j < 3; j++)
    for (int q = 0; q < 8; q++) m->slot[j][q] = m->stage_arena + (size_t)m->N * (8 * j + q);
  if ((e = cudaStreamCreateWithFlags(&m->s_in, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&m->s_out, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&m->ev_done, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&m->ev_out, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "pipeline streams");
  for (int j = 0; j < 3; j++)
    if ((e = cudaEventCreateWithFlags(&m->ev_in[j], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&m->ev_free[j], cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "pipeline events");
  return MHD_OK;
}

int run_steps(mhd_s* m, int nsteps, double cfl) {
  for (int s = 0; s < nsteps; s++) {
    int rc = traced(m, MHD_K_CONTROL, [&] {
      CK(mhd::launch_step_control(&m->sc->rate[m->rcur], &m->sc->rate[1 - m->rcur], &m->sc->tau,
                                  &m->sc->time, cfl, 0.0, m->stream));
      return MHD_OK;
    });
    if (!rc) rc = full_step(m);
    if (rc) return rc;
  }
  return ensure_layout(m, 0);  // consecutive steps share their x-sweep layout
}

// ---- FP64 boxes ----------------------------------------------------------

int fluid64(mhd_s* m, int d, double tau) {
  mhd::Fluid64Args a;
  for (int q = 0; q < 8; q++) {
    a.in[q] = m->cur64[q];
    a.out[q] = m->spare64[q];
  }
  for (int k = 0; k < 3; k++) {
    a.n[k] = m->n[k];
    a.ih[k] = m->cpl[k] > 0.0 ? m->cpl[k] : (double)m->n[k];
  }
  a.gamma = m->gamma;
  a.tau = tau;
  CK(mhd::launch_fluid64(d, a, m->stream));
  for (int q = 0; q < 5; q++) std::swap(m->cur64[q], m->spare64[q]);
  return MHD_OK;
}

int magnetic64(mhd_s* m, int d, double tau) {
  mhd::Mag64Args a;
  for (int q = 0; q < 8; q++) {
    a.in[q] = m->cur64[q];
    a.out[q] = m->spare64[q];
  }
  a.E[0] = m->e64;
  a.E[1] = m->e64 + m->N;
  for (int k = 0; k < 3; k++) {
    a.n[k] = m->n[k];
    a.ih[k] = m->cpl[k] > 0.0 ? m->cpl[k] : (double)m->n[k];
  }
  a.tau = tau;
  CK(mhd::launch_mag64(d, a, m->stream));
  for (int q = 5; q < 8; q++) std::swap(m->cur64[q], m->spare64[q]);
  return MHD_OK;
}

// the schedule of Section II.B, every sweep with tau = dt/2
int full_step64(mhd_s* m, double dt) {
  const double tau = 0.5 * dt;
  int rc;
  for (int d = 0; d < 3; d++) {
    if ((rc = fluid64(m, d, tau))) return rc;
    if ((rc = magnetic64(m, d, tau))) return rc;
  }
  for (int d = 2; d >= 0; d--) {
    if ((rc = magnetic64(m, d, tau))) return rc;
    if ((rc = fluid64(m, d, tau))) return rc;
  }
  return MHD_OK;
}

int cfl_dt64(mhd_s* m, double cfl, double* dt) {
  double ih[3];
  for (int k = 0; k < 3; k++) ih[k] = m->cpl[k] > 0.0 ? m->cpl[k] : (double)m->n[k];
  CK(cudaMemsetAsync(m->rate64, 0, sizeof(unsigned long long), m->stream));
  const double* cf[8];
  for (int q = 0; q < 8; q++) cf[q] = m->cur64[q];
  CK(mhd::launch_cfl64(cf, m->n, ih, m->gamma, m->rate64, m->stream));
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, m->rate64, sizeof bits, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  double r;
  std::memcpy(&r, &bits, sizeof r);
  if (!(r > 0.0) || !std::isfinite(r)) {
    *dt = 0.0;
    return fail(MHD_E_STATE, "invalid state: NaN, rho <= 0 or p <= 0 in some cell");
  }
  *dt = 2.0 * cfl / r;
  return MHD_OK;
}

// calls that FP32 boxes only support
int fp32_only(const mhd_t* m) {
  return m->f64 ? fail(MHD_E_ARG, "not available for FP64 boxes (mhd_create_f64)") : MHD_OK;
}

bool check_box(const mhd_t* m) {
  if (!m) {
    fail(MHD_E_ARG, "null mhd_t");
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

mhd_t* mhd_create(int nx, int ny, int nz, double gamma) {
  if (nx < 4 || ny < 1 || nz < 1 || nx % 4 != 0) {
    fail(MHD_E_ARG, "bad box size (need nx >= 4, nx %% 4 == 0, ny, nz >= 1)");
    return nullptr;
  }
  if (!(gamma > 1.0)) {
    fail(MHD_E_ARG, "gamma must be > 1");
    return nullptr;
  }
  const long long N = (long long)nx * ny * nz;
  if (N >= (1LL << 31)) {
    fail(MHD_E_ARG, "box too large: a field must hold fewer than 2^31 cells");
    return nullptr;
  }
  mhd_s* m = new (std::nothrow) mhd_s;
  if (!m) {
    fail(MHD_E_OOM, "host allocation failed");
    return nullptr;
  }
  m->n[0] = nx;
  m->n[1] = ny;
  m->n[2] = nz;
  m->gamma = gamma;
  m->N = N;
  m->box.n[0] = nx;
  m->box.n[1] = ny;
  m->box.n[2] = nz;
  m->box = mhd::make_box(nx, ny, nz);
  cudaError_t e = mhd::prepare_mag_kernels();
  if (e != cudaSuccess) {
    cuda_fail(e, "kernel attributes");
    delete m;
    return nullptr;
  }
  e = cudaMalloc(&m->arena, sizeof(float) * (size_t)N * 16);
  if (e != cudaSuccess) {
    cuda_fail(e, "cudaMalloc(state)");
    delete m;
    return nullptr;
  }
  for (int q = 0; q < 8; q++) {
    m->cur[q] = m->arena + (size_t)N * q;
    m->spare[q] = m->arena + (size_t)N * (8 + q);
  }
  m->tbox.n[0] = ny;
  m->tbox.n[1] = nx;
  m->tbox.n[2] = nz;
  m->tbox.stride[0] = 1;
  m->tbox.stride[1] = ny;
  m->tbox.stride[2] = (long long)nx * ny;
  m->zbox.n[0] = nz;
  m->zbox.n[1] = ny;
  m->zbox.n[2] = nx;
  m->zbox.stride[0] = 1;
  m->zbox.stride[1] = nz;
  m->zbox.stride[2] = (long long)nz * ny;
  set_geometry(m);
  m->xpath = auto_xpath(m);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int nblk = mhd::diag_blocks(m->box);
  if ((e = cudaMalloc(&m->sc, sizeof(Scalars))) != cudaSuccess ||
      (e = cudaMalloc(&m->diag_partial, sizeof(double) * mhd::kDiagSlots * nblk)) != cudaSuccess ||
      (e = cudaMemset(m->sc, 0, sizeof(Scalars))) != cudaSuccess ||
      (e = cudaMemset(m->arena, 0, sizeof(float) * (size_t)N * 16)) != cudaSuccess) {
    cuda_fail(e, "mhd_create");
    cudaFree(m->arena);
    cudaFree(m->sc);
    cudaFree(m->diag_partial);
    delete m;
    return nullptr;
  }
  for (int d = 0; d < 3; d++) m->seg[d] = choose_seg(m, d);
  return m;
}

mhd_t* mhd_create_f64(int nx, int ny, int nz, double gamma) {
  if (nx < 1 || ny < 1 || nz < 1 || !(gamma > 1.0)) {
    fail(MHD_E_ARG, "need nx, ny, nz >= 1 and gamma > 1");
    return nullptr;
  }
  const long long N = (long long)nx * ny * nz;
  if (N >= (1LL << 31)) {
    fail(MHD_E_ARG, "box too large: a field must hold fewer than 2^31 cells");
    return nullptr;
  }
  mhd_s* m = new (std::nothrow) mhd_s;
  if (!m) {
    fail(MHD_E_OOM, "host allocation failed");
    return nullptr;
  }
  m->n[0] = nx;
  m->n[1] = ny;
  m->n[2] = nz;
  m->gamma = gamma;
  m->N = N;
  m->box = mhd::make_box(nx, ny, nz);
  m->f64 = true;
  cudaError_t e;
  if ((e = cudaMalloc(&m->arena64, sizeof(double) * (size_t)N * 18)) != cudaSuccess ||
      (e = cudaMalloc(&m->rate64, sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMemset(m->arena64, 0, sizeof(double) * (size_t)N * 18)) != cudaSuccess) {
    cuda_fail(e, "mhd_create_f64");
    cudaFree(m->arena64);
    cudaFree(m->rate64);
    delete m;
    return nullptr;
  }
  for (int q = 0; q < 8; q++) {
    m->cur64[q] = m->arena64 + (size_t)N * q;
    m->spare64[q] = m->arena64 + (size_t)N * (8 + q);
  }
  m->e64 = m->arena64 + (size_t)N * 16;
  return m;
}

int mhd_set_state_f64(mhd_t* m, const double* const f[8], int on_device) {
  if (!check_box(m) || !f) return fail(MHD_E_ARG, "null argument");
  if (!m->f64) return fail(MHD_E_ARG, "not an FP64 box (mhd_create_f64)");
  for (int q = 0; q < 8; q++)
    if (!f[q]) return fail(MHD_E_ARG, "null field pointer");
  for (int q = 0; q < 8; q++)
    CK(cudaMemcpyAsync(m->cur64[q], f[q], sizeof(double) * (size_t)m->N,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
  m->time64 = 0.0;
  return MHD_OK;
}

int mhd_get_state_f64(const mhd_t* m, double* const f[8], int on_device) {
  if (!check_box(m) || !f) return fail(MHD_E_ARG, "null argument");
  if (!m->f64) return fail(MHD_E_ARG, "not an FP64 box (mhd_create_f64)");
  for (int q = 0; q < 8; q++)
    if (!f[q]) return fail(MHD_E_ARG, "null field pointer");
  for (int q = 0; q < 8; q++)
    CK(cudaMemcpyAsync(f[q], m->cur64[q], sizeof(double) * (size_t)m->N,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return MHD_OK;
}

void mhd_destroy(mhd_t* m) {
  if (!m) return;
  cudaFree(m->arena64);
  cudaFree(m->rate64);
  free_pipeline(m);
  drop_events(m);
  cudaFree(m->pencil_c);
  cudaFree(m->arena);
  cudaFree(m->sc);
  cudaFree(m->diag_partial);
  delete m;
}

int mhd_set_stream(mhd_t* m, void* cuda_stream) {
  if (!check_box(m)) return MHD_E_ARG;
  m->stream = (cudaStream_t)cuda_stream;
  return MHD_OK;
}

int mhd_set_state(mhd_t* m, const float* const f[8], int on_device) {
  if (!check_box(m) || !f) return fail(MHD_E_ARG, "null argument");
  if (int rc = fp32_only(m)) return rc;
  for (int q = 0; q < 8; q++)
    if (!f[q]) return fail(MHD_E_ARG, "null field pointer");
  if (int rc = join_pipeline(m)) return rc;
  const size_t bytes = sizeof(float) * (size_t)m->N;
  if (m->layout) {  // back to the plain layout (the old state is overwritten)
    const int a = m->layout == 1 ? 2 : 3;  // the slot exchanged with x
    std::swap(m->cur[1], m->cur[a]);
    std::swap(m->spare[1], m->spare[a]);
    std::swap(m->cur[5], m->cur[4 + a]);
    std::swap(m->spare[5], m->spare[4 + a]);
    m->layout = 0;
  }
  for (int q = 0; q < 8; q++)
    CK(cudaMemcpyAsync(m->cur[q], f[q], bytes,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
  CK(cudaMemsetAsync(m->sc, 0, sizeof(Scalars), m->stream));
  m->rcur = 0;
  return state_rate(m, &m->sc->rate[0]);
}

int mhd_get_state(const mhd_t* m, float* const f[8], int on_device) {
  if (!check_box(m) || !f) return fail(MHD_E_ARG, "null argument");
  if (int rc = fp32_only(m)) return rc;
  for (int q = 0; q < 8; q++)
    if (!f[q]) return fail(MHD_E_ARG, "null field pointer");
  const size_t bytes = sizeof(float) * (size_t)m->N;
  if (m->layout) return fail(MHD_E_ARG, "internal: state left in the exchanged layout");
  if (int rc = join_pipeline(const_cast<mhd_s*>(m))) return rc;
  for (int q = 0; q < 8; q++)
    CK(cudaMemcpyAsync(f[q], m->cur[q], bytes,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return MHD_OK;
}

int mhd_cfl_dt(mhd_t* m, double cfl, double* dt_full) {
  if (!check_box(m) || !dt_full) return fail(MHD_E_ARG, "null argument");
  if (!(cfl > 0.0)) return fail(MHD_E_ARG, "cfl must be > 0");
  if (m->f64) return cfl_dt64(m, cfl, dt_full);
  unsigned w[3] = {0, 0, 0};  // rate[0], rate[1], err
  CK(cudaMemcpyAsync(w, &m->sc->rate[0], sizeof w, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  if (w[2]) {
    *dt_full = 0.0;
    return fail(MHD_E_TIMEOUT, "a staged chunk of a sweep did not arrive within the wait bound");
  }
  float r;
  std::memcpy(&r, &w[m->rcur], sizeof r);
  if (!(r > 0.f) || !std::isfinite(r)) {
    *dt_full = 0.0;
    return fail(MHD_E_STATE, "invalid state: NaN, rho <= 0 or p <= 0 in some cell");
  }
  *dt_full = 2.0 * cfl / (double)r;
  return MHD_OK;
}

int mhd_step(mhd_t* m, double dt_full) {
  if (!check_box(m)) return MHD_E_ARG;
  if (!(dt_full >= 0.0) || !std::isfinite(dt_full)) return fail(MHD_E_ARG, "dt must be finite and >= 0");
  if (m->f64) {
    if (int rc = full_step64(m, dt_full)) return rc;
    m->time64 += dt_full;
    return MHD_OK;
  }
  if (int rc = join_pipeline(m)) return rc;
  int rc = traced(m, MHD_K_CONTROL, [&] {
    CK(mhd::launch_step_control(&m->sc->rate[m->rcur], &m->sc->rate[1 - m->rcur], &m->sc->tau,
                                &m->sc->time, -1.0, 0.5 * dt_full, m->stream));
    return MHD_OK;
  });
  if (!rc) rc = full_step(m);
  return rc ? rc : ensure_layout(m, 0);
}

int mhd_run(mhd_t* m, int nsteps, double cfl) {
  if (!check_box(m)) return MHD_E_ARG;
  if (nsteps < 0 || !(cfl > 0.0)) return fail(MHD_E_ARG, "need nsteps >= 0 and cfl > 0");
  if (m->f64) {  // the timestep through the host: one synchronisation per step
    for (int s = 0; s < nsteps; s++) {
      double dt;
      if (int rc = cfl_dt64(m, cfl, &dt)) return rc;
      if (int rc = full_step64(m, dt)) return rc;
      m->time64 += dt;
    }
    return MHD_OK;
  }
  if (int rc = join_pipeline(m)) return rc;
  return run_steps(m, nsteps, cfl);
}

// Pipelined host runs.  Submission k uses staging slot j = k mod 3:
//   s_in:   wait until slot j's arrays are no longer read (ev_free[j]), copy
//           the host input into them, record ev_in[j];
//   stream: wait ev_in[j], adopt slot j's arrays as the state (the arrays of
//           the previous result move into slot j; ev_free[j], recorded on
//           s_out now, marks the end of that result's output copy), reset the
//           CFL rate and time, run nsteps, record ev_done;
//   s_out:  wait ev_done, copy the state out to the host.
// So the steps of submission k overlap the input copy of k+1 and the output
// copy of k-1.
int mhd_submit(mhd_t* m, const float* const in[8], float* const out[8], int nsteps, double cfl) {
  if (!check_box(m) || !in || !out) return fail(MHD_E_ARG, "null argument");
  if (int rc = fp32_only(m)) return rc;
  for (int q = 0; q < 8; q++)
    if (!in[q] || !out[q]) return fail(MHD_E_ARG, "null field pointer");
  if (nsteps < 0 || !(cfl > 0.0)) return fail(MHD_E_ARG, "need nsteps >= 0 and cfl > 0");
  if (m->layout) return fail(MHD_E_ARG, "internal: state left in the exchanged layout");
  if (int rc = make_pipeline(m)) return rc;
  const size_t bytes = sizeof(float) * (size_t)m->N;
  const int j = m->next_slot;
  m->next_slot = (j + 1) % 3;
  if (m->slot_used[j]) CK(cudaStreamWaitEvent(m->s_in, m->ev_free[j], 0));
  m->slot_used[j] = true;
  for (int q = 0; q < 8; q++) CK(cudaMemcpyAsync(m->slot[j][q], in[q], bytes, cudaMemcpyHostToDevice, m->s_in));
  CK(cudaEventRecord(m->ev_in[j], m->s_in));
  CK(cudaStreamWaitEvent(m->stream, m->ev_in[j], 0));
  for (int q = 0; q < 8; q++) std::swap(m->cur[q], m->slot[j][q]);
  CK(cudaEventRecord(m->ev_free[j], m->s_out));
  CK(cudaMemsetAsync(m->sc, 0, sizeof(Scalars), m->stream));
  m->rcur = 0;
  if (int rc = state_rate(m, &m->sc->rate[0])) return rc;
  if (int rc = run_steps(m, nsteps, cfl)) return rc;
  CK(cudaEventRecord(m->ev_done, m->stream));
  CK(cudaStreamWaitEvent(m->s_out, m->ev_done, 0));
  for (int q = 0; q < 8; q++) CK(cudaMemcpyAsync(out[q], m->cur[q], bytes, cudaMemcpyDeviceToHost, m->s_out));
  m->pipe_pending = true;
  return MHD_OK;
}

int mhd_drain(mhd_t* m) {
  if (!check_box(m)) return MHD_E_ARG;
  if (!m->pipe_pending) return MHD_OK;
  if (int rc = join_pipeline(m)) return rc;
  CK(cudaStreamSynchronize(m->s_out));
  CK(cudaStreamSynchronize(m->stream));
  m->pipe_pending = false;
  return MHD_OK;
}

int mhd_time(const mhd_t* m, double* t) {
  if (!check_box(m) || !t) return fail(MHD_E_ARG, "null argument");
  if (m->f64) {
    *t = m->time64;
    return MHD_OK;
  }
  CK(cudaMemcpyAsync(t, &m->sc->time, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return MHD_OK;
}

int mhd_sweep(mhd_t* m, int axis, int kind, double tau) {
  if (!check_box(m)) return MHD_E_ARG;
  if (axis < 0 || axis > 2 || kind < 0 || kind > 1 || !(tau >= 0.0))
    return fail(MHD_E_ARG, "bad axis/kind/tau");
  if (m->f64) return kind == 0 ? fluid64(m, axis, tau) : magnetic64(m, axis, tau);
  // a single sweep does not advance the simulation time; afterwards the CFL
  // rate is recomputed for the new state
  if (int rc = join_pipeline(m)) return rc;
  CK(mhd::launch_set_tau(&m->sc->tau, tau, m->stream));
  int rc = kind == 0 ? fluid(m, axis, false) : magnetic(m, axis);
  if (!rc) rc = ensure_layout(m, 0);
  if (rc) return rc;
  return state_rate(m, &m->sc->rate[m->rcur]);
}

int mhd_set_boundary(mhd_t* m, int axis, int mode) {
  if (!check_box(m)) return MHD_E_ARG;
  if (int rc = fp32_only(m)) return rc;
  if (axis < 0 || axis > 2 || mode < 0 || mode > 2) return fail(MHD_E_ARG, "bad axis or boundary mode");
  if (mode && m->n[axis] < 3 * mhd::kGhost)
    return fail(MHD_E_ARG, "a non-periodic axis needs at least 12 cells (4 ghost cells at each end)");
  if (int rc = join_pipeline(m)) return rc;
  m->bc[axis] = mode;
  // the rate of the current state under the new boundaries
  return state_rate(m, &m->sc->rate[m->rcur]);
}

int mhd_fill_ghosts(mhd_t* m) {
  if (!check_box(m)) return MHD_E_ARG;
  if (int rc = fp32_only(m)) return rc;
  if (int rc = join_pipeline(m)) return rc;
  return fill_ghosts(m);
}

int mhd_set_segments(mhd_t* m, int seg_x, int seg_y, int seg_z) {
  if (!check_box(m)) return MHD_E_ARG;
  if (int rc = fp32_only(m)) return rc;
  const int seg[3] = {seg_x, seg_y, seg_z};
  for (int d = 0; d < 3; d++)
    if (seg[d] != 0 && (seg[d] < 4 || seg[d] % 4 != 0 || m->n[d] % seg[d] != 0))
      return fail(MHD_E_ARG, "segment length must be a multiple of 4 dividing n_d");
  for (int d = 0; d < 3; d++) m->seg[d] = seg[d] ? seg[d] : choose_seg(m, d);
  return MHD_OK;
}

int mhd_set_xpath(mhd_t* m, int mode) {
  if (!check_box(m)) return MHD_E_ARG;
  if (int rc = fp32_only(m)) return rc;
  if (mode < 0 || mode > 3) return fail(MHD_E_ARG, "x path mode must be 0, 1, 2 or 3");
  if (mode == 3 && (m->n[0] % 4 || m->n[1] % 4 || m->n[2] % 4 || m->n[1] > 65535))
    return fail(MHD_E_ARG, "x path 3 needs every extent a multiple of 4 (and ny <= 65535)");
  if (m->layout) return fail(MHD_E_ARG, "internal: state left in the exchanged layout");
  m->xpath_req = mode;
  m->xpath = mode ? mode : auto_xpath(m);
  return MHD_OK;
}

int mhd_set_scheme(mhd_t* m, int limiter, int freezing) {
  if (!check_box(m)) return MHD_E_ARG;
  if (m->f64 && (limiter || freezing)) return fail(MHD_E_ARG, "FP64 boxes run the paper's scheme only");
  if (m->f64) return MHD_OK;
  if (limiter < 0 || limiter > 2 || freezing < 0 || freezing > 2 || (limiter && freezing))
    return fail(MHD_E_ARG, "limiter 0..2, freezing 0..2, one ablation at a time");
  if (freezing == 2 && !m->pencil_c) {  // two speeds per pencil of the longest pencil family
    const int nmin = std::min(m->n[0], std::min(m->n[1], m->n[2]));
    if (cudaMalloc(&m->pencil_c, sizeof(float) * 2 * (size_t)(m->N / nmin)) != cudaSuccess) {
      m->pencil_c = nullptr;
      return fail(MHD_E_OOM, "per-pencil freezing speeds");
    }
  }
  m->lim = limiter;
  m->fast = freezing;
  if (!m->xpath_req && !m->layout) m->xpath = auto_xpath(m);
  return MHD_OK;
}

int mhd_set_resolution(mhd_t* m, double cx, double cy, double cz) {
  if (!check_box(m)) return MHD_E_ARG;
  const double c[3] = {cx, cy, cz};
  for (int d = 0; d < 3; d++)
    if (!(c[d] >= 0.0) || !std::isfinite(c[d]) || c[d] > 3.0e38) return fail(MHD_E_ARG, "cells per unit length must be finite and >= 0");
  for (int d = 0; d < 3; d++) m->cpl[d] = c[d];
  if (m->f64) return MHD_OK;  // the FP64 CFL rate is computed when asked
  if (int rc = join_pipeline(m)) return rc;
  set_geometry(m);
  return state_rate(m, &m->sc->rate[m->rcur]);
}

int mhd_set_interior(mhd_t* m, int axis, int lo, int hi) {
  if (!check_box(m)) return MHD_E_ARG;
  if (int rc = fp32_only(m)) return rc;
  if (axis < 0 || axis > 2 || lo < 0 || hi > m->n[axis] || lo >= hi)
    return fail(MHD_E_ARG, "need 0 <= lo < hi <= n along the axis");
  if (int rc = join_pipeline(m)) return rc;
  m->own_lo[axis] = lo;
  m->own_hi[axis] = hi;
  return state_rate(m, &m->sc->rate[m->rcur]);
}

int mhd_copy_planes(mhd_t* m, int z0, int nplanes, float* const f[8], int into_box, int on_device) {
  if (!check_box(m) || !f) return fail(MHD_E_ARG, "null argument");
  if (int rc = fp32_only(m)) return rc;
  for (int q = 0; q < 8; q++)
    if (!f[q]) return fail(MHD_E_ARG, "null field pointer");
  if (z0 < 0 || nplanes < 0 || z0 + nplanes > m->n[2]) return fail(MHD_E_ARG, "planes outside the box");
  if (m->layout) return fail(MHD_E_ARG, "internal: state left in the exchanged layout");
  if (int rc = join_pipeline(m)) return rc;
  const size_t plane = (size_t)m->n[0] * m->n[1];
  const size_t bytes = sizeof(float) * plane * nplanes;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                        : (into_box ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  for (int q = 0; q < 8; q++) {
    float* boxp = m->cur[q] + plane * z0;
    if (into_box)
      CK(cudaMemcpyAsync(boxp, f[q], bytes, kind, m->stream));
    else
      CK(cudaMemcpyAsync(f[q], boxp, bytes, kind, m->stream));
  }
  if (!on_device) CK(cudaStreamSynchronize(m->stream));
  return MHD_OK;
}

int mhd_set_fusion(mhd_t* m, int on) {
  if (!check_box(m)) return MHD_E_ARG;
  if (on < 0 || on > 1) return fail(MHD_E_ARG, "fusion must be 0 or 1");
  m->fuse = on;
  return MHD_OK;
}

int mhd_set_tma(mhd_t* m, int on) {
  if (!check_box(m)) return MHD_E_ARG;
  if (int rc = fp32_only(m)) return rc;
  if (on < 0 || on > 1) return fail(MHD_E_ARG, "tma must be 0 or 1");
  m->tma = on;
  if (!m->xpath_req && !m->layout) m->xpath = auto_xpath(m);
  return MHD_OK;
}

int mhd_tma_sweeps(const mhd_t* m, long long* count) {
  if (!check_box(m) || !count) return fail(MHD_E_ARG, "null argument");
  *count = m->tma_sweeps;
  return MHD_OK;
}

int mhd_set_pressure_floor(mhd_t* m, double p_floor) {
  if (!check_box(m)) return MHD_E_ARG;
  if (int rc = fp32_only(m)) return rc;
  if (!(p_floor >= 0.0)) return fail(MHD_E_ARG, "pressure floor must be >= 0");
  m->p_floor = (float)p_floor;
  return MHD_OK;
}

int mhd_diagnostics(mhd_t* m, double out[10]) {
  if (!check_box(m) || !out) return fail(MHD_E_ARG, "null argument");
  if (int rc = fp32_only(m)) return rc;
  if (int rc = join_pipeline(m)) return rc;
  const float* cf[8];
  field_ptrs(m, cf);
  if (int rc = traced(m, MHD_K_CONTROL, [&] {
        CK(mhd::launch_diagnostics(cf, m->box, m->gamma, m->diag_partial, m->sc->diag, m->stream));
        return MHD_OK;
      }))
    return rc;
  CK(cudaMemcpyAsync(out, m->sc->diag, sizeof(double) * 10, cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return MHD_OK;
}

int mhd_profile(mhd_t* m, int capacity) {
  if (!check_box(m)) return MHD_E_ARG;
  if (capacity < 0) return fail(MHD_E_ARG, "capacity must be >= 0");
  CK(cudaStreamSynchronize(m->stream));
  drop_events(m);
  m->ev.resize(2 * (size_t)capacity);
  for (auto& e : m->ev) {
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) {
      e = nullptr;
      drop_events(m);
      return cuda_fail(err, "cudaEventCreate");
    }
  }
  m->ev_kind.assign((size_t)capacity, -1);
  return MHD_OK;
}

int mhd_profile_read(mhd_t* m, int counts[], double ms[]) {
  if (!check_box(m) || !counts || !ms) return fail(MHD_E_ARG, "null argument");
  for (int k = 0; k < MHD_K_CLASSES; k++) {
    counts[k] = 0;
    ms[k] = 0.0;
  }
  CK(cudaStreamSynchronize(m->stream));
  for (size_t i = 0; i < m->ev_used; i++) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, m->ev[2 * i], m->ev[2 * i + 1]));
    counts[m->ev_kind[i]] += 1;
    ms[m->ev_kind[i]] += t;
  }
  return MHD_OK;
}

const char* mhd_last_error(void) { return g_err; }

}  // extern "C"
