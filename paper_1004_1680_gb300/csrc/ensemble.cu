// Batched ensembles of independent periodic boxes of uneven sizes.
//
// All boxes live in one concatenated arena (each field's boxes back to back,
// every box starting on a 128-byte boundary) and advance together: each sweep
// of the Section II.B schedule is ONE launch over a work list whose items are
// (box, tile) pairs of every box, with per-box geometry, segment length,
// timestep and CFL accumulator (EnsArgs in mhd_launch.h).  Each box keeps its
// own CFL timestep and simulation time.  A run of steps is captured once into
// a CUDA graph and replayed; graphs are cached by everything they bake in
// (step count, cfl, buffer assignment, accumulator parity).
//
// The per-box arithmetic is exactly that of a single box run with the same
// x path and segments, so an ensemble member is bitwise equal to the same box
// run alone.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "mhd.h"
#include "mhd_launch.h"

namespace {

#define CKE(call)                                                                 \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return mhd::set_error(e_ == cudaErrorMemoryAllocation ? MHD_E_OOM : MHD_E_CUDA, #call, \
                            cudaGetErrorString(e_));                              \
  } while (0)

struct WorkList {
  int4* d = nullptr;
  int n = 0;
  int minext = 0;  // smallest extent along the launch's kernel axis
};

struct GraphKey {
  int nsteps, rcur, layout;
  double cfl;
  float* cur[8];
  float* spare[8];
  bool operator<(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) < 0; }
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  float* cur[8];
  float* spare[8];
  int rcur, layout;
};

// process-wide autotuner cache: dims signature -> (xpath, segment divisor)
std::mutex g_tune_lock;
std::map<std::string, std::pair<int, int>> g_tune_cache;

}  // namespace

struct mhd_ens_s {
  int nbox = 0;
  double gamma = 5.0 / 3.0;
  std::vector<mhd::EnsBox> boxes;
  mhd::EnsBox* boxes_d = nullptr;
  long long ntot = 0;  // cells per field in the arena
  float* arena = nullptr;
  float* cur[8];
  float* spare[8];
  int layout = 0;
  int xpath = 2;
  int segdiv = 1;
  float p_floor = 0.f;
  float* tau = nullptr;
  unsigned* rate[2] = {nullptr, nullptr};
  double* time = nullptr;
  int rcur = 0;
  WorkList fluid[3], mag[3], trans[2];  // sweeps by physical axis; transposes by input layout
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // private stream used to capture graphs
  std::map<GraphKey, GraphEntry> graphs;
  double* diag_partial = nullptr;
  double* diag_out = nullptr;
};

namespace {

void free_lists(mhd_ens_s* e) {
  for (WorkList* l : {&e->fluid[0], &e->fluid[1], &e->fluid[2], &e->mag[0], &e->mag[1], &e->mag[2],
                      &e->trans[0], &e->trans[1]}) {
    cudaFree(l->d);
    l->d = nullptr;
    l->n = 0;
  }
}

void drop_graphs(mhd_ens_s* e) {
  for (auto& kv : e->graphs) cudaGraphExecDestroy(kv.second.exec);
  e->graphs.clear();
}

// the layout a sweep along physical axis d runs in (x: per x path; y, z: plain)
int sweep_layout(const mhd_ens_s* e, int d) { return (d == 0 && e->xpath == 2) ? 1 : 0; }

int kernel_axis(int layout, int d) { return (layout && d < 2) ? 1 - d : d; }

int upload(WorkList* l, const std::vector<int4>& items, int minext) {
  cudaFree(l->d);
  l->d = nullptr;
  l->n = (int)items.size();
  l->minext = minext;
  if (items.empty()) return MHD_OK;
  CKE(cudaMalloc(&l->d, sizeof(int4) * items.size()));
  CKE(cudaMemcpy(l->d, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
  return MHD_OK;
}

// Segment lengths and work lists for the current x path and divisor.
int build_lists(mhd_ens_s* e) {
  for (auto& b : e->boxes) {
    for (int d = 0; d < 3; d++) {
      int seg = b.n[d];
      if (e->segdiv > 1 && b.n[d] % (4 * e->segdiv) == 0 && b.n[d] / e->segdiv >= 16)
        seg = b.n[d] / e->segdiv;
      b.seg[d] = seg;
    }
  }
  CKE(cudaMemcpy(e->boxes_d, e->boxes.data(), sizeof(mhd::EnsBox) * e->nbox, cudaMemcpyHostToDevice));
  for (int kind = 0; kind < 2; kind++) {
    const int W = kind == 0 ? 4 : mhd::kMagWarps;  // rows per block: fluid, magnetic
    for (int d = 0; d < 3; d++) {
      const int L = sweep_layout(e, d), ka = kernel_axis(L, d);
      const int A = (ka == 0) ? 1 : 0, O = (ka == 2) ? 1 : 2;
      std::vector<int4> items;
      int minext = 1 << 30;
      for (int bi = 0; bi < e->nbox; bi++) {
        const mhd::EnsBox& b = e->boxes[bi];
        int n[3] = {L ? b.n[1] : b.n[0], L ? b.n[0] : b.n[1], b.n[2]};
        minext = std::min(minext, n[ka]);
        // fluid y and z kernel axes: runs of 32 W consecutive pencils (the
        // kernel's row-order mapping); otherwise tiles of 32 x W pencils
        const bool runs = kind == 0 && ka != 0;
        const int gx = runs ? (n[A] * n[O] + 32 * W - 1) / (32 * W) : (n[A] + 31) / 32;
        const int gy = runs ? 1 : (n[O] + W - 1) / W, gz = n[ka] / b.seg[d];
        for (int z = 0; z < gz; z++)
          for (int y = 0; y < gy; y++)
            for (int x = 0; x < gx; x++) items.push_back(make_int4(bi, x, y, z));
      }
      int rc = upload(kind == 0 ? &e->fluid[d] : &e->mag[d], items, minext);
      if (rc) return rc;
    }
  }
  for (int L = 0; L < 2; L++) {
    std::vector<int4> items;
    for (int bi = 0; bi < e->nbox; bi++) {
      const mhd::EnsBox& b = e->boxes[bi];
      const int n0 = L ? b.n[1] : b.n[0], n1 = L ? b.n[0] : b.n[1];
      for (int k = 0; k < b.n[2]; k++)
        for (int j = 0; j < (n1 + 31) / 32; j++)
          for (int i = 0; i < (n0 + 31) / 32; i++) items.push_back(make_int4(bi, i, j, k));
    }
    int rc = upload(&e->trans[L], items, 0);
    if (rc) return rc;
  }
  drop_graphs(e);
  return MHD_OK;
}

mhd::EnsArgs ens_args(const mhd_ens_s* e, const WorkList& l, int layout, int d, unsigned* rate) {
  mhd::EnsArgs a;
  a.items = l.d;
  a.boxes = e->boxes_d;
  a.tau_arr = e->tau;
  a.rate_arr = rate;
  a.layout = layout;
  a.phys_axis = d;
  return a;
}

int exchange(mhd_ens_s* e, cudaStream_t s) {
  mhd::TransposeArgs a;
  for (int q = 0; q < 8; q++) {
    a.in[q] = e->cur[q];
    a.out[q] = e->spare[q];
  }
  a.n[0] = a.n[1] = a.n[2] = 32;
  a.ens = ens_args(e, e->trans[e->layout], e->layout, 0, nullptr);
  a.nblocks = e->trans[e->layout].n;
  CKE(mhd::launch_transpose01(a, s));
  static const int relabel[8] = {0, 2, 1, 3, 4, 6, 5, 7};
  float* nc[8];
  float* ns[8];
  for (int q = 0; q < 8; q++) {
    nc[relabel[q]] = e->spare[q];
    ns[relabel[q]] = e->cur[q];
  }
  for (int q = 0; q < 8; q++) {
    e->cur[q] = nc[q];
    e->spare[q] = ns[q];
  }
  e->layout ^= 1;
  return MHD_OK;
}

int ensure_layout(mhd_ens_s* e, int L, cudaStream_t s) { return e->layout == L ? MHD_OK : exchange(e, s); }

int fluid(mhd_ens_s* e, int d, bool rate, cudaStream_t s) {
  int rc = ensure_layout(e, sweep_layout(e, d), s);
  if (rc) return rc;
  const int ka = kernel_axis(e->layout, d);
  mhd::FluidArgs a;
  for (int q = 0; q < 8; q++) {
    a.in[q] = e->cur[q];
    a.out[q] = e->spare[q];
  }
  a.box.n[0] = a.box.n[1] = a.box.n[2] = 32;
  a.box.n[ka] = e->fluid[d].minext;  // selects the short-axis kernel if any box needs it
  a.gamma = (float)e->gamma;
  a.p_floor = e->p_floor;
  a.tau = e->tau;
  a.rate = nullptr;
  a.seg = 1;
  a.ens = ens_args(e, e->fluid[d], e->layout, d, rate ? e->rate[1 - e->rcur] : nullptr);
  a.nblocks = e->fluid[d].n;
  CKE(mhd::launch_fluid(ka, rate, a, s));
  for (int q = 0; q < 5; q++) std::swap(e->cur[q], e->spare[q]);
  return MHD_OK;
}

// passes = 2: the two middle z sweeps of a step in one launch (bitwise the
// same as two)
int magnetic(mhd_ens_s* e, int d, cudaStream_t s, int passes = 1) {
  int rc = ensure_layout(e, sweep_layout(e, d), s);
  if (rc) return rc;
  const int ka = kernel_axis(e->layout, d);
  mhd::MagArgs a;
  for (int q = 0; q < 8; q++) a.in[q] = e->cur[q];
  for (int q = 0; q < 3; q++) a.out[q] = e->spare[5 + q];
  a.box.n[0] = a.box.n[1] = a.box.n[2] = 32;
  a.box.n[ka] = e->mag[d].minext;
  a.tau = e->tau;
  a.seg = 1;
  a.ens = ens_args(e, e->mag[d], e->layout, d, nullptr);
  a.nblocks = e->mag[d].n;
  a.passes = passes;
  CKE(mhd::launch_mag(ka, a, s));
  for (int q = 5; q < 8; q++) std::swap(e->cur[q], e->spare[q]);
  return MHD_OK;
}

// One step of every box (Section II.B schedule), launched on stream s.
int ens_step(mhd_ens_s* e, double cfl, cudaStream_t s) {
  CKE(mhd::launch_ens_control(e->rate[e->rcur], e->rate[1 - e->rcur], e->tau, e->time, e->nbox, cfl, s));
  int rc;
  for (int d = 0; d < 2; d++) {
    if ((rc = fluid(e, d, false, s))) return rc;
    if ((rc = magnetic(e, d, s))) return rc;
  }
  if ((rc = fluid(e, 2, false, s))) return rc;
  if ((rc = magnetic(e, 2, s, 2))) return rc;  // [M_z][M_z] in one launch
  if ((rc = fluid(e, 2, false, s))) return rc;
  for (int d = 1; d >= 0; d--) {
    if ((rc = magnetic(e, d, s))) return rc;
    if ((rc = fluid(e, d, d == 0, s))) return rc;
  }
  e->rcur ^= 1;
  return MHD_OK;
}

int box_ptrs(const mhd_ens_s* e, int b, const float* out[8]) {
  for (int q = 0; q < 8; q++) out[q] = e->cur[q] + e->boxes[b].offset;
  return MHD_OK;
}

mhd::Box plain_box(const mhd::EnsBox& b) { return mhd::make_box(b.n[0], b.n[1], b.n[2]); }

bool bad(const mhd_ens_t* e, int b) { return !e || b < 0 || b >= e->nbox; }

int run_graph(mhd_ens_s* e, int nsteps, double cfl) {
  GraphKey k;
  std::memset(&k, 0, sizeof k);
  k.nsteps = nsteps;
  k.rcur = e->rcur;
  k.layout = e->layout;
  k.cfl = cfl;
  std::memcpy(k.cur, e->cur, sizeof k.cur);
  std::memcpy(k.spare, e->spare, sizeof k.spare);
  auto it = e->graphs.find(k);
  if (it == e->graphs.end()) {
    if (!e->cap) CKE(cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking));
    CKE(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
    int rc = MHD_OK;
    for (int s = 0; s < nsteps && !rc; s++) rc = ens_step(e, cfl, e->cap);
    if (!rc) rc = ensure_layout(e, 0, e->cap);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(e->cap, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ce != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "cudaStreamEndCapture", cudaGetErrorString(ce));
    GraphEntry ent;
    ce = cudaGraphInstantiate(&ent.exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return mhd::set_error(MHD_E_CUDA, "cudaGraphInstantiate", cudaGetErrorString(ce));
    std::memcpy(ent.cur, e->cur, sizeof ent.cur);
    std::memcpy(ent.spare, e->spare, sizeof ent.spare);
    ent.rcur = e->rcur;
    ent.layout = e->layout;
    // capture advanced the bookkeeping without running anything: rewind it
    std::memcpy(e->cur, k.cur, sizeof k.cur);
    std::memcpy(e->spare, k.spare, sizeof k.spare);
    e->rcur = k.rcur;
    e->layout = k.layout;
    it = e->graphs.emplace(k, ent).first;
  }
  CKE(cudaGraphLaunch(it->second.exec, e->stream));
  std::memcpy(e->cur, it->second.cur, sizeof e->cur);
  std::memcpy(e->spare, it->second.spare, sizeof e->spare);
  e->rcur = it->second.rcur;
  e->layout = it->second.layout;
  return MHD_OK;
}

}  // namespace

extern "C" {

mhd_ens_t* mhd_ens_create(int nbox, const int* dims3, double gamma) {
  if (nbox < 1 || !dims3 || !(gamma > 1.0)) {
    mhd::set_error(MHD_E_ARG, "mhd_ens_create", "need nbox >= 1, dims and gamma > 1");
    return nullptr;
  }
  mhd_ens_s* e = new (std::nothrow) mhd_ens_s;
  if (!e) {
    mhd::set_error(MHD_E_OOM, "mhd_ens_create", "host allocation failed");
    return nullptr;
  }
  e->nbox = nbox;
  e->gamma = gamma;
  long long off = 0;
  long long biggest = 0;
  for (int b = 0; b < nbox; b++) {
    mhd::EnsBox x;
    std::memset(&x, 0, sizeof x);
    for (int d = 0; d < 3; d++) x.n[d] = dims3[3 * b + d];
    if (x.n[0] < 4 || x.n[0] % 4 || x.n[1] < 1 || x.n[2] < 1) {
      mhd::set_error(MHD_E_ARG, "mhd_ens_create", "box sizes need nx >= 4, nx % 4 == 0, ny, nz >= 1");
      delete e;
      return nullptr;
    }
    const long long N = (long long)x.n[0] * x.n[1] * x.n[2];
    x.offset = (int)off;
    off += (N + 31) / 32 * 32;
    biggest = std::max(biggest, N);
    e->boxes.push_back(x);
  }
  if (off >= (1LL << 31)) {
    mhd::set_error(MHD_E_ARG, "mhd_ens_create", "ensemble too large: at most 2^31 - 1 cells per field");
    delete e;
    return nullptr;
  }
  e->ntot = off;
  e->xpath = 2;
  const mhd::Box big = mhd::make_box((int)std::min<long long>(biggest, 1 << 30), 1, 1);
  const int nblk = mhd::diag_blocks(big);
  cudaError_t ce;
  if ((ce = mhd::prepare_mag_kernels()) != cudaSuccess ||
      (ce = cudaMalloc(&e->arena, sizeof(float) * (size_t)off * 16)) != cudaSuccess ||
      (ce = cudaMalloc(&e->boxes_d, sizeof(mhd::EnsBox) * nbox)) != cudaSuccess ||
      (ce = cudaMalloc(&e->tau, sizeof(float) * nbox)) != cudaSuccess ||
      (ce = cudaMalloc(&e->rate[0], sizeof(unsigned) * nbox * 2)) != cudaSuccess ||
      (ce = cudaMalloc(&e->time, sizeof(double) * nbox)) != cudaSuccess ||
      (ce = cudaMalloc(&e->diag_partial, sizeof(double) * mhd::kDiagSlots * nblk)) != cudaSuccess ||
      (ce = cudaMalloc(&e->diag_out, sizeof(double) * 10)) != cudaSuccess ||
      (ce = cudaMemset(e->arena, 0, sizeof(float) * (size_t)off * 16)) != cudaSuccess ||
      (ce = cudaMemset(e->rate[0], 0, sizeof(unsigned) * nbox * 2)) != cudaSuccess ||
      (ce = cudaMemset(e->time, 0, sizeof(double) * nbox)) != cudaSuccess) {
    mhd::set_error(ce == cudaErrorMemoryAllocation ? MHD_E_OOM : MHD_E_CUDA, "mhd_ens_create",
                   cudaGetErrorString(ce));
    mhd_ens_destroy(e);
    return nullptr;
  }
  e->rate[1] = e->rate[0] + nbox;
  for (int q = 0; q < 8; q++) {
    e->cur[q] = e->arena + (size_t)off * q;
    e->spare[q] = e->arena + (size_t)off * (8 + q);
  }
  if (build_lists(e)) {
    mhd_ens_destroy(e);
    return nullptr;
  }
  return e;
}

void mhd_ens_destroy(mhd_ens_t* e) {
  if (!e) return;
  drop_graphs(e);
  free_lists(e);
  if (e->cap) cudaStreamDestroy(e->cap);
  cudaFree(e->arena);
  cudaFree(e->boxes_d);
  cudaFree(e->tau);
  cudaFree(e->rate[0]);
  cudaFree(e->time);
  cudaFree(e->diag_partial);
  cudaFree(e->diag_out);
  delete e;
}

int mhd_ens_set_stream(mhd_ens_t* e, void* cuda_stream) {
  if (!e) return mhd::set_error(MHD_E_ARG, "mhd_ens_set_stream", "null ensemble");
  e->stream = (cudaStream_t)cuda_stream;
  return MHD_OK;
}

int mhd_ens_set_state(mhd_ens_t* e, int b, const float* const f[8], int on_device) {
  if (bad(e, b) || !f) return mhd::set_error(MHD_E_ARG, "mhd_ens_set_state", "bad box index or null");
  for (int q = 0; q < 8; q++)
    if (!f[q]) return mhd::set_error(MHD_E_ARG, "mhd_ens_set_state", "null field pointer");
  if (e->layout) return mhd::set_error(MHD_E_ARG, "mhd_ens_set_state", "internal: exchanged layout");
  const mhd::EnsBox& x = e->boxes[b];
  const size_t bytes = sizeof(float) * (size_t)x.n[0] * x.n[1] * x.n[2];
  for (int q = 0; q < 8; q++)
    CKE(cudaMemcpyAsync(e->cur[q] + x.offset, f[q], bytes,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, e->stream));
  CKE(cudaMemsetAsync(e->rate[e->rcur] + b, 0, sizeof(unsigned), e->stream));
  CKE(cudaMemsetAsync(e->time + b, 0, sizeof(double), e->stream));
  const float* p[8];
  box_ptrs(e, b, p);
  CKE(mhd::launch_cfl_rate(p, plain_box(x), (float)e->gamma, e->rate[e->rcur] + b, e->stream));
  return MHD_OK;
}

int mhd_ens_get_state(const mhd_ens_t* e, int b, float* const f[8], int on_device) {
  if (bad(e, b) || !f) return mhd::set_error(MHD_E_ARG, "mhd_ens_get_state", "bad box index or null");
  for (int q = 0; q < 8; q++)
    if (!f[q]) return mhd::set_error(MHD_E_ARG, "mhd_ens_get_state", "null field pointer");
  if (e->layout) return mhd::set_error(MHD_E_ARG, "mhd_ens_get_state", "internal: exchanged layout");
  const mhd::EnsBox& x = e->boxes[b];
  const size_t bytes = sizeof(float) * (size_t)x.n[0] * x.n[1] * x.n[2];
  for (int q = 0; q < 8; q++)
    CKE(cudaMemcpyAsync(f[q], e->cur[q] + x.offset, bytes,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, e->stream));
  CKE(cudaStreamSynchronize(e->stream));
  return MHD_OK;
}

int mhd_ens_run(mhd_ens_t* e, int nsteps, double cfl) {
  if (!e || nsteps < 0 || !(cfl > 0.0)) return mhd::set_error(MHD_E_ARG, "mhd_ens_run", "bad arguments");
  if (nsteps == 0) return MHD_OK;
  return run_graph(e, nsteps, cfl);
}

int mhd_ens_times(const mhd_ens_t* e, double* t_out) {
  if (!e || !t_out) return mhd::set_error(MHD_E_ARG, "mhd_ens_times", "null argument");
  CKE(cudaMemcpyAsync(t_out, e->time, sizeof(double) * e->nbox, cudaMemcpyDeviceToHost, e->stream));
  CKE(cudaStreamSynchronize(e->stream));
  return MHD_OK;
}

int mhd_ens_cfl_dt(mhd_ens_t* e, double cfl, double* dt_out) {
  if (!e || !dt_out || !(cfl > 0.0)) return mhd::set_error(MHD_E_ARG, "mhd_ens_cfl_dt", "bad arguments");
  std::vector<unsigned> bits(e->nbox);
  CKE(cudaMemcpyAsync(bits.data(), e->rate[e->rcur], sizeof(unsigned) * e->nbox, cudaMemcpyDeviceToHost,
                      e->stream));
  CKE(cudaStreamSynchronize(e->stream));
  int rc = MHD_OK;
  for (int b = 0; b < e->nbox; b++) {
    float r;
    std::memcpy(&r, &bits[b], sizeof r);
    if (!(r > 0.f) || !std::isfinite(r)) {
      dt_out[b] = 0.0;
      rc = mhd::set_error(MHD_E_STATE, "mhd_ens_cfl_dt", "invalid state (NaN, rho <= 0 or p <= 0) in a box");
    } else {
      dt_out[b] = 2.0 * cfl / (double)r;
    }
  }
  return rc;
}

int mhd_ens_diagnostics(mhd_ens_t* e, double* out) {
  if (!e || !out) return mhd::set_error(MHD_E_ARG, "mhd_ens_diagnostics", "null argument");
  for (int b = 0; b < e->nbox; b++) {
    const float* p[8];
    box_ptrs(e, b, p);
    CKE(mhd::launch_diagnostics(p, plain_box(e->boxes[b]), e->gamma, e->diag_partial, e->diag_out, e->stream));
    CKE(cudaMemcpyAsync(out + 10 * b, e->diag_out, sizeof(double) * 10, cudaMemcpyDeviceToHost, e->stream));
  }
  CKE(cudaStreamSynchronize(e->stream));
  return MHD_OK;
}

int mhd_ens_set_pressure_floor(mhd_ens_t* e, double p_floor) {
  if (!e || !(p_floor >= 0.0)) return mhd::set_error(MHD_E_ARG, "mhd_ens_set_pressure_floor", "bad arguments");
  e->p_floor = (float)p_floor;
  drop_graphs(e);  // the floor is baked into captured launches
  return MHD_OK;
}

int mhd_ens_set_tuning(mhd_ens_t* e, int xpath, int segdiv) {
  if (!e || xpath < 1 || xpath > 2 || (segdiv != 1 && segdiv != 2 && segdiv != 4))
    return mhd::set_error(MHD_E_ARG, "mhd_ens_set_tuning", "xpath must be 1 or 2, segdiv 1, 2 or 4");
  if (e->layout) return mhd::set_error(MHD_E_ARG, "mhd_ens_set_tuning", "internal: exchanged layout");
  e->xpath = xpath;
  e->segdiv = segdiv;
  return build_lists(e);
}

int mhd_ens_autotune(mhd_ens_t* e, double cfl, int* xpath_out, int* segdiv_out) {
  if (!e || !(cfl > 0.0)) return mhd::set_error(MHD_E_ARG, "mhd_ens_autotune", "bad arguments");
  std::string sig;
  for (auto& b : e->boxes) sig += std::to_string(b.n[0]) + "x" + std::to_string(b.n[1]) + "x" + std::to_string(b.n[2]) + ";";
  {
    std::lock_guard<std::mutex> g(g_tune_lock);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      int rc = mhd_ens_set_tuning(e, it->second.first, it->second.second);
      if (xpath_out) *xpath_out = e->xpath;
      if (segdiv_out) *segdiv_out = e->segdiv;
      return rc;
    }
  }
  // time each candidate on a copy of the state, then restore it
  const size_t bytes = sizeof(float) * (size_t)e->ntot * 8;
  float* backup = nullptr;
  unsigned* rbackup = nullptr;
  double* tbackup = nullptr;
  CKE(cudaMalloc(&backup, bytes));
  CKE(cudaMalloc(&rbackup, sizeof(unsigned) * e->nbox * 2));
  CKE(cudaMalloc(&tbackup, sizeof(double) * e->nbox));
  float* save_cur[8];
  float* save_spare[8];
  std::memcpy(save_cur, e->cur, sizeof save_cur);
  std::memcpy(save_spare, e->spare, sizeof save_spare);
  const int save_rcur = e->rcur;
  for (int q = 0; q < 8; q++)
    CKE(cudaMemcpyAsync(backup + (size_t)e->ntot * q, e->cur[q], sizeof(float) * e->ntot,
                        cudaMemcpyDeviceToDevice, e->stream));
  CKE(cudaMemcpyAsync(rbackup, e->rate[0], sizeof(unsigned) * e->nbox * 2, cudaMemcpyDeviceToDevice, e->stream));
  CKE(cudaMemcpyAsync(tbackup, e->time, sizeof(double) * e->nbox, cudaMemcpyDeviceToDevice, e->stream));
  cudaEvent_t t0, t1;
  CKE(cudaEventCreate(&t0));
  CKE(cudaEventCreate(&t1));
  int best_x = 2, best_s = 1;
  float best = 1e30f;
  int rc = MHD_OK;
  for (int xp = 1; xp <= 2 && !rc; xp++) {
    for (int sd = 1; sd <= 2 && !rc; sd *= 2) {
      rc = mhd_ens_set_tuning(e, xp, sd);
      if (!rc) rc = mhd_ens_run(e, 1, cfl);  // capture + warm-up
      if (rc) break;
      cudaEventRecord(t0, e->stream);
      rc = mhd_ens_run(e, 2, cfl);
      cudaEventRecord(t1, e->stream);
      cudaEventSynchronize(t1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (!rc && ms < best) {
        best = ms;
        best_x = xp;
        best_s = sd;
      }
    }
  }
  // restore the state, the accumulators and the buffer assignment
  std::memcpy(e->cur, save_cur, sizeof save_cur);
  std::memcpy(e->spare, save_spare, sizeof save_spare);
  e->rcur = save_rcur;
  for (int q = 0; q < 8; q++)
    cudaMemcpyAsync(e->cur[q], backup + (size_t)e->ntot * q, sizeof(float) * e->ntot, cudaMemcpyDeviceToDevice,
                    e->stream);
  cudaMemcpyAsync(e->rate[0], rbackup, sizeof(unsigned) * e->nbox * 2, cudaMemcpyDeviceToDevice, e->stream);
  cudaMemcpyAsync(e->time, tbackup, sizeof(double) * e->nbox, cudaMemcpyDeviceToDevice, e->stream);
  cudaStreamSynchronize(e->stream);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(backup);
  cudaFree(rbackup);
  cudaFree(tbackup);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> g(g_tune_lock);
    g_tune_cache[sig] = {best_x, best_s};
  }
  rc = mhd_ens_set_tuning(e, best_x, best_s);
  if (xpath_out) *xpath_out = e->xpath;
  if (segdiv_out) *segdiv_out = e->segdiv;
  return rc;
}

}  // extern "C"
