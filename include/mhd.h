/*
 * mhd.h -- C ABI of the GB300 (sm_103a) dimensionally split ideal-MHD grid
 * update of Pang, Pen & Perrone, "Magnetohydrodynamics on Heterogeneous
 * architectures: a performance comparison".
 *
 * The problem (Section III, first paragraphs): evolve a periodic 3-D box of
 * nx*ny*nz zones of ideal MHD (Eq. 1-5) by one timestep, in single
 * precision, with no host<->device traffic inside the evolution.  One
 * timestep (Section II.B) is a CFL timestep choice followed by sweeps along
 * x, y, z and then z, y, x; every sweep is a relaxing-TVD fluid update
 * (Eq. 6, MUSCL + van Leer, 2-stage Runge-Kutta) and a constrained-transport
 * advection-constraint update of the face-centred magnetic field.
 *
 * Conventions shared by every call:
 *   - Domain: the periodic unit cube, cell size h_d = 1/n_d.
 *   - State: 8 single-precision fields, in this order:
 *       0 rho, 1 m_x, 2 m_y, 3 m_z, 4 e, 5 b_x, 6 b_y, 7 b_z.
 *     Each field is a contiguous array of nx*ny*nz floats, flat index
 *     i + nx*(j + ny*k) (x fastest).  b is in units with 4*pi absorbed
 *     (Section II.A); e = rho v^2/2 + p/(gamma-1) + b^2/2 (Eq. 3).
 *     b_d[i,j,k] is the mean normal field over the LOW face of cell (i,j,k)
 *     along d; the cell-centred field is the mean of the cell's two faces.
 *   - Ownership: every device buffer behind an mhd_t is allocated by
 *     mhd_create and freed by mhd_destroy.  Pointers passed in are borrowed
 *     for the duration of the call only.  No call allocates memory the
 *     caller must free.
 *   - Streams: all device work is ordered on the stream set with
 *     mhd_set_stream (default: the legacy default stream).  Calls that
 *     return host data (mhd_get_state, mhd_cfl_dt, mhd_time,
 *     mhd_diagnostics) synchronise that stream.
 *   - Errors: every int-returning call returns MHD_OK (0) or one of the
 *     codes below; mhd_last_error() then describes the failure (thread-local
 *     string, valid until the next failing call on the same thread).
 *   - Sizes: nx, ny, nz >= 1, nx a multiple of 4 (128-bit loads along x),
 *     and a single field must hold fewer than 2^31 cells.
 */
#ifndef MHD_GB300_H
#define MHD_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

#define MHD_OK 0
#define MHD_E_ARG 1     /* invalid argument: NULL, bad size, gamma <= 1, ...   */
#define MHD_E_CUDA 2    /* a CUDA runtime call failed                          */
#define MHD_E_OOM 3     /* device allocation failed                            */
#define MHD_E_STATE 4   /* NaN, rho <= 0 or p <= 0 found in the state          */
#define MHD_E_TIMEOUT 5 /* a bounded device-side wait gave up                  */

typedef struct mhd_s mhd_t;

/* Create a box of nx*ny*nz zones with adiabatic index gamma (> 1).
 * Allocates two copies of the 8-field state on the current CUDA device
 * (sweeps write out of place).  Returns NULL on failure (see mhd_last_error).
 * The state is zero until mhd_set_state. */
mhd_t *mhd_create(int nx, int ny, int nz, double gamma);

/* Free all device memory of the box.  NULL is ignored. */
void mhd_destroy(mhd_t *m);

/* Order all later work of this box on `cuda_stream` (a cudaStream_t, e.g.
 * torch.cuda.current_stream().cuda_stream).  NULL selects the default stream. */
int mhd_set_stream(mhd_t *m, void *cuda_stream);

/* Copy a state in.  f[q] points at field q (nx*ny*nz floats, layout above),
 * in device memory if on_device != 0, else in host memory (pinned memory
 * gives asynchronous copies).  Also recomputes the CFL rate of the new state
 * and sets the simulation time to 0. */
int mhd_set_state(mhd_t *m, const float *const f[8], int on_device);

/* Copy the current state out into caller-allocated buffers f[q] (device if
 * on_device != 0, else host).  Synchronises the stream. */
int mhd_get_state(const mhd_t *m, float *const f[8], int on_device);

/* Largest stable full timestep of the current state (Section II.B: the
 * fastest wave moves at most `cfl` cells per sweep):
 *   dt_full = 2 * cfl / max_cells max_d (|v_d| + c_f*) / h_d,
 *   c_f* = sqrt((gamma p + |b_c|^2) / rho).
 * Each of the 6 sweeps of a step uses dt_full/2.  Returns MHD_E_STATE if any
 * cell has NaN, rho <= 0 or p <= 0, and MHD_E_TIMEOUT if a TMA-staged sweep
 * since the last mhd_set_state gave up waiting for a chunk (see
 * mhd_set_tma).  Synchronises the stream. */
int mhd_cfl_dt(mhd_t *m, double cfl, double *dt_full);

/* One full timestep of length dt_full (Section II.B): fluid_x, mag_x,
 * fluid_y, mag_y, fluid_z, mag_z, then mag_z, fluid_z, mag_y, fluid_y,
 * mag_x, fluid_x, every sweep with step dt_full/2.  Asynchronous. */
int mhd_step(mhd_t *m, double dt_full);

/* nsteps full timesteps, each with its own CFL timestep computed on the
 * device from the state at the start of that step (no host round trip).
 * Asynchronous.  A step whose starting state is invalid (NaN, rho <= 0 or
 * p <= 0) gets dt = 0; mhd_cfl_dt afterwards reports MHD_E_STATE. */
int mhd_run(mhd_t *m, int nsteps, double cfl);

/* Pipelined host-to-host runs (the paper times the update alone and leaves
 * the host round trip out, Section III; a caller that streams states through
 * the GPU needs it).  mhd_submit enqueues: copy the host state `in` (8 field
 * pointers as in mhd_set_state) to the device, recompute its CFL rate and
 * reset the time (as mhd_set_state), run nsteps steps (as mhd_run), copy the
 * result to the host buffers `out`; it returns without waiting.  The copies
 * run on two copy streams of the box and overlap the steps of the neighbouring
 * submissions: the steps of submission k run while the input of k+1 and the
 * output of k-1 move (three staging copies of the state, allocated on first
 * use).  `in` must stay unchanged and `out` unread until mhd_drain; pinned
 * host memory is needed for the copies to be asynchronous.  Any other call on
 * the box is ordered after the submitted copies.  Returns MHD_E_ARG for NULL
 * pointers, nsteps < 0 or cfl <= 0. */
int mhd_submit(mhd_t *m, const float *const in[8], float *const out[8], int nsteps, double cfl);

/* Wait until every submitted run has its result in the host buffers. */
int mhd_drain(mhd_t *m);

/* Simulation time accumulated by mhd_step / mhd_run since mhd_set_state.
 * Synchronises the stream. */
int mhd_time(const mhd_t *m, double *t);

/* A single sweep along axis (0 = x, 1 = y, 2 = z) with step tau:
 * kind 0 = relaxing-TVD fluid update (b frozen), kind 1 = magnetic
 * advection-constraint update (Section II.B).  Asynchronous.  Used to test
 * the sweeps one by one. */
int mhd_sweep(mhd_t *m, int axis, int kind, double tau);

/* ---- FP64 boxes -----------------------------------------------------------
 * The same grid update computed in FP64 on the GPU (an ablation: the paper
 * computes in FP32, Section III): the scheme of Section II.B with every
 * operation an IEEE double operation rounded once.  FP64 arithmetic runs at
 * a small fraction of the FP32 rate on this GPU; these kernels favour
 * clarity (one thread per whole pencil, the magnetic edge fluxes through a
 * scratch array, the timestep through the host).  An FP64 box supports
 * mhd_set_stream, mhd_cfl_dt, mhd_step, mhd_run (one host synchronisation
 * per step), mhd_time, mhd_sweep, mhd_set_resolution and mhd_destroy, and
 * the paper's scheme only; the other calls return MHD_E_ARG.
 *
 * Create: periodic box, any nx, ny, nz >= 1 (at most 2^31 - 1 cells), gamma
 * > 1; allocates 18 N doubles (two state copies and the edge fluxes) on the
 * current device.  NULL on failure (mhd_last_error). */
mhd_t *mhd_create_f64(int nx, int ny, int nz, double gamma);

/* Copy the 8 FP64 fields in / out (layout of mhd_set_state; host or device
 * pointers, caller-owned).  set_state_f64 resets the time.  get_state_f64
 * synchronises.  MHD_E_ARG for a NULL pointer or a box that is not FP64. */
int mhd_set_state_f64(mhd_t *m, const double *const f[8], int on_device);
int mhd_get_state_f64(const mhd_t *m, double *const f[8], int on_device);

/* ---- Boxes that are part of a larger periodic domain ------------------
 * Section II.B evolves a periodic unit box (h_d = 1/n_d).  Sharding that box
 * across GPUs (the paper's future-work item: MPI across nodes, Section VI)
 * cuts it into slabs along z; each slab box holds its own planes plus halo
 * planes copied from its neighbours.  These calls let one mhd_t be such a
 * slab.  (Extensions: the paper has no counterpart.) */

/* Cells per unit length along x, y, z, i.e. 1/h_d of the sweeps (tau/h_d)
 * and of the CFL rate ((|v_d| + c_f*)/h_d).  0 (the default) means n_d, the
 * unit box.  A slab of a box of nz planes passes cz = nz so that its h_z is
 * the whole box's.  Recomputes the CFL rate.  MHD_E_ARG for a negative or
 * non-finite value. */
int mhd_set_resolution(mhd_t *m, double cx, double cy, double cz);

/* Cells [lo, hi) along axis (0..2) are the box's own; the others are halo
 * copies of cells that another box owns.  The CFL rate (mhd_cfl_dt, the
 * device-resident timestep of mhd_run) covers own cells only (and, on a
 * non-periodic axis, interior cells only), so that the largest rate over all
 * slabs is the whole box's.  Default: the whole box.  Recomputes the rate.
 * MHD_E_ARG unless 0 <= lo < hi <= n_axis. */
int mhd_set_interior(mhd_t *m, int axis, int lo, int hi);

/* Copy the z-planes z0 .. z0+nplanes-1 of all 8 fields between the box and
 * f[q] (nplanes*ny*nx floats each, layout as mhd_set_state): into_box = 1
 * writes the box, 0 reads it.  on_device: f[q] are device pointers (stream
 * ordered, asynchronous); otherwise host pointers (synchronises).  The CFL
 * rate is left as it was (halo planes are not own cells).  MHD_E_ARG for
 * planes outside the box or a NULL pointer. */
int mhd_copy_planes(mhd_t *m, int z0, int nplanes, float *const f[8], int into_box, int on_device);

/* Kernel fusion of the schedule (not a change of the method): with on = 1
 * (the default) the two magnetic z sweeps in the middle of a full step,
 * which follow each other with the same step tau = dt/2, run as one launch
 * that reads and writes the fields once (two advection pipelines per
 * transverse component, the second fed by the first; b_z takes both passes'
 * edge fluxes).  Every value is rounded as in two launches, so the state is
 * bitwise the same either way.  on = 0 runs the twelve sweeps of Section
 * II.B one launch each.  Boxes with non-periodic axes (ghost layers are
 * refilled between the two sweeps) and x path 3 always run them separately.
 * MHD_E_ARG unless on is 0 or 1. */
int mhd_set_fusion(mhd_t *m, int on);

/* Staging of the sweeps (not a change of the method): with on = 1 (the
 * default) the sweeps read their input through the Tensor Memory
 * Accelerator where the box qualifies.  Along the y and z kernel axes one
 * thread per block copies the next chunk of positions of the block's pencils
 * (and of the neighbouring pencils it needs) into shared memory while the
 * block computes the current one: fluid sweeps whose rows are a multiple of
 * 16 bytes, magnetic sweeps whose lane extent (the contiguous axis) is a
 * multiple of 32 and row extent a multiple of 8.  Along x (x path 1, see
 * mhd_set_xpath) whole x rows are copied into shared memory, each thread
 * computing 4 consecutive cells: fluid sweeps with nx a multiple of 128 up
 * to 1024, magnetic sweeps with nx a multiple of 128 up to 1024 and ny a
 * multiple of 4 (2 for nx above 512) (not with the per-pencil freezing
 * speed).  Every other scheme
 * variant of mhd_set_scheme is staged.  The values and their arithmetic are
 * those of the register-load sweeps, except that the staged fluid sweeps
 * take the freezing speeds' square roots from the hardware approximation (a
 * few ulp; the faster choice on each path), so the two paths agree to FP32
 * rounding, not bitwise (the magnetic sweeps bitwise); on = 0 always uses
 * register loads.  Ensembles, pencils shorter than 16 cells and boxes that do
 * not qualify use register loads.  If staged data does not arrive within the
 * bounded wait (about half a second), the block records the failure and
 * stops; mhd_cfl_dt then returns MHD_E_TIMEOUT until the next mhd_set_state.
 * MHD_E_ARG unless on is 0 or 1, or for an FP64 box. */
int mhd_set_tma(mhd_t *m, int on);

/* Number of sweeps (fluid and magnetic) this box has launched TMA-staged so
 * far.  MHD_E_ARG for NULL. */
int mhd_tma_sweeps(const mhd_t *m, long long *count);

/* Optional floor on the gas pressure (not in the paper; 0 = off, the
 * default).  The total-energy scheme leaves e untouched in the magnetic
 * sweeps, so in strongly magnetised, supersonic flow the magnetic energy can
 * outgrow the cell's thermal energy and p falls below zero.  With
 * p_floor > 0, each fluid sweep raises e after its update where needed so
 * that p >= p_floor (mass, momentum and b unchanged; energy is added only
 * where the floor acts). */
int mhd_set_pressure_floor(mhd_t *m, double p_floor);

/* Scheme variants, ablations of the paper's scheme (limiter 0 and freezing 0,
 * the default): limiter 1 = minmod, 2 = superbee instead of van Leer, in the
 * fluid and the magnetic sweeps; freezing 1 = |v_d| + the exact fast
 * magnetosonic speed along the sweep axis instead of the bound
 * |v_d| + sqrt((gamma p + |b|^2)/rho) (Section II.B leaves the freezing speed
 * open); freezing 2 = one speed per pencil and Runge-Kutta stage, the largest
 * bound along the pencil (for the second stage, over the first stage's
 * half-step state), computed by a reduction pass before each fluid sweep.
 * The CFL timestep keeps the bound.  One ablation at a time: MHD_E_ARG for
 * limiter and freezing both non-zero or out of range; MHD_E_OOM if the
 * per-pencil speeds cannot be allocated.  Ensembles always use the paper's
 * scheme. */
int mhd_set_scheme(mhd_t *m, int limiter, int freezing);

/* Boundaries (an extension: the paper's runs are periodic).  mode 0 =
 * periodic (the default), 1 = outflow, 2 = reflecting, for physical axis
 * `axis` (0 = x, 1 = y, 2 = z).  A non-periodic axis keeps 4 ghost cells at
 * each end inside the box (the caller includes them in n_axis, which must be
 * at least 12): interior cells 4 .. n-5, wall faces 4 (low) and n-4 (the low
 * face of the first high ghost cell).  Before every sweep and before every
 * CFL rate the library refills the ghost layers from the interior, axis by
 * axis in the order x, y, z:
 *   outflow:    a ghost cell copies the nearest interior cell; ghost faces of
 *               the normal field copy the wall face (zero gradient);
 *   reflecting: a ghost cell copies its mirror image in the wall with the
 *               normal momentum negated; ghost faces of the normal field copy
 *               their mirror faces, negated.
 * Tangential face fields follow the cell rule.  The sweeps themselves are the
 * periodic ones (a cell reads at most 3 cells along a sweep and 1 pencil
 * across, all inside the ghost layers); what they write into the ghost
 * layers is replaced by the next fill, so after a step the ghost layers hold
 * such values until mhd_fill_ghosts.  The CFL rate is taken over the whole
 * box after a fill (not fused into the last sweep).  Diagnostics sum the
 * whole box, ghost layers included.  Ensembles are always periodic.
 * MHD_E_ARG for a bad axis or mode or too short an axis. */
int mhd_set_boundary(mhd_t *m, int axis, int mode);

/* Refill the ghost layers of the non-periodic axes now (no-op without any):
 * after it the whole box, ghosts included, follows the boundary rules. */
int mhd_fill_ghosts(mhd_t *m);

/* Pencil segment lengths used by the sweeps along x, y and z.  A sweep splits
 * every pencil of n_d cells into n_d/seg_d pieces, each marched by its own
 * thread (more parallelism for small boxes, 8 cells of warm-up re-read per
 * piece).  Each seg_d must be a multiple of 4 that divides n_d; 0 restores
 * the automatic choice.  The arithmetic of every cell is the same for any
 * segmentation, so results are bitwise independent of it. */
int mhd_set_segments(mhd_t *m, int seg_x, int seg_y, int seg_z);

/* How x sweeps read the state: 1 = directly (over whole x rows staged in
 * shared memory where the row sweeps of mhd_set_tma qualify; otherwise a
 * warp stages 8-cell row pieces of its 32 pencils), 2 = through a copy with x
 * and y exchanged (all 8 fields transposed once before a group of x sweeps
 * and once after; consecutive steps share one group, so a run of steps costs
 * two transposes per step), 0 = automatic: 1 where both row sweeps qualify,
 * else 2 once the state exceeds 64 MiB, else 1.  3 = the paper's data flow,
 * as an ablation: every sweep runs along the contiguous axis of a copy
 * transposed so that its axis is fastest (x<->y around the y sweeps, x<->z
 * around the z sweeps; six transposes per step); needs every extent a
 * multiple of 4.  All paths compute the same update; results differ by FP32
 * rounding of sums taken in another order. */
int mhd_set_xpath(mhd_t *m, int mode);

/* FP64 diagnostics of the current state, computed on the device in one pass
 * and a fixed order, so repeated calls on the same state give bitwise
 * identical results.  The sums are compensated (FP32 words per lane, then
 * FP64 with Neumaier merges) to within a few 2^-48 of the absolute sum; the
 * extrema are the exact FP64 values of the formulas below:
 *   out[0..7] = sums over all cells of rho, m_x, m_y, m_z, e, b_x, b_y, b_z;
 *   out[8]    = max over cells of |div b| * h_min, div b the cell's discrete
 *               flux balance sum_d (b_d(high) - b_d(low)) / h_d,
 *               h_min = 1 / max(nx, ny, nz);
 *   out[9]    = min over cells of the gas pressure p.
 * `out` is host memory.  Synchronises the stream. */
int mhd_diagnostics(mhd_t *m, double out[10]);

/* Kernel classes reported by mhd_profile_read. */
#define MHD_K_FLUID_X 0
#define MHD_K_FLUID_Y 1
#define MHD_K_FLUID_Z 2
#define MHD_K_MAG_X 3
#define MHD_K_MAG_Y 4
#define MHD_K_MAG_Z 5
#define MHD_K_CONTROL 6 /* step control, CFL reduction, diagnostics */
#define MHD_K_TRANSPOSE 7 /* x <-> y exchange of the state (x sweep path 2) */
#define MHD_K_CLASSES 8

/* Per-kernel device timing (tracing).  With capacity > 0, every later kernel
 * launch of this box is bracketed by a pair of CUDA events on its stream,
 * for up to `capacity` launches (later launches are not timed); capacity 0
 * stops timing and drops the records.  Events are created here, not at
 * launch time. */
int mhd_profile(mhd_t *m, int capacity);

/* Launch counts and summed device milliseconds per kernel class since
 * mhd_profile (arrays of MHD_K_CLASSES entries, host memory).  Synchronises
 * the stream.  Records are kept, so repeated reads give the same totals. */
int mhd_profile_read(mhd_t *m, int counts[], double ms[]);

/* FP64 diagnostics of caller-owned fields, for callers that cannot allocate
 * device memory (no counterpart in the paper).  Same numbers as
 * mhd_diagnostics, computed by the same kernels, but without an mhd_t and
 * without any allocation: code that runs where a framework's caching
 * allocator owns all device memory, in a latency-critical loop where a
 * cudaMalloc (which can synchronise the device) is not allowed, or in a
 * plug-in with no allocation rights, can still take the conservation sums.
 *   nx, ny, nz, gamma: box and adiabatic index (gamma > 1), at most
 *     2^31 - 1 cells; larger boxes are rejected with MHD_E_ARG.
 *   f[q]: device pointers to the 8 fields, layout as above (read only).
 *   out: host array of 10 doubles (layout of mhd_diagnostics).
 *   cuda_stream: the stream to run on (NULL = default); synchronised before
 *     return.
 * Scratch: a fixed 194 KiB array in the library's device memory, held by
 * every GPU that loads the library until the process exits.  Its device
 * address is looked up in the current context on every call; the first call
 * in a context also loads the library's device code there, so make it
 * before capturing a stream that will contain it.  All calls share the
 * array: calls that overlap on the GPU (different streams, threads or
 * processes sharing a context) race and must be serialised by the caller. */
int mhd_diagnostics_static(int nx, int ny, int nz, double gamma, const float *const f[8],
                           double out[10], void *cuda_stream);

/* ---- Ensembles of independent boxes -------------------------------------
 * Many periodic boxes of uneven sizes advanced together: every sweep of the
 * Section II.B schedule is one launch over all boxes, each box keeps its own
 * CFL timestep and time, and a run of steps is one CUDA graph launch.  (The
 * paper evolves one box; ensembles are an extension.)  Box b has the layout
 * and conventions of a single box with dims3[3b..3b+2] = (nx, ny, nz). */
typedef struct mhd_ens_s mhd_ens_t;

/* Create nbox boxes (nx >= 4, nx % 4 == 0, ny, nz >= 1; at most 2^31 - 1
 * cells in all boxes together).  Allocates two copies of every box's state
 * on the current device.  NULL on failure. */
mhd_ens_t *mhd_ens_create(int nbox, const int *dims3, double gamma);
void mhd_ens_destroy(mhd_ens_t *e);
int mhd_ens_set_stream(mhd_ens_t *e, void *cuda_stream);

/* Copy box b's state in / out (layout of mhd_set_state / mhd_get_state).
 * set_state resets that box's time and recomputes its CFL rate. */
int mhd_ens_set_state(mhd_ens_t *e, int box, const float *const f[8], int on_device);
int mhd_ens_get_state(const mhd_ens_t *e, int box, float *const f[8], int on_device);

/* nsteps full steps of every box, each box with its own CFL timestep computed
 * on the device.  The launches of the whole run are captured into a CUDA
 * graph on first use (cached per step count, cfl and buffer assignment) and
 * replayed.  Asynchronous. */
int mhd_ens_run(mhd_ens_t *e, int nsteps, double cfl);

/* Per-box simulation times (nbox doubles, host).  Synchronises. */
int mhd_ens_times(const mhd_ens_t *e, double *t_out);

/* Per-box full CFL timestep of the current states (nbox doubles, host);
 * MHD_E_STATE if any box is invalid (its entry is 0).  Synchronises. */
int mhd_ens_cfl_dt(mhd_ens_t *e, double cfl, double *dt_out);

/* Per-box FP64 diagnostics (nbox x 10 doubles, host, layout of
 * mhd_diagnostics).  Synchronises. */
int mhd_ens_diagnostics(mhd_ens_t *e, double *out);

/* Pressure floor for every box (see mhd_set_pressure_floor). */
int mhd_ens_set_pressure_floor(mhd_ens_t *e, double p_floor);

/* Tiling of the ensemble launches: x path (1 direct, 2 exchanged layout; see
 * mhd_set_xpath) and pencil segment divisor (1, 2 or 4: each pencil of a box
 * is marched by that many threads when its length allows). */
int mhd_ens_set_tuning(mhd_ens_t *e, int xpath, int segdiv);

/* Pick the fastest tiling by timing two steps of each candidate on a copy of
 * the current states (restored afterwards); the choice is cached per set of
 * box sizes for the process.  Writes the choice if the pointers are not NULL. */
int mhd_ens_autotune(mhd_ens_t *e, double cfl, int *xpath_out, int *segdiv_out);

/* ---- Kernels of the learned coarse-grid correction ----------------------
 * (Not in the paper: a 3-D CNN that corrects a coarse step toward a
 * restricted fine solution.)  Activations are channels-last BF16
 * [cell][channel], cell = i + nx*(j + ny*k); channel counts are 8 or 32.
 * mhd_conv3d needs nx % 8 == 0 and ny % 16 == 0 (tiles of 8 x 16 x 1
 * cells), mhd_conv3d_wgrad a multiple of 64 cells.  All pointers are device
 * memory, all calls asynchronous on `stream`, no call allocates.
 *
 * Weights w[cout][cin][3][3][3] (FP32, cross-correlation: output cell
 * (i,j,k) sees input (i+kx-1, j+ky-1, k+kz-1), periodic) are packed into a
 * BF16 tensor-core image of mhd_conv_pack_bytes() bytes (the three z taps
 * side by side along the GEMM's N); transpose = 1 packs the image used for
 * the input gradient, with the channels exchanged and the taps already
 * mirrored. */
size_t mhd_conv_pack_bytes(int cin, int cout, int transpose);
int mhd_conv_pack(const float *w, int cin, int cout, int transpose, void *img, void *stream);

/* y[cell][co] = sum_{ci, taps} x[cell + s*offset][ci] * W + bias[co]
 * (s = +1, or -1 with flip = 1), accumulated in FP32 on the tensor cores
 * (tcgen05); optional ReLU; where mask != NULL, outputs with
 * mask[cell][co] <= 0 are zeroed (backward through a ReLU); written as BF16
 * (y_bf16) and/or FP32 (y_f32).  The input gradient of a layer with cin_f,
 * cout_f is mhd_conv3d(cin = cout_f, cout = cin_f, img = transposed pack,
 * flip = 1): the mirrored taps come with the transposed pack, so flip = 1
 * goes with a transposed pack and flip = 0 with a forward one.  img_bytes
 * must equal the size of the image for these channel counts (MHD_E_ARG
 * otherwise). */
int mhd_conv3d(int nx, int ny, int nz, int cin, int cout, const void *x, const void *img,
               size_t img_bytes, const float *bias, int relu, int flip, const void *mask, void *y_bf16,
               float *y_f32, void *stream);

/* Weight gradient: gw[co][ci][tap] += sum_cell gy[cell][co] x[cell + offset][ci],
 * gb[co] += sum_cell gy[cell][co] (FP32 atomics: the caller zeroes them; gb
 * may be NULL).  With nx % 8 == 0, ny % 16 == 0 and x, gy 16-byte aligned the
 * sum over cells runs on the tensor cores (tcgen05, FP32 accumulation; a
 * bounded wait that gives up sets the flag mhd_conv_error reads); otherwise
 * on the CUDA cores. */
int mhd_conv3d_wgrad(int nx, int ny, int nz, int cin, int cout, const void *x, const void *gy,
                     float *gw, float *gb, void *stream);

/* Restriction of a fine state (nx, ny, nz) to the grid coarser by r along
 * every axis: cell quantities are r^3 block means, b_d the mean of the r^2
 * fine faces tiling each coarse face (flux preserving: a divergence-free
 * fine field restricts to a divergence-free coarse field). */
int mhd_restrict(int nx, int ny, int nz, int r, const float *const fine[8], float *const coarse[8],
                 void *stream);

/* Network input: x[cell][q] = BF16((s_q[cell] - mu[q]) * inv_sigma[q]). */
int mhd_cnn_normalize(int nx, int ny, int nz, const float *const s[8], const float mu[8],
                      const float inv_sigma[8], void *x_bf16, void *stream);

/* Network output y[cell][8] (FP32) -> correction d (8 SoA fields):
 * d_q = scale[q] y_q for q < 5 with the box mean removed (conservation), and
 * d_b = discrete curl of the edge potential A = scale[5] (y_5, y_6, y_7)
 * (A_x on x-edges (i, j-1/2, k-1/2), A_y on (i-1/2, j, k-1/2), A_z on
 * (i-1/2, j-1/2, k)), so div d_b = 0 up to rounding.  `sums` is 5 doubles
 * of device scratch. */
int mhd_cnn_project(int nx, int ny, int nz, const float *y, const float scale[6], float *const d[8],
                    double *sums, void *stream);

/* loss (device double) = sum_q weight[q] sum_cells (d_q - t_q)^2 and, if g
 * is not NULL, g_q = 2 weight[q] (d_q - t_q). */
int mhd_cnn_loss(int nx, int ny, int nz, const float *const d[8], const float *const t[8],
                 const float weight[8], double *loss, float *const g[8], void *stream);

/* Adjoint of mhd_cnn_project: the gradient with respect to y (BF16
 * channels-last) of a loss whose gradient with respect to d is g. */
int mhd_cnn_project_backward(int nx, int ny, int nz, const float *const g[8], const float scale[6],
                             double *sums, void *gy_bf16, void *stream);

/* Apply a correction d to a state s in place, keeping it physical: b += d_b
 * (divergence-free, never scaled); the density correction is clipped at
 * -rho/2; the cell correction (rho, m, e) is scaled by the largest of 1,
 * 1/2, 1/4, 0 that keeps the thermal energy above half its uncorrected value,
 * and if none does e is raised to that bound.  scratch: nx*ny*nz floats;
 * nclip (device int, may be NULL) counts the cells where a limit acted. */
int mhd_correct(int nx, int ny, int nz, float *const s[8], const float *const d[8], float *scratch,
                int *nclip, void *stream);

/* Adam step on `count` FP32 parameters (step counts from 1). */
int mhd_adam(float *p, const float *g, float *m, float *v, int count, float lr, float beta1, float beta2,
             float eps, int step, void *stream);

/* The whole correction network: 4 periodic 3x3x3 layers 8 -> 32 -> 32 ->
 * 32 -> 8 with ReLU after the first three (mhd_conv3d per layer).  x: input
 * [cell][8] BF16 (normalised); img[l]: forward weight images of layer l
 * (mhd_conv_pack, transpose 0) of img_bytes[l] bytes; bias[l]: [cout_l] FP32
 * or NULL; acts[0..2]: caller-owned BF16 [cell][32] buffers that receive the
 * three hidden activations (the backward reads them); y: FP32 [cell][8].
 * Same box requirements as mhd_conv3d. */
int mhd_cnn_forward(int nx, int ny, int nz, const void *x, const void *const img[4], const size_t img_bytes[4],
                    const float *const bias[4], void *const acts[3], float *y, void *stream);

/* Backward of mhd_cnn_forward for the output gradient gy ([cell][8] BF16):
 * layer by layer from the last, the weight and bias gradient
 * (mhd_conv3d_wgrad, accumulated into gw[l] = [cout_l][cin_l][27] and
 * gb[l] = [cout_l] FP32: the caller zeroes them) and, below the top layer,
 * the input gradient through the ReLU mask of the saved activation
 * (mhd_conv3d with the transposed images imgT[l], flip = 1) into two
 * caller-owned BF16 [cell][32] scratch buffers. */
int mhd_cnn_backward(int nx, int ny, int nz, const void *x, const void *const acts[3], const void *gy,
                     const void *const imgT[4], const size_t imgT_bytes[4], float *const gw[4], float *const gb[4],
                     void *const scratch[2], void *stream);

/* Read and clear the flag raised by a convolution whose bounded tensor-core
 * wait gave up (MHD_E_TIMEOUT if set).  Synchronises the device. */
int mhd_conv_error(int *flag);

/* Description of the last failure on this thread ("" if none). */
const char *mhd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MHD_GB300_H */
