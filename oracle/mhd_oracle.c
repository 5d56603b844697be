/*
 * FP64 CPU oracle for the dimensionally split ideal-MHD grid update of
 * "Magnetohydrodynamics on Heterogeneous architectures: a performance
 * comparison" (Pang, Pen & Perrone), Section II.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes (restated from the equations, not from any code):
 *   - state: cell-centred conserved U = (rho, m_x, m_y, m_z, e) and a
 *     face-centred magnetic field b_x, b_y, b_z (constrained transport,
 *     Section II.B); b is in units where the 4*pi is absorbed (Section II.A),
 *     e = rho v^2/2 + p/(gamma-1) + b^2/2 and P* = p + b^2/2 (Eq. 1-3).
 *   - a fluid sweep along axis d: the 1-D conservation law du/dt + dF/dx = 0
 *     (Eq. 6) with the flux of Eq. 2-3 projected on d, discretised by a
 *     relaxing TVD scheme: per-cell freezing speed c, right/left movers
 *     F^R = (cU+F)/2, F^L = (cU-F)/2, a first-order upwind half step and a
 *     full step with van Leer limited second-order fluxes (2-stage
 *     Runge-Kutta), Section II.B.  b is held fixed during the sweep.
 *   - a magnetic sweep along d: for each transverse axis t, the component b_t
 *     is advected along d by the same upwind + van Leer, 2-stage scheme, and
 *     the edge flux it produces is applied to b_d so that div b is unchanged
 *     (advection-constraint step of Section II.B, Eq. 4-5).
 *   - the timestep: CFL rate, then sweeps x, y, z followed by z, y, x.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - freezing speed per cell c = |v_d| + sqrt((gamma p + |b_c|^2)/rho),
 *     recomputed from each Runge-Kutta stage's state;
 *   - cell-centred b_c is the mean of the two faces of the cell;
 *   - b_d[i] sits on the low face of cell i along d;
 *   - advection velocity of b_t: v_d averaged to the b_t face (cells j, j-1
 *     along t), then to the edge (cells i, i+1 along d);
 *   - second-order magnetic flux: ubar * (q_up + s * phi(dq-, dq+) / 2), with
 *     s = +1 for ubar >= 0 (upwind cell i) and -1 otherwise (upwind cell i+1);
 *   - schedule: forward half [fluid_d, magnetic_d] for d = x, y, z, reverse
 *     half [magnetic_d, fluid_d] for d = z, y, x, every sweep with tau = dt/2;
 *   - CFL: dt = 2 * cfl / max_cells max_d (|v_d| + c_f*) / h_d;
 *   - domain is the periodic unit cube, h_d = 1 / n_d (non-periodic axes: see
 *     the boundaries below); orc_set_resolution gives another number of
 *     cells per unit length along an axis (a box that is part of a larger
 *     periodic domain, such as a slab of it).
 *
 * Layout: 8 arrays (rho, m_x, m_y, m_z, e, b_x, b_y, b_z), each nx*ny*nz
 * doubles, flat index i + nx*(j + ny*k).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BX = 5, BY = 6, BZ = 7 };

/* Optional pressure floor (0 = off, the paper's scheme).  When positive, the
 * fluid sweep raises e after its update wherever the gas pressure would fall
 * below p_floor: e = max(e, |m|^2/(2 rho) + |b_c|^2/2 + p_floor/(gamma-1)).
 * Mass and momentum are untouched; energy is added only where the floor acts.
 * Not in the paper: an extension for strongly magnetised, supersonic runs in
 * which the total-energy scheme drives p negative. */
static double g_pfloor = 0.0;
void orc_set_pressure_floor(double p_floor) { g_pfloor = p_floor > 0.0 ? p_floor : 0.0; }

/* Cells per unit length along each axis, 1 / h_d (0 = the box's own cell
 * count n_d: the periodic unit cube).  A slab of nz_s planes cut from a
 * periodic unit box of nz planes keeps h_z = 1 / nz by giving nz here. */
static double g_cpl[3] = {0.0, 0.0, 0.0};
void orc_set_resolution(double cx, double cy, double cz) {
    g_cpl[0] = cx > 0.0 ? cx : 0.0;
    g_cpl[1] = cy > 0.0 ? cy : 0.0;
    g_cpl[2] = cz > 0.0 ? cz : 0.0;
}
static double cells_per_length(const int n[3], int d) { return g_cpl[d] > 0.0 ? g_cpl[d] : (double)n[d]; }

/* Boundaries (an extension: the paper's runs are periodic).  An axis is
 * periodic (0, the default), outflow (1) or reflecting (2).  A non-periodic
 * axis of n cells keeps GHOST = 4 ghost cells at each end inside the box:
 * interior cells GHOST .. n-GHOST-1, wall faces GHOST (low) and n-GHOST (the
 * low face of the first high ghost cell).  Before every sweep and before the
 * CFL rate the ghost layers are refilled from the interior, axis by axis in
 * the order x, y, z over the whole extent of the other two axes:
 *   outflow:    a ghost cell copies the nearest interior cell; ghost faces of
 *               the normal field copy the wall face (zero gradient);
 *   reflecting: a ghost cell copies its mirror image in the wall with the
 *               normal momentum negated; ghost faces of the normal field copy
 *               their mirror faces, negated.
 * The tangential face fields are cell-like along the axis and follow the
 * cell rule.  The sweeps are then the periodic ones: a cell reads at most 3
 * cells along the sweep and 1 pencil across, all inside the ghost layers,
 * and whatever the sweep writes into the ghost layers is replaced by the next
 * fill.  The CFL rate takes the interior cells only.  A non-periodic axis
 * needs n >= 3 GHOST (the sweeps of a shorter
 * one leave its ghost layers as they are; the Python wrappers refuse it). */
enum { GHOST = 4 };
static int g_bc[3] = {0, 0, 0};
int orc_set_boundary(int axis, int mode) {
    if (axis < 0 || axis > 2 || mode < 0 || mode > 2) return 1;
    g_bc[axis] = mode;
    return 0;
}
int orc_boundary(int axis) { return (axis < 0 || axis > 2) ? -1 : g_bc[axis]; }
static int any_boundary(void) { return g_bc[0] || g_bc[1] || g_bc[2]; }

/* Returns 1 (and writes nothing) if a non-periodic axis is shorter than
 * 3 GHOST cells. */
int orc_fill_ghosts(const int n[3], double *f[8]) {
    int d;
    for (d = 0; d < 3; d++)
        if (g_bc[d] && n[d] < 3 * GHOST) return 1;
    for (d = 0; d < 3; d++) {
        const int mode = g_bc[d], t1 = (d + 1) % 3, t2 = (d + 2) % 3, nd = n[d];
        const int wlo = GHOST, whi = nd - GHOST;  /* wall faces */
        long sd, st1, st2;
        int a1, a2;
        if (!mode) continue;
        sd = d == 0 ? 1 : (d == 1 ? n[0] : (long)n[0] * n[1]);
        st1 = t1 == 0 ? 1 : (t1 == 1 ? n[0] : (long)n[0] * n[1]);
        st2 = t2 == 0 ? 1 : (t2 == 1 ? n[0] : (long)n[0] * n[1]);
        for (a2 = 0; a2 < n[t2]; a2++) {
            for (a1 = 0; a1 < n[t1]; a1++) {
                const long base = a1 * st1 + a2 * st2;
                int k, q;
                for (k = 0; k < GHOST; k++) {
                    /* cells: low ghost k, high ghost nd-1-k */
                    const int lo = k, hi = nd - 1 - k;
                    const int slo = mode == 1 ? wlo : 2 * wlo - 1 - lo;
                    const int shi = mode == 1 ? whi - 1 : 2 * whi - 1 - hi;
                    for (q = 0; q < 8; q++) {
                        double sign = 1.0;
                        if (q == BX + d) continue;
                        if (mode == 2 && q == MX + d) sign = -1.0;
                        f[q][base + lo * sd] = sign * f[q][base + slo * sd];
                        f[q][base + hi * sd] = sign * f[q][base + shi * sd];
                    }
                    /* normal face field: low ghost faces 0..GHOST-1, high
                     * ghost faces whi+1 .. nd-1 (the wall faces stay) */
                    f[BX + d][base + lo * sd] =
                        mode == 1 ? f[BX + d][base + wlo * sd] : -f[BX + d][base + (2 * wlo - lo) * sd];
                    if (hi > whi)
                        f[BX + d][base + hi * sd] =
                            mode == 1 ? f[BX + d][base + whi * sd] : -f[BX + d][base + (2 * whi - hi) * sd];
                }
            }
        }
    }
    return 0;
}

/* periodic wrap of an index */
static int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* flat index of cell c[0..2], wrapped periodically */
static long at(const int n[3], const int c[3]) {
    return (long)wrap(c[0], n[0]) +
           (long)n[0] * ((long)wrap(c[1], n[1]) + (long)n[1] * (long)wrap(c[2], n[2]));
}

/* Scheme variants, ablations of the paper's scheme (which is limiter 0,
 * freezing 0):
 *   limiter 0 = van Leer (Section II.B), 1 = minmod, 2 = superbee
 *     (the two limiters that bound the second-order TVD region of Sweby's
 *     diagram from below and from above);
 *   freezing 0 = the bound |v_d| + sqrt((gamma p + |b_c|^2)/rho),
 *   freezing 1 = |v_d| + the fast magnetosonic speed along d,
 *     c_f^2 = (s + sqrt(s^2 - 4 a^2 v_Ad^2)) / 2, s = a^2 + v_A^2,
 *     a^2 = gamma p / rho, v_A^2 = |b_c|^2 / rho, v_Ad^2 = b_d^2 / rho
 *     (the smallest freezing speed the relaxation scheme allows).
 *   freezing 2 = the largest bound along the pencil, one value per pencil
 *     and Runge-Kutta stage (the first stage's from U, the second's from
 *     the half-step state), the classical global choice of relaxing TVD
 *     schemes applied pencil by pencil.
 * The CFL rate keeps the bound in every variant. */
static int g_limiter = 0, g_freezing = 0;
int orc_set_scheme(int limiter, int freezing) {
    if (limiter < 0 || limiter > 2 || freezing < 0 || freezing > 2) return 1;
    g_limiter = limiter;
    g_freezing = freezing;
    return 0;
}

/* Slope limiter phi(a, b) of two neighbouring differences: 0 unless they
 * have the same sign; van Leer 2ab/(a+b) (Section II.B); minmod, the one of
 * smaller magnitude; superbee, sign(a) max(min(2|a|,|b|), min(|a|,2|b|)). */
double orc_limiter(double a, double b) {
    if (!(a * b > 0.0)) return 0.0;
    if (g_limiter == 1) return fabs(a) < fabs(b) ? a : b;
    if (g_limiter == 2) {
        double A = fabs(a), B = fabs(b);
        double m = fmax(fmin(2.0 * A, B), fmin(A, 2.0 * B));
        return a > 0.0 ? m : -m;
    }
    return 2.0 * a * b / (a + b);
}


/*
 * Flux of Eq. 2-3 projected on the sweep axis, in the sweep's local frame
 * (component 0 = along d, 1 and 2 = the two transverse axes), and the
 * freezing speed c of the relaxation scheme.
 *   u = (rho, m_d, m_t1, m_t2, e), b = cell-centred (b_d, b_t1, b_t2).
 */
static void flux_and_speed(const double u[5], const double b[3], double gamma,
                           double F[5], double *c) {
    double rho = u[0];
    double vd = u[1] / rho, v1 = u[2] / rho, v2 = u[3] / rho;
    double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    double kinetic = 0.5 * (u[1] * vd + u[2] * v1 + u[3] * v2);
    double p = (gamma - 1.0) * (u[4] - kinetic - 0.5 * b2);
    double pstar = p + 0.5 * b2;
    double bv = b[0] * vd + b[1] * v1 + b[2] * v2;
    F[0] = u[1];
    F[1] = u[1] * vd + pstar - b[0] * b[0];
    F[2] = u[2] * vd - b[0] * b[1];
    F[3] = u[3] * vd - b[0] * b[2];
    F[4] = (u[4] + pstar) * vd - b[0] * bv;
    if (g_freezing == 1) {
        double a2 = gamma * p / rho, va2 = b2 / rho, vad2 = b[0] * b[0] / rho;
        double sum = a2 + va2, disc = sum * sum - 4.0 * a2 * vad2;
        *c = fabs(vd) + sqrt(0.5 * (sum + sqrt(disc > 0.0 ? disc : 0.0)));
    } else {
        *c = fabs(vd) + sqrt((gamma * p + b2) / rho);
    }
}

/* The freezing speed of one cell state (u, b in the sweep's local frame),
 * for the tests. */
double orc_freezing_speed(const double u[5], const double b[3], double gamma) {
    double F[5], c;
    flux_and_speed(u, b, gamma, F, &c);
    return c;
}

/*
 * One relaxing-TVD fluid update of a periodic pencil of n cells with step tau
 * and spacing h (Section II.B).  U[q][i] is updated in place; B[q][i] is the
 * frozen cell-centred field.  w is workspace of at least 25*n doubles.
 */
/* freezing 2: every cell of the pencil takes the pencil's largest speed */
static void pencil_max_speed(double *cs, int n) {
    double m = 0.0;
    int i;
    if (g_freezing != 2) return;
    for (i = 0; i < n; i++)
        if (cs[i] > m) m = cs[i];
    for (i = 0; i < n; i++) cs[i] = m;
}

static void fluid_pencil(int n, double h, double tau, double gamma,
                         double *U[5], double *B[3], double *w) {
    double *FR = w;            /* 5*n : right movers of the current stage */
    double *FL = w + 5 * n;    /* 5*n : left movers */
    double *Uh = w + 10 * n;   /* 5*n : half-step state */
    double *fl = w + 15 * n;   /* 5*n : interface flux, fl[q*n+i] at i+1/2 */
    double *cs = w + 20 * n;   /* n   : freezing speed */
    double u[5], b[3], F[5];
    int i, q;

    /* stage 1: first-order upwind fluxes from U, half step tau/2 (FR holds
     * F until the freezing speeds are known) */
    for (i = 0; i < n; i++) {
        for (q = 0; q < 5; q++) u[q] = U[q][i];
        for (q = 0; q < 3; q++) b[q] = B[q][i];
        flux_and_speed(u, b, gamma, F, &cs[i]);
        for (q = 0; q < 5; q++) FR[q * n + i] = F[q];
    }
    pencil_max_speed(cs, n);
    for (i = 0; i < n; i++)
        for (q = 0; q < 5; q++) {
            const double Fq = FR[q * n + i];
            FR[q * n + i] = 0.5 * (cs[i] * U[q][i] + Fq);
            FL[q * n + i] = 0.5 * (cs[i] * U[q][i] - Fq);
        }
    for (q = 0; q < 5; q++)
        for (i = 0; i < n; i++)
            fl[q * n + i] = FR[q * n + i] - FL[q * n + wrap(i + 1, n)];
    for (q = 0; q < 5; q++)
        for (i = 0; i < n; i++)
            Uh[q * n + i] = U[q][i] - (tau / (2.0 * h)) *
                                          (fl[q * n + i] - fl[q * n + wrap(i - 1, n)]);

    /* stage 2: van Leer limited second-order fluxes from the half-step state */
    for (i = 0; i < n; i++) {
        for (q = 0; q < 5; q++) u[q] = Uh[q * n + i];
        for (q = 0; q < 3; q++) b[q] = B[q][i];
        flux_and_speed(u, b, gamma, F, &cs[i]);
        for (q = 0; q < 5; q++) FR[q * n + i] = F[q];
    }
    pencil_max_speed(cs, n);
    for (i = 0; i < n; i++)
        for (q = 0; q < 5; q++) {
            const double Fq = FR[q * n + i];
            FR[q * n + i] = 0.5 * (cs[i] * Uh[q * n + i] + Fq);
            FL[q * n + i] = 0.5 * (cs[i] * Uh[q * n + i] - Fq);
        }
    for (q = 0; q < 5; q++) {
        const double *R = FR + q * n, *L = FL + q * n;
        for (i = 0; i < n; i++) {
            int im = wrap(i - 1, n), ip = wrap(i + 1, n), ipp = wrap(i + 2, n);
            double right = R[i] + 0.5 * orc_limiter(R[i] - R[im], R[ip] - R[i]);
            double left = L[ip] - 0.5 * orc_limiter(L[ip] - L[i], L[ipp] - L[ip]);
            fl[q * n + i] = right - left;
        }
    }
    for (q = 0; q < 5; q++)
        for (i = 0; i < n; i++)
            U[q][i] = U[q][i] - (tau / h) * (fl[q * n + i] - fl[q * n + wrap(i - 1, n)]);
    if (g_pfloor > 0.0) {
        for (i = 0; i < n; i++) {
            double kin = 0.5 * (U[1][i] * U[1][i] + U[2][i] * U[2][i] + U[3][i] * U[3][i]) / U[0][i];
            double mag = 0.5 * (B[0][i] * B[0][i] + B[1][i] * B[1][i] + B[2][i] * B[2][i]);
            double emin = kin + mag + g_pfloor / (gamma - 1.0);
            if (U[4][i] < emin) U[4][i] = emin;
        }
    }
}

/*
 * Edge flux of the advected transverse field along a periodic pencil
 * (Section II.B, magnetic part).  q[i] is b_t on the pencil, ub[i] the
 * advection velocity at edge i+1/2.  Output f[i] at edge i+1/2.
 * w is workspace of at least 2*n doubles.
 */
static void advect_flux(int n, double h, double tau, const double *q,
                        const double *ub, double *f, double *w) {
    double *g = w, *qh = w + n;
    int i;
    /* stage 1: upwind flux, half step */
    for (i = 0; i < n; i++)
        g[i] = ub[i] * (ub[i] >= 0.0 ? q[i] : q[wrap(i + 1, n)]);
    for (i = 0; i < n; i++)
        qh[i] = q[i] - (tau / (2.0 * h)) * (g[i] - g[wrap(i - 1, n)]);
    /* stage 2: upwind value plus half the limited slope of the upwind cell */
    for (i = 0; i < n; i++) {
        int im = wrap(i - 1, n), ip = wrap(i + 1, n), ipp = wrap(i + 2, n);
        if (ub[i] >= 0.0)
            f[i] = ub[i] * (qh[i] + 0.5 * orc_limiter(qh[i] - qh[im], qh[ip] - qh[i]));
        else
            f[i] = ub[i] * (qh[ip] - 0.5 * orc_limiter(qh[ip] - qh[i], qh[ipp] - qh[ip]));
    }
}

/* ------------------------------------------------------------------------ */

/* transverse axes of a sweep along d: cyclic (d+1, d+2) */
static int t1_of(int d) { return (d + 1) % 3; }
static int t2_of(int d) { return (d + 2) % 3; }

/*
 * Fluid sweep along axis d with step tau: every pencil along d independently
 * (the magnetic field is frozen; it only enters through b_c).
 */
void orc_fluid_sweep(const int n[3], double gamma, double *f[8], int d, double tau) {
    if (any_boundary()) orc_fill_ghosts(n, f);
    int t1 = t1_of(d), t2 = t2_of(d);
    int nd = n[d];
    double h = 1.0 / cells_per_length(n, d);
    int np = n[t1] * n[t2];
    int p;
#pragma omp parallel for schedule(static)
    for (p = 0; p < np; p++) {
        double *buf = (double *)malloc(sizeof(double) * (size_t)nd * (5 + 3 + 25));
        double *U[5], *B[3];
        int q, s, c[3], cn[3];
        long id;
        for (q = 0; q < 5; q++) U[q] = buf + q * nd;
        for (q = 0; q < 3; q++) B[q] = buf + (5 + q) * nd;
        c[t1] = p % n[t1];
        c[t2] = p / n[t1];
        for (s = 0; s < nd; s++) {
            c[d] = s;
            id = at(n, c);
            U[0][s] = f[RHO][id];
            U[1][s] = f[MX + d][id];
            U[2][s] = f[MX + t1][id];
            U[3][s] = f[MX + t2][id];
            U[4][s] = f[EN][id];
            /* cell-centred field: mean of the low and high faces (axis a) */
            {
                int ax[3] = {d, t1, t2}, a;
                for (a = 0; a < 3; a++) {
                    memcpy(cn, c, sizeof cn);
                    cn[ax[a]] += 1;
                    B[a][s] = 0.5 * (f[BX + ax[a]][id] + f[BX + ax[a]][at(n, cn)]);
                }
            }
        }
        fluid_pencil(nd, h, tau, gamma, U, B, buf + 8 * nd);
        for (s = 0; s < nd; s++) {
            c[d] = s;
            id = at(n, c);
            f[RHO][id] = U[0][s];
            f[MX + d][id] = U[1][s];
            f[MX + t1][id] = U[2][s];
            f[MX + t2][id] = U[3][s];
            f[EN][id] = U[4][s];
        }
        free(buf);
    }
}

/*
 * Magnetic advection-constraint sweep along axis d with step tau.
 * For each transverse axis t: the edge flux e_t of b_t along d is computed on
 * every pencil from the unmodified state; then
 *   b_t(cell)            -= tau/h_d * (e_t(i+1/2) - e_t(i-1/2))   (advection)
 *   b_d(face i+1/2, j)   += tau/h_t * (e_t(pencil j+1) - e_t(pencil j))
 *                                                               (constraint)
 * where e_t on pencil j lives on the edge (d: i+1/2, t: j-1/2).  The total
 * energy e is not touched (it is the conserved variable of Eq. 3).
 */
void orc_mag_sweep(const int n[3], double *f[8], int d, double tau) {
    if (any_boundary()) orc_fill_ghosts(n, f);
    int nd = n[d];
    double hd = 1.0 / cells_per_length(n, d);
    long N = (long)n[0] * n[1] * n[2];
    int ts[2] = {t1_of(d), t2_of(d)};
    double *E[2];
    int k;

    for (k = 0; k < 2; k++) {
        int t = ts[k], o = 3 - d - t; /* o: the third axis */
        int np = n[t] * n[o];
        int p;
        E[k] = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(static)
        for (p = 0; p < np; p++) {
            double *buf = (double *)malloc(sizeof(double) * (size_t)nd * 6);
            double *q = buf, *u = buf + nd, *ub = buf + 2 * nd, *fe = buf + 3 * nd;
            int s, c[3], cm[3];
            c[t] = p % n[t];
            c[o] = p / n[t];
            for (s = 0; s < nd; s++) {
                long id, idm;
                c[d] = s;
                memcpy(cm, c, sizeof cm);
                cm[t] -= 1;
                id = at(n, c);
                idm = at(n, cm);
                q[s] = f[BX + t][id];
                /* v_d averaged to the b_t face between cells j-1 and j */
                u[s] = 0.5 * (f[MX + d][id] / f[RHO][id] + f[MX + d][idm] / f[RHO][idm]);
            }
            for (s = 0; s < nd; s++) ub[s] = 0.5 * (u[s] + u[wrap(s + 1, nd)]);
            advect_flux(nd, hd, tau, q, ub, fe, buf + 4 * nd);
            for (s = 0; s < nd; s++) {
                c[d] = s;
                E[k][at(n, c)] = fe[s];
            }
            free(buf);
        }
    }
    /* apply: advection of each b_t, then the constraint on b_d */
    for (k = 0; k < 2; k++) {
        int t = ts[k];
        double ht = 1.0 / cells_per_length(n, t);
        long id;
#pragma omp parallel for schedule(static)
        for (id = 0; id < N; id++) {
            int c[3], cm[3];
            c[0] = (int)(id % n[0]);
            c[1] = (int)((id / n[0]) % n[1]);
            c[2] = (int)(id / ((long)n[0] * n[1]));
            memcpy(cm, c, sizeof cm);
            cm[d] -= 1;
            f[BX + t][id] -= (tau / hd) * (E[k][id] - E[k][at(n, cm)]);
        }
#pragma omp parallel for schedule(static)
        for (id = 0; id < N; id++) {
            /* b_d on the low face of cell c along d = face (c_d - 1) + 1/2 */
            int c[3], e0[3], e1[3];
            c[0] = (int)(id % n[0]);
            c[1] = (int)((id / n[0]) % n[1]);
            c[2] = (int)(id / ((long)n[0] * n[1]));
            memcpy(e0, c, sizeof e0);
            e0[d] -= 1;              /* edge (d: c_d - 1/2, t: c_t - 1/2) */
            memcpy(e1, e0, sizeof e1);
            e1[t] += 1;              /* edge (d: c_d - 1/2, t: c_t + 1/2) */
            f[BX + d][id] += (tau / ht) * (E[k][at(n, e1)] - E[k][at(n, e0)]);
        }
    }
    free(E[0]);
    free(E[1]);
}

/* Largest signal rate max_cells max_d (|v_d| + c_f*) / h_d, c_f* the fast-speed
 * bound sqrt((gamma p + |b_c|^2)/rho); the CFL timestep is 2*cfl/rate.  With
 * non-periodic axes: over the interior cells, after refilling the ghosts (a
 * ghost cell next to the periodic wrap pairs faces from both ends). */
double orc_cfl_rate(const int n[3], double gamma, double *const f[8]) {
    long N = (long)n[0] * n[1] * n[2];
    if (any_boundary()) orc_fill_ghosts(n, (double **)f);
    double rmax = 0.0;
    long id;
#pragma omp parallel for reduction(max : rmax) schedule(static)
    for (id = 0; id < N; id++) {
        int c[3], cn[3], a;
        double b[3], v[3], rho = f[RHO][id], b2 = 0.0, kin = 0.0, p, cf, r = 0.0;
        c[0] = (int)(id % n[0]);
        c[1] = (int)((id / n[0]) % n[1]);
        c[2] = (int)(id / ((long)n[0] * n[1]));
        for (a = 0; a < 3; a++)  /* interior cells only along non-periodic axes */
            if (g_bc[a] && (c[a] < GHOST || c[a] >= n[a] - GHOST)) break;
        if (a < 3) continue;
        for (a = 0; a < 3; a++) {
            memcpy(cn, c, sizeof cn);
            cn[a] += 1;
            b[a] = 0.5 * (f[BX + a][id] + f[BX + a][at(n, cn)]);
            v[a] = f[MX + a][id] / rho;
            b2 += b[a] * b[a];
            kin += 0.5 * f[MX + a][id] * v[a];
        }
        p = (gamma - 1.0) * (f[EN][id] - kin - 0.5 * b2);
        cf = sqrt((gamma * p + b2) / rho);
        for (a = 0; a < 3; a++) {
            double ra = (fabs(v[a]) + cf) * cells_per_length(n, a);
            if (ra > r) r = ra;
        }
        if (r > rmax) rmax = r;
    }
    return rmax;
}

/* One full timestep dt: x, y, z then z, y, x, each sweep with tau = dt/2. */
void orc_step(const int n[3], double gamma, double *f[8], double dt) {
    double tau = 0.5 * dt;
    int d;
    for (d = 0; d < 3; d++) {
        orc_fluid_sweep(n, gamma, f, d, tau);
        orc_mag_sweep(n, f, d, tau);
    }
    for (d = 2; d >= 0; d--) {
        orc_mag_sweep(n, f, d, tau);
        orc_fluid_sweep(n, gamma, f, d, tau);
    }
}

/* nsteps full steps, each with its own CFL timestep; returns elapsed time.
 * dts (optional, length nsteps) receives the timesteps taken. */
double orc_run(const int n[3], double gamma, double *f[8], int nsteps, double cfl,
               double *dts) {
    double t = 0.0;
    int s;
    for (s = 0; s < nsteps; s++) {
        double dt = 2.0 * cfl / orc_cfl_rate(n, gamma, f);
        if (dts) dts[s] = dt;
        orc_step(n, gamma, f, dt);
        t += dt;
    }
    return t;
}

/* thread count the OpenMP runtime will use (1 without OpenMP) */
#ifdef _OPENMP
#include <omp.h>
int orc_threads(void) { return omp_get_max_threads(); }
void orc_set_threads(int t) { omp_set_num_threads(t); }
#else
int orc_threads(void) { return 1; }
void orc_set_threads(int t) { (void)t; }
#endif
