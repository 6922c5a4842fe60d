/*
 * sgn.h -- C ABI of the GB300 (sm_103a) explicit finite-volume step for the
 * hyperbolic Serre-Green-Naghdi systems with the transition to the shallow water
 * equations near shore.
 *
 * The method (paper Sec. 3-4): the state q = (h, hu, hv, ...) of one of
 *   SWE    (Eq. NSWEs)   3 fields: eta, hu, hv
 *   mbHSGN (Eq. mbHSGN)  5 fields: eta, hu, hv, hw, hp
 *   HSGN   (Eq. HSGN)    7 fields: eta, hu, hv, hw, h sigma, hp, h p_b
 * advances by operator splitting (Sec. 4): a relaxation-source half step
 * (SDIRK(2,2)), the wave-propagation step (f-wave normal Riemann solver with
 * Roe averages, Einfeldt speeds, well-balanced bathymetry quadrature with the
 * sharpness sensor psi, MC/minmod limiters, transverse Riemann solver), a second
 * source half step, the switch to SWE where phi_T = 0 (Eq. transition_function)
 * and a CFL time step from the maximum wave speed (Eq. eigenvalue_bound).
 * The relaxation parameter is c^2 = alpha^2 g H phi_T (Sec. 3.3).
 *
 * Conventions for every entry point:
 *  - Return 0 on success or a negative SGN_E* code; no entry point aborts.
 *  - Host arrays passed in are copied before the call returns; output arrays
 *    are caller-owned and must hold the stated number of elements.
 *  - Device memory belongs to the handle and comes from the allocator given to
 *    sgn_create (NULL: cudaMalloc/cudaFree).  All work is issued on the stream
 *    given to sgn_create (NULL: the legacy default stream).
 *  - Dense field layout ("SoA"): field-major, each field ny*nx doubles, row-major
 *    with x fastest: q[(k*ny + j)*nx + i].  eta = h + b is the surface elevation
 *    above the still level 0; b < 0 under water.
 *  - A handle is not thread-safe; separate handles are independent.
 *  - Every computation runs in this library's CUDA kernels; there is no CPU path.
 */
#ifndef SGN_H
#define SGN_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define SGN_OK          0
#define SGN_EINVAL     -1   /* invalid argument (null pointer, size, enum value) */
#define SGN_ENOMEM     -2   /* the allocator returned NULL */
#define SGN_ECUDA      -3   /* a CUDA runtime call failed (no device, launch error) */
#define SGN_ENEGDEPTH  -4   /* a depth below -tolerance appeared (positivity lost) */
#define SGN_ENONFINITE -5   /* NaN or Inf in the state */
#define SGN_ECFL       -6   /* a face Courant number above 1 */
#define SGN_ENONHYP    -7   /* g h + p + c^2 < 0 at a wet cell (loss of hyperbolicity) */
#define SGN_EALLDRY    -8   /* no wet cell: no time step can be computed */
#define SGN_ERANGE     -9   /* output buffer too small / gauge outside the grid */

/* status bits reported by sgn_status (set on the device, never cleared by a step) */
#define SGN_ST_NEGDEPTH   1u
#define SGN_ST_NONFINITE  2u
#define SGN_ST_CFL        4u
#define SGN_ST_NONHYP     8u
#define SGN_ST_ALLDRY    16u
#define SGN_ST_GAUGEFULL 32u

typedef enum { SGN_SWE = 0, SGN_MBHSGN = 1, SGN_HSGN = 2 } sgn_model;
typedef enum { SGN_BC_WALL = 0, SGN_BC_EXTRAP = 1, SGN_BC_PERIODIC = 2 } sgn_bc;
typedef enum { SGN_FP64 = 0, SGN_MIXED = 1 } sgn_precision;
typedef enum { SGN_LIM_MINMOD = 0, SGN_LIM_MC = 1, SGN_LIM_NONE = 2 } sgn_limiter;

/* Logically rectangular grid of nx*ny cells of size dx*dy with lower-left corner
 * (x0, y0); cell (i, j) has centre (x0 + (i+1/2) dx, y0 + (j+1/2) dy).
 * bc: boundary condition on the sides x-, x+, y-, y+ (periodic must be paired). */
typedef struct {
  int nx, ny;
  double x0, y0, dx, dy;
  int bc[4];
} sgn_grid;

/* Method parameters (Sec. 4, last paragraph: alpha = 3, xi0 = 0.01, xi1 = 0.05,
 * Courant 0.9-1, n = 1).  precision: SGN_FP64 computes and stores everything in
 * FP64; SGN_MIXED stores the state in FP32 (eta as deviation from the still level)
 * and computes the fluxes and sources in FP32, keeping FP64 for the depth
 * h = eta - b and the hydrostatic term g h_hat d(eta), the positivity guard, the
 * conservative mass update and the mass reduction. */
typedef struct {
  double alpha;        /* dimensionless relaxation parameter, c = alpha sqrt(g H) */
  double h_star;       /* transition depth of phi_T [m] */
  int n_transition;    /* neighbourhood radius n of phi_T in cells, 0..2 */
  double xi0, xi1;     /* sensor parameters */
  double cfl;          /* Courant number of the time step, (0, 1] */
  double g;            /* gravity [m/s^2] */
  double dry_tol;      /* a cell is wet when h > dry_tol [m] */
  int limiter;         /* sgn_limiter */
  int strang;          /* 1: Strang splitting, 0: Lie-Trotter */
  int precision;       /* sgn_precision */
} sgn_params;

/* Device memory provider: alloc(bytes, ctx) returns device memory or NULL,
 * free(ptr, ctx) releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* ctx;
} sgn_allocator;

typedef struct sgn_solver sgn_solver;

/* Fill *p with the defaults: alpha 3, h_star 0, n 1, xi0 0.01, xi1 0.05, cfl 0.9,
 * g 9.81, dry_tol 1e-3, MC limiter, Strang, FP64. */
void sgn_default_params(sgn_params* p);

/* Number of state fields of a model (3, 5, 7) or SGN_EINVAL. */
int sgn_nvar(int model);

/* Human-readable text of an error code (static storage). */
const char* sgn_strerror(int code);

/* Create a solver.  bathymetry: ny*nx doubles (copied).  phi_override: NULL, or
 * ny*nx bytes replacing the computed transition mask phi_T (0: SWE, else
 * dispersive), copied.  The initial state is the lake at rest eta = max(0, b).
 * Needs nx, ny >= 2, dx, dy > 0, 0 < cfl <= 1, n_transition in 0..2.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int sgn_create(const sgn_grid* grid, const double* bathymetry, int model,
               const sgn_params* params, const unsigned char* phi_override,
               const sgn_allocator* allocator, void* cuda_stream, sgn_solver** out);

/* Replace the state: q is nvar*ny*nx doubles in host memory; t is the new time.
 * Pinned, mapped host memory (cudaHostAlloc, cudaMallocHost, a range registered
 * with cudaHostRegister, a pinned torch tensor) is read by the conversion kernel
 * in place over the host link; other host memory is first copied to a device
 * staging buffer.  The SWE/dry switch is
 * applied (auxiliaries zeroed where phi_T = 0 or h <= dry_tol, momenta zeroed
 * where h <= dry_tol), the status word and the gauge records are cleared and the
 * CFL time step of the new state is computed.  Errors: EINVAL, ECUDA. */
int sgn_set_state(sgn_solver* s, const double* q, double t);

/* As sgn_set_state with q in device memory (nvar*ny*nx doubles, dense layout). */
int sgn_set_state_device(sgn_solver* s, const double* q_dev, double t);

/* Advance nsteps CFL-limited time steps (CUDA-graph replays of the kernel
 * sequence; the time step lives on the device, no host synchronisation inside
 * the batch).  Synchronises once at the end, reads the status word and returns
 * the error of the first set bit (ENEGDEPTH, ENONFINITE, ECFL, ENONHYP, EALLDRY).
 * t_out (may be NULL) receives the time reached. */
int sgn_step(sgn_solver* s, int nsteps, double* t_out);

/* Advance one step with the prescribed time step dt > 0 instead of the CFL one
 * (the next CFL step is recomputed from the new state).  Errors as sgn_step. */
int sgn_step_dt(sgn_solver* s, double dt);

/* Copy fields of the state to host memory.  field_mask: bit k selects field k
 * (0: all fields); the selected fields are written consecutively (ny*nx doubles
 * each) into out, which holds out_len doubles.  Pinned, mapped host memory is
 * written by the conversion kernel in place; other host memory through a device
 * staging buffer.  t_out may be NULL.
 * Synchronises the stream.  Errors: EINVAL, ERANGE, ECUDA. */
int sgn_get_state(sgn_solver* s, int field_mask, double* out, size_t out_len, double* t_out);

/* As sgn_get_state into device memory (all fields, nvar*ny*nx doubles); does not
 * synchronise. */
int sgn_get_state_device(sgn_solver* s, double* out_dev, size_t out_len);

/* Gauges: xy holds n (x, y) pairs (copied); each step appends, per gauge, the
 * record (t, eta, hu, hv) of the cell containing the gauge, up to capacity
 * steps (then SGN_ST_GAUGEFULL is set and records stop).  Replaces earlier
 * gauges.  Errors: EINVAL, ERANGE (gauge outside the grid), ENOMEM. */
int sgn_add_gauges(sgn_solver* s, const double* xy, int n, int capacity);

/* Copy the gauge records [rec][gauge][4] (cap doubles available in out) and
 * report the number of records in *nrec; the records stay until the next
 * sgn_set_state / sgn_add_gauges / sgn_clear_gauges.  Errors: EINVAL, ERANGE. */
int sgn_gauges(sgn_solver* s, double* out, size_t cap, int* nrec);
int sgn_clear_gauges(sgn_solver* s);

/* Status word, the last time step taken and the largest face Courant number of
 * the last step (any pointer may be NULL).  Synchronises the stream. */
int sgn_status(sgn_solver* s, unsigned* flags, double* last_dt, double* max_courant);

/* The CFL time step the next sgn_step will take (Eq. (eigenvalue_bound) and the
 * CFL condition of Sec. 4, from the current state; 0 if every cell is dry), so
 * that a caller can end a run exactly at an output time with sgn_step_dt.
 * Synchronises the stream.  Errors: EINVAL. */
int sgn_next_dt(sgn_solver* s, double* dt);

/* Total mass sum(h) dx dy over the grid by a deterministic two-stage FP64
 * reduction.  Synchronises the stream. */
int sgn_mass(sgn_solver* s, double* mass);

/* Relaxation parameter c^2 (ny*nx doubles) and transition mask phi_T (ny*nx
 * bytes) of the interior cells; either pointer may be NULL. */
int sgn_get_aux(sgn_solver* s, double* c2, unsigned char* phi);

/* Well-prepared initial data for mbHSGN (Sec. 3.2): replaces hw and hp of the
 * current state by h w and h p, w from the mbSGN constraint and p from the
 * relation of Sec. 3.2 with d_t u eliminated (w = -(h/2) u_x + u b_x, the sign
 * of Eq. (mbHSGN) and of the kinematic bottom condition; p re-derived from the
 * hw equation and that constraint, as the printed relation is dimensionally
 * inconsistent), for data varying along x: every row is solved independently
 * (one tridiagonal system per row, zero-gradient ends); rows with a dry cell
 * are left unchanged.  mbHSGN solvers only (else EINVAL).  The first call
 * allocates 7 nx ny doubles of scratch through the solver's allocator (ENOMEM).
 * Recomputes the next time step.  Synchronises the stream. */
int sgn_well_prepare(sgn_solver* s);

/* Replace the relaxation parameter c^2 of every cell by a given field (ny*nx
 * doubles, row-major, copied; every value finite and >= 0): the constant-c^2
 * setting of the steady-state test of Sec. 5.3 (Table 3) instead of
 * alpha^2 g H phi_T.  Ghost cells follow the boundary conditions; call it
 * before sgn_set_state (the SWE switch and the first time step use c^2).
 * Synchronises the stream.  Errors: EINVAL. */
int sgn_set_c2(sgn_solver* s, const double* c2);

/* Per-kernel timing: when enabled, steps launch kernels without CUDA graphs and
 * bracket each launch with CUDA events on the solver stream.  sgn_kernel_times
 * returns, for up to n kernels, the name, the accumulated time [ms] and the
 * number of launches since profiling was enabled; the return value is the
 * number of kernel kinds. */
int sgn_set_profiling(sgn_solver* s, int enable);
int sgn_kernel_times(sgn_solver* s, const char** names, double* ms, long* launches, int n);

/* Number of kernel launches one time step issues (for launch accounting). */
int sgn_launches_per_step(sgn_solver* s);

/* Autotuner of the step's launch shapes and schedule.  The paper runs the
 * step on CPUs (Sec. 7) and has no counterpart; it serves the batched form,
 * whose level grids differ in size and shape.
 *
 * A tuning is SGN_TUNE_N option indices, one per slot:
 *   SGN_TUNE_PREP, _FACE_X, _FACE_Y, _TRANS_X, _TRANS_Y, _THETA, _UPDATE: the
 *     thread-block shape of that kernel, 0 .. SGN_TUNE_OPTS-1 (0 = default);
 *     sgn_get_tuning reports the block dimensions each index stands for;
 *   SGN_TUNE_SCHEDULE: 0 = one stream; 1 = the x and y face kernels, then the
 *     two transverse kernels, as two concurrent branches; 2 = the one-pass
 *     kernel: the whole step in one launch that keeps every intermediate
 *     quantity on chip and moves only the state through HBM (mixed precision on
 *     a single grid only: EINVAL for an FP64 solver; a refined level falls back
 *     to 0).  With schedule 2 the SGN_TUNE_UPDATE option selects the rows one
 *     block of the one-pass kernel marches over: at most 128, 64 or 256 (its
 *     block is 128 columns wide), halved down to 32 while the grid would give
 *     fewer tiles than the device holds resident blocks; sgn_get_tuning
 *     reports the rows used.  A new mixed-precision solver starts with
 *     schedule 2 when the grid gives at least half as many 32-row tiles as
 *     resident blocks (on 152 SMs: from about 1024 x 1024 cells), else with
 *     schedule 0, and with option 0 elsewhere; an FP64 solver with schedule 0.
 * The block-shape options and schedules 0 and 1 compute the same values bit
 * for bit; schedule 2 evaluates the same expressions in one kernel and agrees
 * with them to FP32 rounding (the compiler may fuse a different set of
 * multiply-adds).
 *
 * sgn_autotune times, on the current state and in step order, reps launches
 * of each option of each kernel (CUDA events on the solver stream, after one
 * untimed launch), keeps the fastest, then times the whole step as a CUDA graph
 * in every schedule (schedule 2 with each of its row counts) and keeps the
 * fastest.  It leaves
 * the state, time, next dt and status unchanged: the next step is the one that
 * would have run without it.  choice (SGN_TUNE_N ints, may be NULL) receives
 * the tuning kept; ms (SGN_TUNE_N * SGN_TUNE_OPTS doubles, may be NULL) the
 * mean time per launch [ms] of option o of slot k at ms[k*SGN_TUNE_OPTS + o]
 * (for the schedule slot: of the whole step, the best row count for schedule
 * 2; -1 where not measured).
 * Synchronises the stream.  Errors: EINVAL (reps outside 1..10000), ECUDA.
 *
 * sgn_set_tuning installs a tuning (EINVAL for an index out of range);
 * sgn_get_tuning reports the current one and, per slot, the block dimensions
 * (bx, by; 0 for the schedule slot; with schedule 2 the update slot reports
 * 128 columns by the rows per block).  Any pointer of sgn_get_tuning may be
 * NULL. */
#define SGN_TUNE_N 8
#define SGN_TUNE_OPTS 3
enum {
  SGN_TUNE_PREP = 0, SGN_TUNE_FACE_X = 1, SGN_TUNE_FACE_Y = 2, SGN_TUNE_TRANS_X = 3,
  SGN_TUNE_TRANS_Y = 4, SGN_TUNE_THETA = 5, SGN_TUNE_UPDATE = 6, SGN_TUNE_SCHEDULE = 7
};
int sgn_autotune(sgn_solver* s, int reps, int* choice, double* ms);
int sgn_set_tuning(sgn_solver* s, const int* choice);
int sgn_get_tuning(sgn_solver* s, int* choice, int* bx, int* by);

/* Release all device memory and the handle (NULL is ignored). */
void sgn_destroy(sgn_solver* s);

/* Diagnostic: the FP64 reciprocal and square root used inside the kernels (a
 * hardware approximation refined by Newton-Raphson steps) against CUDA's IEEE
 * division and sqrt.  x_dev: n positive doubles in device memory; err_dev: 2n
 * doubles in device memory receiving, per input, the error of the reciprocal and
 * of the square root in units in the last place.  Synchronises the device.
 * Errors: EINVAL, ECUDA. */
int sgn_math_check(const double* x_dev, int n, double* err_dev);

/* Diagnostic: the FP32 reciprocal and square root of the mixed path (the
 * hardware approximations refined by one Newton-Raphson step) against CUDA's
 * correctly rounded FP32 division and square root.  x_dev: n positive floats
 * in device memory, x and 1/x normal (the approximations flush subnormals); err_dev: 2n doubles in device memory receiving the
 * errors in FP32 units in the last place.  Synchronises the device.
 * Errors: EINVAL, ECUDA. */
int sgn_math_check_f32(const float* x_dev, int n, double* err_dev);

/* Total mass without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory where they
 * need the mass (a host that hands the library a fixed memory pool and forbids
 * further allocations, or a latency-critical loop where cudaMalloc / cudaFree,
 * which can synchronise the device, are not acceptable).
 *
 * Computes sum over the nx*ny cells of max(0, eta - b) * dx * dy, like
 * sgn_mass, from caller-owned device arrays: eta_dev and b_dev hold nx*ny
 * doubles each (row-major, x fastest, e.g. field 0 of sgn_get_state_device and
 * the bathymetry), mass_dev receives one double.  Work is issued on cuda_stream
 * (NULL: the legacy default stream) and the call does not synchronise.
 * The per-block partial sums live in a fixed array compiled into the library:
 * SGN_MASS_SCRATCH_MAX doubles, one per 4096 cells, so grids above
 * 4096 * SGN_MASS_SCRATCH_MAX cells are rejected with SGN_ERANGE.  Every call
 * shares that array (it keeps the last call's partials; each call writes every
 * slot it reads), so calls that may overlap on the GPU -- on different streams
 * or from different host threads -- race and must be ordered by the caller.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Errors: EINVAL (null pointer, non-positive size), ERANGE, ECUDA. */
#define SGN_MASS_SCRATCH_MAX 65536
int sgn_mass_static(const double* eta_dev, const double* b_dev, int nx, int ny, double dx, double dy,
                    double* mass_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SGN_H */
