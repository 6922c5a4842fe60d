/*
 * sgn_oracle.h -- plain FP64 CPU oracle for the explicit patch-wise finite-volume
 * step of the hyperbolic Serre-Green-Naghdi systems (mbHSGN, HSGN) with the switch
 * to the shallow water equations near shore.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library.  It shares no code, header,
 * table or helper with the CUDA path in paper_2606_12162_gb300/.
 *
 * Every function in sgn_oracle.c names the passage of the paper it follows
 * (Sec. 2-4, the equations cited there, App. B and App. C).
 *
 * Layout of the state that crosses this interface: field-major SoA, each field a
 * dense ny*nx row-major array (x fastest).  Field order: eta, hu, hv
 * [, hw] [, hsigma], hp [, hp_b]  (SWE: 3, mbHSGN: 5, HSGN: 7 fields).
 * eta = h + b is the surface elevation relative to the still level eta0 = 0.
 */
#ifndef SGN_ORACLE_H
#define SGN_ORACLE_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { OR_SWE = 0, OR_MBHSGN = 1, OR_HSGN = 2 };
enum { OR_BC_WALL = 0, OR_BC_EXTRAP = 1, OR_BC_PERIODIC = 2 };
enum { OR_LIM_MINMOD = 0, OR_LIM_MC = 1, OR_LIM_NONE = 2 };

/* status bits (or_status) */
enum {
  OR_ST_NEGDEPTH = 1u, OR_ST_NONFINITE = 2u, OR_ST_CFL = 4u,
  OR_ST_NONHYP = 8u, OR_ST_ALLDRY = 16u, OR_ST_GAUGE_FULL = 32u
};

typedef struct {
  int nx, ny;
  double x0, y0, dx, dy;
  int bc[4];            /* x-, x+, y-, y+ */
  int model;            /* OR_SWE / OR_MBHSGN / OR_HSGN */
  double alpha;         /* dimensionless relaxation parameter, c = alpha sqrt(gH) */
  double h_star;        /* transition depth of phi_T */
  int n_transition;     /* neighbourhood radius n of phi_T, 0..2 */
  double xi0, xi1;      /* sensor parameters */
  double cfl, g, dry_tol;
  int limiter;          /* OR_LIM_* */
  int strang;           /* 1 Strang, 0 Lie-Trotter */
} or_config;

typedef struct or_solver or_solver;

/* b: ny*nx bathymetry (copied).  phi_override: NULL, or ny*nx bytes that replace
 * the computed transition mask phi_T (copied). Returns NULL on invalid input. */
or_solver* or_create(const or_config* cfg, const double* b, const unsigned char* phi_override);
void or_destroy(or_solver* s);
int or_nvar(const or_solver* s);
int or_set_state(or_solver* s, const double* q, double t);
int or_get_state(const or_solver* s, double* q, double* t);
/* nsteps steps with the CFL time step; returns 0 or -1 (status bits say why). */
int or_step(or_solver* s, int nsteps);
/* one step with a prescribed time step dt (used by crop parity checks). */
int or_step_dt(or_solver* s, double dt);
double or_dt_cfl(or_solver* s);             /* CFL time step of the current state */
double or_mass(const or_solver* s);         /* sum h dx dy, row order */
unsigned or_status(const or_solver* s);
double or_last_dt(const or_solver* s);
double or_max_courant(const or_solver* s);
/* c2 and phi_T of the interior cells (ny*nx each; either may be NULL). */
int or_get_aux(const or_solver* s, double* c2, unsigned char* phi);
/* replace c^2 of the interior cells (ny*nx >= 0; ghosts by the boundary conditions). */
int or_set_c2(or_solver* s, const double* c2);
int or_add_gauges(or_solver* s, const double* xy, int n, int capacity);
/* records: [rec][gauge][t, eta, hu, hv]; returns the number of records. */
int or_gauges(const or_solver* s, double* out, size_t cap);

/* ---- patch mode: one patch of a refined level (block-structured AMR) ----
 * The caller owns the ghost frame: arrays cover the padded patch of
 * (ny+4) x (nx+4) cells (two ghost layers), row-major, field-major for states.
 * A step is or_step_begin (source, faces, limiters, transverse terms,
 * positivity factors of the interior) then or_step_end (update, second source
 * step); ghost-cell factors may be exchanged in between (or_get/set_theta). */
or_solver* or_create_frame(const or_config* cfg, const double* b_frame, const unsigned char* phi_frame);
int or_set_frame(or_solver* s, const double* q, double t);
int or_get_frame(const or_solver* s, double* q);
int or_step_begin(or_solver* s, double dt);
int or_step_end(or_solver* s, double dt);
int or_get_theta(const or_solver* s, double* theta);
int or_set_theta(or_solver* s, const double* theta);
/* theta-weighted mass flux at the faces of the interior cells (dir 0: ny x
 * (nx+1) x faces, dir 1: (ny+1) x nx y faces). */
int or_face_mass(const or_solver* s, int dir, double* out);
double or_max_speed(or_solver* s);

/* ---- single-face and single-cell pieces, exposed for the pin tests ---- */

/* Right eigenvector matrix (App. C, columns are the waves, rows the fields in the
 * order above) for the x-direction with passive v, at the state
 * roe = {h, u, v, w, sigma, p, pb, c2}; s1/sN replace the fast speeds. Row-major
 * nv*nv into R. */
int or_eigvecs(int model, const double* roe, double g, double s1, double sN, double* R);
/* Jacobian dF/dq + A of App. C at the same state (row-major nv*nv). */
int or_jacobian(int model, const double* roe, double g, double* J);
/* One normal Riemann solve in x.  qL/qR: conserved states (field order, eta
 * first), bL/bR bathymetry, c2L/c2R relaxation.  Outputs (any may be NULL):
 * Z[nv*nv] waves (wave-major), s[nv] speeds, Am/Ap[nv] fluctuations,
 * delta[nv] total fluctuation, Fhat mass flux. */
int or_face(const or_config* cfg, const double* qL, const double* qR, double bL, double bR,
            double c2L, double c2R, double* Z, double* s, double* Am, double* Ap,
            double* delta, double* Fhat);
/* SDIRK(2,2) source step of length tau on one cell: aux = (w, p) [mbHSGN] or
 * (w, sigma, p, pb) [HSGN] primitives, updated in place. */
int or_source(int model, double h, double c2, double tau, double* aux);
double or_psi(double bR, double bL, double xi0, double xi1);

#ifdef __cplusplus
}
#endif
#endif
