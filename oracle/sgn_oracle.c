/*
 * sgn_oracle.c -- plain, slow FP64 CPU oracle for one explicit time step of the
 * hyperbolic SGN systems (Sec. 3-4 of the paper) with the transition to SWE.
 *
 * TEST INFRASTRUCTURE ONLY (see sgn_oracle.h).  Built with -O2 -ffp-contract=off.
 * It shares no code with the CUDA path.  Every decomposition is a dense solve of
 * the eigenvector matrix (Gaussian elimination), every implicit stage a dense
 * solve of (I - gamma tau M); the loops run over separate face arrays in the
 * order the method states: ghost fill, source half step, x-faces, y-faces,
 * limiters, transverse propagation, conservative update, source half step.
 * OpenMP only parallelises independent loop iterations (results do not depend
 * on the thread count).
 *
 * Readings of points where the paper is silent, ambiguous or garbled (the
 * letters are used throughout the repository):
 *  G1  c^2 = alpha^2 g H phi_T  (Sec. 3.3 formula vs the definition alpha = c/sqrt(gH))
 *  G7  Strang splitting by default, Lie-Trotter as an option (Sec. 4)
 *  G8  transverse solver: App. C eigenstructure at the Roe average of the cell
 *      receiving the fluctuation and its transverse neighbour; fluctuations and
 *      second-order corrections are both propagated; no bathymetry term
 *  G9  HSGN bathymetry terms: psi multiplies every non-hydrostatic coupling
 *  G11 phi_T neighbourhood: cell centres within n*dx, eta0 = 0 (still level)
 *  G12 psi = 0 when b_i + b_{i-1} = 0
 *  G14 wet/dry: a dry neighbour higher than the wet surface is a wall; limiter
 *      off at faces touching a dry cell; draining-time positivity guard
 *  G23 a wave of speed exactly 0 is split half/half
 *  G24 relaxation term h c^2 d_x u discretised as c^2_hat * jump(hu) (c^2 stays
 *      outside the derivative, as printed in Eq. (mbHSGN)); for constant c^2 this
 *      equals the flux form d_x[h u (p + c^2)] printed for HSGN
 */
#include "sgn_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NG 2          /* ghost layers */
#define NVMAX 7

typedef struct { int nv, hw, hs, hp, hpb; } fields_t;

/* Field lists of the three models: Eq. (NSWEs), Eq. (mbHSGN), Eq. (HSGN). */
static fields_t model_fields(int model) {
  fields_t f = {3, -1, -1, -1, -1};
  if (model == OR_MBHSGN) { f.nv = 5; f.hw = 3; f.hp = 4; }
  else if (model == OR_HSGN) { f.nv = 7; f.hw = 3; f.hs = 4; f.hp = 5; f.hpb = 6; }
  return f;
}

typedef struct {
  double Z[NVMAX][NVMAX];   /* f-waves Z[p][k] */
  double s[NVMAX];          /* wave speeds */
  double Am[NVMAX], Ap[NVMAX];
  double Ftil[NVMAX], Lv[NVMAX], Rv[NVMAX], Pt[NVMAX];
  double d[NVMAX];          /* total fluctuation delta */
  double Fhat, M;
  int active, first_order, wall;
} face_t;

struct or_solver {
  or_config c;
  fields_t f;
  int nxp, nyp;
  double* q;                 /* nv fields, padded */
  double* b;                 /* padded */
  double* c2;                /* padded */
  unsigned char* phi;        /* padded */
  face_t* fx;                /* (nxp+1) x nyp */
  face_t* fy;                /* nxp x (nyp+1) */
  double* theta;             /* padded */
  double t, last_dt, max_courant;
  unsigned status;
  int frame;                 /* ghost frame given by the caller (patch of a refined level) */
  int ngauge, gcap, grec;
  int* gidx;
  double* grec_buf;
};

static void set_status(or_solver* s, unsigned bit) {
#pragma omp atomic
  s->status |= bit;
}

static size_t cidx(const or_solver* s, int I, int J) { return (size_t)J * s->nxp + I; }
static double* fld(or_solver* s, int k) { return s->q + (size_t)k * s->nxp * s->nyp; }

/* ------------------------------------------------------------------------- */
/* Dense linear solve by Gaussian elimination with partial pivoting (n <= 7). */
static int solve_dense(int n, const double* A_in, const double* rhs, double* x) {
  double A[NVMAX][NVMAX + 1];
  for (int i = 0; i < n; i++) {
    for (int j = 0; j < n; j++) A[i][j] = A_in[i * n + j];
    A[i][n] = rhs[i];
  }
  for (int col = 0; col < n; col++) {
    int piv = col;
    for (int r = col + 1; r < n; r++)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (A[piv][col] == 0.0) return -1;
    if (piv != col)
      for (int j = 0; j <= n; j++) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
    for (int r = col + 1; r < n; r++) {
      double m = A[r][col] / A[col][col];
      for (int j = col; j <= n; j++) A[r][j] -= m * A[col][j];
    }
  }
  for (int i = n - 1; i >= 0; i--) {
    double acc = A[i][n];
    for (int j = i + 1; j < n; j++) acc -= A[i][j] * x[j];
    x[i] = acc / A[i][i];
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Boundary conditions (Sec. 5: reflecting walls, zeroth-order extrapolation,
 * periodic).  Maps a padded index to the interior cell it copies; *flip is set
 * when a reflecting wall negates the normal momentum. */
static int bc_map(int i, int n, int bcl, int bcr, int* flip) {
  *flip = 0;
  int k = i - NG;                     /* interior coordinate */
  if (k < 0) {
    int layer = -k - 1;
    if (bcl == OR_BC_WALL) { *flip = 1; return NG + layer; }
    if (bcl == OR_BC_EXTRAP) return NG;
    return NG + n - 1 - layer;        /* periodic */
  }
  if (k >= n) {
    int layer = k - n;
    if (bcr == OR_BC_WALL) { *flip = 1; return NG + n - 1 - layer; }
    if (bcr == OR_BC_EXTRAP) return NG + n - 1;
    return NG + layer;
  }
  return i;
}

/* Fill the ghost frame of nf padded arrays; vector fields hu (index 1) and hv
 * (index 2) are negated across reflecting walls when is_state is set. */
static void fill_ghosts(or_solver* s, double* base, int nf, int is_state) {
  if (s->frame) return;
  size_t np = (size_t)s->nxp * s->nyp;
  for (int J = 0; J < s->nyp; J++)
    for (int I = 0; I < s->nxp; I++) {
      int inx = (I >= NG && I < NG + s->c.nx), iny = (J >= NG && J < NG + s->c.ny);
      if (inx && iny) continue;
      int fxl, fyl;
      int Is = bc_map(I, s->c.nx, s->c.bc[0], s->c.bc[1], &fxl);
      int Js = bc_map(J, s->c.ny, s->c.bc[2], s->c.bc[3], &fyl);
      for (int k = 0; k < nf; k++) {
        double v = base[k * np + cidx(s, Is, Js)];
        if (is_state && k == 1 && fxl) v = -v;
        if (is_state && k == 2 && fyl) v = -v;
        base[k * np + cidx(s, I, J)] = v;
      }
    }
}

static void fill_ghosts_u8(or_solver* s, unsigned char* a) {
  if (s->frame) return;
  for (int J = 0; J < s->nyp; J++)
    for (int I = 0; I < s->nxp; I++) {
      int inx = (I >= NG && I < NG + s->c.nx), iny = (J >= NG && J < NG + s->c.ny);
      if (inx && iny) continue;
      int f1, f2;
      int Is = bc_map(I, s->c.nx, s->c.bc[0], s->c.bc[1], &f1);
      int Js = bc_map(J, s->c.ny, s->c.bc[2], s->c.bc[3], &f2);
      a[cidx(s, I, J)] = a[cidx(s, Is, Js)];
    }
}

/* ------------------------------------------------------------------------- */
/* Bathymetry sharpness sensor psi(b_i, b_{i-1}) of Sec. 4 (reading G12). */
double or_psi(double bR, double bL, double xi0, double xi1) {
  double den = fabs(bR + bL);
  if (den == 0.0) return 0.0;
  double xi = 2.0 * fabs(bR - bL) / den;
  if (xi < xi0) return 1.0;
  if (xi < xi0 + xi1) {
    double t = (xi - xi0) / xi1;
    return -3.0 * t * t + 2.0 * t * t * t + 1.0;
  }
  return 0.0;
}

/* ------------------------------------------------------------------------- */
/* Source step of Sec. 4: the ODEs dq/dt = S(q) are linear in the primitive
 * auxiliary variables with h (and hu, hv) frozen; integrated with SDIRK(2,2)
 * (Kennedy & Carpenter 2016, Sec. 4.1.2): gamma = 1 - 1/sqrt(2),
 *   Y1 = y + gamma tau M Y1,  Y2 = y + (1-gamma) tau M Y1 + gamma tau M Y2,
 *   y_new = Y2 (stiffly accurate).
 * mbHSGN, Eq. (mbHSGN): (hw)' = 3p/2, (hp)' = -2 c^2 w.
 * HSGN,   Eq. (HSGN):   (hw)' = p_b, (h sigma)' = -6 p_b + 12 p,
 *                       (hp)' = -c^2 sigma, (h p_b)' = -6 c^2 (w - sigma/2). */
static void source_matrix(int model, double h, double c2, double* M, int* n) {
  if (model == OR_MBHSGN) {
    *n = 2;
    M[0] = 0.0;               M[1] = 1.5 / h;      /* w' = 3p/(2h)   */
    M[2] = -2.0 * c2 / h;     M[3] = 0.0;          /* p' = -2c^2 w/h */
  } else {
    *n = 4;  /* (w, sigma, p, pb) */
    double z[16] = {0};
    z[0 * 4 + 3] = 1.0 / h;                            /* w'  = pb/h */
    z[1 * 4 + 2] = 12.0 / h;  z[1 * 4 + 3] = -6.0 / h; /* sigma' = (12p - 6pb)/h */
    z[2 * 4 + 1] = -c2 / h;                            /* p'  = -c^2 sigma/h */
    z[3 * 4 + 0] = -6.0 * c2 / h; z[3 * 4 + 1] = 3.0 * c2 / h; /* pb' = -6c^2(w - sigma/2)/h */
    memcpy(M, z, sizeof z);
  }
}

int or_source(int model, double h, double c2, double tau, double* y) {
  if (model == OR_SWE) return 0;
  double M[16]; int n;
  source_matrix(model, h, c2, M, &n);
  const double gam = 1.0 - 1.0 / sqrt(2.0);
  double A[16], Y1[4], Y2[4], r[4];
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) A[i * n + j] = (i == j ? 1.0 : 0.0) - gam * tau * M[i * n + j];
  if (solve_dense(n, A, y, Y1)) return -1;
  for (int i = 0; i < n; i++) {
    double my = 0.0;
    for (int j = 0; j < n; j++) my += M[i * n + j] * Y1[j];
    r[i] = y[i] + (1.0 - gam) * tau * my;
  }
  if (solve_dense(n, A, r, Y2)) return -1;
  for (int i = 0; i < n; i++) y[i] = Y2[i];
  return 0;
}

/* Source step plus the SWE/dry switch on one padded cell (Sec. 3.3, Sec. 4):
 * dry cells (h <= dry_tol) lose momentum and auxiliary variables; wet cells
 * with c^2 = 0 (phi_T = 0 or alpha = 0) keep SWE only (auxiliaries zeroed);
 * the remaining cells take the SDIRK(2,2) step on their primitives. */
static void source_cell(or_solver* s, int I, int J, double tau) {
  size_t id = cidx(s, I, J);
  const fields_t* f = &s->f;
  double h = fld(s, 0)[id] - s->b[id];
  if (h < 0.0) h = 0.0;
  double c2 = s->c2[id];
  int wet = h > s->c.dry_tol;
  if (!wet) {
    for (int k = 1; k < f->nv; k++) fld(s, k)[id] = 0.0;
    return;
  }
  if (s->c.model == OR_SWE) return;
  if (!(c2 > 0.0)) {
    for (int k = 3; k < f->nv; k++) fld(s, k)[id] = 0.0;
    return;
  }
  if (tau == 0.0) return;
  double y[4];
  if (s->c.model == OR_MBHSGN) {
    y[0] = fld(s, f->hw)[id] / h; y[1] = fld(s, f->hp)[id] / h;
    or_source(OR_MBHSGN, h, c2, tau, y);
    fld(s, f->hw)[id] = h * y[0]; fld(s, f->hp)[id] = h * y[1];
  } else {
    y[0] = fld(s, f->hw)[id] / h; y[1] = fld(s, f->hs)[id] / h;
    y[2] = fld(s, f->hp)[id] / h; y[3] = fld(s, f->hpb)[id] / h;
    or_source(OR_HSGN, h, c2, tau, y);
    fld(s, f->hw)[id] = h * y[0]; fld(s, f->hs)[id] = h * y[1];
    fld(s, f->hp)[id] = h * y[2]; fld(s, f->hpb)[id] = h * y[3];
  }
}

/* ------------------------------------------------------------------------- */
/* Cell data for the Riemann problems. */
typedef struct {
  double h, eta, b, c2;
  double q[NVMAX];
  double vel[2];            /* u, v */
  double w, sg, p, pb;      /* auxiliary primitives (0 if absent) */
  int wet;
} cell_t;

static cell_t load_cell(or_solver* s, int I, int J) {
  cell_t c; memset(&c, 0, sizeof c);
  size_t id = cidx(s, I, J);
  c.eta = fld(s, 0)[id]; c.b = s->b[id]; c.c2 = s->c2[id];
  c.h = c.eta - c.b; if (c.h < 0.0) c.h = 0.0;
  c.wet = c.h > s->c.dry_tol;
  c.q[0] = c.eta;
  for (int k = 1; k < s->f.nv; k++) c.q[k] = c.wet ? fld(s, k)[id] : 0.0;
  if (c.wet) {
    c.vel[0] = c.q[1] / c.h; c.vel[1] = c.q[2] / c.h;
    if (s->f.hw >= 0) c.w = c.q[s->f.hw] / c.h;
    if (s->f.hs >= 0) c.sg = c.q[s->f.hs] / c.h;
    if (s->f.hp >= 0) c.p = c.q[s->f.hp] / c.h;
    if (s->f.hpb >= 0) c.pb = c.q[s->f.hpb] / c.h;
  }
  return c;
}

static cell_t mirror_cell(cell_t c, int dir) {
  c.q[1 + dir] = -c.q[1 + dir];
  c.vel[dir] = -c.vel[dir];
  return c;
}

/* Roe-type interface state of Sec. 4: arithmetic means of h and c^2, sqrt(h)
 * weighted means of the primitives u, v, w, p (and sigma, p_b). */
typedef struct { double h, c2, vel[2], w, sg, p, pb; } roe_t;

static roe_t roe_average(const cell_t* L, const cell_t* R) {
  roe_t r;
  double sl = sqrt(L->h), sr = sqrt(R->h), den = sl + sr;
  r.h = 0.5 * (L->h + R->h);
  r.c2 = 0.5 * (L->c2 + R->c2);
  r.vel[0] = (sr * R->vel[0] + sl * L->vel[0]) / den;
  r.vel[1] = (sr * R->vel[1] + sl * L->vel[1]) / den;
  r.w = (sr * R->w + sl * L->w) / den;
  r.sg = (sr * R->sg + sl * L->sg) / den;
  r.p = (sr * R->p + sl * L->p) / den;
  r.pb = (sr * R->pb + sl * L->pb) / den;
  return r;
}

/* Right eigenvectors of App. C for the normal direction dir (0: x, 1: y; the
 * tangential velocity is the passive tracer).  Wave families, in order: the
 * left fast wave (speed s1), the pressure wave r2 = (1, u_n, 0.., -g h, ..)
 * when the model has p, one passive unit wave per passive field (tangential
 * momentum, hw, h sigma, h p_b), and the right fast wave (speed sN).
 * R is row-major (field, wave).  Speeds of r2 and of the passive waves: u_n. */
static void eig_matrix(const fields_t* f, int dir, const roe_t* r, double g, double s1,
                       double sN, double* R, double* spd) {
  int nv = f->nv, kn = 1 + dir, kt = 2 - dir;
  double K = r->c2 + r->p;
  memset(R, 0, sizeof(double) * nv * nv);
  int p = 0;
  /* fast left */
  R[0 * nv + p] = 1.0; R[kn * nv + p] = s1; R[kt * nv + p] = r->vel[1 - dir];
  if (f->hw >= 0) R[f->hw * nv + p] = r->w;
  if (f->hs >= 0) R[f->hs * nv + p] = r->sg;
  if (f->hp >= 0) R[f->hp * nv + p] = K;
  if (f->hpb >= 0) R[f->hpb * nv + p] = r->pb;
  spd[p++] = s1;
  if (f->hp >= 0) {
    R[0 * nv + p] = 1.0; R[kn * nv + p] = r->vel[dir]; R[f->hp * nv + p] = -g * r->h;
    spd[p++] = r->vel[dir];
  }
  int passive[4], np = 0;
  passive[np++] = kt;
  if (f->hw >= 0) passive[np++] = f->hw;
  if (f->hs >= 0) passive[np++] = f->hs;
  if (f->hpb >= 0) passive[np++] = f->hpb;
  for (int i = 0; i < np; i++) { R[passive[i] * nv + p] = 1.0; spd[p++] = r->vel[dir]; }
  /* fast right */
  R[0 * nv + p] = 1.0; R[kn * nv + p] = sN; R[kt * nv + p] = r->vel[1 - dir];
  if (f->hw >= 0) R[f->hw * nv + p] = r->w;
  if (f->hs >= 0) R[f->hs * nv + p] = r->sg;
  if (f->hp >= 0) R[f->hp * nv + p] = K;
  if (f->hpb >= 0) R[f->hpb * nv + p] = r->pb;
  spd[p++] = sN;
}

static double fast_speed2(double g, double h, double p, double c2) { return g * h + p + c2; }

/* Normal Riemann solver at the interface L|R in direction dir (Sec. 4):
 * total fluctuation of Eq. (total fluctuation) with the one-point quadrature of
 * the non-conservative products at the Roe state, the well-balanced bathymetry
 * terms with the sensor psi, Einfeldt speeds for the fast waves, and its
 * decomposition into f-waves proportional to the eigenvectors of App. C. */
static void normal_solve(or_solver* s, int dir, cell_t L, cell_t R, double dtdx, face_t* F) {
  const fields_t* f = &s->f;
  int nv = f->nv, kn = 1 + dir, kt = 2 - dir;
  double g = s->c.g;
  memset(F, 0, sizeof *F);
  int wetL = L.wet, wetR = R.wet;
  if (!wetL && !wetR) return;
  F->active = 1;
  F->first_order = !(wetL && wetR);
  if (wetL && !wetR && R.b > L.eta) { R = mirror_cell(L, dir); F->wall = 2; }
  else if (wetR && !wetL && L.b > R.eta) { L = mirror_cell(R, dir); F->wall = 1; }

  roe_t r = roe_average(&L, &R);
  double deta = R.eta - L.eta, db = R.b - L.b, dh = R.h - L.h;
  double psi = or_psi(R.b, L.b, s->c.xi0, s->c.xi1);
  double un = r.vel[dir];
  double cl2 = fast_speed2(g, L.h, L.p, L.c2), cr2 = fast_speed2(g, R.h, R.p, R.c2);
  double ch2 = fast_speed2(g, r.h, r.p, r.c2);
  if (cl2 < 0 || cr2 < 0 || ch2 < 0) set_status(s, OR_ST_NONHYP);
  double CL = sqrt(cl2 > 0 ? cl2 : 0), CR = sqrt(cr2 > 0 ? cr2 : 0), CH = sqrt(ch2 > 0 ? ch2 : 0);
  double s1 = fmin(un - CH, L.vel[dir] - CL);
  double sN = fmax(un + CH, R.vel[dir] + CR);

  /* total fluctuation delta = dF + A(Qhat) dQ + B dB (Sec. 4) */
  double d[NVMAX] = {0};
  double hnL = L.q[kn], hnR = R.q[kn];
  d[0] = hnR - hnL;
  double hpL = f->hp >= 0 ? L.q[f->hp] : 0.0, hpR = f->hp >= 0 ? R.q[f->hp] : 0.0;
  d[kn] = (hnR * R.vel[dir] + hpR) - (hnL * L.vel[dir] + hpL) + g * r.h * deta;
  if (s->c.model == OR_MBHSGN) d[kn] += 1.5 * psi * r.p * db;
  if (s->c.model == OR_HSGN) d[kn] += psi * r.pb * db;
  d[kt] = hnR * R.vel[1 - dir] - hnL * L.vel[1 - dir];
  if (f->hw >= 0) d[f->hw] = hnR * R.w - hnL * L.w;
  if (f->hs >= 0) d[f->hs] = hnR * R.sg - hnL * L.sg;
  if (f->hp >= 0) {
    /* relaxation term h c^2 d_x u of Eq. (mbHSGN) kept non-conservative in c^2
     * (reading G24): c^2 multiplies the jump of hu at the Roe state, so that a
     * jump of c^2 (the SWE transition) adds no hu d_x(c^2) term */
    d[f->hp] = hnR * R.p - hnL * L.p + r.c2 * (hnR - hnL);
    if (s->c.model == OR_MBHSGN) d[f->hp] -= r.c2 * un * (deta + psi * db);
    else d[f->hp] -= r.c2 * un * dh;
  }
  if (f->hpb >= 0) d[f->hpb] = hnR * R.pb - hnL * L.pb - 6.0 * r.c2 * un * psi * db;

  double Rm[NVMAX * NVMAX], spd[NVMAX], beta[NVMAX];
  eig_matrix(f, dir, &r, g, s1, sN, Rm, spd);
  if (solve_dense(nv, Rm, d, beta)) { memset(beta, 0, sizeof beta); set_status(s, OR_ST_NONHYP); }
  for (int k = 0; k < nv; k++) F->d[k] = d[k];
  for (int p = 0; p < nv; p++) {
    F->s[p] = spd[p];
    for (int k = 0; k < nv; k++) F->Z[p][k] = beta[p] * Rm[k * nv + p];
  }
  for (int k = 0; k < nv; k++) {
    double am = 0.0, ap = 0.0;
    for (int p = 0; p < nv; p++) {
      if (F->s[p] < 0) am += F->Z[p][k];
      else if (F->s[p] > 0) ap += F->Z[p][k];
      else { am += 0.5 * F->Z[p][k]; ap += 0.5 * F->Z[p][k]; }
    }
    F->Am[k] = am; F->Ap[k] = ap;
  }
  F->Fhat = hnL + F->Am[0];
  if (F->wall == 2) { for (int k = 0; k < nv; k++) F->Ap[k] = 0.0; F->Fhat = 0.0; }
  if (F->wall == 1) { for (int k = 0; k < nv; k++) F->Am[k] = 0.0; F->Fhat = 0.0; }
  (void)dtdx;
}

/* Wave limiter (Sec. 4: minmod or MC) and the second-order correction flux
 * Ftil = 1/2 sum_p sgn(s_p) (1 - dt/dx |s_p|) phi(theta_p) Z_p, with theta the
 * ratio of the upwind wave projected on the local wave. */
static double limiter_fn(int kind, double th) {
  if (kind == OR_LIM_MINMOD) return fmax(0.0, fmin(1.0, th));
  double a = fmin(0.5 * (1.0 + th), fmin(2.0, 2.0 * th));
  return fmax(0.0, a);
}

static void limit_face(or_solver* s, face_t* F, const face_t* Fm, const face_t* Fp, double dtdx) {
  int nv = s->f.nv;
  for (int k = 0; k < nv; k++) F->Ftil[k] = 0.0;
  if (F->active && !F->first_order && s->c.limiter != OR_LIM_NONE) {
    for (int p = 0; p < nv; p++) {
      double sp = F->s[p];
      if (sp == 0.0) continue;
      const face_t* U = sp > 0 ? Fm : Fp;
      double zz = 0.0, zu = 0.0;
      for (int k = 0; k < nv; k++) { zz += F->Z[p][k] * F->Z[p][k]; zu += U->Z[p][k] * F->Z[p][k]; }
      double phi = zz > 0.0 ? limiter_fn(s->c.limiter, zu / zz) : 0.0;
      double sg = sp > 0 ? 1.0 : -1.0;
      double cf = 0.5 * sg * (1.0 - dtdx * fabs(sp)) * phi;
      for (int k = 0; k < nv; k++) F->Ftil[k] += cf * F->Z[p][k];
    }
  }
  for (int k = 0; k < nv; k++) {
    F->Lv[k] = F->Am[k] + F->Ftil[k];
    F->Rv[k] = F->Ap[k] - F->Ftil[k];
  }
  F->M = F->Fhat + F->Ftil[0];
}

/* Transverse split (reading G8): A^+ Vl + A^- Vr in direction dir at the Roe
 * state of the two cells, with the exact eigenvalues u_n -+ C of App. C. */
static void transverse_split(or_solver* s, int dir, const cell_t* L, const cell_t* R,
                             const double* Vl, const double* Vr, double* out) {
  const fields_t* f = &s->f;
  int nv = f->nv;
  roe_t r = roe_average(L, R);
  double ch2 = fast_speed2(s->c.g, r.h, r.p, r.c2);
  double CH = sqrt(ch2 > 0 ? ch2 : 0);
  double un = r.vel[dir];
  double Rm[NVMAX * NVMAX], lam[NVMAX], bl[NVMAX], br[NVMAX];
  eig_matrix(f, dir, &r, s->c.g, un - CH, un + CH, Rm, lam);
  for (int k = 0; k < nv; k++) out[k] = 0.0;
  if (solve_dense(nv, Rm, Vl, bl) || solve_dense(nv, Rm, Vr, br)) { set_status(s, OR_ST_NONHYP); return; }
  for (int p = 0; p < nv; p++) {
    double cp = fmax(lam[p], 0.0) * bl[p] + fmin(lam[p], 0.0) * br[p];
    for (int k = 0; k < nv; k++) out[k] += cp * Rm[k * nv + p];
  }
}

/* ------------------------------------------------------------------------- */
/* Transition function phi_T of Eq. (transition_function), reading G11, and the
 * space-varying relaxation parameter c^2 = alpha^2 g H phi_T (reading G1). */
static void setup_aux(or_solver* s, const unsigned char* phi_override) {
  int nx = s->c.nx, ny = s->c.ny, n = s->c.n_transition;
  double dx = s->c.dx, dy = s->c.dy;
  for (int J = NG; J < NG + ny; J++)
    for (int I = NG; I < NG + nx; I++) {
      unsigned char ph;
      if (phi_override) ph = phi_override[(size_t)(J - NG) * nx + (I - NG)] ? 1 : 0;
      else {
        double mn = INFINITY;
        for (int dj = -n; dj <= n; dj++)
          for (int di = -n; di <= n; di++) {
            if ((di * dx) * (di * dx) + (dj * dy) * (dj * dy) > (n * dx) * (n * dx)) continue;
            double H = -s->b[cidx(s, I + di, J + dj)];
            if (H < 0.0) H = 0.0;
            if (H < mn) mn = H;
          }
        ph = mn > s->c.h_star ? 1 : 0;
      }
      s->phi[cidx(s, I, J)] = ph;
    }
  fill_ghosts_u8(s, s->phi);
  for (int J = NG; J < NG + ny; J++)
    for (int I = NG; I < NG + nx; I++) {
      size_t id = cidx(s, I, J);
      double H = -s->b[id]; if (H < 0.0) H = 0.0;
      s->c2[id] = s->c.alpha * s->c.alpha * s->c.g * H * (double)s->phi[id];
    }
  fill_ghosts(s, s->c2, 1, 0);
}

or_solver* or_create(const or_config* cfg, const double* b, const unsigned char* phi_override) {
  if (!cfg || !b) return NULL;
  if (cfg->nx < 2 || cfg->ny < 2 || !(cfg->dx > 0) || !(cfg->dy > 0)) return NULL;
  if (cfg->model < 0 || cfg->model > 2) return NULL;
  if (cfg->n_transition < 0 || cfg->n_transition > NG) return NULL;
  for (int i = 0; i < 4; i++) if (cfg->bc[i] < 0 || cfg->bc[i] > 2) return NULL;
  if ((cfg->bc[0] == OR_BC_PERIODIC) != (cfg->bc[1] == OR_BC_PERIODIC)) return NULL;
  if ((cfg->bc[2] == OR_BC_PERIODIC) != (cfg->bc[3] == OR_BC_PERIODIC)) return NULL;
  or_solver* s = (or_solver*)calloc(1, sizeof *s);
  s->c = *cfg;
  s->f = model_fields(cfg->model);
  s->nxp = cfg->nx + 2 * NG; s->nyp = cfg->ny + 2 * NG;
  size_t np = (size_t)s->nxp * s->nyp;
  s->q = (double*)calloc(np * s->f.nv, sizeof(double));
  s->b = (double*)calloc(np, sizeof(double));
  s->c2 = (double*)calloc(np, sizeof(double));
  s->phi = (unsigned char*)calloc(np, 1);
  s->theta = (double*)calloc(np, sizeof(double));
  s->fx = (face_t*)calloc((size_t)(s->nxp + 1) * s->nyp, sizeof(face_t));
  s->fy = (face_t*)calloc((size_t)s->nxp * (s->nyp + 1), sizeof(face_t));
  if (!s->q || !s->b || !s->c2 || !s->phi || !s->theta || !s->fx || !s->fy) { or_destroy(s); return NULL; }
  for (int j = 0; j < cfg->ny; j++)
    for (int i = 0; i < cfg->nx; i++) s->b[cidx(s, i + NG, j + NG)] = b[(size_t)j * cfg->nx + i];
  fill_ghosts(s, s->b, 1, 0);
  setup_aux(s, phi_override);
  /* still water at rest: eta = max(0, b) so that h = max(0, -b) */
  for (size_t i = 0; i < np; i++) s->q[i] = s->b[i] > 0 ? s->b[i] : 0.0;
  return s;
}

void or_destroy(or_solver* s) {
  if (!s) return;
  free(s->q); free(s->b); free(s->c2); free(s->phi); free(s->theta);
  free(s->fx); free(s->fy); free(s->gidx); free(s->grec_buf);
  free(s);
}

int or_nvar(const or_solver* s) { return s->f.nv; }

int or_set_state(or_solver* s, const double* q, double t) {
  if (!s || !q) return -1;
  int nx = s->c.nx, ny = s->c.ny;
  for (int k = 0; k < s->f.nv; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++)
        fld(s, k)[cidx(s, i + NG, j + NG)] = q[((size_t)k * ny + j) * nx + i];
  /* every state the solver holds satisfies the SWE/dry switch (Sec. 3.3) */
  for (int J = NG; J < NG + ny; J++)
    for (int I = NG; I < NG + nx; I++) source_cell(s, I, J, 0.0);
  s->t = t; s->status = 0; s->grec = 0;
  return 0;
}

int or_get_state(const or_solver* s, double* q, double* t) {
  if (!s || !q) return -1;
  int nx = s->c.nx, ny = s->c.ny;
  for (int k = 0; k < s->f.nv; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++)
        q[((size_t)k * ny + j) * nx + i] = s->q[(size_t)k * s->nxp * s->nyp + cidx(s, i + NG, j + NG)];
  if (t) *t = s->t;
  return 0;
}

/* Replace the relaxation parameter c^2 of the interior cells (ny*nx, copied;
 * the constant-c^2 setting of the steady-state test of Sec. 5.3, Table 3);
 * ghost cells follow the boundary conditions. */
int or_set_c2(or_solver* s, const double* c2) {
  if (!s || !c2) return -1;
  for (int j = 0; j < s->c.ny; j++)
    for (int i = 0; i < s->c.nx; i++) {
      double v = c2[(size_t)j * s->c.nx + i];
      if (!(v >= 0.0)) return -1;
      s->c2[cidx(s, i + NG, j + NG)] = v;
    }
  fill_ghosts(s, s->c2, 1, 0);
  return 0;
}

int or_get_aux(const or_solver* s, double* c2, unsigned char* phi) {
  int nx = s->c.nx, ny = s->c.ny;
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      size_t id = cidx(s, i + NG, j + NG);
      if (c2) c2[(size_t)j * nx + i] = s->c2[id];
      if (phi) phi[(size_t)j * nx + i] = s->phi[id];
    }
  return 0;
}

/* CFL time step from the cell speeds, Eq. (eigenvalue_bound) and Sec. 4:
 * dt = CFL / max over wet cells of max((|u| + C_e)/dx, (|v| + C_e)/dy). */
double or_dt_cfl(or_solver* s) {
  double smax = 0.0; int anywet = 0;
  for (int J = NG; J < NG + s->c.ny; J++)
    for (int I = NG; I < NG + s->c.nx; I++) {
      cell_t c = load_cell(s, I, J);
      if (!c.wet) continue;
      anywet = 1;
      double c2e = fast_speed2(s->c.g, c.h, c.p, c.c2);
      if (c2e < 0) { s->status |= OR_ST_NONHYP; c2e = 0; }
      double C = sqrt(c2e);
      double sx = (fabs(c.vel[0]) + C) / s->c.dx, sy = (fabs(c.vel[1]) + C) / s->c.dy;
      double sp = sx > sy ? sx : sy;
      if (sp > smax) smax = sp;
    }
  if (!anywet || !(smax > 0)) { s->status |= OR_ST_ALLDRY; return 0.0; }
  return s->c.cfl / smax;
}

/* One time step: S(dt/2) H(dt) S(dt/2) (Strang) or H(dt) S(dt) (Lie), Sec. 4,
 * in two phases: step_begin runs everything up to the positivity factors,
 * step_end the update and the second source step.  A patch of a refined level
 * exchanges the factors of its ghost cells in between. */
static void step_begin(or_solver* s, double dt) {
  int nx = s->c.nx, ny = s->c.ny, nxp = s->nxp, nyp = s->nyp, nv = s->f.nv;
  double dtdx = dt / s->c.dx, dtdy = dt / s->c.dy;
  double tau1 = s->c.strang ? 0.5 * dt : 0.0;

  /* 1. ghost cells, 2. first source half step on every cell */
  fill_ghosts(s, s->q, nv, 1);
#pragma omp parallel for schedule(static)
  for (int J = 0; J < nyp; J++)
    for (int I = 0; I < nxp; I++) source_cell(s, I, J, tau1);

  /* 3. normal Riemann problems: x faces I (between I-1 and I), y faces J */
#pragma omp parallel for schedule(static)
  for (int J = 0; J < nyp; J++)
    for (int I = 1; I < nxp; I++)
      normal_solve(s, 0, load_cell(s, I - 1, J), load_cell(s, I, J), dtdx, &s->fx[(size_t)J * (nxp + 1) + I]);
#pragma omp parallel for schedule(static)
  for (int J = 1; J < nyp; J++)
    for (int I = 0; I < nxp; I++)
      normal_solve(s, 1, load_cell(s, I, J - 1), load_cell(s, I, J), dtdy, &s->fy[(size_t)J * nxp + I]);

  /* 4. limiters and second-order corrections */
#pragma omp parallel for schedule(static)
  for (int J = 0; J < nyp; J++)
    for (int I = 2; I < nxp - 1; I++) {
      face_t* F = &s->fx[(size_t)J * (nxp + 1) + I];
      limit_face(s, F, F - 1, F + 1, dtdx);
    }
#pragma omp parallel for schedule(static)
  for (int J = 2; J < nyp - 1; J++)
    for (int I = 0; I < nxp; I++) {
      face_t* F = &s->fy[(size_t)J * nxp + I];
      limit_face(s, F, F - nxp, F + nxp, dtdy);
    }

  /* Courant number of this step from the face speeds (reading G15) */
  double cmax = 0.0;
  for (int J = NG; J < NG + ny; J++)
    for (int I = NG; I <= NG + nx; I++) {
      face_t* F = &s->fx[(size_t)J * (nxp + 1) + I];
      if (!F->active) continue;
      for (int p = 0; p < nv; p++) cmax = fmax(cmax, fabs(F->s[p]) * dtdx);
    }
  for (int J = NG; J <= NG + ny; J++)
    for (int I = NG; I < NG + nx; I++) {
      face_t* F = &s->fy[(size_t)J * nxp + I];
      if (!F->active) continue;
      for (int p = 0; p < nv; p++) cmax = fmax(cmax, fabs(F->s[p]) * dtdy);
    }
  s->max_courant = cmax;
  if (cmax > 1.0) s->status |= OR_ST_CFL;

  /* 5. transverse propagation (reading G8) at the faces of interior cells */
#pragma omp parallel for schedule(static)
  for (int J = NG; J < NG + ny; J++)
    for (int I = NG; I <= NG + nx; I++) {
      face_t* F = &s->fx[(size_t)J * (nxp + 1) + I];
      for (int k = 0; k < nv; k++) F->Pt[k] = 0.0;
      cell_t L = load_cell(s, I - 1, J), R = load_cell(s, I, J);
      if (L.wet && R.wet) {
        double Vl[NVMAX], Vr[NVMAX], out[NVMAX];
        const face_t* bl = &s->fy[(size_t)J * nxp + (I - 1)];
        const face_t* tl = &s->fy[(size_t)(J + 1) * nxp + (I - 1)];
        const face_t* br = &s->fy[(size_t)J * nxp + I];
        const face_t* tr = &s->fy[(size_t)(J + 1) * nxp + I];
        for (int k = 0; k < nv; k++) { Vl[k] = bl->Rv[k] + tl->Lv[k]; Vr[k] = br->Rv[k] + tr->Lv[k]; }
        transverse_split(s, 0, &L, &R, Vl, Vr, out);
        for (int k = 0; k < nv; k++) F->Pt[k] = -0.5 * dtdy * out[k];
      }
    }
#pragma omp parallel for schedule(static)
  for (int J = NG; J <= NG + ny; J++)
    for (int I = NG; I < NG + nx; I++) {
      face_t* F = &s->fy[(size_t)J * nxp + I];
      for (int k = 0; k < nv; k++) F->Pt[k] = 0.0;
      cell_t B = load_cell(s, I, J - 1), T = load_cell(s, I, J);
      if (B.wet && T.wet) {
        double Vb[NVMAX], Vt[NVMAX], out[NVMAX];
        const face_t* lb = &s->fx[(size_t)(J - 1) * (nxp + 1) + I];
        const face_t* rb = &s->fx[(size_t)(J - 1) * (nxp + 1) + I + 1];
        const face_t* lt = &s->fx[(size_t)J * (nxp + 1) + I];
        const face_t* rt = &s->fx[(size_t)J * (nxp + 1) + I + 1];
        for (int k = 0; k < nv; k++) { Vb[k] = lb->Rv[k] + rb->Lv[k]; Vt[k] = lt->Rv[k] + rt->Lv[k]; }
        transverse_split(s, 1, &B, &T, Vb, Vt, out);
        for (int k = 0; k < nv; k++) F->Pt[k] = -0.5 * dtdx * out[k];
      }
    }

  /* 6. draining-time positivity guard (reading G14): theta_c = h_c / outflow_c
   * when the outflow of mass in this step exceeds the water in the cell. */
  for (size_t i = 0; i < (size_t)nxp * nyp; i++) s->theta[i] = 1.0;
#pragma omp parallel for schedule(static)
  for (int J = NG; J < NG + ny; J++)
    for (int I = NG; I < NG + nx; I++) {
      double Ml = s->fx[(size_t)J * (nxp + 1) + I].M + s->fx[(size_t)J * (nxp + 1) + I].Pt[0];
      double Mr = s->fx[(size_t)J * (nxp + 1) + I + 1].M + s->fx[(size_t)J * (nxp + 1) + I + 1].Pt[0];
      double Mb = s->fy[(size_t)J * nxp + I].M + s->fy[(size_t)J * nxp + I].Pt[0];
      double Mt = s->fy[(size_t)(J + 1) * nxp + I].M + s->fy[(size_t)(J + 1) * nxp + I].Pt[0];
      double out = dtdx * (fmax(Mr, 0.0) + fmax(-Ml, 0.0)) + dtdy * (fmax(Mt, 0.0) + fmax(-Mb, 0.0));
      size_t id = cidx(s, I, J);
      double h = fld(s, 0)[id] - s->b[id]; if (h < 0.0) h = 0.0;
      s->theta[id] = out > h ? h / out : 1.0;
    }
}

static int step_end(or_solver* s, double dt) {
  int nx = s->c.nx, ny = s->c.ny, nxp = s->nxp, nv = s->f.nv;
  double dtdx = dt / s->c.dx, dtdy = dt / s->c.dy;
  double tau2 = s->c.strang ? 0.5 * dt : dt;

  /* 7. conservative update of the interior cells (Sec. 4, wave propagation
   * form; the mass row in flux form so that it telescopes) */
  double* qn = (double*)malloc(sizeof(double) * (size_t)nv * nx * ny);
  unsigned st = 0;
#pragma omp parallel for schedule(static) reduction(| : st)
  for (int J = NG; J < NG + ny; J++)
    for (int I = NG; I < NG + nx; I++) {
      const face_t* Fl = &s->fx[(size_t)J * (nxp + 1) + I];
      const face_t* Fr = Fl + 1;
      const face_t* Gb = &s->fy[(size_t)J * nxp + I];
      const face_t* Gt = Gb + nxp;
      double Ml = Fl->M + Fl->Pt[0], Mr = Fr->M + Fr->Pt[0];
      double Mb = Gb->M + Gb->Pt[0], Mt = Gt->M + Gt->Pt[0];
      double tl = Ml > 0 ? s->theta[cidx(s, I - 1, J)] : (Ml < 0 ? s->theta[cidx(s, I, J)] : 1.0);
      double tr = Mr > 0 ? s->theta[cidx(s, I, J)] : (Mr < 0 ? s->theta[cidx(s, I + 1, J)] : 1.0);
      double tb = Mb > 0 ? s->theta[cidx(s, I, J - 1)] : (Mb < 0 ? s->theta[cidx(s, I, J)] : 1.0);
      double tt = Mt > 0 ? s->theta[cidx(s, I, J)] : (Mt < 0 ? s->theta[cidx(s, I, J + 1)] : 1.0);
      size_t id = cidx(s, I, J);
      size_t od = (size_t)(J - NG) * nx + (I - NG);
      double eta = fld(s, 0)[id];
      double en = eta - dtdx * (tr * Mr - tl * Ml) - dtdy * (tt * Mt - tb * Mb);
      qn[od] = en;
      for (int k = 1; k < nv; k++) {
        double v = fld(s, k)[id]
                 - dtdx * (tl * (Fl->Rv[k] - Fl->Pt[k]) + tr * (Fr->Lv[k] + Fr->Pt[k]))
                 - dtdy * (tb * (Gb->Rv[k] - Gb->Pt[k]) + tt * (Gt->Lv[k] + Gt->Pt[k]));
        qn[(size_t)k * nx * ny + od] = v;
        if (!isfinite(v)) st |= OR_ST_NONFINITE;
      }
      if (!isfinite(en)) st |= OR_ST_NONFINITE;
      double hb = s->b[id];
      double tol = 1e-12 * (1.0 + fabs(hb));
      if (en - hb < -tol) st |= OR_ST_NEGDEPTH;
    }
  s->status |= st;
  for (int k = 0; k < nv; k++)
    for (int J = NG; J < NG + ny; J++)
      for (int I = NG; I < NG + nx; I++)
        fld(s, k)[cidx(s, I, J)] = qn[(size_t)k * nx * ny + (size_t)(J - NG) * nx + (I - NG)];
  free(qn);

  /* 8. second source half step and SWE switch on the interior cells */
#pragma omp parallel for schedule(static)
  for (int J = NG; J < NG + ny; J++)
    for (int I = NG; I < NG + nx; I++) source_cell(s, I, J, tau2);

  s->t += dt;
  s->last_dt = dt;
  /* gauges: the cell containing each gauge (reading G20) */
  if (s->ngauge > 0) {
    if (s->grec < s->gcap) {
      double* r = s->grec_buf + (size_t)s->grec * s->ngauge * 4;
      for (int gi = 0; gi < s->ngauge; gi++) {
        size_t id = (size_t)s->gidx[gi];
        r[gi * 4 + 0] = s->t; r[gi * 4 + 1] = fld(s, 0)[id];
        r[gi * 4 + 2] = fld(s, 1)[id]; r[gi * 4 + 3] = fld(s, 2)[id];
      }
      s->grec++;
    } else s->status |= OR_ST_GAUGE_FULL;
  }
  return (s->status & (OR_ST_NEGDEPTH | OR_ST_NONFINITE | OR_ST_CFL | OR_ST_NONHYP | OR_ST_ALLDRY)) ? -1 : 0;
}

static int step_once(or_solver* s, double dt) {
  step_begin(s, dt);
  return step_end(s, dt);
}

int or_step(or_solver* s, int nsteps) {
  for (int n = 0; n < nsteps; n++) {
    double dt = or_dt_cfl(s);
    if (s->status & OR_ST_ALLDRY) return -1;
    if (step_once(s, dt)) return -1;
  }
  return 0;
}

int or_step_dt(or_solver* s, double dt) {
  if (!(dt > 0)) return -1;
  return step_once(s, dt);
}

double or_mass(const or_solver* s) {
  double m = 0.0;
  for (int J = NG; J < NG + s->c.ny; J++)
    for (int I = NG; I < NG + s->c.nx; I++) {
      size_t id = cidx(s, I, J);
      double h = s->q[id] - s->b[id];
      m += h > 0 ? h : 0.0;
    }
  return m * s->c.dx * s->c.dy;
}

unsigned or_status(const or_solver* s) { return s->status; }
double or_last_dt(const or_solver* s) { return s->last_dt; }
double or_max_courant(const or_solver* s) { return s->max_courant; }

int or_add_gauges(or_solver* s, const double* xy, int n, int capacity) {
  if (!s || n < 0 || (n > 0 && !xy) || capacity < 0) return -1;
  free(s->gidx); free(s->grec_buf);
  s->gidx = (int*)calloc(n > 0 ? n : 1, sizeof(int));
  s->grec_buf = (double*)calloc((size_t)(n > 0 ? n : 1) * 4 * (capacity > 0 ? capacity : 1), sizeof(double));
  for (int g = 0; g < n; g++) {
    double fx = (xy[2 * g] - s->c.x0) / s->c.dx, fy = (xy[2 * g + 1] - s->c.y0) / s->c.dy;
    int i = (int)floor(fx), j = (int)floor(fy);
    if (i < 0 || j < 0 || i >= s->c.nx || j >= s->c.ny) return -1;
    s->gidx[g] = (int)cidx(s, i + NG, j + NG);
  }
  s->ngauge = n; s->gcap = capacity; s->grec = 0;
  return 0;
}

int or_gauges(const or_solver* s, double* out, size_t cap) {
  size_t need = (size_t)s->grec * s->ngauge * 4;
  if (out && cap >= need) memcpy(out, s->grec_buf, need * sizeof(double));
  return s->grec;
}

/* ---- pieces exposed for the pin tests ---------------------------------- */
/* ------------------------------------------------------------------------- */
/* Patch mode (block-structured refinement of Sec. 4): the caller owns the
 * ghost frame.  b_frame and phi_frame cover the padded patch, (ny+4) x (nx+4)
 * cells; c^2 = alpha^2 g max(-b, 0) phi_T of every cell (reading G1). */
or_solver* or_create_frame(const or_config* cfg, const double* b_frame, const unsigned char* phi_frame) {
  if (!cfg || !b_frame || !phi_frame) return NULL;
  if (cfg->nx < 2 || cfg->ny < 2 || !(cfg->dx > 0) || !(cfg->dy > 0)) return NULL;
  if (cfg->model < 0 || cfg->model > 2) return NULL;
  or_solver* s = (or_solver*)calloc(1, sizeof *s);
  s->c = *cfg;
  s->frame = 1;
  s->f = model_fields(cfg->model);
  s->nxp = cfg->nx + 2 * NG; s->nyp = cfg->ny + 2 * NG;
  size_t np = (size_t)s->nxp * s->nyp;
  s->q = (double*)calloc(np * s->f.nv, sizeof(double));
  s->b = (double*)calloc(np, sizeof(double));
  s->c2 = (double*)calloc(np, sizeof(double));
  s->phi = (unsigned char*)calloc(np, 1);
  s->theta = (double*)calloc(np, sizeof(double));
  s->fx = (face_t*)calloc((size_t)(s->nxp + 1) * s->nyp, sizeof(face_t));
  s->fy = (face_t*)calloc((size_t)s->nxp * (s->nyp + 1), sizeof(face_t));
  if (!s->q || !s->b || !s->c2 || !s->phi || !s->theta || !s->fx || !s->fy) { or_destroy(s); return NULL; }
  for (size_t i = 0; i < np; i++) {
    s->b[i] = b_frame[i];
    s->phi[i] = phi_frame[i] ? 1 : 0;
    double H = -s->b[i]; if (H < 0.0) H = 0.0;
    s->c2[i] = s->c.alpha * s->c.alpha * s->c.g * H * (double)s->phi[i];
    s->q[i] = s->b[i] > 0 ? s->b[i] : 0.0;
  }
  return s;
}

/* The whole padded state (nv fields of (ny+4) x (nx+4)), copied as given. */
int or_set_frame(or_solver* s, const double* q, double t) {
  if (!s || !q) return -1;
  memcpy(s->q, q, sizeof(double) * (size_t)s->f.nv * s->nxp * s->nyp);
  s->t = t;
  return 0;
}

int or_get_frame(const or_solver* s, double* q) {
  if (!s || !q) return -1;
  memcpy(q, s->q, sizeof(double) * (size_t)s->f.nv * s->nxp * s->nyp);
  return 0;
}

int or_step_begin(or_solver* s, double dt) {
  if (!s || !(dt > 0)) return -1;
  step_begin(s, dt);
  return 0;
}

int or_step_end(or_solver* s, double dt) {
  if (!s || !(dt > 0)) return -1;
  return step_end(s, dt);
}

/* Positivity factors of the padded cells (1 outside the interior unless set). */
int or_get_theta(const or_solver* s, double* th) {
  if (!s || !th) return -1;
  memcpy(th, s->theta, sizeof(double) * (size_t)s->nxp * s->nyp);
  return 0;
}

int or_set_theta(or_solver* s, const double* th) {
  if (!s || !th) return -1;
  memcpy(s->theta, th, sizeof(double) * (size_t)s->nxp * s->nyp);
  return 0;
}

/* Mass flux through the faces of the interior cells as the update applies it:
 * theta of the cell the water leaves times (M + the transverse mass term).
 * dir 0: x faces, ny rows of nx+1 faces (face i between cells i-1 and i);
 * dir 1: y faces, ny+1 rows of nx faces.  Valid after or_step_begin (and the
 * exchange of theta), until the next step. */
int or_face_mass(const or_solver* s, int dir, double* out) {
  if (!s || !out || dir < 0 || dir > 1) return -1;
  int nx = s->c.nx, ny = s->c.ny, nxp = s->nxp;
  if (dir == 0) {
    for (int j = 0; j < ny; j++)
      for (int i = 0; i <= nx; i++) {
        int I = i + NG, J = j + NG;
        const face_t* F = &s->fx[(size_t)J * (nxp + 1) + I];
        double M = F->M + F->Pt[0];
        double t = M > 0 ? s->theta[cidx(s, I - 1, J)] : (M < 0 ? s->theta[cidx(s, I, J)] : 1.0);
        out[(size_t)j * (nx + 1) + i] = t * M;
      }
  } else {
    for (int j = 0; j <= ny; j++)
      for (int i = 0; i < nx; i++) {
        int I = i + NG, J = j + NG;
        const face_t* F = &s->fy[(size_t)J * nxp + I];
        double M = F->M + F->Pt[0];
        double t = M > 0 ? s->theta[cidx(s, I, J - 1)] : (M < 0 ? s->theta[cidx(s, I, J)] : 1.0);
        out[(size_t)j * nx + i] = t * M;
      }
  }
  return 0;
}

/* Largest cell speed max((|u| + C_e)/dx, (|v| + C_e)/dy) over the wet interior
 * cells, Eq. (eigenvalue_bound) (0 if none is wet). */
double or_max_speed(or_solver* s) {
  double smax = 0.0;
  for (int J = NG; J < NG + s->c.ny; J++)
    for (int I = NG; I < NG + s->c.nx; I++) {
      cell_t c = load_cell(s, I, J);
      if (!c.wet) continue;
      double c2e = fast_speed2(s->c.g, c.h, c.p, c.c2);
      if (c2e < 0) { s->status |= OR_ST_NONHYP; c2e = 0; }
      double C = sqrt(c2e);
      double sx = (fabs(c.vel[0]) + C) / s->c.dx, sy = (fabs(c.vel[1]) + C) / s->c.dy;
      double sp = sx > sy ? sx : sy;
      if (sp > smax) smax = sp;
    }
  return smax;
}

int or_eigvecs(int model, const double* roe, double g, double s1, double sN, double* R) {
  fields_t f = model_fields(model);
  roe_t r = {roe[0], roe[7], {roe[1], roe[2]}, roe[3], roe[4], roe[5], roe[6]};
  double spd[NVMAX];
  eig_matrix(&f, 0, &r, g, s1, sN, R, spd);
  return f.nv;
}

/* Jacobian dF/dq + A (x-direction, passive v) of the quasi-linear form of
 * Eq. (mbHSGN) / Eq. (HSGN) at (h, u, v, w, sigma, p, pb, c2). */
int or_jacobian(int model, const double* st, double g, double* J) {
  fields_t f = model_fields(model);
  int n = f.nv;
  double h = st[0], u = st[1], v = st[2], w = st[3], sg = st[4], p = st[5], pb = st[6], c2 = st[7];
  memset(J, 0, sizeof(double) * n * n);
  J[0 * n + 1] = 1.0;
  J[1 * n + 0] = g * h - u * u; J[1 * n + 1] = 2.0 * u;
  if (f.hp >= 0) J[1 * n + f.hp] = 1.0;
  J[2 * n + 0] = -u * v; J[2 * n + 1] = v; J[2 * n + 2] = u;
  if (f.hw >= 0) { J[f.hw * n + 0] = -u * w; J[f.hw * n + 1] = w; J[f.hw * n + f.hw] = u; }
  if (f.hs >= 0) { J[f.hs * n + 0] = -u * sg; J[f.hs * n + 1] = sg; J[f.hs * n + f.hs] = u; }
  if (f.hp >= 0) { J[f.hp * n + 0] = -c2 * u - p * u; J[f.hp * n + 1] = c2 + p; J[f.hp * n + f.hp] = u; }
  if (f.hpb >= 0) { J[f.hpb * n + 0] = -u * pb; J[f.hpb * n + 1] = pb; J[f.hpb * n + f.hpb] = u; }
  return n;
}

int or_face(const or_config* cfg, const double* qL, const double* qR, double bL, double bR,
            double c2L, double c2R, double* Z, double* s_out, double* Am, double* Ap,
            double* delta, double* Fhat) {
  or_solver tmp; memset(&tmp, 0, sizeof tmp);
  tmp.c = *cfg; tmp.f = model_fields(cfg->model);
  int nv = tmp.f.nv;
  /* build the two cells the way load_cell does */
  cell_t c[2]; const double* qs[2] = {qL, qR}; double bs[2] = {bL, bR}, cs[2] = {c2L, c2R};
  for (int i = 0; i < 2; i++) {
    memset(&c[i], 0, sizeof c[i]);
    c[i].eta = qs[i][0]; c[i].b = bs[i]; c[i].c2 = cs[i];
    c[i].h = c[i].eta - c[i].b; if (c[i].h < 0) c[i].h = 0;
    c[i].wet = c[i].h > cfg->dry_tol;
    c[i].q[0] = c[i].eta;
    for (int k = 1; k < nv; k++) c[i].q[k] = c[i].wet ? qs[i][k] : 0.0;
    if (c[i].wet) {
      c[i].vel[0] = c[i].q[1] / c[i].h; c[i].vel[1] = c[i].q[2] / c[i].h;
      if (tmp.f.hw >= 0) c[i].w = c[i].q[tmp.f.hw] / c[i].h;
      if (tmp.f.hs >= 0) c[i].sg = c[i].q[tmp.f.hs] / c[i].h;
      if (tmp.f.hp >= 0) c[i].p = c[i].q[tmp.f.hp] / c[i].h;
      if (tmp.f.hpb >= 0) c[i].pb = c[i].q[tmp.f.hpb] / c[i].h;
    }
  }
  face_t F;
  normal_solve(&tmp, 0, c[0], c[1], 0.0, &F);
  for (int p = 0; p < nv; p++) {
    if (s_out) s_out[p] = F.s[p];
    for (int k = 0; k < nv; k++) if (Z) Z[p * nv + k] = F.Z[p][k];
  }
  for (int k = 0; k < nv; k++) {
    if (Am) Am[k] = F.Am[k];
    if (Ap) Ap[k] = F.Ap[k];
  }
  if (delta) for (int k = 0; k < nv; k++) delta[k] = F.d[k];
  if (Fhat) *Fhat = F.Fhat;
  return F.active ? nv : 0;
}
