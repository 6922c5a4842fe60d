// sgn_amr.cuh -- refined hierarchy (block-structured AMR, Sec. 4 of the paper:
// patches, refinement ratio r, subcycling in time).
//
// Each level is one padded "atlas" grid holding all of its patches (runs of
// patches with the same rows that abut in x share one ghost frame; the
// regions' frames are packed on shelves), stepped with a kind mask (patch
// interior / covered / sibling ghost / exported cell): every stage is one
// launch over all patches of the level.
//
// Mixed precision: the frames are three cells deep and each level step (on a
// level whose atlas is large enough to fill the GPU) is ONE launch of the
// one-pass kernel k_step_fused over the atlas: it computes the positivity
// factors of the sibling ghosts next to a patch edge itself (the third layer
// makes them equal to the sibling's own) and writes the theta-weighted mass
// fluxes of the cells beside coarse/fine faces to the level's export buffer.
// FP64, and mixed levels on the kernel sequence: the seven-kernel sequence
// (two-layer frames in FP64), k_amr_theta copies the sibling ghosts'
// positivity factors and k_amr_export reads the exported fluxes from the face
// planes.  Around the step, per level:
//   k_amr_fill       ghost cells from siblings (copy) and the parent (limited
//                    interpolation in space of the surface and primitives,
//                    linear in time; one thread per parent cell and up to four
//                    of its ghosts), k_amr_fill_bc the boundary-condition ghosts,
//   k_amr_avg_reflux average-down and the mass correction at coarse/fine faces
//                    from the exported fluxes of both levels (one launch),
//   k_amr_finalize   the level-0 step from the speeds of all levels.
// A level-0 step with all substeps is captured once per ping-pong state and
// replayed as a CUDA graph.
#pragma once
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <vector>

#include "../../include/sgn_amr.h"
#include "sgn_solver.cuh"

namespace sgn {

constexpr int AMR_MAXL = 8;

// ghost-table entry: dst/src padded indices; info: bits 0-1 type, BC: bit 2/3
// flip hu/hv.
struct GEnt { int dst, src, info; };
enum { GE_SIB = 0, GE_PAR = 1, GE_BC = 2 };

// Ghost cells filled from the parent level, grouped by parent cell: group g
// holds the padded index of the parent cell (src[g]), its stencil W, E, S, N
// (nb[g]: padded indices into the parent level's atlas, -1 where the level
// has no patch there or the cell is outside the domain -- each stencil cell is
// read from the patch that holds it, so a ghost's value depends only on where
// it is, not on which patch's frame holds it) and its ghost cells first[g] ..
// first[g+1]-1: padded index dst and sub-cell offsets sub = sx | sy << 8.
struct ParTab {
  const int* src;
  const int4* nb;
  const int* first;
  const int* dst;
  const int* sub;
  int n;
};

// Ghost fill of a level before its step (one launch).  Threads [0, par.n):
// one parent cell each -- its surface and primitives at the substep's time
// weight a and the minmod slopes of its stencil, once -- then the limited
// interpolation of each of its ghost cells (depth from the surface, conserved
// values no larger than the parent cell's own).  Threads [par.n, par.n + ns):
// copies from sibling patches (sib, type GE_SIB).
template <int MODEL, typename Real>
__global__ void k_amr_fill(Dev<Real> c, Dev<Real> p, ParTab par, const GEnt* __restrict__ sib, int ns, int cc,
                           int pold, int pnew, double a, int r) {
  constexpr int NV = MT<MODEL>::NV;
  // the interpolation runs in the bulk type (the depth of a parent cell, which
  // decides dry or wet, in FP64): a ghost value is an input of the step, not
  // one of its balanced or positivity-critical terms
  typedef Real A;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  Real* qc = c.q[cc];
  if (e >= par.n) {
    e -= par.n;
    if (e >= ns) return;
    const GEnt g = sib[e];
#pragma unroll
    for (int k = 0; k < NV; k++) qc[k * c.fs + g.dst] = qc[k * c.fs + g.src];
    return;
  }
  const int4 nv = par.nb[e];
  const int c0 = par.first[e], c1 = par.first[e + 1];
  const Real* qo = p.q[pold];
  const Real* qn = p.q[pnew];
  const A a1 = A(a), a0 = A(1.0 - a);
  // surface and primitives of a parent cell at the time weight (false: dry)
  auto prim = [&](size_t id, A* o) -> bool {
    A v[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = a0 * (A)qo[k * p.fs + id] + a1 * (A)qn[k * p.fs + id];
    double hd = (1.0 - a) * (double)qo[id] + a * (double)qn[id] - (double)p.b[id];
    if (!(hd > c.dry_tol)) return false;
    A ih = A(1) / A(hd);
    o[0] = v[0];
#pragma unroll
    for (int k = 1; k < NV; k++) o[k] = v[k] * ih;
    return true;
  };
  A pc[NV], pw[NV], pe[NV], ps[NV], pn[NV], slx[NV], sly[NV], cv[NV];
  const size_t ic = (size_t)par.src[e];
  if (!prim(ic, pc)) {
    for (int ch = c0; ch < c1; ch++) {
      const size_t d = (size_t)par.dst[ch];
      const double bf = (double)c.b[d];
      qc[d] = (Real)(bf > 0.0 ? bf : 0.0);
#pragma unroll
      for (int k = 1; k < NV; k++) qc[k * c.fs + d] = Real(0);
    }
    return;
  }
  const bool hx = nv.x >= 0 && nv.y >= 0 && prim((size_t)nv.x, pw) && prim((size_t)nv.y, pe);
  const bool hy = nv.z >= 0 && nv.w >= 0 && prim((size_t)nv.z, ps) && prim((size_t)nv.w, pn);
  auto mm = [](A u, A v) -> A { return u * v <= A(0) ? A(0) : (fabs(u) < fabs(v) ? u : v); };
#pragma unroll
  for (int k = 0; k < NV; k++) {
    slx[k] = hx ? mm(pc[k] - pw[k], pe[k] - pc[k]) : A(0);
    sly[k] = hy ? mm(pc[k] - ps[k], pn[k] - pc[k]) : A(0);
    cv[k] = a0 * (A)qo[k * p.fs + ic] + a1 * (A)qn[k * p.fs + ic];   // conserved values of the parent cell
  }
  for (int ch = c0; ch < c1; ch++) {
    const size_t d = (size_t)par.dst[ch];
    const int sx = par.sub[ch] & 255, sy = par.sub[ch] >> 8;
    const A xi = A((sx + 0.5) / r - 0.5), yi = A((sy + 0.5) / r - 0.5);
    const double bf = (double)c.b[d];
    A out[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) out[k] = pc[k] + xi * slx[k] + yi * sly[k];
    double eta = (double)out[0];
    if (eta < bf) eta = bf;
    const double hf = eta - bf;
    qc[d] = (Real)eta;
#pragma unroll
    for (int k = 1; k < NV; k++) {
      // depth x primitive, no larger than the parent cell's own conserved value
      // (a mostly dry parent has a small mean depth and an unreliable velocity)
      const A v = hf > c.dry_tol ? A(hf) * out[k] : A(0);
      qc[k * c.fs + d] = (Real)(v * cv[k] > A(0) ? (fabs(v) <= fabs(cv[k]) ? v : cv[k]) : A(0));
    }
  }
}

template <int MODEL, typename Real>
__global__ void k_amr_fill_bc(Dev<Real> c, const GEnt* __restrict__ t, int n, int cc) {
  constexpr int NV = MT<MODEL>::NV;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const GEnt g = t[e];
  Real* q = c.q[cc];
#pragma unroll
  for (int k = 0; k < NV; k++) {
    Real v = q[k * c.fs + g.src];
    if ((k == 1 && (g.info & 4)) || (k == 2 && (g.info & 8))) v = -v;
    q[k * c.fs + g.dst] = v;
  }
}

template <typename Real>
__global__ void k_amr_theta(Dev<Real> c, const GEnt* __restrict__ t, int n) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const GEnt g = t[e];
  if ((g.info & 3) == GE_SIB) c.theta[g.dst] = c.theta[g.src];
}

// regridding: interior cell dst of the new level atlas takes every field of
// cell src of the old atlas of the same level
template <int MODEL, typename Real>
__global__ void k_amr_copy(Dev<Real> c, Dev<Real> o, const int* __restrict__ dst, const int* __restrict__ src,
                           int n, int cc, int oc) {
  constexpr int NV = MT<MODEL>::NV;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int d = dst[e], s = src[e];
#pragma unroll
  for (int k = 0; k < NV; k++) c.q[cc][k * c.fs + d] = o.q[oc][k * o.fs + s];
}

// refinement flag (Sec. 6.3: the surface jump between neighbouring cells
// exceeds tol), over the wet patch interiors of a level's atlas; neighbours
// that are dry or not interior cells of the same patch are not compared (a dry
// cell's eta is its bathymetry, not a free surface; kind bit 5 marks a cell
// whose left neighbour in the atlas is another patch of its region)
template <typename Real>
__global__ void k_amr_flag(Dev<Real> d, int cur, double tol, unsigned char* __restrict__ out) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= d.nxp || J >= d.nyp) return;
  const size_t id = at(d.pitch, I, J);
  const Real* e = d.q[cur];
  auto wet = [&](size_t c) { return (double)e[c] - (double)d.b[c] > d.dry_tol; };
  unsigned char f = 0;
  if ((d.kind[id] & 1) && wet(id)) {
    const double c = (double)e[id];
    const size_t nb[4] = {id - 1, id + 1, id - d.pitch, id + d.pitch};
    const bool other[4] = {(d.kind[id] & 32) != 0, (d.kind[id + 1] & 32) != 0, false, false};
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (!other[k] && (d.kind[nb[k]] & 1) && wet(nb[k]) && fabs((double)e[nb[k]] - c) > tol) f = 1;
  }
  out[id] = f;
}

// Kernel-sequence levels: the theta-weighted mass fluxes of the four faces
// (left, right, bottom, top) of every exported cell, in the bulk type, from
// the face planes as k_update applies them; cells[k] has export slot k.  The
// one-pass kernel writes the same values itself.
template <typename Real>
__global__ void k_amr_export(Dev<Real> d, const int* __restrict__ cells, int n, Real* __restrict__ xphi) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const size_t id = (size_t)cells[e];
  auto phi = [&](size_t f, size_t fl, Real M) {   // face f between cells fl and f
    const Real t = M > Real(0) ? d.theta[fl] : (M < Real(0) ? d.theta[f] : Real(1));
    return t * M;
  };
  Real* o = xphi + 4 * (size_t)e;
  o[0] = phi(id, id - 1, d.TX[id]);
  o[1] = phi(id + 1, id, d.TX[id + 1]);
  o[2] = phi(id, id - d.pitch, d.TY[id]);
  o[3] = phi(id + d.pitch, id, d.TY[id + d.pitch]);
}

// Average-down and reflux of a coarse level after its finer level's r
// substeps (one launch; the two touch disjoint cells).  Threads [0, navg):
// covered coarse cell ci[g] takes the mean of its r x r children (the surface
// summed in FP64).  Threads [navg, navg + m): uncovered coarse cell cell[g]
// next to the finer patches gets the mass correction of its coarse/fine faces
// (registers first[g] .. first[g+1]-1, fixed order): for register i with
// direction dir[i] and sign sgn[i],
//   v_i = sgn lam_c phi_c[cref[i]] - sum_k sgn (lam_f / r^2) sum_m phi_f[k][fref[i r + m]],
// phi_c: the coarse level's exported fluxes of this step, phi_f: the finer
// level's of its substeps k = 0 .. r-1 (nf4 values apart); a correction that
// would leave a negative depth is clipped and the water added accumulated.
template <int MODEL, typename Real>
__global__ void k_amr_avg_reflux(Dev<Real> cd, Dev<Real> fd, const int* __restrict__ ci, const int* __restrict__ fi,
                                 int navg, const int* __restrict__ cell, const int* __restrict__ first, int m,
                                 const int* __restrict__ cref, const signed char* __restrict__ dir,
                                 const signed char* __restrict__ sgn, const int* __restrict__ fref,
                                 const Real* __restrict__ phic, const Real* __restrict__ phif, size_t nf4, int cc,
                                 int fc, int r, double area, double* clipped) {
  constexpr int NV = MT<MODEL>::NV;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < navg) {
    const size_t f0 = (size_t)fi[g];
    {
      double s = 0.0;
      for (int dj = 0; dj < r; dj++)
        for (int di = 0; di < r; di++) s += (double)fd.q[fc][f0 + (size_t)dj * fd.pitch + di];
      cd.q[cc][ci[g]] = (Real)(s / (double)(r * r));
    }
#pragma unroll
    for (int k = 1; k < NV; k++) {
      Real s = Real(0);
      for (int dj = 0; dj < r; dj++)
        for (int di = 0; di < r; di++) s += fd.q[fc][k * fd.fs + f0 + (size_t)dj * fd.pitch + di];
      cd.q[cc][k * cd.fs + ci[g]] = s / Real(r * r);
    }
    return;
  }
  g -= navg;
  if (g >= m) return;
  double corr = 0.0;
  for (int i = first[g]; i < first[g + 1]; i++) {
    const int dr = dir[i];
    double v = ((double)sgn[i] * cd.lam[dr]) * (double)phic[cref[i]];
    const double coef = fd.lam[dr] / (double)(r * r);
    for (int k = 0; k < r; k++) {
      double s = 0.0;
      for (int q = 0; q < r; q++) s += (double)phif[(size_t)k * nf4 + fref[(size_t)i * r + q]];
      v -= ((double)sgn[i] * coef) * s;
    }
    corr += v;
  }
  const size_t id = (size_t)cell[g];
  double e = (double)cd.q[cc][id] + corr;
  const double b = (double)cd.b[id];
  if (e < b) {
    atomicAdd(clipped, (b - e) * area);
    e = b;
  }
  cd.q[cc][id] = (Real)e;
}

// mass partials over uncovered patch interiors (kind == 1)
template <typename Real>
__global__ void k_amr_mass1(Dev<Real> d, int cur) {
  __shared__ double red[256];
  double s = 0.0;
  size_t n = (size_t)d.nx * d.ny;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(c % d.nx), j = (int)(c / d.nx);
    size_t id = at(d.pitch, i + NG, j + NG);
    if ((d.kind[id] & 3) != 1) continue;
    double h = (double)d.q[cur][id] - (double)d.b[id];
    s += h > 0 ? h : 0.0;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) d.mass_part[blockIdx.x] = red[0];
}

// copy one patch interior between a dense nv x ny x nx buffer and the atlas;
// (px, py): padded atlas index of the patch's first interior cell
template <int MODEL, typename Real>
__global__ void k_amr_pack(Dev<Real> d, const double* qd, int px, int py, int nx, int ny, int cur) {
  constexpr int NV = MT<MODEL>::NV;
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  size_t id = at(d.pitch, px + i, py + j), n = (size_t)nx * ny, s = (size_t)j * nx + i;
  Real q[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) q[k] = (Real)qd[k * n + s];
  Crit h = (Crit)q[0] - (Crit)d.b[id];
  h = h > 0 ? h : 0;
  source_switch<MODEL, Real>(q, h > d.dry_tol, Real(h), d.c2[id], Real(0));
#pragma unroll
  for (int k = 0; k < NV; k++) d.q[cur][k * d.fs + id] = q[k];
}

template <int MODEL, typename Real>
__global__ void k_amr_unpack(Dev<Real> d, double* qd, int px, int py, int nx, int ny, int cur) {
  constexpr int NV = MT<MODEL>::NV;
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  size_t id = at(d.pitch, px + i, py + j), n = (size_t)nx * ny, s = (size_t)j * nx + i;
#pragma unroll
  for (int k = 0; k < NV; k++) qd[k * n + s] = (double)d.q[cur][k * d.fs + id];
}

// Interior cells of every patch of a level into a dense device field
// (fields [0, nf) of [field][NY][NX]); tab: px, py (padded index of the first
// interior cell), nx, ny, i0, j0 per patch, one patch per blockIdx.z.
template <int MODEL, typename Real>
__global__ void k_amr_scatter(Dev<Real> d, const int* __restrict__ tab, int nf, double* __restrict__ out, int NX,
                              int NY, int cur) {
  const int* t = tab + 6 * blockIdx.z;
  const int px = t[0], py = t[1], nx = t[2], ny = t[3], i0 = t[4], j0 = t[5];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t id = at(d.pitch, px + i, py + j);
  const size_t o = (size_t)(j0 + j) * NX + (i0 + i), plane = (size_t)NX * NY;
  for (int k = 0; k < nf; k++) out[k * plane + o] = (double)d.q[cur][k * d.fs + id];
}

struct AmrDt {
  int L, strang;
  double cfl;
  double R[AMR_MAXL], dx[AMR_MAXL], dy[AMR_MAXL];
  unsigned long long* smax[AMR_MAXL];
  unsigned long long* cmax[AMR_MAXL];
  double* dt[AMR_MAXL];
  double* lam[AMR_MAXL];
  float* lamf[AMR_MAXL];    // bulk-type copies of lam (one of the two is set)
  double* lamd[AMR_MAXL];
  unsigned* status;
  double* sc;   // dt0, t, last_dt, courant, clipped
};

__device__ __forceinline__ void amr_level_steps(const AmrDt& a, double dt0) {
  for (int l = 0; l < a.L; l++) {
    double dtl = dt0 / a.R[l];
    *a.dt[l] = dtl;
    a.lam[l][0] = dtl / a.dx[l];
    a.lam[l][1] = dtl / a.dy[l];
    a.lam[l][2] = a.strang ? 0.5 * dtl : 0.0;
    a.lam[l][3] = a.strang ? 0.5 * dtl : dtl;
    for (int k = 0; k < 4; k++) {
      if (a.lamf[l]) a.lamf[l][k] = (float)a.lam[l][k];
      if (a.lamd[l]) a.lamd[l][k] = a.lam[l][k];
    }
  }
}

// Level-0 step bookkeeping (one thread): dt0 = min_l CFL r^l / smax_l, the
// level steps dt0 / r^l with their dt/dx, dt/dy and source sub-steps; the
// accumulators are cleared for the next level-0 step.
static __global__ void k_amr_finalize(AmrDt a, int advance) {
  if (threadIdx.x != 0) return;
  if (advance) {
    double dt = a.sc[0];
    a.sc[1] += dt;
    a.sc[2] = dt;
    double cr = 0.0;
    for (int l = 0; l < a.L; l++) cr = fmax(cr, __longlong_as_double((long long)*a.cmax[l]));
    a.sc[3] = cr;
    if (cr > 1.0) set_status(a.status, ST_CFL);
  }
  double best = 0.0;
  bool any = false;
  for (int l = 0; l < a.L; l++) {
    double sp = __longlong_as_double((long long)*a.smax[l]);
    if (sp > 0.0) {
      double d = a.cfl * a.R[l] / sp;
      if (!any || d < best) best = d;
      any = true;
    }
  }
  if (!any) set_status(a.status, ST_ALLDRY);
  a.sc[0] = best;
  amr_level_steps(a, best);
  for (int l = 0; l < a.L; l++) {
    *a.smax[l] = 0ull;
    *a.cmax[l] = 0ull;
  }
}

// a prescribed level-0 step
static __global__ void k_amr_setdt(AmrDt a, double dt0) {
  if (threadIdx.x != 0) return;
  a.sc[0] = dt0;
  amr_level_steps(a, dt0);
}

struct AmrArgs {
  sgn_grid grid;
  sgn_params prm;
  int model, L, r;
  const double* b;
  std::vector<std::vector<int>> boxes;   // per level >= 1: 4 ints per box
  const sgn_allocator* alloc;
  cudaStream_t stream;
  const struct AmrBase* prev = nullptr;  // regrid: the hierarchy whose state the new one takes
};

// Bathymetry of the levels coarser than the finest (block means), kept by a
// hierarchy and shared with the hierarchies its regrids build (the finest
// bathymetry, and so these means, do not change between regrids).
typedef std::shared_ptr<const std::vector<std::vector<double>>> CoarseBath;

struct AmrBase {
  virtual ~AmrBase() {}
  virtual CoarseBath coarse_bath() const = 0;
  virtual int init(const AmrArgs& a) = 0;
  virtual int npatches(int l) const = 0;
  virtual int set_patch(int l, int k, const double* q) = 0;
  virtual int get_patch(int l, int k, double* q) = 0;
  virtual int step(int n, double* t_out) = 0;
  virtual int step_dt(double dt0) = 0;
  virtual int next_dt(double* dt0) = 0;
  virtual int mass(double* m, double* clipped) = 0;
  virtual int status(unsigned* f) = 0;
  virtual int info(long long* cells, long long* atlas) const = 0;
  virtual int launches_per_step() const = 0;
  virtual int autotune(int reps, int* choice, double* ms) = 0;
  virtual int set_tuning(const int* choice) = 0;
  virtual int take_state(AmrBase* old) = 0;
  // level sizes, boxes (4 ints each), and the flags of a level on its full
  // grid (dense NX x NY; have = 1 where a patch of the level holds the cell)
  virtual void dims(int l, int* NX, int* NY) const = 0;
  virtual void boxes(int l, std::vector<int>& out) const = 0;
  virtual int flags(int l, double tol, std::vector<unsigned char>& flag, std::vector<unsigned char>& have) = 0;
  // fields [0, nf) of every patch of level l into out (device, [nf][NY][NX] of
  // the level's full grid); cells without a patch are left as they are
  virtual int get_level_device(int l, int nf, double* out) = 0;
  // retaking of level-0 steps that break the CFL limit (0: off), and the
  // number of steps retaken so far
  virtual int set_retake(int max_retakes) = 0;
  virtual long long retakes() const = 0;
};

AmrBase* make_amr_f64(int model);
AmrBase* make_amr_mixed(int model);

// ---------------------------------------------------------------------------
// host side: hierarchy geometry, atlas packing, tables
// (px, py): padded atlas index of the frame corner (frame cell (0, 0); the
// first interior cell is frame cell (G, G), G the frame depth)
struct Box { int i0, j0, nx, ny; int px, py; int parent; };

inline int bc_index(int X, int N, int lo, int hi, bool& flip) {
  flip = false;
  if (X < 0) { if (lo == SGN_BC_WALL) { flip = true; return -X - 1; } return 0; }
  if (X >= N) { if (hi == SGN_BC_WALL) { flip = true; return 2 * N - 1 - X; } return N - 1; }
  return X;
}

// spatial buckets of a level's boxes for owner lookups
struct Owner {
  int B = 64, nbx = 1, nby = 1;
  std::vector<std::vector<int>> bk;
  const std::vector<Box>* bx = nullptr;
  void build(const std::vector<Box>& boxes, int NX, int NY) {
    bx = &boxes;
    nbx = (NX + B - 1) / B; nby = (NY + B - 1) / B;
    bk.assign((size_t)nbx * nby, {});
    for (int k = 0; k < (int)boxes.size(); k++) {
      const Box& b = boxes[k];
      int x0 = std::max(0, b.i0) / B, x1 = std::min(NX - 1, b.i0 + b.nx - 1) / B;
      int y0 = std::max(0, b.j0) / B, y1 = std::min(NY - 1, b.j0 + b.ny - 1) / B;
      for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++) bk[(size_t)y * nbx + x].push_back(k);
    }
  }
  int find(int X, int Y, int skip = -1) const {
    if (X < 0 || Y < 0 || X / B >= nbx || Y / B >= nby) return -1;
    for (int k : bk[(size_t)(Y / B) * nbx + X / B]) {
      const Box& b = (*bx)[k];
      if (k != skip && X >= b.i0 && X < b.i0 + b.nx && Y >= b.j0 && Y < b.j0 + b.ny) return k;
    }
    return -1;
  }
};

template <int MODEL, typename Real>
class Amr : public AmrBase {
  static constexpr int NV = MT<MODEL>::NV;
  // ghost layers of a patch frame: three in mixed precision, where the
  // one-pass kernel computes the positivity factors of sibling ghosts next to
  // a patch edge itself (their faces' fluxes reach two cells further out); two
  // where the kernel sequence copies them from the sibling
  static constexpr int G = sizeof(Real) == 4 ? 3 : 2;
  int L_ = 1, r_ = 2;
  sgn_grid g0_{};
  sgn_params prm_{};
  std::vector<Solver<MODEL, Real>*> lv_;
  std::vector<std::vector<Box>> bx_;
  std::vector<int> NX_, NY_;
  std::vector<double> dx_;
  struct Tabs {
    GEnt* fill = nullptr; int nfill = 0;      // copies from sibling patches (GE_SIB)
    ParTab par{};                             // ghosts from the parent level, by parent cell
    GEnt* bc = nullptr; int nbc = 0;
    int* xcell = nullptr; int nxc = 0;        // exported cells of this level, by slot
    Real* xphi = nullptr;                     // their face fluxes: (l ? r : 1) substeps x nxc x 4
    // registers of this level as the coarse side, grouped by corrected cell
    int* rcref = nullptr; int* rfref = nullptr; signed char* rdir = nullptr; signed char* rsgn = nullptr;
    int nreg = 0;
    int* rcell = nullptr; int* rfirst = nullptr; int ncell = 0;
    int* acoarse = nullptr; int* afine = nullptr; int navg = 0;
  };
  std::vector<Owner> own_;     // per level: box lookup by cell
  // per level >= 1: the regions of the atlas (runs of boxes of equal rows that
  // abut in x), each with one frame; Box::parent holds the region's first box
  std::vector<std::vector<Box>> rg_;
  std::vector<Tabs> tb_;
  std::vector<long long> cells_, atlas_;
  CoarseBath bath_;            // bathymetry of levels 0 .. L-2
  double* sc_ = nullptr;       // dt0, t, last_dt, courant, clipped
  double* staging_ = nullptr;
  size_t stage_bytes_ = 0;
  unsigned char* flag_buf_ = nullptr;   // atlas-sized flag plane (when staging_ is smaller)
  int* scat_[AMR_MAXL] = {};            // per level: patch table of k_amr_scatter (built on first use)
  int scat_mx_[AMR_MAXL] = {}, scat_my_[AMR_MAXL] = {};
  size_t flag_cap_ = 0;
  double* hsc_ = nullptr;      // pinned host scalars
  cudaStream_t st_ = nullptr, cap_ = nullptr;
  std::map<unsigned, std::pair<cudaGraphExec_t, unsigned>> graphs_;   // cur bits -> (graph, cur bits after)
  bool fresh_ = true;
  int launches_ = 0;
  AmrDt dt_{};
  // step retaking: the states of levels >= 1 before a level-0 step (level 0
  // keeps its own in the buffer the step does not write), and the scalars and
  // status words (device)
  int retake_max_ = 0;
  long long retakes_ = 0;
  std::vector<Real*> bak_;
  double* bsc_ = nullptr;      // 8 scalars, then AMR_MAXL status words

  // device memory of the hierarchy's own tables and buffers (the level
  // solvers hold their planes), from the caller's allocator or cudaMalloc,
  // freed with the hierarchy
  sgn_allocator al_{};
  bool has_al_ = false;
  std::vector<void*> mine_;
  // a regrid's hierarchy takes over the level-0 solver of the one it
  // replaces (level 0 does not change); until it is committed the donor
  // gets it back if this hierarchy is destroyed
  Amr* donor_ = nullptr;
  std::vector<unsigned char> kd0_;   // level 0's kind plane (dense) ...
  std::vector<int> xs0_;             // ... and export slots, as this hierarchy set them
  template <typename T> T* adev(size_t n) {
    const size_t bytes = n * sizeof(T) + 256;
    void* p = nullptr;
    if (has_al_) p = al_.alloc(bytes, al_.ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) mine_.push_back(p);
    return (T*)p;
  }

  template <typename T> T* up(const std::vector<T>& h) {
    if (h.empty()) return nullptr;
    T* d = adev<T>(h.size());
    if (!d) return nullptr;
    if (cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st_) != cudaSuccess) return nullptr;
    return d;
  }

  static unsigned grid1(int n) { return (unsigned)((n + 255) / 256); }

 public:
  ~Amr() override {
    if (st_) cudaStreamSynchronize(st_);
    for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second.first);
    if (donor_ && !lv_.empty() && lv_[0] && donor_->lv_.size() && !donor_->lv_[0]) {
      donor_->lv_[0] = lv_[0];
      lv_[0] = nullptr;
      if (!donor_->kd0_.empty()) donor_->lv_[0]->set_kind(donor_->kd0_.data());
      if (!donor_->xs0_.empty()) donor_->lv_[0]->set_xslot(donor_->xs0_.data());
    }
    for (int l = (int)lv_.size() - 1; l >= 0; l--) delete lv_[l];
    for (void* p : mine_) {
      if (has_al_) al_.free(p, al_.ctx);
      else cudaFree(p);
    }
    if (hsc_) cudaFreeHost(hsc_);
    if (cap_) cudaStreamDestroy(cap_);
  }

  CoarseBath coarse_bath() const override { return bath_; }
  int npatches(int l) const override { return (l >= 0 && l < L_) ? (int)bx_[l].size() : SGN_EINVAL; }
  int launches_per_step() const override { return launches_; }
  int info(long long* cells, long long* atlas) const override {
    for (int l = 0; l < L_; l++) {
      if (cells) cells[l] = cells_[l];
      if (atlas) atlas[l] = atlas_[l];
    }
    return SGN_OK;
  }

  int init(const AmrArgs& a) override {
    L_ = a.L; r_ = a.r; g0_ = a.grid; prm_ = a.prm; st_ = a.stream;
    if (a.alloc && a.alloc->alloc && a.alloc->free) { al_ = *a.alloc; has_al_ = true; }
    const int r = r_, L = L_;
    SGN_CK(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
    SGN_CK(cudaMallocHost((void**)&hsc_, 16 * sizeof(double)));
    NX_.resize(L); NY_.resize(L); dx_.resize(L);
    long long R = 1;
    for (int l = 0; l < L; l++) {
      NX_[l] = (int)(g0_.nx * R); NY_[l] = (int)(g0_.ny * R);
      dx_[l] = g0_.dx / (double)R;
      R *= r;
    }
    // boxes (level 0: the grid)
    bx_.assign(L, {});
    bx_[0].push_back(Box{0, 0, g0_.nx, g0_.ny, 0, 0, -1});
    for (int l = 1; l < L; l++) {
      const std::vector<int>& v = a.boxes[l - 1];
      for (size_t k = 0; k + 3 < v.size(); k += 4) bx_[l].push_back(Box{v[k], v[k + 1], v[k + 2], v[k + 3], 0, 0, -1});
    }
    // validation (the rules of the header)
    own_.assign(L, Owner{});
    std::vector<Owner>& own = own_;
    for (int l = 1; l < L; l++)
      for (const Box& b : bx_[l])
        if (b.i0 < 0 || b.j0 < 0 || b.nx < 2 || b.ny < 2 || b.i0 + b.nx > NX_[l] || b.j0 + b.ny > NY_[l] ||
            b.i0 % r || b.j0 % r || b.nx % r || b.ny % r)
          return SGN_EINVAL;
    for (int l = 0; l < L; l++) own[l].build(bx_[l], NX_[l], NY_[l]);
    for (int l = 1; l < L; l++) {
      for (int k = 0; k < (int)bx_[l].size(); k++) {
        Box& b = bx_[l][k];
        int c0 = b.i0 / r, c1 = (b.i0 + b.nx) / r, d0 = b.j0 / r, d1 = (b.j0 + b.ny) / r;
        int pi = -1;
        for (int q = 0; q < (int)bx_[l - 1].size(); q++) {
          const Box& p = bx_[l - 1][q];
          if (p.i0 <= c0 && c1 <= p.i0 + p.nx && p.j0 <= d0 && d1 <= p.j0 + p.ny) { pi = q; break; }
        }
        if (pi < 0) return SGN_EINVAL;
        const Box& p = bx_[l - 1][pi];
        int gaps[4] = {c0 - p.i0, p.i0 + p.nx - c1, d0 - p.j0, p.j0 + p.ny - d1};
        bool edge[4] = {c0 == 0, c1 == NX_[l - 1], d0 == 0, d1 == NY_[l - 1]};
        for (int s = 0; s < 4; s++)
          if (gaps[s] < 2 && !edge[s]) return SGN_EINVAL;
        b.parent = pi;
        // overlap: another box owns a cell on this machine's boundary (covers
        // partial overlap and containment either way)
        for (int x = b.i0; x < b.i0 + b.nx; x++)
          if (own[l].find(x, b.j0, k) >= 0 || own[l].find(x, b.j0 + b.ny - 1, k) >= 0) return SGN_EINVAL;
        for (int y = b.j0; y < b.j0 + b.ny; y++)
          if (own[l].find(b.i0, y, k) >= 0 || own[l].find(b.i0 + b.nx - 1, y, k) >= 0) return SGN_EINVAL;
      }
    }
    // bathymetry of every level: the finest as given (read in place), block
    // means upward -- computed once and shared with the hierarchies of later
    // regrids
    if (a.prev && a.prev->coarse_bath() && (int)a.prev->coarse_bath()->size() == L - 1) {
      bath_ = a.prev->coarse_bath();
    } else {
      auto bl = std::make_shared<std::vector<std::vector<double>>>(L > 1 ? L - 1 : 0);
      for (int l = L - 2; l >= 0; l--) {
        std::vector<double>& c = (*bl)[l];
        c.assign((size_t)NX_[l] * NY_[l], 0.0);
        const int NXf = NX_[l + 1];
        const double* f = l + 1 == L - 1 ? a.b : (*bl)[l + 1].data();
        for (int j = 0; j < NY_[l]; j++)
          for (int i = 0; i < NX_[l]; i++) {
            double s = 0.0;
            for (int dj = 0; dj < r; dj++)
              for (int di = 0; di < r; di++) s += f[(size_t)(j * r + dj) * NXf + (i * r + di)];
            c[(size_t)j * NX_[l] + i] = s / (double)(r * r);
          }
      }
      bath_ = bl;
    }
    auto blev = [&](int l) -> const double* { return l == L - 1 ? a.b : (*bath_)[l].data(); };
    auto bval = [&](int l, int X, int Y) {
      bool f;
      int Xs = bc_index(X, NX_[l], g0_.bc[0], g0_.bc[1], f), Ys = bc_index(Y, NY_[l], g0_.bc[2], g0_.bc[3], f);
      return blev(l)[(size_t)Ys * NX_[l] + Xs];
    };
    // phi_T of a level cell by the uniform-grid rule (boundary-mapped first)
    auto phival = [&](int l, int X, int Y) -> unsigned char {
      bool f;
      int Xs = bc_index(X, NX_[l], g0_.bc[0], g0_.bc[1], f), Ys = bc_index(Y, NY_[l], g0_.bc[2], g0_.bc[3], f);
      int n = prm_.n_transition;
      double dx = dx_[l], dy = dx_[l];
      double r2 = (n * dx) * (n * dx), mn = 1e300;
      for (int dj = -n; dj <= n; dj++)
        for (int di = -n; di <= n; di++) {
          if ((di * dx) * (di * dx) + (dj * dy) * (dj * dy) > r2) continue;
          double H = -bval(l, Xs + di, Ys + dj);
          H = H > 0.0 ? H : 0.0;
          mn = H < mn ? H : mn;
        }
      return mn > prm_.h_star ? 1 : 0;
    };
    // atlases and level solvers
    lv_.assign(L, nullptr);
    rg_.assign(L, {});
    cells_.assign(L, 0); atlas_.assign(L, 0);
    std::vector<int> NXA(L), NYA(L);
    for (int l = 0; l < L; l++) {
      CreateArgs ca{};
      ca.prm = prm_; ca.model = a.model; ca.alloc = a.alloc; ca.stream = st_;
      ca.no_initial_state = a.prev != nullptr;   // a regrid fills every level from the old hierarchy
      std::vector<double> bd;
      std::vector<unsigned char> pd;
      int nxa, nya;
      for (auto& b : bx_[l]) cells_[l] += (long long)b.nx * b.ny;
      if (l == 0) {
        nxa = g0_.nx; nya = g0_.ny;
        ca.grid = g0_;
        bx_[0][0].px = NG - G;   // level 0's frame is the atlas's own
        bx_[0][0].py = NG - G;
        if (a.prev) {
          // a regrid: level 0 is the replaced hierarchy's, state included
          auto* o = dynamic_cast<Amr<MODEL, Real>*>(const_cast<AmrBase*>(a.prev));
          if (o && !o->lv_.empty() && o->lv_[0] && !o->NX_.empty() && o->NX_[0] == NX_[0] && o->NY_[0] == NY_[0]) {
            lv_[0] = o->lv_[0];
            o->lv_[0] = nullptr;
            donor_ = o;
            NXA[0] = nxa; NYA[0] = nya;
            atlas_[0] = (long long)(nxa + 4) * (nya + 4);
            continue;
          }
        }
        bd.assign(blev(0), blev(0) + (size_t)NX_[0] * NY_[0]);
      } else {
        // regions: runs of boxes of equal rows that abut in x share one frame
        // (the faces between them are interior faces of the atlas, without
        // ghost cells); each box keeps its place inside its region
        std::vector<Box>& rg = rg_[l];
        std::vector<int> byrow(bx_[l].size());
        for (size_t k = 0; k < byrow.size(); k++) byrow[k] = (int)k;
        std::stable_sort(byrow.begin(), byrow.end(), [&](int u, int v) {
          const Box &a = bx_[l][u], &b = bx_[l][v];
          return a.j0 != b.j0 ? a.j0 < b.j0 : (a.ny != b.ny ? a.ny < b.ny : a.i0 < b.i0);
        });
        std::vector<int> regof(bx_[l].size());
        for (int k : byrow) {
          const Box& b = bx_[l][k];
          if (!rg.empty() && rg.back().j0 == b.j0 && rg.back().ny == b.ny && rg.back().i0 + rg.back().nx == b.i0) {
            rg.back().nx += b.nx;
          } else {
            rg.push_back(Box{b.i0, b.j0, b.nx, b.ny, 0, 0, k});   // parent: the region's first box
          }
          regof[k] = (int)rg.size() - 1;
        }
        // shelf packing of the (nx + 2G) x (ny + 2G) region frames, tallest
        // first, at the shelf width (from 0.6 to 1.8 x sqrt(area)) that gives
        // the smallest atlas
        std::vector<int> ord(rg.size());
        for (size_t k = 0; k < ord.size(); k++) ord[k] = (int)k;
        std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) { return rg[u].ny > rg[v].ny; });
        double area = 0;
        int maxw = 2;
        for (auto& b : rg) { area += (double)(b.nx + 2 * G) * (b.ny + 2 * G); maxw = std::max(maxw, b.nx + 2 * G); }
        auto shelves = [&](int w, bool place) {
          int x = 0, y = 0, sh = 0;
          for (int k : ord) {
            Box& b = rg[k];
            if (x + b.nx + 2 * G > w) { x = 0; y += sh; sh = 0; }
            if (place) { b.px = x + NG; b.py = y + NG; }   // the atlas has its own two-cell frame
            x += b.nx + 2 * G;
            sh = std::max(sh, b.ny + 2 * G);
          }
          return std::max(2, y + sh);
        };
        nxa = std::max(maxw, (int)std::ceil(std::sqrt(area * 1.1)));
        long long best = (long long)nxa * shelves(nxa, false);
        for (int i = 0; i <= 60; i++) {
          const int w = std::max(maxw, (int)(std::sqrt(area) * (0.6 + 0.02 * i)));
          const long long a = (long long)w * shelves(w, false);
          if (a < best) { best = a; nxa = w; }
        }
        nya = shelves(nxa, true);
        for (int k = 0; k < (int)bx_[l].size(); k++) {
          Box& b = bx_[l][k];
          const Box& R = rg[regof[k]];
          b.px = R.px + (b.i0 - R.i0);
          b.py = R.py;
        }
        ca.grid = g0_;
        ca.grid.nx = nxa; ca.grid.ny = nya;
        ca.grid.dx = dx_[l]; ca.grid.dy = dx_[l];
        for (int s = 0; s < 4; s++) ca.grid.bc[s] = SGN_BC_EXTRAP;
        bd.assign((size_t)nxa * nya, 1000.0);   // empty atlas cells: dry land
        pd.assign((size_t)nxa * nya, 0);
        // bathymetry and phi_T of every region's frame: b read once per cell
        // of the frame and an n-cell margin, phi_T from those values (the
        // boundary-mapped rule of phival where a cell lies outside the domain)
        const int n = prm_.n_transition;
        std::vector<std::pair<int, int>> nbh;
        {
          const double dxl = dx_[l], r2 = (n * dxl) * (n * dxl);
          for (int dj = -n; dj <= n; dj++)
            for (int di = -n; di <= n; di++)
              if ((di * dxl) * (di * dxl) + (dj * dxl) * (dj * dxl) <= r2) nbh.push_back(std::make_pair(di, dj));
        }
        std::vector<double> loc;
        for (auto& b : rg) {
          const int Wl = b.nx + 2 * G + 2 * n, Hl = b.ny + 2 * G + 2 * n;
          loc.resize((size_t)Wl * Hl);
          for (int JJ = 0; JJ < Hl; JJ++)
            for (int II = 0; II < Wl; II++) loc[(size_t)JJ * Wl + II] = bval(l, b.i0 - G - n + II, b.j0 - G - n + JJ);
          for (int J = 0; J < b.ny + 2 * G; J++)
            for (int I = 0; I < b.nx + 2 * G; I++) {
              const int X = b.i0 - G + I, Y = b.j0 - G + J;
              const size_t o = (size_t)(b.py - NG + J) * nxa + (b.px - NG + I);
              const size_t c = (size_t)(J + n) * Wl + (I + n);
              bd[o] = loc[c];
              if (X < 0 || Y < 0 || X >= NX_[l] || Y >= NY_[l]) {
                pd[o] = phival(l, X, Y);
                continue;
              }
              double mn = 1e300;
              for (const auto& q : nbh) {
                double H = -loc[c + (long)q.second * Wl + q.first];
                H = H > 0.0 ? H : 0.0;
                mn = H < mn ? H : mn;
              }
              pd[o] = mn > prm_.h_star ? 1 : 0;
            }
        }
      }
      NXA[l] = nxa; NYA[l] = nya;
      atlas_[l] = (long long)(nxa + 4) * (nya + 4);
      if ((long long)((nxa + 5 + 31) / 32 * 32) * (nya + 5) >= (1LL << 31)) return SGN_EINVAL;
      ca.b = bd.data();
      ca.phi = l == 0 ? nullptr : pd.data();
      lv_[l] = new Solver<MODEL, Real>();
      int rc = lv_[l]->init(ca);
      if (rc) return rc;
    }
    // kind planes (bit 0 interior, 1 covered by the next level, 2 sibling
    // ghost next to a patch edge, 3 exported cell) and export slots, dense
    // over each atlas; frame cell (I, J) of box b is dense atlas cell
    // (px - NG + I, py - NG + J)
    std::vector<std::vector<unsigned char>> kd(L);
    std::vector<std::vector<int>> xs(L);
    std::vector<std::vector<int>> xcells(L);
    auto dense = [&](int l, const Box& b, int I, int J) {
      return (size_t)(b.py - NG + J) * NXA[l] + (size_t)(b.px - NG + I);
    };
    for (int l = 0; l < L; l++) {
      kd[l].assign((size_t)NXA[l] * NYA[l], 0);
      xs[l].assign((size_t)NXA[l] * NYA[l], -1);
      for (int k = 0; k < (int)bx_[l].size(); k++) {
        const Box& b = bx_[l][k];
        for (int j = 0; j < b.ny; j++) {
          unsigned char* row = &kd[l][dense(l, b, G, G + j)];
          std::fill(row, row + b.nx, (unsigned char)1);
        }
      }
      // bit 5: the first column of a patch that follows another in its region
      if (l > 0)
        for (const Box& b : bx_[l])
          for (const Box& R : rg_[l])
            if (R.j0 == b.j0 && R.ny == b.ny && R.i0 < b.i0 && b.i0 < R.i0 + R.nx)
              for (int j = 0; j < b.ny; j++) kd[l][dense(l, b, G, G + j)] |= 32;
      // covered: the footprint of every box of the next level, in its parent
      if (l + 1 < L)
        for (const Box& c : bx_[l + 1]) {
          const Box& P = bx_[l][c.parent];
          for (int jc = c.j0 / r; jc < (c.j0 + c.ny) / r; jc++)
            for (int ic = c.i0 / r; ic < (c.i0 + c.nx) / r; ic++) kd[l][dense(l, P, G + ic - P.i0, G + jc - P.j0)] |= 2;
        }
    }
    // export slot of a cell (assigned on first use)
    auto slot_of = [&](int l, const Box& b, int I, int J) {
      const size_t o = dense(l, b, I, J);
      if (xs[l][o] < 0) {
        xs[l][o] = (int)xcells[l].size();
        xcells[l].push_back(pidx(l, b, I, J));
        kd[l][o] |= 8;
      }
      return xs[l][o];
    };
    tb_.assign(L, Tabs{});
    for (int l = 1; l < L; l++) {
      std::vector<GEnt> fill, bcs;
      std::vector<ParEnt> pe;
      // the ghost cells of every region's frame (b: the region)
      for (const Box& b : rg_[l]) {
        for (int J = 0; J < b.ny + 2 * G; J++)
          for (int I = 0; I < b.nx + 2 * G; I++) {
            if (I >= G && I < b.nx + G && J >= G && J < b.ny + G) continue;
            int X = b.i0 - G + I, Y = b.j0 - G + J;
            int dst = pidx(l, b, I, J);
            if (X < 0 || Y < 0 || X >= NX_[l] || Y >= NY_[l]) {
              bool fx, fy;
              int Xs = bc_index(X, NX_[l], g0_.bc[0], g0_.bc[1], fx);
              int Ys = bc_index(Y, NY_[l], g0_.bc[2], g0_.bc[3], fy);
              int Is = Xs - b.i0 + G, Js = Ys - b.j0 + G;
              if (Is < 0 || Js < 0 || Is >= b.nx + 2 * G || Js >= b.ny + 2 * G) return SGN_EINVAL;
              bcs.push_back(GEnt{dst, pidx(l, b, Is, Js), GE_BC | (fx ? 4 : 0) | (fy ? 8 : 0)});
              continue;
            }
            int o = own[l].find(X, Y);
            if (o >= 0) {
              const Box& s = bx_[l][o];
              fill.push_back(GEnt{dst, pidx(l, s, X - s.i0 + G, Y - s.j0 + G), GE_SIB});
              // a sibling ghost sharing a face with an interior cell
              const bool side = ((I == G - 1 || I == G + b.nx) && J >= G && J < G + b.ny) ||
                                ((J == G - 1 || J == G + b.ny) && I >= G && I < G + b.nx);
              if (side) kd[l][dense(l, b, I, J)] |= 4;
              continue;
            }
            // interpolated from the parent of the region's box nearest in x
            const int kb = own[l].find(std::min(std::max(X, b.i0), b.i0 + b.nx - 1), b.j0);
            ParEnt q;
            if (kb < 0 || !par_entry(l, bx_[l][kb], X, Y, dst, q)) return SGN_EINVAL;
            pe.push_back(q);
          }
      }
      tb_[l].fill = up(fill); tb_[l].nfill = (int)fill.size();
      tb_[l].bc = up(bcs); tb_[l].nbc = (int)bcs.size();
      if ((tb_[l].nfill && !tb_[l].fill) || (tb_[l].nbc && !tb_[l].bc)) return SGN_ENOMEM;
      if (!upload_par(pe, tb_[l].par)) return SGN_ENOMEM;
    }
    // registers and average-down maps of level l (coarse side).  A register
    // is a coarse face between an uncovered cell u and a covered one: its
    // coarse flux is exported by u (the face of u it is), its r fine fluxes by
    // the fine interior cells along the patch edge.
    for (int l = 0; l + 1 < L; l++) {
      std::vector<int> af, ac, cellof, cref, fref;
      std::vector<signed char> dr, sg;
      for (int ci = 0; ci < (int)bx_[l + 1].size(); ci++) {
        const Box& c = bx_[l + 1][ci];
        const Box& P = bx_[l][c.parent];
        int c0 = c.i0 / r, d0 = c.j0 / r, cw = c.nx / r, ch = c.ny / r;
        for (int jc = d0; jc < d0 + ch; jc++)
          for (int ic = c0; ic < c0 + cw; ic++) {
            ac.push_back(pidx(l, P, ic - P.i0 + G, jc - P.j0 + G));
            af.push_back(pidx(l + 1, c, (ic - c0) * r + G, (jc - d0) * r + G));
          }
        // d: direction; (ux, uy): the uncovered coarse cell; s: sign; fu: the
        // face of u; (fI, fJ): frame index of the first fine cell along the
        // edge, (sI, sJ) the step to the next; ff: their face on the edge
        struct Cand { int d, ux, uy, s, fu, fI, fJ, sI, sJ, ff; };
        std::vector<Cand> cand;
        for (int jc = d0; jc < d0 + ch; jc++) {
          cand.push_back(Cand{0, c0 - 1, jc, +1, 1, G, (jc - d0) * r + G, 0, 1, 0});
          cand.push_back(Cand{0, c0 + cw, jc, -1, 0, G + c.nx - 1, (jc - d0) * r + G, 0, 1, 1});
        }
        for (int ic = c0; ic < c0 + cw; ic++) {
          cand.push_back(Cand{1, ic, d0 - 1, +1, 3, (ic - c0) * r + G, G, 1, 0, 2});
          cand.push_back(Cand{1, ic, d0 + ch, -1, 2, (ic - c0) * r + G, G + c.ny - 1, 1, 0, 3});
        }
        for (const Cand& q : cand) {
          if (q.ux < 0 || q.uy < 0 || q.ux >= NX_[l] || q.uy >= NY_[l]) continue;
          if (own[l + 1].find(q.ux * r, q.uy * r) >= 0) continue;   // covered: a sibling face
          const int uI = q.ux - P.i0 + G, uJ = q.uy - P.j0 + G;
          cref.push_back(4 * slot_of(l, P, uI, uJ) + q.fu);
          for (int m = 0; m < r; m++) fref.push_back(4 * slot_of(l + 1, c, q.fI + m * q.sI, q.fJ + m * q.sJ) + q.ff);
          dr.push_back((signed char)q.d);
          sg.push_back((signed char)q.s);
          cellof.push_back(pidx(l, P, uI, uJ));
        }
      }
      // group the registers by corrected cell (creation order within a cell)
      std::vector<int> order(cellof.size());
      for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
      std::stable_sort(order.begin(), order.end(), [&](int u, int v) { return cellof[u] < cellof[v]; });
      std::vector<int> cref2, fref2, cells, first;
      std::vector<signed char> dr2, sg2;
      for (size_t i = 0; i < order.size(); i++) {
        int g = order[i];
        if (i == 0 || cellof[g] != cellof[order[i - 1]]) { cells.push_back(cellof[g]); first.push_back((int)i); }
        cref2.push_back(cref[g]);
        for (int m = 0; m < r; m++) fref2.push_back(fref[(size_t)g * r + m]);
        dr2.push_back(dr[g]); sg2.push_back(sg[g]);
      }
      first.push_back((int)order.size());
      Tabs& t = tb_[l];
      t.nreg = (int)cref2.size();
      if (t.nreg) {
        t.rcref = up(cref2); t.rfref = up(fref2); t.rdir = up(dr2); t.rsgn = up(sg2);
        t.ncell = (int)cells.size();
        t.rcell = up(cells); t.rfirst = up(first);
        if (!t.rcref || !t.rfref || !t.rdir || !t.rsgn || !t.rcell || !t.rfirst) return SGN_ENOMEM;
      }
      t.navg = (int)ac.size();
      if (t.navg) {
        t.acoarse = up(ac); t.afine = up(af);
        if (!t.acoarse || !t.afine) return SGN_ENOMEM;
      }
    }
    for (int l = 0; l < L; l++) {
      Tabs& t = tb_[l];
      t.nxc = (int)xcells[l].size();
      if (t.nxc) {
        t.xcell = up(xcells[l]);
        t.xphi = adev<Real>((size_t)(l ? r : 1) * t.nxc * 4);
        if (!t.xcell || !t.xphi) return SGN_ENOMEM;
        SGN_CK(cudaMemsetAsync(t.xphi, 0, (size_t)(l ? r : 1) * t.nxc * 4 * sizeof(Real), st_));
      }
      int rc = lv_[l]->set_kind(kd[l].data());
      if (rc) return rc;
      rc = lv_[l]->set_xslot(xs[l].data());
      if (rc) return rc;
    }
    // level 0's planes, to give them back if a regrid's hierarchy that took
    // over this level 0 is deleted before it is committed
    kd0_ = std::move(kd[0]);
    xs0_ = std::move(xs[0]);
    // each level keeps its solver's default schedule: the one-pass kernel in
    // mixed precision where the atlas gives the resident blocks enough tiles,
    // else the kernel sequence (both export the same fluxes and give sibling
    // ghosts the same positivity factors, so the levels may differ)
    sc_ = adev<double>(8);
    if (!sc_) return SGN_ENOMEM;
    SGN_CK(cudaMemsetAsync(sc_, 0, 8 * sizeof(double), st_));
    size_t mx = 0;
    for (auto& v : bx_)
      for (auto& b : v) mx = std::max(mx, (size_t)b.nx * b.ny);
    staging_ = adev<double>(mx * NV);
    if (!staging_) return SGN_ENOMEM;
    stage_bytes_ = mx * NV * sizeof(double);
    // step bookkeeping
    dt_.L = L; dt_.strang = prm_.strang; dt_.cfl = prm_.cfl;
    double Rl = 1.0;
    for (int l = 0; l < L; l++) {
      Dev<Real>& d = lv_[l]->dev();
      dt_.R[l] = Rl; Rl *= r;
      dt_.dx[l] = d.dx; dt_.dy[l] = d.dy;
      dt_.smax[l] = d.smax; dt_.cmax[l] = d.cmax; dt_.dt[l] = d.dt; dt_.lam[l] = d.lam;
      dt_.lamf[l] = sizeof(Real) == 4 ? (float*)d.lamr : nullptr;
      dt_.lamd[l] = sizeof(Real) == 8 ? (double*)d.lamr : nullptr;
    }
    dt_.status = lv_[0]->dev().status;
    dt_.sc = sc_;
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaStreamSynchronize(st_));
    fresh_ = true;
    return SGN_OK;
  }

  // padded atlas index of frame cell (I, J) of box b on level l
  int pidx(int l, const Box& b, int I, int J) const {
    return (int)((size_t)(b.py + J) * lv_[l]->dev().pitch + (b.px + I));
  }

  // a cell filled from the parent level: parent cell (padded), its stencil,
  // the cell (padded) and its sub-cell offsets sx | sy << 8
  struct ParEnt { int src; int4 nb; int dst, sub; };

  // Ghost cell (X, Y) of a level-l patch b (inside the domain, no level-l
  // patch holds it): limited interpolation from its parent cell, which lies in
  // b's parent box P; the stencil cells come from whichever level-(l-1) patch
  // holds them (-1: none, or outside the domain).  False if the parent cell is
  // not inside P (the box rules exclude this).
  bool par_entry(int l, const Box& b, int X, int Y, int dst, ParEnt& e) const {
    const int r = r_, ic = X / r, jc = Y / r;
    const Box& P = bx_[l - 1][b.parent];
    if (ic < P.i0 || ic >= P.i0 + P.nx || jc < P.j0 || jc >= P.j0 + P.ny) return false;
    e.src = pidx(l - 1, P, ic - P.i0 + G, jc - P.j0 + G);
    e.dst = dst;
    e.sub = (X % r) | ((Y % r) << 8);
    auto nb = [&](int x, int y) -> int {
      if (x < 0 || y < 0 || x >= NX_[l - 1] || y >= NY_[l - 1]) return -1;
      const int o = own_[l - 1].find(x, y);
      if (o < 0) return -1;
      const Box& Q = bx_[l - 1][o];
      return pidx(l - 1, Q, x - Q.i0 + G, y - Q.j0 + G);
    };
    e.nb = make_int4(nb(ic - 1, jc), nb(ic + 1, jc), nb(ic, jc - 1), nb(ic, jc + 1));
    return true;
  }

  // groups of parent-filled cells by parent cell (parent order, cells in
  // creation order), at most kParChunk cells a group -- a parent cell with
  // more starts another group, so that small fills keep enough threads --
  // uploaded; false: out of device memory
  static constexpr int kParChunk = 4;
  bool upload_par(const std::vector<ParEnt>& v, ParTab& t) {
    t = ParTab{};
    if (v.empty()) return true;
    std::vector<int> ord(v.size());
    for (size_t i = 0; i < ord.size(); i++) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return v[a].src < v[b].src; });
    std::vector<int> src, first, dst, sub;
    std::vector<int4> nb;
    for (size_t i = 0; i < ord.size(); i++) {
      const ParEnt& e = v[ord[i]];
      if (i == 0 || e.src != v[ord[i - 1]].src || (int)dst.size() - first.back() >= kParChunk) {
        src.push_back(e.src);
        nb.push_back(e.nb);
        first.push_back((int)dst.size());
      }
      dst.push_back(e.dst);
      sub.push_back(e.sub);
    }
    first.push_back((int)dst.size());
    t.src = up(src); t.nb = up(nb); t.first = up(first); t.dst = up(dst); t.sub = up(sub);
    t.n = (int)src.size();
    return t.src && t.nb && t.first && t.dst && t.sub;
  }

  int set_patch(int l, int k, const double* q) override {
    if (l < 0 || l >= L_ || k < 0 || k >= (int)bx_[l].size() || !q) return SGN_EINVAL;
    const Box& b = bx_[l][k];
    size_t n = (size_t)b.nx * b.ny * NV;
    SGN_CK(cudaMemcpyAsync(staging_, q, n * sizeof(double), cudaMemcpyHostToDevice, st_));
    dim3 gr((b.nx + 31) / 32, (b.ny + 7) / 8);
    k_amr_pack<MODEL, Real><<<gr, dim3(32, 8), 0, st_>>>(lv_[l]->dev(), staging_, b.px + G, b.py + G, b.nx, b.ny,
                                                          lv_[l]->cur());
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaStreamSynchronize(st_));
    fresh_ = true;
    return SGN_OK;
  }

  int get_patch(int l, int k, double* q) override {
    if (l < 0 || l >= L_ || k < 0 || k >= (int)bx_[l].size() || !q) return SGN_EINVAL;
    const Box& b = bx_[l][k];
    size_t n = (size_t)b.nx * b.ny * NV;
    dim3 gr((b.nx + 31) / 32, (b.ny + 7) / 8);
    k_amr_unpack<MODEL, Real><<<gr, dim3(32, 8), 0, st_>>>(lv_[l]->dev(), staging_, b.px + G, b.py + G, b.nx,
                                                            b.ny, lv_[l]->cur());
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaMemcpyAsync(q, staging_, n * sizeof(double), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    return SGN_OK;
  }

  // speeds of the current states -> dt0 and the level steps; clears time,
  // status and clipping
  int begin() {
    for (int l = 0; l < L_; l++) {
      Dev<Real>& d = lv_[l]->dev();
      SGN_CK(cudaMemsetAsync(d.status, 0, sizeof(unsigned), st_));
      SGN_CK(cudaMemsetAsync(d.smax, 0, 2 * sizeof(unsigned long long), st_));
      k_speed<MODEL, Real><<<lv_[l]->grid_interior(), dim3(32, 8), 0, st_>>>(d, lv_[l]->cur());
    }
    SGN_CK(cudaMemsetAsync(sc_ + 1, 0, 4 * sizeof(double), st_));
    k_amr_finalize<<<1, 32, 0, st_>>>(dt_, 0);
    SGN_CK(cudaGetLastError());
    fresh_ = false;
    return SGN_OK;
  }

  // one level-l step at substep ksub of its parent, then the finer levels
  void run_level(cudaStream_t s, int l, int ksub, int& nl) {
    Solver<MODEL, Real>* S = lv_[l];
    Tabs& t = tb_[l];
    const int c = S->cur();
    if (l > 0) {
      Solver<MODEL, Real>* P = lv_[l - 1];
      const int pnew = P->cur(), pold = 1 - pnew;   // the parent has stepped already
      if (t.nfill || t.par.n) {
        k_amr_fill<MODEL, Real><<<grid1(t.par.n + t.nfill), 256, 0, s>>>(S->dev(), P->dev(), t.par, t.fill, t.nfill,
                                                                           c, pold, pnew, (double)ksub / r_, r_);
        nl++;
      }
      if (t.nbc) { k_amr_fill_bc<MODEL, Real><<<grid1(t.nbc), 256, 0, s>>>(S->dev(), t.bc, t.nbc, c); nl++; }
    }
    // this step's slice of the level's export buffer
    Real* xp = t.nxc ? t.xphi + (size_t)ksub * t.nxc * 4 : nullptr;
    if (S->schedule() == SCHED_FUSED) {
      S->launch_fused(s, c, xp);
      nl++;
    } else {
      S->launch_phase1(s, c);
      nl += 6;
      if (l > 0 && t.nfill) { k_amr_theta<Real><<<grid1(t.nfill), 256, 0, s>>>(S->dev(), t.fill, t.nfill); nl++; }
      if (t.nxc) { k_amr_export<Real><<<grid1(t.nxc), 256, 0, s>>>(S->dev(), t.xcell, t.nxc, xp); nl++; }
      S->launch_phase2(s, c);
      nl++;
    }
    S->flip();
    if (l + 1 < L_) {
      for (int k = 0; k < r_; k++) run_level(s, l + 1, k, nl);
      if (t.navg || t.ncell) {
        const Tabs& u = tb_[l + 1];
        k_amr_avg_reflux<MODEL, Real><<<grid1(t.navg + t.ncell), 256, 0, s>>>(
            S->dev(), lv_[l + 1]->dev(), t.acoarse, t.afine, t.navg, t.rcell, t.rfirst, t.ncell, t.rcref, t.rdir,
            t.rsgn, t.rfref, xp, u.xphi, (size_t)u.nxc * 4, S->cur(), lv_[l + 1]->cur(), r_, dx_[l] * dx_[l],
            sc_ + 4);
        nl++;
      }
    }
  }

  unsigned curbits() const {
    unsigned v = 0;
    for (int l = 0; l < L_; l++) v |= (unsigned)lv_[l]->cur() << l;
    return v;
  }
  void setcur(unsigned v) {
    for (int l = 0; l < L_; l++)
      if (((v >> l) & 1u) != (unsigned)lv_[l]->cur()) lv_[l]->flip();
  }

  int launch_one() {
    unsigned key = curbits();
    auto it = graphs_.find(key);
    if (it == graphs_.end()) {
      cudaGraph_t gr;
      SGN_CK(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
      int nl = 0;
      run_level(cap_, 0, 0, nl);
      k_amr_finalize<<<1, 32, 0, cap_>>>(dt_, 1);
      nl++;
      unsigned after = curbits();
      setcur(key);
      cudaError_t e = cudaStreamEndCapture(cap_, &gr);
      if (e != cudaSuccess) return SGN_ECUDA;
      cudaGraphExec_t gx;
      e = cudaGraphInstantiate(&gx, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) return SGN_ECUDA;
      it = graphs_.emplace(key, std::make_pair(gx, after)).first;
      launches_ = nl;
    }
    SGN_CK(cudaGraphLaunch(it->second.first, st_));
    setcur(it->second.second);
    return SGN_OK;
  }

  int finish(double* t_out) {
    unsigned st = 0;
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaMemcpyAsync(hsc_, sc_ + 1, sizeof(double), cudaMemcpyDeviceToHost, st_));
    for (int l = 0; l < L_; l++)
      SGN_CK(cudaMemcpyAsync((unsigned*)(hsc_ + 2) + l, lv_[l]->dev().status, sizeof(unsigned),
                             cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    for (int l = 0; l < L_; l++) st |= ((unsigned*)(hsc_ + 2))[l];
    if (t_out) *t_out = hsc_[0];
    return status_to_error(st);
  }

  int set_retake(int max_retakes) override {
    if (max_retakes < 0 || max_retakes > 16) return SGN_EINVAL;
    if (max_retakes > 0 && !bsc_) {
      bsc_ = adev<double>(8 + AMR_MAXL);
      if (!bsc_) return SGN_ENOMEM;
      bak_.assign(L_, nullptr);
      for (int l = 1; l < L_; l++) {
        bak_[l] = adev<Real>((size_t)NV * lv_[l]->dev().fs);
        if (!bak_[l]) return SGN_ENOMEM;
      }
    }
    retake_max_ = max_retakes;
    return SGN_OK;
  }
  long long retakes() const override { return retakes_; }

  // the scalars, status words and finer states before a level-0 step
  void backup() {
    cudaMemcpyAsync(bsc_, sc_, 8 * sizeof(double), cudaMemcpyDeviceToDevice, st_);
    for (int l = 0; l < L_; l++)
      cudaMemcpyAsync((unsigned*)(bsc_ + 8) + l, lv_[l]->dev().status, sizeof(unsigned), cudaMemcpyDeviceToDevice,
                      st_);
    for (int l = 1; l < L_; l++) {
      const Dev<Real>& d = lv_[l]->dev();
      cudaMemcpyAsync(bak_[l], d.q[lv_[l]->cur()], (size_t)NV * d.fs * sizeof(Real), cudaMemcpyDeviceToDevice, st_);
    }
  }
  void restore(unsigned key) {
    setcur(key);
    cudaMemcpyAsync(sc_, bsc_, 8 * sizeof(double), cudaMemcpyDeviceToDevice, st_);
    for (int l = 0; l < L_; l++)
      cudaMemcpyAsync(lv_[l]->dev().status, (unsigned*)(bsc_ + 8) + l, sizeof(unsigned), cudaMemcpyDeviceToDevice,
                      st_);
    for (int l = 1; l < L_; l++) {
      const Dev<Real>& d = lv_[l]->dev();
      cudaMemcpyAsync(d.q[lv_[l]->cur()], bak_[l], (size_t)NV * d.fs * sizeof(Real), cudaMemcpyDeviceToDevice, st_);
    }
  }

  // One level-0 step (its dt already on the device) with retaking: a step
  // whose largest face Courant number exceeded 1 on any level is undone and
  // taken again with dt0 * CFL / Courant, up to retake_max_ times (Sec. 4:
  // CFL step with subcycling; the step-size controller of Sec. 7 acts on wave
  // speeds that can grow within a level-0 step).
  int step_retake() {
    const unsigned key = curbits();
    backup();
    for (int k = 0;; k++) {
      int rc = launch_one();
      if (rc) return rc;
      SGN_CK(cudaMemcpyAsync(hsc_ + 10, sc_ + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st_));
      for (int l = 0; l < L_; l++) {
        SGN_CK(cudaMemcpyAsync((unsigned*)(hsc_ + 2) + l, lv_[l]->dev().status, sizeof(unsigned),
                               cudaMemcpyDeviceToHost, st_));
        SGN_CK(cudaMemcpyAsync((unsigned*)(hsc_ + 12) + l, (unsigned*)(bsc_ + 8) + l, sizeof(unsigned),
                               cudaMemcpyDeviceToHost, st_));
      }
      SGN_CK(cudaStreamSynchronize(st_));
      unsigned now = 0, before = 0;
      for (int l = 0; l < L_; l++) {
        now |= ((unsigned*)(hsc_ + 2))[l];
        before |= ((unsigned*)(hsc_ + 12))[l];
      }
      // only a CFL flag this step raised, on a step that stayed finite
      if (!(now & ST_CFL) || (before & ST_CFL) || (now & (ST_NONFINITE | ST_NEGDEPTH))) return SGN_OK;
      const double dt_used = hsc_[10], courant = hsc_[11];
      if (k >= retake_max_ || !(courant > 1.0) || !(dt_used > 0.0)) return SGN_ECFL;
      restore(key);
      k_amr_setdt<<<1, 32, 0, st_>>>(dt_, dt_used * prm_.cfl / courant);
      SGN_CK(cudaGetLastError());
      retakes_++;
    }
  }

  int step(int n, double* t_out) override {
    if (n < 0) return SGN_EINVAL;
    if (fresh_) { int rc = begin(); if (rc) return rc; }
    for (int i = 0; i < n; i++) {
      int rc = retake_max_ > 0 ? step_retake() : launch_one();
      if (rc == SGN_ECFL) break;
      if (rc) return rc;
    }
    return finish(t_out);
  }

  int step_dt(double dt0) override {
    if (!(dt0 > 0)) return SGN_EINVAL;
    if (fresh_) { int rc = begin(); if (rc) return rc; }
    k_amr_setdt<<<1, 32, 0, st_>>>(dt_, dt0);
    int rc = retake_max_ > 0 ? step_retake() : launch_one();
    if (rc && rc != SGN_ECFL) return rc;
    return finish(nullptr);
  }

  int next_dt(double* dt0) override {
    if (fresh_) { int rc = begin(); if (rc) return rc; }
    SGN_CK(cudaMemcpyAsync(hsc_, sc_, sizeof(double), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    *dt0 = hsc_[0];
    return SGN_OK;
  }

  int mass(double* m, double* clipped) override {
    double tot = 0.0;
    for (int l = 0; l < L_; l++) {
      Dev<Real>& d = lv_[l]->dev();
      k_amr_mass1<Real><<<592, 256, 0, st_>>>(d, lv_[l]->cur());
      k_mass2<Real><<<1, 256, 0, st_>>>(d, 592);
      SGN_CK(cudaGetLastError());
      SGN_CK(cudaMemcpyAsync(hsc_ + 8, d.mass, sizeof(double), cudaMemcpyDeviceToHost, st_));
      SGN_CK(cudaStreamSynchronize(st_));
      tot += hsc_[8];
    }
    SGN_CK(cudaMemcpyAsync(hsc_ + 9, sc_ + 4, sizeof(double), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    if (m) *m = tot;
    if (clipped) *clipped = hsc_[9];
    return SGN_OK;
  }

  void drop_amr_graphs() {
    for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second.first);
    graphs_.clear();
  }

  // Tunes each level (launch shapes and schedule, the one-pass kernel among
  // them in mixed precision) on its own atlas.
  int autotune(int reps, int* ch, double* ms) override {
    if (reps < 1 || reps > 10000) return SGN_EINVAL;
    SGN_CK(cudaStreamSynchronize(st_));
    for (int l = 0; l < L_; l++) {
      int rc = lv_[l]->autotune(reps, ch ? ch + l * TU_N : nullptr, ms ? ms + l * TU_N * TU_OPTS : nullptr);
      if (rc) return rc;
    }
    drop_amr_graphs();
    return SGN_OK;
  }

  // One tuning per level (the one-pass schedule only in mixed precision).
  int set_tuning(const int* ch) override {
    if (!ch) return SGN_EINVAL;
    for (int l = 0; l < L_; l++)
      for (int k = 0; k < TU_N; k++)
        if (ch[l * TU_N + k] < 0 || ch[l * TU_N + k] >= (k == TU_SCHED ? SCHED_N : TU_OPTS)) return SGN_EINVAL;
    for (int l = 0; l < L_; l++)
      if (ch[l * TU_N + TU_SCHED] == SCHED_FUSED && sizeof(Real) != 4) return SGN_EINVAL;
    for (int l = 0; l < L_; l++) {
      int rc = lv_[l]->set_tuning(ch + l * TU_N);
      if (rc) return rc;
    }
    drop_amr_graphs();
    return SGN_OK;
  }

  void dims(int l, int* NX, int* NY) const override { *NX = NX_[l]; *NY = NY_[l]; }

  int get_level_device(int l, int nf, double* out) override {
    if (l < 0 || l >= L_ || nf < 1 || nf > NV || !out) return SGN_EINVAL;
    const int nb = (int)bx_[l].size();
    if (nb == 0) return SGN_OK;
    if (nb > 65535) return SGN_ERANGE;
    if (!scat_[l]) {
      std::vector<int> t(6 * (size_t)nb);
      int mx = 1, my = 1;
      for (int k = 0; k < nb; k++) {
        const Box& b = bx_[l][k];
        int* e = &t[6 * (size_t)k];
        e[0] = b.px + G; e[1] = b.py + G; e[2] = b.nx; e[3] = b.ny; e[4] = b.i0; e[5] = b.j0;
        mx = std::max(mx, b.nx);
        my = std::max(my, b.ny);
      }
      int* dt = adev<int>(t.size());
      if (!dt) return SGN_ENOMEM;
      SGN_CK(cudaMemcpyAsync(dt, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice, st_));
      SGN_CK(cudaStreamSynchronize(st_));
      scat_[l] = dt;
      scat_mx_[l] = mx;
      scat_my_[l] = my;
    }
    dim3 gr((scat_mx_[l] + 31) / 32, (scat_my_[l] + 7) / 8, nb);
    k_amr_scatter<MODEL, Real><<<gr, dim3(32, 8), 0, st_>>>(lv_[l]->dev(), scat_[l], nf, out, NX_[l], NY_[l],
                                                             lv_[l]->cur());
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaStreamSynchronize(st_));
    return SGN_OK;
  }

  void boxes(int l, std::vector<int>& out) const override {
    out.clear();
    for (const Box& b : bx_[l]) out.insert(out.end(), {b.i0, b.j0, b.nx, b.ny});
  }

  int flags(int l, double tol, std::vector<unsigned char>& flag, std::vector<unsigned char>& have) override {
    Dev<Real>& d = lv_[l]->dev();
    unsigned char* fd = (unsigned char*)staging_;   // >= nvar doubles per cell of the largest patch
    std::vector<unsigned char> atl(d.fs);
    if ((size_t)d.fs > stage_bytes_) {
      if (!flag_buf_ || flag_cap_ < d.fs) {
        flag_buf_ = adev<unsigned char>(d.fs);
        if (!flag_buf_) return SGN_ENOMEM;
        flag_cap_ = d.fs;
      }
      fd = flag_buf_;
    }
    dim3 gr((d.nxp + 31) / 32, (d.nyp + 7) / 8);
    k_amr_flag<Real><<<gr, dim3(32, 8), 0, st_>>>(d, lv_[l]->cur(), tol, fd);
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaMemcpyAsync(atl.data(), fd, d.fs, cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    flag.assign((size_t)NX_[l] * NY_[l], 0);
    have.assign((size_t)NX_[l] * NY_[l], 0);
    for (const Box& b : bx_[l])
      for (int j = 0; j < b.ny; j++)
        for (int i = 0; i < b.nx; i++) {
          const size_t o = (size_t)(b.j0 + j) * NX_[l] + (b.i0 + i);
          flag[o] = atl[(size_t)pidx(l, b, i + G, j + G)];
          have[o] = 1;
        }
    return SGN_OK;
  }

  // Regridding (reading A11 of the refinement oracle): this hierarchy, just
  // created with new boxes over the same grid, takes the state of `ob`.
  // Level 0 is copied; then, coarse to fine, every interior cell of a new
  // patch takes the old patch's cell of the same level where one covered it,
  // else the limited interpolation of the ghost cells (A4) from the new parent
  // at its current state; then every level is averaged down (A8), finest
  // first.  The time and the clipped water carry over; the time step is
  // recomputed from the new states; the status starts clear.
  int take_state(AmrBase* ob) override {
    auto* o = dynamic_cast<Amr<MODEL, Real>*>(ob);
    if (!o || o->L_ != L_ || o->r_ != r_ || o->NX_ != NX_ || o->NY_ != NY_) return SGN_EINVAL;
    const int r = r_;
    SGN_CK(cudaStreamSynchronize(o->st_));
    SGN_CK(cudaStreamSynchronize(st_));
    if (o->lv_[0]) {   // level 0 not taken over: copy its state
      Dev<Real>& n0 = lv_[0]->dev();
      Dev<Real>& o0 = o->lv_[0]->dev();
      if (n0.fs != o0.fs || n0.pitch != o0.pitch) return SGN_EINVAL;
      SGN_CK(cudaMemcpyAsync(n0.q[lv_[0]->cur()], o0.q[o->lv_[0]->cur()], (size_t)NV * n0.fs * sizeof(Real),
                             cudaMemcpyDeviceToDevice, st_));
    }
    for (int l = 1; l < L_; l++) {
      Owner oo;
      oo.build(o->bx_[l], NX_[l], NY_[l]);
      std::vector<int> cd, cs;
      std::vector<ParEnt> par;
      for (const Box& b : bx_[l]) {
        for (int j = 0; j < b.ny; j++)
          for (int i = 0; i < b.nx;) {
            const int X = b.i0 + i, Y = b.j0 + j, dst = pidx(l, b, i + G, j + G);
            const int k = oo.find(X, Y);
            if (k >= 0) {
              // the run of this row that the old box covers
              const Box& s = o->bx_[l][k];
              const int m = std::min(b.nx - i, s.i0 + s.nx - X);
              const int src = o->pidx(l, s, X - s.i0 + G, Y - s.j0 + G);
              for (int q = 0; q < m; q++) {
                cd.push_back(dst + q);
                cs.push_back(src + q);
              }
              i += m;
              continue;
            }
            ParEnt e;
            if (!par_entry(l, b, X, Y, dst, e)) return SGN_EINVAL;
            par.push_back(e);
            i++;
          }
      }
      if (!cd.empty()) {
        int* dd = up(cd);
        int* ds = up(cs);
        if (!dd || !ds) return SGN_ENOMEM;
        k_amr_copy<MODEL, Real><<<grid1((int)cd.size()), 256, 0, st_>>>(
            lv_[l]->dev(), o->lv_[l]->dev(), dd, ds, (int)cd.size(), lv_[l]->cur(), o->lv_[l]->cur());
      }
      if (!par.empty()) {
        ParTab pt;
        if (!upload_par(par, pt)) return SGN_ENOMEM;
        const int pc = lv_[l - 1]->cur();
        k_amr_fill<MODEL, Real><<<grid1(pt.n), 256, 0, st_>>>(lv_[l]->dev(), lv_[l - 1]->dev(), pt, nullptr, 0,
                                                               lv_[l]->cur(), pc, pc, 0.0, r);
      }
      SGN_CK(cudaGetLastError());
    }
    for (int l = L_ - 2; l >= 0; l--)
      if (tb_[l].navg)
        k_amr_avg_reflux<MODEL, Real><<<grid1(tb_[l].navg), 256, 0, st_>>>(
            lv_[l]->dev(), lv_[l + 1]->dev(), tb_[l].acoarse, tb_[l].afine, tb_[l].navg, nullptr, nullptr, 0, nullptr,
            nullptr, nullptr, nullptr, nullptr, nullptr, 0, lv_[l]->cur(), lv_[l + 1]->cur(), r, 0.0, nullptr);
    SGN_CK(cudaGetLastError());
    int rc = begin();
    if (rc) return rc;
    SGN_CK(cudaMemcpyAsync(sc_ + 1, o->sc_ + 1, sizeof(double), cudaMemcpyDeviceToDevice, st_));
    SGN_CK(cudaMemcpyAsync(sc_ + 4, o->sc_ + 4, sizeof(double), cudaMemcpyDeviceToDevice, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    donor_ = nullptr;   // committed: the level-0 solver is this hierarchy's
    return SGN_OK;
  }

  int status(unsigned* f) override {
    for (int l = 0; l < L_; l++)
      SGN_CK(cudaMemcpyAsync((unsigned*)(hsc_ + 2) + l, lv_[l]->dev().status, sizeof(unsigned),
                             cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    unsigned s = 0;
    for (int l = 0; l < L_; l++) s |= ((unsigned*)(hsc_ + 2))[l];
    if (f) *f = s;
    return SGN_OK;
  }
};

}  // namespace sgn
