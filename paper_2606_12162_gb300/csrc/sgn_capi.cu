// sgn_capi.cu -- the extern "C" entry points of include/sgn.h: argument checks,
// then dispatch to the solver object of the model and precision.
#include <math.h>
#include <new>

#include "sgn_solver.cuh"

struct sgn_solver {
  sgn::SolverBase* impl;
  int model;
};

// Error of the kernels' FP64 reciprocal and square root against the IEEE
// results of CUDA's division and sqrt, in units in the last place of the IEEE
// result: err[2i] for rcp(x[i]), err[2i+1] for sqrt(x[i]).
__global__ void k_math_check(const double* x, int n, double* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = x[i];
  double r0 = 1.0 / v, r1 = sgn::rcp(v);
  double q0 = sqrt(v), q1 = sgn::sqrt_nr(v);
  // one unit in the last place: the distance to the next representable double
  double ur = fabs(__longlong_as_double(__double_as_longlong(r0) + 1) - r0);
  double uq = fabs(__longlong_as_double(__double_as_longlong(q0) + 1) - q0);
  err[2 * i] = ur > 0 ? fabs(r1 - r0) / ur : 0.0;
  err[2 * i + 1] = uq > 0 ? fabs(q1 - q0) / uq : 0.0;
}

// The same for the FP32 reciprocal and square root of the mixed path, in units
// in the last place of the FP32 IEEE result (correctly rounded division and sqrtf).
__global__ void k_math_check_f32(const float* x, int n, double* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = x[i];
  float r0 = __fdiv_rn(1.0f, v), r1 = sgn::rcp(v);
  float q0 = __fsqrt_rn(v), q1 = sgn::sqrt_nr(v);
  float ur = fabsf(__int_as_float(__float_as_int(r0) + 1) - r0);
  float uq = fabsf(__int_as_float(__float_as_int(q0) + 1) - q0);
  err[2 * i] = ur > 0 ? fabs((double)r1 - (double)r0) / ur : 0.0;
  err[2 * i + 1] = uq > 0 ? fabs((double)q1 - (double)q0) / uq : 0.0;
}

extern "C" {

int sgn_math_check_f32(const float* x_dev, int n, double* err_dev) {
  if (!x_dev || !err_dev || n < 0) return SGN_EINVAL;
  if (n == 0) return SGN_OK;
  k_math_check_f32<<<(n + 255) / 256, 256>>>(x_dev, n, err_dev);
  if (cudaGetLastError() != cudaSuccess) return SGN_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? SGN_OK : SGN_ECUDA;
}

int sgn_math_check(const double* x_dev, int n, double* err_dev) {
  if (!x_dev || !err_dev || n < 0) return SGN_EINVAL;
  if (n == 0) return SGN_OK;
  k_math_check<<<(n + 255) / 256, 256>>>(x_dev, n, err_dev);
  if (cudaGetLastError() != cudaSuccess) return SGN_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? SGN_OK : SGN_ECUDA;
}

void sgn_default_params(sgn_params* p) {
  if (!p) return;
  p->alpha = 3.0;
  p->h_star = 0.0;
  p->n_transition = 1;
  p->xi0 = 0.01;
  p->xi1 = 0.05;
  p->cfl = 0.9;
  p->g = 9.81;
  p->dry_tol = 1e-3;
  p->limiter = SGN_LIM_MC;
  p->strang = 1;
  p->precision = SGN_FP64;
}

int sgn_nvar(int model) {
  switch (model) {
    case SGN_SWE: return 3;
    case SGN_MBHSGN: return 5;
    case SGN_HSGN: return 7;
  }
  return SGN_EINVAL;
}

const char* sgn_strerror(int code) {
  switch (code) {
    case SGN_OK: return "ok";
    case SGN_EINVAL: return "invalid argument";
    case SGN_ENOMEM: return "device allocation failed";
    case SGN_ECUDA: return "CUDA runtime error";
    case SGN_ENEGDEPTH: return "negative water depth";
    case SGN_ENONFINITE: return "non-finite value in the state";
    case SGN_ECFL: return "face Courant number above 1";
    case SGN_ENONHYP: return "loss of hyperbolicity (g h + p + c^2 < 0)";
    case SGN_EALLDRY: return "no wet cell";
    case SGN_ERANGE: return "buffer too small or gauge outside the grid";
  }
  return "unknown error";
}

static int check_args(const sgn_grid* g, const double* b, int model, const sgn_params* p) {
  if (!g || !b || !p) return SGN_EINVAL;
  if (g->nx < 2 || g->ny < 2) return SGN_EINVAL;
  if ((long long)g->nx * g->ny > (1LL << 31)) return SGN_EINVAL;
  if (!(g->dx > 0) || !(g->dy > 0) || !isfinite(g->dx) || !isfinite(g->dy)) return SGN_EINVAL;
  for (int i = 0; i < 4; i++)
    if (g->bc[i] < SGN_BC_WALL || g->bc[i] > SGN_BC_PERIODIC) return SGN_EINVAL;
  if ((g->bc[0] == SGN_BC_PERIODIC) != (g->bc[1] == SGN_BC_PERIODIC)) return SGN_EINVAL;
  if ((g->bc[2] == SGN_BC_PERIODIC) != (g->bc[3] == SGN_BC_PERIODIC)) return SGN_EINVAL;
  if (sgn_nvar(model) < 0) return SGN_EINVAL;
  if (!(p->cfl > 0) || p->cfl > 1.0) return SGN_EINVAL;
  if (!(p->g > 0) || !(p->dry_tol >= 0) || !(p->alpha >= 0)) return SGN_EINVAL;
  if (p->n_transition < 0 || p->n_transition > 2) return SGN_EINVAL;
  if (p->limiter < SGN_LIM_MINMOD || p->limiter > SGN_LIM_NONE) return SGN_EINVAL;
  if (p->precision != SGN_FP64 && p->precision != SGN_MIXED) return SGN_EINVAL;
  if (!(p->xi0 >= 0) || !(p->xi1 > 0)) return SGN_EINVAL;
  return SGN_OK;
}

int sgn_create(const sgn_grid* grid, const double* bathymetry, int model, const sgn_params* params,
               const unsigned char* phi_override, const sgn_allocator* allocator, void* cuda_stream,
               sgn_solver** out) {
  if (!out) return SGN_EINVAL;
  *out = nullptr;
  int r = check_args(grid, bathymetry, model, params);
  if (r) return r;
  if (allocator && (!allocator->alloc || !allocator->free)) return SGN_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SGN_ECUDA;
  sgn::SolverBase* impl = params->precision == SGN_MIXED ? sgn::make_solver_mixed(model)
                                                          : sgn::make_solver_f64(model);
  if (!impl) return SGN_ENOMEM;
  sgn::CreateArgs a;
  a.grid = *grid;
  a.prm = *params;
  a.model = model;
  a.b = bathymetry;
  a.phi = phi_override;
  a.alloc = allocator;
  a.stream = (cudaStream_t)cuda_stream;
  r = impl->init(a);
  if (r) {
    delete impl;
    return r;
  }
  sgn_solver* s = new (std::nothrow) sgn_solver;
  if (!s) { delete impl; return SGN_ENOMEM; }
  s->impl = impl;
  s->model = model;
  *out = s;
  return SGN_OK;
}

int sgn_set_state(sgn_solver* s, const double* q, double t) {
  if (!s || !q || !isfinite(t)) return SGN_EINVAL;
  return s->impl->set_state(q, t, false);
}

int sgn_set_state_device(sgn_solver* s, const double* q_dev, double t) {
  if (!s || !q_dev || !isfinite(t)) return SGN_EINVAL;
  return s->impl->set_state(q_dev, t, true);
}

int sgn_step(sgn_solver* s, int nsteps, double* t_out) {
  if (!s || nsteps < 0) return SGN_EINVAL;
  return s->impl->step(nsteps, t_out);
}

int sgn_step_dt(sgn_solver* s, double dt) {
  if (!s || !(dt > 0) || !isfinite(dt)) return SGN_EINVAL;
  return s->impl->step_dt(dt);
}

int sgn_get_state(sgn_solver* s, int field_mask, double* out, size_t out_len, double* t_out) {
  if (!s || !out || field_mask < 0) return SGN_EINVAL;
  return s->impl->get_state(field_mask, out, out_len, t_out, false);
}

int sgn_get_state_device(sgn_solver* s, double* out_dev, size_t out_len) {
  if (!s || !out_dev) return SGN_EINVAL;
  return s->impl->get_state(0, out_dev, out_len, nullptr, true);
}

int sgn_add_gauges(sgn_solver* s, const double* xy, int n, int capacity) {
  if (!s) return SGN_EINVAL;
  return s->impl->add_gauges(xy, n, capacity);
}

int sgn_gauges(sgn_solver* s, double* out, size_t cap, int* nrec) {
  if (!s) return SGN_EINVAL;
  return s->impl->gauges(out, cap, nrec);
}

int sgn_clear_gauges(sgn_solver* s) {
  if (!s) return SGN_EINVAL;
  return s->impl->clear_gauges();
}

int sgn_status(sgn_solver* s, unsigned* flags, double* last_dt, double* max_courant) {
  if (!s) return SGN_EINVAL;
  return s->impl->status(flags, last_dt, max_courant);
}

int sgn_next_dt(sgn_solver* s, double* dt) {
  if (!s || !s->impl || !dt) return SGN_EINVAL;
  return s->impl->next_dt(dt);
}

int sgn_mass(sgn_solver* s, double* mass) {
  if (!s || !mass) return SGN_EINVAL;
  return s->impl->mass(mass);
}

int sgn_set_c2(sgn_solver* s, const double* c2) {
  if (!s || !c2) return SGN_EINVAL;
  return s->impl->set_c2(c2);
}

int sgn_well_prepare(sgn_solver* s) {
  if (!s) return SGN_EINVAL;
  return s->impl->well_prepare();
}

int sgn_get_aux(sgn_solver* s, double* c2, unsigned char* phi) {
  if (!s) return SGN_EINVAL;
  return s->impl->get_aux(c2, phi);
}

int sgn_set_profiling(sgn_solver* s, int enable) {
  if (!s) return SGN_EINVAL;
  return s->impl->set_profiling(enable);
}

int sgn_kernel_times(sgn_solver* s, const char** names, double* ms, long* launches, int n) {
  if (!s || n < 0) return SGN_EINVAL;
  return s->impl->kernel_times(names, ms, launches, n);
}

int sgn_launches_per_step(sgn_solver* s) {
  if (!s) return SGN_EINVAL;
  return s->impl->launches_per_step();
}

int sgn_autotune(sgn_solver* s, int reps, int* choice, double* ms) {
  if (!s) return SGN_EINVAL;
  return s->impl->autotune(reps, choice, ms);
}

int sgn_set_tuning(sgn_solver* s, const int* choice) {
  if (!s || !choice) return SGN_EINVAL;
  return s->impl->set_tuning(choice);
}

int sgn_get_tuning(sgn_solver* s, int* choice, int* bx, int* by) {
  if (!s) return SGN_EINVAL;
  return s->impl->get_tuning(choice, bx, by);
}

void sgn_destroy(sgn_solver* s) {
  if (!s) return;
  delete s->impl;
  delete s;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// refined hierarchy (include/sgn_amr.h)
#include "sgn_amr.cuh"

struct sgn_amr {
  sgn::AmrBase* impl;
  sgn::AmrArgs args;        // creation arguments (boxes and bathymetry pointer not kept)
  sgn_allocator alloc;
  bool has_alloc;
  int retake = 0;           // retakes per level-0 step (kept across regrids)
  long long retaken = 0;    // steps retaken by the hierarchies that regrids replaced
};

// a hierarchy from creation arguments and a box list (validated by init)
static int amr_build(sgn::AmrArgs& a, const int* nboxes, const int* boxes, sgn::AmrBase** out) {
  *out = nullptr;
  a.boxes.clear();
  int off = 0;
  for (int l = 1; l < a.L; l++) {
    if (nboxes[l - 1] < 0) return SGN_EINVAL;
    a.boxes.emplace_back(boxes + 4 * off, boxes + 4 * (off + nboxes[l - 1]));
    off += nboxes[l - 1];
  }
  sgn::AmrBase* impl = a.prm.precision == SGN_MIXED ? sgn::make_amr_mixed(a.model) : sgn::make_amr_f64(a.model);
  if (!impl) return SGN_ENOMEM;
  int r = impl->init(a);
  if (r) {
    delete impl;
    return r;
  }
  *out = impl;
  return SGN_OK;
}

// Box lists from refinement flags (reading A12 of the refinement oracle):
// level by level from the coarsest, flag the level's cells (surface jump to a
// neighbour above tol; where the level has no patch, the flag of the parent
// cell), widen the flags by `buffer` cells, and cut the refinable part of each
// new box of the level (two cells inside its edges except along the domain
// boundary) into tile x tile squares, the last ones clipped (a one-cell
// remainder joins the square before it); every square holding a widened flag
// becomes a box of the next level.
static int flagged_boxes(sgn::AmrBase* impl, int L, int r, double tol, int tile, int buffer,
                         std::vector<std::vector<int>>& out) {
  out.assign(L > 1 ? L - 1 : 0, {});
  std::vector<int> parents;
  impl->boxes(0, parents);
  std::vector<unsigned char> prev;    // final flags of the previous level
  int pNX = 0;
  for (int l = 0; l + 1 < L; l++) {
    int NX, NY;
    impl->dims(l, &NX, &NY);
    std::vector<unsigned char> f, have;
    int rc = impl->flags(l, tol, f, have);
    if (rc) return rc;
    if (l > 0)
      for (int Y = 0; Y < NY; Y++)
        for (int X = 0; X < NX; X++) {
          const size_t o = (size_t)Y * NX + X;
          if (!have[o]) f[o] = prev[(size_t)(Y / r) * pNX + X / r];
        }
    // widen by buffer cells: rows, then columns
    std::vector<unsigned char> t(f.size(), 0), w(f.size(), 0);
    for (int Y = 0; Y < NY; Y++)
      for (int X = 0; X < NX; X++)
        if (f[(size_t)Y * NX + X])
          for (int x = std::max(0, X - buffer); x <= std::min(NX - 1, X + buffer); x++) t[(size_t)Y * NX + x] = 1;
    for (int Y = 0; Y < NY; Y++)
      for (int X = 0; X < NX; X++)
        if (t[(size_t)Y * NX + X])
          for (int y = std::max(0, Y - buffer); y <= std::min(NY - 1, Y + buffer); y++) w[(size_t)y * NX + X] = 1;
    std::vector<int>& nb = out[l];
    for (size_t k = 0; k + 3 < parents.size(); k += 4) {
      const int i0 = parents[k], j0 = parents[k + 1], nx = parents[k + 2], ny = parents[k + 3];
      const int x0 = i0 + (i0 == 0 ? 0 : 2), x1 = i0 + nx - (i0 + nx == NX ? 0 : 2);
      const int y0 = j0 + (j0 == 0 ? 0 : 2), y1 = j0 + ny - (j0 + ny == NY ? 0 : 2);
      // tile x tile squares from the low corner, the last ones clipped; a
      // one-cell remainder joins the square before it (no box may end one
      // parent cell short of its parent's edge when that edge is the domain's)
      auto piece = [&](int a, int a1) {
        int w = std::min(tile, a1 - a);
        return a1 - (a + w) == 1 ? w + 1 : w;
      };
      for (int ty = y0, th = 0; ty < y1; ty += th) {
        th = piece(ty, y1);
        for (int tx = x0, tw = 0; tx < x1; tx += tw) {
          tw = piece(tx, x1);
          bool any = false;
          for (int y = ty; y < ty + th && !any; y++)
            for (int x = tx; x < tx + tw; x++)
              if (w[(size_t)y * NX + x]) { any = true; break; }
          if (any) nb.insert(nb.end(), {tx * r, ty * r, tw * r, th * r});
        }
      }
    }
    parents = nb;
    prev.swap(f);
    pNX = NX;
  }
  return SGN_OK;
}

extern "C" {

int sgn_amr_create(const sgn_grid* grid0, const double* b_finest, int nlevels, int ratio, const int* nboxes,
                   const int* boxes, int model, const sgn_params* params, const sgn_allocator* allocator,
                   void* cuda_stream, sgn_amr** out) {
  if (!out) return SGN_EINVAL;
  *out = nullptr;
  if (!grid0 || !b_finest || !params || nlevels < 1 || nlevels > sgn::AMR_MAXL || ratio < 2 || ratio > 8)
    return SGN_EINVAL;
  if (nlevels > 1 && (!nboxes || !boxes)) return SGN_EINVAL;
  for (int i = 0; i < 4; i++)
    if (grid0->bc[i] != SGN_BC_WALL && grid0->bc[i] != SGN_BC_EXTRAP) return SGN_EINVAL;
  if (grid0->dx != grid0->dy) return SGN_EINVAL;
  long long R = 1;
  for (int l = 1; l < nlevels; l++) R *= ratio;
  if ((long long)grid0->nx * R > (1LL << 30) || (long long)grid0->ny * R > (1LL << 30)) return SGN_EINVAL;
  int r = check_args(grid0, b_finest, model, params);
  if (r) return r;
  if (allocator && (!allocator->alloc || !allocator->free)) return SGN_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return SGN_ECUDA;
  sgn_amr* h = new (std::nothrow) sgn_amr;
  if (!h) return SGN_ENOMEM;
  h->has_alloc = allocator != nullptr;
  if (allocator) h->alloc = *allocator;
  sgn::AmrArgs& a = h->args;
  a.grid = *grid0;
  a.prm = *params;
  a.model = model;
  a.L = nlevels;
  a.r = ratio;
  a.b = b_finest;
  a.alloc = h->has_alloc ? &h->alloc : nullptr;
  a.stream = (cudaStream_t)cuda_stream;
  r = amr_build(a, nboxes, boxes, &h->impl);
  a.b = nullptr;
  a.boxes.clear();
  if (r) {
    delete h;
    return r;
  }
  *out = h;
  return SGN_OK;
}

int sgn_amr_regrid(sgn_amr* h, const double* b_finest, const int* nboxes, const int* boxes) {
  if (!h || !b_finest) return SGN_EINVAL;
  if (h->args.L > 1 && (!nboxes || !boxes)) return SGN_EINVAL;
  sgn::AmrBase* impl = nullptr;
  h->args.b = b_finest;
  h->args.prev = h->impl;
  int r = amr_build(h->args, nboxes, boxes, &impl);
  h->args.b = nullptr;
  h->args.prev = nullptr;
  h->args.boxes.clear();
  if (r) return r;
  // (the new hierarchy may take over the old one's level 0: it hands it
  // back if it is deleted before take_state has succeeded)
  if (h->retake) r = impl->set_retake(h->retake);
  if (!r) r = impl->take_state(h->impl);
  if (r) {
    delete impl;
    return r;
  }
  h->retaken += h->impl->retakes();
  delete h->impl;
  h->impl = impl;
  return SGN_OK;
}

void sgn_amr_destroy(sgn_amr* a) {
  if (!a) return;
  delete a->impl;
  delete a;
}

int sgn_amr_regrid_flagged(sgn_amr* h, const double* b_finest, double tol, int tile, int buffer, int* nboxes) {
  if (!h || !b_finest || !(tol > 0) || !isfinite(tol) || tile < 2 || buffer < 0) return SGN_EINVAL;
  const int L = h->args.L;
  if (L < 2) return SGN_EINVAL;
  std::vector<std::vector<int>> bl;
  int rc = flagged_boxes(h->impl, L, h->args.r, tol, tile, buffer, bl);
  if (rc) return rc;
  std::vector<int> nb(L - 1), flat;
  for (int l = 0; l + 1 < L; l++) {
    nb[l] = (int)bl[l].size() / 4;
    flat.insert(flat.end(), bl[l].begin(), bl[l].end());
  }
  if (flat.empty()) flat.push_back(0);
  rc = sgn_amr_regrid(h, b_finest, nb.data(), flat.data());
  if (rc) return rc;
  if (nboxes)
    for (int l = 0; l + 1 < L; l++) nboxes[l] = nb[l];
  return SGN_OK;
}

int sgn_amr_get_boxes(const sgn_amr* h, int level, int* boxes, int cap) {
  if (!h || level < 0 || level >= h->args.L || cap < 0) return SGN_EINVAL;
  std::vector<int> v;
  h->impl->boxes(level, v);
  const int n = (int)v.size() / 4;
  if (boxes) {
    if (cap < n) return SGN_ERANGE;
    for (size_t i = 0; i < v.size(); i++) boxes[i] = v[i];
  }
  return n;
}

int sgn_amr_npatches(const sgn_amr* a, int level) { return a ? a->impl->npatches(level) : SGN_EINVAL; }

int sgn_amr_set_patch(sgn_amr* a, int level, int patch, const double* q) {
  return (a && q) ? a->impl->set_patch(level, patch, q) : SGN_EINVAL;
}

int sgn_amr_get_level_device(sgn_amr* a, int level, int nfields, double* out_dev) {
  if (!a || !out_dev) return SGN_EINVAL;
  return a->impl->get_level_device(level, nfields, out_dev);
}

int sgn_amr_get_patch(sgn_amr* a, int level, int patch, double* q) {
  return (a && q) ? a->impl->get_patch(level, patch, q) : SGN_EINVAL;
}

int sgn_amr_step(sgn_amr* a, int n, double* t_out) { return a ? a->impl->step(n, t_out) : SGN_EINVAL; }

int sgn_amr_step_dt(sgn_amr* a, double dt0) { return a ? a->impl->step_dt(dt0) : SGN_EINVAL; }

int sgn_amr_next_dt(sgn_amr* a, double* dt0) { return (a && dt0) ? a->impl->next_dt(dt0) : SGN_EINVAL; }

int sgn_amr_mass(sgn_amr* a, double* mass, double* clipped) {
  return a ? a->impl->mass(mass, clipped) : SGN_EINVAL;
}

int sgn_amr_status(sgn_amr* a, unsigned* flags) { return a ? a->impl->status(flags) : SGN_EINVAL; }

int sgn_amr_info(const sgn_amr* a, long long* cells, long long* atlas_cells) {
  return a ? a->impl->info(cells, atlas_cells) : SGN_EINVAL;
}

int sgn_amr_launches_per_step(const sgn_amr* a) { return a ? a->impl->launches_per_step() : SGN_EINVAL; }

int sgn_amr_autotune(sgn_amr* a, int reps, int* choice, double* ms) {
  return a ? a->impl->autotune(reps, choice, ms) : SGN_EINVAL;
}

int sgn_amr_set_tuning(sgn_amr* a, const int* choice) {
  return (a && choice) ? a->impl->set_tuning(choice) : SGN_EINVAL;
}

int sgn_amr_set_retake(sgn_amr* a, int max_retakes) {
  if (!a) return SGN_EINVAL;
  const int r = a->impl->set_retake(max_retakes);
  if (!r) a->retake = max_retakes;
  return r;
}

int sgn_amr_retakes(const sgn_amr* a, long long* count) {
  if (!a || !count) return SGN_EINVAL;
  *count = a->retaken + a->impl->retakes();
  return SGN_OK;
}

}  // extern "C"
