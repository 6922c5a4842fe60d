// sgn_solver.cuh -- host-side solver object: device buffers, the launch sequence
// of one time step, CUDA-graph replay of that sequence, per-kernel timing.
#pragma once
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>
#include <cmath>
#include <vector>

#include "../../include/sgn.h"
#include "sgn_kernels.cuh"
#include "sgn_fused.cuh"

namespace sgn {

struct CreateArgs {
  sgn_grid grid;
  sgn_params prm;
  int model;
  const double* b;
  const unsigned char* phi;
  const sgn_allocator* alloc;
  cudaStream_t stream;
  bool no_initial_state = false;   // leave the state zero (a caller fills it right away)
};

struct SolverBase {
  virtual ~SolverBase() {}
  virtual int init(const CreateArgs& a) = 0;
  virtual int set_state(const double* q, double t, bool device) = 0;
  virtual int step(int n, double* t_out) = 0;
  virtual int step_dt(double dt) = 0;
  virtual int get_state(int mask, double* out, size_t len, double* t_out, bool device) = 0;
  virtual int add_gauges(const double* xy, int n, int cap) = 0;
  virtual int gauges(double* out, size_t cap, int* nrec) = 0;
  virtual int clear_gauges() = 0;
  virtual int status(unsigned* f, double* dt, double* cr) = 0;
  virtual int next_dt(double* dt) = 0;
  virtual int mass(double* m) = 0;
  virtual int get_aux(double* c2, unsigned char* phi) = 0;
  virtual int well_prepare() = 0;
  virtual int set_c2(const double* c2) = 0;
  virtual int set_profiling(int on) = 0;
  virtual int kernel_times(const char** names, double* ms, long* launches, int n) = 0;
  virtual int launches_per_step() = 0;
  virtual int autotune(int reps, int* choice, double* ms) = 0;
  virtual int set_tuning(const int* choice) = 0;
  virtual int get_tuning(int* choice, int* bx, int* by) = 0;
};

SolverBase* make_solver_f64(int model);
SolverBase* make_solver_mixed(int model);

inline int status_to_error(unsigned st) {
  if (st & ST_NONFINITE) return SGN_ENONFINITE;
  if (st & ST_NEGDEPTH) return SGN_ENEGDEPTH;
  if (st & ST_NONHYP) return SGN_ENONHYP;
  if (st & ST_ALLDRY) return SGN_EALLDRY;
  if (st & ST_CFL) return SGN_ECFL;
  return SGN_OK;
}

#define SGN_CK(x)                        \
  do {                                   \
    cudaError_t e_ = (x);                \
    if (e_ != cudaSuccess) return SGN_ECUDA; \
  } while (0)

enum { KN_PREP, KN_FACEX, KN_FACEY, KN_TRANSX, KN_TRANSY, KN_THETA, KN_UPDATE, KN_FINAL, KN_GAUGE, KN_FUSED,
       KN_COUNT };
static const char* const kKernelNames[KN_COUNT] = {"k_prep",   "k_face_x",   "k_face_y", "k_trans_x",
                                                   "k_trans_y", "k_theta",   "k_update", "k_finalize",
                                                   "k_gauge",  "k_step_fused"};

// Autotuner choices (include/sgn.h, SGN_TUNE_*): one launch-shape option per
// tuned kernel, in step order, then the schedule of the step.  Option 0
// is the default of each slot.
enum { TU_PREP, TU_FACEX, TU_FACEY, TU_TRANSX, TU_TRANSY, TU_THETA, TU_UPDATE, TU_SCHED, TU_N };
static const int TU_OPTS = 3;
// schedules of the step: serial, two branches in the first phase, and the one-pass kernel
// (k_step_fused: the whole step in one launch; FP32 bulk, uniform grids only)
enum { SCHED_SERIAL = 0, SCHED_FORK = 1, SCHED_FUSED = 2, SCHED_N = 3 };
// rows per block of the one-pass kernel, by the option of its slot (SGN_TUNE_UPDATE)
static const int kFusedRows[3] = {128, 64, 256};
static_assert(TU_N == SGN_TUNE_N && TU_OPTS == SGN_TUNE_OPTS, "tuning table size");

// Face block shapes (BX, BY) per option; they are template arguments of
// k_face (the shared-memory wave records are sized by them).  FP32: 256 or 512
// threads, 64 registers; FP64: records of 16 values x 8 B x BX x BY within
// 48 KB of static shared memory.
template <bool F32> struct FaceShapes;
template <> struct FaceShapes<true> {
  static constexpr int XB[3] = {128, 64, 256}, XY[3] = {2, 4, 1};
  static constexpr int YB[3] = {32, 32, 64}, YY[3] = {8, 16, 4};
};
template <> struct FaceShapes<false> {
  static constexpr int XB[3] = {64, 32, 128}, XY[3] = {4, 8, 2};
  static constexpr int YB[3] = {16, 32, 16}, YY[3] = {16, 8, 8};
};
// blocks of the kernels that take their shape at run time
static const int kTransShape[3][2] = {{32, 4}, {32, 8}, {64, 4}};
static const int kCellShape[3][2] = {{32, 8}, {32, 4}, {64, 4}};

template <int MODEL, typename Real>
class Solver : public SolverBase {
  static constexpr int NV = MT<MODEL>::NV;
  static constexpr int NF = FT<MODEL>::NF;
  // Face blocks of 256 threads in FP32 (four resident blocks per SM within the
  // 64-register bound; fewer, larger blocks or more registers per thread
  // measured slower): x faces 128 x 2 (one halo face per 126), y faces 32 x 8.
  // FP64: x 64 x 4, y 16 x 16 (the FP64 records of 32 x 16 would exceed 48 KB
  // of static shared memory).
  // These are option 0 of FaceShapes; the autotuner may pick another.
  typedef FaceShapes<sizeof(Real) == 4> FS;
  typedef void (*KFace)(Dev<Real>);
  template <int DIR, int O> static KFace face_fn() {
    return DIR == 0 ? (KFace)k_face<MODEL, Real, 0, FS::XB[O], FS::XY[O]>
                    : (KFace)k_face<MODEL, Real, 1, FS::YB[O], FS::YY[O]>;
  }
  KFace kface_[2][TU_OPTS] = {{face_fn<0, 0>(), face_fn<0, 1>(), face_fn<0, 2>()},
                              {face_fn<1, 0>(), face_fn<1, 1>(), face_fn<1, 2>()}};
  int tune_[TU_N] = {0, 0, 0, 0, 0, 0, 0, 0};
  dim3 tg_[TU_N], tb_[TU_N];    // grid and block of each tuned kernel for the current choices
  cudaStream_t aux_ = nullptr;  // second branch of the forked schedule
  cudaEvent_t fork_[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned long long* save_ = nullptr;   // accumulators kept across autotuning
  float ms_sched_[SCHED_N] = {0.f, 0.f, 0.f};   // autotuner: best step time per schedule

  Dev<Real> d_{};
  sgn_allocator al_{};
  bool own_alloc_ = true;
  cudaStream_t st_ = nullptr, cap_ = nullptr;
  std::vector<void*> bufs_;
  int cur_ = 0;
  double* staging_ = nullptr;   // dense double nv*nx*ny
  double* hscal_ = nullptr;     // pinned host scalars
  cudaGraphExec_t gx_[2] = {nullptr, nullptr};
  bool prof_ = false;
  struct Ev { int k; cudaEvent_t a, b; };
  std::vector<Ev> evs_;
  double kms_[KN_COUNT] = {0};
  long kcnt_[KN_COUNT] = {0};
  dim3 gPad_, gInt_;
  int nmass_ = 0;

  void* dalloc(size_t bytes) {
    void* p = nullptr;
    if (own_alloc_) {
      if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    } else {
      p = al_.alloc(bytes, al_.ctx);
    }
    if (p) bufs_.push_back(p);
    return p;
  }
  template <typename T> T* dnew(size_t n) { return (T*)dalloc(n * sizeof(T) + 256); }

  // grid and block of every tuned kernel from tune_.  Face kernels solve one
  // extra face on each side of a block along their direction: x faces
  // I in [1, nx+3] (BX - 2 per block), y faces J in [1, ny+3] (BY - 2 per block).
  void set_geometry() {
    const int nx = d_.nx, ny = d_.ny;
    auto cell = [&](int k, int w, int h) {
      const int* sh = kCellShape[tune_[k]];
      tb_[k] = dim3(sh[0], sh[1]);
      tg_[k] = dim3((w + sh[0] - 1) / sh[0], (h + sh[1] - 1) / sh[1]);
    };
    cell(TU_PREP, d_.nxp, d_.nyp);
    cell(TU_THETA, nx, ny);
    cell(TU_UPDATE, nx, ny);
    {
      const int bx = FS::XB[tune_[TU_FACEX]], by = FS::XY[tune_[TU_FACEX]];
      tb_[TU_FACEX] = dim3(bx, by);
      tg_[TU_FACEX] = dim3((nx + 1 + bx - 3) / (bx - 2), (ny + 2 + by - 1) / by);
    }
    {
      const int bx = FS::YB[tune_[TU_FACEY]], by = FS::YY[tune_[TU_FACEY]];
      tb_[TU_FACEY] = dim3(bx, by);
      tg_[TU_FACEY] = dim3((nx + 2 + bx - 1) / bx, (ny + 1 + by - 3) / (by - 2));
    }
    {
      const int* sh = kTransShape[tune_[TU_TRANSX]];
      tb_[TU_TRANSX] = dim3(sh[0], sh[1]);
      tg_[TU_TRANSX] = dim3((nx + 3 + sh[0] - 1) / sh[0], (ny + 2 + sh[1] - 1) / sh[1]);
    }
    {
      const int* sh = kTransShape[tune_[TU_TRANSY]];
      tb_[TU_TRANSY] = dim3(sh[0], sh[1]);
      tg_[TU_TRANSY] = dim3((nx + 2 + sh[0] - 1) / sh[0], (ny + 3 + sh[1] - 1) / sh[1]);
    }
  }

  void drop_graphs() {
    for (int i = 0; i < 2; i++)
      if (gx_[i]) { cudaGraphExecDestroy(gx_[i]); gx_[i] = nullptr; }
  }

 public:
  ~Solver() override {
    if (st_) cudaStreamSynchronize(st_);
    drop_graphs();
    for (auto& e : evs_) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (void* p : bufs_) {
      if (own_alloc_) cudaFree(p);
      else al_.free(p, al_.ctx);
    }
    if (hscal_) cudaFreeHost(hscal_);
    if (cap_) cudaStreamDestroy(cap_);
    if (aux_) cudaStreamDestroy(aux_);
    for (auto& e : fork_)
      if (e) cudaEventDestroy(e);
  }

  int init(const CreateArgs& a) override {
    st_ = a.stream;
    if (a.alloc && a.alloc->alloc && a.alloc->free) { al_ = *a.alloc; own_alloc_ = false; }
    int dev = -1;
    SGN_CK(cudaGetDevice(&dev));
    SGN_CK(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
    SGN_CK(cudaMallocHost((void**)&hscal_, 64 * sizeof(double)));
    const sgn_grid& g = a.grid;
    const sgn_params& p = a.prm;
    d_.nx = g.nx; d_.ny = g.ny;
    d_.nxp = g.nx + 2 * NG; d_.nyp = g.ny + 2 * NG;
    d_.pitch = ((d_.nxp + 1) + 31) / 32 * 32;
    d_.fs = (size_t)d_.pitch * (d_.nyp + 1);
    for (int i = 0; i < 4; i++) d_.bc[i] = g.bc[i];
    x0_ = g.x0; y0_ = g.y0;
    d_.dx = g.dx; d_.dy = g.dy; d_.g = p.g; d_.dry_tol = p.dry_tol; d_.cfl = p.cfl;
    d_.xi0 = p.xi0; d_.xi1 = p.xi1; d_.alpha = p.alpha; d_.h_star = p.h_star;
    d_.limiter = p.limiter; d_.strang = p.strang; d_.n_transition = p.n_transition;
    size_t fs = d_.fs;
    d_.q[0] = dnew<Real>(NV * fs); d_.q[1] = dnew<Real>(NV * fs);
    d_.b = dnew<Real>(fs); d_.c2 = dnew<Real>(fs); d_.psx = dnew<Real>(fs); d_.psy = dnew<Real>(fs);
    d_.phi = dnew<unsigned char>(fs);
    d_.W = dnew<Real>(NV * fs);
    if (sizeof(Real) == 8) d_.P = dnew<Real>((size_t)PT<MODEL>::NP * fs);   // primitives: FP64 path only
    d_.FX = dnew<Real>(NF * fs); d_.FY = dnew<Real>(NF * fs);
    d_.TX = dnew<Real>(NV * fs); d_.TY = dnew<Real>(NV * fs);
    d_.theta = dnew<Real>(fs);
    d_.G2 = dnew<double>(fs);
    double* sc = dnew<double>(16);
    unsigned* si = dnew<unsigned>(16);
    staging_ = dnew<double>((size_t)NV * g.nx * g.ny);
    if (!d_.q[0] || !d_.q[1] || !d_.b || !d_.c2 || !d_.psx || !d_.psy || !d_.phi || !d_.W || (sizeof(Real) == 8 && !d_.P) ||
        !d_.FX || !d_.FY || !d_.TX || !d_.TY || !d_.theta || !d_.G2 || !sc || !si || !staging_)
      return SGN_ENOMEM;
    d_.dt = sc; d_.t = sc + 1; d_.last_dt = sc + 2; d_.courant = sc + 3; d_.mass = sc + 4;
    d_.lam = sc + 5;                                   // 4 doubles
    d_.lamr = (Real*)(sc + 12);                        // 4 bulk-type values
    d_.smax = (unsigned long long*)(sc + 10);
    d_.cmax = (unsigned long long*)(sc + 11);
    d_.rdry_tol = (Real)p.dry_tol;
    d_.two_over_g = 2.0 / p.g;
    d_.two_over_g_r = (Real)d_.two_over_g;
    d_.half_g = 0.5 * p.g;
    d_.inv_dx = 1.0 / g.dx;
    d_.inv_dy = 1.0 / g.dy;
    d_.g_r = (Real)p.g;
    d_.inv_dx_r = (Real)d_.inv_dx;
    d_.inv_dy_r = (Real)d_.inv_dy;
    d_.status = si; d_.gn = (int*)(si + 1);
    d_.tiles = si + 4;   // two words, zeroed below and by the last block of every one-pass launch
    // launch geometry
    gPad_ = dim3((d_.nxp + 31) / 32, (d_.nyp + 7) / 8);
    gInt_ = dim3((g.nx + 31) / 32, (g.ny + 7) / 8);
    set_geometry();
    SGN_CK(cudaStreamCreateWithFlags(&aux_, cudaStreamNonBlocking));
    if constexpr (kFusedBuilt) {
      const int smb = (int)sizeof(FusedSmem<MODEL, Real>);
      SGN_CK(cudaFuncSetAttribute(k_step_fused<MODEL, Real, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
      SGN_CK(cudaFuncSetAttribute(k_step_fused<MODEL, Real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
      int per_sm = 0, per_sm_kd = 0, nsm = 0;
      SGN_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_fused<MODEL, Real, false>, FUSED_NT, smb));
      SGN_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_kd, k_step_fused<MODEL, Real, true>, FUSED_NT, smb));
      if (per_sm_kd < per_sm) per_sm = per_sm_kd;
      SGN_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      fused_resident_ = (per_sm > 0 ? per_sm : 1) * (nsm > 0 ? nsm : 1);
      // the default schedule of the mixed path on a single grid, unless the grid
      // is too small to give the resident blocks tiles of at least 32 rows
      if (fused_plan(g.nx, g.ny, 32).ntiles * 2 >= fused_resident_) tune_[TU_SCHED] = SCHED_FUSED;
    }
    for (int k = 0; k < 4; k++) SGN_CK(cudaEventCreateWithFlags(&fork_[k], cudaEventDisableTiming));
    save_ = dnew<unsigned long long>(4);
    if (!save_) return SGN_ENOMEM;
    nmass_ = 1024;
    d_.mass_part = dnew<double>(nmass_);
    if (!d_.mass_part) return SGN_ENOMEM;
    // zero every buffer (faces outside the computed ranges stay 0), theta = 1
    for (size_t k = 0; k < 2; k++) SGN_CK(cudaMemsetAsync(d_.q[k], 0, NV * fs * sizeof(Real), st_));
    SGN_CK(cudaMemsetAsync(d_.W, 0, NV * fs * sizeof(Real), st_));
    if (d_.P) SGN_CK(cudaMemsetAsync(d_.P, 0, PT<MODEL>::NP * fs * sizeof(Real), st_));
    SGN_CK(cudaMemsetAsync(d_.FX, 0, NF * fs * sizeof(Real), st_));
    SGN_CK(cudaMemsetAsync(d_.FY, 0, NF * fs * sizeof(Real), st_));
    SGN_CK(cudaMemsetAsync(d_.TX, 0, NV * fs * sizeof(Real), st_));
    SGN_CK(cudaMemsetAsync(d_.TY, 0, NV * fs * sizeof(Real), st_));
    SGN_CK(cudaMemsetAsync(d_.psx, 0, fs * sizeof(Real), st_));
    SGN_CK(cudaMemsetAsync(d_.psy, 0, fs * sizeof(Real), st_));
    SGN_CK(cudaMemsetAsync(d_.phi, 0, fs, st_));
    SGN_CK(cudaMemsetAsync(sc, 0, 16 * sizeof(double), st_));
    SGN_CK(cudaMemsetAsync(si, 0, 16 * sizeof(unsigned), st_));
    k_fill_one<Real><<<(unsigned)((fs + 255) / 256), 256, 0, st_>>>(d_.theta, fs);
    // setup: padded b and phi override, phi_T, c^2, psi
    size_t n = (size_t)g.nx * g.ny;
    SGN_CK(cudaMemcpyAsync(staging_, a.b, n * sizeof(double), cudaMemcpyHostToDevice, st_));
    unsigned char* phid = nullptr;
    if (a.phi) {
      phid = (unsigned char*)(staging_ + n);
      SGN_CK(cudaMemcpyAsync(phid, a.phi, n, cudaMemcpyHostToDevice, st_));
    }
    k_pack_b<Real><<<gPad_, dim3(32, 8), 0, st_>>>(d_, staging_, phid);
    k_phi<Real><<<gInt_, dim3(32, 8), 0, st_>>>(d_, a.phi ? 1 : 0);
    k_aux<Real><<<dim3((d_.nxp + 1 + 31) / 32, (d_.nyp + 1 + 7) / 8), dim3(32, 8), 0, st_>>>(d_);
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaStreamSynchronize(st_));
    if (a.no_initial_state) return SGN_OK;
    // initial state: lake at rest
    std::vector<double> q0(n * NV, 0.0);
    for (size_t i = 0; i < n; i++) q0[i] = a.b[i] > 0 ? a.b[i] : 0.0;
    return set_state(q0.data(), 0.0, false);
  }

  // Device address of a host buffer the GPU can reach (pinned and mapped:
  // cudaHostAlloc, cudaMallocHost or a registered range), else null.
  static const void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
  }

  int set_state(const double* q, double t, bool device) override {
    size_t n = (size_t)d_.nx * d_.ny * NV;
    // device memory and mapped pinned host memory are read by the pack kernel
    // in place; other host memory goes through the staging buffer
    const double* src = device ? q : (const double*)mapped_host(q);
    if (!src) {
      SGN_CK(cudaMemcpyAsync(staging_, q, n * sizeof(double), cudaMemcpyHostToDevice, st_));
      src = staging_;
    }
    cur_ = 0;
    k_pack_state<MODEL, Real><<<gInt_, dim3(32, 8), 0, st_>>>(d_, src, 0);
    hscal_[0] = t;
    SGN_CK(cudaMemcpyAsync(d_.t, hscal_, sizeof(double), cudaMemcpyHostToDevice, st_));
    SGN_CK(cudaMemsetAsync(d_.status, 0, sizeof(unsigned), st_));
    SGN_CK(cudaMemsetAsync(d_.gn, 0, sizeof(int), st_));
    SGN_CK(cudaMemsetAsync(d_.last_dt, 0, 2 * sizeof(double), st_));
    SGN_CK(cudaMemsetAsync(d_.smax, 0, 2 * sizeof(unsigned long long), st_));
    k_speed<MODEL, Real><<<gInt_, dim3(32, 8), 0, st_>>>(d_, 0);
    k_finalize<Real><<<1, 32, 0, st_>>>(d_, 0);
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaStreamSynchronize(st_));
    return SGN_OK;
  }

  void pre(cudaStream_t s, int k) {
    if (!prof_) return;
    Ev e; e.k = k; cudaEventCreate(&e.a); cudaEventCreate(&e.b);
    cudaEventRecord(e.a, s); evs_.push_back(e);
  }
  void post(cudaStream_t s) { if (prof_) cudaEventRecord(evs_.back().b, s); }

  // One time step from q[c] into q[1-c]: the kernel sequence of the method,
  // in two phases (a refined level exchanges ghost positivity factors and
  // records reflux fluxes in between).
  void launch_step(cudaStream_t s, int c) {
    if (tune_[TU_SCHED] == SCHED_FUSED) {
      pre(s, KN_FUSED);
      launch_fused(s, c);
      post(s);
    } else {
      launch_phase1(s, c);
      launch_phase2(s, c);
    }
    pre(s, KN_FINAL);
    k_finalize<Real><<<1, 32, 0, s>>>(d_, 1); post(s);
    if (d_.ngauge > 0) {
      pre(s, KN_GAUGE);
      k_gauge<Real><<<1, 256, 0, s>>>(d_, 1 - c); post(s);
    }
  }

  // The one-pass step (k_step_fused): strips of FUSED_OUT columns by chunks of
  // fused_rows() rows (the long chunks), one block each.
  static constexpr bool kFusedBuilt = sizeof(Real) == 4;
  bool fused_ok() const { return kFusedBuilt; }
  int fused_resident_ = 0;   // blocks of the one-pass kernel resident on the device
  // rows of the long chunks: the option's, halved (not below 32) while the grid
  // would give fewer tiles than there are resident blocks
  int fused_rows() const {
    int H = kFusedRows[tune_[TU_UPDATE]];
    while (H > 32 && fused_plan(d_.nx, d_.ny, H).ntiles < fused_resident_) H /= 2;
    return H;
  }
  // xphi: a refined level's export buffer for this step (see fused_tile).
  void launch_fused(cudaStream_t s, int c, Real* xphi = nullptr) {
    if constexpr (kFusedBuilt) {
      const FusedPlan p = fused_plan(d_.nx, d_.ny, fused_rows());
      const int nb = p.ntiles < fused_resident_ ? p.ntiles : fused_resident_;
      const size_t smb = sizeof(FusedSmem<MODEL, Real>);
      if (d_.kind) k_step_fused<MODEL, Real, true><<<nb, FUSED_NT, smb, s>>>(d_, c, p, xphi);
      else k_step_fused<MODEL, Real, false><<<nb, FUSED_NT, smb, s>>>(d_, c, p, xphi);
    }
  }

  // one launch of tuned kernel k (TU_PREP .. TU_UPDATE) with its current shape
  void launch_kernel(cudaStream_t s, int k, int c) {
    switch (k) {
      case TU_PREP: k_prep<MODEL, Real><<<tg_[k], tb_[k], 0, s>>>(d_, c); break;
      case TU_FACEX: kface_[0][tune_[k]]<<<tg_[k], tb_[k], 0, s>>>(d_); break;
      case TU_FACEY: kface_[1][tune_[k]]<<<tg_[k], tb_[k], 0, s>>>(d_); break;
      case TU_TRANSX: k_trans<MODEL, Real, 0><<<tg_[k], tb_[k], 0, s>>>(d_); break;
      case TU_TRANSY: k_trans<MODEL, Real, 1><<<tg_[k], tb_[k], 0, s>>>(d_); break;
      case TU_THETA: k_theta<MODEL, Real><<<tg_[k], tb_[k], 0, s>>>(d_); break;
      case TU_UPDATE: k_update<MODEL, Real><<<tg_[k], tb_[k], 0, s>>>(d_, c); break;
    }
  }
  void timed(cudaStream_t s, int k, int c) {   // KN_* and TU_* agree for k <= TU_UPDATE
    pre(s, k);
    launch_kernel(s, k, c);
    post(s);
  }

  // Prep, faces, transverse kernels and positivity factors.  Schedule 1 runs
  // the x and y face kernels, then the two transverse kernels, as two
  // concurrent branches (they read the same inputs and write disjoint planes);
  // profiling keeps the serial order so that each launch is timed alone.
  void launch_phase1(cudaStream_t s, int c) {
    timed(s, TU_PREP, c);
    if (tune_[TU_SCHED] == 1 && !prof_) {
      cudaEventRecord(fork_[0], s);
      cudaStreamWaitEvent(aux_, fork_[0], 0);
      launch_kernel(aux_, TU_FACEY, c);
      launch_kernel(s, TU_FACEX, c);
      cudaEventRecord(fork_[1], aux_);
      cudaEventRecord(fork_[2], s);
      cudaStreamWaitEvent(aux_, fork_[2], 0);   // transverse x reads the y faces and vice versa
      cudaStreamWaitEvent(s, fork_[1], 0);
      launch_kernel(aux_, TU_TRANSY, c);
      launch_kernel(s, TU_TRANSX, c);
      cudaEventRecord(fork_[3], aux_);
      cudaStreamWaitEvent(s, fork_[3], 0);
    } else {
      timed(s, TU_FACEX, c);
      timed(s, TU_FACEY, c);
      timed(s, TU_TRANSX, c);
      timed(s, TU_TRANSY, c);
    }
    timed(s, TU_THETA, c);
  }

  void launch_phase2(cudaStream_t s, int c) { timed(s, TU_UPDATE, c); }

  // access for the refined hierarchy (sgn_amr.cuh)
  Dev<Real>& dev() { return d_; }
  int cur() const { return cur_; }
  void flip() { cur_ ^= 1; }
  dim3 grid_interior() const { return gInt_; }
  template <typename T> T* alloc_dev(size_t n) { return dnew<T>(n); }
  // kind plane from a dense ny*nx host array (ghost frame 0)
  unsigned char* kind_buf_ = nullptr;   // the kind plane (kept across calls)
  int* xslot_buf_ = nullptr;            // the export slot plane (likewise)
  int set_kind(const unsigned char* kind_dense) {
    unsigned char* kp = kind_buf_ ? kind_buf_ : dnew<unsigned char>(d_.fs);
    if (!kp) return SGN_ENOMEM;
    kind_buf_ = kp;
    std::vector<unsigned char> h(d_.fs, 0);
    for (int j = 0; j < d_.ny; j++)
      for (int i = 0; i < d_.nx; i++)
        h[(size_t)(j + NG) * d_.pitch + (i + NG)] = kind_dense[(size_t)j * d_.nx + i];
    SGN_CK(cudaMemcpyAsync(kp, h.data(), d_.fs, cudaMemcpyHostToDevice, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    d_.kind = kp;
    drop_graphs();
    return SGN_OK;
  }
  // export slots of a refined level (dense ny*nx host array, -1: none)
  int set_xslot(const int* slot_dense) {
    int* sp = xslot_buf_ ? xslot_buf_ : dnew<int>(d_.fs);
    if (!sp) return SGN_ENOMEM;
    xslot_buf_ = sp;
    std::vector<int> h(d_.fs, -1);
    for (int j = 0; j < d_.ny; j++)
      for (int i = 0; i < d_.nx; i++) h[(size_t)(j + NG) * d_.pitch + (i + NG)] = slot_dense[(size_t)j * d_.nx + i];
    SGN_CK(cudaMemcpyAsync(sp, h.data(), d_.fs * sizeof(int), cudaMemcpyHostToDevice, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    d_.xslot = sp;
    drop_graphs();
    return SGN_OK;
  }
  int schedule() const { return tune_[TU_SCHED]; }

  int launches_per_step() override {
    const int n = tune_[TU_SCHED] == SCHED_FUSED ? 2 : 8;
    return d_.ngauge > 0 ? n + 1 : n;
  }

  int build_graph(int c) {
    cudaGraph_t gr;
    SGN_CK(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
    launch_step(cap_, c);
    cudaError_t e = cudaStreamEndCapture(cap_, &gr);
    if (e != cudaSuccess) return SGN_ECUDA;
    e = cudaGraphInstantiate(&gx_[c], gr, 0);
    cudaGraphDestroy(gr);
    return e == cudaSuccess ? SGN_OK : SGN_ECUDA;
  }

  int finish_batch(double* t_out) {
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaMemcpyAsync(hscal_, d_.t, sizeof(double), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaMemcpyAsync(hscal_ + 1, d_.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    if (t_out) *t_out = hscal_[0];
    unsigned stv;
    memcpy(&stv, hscal_ + 1, sizeof(unsigned));
    return status_to_error(stv);
  }

  int step(int n, double* t_out) override {
    if (n < 0) return SGN_EINVAL;
    for (int i = 0; i < n; i++) {
      if (prof_) {
        launch_step(st_, cur_);
      } else {
        if (!gx_[cur_]) { int r = build_graph(cur_); if (r) return r; }
        SGN_CK(cudaGraphLaunch(gx_[cur_], st_));
      }
      cur_ ^= 1;
    }
    return finish_batch(t_out);
  }

  int step_dt(double dt) override {
    hscal_[2] = dt;
    hscal_[8] = dt / d_.dx;
    hscal_[9] = dt / d_.dy;
    hscal_[10] = d_.strang ? 0.5 * dt : 0.0;
    hscal_[11] = d_.strang ? 0.5 * dt : dt;
    SGN_CK(cudaMemcpyAsync(d_.dt, hscal_ + 2, sizeof(double), cudaMemcpyHostToDevice, st_));
    SGN_CK(cudaMemcpyAsync(d_.lam, hscal_ + 8, 4 * sizeof(double), cudaMemcpyHostToDevice, st_));
    Real* hr = (Real*)(hscal_ + 16);
    for (int k = 0; k < 4; k++) hr[k] = (Real)hscal_[8 + k];
    SGN_CK(cudaMemcpyAsync(d_.lamr, hr, 4 * sizeof(Real), cudaMemcpyHostToDevice, st_));
    launch_step(st_, cur_);
    cur_ ^= 1;
    return finish_batch(nullptr);
  }

  int get_state(int mask, double* out, size_t len, double* t_out, bool device) override {
    size_t n = (size_t)d_.nx * d_.ny;
    if (mask == 0) mask = (1 << NV) - 1;
    if (mask & ~((1 << NV) - 1)) return SGN_EINVAL;
    int nsel = 0;
    for (int k = 0; k < NV; k++) nsel += (mask >> k) & 1;
    if (len < nsel * n) return SGN_ERANGE;
    // device memory and mapped pinned host memory are written by the unpack
    // kernel in place; other host memory through the staging buffer
    double* dst = device ? out : (double*)mapped_host(out);
    k_unpack_state<MODEL, Real><<<gInt_, dim3(32, 8), 0, st_>>>(d_, dst ? dst : staging_, cur_, mask);
    SGN_CK(cudaGetLastError());
    if (!dst) SGN_CK(cudaMemcpyAsync(out, staging_, nsel * n * sizeof(double), cudaMemcpyDeviceToHost, st_));
    if (t_out || !device) {
      SGN_CK(cudaMemcpyAsync(hscal_, d_.t, sizeof(double), cudaMemcpyDeviceToHost, st_));
      SGN_CK(cudaStreamSynchronize(st_));
      if (t_out) *t_out = hscal_[0];
    }
    return SGN_OK;
  }

  int add_gauges(const double* xy, int n, int cap) override {
    if (n < 0 || cap < 0 || (n > 0 && !xy)) return SGN_EINVAL;
    std::vector<int> idx(n > 0 ? n : 1);
    for (int g = 0; g < n; g++) {
      double fx = (xy[2 * g] - x0_) / d_.dx, fy = (xy[2 * g + 1] - y0_) / d_.dy;
      if (!(fx >= 0) || !(fy >= 0)) return SGN_ERANGE;
      long i = (long)fx, j = (long)fy;
      if (i >= d_.nx || j >= d_.ny) return SGN_ERANGE;
      idx[g] = (int)((j + NG) * (long)d_.pitch + (i + NG));
    }
    drop_graphs();
    d_.gidx = dnew<int>(idx.size());
    d_.grec = dnew<double>((size_t)(n > 0 ? n : 1) * 4 * (cap > 0 ? cap : 1));
    if (!d_.gidx || !d_.grec) return SGN_ENOMEM;
    SGN_CK(cudaMemcpyAsync(d_.gidx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, st_));
    SGN_CK(cudaMemsetAsync(d_.gn, 0, sizeof(int), st_));
    SGN_CK(cudaStreamSynchronize(st_));
    d_.ngauge = n; d_.gcap = cap;
    return SGN_OK;
  }

  int gauges(double* out, size_t cap, int* nrec) override {
    int n = 0;
    SGN_CK(cudaMemcpyAsync(hscal_ + 3, d_.gn, sizeof(int), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    memcpy(&n, hscal_ + 3, sizeof(int));
    if (nrec) *nrec = n;
    size_t need = (size_t)n * d_.ngauge * 4;
    if (!out) return SGN_OK;
    if (cap < need) return SGN_ERANGE;
    if (need) SGN_CK(cudaMemcpy(out, d_.grec, need * sizeof(double), cudaMemcpyDeviceToHost));
    return SGN_OK;
  }

  int clear_gauges() override {
    SGN_CK(cudaMemsetAsync(d_.gn, 0, sizeof(int), st_));
    return SGN_OK;
  }

  int status(unsigned* f, double* dt, double* cr) override {
    SGN_CK(cudaMemcpyAsync(hscal_ + 4, d_.last_dt, 2 * sizeof(double), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaMemcpyAsync(hscal_ + 6, d_.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    if (dt) *dt = hscal_[4];
    if (cr) *cr = hscal_[5];
    if (f) memcpy(f, hscal_ + 6, sizeof(unsigned));
    return SGN_OK;
  }

  int next_dt(double* dt) override {
    SGN_CK(cudaMemcpyAsync(hscal_ + 12, d_.dt, sizeof(double), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    *dt = hscal_[12];
    return SGN_OK;
  }

  int mass(double* m) override {
    int nb = 592;   // 152 SMs x 4
    k_mass1<Real><<<nb, 256, 0, st_>>>(d_, cur_);
    k_mass2<Real><<<1, 256, 0, st_>>>(d_, nb);
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaMemcpyAsync(hscal_ + 7, d_.mass, sizeof(double), cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    *m = hscal_[7];
    return SGN_OK;
  }

  int set_c2(const double* c2) override {
    size_t n = (size_t)d_.nx * d_.ny;
    for (size_t i = 0; i < n; i++)
      if (!(c2[i] >= 0.0) || !std::isfinite(c2[i])) return SGN_EINVAL;
    SGN_CK(cudaMemcpyAsync(staging_, c2, n * sizeof(double), cudaMemcpyHostToDevice, st_));
    k_set_c2<Real><<<gPad_, dim3(32, 8), 0, st_>>>(d_, staging_);
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaStreamSynchronize(st_));
    return SGN_OK;
  }

  double* wp_scratch_ = nullptr;
  int well_prepare() override {
    if (MODEL != 1) return SGN_EINVAL;
    if (!wp_scratch_) {
      wp_scratch_ = dnew<double>((size_t)7 * d_.nx * d_.ny);
      if (!wp_scratch_) return SGN_ENOMEM;
    }
    k_well_prepared<Real><<<(d_.ny + 127) / 128, 128, 0, st_>>>(d_, cur_, wp_scratch_);
    SGN_CK(cudaGetLastError());
    // the time step of the next step from the new state
    SGN_CK(cudaMemsetAsync(d_.smax, 0, sizeof(unsigned long long), st_));
    k_speed<MODEL, Real><<<gInt_, dim3(32, 8), 0, st_>>>(d_, cur_);
    k_finalize<Real><<<1, 32, 0, st_>>>(d_, 0);
    SGN_CK(cudaGetLastError());
    SGN_CK(cudaStreamSynchronize(st_));
    return SGN_OK;
  }

  int get_aux(double* c2, unsigned char* phi) override {
    size_t n = (size_t)d_.nx * d_.ny;
    unsigned char* pd = (unsigned char*)(staging_ + n);
    k_aux_out<Real><<<gInt_, dim3(32, 8), 0, st_>>>(d_, staging_, pd);
    SGN_CK(cudaGetLastError());
    if (c2) SGN_CK(cudaMemcpyAsync(c2, staging_, n * sizeof(double), cudaMemcpyDeviceToHost, st_));
    if (phi) SGN_CK(cudaMemcpyAsync(phi, pd, n, cudaMemcpyDeviceToHost, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    return SGN_OK;
  }

  int set_profiling(int on) override {
    SGN_CK(cudaStreamSynchronize(st_));
    collect();
    prof_ = on != 0;
    for (int k = 0; k < KN_COUNT; k++) { kms_[k] = 0; kcnt_[k] = 0; }
    return SGN_OK;
  }

  void collect() {
    for (auto& e : evs_) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) { kms_[e.k] += ms; kcnt_[e.k]++; }
      cudaEventDestroy(e.a); cudaEventDestroy(e.b);
    }
    evs_.clear();
  }

  int kernel_times(const char** names, double* ms, long* launches, int n) override {
    SGN_CK(cudaStreamSynchronize(st_));
    collect();
    for (int k = 0; k < n && k < KN_COUNT; k++) {
      if (names) names[k] = kKernelNames[k];
      if (ms) ms[k] = kms_[k];
      if (launches) launches[k] = kcnt_[k];
    }
    return KN_COUNT;
  }

  int set_tuning(const int* ch) override {
    if (!ch) return SGN_EINVAL;
    for (int k = 0; k < TU_N; k++)
      if (ch[k] < 0 || ch[k] >= (k == TU_SCHED ? SCHED_N : TU_OPTS)) return SGN_EINVAL;
    if (ch[TU_SCHED] == SCHED_FUSED && !fused_ok()) return SGN_EINVAL;
    SGN_CK(cudaStreamSynchronize(st_));
    for (int k = 0; k < TU_N; k++) tune_[k] = ch[k];
    set_geometry();
    drop_graphs();
    return SGN_OK;
  }

  int get_tuning(int* ch, int* bx, int* by) override {
    const bool fz = tune_[TU_SCHED] == SCHED_FUSED;
    for (int k = 0; k < TU_N; k++) {
      if (ch) ch[k] = tune_[k];
      // with the one-pass schedule the update slot stands for its block: NT columns by H rows
      const int x = k == TU_SCHED ? 0 : (fz && k == TU_UPDATE ? FUSED_NT : (int)tb_[k].x);
      const int y = k == TU_SCHED ? 0 : (fz && k == TU_UPDATE ? fused_rows() : (int)tb_[k].y);
      if (bx) bx[k] = x;
      if (by) by[k] = y;
    }
    return SGN_OK;
  }

  // Times every option of each tuned kernel on the current state, in step
  // order, keeping the fastest (ties keep the lower option), then the whole
  // step in every schedule replayed as a graph (the one-pass kernel with each
  // row count).  Every option of a kernel writes the same values (a block shape
  // changes only which thread computes what), so each kernel leaves the next
  // one's inputs as a step would; every trial reads q[cur] and writes only
  // scratch planes or q[1 - cur].  The speed and Courant maxima and the status
  // word are saved first and put back at the end, so the next step is the one
  // that would have run without tuning (on the schedule kept).
  int autotune(int reps, int* ch, double* ms) override {
    if (reps < 1 || reps > 10000) return SGN_EINVAL;
    if (ms)
      for (int i = 0; i < TU_N * TU_OPTS; i++) ms[i] = -1.0;
    const int c = cur_;
    const bool prof = prof_;
    prof_ = false;
    SGN_CK(cudaStreamSynchronize(st_));
    SGN_CK(cudaMemcpyAsync(save_, d_.smax, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st_));
    SGN_CK(cudaMemcpyAsync(save_ + 2, d_.status, sizeof(unsigned), cudaMemcpyDeviceToDevice, st_));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SGN_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SGN_ECUDA;
    // mean time of one launch over reps, after one untimed launch
    auto time_it = [&](auto&& launch, float* out) -> int {
      launch();
      cudaEventRecord(e0, st_);
      for (int r = 0; r < reps; r++) launch();
      cudaEventRecord(e1, st_);
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return SGN_ECUDA;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return SGN_ECUDA;
      *out = t / reps;
      return SGN_OK;
    };
    for (int k = 0; k < TU_SCHED && rc == SGN_OK; k++) {
      float best = 0.f;
      int bo = 0;
      for (int o = 0; o < TU_OPTS && rc == SGN_OK; o++) {
        tune_[k] = o;
        set_geometry();
        float t = 0.f;
        rc = time_it([&]() { launch_kernel(st_, k, c); }, &t);
        if (ms) ms[k * TU_OPTS + o] = t;
        if (o == 0 || t < best) { best = t; bo = o; }
      }
      tune_[k] = bo;
      set_geometry();
    }
    // schedules: the whole step (first phase and update, or the one-pass
    // kernel with each of its row counts) replayed as a CUDA graph
    {
      const int upd0 = tune_[TU_UPDATE];
      float best = 0.f;
      int bo = -1, bu = upd0;
      for (int o = 0; o < SCHED_N && rc == SGN_OK; o++) {
        if (o == SCHED_FUSED && !fused_ok()) continue;
        const int nu = o == SCHED_FUSED ? TU_OPTS : 1;
        for (int u = 0; u < nu && rc == SGN_OK; u++) {
          tune_[TU_SCHED] = o;
          tune_[TU_UPDATE] = o == SCHED_FUSED ? u : upd0;
          set_geometry();
          cudaGraph_t gr = nullptr;
          cudaGraphExec_t gx = nullptr;
          if (cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = SGN_ECUDA; break; }
          if (o == SCHED_FUSED) launch_fused(cap_, c);
          else { launch_phase1(cap_, c); launch_phase2(cap_, c); }
          if (cudaStreamEndCapture(cap_, &gr) != cudaSuccess) { rc = SGN_ECUDA; break; }
          cudaError_t e = cudaGraphInstantiate(&gx, gr, 0);
          cudaGraphDestroy(gr);
          if (e != cudaSuccess) { rc = SGN_ECUDA; break; }
          float t = 0.f;
          rc = time_it([&]() { cudaGraphLaunch(gx, st_); }, &t);
          cudaGraphExecDestroy(gx);
          if (rc) break;
          float& slot = ms_sched_[o];
          if (u == 0 || t < slot) slot = t;
          if (bo < 0 || t < best) { best = t; bo = o; bu = tune_[TU_UPDATE]; }
        }
        if (ms && rc == SGN_OK) ms[TU_SCHED * TU_OPTS + o] = ms_sched_[o];
      }
      tune_[TU_SCHED] = bo < 0 ? SCHED_SERIAL : bo;
      tune_[TU_UPDATE] = bo == SCHED_FUSED ? bu : upd0;
      set_geometry();
    }
    if (rc) tune_[TU_SCHED] = 0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    prof_ = prof;
    drop_graphs();
    SGN_CK(cudaMemcpyAsync(d_.smax, save_, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st_));
    SGN_CK(cudaMemcpyAsync(d_.status, save_ + 2, sizeof(unsigned), cudaMemcpyDeviceToDevice, st_));
    SGN_CK(cudaStreamSynchronize(st_));
    if (rc) return rc;
    return get_tuning(ch, nullptr, nullptr);
  }

  double x0_ = 0, y0_ = 0;
  void set_origin(double x0, double y0) { x0_ = x0; y0_ = y0; }
};

}  // namespace sgn
