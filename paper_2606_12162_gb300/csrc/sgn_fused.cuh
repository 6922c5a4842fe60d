// sgn_fused.cuh -- the whole time step of a uniform grid in one pass over the
// state (paper Sec. 4: first source half step, x and y normal Riemann solves with
// the limiter, transverse propagation, positivity factors, conservative update,
// second source half step and SWE switch, speed of the new state for the next
// CFL step).  It computes exactly what the kernel sequence k_prep .. k_update of
// sgn_kernels.cuh computes, with the same device functions, but keeps every
// intermediate quantity on chip: only the state, b, c^2 and the sensor values
// are read from HBM and only the new state is written.
//
// Work split.  A block of NT threads owns a strip of NT - 6 output columns and a
// chunk of rows.  Thread t holds column I = x0 + t of the strip window, which
// reaches three columns beyond the strip on each side: the normal solves of
// the x faces feed the limiter of their neighbours, the limited fluxes feed the
// transverse corrections of the neighbouring faces, and those feed the
// positivity factors of the ring of cells around each updated cell.  The
// thread marches up the rows; at iteration r it
//   A  stages row r + 2 into shared memory with cp.async (ghost cells through
//      the boundary index map), builds the record of cell (I, r) (first source
//      half step, primitives, FP64 g h / 2), solves the y face below row r and
//      limits the y face below row r - 1 (the faces below and above it are the
//      thread's own, in registers);
//   B  solves the x face I of row r - 1 (left cell record from shared memory);
//   C  limits it with the x faces I - 1 and I + 1 (shared memory);
//   D  transverse corrections of the y face below row r - 1 (x fluctuations of
//      rows r - 2 and r - 1) and of the x face I of row r - 2 (y fluctuations of
//      columns I - 1 and I);
//   E  positivity factor of cell (I, r - 2) and the update of cell (I, r - 3).
// Values along a column stay in the thread's registers from row to row; values
// of neighbouring columns pass through shared memory (four barriers per row).
// The index ranges over which each quantity is computed are those of the
// kernel sequence (faces of ghost rows and columns included), so the result is
// the same.
#pragma once
#include "sgn_kernels.cuh"

namespace sgn {

#ifndef SGN_FUSED_NT
#define SGN_FUSED_NT 128
#endif
#ifndef SGN_FUSED_UNROLL
#define SGN_FUSED_UNROLL 1
#endif
constexpr int FUSED_NT = SGN_FUSED_NT;  // threads (columns) per block
constexpr int FUSED_UNROLL = SGN_FUSED_UNROLL;   // rows per unrolled march iteration
#ifndef SGN_FUSED_MINB
#define SGN_FUSED_MINB 2                // resident blocks per SM the register bound aims at
#endif
constexpr int FUSED_OUT = FUSED_NT - 6; // output columns per block

// cp.async of one 4- or 8-byte word (global -> shared, L1-allocating), its group
// commit and wait (sm_80+ asynchronous copy; PTX ISA "cp.async").
template <typename T> __device__ __forceinline__ void cp_async_word(T* smem, const T* gmem) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "word copies only");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// A cell after the first source half step: the post-source state W, b, c^2,
// the bulk-type depth, the primitives (slot k-1: field k divided by h),
// sqrt(h), C = sqrt(g h + p + c^2), FP64 g h / 2, the wet flag and the sensor
// value of its x face (kept for the x solve one row later).
template <int MODEL, typename Real> struct Rec {
  static constexpr int NV = MT<MODEL>::NV;
  Real W[NV];
  Real P[NV - 1];
  Real b, c2, hr, sqh, C, psx;
  double g2, e64;   // FP64 g h / 2 and eta
  bool wet;
  unsigned char kind;   // refined levels: the cell's kind bits (else unused)
};

// Primitives of a record from its W, b and c^2 (the mixed path's load_side
// arithmetic: h = max(0, eta - b) in the bulk type, wet when h > dry_tol).
template <int MODEL, typename Real>
__device__ __forceinline__ void rec_prims(const Dev<Real>& d, Rec<MODEL, Real>& r) {
  typedef MT<MODEL> M;
  Real hr = r.W[0] - r.b;
  hr = hr > Real(0) ? hr : Real(0);
  r.hr = hr;
  r.wet = hr > d.rdry_tol;
  const Real ih = r.wet ? rcp(hr) : Real(0);
#pragma unroll
  for (int k = 1; k < M::NV; k++) r.P[k - 1] = r.W[k] * ih;
  const Real p = M::HP > 0 ? r.P[(M::HP > 0 ? M::HP : 1) - 1] : Real(0);
  r.sqh = sqrt_nr(hr);
  r.C = sqrt_nr(d.g_r * hr + p + r.c2);
}

template <int MODEL, typename Real, int DIR>
__device__ __forceinline__ Side<MODEL, Real> rec_side(const Rec<MODEL, Real>& r) {
  typedef MT<MODEL> M;
  Side<MODEL, Real> s;
  s.g2 = r.g2;
  s.e64 = r.e64;
  s.hr = r.hr;
  s.eta = r.W[0];
  s.b = r.b;
  s.c2 = r.c2;
  s.hn = r.W[1 + DIR];
  s.ht = r.W[2 - DIR];
  s.hw = M::HW > 0 ? r.W[M::HW > 0 ? M::HW : 0] : Real(0);
  s.hs = M::HS > 0 ? r.W[M::HS > 0 ? M::HS : 0] : Real(0);
  s.hp = M::HP > 0 ? r.W[M::HP > 0 ? M::HP : 0] : Real(0);
  s.hpb = M::HPB > 0 ? r.W[M::HPB > 0 ? M::HPB : 0] : Real(0);
  s.un = r.P[DIR];
  s.ut = r.P[1 - DIR];
  s.w = M::HW > 0 ? r.P[(M::HW > 0 ? M::HW : 1) - 1] : Real(0);
  s.sg = M::HS > 0 ? r.P[(M::HS > 0 ? M::HS : 1) - 1] : Real(0);
  s.p = M::HP > 0 ? r.P[(M::HP > 0 ? M::HP : 1) - 1] : Real(0);
  s.pb = M::HPB > 0 ? r.P[(M::HPB > 0 ? M::HPB : 1) - 1] : Real(0);
  s.sqh = r.sqh;
  s.C = r.C;
  s.wet = r.wet;
  return s;
}

template <typename Real> __device__ __forceinline__ Waves<Real> zero_waves() {
  Waves<Real> v;
  v.b1 = v.b2 = v.bt = v.bw = v.bs = v.bpb = v.bN = Real(0);
  v.s1 = v.un = v.sN = v.ut = v.w = v.sg = v.K = v.pb = v.gh = v.C = v.hnL = Real(0);
  v.wall = 0;
  v.active = false;
  v.first = true;
  return v;
}

// The 16 fields of a wave record that the limiter of a neighbouring face reads
// (WR_* order).
template <typename Real> __device__ __forceinline__ Real wr_get(const Waves<Real>& v, int f) {
  switch (f) {
    case WR_B1: return v.b1;
    case WR_B2: return v.b2;
    case WR_BT: return v.bt;
    case WR_BW: return v.bw;
    case WR_BS: return v.bs;
    case WR_BPB: return v.bpb;
    case WR_BN: return v.bN;
    case WR_S1: return v.s1;
    case WR_UN: return v.un;
    case WR_SN: return v.sN;
    case WR_UT: return v.ut;
    case WR_W: return v.w;
    case WR_SG: return v.sg;
    case WR_K: return v.K;
    case WR_PB: return v.pb;
    default: return v.gh;
  }
}

// Fluctuations and second-order correction of one face from its wave record v
// and its neighbours' (nb(f, left): field f of the face before it, left = true,
// or after it): Lo = A^- dQ + Ftil, Ro = A^+ dQ - Ftil, Mo = Fhat + Ftil_h --
// the values k_face writes to the face planes (same arithmetic).
template <int MODEL, typename Real, int DIR, typename NB>
__device__ __forceinline__ void face_out(const Dev<Real>& d, const Waves<Real>& v, NB nb, Real lam, Real* Lo,
                                         Real* Ro, Real& Mo) {
  constexpr int NV = MT<MODEL>::NV;
  auto wneg = [](Real s) { return s < Real(0) ? Real(1) : (s > Real(0) ? Real(0) : Real(0.5)); };
  Real m1 = wneg(v.s1), m0 = wneg(v.un), mN = wneg(v.sN);
  Real Am[NV], Ap[NV], Ft[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) { Am[k] = Real(0); Ap[k] = Real(0); Ft[k] = Real(0); }
  combine<MODEL, Real, DIR>(v, m1, m0, m0, m0, m0, m0, mN, Am);
  combine<MODEL, Real, DIR>(v, Real(1) - m1, Real(1) - m0, Real(1) - m0, Real(1) - m0, Real(1) - m0,
                            Real(1) - m0, Real(1) - mN, Ap);
  Real Fhat = v.hnL + Am[0];
  if (v.wall == 2) {
#pragma unroll
    for (int k = 0; k < NV; k++) Ap[k] = Real(0);
    Fhat = Real(0);
  }
  if (v.wall == 1) {
#pragma unroll
    for (int k = 0; k < NV; k++) Am[k] = Real(0);
    Fhat = Real(0);
  }
  if (v.active && !v.first && d.limiter != 2) {
    auto rdot = [&](Real s, Real so, Real uto, Real wo, Real sgo, Real Ko, Real pbo) {
      Real r = Real(1) + s * so + v.ut * uto;
      if (MODEL > 0) r += v.w * wo + v.K * Ko;
      if (MODEL == 2) r += v.sg * sgo + v.pb * pbo;
      return r;
    };
    const int lk = d.limiter;
    const bool l1 = v.s1 > Real(0), l0 = v.un > Real(0), lN = v.sN > Real(0);
    Real c1, cN;
    {
      Real us = nb(WR_S1, l1), uut = nb(WR_UT, l1), uw = MODEL > 0 ? nb(WR_W, l1) : Real(0);
      Real usg = MODEL == 2 ? nb(WR_SG, l1) : Real(0), uK = MODEL > 0 ? nb(WR_K, l1) : Real(0);
      Real upb = MODEL == 2 ? nb(WR_PB, l1) : Real(0);
      Real pr = nb(WR_B1, l1) * rdot(v.s1, us, uut, uw, usg, uK, upb) *
                rcp(rdot(v.s1, v.s1, v.ut, v.w, v.sg, v.K, v.pb));
      c1 = lim_wave<Real>(lk, lam, v.s1, v.b1, pr);
    }
    {
      Real us = nb(WR_SN, lN), uut = nb(WR_UT, lN), uw = MODEL > 0 ? nb(WR_W, lN) : Real(0);
      Real usg = MODEL == 2 ? nb(WR_SG, lN) : Real(0), uK = MODEL > 0 ? nb(WR_K, lN) : Real(0);
      Real upb = MODEL == 2 ? nb(WR_PB, lN) : Real(0);
      Real pr = nb(WR_BN, lN) * rdot(v.sN, us, uut, uw, usg, uK, upb) *
                rcp(rdot(v.sN, v.sN, v.ut, v.w, v.sg, v.K, v.pb));
      cN = lim_wave<Real>(lk, lam, v.sN, v.bN, pr);
    }
    Real c2 = Real(0), cw = Real(0), cs = Real(0), cpb = Real(0);
    Real ct = lim_wave<Real>(lk, lam, v.un, v.bt, nb(WR_BT, l0));
    if (MODEL > 0) {
      Real r22 = Real(1) + v.un * v.un + v.gh * v.gh;
      Real r2u = Real(1) + v.un * nb(WR_UN, l0) + v.gh * nb(WR_GH, l0);
      c2 = lim_wave<Real>(lk, lam, v.un, v.b2, nb(WR_B2, l0) * r2u * rcp(r22));
      cw = lim_wave<Real>(lk, lam, v.un, v.bw, nb(WR_BW, l0));
    }
    if (MODEL == 2) {
      cs = lim_wave<Real>(lk, lam, v.un, v.bs, nb(WR_BS, l0));
      cpb = lim_wave<Real>(lk, lam, v.un, v.bpb, nb(WR_BPB, l0));
    }
    combine_amp<MODEL, Real, DIR>(v, c1, c2, ct, cw, cs, cpb, cN, Ft);
  }
#pragma unroll
  for (int k = 0; k < NV; k++) {
    Lo[k] = Am[k] + Ft[k];
    Ro[k] = Ap[k] - Ft[k];
  }
  Mo = Fhat + Ft[0];
}

// Roe data of a face kept for its transverse correction (the ROE slots of the
// face planes): u_n, u_t, w, sigma, p_b, K, g h, C (C = 0: not both cells wet).
template <typename Real> struct Roe {
  Real un, ut, w, sg, pb, K, gh, C;
};
template <typename Real> __device__ __forceinline__ Roe<Real> roe_of(const Waves<Real>& v) {
  Roe<Real> e;
  e.un = v.un; e.ut = v.ut; e.w = v.w; e.sg = v.sg; e.pb = v.pb; e.K = v.K; e.gh = v.gh; e.C = v.C;
  return e;
}

// Transverse correction of one face (the body of k_trans): out = the total flux
// of the face's row plus the split of the other direction's fluctuations Va
// (entering the cell before the face) and Vb (the cell after it).
template <int MODEL, typename Real, int DIR>
__device__ __forceinline__ void trans_out(const Dev<Real>& d, const Roe<Real>& e, Real M, const Real* Va,
                                          const Real* Vb, Real* out) {
  constexpr int NV = MT<MODEL>::NV;
#pragma unroll
  for (int k = 0; k < NV; k++) out[k] = Real(0);
  if (e.C > Real(0)) {
    Real iKg = MODEL > 0 ? rcp(e.K + e.gh) : Real(0);
    Real i2C = rcp(Real(2) * e.C);
    tsplit<MODEL, Real, DIR>(Va, e.un, e.ut, e.w, e.sg, e.pb, e.K, e.gh, e.C, iKg, i2C, true, out);
    tsplit<MODEL, Real, DIR>(Vb, e.un, e.ut, e.w, e.sg, e.pb, e.K, e.gh, e.C, iKg, i2C, false, out);
    const Real c = Real(-0.5) * d.lamr[1 - DIR];
#pragma unroll
    for (int k = 0; k < NV; k++) out[k] *= c;
  }
  out[0] = M + out[0];
}

// Shared memory of one block: the exchange between neighbouring columns and
// the cp.async staging ring of the input rows (3 rows in flight).
template <int MODEL, typename Real> struct FusedSmem {
  static constexpr int NV = MT<MODEL>::NV;
  static constexpr int NX = 2 * NV + 4;   // record fields passed to the right neighbour:
                                          // W, P, b, c^2, h, sqrt(h), C
  static constexpr int NIN = NV + 4;      // staged fields: state, b, c^2, psi_x, psi_y
  Real in[2][NIN][FUSED_NT];
  Real rec[NX][FUSED_NT];
  double g2[FUSED_NT];
  double e64[FUSED_NT];
  unsigned char wet[FUSED_NT];
  unsigned char kind[FUSED_NT];           // kind bits of the record (refined levels)
  Real xw[WR_N][FUSED_NT];                // x-face wave records of the row being limited
  Real lx[NV][FUSED_NT];                  // A^- + Ftil of each x face (for the transverse sums)
  Real uy[NV][FUSED_NT];                  // sum of the y fluctuations entering each cell
  Real gx[2][NV][FUSED_NT];               // slot 0: total x mass flux, 1..: L + T of each x face (by row parity)
  Real th[2][FUSED_NT];                   // positivity factors (by row parity)
  int tile;                               // tile taken by the block
};

// Tiles of the one-pass kernel: strips of FUSED_OUT output columns by chunks of
// rows.  The rows are cut into three bands -- chunks of H1 rows up to R1, of H2
// up to R2, of H3 to the top -- and the tiles are numbered band by band, strip
// fastest: blocks take tiles in that order, so the last tiles handed out are
// the shortest and the blocks finish close together, while most rows pay the
// small march start-up of the long chunks.
struct FusedPlan {
  int nsx;              // strips
  int H1, R1, H2, R2, H3;
  int n1, n2, ntiles;   // tiles in band 1, in band 2, in all
};

inline FusedPlan fused_plan(int nx, int ny, int H) {
  FusedPlan p;
  p.nsx = (nx + FUSED_OUT - 1) / FUSED_OUT;
  p.H1 = H;
  p.H2 = H / 2 > 16 ? H / 2 : 16;
  p.H3 = H / 4 > 16 ? H / 4 : 16;
  p.R1 = (ny - ny / 4) / p.H1 * p.H1;                       // about 3/4 of the rows in long chunks
  p.R2 = p.R1 + (ny - p.R1) / 2 / p.H2 * p.H2;              // half of the rest in half chunks
  p.n1 = p.nsx * (p.R1 / p.H1);
  p.n2 = p.nsx * ((p.R2 - p.R1) / p.H2);
  p.ntiles = p.n1 + p.n2 + p.nsx * ((ny - p.R2 + p.H3 - 1) / p.H3);
  return p;
}

// One tile: the strip `sx` by the output rows [r0, r0 + nr) (interior row
// indices), marched by the block.
//
// KD: the grid is the atlas of a refined level, with a kind plane (bit 0 patch
// interior, bit 1 covered by a finer patch, bit 2 ghost cell copied from a
// sibling patch next to a patch edge, bit 3 cell whose four face mass fluxes
// are exported for the coarse/fine flux correction).  Then only interior
// cells are updated, the Courant number is taken over faces of interior
// cells, positivity factors are computed for interior cells and for bit-2
// ghosts (whose frame is deep enough that the factor equals the sibling's own,
// so that both sides of a sibling face move the same mass) and are 1 for
// every other ghost, and the theta-weighted mass fluxes of the four faces of
// every bit-3 cell go to xphi[4 * xslot[cell] + {left, right, bottom, top}]
// (nothing is exported when xphi is null).
template <int MODEL, typename Real, bool KD>
__device__ __forceinline__ void fused_tile(const Dev<Real>& d, FusedSmem<MODEL, Real>& sm, int cur, int sx, int r0,
                                           int nr, Real& courmax, Real& spmax, Real* __restrict__ xphi) {
  typedef MT<MODEL> M;
  constexpr int NV = M::NV;
  const int t = threadIdx.x;
  const int nx = d.nx, ny = d.ny, nxp = d.nxp, nyp = d.nyp;
  const int a0 = NG + sx * FUSED_OUT;               // first output column of the strip
  const int I = a0 - 3 + t;                         // this thread's column
  const int b0 = NG + r0;                           // first output row of the chunk
  const int b1 = min(b0 + nr, NG + ny);             // one past the last output row
  const int rs = b0 - 3;                            // first row of the march
  const int re = b1 + 2;                            // last row of the march
  const bool colok = I >= 0 && I < nxp;
  bool fx = false;
  const int Is = colok ? bc_src(I, nx, d.bc[0], d.bc[1], fx) : 0;

  // ---- staging of one input row (own column; ghost rows/columns mapped)
  auto stage = [&](int row) {
    if (row <= re && colok && row >= 0 && row < nyp) {
      bool fy;
      const int Js = bc_src(row, ny, d.bc[2], d.bc[3], fy);
      const int sl = (row - rs) & 1;
      const size_t src = at(d.pitch, Is, Js), id = at(d.pitch, I, row);
      const Real* q = d.q[cur];
#pragma unroll
      for (int k = 0; k < NV; k++) cp_async_word(&sm.in[sl][k][t], q + k * d.fs + src);
      cp_async_word(&sm.in[sl][NV][t], d.b + id);
      cp_async_word(&sm.in[sl][NV + 1][t], d.c2 + id);
      cp_async_word(&sm.in[sl][NV + 2][t], d.psx + id);
      cp_async_word(&sm.in[sl][NV + 3][t], d.psy + id);
    }
    cp_async_commit();
  };

  // ---- per-column state carried from row to row
  Rec<MODEL, Real> rp;            // record of row r - 1
  Waves<Real> y1 = zero_waves<Real>();   // y face below row r - 1
  Real y2[WR_N];                  // wave fields of the y face below row r - 2
  Real vx1[NV];                   // x fluctuations entering cell (I, r - 2): R_x(I) + L_x(I + 1)
  Real fxL[NV], fxR[NV], fxM = Real(0);   // limited x face I of row r - 2
  Roe<Real> fxE;
  Real ry1[NV];                   // A^+ - Ftil of the y face below row r - 2
  Real hy2[NV], hy3[NV];          // R_y - T_y of the y faces below rows r - 2 and r - 3 (k >= 1)
  Real gy2[NV];                   // L_y + T_y of the y face below row r - 2 (k >= 1)
  Real my2 = Real(0), my3 = Real(0);   // total y mass fluxes of the faces below rows r - 2, r - 3
  Real hx3[NV], mx3 = Real(0);    // R_x - T_x and total mass flux of x face I, row r - 3
  Real wa[NV], wab = Real(0), wac = Real(0);   // W, b, c^2 of cell (I, r - 2)
  Real wb[NV], wbb = Real(0), wbc = Real(0);   // of cell (I, r - 3)
  Real th3 = Real(1), th4 = Real(1);            // positivity factors of rows r - 3, r - 4
#pragma unroll
  for (int k = 0; k < NV; k++) {
    vx1[k] = fxL[k] = fxR[k] = ry1[k] = hy2[k] = hy3[k] = gy2[k] = hx3[k] = Real(0);
    wa[k] = wb[k] = rp.W[k] = Real(0);
  }
#pragma unroll
  for (int f = 0; f < WR_N; f++) y2[f] = Real(0);
#pragma unroll
  for (int k = 0; k < NV - 1; k++) rp.P[k] = Real(0);
  rp.b = rp.c2 = rp.hr = rp.sqh = rp.C = rp.psx = Real(0);
  rp.g2 = rp.e64 = 0.0;
  rp.wet = false;
  rp.kind = 0;
  unsigned ka = 0, kb = 0;        // kind bits of cells (I, r - 2), (I, r - 3)
  fxE.un = fxE.ut = fxE.w = fxE.sg = fxE.pb = fxE.K = fxE.gh = fxE.C = Real(0);

  // outputs of this thread: strip columns, inside the grid
  const bool outcol = t >= 3 && t < 3 + FUSED_OUT && I < NG + nx;

  stage(rs);
#pragma unroll FUSED_UNROLL
  for (int r = rs; r <= re; r++) {
    const int par = r & 1;
    stage(r + 1);
    cp_async_wait<1>();

    // ===== A: cell record of row r, y face below row r, limited y face below row r - 1
    Rec<MODEL, Real> rc;
    {
      const bool ok = colok && r >= 0 && r < nyp;
      const int sl = (r - rs) & 1;
      Real q[NV];
      bool fy = false;
      if (ok) (void)bc_src(r, ny, d.bc[2], d.bc[3], fy);
#pragma unroll
      for (int k = 0; k < NV; k++) q[k] = ok ? sm.in[sl][k][t] : Real(0);
      if (fx) q[1] = -q[1];
      if (fy) q[2] = -q[2];
      const Real b = ok ? sm.in[sl][NV][t] : Real(0);
      const Real c2 = ok ? sm.in[sl][NV + 1][t] : Real(0);
      rc.psx = ok ? sm.in[sl][NV + 2][t] : Real(0);
      Real hr = q[0] - b;
      const Crit e64 = (Crit)q[0];
      Crit h = hr > Real(0) ? e64 - (Crit)b : Crit(0);
      hr = hr > Real(0) ? hr : Real(0);
      const bool wet = hr > d.rdry_tol;
      source_switch<MODEL, Real>(q, wet, hr, c2, d.lamr[2]);
#pragma unroll
      for (int k = 0; k < NV; k++) rc.W[k] = q[k];
      rc.b = b; rc.c2 = c2;
      if (KD) rc.kind = ok ? d.kind[at(d.pitch, I, r)] : (unsigned char)0;
      rc.g2 = d.half_g * h;
      rc.e64 = e64;
      rec_prims<MODEL, Real>(d, rc);
      if (M::HP > 0 && wet) {
        const Real p = rc.P[(M::HP > 0 ? M::HP : 1) - 1];
        if (d.g_r * rc.hr + p + c2 < Real(0)) set_status(d.status, ST_NONHYP);
      }
    }
    // y face J = r between rows r - 1 and r: solved for J in [1, ny+3], I in [1, nx+2]
    Waves<Real> y0 = zero_waves<Real>();
    if (r >= 1 && r <= ny + 3 && I >= 1 && I <= nx + 2 && r - 1 >= rs) {
      const Real psi = sm.in[(r - rs) & 1][NV + 3][t];
      y0 = normal_solve<MODEL, Real>(d, rec_side<MODEL, Real, 1>(rp), rec_side<MODEL, Real, 1>(rc), psi);
    }
    // limited y face J = r - 1: J in [2, ny+2], I in [1, nx+2], its neighbours solved here
    Real fyL[NV], fyR[NV], fyM = Real(0);
    Roe<Real> fyE;
    {
      const int J = r - 1;
      const bool go = J >= 2 && J <= ny + 2 && I >= 1 && I <= nx + 2 && J - 2 >= rs;
      if (go) {
        auto nb = [&](int f, bool below) -> Real { return below ? y2[f] : wr_get(y0, f); };
        face_out<MODEL, Real, 1>(d, y1, nb, d.lamr[1], fyL, fyR, fyM);
        fyE = roe_of(y1);
        if (J <= NG + ny && I >= NG && I < NG + nx && y1.active && (!KD || ((rp.kind | ka) & 1u)))
          courmax = fmax(courmax, fmax(fabs(y1.s1), fabs(y1.sN)) * d.lamr[1]);
      } else {
#pragma unroll
        for (int k = 0; k < NV; k++) fyL[k] = fyR[k] = Real(0);
        fyE.un = fyE.ut = fyE.w = fyE.sg = fyE.pb = fyE.K = fyE.gh = fyE.C = Real(0);
      }
    }
    // y fluctuations entering cell (I, r - 2): R_y(I, r - 2) + L_y(I, r - 1)
    Real uy[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) { uy[k] = ry1[k] + fyL[k]; sm.uy[k][t] = uy[k]; }
    // record of row r - 1 for the x solve of its right neighbour
    {
#pragma unroll
      for (int k = 0; k < NV; k++) sm.rec[k][t] = rp.W[k];
#pragma unroll
      for (int k = 0; k < NV - 1; k++) sm.rec[NV + k][t] = rp.P[k];
      sm.rec[2 * NV - 1][t] = rp.b;
      sm.rec[2 * NV][t] = rp.c2;
      sm.rec[2 * NV + 1][t] = rp.hr;
      sm.rec[2 * NV + 2][t] = rp.sqh;
      sm.rec[2 * NV + 3][t] = rp.C;
      sm.wet[t] = rp.wet ? 1 : 0;
      if (KD) sm.kind[t] = rp.kind;
      sm.g2[t] = rp.g2;
      sm.e64[t] = rp.e64;
    }
    __syncthreads();

    // ===== B: x face I of row r - 1 (between columns I - 1 and I)
    Waves<Real> xv = zero_waves<Real>();
    {
      const int J = r - 1;
      if (t >= 1 && J >= 1 && J <= ny + 2 && I >= 1 && I <= nx + 3 && J >= rs) {
        Rec<MODEL, Real> lf;
#pragma unroll
        for (int k = 0; k < NV; k++) lf.W[k] = sm.rec[k][t - 1];
#pragma unroll
        for (int k = 0; k < NV - 1; k++) lf.P[k] = sm.rec[NV + k][t - 1];
        lf.b = sm.rec[2 * NV - 1][t - 1];
        lf.c2 = sm.rec[2 * NV][t - 1];
        lf.hr = sm.rec[2 * NV + 1][t - 1];
        lf.sqh = sm.rec[2 * NV + 2][t - 1];
        lf.C = sm.rec[2 * NV + 3][t - 1];
        lf.wet = sm.wet[t - 1] != 0;
        lf.g2 = sm.g2[t - 1];
        lf.e64 = sm.e64[t - 1];
        lf.psx = Real(0);
        xv = normal_solve<MODEL, Real>(d, rec_side<MODEL, Real, 0>(lf), rec_side<MODEL, Real, 0>(rp), rp.psx);
      }
#pragma unroll
      for (int f = 0; f < WR_N; f++) sm.xw[f][t] = wr_get(xv, f);
    }
    __syncthreads();

    // ===== C: limited x face I of row r - 1: I in [2, nx+2], J in [1, ny+2]
    Real nL[NV], nR[NV], nM = Real(0);
    Roe<Real> nE;
    {
      const int J = r - 1;
      const bool go = t >= 2 && t <= FUSED_NT - 2 && J >= 1 && J <= ny + 2 && I >= 2 && I <= nx + 2 && J >= rs;
      if (go) {
        auto nb = [&](int f, bool left) -> Real { return sm.xw[f][left ? t - 1 : t + 1]; };
        face_out<MODEL, Real, 0>(d, xv, nb, d.lamr[0], nL, nR, nM);
        nE = roe_of(xv);
        if (I <= NG + nx && J >= NG && J < NG + ny && xv.active && (!KD || ((rp.kind | sm.kind[t - 1]) & 1u)))
          courmax = fmax(courmax, fmax(fabs(xv.s1), fabs(xv.sN)) * d.lamr[0]);
      } else {
#pragma unroll
        for (int k = 0; k < NV; k++) nL[k] = nR[k] = Real(0);
        nE.un = nE.ut = nE.w = nE.sg = nE.pb = nE.K = nE.gh = nE.C = Real(0);
      }
#pragma unroll
      for (int k = 0; k < NV; k++) sm.lx[k][t] = nL[k];
    }
    __syncthreads();

    // ===== D: transverse corrections
    // x fluctuations entering cell (I, r - 1): R_x(I) + L_x(I + 1) of row r - 1
    Real vx0[NV];
    {
      const bool nbok = t + 1 < FUSED_NT;
#pragma unroll
      for (int k = 0; k < NV; k++) vx0[k] = nR[k] + (nbok ? sm.lx[k][t + 1] : Real(0));
    }
    // y face J = r - 1: I in [2, nx+1], J in [2, ny+2]
    Real gyn[NV], hyn[NV], myn = Real(0);
    {
      const int J = r - 1;
      Real T[NV];
      const bool go = t >= 2 && t <= FUSED_NT - 3 && I >= 2 && I <= nx + 1 && J >= 2 && J <= ny + 2 && J - 2 >= rs;
      if (go) {
        trans_out<MODEL, Real, 1>(d, fyE, fyM, vx1, vx0, T);
      } else {
#pragma unroll
        for (int k = 0; k < NV; k++) T[k] = Real(0);
      }
      myn = T[0];
#pragma unroll
      for (int k = 1; k < NV; k++) { gyn[k] = fyL[k] + T[k]; hyn[k] = fyR[k] - T[k]; }
      gyn[0] = hyn[0] = Real(0);
    }
    // x face I of row J = r - 2: I in [2, nx+2], J in [2, ny+1]
    Real hxn[NV], mxn = Real(0);
    {
      const int J = r - 2;
      Real T[NV];
      const bool go = t >= 2 && t <= FUSED_NT - 2 && I >= 2 && I <= nx + 2 && J >= 2 && J <= ny + 1 && J - 2 >= rs;
      if (go) {
        Real Va[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) Va[k] = sm.uy[k][t - 1];
        trans_out<MODEL, Real, 0>(d, fxE, fxM, Va, uy, T);
      } else {
#pragma unroll
        for (int k = 0; k < NV; k++) T[k] = Real(0);
      }
      mxn = T[0];
      sm.gx[par][0][t] = T[0];
#pragma unroll
      for (int k = 1; k < NV; k++) {
        sm.gx[par][k][t] = fxL[k] + T[k];
        hxn[k] = fxR[k] - T[k];
      }
      hxn[0] = Real(0);
    }
    __syncthreads();

    // ===== E: positivity factor of cell (I, r - 2), update of cell (I, r - 3)
    Real thn = Real(1);
    {
      const int J = r - 2;
      const bool go = t >= 2 && t <= FUSED_NT - 3 && I >= NG && I < NG + nx && J >= NG && J < NG + ny &&
                      J - 2 >= rs && (!KD || (ka & 5u));
      if (go) {
        const Real fl = mxn, fr = sm.gx[par][0][t + 1], fb = my2, ft = myn;
        bool done = false;
        if (sizeof(Real) == 4) {
          Real o = d.lamr[0] * (fmax(fr, Real(0)) + fmax(-fl, Real(0))) +
                   d.lamr[1] * (fmax(ft, Real(0)) + fmax(-fb, Real(0)));
          Real hf = wa[0] - wab;
          if (o <= Real(0.5) * hf) done = true;
        }
        if (!done) {
          Crit Ml = (Crit)fl, Mr = (Crit)fr, Mb = (Crit)fb, Mt = (Crit)ft;
          Crit out = d.lam[0] * (fmax(Mr, 0.0) + fmax(-Ml, 0.0)) + d.lam[1] * (fmax(Mt, 0.0) + fmax(-Mb, 0.0));
          Crit h = (Crit)wa[0] - (Crit)wab;
          h = h > 0 ? h : 0;
          thn = Real(out > h ? h / out : 1.0);
        }
      }
      sm.th[par][t] = thn;
    }
    {
      const int J = r - 3;
      if (outcol && J >= b0 && J < b1 && (!KD || (kb & 1u))) {
        const int po = par ^ 1;
        const Real Ml = mx3, Mr = sm.gx[po][0][t + 1], Mb = my3, Mt = my2;
        const Real th = th3;
        const Real tl = Ml > Real(0) ? sm.th[po][t - 1] : (Ml < Real(0) ? th : Real(1));
        const Real tr = Mr > Real(0) ? th : (Mr < Real(0) ? sm.th[po][t + 1] : Real(1));
        const Real tb = Mb > Real(0) ? th4 : (Mb < Real(0) ? th : Real(1));
        const Real tt = Mt > Real(0) ? th : (Mt < Real(0) ? thn : Real(1));
        const Real lx = d.lamr[0], ly = d.lamr[1];   // the FP64 factors rounded once (the same values)
        if (KD && (kb & 8u) && xphi) {
          Real* o = xphi + 4 * (size_t)d.xslot[at(d.pitch, I, J)];
          o[0] = tl * Ml;
          o[1] = tr * Mr;
          o[2] = tb * Mb;
          o[3] = tt * Mt;
        }
        Real en = wb[0] - lx * (tr * Mr - tl * Ml) - ly * (tt * Mt - tb * Mb);
        Real q[NV];
        bool bad = !isfinite(en);
#pragma unroll
        for (int k = 1; k < NV; k++) {
          Real v = wb[k] - lx * (tl * hx3[k] + tr * sm.gx[po][k][t + 1]) - ly * (tb * hy3[k] + tt * gy2[k]);
          bad = bad || !isfinite(v);
          q[k] = v;
        }
        const Real b = wbb, c2 = wbc;
        const Real ntol = Real(sizeof(Real) == 8 ? 1e-12 : 1e-6);
        if ((en - b) < -ntol * (Real(1) + fabs(b))) set_status(d.status, ST_NEGDEPTH);
        if (bad) set_status(d.status, ST_NONFINITE);
        q[0] = en;
        Real hr = en - b;
        hr = hr > Real(0) ? hr : Real(0);
        const bool wet = hr > d.rdry_tol;
        source_switch<MODEL, Real>(q, wet, hr, c2, d.lamr[3]);
        Real* qo = d.q[1 - cur];
        const size_t id = at(d.pitch, I, J);
#pragma unroll
        for (int k = 0; k < NV; k++) qo[k * d.fs + id] = q[k];
        spmax = fmax(spmax, cell_speed<MODEL, Real>(d, q, wet, hr, c2));
      }
    }

    // ===== shift the column state by one row
#pragma unroll
    for (int k = 0; k < NV; k++) {
      wb[k] = wa[k];
      wa[k] = rp.W[k];
      hy3[k] = hy2[k];
      hy2[k] = hyn[k];
      gy2[k] = gyn[k];
      hx3[k] = hxn[k];
      vx1[k] = vx0[k];
      fxL[k] = nL[k];
      fxR[k] = nR[k];
      ry1[k] = fyR[k];
    }
    wbb = wab; wbc = wac;
    wab = rp.b; wac = rp.c2;
    my3 = my2; my2 = myn;
    mx3 = mxn;
    th4 = th3; th3 = thn;
    if (KD) { kb = ka; ka = rp.kind; }
    fxM = nM; fxE = nE;
#pragma unroll
    for (int f = 0; f < WR_N; f++) y2[f] = wr_get(y1, f);
    y1 = y0;
    rp = rc;
  }
  cp_async_wait<0>();
}

// The one-pass step.  A persistent grid (as many blocks as stay resident) takes
// tiles in row-chunk-major order from a device counter, so that the blocks in
// flight work on neighbouring strips of the same rows (their halo columns meet
// in L2) and wet and dry tiles, whose costs differ, balance over the SMs.  The
// last block to finish clears the counters for the next launch.
template <int MODEL, typename Real, bool KD>
__global__ void __launch_bounds__(FUSED_NT, SGN_FUSED_MINB)
    k_step_fused(Dev<Real> d, int cur, FusedPlan p, Real* __restrict__ xphi) {
  typedef FusedSmem<MODEL, Real> SM;
  extern __shared__ __align__(16) unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>(smraw);
  Real courmax = Real(0), spmax = Real(0);
  for (;;) {
    if (threadIdx.x == 0) sm.tile = (int)atomicAdd(&d.tiles[0], 1u);
    __syncthreads();
    const int tile = sm.tile;
    __syncthreads();
    if (tile >= p.ntiles) break;
    int r0, nr, u = tile;
    if (u < p.n1) {
      r0 = u / p.nsx * p.H1; nr = p.H1;
    } else if ((u -= p.n1) < p.n2) {
      r0 = p.R1 + u / p.nsx * p.H2; nr = p.H2;
    } else {
      u -= p.n2;
      r0 = p.R2 + u / p.nsx * p.H3; nr = p.H3;
    }
    fused_tile<MODEL, Real, KD>(d, sm, cur, tile % p.nsx, r0, nr, courmax, spmax, xphi);
  }
  warp_max_to(d.cmax, courmax);
  warp_max_to(d.smax, spmax);
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&d.tiles[1], 1u) == gridDim.x - 1) {
      d.tiles[0] = 0u;
      d.tiles[1] = 0u;
    }
  }
}

}  // namespace sgn
