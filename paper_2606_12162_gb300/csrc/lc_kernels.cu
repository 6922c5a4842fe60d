// lc_kernels.cu -- learned coarse-to-fine corrector: 3x3 convolution network
// with hand-written forward, backward (data and weight gradients), loss and Adam
// kernels, plus the data kernels that turn solver states into inputs/targets.
//
// Convolutions run on the CUDA cores: weights stored as BF16 and expanded to
// FP32 in shared memory, FP32 activations and accumulation.  The weight
// gradients are formed per 16x16 pixel tile and summed over tiles in a fixed
// order, so training is run-to-run reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/lc.h"

namespace {

constexpr int TS = 16;        // output tile edge
constexpr int CIC = 8;        // input channels per shared-memory chunk
constexpr int COT = 16;       // output channels per block (forward)

// Forward 3x3 convolution, padding 1: out[co][y][x] = bias[co] +
// sum_ci sum_k w[co][ci][k] in[ci][y+ky-1][x+kx-1], then optional ReLU and an
// optional multiplication by the mask (mask_src > 0) used by the backward pass.
// WT: weight element type (BF16 network weights or FP32 flipped weights).
// A block of TS x TS threads computes a TS x (PX TS) output tile: each thread
// PX pixels TS columns apart, so every weight vector read from shared memory
// feeds PX pixels' FMAs.
constexpr int PX = 4;          // output pixels per thread (along x)
constexpr int TSX = PX * TS;   // output tile width of the convolution
template <typename WT>
__global__ void __launch_bounds__(TS * TS) k_conv3x3(const float* __restrict__ in, int cin, int H, int W,
                                                     const WT* __restrict__ w, const float* __restrict__ bias,
                                                     int cout, int relu, const float* __restrict__ mask_src,
                                                     float* __restrict__ out) {
  __shared__ float sin_[CIC][TS + 2][TSX + 2];
  __shared__ __align__(16) float sw[CIC][9][COT];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TS + tx;
  const int x0 = blockIdx.x * TSX + tx, y = blockIdx.y * TS + ty;
  const int co0 = blockIdx.z * COT;
  float acc[PX][COT];
#pragma unroll
  for (int h = 0; h < PX; h++)
#pragma unroll
    for (int c = 0; c < COT; c++) acc[h][c] = 0.f;
  for (int c0 = 0; c0 < cin; c0 += CIC) {
    __syncthreads();
    for (int t = tid; t < CIC * (TS + 2) * (TSX + 2); t += TS * TS) {
      int ci = t / ((TS + 2) * (TSX + 2)), r = t - ci * (TS + 2) * (TSX + 2);
      int yy = r / (TSX + 2), xx = r - yy * (TSX + 2);
      int gy = blockIdx.y * TS + yy - 1, gx = blockIdx.x * TSX + xx - 1;
      float v = 0.f;
      if (c0 + ci < cin && gy >= 0 && gy < H && gx >= 0 && gx < W) v = in[((size_t)(c0 + ci) * H + gy) * W + gx];
      sin_[ci][yy][xx] = v;
    }
    for (int t = tid; t < CIC * 9 * COT; t += TS * TS) {
      int ci = t / (9 * COT), r = t - ci * 9 * COT;
      int k = r / COT, co = r - k * COT;
      float v = 0.f;
      if (c0 + ci < cin && co0 + co < cout) v = (float)w[((size_t)(co0 + co) * cin + (c0 + ci)) * 9 + k];
      sw[ci][k][co] = v;
    }
    __syncthreads();
    for (int ci = 0; ci < CIC; ci++) {
#pragma unroll
      for (int k = 0; k < 9; k++) {
        float v[PX];
#pragma unroll
        for (int h = 0; h < PX; h++) v[h] = sin_[ci][ty + k / 3][tx + h * TS + k % 3];
#pragma unroll
        for (int c = 0; c < COT; c += 4) {
          const float4 w4 = *reinterpret_cast<const float4*>(&sw[ci][k][c]);
#pragma unroll
          for (int h = 0; h < PX; h++) {
            acc[h][c] += w4.x * v[h];
            acc[h][c + 1] += w4.y * v[h];
            acc[h][c + 2] += w4.z * v[h];
            acc[h][c + 3] += w4.w * v[h];
          }
        }
      }
    }
  }
  if (y >= H) return;
#pragma unroll
  for (int h = 0; h < PX; h++) {
    const int x = x0 + h * TS;
    if (x >= W) break;
#pragma unroll
    for (int c = 0; c < COT; c++) {
      int co = co0 + c;
      if (co >= cout) break;
      float v = acc[h][c] + (bias ? bias[co] : 0.f);
      if (relu) v = v > 0.f ? v : 0.f;
      size_t o = ((size_t)co * H + y) * W + x;
      if (mask_src && !(mask_src[o] > 0.f)) v = 0.f;
      out[o] = v;
    }
  }
}

// Weights for the input gradient: wf[ci][co][k] = w[co][ci][8 - k] (the
// transposed, flipped kernel), so that dL/din = conv3x3(dL/dout, wf).
__global__ void k_flip(const __nv_bfloat16* __restrict__ w, int cin, int cout, float* __restrict__ wf) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cin * cout * 9) return;
  int ci = t / (cout * 9), r = t - ci * cout * 9;
  int co = r / 9, k = r - co * 9;
  wf[t] = (float)w[((size_t)co * cin + ci) * 9 + (8 - k)];
}

// Weight and bias gradient partials of one 16x16 pixel tile:
// part[tile][co][ci][k] = sum_p g[co][p] in[ci][p + off_k], part[tile][bias co] =
// sum_p g[co][p].  Summed over tiles by k_sum_tiles.
__global__ void __launch_bounds__(TS * TS) k_wgrad(const float* __restrict__ in, int cin, int H, int W,
                                                   const float* __restrict__ g, int cout, float* __restrict__ part,
                                                   long nper) {
  __shared__ float sg[COT][TS][TS];
  __shared__ float sin_[CIC][TS + 2][TS + 2];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TS + tx;
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  float* pt = part + (size_t)tile * nper;
  for (int co0 = 0; co0 < cout; co0 += COT) {
    __syncthreads();
    for (int t = tid; t < COT * TS * TS; t += TS * TS) {
      int c = t / (TS * TS), r = t - c * TS * TS;
      int yy = r / TS, xx = r - yy * TS;
      int gy = blockIdx.y * TS + yy, gx = blockIdx.x * TS + xx;
      float v = 0.f;
      if (co0 + c < cout && gy < H && gx < W) v = g[((size_t)(co0 + c) * H + gy) * W + gx];
      sg[c][yy][xx] = v;
    }
    __syncthreads();
    // bias partials
    if (tid < COT && co0 + tid < cout) {
      float s = 0.f;
      for (int p = 0; p < TS * TS; p++) s += sg[tid][p / TS][p % TS];
      pt[(size_t)cout * cin * 9 + co0 + tid] = s;
    }
    for (int c0 = 0; c0 < cin; c0 += CIC) {
      __syncthreads();
      for (int t = tid; t < CIC * (TS + 2) * (TS + 2); t += TS * TS) {
        int ci = t / ((TS + 2) * (TS + 2)), r = t - ci * (TS + 2) * (TS + 2);
        int yy = r / (TS + 2), xx = r - yy * (TS + 2);
        int gy = blockIdx.y * TS + yy - 1, gx = blockIdx.x * TS + xx - 1;
        float v = 0.f;
        if (c0 + ci < cin && gy >= 0 && gy < H && gx >= 0 && gx < W) v = in[((size_t)(c0 + ci) * H + gy) * W + gx];
        sin_[ci][yy][xx] = v;
      }
      __syncthreads();
      for (int t = tid; t < COT * CIC * 9; t += TS * TS) {
        int c = t / (CIC * 9), r = t - c * CIC * 9;
        int ci = r / 9, k = r - ci * 9;
        if (co0 + c >= cout || c0 + ci >= cin) continue;
        const int ky = k / 3, kx = k % 3;
        float s = 0.f;
        for (int yy = 0; yy < TS; yy++)
#pragma unroll 4
          for (int xx = 0; xx < TS; xx++) s += sg[c][yy][xx] * sin_[ci][yy + ky][xx + kx];
        pt[((size_t)(co0 + c) * cin + (c0 + ci)) * 9 + k] = s;
      }
    }
  }
}

// grad[i] = sum over tiles of part[tile][i], in tile order.
__global__ void k_sum_tiles(const float* __restrict__ part, int ntiles, long n, float* __restrict__ grad) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int t = 0; t < ntiles; t++) s += part[(size_t)t * n + i];
  grad[i] = s;
}

// Loss of the pixel-shuffled output against the fine target and its gradient:
// channel f*r*r + sy*r + sx of coarse pixel (y, x) is fine cell (r y + sy, r x + sx)
// of field f.  Per-block loss partials are summed in order by k_sum_loss.
__global__ void k_loss(const float* __restrict__ yv, const float* __restrict__ tgt, int H, int W, int r, int nout,
                       const float* __restrict__ fw, float* __restrict__ gy, double* __restrict__ lpart) {
  __shared__ double red[256];
  long n = (long)nout * r * r * H * W;
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    int c = (int)(i / ((long)H * W));
    long p = i - (long)c * H * W;
    int yy = (int)(p / W), xx = (int)(p - (long)yy * W);
    int f = c / (r * r), s = c - f * r * r, sy = s / r, sx = s - sy * r;
    int Wf = W * r;
    float d = yv[i] - tgt[((size_t)f * H * r + (size_t)(yy * r + sy)) * Wf + (xx * r + sx)];
    float inv = 1.f / (float)((long)H * W * r * r);
    gy[i] = 2.f * fw[f] * d * inv;
    l = (double)fw[f] * (double)d * (double)d * (double)inv;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) lpart[blockIdx.x] = red[0];
}

__global__ void k_sum_loss(const double* __restrict__ lpart, int n, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; i++) s += lpart[i];
  *out = s;
}

// Adam on the FP32 master parameters and refresh of their BF16 copy.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, long n, float lr, float bc1,
                       float bc2) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = 0.9f * m[i] + 0.1f * gi;
  float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
  p[i] = pi;
  pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

// --- data kernels -----------------------------------------------------------
__global__ void k_make_input(const double* __restrict__ q, const double* __restrict__ b,
                             const unsigned char* __restrict__ phi, int H, int W, float se, float sq, float sb,
                             float* __restrict__ x) {
  long n = (long)H * W;
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double bb = b[i];
  double eta = q[i];
  x[i] = (float)((bb < 0.0 ? eta : 0.0) / se);         // surface deviation over the ocean
  x[n + i] = (float)(q[n + i] / sq);
  x[2 * n + i] = (float)(q[2 * n + i] / sq);
  x[3 * n + i] = (float)(bb / sb);
  x[4 * n + i] = phi ? (float)phi[i] : 0.f;
}

__global__ void k_make_target(const double* __restrict__ qf, const double* __restrict__ qc,
                              const double* __restrict__ bf, const double* __restrict__ bc, int Hc, int Wc, int r,
                              float se, float sq, float* __restrict__ t) {
  long Wf = (long)Wc * r, n = (long)Hc * r * Wf;
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  int f = (int)(i / n);
  long p = i - (long)f * n;
  long Y = p / Wf, X = p - Y * Wf;
  size_t ic = (size_t)f * Hc * Wc + (size_t)(Y / r) * Wc + (X / r);
  float s = f == 0 ? se : sq;
  // fine land, or a fine cell whose coarse cell is land, at or above the still
  // level: no surface target (its eta is bathymetry, not a wave)
  if (f == 0 && ((bf && bf[p] >= 0.0) || (bc && bc[ic] >= 0.0))) { t[i] = 0.f; return; }
  t[i] = (float)((qf[i] - qc[ic]) / s);
}

__global__ void k_apply(const double* __restrict__ qc, const float* __restrict__ y, int Hc, int Wc, int r, float se,
                        float sq, int use_net, double* __restrict__ out) {
  long Wf = (long)Wc * r, n = (long)Hc * r * Wf;
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  int f = (int)(i / n);
  long p = i - (long)f * n;
  long Y = p / Wf, X = p - Y * Wf;
  long yc = Y / r, xc = X / r;
  double v = qc[(size_t)f * Hc * Wc + (size_t)yc * Wc + xc];
  if (use_net) {
    int c = f * r * r + (int)(Y - yc * r) * r + (int)(X - xc * r);
    v += (double)(f == 0 ? se : sq) * (double)y[((size_t)c * Hc + yc) * Wc + xc];
  }
  out[i] = v;
}

__global__ void k_restrict(const double* __restrict__ fine, int Hc, int Wc, int r, double* __restrict__ coarse) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)Hc * Wc) return;
  long yc = i / Wc, xc = i - yc * Wc;
  long Wf = (long)Wc * r;
  double s = 0.0;
  for (int a = 0; a < r; a++)
    for (int b = 0; b < r; b++) s += fine[(yc * r + a) * Wf + xc * r + b];
  coarse[i] = s / (double)(r * r);
}

unsigned long long splitmix(unsigned long long& s) {
  unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct lc_net {
  int cin, width, depth, cout;
  long max_hw;
  cudaStream_t st;
  std::vector<int> ci, co;
  std::vector<long> woff, boff;
  long np;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* pb = nullptr;
  std::vector<float*> act;      // act[l]: output of layer l (l = 0..depth-1)
  float *ga = nullptr, *gb = nullptr, *wf = nullptr, *part = nullptr;
  double *lpart = nullptr, *lsum = nullptr;
  float* fw = nullptr;          // loss field weights (device copy)
  long max_layer;
  int max_tiles, max_lblocks;
  long step = 0;
  std::vector<void*> bufs;
};

static void* dmalloc(lc_net* n, size_t bytes) {
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
  n->bufs.push_back(q);
  return q;
}

extern "C" {

int lc_create(int cin, int width, int depth, int cout, long max_hw, unsigned long long seed, void* cuda_stream,
              lc_net** out) {
  if (!out || cin <= 0 || width <= 0 || depth < 2 || cout <= 0 || max_hw <= 0) return -1;
  *out = nullptr;
  lc_net* n = new (std::nothrow) lc_net;
  if (!n) return -2;
  n->cin = cin; n->width = width; n->depth = depth; n->cout = cout; n->max_hw = max_hw;
  n->st = (cudaStream_t)cuda_stream;
  long off = 0;
  n->max_layer = 0;
  for (int l = 0; l < depth; l++) {
    int a = l == 0 ? cin : width, b = l == depth - 1 ? cout : width;
    n->ci.push_back(a); n->co.push_back(b);
    n->woff.push_back(off); off += (long)a * b * 9;
    n->boff.push_back(off); off += b;
    n->max_layer = std::max(n->max_layer, (long)a * b * 9 + b);
  }
  n->np = off;
  long maxc = std::max(width, cout);
  // ceil(H/16) ceil(W/16) <= HW/256 + (H + W)/16 + 1 <= HW/15 + 2 for any H, W >= 1
  n->max_tiles = (int)((max_hw + 14) / 15 + 2);
  n->max_lblocks = (int)((max_hw * cout + 255) / 256) + 1;
  n->p = (float*)dmalloc(n, n->np * 4); n->g = (float*)dmalloc(n, n->np * 4);
  n->m = (float*)dmalloc(n, n->np * 4); n->v = (float*)dmalloc(n, n->np * 4);
  n->pb = (__nv_bfloat16*)dmalloc(n, n->np * 2);
  for (int l = 0; l < depth; l++) n->act.push_back((float*)dmalloc(n, (size_t)n->co[l] * max_hw * 4));
  n->ga = (float*)dmalloc(n, (size_t)maxc * max_hw * 4);
  n->gb = (float*)dmalloc(n, (size_t)maxc * max_hw * 4);
  n->wf = (float*)dmalloc(n, (size_t)n->max_layer * 4);
  n->part = (float*)dmalloc(n, (size_t)n->max_tiles * n->max_layer * 4);
  n->lpart = (double*)dmalloc(n, (size_t)n->max_lblocks * 8);
  n->lsum = (double*)dmalloc(n, 8);
  n->fw = (float*)dmalloc(n, 8 * sizeof(float));
  bool ok = n->p && n->g && n->m && n->v && n->pb && n->ga && n->gb && n->wf && n->part && n->lpart && n->lsum &&
            n->fw;
  for (auto a : n->act) ok = ok && a;
  if (!ok) { lc_destroy(n); return -2; }
  // He initialisation from a counter-based generator (splitmix64 + Box-Muller)
  std::vector<float> h(n->np, 0.f);
  unsigned long long s = seed;
  for (int l = 0; l < depth; l++) {
    double sd = std::sqrt(2.0 / (9.0 * n->ci[l]));
    if (l == depth - 1) sd *= 0.1;   // small initial corrections
    for (long i = 0; i < (long)n->ci[l] * n->co[l] * 9; i++) {
      double u1 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      double u2 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      h[n->woff[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  int r = lc_set_params(n, h.data(), n->np);
  if (r) { lc_destroy(n); return r; }
  *out = n;
  return 0;
}

void lc_destroy(lc_net* n) {
  if (!n) return;
  if (n->st) cudaStreamSynchronize(n->st);
  for (void* q : n->bufs) cudaFree(q);
  delete n;
}

long lc_num_params(lc_net* n) { return n ? n->np : -1; }

int lc_get_params(lc_net* n, float* host, long count) {
  if (!n || !host || count < n->np) return -1;
  if (cudaMemcpyAsync(host, n->p, n->np * 4, cudaMemcpyDeviceToHost, n->st) != cudaSuccess) return -3;
  return cudaStreamSynchronize(n->st) == cudaSuccess ? 0 : -3;
}

int lc_set_params(lc_net* n, const float* host, long count) {
  if (!n || !host || count < n->np) return -1;
  if (cudaMemcpyAsync(n->p, host, n->np * 4, cudaMemcpyHostToDevice, n->st) != cudaSuccess) return -3;
  if (cudaMemsetAsync(n->m, 0, n->np * 4, n->st) != cudaSuccess) return -3;
  if (cudaMemsetAsync(n->v, 0, n->np * 4, n->st) != cudaSuccess) return -3;
  k_to_bf16<<<nblk(n->np, 256), 256, 0, n->st>>>(n->p, n->pb, n->np);
  n->step = 0;
  if (cudaGetLastError() != cudaSuccess) return -3;
  return cudaStreamSynchronize(n->st) == cudaSuccess ? 0 : -3;
}

static void conv_fwd(lc_net* n, int l, const float* in, int H, int W, float* out) {
  dim3 grid((W + TSX - 1) / TSX, (H + TS - 1) / TS, (n->co[l] + COT - 1) / COT);
  k_conv3x3<__nv_bfloat16><<<grid, dim3(TS, TS), 0, n->st>>>(in, n->ci[l], H, W, n->pb + n->woff[l],
                                                               n->p + n->boff[l], n->co[l],
                                                               l < n->depth - 1 ? 1 : 0, nullptr, out);
}

int lc_forward(lc_net* n, const float* x_dev, int H, int W, float* y_dev) {
  if (!n || !x_dev || !y_dev || H <= 0 || W <= 0 || (long)H * W > n->max_hw) return -1;
  const float* in = x_dev;
  for (int l = 0; l < n->depth; l++) {
    float* o = l == n->depth - 1 ? y_dev : n->act[l];
    conv_fwd(n, l, in, H, W, o);
    in = o;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lc_train_step(lc_net* n, const float* x_dev, const float* target_dev, int H, int W, int r, int nout,
                  const float* field_w, float lr, double* loss, float* grad_host) {
  if (!n || !x_dev || !target_dev || !field_w || H <= 0 || W <= 0 || r <= 0 || nout <= 0) return -1;
  if ((long)H * W > n->max_hw || nout * r * r != n->cout || nout > 8 || lr < 0) return -1;
  // forward, keeping every layer's output
  const float* in = x_dev;
  for (int l = 0; l < n->depth; l++) {
    conv_fwd(n, l, in, H, W, n->act[l]);
    in = n->act[l];
  }
  // loss and dL/dy
  long ny = (long)n->cout * H * W;
  int lb = (int)nblk(ny, 256);
  if (lb > n->max_lblocks) return -1;
  if (cudaMemcpyAsync(n->fw, field_w, nout * sizeof(float), cudaMemcpyHostToDevice, n->st) != cudaSuccess) return -3;
  k_loss<<<lb, 256, 0, n->st>>>(n->act[n->depth - 1], target_dev, H, W, r, nout, n->fw, n->ga, n->lpart);
  k_sum_loss<<<1, 32, 0, n->st>>>(n->lpart, lb, n->lsum);
  // backward: g (in ga) is dL/d(pre-activation) of layer l
  dim3 tiles((W + TS - 1) / TS, (H + TS - 1) / TS);
  int ntiles = tiles.x * tiles.y;
  if (ntiles > n->max_tiles) return -1;
  for (int l = n->depth - 1; l >= 0; l--) {
    const float* lin = l == 0 ? x_dev : n->act[l - 1];
    long nl = (long)n->ci[l] * n->co[l] * 9 + n->co[l];
    k_wgrad<<<tiles, dim3(TS, TS), 0, n->st>>>(lin, n->ci[l], H, W, n->ga, n->co[l], n->part, nl);
    k_sum_tiles<<<nblk(nl, 256), 256, 0, n->st>>>(n->part, ntiles, nl, n->g + n->woff[l]);
    if (l > 0) {
      int a = n->ci[l], b = n->co[l];
      k_flip<<<nblk((long)a * b * 9, 256), 256, 0, n->st>>>(n->pb + n->woff[l], a, b, n->wf);
      dim3 grid((W + TSX - 1) / TSX, (H + TS - 1) / TS, (a + COT - 1) / COT);
      // dL/d(out of layer l-1), times ReLU'(out of layer l-1)
      k_conv3x3<float><<<grid, dim3(TS, TS), 0, n->st>>>(n->ga, b, H, W, n->wf, nullptr, a, 0, n->act[l - 1],
                                                         n->gb);
      float* t = n->ga; n->ga = n->gb; n->gb = t;
    }
  }
  if (cudaGetLastError() != cudaSuccess) return -3;
  if (cudaMemcpyAsync(loss, n->lsum, 8, cudaMemcpyDeviceToHost, n->st) != cudaSuccess) return -3;
  if (lr > 0) {
    n->step++;
    float bc1 = 1.f - powf(0.9f, (float)n->step), bc2 = 1.f - powf(0.999f, (float)n->step);
    k_adam<<<nblk(n->np, 256), 256, 0, n->st>>>(n->p, n->g, n->m, n->v, n->pb, n->np, lr, bc1, bc2);
  } else if (grad_host) {
    if (cudaMemcpyAsync(grad_host, n->g, n->np * 4, cudaMemcpyDeviceToHost, n->st) != cudaSuccess) return -3;
  }
  if (cudaGetLastError() != cudaSuccess) return -3;
  return cudaStreamSynchronize(n->st) == cudaSuccess ? 0 : -3;
}

int lc_make_input(const double* q_dev, const double* b_dev, const unsigned char* phi_dev, int Hc, int Wc,
                  float s_eta, float s_q, float s_b, float* x_dev, void* cuda_stream) {
  if (!q_dev || !b_dev || !x_dev || Hc <= 0 || Wc <= 0) return -1;
  long nn = (long)Hc * Wc;
  k_make_input<<<nblk(nn, 256), 256, 0, (cudaStream_t)cuda_stream>>>(q_dev, b_dev, phi_dev, Hc, Wc, s_eta, s_q,
                                                                       s_b, x_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lc_make_target(const double* qf_dev, const double* qc_dev, const double* bf_dev, const double* bc_dev, int Hc,
                   int Wc, int r, float s_eta, float s_q, float* t_dev, void* cuda_stream) {
  if (!qf_dev || !qc_dev || !t_dev || Hc <= 0 || Wc <= 0 || r <= 0) return -1;
  long nn = 3L * Hc * r * Wc * r;
  k_make_target<<<nblk(nn, 256), 256, 0, (cudaStream_t)cuda_stream>>>(qf_dev, qc_dev, bf_dev, bc_dev, Hc, Wc, r,
                                                                        s_eta, s_q, t_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lc_apply(const double* qc_dev, const float* y_dev, int Hc, int Wc, int r, float s_eta, float s_q, int use_net,
             double* out_dev, void* cuda_stream) {
  if (!qc_dev || !out_dev || (use_net && !y_dev) || Hc <= 0 || Wc <= 0 || r <= 0) return -1;
  long nn = 3L * Hc * r * Wc * r;
  k_apply<<<nblk(nn, 256), 256, 0, (cudaStream_t)cuda_stream>>>(qc_dev, y_dev, Hc, Wc, r, s_eta, s_q, use_net,
                                                                  out_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lc_restrict(const double* fine_dev, int Hc, int Wc, int r, double* coarse_dev, void* cuda_stream) {
  if (!fine_dev || !coarse_dev || Hc <= 0 || Wc <= 0 || r <= 0) return -1;
  k_restrict<<<nblk((long)Hc * Wc, 256), 256, 0, (cudaStream_t)cuda_stream>>>(fine_dev, Hc, Wc, r, coarse_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
