// lc_kernels.cu -- learned coarse-to-fine corrector: 3x3 convolution network
// with hand-written forward, backward (data and weight gradients), loss and Adam
// kernels, plus the data kernels that turn solver states into inputs/targets.
//
// Convolutions run on the tensor cores (mma.sync, BF16 operands: the BF16
// weights and the activations or gradients rounded to BF16 as they are staged;
// FP32 accumulation; FP32 activations, biases, losses and master weights).  The
// weight gradients are summed per block of a fixed persistent grid, then over
// blocks in a fixed order, so training is run-to-run reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/lc.h"

namespace {

// ---------------------------------------------------------------------------
// 3x3 convolutions as implicit GEMMs on the tensor cores: mma.sync m16n8k16
// with BF16 operands and FP32 accumulation.
//
// Layouts.  The network input x and its output y are FP32 channel-major planes
// [c][y][x] (the data kernels' layout).  Everything in between -- hidden
// activations and the gradients flowing back through them -- is stored as BF16
// pixel-major rows [y][x][c] of CS = channels rounded up to 16 (the padding
// stays zero): the values the tensor cores multiply are BF16 anyway, so this
// changes no result and halves the bytes.  A block stages a tile of the input
// in shared memory as [pixel][channel] rows of CS + 8 BF16 (the 8 extra keep
// the 16-byte ldmatrix rows of consecutive pixels on different banks), so any
// 3x3 tap offset is a whole-row shift and every operand row stays 16-byte
// aligned: pixel-major inputs arrive by 16-byte cp.async (zero-filled outside
// the image), double-buffered across tiles; channel-major FP32 inputs are read,
// rounded and stored by the threads.
constexpr int CT_H = 8;              // output tile rows (one per warp)
constexpr int CT_W = 32;             // output tile columns (two 16-pixel MMA rows)
constexpr int CT_PIX = (CT_H + 2) * (CT_W + 2);   // staged input pixels (tile + halo)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
// D = A B + D for one 16x8x16 tile (A row-major 16x16, B column-major 16x8).
__device__ __forceinline__ void mma_bf16(float* d, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}
// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros
// without reading (the address passed is then any valid one).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Stage rows [y0, y0 + ROWS) x columns [x0, x0 + COLS) of an input into
// shared-memory rows of PS BF16 (channels 0..CP-1), zero outside the image.
// Pixel-major BF16 source (nhwc, CP channels per pixel): 16-byte cp.async
// copies, committed as one group by the caller.  Channel-major FP32 source
// (planes [0, c)): loads go out in batches of SB element pairs per thread
// before any of them is stored, so a thread waits for one memory latency per
// batch, not per pair.
template <int CP, int PS, int ROWS, int COLS, int SB = 8>
__device__ __forceinline__ void stage_tile(const void* __restrict__ srcv, int nhwc, int c, int H, int W, int y0,
                                           int x0, __nv_bfloat16* dst) {
  if (nhwc) {
    const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(srcv);
    constexpr int CH = CP / 8, N = ROWS * COLS * CH;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
      const int ch = t % CH, pix = t / CH;
      const int yy = pix / COLS, xx = pix - yy * COLS;
      const int gy = y0 + yy, gx = x0 + xx;
      const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
      const __nv_bfloat16* s = in ? src + ((size_t)gy * W + gx) * CP + 8 * ch : src;
      cp_async16(dst + (size_t)pix * PS + 8 * ch, s, in ? 16 : 0);
    }
    return;
  }
  const float* src = static_cast<const float*>(srcv);
  constexpr int N = ROWS * COLS * (CP / 2);
  const size_t pl = (size_t)H * W;
  for (int base = threadIdx.x; base < N; base += SB * blockDim.x) {
    float v0[SB], v1[SB];
#pragma unroll
    for (int j = 0; j < SB; j++) {
      const int t = base + j * blockDim.x;
      const int xx = t % COLS, r = t / COLS;
      const int yy = r % ROWS, ch = 2 * (r / ROWS);
      const int gy = y0 + yy, gx = x0 + xx;
      v0[j] = v1[j] = 0.f;
      if (t < N && gy >= 0 && gy < H && gx >= 0 && gx < W) {
        const size_t o = (size_t)gy * W + gx;
        if (ch < c) v0[j] = __ldg(src + (size_t)ch * pl + o);
        if (ch + 1 < c) v1[j] = __ldg(src + (size_t)(ch + 1) * pl + o);
      }
    }
#pragma unroll
    for (int j = 0; j < SB; j++) {
      const int t = base + j * blockDim.x;
      if (t >= N) break;
      const int xx = t % COLS, r = t / COLS;
      const int yy = r % ROWS, ch = 2 * (r / ROWS);
      *reinterpret_cast<unsigned*>(dst + (size_t)(yy * COLS + xx) * PS + ch) = pack_bf16(v0[j], v1[j]);
    }
  }
}

// Convolution with padding 1: out[o][y][x] = bias[o] + sum_c sum_k
// B(o, c, k) in[c][y + ky - 1][x + kx - 1] (k = 3 ky + kx), then optional ReLU
// and an optional mask (out = 0 where mask <= 0; mask pixel-major BF16 like a
// pixel-major output).  in: pixel-major BF16 with CP channels (in_nhwc) or
// channel-major FP32 with cin planes; out: pixel-major BF16 with NT*8 channels,
// padding included (out_nhwc), or channel-major FP32 with cout planes.  The
// weights B are read from the network's BF16 tensor w: transpose = 0,
// B(o, c, k) = w[o][c][k] (the layer itself, w of shape cout x cin x 9);
// transpose = 1, B(o, c, k) = w[c][o][8 - k] (w of shape cin x cout x 9: the
// transposed, flipped kernel that maps dL/d(out) of that layer to dL/d(in)).
// Persistent blocks of 8 warps take tiles of 8 x 32 output pixels; warp w
// computes row w of the tile: 2 m-tiles of 16 pixels x NT n-tiles of 8 output
// channels, K = 9 taps x CP channels in steps of 16.
template <int CP, int NT>
__global__ void __launch_bounds__(256, 2) k_conv_mma(const void* __restrict__ in, int in_nhwc, int cin, int H, int W,
                                                     const __nv_bfloat16* __restrict__ w, int transpose,
                                                     const float* __restrict__ bias, int cout, int relu,
                                                     const __nv_bfloat16* __restrict__ mask, void* __restrict__ out,
                                                     int out_nhwc, int ntx, int ntiles) {
  constexpr int PS = CP + 8;
  constexpr int NO = NT * 8;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __nv_bfloat16* sB = reinterpret_cast<__nv_bfloat16*>(sm_raw);    // [9][NO][PS]
  __nv_bfloat16* sA0 = sB + 9 * NO * PS;                            // [2][CT_PIX][PS]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // weights, once per block: sB[k][o][c] = B(o, c, k), zero-padded
  for (int t = threadIdx.x; t < 9 * NO * CP; t += blockDim.x) {
    const int c = t % CP, r = t / CP, o = r % NO, k = r / NO;
    float v = 0.f;
    if (o < cout && c < cin)
      v = (float)(transpose ? w[((size_t)c * cout + o) * 9 + (8 - k)] : w[((size_t)o * cin + c) * 9 + k]);
    sB[(size_t)(k * NO + o) * PS + c] = __float2bfloat16_rn(v);
  }
  const int g = lane >> 2, tq = lane & 3;
  auto tile_origin = [&](int tile, int& ty0, int& tx0) {
    ty0 = (tile / ntx) * CT_H;
    tx0 = (tile % ntx) * CT_W;
  };
  if (in_nhwc && (int)blockIdx.x < ntiles) {
    int ty0, tx0;
    tile_origin(blockIdx.x, ty0, tx0);
    stage_tile<CP, PS, CT_H + 2, CT_W + 2>(in, 1, cin, H, W, ty0 - 1, tx0 - 1, sA0);
    cp_commit();
  }
  int it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
    int ty0, tx0;
    tile_origin(tile, ty0, tx0);
    __nv_bfloat16* sA = sA0 + (size_t)(in_nhwc ? (it & 1) : 0) * CT_PIX * PS;
    if (in_nhwc) {
      // prefetch the next tile into the other buffer (read by every thread in
      // the previous iteration, which ended with a barrier), then wait for this one
      const int nt = tile + gridDim.x;
      if (nt < ntiles) {
        int ny0, nx0;
        tile_origin(nt, ny0, nx0);
        stage_tile<CP, PS, CT_H + 2, CT_W + 2>(in, 1, cin, H, W, ny0 - 1, nx0 - 1,
                                               sA0 + (size_t)((it + 1) & 1) * CT_PIX * PS);
      }
      cp_commit();
      cp_wait<1>();
    } else {
      stage_tile<CP, PS, CT_H + 2, CT_W + 2>(in, 0, cin, H, W, ty0 - 1, tx0 - 1, sA);
    }
    __syncthreads();
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
      for (int n = 0; n < NT; n++)
#pragma unroll
        for (int e = 0; e < 4; e++) acc[m][n][e] = 0.f;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const int ky = k / 3, kx = k % 3;
#pragma unroll
      for (int c0 = 0; c0 < CP; c0 += 16) {
        unsigned a[2][4];
#pragma unroll
        for (int m = 0; m < 2; m++) {
          // A rows: pixels x = 16 m + (lane & 15) of output row `warp`, shifted by the tap
          const int px = 16 * m + (lane & 15) + kx, py = warp + ky;
          const __nv_bfloat16* pa = sA + (size_t)(py * (CT_W + 2) + px) * PS + c0 + 8 * (lane >> 4);
          ldsm_x4(smem_u32(pa), a[m][0], a[m][1], a[m][2], a[m][3]);
        }
#pragma unroll
        for (int n = 0; n < NT; n += 2) {
          unsigned b0, b1, b2, b3;
          const int o = 8 * (n + (lane >> 4)) + (lane & 7);
          const __nv_bfloat16* pb = sB + (size_t)(k * NO + o) * PS + c0 + 8 * ((lane >> 3) & 1);
          ldsm_x4(smem_u32(pb), b0, b1, b2, b3);
#pragma unroll
          for (int m = 0; m < 2; m++) {
            mma_bf16(acc[m][n], a[m][0], a[m][1], a[m][2], a[m][3], b0, b1);
            mma_bf16(acc[m][n + 1], a[m][0], a[m][1], a[m][2], a[m][3], b2, b3);
          }
        }
      }
    }
    // epilogue: rows g and g + 8 of each m-tile are pixels, columns 2 tq, 2 tq + 1 channels
    const int y = ty0 + warp;
    if (y < H) {
#pragma unroll
      for (int m = 0; m < 2; m++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int x = tx0 + 16 * m + g + 8 * h;
          if (x >= W) continue;
          const size_t pix = (size_t)y * W + x;
#pragma unroll
          for (int n = 0; n < NT; n++) {
            const int o = 8 * n + 2 * tq;
            float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
            if (bias) {
              if (o < cout) v0 += bias[o];
              if (o + 1 < cout) v1 += bias[o + 1];
            }
            if (relu) { v0 = v0 > 0.f ? v0 : 0.f; v1 = v1 > 0.f ? v1 : 0.f; }
            if (mask) {
              const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + pix * NO + o);
              if (!(__low2float(mk) > 0.f)) v0 = 0.f;
              if (!(__high2float(mk) > 0.f)) v1 = 0.f;
            }
            if (out_nhwc) {
              *reinterpret_cast<unsigned*>(static_cast<__nv_bfloat16*>(out) + pix * NO + o) = pack_bf16(v0, v1);
            } else {
              float* of = static_cast<float*>(out);
              if (o < cout) of[(size_t)o * H * W + pix] = v0;
              if (o + 1 < cout) of[(size_t)(o + 1) * H * W + pix] = v1;
            }
          }
        }
    }
    __syncthreads();   // this tile's buffer and the other one may be overwritten next
  }
  cp_wait<0>();
}

// Weight gradient partials: part[blk][o][c][k] = sum over the block's pixels
// p of g[o][p] in[c][p + off_k] (BF16 operands, FP32 accumulation), as a GEMM
// with M = output channels, N = input channels and K = pixels.  Both tiles are
// staged as [pixel][channel] rows (either source layout); ldmatrix.trans turns
// them into the A (o x p) and B (p x c) fragments.  Nine warps, one per tap;
// each block sums the tiles blockIdx.x, blockIdx.x + gridDim.x, ... in that
// order, and the partials of the blocks are summed in block order by
// k_sum_tiles, so the result does not depend on the schedule.
template <int OP, int CP>
__global__ void __launch_bounds__(288, 2) k_wgrad_mma(const void* __restrict__ in, int in_nhwc, int cin, int H,
                                                      int W, const void* __restrict__ g, int g_nhwc, int cout,
                                                      float* __restrict__ part, int ntx, int ntiles) {
  constexpr int PSI = CP + 8, PSG = OP + 8;
  constexpr int MT = OP / 16, NT = CP / 8;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __nv_bfloat16* sI = reinterpret_cast<__nv_bfloat16*>(sm_raw);     // [CT_PIX][PSI]
  __nv_bfloat16* sG = sI + CT_PIX * PSI;                             // [CT_H * CT_W][PSG]
  const int lane = threadIdx.x & 31, tap = threadIdx.x >> 5;
  const int ky = tap / 3, kx = tap % 3;
  float acc[MT][NT][4];
#pragma unroll
  for (int m = 0; m < MT; m++)
#pragma unroll
    for (int n = 0; n < NT; n++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[m][n][e] = 0.f;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ty0 = (tile / ntx) * CT_H, tx0 = (tile % ntx) * CT_W;
    __syncthreads();
    stage_tile<CP, PSI, CT_H + 2, CT_W + 2, 4>(in, in_nhwc, cin, H, W, ty0 - 1, tx0 - 1, sI);
    stage_tile<OP, PSG, CT_H, CT_W, 4>(g, g_nhwc, cout, H, W, ty0, tx0, sG);
    cp_commit();
    cp_wait<0>();
    __syncthreads();
    // K: the 256 pixels of the tile, 16 at a time (half a tile row)
    for (int ks = 0; ks < CT_H * CT_W / 16; ks++) {
      const int row = ks >> 1, xs = 16 * (ks & 1);
      unsigned a[MT][4];
#pragma unroll
      for (int m = 0; m < MT; m++) {
        // A (o x p) from sG rows = pixels: matrices (o 0-7, p 0-7), (o 8-15, p 0-7), (o 0-7, p 8-15), (o 8-15, p 8-15)
        const int p = xs + (lane & 7) + 8 * (lane >> 4);
        const __nv_bfloat16* pa = sG + (size_t)(row * CT_W + p) * PSG + 16 * m + 8 * ((lane >> 3) & 1);
        ldsm_x4_t(smem_u32(pa), a[m][0], a[m][1], a[m][2], a[m][3]);
      }
#pragma unroll
      for (int n = 0; n < NT; n += 2) {
        // B (p x c) from sI rows = pixels shifted by the tap: (p 0-7, c), (p 8-15, c), (p 0-7, c+8), (p 8-15, c+8)
        const int p = xs + (lane & 7) + 8 * ((lane >> 3) & 1) + kx;
        const __nv_bfloat16* pb = sI + (size_t)((row + ky) * (CT_W + 2) + p) * PSI + 8 * (n + (lane >> 4));
        unsigned b0, b1, b2, b3;
        ldsm_x4_t(smem_u32(pb), b0, b1, b2, b3);
#pragma unroll
        for (int m = 0; m < MT; m++) {
          mma_bf16(acc[m][n], a[m][0], a[m][1], a[m][2], a[m][3], b0, b1);
          mma_bf16(acc[m][n + 1], a[m][0], a[m][1], a[m][2], a[m][3], b2, b3);
        }
      }
    }
  }
  // this block's partial: rows g, g + 8 are output channels, columns 2 tq, 2 tq + 1 input channels
  const long nper = (long)cout * cin * 9;
  float* pt = part + (size_t)blockIdx.x * nper;
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int m = 0; m < MT; m++)
#pragma unroll
    for (int n = 0; n < NT; n++)
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int o = 16 * m + gq + 8 * (e >> 1), c = 8 * n + 2 * tq + (e & 1);
        if (o < cout && c < cin) pt[((size_t)o * cin + c) * 9 + tap] = acc[m][n][e];
      }
}

// Bias gradient partials of a hidden layer: part[chunk][o] = sum of g[p][o]
// over the pixels of chunk blockIdx.x (gridDim.x contiguous ranges), in FP32, in
// a fixed order; k_sum_chunks adds the chunks.  g: pixel-major BF16 with cs
// channels per pixel; thread t reads channel t % cs of every (blockDim / cs)-th
// pixel, so a warp reads consecutive bytes; the threads of one channel are then
// summed in thread order.
constexpr int BG_CHUNKS = 1024;
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ gb, int cs, long hw, int cout,
                            float* __restrict__ part) {
  __shared__ float red[256];
  const long p0 = hw * blockIdx.x / gridDim.x, p1 = hw * (blockIdx.x + 1) / gridDim.x;
  const int ppi = blockDim.x / cs;                     // pixels per pass
  const int o = threadIdx.x % cs, pk = threadIdx.x / cs;
  float s = 0.f;
  if (pk < ppi)
    for (long p = p0 + pk; p < p1; p += ppi) s += (float)gb[(size_t)p * cs + o];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < cout) {
    float t = 0.f;
    for (int k = 0; k < ppi; k++) t += red[k * cs + threadIdx.x];
    part[(size_t)blockIdx.x * cout + threadIdx.x] = t;
  }
}

// out[o] = sum over chunks k of part[k][o] (n values per chunk): one block per
// o; thread t adds chunks t, t + 256, ... in order, then a fixed tree.
__global__ void __launch_bounds__(256) k_sum_chunks(const float* __restrict__ part, int nchunks, int n,
                                                    float* __restrict__ out) {
  __shared__ float red[256];
  const int o = blockIdx.x;
  float s = 0.f;
  for (int k = threadIdx.x; k < nchunks; k += 256) s += part[(size_t)k * n + o];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[o] = red[0];
}

// grad[i] = sum over tiles t of part[t][i].  A block takes 32 consecutive i
// and splits the tiles into 8 classes (t mod 8): thread (class, i) adds its
// class in tile order, then the class sums are added in class order.
__global__ void __launch_bounds__(256) k_sum_tiles(const float* __restrict__ part, int ntiles, long n,
                                                   float* __restrict__ grad) {
  __shared__ float red[8][33];
  const int j = threadIdx.x & 31, c = threadIdx.x >> 5;
  const long i = (long)blockIdx.x * 32 + j;
  float a = 0.f;
  if (i < n)
    for (int t = c; t < ntiles; t += 8) a += part[(size_t)t * n + i];
  red[c][j] = a;
  __syncthreads();
  if (c == 0 && i < n) {
    float b = 0.f;
    for (int k = 0; k < 8; k++) b += red[k][j];
    grad[i] = b;
  }
}

// Loss of the pixel-shuffled output against the fine target, dL/dy and the
// last layer's bias-gradient partials.  Channel f r^2 + sy r + sx of coarse
// pixel (y, x) is fine cell (r y + sy, r x + sx) of field f.  Block (k, g)
// takes row group g = (f, sy) -- output channels c0 + [0, r), c0 = f r^2 + sy r,
// and fine rows r y + sy of field f -- for the coarse rows y = k, k +
// LOSS_CHUNKS, ...: a thread reads the r output planes at its pixel and r
// consecutive target values (one 16-byte load when r = 4).  dL/dy goes out
// pixel-major BF16 with cs channels per pixel, the operand layout of the
// backward convolutions (which multiply it in BF16); the bias partials use the
// FP32 values.  Loss and bias partials per block are summed in a fixed order
// by k_sum_loss and k_sum_chunks.
constexpr int LOSS_CHUNKS = 64, LOSS_MAXR = 8;
template <bool R4>
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ yv, const float* __restrict__ tgt, int H,
                                              int W, int r, int cs, const float* __restrict__ fw,
                                              __nv_bfloat16* __restrict__ gy, double* __restrict__ lpart,
                                              float* __restrict__ bpart, int cout) {
  __shared__ float red[LOSS_MAXR + 1][256];
  const int g = blockIdx.y, f = g / r, sy = g - f * r, c0 = f * r * r + sy * r;
  const size_t hw = (size_t)H * W, Wf = (size_t)W * r;
  const float inv = 1.f / (float)(hw * r * r), wf = fw[f];
  float l = 0.f, bs[LOSS_MAXR];
#pragma unroll
  for (int j = 0; j < LOSS_MAXR; j++) bs[j] = 0.f;
  for (int y = blockIdx.x; y < H; y += LOSS_CHUNKS) {
    const float* trow = tgt + ((size_t)f * H * r + (size_t)y * r + sy) * Wf;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
      const size_t p = (size_t)y * W + x;
      if constexpr (R4) {
        const float4 t4 = *reinterpret_cast<const float4*>(trow + (size_t)x * 4);
        const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
        float gv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const float d = yv[(size_t)(c0 + j) * hw + p] - tv[j];
          gv[j] = 2.f * wf * d * inv;
          bs[j] += gv[j];
          l += wf * d * d * inv;
        }
        uint2 pk;
        pk.x = pack_bf16(gv[0], gv[1]);
        pk.y = pack_bf16(gv[2], gv[3]);
        *reinterpret_cast<uint2*>(gy + p * cs + c0) = pk;
      } else {
#pragma unroll
        for (int j = 0; j < LOSS_MAXR; j++) {
          if (j < r) {
            const float d = yv[(size_t)(c0 + j) * hw + p] - trow[(size_t)x * r + j];
            const float gv = 2.f * wf * d * inv;
            gy[p * cs + c0 + j] = __float2bfloat16_rn(gv);
            bs[j] += gv;
            l += wf * d * d * inv;
          }
        }
      }
    }
  }
  red[0][threadIdx.x] = l;
#pragma unroll
  for (int j = 0; j < LOSS_MAXR; j++) red[1 + j][threadIdx.x] = bs[j];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int j = 0; j <= r; j++) red[j][threadIdx.x] += red[j][threadIdx.x + h];
    __syncthreads();
  }
  const int k = blockIdx.x;
  if (threadIdx.x == 0) lpart[(size_t)g * LOSS_CHUNKS + k] = (double)red[0][0];
  if (threadIdx.x < r) bpart[(size_t)k * cout + c0 + threadIdx.x] = red[1 + threadIdx.x][0];
}

// Sum of the n block partials in FP64: one block, strided per-thread sums and a
// fixed tree (the same order every call).
__global__ void __launch_bounds__(1024) k_sum_loss(const double* __restrict__ lpart, int n, double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += lpart[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
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

// ---- launch helpers of the tensor-core kernels: padded channel counts are
// template arguments (16, 32, 48 channels; 2, 4, 6 n-tiles of 8 outputs)
typedef void (*ConvFn)(const void*, int, int, int, int, const __nv_bfloat16*, int, const float*, int, int,
                       const __nv_bfloat16*, void*, int, int, int);
typedef void (*WgradFn)(const void*, int, int, int, int, const void*, int, int, float*, int, int);
static int pad16(int c) { return (c + 15) / 16 * 16; }
static ConvFn conv_fn(int cp, int nt) {
#define CF(C, N) if (cp == C && nt == N) return k_conv_mma<C, N>;
  CF(16, 2) CF(16, 4) CF(16, 6) CF(32, 2) CF(32, 4) CF(32, 6) CF(48, 2) CF(48, 4) CF(48, 6)
#undef CF
  return nullptr;
}
static WgradFn wgrad_fn(int op, int cp) {
#define WF(O, C) if (op == O && cp == C) return k_wgrad_mma<O, C>;
  WF(16, 16) WF(16, 32) WF(16, 48) WF(32, 16) WF(32, 32) WF(32, 48) WF(48, 16) WF(48, 32) WF(48, 48)
#undef WF
  return nullptr;
}
static size_t conv_smem(int cp, int nt) { return (size_t)(9 * nt * 8 + 2 * CT_PIX) * (cp + 8) * 2; }
static size_t wgrad_smem(int op, int cp) { return ((size_t)CT_PIX * (cp + 8) + (size_t)CT_H * CT_W * (op + 8)) * 2; }
static int set_smem_attrs() {
  for (int cp = 16; cp <= 48; cp += 16)
    for (int k = 2; k <= 6; k += 2) {
      if (cudaFuncSetAttribute(conv_fn(cp, k), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv_smem(cp, k)) !=
          cudaSuccess)
        return -3;
      const int op = 8 * k;   // 16, 32, 48
      if (cudaFuncSetAttribute(wgrad_fn(op, cp), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)wgrad_smem(op, cp)) != cudaSuccess)
        return -3;
    }
  return 0;
}

struct lc_net {
  int cin, width, depth, cout;
  long max_hw;
  cudaStream_t st;
  std::vector<int> ci, co;
  std::vector<long> woff, boff;
  long np;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* pb = nullptr;
  // act[l]: output of layer l -- pixel-major BF16 rows of pad16(co[l]) channels
  // for the hidden layers, channel-major FP32 for the last one
  std::vector<void*> act;
  __nv_bfloat16* gh[2] = {nullptr, nullptr};   // pixel-major BF16 gradients of hidden outputs
  __nv_bfloat16* ga = nullptr;  // dL/dy, pixel-major BF16 with pad16(cout) channels (padding zero)
  float *part = nullptr, *bpart = nullptr;
  double *lpart = nullptr, *lsum = nullptr;
  float* fw = nullptr;          // loss field weights (device copy)
  long max_layer;
  int max_tiles;
  int nsm = 1;                  // SMs of the device (persistent grids: 2 blocks per SM)
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
  if (cin > 48 || width > 48 || cout > 48) return -1;   // tensor-core kernels: at most 48 channels
  if ((long)cout * max_hw >= (1L << 31)) return -1;       // 32-bit element indices of the loss
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
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n->nsm < 1)
      n->nsm = 1;
    if (set_smem_attrs()) { delete n; return -3; }
  }
  // weight-gradient partials: one per block of the persistent grid
  n->max_tiles = 2 * n->nsm;
  n->p = (float*)dmalloc(n, n->np * 4); n->g = (float*)dmalloc(n, n->np * 4);
  n->m = (float*)dmalloc(n, n->np * 4); n->v = (float*)dmalloc(n, n->np * 4);
  n->pb = (__nv_bfloat16*)dmalloc(n, n->np * 2);
  for (int l = 0; l < depth; l++)
    n->act.push_back(dmalloc(n, l < depth - 1 ? (size_t)pad16(n->co[l]) * max_hw * 2 : (size_t)n->co[l] * max_hw * 4));
  n->ga = (__nv_bfloat16*)dmalloc(n, (size_t)pad16(cout) * max_hw * 2);
  for (int k = 0; k < 2; k++) n->gh[k] = (__nv_bfloat16*)dmalloc(n, (size_t)pad16(width) * max_hw * 2);
  n->part = (float*)dmalloc(n, (size_t)n->max_tiles * n->max_layer * 4);
  n->lpart = (double*)dmalloc(n, (size_t)LOSS_CHUNKS * cout * 8);
  n->bpart = (float*)dmalloc(n, (size_t)std::max(BG_CHUNKS, LOSS_CHUNKS) * maxc * 4);
  n->lsum = (double*)dmalloc(n, 8);
  n->fw = (float*)dmalloc(n, 8 * sizeof(float));
  bool ok = n->p && n->g && n->m && n->v && n->pb && n->ga && n->gh[0] && n->gh[1] && n->part && n->bpart &&
            n->lpart && n->lsum && n->fw;
  for (auto a : n->act) ok = ok && a;
  if (!ok) { lc_destroy(n); return -2; }
  if (cudaMemset(n->ga, 0, (size_t)pad16(cout) * max_hw * 2) != cudaSuccess) { lc_destroy(n); return -3; }
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

// 3x3 convolution of `in` (cin planes) into `out` (cout planes) on the tensor
// cores with the BF16 weights w (transpose: see k_conv_mma).
static void conv(lc_net* n, const void* in, int in_nhwc, int cin, int H, int W, const __nv_bfloat16* w,
                 int transpose, const float* bias, int cout, int relu, const __nv_bfloat16* mask, void* out,
                 int out_nhwc) {
  const int cp = pad16(cin), nt = (cout + 15) / 16 * 2;
  const int ntx = (W + CT_W - 1) / CT_W, ntiles = ntx * ((H + CT_H - 1) / CT_H);
  const int nb = std::min(ntiles, 2 * n->nsm);
  conv_fn(cp, nt)<<<nb, 256, conv_smem(cp, nt), n->st>>>(in, in_nhwc, cin, H, W, w, transpose, bias, cout, relu,
                                                          mask, out, out_nhwc, ntx, ntiles);
}

// Layer l forward: its input is x (channel-major FP32) for l = 0, else the
// previous hidden output; hidden outputs are pixel-major BF16, the last
// layer's channel-major FP32 (out).
static void conv_fwd(lc_net* n, int l, const float* x, int H, int W, void* out) {
  const bool last = l == n->depth - 1;
  conv(n, l == 0 ? (const void*)x : n->act[l - 1], l == 0 ? 0 : 1, n->ci[l], H, W, n->pb + n->woff[l], 0,
       n->p + n->boff[l], n->co[l], last ? 0 : 1, nullptr, out, last ? 0 : 1);
}

int lc_forward(lc_net* n, const float* x_dev, int H, int W, float* y_dev) {
  if (!n || !x_dev || !y_dev || H <= 0 || W <= 0 || (long)H * W > n->max_hw) return -1;
  for (int l = 0; l < n->depth; l++) conv_fwd(n, l, x_dev, H, W, l == n->depth - 1 ? (void*)y_dev : n->act[l]);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lc_train_step(lc_net* n, const float* x_dev, const float* target_dev, int H, int W, int r, int nout,
                  const float* field_w, float lr, double* loss, float* grad_host) {
  if (!n || !x_dev || !target_dev || !field_w || H <= 0 || W <= 0 || r <= 0 || nout <= 0) return -1;
  if ((long)H * W > n->max_hw || nout * r * r != n->cout || nout > 8 || lr < 0) return -1;
  // forward, keeping every layer's output
  for (int l = 0; l < n->depth; l++) conv_fwd(n, l, x_dev, H, W, n->act[l]);
  // loss, dL/dy and the last layer's bias-gradient partials
  const int ng = n->cout / r;                    // row groups (field, sub-row)
  if (cudaMemcpyAsync(n->fw, field_w, nout * sizeof(float), cudaMemcpyHostToDevice, n->st) != cudaSuccess) return -3;
  const int cs = pad16(n->cout);
  if (r == 4 && ((uintptr_t)target_dev & 15) == 0)
    k_loss<true><<<dim3(LOSS_CHUNKS, ng), 256, 0, n->st>>>(static_cast<const float*>(n->act[n->depth - 1]),
                                                           target_dev, H, W, r, cs, n->fw, n->ga, n->lpart,
                                                           n->bpart, n->cout);
  else
    k_loss<false><<<dim3(LOSS_CHUNKS, ng), 256, 0, n->st>>>(static_cast<const float*>(n->act[n->depth - 1]),
                                                            target_dev, H, W, r, cs, n->fw, n->ga, n->lpart,
                                                            n->bpart, n->cout);
  k_sum_loss<<<1, 1024, 0, n->st>>>(n->lpart, ng * LOSS_CHUNKS, n->lsum);
  // backward: g is dL/d(pre-activation) of layer l, pixel-major BF16
  const int ntx = (W + CT_W - 1) / CT_W, ntiles = ntx * ((H + CT_H - 1) / CT_H);
  const int nbw = std::min(ntiles, n->max_tiles);
  // g: dL/dy for the last layer, then the gradients of the hidden outputs,
  // alternating between gh[0] and gh[1]
  const __nv_bfloat16* g = n->ga;
  int gk = 0;
  for (int l = n->depth - 1; l >= 0; l--) {
    const void* lin = l == 0 ? (const void*)x_dev : n->act[l - 1];
    const int a = n->ci[l], b = n->co[l];
    const long nw = (long)a * b * 9;
    const int op = pad16(b), cp = pad16(a);
    wgrad_fn(op, cp)<<<nbw, 288, wgrad_smem(op, cp), n->st>>>(lin, l == 0 ? 0 : 1, a, H, W, g, 1, b, n->part,
                                                               ntx, ntiles);
    k_sum_tiles<<<(unsigned)((nw + 31) / 32), 256, 0, n->st>>>(n->part, nbw, nw, n->g + n->woff[l]);
    if (l == n->depth - 1) {
      k_sum_chunks<<<b, 256, 0, n->st>>>(n->bpart, LOSS_CHUNKS, b, n->g + n->boff[l]);
    } else {
      k_bias_grad<<<BG_CHUNKS, 256 / op * op, 0, n->st>>>(g, op, (long)H * W, b, n->bpart);
      k_sum_chunks<<<b, 256, 0, n->st>>>(n->bpart, BG_CHUNKS, b, n->g + n->boff[l]);
    }
    if (l > 0) {
      // dL/d(out of layer l-1) = transposed, flipped convolution of g, times ReLU'(out of layer l-1)
      conv(n, g, 1, b, H, W, n->pb + n->woff[l], 1, nullptr, a, 0,
           static_cast<const __nv_bfloat16*>(n->act[l - 1]), n->gh[gk], 1);
      g = n->gh[gk];
      gk ^= 1;
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
