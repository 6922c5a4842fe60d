// lc_kernels.cu -- learned coarse-to-fine corrector: 3x3 convolution network
// with hand-written forward, backward (data and weight gradients), loss and Adam
// kernels, plus the data kernels that turn solver states into inputs/targets.
//
// Convolutions run on the tensor cores (mma.sync, BF16 operands: the BF16
// weights and the activations or gradients rounded to BF16 as they are staged;
// FP32 accumulation; FP32 activations, biases, losses and master weights).  The
// weight gradients are summed per block of a fixed persistent grid, then over
// blocks in a fixed order, so training is run-to-run reproducible.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/lc.h"

namespace {

// ---------------------------------------------------------------------------
// Layouts.  The network input x and its output y are FP32 channel-major planes
// [c][y][x] (the data kernels' layout).  Everything in between -- hidden
// activations and the gradients flowing back through them -- is stored in BF16,
// channel-blocked: [c / 8][y][x][c % 8] with CS = channels rounded up to 16
// (the padding stays zero).  The values the tensor cores multiply are BF16
// anyway, so this changes no result and halves the bytes; each block of 8
// channels is a dense [y][x] image of 16-byte pixels, which is both what the
// tensor-core descriptors read and what a TMA box copies in long contiguous
// rows.
//
// Weight gradients (k_wgrad_mma) run on the warp-level tensor-core
// instructions, mma.sync m16n8k16 with BF16 operands and FP32 accumulation: a
// block stages a tile of the layer input and of the gradient in shared memory
// as [pixel][channel] rows of CS + 8 BF16 (the 8 extra keep the 16-byte
// ldmatrix rows of consecutive pixels on different banks); channel-blocked
// inputs arrive by 16-byte cp.async (zero-filled outside the image), channel-major
// FP32 inputs are read, rounded and stored by the threads.  The convolutions
// themselves (forward and input gradient) run on tcgen05 (k_conv_tc, below).
constexpr int CT_H = 8;              // weight-gradient tile rows
constexpr int CT_W = 32;             // weight-gradient tile columns
constexpr int CT_PIX = (CT_H + 2) * (CT_W + 2);   // staged input pixels (tile + halo)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

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
// Channel-blocked BF16 source (blk, CP channels): 16-byte cp.async
// copies, committed as one group by the caller.  Channel-major FP32 source
// (planes [0, c)): loads go out in batches of SB element pairs per thread
// before any of them is stored, so a thread waits for one memory latency per
// batch, not per pair.
template <int CP, int PS, int ROWS, int COLS, int SB = 8>
__device__ __forceinline__ void stage_tile(const void* __restrict__ srcv, int blk, int c, int H, int W, int y0,
                                           int x0, __nv_bfloat16* dst) {
  if (blk) {
    const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(srcv);
    constexpr int CH = CP / 8, N = ROWS * COLS * CH;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
      const int pix = t % (ROWS * COLS), ch = t / (ROWS * COLS);   // consecutive threads: consecutive pixels
      const int yy = pix / COLS, xx = pix - yy * COLS;
      const int gy = y0 + yy, gx = x0 + xx;
      const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
      const __nv_bfloat16* s = in ? src + ((size_t)ch * H * W + (size_t)gy * W + gx) * 8 : src;
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

// ---------------------------------------------------------------------------
// 3x3 convolutions on the fifth-generation tensor cores (tcgen05): implicit
// GEMM with M = 128 pixels of one tile row, N = the output channels
// (16, 32 or 48, padding included), K = 16 input channels of one tap per
// instruction; BF16 operands read by the tensor cores from shared memory
// through matrix descriptors, FP32 accumulators in tensor memory (TMEM).
//
// Shared-memory operand layout (the "no swizzle, K-major" canonical layout of
// the tcgen05 descriptors: 8 x 16-byte core matrices; LBO = byte distance
// between the two 8-channel halves of an instruction's K = 16, SBO = byte
// distance between groups of 8 rows):
//   A (input tile, TC_R + 2 rows x TC_SW = 128 columns, starting one row and
//     one column before the tile's TC_W = 126 output columns):
//     [channel / 8][row][column][channel % 8], planes TC_BOX bytes apart, so
//     the 128 pixels x 16 channels of staged row t shifted by kx start at pixel
//     t * TC_SW + kx of planes 2j, 2j + 1 (LBO = TC_BOX, SBO = 128): a tap
//     shift is a shift of the descriptor's start address.  Output pixels 126
//     and 127 of an instruction read past the row and are discarded.  The tile
//     is one TMA box of the channel-blocked input seen as 8-byte elements
//     (256 elements = 128 pixels x TC_R + 2 rows x CP / 8 blocks, zero-filled
//     outside the image): each box row is 2 KB contiguous in global memory.
//   B (weights): [kx][channel / 8][n][channel % 8] with n = (2 - ky) NO + o:
//     the three row taps of one column tap stacked along N (LBO = 3 NO * 16,
//     SBO = 128).
// One instruction multiplies staged row t (shifted by kx) by the stacked
// weights of the row taps ky that map it to output rows of the tile (output
// row t - ky, 0 <= t - ky < TC_R): N = NO, 2 NO or 3 NO columns, written to the
// TMEM columns of output rows t - ky_hi .. t - ky_lo (lane p = output pixel p,
// column r * NO + o = channel o of output row r), which are zero before the
// tile.  Per tile that is (TC_R + 2) x 3 x CP / 16 instructions of up to
// 3 NO columns instead of TC_R x 9 x CP / 16 of NO columns: each staged row
// shift is read from shared memory once for its three row taps.
//
// Pipeline (one persistent block per SM, warp-specialised): warp TC_TMA_WARP
// loads input tiles by TMA into a ring of tc_stages(CP) shared-memory stages
// (full / empty mbarriers); warp TC_MMA_WARP issues each tile's instructions
// into one of two
// TMEM accumulator buffers and commits them to the stage's empty barrier and
// the buffer's full barrier; the write-back warps (warp w: lanes 32 (w % 4) ..
// 32 (w % 4) + 31, tile row w / 4) read their part of a full buffer back
// (tcgen05.ld 32x32b), write bias + ReLU (+ mask) pixel by pixel --
// channel-blocked BF16 (16-byte stores) or channel-major FP32 planes, both
// coalesced along x -- clear the buffer and release it.  Loads, tensor-core
// work and write-back of different tiles overlap.
constexpr int TC_R = 4;                         // output rows per tile
constexpr int TC_M = 128;                       // pixels per instruction (M)
constexpr int TC_SW = TC_M;                     // staged columns: one TMA box row of 256 8-byte elements
constexpr int TC_W = TC_SW - 2;                 // output columns per tile
constexpr int TC_SPIX = (TC_R + 2) * TC_SW;     // staged pixels
constexpr int TC_BOX = TC_SPIX * 16;            // bytes of one 8-channel plane of the staged tile
constexpr int TC_EW = 4 * TC_R;                 // write-back warps: one per TMEM lane quarter and tile row
constexpr int TC_TMA_WARP = TC_EW, TC_MMA_WARP = TC_EW + 1;
constexpr int TC_THREADS = 32 * (TC_EW + 2);

__host__ __device__ constexpr int tc_stages(int cp) { return cp == 48 ? 2 : 3; }
__host__ __device__ constexpr int tc_bufcols(int no) { return TC_R * no; }   // TMEM columns of one buffer
// bytes of one stage: the planes plus 128 (the two pixels the last row's
// shifted instructions read past the end)
__host__ __device__ constexpr int tc_stage_bytes(int cp) { return cp / 8 * TC_BOX + 128; }
__host__ __device__ constexpr int tc_cols(int no) {   // TMEM columns to allocate: a power of 2 >= 2 buffers
  return 2 * TC_R * no <= 32 ? 32 : 2 * TC_R * no <= 64 ? 64 : 2 * TC_R * no <= 128 ? 128
         : 2 * TC_R * no <= 256 ? 256 : 512;
}
__host__ __device__ constexpr int tc_smem_used(int cp, int no) {
  // alignment slack, stages, B, bias, 2 S + 4 mbarriers, TMEM address + abort flag
  return 128 + tc_stages(cp) * tc_stage_bytes(cp) + 9 * cp * no * 2 + 256 + (2 * tc_stages(cp) + 4) * 8 + 16;
}

static_assert(TC_BOX % 128 == 0, "stages stay 128-byte aligned");

// Shared-memory matrix descriptor: start address, LBO and SBO in 16-byte units,
// descriptor version 1 (bits 46-47), no swizzle, base offset 0.
__device__ __forceinline__ unsigned long long tc_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 (bits 17-22),
// M >> 4 (bits 24-28).
__device__ __forceinline__ unsigned tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       int accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
// Wait until the mbarrier has completed the phase of the given parity; gives up
// after about two seconds, or as soon as *abort is set (returns false).
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity, const volatile int* abort) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort || global_ns() - t0 > 2000000000ull) return false;
  }
}
__device__ __forceinline__ void mbar_arrive(unsigned addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(addr) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(addr), "r"(bytes) : "memory");
}
// TMA: box at coordinates (c0, c1, c2) of a 3-D tensor map into shared memory,
// completion counted on the mbarrier in bytes.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}
// The NO consecutive FP32 columns (16, 32 or 48) of this thread's TMEM lane,
// waited for in the same statement (the registers are only valid after
// tcgen05.wait::ld).
#define TC_R16(i) "=r"(r[i]), "=r"(r[i + 1]), "=r"(r[i + 2]), "=r"(r[i + 3]), "=r"(r[i + 4]), "=r"(r[i + 5]), \
                  "=r"(r[i + 6]), "=r"(r[i + 7]), "=r"(r[i + 8]), "=r"(r[i + 9]), "=r"(r[i + 10]),          \
                  "=r"(r[i + 11]), "=r"(r[i + 12]), "=r"(r[i + 13]), "=r"(r[i + 14]), "=r"(r[i + 15])
template <int NO> __device__ __forceinline__ void tmem_ld(unsigned taddr, float* v) {
  unsigned r[NO];
  if constexpr (NO == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : TC_R16(0)
        : "r"(taddr)
        : "memory");
  } else if constexpr (NO == 32) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : TC_R16(0), TC_R16(16)
        : "r"(taddr)
        : "memory");
  } else {
    static_assert(NO == 48, "16, 32 or 48 output channels");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%48];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,"
        "%47}, [%49];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : TC_R16(0), TC_R16(16), TC_R16(32)
        : "r"(taddr), "r"(taddr + 32)
        : "memory");
  }
#pragma unroll
  for (int i = 0; i < NO; i++) v[i] = __uint_as_float(r[i]);
}
#undef TC_R16
// Zero 32 (or 16) consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_zero32(unsigned taddr) {
  const unsigned z = 0;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
      "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(taddr),
      "r"(z)
      : "memory");
}
__device__ __forceinline__ void tmem_zero16(unsigned taddr) {
  const unsigned z = 0;
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(
                   taddr),
               "r"(z)
               : "memory");
}
// Zero NO (16, 32 or 48) consecutive TMEM columns of this warp's lanes.
template <int NO> __device__ __forceinline__ void tmem_zero(unsigned taddr) {
  if constexpr (NO >= 32) tmem_zero32(taddr);
  if constexpr (NO != 32) tmem_zero16(taddr + (NO >= 32 ? 32 : 0));
}

// Convolution with padding 1: out[o][y][x] =
// bias[o] + sum_c sum_k B(o, c, k) in[c][y + ky - 1][x + kx - 1], optional
// ReLU, optional mask (out = 0 where mask <= 0).  transpose = 0: B(o, c, k) =
// w[o][c][k]; transpose = 1: B(o, c, k) = w[c][o][8 - k] (the transposed,
// flipped kernel mapping dL/d(out) of that layer to dL/d(in)).  in: the
// channel-blocked BF16 tensor (CP channels) behind the tensor map; out:
// channel-blocked BF16 with NO channels (out_blk) or channel-major FP32
// planes (cout); mask: channel-blocked BF16 with NO channels.  Persistent blocks (one per SM) take tiles of TC_R x TC_W
// output pixels in the pipeline described above.  Every wait is bounded
// (about two seconds); one that runs out sets *err and a shared abort flag
// that ends the other roles' waits, and the block releases its TMEM and ends.
template <int CP, int NO>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap map, int cin, int H, int W, const __nv_bfloat16* __restrict__ w,
              int transpose, const float* __restrict__ bias, int cout, int relu,
              const __nv_bfloat16* __restrict__ mask, void* __restrict__ out, int out_blk, int ntx, int ntiles,
              int* __restrict__ err) {
  constexpr int C8 = CP / 8, S = tc_stages(CP);
  constexpr int A_STAGE = tc_stage_bytes(CP), B_BYTES = 9 * CP * NO * 2, TB = tc_bufcols(NO);
  constexpr unsigned NCOL = tc_cols(NO);
  extern __shared__ __align__(16) unsigned char tc_raw[];
  const unsigned raw = smem_u32(tc_raw), base = (raw + 127) & ~127u;
  unsigned char* g0 = tc_raw + (base - raw);                 // 128-byte aligned
  __nv_bfloat16* sB = reinterpret_cast<__nv_bfloat16*>(g0 + S * A_STAGE);
  float* sBias = reinterpret_cast<float*>(g0 + S * A_STAGE + B_BYTES);
  const unsigned bars = base + S * A_STAGE + B_BYTES + 256;  // full[S], empty[S], tfull[2], tempty[2]
  unsigned* tslot = reinterpret_cast<unsigned*>(g0 + S * A_STAGE + B_BYTES + 256 + (2 * S + 4) * 8);
  volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);
  auto full = [&](int st) { return bars + 8 * st; };
  auto empty = [&](int st) { return bars + 8 * (S + st); };
  auto tfull = [&](int b) { return bars + 8 * (2 * S + b); };
  auto tempty = [&](int b) { return bars + 8 * (2 * S + 2 + b); };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights once per block: sB[kx][c / 8][(2 - ky) NO + o][c % 8] = B(o, c, 3 ky + kx),
  // zero-padded
  for (int e = tid; e < 9 * CP * NO; e += TC_THREADS) {
    const int c = e % CP, o = (e / CP) % NO, k = e / (CP * NO);
    const int ky = k / 3, kx = k - 3 * ky;
    float v = 0.f;
    if (o < cout && c < cin)
      v = (float)(transpose ? w[((size_t)c * cout + o) * 9 + (8 - k)] : w[((size_t)o * cin + c) * 9 + k]);
    sB[((size_t)(kx * C8 + c / 8) * (3 * NO) + (2 - ky) * NO + o) * 8 + (c & 7)] = __float2bfloat16_rn(v);
  }
  for (int o = tid; o < NO; o += TC_THREADS) sBias[o] = (bias && o < cout) ? bias[o] : 0.f;
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // the weights, for the tensor cores
  if (tid == 0) {
    for (int st = 0; st < S; st++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(full(st)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(empty(st)) : "memory");
    }
    for (int b = 0; b < 2; b++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tfull(b)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tempty(b)), "r"(TC_EW) : "memory");
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tslot;
  if (warp < 4) {   // both accumulator buffers start at zero (each lane quarter's warp clears its lanes)
    const unsigned tl = tmem + ((unsigned)(32 * warp) << 16);
#pragma unroll
    for (int c = 0; c < 2 * TB; c += 32) tmem_zero32(tl + c);
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  bool failed = false;
  if (warp == TC_TMA_WARP) {
    // ---- TMA producer
    if (lane == 0) {
      int i = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, i++) {
        const int st = i % S;
        if (!mbar_wait(empty(st), ((i / S) & 1) ^ 1, abort)) { failed = true; break; }
        const int ty0 = (tile / ntx) * TC_R, tx0 = (tile % ntx) * TC_W;
        mbar_expect_tx(full(st), C8 * TC_BOX);
        tma_load_3d(base + st * A_STAGE, &map, 2 * (tx0 - 1), ty0 - 1, 0, full(st));
      }
    }
  } else if (warp == TC_MMA_WARP) {
    // ---- tensor-core issue
    if (lane == 0) {
      int i = 0;
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, i++) {
        const int st = i % S, b = i & 1;
        if (!mbar_wait(full(st), (i / S) & 1, abort) || !mbar_wait(tempty(b), ((i >> 1) & 1) ^ 1, abort)) {
          failed = true;
          break;
        }
        tc_fence_after();
        const unsigned aBase = base + st * A_STAGE, bBase = smem_u32(sB), dBase = tmem + b * TB;
#pragma unroll 1
        for (int t = 0; t < TC_R + 2; t++) {
          // row taps that map staged row t to an output row of the tile
          const int ky_lo = t - (TC_R - 1) > 0 ? t - (TC_R - 1) : 0, ky_hi = t < 2 ? t : 2;
          const unsigned id = tc_idesc((ky_hi - ky_lo + 1) * NO);
          const unsigned d = dBase + (t - ky_hi) * NO;
          const unsigned boff = (2 - ky_hi) * NO / 8 * 128;
#pragma unroll
          for (int kx = 0; kx < 3; kx++)
#pragma unroll
            for (int j = 0; j < CP / 16; j++) {
              const unsigned long long ad =
                  tc_desc(aBase + 2 * j * TC_BOX + (t * TC_SW + kx) * 16, TC_BOX, 128);
              const unsigned long long bd =
                  tc_desc(bBase + (kx * C8 + 2 * j) * (3 * NO) * 16 + boff, 3 * NO * 16, 128);
              tc_mma(d, ad, bd, id, 1);
            }
        }
        // the stage is free and the buffer full once these instructions complete
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         empty(st))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         tfull(b))
                     : "memory");
      }
    }
  } else {
    // ---- write-back: warp w owns TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 =
    // output pixels of tile row w / 4
    const int q = warp & 3, r = warp >> 2;
    const unsigned tl = tmem + ((unsigned)(32 * q) << 16);
    const size_t hw = (size_t)H * W;
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, i++) {
      const int b = i & 1;
      const int ok = __shfl_sync(0xffffffffu, lane == 0 ? (int)mbar_wait(tfull(b), (i >> 1) & 1, abort) : 0, 0);
      if (!ok) { failed = true; break; }
      tc_fence_after();
      const int ty0 = (tile / ntx) * TC_R, tx0 = (tile % ntx) * TC_W;
      const int x = tx0 + 32 * q + lane;
      {
        float v[NO];
        tmem_ld<NO>(tl + b * TB + r * NO, v);
        const int y = ty0 + r;
        if (y < H && x < W && 32 * q + lane < TC_W) {
        const size_t pix = (size_t)y * W + x;
#pragma unroll
        for (int o = 0; o < NO; o++) {
          v[o] += sBias[o];
          if (relu) v[o] = v[o] > 0.f ? v[o] : 0.f;
        }
        if (mask) {
          const uint4* mk = reinterpret_cast<const uint4*>(mask) + pix;
#pragma unroll
          for (int c = 0; c < NO / 8; c++) {
            const uint4 m4 = __ldg(mk + c * hw);
            const unsigned mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
              const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mw[e]);
              if (!(__low2float(m2) > 0.f)) v[8 * c + 2 * e] = 0.f;
              if (!(__high2float(m2) > 0.f)) v[8 * c + 2 * e + 1] = 0.f;
            }
          }
        }
        if (out_blk) {
          uint4* op = reinterpret_cast<uint4*>(out) + pix;
#pragma unroll
          for (int c = 0; c < NO / 8; c++) {
            uint4 u;
            u.x = pack_bf16(v[8 * c], v[8 * c + 1]);
            u.y = pack_bf16(v[8 * c + 2], v[8 * c + 3]);
            u.z = pack_bf16(v[8 * c + 4], v[8 * c + 5]);
            u.w = pack_bf16(v[8 * c + 6], v[8 * c + 7]);
            op[c * hw] = u;
          }
        } else {
          float* of = static_cast<float*>(out);
#pragma unroll
          for (int o = 0; o < NO; o++)
            if (o < cout) of[(size_t)o * hw + pix] = v[o];
        }
        }
      }
      // clear this warp's part of the buffer for its next tile and hand it back
      tmem_zero<NO>(tl + b * TB + r * NO);
      asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(b));
    }
  }
  if (failed) {
    *abort = 1;
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL) : "memory");
  }
}

// FP32 channel-major planes (cin) -> channel-blocked BF16 with cp channels
// (zero-padded): the network input in the layout the convolutions load.
__global__ void k_to_blk(const float* __restrict__ x, int cin, long hw, int cp, __nv_bfloat16* __restrict__ y) {
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= hw) return;
  for (int c0 = 0; c0 < cp; c0 += 8) {
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = c0 + i < cin ? x[(size_t)(c0 + i) * hw + p] : 0.f;
    uint4 u;
    u.x = pack_bf16(v[0], v[1]);
    u.y = pack_bf16(v[2], v[3]);
    u.z = pack_bf16(v[4], v[5]);
    u.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(y + ((size_t)(c0 / 8) * hw + p) * 8) = u;
  }
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
__global__ void __launch_bounds__(288, 2) k_wgrad_mma(const void* __restrict__ in, int in_blk, int cin, int H,
                                                      int W, const void* __restrict__ g, int g_blk, int cout,
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
    stage_tile<CP, PSI, CT_H + 2, CT_W + 2, 4>(in, in_blk, cin, H, W, ty0 - 1, tx0 - 1, sI);
    stage_tile<OP, PSG, CT_H, CT_W, 4>(g, g_blk, cout, H, W, ty0, tx0, sG);
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

// Bias gradient partials of a hidden layer: part[chunk][o] = sum of g[o][p]
// over the pixels of chunk blockIdx.x (gridDim.x contiguous ranges), in FP32, in
// a fixed order; k_sum_chunks adds the chunks.  g: channel-blocked BF16 with cs
// channels; thread t reads the 16-byte pixel (t % 32 + 32 i) of channel block
// t / 32 (a warp reads 512 contiguous bytes), sums its 8 channels separately,
// and the 32 lanes of each block are then summed in lane order.
constexpr int BG_CHUNKS = 1024;
__global__ void __launch_bounds__(192) k_bias_grad(const __nv_bfloat16* __restrict__ gb, int cs, long hw, int cout,
                                                   float* __restrict__ part) {
  __shared__ float red[6][32][9];
  const long p0 = hw * blockIdx.x / gridDim.x, p1 = hw * (blockIdx.x + 1) / gridDim.x;
  const int lane = threadIdx.x & 31, cb = threadIdx.x >> 5;   // channel block of this warp
  float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (cb < cs / 8) {
    const uint4* src = reinterpret_cast<const uint4*>(gb) + (size_t)cb * hw;
    for (long p = p0 + lane; p < p1; p += 32) {
      const uint4 u = src[p];
      const unsigned w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const __nv_bfloat162 b2 = *reinterpret_cast<const __nv_bfloat162*>(&w4[q]);
        s[2 * q] += __low2float(b2);
        s[2 * q + 1] += __high2float(b2);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; q++) red[cb][lane][q] = s[q];
  }
  __syncthreads();
  if (threadIdx.x < cout) {
    const int o = threadIdx.x;
    float t = 0.f;
    for (int k = 0; k < 32; k++) t += red[o / 8][k][o % 8];
    part[(size_t)blockIdx.x * cout + o] = t;
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
// channel-blocked BF16 (cs channels), the operand layout of the backward
// convolutions (which multiply it in BF16); the bias partials use the FP32
// values.  Loss and bias partials per block are summed in a fixed order
// by k_sum_loss and k_sum_chunks.
constexpr int LOSS_CHUNKS = 64, LOSS_MAXR = 8;
template <bool R4>
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ yv, const float* __restrict__ tgt, int H,
                                              int W, int r, const float* __restrict__ fw,
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
        *reinterpret_cast<uint2*>(gy + ((size_t)(c0 / 8) * hw + p) * 8 + (c0 & 7)) = pk;
      } else {
#pragma unroll
        for (int j = 0; j < LOSS_MAXR; j++) {
          if (j < r) {
            const float d = yv[(size_t)(c0 + j) * hw + p] - trow[(size_t)x * r + j];
            const float gv = 2.f * wf * d * inv;
            gy[((size_t)((c0 + j) / 8) * hw + p) * 8 + ((c0 + j) & 7)] = __float2bfloat16_rn(gv);
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

// The learned form's fallback flag (the paper's refinement flag, a surface jump
// between neighbouring cells, Sec. 6.3) on the coarse state: cell c is flagged
// when a face neighbour n and c are both deeper than hmin (eta - b > hmin) and
// |eta_c - eta_n| > thr.  Tiles: `tile` cells from the low corner, a one-cell
// remainder joined to the tile before it.  A tile is selected when a flagged
// cell lies within Chebyshev distance `buffer` of it and none of its own cells
// is shallower than hmin.  One block per tile; the FP64 comparisons are those
// of the definition.
__device__ __forceinline__ void tile_span(int k, int n, int nt, int tile, int& a0, int& a1) {
  a0 = k * tile;
  a1 = k == nt - 1 ? n : a0 + tile;
}
__global__ void k_fallback_tiles(const double* __restrict__ eta, const double* __restrict__ b, int H, int W, double thr,
                                 double hmin, int tile, int buffer, int ntx, int nty, unsigned char* __restrict__ sel) {
  int x0, x1, y0, y1;
  tile_span(blockIdx.x, W, ntx, tile, x0, x1);
  tile_span(blockIdx.y, H, nty, tile, y0, y1);
  const int ex0 = max(0, x0 - buffer), ex1 = min(W, x1 + buffer), ey0 = max(0, y0 - buffer), ey1 = min(H, y1 + buffer);
  const int ew = ex1 - ex0, ne = ew * (ey1 - ey0);
  int any = 0;
  for (int e = threadIdx.x; e < ne && !any; e += blockDim.x) {
    const int y = ey0 + e / ew, x = ex0 + e % ew;
    const size_t c = (size_t)y * W + x;
    const double ec = eta[c];
    if (!(ec - b[c] > hmin)) continue;
    const int nx[4] = {x - 1, x + 1, x, x}, ny[4] = {y, y, y - 1, y + 1};
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (nx[q] < 0 || nx[q] >= W || ny[q] < 0 || ny[q] >= H) continue;
      const size_t m = (size_t)ny[q] * W + nx[q];
      const double em = eta[m];
      if (em - b[m] > hmin && fabs(ec - em) > thr) any = 1;
    }
  }
  const int tw = x1 - x0, nt = tw * (y1 - y0);
  int shallow = 0;
  for (int e = threadIdx.x; e < nt; e += blockDim.x) {
    const size_t c = (size_t)(y0 + e / tw) * W + x0 + e % tw;
    if (!(eta[c] - b[c] > hmin)) shallow = 1;
  }
  any = __syncthreads_or(any);
  shallow = __syncthreads_or(shallow);
  if (threadIdx.x == 0) sel[(size_t)blockIdx.y * ntx + blockIdx.x] = any && !shallow;
}

}  // namespace

// ---- launch helpers of the tensor-core kernels: padded channel counts are
// template arguments (16, 32, 48 channels; 2, 4, 6 n-tiles of 8 outputs)
typedef void (*WgradFn)(const void*, int, int, int, int, const void*, int, int, float*, int, int);
static int pad16(int c) { return (c + 15) / 16 * 16; }
static WgradFn wgrad_fn(int op, int cp) {
#define WF(O, C) if (op == O && cp == C) return k_wgrad_mma<O, C>;
  WF(16, 16) WF(16, 32) WF(16, 48) WF(32, 16) WF(32, 32) WF(32, 48) WF(48, 16) WF(48, 32) WF(48, 48)
#undef WF
  return nullptr;
}
static size_t wgrad_smem(int op, int cp) { return ((size_t)CT_PIX * (cp + 8) + (size_t)CT_H * CT_W * (op + 8)) * 2; }
typedef void (*TcFn)(const CUtensorMap, int, int, int, const __nv_bfloat16*, int, const float*, int, int,
                     const __nv_bfloat16*, void*, int, int, int, int*);
static PFN_cuTensorMapEncodeTiled_v12000 tma_encode = nullptr;   // driver entry point
static TcFn tc_fn(int cp, int no) {
#define TF(C, N) if (cp == C && no == N) return k_conv_tc<C, N>;
  TF(16, 16) TF(16, 32) TF(16, 48) TF(32, 16) TF(32, 32) TF(32, 48) TF(48, 16) TF(48, 32) TF(48, 48)
#undef TF
  return nullptr;
}
// Launch configuration of each tensor-core convolution: dynamic shared memory
// (padded where needed so that the blocks resident on one SM never ask for more
// than the 512 TMEM columns between them) and resident blocks per SM.
struct TcCfg {
  int smem = 0, per_sm = 0;
};
static TcCfg tc_cfg[3][3];
static int set_smem_attrs() {
  for (int cp = 16; cp <= 48; cp += 16)
    for (int op = 16; op <= 48; op += 16)
      if (cudaFuncSetAttribute(wgrad_fn(op, cp), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)wgrad_smem(op, cp)) != cudaSuccess)
        return -3;
  // resident blocks of a tensor-core convolution = what the SM's shared memory
  // holds; the request is padded until that is at most 512 / (its TMEM columns)
  if (!tma_encode) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", reinterpret_cast<void**>(&tma_encode), 12000,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !tma_encode) {
      tma_encode = nullptr;
      return -3;
    }
  }
  int dev = 0, smax = 0, ssm = 0, sres = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&ssm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sres, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
    return -3;
  for (int cp = 16; cp <= 48; cp += 16)
    for (int no = 16; no <= 48; no += 16) {
      TcFn f = tc_fn(cp, no);
      const int allowed = 512 / tc_cols(no);
      int sm = tc_smem_used(cp, no);
      while (ssm / (sm + sres) > allowed) sm += 1024;
      if (sm > smax) return -3;
      if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return -3;
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return -3;
      const int regs = (fa.numRegs + 7) / 8 * 8;   // per-thread allocation granularity
      int occ = std::min(ssm / (sm + sres), allowed);
      occ = std::min(occ, 65536 / (regs * TC_THREADS));
      if (occ < 1) return -3;
      tc_cfg[cp / 16 - 1][no / 16 - 1] = {sm, occ};
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
  // act[l]: output of layer l -- channel-blocked BF16 with pad16(co[l]) channels
  // for the hidden layers, channel-major FP32 for the last one
  std::vector<void*> act;
  __nv_bfloat16* gh[2] = {nullptr, nullptr};   // channel-blocked BF16 gradients of hidden outputs
  __nv_bfloat16* ga = nullptr;  // dL/dy, channel-blocked BF16 with pad16(cout) channels (padding zero)
  __nv_bfloat16* x16 = nullptr; // the network input, channel-blocked BF16 with pad16(cin) channels
  float *part = nullptr, *bpart = nullptr;
  double *lpart = nullptr, *lsum = nullptr;
  float* fw = nullptr;          // loss field weights (device copy)
  int* err = nullptr;           // set by a kernel whose bounded wait ran out
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
  n->x16 = (__nv_bfloat16*)dmalloc(n, (size_t)pad16(cin) * max_hw * 2);
  for (int k = 0; k < 2; k++) n->gh[k] = (__nv_bfloat16*)dmalloc(n, (size_t)pad16(width) * max_hw * 2);
  n->part = (float*)dmalloc(n, (size_t)n->max_tiles * n->max_layer * 4);
  n->lpart = (double*)dmalloc(n, (size_t)LOSS_CHUNKS * cout * 8);
  n->bpart = (float*)dmalloc(n, (size_t)std::max(BG_CHUNKS, LOSS_CHUNKS) * maxc * 4);
  n->lsum = (double*)dmalloc(n, 8);
  n->fw = (float*)dmalloc(n, 8 * sizeof(float));
  n->err = (int*)dmalloc(n, sizeof(int));
  bool ok = n->p && n->g && n->m && n->v && n->pb && n->ga && n->gh[0] && n->gh[1] && n->part && n->bpart &&
            n->lpart && n->lsum && n->fw && n->err && n->x16;
  for (auto a : n->act) ok = ok && a;
  if (!ok) { lc_destroy(n); return -2; }
  if (cudaMemset(n->ga, 0, (size_t)pad16(cout) * max_hw * 2) != cudaSuccess ||
      cudaMemset(n->err, 0, sizeof(int)) != cudaSuccess) {
    lc_destroy(n);
    return -3;
  }
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

// 3x3 convolution of `in` (cin channels) into `out` (cout channels) on the
// tensor cores with the BF16 weights w (transpose: see k_conv_tc).  A
// channel-major FP32 input (in_blk = 0, the network input) is first rounded
// into the channel-blocked BF16 buffer the TMA loads read.
static int conv(lc_net* n, const void* in, int in_blk, int cin, int H, int W, const __nv_bfloat16* w,
                int transpose, const float* bias, int cout, int relu, const __nv_bfloat16* mask, void* out,
                int out_blk) {
  const int cp = pad16(cin), no = pad16(cout);
  const long hw = (long)H * W;
  if (!in_blk) {
    k_to_blk<<<nblk(hw, 256), 256, 0, n->st>>>(static_cast<const float*>(in), cin, hw, cp, n->x16);
    in = n->x16;
  }
  // the input as a 3-D tensor of 8-byte elements (2 W per channel-block row, H
  // rows, cp / 8 blocks); boxes of 2 TC_SW x (TC_R + 2) x cp / 8, zero fill
  // outside
  CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)W * 2, (cuuint64_t)H, (cuuint64_t)(cp / 8)};
  const cuuint64_t strides[2] = {(cuuint64_t)W * 16, (cuuint64_t)hw * 16};
  const cuuint32_t box[3] = {2 * TC_SW, TC_R + 2, (cuuint32_t)(cp / 8)}, estr[3] = {1, 1, 1};
  if (tma_encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(in), dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return -3;
  const TcCfg& c = tc_cfg[cp / 16 - 1][no / 16 - 1];
  const int ntx = (W + TC_W - 1) / TC_W, ntiles = ntx * ((H + TC_R - 1) / TC_R);
  const int nb = std::min(ntiles, c.per_sm * n->nsm);
  tc_fn(cp, no)<<<nb, TC_THREADS, c.smem, n->st>>>(map, cin, H, W, w, transpose, bias, cout, relu, mask, out,
                                                    out_blk, ntx, ntiles, n->err);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Layer l forward: its input is x (channel-major FP32) for l = 0, else the
// previous hidden output; hidden outputs are channel-blocked BF16, the last
// layer's channel-major FP32 (out).
static int conv_fwd(lc_net* n, int l, const float* x, int H, int W, void* out) {
  const bool last = l == n->depth - 1;
  return conv(n, l == 0 ? (const void*)x : n->act[l - 1], l == 0 ? 0 : 1, n->ci[l], H, W, n->pb + n->woff[l], 0,
       n->p + n->boff[l], n->co[l], last ? 0 : 1, nullptr, out, last ? 0 : 1);
}

int lc_forward(lc_net* n, const float* x_dev, int H, int W, float* y_dev) {
  if (!n || !x_dev || !y_dev || H <= 0 || W <= 0 || (long)H * W > n->max_hw) return -1;
  for (int l = 0; l < n->depth; l++)
    if (conv_fwd(n, l, x_dev, H, W, l == n->depth - 1 ? (void*)y_dev : n->act[l])) return -3;
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lc_train_step(lc_net* n, const float* x_dev, const float* target_dev, int H, int W, int r, int nout,
                  const float* field_w, float lr, double* loss, float* grad_host) {
  if (!n || !x_dev || !target_dev || !field_w || H <= 0 || W <= 0 || r <= 0 || nout <= 0) return -1;
  if ((long)H * W > n->max_hw || nout * r * r != n->cout || nout > 8 || lr < 0) return -1;
  // forward, keeping every layer's output
  for (int l = 0; l < n->depth; l++)
    if (conv_fwd(n, l, x_dev, H, W, n->act[l])) return -3;
  // loss, dL/dy and the last layer's bias-gradient partials
  const int ng = n->cout / r;                    // row groups (field, sub-row)
  if (cudaMemcpyAsync(n->fw, field_w, nout * sizeof(float), cudaMemcpyHostToDevice, n->st) != cudaSuccess) return -3;
  if (r == 4 && ((uintptr_t)target_dev & 15) == 0)
    k_loss<true><<<dim3(LOSS_CHUNKS, ng), 256, 0, n->st>>>(static_cast<const float*>(n->act[n->depth - 1]),
                                                           target_dev, H, W, r, n->fw, n->ga, n->lpart,
                                                           n->bpart, n->cout);
  else
    k_loss<false><<<dim3(LOSS_CHUNKS, ng), 256, 0, n->st>>>(static_cast<const float*>(n->act[n->depth - 1]),
                                                            target_dev, H, W, r, n->fw, n->ga, n->lpart,
                                                            n->bpart, n->cout);
  k_sum_loss<<<1, 1024, 0, n->st>>>(n->lpart, ng * LOSS_CHUNKS, n->lsum);
  // backward: g is dL/d(pre-activation) of layer l, channel-blocked BF16
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
      k_bias_grad<<<BG_CHUNKS, 192, 0, n->st>>>(g, op, (long)H * W, b, n->bpart);
      k_sum_chunks<<<b, 256, 0, n->st>>>(n->bpart, BG_CHUNKS, b, n->g + n->boff[l]);
    }
    if (l > 0) {
      // dL/d(out of layer l-1) = transposed, flipped convolution of g, times ReLU'(out of layer l-1)
      if (conv(n, g, 1, b, H, W, n->pb + n->woff[l], 1, nullptr, a, 0,
               static_cast<const __nv_bfloat16*>(n->act[l - 1]), n->gh[gk], 1))
        return -3;
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
  return lc_sync(n);
}

int lc_sync(lc_net* n) {
  if (!n) return -1;
  int e = 0;
  if (cudaMemcpyAsync(&e, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->st) != cudaSuccess) return -3;
  if (cudaStreamSynchronize(n->st) != cudaSuccess) return -3;
  return e ? -4 : 0;
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

static int tile_count(int n, int tile) { return n < tile + 2 ? 1 : n / tile + (n % tile >= 2 ? 1 : 0); }

int lc_fallback_tiles(const double* eta_dev, const double* b_dev, int H, int W, double thr, double hmin, int tile,
                      int buffer, unsigned char* sel_dev, void* cuda_stream) {
  if (!eta_dev || !b_dev || !sel_dev || H <= 0 || W <= 0 || tile < 2 || buffer < 0 || !(thr >= 0) ||
      !std::isfinite(thr) || !std::isfinite(hmin))
    return -1;
  const int ntx = tile_count(W, tile), nty = tile_count(H, tile);
  k_fallback_tiles<<<dim3(ntx, nty), 256, 0, (cudaStream_t)cuda_stream>>>(eta_dev, b_dev, H, W, thr, hmin, tile,
                                                                           buffer, ntx, nty, sel_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lc_restrict(const double* fine_dev, int Hc, int Wc, int r, double* coarse_dev, void* cuda_stream) {
  if (!fine_dev || !coarse_dev || Hc <= 0 || Wc <= 0 || r <= 0) return -1;
  k_restrict<<<nblk((long)Hc * Wc, 256), 256, 0, (cudaStream_t)cuda_stream>>>(fine_dev, Hc, Wc, r, coarse_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
