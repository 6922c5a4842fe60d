// sgn_noalloc.cu -- total-mass reduction that allocates no device memory.
//
// Who needs it: callers that may not allocate device memory at the point where
// they want the mass -- a host that gives this library a fixed memory pool and
// forbids further device allocations (for instance a framework whose caching
// allocator owns all device memory), or a latency-critical loop in which
// cudaMalloc / cudaFree, which can synchronise the whole device, are not
// acceptable.  The reduction below keeps its per-block partial sums in a fixed
// array compiled into this library instead of in allocated scratch.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/sgn.h"

// Partial sums of the first stage.  A file-scope __device__ array: every GPU
// that loads the library holds these SGN_MASS_SCRATCH_MAX doubles (512 KiB)
// until the process exits.  In host code the name is only a stand-in for the
// symbol, never a device address; the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_mass_scratch[SGN_MASS_SCRATCH_MAX];

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;

// Stage 1: block k sums h = max(0, eta - b) over the cells
// [k*kCellsPerBlock, (k+1)*kCellsPerBlock) in a fixed order (each thread a
// strided run of kCellsPerThread cells, then a fixed shared-memory tree) and
// writes one partial.  Every slot that stage 2 reads is written here first, so
// no slot has to start at zero.
__global__ void k_mass_static1(const double* __restrict__ eta, const double* __restrict__ b, long long n,
                               double* partial) {
  __shared__ double red[kThreads];
  long long base = (long long)blockIdx.x * kCellsPerBlock + threadIdx.x;
  double s = 0.0;
  for (int r = 0; r < kCellsPerThread; r++) {
    long long c = base + (long long)r * kThreads;
    if (c < n) {
      double h = eta[c] - b[c];
      s += h > 0.0 ? h : 0.0;
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Stage 2: one block sums the nb partials in a fixed order and scales by the
// cell area.
__global__ void k_mass_static2(const double* partial, int nb, double area, double* out) {
  __shared__ double red[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += kThreads) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * area;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_mass_scratch on the current device, looked up once per
// device (with that device current) and cached.
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SGN_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mass_scratch) != cudaSuccess || !p) return SGN_ECUDA;
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return SGN_OK;
}

}  // namespace

extern "C" int sgn_mass_static(const double* eta_dev, const double* b_dev, int nx, int ny, double dx,
                               double dy, double* mass_dev, void* cuda_stream) {
  if (!eta_dev || !b_dev || !mass_dev || nx <= 0 || ny <= 0 || !(dx > 0) || !(dy > 0)) return SGN_EINVAL;
  long long n = (long long)nx * ny;
  long long nb = (n + kCellsPerBlock - 1) / kCellsPerBlock;
  if (nb > SGN_MASS_SCRATCH_MAX) return SGN_ERANGE;   // the grid needs more partials than the array holds
  double* scratch = nullptr;
  int r = scratch_address(&scratch);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_mass_static1<<<(unsigned)nb, kThreads, 0, st>>>(eta_dev, b_dev, n, scratch);
  k_mass_static2<<<1, kThreads, 0, st>>>(scratch, (int)nb, dx * dy, mass_dev);
  return cudaGetLastError() == cudaSuccess ? SGN_OK : SGN_ECUDA;
}
