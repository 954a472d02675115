// Residual norms without any device allocation.
//
// Some callers of this library cannot allocate device memory at the moment they
// need the residual norm: a framework that owns all device memory through its own
// pool allocator and forbids raw cudaMalloc (it would bypass the pool's
// accounting and fragment memory), or a long-running service that reserves all of
// its memory at start-up and must never allocate in its steady state, where a
// cudaMalloc could implicitly synchronise the device, add latency spikes, or fail
// close to the HBM limit.  rccsdt_residual_norms_noalloc serves them: it needs no
// context (creating one allocates) and takes its scratch from a fixed array in
// the library image instead of the heap.
//
// The scratch is one file-scope device array of kNoallocSlots doubles (32 KiB plus
// two slots), held by every GPU that loads the library until the process exits.
// Every call on a device shares it: two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on it and may return wrong
// norms; order such calls on one stream or with events.  Each call writes every
// slot it reads before reading it, so the contents left by the previous call are
// never used.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rccsdt.h"
#include "common.cuh"

namespace {

using rcc::i64;

constexpr int kMaxBlocks = 4096;              // n3 = o(o+1)(o+2)/6 <= 4096, i.e. o <= 28
constexpr int kNoallocSlots = kMaxBlocks + 2; // per-block R3 partials, then |R1|^2, |R2|^2
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kNoallocSlots];

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) x += __shfl_xor_sync(0xffffffffu, x, s);
  return x;
}

__device__ double block_sum(double x) {
  __shared__ double ws[32];
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    x = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    x = warp_sum(x);
  }
  return x;
}

// Block b < n3 sums r3c[b]^2; block n3 sums r1^2; block n3 + 1 sums r2^2.
// Every scratch slot read by k_noalloc_finish is written here first.
__global__ void __launch_bounds__(256) k_noalloc_partials(double* scratch, const double* __restrict__ r1, i64 n1,
                                                          const double* __restrict__ r2, i64 n2,
                                                          const double* __restrict__ r3c, i64 V3, int n3) {
  const int b = blockIdx.x;
  const double* p;
  i64 n;
  int slot;
  if (b < n3) {
    p = r3c + (i64)b * V3; n = V3; slot = b;
  } else if (b == n3) {
    p = r1; n = n1; slot = kMaxBlocks;
  } else {
    p = r2; n = n2; slot = kMaxBlocks + 1;
  }
  double s = 0.0;
  for (i64 i = threadIdx.x; i < n; i += blockDim.x) s += p[i] * p[i];
  s = block_sum(s);
  if (threadIdx.x == 0) scratch[slot] = s;
}

// One thread: weights each stored block by the number of occupied triples it
// stands for (6, 3 or 1; colex order blk = C(k+2,3) + C(j+1,2) + i) and sums in
// block order, so the result is deterministic.
__global__ void k_noalloc_finish(const double* __restrict__ scratch, int o, double* __restrict__ norms) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s3 = 0.0;
  int b = 0;
  for (int k = 0; k < o; ++k)
    for (int j = 0; j <= k; ++j)
      for (int i = 0; i <= j; ++i, ++b) {
        const double m = (i == j && j == k) ? 1.0 : ((i == j || j == k) ? 3.0 : 6.0);
        s3 += m * scratch[b];
      }
  const double s1 = scratch[kMaxBlocks], s2 = scratch[kMaxBlocks + 1];
  norms[0] = sqrt(s1);
  norms[1] = sqrt(s2);
  norms[2] = sqrt(s3);
  norms[3] = sqrt(s1 + s2 + s3);
}

// Device address of g_scratch, looked up once per device with that device current.
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {nullptr};

int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RCCSDT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();  // this lookup's own (non-sticky) error; nothing else is pending here
      return RCCSDT_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = (double*)g_addr[dev];
  return RCCSDT_OK;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int rccsdt_residual_norms_noalloc(
    int o, int v, const double* r1, const double* r2, const double* r3c, double* norms, void* stream) {
  if (o < 1 || v < 1 || !r1 || !r2 || !r3c || !norms) return RCCSDT_ERR_ARG;
  const i64 n3 = (i64)o * (o + 1) * (o + 2) / 6;
  if (n3 > kMaxBlocks) return RCCSDT_ERR_ARG;  // o > 28 exceeds the fixed scratch
  // an error left pending by the caller's earlier work is reported and left in place
  // (peek, not get), so the caller can still read its own error state
  if (cudaPeekAtLastError() != cudaSuccess) return RCCSDT_ERR_CUDA;
  double* scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st) return st;
  const i64 V3 = (i64)v * v * v;
  cudaStream_t s = (cudaStream_t)stream;
  k_noalloc_partials<<<(unsigned)n3 + 2, 256, 0, s>>>(scratch, r1, (i64)o * v, r2, (i64)o * o * v * v, r3c, V3,
                                                     (int)n3);
  k_noalloc_finish<<<1, 32, 0, s>>>(scratch, o, norms);
  // nothing was pending before the launches, so an error here is theirs
  return cudaGetLastError() == cudaSuccess ? RCCSDT_OK : RCCSDT_ERR_CUDA;
}
