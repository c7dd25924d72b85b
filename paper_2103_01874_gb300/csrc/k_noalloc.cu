// ppe_rho0_noalloc: rho_0 = min(rho) without any device allocation.
//
// The plan-based entry points take their scratch (reduction slots, spectrum,
// tables) from memory that ppe_plan obtains with cudaMalloc.  Some callers
// cannot do that: code whose device memory is owned by someone else's budget
// (a framework's caching allocator, or the serving loop's admission control,
// where an extra cudaMalloc can fail or push the process over its budget), and
// latency-critical code for which cudaMalloc may synchronise the device.  For
// them this file provides the min-reduction that ppe_rhs / ppe_project run when
// rho0 <= 0, with its scratch in a fixed, file-scope device array.
//
// Scratch: per-block minima plus a completion counter, 16384 * 8 + 4 bytes
// (about 128 KiB).  Every GPU that loads libppe holds one copy of it until the
// process exits.  The largest accepted input is 16384 blocks of 4096 cells,
// i.e. 67,108,864 values.  All calls share the one copy: calls that overlap on
// the GPU race on it and must be serialised by the caller.  The counter is
// cleared at the start of each call; the partials are always written before
// they are read.
#include <mutex>

#include "../../include/ppe.h"
#include "ppe_internal.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 16;
constexpr size_t kNaCellsPerBlock = (size_t)kNaThreads * kNaPerThread;  // 4096
constexpr unsigned kNaMaxBlocks = 16384;                                 // -> 67,108,864 cells
constexpr int kNaMaxDevices = 64;

struct NoallocScratch {
  unsigned long long partial[kNaMaxBlocks];  // per-block minimum, as FP64 bit patterns
  unsigned int blocks_done;                  // must be 0 when the kernel starts
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// One pass: each block reduces its 4096 cells and stores its minimum; the
// block that finishes last reduces the partials and writes *out.  rho > 0 (a
// density), so the IEEE bit patterns order like the values and the reduction
// runs on integers.
__global__ void __launch_bounds__(kNaThreads) k_rho_min_noalloc(const double* __restrict__ rho, size_t n,
                                                                NoallocScratch* s, double* out) {
  __shared__ unsigned long long red[kNaThreads / 32];
  __shared__ int is_last;
  const size_t base = (size_t)blockIdx.x * kNaCellsPerBlock;
  unsigned long long m = 0x7FF0000000000000ull;  // +inf
#pragma unroll
  for (int u = 0; u < kNaPerThread; ++u) {
    const size_t i = base + (size_t)u * kNaThreads + threadIdx.x;
    if (i < n) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(__ldg(rho + i));
      m = b < m ? b : m;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t < m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kNaThreads / 32; ++w) m = red[w] < m ? red[w] : m;
    s->partial[blockIdx.x] = m;
    __threadfence();
    is_last = (atomicAdd(&s->blocks_done, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  m = 0x7FF0000000000000ull;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += kNaThreads) {
    const unsigned long long t = __ldcg(&s->partial[b]);
    m = t < m ? t : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t < m ? t : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kNaThreads / 32; ++w) m = red[w] < m ? red[w] : m;
    *out = __longlong_as_double((long long)m);
    s->blocks_done = 0u;
  }
}

std::mutex g_na_mutex;
NoallocScratch* g_na_ptr[kNaMaxDevices] = {};

// Set-up, once per device with that device current: the device address of the
// static array (its name in host code is only a host-side stand-in).
ppe_status noalloc_scratch(NoallocScratch** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return PPE_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PPE_ERR_CUDA;
    }
    g_na_ptr[dev] = static_cast<NoallocScratch*>(p);
  }
  *out = g_na_ptr[dev];
  return PPE_OK;
}

}  // namespace

extern "C" ppe_status ppe_rho0_noalloc(const double* rho, size_t n, double* rho0_out, void* stream) {
  if (!rho || !rho0_out || n == 0) return PPE_ERR_INVALID_ARG;
  const size_t blocks = (n + kNaCellsPerBlock - 1) / kNaCellsPerBlock;
  if (blocks > kNaMaxBlocks) return PPE_ERR_UNSUPPORTED_SIZE;
  NoallocScratch* s = nullptr;
  ppe_status st = noalloc_scratch(&s);
  if (st != PPE_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  if (cudaMemsetAsync(&s->blocks_done, 0, sizeof(unsigned int), cs) != cudaSuccess) return PPE_ERR_CUDA;
  k_rho_min_noalloc<<<(unsigned)blocks, kNaThreads, 0, cs>>>(rho, n, s, rho0_out);
  return cudaGetLastError() == cudaSuccess ? PPE_OK : PPE_ERR_CUDA;
}
