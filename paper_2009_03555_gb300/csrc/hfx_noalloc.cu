// hfx_noalloc.cu -- an exchange-energy entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs under a custom or
// pre-reserved device-memory budget (a serving process that must not grow its
// footprint mid-request), code inside a framework that owns every allocation,
// or a plugin loaded into a process whose allocator forbids foreign
// allocations.  hfx_exchange_energy keeps its scratch in the quartet-list
// handle, which hfx_build_quartets allocates; this variant needs no handle and
// keeps its scratch in a file-scope device array instead.
//
// Scratch: g_partials, kNoAllocMaxPartials doubles (64 Ki doubles = 512 KiB),
// one partial sum per block of kValuesPerBlock values, so inputs of up to
// kNoAllocMaxPartials * kValuesPerBlock values (2^28, 2 GiB of doubles per
// array) are accepted.  The array lives for as long as the library is loaded
// and is held on every GPU the library touches.  The first pass writes every
// partial slot it later reads, so nothing has to be cleared.  Every call
// shares the array: calls whose work overlaps on the GPU (several streams,
// several host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <string>

#include "hfx.h"

// Sets the message hfx_last_error() returns (defined with it in hfx_core.cu).
void hfx_set_last_error(const std::string& m);

namespace {

constexpr int kNoAllocMaxPartials = 1 << 16;
constexpr int kNoAllocThreads = 256;
constexpr long long kValuesPerBlock = 4096;  // 16 values per thread

static __device__ __align__(256) double g_partials[kNoAllocMaxPartials];


hfx_status noalloc_fail(hfx_status s, const std::string& m) {
  hfx_set_last_error(m);
  return s;
}

// Pass 1: block b sums P_i K_i over its kValuesPerBlock values and writes the
// sum to partial[b] (fixed order inside the block: deterministic).
__global__ void k_dot_partials(long long n, const double* __restrict__ P, const double* __restrict__ K,
                               double* __restrict__ partial) {
  const long long base = (long long)blockIdx.x * kValuesPerBlock;
  long long end = base + kValuesPerBlock;
  if (end > n) end = n;
  double s = 0.0;
  for (long long i = base + threadIdx.x; i < end; i += blockDim.x) s = fma(__ldg(P + i), __ldg(K + i), s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[kNoAllocThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// Pass 2: one block sums the nb partials and writes E_x = -sum / 2.
__global__ void k_dot_final(int nb, const double* __restrict__ partial, double* __restrict__ E_x) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[kNoAllocThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) t += ws[w];
    *E_x = -0.5 * t;
  }
}

}  // namespace

extern "C" {

hfx_status hfx_exchange_energy_noalloc(const double* P_val, const double* K_val, long long n_values, double* E_x,
                                       void* stream) {
  if (!P_val || !K_val || !E_x) return noalloc_fail(HFX_ERR_INVALID_ARG, "NULL argument");
  if (n_values < 0) return noalloc_fail(HFX_ERR_INVALID_ARG, "n_values must be >= 0");
  const long long nb = (n_values + kValuesPerBlock - 1) / kValuesPerBlock;
  if (nb > kNoAllocMaxPartials)
    return noalloc_fail(HFX_ERR_INVALID_ARG,
                        "n_values exceeds the no-allocation limit of " +
                            std::to_string((long long)kNoAllocMaxPartials * kValuesPerBlock) + " values");
  // the array's device address on the current device (the host-side symbol
  // only stands in for it), asked for on every call: after a device reset
  // the module can be loaded again at another address
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
  if (e != cudaSuccess) return noalloc_fail(HFX_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  double* partial = static_cast<double*>(p);
  cudaStream_t s = (cudaStream_t)stream;
  if (nb > 0) k_dot_partials<<<(unsigned)nb, kNoAllocThreads, 0, s>>>(n_values, P_val, K_val, partial);
  k_dot_final<<<1, kNoAllocThreads, 0, s>>>((int)nb, partial, E_x);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(HFX_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return HFX_OK;
}

}  // extern "C"
