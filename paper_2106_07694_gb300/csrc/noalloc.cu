// Total mass of a concentration field without any device allocation.
//
// Some callers cannot allocate device memory at all: a host application that hands
// this library a fixed device arena and forbids further cudaMalloc calls, a plugin
// that runs inside another framework's allocator, or a monitoring tool that only holds
// a pointer to a field someone else owns.  The workspace-based lbm_wenoc_total_mass()
// needs a handle and its caller-sized workspace for the per-block partial sums; this
// entry point keeps those partial sums in a fixed file-scope device array instead.
//
// Scratch: kNoAllocMaxBlocks FP64 partial sums plus a ticket and the result slot, in
// one static __device__ array (about 16 KB) that every GPU which loads the library
// holds until the process exits.  Each block sums kNoAllocChunk consecutive elements,
// so at most kNoAllocMaxBlocks * kNoAllocChunk elements can be summed per call; larger
// fields are rejected with LW_EINVAL.
//
// All calls share the array: the ticket is cleared at the start of every call, the
// partial sums are overwritten before they are read, and the array keeps the last
// call's contents.  Two calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on it and give wrong totals.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm_wenoc.h"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 2048;
constexpr long long kNoAllocChunk = 32768;  // elements per block
constexpr int kNoAllocMaxDevices = 64;

// [0, kNoAllocMaxBlocks): partial sums; [kNoAllocMaxBlocks]: result; then the ticket.
constexpr int kNoAllocWords = kNoAllocMaxBlocks + 2;
static __device__ __align__(256) double noalloc_scratch[kNoAllocWords];

std::mutex g_setup_mutex;
double* g_scratch_addr[kNoAllocMaxDevices] = {nullptr};

template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_sum_kernel(const T* __restrict__ c, long long n,
                                                                       double* scratch, double* out) {
  __shared__ double sh[kNoAllocThreads / 32];
  __shared__ bool last;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kNoAllocMaxBlocks + 1);
  const long long begin = (long long)blockIdx.x * kNoAllocChunk;
  const long long end = begin + kNoAllocChunk < n ? begin + kNoAllocChunk : n;
  double acc = 0.0;
  for (long long k = begin + threadIdx.x; k < end; k += kNoAllocThreads) acc += (double)c[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) s += sh[w];
    scratch[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    const volatile double* vp = scratch;
    double tot = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) tot += vp[b];  // fixed order
    scratch[kNoAllocMaxBlocks] = tot;
    *out = tot;
    *ticket = 0u;
  }
}

// Device address of the scratch array on the current device.  The array's name is
// only a host-side stand-in in host code, so the address is looked up once per device
// (with that device current) and cached for the life of the process; a device reset
// (cudaDeviceReset, or the primary context torn down) makes the cached address stale.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LW_ECUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return LW_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LW_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return LW_OK;
}

}  // namespace

extern "C" int lbm_wenoc_total_mass_noalloc(const void* c_dev, int64_t n, int32_t fp64, void* cuda_stream,
                                            double* out_dev) {
  if (!c_dev || !out_dev || n < 1) return LW_EINVAL;
  if (n > (int64_t)kNoAllocMaxBlocks * kNoAllocChunk) return LW_EINVAL;  // beyond the fixed scratch
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != LW_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the ticket must start at zero (an earlier failed call may have left it set)
  if (cudaMemsetAsync(scratch + kNoAllocMaxBlocks + 1, 0, sizeof(double), s) != cudaSuccess) return LW_ECUDA;
  const int blocks = (int)((n + kNoAllocChunk - 1) / kNoAllocChunk);
  if (fp64)
    noalloc_sum_kernel<double><<<blocks, kNoAllocThreads, 0, s>>>(static_cast<const double*>(c_dev), n, scratch,
                                                                   out_dev);
  else
    noalloc_sum_kernel<float><<<blocks, kNoAllocThreads, 0, s>>>(static_cast<const float*>(c_dev), n, scratch,
                                                                  out_dev);
  return cudaGetLastError() == cudaSuccess ? LW_OK : LW_ECUDA;
}
