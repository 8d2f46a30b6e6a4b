// FP64 reductions: the floor deposit of one step (a9) and the total mass.
//
// Deterministic: each block sums a fixed slice in a fixed tree order into
// partials[block]; the block that takes the last ticket sums the partials in index
// order and resets the ticket.  No floating-point atomics.
#pragma once
#include "common.cuh"

namespace lw {

constexpr int kReduceThreads = 256;
constexpr int kMaxReduceBlocks = 1024;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;  // valid in thread 0
}

// Finish: the last block folds partials[0..nblocks) into *target (target += sum, or
// target = sum when accumulate == 0).
__device__ __forceinline__ void finish_reduction(double block_total, double* partials, unsigned* ticket,
                                                 double* target, int accumulate) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = block_total;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s = 0.0;
    const volatile double* vp = partials;
    for (unsigned b = 0; b < gridDim.x; ++b) s += vp[b];
    *target = accumulate ? *target + s : s;
    *ticket = 0u;
  }
}

// a9: deposit += Vs * sum over the floor (v = 0) of c/6 + c1/6 + 2 c2/3 (RK3 b-weights,
// so that sum c + deposit is invariant).  The floor is the first nfloor nodes.
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) deposit_kernel(Args<T> a, long long nfloor) {
  __shared__ double sh[kReduceThreads / 32];
  double acc = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nfloor;
       k += (long long)gridDim.x * blockDim.x) {
    const double b = ((double)a.c[k] + (double)a.c1[k]) * (1.0 / 6.0) + (double)a.c2[k] * (2.0 / 3.0);
    acc += a.S ? (double)settling_at(a, k) * b : b;  // with sugar Vs(S) per floor node
  }
  double s = block_sum(acc, sh);
  finish_reduction(a.S ? s : s * (double)a.vs, a.partials, a.ticket, &a.scalars[0], 1);
}

// scalars[1] = sum of src[0..count)
template <typename T>
__global__ void __launch_bounds__(kReduceThreads) sum_kernel(Args<T> a, const T* src, long long count) {
  __shared__ double sh[kReduceThreads / 32];
  double acc = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x)
    acc += (double)src[k];
  double s = block_sum(acc, sh);
  finish_reduction(s, a.partials, a.ticket, &a.scalars[1], 0);
}

// Polydisperse particles: phi_tot / phi0 = sum of the classes (in class order), the
// concentration the force reads (Eqs. forceterm_poly, poly).
template <typename T>
struct ClassPtrs {
  const T* c[8];
  int count;
};

// The loads of every class are issued before the sums (unrolled to the 8-class maximum);
// the sum runs in class order.
template <typename T>
__global__ void class_sum_kernel(ClassPtrs<T> cp, T* out, long long n) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  T v[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = m < cp.count ? __ldg(cp.c[m] + k) : T(0);
  T acc = v[0];
#pragma unroll
  for (int m = 1; m < 8; ++m)
    if (m < cp.count) acc += v[m];
  out[k] = acc;
}

}  // namespace lw
