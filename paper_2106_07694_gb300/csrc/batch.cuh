// Batched launches: many independent 2D FP32 simulations of different sizes and
// parameters advanced by one launch per kernel type (the paper's parameter sweep over
// initial concentration and particle diameter, Sec. 2.2 Table 1, run as one job).
//
// Each launch covers the blocks of every instance back to back.  Block b finds its
// instance i by a binary search in the prefix table start[] (start[i] = first block of
// instance i), copies that instance's argument block into shared memory and runs the
// same body as the single-instance kernel on its local block coordinates.  The deposit
// of each instance is folded by that instance's floor CTAs with its own ticket.
#pragma once
#include "common.cuh"
#include "lbm_kernels.cuh"
#include "transport_stage2d_wide.cuh"

namespace lw {

struct BatchTables {
  const Args<float>* args;  // [count]
  const int* lbm_start;     // [count + 1] prefix of fluid-kernel blocks
  const int* lbm_gx;        // [count] fluid blocks per row
  const int* st_start;      // [count + 1] prefix of stage-kernel blocks
  const int* st_strips;     // [count] strips per instance
  const int* st_rows;       // [count] rows per segment
  int count;
};

__device__ __forceinline__ int find_instance(const int* start, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <int PARITY>
__global__ void __launch_bounds__(128) lbm_d2q9_batch_kernel(BatchTables t) {
  __shared__ Args<float> sa;
  __shared__ int s_local[2];
  if (threadIdx.x == 0) {
    const int i = find_instance(t.lbm_start, t.count, blockIdx.x);
    sa = t.args[i];
    const int local = blockIdx.x - t.lbm_start[i];
    const int gx = t.lbm_gx[i];
    s_local[0] = local % gx;
    s_local[1] = local / gx;
  }
  __syncthreads();
  lbm_d2q9_body<float, PARITY>(sa, s_local[0], s_local[1]);
}

template <int STAGE>
__global__ void __launch_bounds__(kWT) stage2d_batch_kernel(BatchTables t) {
  __shared__ Args<float> sa;
  __shared__ int s_meta[4];
  if (threadIdx.x == 0) {
    const int i = find_instance(t.st_start, t.count, blockIdx.x);
    sa = t.args[i];
    const int local = blockIdx.x - t.st_start[i];
    const int strips = t.st_strips[i];
    s_meta[0] = local % strips;
    s_meta[1] = local / strips;
    s_meta[2] = strips;
    s_meta[3] = t.st_rows[i];
  }
  __syncthreads();
  Stage2dParams sp;
  sp.cin = STAGE == 1 ? sa.c : (STAGE == 2 ? sa.c1 : sa.c2);
  sp.cout = STAGE == 1 ? sa.c1 : (STAGE == 2 ? sa.c2 : sa.c);
  sp.H = s_meta[3];
  stage2d_wide_body<STAGE>(sa, sp, s_meta[0], s_meta[1], s_meta[2]);
}

}  // namespace lw
