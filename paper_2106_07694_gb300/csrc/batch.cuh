// Batched simulations: many independent 2D FP32 simulations of different sizes and
// parameters advanced together (the paper's parameter sweep over initial concentration
// and particle diameter, Sec. 2.2 Table 1, run as one job).
//
// Persistent form (default): one cooperative launch of as many CTAs as the SMs hold at
// once advances every instance by up to kPersistSteps steps.  A step is four phases --
// the fluid part (collide-stream), then the three RK3 stages of the transport -- over a
// work list of (instance, tile) items; a grid barrier separates the phases.  Fluid items
// are one row by 128 columns, one contiguous run per CTA (uniform cost); stage items are one
// four-column-kernel strip by one row segment (the segment height is the instance's own,
// chosen by the autotuner), taken from a per-phase counter so that uneven items balance.
// The barrier waits on a generation word with a clock64 bound: a CTA that waits longer
// than the limit sets kStatusTimeout in the batch status word and returns, and every
// other CTA leaves at its next wait, so the launch ends and the host reads LW_ETIMEOUT.
// Every field the launch writes is read back at L2 (LoadL2): L1 is not coherent between
// SMs within a launch.
//
// Split form: per step the fluid part as one grouped launch (below; a short memory-bound
// kernel with 128-thread CTAs keeps more bytes in flight than the persistent CTAs, whose
// registers are sized for the stage body), then the three RK3 stages in one persistent
// launch as above.
//
// Grouped form: one launch per kernel type and step; block b finds its instance by a
// binary search in the prefix table of block counts and runs the single-instance body.
// All forms run the same per-node arithmetic as the single-instance kernels.
#pragma once
#include "common.cuh"
#include "lbm_kernels.cuh"
#include "transport_stage2d_wide.cuh"
#include "fluid_rows.cuh"

namespace lw {

constexpr int kPersistSteps = 16;  // steps per persistent launch (work counters per launch)
constexpr int kPersistMinB = 8;    // CTAs per SM the persistent kernel's registers must allow

struct BatchTables {
  const Args<float>* args;  // [count]
  const int* lbm_start;     // [count + 1] prefix of fluid-kernel blocks (grouped form)
  const int* lbm_gx;        // [count] fluid blocks per row (grouped form)
  const int* st_start;      // [count + 1] prefix of stage items / blocks
  const int* st_strips;     // [count] strips per instance
  const int* st_rows;       // [count] rows per segment
  const int* fl_start;      // [count + 1] prefix of fluid items (persistent form)
  const int* fl_chunks;     // [count] 256-column chunks per row
  int count;
  unsigned* bar;     // [0] arrivals at the current barrier, [1] generation (zeroed per launch)
  unsigned* status;  // [0] batch status (kStatusTimeout)
  unsigned* queue;   // stage-item counters, 3 per step (zeroed per launch)
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

// ------------------------------------------------------------------ grouped form

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
  __shared__ __align__(16) StageWideSmem S;
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
  stage2d_wide_body<STAGE>(S, sa, sp, s_meta[0], s_meta[1], s_meta[2]);
}

// ------------------------------------------------------------------ persistent form

// Grid barrier with a bounded wait.  Returns false (and leaves kStatusTimeout set) when
// this CTA gave up or another one already had.
__device__ __forceinline__ bool batch_grid_sync(const BatchTables& t, unsigned nblocks, long long limit,
                                                int& s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = t.bar + 1;
    volatile unsigned* st = t.status;
    const unsigned g0 = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(t.bar, 1u) + 1u == nblocks) {
      t.bar[0] = 0u;  // only this CTA touches the count until the generation moves
      __threadfence();
      atomicAdd(t.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (*st & kStatusTimeout) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > limit) {
          atomicOr(t.status, kStatusTimeout);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Fluid phase of every instance: item = one row by kFluidCols columns (fluid_rows.cuh);
// the window buffers overlay the stage phases' shared block.
constexpr size_t kPersistSmem = sizeof(StageWideSmem) > sizeof(FluidStage) ? sizeof(StageWideSmem) : sizeof(FluidStage);

// Instance of a run of fluid items, kept while the items stay in it: a CTA's items are
// consecutive, so the table lookup (a chain of dependent loads) is rare.
struct FluidCursor {
  int start = 0, end = 0, i = -1, chunks = 1;
  const float* G = nullptr;
  const float* C = nullptr;
  unsigned n = 0;
  int nx = 0, ny = 0;
};

__device__ __forceinline__ void fluid_seek(const BatchTables& t, FluidCursor& c, int item) {
  if (item >= c.start && item < c.end) return;
  const int i = find_instance(t.fl_start, t.count, item);
  c.i = i;
  c.start = __ldg(t.fl_start + i);
  c.end = __ldg(t.fl_start + i + 1);
  c.chunks = __ldg(t.fl_chunks + i);
  const Args<float>* A = t.args + i;
  c.G = A->g;
  c.C = A->c;
  c.n = (unsigned)A->n;
  c.nx = A->nx;
  c.ny = A->ny;
}

template <int PARITY>
__device__ __forceinline__ void fluid_issue(const BatchTables& t, FluidCursor& c, int item, FluidStage& st, int buf) {
  fluid_seek(t, c, item);
  const int local = item - c.start;
  fluid_issue_row<PARITY>(c.G, c.C, c.n, c.nx, c.ny, local / c.chunks, (local % c.chunks) * kFluidCols, st, buf);
}

// Fluid items are uniform in cost, so each CTA takes one contiguous run of them (rows of
// one instance in order, which also keeps a row's windows in L2 for the next row's odd-step
// pulls); the next item's windows are copied while the current one is collided.
template <int PARITY>
__device__ __forceinline__ void batch_fluid_phase(const BatchTables& t, FluidStage& st, Args<float>& sa,
                                                  int& s_inst) {
  const int total = __ldg(t.fl_start + t.count);
  const int per = (total + (int)gridDim.x - 1) / (int)gridDim.x;
  const int first = (int)blockIdx.x * per, last = min(total, first + per);
  constexpr int kAhead = kFluidBufs - 1;
  FluidCursor ci, cc;  // the issuing side (kAhead items ahead) and the computing side
  int inst = s_inst;   // the instance in sa (the same in every thread)
#pragma unroll
  for (int j = 0; j < kAhead; ++j) {
    if (first + j < last) fluid_issue<PARITY>(t, ci, first + j, st, j);
    cp_async_commit();
  }
  int buf = 0;
  for (int item = first; item < last; ++item, buf = buf == kFluidBufs - 1 ? 0 : buf + 1) {
    const int ahead = item + kAhead;
    if (ahead < last) fluid_issue<PARITY>(t, ci, ahead, st, buf == 0 ? kFluidBufs - 1 : buf - 1);
    cp_async_commit();
    cp_async_wait<kAhead>();  // this item's windows (the later items' copies may still fly)
    fluid_seek(t, cc, item);
    __syncthreads();     // every thread's copies have landed; sa is no longer read
    if (cc.i != inst) {  // uniform: every thread computed the same cursor
      if (threadIdx.x == 0) {
        sa = t.args[cc.i];
        s_inst = cc.i;
      }
      inst = cc.i;
      __syncthreads();
    }
    const int local = item - cc.start;
    fluid_compute_row<PARITY>(sa, local / cc.chunks, (local % cc.chunks) * kFluidCols, st, buf);
    __syncthreads();  // buffer `buf` is refilled by the next item's issue
  }
  cp_async_wait<0>();
  __syncthreads();
}

// One RK3 stage of every instance: items taken from the phase's counter.
template <int STAGE>
__device__ __forceinline__ void batch_stage_phase(const BatchTables& t, unsigned* counter, StageWideSmem& S,
                                                  Args<float>& sa, int& s_inst, int* s_meta) {
  const int total = __ldg(t.st_start + t.count);
  for (;;) {
    if (threadIdx.x == 0) {
      const int item = (int)atomicAdd(counter, 1u);
      s_meta[0] = item;
      if (item < total) {
        const int i = find_instance(t.st_start, t.count, item);
        if (i != s_inst) {
          sa = t.args[i];
          s_inst = i;
        }
        const int local = item - __ldg(t.st_start + i);
        const int strips = __ldg(t.st_strips + i);
        s_meta[1] = local % strips;
        s_meta[2] = local / strips;
        s_meta[3] = strips;
        s_meta[4] = __ldg(t.st_rows + i);
      }
    }
    __syncthreads();
    if (s_meta[0] >= total) break;
    Stage2dParams sp;
    sp.cin = STAGE == 1 ? sa.c : (STAGE == 2 ? sa.c1 : sa.c2);
    sp.cout = STAGE == 1 ? sa.c1 : (STAGE == 2 ? sa.c2 : sa.c);
    sp.H = s_meta[4];
    stage2d_wide_body<STAGE, LoadL2>(S, sa, sp, s_meta[1], s_meta[2], s_meta[3]);
    __syncthreads();
  }
  __syncthreads();
}

// nsteps (<= kPersistSteps) coupled steps of every instance from AA parity `parity`.
// with_fluid = 0: the three RK3 stages of one step only (nsteps = 1), the fluid part having
// run in a grouped launch before this one.  skip_cta >= 0: that CTA leaves before its first
// barrier (a host-made fault that the bounded wait turns into LW_ETIMEOUT).
__global__ void __launch_bounds__(kWT, kPersistMinB) batch_persistent_kernel(BatchTables t, int parity, int nsteps,
                                                               long long wait_limit, int skip_cta,
                                                               int with_fluid) {
  __shared__ __align__(16) unsigned char smem_buf[kPersistSmem];
  StageWideSmem& S = *reinterpret_cast<StageWideSmem*>(smem_buf);
  __shared__ Args<float> sa;
  __shared__ int s_inst, s_ok;
  __shared__ int s_meta[5];
  // a launch after a timeout that has not been read yet does nothing (the state is undefined)
  if ((int)blockIdx.x == skip_cta || (*reinterpret_cast<volatile unsigned*>(t.status) & kStatusTimeout)) return;
  if (threadIdx.x == 0) s_inst = -1;
  __syncthreads();
  const unsigned nb = gridDim.x;
  if (!with_fluid) nsteps = min(nsteps, 1);
  for (int k = 0; k < nsteps; ++k) {
    if (with_fluid) {
      FluidStage& fs = *reinterpret_cast<FluidStage*>(smem_buf);
      if (((parity + k) & 1) == 0)
        batch_fluid_phase<0>(t, fs, sa, s_inst);
      else
        batch_fluid_phase<1>(t, fs, sa, s_inst);
      if (!batch_grid_sync(t, nb, wait_limit, s_ok)) return;
    }
    batch_stage_phase<1>(t, t.queue + 3 * k, S, sa, s_inst, s_meta);
    if (!batch_grid_sync(t, nb, wait_limit, s_ok)) return;
    batch_stage_phase<2>(t, t.queue + 3 * k + 1, S, sa, s_inst, s_meta);
    if (!batch_grid_sync(t, nb, wait_limit, s_ok)) return;
    batch_stage_phase<3>(t, t.queue + 3 * k + 2, S, sa, s_inst, s_meta);
    if (k + 1 < nsteps && !batch_grid_sync(t, nb, wait_limit, s_ok)) return;
  }
}

}  // namespace lw
