// The fluid part of a coupled step (collide-stream, AA pattern) over row items of
// kFluidCols columns, for kernels whose CTAs take such items between other work: 64 threads
// x kFluidCols / 64 nodes (x = x0 + t + 64 q).  The populations an item reads -- for each
// direction i one row window of kFluidCols + 8 columns (the item's columns and a four-column
// quad on each side, for the x-shifted pulls of the odd AA step) -- are copied into shared
// memory with asynchronous 16-byte copies (cp.async.cg: at L2, no L1 line), kFluidBufs - 1
// items ahead, so that many bytes are in flight per SM without holding registers; the
// collision then reads them from shared memory.
#pragma once
#include "common.cuh"
#include "lattice.cuh"
#include "lbm_kernels.cuh"

namespace lw {

constexpr int kFluidCols = 128;                 // columns of a fluid item (64 threads x 2 nodes)
constexpr int kFluidBufs = 4;                   // item buffers: one collided, the others in flight
constexpr int kFlQuads = kFluidCols / 4 + 2;    // 16-byte quads of a population row window
constexpr int kFluidPair = 2;                   // nodes a thread collides together
constexpr int kFluidNodes = kFluidCols / 64;    // nodes per thread and item
struct FluidStage {
  float4 w[kFluidBufs][9][kFlQuads];     // items' population windows
  float4 c[kFluidBufs][kFluidCols / 4];  // and their c (the force)
};

// Column offset of direction i's source window for this parity and row (the odd step pulls
// g_opp(i) from x - c_i, or its own g_i when x - c_i is behind a wall).
template <int PARITY>
__device__ __forceinline__ int fluid_src_shift(int i, bool wall) {
  return (PARITY == 1 && !wall) ? D2Q9::cx(i) : 0;
}

// Issue the copies of row y, columns x0 .. x0 + 255 of populations G and concentration C
// (n nodes, nx x ny) into buffer buf (every thread of the CTA takes part, blockDim.x = 64;
// commit separately).
template <int PARITY>
__device__ __forceinline__ void fluid_issue_row(const float* G, const float* C, unsigned n, int nx, int ny, int y,
                                                int x0, FluidStage& st, int buf) {
  // this thread's quads of every window: q = t and q = t + 64
  const int t = (int)threadIdx.x;
  int col0 = x0 - 4 + 4 * t;  // wrapped into [0, nx): quads never straddle the wrap (nx % 4 == 0)
  while (col0 < 0) col0 += nx;
  while (col0 >= nx) col0 -= nx;
  int col1 = x0 - 4 + 4 * (t + 64);
  while (col1 >= nx) col1 -= nx;
  const bool one = t < kFlQuads, two = t + 64 < kFlQuads;
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    int plane = d, row = y;
    if (PARITY == 1) {
      const int ys = y - D2Q9::cy(d);
      if (ys >= 0 && ys < ny) {  // pull g_opp(d) from the row below/above; behind a wall: own g_d
        plane = D2Q9::opp(d);
        row = ys;
      }
    }
    const float* src = G + (size_t)plane * n + (size_t)row * nx;
    if (one) cp_async16(&st.w[buf][d][t], src + col0);
    if (two) cp_async16(&st.w[buf][d][t + 64], src + col1);
  }
  if (t < kFluidCols / 4) {
    int cc = x0 + 4 * t;  // this thread's quad of c
    while (cc >= nx) cc -= nx;
    cp_async16(&st.c[buf][t], C + (size_t)y * nx + cc);
  }
}

// Collide-stream the item's nodes from the windows in buffer buf; u goes to a.u.
template <int PARITY>
__device__ __forceinline__ void fluid_compute_row(const Args<float>& sa, int y, int x0, const FluidStage& st,
                                                  int buf) {
  const float* W = reinterpret_cast<const float*>(&st.w[buf][0][0]);
#pragma unroll 1
  for (int q0 = 0; q0 < kFluidNodes; q0 += kFluidPair) {  // kFluidPair nodes interleaved
    D2Q9Node nd[kFluidPair];
    float g[kFluidPair][9];
#pragma unroll
    for (int h = 0; h < kFluidPair; ++h) {
      const int x = x0 + (int)threadIdx.x + 64 * (q0 + h);
      nd[h] = d2q9_node(sa, x < sa.nx ? x : 0, y);
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int shift = fluid_src_shift<PARITY>(i, nd[h].behind_wall(i, -1));
        g[h][i] = W[i * 4 * kFlQuads + (x - x0 + 4 - shift)];
      }
    }
#pragma unroll
    for (int h = 0; h < kFluidPair; ++h)
      if (x0 + (int)threadIdx.x + 64 * (q0 + h) < sa.nx)
        d2q9_collide_store_c<float, PARITY, false, false, LoadL2>(
            sa, nd[h], g[h], nullptr, reinterpret_cast<const float*>(&st.c[buf][0])[(int)threadIdx.x + 64 * (q0 + h)]);
  }
}

}  // namespace lw
