// 2D FP32 production transport kernel (all three RK3 stages in one pass).
#pragma once
#include "common.cuh"

namespace lw {

inline bool sweep2d_supported(int, int) { return false; }
inline void launch_sweep2d(const Args<float>&, cudaStream_t) {}

}  // namespace lw
