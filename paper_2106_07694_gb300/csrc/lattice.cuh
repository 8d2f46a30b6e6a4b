// Velocity sets of the fluid solver (Sec. 2.3.1: "DrQm" lattices; D3Q19 as in the
// paper's Fig. 3, D2Q9 its 2D counterpart).  Directions are stored in opposite
// pairs (1,2), (3,4), ... so that opp(i) is computed, not looked up.
#pragma once

struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int DIM = 2;
  static constexpr int VAXIS = 1;  // vertical = y
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int v[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
    return v[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int v[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int DIM = 3;
  static constexpr int VAXIS = 2;  // vertical = z
  // rest; 6 axis directions; 12 plane diagonals, each followed by its opposite
  __host__ __device__ static constexpr int cx(int i) {
    constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[i];
  }
  __host__ __device__ static constexpr int cy(int i) {
    constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[i];
  }
  __host__ __device__ static constexpr int cz(int i) {
    constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[i];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
};
