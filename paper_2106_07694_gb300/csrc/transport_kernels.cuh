// Particle half of the coupled step: WENO5 + central diffusion + settling, SSP-RK3.
//
//   a4  global Lax-Friedrichs split of the advective flux h = w c, w = u - Vs e_v:
//       h+- = (w +- alpha) c / 2   (the "upwind splitting" after Supplement Eq. S16,
//       with the split speed a constant alpha so that no reduction is needed)
//   a5  WENO5-JS face values (Jiang & Shu 1996, the scheme the paper cites, at fifth
//       order instead of the third order of Eqs. S10-S16): h+ upwind from the left
//       (points i-2..i+2), h- its mirror image (points i+3..i-1)
//   a6  diffusion flux -kappa (c_{i+1} - c_i) (second-order central, Eq. S4)
//   a7  L(c)_i = -sum_d (F_{i+1/2} - F_{i-1/2}) (conservative form, Eq. S9 / Eq. ADS)
//   a8  SSP-RK3 (Eqs. S21-S23): c1 = c + L(c); c2 = 3/4 c + 1/4 c1 + 1/4 L(c1);
//       c_new = 1/3 c + 2/3 c2 + 2/3 L(c2), with u frozen at the step's value
//   walls: fluid nodes v = 0..N-1, walls at v = -1/2 and N-1/2.  Stencils that cross
//       a wall read ghosts (c even, fluid velocity odd, Vs unchanged); the lid face
//       carries no flux; the floor face carries the settling outflow -Vs c_0.
//
// Variants (Args::scheme): kSchemeWeno3, the paper's third-order WENO (Supplement Eqs.
// S10-S20) instead of WENO5; kSchemeSignSplit, the whole flux w c reconstructed from the
// side the face velocity comes from instead of the Lax-Friedrichs split.
//
// This file holds the generic one-node-per-thread form used for every lattice, precision
// and variant; the 2D/3D FP32 production kernels live in transport_stage2d.cuh,
// transport_sweep2d.cuh and transport_sweep3d.cuh.
#pragma once
#include "common.cuh"

namespace lw {

// WENO5-JS face value, written with one division: with a_k = (eps + beta_k)^2 the
// normalised weights are d_k prod_{j!=k} a_j / sum_m d_m prod_{j!=m} a_j.  Inputs are
// the split flux divided by alpha, so eps = 1e-6 here is eps = 1e-6 alpha^2 on the
// unscaled flux.  The face value (in units of alpha) is num / den.
template <typename T>
__device__ __forceinline__ void weno5_face(T a, T b, T c, T d, T e, T& num, T& den) {
  const T eps = T(1e-6);
  const T s0 = a - T(2) * b + c;
  const T s1 = b - T(2) * c + d;
  const T s2 = c - T(2) * d + e;
  const T t0 = a - T(4) * b + T(3) * c;
  const T t1 = b - d;
  const T t2 = T(3) * c - T(4) * d + e;
  T a0 = eps + T(13.0 / 12.0) * s0 * s0 + T(0.25) * t0 * t0;
  T a1 = eps + T(13.0 / 12.0) * s1 * s1 + T(0.25) * t1 * t1;
  T a2 = eps + T(13.0 / 12.0) * s2 * s2 + T(0.25) * t2 * t2;
  a0 *= a0;
  a1 *= a1;
  a2 *= a2;
  const T p0 = T(0.1) * a1 * a2;
  const T p1 = T(0.6) * a0 * a2;
  const T p2 = T(0.3) * a0 * a1;
  const T q0 = T(2) * a - T(7) * b + T(11) * c;
  const T q1 = -b + T(5) * c + T(2) * d;
  const T q2 = T(2) * c + T(5) * d - e;
  num = p0 * q0 + p1 * q1 + p2 * q2;
  den = T(6) * (p0 + p1 + p2);
}

// The paper's third-order WENO face value (Supplement Eqs. S10, S11, S14-S16), upwind side
// on the left: a, b, c = h_{i-1}, h_i, h_{i+1} (scaled by 1/alpha, eps as above);
// candidates (b + c)/2 and (3b - a)/2, indicators (c - b)^2 and (b - a)^2, linear
// weights (2/3, 1/3); one division: face value = num / den.
template <typename T>
__device__ __forceinline__ void weno3_face(T a, T b, T c, T& num, T& den) {
  const T eps = T(1e-6);
  T a1 = eps + (c - b) * (c - b);
  T a2 = eps + (b - a) * (b - a);
  a1 *= a1;
  a2 *= a2;
  const T p1 = T(2) * a2;  // (2/3)/a1 and (1/3)/a2 over the common factor 1/(3 a1 a2)
  const T p2 = a1;
  num = p1 * (b + c) + p2 * (T(3) * b - a);
  den = T(2) * (p1 + p2);
}

template <typename T>
__device__ __forceinline__ T fast_div(T x, T y) { return x / y; }
template <>
__device__ __forceinline__ float fast_div<float>(float x, float y) { return __fdividef(x, y); }

// Total flux through the face between node (x,y,z) and its +1 neighbour along axis d:
// reads c and u at offsets -2..3 along d (periodic wrap, or reflected ghosts across a
// wall).  Never called for the wall faces themselves.
template <typename T, int DIM>
__device__ __forceinline__ T face_flux(const Args<T>& a, const T* __restrict__ cin, int x, int y, int z,
                                       int d) {
  const int VA = DIM - 1;
  const int ext[3] = {a.nx, a.ny, a.nz};
  const int pos0[3] = {x, y, z};
  const long long stride[3] = {1, a.nx, (long long)a.nx * a.ny};
  const long long base = ((long long)z * a.ny + y) * a.nx + x - (long long)pos0[d] * stride[d];
  const bool wall_axis = (d == VA) && a.walls;
  T hp[6], hm[6], cv[6], wsv[6];
#pragma unroll
  for (int k = -2; k <= 3; ++k) {
    int p = pos0[d] + k;
    bool ghost = false;
    if (wall_axis) {
      if (p < 0) {
        p = -1 - p;
        ghost = true;
      } else if (p >= ext[d]) {
        p = 2 * ext[d] - 1 - p;
        ghost = true;
      }
    } else {
      p = wrap_any(p, ext[d]);
    }
    const long long m = base + (long long)p * stride[d];
    const T cval = cin[m];
    T ud = a.u[(long long)d * a.n + m];
    if (ghost) ud = -ud;
    const T sv = (d == VA) ? settling_at(a, m) : T(0);  // Vs, or Vs(S) with sugar
    const T ws = (ud - sv) * a.inv_alpha;               // w / alpha
    cv[k + 2] = cval;
    wsv[k + 2] = ws;
    hp[k + 2] = T(0.5) * (ws + T(1)) * cval;
    hm[k + 2] = T(0.5) * (ws - T(1)) * cval;
  }
  const T diff = a.kappa * (cv[3] - cv[2]);
  if (a.scheme & kSchemeSignSplit) {
    // whole flux w c from the side the face velocity (w_i + w_{i+1})/2 comes from
    T h[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = wsv[k] * cv[k];
    const bool left = wsv[2] + wsv[3] >= T(0);
    T n_, d_;
    if (a.scheme & kSchemeWeno3) {
      if (left)
        weno3_face<T>(h[1], h[2], h[3], n_, d_);
      else
        weno3_face<T>(h[4], h[3], h[2], n_, d_);
    } else {
      if (left)
        weno5_face<T>(h[0], h[1], h[2], h[3], h[4], n_, d_);
      else
        weno5_face<T>(h[5], h[4], h[3], h[2], h[1], n_, d_);
    }
    return a.alpha * fast_div(n_, d_) - diff;
  }
  T np, dp, nm, dm;
  if (a.scheme & kSchemeWeno3) {
    weno3_face<T>(hp[1], hp[2], hp[3], np, dp);
    weno3_face<T>(hm[4], hm[3], hm[2], nm, dm);
  } else {
    weno5_face<T>(hp[0], hp[1], hp[2], hp[3], hp[4], np, dp);
    weno5_face<T>(hm[5], hm[4], hm[3], hm[2], hm[1], nm, dm);
  }
  return a.alpha * (fast_div(np, dp) + fast_div(nm, dm)) - diff;
}

// One RK3 stage on every node.  STAGE 1: c1 = c + L(c).  STAGE 2: c2 = 3/4 c + 1/4 c1 +
// 1/4 L(c1).  STAGE 3: c = 1/3 c + 2/3 c2 + 2/3 L(c2) (in place: c is read only at the
// node itself in this stage).
template <typename T, int DIM, int STAGE>
__global__ void __launch_bounds__(128) rk_stage_kernel(Args<T> a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx) return;
  const int VA = DIM - 1;
  const long long node = ((long long)z * a.ny + y) * a.nx + x;
  const T* __restrict__ cin = STAGE == 1 ? a.c : (STAGE == 2 ? a.c1 : a.c2);
  const int pos[3] = {x, y, z};
  const int ext[3] = {a.nx, a.ny, a.nz};
  T L = T(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const bool wall_axis = (d == VA) && a.walls;
    T fplus, fminus;
    if (wall_axis && pos[d] == ext[d] - 1)
      fplus = T(0);  // lid
    else
      fplus = face_flux<T, DIM>(a, cin, x, y, z, d);
    if (wall_axis && pos[d] == 0) {
      fminus = -settling_at(a, node) * cin[node];  // floor: settling outflow
    } else {
      int q[3] = {x, y, z};
      q[d] = wrap_dec(pos[d] - 1, ext[d]);
      fminus = face_flux<T, DIM>(a, cin, q[0], q[1], q[2], d);
    }
    L -= fplus - fminus;
  }
  if (STAGE == 1) {
    a.c1[node] = a.c[node] + L;
  } else if (STAGE == 2) {
    a.c2[node] = T(0.75) * a.c[node] + T(0.25) * a.c1[node] + T(0.25) * L;
  } else {
    // 1/3 c + 2/3 (c2 + L) written as s + 1/3 (c - s): the FP32 roundings of 1/3 and
    // 2/3 sum to 1 + 3e-8, which would add a bias to c every step.
    const T s = a.c2[node] + L;
    const T out = s + T(1.0 / 3.0) * (a.c[node] - s);
    a.c[node] = out;
    report_status(a.status, !finite_val(out));
  }
}

// Sugar (the paper's density-altering scalar): one explicit first-order upwind step per
// axis in the advective form of Supplement Eqs. S5 (u > 0: backward difference) and S6
// (u < 0: forward difference), with the velocity of this step's fluid update, plus
// central diffusion D_s; walls mirror S (Neumann).  Writes S2.
template <typename T, int DIM>
__global__ void __launch_bounds__(128) sugar_kernel(Args<T> a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  if (x >= nx) return;
  const bool walls = a.walls != 0;
  const unsigned n = (unsigned)a.n;  // Q n < 2^31 (checked at create)
  const unsigned node = ((unsigned)z * (unsigned)ny + (unsigned)y) * (unsigned)nx + (unsigned)x;
  // neighbour offsets along each axis: x (and y in 3D) periodic; the vertical axis wraps, or
  // at a wall takes offset 0 (the ghost mirrors the boundary node: no flux through the wall)
  int off_m[3] = {x == 0 ? nx - 1 : -1, 0, 0}, off_p[3] = {x == nx - 1 ? -(nx - 1) : 1, 0, 0};
  if (DIM == 2) {
    off_m[1] = y == 0 ? (walls ? 0 : (ny - 1) * nx) : -nx;
    off_p[1] = y == ny - 1 ? (walls ? 0 : -(ny - 1) * nx) : nx;
  } else {
    const int plane = nx * ny;
    off_m[1] = y == 0 ? (ny - 1) * nx : -nx;
    off_p[1] = y == ny - 1 ? -(ny - 1) * nx : nx;
    off_m[2] = z == 0 ? (walls ? 0 : (nz - 1) * plane) : -plane;
    off_p[2] = z == nz - 1 ? (walls ? 0 : -(nz - 1) * plane) : plane;
  }
  const T s0 = a.S[node];
  T next = s0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const T sm = a.S[(unsigned)((int)node + off_m[d])];
    const T sp = a.S[(unsigned)((int)node + off_p[d])];
    const T u = a.u[(unsigned)d * n + node];
    next -= u > T(0) ? u * (s0 - sm) : u * (sp - s0);
    next += a.Ds * (sp - T(2) * s0 + sm);
  }
  a.S2[node] = next;
}

}  // namespace lw
