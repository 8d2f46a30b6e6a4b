// 2D FP32 production transport kernel: the three SSP-RK3 stages of the WENO5 +
// diffusion + settling update of c (steps a4..a9 of the coupled step) in ONE pass.
//
// Decomposition.  A CTA owns a strip of W output columns and a segment of H output
// rows.  Its NT threads hold one column each: the W output columns plus a 9-column
// halo on each side (3 columns of stencil per RK stage).  The CTA sweeps its rows
// bottom to top.  At sweep position r0 it loads input row r0 (c^n and the velocity)
// and advances stage 1 at row r0-3, stage 2 at row r0-6 and stage 3 at row r0-9:
// each stage lags the previous one by the stencil radius, so every value it needs has
// already been produced by the stage below.  Intermediate fields (c1, c2) never
// leave shared memory; each face flux is computed once (the x face on the left of
// every column, the y face above every row, carried in a register to the next row).
// HBM traffic per node: c^n (4 B) and u (8 B) in, c^{n+1} (4 B) out, plus the
// halo overlap.
//
// Arithmetic.  Scalar FP32 (packed f32x2 instructions issue to the FP64 pipe on
// this part, which is far narrower).  The WENO5-JS reconstruction is written on
// first differences with a single division per face half.  Split fluxes are kept
// divided by alpha (epsilon = 1e-6 alpha^2 on the unscaled flux, as in the generic
// kernel).
//
// Walls.  Ghost rows -2, -1 and ny, ny+1 hold the even reflection of c and the odd
// reflection of the fluid velocity (Vs unchanged); the floor face carries -Vs c_0,
// the lid face 0.  Deposit: the CTAs that hold row 0 accumulate
// Vs (c/6 + c1/6 + 2 c2/3) of the floor in FP64 and fold it with a fixed-order,
// last-block reduction.
//
// The output goes to a second c buffer (neighbouring CTAs read this one's input halo).
#pragma once
#include "common.cuh"
#include "reduce_kernels.cuh"

#include <type_traits>

namespace lw {

// ---------------------------------------------------------------- WENO5-JS, scalar FP32
// Written on the first differences d1..d4 of the five upwind-side values a..e, which
// the smoothness indicators and the three candidates share:
//   beta_0 = 13/12 (d2-d1)^2 + 1/4 (3 d2 - d1)^2,  beta_1 = 13/12 (d3-d2)^2 + 1/4 (d2+d3)^2,
//   beta_2 = 13/12 (d4-d3)^2 + 1/4 (d4 - 3 d3)^2;
//   6 (q_k - c) = 5 d2 - 2 d1,  d2 + 2 d3,  4 d3 - d4;
// and one division.  The weights are proportional to d_k prod_{j != k} A_j with
// A_k = (eps + beta_k)^2, and only their ratios matter, so beta_k and eps are both scaled
// by 12/13 (beta_k' = s_k^2 + 3/13 t_k^2) and the linear weights (1, 6, 3)/10 by 10:
//   q-weights  A1 A2,  6 A0 A2,  3 A0 A1;
//   numerator  A1 (A2 r0 + 3 A0 r2) + 6 A0 A2 r1,  denominator  A1 (A2 + 3 A0) + 6 A0 A2.
// Returns the face value c + sum_k w_k (q_k - c).
//
// weno5_q takes the differences d1..d4 and the second differences s_k = d_{k+2} - d_{k+1}
// and returns 6 sum_k w_k (q_k - c) = num / den, so that kernels which reconstruct several
// adjacent faces can share the differences between them.  Rounding is sign-symmetric, so
// b - a = -(a - b) bit for bit: a mirrored (h-) reconstruction may pass the negated
// differences of the stored order and gets the same bits as weno5_face_value.
__device__ __forceinline__ float weno5_q(float d1, float d2, float d3, float d4, float s0, float s1, float s2) {
  const float t0 = fmaf(3.f, d2, -d1), t1 = d2 + d3, t2 = fmaf(-3.f, d3, d4);
  const float q = 3.f / 13.f, eps = 1e-6f * (12.f / 13.f);
  float A0 = fmaf(s0, s0, fmaf(q * t0, t0, eps));
  float A1 = fmaf(s1, s1, fmaf(q * t1, t1, eps));
  float A2 = fmaf(s2, s2, fmaf(q * t2, t2, eps));
  A0 *= A0;
  A1 *= A1;
  A2 *= A2;
  const float r0 = fmaf(5.f, d2, -2.f * d1), r1 = fmaf(2.f, d3, d2), r2 = fmaf(4.f, d3, -d4);
  const float A02x6 = 6.f * (A0 * A2);
  const float num = fmaf(A1, fmaf(3.f * A0, r2, A2 * r0), A02x6 * r1);
  const float den = fmaf(A1, fmaf(3.f, A0, A2), A02x6);
  return __fdividef(num, den);
}

__device__ __forceinline__ float weno5_face_value(float a, float b, float c, float d, float e) {
  const float d1 = b - a, d2 = c - b, d3 = d - c, d4 = e - d;
  return fmaf(weno5_q(d1, d2, d3, d4, d2 - d1, d3 - d2, d4 - d3), 1.f / 6.f, c);
}

// The paper's third-order WENO face value (Supplement Eqs. S10, S11, S14-S16) on the
// upwind-side values a, b, c = h_{i-1}, h_i, h_{i+1}: candidates (b + c)/2 and (3b - a)/2,
// indicators (c - b)^2 and (b - a)^2, linear weights 2/3 and 1/3; one division.
__device__ __forceinline__ float weno3_face_value(float a, float b, float c) {
  const float eps = 1e-6f;
  float a1 = fmaf(c - b, c - b, eps), a2 = fmaf(b - a, b - a, eps);
  a1 *= a1;
  a2 *= a2;
  const float p1 = 2.f * a2;  // (2/3)/a1 : (1/3)/a2 over the common factor 1/(3 a1 a2)
  return __fdividef(fmaf(p1, b + c, a1 * fmaf(3.f, b, -a)), 2.f * (p1 + a1));
}

// FP64 forms of the same face values (the validation build): the same algebra with fma
// and an IEEE division.
__device__ __forceinline__ double weno5_q(double d1, double d2, double d3, double d4, double s0, double s1,
                                          double s2) {
  const double t0 = fma(3.0, d2, -d1), t1 = d2 + d3, t2 = fma(-3.0, d3, d4);
  const double q = 3.0 / 13.0, eps = 1e-6 * (12.0 / 13.0);
  double A0 = fma(s0, s0, fma(q * t0, t0, eps));
  double A1 = fma(s1, s1, fma(q * t1, t1, eps));
  double A2 = fma(s2, s2, fma(q * t2, t2, eps));
  A0 *= A0;
  A1 *= A1;
  A2 *= A2;
  const double r0 = fma(5.0, d2, -2.0 * d1), r1 = fma(2.0, d3, d2), r2 = fma(4.0, d3, -d4);
  const double A02x6 = 6.0 * (A0 * A2);
  const double num = fma(A1, fma(3.0 * A0, r2, A2 * r0), A02x6 * r1);
  const double den = fma(A1, fma(3.0, A0, A2), A02x6);
  return num / den;
}

__device__ __forceinline__ double weno5_face_value(double a, double b, double c, double d, double e) {
  const double d1 = b - a, d2 = c - b, d3 = d - c, d4 = e - d;
  return fma(weno5_q(d1, d2, d3, d4, d2 - d1, d3 - d2, d4 - d3), 1.0 / 6.0, c);
}

__device__ __forceinline__ double weno3_face_value(double a, double b, double c) {
  const double eps = 1e-6;
  double a1 = fma(c - b, c - b, eps), a2 = fma(b - a, b - a, eps);
  a1 *= a1;
  a2 *= a2;
  const double p1 = 2.0 * a2;
  return fma(p1, b + c, a1 * fma(3.0, b, -a)) / (2.0 * (p1 + a1));
}

// Face flux of a transport-scheme variant (SCHEME = kSchemeWeno3 | kSchemeSignSplit bits;
// 0 is the Lax-Friedrichs WENO5 of face_flux_x) from the staged pairs of the six points
// i-2 .. i+3 around the face i+1/2 (p[k], m[k] = point i-2+k).  Lax-Friedrichs schemes
// stage p = h+/alpha, m = h-/alpha; the sign split stages p = w c/alpha, m = w/alpha and
// reconstructs w c from the side the face velocity (w_i + w_{i+1})/2 comes from (ties
// to the left).  T = float or double.
template <int SCHEME, typename T>
__device__ __forceinline__ T face_flux_scheme(const T (&p)[6], const T (&m)[6], T alpha, T kappa, T cl, T cr) {
  constexpr bool W3 = (SCHEME & kSchemeWeno3) != 0, SIGN = (SCHEME & kSchemeSignSplit) != 0;
  T h;
  if (SIGN) {
    const bool left = m[2] + m[3] >= T(0);
    if (W3) {
      h = weno3_face_value(left ? p[1] : p[4], left ? p[2] : p[3], left ? p[3] : p[2]);
    } else {
      h = weno5_face_value(left ? p[0] : p[5], left ? p[1] : p[4], left ? p[2] : p[3], left ? p[3] : p[2],
                           left ? p[4] : p[1]);
    }
  } else if (W3) {
    h = weno3_face_value(p[1], p[2], p[3]) + weno3_face_value(m[4], m[3], m[2]);
  } else {
    h = weno5_face_value(p[0], p[1], p[2], p[3], p[4]) + weno5_face_value(m[5], m[4], m[3], m[2], m[1]);
  }
  return fma_t(alpha, h, kappa * (cl - cr));
}

// Total face flux (unscaled): alpha (h+ + h-) + kappa (cl - cr), with h+ from the
// left-biased values p0..p4 and h- from the right-biased values m0..m4 (already mirrored).
template <typename T>
__device__ __forceinline__ T face_flux_x(T p0, T p1, T p2, T p3, T p4, T m0, T m1, T m2, T m3, T m4, T alpha, T kappa,
                                         T cl, T cr) {
  const T hp = weno5_face_value(p0, p1, p2, p3, p4);
  const T hm = weno5_face_value(m0, m1, m2, m3, m4);
  return fma_t(alpha, hp + hm, kappa * (cl - cr));
}

// ---------------------------------------------------------------- geometry / smem

constexpr int kSwThreads = 256;         // columns per CTA including both halos
constexpr int kSwHalo = 9;              // 3 stages x stencil radius 3
constexpr int kSwPad = 4;               // smem padding of x-indexed rows
constexpr int kSwRowX = kSwThreads + 2 * kSwPad;
constexpr int kRx = 4;                  // x-split ring depth (rows)
constexpr int kRy = 6;                  // y-split ring depth
constexpr int kRw = 8;                  // velocity ring depth
constexpr int kRc0 = 16;                // c^n ring depth (rows r0-9..r0 live)
constexpr int kRc = 4;                  // c1, c2 ring depth

struct SweepSmem {
  float xp[3][kRx][kSwRowX];   // x-split h+/alpha of the stage input (stage 0: c^n, 1: c1, 2: c2)
  float xm[3][kRx][kSwRowX];
  float yp[3][kRy][kSwThreads];
  float ym[3][kRy][kSwThreads];
  float wsx[kRw][kSwThreads];  // u_x / alpha
  float wsy[kRw][kSwThreads];  // (u_y - Vs) / alpha
  float c0[kRc0][kSwRowX];     // c^n
  float c1[kRc][kSwRowX];
  float c2[kRc][kSwRowX];
  float fx[2][3][kSwRowX];     // left-face x flux per stage, double-buffered by row parity
  double red[kSwThreads / 32];
};

__device__ __forceinline__ int ring(int row, int depth) { return (row + 4 * depth) % depth; }

struct SweepParams {
  float* c_out;
  int W;        // output columns per strip
  int H;        // output rows per segment
  float alpha;  // Lax-Friedrichs split speed
  float ghost_shift;  // 2 Vs / alpha
};

// Store the x- and y-splits of a stage input at (row, this column); ry = y-ring slot.
__device__ __forceinline__ void put_splits(SweepSmem& S, int stage, int row, int ry, int t, float c, float wx,
                                           float wy, bool store_x) {
  const float h = 0.5f * c;
  if (store_x) {
    S.xp[stage][row & (kRx - 1)][t + kSwPad] = fmaf(wx, h, h);
    S.xm[stage][row & (kRx - 1)][t + kSwPad] = fmaf(wx, h, -h);
  }
  S.yp[stage][ry][t] = fmaf(wy, h, h);
  S.ym[stage][ry][t] = fmaf(wy, h, -h);
}

// Left x-face flux of column t at `row` for a stage (reads its x-split ring).
__device__ __forceinline__ float xface(const SweepSmem& S, int stage, const float* crow, int row, int t,
                                       float alpha, float kappa) {
  const float* P = S.xp[stage][row & (kRx - 1)] + kSwPad + t;
  const float* M = S.xm[stage][row & (kRx - 1)] + kSwPad + t;
  return face_flux_x(P[-3], P[-2], P[-1], P[0], P[1], M[2], M[1], M[0], M[-1], M[-2], alpha, kappa,
                     crow[kSwPad + t - 1], crow[kSwPad + t]);
}

// Upper y-face flux (row + 1/2) of column t for a stage (reads its y-split ring).
// For the produced stages (c1, c2) the ghost rows above the lid are not stored: they
// are rebuilt from the reflected row, h+_g = -h- - sigma c and h-_g = -h+ - sigma c
// with c = h+ - h- and sigma = Vs/alpha (even c, odd fluid velocity, Vs unchanged).
__device__ __forceinline__ void y_split(const SweepSmem& S, int stage, int rr, int t, int ny, float sigma,
                                        float& p, float& m) {
  if (stage > 0 && rr >= ny) {
    const int rf = ring(2 * ny - 1 - rr, kRy);
    const float P = S.yp[stage][rf][t], M = S.ym[stage][rf][t];
    const float c = P - M;
    p = fmaf(-sigma, c, -M);
    m = fmaf(-sigma, c, -P);
  } else {
    p = S.yp[stage][ring(rr, kRy)][t];
    m = S.ym[stage][ring(rr, kRy)][t];
  }
}

// yo[k] = slot of row (row - 2 + k) in the stage's y ring, k = 0..5.
__device__ __forceinline__ float yface(const SweepSmem& S, int stage, int row, int t, int ny, float sigma,
                                       const int (&yo)[6], float alpha, float kappa, float c_here,
                                       float c_above) {
  const float* P = &S.yp[stage][0][t];
  const float* M = &S.ym[stage][0][t];
  if (stage > 0 && row + 3 >= ny) {  // near the lid: rebuild the ghost rows
    float p[5], m[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float dummy;
      y_split(S, stage, row - 2 + k, t, ny, sigma, p[k], dummy);
      y_split(S, stage, row + 3 - k, t, ny, sigma, dummy, m[k]);
    }
    return face_flux_x(p[0], p[1], p[2], p[3], p[4], m[0], m[1], m[2], m[3], m[4], alpha, kappa, c_here,
                       c_above);
  }
  const int R = kSwThreads;
  return face_flux_x(P[yo[0] * R], P[yo[1] * R], P[yo[2] * R], P[yo[3] * R], P[yo[4] * R], M[yo[5] * R],
                     M[yo[4] * R], M[yo[3] * R], M[yo[2] * R], M[yo[1] * R], alpha, kappa, c_here, c_above);
}

__global__ void __launch_bounds__(kSwThreads, 2) rk3_sweep2d_kernel(Args<float> a, SweepParams sp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SweepSmem& S = *reinterpret_cast<SweepSmem*>(smem_raw);
  const int t = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  const int x0 = blockIdx.x * sp.W;
  int X = (x0 - kSwHalo + t) % nx;
  if (X < 0) X += nx;
  const bool out_col = t >= kSwHalo && t < kSwHalo + sp.W && (x0 + t - kSwHalo) < nx;
  const int y0 = blockIdx.y * sp.H;
  const int y1 = min(ny, y0 + sp.H);
  const float kappa = a.kappa, alpha = sp.alpha, vs = a.vs;
  const float inv_alpha = a.inv_alpha, vs_a = a.vs * a.inv_alpha, sigma = 0.5f * sp.ghost_shift;
  const float* __restrict__ cin = a.c + X;
  const float* __restrict__ ux = a.u + X;
  const float* __restrict__ uy = a.u + a.n + X;
  float* __restrict__ cout = sp.c_out + X;

  // real rows of each stage in this segment (the row below the first one, if any,
  // is a priming row: only its upper face is computed, to seed the carried flux)
  const int lo1 = max(0, y0 - 6), hi1 = min(ny, y1 + 6);
  const int lo2 = max(0, y0 - 3), hi2 = min(ny, y1 + 3);
  const int lo3 = y0, hi3 = y1;
  const int r_begin = lo1 == 0 ? -2 : lo1 - 3;
  const int r_load_end = min(hi1 + 2, ny + 1);
  const int r_end = hi3 - 1 + 9;

  // input rows prefetched three rows ahead (ghost rows reflect into the fluid)
  // Two register sets, used alternately by the even and odd iterations of the unrolled
  // loop: the loads of row r0 + 2 go into the set row r0 has just released, so a load
  // has two iterations to land and no register is moved while it is in flight.
  float qc[2] = {0.f, 0.f}, qx[2] = {0.f, 0.f}, qy[2] = {0.f, 0.f};
  auto fetch = [&](int r, float& c, float& vx, float& vy) {
    if (r > r_load_end) return;
    const int rr = r < 0 ? -1 - r : (r >= ny ? 2 * ny - 1 - r : r);
    const unsigned off = (unsigned)rr * (unsigned)nx;
    c = __ldg(cin + off);
    vx = __ldg(ux + off);
    vy = __ldg(uy + off);
  };
  fetch(r_begin, qc[0], qx[0], qy[0]);
  fetch(r_begin + 1, qc[1], qx[1], qy[1]);

  float carry[3] = {0.f, 0.f, 0.f};
  float dep_c = 0.f, dep_c1 = 0.f, dep_c2 = 0.f;  // floor values (this column) for the deposit
  int sy = ((r_begin % kRy) + kRy) % kRy;         // y-ring slot of row r0

  auto body = [&](auto P, const int r0) {
    constexpr int par = decltype(P)::value;  // register set and fx buffer of this iteration
    const int r1 = r0 - 3, r2 = r0 - 6, r3 = r0 - 9;
    const bool act1 = r1 >= lo1 && r1 < hi1, act2 = r2 >= lo2 && r2 < hi2, act3 = r3 >= lo3 && r3 < hi3;
    const bool prime1 = lo1 > 0 && r1 == lo1 - 1, prime2 = lo2 > 0 && r2 == lo2 - 1, prime3 = lo3 > 0 && r3 == lo3 - 1;

    // y-ring slots: yo13[k] = slot of row r0-5+k (stages 1 and 3 read rows
    // r-2..r+3 around their row, which fall on the same slots); stage 2 is rotated by 3.
    int yo13[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      int v = sy + 1 + k;
      v = v >= kRy ? v - kRy : v;
      v = v >= kRy ? v - kRy : v;
      yo13[k] = v;
    }
    const int yo2[6] = {yo13[3], yo13[4], yo13[5], yo13[0], yo13[1], yo13[2]};
    const int c0s0 = r0 & (kRc0 - 1), c0s1 = r1 & (kRc0 - 1), c0s1u = (r1 + 1) & (kRc0 - 1);
    const int c0s2 = r2 & (kRc0 - 1), c0s3 = r3 & (kRc0 - 1);

    // ---- phase A: x faces of the three stages (data from earlier rows) and the new input row
    if (act1) S.fx[par][0][kSwPad + t] = xface(S, 0, S.c0[c0s1], r1, t, alpha, kappa);
    if (act2) S.fx[par][1][kSwPad + t] = xface(S, 1, S.c1[r2 & (kRc - 1)], r2, t, alpha, kappa);
    if (act3) S.fx[par][2][kSwPad + t] = xface(S, 2, S.c2[r3 & (kRc - 1)], r3, t, alpha, kappa);
    if (r0 <= r_load_end) {
      const float c = qc[par], vx = qx[par], vy = qy[par];
      fetch(r0 + 2, qc[par], qx[par], qy[par]);
      if (r0 >= 0 && r0 < ny) {
        const float wx = vx * inv_alpha;
        const float wy = fmaf(vy, inv_alpha, -vs_a);
        S.wsx[r0 & (kRw - 1)][t] = wx;
        S.wsy[r0 & (kRw - 1)][t] = wy;
        S.c0[c0s0][kSwPad + t] = c;
        put_splits(S, 0, r0, sy, t, c, wx, wy, true);
      } else {  // ghost row: c even, fluid velocity odd, Vs unchanged
        put_splits(S, 0, r0, sy, t, c, 0.f, fmaf(-vy, inv_alpha, -vs_a), false);
      }
    }
    __syncthreads();

    // ---- phase B: stage 1 at r1:  c1 = c + L(c)
    if (act1 || prime1) {
      const float chere = S.c0[c0s1][kSwPad + t];
      const float fup =
          (r1 == ny - 1) ? 0.f : yface(S, 0, r1, t, ny, sigma, yo13, alpha, kappa, chere, S.c0[c0s1u][kSwPad + t]);
      if (act1) {
        const float fdn = (r1 == 0) ? -vs * chere : carry[0];
        const float L = S.fx[par][0][kSwPad + t] - S.fx[par][0][kSwPad + t + 1] + fdn - fup;
        const float c1 = chere + L;
        S.c1[r1 & (kRc - 1)][kSwPad + t] = c1;
        const float wx = S.wsx[r1 & (kRw - 1)][t], wy = S.wsy[r1 & (kRw - 1)][t];
        put_splits(S, 1, r1, yo13[2], t, c1, wx, wy, true);
        if (r1 <= 1) {  // ghost rows -1, -2 below the floor (slots 5, 4)
          put_splits(S, 1, -1 - r1, 5 - r1, t, c1, 0.f, -wy - sp.ghost_shift, false);
          if (r1 == 0) {
            dep_c = chere;
            dep_c1 = c1;
          }
        }
      }
      carry[0] = fup;
    }
    __syncthreads();

    // ---- phase C: stage 2 at r2:  c2 = 3/4 c + 1/4 (c1 + L(c1))
    if (act2 || prime2) {
      const float chere = S.c1[r2 & (kRc - 1)][kSwPad + t];
      const float fup = (r2 == ny - 1) ? 0.f
                                       : yface(S, 1, r2, t, ny, sigma, yo2, alpha, kappa, chere,
                                               S.c1[(r2 + 1) & (kRc - 1)][kSwPad + t]);
      if (act2) {
        const float fdn = (r2 == 0) ? -vs * chere : carry[1];
        const float L = S.fx[par][1][kSwPad + t] - S.fx[par][1][kSwPad + t + 1] + fdn - fup;
        const float c2 = fmaf(0.75f, S.c0[c0s2][kSwPad + t], 0.25f * (chere + L));
        S.c2[r2 & (kRc - 1)][kSwPad + t] = c2;
        const float wx = S.wsx[r2 & (kRw - 1)][t], wy = S.wsy[r2 & (kRw - 1)][t];
        put_splits(S, 2, r2, sy, t, c2, wx, wy, true);
        if (r2 <= 1) {
          put_splits(S, 2, -1 - r2, 5 - r2, t, c2, 0.f, -wy - sp.ghost_shift, false);
          if (r2 == 0) dep_c2 = c2;
        }
      }
      carry[1] = fup;
    }
    __syncthreads();

    // ---- phase D: stage 3 at r3:  c_new = 1/3 c + 2/3 (c2 + L(c2)), written as s + (c - s)/3
    if (act3 || prime3) {
      const float chere = S.c2[r3 & (kRc - 1)][kSwPad + t];
      const float fup = (r3 == ny - 1) ? 0.f
                                       : yface(S, 2, r3, t, ny, sigma, yo13, alpha, kappa, chere,
                                               S.c2[(r3 + 1) & (kRc - 1)][kSwPad + t]);
      if (act3) {
        const float fdn = (r3 == 0) ? -vs * chere : carry[2];
        const float L = S.fx[par][2][kSwPad + t] - S.fx[par][2][kSwPad + t + 1] + fdn - fup;
        const float s = chere + L;
        const float out = fmaf(1.f / 3.f, S.c0[c0s3][kSwPad + t] - s, s);
        if (out_col) {
          cout[(unsigned)r3 * (unsigned)nx] = out;
          report_status(a.status, !isfinite(out));
        }
      }
      carry[2] = fup;
    }
    sy = sy == kRy - 1 ? 0 : sy + 1;
  };
  for (int r0 = r_begin; r0 <= r_end; r0 += 2) {
    body(std::integral_constant<int, 0>(), r0);
    if (r0 + 1 <= r_end) body(std::integral_constant<int, 1>(), r0 + 1);
  }

  // ---- deposit of this step: Vs * sum over the floor of c/6 + c1/6 + 2 c2/3, in FP64;
  // the floor CTAs fold their partial sums in a fixed order
  if (y0 == 0) {
    double v = out_col ? ((double)dep_c + (double)dep_c1) * (1.0 / 6.0) + (double)dep_c2 * (2.0 / 3.0) : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) S.red[t >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (t == 0)
      for (int w = 0; w < kSwThreads / 32; ++w) s += S.red[w];
    __shared__ bool last;
    if (t == 0) {
      a.partials[blockIdx.x] = s * (double)a.vs;
      __threadfence();
      last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && t == 0) {
      __threadfence();
      const volatile double* vp = a.partials;
      double tot = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) tot += vp[b];
      a.scalars[0] += tot;
      *a.ticket = 0u;
    }
  }
}

inline bool sweep2d_supported(int nx, int ny, bool walls) { return walls && nx >= 4 && ny >= 4; }

struct SweepLaunch {
  int W, H, strips, segs;
};

inline SweepLaunch sweep2d_geometry(int nx, int ny, int sm_count, int H_override) {
  SweepLaunch g{};
  const int wmax = kSwThreads - 2 * kSwHalo;
  g.strips = (nx + wmax - 1) / wmax;
  g.W = (nx + g.strips - 1) / g.strips;
  if (H_override > 0) {
    g.H = H_override;
  } else {
    // about two CTAs per SM in one wave, segments no shorter than 64 rows
    int segs = max(1, (2 * sm_count) / g.strips);
    g.H = max(64, (ny + segs - 1) / segs);
  }
  g.H = min(g.H, ny);
  g.segs = (ny + g.H - 1) / g.H;
  return g;
}

inline size_t sweep2d_smem() { return sizeof(SweepSmem); }

inline cudaError_t launch_sweep2d(const Args<float>& a, float* c_out, const SweepLaunch& g, cudaStream_t s) {
  SweepParams sp;
  sp.c_out = c_out;
  sp.W = g.W;
  sp.H = g.H;
  sp.alpha = a.alpha;
  sp.ghost_shift = 2.f * a.vs * a.inv_alpha;
  rk3_sweep2d_kernel<<<dim3(g.strips, g.segs), kSwThreads, sizeof(SweepSmem), s>>>(a, sp);
  return cudaGetLastError();
}

}  // namespace lw
