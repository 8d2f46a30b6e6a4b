// Reverse-mode (adjoint) kernels of the 2D coupled step, for the gradient of the
// deposited mass (Sec. 4, m_b) with respect to the initial concentration and to Vs.
//
// Forward step n (lbm_kernels.cuh, transport kernels):
//   u = U(g, c); g' = Stream(Collide(g, F(c)));
//   c1 = c + L(c; u); c2 = 3/4 c + 1/4 c1 + 1/4 L(c1; u); c' = 1/3 c + 2/3 c2 + 2/3 L(c2; u);
//   J += Vs sum_floor(c/6 + c1/6 + 2 c2/3).
// Given lambda(c') and lambda(g') and the recorded c, c1, c2, u, rho of the step, one
// reverse step is six launches: the three transport stages backwards (for each,
// adj_faces_kernel records every face's flux derivatives once and a gather sums, per node,
// the records of the faces whose stencils contain it: the Jacobian-transpose of L with
// respect to its input and to u, WENO5-JS nonlinear weights included), the last gather
// fused with the fluid step backwards (reverse streaming with bounce-back, transpose of
// the BGK-Guo collision, the velocity chain u = (j + F/2)/rho, the buoyancy F_y = -A c).
// The Lax-Friedrichs alpha is a fixed parameter here (the caller sets lf_alpha), so d/dVs
// holds alpha fixed.  No atomics: results are bitwise reproducible and independent of the
// checkpoint spacing.
#pragma once
#include "common.cuh"
#include "lattice.cuh"
#include "lbm_kernels.cuh"

namespace lw {

// Adjoint fields of one reverse step.  mu = lambda(c^{n+1}) (read by stage 3, then
// overwritten with lambda(c^n) by the fluid kernel); lc2, lc1, lc accumulate lambda of
// c2, c1 and c^n (each written whole by its stage kernel); lam_u = lambda(u) [2][n]
// (written by stage 3, accumulated by stages 2 and 1).
template <typename T>
struct AdjFields {
  T* mu;
  T* lc2;
  T* lc1;
  T* lc;
  T* lam_u;
  double* lam_vs;   // dJ/dVs (written once at the end)
  double* vs_part;  // per-CTA partial sums of dJ/dVs, accumulated over stages and steps
};

// Fused multiply-add in the working precision.
__device__ __forceinline__ float fmaf_t(float x, float y, float z) { return fmaf(x, y, z); }
__device__ __forceinline__ double fmaf_t(double x, double y, double z) { return fma(x, y, z); }

// Reciprocal for the derivative weights: MUFU reciprocal (2 ulp) in FP32, exact in FP64.
__device__ __forceinline__ float adj_rcp(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double adj_rcp(double x) { return 1.0 / x; }

// WENO5-JS face value of the scaled values v[0..4] (upwind side first) and its partial
// derivatives dv[0..4]: sum_k w_k dq_k/dv_j + sum_m (q_m - val) w_m (-2/(eps+beta_m)) dbeta_m/dv_j.
// Written on the first differences d1..d4 (candidates relative to the centre value c:
// 6 (q_m - c) = 5 d2 - 2 d1, d2 + 2 d3, 4 d3 - d4; s_m, t_m as in the indicators below).
// The weights depend only on ratios of (eps + beta_m)^2, so beta_m and eps are scaled by
// 12/13: beta'_m = s_m^2 + k t_m^2 with k = 3/13, and d beta'_m/dv = 2 (s_m ds_m + k t_m dt_m),
// the factor 2 folded into the weight-sensitivity factors r_m.
template <typename T>
__device__ __forceinline__ T weno5_value_grad(const T (&v)[5], T (&dv)[5]) {
  const T a = v[0], b = v[1], c = v[2], d = v[3], e = v[4];
  const T d1 = b - a, d2 = c - b, d3 = d - c, d4 = e - d;
  const T dq0 = fmaf_t(T(5.0 / 6.0), d2, T(-1.0 / 3.0) * d1);
  const T dq1 = fmaf_t(T(1.0 / 3.0), d3, T(1.0 / 6.0) * d2);
  const T dq2 = fmaf_t(T(2.0 / 3.0), d3, T(-1.0 / 6.0) * d4);
  const T s0 = d2 - d1, s1 = d3 - d2, s2 = d4 - d3;            // a - 2b + c, b - 2c + d, c - 2d + e
  const T t0 = fmaf_t(T(3), d2, -d1), t1 = d2 + d3, t2 = fmaf_t(T(-3), d3, d4);  // a - 4b + 3c, d - b, 3c - 4d + e
  const T k = T(3.0 / 13.0), eps = T(1e-6 * 12.0 / 13.0);
  const T kt0 = k * t0, kt1 = k * t1, kt2 = k * t2;
  // reciprocals of eps' + beta'_m and of the weight sum: four in all
  const T i0 = adj_rcp(fmaf_t(s0, s0, fmaf_t(kt0, t0, eps)));
  const T i1 = adj_rcp(fmaf_t(s1, s1, fmaf_t(kt1, t1, eps)));
  const T i2 = adj_rcp(fmaf_t(s2, s2, fmaf_t(kt2, t2, eps)));
  const T a0 = T(0.1) * i0 * i0, a1 = T(0.6) * i1 * i1, a2 = T(0.3) * i2 * i2;
  const T inv = adj_rcp(a0 + a1 + a2);
  const T w0 = a0 * inv, w1 = a1 * inv, w2 = a2 * inv;
  const T dval = fmaf_t(w2, dq2, fmaf_t(w1, dq1, w0 * dq0));  // val - c
  // weight-sensitivity factors 2 r_m = -4 (q_m - val) w_m / (eps' + beta'_m)
  const T r0 = T(-4) * (dq0 - dval) * (w0 * i0);
  const T r1 = T(-4) * (dq1 - dval) * (w1 * i1);
  const T r2 = T(-4) * (dq2 - dval) * (w2 * i2);
  dv[0] = w0 * T(1.0 / 3.0) + r0 * (s0 + kt0);
  dv[1] = w0 * T(-7.0 / 6.0) + w1 * T(-1.0 / 6.0) + r0 * (T(-2) * s0 - T(4) * kt0) + r1 * (s1 - kt1);
  dv[2] = w0 * T(11.0 / 6.0) + w1 * T(5.0 / 6.0) + w2 * T(1.0 / 3.0) + r0 * (s0 + T(3) * kt0) +
          r1 * (T(-2) * s1) + r2 * (s2 + T(3) * kt2);
  dv[3] = w1 * T(1.0 / 3.0) + w2 * T(5.0 / 6.0) + r1 * (s1 + kt1) + r2 * (T(-2) * s2 - T(4) * kt2);
  dv[4] = w2 * T(-1.0 / 6.0) + r2 * (s2 + kt2);
  return c + dval;
}

// Adjoint of one face flux F = alpha (v+ + v-) + kappa (c_0 - c_1) (face between stencil
// positions 2 and 3 of the six values c[0..5], w[0..5] = velocity / alpha): dc[k] =
// lamF dF/dc_k and dw[k] = lamF dF/dw_k (w the physical face-normal velocity).  With
// h = (w/alpha +- 1) c / 2 (scaled by 1/alpha), dF/dh = alpha dv, dh/dc = (w/alpha +- 1)/2
// and dF/dw = dv c / 2.
template <typename T>
__device__ __forceinline__ void face_adjoint(const T (&cv)[6], const T (&wv)[6], T alpha, T kappa, T lamF,
                                             T (&dc)[6], T (&dw)[6]) {
  T hp[5], hm[5], gp[5], gm[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    hp[k] = T(0.5) * (wv[k] + T(1)) * cv[k];          // h+ at stencil k
    hm[k] = T(0.5) * (wv[5 - k] - T(1)) * cv[5 - k];  // h- mirrored: stencil 5..1
  }
  weno5_value_grad<T>(hp, gp);
  weno5_value_grad<T>(hm, gm);
  const T la = lamF * alpha, lh = T(0.5) * lamF;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    dc[k] = T(0);
    dw[k] = T(0);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    dc[k] += la * gp[k] * T(0.5) * (wv[k] + T(1));
    dw[k] += lh * gp[k] * cv[k];
    dc[5 - k] += la * gm[k] * T(0.5) * (wv[5 - k] - T(1));
    dw[5 - k] += lh * gm[k] * cv[5 - k];
  }
  dc[2] += lamF * kappa;
  dc[3] -= lamF * kappa;
}

// Per-face derivative records of one stage (scratch, [k][node] layout, k = stencil
// position 0..5 of the face node + 1/2): dcx/dwx for the face on the +x side of each
// node, dcy/dwy for the +y side (zero on the lid row).  dw is the derivative with
// respect to the physical face-normal velocity w at that stencil position.
template <typename T>
struct FaceRecords {
  T* dcx;
  T* dwx;
  T* dcy;
  T* dwy;
};

constexpr int kAdjThreads = 128;

// Adjoint of SSP-RK3 stage STAGE of the transport, part 1: every face once.
//   STAGE 3: c' = 1/3 c + 2/3 (c2 + L(c2)):  lamL = 2/3 mu
//   STAGE 2: c2 = 3/4 c + 1/4 (c1 + L(c1)):  lamL = 1/4 lc2
//   STAGE 1: c1 = c + L(c):                  lamL = lc1
// The thread of node i records, for the faces on its +x and +y sides, lamF = lamL[next] -
// lamL[i] (the face flux leaves i and enters next) times the flux derivatives with respect
// to the six stencil values of c and of w (WENO5-JS nonlinear weights included; ghost rows
// mirror c and flip u).  The Vs terms go to a per-CTA partial: -lamF dF/dw on vertical
// faces (w = +-u - Vs), the floor face F = -Vs c_0, and the deposit's RK3 b-weights
// (2/3, 1/6, 1/6 of c2, c1, c on the floor).
template <typename T, int STAGE>
__global__ void __launch_bounds__(kAdjThreads) adj_faces_kernel(Args<T> a, AdjFields<T> f, FaceRecords<T> fr) {
  __shared__ double red[kAdjThreads / 32];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int nx = a.nx, ny = a.ny;
  const unsigned n = (unsigned)a.n;  // 24 n < 2^31 (checked by the host)
  const T* __restrict__ cs = STAGE == 3 ? a.c2 : (STAGE == 2 ? a.c1 : a.c);
  const T* __restrict__ lsrc = STAGE == 3 ? f.mu : (STAGE == 2 ? f.lc2 : f.lc1);
  const T* __restrict__ U = a.u;
  const T lscale = STAGE == 3 ? T(2.0 / 3.0) : (STAGE == 2 ? T(0.25) : T(1));
  T vs_acc = T(0);  // this thread's Vs terms (FP64 from the block sum on)
  if (x < nx) {
    const int node = y * nx + x;
    const int row = node - x;
    const T alpha = a.alpha, ia = a.inv_alpha, kappa = a.kappa, vs = a.vs;
    const T lam_here = lscale * lsrc[node];
    // +x face (periodic)
    {
      T cv[6], wv[6], dc[6], dw[6];
      if (x >= 2 && x + 3 < nx) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          cv[k] = cs[node - 2 + k];
          wv[k] = U[node - 2 + k] * ia;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int q = row + wrap_any(x - 2 + k, nx);
          cv[k] = cs[q];
          wv[k] = U[q] * ia;
        }
      }
      const T lamF = lscale * lsrc[x + 1 == nx ? row : node + 1] - lam_here;
      face_adjoint<T>(cv, wv, alpha, kappa, lamF, dc, dw);
      T* __restrict__ pc = fr.dcx + node;
      T* __restrict__ pw = fr.dwx + node;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        pc[k * n] = dc[k];
        pw[k * n] = dw[k];
      }
    }
    // +y face (none on the lid row); ghost rows beyond the floor and lid mirror c, flip u
    T* __restrict__ pc = fr.dcy + node;
    T* __restrict__ pw = fr.dwy + node;
    if (y < ny - 1) {
      T cv[6], wv[6], dc[6], dw[6];
      const T* __restrict__ V = U + n;
      if (y >= 2 && y + 3 < ny) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int q = node + (k - 2) * nx;
          cv[k] = cs[q];
          wv[k] = (V[q] - vs) * ia;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const int p = y - 2 + k;
          const bool ghost = p < 0 || p >= ny;
          const int pr = p < 0 ? -1 - p : (p >= ny ? 2 * ny - 1 - p : p);
          const int q = pr * nx + x;
          cv[k] = cs[q];
          const T u = V[q];
          wv[k] = ((ghost ? -u : u) - vs) * ia;
        }
      }
      const T lamF = lscale * lsrc[node + nx] - lam_here;
      face_adjoint<T>(cv, wv, alpha, kappa, lamF, dc, dw);
      T sw = T(0);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        pc[k * n] = dc[k];
        pw[k * n] = dw[k];
        sw += dw[k];
      }
      vs_acc -= sw;
    } else {
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        pc[k * n] = T(0);
        pw[k * n] = T(0);
      }
    }
    if (y == 0) {
      const T c0 = cs[node];
      vs_acc += c0 * (STAGE == 3 ? T(2.0 / 3.0) : T(1.0 / 6.0)) - c0 * lam_here;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vs_acc += __shfl_down_sync(0xffffffffu, vs_acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)vs_acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) s += red[w];
    f.vs_part[blockIdx.y * gridDim.x + blockIdx.x] += s;  // own slot, fixed order over steps
  }
}

// Part 2: each node gathers the records of the faces whose stencils contain it (x faces
// x + 2 - k at position k, periodic; y faces y + 2 - k for existing faces, plus the ghost
// positions that mirror onto rows 0, 1, ny - 2, ny - 1, with u odd):
//   STAGE 3: lc2 = lamL + L^T lamL
//   STAGE 2: lc1 = lamL + L^T lamL
//   STAGE 1: lc  = 1/3 mu + 3/4 lc2 + lamL + L^T lamL
// with the deposit's floor terms and the floor face; gx, gy = this stage's part of
// lambda(u).
template <typename T, int STAGE>
__device__ __forceinline__ void gather_node(const Args<T>& a, const AdjFields<T>& f, const FaceRecords<T>& fr,
                                            int x, int y, T& v, T& gx, T& gy) {
  const int nx = a.nx, ny = a.ny;
  const unsigned n = (unsigned)a.n;
  const int node = y * nx + x;
  const int row = node - x;
  const T* __restrict__ lsrc = STAGE == 3 ? f.mu : (STAGE == 2 ? f.lc2 : f.lc1);
  const T lscale = STAGE == 3 ? T(2.0 / 3.0) : (STAGE == 2 ? T(0.25) : T(1));
  const T vs = a.vs;
  const T* __restrict__ DCX = fr.dcx;
  const T* __restrict__ DWX = fr.dwx;
  const T* __restrict__ DCY = fr.dcy;
  const T* __restrict__ DWY = fr.dwy;
  T gc = T(0);
  gx = T(0);
  gy = T(0);
  if (x >= 3 && x + 2 < nx) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const unsigned q = k * n + (unsigned)(node + 2 - k);
      gc += DCX[q];
      gx += DWX[q];
    }
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const unsigned q = k * n + (unsigned)(row + wrap_any(x + 2 - k, nx));
      gc += DCX[q];
      gx += DWX[q];
    }
  }
  if (y >= 3 && y + 4 <= ny) {  // faces y - 3 .. y + 2 all exist, no ghost lands here
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const unsigned q = k * n + (unsigned)(node + (2 - k) * nx);
      gc += DCY[q];
      gy += DWY[q];
    }
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int yf = y + 2 - k;
      if (yf >= 0 && yf <= ny - 2) {
        const unsigned q = k * n + (unsigned)(yf * nx + x);
        gc += DCY[q];
        gy += DWY[q];
      }
    }
    // ghost stencil positions folded onto the mirror rows (p = -1 -> 0, -2 -> 1, ny -> ny-1,
    // ny+1 -> ny-2); face yf has position p at k = p - yf + 2
    auto ghost = [&](int yf, int k) {
      const unsigned q = k * n + (unsigned)(yf * nx + x);
      gc += DCY[q];
      gy -= DWY[q];
    };
    if (y == 0) {
      ghost(0, 1);
      if (ny - 2 >= 1) ghost(1, 0);
    }
    if (y == 1) ghost(0, 0);
    if (y == ny - 1) {
      ghost(ny - 2, 4);
      if (ny - 3 >= 0) ghost(ny - 3, 5);
    }
    if (y == ny - 2) ghost(ny - 2, 5);
  }
  const T lam_here = lscale * lsrc[node];
  v = lam_here + gc;
  if (STAGE == 1) v += T(1.0 / 3.0) * f.mu[node] + T(0.75) * f.lc2[node];
  if (y == 0) {
    v += (STAGE == 3 ? T(2.0 / 3.0) : T(1.0 / 6.0)) * vs;  // deposit b-weight
    v -= vs * lam_here;                                    // floor face
  }
}

// Stages 3 and 2: write lc2 / lc1 and lambda(u) (written by stage 3, accumulated by 2).
template <typename T, int STAGE>
__global__ void __launch_bounds__(kAdjThreads) adj_gather_kernel(Args<T> a, AdjFields<T> f, FaceRecords<T> fr) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= a.nx) return;
  const long long n = a.n;
  const long long node = (long long)y * a.nx + x;
  T v, gx, gy;
  gather_node<T, STAGE>(a, f, fr, x, y, v, gx, gy);
  (STAGE == 3 ? f.lc2 : f.lc1)[node] = v;
  if (STAGE == 3) {
    f.lam_u[node] = gx;
    f.lam_u[n + node] = gy;
  } else {
    f.lam_u[node] += gx;
    f.lam_u[n + node] += gy;
  }
}

// State before the last reverse step: J does not depend on c^N or the final populations.
template <typename T>
__global__ void adj_init_kernel(AdjFields<T> f, long long n, int nparts) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) f.mu[k] = T(0);
  if (k < nparts) f.vs_part[k] = 0.0;
}

// dJ/dVs = sum of the per-CTA partials in index order (one block).
__global__ void adj_vs_finish_kernel(const double* part, int nparts, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x) s += part[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) tot += sh[k];
    *out = tot;
  }
}

// Adjoint of the fluid step at one node, fused with the stage-1 gather (which completes
// lambda(c^n)'s transport part lc and lambda(u) at this node).  Inputs: rho and u of step
// n as the forward step computed them (recorded), c^n, lambda of the streamed populations
// of step n+1 (natural layout lam_next[i][node]).  Outputs: lambda of the populations of
// step n (natural layout) and lambda(c^n) = lc - A lambda(F_y) in mu.  The collision
// g* = (1 - w) g + w geq(rho - 1, u) + src(u, F) and u = (j + F/2)/rho depend on the
// populations only through rho and j.
template <typename T>
__global__ void __launch_bounds__(128) adj_gather_fluid_kernel(Args<T> a, AdjFields<T> f, FaceRecords<T> fr,
                                                               const T* rho_rec, const T* lam_next, T* lam_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= a.nx) return;
  const unsigned n = (unsigned)a.n;  // 24 n < 2^31 (checked by the host)
  const D2Q9Node nd = d2q9_node(a, x, y);
  const unsigned node = nd.node;
  T lc, gx, gy;
  gather_node<T, 1>(a, f, fr, x, y, lc, gx, gy);
  const T Fx = a.bf[0], Fy = a.bf[1] - a.A * a.c[node];
  const T rho = rho_rec[node];
  const T ux = a.u[node], uy = a.u[n + node];
  const T uu = ux * ux + uy * uy;
  // adjoint of the post-collision populations: reverse streaming with bounce-back (the
  // population pushed to node + c_i, or bounced back into opp(i) here at a wall)
  T mu[9];
#pragma unroll
  for (int i = 0; i < 9; ++i)
    mu[i] = nd.behind_wall(i, +1) ? lam_next[D2Q9::opp(i) * n + node]
                                  : lam_next[i * n + (unsigned)((int)node + nd.off(i, +1))];
  T lam_drho = T(0), lux = f.lam_u[node] + gx, luy = f.lam_u[n + node] + gy, lFy = T(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const T wi = T(D2Q9::w(i));
    const T cx = T(D2Q9::cx(i)), cy = T(D2Q9::cy(i));
    const T cu = cx * ux + cy * uy, cF = cx * Fx + cy * Fy;
    const T lgeq = a.omega * mu[i], lsrc = mu[i];
    const T P = T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu;
    lam_drho += lgeq * wi * (T(1) + P);
    const T kq = lgeq * wi * rho, ks = lsrc * a.guo * wi;
    lux += kq * (T(3) * cx + T(9) * cu * cx - T(3) * ux) + ks * (T(-3) * Fx + T(9) * cx * cF);
    luy += kq * (T(3) * cy + T(9) * cu * cy - T(3) * uy) + ks * (T(-3) * Fy + T(9) * cy * cF);
    lFy += ks * (T(3) * cy - T(3) * uy + T(9) * cu * cy);
  }
  // u = (j + F/2)/rho
  const T irho = T(1) / rho;
  const T ljx = lux * irho, ljy = luy * irho;
  lFy += T(0.5) * ljy;
  lam_drho -= (lux * ux + luy * uy) * irho;
  const T keep = T(1) - a.omega;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    lam_out[i * n + node] = keep * mu[i] + lam_drho + ljx * T(D2Q9::cx(i)) + ljy * T(D2Q9::cy(i));
  f.mu[node] = lc - a.A * lFy;
}

}  // namespace lw
