// Reverse-mode (adjoint) kernels of the 2D coupled step, for the gradient of the
// deposited mass (Sec. 4, m_b) with respect to the initial concentration and to Vs.
//
// Forward step n (lbm_kernels.cuh, transport kernels):
//   u = U(g, c); g' = Stream(Collide(g, F(c)));
//   c1 = c + L(c; u); c2 = 3/4 c + 1/4 c1 + 1/4 L(c1; u); c' = 1/3 c + 2/3 c2 + 2/3 L(c2; u);
//   J += Vs sum_floor(c/6 + c1/6 + 2 c2/3).
// Given lambda(c') and lambda(g') and the stored u, c1, c2 of the step, one reverse step
// is four launches: the three transport stages backwards (adj_stage_kernel<3,2,1>:
// Jacobian-transpose of L with respect to its input and to u, WENO5-JS nonlinear weights
// included, scattered with atomics), then the fluid step backwards (adj_fluid_kernel:
// reverse streaming with bounce-back, transpose of the BGK-Guo collision, the velocity
// chain u = (j + F/2)/rho, the buoyancy F_y = -A c), which also sets up the accumulators
// of the next reverse step.  The Lax-Friedrichs alpha is a fixed parameter here (the
// caller sets lf_alpha), so d/dVs holds alpha fixed.
#pragma once
#include "common.cuh"
#include "lattice.cuh"
#include "lbm_kernels.cuh"

namespace lw {

// Adjoint fields of one reverse step.  mu = lambda(c^{n+1}) (read by stage 3, then
// overwritten with lambda(c^n) by the fluid kernel); lc2, lc1, lc accumulate lambda of
// c2, c1 and c^n; lam_u = lambda(u) [2][n], zeroed again by the fluid kernel.
template <typename T>
struct AdjFields {
  T* mu;
  T* lc2;
  T* lc1;
  T* lc;
  T* lam_u;
  double* lam_vs;
};

// WENO5-JS face value of the scaled values v[0..4] (upwind side first) and its partial
// derivatives dv[0..4]: sum_k w_k dq_k/dv_j + sum_m (q_m - val) w_m (-2/(eps+beta_m)) dbeta_m/dv_j.
template <typename T>
__device__ __forceinline__ T weno5_value_grad(const T (&v)[5], T (&dv)[5]) {
  const T a = v[0], b = v[1], c = v[2], d = v[3], e = v[4];
  const T eps = T(1e-6);
  const T q0 = (T(2) * a - T(7) * b + T(11) * c) / T(6);
  const T q1 = (-b + T(5) * c + T(2) * d) / T(6);
  const T q2 = (T(2) * c + T(5) * d - e) / T(6);
  const T s0 = a - T(2) * b + c, s1 = b - T(2) * c + d, s2 = c - T(2) * d + e;
  const T t0 = a - T(4) * b + T(3) * c, t1 = b - d, t2 = T(3) * c - T(4) * d + e;
  const T A0 = eps + T(13.0 / 12.0) * s0 * s0 + T(0.25) * t0 * t0;
  const T A1 = eps + T(13.0 / 12.0) * s1 * s1 + T(0.25) * t1 * t1;
  const T A2 = eps + T(13.0 / 12.0) * s2 * s2 + T(0.25) * t2 * t2;
  const T a0 = T(0.1) / (A0 * A0), a1 = T(0.6) / (A1 * A1), a2 = T(0.3) / (A2 * A2);
  const T inv = T(1) / (a0 + a1 + a2);
  const T w0 = a0 * inv, w1 = a1 * inv, w2 = a2 * inv;
  const T val = w0 * q0 + w1 * q1 + w2 * q2;
  // weight-sensitivity factors r_m = (q_m - val) w_m (-2 / A_m)
  const T r0 = (q0 - val) * w0 * (T(-2) / A0);
  const T r1 = (q1 - val) * w1 * (T(-2) / A1);
  const T r2 = (q2 - val) * w2 * (T(-2) / A2);
  // dbeta_m/dv = 13/6 s_m ds_m + 1/2 t_m dt_m
  const T u0 = T(13.0 / 6.0) * s0, p0 = T(0.5) * t0;
  const T u1 = T(13.0 / 6.0) * s1, p1 = T(0.5) * t1;
  const T u2 = T(13.0 / 6.0) * s2, p2 = T(0.5) * t2;
  dv[0] = w0 * T(1.0 / 3.0) + r0 * (u0 + p0);
  dv[1] = w0 * T(-7.0 / 6.0) + w1 * T(-1.0 / 6.0) + r0 * (T(-2) * u0 - T(4) * p0) + r1 * (u1 + p1);
  dv[2] = w0 * T(11.0 / 6.0) + w1 * T(5.0 / 6.0) + w2 * T(1.0 / 3.0) + r0 * (u0 + T(3) * p0) +
          r1 * (T(-2) * u1) + r2 * (u2 + T(3) * p2);
  dv[3] = w1 * T(1.0 / 3.0) + w2 * T(5.0 / 6.0) + r1 * (u1 - p1) + r2 * (T(-2) * u2 - T(4) * p2);
  dv[4] = w2 * T(-1.0 / 6.0) + r2 * (u2 + p2);
  return val;
}

__device__ __forceinline__ void atomic_add_t(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_t(double* p, double v) { atomicAdd(p, v); }

// Adjoint of SSP-RK3 stage STAGE of the transport, one node per thread.
//   STAGE 3: c' = 1/3 c + 2/3 (c2 + L(c2)):  lamL = 2/3 mu, scatter into lc2;
//   STAGE 2: c2 = 3/4 c + 1/4 (c1 + L(c1)):  lamL = 1/4 lc2, scatter into lc1; direct
//            terms lc1 += 1/4 lc2, lc += 3/4 lc2;
//   STAGE 1: c1 = c + L(c):                  lamL = lc1, scatter into lc; lc += lc1.
// The thread of node i handles the faces on its + side along x and along y: for each, the
// adjoint of the face flux lamF = lamL[i+1] - lamL[i] times the flux derivatives with
// respect to the six stencil values of c and of the velocity, added with atomics (the
// node's own entry merged into one add).  The floor face below row 0 (F = -Vs c) and the
// deposit's RK3 b-weights (c/6 + c1/6 + 2 c2/3 on the floor, times Vs) give the Vs adjoint.
template <typename T, int STAGE>
__global__ void __launch_bounds__(128) adj_stage_kernel(Args<T> a, AdjFields<T> f) {
  __shared__ double sh[4];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int nx = a.nx, ny = a.ny;
  const T* __restrict__ cs = STAGE == 3 ? a.c2 : (STAGE == 2 ? a.c1 : a.c);
  const T* lsrc = STAGE == 3 ? f.mu : (STAGE == 2 ? f.lc2 : f.lc1);
  const T lscale = STAGE == 3 ? T(2.0 / 3.0) : (STAGE == 2 ? T(0.25) : T(1));
  T* lam_cs = STAGE == 3 ? f.lc2 : (STAGE == 2 ? f.lc1 : f.lc);
  double vs_acc = 0.0;
  if (x < nx) {
    const long long n = a.n;
    const long long node = (long long)y * nx + x;
    const T alpha = a.alpha, ia = a.inv_alpha;
    const T lam_here = lscale * lsrc[node];
    T own = T(0);  // everything this thread adds to lam_cs[node]
    if (STAGE == 2) {
      own = lam_here;                 // 1/4 lc2: c1 enters c2 directly
      f.lc[node] += T(3) * lam_here;  // 3/4 lc2: c^n enters c2 (no other writer of lc here)
    } else if (STAGE == 1) {
      own = lam_here;                 // lc1: c^n enters c1 directly
    }
    for (int d = 0; d < 2; ++d) {
      const bool vert = d == 1;
      if (vert && y == ny - 1) continue;  // lid: no flux
      const long long next = vert ? node + nx : (long long)y * nx + (x + 1 == nx ? 0 : x + 1);
      const T lamF = lscale * lsrc[next] - lam_here;  // F_{+1/2} leaves node, enters next
      long long idx[6];
      bool ghost[6];
      T cv[6], wv[6];
#pragma unroll
      for (int k = -2; k <= 3; ++k) {
        int p = (vert ? y : x) + k;
        bool g = false;
        if (vert) {
          if (p < 0) {
            p = -1 - p;
            g = true;
          } else if (p >= ny) {
            p = 2 * ny - 1 - p;
            g = true;
          }
          idx[k + 2] = (long long)p * nx + x;
        } else {
          p = p < 0 ? p + nx : (p >= nx ? p - nx : p);
          idx[k + 2] = (long long)y * nx + p;
        }
        ghost[k + 2] = g;
        cv[k + 2] = cs[idx[k + 2]];
        T ud = a.u[(long long)d * n + idx[k + 2]];
        if (g) ud = -ud;
        wv[k + 2] = (ud - (vert ? a.vs : T(0))) * ia;  // w / alpha
      }
      T hp[5], hm[5], gp[5], gm[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        hp[k] = T(0.5) * (wv[k] + T(1)) * cv[k];          // h+ at stencil k-2
        hm[k] = T(0.5) * (wv[5 - k] - T(1)) * cv[5 - k];  // h- mirrored: stencil 3..-1
      }
      weno5_value_grad<T>(hp, gp);
      weno5_value_grad<T>(hm, gm);
      // F = alpha (v+ + v-) + kappa (c_0 - c_1): dF/dh = alpha dv; dh/dc = (w/alpha +- 1)/2,
      // dF/dw_phys = dv c / 2
      T dFdc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
      T dFdw[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        dFdc[k] += alpha * gp[k] * T(0.5) * (wv[k] + T(1));
        dFdw[k] += gp[k] * T(0.5) * cv[k];
        dFdc[5 - k] += alpha * gm[k] * T(0.5) * (wv[5 - k] - T(1));
        dFdw[5 - k] += gm[k] * T(0.5) * cv[5 - k];
      }
      dFdc[2] += a.kappa;
      dFdc[3] -= a.kappa;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        if (k == 2)  // the node itself (never a ghost: y is inside the lattice)
          own += lamF * dFdc[k];
        else
          atomic_add_t(lam_cs + idx[k], lamF * dFdc[k]);
        const T du = ghost[k] ? -dFdw[k] : dFdw[k];  // w = +-u - Vs (vertical) or u (horizontal)
        atomic_add_t(f.lam_u + (long long)d * n + idx[k], lamF * du);
        if (vert) vs_acc -= (double)(lamF * dFdw[k]);
      }
    }
    if (y == 0) {
      own -= a.vs * lam_here;  // floor face below row 0: F = -Vs c_0 enters L_0 with +
      vs_acc -= (double)(cs[node] * lam_here);
      vs_acc += (double)cs[node] * (STAGE == 3 ? 2.0 / 3.0 : 1.0 / 6.0);  // deposit b-weights
    }
    atomic_add_t(lam_cs + node, own);
  }
  // block sum of the Vs adjoint, one double atomic per block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vs_acc += __shfl_down_sync(0xffffffffu, vs_acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = vs_acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    if (s != 0.0) atomicAdd(f.lam_vs, s);
  }
}

// Seed the accumulators of a reverse step at node k from m = lambda(c') there: the
// direct terms 2/3 m (into lc2) and 1/3 m (into lc), and the floor terms of the deposit.
template <typename T>
__device__ __forceinline__ void adj_seed(const AdjFields<T>& f, long long k, bool floor, T m, T vs) {
  f.lc2[k] = T(2.0 / 3.0) * m + (floor ? T(2.0 / 3.0) * vs : T(0));
  f.lc1[k] = floor ? vs / T(6) : T(0);
  f.lc[k] = T(1.0 / 3.0) * m + (floor ? vs / T(6) : T(0));
}

// State before the last reverse step: J does not depend on c^N or the final populations,
// so mu = 0 and lambda(u) = 0.
template <typename T>
__global__ void adj_init_kernel(AdjFields<T> f, long long n, int nx, T vs) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  f.mu[k] = T(0);
  adj_seed<T>(f, k, k < nx, T(0), vs);
  f.lam_u[k] = T(0);
  f.lam_u[n + k] = T(0);
  if (k == 0) *f.lam_vs = 0.0;
}

// Adjoint of the fluid step at each node.  Inputs: the populations of step n (AA layout
// with its parity), c^n, lambda of the streamed populations of step n+1 (natural layout
// lam_next[i][node]), lambda(u) and the transport part of lambda(c^n) in lc.  Outputs:
// lambda of the populations of step n (natural layout) and lambda(c^n) = lc - A
// lambda(F_y) in mu; then seeds lc2, lc1, lc for the step before and zeroes lambda(u).
template <typename T, int PARITY>
__global__ void __launch_bounds__(128) adj_fluid_kernel(Args<T> a, AdjFields<T> f, const T* lam_next,
                                                        T* lam_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= a.nx) return;
  const long long n = a.n;
  const long long node = (long long)y * a.nx + x;
  T g[9];
  load_populations<D2Q9, T, PARITY>(a, x, y, 0, node, g);
  T drho = T(0), jx = T(0), jy = T(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    drho += g[i];
    jx += D2Q9::cx(i) * g[i];
    jy += D2Q9::cy(i) * g[i];
  }
  const T Fx = a.bf[0], Fy = a.bf[1] - a.A * a.c[node];
  const T rho = T(1) + drho;
  const T ux = (jx + T(0.5) * Fx) / rho, uy = (jy + T(0.5) * Fy) / rho;
  const T uu = ux * ux + uy * uy;
  // adjoint of the post-collision populations: reverse streaming with bounce-back
  T mu[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    long long dst;
    if (neighbour<D2Q9>(i, +1, x, y, 0, a.nx, a.ny, 1, a.walls != 0, dst))
      mu[i] = lam_next[i * n + dst];
    else
      mu[i] = lam_next[D2Q9::opp(i) * n + node];
  }
  // collision g* = (1 - w) g + w geq(drho, u) + src(u, F)
  T lam_drho = T(0), lux = f.lam_u[node], luy = f.lam_u[n + node], lFy = T(0);
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
  const T ljx = lux / rho, ljy = luy / rho;
  lFy += luy / (T(2) * rho);
  lam_drho -= (lux * ux + luy * uy) / rho;
  const T keep = T(1) - a.omega;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    lam_out[i * n + node] = keep * mu[i] + lam_drho + ljx * T(D2Q9::cx(i)) + ljy * T(D2Q9::cy(i));
  const T lam_c = f.lc[node] - a.A * lFy;
  f.mu[node] = lam_c;
  adj_seed<T>(f, node, y == 0, lam_c, a.vs);
  f.lam_u[node] = T(0);
  f.lam_u[n + node] = T(0);
}

}  // namespace lw
