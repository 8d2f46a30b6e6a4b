// Reverse-mode (adjoint) kernels of the 2D coupled step, for the gradient of the
// deposited mass (Sec. 4, m_b) with respect to the initial concentration and to Vs.
//
// Forward step n (see lbm_kernels.cuh, transport_kernels.cuh):
//   u = U(g, c); g' = Stream(Collide(g, F(c)));
//   c1 = c + L(c; u); c2 = 3/4 c + 1/4 c1 + 1/4 L(c1; u); c' = 1/3 c + 2/3 c2 + 2/3 L(c2; u);
//   J += Vs sum_floor(c/6 + c1/6 + 2 c2/3).
// Its adjoint, given lambda(c'), lambda(g') and the recomputed u, c1, c2, runs the three
// transport stages backwards (adj_stage_kernel scatters the face-flux derivatives with
// atomics: Jacobian-transpose of L with respect to its input and to u, including the
// WENO5-JS nonlinear weights), then the fluid step backwards (adj_fluid_kernel: reverse
// streaming with bounce-back, transpose of the BGK-Guo collision, the velocity chain
// u = (j + F/2)/rho, and the buoyancy F_y = -A c).  Lax-Friedrichs alpha is a fixed
// parameter here (the caller sets lf_alpha), so d/dVs holds alpha fixed.
#pragma once
#include "common.cuh"
#include "lattice.cuh"
#include "lbm_kernels.cuh"

namespace lw {

template <typename T>
struct AdjArgs {
  const T* cs;    // stage input field (c, c1 or c2)
  const T* lamL;  // adjoint of the stage rate L(cs)
  T* lam_cs;      // adjoint of cs (accumulated)
  T* lam_u;       // adjoint of u, [2][n] (accumulated)
  double* lam_vs; // adjoint of Vs (accumulated)
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

// Adjoint of one stage's rate L(cs; u): one thread per node handles the face on its +
// side along x and along y (and the floor face below row 0).
template <typename T>
__global__ void __launch_bounds__(128) adj_stage_kernel(Args<T> a, AdjArgs<T> j) {
  __shared__ double sh[4];
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int nx = a.nx, ny = a.ny;
  double vs_acc = 0.0;
  if (x < nx) {
    const long long n = a.n;
    const long long node = (long long)y * nx + x;
    const T alpha = a.alpha, ia = a.inv_alpha;
    for (int d = 0; d < 2; ++d) {
      const bool vert = d == 1;
      if (vert && y == ny - 1) continue;  // lid: no flux
      // adjoint of the face flux F_{+1/2}: L_node -= F, L_next += F
      long long next;
      if (!vert)
        next = (long long)y * nx + (x + 1 == nx ? 0 : x + 1);
      else
        next = node + nx;
      const T lamF = j.lamL[next] - j.lamL[node];
      // stencil k = -2..3 along d: node index, ghost flag
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
        cv[k + 2] = j.cs[idx[k + 2]];
        T ud = a.u[(long long)d * n + idx[k + 2]];
        if (g) ud = -ud;
        wv[k + 2] = (ud - (vert ? a.vs : T(0))) * ia;  // w / alpha
      }
      T hp[5], hm[5], gp[5], gm[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        hp[k] = T(0.5) * (wv[k] + T(1)) * cv[k];       // h+ at stencil k-2 (k = 0..4)
        hm[k] = T(0.5) * (wv[5 - k] - T(1)) * cv[5 - k];  // h- mirrored: stencil 3..-1
      }
      weno5_value_grad<T>(hp, gp);
      weno5_value_grad<T>(hm, gm);
      // F = alpha (v+ + v-) + kappa (c_0 - c_1): dF/dh = alpha dv; dh/dc = (w/alpha +- 1)/2,
      // dh/dw_phys = c / (2 alpha) -> dF/dw_phys = dv c / 2
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
        atomic_add_t(j.lam_cs + idx[k], lamF * dFdc[k]);
        const T du = ghost[k] ? -dFdw[k] : dFdw[k];  // w = +-u - Vs (vertical) or u (horizontal)
        atomic_add_t(j.lam_u + (long long)d * n + idx[k], lamF * du);
        if (vert) vs_acc -= (double)(lamF * dFdw[k]);
      }
    }
    if (y == 0) {  // floor face below row 0: F = -Vs c_0, enters L_0 with +
      const T lam = j.lamL[node];
      atomic_add_t(j.lam_cs + node, -a.vs * lam);
      vs_acc -= (double)(j.cs[node] * lam);
    }
  }
  // block sum of the Vs adjoint, one double atomic per block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vs_acc += __shfl_down_sync(0xffffffffu, vs_acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = vs_acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    if (s != 0.0) atomicAdd(j.lam_vs, s);
  }
}

// Elementwise combinations of the adjoint fields (n nodes):
// out = ca * A + cb * B (+ floor term: fl on the first nfloor nodes)
template <typename T>
__global__ void adj_axpby_kernel(T* out, const T* A, T ca, const T* B, T cb, long long n, long long nfloor, T fl) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  T v = ca * A[k];
  if (B) v += cb * B[k];
  if (k < nfloor) v += fl;
  out[k] = v;
}

// Deposit's direct dependence on Vs: lam_vs += sum_floor(c/6 + c1/6 + 2 c2/3)
template <typename T>
__global__ void adj_deposit_vs_kernel(const T* c, const T* c1, const T* c2, long long nfloor, double* lam_vs) {
  __shared__ double sh[8];
  double acc = 0.0;
  for (long long k = threadIdx.x; k < nfloor; k += blockDim.x)
    acc += ((double)c[k] + (double)c1[k]) / 6.0 + (double)c2[k] * (2.0 / 3.0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    *lam_vs += s;
  }
}

// Adjoint of the fluid step at each node.  Inputs: the populations of step n (AA layout
// with its parity), c^n, lambda of the streamed populations of step n+1 (natural layout
// lam_next[i][node]), lambda(u) from the transport.  Outputs: lambda of the populations
// of step n (natural layout), and -A lambda(F_y) added to lambda(c^n).
template <typename T, int PARITY>
__global__ void __launch_bounds__(128) adj_fluid_kernel(Args<T> a, const T* lam_next, const T* lam_u, T* lam_out,
                                                        T* lam_c) {
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
  T lam_drho = T(0), lux = lam_u[node], luy = lam_u[n + node], lFx = T(0), lFy = T(0);
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
    lFx += ks * (T(3) * cx - T(3) * ux + T(9) * cu * cx);
    lFy += ks * (T(3) * cy - T(3) * uy + T(9) * cu * cy);
  }
  // u = (j + F/2)/rho
  const T ljx = lux / rho, ljy = luy / rho;
  lFx += lux / (T(2) * rho);
  lFy += luy / (T(2) * rho);
  lam_drho -= (lux * ux + luy * uy) / rho;
  const T keep = T(1) - a.omega;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    lam_out[i * n + node] = keep * mu[i] + lam_drho + ljx * T(D2Q9::cx(i)) + ljy * T(D2Q9::cy(i));
  lam_c[node] += -a.A * lFy;
  (void)lFx;
}

}  // namespace lw
