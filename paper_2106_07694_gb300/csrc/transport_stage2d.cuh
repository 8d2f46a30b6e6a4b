// 2D transport (FP32; FP64 in the validation build): one SSP-RK3 stage of the WENO5 + diffusion + settling update of c
// (steps a4..a8) as a row sweep, the 2D counterpart of the 3D stage kernels.
//
// A CTA owns a strip of 128 columns and a segment of rows and sweeps it upward.  At row
// k it stages the x-split fluxes of the stage input on the strip plus a 3-column halo
// in shared memory (prefetched one row ahead), computes the left x face of every column
// (the strip's right edge face by one lane of warp 0), and the upper y face of its own
// column from a ring of y-split fluxes running three rows ahead; the lower y face is
// carried from the previous row.  Every face of the stage is computed once.  The ring
// holds six rows, each stored twice (slots r and r + 6), so a face reads its six rows
// from one base slot without wrap-around arithmetic.  Small shared-memory footprint
// (about 21 KB), so many CTAs share an SM.  Three launches make
// a step (the stage-3 kernel also folds the floor deposit); c1 and c2 go through L2/HBM.
#pragma once
#include "common.cuh"
#include "transport_sweep2d.cuh"  // weno5_face_value, face_flux_x

namespace lw {

constexpr int kS2T = 128;             // columns per CTA (threads)
constexpr int kS2h = 3;               // stencil radius
constexpr int kS2X = kS2T + 2 * kS2h;
constexpr int kS2r = 6;               // y ring depth (rows k-2 .. k+3), stored twice

template <typename T>
struct Stage2dSmem {
  T xp[kS2X];  // x-split h+/alpha of the current row (strip + halo)
  T xm[kS2X];
  T c[kS2X];   // stage input value of the current row
  T yp[2 * kS2r][kS2T];  // y-split ring of each column; slot r and r + 6 hold the same
  T ym[2 * kS2r][kS2T];  // row, so the six rows of a face are read without wrap-around
  T cy[2 * kS2r][kS2T];  // stage input value ring of each column, stored the same way
  T fx[kS2T + 1];    // left x faces (+ right edge)
};

template <typename T>
struct Stage2dParamsT {
  const T* cin;  // stage input (c, c1 or c2)
  T* cout;       // stage output (c1, c2 or c in place)
  int H;         // rows per segment
};
using Stage2dParams = Stage2dParamsT<float>;

// Body of the stage kernel for strip bx, segment by; `strips` = number of strips (the
// floor CTAs that fold the deposit).  SCHEME: transport-scheme variant bits (kSchemeWeno3,
// kSchemeSignSplit; 0 = Lax-Friedrichs WENO5), see face_flux_scheme.  T = float (the
// production path) or double (the validation build: the same sweep in FP64).
template <int STAGE, bool SUGAR = false, int SCHEME = 0, typename T = float>
__device__ __forceinline__ void stage2d_body(const Args<T>& a, const Stage2dParamsT<T>& sp, int bx, int by,
                                             int strips) {
  __shared__ __align__(16) Stage2dSmem<T> S;
  const int t = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  const int x0 = bx * kS2T;
  const int y0 = by * sp.H, y1 = min(ny, y0 + sp.H);
  const int X = (x0 + t) % nx;
  const bool out = x0 + t < nx;
  const T inv_alpha = a.inv_alpha, vs_a = a.vs * a.inv_alpha, alpha = a.alpha, kappa = a.kappa;
  const T* __restrict__ cin = sp.cin;
  const T* __restrict__ ux = a.u;
  const T* __restrict__ uy = a.u + a.n;

  // staging positions of this thread in the strip + halo row (fixed for the sweep)
  const int j1 = t + kS2T;  // second position, only for the 6 halo columns
  const unsigned gx1 = (unsigned)((x0 - kS2h + j1 + 4 * nx) % nx);
  const unsigned gxs = (unsigned)((x0 - kS2h + t + 4 * nx) % nx);
  const bool has2 = j1 < kS2X;
  T p0c = T(0), p0u = T(0), p1c = T(0), p1u = T(0);
  auto fetch_row = [&](int k) {
    if (k >= y1) return;
    const unsigned row = (unsigned)k * (unsigned)nx;
    p0c = __ldg(cin + row + gxs);
    p0u = __ldg(ux + row + gxs);
    if (has2) {
      p1c = __ldg(cin + row + gx1);
      p1u = __ldg(ux + row + gx1);
    }
  };
  // own column, row l (ghost rows reflect): value and scaled vertical velocity
  T qc = T(0), qw = T(0), qn = T(0);
  auto col_fetch = [&](int l) {
    const bool ghost = l < 0 || l >= ny;
    const int lr = l < 0 ? -1 - l : (l >= ny ? 2 * ny - 1 - l : l);
    const unsigned k = (unsigned)lr * (unsigned)nx + X;
    qc = __ldg(cin + k);
    const T u = __ldg(uy + k);
    // with sugar the settling velocity of the node (a ghost reads its mirror's) is Vs (1 - ks S)
    const T vsa = SUGAR ? vs_a * fma_t(-a.ks, __ldg(a.S + k), T(1)) : vs_a;
    qw = fma_t(ghost ? -u : u, inv_alpha, -vsa);
  };
  constexpr bool SIGN = (SCHEME & kSchemeSignSplit) != 0;
  auto col_put = [&](int slot) {
    const T h = T(0.5) * qc, p = SIGN ? qw * qc : fma_t(qw, h, h), m = SIGN ? qw : fma_t(qw, h, -h);
    S.yp[slot][t] = p;
    S.yp[slot + kS2r][t] = p;
    S.ym[slot][t] = m;
    S.ym[slot + kS2r][t] = m;
    S.cy[slot][t] = qc;
    S.cy[slot + kS2r][t] = qc;
  };
  auto cn_fetch = [&](int k) {
    if (STAGE > 1 && k < y1) qn = a.c[(unsigned)k * (unsigned)nx + X];
  };

  const int kb = y0 == 0 ? 0 : y0 - 1;  // first row: y0, or the priming row below it
  for (int l = kb - 2; l < kb + 3; ++l) {
    col_fetch(l);
    col_put(((l % kS2r) + kS2r) % kS2r);
  }
  col_fetch(kb + 3);
  int slot = (kb + 3) % kS2r;  // ring slot of row k + 3
  fetch_row(kb);
  cn_fetch(kb);
  T carry = T(0);
  double dep = 0.0;  // stage 3, floor row: this column's Vs-free deposit term

  for (int k = kb; k < y1; ++k) {
    const bool prime = k < y0;
    // ---- stage row k (prefetched), own column three rows ahead
    {
      const T h0 = T(0.5) * p0c, w0 = p0u * inv_alpha;
      S.c[t] = p0c;
      S.xp[t] = SIGN ? w0 * p0c : fma_t(w0, h0, h0);
      S.xm[t] = SIGN ? w0 : fma_t(w0, h0, -h0);
      if (has2) {
        const T h1 = T(0.5) * p1c, w1 = p1u * inv_alpha;
        S.c[j1] = p1c;
        S.xp[j1] = SIGN ? w1 * p1c : fma_t(w1, h1, h1);
        S.xm[j1] = SIGN ? w1 : fma_t(w1, h1, -h1);
      }
    }
    fetch_row(k + 1);
    col_put(slot);
    col_fetch(k + 4);
    const T cn_here = qn;
    cn_fetch(k + 1);
    __syncthreads();

    // ---- faces: left x face of this column (and the strip's right edge), upper y face
    if (!prime) {
      if constexpr (SCHEME == 0) {
        S.fx[t] = face_flux_x(S.xp[t], S.xp[t + 1], S.xp[t + 2], S.xp[t + 3], S.xp[t + 4], S.xm[t + 5],
                              S.xm[t + 4], S.xm[t + 3], S.xm[t + 2], S.xm[t + 1], alpha, kappa, S.c[t + kS2h - 1],
                              S.c[t + kS2h]);
        if (t == 0) {
          const int e = kS2T;
          S.fx[e] = face_flux_x(S.xp[e], S.xp[e + 1], S.xp[e + 2], S.xp[e + 3], S.xp[e + 4], S.xm[e + 5],
                                S.xm[e + 4], S.xm[e + 3], S.xm[e + 2], S.xm[e + 1], alpha, kappa, S.c[e + kS2h - 1],
                                S.c[e + kS2h]);
        }
      } else {
        auto xface = [&](int j) {  // face between staging positions j + 2 and j + 3
          T p[6], m[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            p[q] = S.xp[j + q];
            m[q] = S.xm[j + q];
          }
          return face_flux_scheme<SCHEME>(p, m, alpha, kappa, S.c[j + kS2h - 1], S.c[j + kS2h]);
        };
        S.fx[t] = xface(t);
        if (t == 0) S.fx[kS2T] = xface(kS2T);
      }
    }
    const int rb = slot == kS2r - 1 ? 0 : slot + 1;  // ring slot of row k - 2 (= that of row k + 4)
    const T chere = S.cy[rb + 2][t], cnext = S.cy[rb + 3][t];
    T fup = T(0);
    if (k != ny - 1) {
      const T* P = &S.yp[rb][t];
      const T* M = &S.ym[rb][t];
      if constexpr (SCHEME == 0) {
        fup = face_flux_x(P[0], P[kS2T], P[2 * kS2T], P[3 * kS2T], P[4 * kS2T], M[5 * kS2T], M[4 * kS2T],
                          M[3 * kS2T], M[2 * kS2T], M[kS2T], alpha, kappa, chere, cnext);
      } else {
        T p[6], m[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          p[q] = P[q * kS2T];
          m[q] = M[q * kS2T];
        }
        fup = face_flux_scheme<SCHEME>(p, m, alpha, kappa, chere, cnext);
      }
    }
    __syncthreads();

    // ---- divergence and the Shu-Osher combination of this stage
    if (!prime) {
      const T vs_floor = SUGAR && k == 0 ? a.vs * fma_t(-a.ks, __ldg(a.S + X), T(1)) : a.vs;
      const T fdn = k == 0 ? -vs_floor * chere : carry;
      const T L = S.fx[t] - S.fx[t + 1] + fdn - fup;
      if (out) {
        T v;
        if (STAGE == 1) {
          v = chere + L;
        } else if (STAGE == 2) {
          v = fma_t(T(0.75), cn_here, T(0.25) * (chere + L));
        } else {
          const T s = chere + L;
          v = fma_t(T(1) / T(3), cn_here - s, s);
        }
        sp.cout[(unsigned)k * (unsigned)nx + X] = v;
        if (STAGE == 3) {
          report_status(a.status, !isfinite(v));
          if (k == 0) {  // RK3 b-weights of the floor flux: c^n/6 + c1/6 + 2 c2/3
            dep = ((double)cn_here + (double)a.c1[X]) * (1.0 / 6.0) + (double)chere * (2.0 / 3.0);
            if (SUGAR) dep *= (double)vs_floor;  // Vs(S) per floor node, no common factor
          }
        }
      }
    }
    carry = fup;
    slot = rb;
  }

  // stage 3: the CTAs holding the floor row fold the deposit of this step (FP64,
  // fixed order: warp shuffles, then the last CTA sums the per-CTA partials)
  if (STAGE == 3 && y0 == 0) {
    __shared__ double red[kS2T / 32];
    __shared__ bool last;
    double v = dep;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
      double s2 = 0.0;
      for (int w = 0; w < kS2T / 32; ++w) s2 += red[w];
      a.partials[bx] = SUGAR ? s2 : s2 * (double)a.vs;
      __threadfence();
      last = atomicAdd(a.ticket, 1u) == (unsigned)strips - 1;
    }
    __syncthreads();
    if (last && t == 0) {
      __threadfence();
      const volatile double* vp = a.partials;
      double tot = 0.0;
      for (int b = 0; b < strips; ++b) tot += vp[b];
      a.scalars[0] += tot;
      *a.ticket = 0u;
    }
  }
}

template <int STAGE, bool SUGAR = false, int SCHEME = 0, typename T = float>
__global__ void __launch_bounds__(kS2T) rk_stage2d_kernel(Args<T> a, Stage2dParamsT<T> sp) {
  stage2d_body<STAGE, SUGAR, SCHEME, T>(a, sp, blockIdx.x, blockIdx.y, gridDim.x);
}

inline int stage2d_rows(int nx, int ny, int sm_count, int override_rows) {
  if (override_rows > 0) return min(override_rows, ny);
  const long long strips = (nx + kS2T - 1) / kS2T;
  // the longest segment (fewest priming rows) that still gives about 8.5 CTAs per SM;
  // measured best: 16 rows on 2048 x 4096 and 1024 x 2048, 3-4 on 512 x 1024, 2 on 256 x 512
  const int cand[] = {16, 12, 8, 6, 4, 3, 2};
  for (int H : cand) {
    if (strips * ((ny + H - 1) / H) >= 17LL * sm_count / 2) return min(H, ny);
  }
  return min(2, ny);
}

// The stage kernel of the handle's transport scheme (runtime field) as a compile-time variant.
template <int STAGE, bool SUGAR, typename T>
inline void launch_stage2d_scheme(const Args<T>& a, const Stage2dParamsT<T>& sp, dim3 grid, cudaStream_t s) {
  switch (a.scheme) {
    case kSchemeWeno3:
      rk_stage2d_kernel<STAGE, SUGAR, kSchemeWeno3, T><<<grid, kS2T, 0, s>>>(a, sp);
      break;
    case kSchemeSignSplit:
      rk_stage2d_kernel<STAGE, SUGAR, kSchemeSignSplit, T><<<grid, kS2T, 0, s>>>(a, sp);
      break;
    case kSchemeWeno3 | kSchemeSignSplit:
      rk_stage2d_kernel<STAGE, SUGAR, kSchemeWeno3 | kSchemeSignSplit, T><<<grid, kS2T, 0, s>>>(a, sp);
      break;
    default:
      rk_stage2d_kernel<STAGE, SUGAR, 0, T><<<grid, kS2T, 0, s>>>(a, sp);
  }
}

template <int STAGE, typename T>
inline cudaError_t launch_stage2d(const Args<T>& a, const T* cin, T* cout, int H, cudaStream_t s) {
  Stage2dParamsT<T> sp;
  sp.cin = cin;
  sp.cout = cout;
  sp.H = H;
  const dim3 grid((a.nx + kS2T - 1) / kS2T, (a.ny + H - 1) / H);
  if (a.S)
    launch_stage2d_scheme<STAGE, true, T>(a, sp, grid, s);
  else
    launch_stage2d_scheme<STAGE, false, T>(a, sp, grid, s);
  return cudaGetLastError();
}

}  // namespace lw
