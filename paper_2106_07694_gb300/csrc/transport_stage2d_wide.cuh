// 2D FP32 transport with four adjacent columns per thread: one SSP-RK3 stage of the
// WENO5 + diffusion + settling update of c (steps a4..a8; the stage-3 kernel also folds
// the floor deposit, a9).  Default scheme (Lax-Friedrichs WENO5), no sugar; the scheme
// variants and the sugar scalar keep the one-column kernel of transport_stage2d.cuh.
//
// A CTA of kWT threads owns a strip of kWW = 4 kWT columns and a segment of rows and
// sweeps it upward.  At row k:
//  - the x-split fluxes and c of row k+1 on the strip plus one four-column halo quad on
//    each side are staged in shared memory as float4 quads, double-buffered by row
//    parity and loaded one row ahead, so the row needs a single barrier;
//  - each thread reconstructs the left x faces of its four columns from three quads of
//    h+/alpha, three of h-/alpha and two of c, sharing the first and second differences
//    of the split fluxes between the four faces; the right face of its last column is
//    its neighbour's first face, and for the strip's last column it is computed for the
//    whole segment before the sweep;
//  - the upper y face of each of its columns comes from a private ring of the y-split
//    fluxes of rows k-2 .. k+3 (one float4 per row and split half), filled three rows
//    ahead; the lower y face is carried from the previous row;
//  - stages 2 and 3 also combine with c^n at the node, copied two rows ahead by cp.async
//    into a three-row ring in shared memory (no registers held while it is in flight).
// Every face is computed once, with the arithmetic of weno5_face_value/face_flux_x, so
// the faces and the updated c are bitwise those of the one-column kernel.
#pragma once
#include "common.cuh"
#include "transport_sweep2d.cuh"  // weno5_q, weno5_face_value, face_flux_x
#include "transport_stage2d.cuh"  // Stage2dParams

namespace lw {

constexpr int kWq = 4;           // columns per thread (one float4)
constexpr int kWT = 64;          // threads per CTA
constexpr int kWW = kWq * kWT;   // columns per strip
constexpr int kWQ = kWT + 2;     // staged quads per row: the strip and one halo quad per side
constexpr int kWring = 6;        // y ring rows (k-2 .. k+3)
constexpr int kWmaxH = 64;       // longest row segment (its strip-edge faces are held in smem)
constexpr int kWminB = 1;        // CTAs per SM the register allocation must allow

struct StageWideSmem {
  float4 xp[2][kWQ];  // x-split h+/alpha of the staged row, by row parity
  float4 xm[2][kWQ];  // x-split h-/alpha
  float4 xc[2][kWQ];  // stage input c
  float4 yp[kWring][kWT];  // y-split ring of each thread's four columns
  float4 ym[kWring][kWT];
  float fx[2][kWT + 1];  // first left x face of each thread (+ the strip's right edge), by row parity
  float edge[kWmaxH];    // the strip's right-edge x face for each row of the segment
  float4 cn[3][kWT];     // stages 2, 3: c^n of rows k .. k+2 at each thread's columns (cp.async ring)
  double red[kWT / 32];
  bool last;
};

// Lax-Friedrichs split of one node: p = h+/alpha, m = h-/alpha with h = c/2, w = u/alpha.
__device__ __forceinline__ void lf_split(float c, float w, float& p, float& m) {
  const float h = 0.5f * c;
  p = fmaf(w, h, h);
  m = fmaf(w, h, -h);
}

// LD: the global-load policy (LoadNC for a launch of its own, LoadL2 inside a kernel
// whose earlier phases wrote the fields).
template <int STAGE, class LD = LoadNC>
__device__ __forceinline__ void stage2d_wide_body(StageWideSmem& S, const Args<float>& a, const Stage2dParams& sp,
                                                  int bx, int by, int strips) {
  const int t = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  const int x0 = bx * kWW;
  const int y0 = by * sp.H, y1 = min(ny, y0 + sp.H);
  const int xl = x0 + kWq * t;  // first column of this thread (past a ragged strip end: wrapped)
  const bool out = xl < nx;
  const unsigned X = (unsigned)(xl % nx);
  const float ia = a.inv_alpha, vs_a = a.vs * a.inv_alpha, alpha = a.alpha, kappa = a.kappa;
  const float* __restrict__ cin = sp.cin;
  const float* __restrict__ ux = a.u;
  const float* __restrict__ uy = a.u + a.n;

  // halo quads of the staged row: thread 0 the quad left of the strip, thread 1 the one right of it
  const bool halo = t < 2;
  const int hslot = t == 0 ? 0 : kWQ - 1;
  const unsigned hX = (unsigned)(t == 0 ? ((x0 - kWq) % nx + nx) % nx : (x0 + kWW) % nx);

  float4 Xc, Xu, Hc = make_float4(0.f, 0.f, 0.f, 0.f), Hu = Hc;
  auto fetch_x = [&](int r) {
    const unsigned row = (unsigned)r * (unsigned)nx;
    Xc = LD::v4(cin + row + X);
    Xu = LD::v4(ux + row + X);
    if (halo) {
      Hc = LD::v4(cin + row + hX);
      Hu = LD::v4(ux + row + hX);
    }
  };
  auto put_quad = [&](int b, int q, const float4& c, const float4& u) {
    float4 p, m;
    lf_split(c.x, u.x * ia, p.x, m.x);
    lf_split(c.y, u.y * ia, p.y, m.y);
    lf_split(c.z, u.z * ia, p.z, m.z);
    lf_split(c.w, u.w * ia, p.w, m.w);
    S.xp[b][q] = p;
    S.xm[b][q] = m;
    S.xc[b][q] = c;
  };
  auto stage_x = [&](int b) {
    put_quad(b, t + 1, Xc, Xu);
    if (halo) put_quad(b, hslot, Hc, Hu);
  };

  // own columns, ring row l (ghost rows reflect: c even, u_y odd); rows past the ones any
  // face reads are clamped into the lattice and never used
  float4 Rc, Ru;
  bool Rg = false;
  auto fetch_r = [&](int l) {
    Rg = l < 0 || l >= ny;
    int lr = l < 0 ? -1 - l : (l >= ny ? 2 * ny - 1 - l : l);
    lr = max(0, min(ny - 1, lr));
    const unsigned row = (unsigned)lr * (unsigned)nx;
    Rc = LD::v4(cin + row + X);
    Ru = LD::v4(uy + row + X);
  };
  // ring entries are addressed by byte offset (slot * kWT + t) * 16, rotated as the sweep advances
  auto ring_at = [&](float4 (*arr)[kWT], unsigned off) -> float4& {
    return *reinterpret_cast<float4*>(reinterpret_cast<char*>(&arr[0][0]) + off);
  };
  auto put_r = [&](unsigned off) {
    const float s = Rg ? -ia : ia;
    float4 p, m;
    lf_split(Rc.x, fmaf(Ru.x, s, -vs_a), p.x, m.x);
    lf_split(Rc.y, fmaf(Ru.y, s, -vs_a), p.y, m.y);
    lf_split(Rc.z, fmaf(Ru.z, s, -vs_a), p.z, m.z);
    lf_split(Rc.w, fmaf(Ru.w, s, -vs_a), p.w, m.w);
    ring_at(S.yp, off) = p;
    ring_at(S.ym, off) = m;
  };

  // right-edge x face of every row of the segment (full strips; a ragged strip's last
  // column takes the first face of the next, wrapped, thread)
  for (int r = t; r < y1 - y0; r += kWT) {
    float e = 0.f;
    if (x0 + kWW <= nx) {
      const unsigned row = (unsigned)(y0 + r) * (unsigned)nx;
      float P[6], M[6], C[6];
#pragma unroll
      for (int o = 0; o < 6; ++o) {
        const unsigned col = (unsigned)((x0 + kWW - 3 + o) % nx);
        C[o] = LD::s(cin + row + col);
        lf_split(C[o], LD::s(ux + row + col) * ia, P[o], M[o]);
      }
      e = face_flux_x(P[0], P[1], P[2], P[3], P[4], M[5], M[4], M[3], M[2], M[1], alpha, kappa, C[2], C[3]);
    }
    S.edge[r] = e;
  }

  const int kb = y0 == 0 ? 0 : y0 - 1;  // first row: y0, or the priming row below it
  unsigned ring[kWring];  // rows k-2 .. k+3
#pragma unroll
  for (int j = 0; j < kWring; ++j) {
    ring[j] = (unsigned)((j * kWT + t) * sizeof(float4));
    fetch_r(kb - 2 + j);
    put_r(ring[j]);
  }
  fetch_r(kb + 4);
  fetch_x(kb);
  stage_x(kb & 1);
  fetch_x(kb + 1);  // kb + 1 <= y0 < ny
  // stages 2, 3: c^n of this thread's columns, copied two rows ahead into a three-row ring
  // (each thread reads back only its own copies: a wait per thread, no barrier)
  auto fetch_cn = [&](int r) {
    if (STAGE > 1 && r < y1) cp_async16(&S.cn[r % 3][t], a.c + (unsigned)r * (unsigned)nx + X);
    if (STAGE > 1) cp_async_commit();
  };
  fetch_cn(kb);
  fetch_cn(kb + 1);
  float4 carry = make_float4(0.f, 0.f, 0.f, 0.f);
  double dep = 0.0;  // stage 3, floor row: this thread's Vs-free deposit term
  __syncthreads();

  for (int k = kb; k < y1; ++k) {
    const int b = k & 1;
    const bool prime = k < y0;
    // ---- stage row k + 1 into the other buffer, fetch row k + 2
    const float4 cnext = Xc;  // c of row k + 1 at this thread's columns
    if (k + 1 < y1) stage_x(b ^ 1);
    if (k + 1 < y1 && k + 2 < ny) fetch_x(k + 2);
    const float4 cq = S.xc[b][t + 1];  // c of row k at this thread's columns

    // ---- left x faces of this thread's four columns
    float fxq[4] = {0.f, 0.f, 0.f, 0.f};
    if (!prime) {
      const float4 p0 = S.xp[b][t], p1 = S.xp[b][t + 1], p2 = S.xp[b][t + 2];
      const float4 m0 = S.xm[b][t], m1 = S.xm[b][t + 1], m2 = S.xm[b][t + 2];
      const float c0w = S.xc[b][t].w;
      const float P[8] = {p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x};  // h+ at columns x-3 .. x+4
      const float M[8] = {m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x, m2.y};  // h- at columns x-2 .. x+5
      const float C[5] = {c0w, cq.x, cq.y, cq.z, cq.w};                     // c at columns x-1 .. x+3
      float D[7], E[7], SD[6], SE[6];
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        D[j] = P[j + 1] - P[j];
        E[j] = M[j + 1] - M[j];
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        SD[j] = D[j + 1] - D[j];
        SE[j] = E[j + 1] - E[j];
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {  // face between columns x - 1 + f and x + f
        const float hp = fmaf(weno5_q(D[f], D[f + 1], D[f + 2], D[f + 3], SD[f], SD[f + 1], SD[f + 2]),
                              1.f / 6.f, P[f + 2]);
        const float hm = fmaf(weno5_q(-E[f + 3], -E[f + 2], -E[f + 1], -E[f], SE[f + 2], SE[f + 1], SE[f]),
                              1.f / 6.f, M[f + 2]);
        fxq[f] = fmaf(alpha, hp + hm, kappa * (C[f] - C[f + 1]));
      }
      S.fx[b][t] = fxq[0];
      if (t == kWT - 1) S.fx[b][kWT] = S.edge[k - y0];
    }

    // ---- upper y face of each column (the lid face carries nothing)
    float fup[4] = {0.f, 0.f, 0.f, 0.f};
    if (k != ny - 1) {
      const float4 P0 = ring_at(S.yp, ring[0]), P1 = ring_at(S.yp, ring[1]), P2 = ring_at(S.yp, ring[2]),
                   P3 = ring_at(S.yp, ring[3]), P4 = ring_at(S.yp, ring[4]);
      const float4 M1 = ring_at(S.ym, ring[1]), M2 = ring_at(S.ym, ring[2]), M3 = ring_at(S.ym, ring[3]),
                   M4 = ring_at(S.ym, ring[4]), M5 = ring_at(S.ym, ring[5]);
      fup[0] = face_flux_x(P0.x, P1.x, P2.x, P3.x, P4.x, M5.x, M4.x, M3.x, M2.x, M1.x, alpha, kappa, cq.x, cnext.x);
      fup[1] = face_flux_x(P0.y, P1.y, P2.y, P3.y, P4.y, M5.y, M4.y, M3.y, M2.y, M1.y, alpha, kappa, cq.y, cnext.y);
      fup[2] = face_flux_x(P0.z, P1.z, P2.z, P3.z, P4.z, M5.z, M4.z, M3.z, M2.z, M1.z, alpha, kappa, cq.z, cnext.z);
      fup[3] = face_flux_x(P0.w, P1.w, P2.w, P3.w, P4.w, M5.w, M4.w, M3.w, M2.w, M1.w, alpha, kappa, cq.w, cnext.w);
    }
    // ---- ring: row k + 4 replaces row k - 2; fetch row k + 5
    put_r(ring[0]);
    fetch_r(k + 5);
    {
      const unsigned r0 = ring[0];
#pragma unroll
      for (int j = 0; j < kWring - 1; ++j) ring[j] = ring[j + 1];
      ring[kWring - 1] = r0;
    }
    __syncthreads();

    // ---- divergence and the Shu-Osher combination of this stage
    float4 cn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (STAGE > 1) {
      cp_async_wait<1>();  // row k landed (row k + 1 may still fly)
      cn = S.cn[k % 3][t];
    }
    if (!prime) {
      const float fr[4] = {fxq[1], fxq[2], fxq[3], S.fx[b][t + 1]};
      const float ch[4] = {cq.x, cq.y, cq.z, cq.w};
      const float cnv[4] = {cn.x, cn.y, cn.z, cn.w};
      const float cy[4] = {carry.x, carry.y, carry.z, carry.w};
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float fdn = k == 0 ? -a.vs * ch[j] : cy[j];
        const float L = fxq[j] - fr[j] + fdn - fup[j];
        if (STAGE == 1) {
          v[j] = ch[j] + L;
        } else if (STAGE == 2) {
          v[j] = fmaf(0.75f, cnv[j], 0.25f * (ch[j] + L));
        } else {
          const float s = ch[j] + L;
          v[j] = fmaf(1.f / 3.f, cnv[j] - s, s);
        }
      }
      if (out) {
        *reinterpret_cast<float4*>(sp.cout + (unsigned)k * (unsigned)nx + X) = make_float4(v[0], v[1], v[2], v[3]);
        if (STAGE == 3) {
          report_status(a.status, !(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3])));
          if (k == 0) {  // RK3 b-weights of the floor flux: c^n/6 + c1/6 + 2 c2/3
            const float4 c1 = LD::v4(a.c1 + X);
            const float c1v[4] = {c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int j = 0; j < 4; ++j)
              dep += fma((double)cnv[j] + (double)c1v[j], 1.0 / 6.0, (double)ch[j] * (2.0 / 3.0));
          }
        }
      }
    }
    carry = make_float4(fup[0], fup[1], fup[2], fup[3]);
    fetch_cn(k + 2);
  }
  if (STAGE > 1) cp_async_wait<0>();

  // stage 3: the CTAs holding the floor row fold the deposit of this step (FP64, fixed
  // order: warp shuffles, then the last CTA sums the per-CTA partials in strip order)
  if (STAGE == 3 && y0 == 0) {
    double v = dep;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) S.red[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
      double s2 = 0.0;
      for (int w = 0; w < kWT / 32; ++w) s2 += S.red[w];
      a.partials[bx] = s2 * (double)a.vs;
      __threadfence();
      S.last = atomicAdd(a.ticket, 1u) == (unsigned)strips - 1;
    }
    __syncthreads();
    if (S.last && t == 0) {
      __threadfence();
      const volatile double* vp = a.partials;
      double tot = 0.0;
      for (int s = 0; s < strips; ++s) tot += vp[s];
      const double prev = *reinterpret_cast<volatile double*>(a.scalars);  // written by earlier steps
      a.scalars[0] = prev + tot;
      *a.ticket = 0u;
    }
  }
}

template <int STAGE>
__global__ void __launch_bounds__(kWT, kWminB) rk_stage2d_wide_kernel(Args<float> a, Stage2dParams sp) {
  __shared__ __align__(16) StageWideSmem S;
  stage2d_wide_body<STAGE>(S, a, sp, blockIdx.x, blockIdx.y, gridDim.x);
}

// Rows per segment of the four-column kernel.  The CTAs of a launch run in waves of
// sm_count x per_sm (the CTAs the SMs hold at once), and a CTA's time grows with its rows
// plus about two rows of set-up (ring fill, priming row), so take the height that
// minimises waves x (H + 2); ties go to the fuller last wave.  Capped at kWmaxH.
inline int stage2d_wide_rows(int nx, int ny, int sm_count, int per_sm, int override_rows) {
  if (override_rows > 0) return min(min(override_rows, ny), kWmaxH);
  const long long strips = (nx + kWW - 1) / kWW;
  const long long slots = (long long)max(1, per_sm) * max(1, sm_count);
  int best = min(2, ny);
  double best_cost = 1e300;
  for (int H = 2; H <= kWmaxH; ++H) {
    const long long ctas = strips * ((ny + H - 1) / H);
    const long long waves = (ctas + slots - 1) / slots;
    const double cost = (double)waves * (H + 2) - 1e-6 * (double)ctas / (double)(waves * slots);
    if (cost < best_cost) {
      best_cost = cost;
      best = H;
    }
    if (H >= ny) break;
  }
  return min(best, ny);
}

template <int STAGE>
inline cudaError_t launch_stage2d_wide(const Args<float>& a, const float* cin, float* cout, int H, cudaStream_t s) {
  Stage2dParams sp;
  sp.cin = cin;
  sp.cout = cout;
  sp.H = H;
  const dim3 grid((a.nx + kWW - 1) / kWW, (a.ny + H - 1) / H);
  rk_stage2d_wide_kernel<STAGE><<<grid, kWT, 0, s>>>(a, sp);
  return cudaGetLastError();
}

}  // namespace lw
