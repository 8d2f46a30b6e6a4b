// 3D FP32 transport with four adjacent x columns per thread: one SSP-RK3 stage of the
// WENO5 + diffusion + settling update of c (steps a4..a8) as a tiled sweep along the
// vertical axis z.  Default scheme (Lax-Friedrichs WENO5), no sugar; the scheme variants
// and the sugar scalar keep the one-column kernel of transport_sweep3d.cuh.
//
// A CTA of kV3x x kV3y threads owns a tile of 4 kV3x x kV3y (x, y) columns and a segment
// of z levels and sweeps it upward.  At level k:
//  - the x-split fluxes of the tile rows with a four-column halo quad on each side, the
//    y-split fluxes of the tile columns with a three-row halo below and above, and c on
//    both, are staged in shared memory as float4 quads (loaded one level ahead; one buffer,
//    refilled between two barriers, so that four CTAs fit an SM);
//  - a thread reconstructs the left x faces of its four columns (first and second
//    differences of the split fluxes shared between the four faces) and the lower y face
//    of each of them; the x face right of its last column is its neighbour's first one,
//    the y face above is the lower face of the thread above; for the tile's right column
//    and top row these faces are computed for every level of the segment before the
//    sweep;
//  - the upper z face of each column comes from a private ring of the z-split fluxes of
//    levels k-2 .. k+3, filled three levels ahead; the lower z face is carried.
// Every face is computed once with the arithmetic of weno5_face_value/face_flux_x, so c is
// bitwise that of the one-column kernel.
//
// Walls: ghost levels -2, -1, nz, nz+1 reflect c (even) and the fluid velocity (odd, Vs
// unchanged); the floor face carries -Vs c(0), the lid 0 (the floor deposit is folded by
// its own kernel in 3D).
#pragma once
#include "common.cuh"
#include "transport_sweep2d.cuh"       // weno5_q, weno5_face_value, face_flux_x
#include "transport_sweep3d.cuh"       // Sweep3dParams
#include "transport_stage2d_wide.cuh"  // lf_split

namespace lw {

constexpr int kV3x = 8;                 // threads along x (4 columns each)
constexpr int kV3y = 16;                // threads along y
constexpr int kV3T = kV3x * kV3y;       // threads per CTA
constexpr int kV3W = 4 * kV3x;          // tile width in columns
constexpr int kV3Qx = kV3x + 2;         // staged quads per row (tile and one halo quad per side)
constexpr int kV3Ry = kV3y + 6;         // staged rows of the y stencil (three-row halo per side)
constexpr int kV3maxH = 32;             // longest z segment (its edge faces are held in smem)
constexpr int kV3Buf = 1;               // staging buffers: 1 (two barriers a level, four CTAs an SM)

struct Sweep3dWideSmem {
  float4 xp[kV3Buf][kV3y][kV3Qx];   // x-split h+/alpha of the tile rows (by level parity if two)
  float4 xm[kV3Buf][kV3y][kV3Qx];
  float4 yp[kV3Buf][kV3Ry][kV3x];   // y-split h+/alpha of the tile columns (rows -3 .. kV3y + 2)
  float4 ym[kV3Buf][kV3Ry][kV3x];
  float4 c[kV3Buf][kV3Ry][kV3Qx];   // stage input c (rows -3 .. kV3y + 2, quads -1 .. kV3x)
  float4 zp[6][kV3T];          // z-split ring of each thread's four columns
  float4 zm[6][kV3T];
  float fx[2][kV3y][kV3x + 1];     // first left x face of each thread (+ the tile's right edge)
  float4 fy[2][kV3y + 1][kV3x];    // lower y faces of each thread's columns (+ the tile's top edge)
  float xedge[kV3maxH][kV3y];      // right-edge x face of each tile row at each level
  float4 yedge[kV3maxH][kV3x];     // top-edge y faces of the tile columns at each level
};

template <int STAGE>
__device__ __forceinline__ void sweep3d_wide_body(Sweep3dWideSmem& S, const Args<float>& a, const Sweep3dParams& sp) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kV3x + tx;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x0 = blockIdx.x * kV3W, y0 = blockIdx.y * kV3y;
  const int z0 = blockIdx.z * sp.H, z1 = min(nz, z0 + sp.H);
  const int xl = x0 + 4 * tx, yl = y0 + ty;
  const bool out = xl < nx && yl < ny;
  const unsigned X = (unsigned)(xl % nx), Y = (unsigned)(yl % ny);
  const unsigned plane = (unsigned)nx * (unsigned)ny, n = (unsigned)a.n;
  const unsigned col = Y * (unsigned)nx + X;
  const float ia = a.inv_alpha, vs_a = a.vs * a.inv_alpha, alpha = a.alpha, kappa = a.kappa;
  const float* __restrict__ cin = sp.cin;
  const float* __restrict__ ux = a.u;
  const float* __restrict__ uy = a.u + n;
  const float* __restrict__ uz = a.u + 2 * n;

  // staging positions: the cross of tile rows x [quads -1 .. kV3x] and rows [-3 .. kV3y+2]
  // x tile quads (the corners are not needed); each thread takes up to two
  constexpr int kPos = kV3y * kV3Qx + 6 * kV3x;  // tile rows (with x halo) + the 6 halo rows
  constexpr int kSl = (kPos + kV3T - 1) / kV3T;
  int sl_r[kSl], sl_q[kSl];  // staged row (0 .. kV3Ry-1) and quad (0 .. kV3Qx-1)
  unsigned sl_off[kSl];
  bool sl_on[kSl], sl_x[kSl], sl_y[kSl];
#pragma unroll
  for (int s = 0; s < kSl; ++s) {
    const int j = tid + s * kV3T;
    int r, q;
    if (j < kV3y * kV3Qx) {  // a tile row, any quad
      r = 3 + j / kV3Qx;
      q = j % kV3Qx;
    } else {  // a halo row, a tile quad
      const int h = j - kV3y * kV3Qx;
      const int hr = h / kV3x;  // 0..5: rows -3, -2, -1, kV3y, kV3y + 1, kV3y + 2
      r = hr < 3 ? hr : kV3y + hr;
      q = 1 + h % kV3x;
    }
    sl_on[s] = j < kPos;
    sl_r[s] = r;
    sl_q[s] = q;
    sl_x[s] = r >= 3 && r < 3 + kV3y;
    sl_y[s] = q >= 1 && q <= kV3x;
    const int gx = ((x0 - 4 + 4 * q) % nx + nx) % nx, gy = ((y0 - 3 + r) % ny + ny) % ny;
    sl_off[s] = (unsigned)gy * (unsigned)nx + (unsigned)gx;
  }
  float4 pc[kSl], pu[kSl], pv[kSl];
  auto fetch_tile = [&](int l) {
    const unsigned lv = (unsigned)l * plane;
#pragma unroll
    for (int s = 0; s < kSl; ++s) {
      if (sl_on[s]) {
        pc[s] = LoadNC::v4(cin + lv + sl_off[s]);
        if (sl_x[s]) pu[s] = LoadNC::v4(ux + lv + sl_off[s]);
        if (sl_y[s]) pv[s] = LoadNC::v4(uy + lv + sl_off[s]);
      }
    }
  };
  auto stage_tile = [&](int b) {
#pragma unroll
    for (int s = 0; s < kSl; ++s) {
      if (sl_on[s]) {
        const float4 c = pc[s];
        S.c[b][sl_r[s]][sl_q[s]] = c;
        if (sl_x[s]) {
          const float4 u = pu[s];
          float4 p, m;
          lf_split(c.x, u.x * ia, p.x, m.x);
          lf_split(c.y, u.y * ia, p.y, m.y);
          lf_split(c.z, u.z * ia, p.z, m.z);
          lf_split(c.w, u.w * ia, p.w, m.w);
          S.xp[b][sl_r[s] - 3][sl_q[s]] = p;
          S.xm[b][sl_r[s] - 3][sl_q[s]] = m;
        }
        if (sl_y[s]) {
          const float4 u = pv[s];
          float4 p, m;
          lf_split(c.x, u.x * ia, p.x, m.x);
          lf_split(c.y, u.y * ia, p.y, m.y);
          lf_split(c.z, u.z * ia, p.z, m.z);
          lf_split(c.w, u.w * ia, p.w, m.w);
          S.yp[b][sl_r[s]][sl_q[s] - 1] = p;
          S.ym[b][sl_r[s]][sl_q[s] - 1] = m;
        }
      }
    }
  };

  // own columns, ring level l (ghost levels reflect: c even, u_z odd); levels past the
  // ones any face reads are clamped into the lattice and never used
  float4 Rc, Ru;
  bool Rg = false;
  auto fetch_r = [&](int l) {
    Rg = l < 0 || l >= nz;
    int lr = l < 0 ? -1 - l : (l >= nz ? 2 * nz - 1 - l : l);
    lr = max(0, min(nz - 1, lr));
    const unsigned k3 = (unsigned)lr * plane + col;
    Rc = LoadNC::v4(cin + k3);
    Ru = LoadNC::v4(uz + k3);
  };
  auto put_r = [&](int slot) {
    const float s = Rg ? -ia : ia;
    float4 p, m;
    lf_split(Rc.x, fmaf(Ru.x, s, -vs_a), p.x, m.x);
    lf_split(Rc.y, fmaf(Ru.y, s, -vs_a), p.y, m.y);
    lf_split(Rc.z, fmaf(Ru.z, s, -vs_a), p.z, m.z);
    lf_split(Rc.w, fmaf(Ru.w, s, -vs_a), p.w, m.w);
    S.zp[slot][tid] = p;
    S.zm[slot][tid] = m;
  };

  // edge faces of every level of the segment: right x edge of each tile row and top y edge
  // of each tile column (the first faces of the neighbouring tiles)
  for (int e = tid; e < (z1 - z0) * (kV3y + kV3W); e += kV3T) {
    const int h = e / (kV3y + kV3W), w = e % (kV3y + kV3W);
    const unsigned lv = (unsigned)(z0 + h) * plane;
    float P[6], M[6], C[6];
    if (w < kV3y) {  // x face between columns x0 + kV3W - 1 and x0 + kV3W, tile row w
      const unsigned row = (unsigned)((y0 + w) % ny) * (unsigned)nx;
#pragma unroll
      for (int o = 0; o < 6; ++o) {
        const unsigned cx = (unsigned)((x0 + kV3W - 3 + o) % nx);
        C[o] = __ldg(cin + lv + row + cx);
        lf_split(C[o], __ldg(ux + lv + row + cx) * ia, P[o], M[o]);
      }
      S.xedge[h][w] = face_flux_x(P[0], P[1], P[2], P[3], P[4], M[5], M[4], M[3], M[2], M[1], alpha, kappa, C[2], C[3]);
    } else {  // y face between rows y0 + kV3y - 1 and y0 + kV3y, tile column w - kV3y
      const int cl = w - kV3y;
      const unsigned cx = (unsigned)((x0 + cl) % nx);
#pragma unroll
      for (int o = 0; o < 6; ++o) {
        const unsigned row = (unsigned)((y0 + kV3y - 3 + o) % ny) * (unsigned)nx;
        C[o] = __ldg(cin + lv + row + cx);
        lf_split(C[o], __ldg(uy + lv + row + cx) * ia, P[o], M[o]);
      }
      reinterpret_cast<float*>(&S.yedge[h][0])[cl] =
          face_flux_x(P[0], P[1], P[2], P[3], P[4], M[5], M[4], M[3], M[2], M[1], alpha, kappa, C[2], C[3]);
    }
  }

  const int kb = z0 == 0 ? 0 : z0 - 1;  // first level: z0, or the priming level below it
  int ring[6];                          // slots of levels k-2 .. k+3
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    ring[j] = j;
    fetch_r(kb - 2 + j);
    put_r(j);
  }
  fetch_r(kb + 4);
  fetch_tile(kb);
  stage_tile(kV3Buf == 2 ? (kb & 1) : 0);
  fetch_tile(kb + 1);  // kb + 1 <= z0 < nz
  float4 cn = make_float4(0.f, 0.f, 0.f, 0.f);
  if (STAGE > 1) cn = LoadNC::v4(a.c + (unsigned)kb * plane + col);
  float4 carry = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();

  for (int k = kb; k < z1; ++k) {
    const int b = k & 1;                           // face exchange buffers
    const int sb = kV3Buf == 2 ? b : 0;            // staging buffer of level k
    const int sn = kV3Buf == 2 ? (b ^ 1) : 0;      // staging buffer of level k + 1
    const bool prime = k < z0;
    if (kV3Buf == 2 && k + 1 < nz) stage_tile(sn);  // level k + 1 (its c at the own columns: the z face)
    if (kV3Buf == 2 && k + 1 < z1 && k + 2 < nz) fetch_tile(k + 2);
    const float4 cq = S.c[sb][3 + ty][1 + tx];  // c of level k at this thread's columns

    float fxq[4] = {0.f, 0.f, 0.f, 0.f};
    float4 fyl = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!prime) {
      // left x faces of the four columns (shared differences, as in the 2D kernel)
      {
        const float4 p0 = S.xp[sb][ty][tx], p1 = S.xp[sb][ty][tx + 1], p2 = S.xp[sb][ty][tx + 2];
        const float4 m0 = S.xm[sb][ty][tx], m1 = S.xm[sb][ty][tx + 1], m2 = S.xm[sb][ty][tx + 2];
        const float c0w = S.c[sb][3 + ty][tx].w;
        const float P[8] = {p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w, p2.x};
        const float M[8] = {m0.z, m0.w, m1.x, m1.y, m1.z, m1.w, m2.x, m2.y};
        const float C[5] = {c0w, cq.x, cq.y, cq.z, cq.w};
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
        for (int f = 0; f < 4; ++f) {
          const float hp = fmaf(weno5_q(D[f], D[f + 1], D[f + 2], D[f + 3], SD[f], SD[f + 1], SD[f + 2]),
                                1.f / 6.f, P[f + 2]);
          const float hm = fmaf(weno5_q(-E[f + 3], -E[f + 2], -E[f + 1], -E[f], SE[f + 2], SE[f + 1], SE[f]),
                                1.f / 6.f, M[f + 2]);
          fxq[f] = fmaf(alpha, hp + hm, kappa * (C[f] - C[f + 1]));
        }
        S.fx[b][ty][tx] = fxq[0];
        if (tx == kV3x - 1) S.fx[b][ty][kV3x] = S.xedge[k - z0][ty];
      }
      // lower y face of each column: y-split rows ty-3 .. ty+2 (staged rows ty .. ty+5)
      {
        const float4 P0 = S.yp[sb][ty][tx], P1 = S.yp[sb][ty + 1][tx], P2 = S.yp[sb][ty + 2][tx],
                     P3 = S.yp[sb][ty + 3][tx], P4 = S.yp[sb][ty + 4][tx];
        const float4 M1 = S.ym[sb][ty + 1][tx], M2 = S.ym[sb][ty + 2][tx], M3 = S.ym[sb][ty + 3][tx],
                     M4 = S.ym[sb][ty + 4][tx], M5 = S.ym[sb][ty + 5][tx];
        const float4 cb = S.c[sb][2 + ty][1 + tx];  // c of the row below
        fyl.x = face_flux_x(P0.x, P1.x, P2.x, P3.x, P4.x, M5.x, M4.x, M3.x, M2.x, M1.x, alpha, kappa, cb.x, cq.x);
        fyl.y = face_flux_x(P0.y, P1.y, P2.y, P3.y, P4.y, M5.y, M4.y, M3.y, M2.y, M1.y, alpha, kappa, cb.y, cq.y);
        fyl.z = face_flux_x(P0.z, P1.z, P2.z, P3.z, P4.z, M5.z, M4.z, M3.z, M2.z, M1.z, alpha, kappa, cb.z, cq.z);
        fyl.w = face_flux_x(P0.w, P1.w, P2.w, P3.w, P4.w, M5.w, M4.w, M3.w, M2.w, M1.w, alpha, kappa, cb.w, cq.w);
        S.fy[b][ty][tx] = fyl;
        if (ty == kV3y - 1) S.fy[b][kV3y][tx] = S.yedge[k - z0][tx];
      }
    }

    __syncthreads();
    if (kV3Buf == 1) {  // one staging buffer: level k + 1 replaces level k once every face has read it
      if (k + 1 < nz) stage_tile(0);
      if (k + 1 < z1 && k + 2 < nz) fetch_tile(k + 2);
      __syncthreads();
    }

    // upper z face of each column from the ring (the lid face carries nothing); c of
    // level k + 1 at the own columns was staged before the barrier
    float fup[4] = {0.f, 0.f, 0.f, 0.f};
    if (k != nz - 1) {
      const float4 cnext = S.c[sn][3 + ty][1 + tx];
      const float4 P0 = S.zp[ring[0]][tid], P1 = S.zp[ring[1]][tid], P2 = S.zp[ring[2]][tid],
                   P3 = S.zp[ring[3]][tid], P4 = S.zp[ring[4]][tid];
      const float4 M1 = S.zm[ring[1]][tid], M2 = S.zm[ring[2]][tid], M3 = S.zm[ring[3]][tid],
                   M4 = S.zm[ring[4]][tid], M5 = S.zm[ring[5]][tid];
      fup[0] = face_flux_x(P0.x, P1.x, P2.x, P3.x, P4.x, M5.x, M4.x, M3.x, M2.x, M1.x, alpha, kappa, cq.x, cnext.x);
      fup[1] = face_flux_x(P0.y, P1.y, P2.y, P3.y, P4.y, M5.y, M4.y, M3.y, M2.y, M1.y, alpha, kappa, cq.y, cnext.y);
      fup[2] = face_flux_x(P0.z, P1.z, P2.z, P3.z, P4.z, M5.z, M4.z, M3.z, M2.z, M1.z, alpha, kappa, cq.z, cnext.z);
      fup[3] = face_flux_x(P0.w, P1.w, P2.w, P3.w, P4.w, M5.w, M4.w, M3.w, M2.w, M1.w, alpha, kappa, cq.w, cnext.w);
    }
    // ring: level k + 4 replaces level k - 2; fetch level k + 5
    put_r(ring[0]);
    fetch_r(k + 5);
    {
      const int r0 = ring[0];
#pragma unroll
      for (int j = 0; j < 5; ++j) ring[j] = ring[j + 1];
      ring[5] = r0;
    }

    // ---- divergence and the Shu-Osher combination of this stage
    if (!prime) {
      const float fr[4] = {fxq[1], fxq[2], fxq[3], S.fx[b][ty][tx + 1]};
      const float4 fyu = S.fy[b][ty + 1][tx];
      const float fyl4[4] = {fyl.x, fyl.y, fyl.z, fyl.w}, fyu4[4] = {fyu.x, fyu.y, fyu.z, fyu.w};
      const float ch[4] = {cq.x, cq.y, cq.z, cq.w};
      const float cnv[4] = {cn.x, cn.y, cn.z, cn.w};
      const float cy[4] = {carry.x, carry.y, carry.z, carry.w};
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float fdn = k == 0 ? -a.vs * ch[j] : cy[j];
        const float L = fxq[j] - fr[j] + fyl4[j] - fyu4[j] + fdn - fup[j];
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
        *reinterpret_cast<float4*>(sp.cout + (unsigned)k * plane + col) = make_float4(v[0], v[1], v[2], v[3]);
        if (STAGE == 3)
          report_status(a.status, !(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3])));
      }
    }
    carry = make_float4(fup[0], fup[1], fup[2], fup[3]);
    if (STAGE > 1 && k + 1 < z1) cn = LoadNC::v4(a.c + (unsigned)(k + 1) * plane + col);
  }
}

template <int STAGE>
__global__ void __launch_bounds__(kV3T, 4) rk_sweep3d_wide_kernel(Args<float> a, Sweep3dParams sp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sweep3d_wide_body<STAGE>(*reinterpret_cast<Sweep3dWideSmem*>(smem_raw), a, sp);
}

inline size_t sweep3d_wide_smem() { return sizeof(Sweep3dWideSmem); }

inline cudaError_t sweep3d_wide_prepare() {
  const int bytes = (int)sizeof(Sweep3dWideSmem);
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(rk_sweep3d_wide_kernel<1>, at, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(rk_sweep3d_wide_kernel<2>, at, bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(rk_sweep3d_wide_kernel<3>, at, bytes);
  return e;
}

// Levels per segment of the four-column kernel: the height that minimises launch waves x
// (H + 2) for the resident CTA count, as for the 2D kernel; capped at kV3maxH.
inline int sweep3d_wide_rows(int nx, int ny, int nz, int sm_count, int per_sm, int override_rows) {
  if (override_rows > 0) return min(min(override_rows, nz), kV3maxH);
  const long long tiles = (long long)((nx + kV3W - 1) / kV3W) * ((ny + kV3y - 1) / kV3y);
  const long long slots = (long long)max(1, per_sm) * max(1, sm_count);
  int best = min(2, nz);
  double best_cost = 1e300;
  for (int H = 2; H <= kV3maxH; ++H) {
    const long long ctas = tiles * ((nz + H - 1) / H);
    const long long waves = (ctas + slots - 1) / slots;
    const double cost = (double)waves * (H + 2) - 1e-6 * (double)ctas / (double)(waves * slots);
    if (cost < best_cost) {
      best_cost = cost;
      best = H;
    }
    if (H >= nz) break;
  }
  return min(best, nz);
}

template <int STAGE>
inline cudaError_t launch_sweep3d_wide(const Args<float>& a, const float* cin, float* cout, int H, cudaStream_t s) {
  Sweep3dParams sp;
  sp.cin = cin;
  sp.cout = cout;
  sp.H = H;
  sp.ghost_shift = 2.f * a.vs * a.inv_alpha;
  const dim3 grid((a.nx + kV3W - 1) / kV3W, (a.ny + kV3y - 1) / kV3y, (a.nz + H - 1) / H);
  rk_sweep3d_wide_kernel<STAGE><<<grid, dim3(kV3x, kV3y), sizeof(Sweep3dWideSmem), s>>>(a, sp);
  return cudaGetLastError();
}

}  // namespace lw
