// 3D FP32 transport: one SSP-RK3 stage of the WENO5 + diffusion + settling update of c
// (steps a4..a8) as a tiled sweep along the vertical axis z.
//
// A CTA owns a 32 x 8 tile of (x, y) columns and a segment of z levels and sweeps it
// upward.  At level k it stages the x- and y-split fluxes of the stage input on the
// tile plus a 3-column halo in shared memory (loaded from L2), computes the left
// x face and the lower y face of every column (the tile's right and upper edge faces by
// two dedicated warps), and the upper z face of its own column from a per-column ring
// of z-split fluxes that runs three levels ahead; the lower z face is carried from the
// previous level.  Every face of the stage is computed once.  Three launches make a
// step (the intermediate fields go through HBM/L2); the stage kernels of the generic
// path (transport_kernels.cuh) remain for FP64, periodic-vertical and 2D.
//
// Walls as in the rest of the library: ghost levels -2, -1, nz, nz+1 reflect c (even)
// and the fluid velocity (odd, Vs unchanged); the floor face carries -Vs c(0), the lid 0.
#pragma once
#include "common.cuh"
#include "transport_sweep2d.cuh"  // weno5_face_value, face_flux_x

namespace lw {

constexpr int kT3x = 32, kT3y = 8;           // tile (threads)
constexpr int kT3h = 3;                      // stencil radius
constexpr int kT3X = kT3x + 2 * kT3h;        // tile + halo, x
constexpr int kT3Y = kT3y + 2 * kT3h;        // tile + halo, y
constexpr int kT3r = 8;                      // z ring depth

struct Sweep3dSmem {
  float xp[kT3y][kT3X];  // x-split h+/alpha, tile rows, x halo
  float xm[kT3y][kT3X];
  float yp[kT3Y][kT3x];  // y-split, tile columns, y halo
  float ym[kT3Y][kT3x];
  float c[kT3Y][kT3X];   // stage input value (diffusion)
  float zp[kT3r][kT3y][kT3x];  // z-split ring of each column
  float zm[kT3r][kT3y][kT3x];
  float cz[kT3r][kT3y][kT3x];  // stage input value ring of each column
  float fx[kT3y][kT3x + 1];    // left x faces (+ right edge)
  float fy[kT3y + 1][kT3x];    // lower y faces (+ upper edge)
};

struct Sweep3dParams {
  const float* cin;  // stage input field (c, c1 or c2)
  float* cout;       // stage output field (c1, c2 or c in place)
  int H;             // z levels per segment
  float ghost_shift; // 2 Vs / alpha
};

// SCHEME: transport-scheme variant bits (kSchemeWeno3, kSchemeSignSplit; 0 = Lax-Friedrichs
// WENO5), see face_flux_scheme.
template <int STAGE, bool SUGAR, int SCHEME>
__device__ __forceinline__ void rk_sweep3d_body(const Args<float>& a, const Sweep3dParams& sp) {
  constexpr bool SIGN = (SCHEME & kSchemeSignSplit) != 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Sweep3dSmem& S = *reinterpret_cast<Sweep3dSmem*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kT3x + tx;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x0 = blockIdx.x * kT3x, y0 = blockIdx.y * kT3y;
  const int z0 = blockIdx.z * sp.H, z1 = min(nz, z0 + sp.H);
  const int X = (x0 + tx) % nx, Y = (y0 + ty) % ny;
  const bool out = (x0 + tx) < nx && (y0 + ty) < ny;
  const unsigned plane = (unsigned)nx * (unsigned)ny, n = (unsigned)a.n;
  const float inv_alpha = a.inv_alpha, vs_a = a.vs * a.inv_alpha, alpha = a.alpha, kappa = a.kappa;
  const float* __restrict__ cin = sp.cin;
  const float* __restrict__ ux = a.u;
  const float* __restrict__ uy = a.u + n;
  const float* __restrict__ uz = a.u + 2 * n;
  const unsigned col = (unsigned)Y * (unsigned)nx + (unsigned)X;

  // own column, level l (ghosts reflect): c and scaled vertical transport velocity,
  // loaded one level before they enter the ring (software pipelining)
  float qc = 0.f, qw = 0.f, qn = 0.f;
  auto col_fetch = [&](int l) {
    const bool ghost = l < 0 || l >= nz;
    const int lr = l < 0 ? -1 - l : (l >= nz ? 2 * nz - 1 - l : l);
    const unsigned k = (unsigned)lr * plane + col;
    qc = __ldg(cin + k);
    const float u = __ldg(uz + k);
    // with sugar the settling velocity of the node (a ghost reads its mirror's) is Vs (1 - ks S)
    const float vsa = SUGAR ? vs_a * fmaf(-a.ks, __ldg(a.S + k), 1.f) : vs_a;
    qw = fmaf(ghost ? -u : u, inv_alpha, -vsa);
  };
  auto col_put = [&](int l) {
    const float h = 0.5f * qc;
    S.zp[l & (kT3r - 1)][ty][tx] = SIGN ? qw * qc : fmaf(qw, h, h);
    S.zm[l & (kT3r - 1)][ty][tx] = SIGN ? qw : fmaf(qw, h, -h);
    S.cz[l & (kT3r - 1)][ty][tx] = qc;
  };
  auto col_split = [&](int l) {
    col_fetch(l);
    col_put(l);
  };
  // c^n at the own column, one level ahead (stages 2 and 3 combine with it)
  auto cn_fetch = [&](int k) {
    if (STAGE > 1 && k < z1) qn = a.c[(unsigned)k * plane + col];
  };

  // Each thread stages up to three positions of the tile + halo cross (the corners are
  // not needed); their smem slots and in-plane offsets are fixed for the whole sweep.
  constexpr int kSlots = (kT3X * kT3Y + kT3x * kT3y - 1) / (kT3x * kT3y);
  int sl_ry[kSlots], sl_rx[kSlots];
  unsigned sl_off[kSlots];
  bool sl_x[kSlots], sl_y[kSlots], sl_on[kSlots];
#pragma unroll
  for (int q = 0; q < kSlots; ++q) {
    const int j = tid + q * kT3x * kT3y;
    const int rx = j % kT3X, ry = j / kT3X;
    sl_rx[q] = rx;
    sl_ry[q] = ry;
    sl_x[q] = ry >= kT3h && ry < kT3h + kT3y;
    sl_y[q] = rx >= kT3h && rx < kT3h + kT3x;
    sl_on[q] = j < kT3X * kT3Y && (sl_x[q] || sl_y[q]);
    const int gx = (x0 - kT3h + rx + 4 * nx) % nx, gy = (y0 - kT3h + ry + 4 * ny) % ny;
    sl_off[q] = (unsigned)gy * (unsigned)nx + (unsigned)gx;
  }
  // registers holding the next level's staged values (software pipelining)
  float pc[kSlots], pu[kSlots], pv[kSlots];
  auto fetch_tile = [&](int k) {
    const unsigned lv = (unsigned)k * plane;
#pragma unroll
    for (int q = 0; q < kSlots; ++q) {
      if (sl_on[q] && k < z1) {
        const unsigned k3 = lv + sl_off[q];
        pc[q] = __ldg(cin + k3);
        pu[q] = sl_x[q] ? __ldg(ux + k3) : 0.f;
        pv[q] = sl_y[q] ? __ldg(uy + k3) : 0.f;
      }
    }
  };

  const int kb = z0 == 0 ? 0 : z0 - 1;  // first level: z0, or the priming level below it
  for (int l = kb - 2; l < kb + 3; ++l) col_split(l);
  col_fetch(kb + 3);
  float carry = 0.f;
  fetch_tile(kb);
  cn_fetch(kb);

  for (int k = kb; k < z1; ++k) {
    const bool prime = k < z0;
    const unsigned lv = (unsigned)k * plane;
    // ---- stage the tile and its halo at level k (prefetched); own column three levels ahead
#pragma unroll
    for (int q = 0; q < kSlots; ++q) {
      if (sl_on[q]) {
        const float c = pc[q], h = 0.5f * c;
        const int rx = sl_rx[q], ry = sl_ry[q];
        S.c[ry][rx] = c;
        if (sl_x[q]) {
          const float w = pu[q] * inv_alpha;
          S.xp[ry - kT3h][rx] = SIGN ? w * c : fmaf(w, h, h);
          S.xm[ry - kT3h][rx] = SIGN ? w : fmaf(w, h, -h);
        }
        if (sl_y[q]) {
          const float w = pv[q] * inv_alpha;
          S.yp[ry][rx - kT3h] = SIGN ? w * c : fmaf(w, h, h);
          S.ym[ry][rx - kT3h] = SIGN ? w : fmaf(w, h, -h);
        }
      }
    }
    fetch_tile(k + 1);
    col_put(k + 3);
    col_fetch(k + 4);
    const float cn_here = qn;
    cn_fetch(k + 1);
    __syncthreads();

    // ---- faces: left x face and lower y face of this column, upper z face
    float chere, fup = 0.f;
    if constexpr (SCHEME == 0) {
      if (!prime) {
        const float* P = &S.xp[ty][tx];
        const float* M = &S.xm[ty][tx];
        S.fx[ty][tx] = face_flux_x(P[0], P[1], P[2], P[3], P[4], M[5], M[4], M[3], M[2], M[1], alpha, kappa,
                                   S.c[ty + kT3h][tx + kT3h - 1], S.c[ty + kT3h][tx + kT3h]);
        S.fy[ty][tx] = face_flux_x(S.yp[ty][tx], S.yp[ty + 1][tx], S.yp[ty + 2][tx], S.yp[ty + 3][tx],
                                   S.yp[ty + 4][tx], S.ym[ty + 5][tx], S.ym[ty + 4][tx], S.ym[ty + 3][tx],
                                   S.ym[ty + 2][tx], S.ym[ty + 1][tx], alpha, kappa, S.c[ty + kT3h - 1][tx + kT3h],
                                   S.c[ty + kT3h][tx + kT3h]);
        if (ty == 0 && tx < kT3y) {  // right edge x faces (column 32) of the tile rows
          const float* Pe = &S.xp[tx][kT3x];
          const float* Me = &S.xm[tx][kT3x];
          S.fx[tx][kT3x] = face_flux_x(Pe[0], Pe[1], Pe[2], Pe[3], Pe[4], Me[5], Me[4], Me[3], Me[2], Me[1], alpha,
                                       kappa, S.c[tx + kT3h][kT3x + kT3h - 1], S.c[tx + kT3h][kT3x + kT3h]);
        }
        if (ty == 1) {  // upper edge y faces (row 8) of the tile columns
          S.fy[kT3y][tx] = face_flux_x(S.yp[kT3y][tx], S.yp[kT3y + 1][tx], S.yp[kT3y + 2][tx], S.yp[kT3y + 3][tx],
                                       S.yp[kT3y + 4][tx], S.ym[kT3y + 5][tx], S.ym[kT3y + 4][tx],
                                       S.ym[kT3y + 3][tx], S.ym[kT3y + 2][tx], S.ym[kT3y + 1][tx], alpha, kappa,
                                       S.c[kT3y + kT3h - 1][tx + kT3h], S.c[kT3y + kT3h][tx + kT3h]);
        }
      }
      chere = S.cz[k & (kT3r - 1)][ty][tx];
      if (k != nz - 1) {
        fup = face_flux_x(S.zp[(k - 2) & (kT3r - 1)][ty][tx], S.zp[(k - 1) & (kT3r - 1)][ty][tx],
                          S.zp[k & (kT3r - 1)][ty][tx], S.zp[(k + 1) & (kT3r - 1)][ty][tx],
                          S.zp[(k + 2) & (kT3r - 1)][ty][tx], S.zm[(k + 3) & (kT3r - 1)][ty][tx],
                          S.zm[(k + 2) & (kT3r - 1)][ty][tx], S.zm[(k + 1) & (kT3r - 1)][ty][tx],
                          S.zm[k & (kT3r - 1)][ty][tx], S.zm[(k - 1) & (kT3r - 1)][ty][tx], alpha, kappa, chere,
                          S.cz[(k + 1) & (kT3r - 1)][ty][tx]);
      }
    } else {
      // the six staged pairs of a face at stride st from P, M (points i-2 .. i+3)
      auto face6 = [&](const float* P, const float* M, int st, float cl, float cr) {
        float p[6], m[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          p[q] = P[q * st];
          m[q] = M[q * st];
        }
        return face_flux_scheme<SCHEME>(p, m, alpha, kappa, cl, cr);
      };
      if (!prime) {
        S.fx[ty][tx] =
            face6(&S.xp[ty][tx], &S.xm[ty][tx], 1, S.c[ty + kT3h][tx + kT3h - 1], S.c[ty + kT3h][tx + kT3h]);
        S.fy[ty][tx] = face6(&S.yp[ty][tx], &S.ym[ty][tx], kT3x, S.c[ty + kT3h - 1][tx + kT3h],
                             S.c[ty + kT3h][tx + kT3h]);
        if (ty == 0 && tx < kT3y)  // right edge x faces (column 32) of the tile rows
          S.fx[tx][kT3x] = face6(&S.xp[tx][kT3x], &S.xm[tx][kT3x], 1, S.c[tx + kT3h][kT3x + kT3h - 1],
                                 S.c[tx + kT3h][kT3x + kT3h]);
        if (ty == 1)  // upper edge y faces (row 8) of the tile columns
          S.fy[kT3y][tx] = face6(&S.yp[kT3y][tx], &S.ym[kT3y][tx], kT3x, S.c[kT3y + kT3h - 1][tx + kT3h],
                                 S.c[kT3y + kT3h][tx + kT3h]);
      }
      chere = S.cz[k & (kT3r - 1)][ty][tx];
      if (k != nz - 1) {
        float p[6], m[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          p[q] = S.zp[(k - 2 + q) & (kT3r - 1)][ty][tx];
          m[q] = S.zm[(k - 2 + q) & (kT3r - 1)][ty][tx];
        }
        fup = face_flux_scheme<SCHEME>(p, m, alpha, kappa, chere, S.cz[(k + 1) & (kT3r - 1)][ty][tx]);
      }
    }
    __syncthreads();

    // ---- divergence and the Shu-Osher combination of this stage
    if (!prime) {
      const float vs_floor = SUGAR && k == 0 ? a.vs * fmaf(-a.ks, __ldg(a.S + col), 1.f) : a.vs;
      const float fdn = k == 0 ? -vs_floor * chere : carry;
      const float L = S.fx[ty][tx] - S.fx[ty][tx + 1] + S.fy[ty][tx] - S.fy[ty + 1][tx] + fdn - fup;
      if (out) {
        const unsigned node = lv + col;
        float v;
        if (STAGE == 1) {
          v = chere + L;
        } else if (STAGE == 2) {
          v = fmaf(0.75f, cn_here, 0.25f * (chere + L));
        } else {
          const float s = chere + L;
          v = fmaf(1.f / 3.f, cn_here - s, s);
        }
        sp.cout[node] = v;
        if (STAGE == 3) report_status(a.status, !isfinite(v));
      }
    }
    carry = fup;
  }
}

// Two entry points with the same body: uncapped (57-62 registers for stages 1 and 2), and
// capped at 64 registers (four resident 256-thread CTAs per SM) for the instantiations the
// compiler would otherwise give more (stage 3: 72; stage 1 with sugar).  An explicit
// minimum of one block is not the same as none: it lets stages 1 and 2 grow to 72.
template <int STAGE, bool SUGAR = false, int SCHEME = 0>
__global__ void __launch_bounds__(kT3x * kT3y) rk_sweep3d_kernel(Args<float> a, Sweep3dParams sp) {
  rk_sweep3d_body<STAGE, SUGAR, SCHEME>(a, sp);
}

template <int STAGE, bool SUGAR = false, int SCHEME = 0>
__global__ void __launch_bounds__(kT3x * kT3y, 4) rk_sweep3d_capped_kernel(Args<float> a, Sweep3dParams sp) {
  rk_sweep3d_body<STAGE, SUGAR, SCHEME>(a, sp);
}

template <int STAGE, bool SUGAR>
constexpr bool sweep3d_capped() { return (STAGE == 3 && !SUGAR) || (STAGE == 1 && SUGAR); }

template <int STAGE, bool SUGAR, int SCHEME = 0>
inline void (*sweep3d_entry())(Args<float>, Sweep3dParams) {
  if constexpr (sweep3d_capped<STAGE, SUGAR>())
    return rk_sweep3d_capped_kernel<STAGE, SUGAR, SCHEME>;
  else
    return rk_sweep3d_kernel<STAGE, SUGAR, SCHEME>;
}

// The entry point of a stage for the handle's arguments: sugar and the transport scheme
// (runtime fields) as compile-time variants.
template <int STAGE, bool SUGAR>
inline void (*sweep3d_entry_scheme(int scheme))(Args<float>, Sweep3dParams) {
  switch (scheme) {
    case kSchemeWeno3: return sweep3d_entry<STAGE, SUGAR, kSchemeWeno3>();
    case kSchemeSignSplit: return sweep3d_entry<STAGE, SUGAR, kSchemeSignSplit>();
    case kSchemeWeno3 | kSchemeSignSplit: return sweep3d_entry<STAGE, SUGAR, kSchemeWeno3 | kSchemeSignSplit>();
    default: return sweep3d_entry<STAGE, SUGAR>();
  }
}

template <int STAGE>
inline void (*sweep3d_entry_for(const Args<float>& a))(Args<float>, Sweep3dParams) {
  return a.S ? sweep3d_entry_scheme<STAGE, true>(a.scheme) : sweep3d_entry_scheme<STAGE, false>(a.scheme);
}

inline size_t sweep3d_smem() { return sizeof(Sweep3dSmem); }

inline bool sweep3d_supported(int nz, bool walls) { return walls && nz >= 4; }

inline cudaError_t sweep3d_prepare() {
  const int b = (int)sizeof(Sweep3dSmem);
  const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  for (int scheme = 0; scheme < 4; ++scheme) {  // every stage x sugar x scheme entry point
    void (*const entries[])(Args<float>, Sweep3dParams) = {
        sweep3d_entry_scheme<1, false>(scheme), sweep3d_entry_scheme<2, false>(scheme),
        sweep3d_entry_scheme<3, false>(scheme), sweep3d_entry_scheme<1, true>(scheme),
        sweep3d_entry_scheme<2, true>(scheme), sweep3d_entry_scheme<3, true>(scheme)};
    for (auto f : entries)
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, at, b);
  }
  return e;
}

inline int sweep3d_rows(int nx, int ny, int nz, int sm_count, int override_rows) {
  if (override_rows > 0) return min(override_rows, nz);
  const long long tiles = (long long)((nx + kT3x - 1) / kT3x) * ((ny + kT3y - 1) / kT3y);
  // at least 21 CTAs per SM in total (five waves at four resident CTAs per SM: on the
  // 256 x 256 x 512 lattice 40-level segments, 0.6 % faster than 52), segments no shorter
  // than 24 levels
  long long segs = (21LL * sm_count + tiles - 1) / tiles;
  int H = (int)((nz + segs - 1) / segs);
  return max(min(24, nz), H);
}

template <int STAGE>
inline cudaError_t launch_sweep3d(const Args<float>& a, const float* cin, float* cout, int H, cudaStream_t s) {
  Sweep3dParams sp;
  sp.cin = cin;
  sp.cout = cout;
  sp.H = H;
  sp.ghost_shift = 2.f * a.vs * a.inv_alpha;
  const dim3 grid((a.nx + kT3x - 1) / kT3x, (a.ny + kT3y - 1) / kT3y, (a.nz + H - 1) / H);
  sweep3d_entry_for<STAGE>(a)<<<grid, dim3(kT3x, kT3y), sizeof(Sweep3dSmem), s>>>(a, sp);
  return cudaGetLastError();
}

}  // namespace lw
