// Fluid half of the coupled step: moments with the half force, BGK collision with
// the Guo source, streaming with halfway bounce-back -- fused in one in-place pass
// over a single population array with the AA access pattern.
//
//   a1  rho = 1 + sum g_i,  rho u = sum g_i c_i + F/2,  F = body - A c e_v
//       (Sec. 2.3.1, Eqs. dens, mom_dens; rho u* of Eq. LBE_Guo with b = 1/2)
//   a2  g_i* = g_i - (g_i - g_i^eq)/tau + (1 - 1/(2 tau)) w_i [3(c_i - u) + 9 (c_i.u) c_i].F
//       (Eqs. LBE, LBE_Guo; Guo 2002 source; g = f - w_i so that FP32 keeps the
//       small deviations from rest)
//   a3  streaming along c_i; populations that would cross the floor or lid are
//       reflected back to the node they left (halfway bounce-back, no-slip walls).
//
// AA pattern: one array, no second copy.  On an even step a node reads its own
// slots and writes the post-collision g_i* into slot opp(i) of the same node.  On an
// odd step it pulls g_i from slot opp(i) of node x - c_i (slot i of itself when
// x - c_i is behind a wall) and pushes g_i* to slot i of x + c_i (slot opp(i) of
// itself when x + c_i is behind a wall).  Every location is read and written by
// one thread only, so the pass is in place.  After an odd number of steps the
// array holds post-collision values (parity 1); after an even number it holds the
// streamed populations (parity 0).
#pragma once
#include "common.cuh"
#include "lattice.cuh"

namespace lw {

// Neighbour of (x,y,z) along direction i, sign s = +1 (x + c_i) or -1 (x - c_i).
// Returns false when the neighbour is behind a no-slip wall.
template <class LAT>
__device__ __forceinline__ bool neighbour(int i, int s, int x, int y, int z, int nx, int ny, int nz,
                                          bool walls, long long& out) {
  int xx = wrap_any(x + s * LAT::cx(i), nx);
  int yy = y + s * LAT::cy(i);
  int zz = z + s * LAT::cz(i);
  if (LAT::VAXIS == 1) {
    if (yy < 0 || yy >= ny) {
      if (walls) return false;
      yy = wrap_any(yy, ny);
    }
  } else {
    yy = wrap_any(yy, ny);
    if (zz < 0 || zz >= nz) {
      if (walls) return false;
      zz = wrap_any(zz, nz);
    }
  }
  out = ((long long)zz * ny + yy) * nx + xx;
  return true;
}

// Load the populations of node (x,y,z) as they stand at the start of a step with
// the given parity (0: natural layout; 1: post-collision layout, pull from neighbours).
template <class LAT, typename T, int PARITY>
__device__ __forceinline__ void load_populations(const Args<T>& a, int x, int y, int z, long long node,
                                                 T (&g)[LAT::Q]) {
  const long long n = a.n;
#pragma unroll
  for (int i = 0; i < LAT::Q; ++i) {
    if (PARITY == 0) {
      g[i] = a.g[i * n + node];
    } else {
      long long src;
      if (neighbour<LAT>(i, -1, x, y, z, a.nx, a.ny, a.nz, a.walls != 0, src))
        g[i] = a.g[LAT::opp(i) * n + src];
      else
        g[i] = a.g[i * n + node];
    }
  }
}

// Force at a node: body force - A c along the vertical, and with sugar also
// - g S* S (1 - phi0 c) (the density-altering term of the force).
template <class LAT, typename T>
__device__ __forceinline__ void node_force(const Args<T>& a, long long node, T (&F)[3]) {
  const T cval = a.c[node];
  F[0] = a.bf[0];
  F[1] = a.bf[1];
  F[2] = a.bf[2];
  F[LAT::VAXIS] -= a.A * cval;
  if (a.S) F[LAT::VAXIS] -= a.gS * a.S[node] * (T(1) - a.phi0 * cval);
}

template <class LAT, typename T, int PARITY>
__global__ void __launch_bounds__(128) lbm_step_kernel(Args<T> a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx) return;
  const long long n = a.n;
  const long long node = ((long long)z * a.ny + y) * a.nx + x;

  T g[LAT::Q];
  load_populations<LAT, T, PARITY>(a, x, y, z, node, g);

  // a1: moments (rho - 1 and momentum of g; sum w_i c_i = 0) and the force from c^n
  T drho = T(0), j[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < LAT::Q; ++i) {
    drho += g[i];
    if (LAT::cx(i)) j[0] += LAT::cx(i) * g[i];
    if (LAT::cy(i)) j[1] += LAT::cy(i) * g[i];
    if (LAT::cz(i)) j[2] += LAT::cz(i) * g[i];
  }
  T F[3];
  node_force<LAT, T>(a, node, F);
  const T rho = T(1) + drho;
  const T inv_rho = T(1) / rho;
  T u[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) u[d] = (j[d] + T(0.5) * F[d]) * inv_rho;
  bool bad = !finite_val(rho);
#pragma unroll
  for (int d = 0; d < LAT::DIM; ++d) {
    a.u[d * n + node] = u[d];
    bad = bad || !(fabs(u[d]) <= a.u_cap);
  }
  report_status(a.status, bad);

  // a2: BGK collision with the Guo source, in the g = f - w variables
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
#pragma unroll
  for (int i = 0; i < LAT::Q; ++i) {
    const T wi = T(LAT::w(i));
    const T cu = LAT::cx(i) * u[0] + LAT::cy(i) * u[1] + LAT::cz(i) * u[2];
    const T cF = LAT::cx(i) * F[0] + LAT::cy(i) * F[1] + LAT::cz(i) * F[2];
    const T geq = wi * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu));
    const T src = a.guo * wi * (T(3) * (cF - uF) + T(9) * cu * cF);
    g[i] = g[i] - a.omega * (g[i] - geq) + src;
  }

  // a3: store (even: swap slots in place; odd: push to neighbours / bounce back)
#pragma unroll
  for (int i = 0; i < LAT::Q; ++i) {
    if (PARITY == 0) {
      a.g[LAT::opp(i) * n + node] = g[i];
    } else {
      long long dst;
      if (neighbour<LAT>(i, +1, x, y, z, a.nx, a.ny, a.nz, a.walls != 0, dst))
        a.g[i * n + dst] = g[i];
      else
        a.g[LAT::opp(i) * n + node] = g[i];
    }
  }
}

// D2Q9 specialisation of the fused collide-stream (same arithmetic as lbm_step_kernel):
// 32-bit node offsets, the three source rows and columns hoisted, the wall test of
// a row taken once per block (a block is one row segment).  The population traffic
// uses plain cached loads and stores: evict-first streaming hints on it were measured
// 5 % slower (the odd step's shifted accesses reuse lines between neighbouring rows).
template <typename T, int PARITY, bool RHO = false, bool SUGAR = false>
__device__ __forceinline__ void lbm_d2q9_body(const Args<T>& a, int bx, int by, T* rho_out = nullptr);

template <typename T, int PARITY, bool SUGAR = false>
__global__ void __launch_bounds__(128) lbm_d2q9_kernel(Args<T> a) {
  lbm_d2q9_body<T, PARITY, false, SUGAR>(a, blockIdx.x, blockIdx.y);
}

// The same step that also stores rho (the steps recorded for the adjoint).
template <typename T, int PARITY>
__global__ void __launch_bounds__(128) lbm_d2q9_record_kernel(Args<T> a, T* rho_out) {
  lbm_d2q9_body<T, PARITY, true>(a, blockIdx.x, blockIdx.y, rho_out);
}

// One D2Q9 node's neighbour offsets along x and y (periodic x; y periodic or walled) and
// its wall flags.
struct D2Q9Node {
  unsigned node;
  int dxm, dxp, dym, dyp;  // offsets of x-1, x+1, y-1, y+1 (0 behind a wall)
  bool wall_m, wall_p;     // floor below / lid above
  __device__ __forceinline__ int off(int i, int s) const {  // node + s c_i, without the wall test
    const int cx = s * D2Q9::cx(i), cy = s * D2Q9::cy(i);
    return (cx > 0 ? dxp : (cx < 0 ? dxm : 0)) + (cy > 0 ? dyp : (cy < 0 ? dym : 0));
  }
  __device__ __forceinline__ bool behind_wall(int i, int s) const {
    const int cy = s * D2Q9::cy(i);
    return (cy < 0 && wall_m) || (cy > 0 && wall_p);
  }
};

template <typename T>
__device__ __forceinline__ D2Q9Node d2q9_node(const Args<T>& a, int x, int y) {
  const int nx = a.nx, ny = a.ny;
  const bool walls = a.walls != 0;
  D2Q9Node nd;
  nd.node = (unsigned)y * (unsigned)nx + (unsigned)x;
  nd.dxm = x == 0 ? nx - 1 : -1;
  nd.dxp = x == nx - 1 ? -(nx - 1) : 1;
  const bool bot = y == 0, top = y == ny - 1;
  nd.dym = bot ? (walls ? 0 : (ny - 1) * nx) : -nx;
  nd.dyp = top ? (walls ? 0 : -(ny - 1) * nx) : nx;
  nd.wall_m = walls && bot;
  nd.wall_p = walls && top;
  return nd;
}

// The node's populations as they stand at the start of a step of this parity (AA pattern).
template <typename T, int PARITY, class LD = LoadNC>
__device__ __forceinline__ void d2q9_load(const Args<T>& a, const D2Q9Node& nd, T (&g)[9]) {
  const unsigned n = (unsigned)a.n;
  const T* __restrict__ G = a.g;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if (PARITY == 0) {
      g[i] = LD::s(G + i * n + nd.node);
    } else {
      g[i] = nd.behind_wall(i, -1) ? LD::s(G + i * n + nd.node)
                                   : LD::s(G + D2Q9::opp(i) * n + (unsigned)((int)nd.node + nd.off(i, -1)));
    }
  }
}

// Moments, BGK-Guo collision and the in-place AA store of one node whose concentration
// (the force's c) is cn (LD: how S is read, see common.cuh).
template <typename T, int PARITY, bool RHO, bool SUGAR, class LD = LoadPlain>
__device__ __forceinline__ void d2q9_collide_store_c(const Args<T>& a, const D2Q9Node& nd, const T (&g)[9],
                                                     T* rho_out, const T cn) {
  const unsigned n = (unsigned)a.n;
  const unsigned node = nd.node;
  T* __restrict__ G = a.g;
  T drho = T(0), jx = T(0), jy = T(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    drho += g[i];
    if (D2Q9::cx(i)) jx += D2Q9::cx(i) * g[i];
    if (D2Q9::cy(i)) jy += D2Q9::cy(i) * g[i];
  }
  T Fy = a.bf[1] - a.A * cn;
  if (SUGAR) Fy -= a.gS * LD::s(a.S + node) * (T(1) - a.phi0 * cn);
  const T Fx = a.bf[0];
  const T rho = T(1) + drho;
  const T inv_rho = T(1) / rho;
  const T ux = (jx + T(0.5) * Fx) * inv_rho, uy = (jy + T(0.5) * Fy) * inv_rho;
  a.u[node] = ux;
  a.u[n + node] = uy;
  if (RHO) rho_out[node] = rho;
  report_status(a.status, !finite_val(rho) || !(fabs(ux) <= a.u_cap) || !(fabs(uy) <= a.u_cap));
  const T uu = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
  const T om = a.omega, keep = T(1) - a.omega;
  auto store = [&](int i, T gs) {
    if (PARITY == 0) {
      G[D2Q9::opp(i) * n + node] = gs;
    } else {
      if (nd.behind_wall(i, +1))
        G[D2Q9::opp(i) * n + node] = gs;
      else
        G[i * n + (unsigned)((int)node + nd.off(i, +1))] = gs;
    }
  };
  // rest population
  {
    const T w0 = T(D2Q9::w(0));
    const T geq = w0 * (drho - rho * T(1.5) * uu);
    const T src = a.guo * w0 * (T(-3) * uF);
    store(0, keep * g[0] + om * geq + src);
  }
  // opposite pairs (i, i+1) share c.u and c.F up to sign: split the equilibrium and
  // the Guo source into parts even and odd in c_i
#pragma unroll
  for (int i = 1; i < 9; i += 2) {
    const T wi = T(D2Q9::w(i));
    const T cu = D2Q9::cx(i) * ux + D2Q9::cy(i) * uy;
    const T cF = D2Q9::cx(i) * Fx + D2Q9::cy(i) * Fy;
    const T even = wi * (drho + rho * (T(4.5) * cu * cu - T(1.5) * uu));
    const T odd = wi * rho * T(3) * cu;
    const T seven = a.guo * wi * (T(9) * cu * cF - T(3) * uF);
    const T sodd = a.guo * wi * T(3) * cF;
    store(i, keep * g[i] + om * (even + odd) + (seven + sodd));
    store(i + 1, keep * g[i + 1] + om * (even - odd) + (seven - sodd));
  }
}

// The same with c (and S) read at the node through LD.
template <typename T, int PARITY, bool RHO, bool SUGAR, class LD = LoadPlain>
__device__ __forceinline__ void d2q9_collide_store(const Args<T>& a, const D2Q9Node& nd, const T (&g)[9],
                                                   T* rho_out) {
  d2q9_collide_store_c<T, PARITY, RHO, SUGAR, LD>(a, nd, g, rho_out, LD::s(a.c + nd.node));
}

// Body of the D2Q9 kernel for block (bx, by): nodes x = bx*128 + thread, row y = by.
template <typename T, int PARITY, bool RHO, bool SUGAR>
__device__ __forceinline__ void lbm_d2q9_body(const Args<T>& a, int bx, int by, T* rho_out) {
  const int x = bx * blockDim.x + threadIdx.x;
  if (x >= a.nx) return;
  const D2Q9Node nd = d2q9_node(a, x, by);
  T g[9];
  d2q9_load<T, PARITY>(a, nd, g);
  d2q9_collide_store<T, PARITY, RHO, SUGAR>(a, nd, g, rho_out);
}

// D3Q19 specialisation (same arithmetic as lbm_step_kernel): 32-bit offsets with the
// neighbour offsets along x, y (periodic) and z (walls or periodic) hoisted, the wall
// tests taken once per block (a block is one x segment of one (y, z) row), plain cached
// population traffic as in D2Q9.
// One D3Q19 node's neighbour offsets (periodic x and y; z periodic or walled) and wall
// flags.
struct D3Q19Node {
  unsigned node;
  int dxm, dxp, dym, dyp, dzm, dzp;  // offsets of the six face neighbours (0 behind a wall)
  bool wall_m, wall_p;               // floor below / lid above
  __device__ __forceinline__ int off(int i, int s) const {  // node + s c_i, without the wall test
    const int cx = s * D3Q19::cx(i), cy = s * D3Q19::cy(i), cz = s * D3Q19::cz(i);
    return (cx > 0 ? dxp : (cx < 0 ? dxm : 0)) + (cy > 0 ? dyp : (cy < 0 ? dym : 0)) +
           (cz > 0 ? dzp : (cz < 0 ? dzm : 0));
  }
  __device__ __forceinline__ bool behind_wall(int i, int s) const {
    const int cz = s * D3Q19::cz(i);
    return (cz < 0 && wall_m) || (cz > 0 && wall_p);
  }
};

template <typename T>
__device__ __forceinline__ D3Q19Node d3q19_node(const Args<T>& a, int x, int y, int z) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int plane = nx * ny;
  const bool walls = a.walls != 0;
  D3Q19Node nd;
  nd.node = (unsigned)z * (unsigned)plane + (unsigned)y * (unsigned)nx + (unsigned)x;
  nd.dxm = x == 0 ? nx - 1 : -1;
  nd.dxp = x == nx - 1 ? -(nx - 1) : 1;
  nd.dym = y == 0 ? (ny - 1) * nx : -nx;
  nd.dyp = y == ny - 1 ? -(ny - 1) * nx : nx;
  const bool bot = z == 0, top = z == nz - 1;
  nd.dzm = bot ? (walls ? 0 : (nz - 1) * plane) : -plane;
  nd.dzp = top ? (walls ? 0 : -(nz - 1) * plane) : plane;
  nd.wall_m = walls && bot;
  nd.wall_p = walls && top;
  return nd;
}

template <typename T, int PARITY>
__device__ __forceinline__ void d3q19_load(const Args<T>& a, const D3Q19Node& nd, T (&g)[19]) {
  const unsigned n = (unsigned)a.n;
  const T* __restrict__ G = a.g;
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    if (PARITY == 0) {
      g[i] = __ldg(G + i * n + nd.node);
    } else {
      g[i] = nd.behind_wall(i, -1) ? __ldg(G + i * n + nd.node)
                                   : __ldg(G + D3Q19::opp(i) * n + (unsigned)((int)nd.node + nd.off(i, -1)));
    }
  }
}

template <typename T, int PARITY, bool SUGAR>
__device__ __forceinline__ void d3q19_collide_store(const Args<T>& a, const D3Q19Node& nd, const T (&g)[19]) {
  const unsigned n = (unsigned)a.n;
  const unsigned node = nd.node;
  T* __restrict__ G = a.g;
  T drho = T(0), jx = T(0), jy = T(0), jz = T(0);
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    drho += g[i];
    if (D3Q19::cx(i)) jx += D3Q19::cx(i) * g[i];
    if (D3Q19::cy(i)) jy += D3Q19::cy(i) * g[i];
    if (D3Q19::cz(i)) jz += D3Q19::cz(i) * g[i];
  }
  const T cn = a.c[node];
  T Fz = a.bf[2] - a.A * cn;
  if (SUGAR) Fz -= a.gS * a.S[node] * (T(1) - a.phi0 * cn);
  const T Fx = a.bf[0], Fy = a.bf[1];
  const T rho = T(1) + drho;
  const T inv_rho = T(1) / rho;
  const T ux = (jx + T(0.5) * Fx) * inv_rho, uy = (jy + T(0.5) * Fy) * inv_rho, uz = (jz + T(0.5) * Fz) * inv_rho;
  a.u[node] = ux;
  a.u[n + node] = uy;
  a.u[2 * n + node] = uz;
  report_status(a.status, !finite_val(rho) || !(fabs(ux) <= a.u_cap) || !(fabs(uy) <= a.u_cap) ||
                              !(fabs(uz) <= a.u_cap));
  const T uu = ux * ux + uy * uy + uz * uz, uF = ux * Fx + uy * Fy + uz * Fz;
  const T om = a.omega, keep = T(1) - a.omega;
  auto store = [&](int i, T gs) {
    if (PARITY == 0) {
      G[D3Q19::opp(i) * n + node] = gs;
    } else {
      if (nd.behind_wall(i, +1))
        G[D3Q19::opp(i) * n + node] = gs;
      else
        G[i * n + (unsigned)((int)node + nd.off(i, +1))] = gs;
    }
  };
  {
    const T w0 = T(D3Q19::w(0));
    const T geq = w0 * (drho - rho * T(1.5) * uu);
    const T src = a.guo * w0 * (T(-3) * uF);
    store(0, keep * g[0] + om * geq + src);
  }
#pragma unroll
  for (int i = 1; i < 19; i += 2) {  // opposite pairs (i, i+1)
    const T wi = T(D3Q19::w(i));
    const T cu = D3Q19::cx(i) * ux + D3Q19::cy(i) * uy + D3Q19::cz(i) * uz;
    const T cF = D3Q19::cx(i) * Fx + D3Q19::cy(i) * Fy + D3Q19::cz(i) * Fz;
    const T even = wi * (drho + rho * (T(4.5) * cu * cu - T(1.5) * uu));
    const T odd = wi * rho * T(3) * cu;
    const T seven = a.guo * wi * (T(9) * cu * cF - T(3) * uF);
    const T sodd = a.guo * wi * T(3) * cF;
    store(i, keep * g[i] + om * (even + odd) + (seven + sodd));
    store(i + 1, keep * g[i + 1] + om * (even - odd) + (seven - sodd));
  }
}

template <typename T, int PARITY, bool SUGAR = false>
__global__ void __launch_bounds__(128) lbm_d3q19_kernel(Args<T> a) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= a.nx) return;
  const D3Q19Node nd = d3q19_node(a, x, blockIdx.y, blockIdx.z);
  T g[19];
  d3q19_load<T, PARITY>(a, nd, g);
  d3q19_collide_store<T, PARITY, SUGAR>(a, nd, g);
}

// Macroscopic fields of the current state (parity as in load_populations):
// rho, u = (sum g c + F/2)/rho with the current c.
template <class LAT, typename T, int PARITY>
__global__ void __launch_bounds__(128) fields_kernel(Args<T> a, T* rho_out, T* u_out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx) return;
  const long long n = a.n;
  const long long node = ((long long)z * a.ny + y) * a.nx + x;
  T g[LAT::Q];
  load_populations<LAT, T, PARITY>(a, x, y, z, node, g);
  T drho = T(0), j[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int i = 0; i < LAT::Q; ++i) {
    drho += g[i];
    j[0] += LAT::cx(i) * g[i];
    j[1] += LAT::cy(i) * g[i];
    j[2] += LAT::cz(i) * g[i];
  }
  T F[3];
  node_force<LAT, T>(a, node, F);
  const T rho = T(1) + drho;
  if (rho_out) rho_out[node] = rho;
  if (u_out) {
#pragma unroll
    for (int d = 0; d < LAT::DIM; ++d) u_out[d * n + node] = (j[d] + T(0.5) * F[d]) / rho;
  }
}

// Initial state: g_i = f_i^eq(1, u0) - w_i, u = u0 (or 0).  c is already in place.
template <class LAT, typename T>
__global__ void __launch_bounds__(128) init_kernel(Args<T> a, const T* u0) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= a.nx) return;
  const long long n = a.n;
  const long long node = ((long long)z * a.ny + y) * a.nx + x;
  T u[3] = {T(0), T(0), T(0)};
  if (u0) {
#pragma unroll
    for (int d = 0; d < LAT::DIM; ++d) u[d] = u0[d * n + node];
  }
#pragma unroll
  for (int d = 0; d < LAT::DIM; ++d) a.u[d * n + node] = u[d];
  const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
  for (int i = 0; i < LAT::Q; ++i) {
    const T cu = LAT::cx(i) * u[0] + LAT::cy(i) * u[1] + LAT::cz(i) * u[2];
    a.g[i * n + node] = T(LAT::w(i)) * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * uu);
  }
}

}  // namespace lw
