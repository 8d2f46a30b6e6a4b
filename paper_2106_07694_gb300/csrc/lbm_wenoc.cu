// Host side of the lbm_wenoc C ABI (include/lbm_wenoc.h): parameter checks, the
// carve-up of the caller's workspace, kernel launches, CUDA-graph replay of whole
// steps, FP64 read-backs and per-kernel event timing.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <string>
#include <vector>

#include "lbm_wenoc.h"
#include "common.cuh"
#include "lattice.cuh"
#include "lbm_kernels.cuh"
#include "reduce_kernels.cuh"
#include "transport_kernels.cuh"
#include "transport_sweep2d.cuh"
#include "transport_sweep3d.cuh"
#include "transport_stage2d.cuh"
#include "transport_stage2d_wide.cuh"
#include "transport_sweep3d_wide.cuh"
#include "batch.cuh"
#include "adjoint.cuh"

namespace {

using lw::Args;

constexpr int kLbmThreads = 128;

// Velocity sets must come in opposite pairs with isotropic second moments.
template <class LAT>
constexpr bool lattice_ok() {
  double s = 0, sxx = 0, syy = 0, szz = 0, sxy = 0;
  for (int i = 0; i < LAT::Q; ++i) {
    const int o = LAT::opp(i);
    if (LAT::cx(o) != -LAT::cx(i) || LAT::cy(o) != -LAT::cy(i) || LAT::cz(o) != -LAT::cz(i)) return false;
    s += LAT::w(i);
    sxx += LAT::w(i) * LAT::cx(i) * LAT::cx(i);
    syy += LAT::w(i) * LAT::cy(i) * LAT::cy(i);
    szz += LAT::w(i) * LAT::cz(i) * LAT::cz(i);
    sxy += LAT::w(i) * LAT::cx(i) * LAT::cy(i);
  }
  auto close = [](double a, double b) { return a - b < 1e-12 && b - a < 1e-12; };
  return close(s, 1.0) && close(sxx, 1.0 / 3.0) && close(syy, 1.0 / 3.0) && close(sxy, 0.0) &&
         (LAT::DIM == 2 ? close(szz, 0.0) : close(szz, 1.0 / 3.0));
}
static_assert(lattice_ok<D2Q9>(), "D2Q9 table");
static_assert(lattice_ok<D3Q19>(), "D3Q19 table");

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
  size_t g, c, c1, c2, u, partials, scalars, status, sa, sb, cls, ctot, total;
};

// scalars[0] deposit (one class), [1] reduction result, [4 + k] deposit of class k
constexpr int kScalars = 16;
constexpr int kClassDeposit = 4;

int classes_of(const lbm_wenoc_params& p) { return p.n_classes >= 2 ? p.n_classes : 1; }

Layout make_layout(const lbm_wenoc_params& p) {
  const size_t n = (size_t)p.nx * p.ny * (p.dim == 3 ? p.nz : 1);
  const size_t es = (p.flags & LW_FP64) ? 8 : 4;
  const int Q = p.dim == 2 ? 9 : 19;
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  L.g = take((size_t)Q * n * es);
  L.c = take(n * es);
  L.c1 = take(n * es);
  L.c2 = take(n * es);
  L.u = take((size_t)p.dim * n * es);
  L.partials = take(sizeof(double) * lw::kMaxReduceBlocks);
  L.scalars = take(sizeof(double) * kScalars);
  L.status = take(sizeof(unsigned) * 4);
  const bool sugar = (p.flags & LW_SUGAR) != 0;
  L.sa = take(sugar ? n * es : 0);  // sugar of step n and n + 1 (ping-pong)
  L.sb = take(sugar ? n * es : 0);
  const int ncls = classes_of(p);
  L.cls = take(ncls > 1 ? (size_t)(ncls - 1) * align_up(n * es, 256) : 0);  // classes 1..ncls-1
  L.ctot = take(ncls > 1 ? n * es : 0);                                   // their sum with class 0
  L.total = off;
  return L;
}

int check_params(const lbm_wenoc_params* p) {
  if (!p) return LW_EINVAL;
  if (p->dim != 2 && p->dim != 3) return LW_EINVAL;
  if (p->nx < 4 || p->ny < 4 || (p->nx % 4) != 0) return LW_EINVAL;
  if (p->dim == 3 && p->nz < 4) return LW_EINVAL;
  if (p->dim == 2 && p->ny > 65535) return LW_EINVAL;          // grid.y
  if (p->dim == 3 && (p->ny > 65535 || p->nz > 65535)) return LW_EINVAL;
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return LW_EINVAL;  // stability needs tau > 1/2
  if (!(p->settling_velocity >= 0.0) || !(p->diffusivity >= 0.0)) return LW_EINVAL;
  if (!(p->lf_alpha >= 0.0) || !(p->u_cap >= 0.0)) return LW_EINVAL;
  if ((p->flags & (LW_WENO3 | LW_SIGN_SPLIT)) && (p->flags & LW_FUSED_RK3)) return LW_EINVAL;
  if (p->n_classes < 0 || p->n_classes > 8) return LW_EINVAL;
  if (p->n_classes >= 2) {
    if (p->flags & LW_FUSED_RK3) return LW_EINVAL;
    for (int k = 0; k < p->n_classes; ++k)
      if (!(p->class_vs[k] >= 0.0) || !std::isfinite(p->class_vs[k])) return LW_EINVAL;
  }
  if ((p->flags & LW_SUGAR) && ((p->flags & LW_FUSED_RK3) || !(p->sugar_diffusivity >= 0.0) ||
                                !std::isfinite(p->sugar_contrast) || !std::isfinite(p->phi0) ||
                                !std::isfinite(p->vs_sugar)))
    return LW_EINVAL;
  const double nn = (double)p->nx * p->ny * (p->dim == 3 ? p->nz : 1);
  if (nn > 4.0e9) return LW_EINVAL;
  if ((double)(p->dim == 2 ? 9 : 19) * nn >= 2147483647.0) return LW_EINVAL;  // 32-bit population offsets
  return LW_OK;
}

}  // namespace

struct lbm_wenoc {
  lbm_wenoc_params p{};
  Layout L{};
  unsigned char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool fp64 = false, walls = true, frozen = false, use_graphs = true;
  long long n = 0;
  int parity = 0;  // AA-pattern parity of the population array
  int cur = 0;     // ping-pong index: c^n in c or c1 (fused sweep), S^n in sa or sb (sugar)
  bool sweep = false;
  lw::SweepLaunch sweep_geom{};
  bool sweep3d = false;  // 3D FP32 with walls: tiled z-sweep stage kernels
  int sweep3d_rows = 0;
  bool wide3d = false;   // ... with four columns per thread (default scheme, no sugar)
  int wide3d_per_sm = 1;
  bool stage2d = false;  // 2D FP32 with walls: three row-sweep stage kernels
  int stage2d_rows = 0;
  bool wide = false;     // ... with four columns per thread (default scheme, no sugar)
  int wide_per_sm = 1;   // CTAs of the four-column stage kernel one SM holds at once
  bool initialised = false;
  bool sugar = false;  // LW_SUGAR: S in L.sa / L.sb, selected by cur (the generic transport path)
  int ncls = 1;        // particle classes
  int64_t steps = 0;
  int64_t launches = 0;
  double alpha = 0.0;
  // graphs keyed by (AA parity, c buffer) at their first step: kGraphSteps steps, and 1 step
  static constexpr int kGraphSteps = 16;
  cudaGraphExec_t graph_many[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t graph_one[4] = {nullptr, nullptr, nullptr, nullptr};
  // profiling
  bool profiling = false;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<std::string> kind_names;
  std::vector<int64_t> kind_launches;
  std::vector<double> kind_ms;
};

namespace {

template <typename T>
Args<T> make_args(const lbm_wenoc* h) {
  Args<T> a{};
  unsigned char* b = h->ws;
  a.g = reinterpret_cast<T*>(b + h->L.g);
  a.c = reinterpret_cast<T*>(b + (h->sweep && h->cur ? h->L.c1 : h->L.c));
  a.c1 = reinterpret_cast<T*>(b + h->L.c1);
  a.c2 = reinterpret_cast<T*>(b + h->L.c2);
  a.u = reinterpret_cast<T*>(b + h->L.u);
  a.partials = reinterpret_cast<double*>(b + h->L.partials);
  a.scalars = reinterpret_cast<double*>(b + h->L.scalars);
  a.status = reinterpret_cast<unsigned*>(b + h->L.status);
  a.ticket = a.status + 1;
  const lbm_wenoc_params& p = h->p;
  a.nx = p.nx;
  a.ny = p.ny;
  a.nz = p.dim == 3 ? p.nz : 1;
  a.n = h->n;
  a.walls = h->walls ? 1 : 0;
  a.omega = T(1.0 / p.tau);
  a.guo = T(1.0 - 0.5 / p.tau);
  a.A = T(p.gravity * p.density_contrast);
  for (int d = 0; d < 3; ++d) a.bf[d] = T(p.body_force[d]);
  a.vs = T(p.settling_velocity);
  a.kappa = T(p.diffusivity);
  a.alpha = T(h->alpha);
  a.inv_alpha = T(1.0 / h->alpha);
  a.u_cap = T(p.u_cap);
  a.scheme = ((p.flags & LW_WENO3) ? lw::kSchemeWeno3 : 0) | ((p.flags & LW_SIGN_SPLIT) ? lw::kSchemeSignSplit : 0);
  if (h->sugar) {
    a.S = reinterpret_cast<T*>(b + (h->cur ? h->L.sb : h->L.sa));
    a.S2 = reinterpret_cast<T*>(b + (h->cur ? h->L.sa : h->L.sb));
    a.gS = T(p.gravity * p.sugar_contrast);
    a.phi0 = T(p.phi0);
    a.ks = T(p.vs_sugar);
    a.Ds = T(p.sugar_diffusivity);
  }
  return a;
}

// Kernel families for timing.
enum Kind {
  K_LBM = 0, K_STAGE1, K_STAGE2, K_STAGE3, K_DEPOSIT, K_RK3_SWEEP, K_OTHER,
  K_ADJ_FACES, K_ADJ_GATHER, K_ADJ_FLUID, K_SUGAR, K_COUNT
};
const char* kKindNames[K_COUNT] = {"lbm_collide_stream", "rk_stage1",  "rk_stage2",  "rk_stage3",
                                   "deposit_reduce",     "rk3_sweep2d", "other",     "adj_faces",
                                   "adj_gather",         "adj_gather_fluid", "sugar_upwind"};
// The 3D FP32 stage kernels are timed under the rk_stage* names.

// NVTX range over a scope (an API call, or a kernel enqueued outside graph capture), for
// profilers that show them (nsys, ncu --nvtx); without an attached tool a push is a test.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

cudaEvent_t take_event(lbm_wenoc* h) {
  if (h->event_pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = h->event_pool.back();
  h->event_pool.pop_back();
  return e;
}

void fold_pending(lbm_wenoc* h) {
  for (auto& pe : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
      h->kind_ms[pe.kind] += ms;
      h->kind_launches[pe.kind] += 1;
    }
    h->event_pool.push_back(pe.a);
    h->event_pool.push_back(pe.b);
  }
  h->pending.clear();
}

// Wrap one launch: optional event pair, launch counting.
template <typename F>
void launch(lbm_wenoc* h, int kind, F&& f) {
  NvtxRange range(kKindNames[kind]);
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (h->profiling) {
    if (h->pending.size() >= 4096) {
      cudaStreamSynchronize(h->stream);
      fold_pending(h);
    }
    ea = take_event(h);
    eb = take_event(h);
    if (ea) cudaEventRecord(ea, h->stream);
  }
  f();
  h->launches++;
  if (ea && eb) {
    cudaEventRecord(eb, h->stream);
    h->pending.push_back({kind, ea, eb});
  }
}

template <class LAT, typename T>
void enqueue_transport(lbm_wenoc* h, const Args<T>& a);

// Sugar: S^{n+1} from S^n and u^n into the other buffer (after the transport of c, which
// reads S^n).
template <class LAT, typename T>
void enqueue_sugar(lbm_wenoc* h, const Args<T>& a) {
  if (!h->sugar) return;
  const dim3 blk(kLbmThreads);
  const dim3 grd((a.nx + kLbmThreads - 1) / kLbmThreads, a.ny, a.nz);
  cudaStream_t s = h->stream;
  launch(h, K_SUGAR, [&] { lw::sugar_kernel<T, LAT::DIM><<<grd, blk, 0, s>>>(a); });
  h->cur ^= 1;
}

// Particle class k's concentration buffer (class 0 is c).
template <typename T>
T* class_ptr(const lbm_wenoc* h, int k) {
  if (k == 0) return reinterpret_cast<T*>(h->ws + h->L.c);
  const size_t stride = align_up((size_t)h->n * sizeof(T), 256);
  return reinterpret_cast<T*>(h->ws + h->L.cls + (size_t)(k - 1) * stride);
}

// phi_tot / phi0 = sum of the classes, into L.ctot (the force's concentration).
template <typename T>
void enqueue_class_sum(lbm_wenoc* h) {
  lw::ClassPtrs<T> cp{};
  cp.count = h->ncls;
  for (int k = 0; k < h->ncls; ++k) cp.c[k] = class_ptr<T>(h, k);
  const long long n = h->n;
  T* out = reinterpret_cast<T*>(h->ws + h->L.ctot);
  launch(h, K_OTHER, [&] {
    lw::class_sum_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(cp, out, n);
  });
}

template <class LAT, typename T>
void enqueue_step(lbm_wenoc* h, int parity) {
  Args<T> a = make_args<T>(h);
  const dim3 blk(kLbmThreads);
  const dim3 grd((a.nx + kLbmThreads - 1) / kLbmThreads, a.ny, a.nz);
  cudaStream_t s = h->stream;
  Args<T> af = a;  // the fluid step's force reads phi_tot with several classes
  if (h->ncls > 1) af.c = reinterpret_cast<T*>(h->ws + h->L.ctot);
  if (!h->frozen) {
    launch(h, K_LBM, [&] {
      if (LAT::DIM == 2) {
        if (h->sugar)
          parity == 0 ? lw::lbm_d2q9_kernel<T, 0, true><<<grd, blk, 0, s>>>(af)
                      : lw::lbm_d2q9_kernel<T, 1, true><<<grd, blk, 0, s>>>(af);
        else if (parity == 0)
          lw::lbm_d2q9_kernel<T, 0><<<grd, blk, 0, s>>>(af);
        else
          lw::lbm_d2q9_kernel<T, 1><<<grd, blk, 0, s>>>(af);
      } else {
        if (h->sugar)
          parity == 0 ? lw::lbm_d3q19_kernel<T, 0, true><<<grd, blk, 0, s>>>(af)
                      : lw::lbm_d3q19_kernel<T, 1, true><<<grd, blk, 0, s>>>(af);
        else if (parity == 0)
          lw::lbm_d3q19_kernel<T, 0><<<grd, blk, 0, s>>>(af);
        else
          lw::lbm_d3q19_kernel<T, 1><<<grd, blk, 0, s>>>(af);
      }
    });
  }
  if (h->ncls == 1) {
    enqueue_transport<LAT, T>(h, a);
  } else {
    // each class with its own settling velocity and deposit slot
    for (int k = 0; k < h->ncls; ++k) {
      Args<T> ak = a;
      ak.c = class_ptr<T>(h, k);
      ak.vs = T(h->p.class_vs[k]);
      ak.scalars = a.scalars + kClassDeposit + k;
      enqueue_transport<LAT, T>(h, ak);
    }
    enqueue_class_sum<T>(h);
  }
  enqueue_sugar<LAT, T>(h, a);
}

// The three RK stages (and the deposit) of one step on the fields a points at.
template <class LAT, typename T>
void enqueue_transport(lbm_wenoc* h, const Args<T>& a) {
  const dim3 blk(kLbmThreads);
  const dim3 grd((a.nx + kLbmThreads - 1) / kLbmThreads, a.ny, a.nz);
  cudaStream_t s = h->stream;
  const long long nfloor = (long long)a.nx * (LAT::DIM == 3 ? a.ny : 1);
  const int dep_blocks = (int)std::min<long long>(lw::kMaxReduceBlocks, (nfloor + 4095) / 4096);
  if (std::is_same<T, float>::value && LAT::DIM == 2 && h->sweep) {
    const Args<float>& af = reinterpret_cast<const Args<float>&>(a);
    float* c_out = reinterpret_cast<float*>(h->ws + (h->cur ? h->L.c : h->L.c1));
    launch(h, K_RK3_SWEEP, [&] { lw::launch_sweep2d(af, c_out, h->sweep_geom, s); });
    h->cur ^= 1;
    return;
  }
  if (LAT::DIM == 2 && h->stage2d) {
    const int H = h->stage2d_rows;
    if (std::is_same<T, float>::value && h->wide) {
      const Args<float>& af = reinterpret_cast<const Args<float>&>(a);
      launch(h, K_STAGE1, [&] { lw::launch_stage2d_wide<1>(af, af.c, af.c1, H, s); });
      launch(h, K_STAGE2, [&] { lw::launch_stage2d_wide<2>(af, af.c1, af.c2, H, s); });
      launch(h, K_STAGE3, [&] { lw::launch_stage2d_wide<3>(af, af.c2, af.c, H, s); });  // + deposit
      return;
    }
    // one column per thread, FP32 or FP64 (the validation build's 2D path)
    launch(h, K_STAGE1, [&] { lw::launch_stage2d<1, T>(a, a.c, a.c1, H, s); });
    launch(h, K_STAGE2, [&] { lw::launch_stage2d<2, T>(a, a.c1, a.c2, H, s); });
    launch(h, K_STAGE3, [&] { lw::launch_stage2d<3, T>(a, a.c2, a.c, H, s); });  // + deposit
    return;
  }
  if (std::is_same<T, float>::value && LAT::DIM == 3 && h->sweep3d && h->wide3d) {
    const Args<float>& af = reinterpret_cast<const Args<float>&>(a);
    const int H = h->sweep3d_rows;
    launch(h, K_STAGE1, [&] { lw::launch_sweep3d_wide<1>(af, af.c, af.c1, H, s); });
    launch(h, K_STAGE2, [&] { lw::launch_sweep3d_wide<2>(af, af.c1, af.c2, H, s); });
    launch(h, K_DEPOSIT, [&] {
      lw::deposit_kernel<T><<<dep_blocks, lw::kReduceThreads, 0, s>>>(a, nfloor);
    });
    launch(h, K_STAGE3, [&] { lw::launch_sweep3d_wide<3>(af, af.c2, af.c, H, s); });
    return;
  }
  if (std::is_same<T, float>::value && LAT::DIM == 3 && h->sweep3d) {
    const Args<float>& af = reinterpret_cast<const Args<float>&>(a);
    const int H = h->sweep3d_rows;
    launch(h, K_STAGE1, [&] { lw::launch_sweep3d<1>(af, af.c, af.c1, H, s); });
    launch(h, K_STAGE2, [&] { lw::launch_sweep3d<2>(af, af.c1, af.c2, H, s); });
    launch(h, K_DEPOSIT, [&] {
      lw::deposit_kernel<T><<<dep_blocks, lw::kReduceThreads, 0, s>>>(a, nfloor);
    });
    launch(h, K_STAGE3, [&] { lw::launch_sweep3d<3>(af, af.c2, af.c, H, s); });
    return;
  }
  launch(h, K_STAGE1, [&] { lw::rk_stage_kernel<T, LAT::DIM, 1><<<grd, blk, 0, s>>>(a); });
  launch(h, K_STAGE2, [&] { lw::rk_stage_kernel<T, LAT::DIM, 2><<<grd, blk, 0, s>>>(a); });
  if (h->walls)
    launch(h, K_DEPOSIT, [&] {
      lw::deposit_kernel<T><<<dep_blocks, lw::kReduceThreads, 0, s>>>(a, nfloor);
    });
  launch(h, K_STAGE3, [&] { lw::rk_stage_kernel<T, LAT::DIM, 3><<<grd, blk, 0, s>>>(a); });
}

void enqueue_one(lbm_wenoc* h, int parity) {
  if (h->p.dim == 2) {
    if (h->fp64)
      enqueue_step<D2Q9, double>(h, parity);
    else
      enqueue_step<D2Q9, float>(h, parity);
  } else {
    if (h->fp64)
      enqueue_step<D3Q19, double>(h, parity);
    else
      enqueue_step<D3Q19, float>(h, parity);
  }
}

// `count` steps from AA parity `parity`.
void enqueue_many(lbm_wenoc* h, int parity, int64_t count) {
  for (int64_t k = 0; k < count; ++k) enqueue_one(h, h->frozen ? 0 : (int)((parity + k) & 1));
}

void destroy_graphs(lbm_wenoc* h) {
  for (int i = 0; i < 4; ++i) {
    if (h->graph_many[i]) cudaGraphExecDestroy(h->graph_many[i]);
    if (h->graph_one[i]) cudaGraphExecDestroy(h->graph_one[i]);
    h->graph_many[i] = h->graph_one[i] = nullptr;
  }
}

// Capture `count` steps starting at `parity` on a private stream.
int capture_graph(lbm_wenoc* h, int parity, int count, cudaGraphExec_t* out) {
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return LW_ECUDA;
  cudaStream_t saved = h->stream;
  const int64_t saved_launches = h->launches;
  const int saved_cur = h->cur;
  h->stream = cap;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue_many(h, parity, count);
    e = cudaStreamEndCapture(cap, &g);
  }
  h->stream = saved;
  h->launches = saved_launches;
  h->cur = saved_cur;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  return e == cudaSuccess ? LW_OK : LW_ECUDA;
}

int launches_per_step(const lbm_wenoc* h) {
  if (h->sweep) return h->frozen ? 1 : 2;
  const int classes = h->ncls > 1 ? h->ncls : 1, sum = h->ncls > 1 ? 1 : 0;
  const int per_class = (h->stage2d || h->sweep3d) ? (h->sweep3d ? 4 : 3) : 3 + (h->walls ? 1 : 0);
  return (h->frozen ? 0 : 1) + classes * per_class + sum + (h->sugar ? 1 : 0);
}

int64_t launches_for(const lbm_wenoc* h, int64_t count) { return (int64_t)launches_per_step(h) * count; }

int sync_and_status(lbm_wenoc* h) {
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
  unsigned st[2] = {0, 0};
  if (cudaMemcpy(st, h->ws + h->L.status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return LW_ECUDA;
  if (st[0] & lw::kStatusTimeout) return LW_ETIMEOUT;
  if (st[0] & lw::kStatusUnstable) return LW_EUNSTABLE;
  return LW_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class LAT, typename T>
void launch_fields(lbm_wenoc* h, T* rho, T* u) {
  Args<T> a = make_args<T>(h);
  if (h->ncls > 1) a.c = reinterpret_cast<T*>(h->ws + h->L.ctot);  // the force reads phi_tot
  const dim3 blk(kLbmThreads);
  const dim3 grd((a.nx + kLbmThreads - 1) / kLbmThreads, a.ny, a.nz);
  if (h->parity == 0)
    lw::fields_kernel<LAT, T, 0><<<grd, blk, 0, h->stream>>>(a, rho, u);
  else
    lw::fields_kernel<LAT, T, 1><<<grd, blk, 0, h->stream>>>(a, rho, u);
}

template <class LAT, typename T>
void launch_init(lbm_wenoc* h, const T* u0) {
  Args<T> a = make_args<T>(h);
  const dim3 blk(kLbmThreads);
  const dim3 grd((a.nx + kLbmThreads - 1) / kLbmThreads, a.ny, a.nz);
  lw::init_kernel<LAT, T><<<grd, blk, 0, h->stream>>>(a, u0);
}

template <typename T>
__global__ void fill_kernel(T* p, long long n, T v) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) p[k] = v;
}

}  // namespace

extern "C" {

int lbm_wenoc_workspace_bytes(const lbm_wenoc_params* p, size_t* bytes) {
  if (!bytes) return LW_EINVAL;
  int rc = check_params(p);
  if (rc != LW_OK) return rc;
  *bytes = make_layout(*p).total;
  return LW_OK;
}

int lbm_wenoc_create(const lbm_wenoc_params* p, void* dev_workspace, size_t bytes, void* cuda_stream,
                     lbm_wenoc** out) {
  if (!out) return LW_EINVAL;
  *out = nullptr;
  int rc = check_params(p);
  if (rc != LW_OK) return rc;
  if (!dev_workspace || (reinterpret_cast<uintptr_t>(dev_workspace) & 255u) != 0) return LW_EINVAL;
  Layout L = make_layout(*p);
  if (bytes < L.total) return LW_ENOMEM;
  lbm_wenoc* h = new (std::nothrow) lbm_wenoc();
  if (!h) return LW_ENOMEM;
  h->p = *p;
  if (h->p.dim == 2) h->p.nz = 1;
  if (h->p.u_cap <= 0.0) h->p.u_cap = 0.1;
  h->L = L;
  h->ws = static_cast<unsigned char*>(dev_workspace);
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->fp64 = (p->flags & LW_FP64) != 0;
  h->walls = (p->flags & LW_PERIODIC_VERTICAL) == 0;
  h->frozen = (p->flags & LW_FROZEN_VELOCITY) != 0;
  h->sugar = (p->flags & LW_SUGAR) != 0;
  const bool variant = (p->flags & (LW_WENO3 | LW_SIGN_SPLIT)) != 0;  // transport-scheme variant
  h->use_graphs = (p->flags & LW_NO_GRAPH) == 0;
  h->n = (long long)p->nx * p->ny * (p->dim == 3 ? p->nz : 1);
  h->ncls = classes_of(*p);
  double vs_max = p->settling_velocity;
  if (h->ncls > 1) {
    vs_max = p->class_vs[0];
    for (int k = 1; k < h->ncls; ++k) vs_max = std::max(vs_max, p->class_vs[k]);
  }
  h->alpha = p->lf_alpha > 0.0 ? p->lf_alpha : vs_max + h->p.u_cap;
  cudaGetDevice(&h->device);
  h->sweep = !h->fp64 && !variant && h->p.dim == 2 && lw::sweep2d_supported(p->nx, p->ny, h->walls) &&
             (p->flags & LW_FUSED_RK3) != 0;
  // the row-sweep stage kernels take the scheme variants and the sugar scalar too
  // (FP64 too: the validation build runs the one-column form)
  h->stage2d = h->p.dim == 2 && h->walls && !h->sweep && (p->nx + lw::kS2T - 1) / lw::kS2T <= lw::kMaxReduceBlocks;
  h->wide = h->stage2d && !h->fp64 && !h->sugar && !variant && !(p->flags & LW_ONE_COLUMN);
  if (h->stage2d) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms <= 0) sms = 148;
    if (h->wide) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lw::rk_stage2d_wide_kernel<3>, lw::kWT, 0) !=
              cudaSuccess ||
          per_sm <= 0)
        per_sm = 1;
      h->wide_per_sm = per_sm;
      h->stage2d_rows = lw::stage2d_wide_rows(p->nx, p->ny, sms, per_sm, 0);
    } else {
      h->stage2d_rows = lw::stage2d_rows(p->nx, p->ny, sms, 0);
    }
  }
  if (h->sweep) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms <= 0) sms = 148;
    h->sweep_geom = lw::sweep2d_geometry(p->nx, p->ny, sms, 0);
    if (cudaFuncSetAttribute(lw::rk3_sweep2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lw::sweep2d_smem()) != cudaSuccess) {
      delete h;
      return LW_ECUDA;
    }
  }
  h->sweep3d = !h->fp64 && h->p.dim == 3 && lw::sweep3d_supported(h->p.nz, h->walls);
  if (h->sweep3d) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms <= 0) sms = 148;
    h->wide3d = !h->sugar && !variant && !(p->flags & LW_ONE_COLUMN);
    if (lw::sweep3d_prepare() != cudaSuccess || (h->wide3d && lw::sweep3d_wide_prepare() != cudaSuccess)) {
      delete h;
      return LW_ECUDA;
    }
    if (h->wide3d) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lw::rk_sweep3d_wide_kernel<3>, lw::kV3T,
                                                        lw::sweep3d_wide_smem()) != cudaSuccess ||
          per_sm <= 0)
        per_sm = 1;
      h->wide3d_per_sm = per_sm;
      h->sweep3d_rows = lw::sweep3d_wide_rows(p->nx, p->ny, p->nz, sms, per_sm, 0);
    } else {
      h->sweep3d_rows = lw::sweep3d_rows(p->nx, p->ny, p->nz, sms, 0);
    }
  }
  h->kind_names.assign(kKindNames, kKindNames + K_COUNT);
  h->kind_launches.assign(K_COUNT, 0);
  h->kind_ms.assign(K_COUNT, 0.0);
  *out = h;
  return LW_OK;
}

int lbm_wenoc_init(lbm_wenoc* h, const void* c0, const void* u0) {
  NvtxRange range("lbm_wenoc_init");
  if (!h || !c0) return LW_EINVAL;
  h->cur = 0;
  const size_t es = h->fp64 ? 8 : 4;
  const size_t cbytes = (size_t)h->n * es;
  const size_t ubytes = cbytes * h->p.dim;
  // c0 -> c buffer (device or host source); u0 -> c1 scratch first (init reads it)
  cudaMemcpyKind kc = is_device_pointer(c0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(h->ws + h->L.c, c0, cbytes, kc, h->stream) != cudaSuccess) return LW_ECUDA;
  const void* u0dev = nullptr;
  if (u0) {
    cudaMemcpyKind ku = is_device_pointer(u0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // stage through the population buffer's tail is unsafe; use u itself then copy in kernel
    if (cudaMemcpyAsync(h->ws + h->L.u, u0, ubytes, ku, h->stream) != cudaSuccess) return LW_ECUDA;
    u0dev = h->ws + h->L.u;
  }
  if (cudaMemsetAsync(h->ws + h->L.scalars, 0, sizeof(double) * kScalars, h->stream) != cudaSuccess)
    return LW_ECUDA;
  if (cudaMemsetAsync(h->ws + h->L.status, 0, sizeof(unsigned) * 4, h->stream) != cudaSuccess) return LW_ECUDA;
  if (h->sugar && cudaMemsetAsync(h->ws + h->L.sa, 0, cbytes, h->stream) != cudaSuccess) return LW_ECUDA;
  if (h->ncls > 1) {  // c0 is class 0; the others start empty, so phi_tot = c0
    if (cudaMemsetAsync(h->ws + h->L.cls, 0, h->L.ctot - h->L.cls, h->stream) != cudaSuccess) return LW_ECUDA;
    if (cudaMemcpyAsync(h->ws + h->L.ctot, h->ws + h->L.c, cbytes, cudaMemcpyDeviceToDevice, h->stream) !=
        cudaSuccess)
      return LW_ECUDA;
  }
  if (h->p.dim == 2) {
    if (h->fp64)
      launch_init<D2Q9, double>(h, static_cast<const double*>(u0dev));
    else
      launch_init<D2Q9, float>(h, static_cast<const float*>(u0dev));
  } else {
    if (h->fp64)
      launch_init<D3Q19, double>(h, static_cast<const double*>(u0dev));
    else
      launch_init<D3Q19, float>(h, static_cast<const float*>(u0dev));
  }
  if (cudaGetLastError() != cudaSuccess) return LW_ECUDA;
  // host sources may be pageable: make the call safe to return
  if (kc == cudaMemcpyHostToDevice || (u0 && !is_device_pointer(u0)))
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
  h->parity = 0;
  h->cur = 0;
  h->steps = 0;
  h->initialised = true;
  return LW_OK;
}

int lbm_wenoc_step(lbm_wenoc* h, int64_t nsteps) {
  NvtxRange range("lbm_wenoc_step");
  if (!h || nsteps < 0) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  int64_t left = nsteps;
  if (h->use_graphs && !h->profiling) {
    while (left > 0) {
      const int par = h->frozen ? 0 : h->parity;
      const int key = par * 2 + h->cur;
      cudaGraphExec_t* slot;
      int count;
      if (left >= lbm_wenoc::kGraphSteps) {
        slot = &h->graph_many[key];
        count = lbm_wenoc::kGraphSteps;
      } else {
        slot = &h->graph_one[key];
        count = 1;
      }
      if (!*slot) {
        int rc = capture_graph(h, par, count, slot);
        if (rc != LW_OK) return rc;
      }
      if (cudaGraphLaunch(*slot, h->stream) != cudaSuccess) return LW_ECUDA;
      h->launches += launches_for(h, count);
      if (!h->frozen) h->parity = (h->parity + count) & 1;
      if (h->sweep || h->sugar) h->cur = (h->cur + count) & 1;
      h->steps += count;
      left -= count;
    }
  } else {
    if (left > 0) {
      enqueue_many(h, h->frozen ? 0 : h->parity, left);
      if (!h->frozen) h->parity = (int)((h->parity + left) & 1);
      h->steps += left;
    }
  }
  if (cudaGetLastError() != cudaSuccess) return LW_ECUDA;
  return LW_OK;
}

int lbm_wenoc_deposited_mass(lbm_wenoc* h, double* out) {
  if (!h || !out) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  int rc = sync_and_status(h);
  if (rc == LW_ECUDA) return rc;
  if (h->ncls > 1) {
    double dep[kScalars];
    if (cudaMemcpy(dep, h->ws + h->L.scalars, sizeof(dep), cudaMemcpyDeviceToHost) != cudaSuccess) return LW_ECUDA;
    double tot = 0.0;
    for (int k = 0; k < h->ncls; ++k) tot += dep[kClassDeposit + k];
    *out = tot;
    return rc;
  }
  if (cudaMemcpy(out, h->ws + h->L.scalars, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LW_ECUDA;
  return rc;
}

// Sum of c (or of the classes) over the first `count` nodes, FP64 in a fixed order, into *out.
static int sum_c(lbm_wenoc* h, long long count, double* out) {
  if (count <= 0) {
    *out = 0.0;
    return LW_OK;
  }
  const int blocks = (int)std::min<long long>(lw::kMaxReduceBlocks, (count + 8191) / 8192);
  const bool classes = h->ncls > 1;  // the sum of the classes
  if (h->fp64) {
    Args<double> a = make_args<double>(h);
    const double* src = classes ? reinterpret_cast<const double*>(h->ws + h->L.ctot) : a.c;
    lw::sum_kernel<double><<<blocks, lw::kReduceThreads, 0, h->stream>>>(a, src, count);
  } else {
    Args<float> a = make_args<float>(h);
    const float* src = classes ? reinterpret_cast<const float*>(h->ws + h->L.ctot) : a.c;
    lw::sum_kernel<float><<<blocks, lw::kReduceThreads, 0, h->stream>>>(a, src, count);
  }
  if (cudaGetLastError() != cudaSuccess) return LW_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
  if (cudaMemcpy(out, h->ws + h->L.scalars + sizeof(double), sizeof(double), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return LW_ECUDA;
  return LW_OK;
}

int lbm_wenoc_total_mass(lbm_wenoc* h, double* out) {
  if (!h || !out) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  return sum_c(h, h->n, out);
}

int lbm_wenoc_mass_below(lbm_wenoc* h, int32_t level, double* out) {
  if (!h || !out) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  const int nv = h->p.dim == 3 ? h->p.nz : h->p.ny;
  if (level < 0 || level > nv) return LW_EINVAL;
  // the vertical axis is the slowest: the levels below the plane are the first nodes
  double below = 0.0, dep = 0.0;
  int rc = sum_c(h, (long long)level * (h->n / nv), &below);
  if (rc != LW_OK) return rc;
  rc = lbm_wenoc_deposited_mass(h, &dep);
  if (rc != LW_OK && rc != LW_EUNSTABLE) return rc;
  *out = below + dep;
  return rc;
}

int lbm_wenoc_fields(lbm_wenoc* h, void* rho, void* u, void* c) {
  NvtxRange range("lbm_wenoc_fields");
  if (!h) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  const size_t es = h->fp64 ? 8 : 4;
  const size_t cbytes = (size_t)h->n * es;
  // Compute rho and u into the stage buffers (free between steps), then copy out.
  unsigned char* rho_dev = h->ws + h->L.c2;  // free between steps on every path
  unsigned char* u_dev = h->ws + h->L.u;
  if (rho || u) {
    if (h->frozen) {
      const int blocks = (int)((h->n + 255) / 256);
      if (h->fp64)
        fill_kernel<double><<<blocks, 256, 0, h->stream>>>(reinterpret_cast<double*>(rho_dev), h->n, 1.0);
      else
        fill_kernel<float><<<blocks, 256, 0, h->stream>>>(reinterpret_cast<float*>(rho_dev), h->n, 1.0f);
    } else {
      // The velocity buffer is scratch between steps (rewritten by the next step), so
      // the fields kernel may overwrite it with the velocity of the current state.
      if (h->p.dim == 2) {
        if (h->fp64)
          launch_fields<D2Q9, double>(h, reinterpret_cast<double*>(rho_dev), reinterpret_cast<double*>(u_dev));
        else
          launch_fields<D2Q9, float>(h, reinterpret_cast<float*>(rho_dev), reinterpret_cast<float*>(u_dev));
      } else {
        if (h->fp64)
          launch_fields<D3Q19, double>(h, reinterpret_cast<double*>(rho_dev), reinterpret_cast<double*>(u_dev));
        else
          launch_fields<D3Q19, float>(h, reinterpret_cast<float*>(rho_dev), reinterpret_cast<float*>(u_dev));
      }
    }
    if (cudaGetLastError() != cudaSuccess) return LW_ECUDA;
  }
  auto copy_out = [&](void* dst, const void* src, size_t nbytes) -> bool {
    cudaMemcpyKind k = is_device_pointer(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    return cudaMemcpyAsync(dst, src, nbytes, k, h->stream) == cudaSuccess;
  };
  if (rho && !copy_out(rho, rho_dev, cbytes)) return LW_ECUDA;
  if (u && !copy_out(u, u_dev, cbytes * h->p.dim)) return LW_ECUDA;
  const size_t c_off = h->ncls > 1 ? h->L.ctot : (h->sweep && h->cur ? h->L.c1 : h->L.c);
  if (c && !copy_out(c, h->ws + c_off, cbytes)) return LW_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
  return LW_OK;
}

// ---- resumable state: a header, then the fields a step reads (populations, the current c,
// u, the current S, the class fields) and the FP64 deposit scalars
namespace {

constexpr uint32_t kStateMagic = 0x5453574cu;  // "LWST"
constexpr uint32_t kStateVersion = 1;

struct StateHeader {
  uint32_t magic, version;
  lbm_wenoc_params p;
  int32_t parity, cur;
  int64_t steps;
  uint64_t bytes;
};

struct StateRegion {
  size_t off, bytes;  // in the workspace
};

std::vector<StateRegion> state_regions(const lbm_wenoc* h) {
  const size_t es = h->fp64 ? 8 : 4, n = (size_t)h->n;
  const Layout& L = h->L;
  std::vector<StateRegion> r;
  r.push_back({L.g, (size_t)(h->p.dim == 2 ? 9 : 19) * n * es});
  r.push_back({h->sweep && h->cur ? L.c1 : L.c, n * es});
  r.push_back({L.u, (size_t)h->p.dim * n * es});  // read by a frozen-velocity step
  if (h->sugar) r.push_back({h->cur ? L.sb : L.sa, n * es});
  if (h->ncls > 1) r.push_back({L.cls, L.ctot + n * es - L.cls});
  r.push_back({L.scalars, sizeof(double) * kScalars});
  return r;
}

// the same simulation (field by field: the struct has padding); LW_NO_GRAPH only changes
// how steps are launched
bool same_params(const lbm_wenoc_params& a, const lbm_wenoc_params& b) {
  bool eq = a.dim == b.dim && a.nx == b.nx && a.ny == b.ny && (a.dim == 2 || a.nz == b.nz) && a.tau == b.tau &&
            a.gravity == b.gravity && a.density_contrast == b.density_contrast &&
            a.settling_velocity == b.settling_velocity && a.diffusivity == b.diffusivity &&
            a.lf_alpha == b.lf_alpha && a.u_cap == b.u_cap && (a.flags | LW_NO_GRAPH) == (b.flags | LW_NO_GRAPH) &&
            a.sugar_contrast == b.sugar_contrast && a.sugar_diffusivity == b.sugar_diffusivity && a.phi0 == b.phi0 &&
            a.vs_sugar == b.vs_sugar && a.n_classes == b.n_classes;
  for (int d = 0; d < 3; ++d) eq = eq && a.body_force[d] == b.body_force[d];
  for (int k = 0; k < 8; ++k) eq = eq && a.class_vs[k] == b.class_vs[k];
  return eq;
}

size_t state_bytes(const lbm_wenoc* h) {
  size_t b = align_up(sizeof(StateHeader), 256);
  for (const StateRegion& r : state_regions(h)) b += align_up(r.bytes, 256);
  return b;
}

}  // namespace

int lbm_wenoc_state_bytes(const lbm_wenoc* h, size_t* bytes) {
  if (!h || !bytes) return LW_EINVAL;
  *bytes = state_bytes(h);
  return LW_OK;
}

int lbm_wenoc_save_state(lbm_wenoc* h, void* dst, size_t bytes) {
  if (!h || !dst) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  const size_t need = state_bytes(h);
  if (bytes < need) return LW_ENOMEM;
  StateHeader hd{};
  hd.magic = kStateMagic;
  hd.version = kStateVersion;
  hd.p = h->p;
  hd.parity = h->parity;
  hd.cur = h->cur;
  hd.steps = h->steps;
  hd.bytes = need;
  unsigned char* d = static_cast<unsigned char*>(dst);
  if (cudaMemcpyAsync(d, &hd, sizeof(hd), cudaMemcpyDefault, h->stream) != cudaSuccess) return LW_ECUDA;
  size_t off = align_up(sizeof(StateHeader), 256);
  for (const StateRegion& r : state_regions(h)) {
    if (cudaMemcpyAsync(d + off, h->ws + r.off, r.bytes, cudaMemcpyDefault, h->stream) != cudaSuccess)
      return LW_ECUDA;
    off += align_up(r.bytes, 256);
  }
  // the header lives on this stack frame and dst may be pageable host memory
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? LW_OK : LW_ECUDA;
}

int lbm_wenoc_load_state(lbm_wenoc* h, const void* src, size_t bytes) {
  if (!h || !src || bytes < sizeof(StateHeader)) return LW_EINVAL;
  StateHeader hd{};
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
  if (cudaMemcpy(&hd, src, sizeof(hd), cudaMemcpyDefault) != cudaSuccess) return LW_ECUDA;
  if (hd.magic != kStateMagic || hd.version != kStateVersion || !same_params(hd.p, h->p) ||
      hd.parity < 0 || hd.parity > 1 || hd.cur < 0 || hd.cur > 1 || hd.steps < 0)
    return LW_EINVAL;
  h->cur = hd.cur;  // selects the buffers the regions go to
  if (hd.bytes != state_bytes(h) || bytes < hd.bytes) return LW_EINVAL;
  const unsigned char* sp = static_cast<const unsigned char*>(src);
  size_t off = align_up(sizeof(StateHeader), 256);
  for (const StateRegion& r : state_regions(h)) {
    if (cudaMemcpyAsync(h->ws + r.off, sp + off, r.bytes, cudaMemcpyDefault, h->stream) != cudaSuccess)
      return LW_ECUDA;
    off += align_up(r.bytes, 256);
  }
  if (cudaMemsetAsync(h->ws + h->L.status, 0, sizeof(unsigned) * 4, h->stream) != cudaSuccess) return LW_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
  h->parity = hd.parity;
  h->steps = hd.steps;
  h->initialised = true;
  return LW_OK;
}

int lbm_wenoc_status(lbm_wenoc* h) {
  if (!h) return LW_EINVAL;
  return sync_and_status(h);
}

int64_t lbm_wenoc_steps(const lbm_wenoc* h) { return h ? h->steps : -1; }

int64_t lbm_wenoc_launch_count(const lbm_wenoc* h) { return h ? h->launches : -1; }

int lbm_wenoc_set_sugar(lbm_wenoc* h, const void* S0) {
  if (!h || !S0 || !h->sugar) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  const size_t bytes = (size_t)h->n * (h->fp64 ? 8 : 4);
  cudaMemcpyKind k = is_device_pointer(S0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(h->ws + (h->cur ? h->L.sb : h->L.sa), S0, bytes, k, h->stream) != cudaSuccess)
    return LW_ECUDA;
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? LW_OK : LW_ECUDA;
}

int lbm_wenoc_set_class(lbm_wenoc* h, int32_t k, const void* ck) {
  if (!h || !ck || h->ncls < 2 || k < 0 || k >= h->ncls) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  const size_t bytes = (size_t)h->n * (h->fp64 ? 8 : 4);
  void* dst = h->fp64 ? (void*)class_ptr<double>(h, k) : (void*)class_ptr<float>(h, k);
  cudaMemcpyKind kind = is_device_pointer(ck) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpyAsync(dst, ck, bytes, kind, h->stream) != cudaSuccess) return LW_ECUDA;
  if (h->fp64)
    enqueue_class_sum<double>(h);
  else
    enqueue_class_sum<float>(h);
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? LW_OK : LW_ECUDA;
}

int lbm_wenoc_class(lbm_wenoc* h, int32_t k, void* out) {
  if (!h || !out || h->ncls < 2 || k < 0 || k >= h->ncls) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  const size_t bytes = (size_t)h->n * (h->fp64 ? 8 : 4);
  const void* src = h->fp64 ? (const void*)class_ptr<double>(h, k) : (const void*)class_ptr<float>(h, k);
  cudaMemcpyKind kind = is_device_pointer(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (cudaMemcpyAsync(out, src, bytes, kind, h->stream) != cudaSuccess) return LW_ECUDA;
  return sync_and_status(h);
}

int lbm_wenoc_class_deposit(lbm_wenoc* h, int32_t k, double* out) {
  if (!h || !out || h->ncls < 2 || k < 0 || k >= h->ncls) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  int rc = sync_and_status(h);
  if (rc == LW_ECUDA) return rc;
  if (cudaMemcpy(out, h->ws + h->L.scalars + sizeof(double) * (kClassDeposit + k), sizeof(double),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return LW_ECUDA;
  return rc;
}

int lbm_wenoc_sugar(lbm_wenoc* h, void* S_out) {
  if (!h || !S_out || !h->sugar) return LW_EINVAL;
  if (!h->initialised) return LW_ESTATE;
  const size_t bytes = (size_t)h->n * (h->fp64 ? 8 : 4);
  cudaMemcpyKind k = is_device_pointer(S_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (cudaMemcpyAsync(S_out, h->ws + (h->cur ? h->L.sb : h->L.sa), bytes, k, h->stream) != cudaSuccess)
    return LW_ECUDA;
  return sync_and_status(h);
}

int lbm_wenoc_profile_enable(lbm_wenoc* h, int enable) {
  if (!h) return LW_EINVAL;
  h->profiling = enable != 0;
  return LW_OK;
}

int lbm_wenoc_profile_read(lbm_wenoc* h, lbm_wenoc_kernel_stat* out, int max, int* count, int reset) {
  if (!h || !count) return LW_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
  fold_pending(h);
  int k = 0;
  for (int i = 0; i < K_COUNT; ++i) {
    if (h->kind_launches[i] == 0) continue;
    if (out && k < max) {
      std::memset(out[k].name, 0, sizeof(out[k].name));
      std::strncpy(out[k].name, h->kind_names[i].c_str(), sizeof(out[k].name) - 1);
      out[k].launches = h->kind_launches[i];
      out[k].total_ms = h->kind_ms[i];
    }
    ++k;
  }
  *count = k;
  if (reset) {
    std::fill(h->kind_launches.begin(), h->kind_launches.end(), 0);
    std::fill(h->kind_ms.begin(), h->kind_ms.end(), 0.0);
  }
  return LW_OK;
}

int lbm_wenoc_set_segment_rows(lbm_wenoc* h, int32_t rows) {
  if (!h || rows < 0) return LW_EINVAL;
  if (h->sweep3d || h->stage2d) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms <= 0) sms = 148;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
    destroy_graphs(h);
    if (h->sweep3d)
      h->sweep3d_rows = h->wide3d ? lw::sweep3d_wide_rows(h->p.nx, h->p.ny, h->p.nz, sms, h->wide3d_per_sm, rows)
                                  : lw::sweep3d_rows(h->p.nx, h->p.ny, h->p.nz, sms, rows);
    if (h->stage2d)
      h->stage2d_rows = h->wide ? lw::stage2d_wide_rows(h->p.nx, h->p.ny, sms, h->wide_per_sm, rows)
                                : lw::stage2d_rows(h->p.nx, h->p.ny, sms, rows);
    return LW_OK;
  }
  if (!h->sweep) return LW_OK;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms <= 0) sms = 148;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LW_ECUDA;
  destroy_graphs(h);
  h->sweep_geom = lw::sweep2d_geometry(h->p.nx, h->p.ny, sms, rows);
  return LW_OK;
}

void lbm_wenoc_destroy(lbm_wenoc* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  fold_pending(h);
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  destroy_graphs(h);
  delete h;
}


}  // extern "C"

// ------------------------------------------------------------------------------------
// Batched simulations: one handle per instance over consecutive slices of one
// workspace, plus device tables, advanced together by one launch per kernel type.

struct lbm_wenoc_batch {
  std::vector<lbm_wenoc*> inst;
  std::vector<size_t> offsets;  // workspace offset of each instance
  std::vector<int> rows;        // segment rows of each instance's stage items
  unsigned char* ws = nullptr;
  size_t tables_off = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int lbm_blocks = 0, st_blocks = 0;
  lw::BatchTables tab{};
  int mode = 1;                  // 1: one cooperative launch per graph of steps; 2: per step a grouped
                                 // fluid launch and a cooperative stage launch; 0: grouped launches
  int grid = 0;                  // CTAs of the persistent launch (all resident at once)
  int64_t wait_limit = 1LL << 31;  // clock64 cycles a barrier wait may take (about 1 s)
  int skip_cta = -1;             // testing: this CTA leaves the next launch before its first barrier
  static constexpr int kGraphSteps = lw::kPersistSteps;
  cudaGraphExec_t graph_many[2] = {nullptr, nullptr};
  cudaGraphExec_t graph_one[2] = {nullptr, nullptr};
  int64_t launches = 0;
};

namespace {

bool batch_params_ok(const lbm_wenoc_params& p) {
  return check_params(&p) == LW_OK && p.dim == 2 && !(p.flags & LW_FP64) && !(p.flags & LW_PERIODIC_VERTICAL) &&
         !(p.flags & (LW_FROZEN_VELOCITY | LW_FUSED_RK3 | LW_SUGAR | LW_WENO3 | LW_SIGN_SPLIT | LW_ONE_COLUMN)) &&
         p.n_classes < 2 && (p.nx + lw::kWW - 1) / lw::kWW <= lw::kMaxReduceBlocks;
}

// Tables: the argument blocks, eight int tables, the barrier, status and work-counter words.
constexpr int kBatchSyncWords = 8 + 3 * lw::kPersistSteps;  // bar[2], status[2], pad, queue

size_t batch_tables_bytes(int count) {
  return align_up(sizeof(Args<float>) * count, 256) + align_up(sizeof(int) * (count + 1), 256) * 3 +
         align_up(sizeof(int) * count, 256) * 4 + align_up(sizeof(unsigned) * kBatchSyncWords, 256);
}

void batch_destroy_graphs(lbm_wenoc_batch* b) {
  for (int i = 0; i < 2; ++i) {
    if (b->graph_many[i]) cudaGraphExecDestroy(b->graph_many[i]);
    if (b->graph_one[i]) cudaGraphExecDestroy(b->graph_one[i]);
    b->graph_many[i] = b->graph_one[i] = nullptr;
  }
}

// Fill the device tables from the instances' current argument blocks and geometries.
int batch_upload_tables(lbm_wenoc_batch* b) {
  const int count = (int)b->inst.size();
  std::vector<Args<float>> args(count);
  std::vector<int> lstart(count + 1), lgx(count), sstart(count + 1), sstrips(count), srows(count), fstart(count + 1),
      fchunks(count);
  lstart[0] = sstart[0] = fstart[0] = 0;
  for (int i = 0; i < count; ++i) {
    lbm_wenoc* h = b->inst[i];
    args[i] = make_args<float>(h);
    lgx[i] = (h->p.nx + kLbmThreads - 1) / kLbmThreads;
    lstart[i + 1] = lstart[i] + lgx[i] * h->p.ny;
    sstrips[i] = (h->p.nx + lw::kWW - 1) / lw::kWW;
    srows[i] = std::min(std::min(b->rows[i] > 0 ? b->rows[i] : h->stage2d_rows, h->p.ny), lw::kWmaxH);
    const int segs = (h->p.ny + srows[i] - 1) / srows[i];
    sstart[i + 1] = sstart[i] + sstrips[i] * segs;
    fchunks[i] = (h->p.nx + lw::kFluidCols - 1) / lw::kFluidCols;
    fstart[i + 1] = fstart[i] + fchunks[i] * h->p.ny;
  }
  b->lbm_blocks = lstart[count];
  b->st_blocks = sstart[count];
  unsigned char* base = b->ws + b->tables_off;
  size_t off = 0;
  auto put = [&](const void* src, size_t nbytes) -> void* {
    unsigned char* dst = base + off;
    off += align_up(nbytes, 256);
    if (src && cudaMemcpyAsync(dst, src, nbytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess) return nullptr;
    return dst;
  };
  b->tab.args = static_cast<const Args<float>*>(put(args.data(), sizeof(Args<float>) * count));
  b->tab.lbm_start = static_cast<const int*>(put(lstart.data(), sizeof(int) * (count + 1)));
  b->tab.st_start = static_cast<const int*>(put(sstart.data(), sizeof(int) * (count + 1)));
  b->tab.fl_start = static_cast<const int*>(put(fstart.data(), sizeof(int) * (count + 1)));
  b->tab.lbm_gx = static_cast<const int*>(put(lgx.data(), sizeof(int) * count));
  b->tab.st_strips = static_cast<const int*>(put(sstrips.data(), sizeof(int) * count));
  b->tab.st_rows = static_cast<const int*>(put(srows.data(), sizeof(int) * count));
  b->tab.fl_chunks = static_cast<const int*>(put(fchunks.data(), sizeof(int) * count));
  unsigned* sync = static_cast<unsigned*>(put(nullptr, sizeof(unsigned) * kBatchSyncWords));
  b->tab.bar = sync;
  b->tab.status = sync + 2;
  b->tab.queue = sync + 8;
  b->tab.count = count;
  if (!b->tab.args || !b->tab.lbm_start || !b->tab.st_start || !b->tab.fl_start || !b->tab.lbm_gx ||
      !b->tab.st_strips || !b->tab.st_rows || !b->tab.fl_chunks)
    return LW_ECUDA;
  if (cudaMemsetAsync(sync, 0, sizeof(unsigned) * kBatchSyncWords, b->stream) != cudaSuccess) return LW_ECUDA;
  // the host vectors go out of scope: wait for the copies
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LW_ECUDA;
  batch_destroy_graphs(b);
  return LW_OK;
}

// `count` steps from AA parity `parity`: one persistent launch (count <= kPersistSteps), or
// four grouped launches per step.
cudaError_t batch_enqueue(lbm_wenoc_batch* b, cudaStream_t s, int parity, int count) {
  const lw::BatchTables t = b->tab;
  // one cooperative launch: the barrier words and the work counters start at zero (the
  // status word is kept)
  auto persistent_launch = [&](int par, int steps, int with_fluid) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(t.bar, 0, sizeof(unsigned) * 2, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t.queue, 0, sizeof(unsigned) * 3 * steps, s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(lw::kWT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const long long limit = (long long)b->wait_limit;
    return cudaLaunchKernelEx(&cfg, lw::batch_persistent_kernel, t, par, steps, limit, b->skip_cta, with_fluid);
  };
  if (b->mode == 1) return persistent_launch(parity, count, 1);
  if (b->mode == 2) {
    for (int k = 0; k < count; ++k) {
      const int par = (parity + k) & 1;
      if (par == 0)
        lw::lbm_d2q9_batch_kernel<0><<<b->lbm_blocks, kLbmThreads, 0, s>>>(t);
      else
        lw::lbm_d2q9_batch_kernel<1><<<b->lbm_blocks, kLbmThreads, 0, s>>>(t);
      const cudaError_t e = persistent_launch(par, 1, 0);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }
  for (int k = 0; k < count; ++k) {
    const int par = (parity + k) & 1;
    if (par == 0)
      lw::lbm_d2q9_batch_kernel<0><<<b->lbm_blocks, kLbmThreads, 0, s>>>(t);
    else
      lw::lbm_d2q9_batch_kernel<1><<<b->lbm_blocks, kLbmThreads, 0, s>>>(t);
    lw::stage2d_batch_kernel<1><<<b->st_blocks, lw::kWT, 0, s>>>(t);
    lw::stage2d_batch_kernel<2><<<b->st_blocks, lw::kWT, 0, s>>>(t);
    lw::stage2d_batch_kernel<3><<<b->st_blocks, lw::kWT, 0, s>>>(t);
  }
  return cudaGetLastError();
}

int batch_capture(lbm_wenoc_batch* b, int parity, int count, cudaGraphExec_t* out) {
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return LW_ECUDA;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = batch_enqueue(b, cap, parity, count);
    e = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  return e == cudaSuccess ? LW_OK : LW_ECUDA;
}

int64_t batch_launches(const lbm_wenoc_batch* b, int count) {
  return b->mode == 1 ? 1 : (b->mode == 2 ? 2LL * count : 4LL * count);
}

// Advance every instance; requires equal step counts (shared AA parity).  Graphs of
// kGraphSteps steps (and of one step for the rest) are captured once per parity.
int batch_advance(lbm_wenoc_batch* b, int64_t nsteps, bool require_init) {
  if (nsteps < 0) return LW_EINVAL;
  const int par = b->inst[0]->parity;
  for (lbm_wenoc* h : b->inst) {
    if (require_init && !h->initialised) return LW_ESTATE;
    if (h->parity != par || h->steps != b->inst[0]->steps) return LW_ESTATE;
  }
  int64_t left = nsteps;
  int parity = par;
  int64_t launches = 0;
  while (left > 0) {
    const bool many = left >= lbm_wenoc_batch::kGraphSteps;
    const int count = many ? lbm_wenoc_batch::kGraphSteps : 1;
    if (b->skip_cta >= 0) {  // testing launch: not captured
      if (batch_enqueue(b, b->stream, parity, count) != cudaSuccess) return LW_ECUDA;
      b->skip_cta = -1;
    } else {
      cudaGraphExec_t* slot = many ? &b->graph_many[parity] : &b->graph_one[parity];
      if (!*slot) {
        int rc = batch_capture(b, parity, count, slot);
        if (rc != LW_OK) return rc;
      }
      if (cudaGraphLaunch(*slot, b->stream) != cudaSuccess) return LW_ECUDA;
    }
    launches += batch_launches(b, count);
    parity = (parity + count) & 1;
    left -= count;
  }
  b->launches += launches;
  for (lbm_wenoc* h : b->inst) {
    h->parity = parity;
    h->steps += nsteps;
    h->launches += 4 * nsteps;
  }
  return cudaGetLastError() == cudaSuccess ? LW_OK : LW_ECUDA;
}

// Trial state of the autotuner: c = 0 and the fluid at rest in every instance.
int batch_trial_state(lbm_wenoc_batch* b) {
  for (lbm_wenoc* h : b->inst) {
    if (cudaMemsetAsync(h->ws + h->L.c, 0, (size_t)h->n * sizeof(float), b->stream) != cudaSuccess) return LW_ECUDA;
    if (cudaMemsetAsync(h->ws + h->L.scalars, 0, sizeof(double) * kScalars, b->stream) != cudaSuccess)
      return LW_ECUDA;
    if (cudaMemsetAsync(h->ws + h->L.status, 0, sizeof(unsigned) * 4, b->stream) != cudaSuccess) return LW_ECUDA;
    h->cur = 0;
    launch_init<D2Q9, float>(h, nullptr);
    h->parity = 0;
    h->steps = 0;
  }
  return LW_OK;
}

// Milliseconds of `steps` batched steps (after one untimed step).
int batch_time(lbm_wenoc_batch* b, int steps, cudaEvent_t e0, cudaEvent_t e1, float* ms) {
  int rc = batch_advance(b, 1, false);
  if (rc != LW_OK) return rc;
  cudaEventRecord(e0, b->stream);
  if ((rc = batch_advance(b, steps, false)) != LW_OK) return rc;
  cudaEventRecord(e1, b->stream);
  if (cudaEventSynchronize(e1) != cudaSuccess) return LW_ECUDA;
  return cudaEventElapsedTime(ms, e0, e1) == cudaSuccess ? LW_OK : LW_ECUDA;
}

}  // namespace

extern "C" {

int lbm_wenoc_batch_workspace_bytes(const lbm_wenoc_params* p, int32_t count, size_t* bytes) {
  if (!p || !bytes || count < 1) return LW_EINVAL;
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    if (!batch_params_ok(p[i])) return LW_EINVAL;
    total += align_up(make_layout(p[i]).total, 256);
  }
  *bytes = total + batch_tables_bytes(count);
  return LW_OK;
}

int lbm_wenoc_batch_create(const lbm_wenoc_params* p, int32_t count, void* dev_workspace, size_t bytes,
                           void* cuda_stream, lbm_wenoc_batch** out) {
  if (!out) return LW_EINVAL;
  *out = nullptr;
  size_t need = 0;
  int rc = lbm_wenoc_batch_workspace_bytes(p, count, &need);
  if (rc != LW_OK) return rc;
  if (!dev_workspace || (reinterpret_cast<uintptr_t>(dev_workspace) & 255u) != 0) return LW_EINVAL;
  if (bytes < need) return LW_ENOMEM;
  lbm_wenoc_batch* b = new (std::nothrow) lbm_wenoc_batch();
  if (!b) return LW_ENOMEM;
  b->ws = static_cast<unsigned char*>(dev_workspace);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&b->device);
  // every CTA of the persistent launch must be resident at once (the grid barrier waits
  // for all of them): as many as the SMs hold
  int sms = 0, per_sm = 0, coop = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || sms <= 0 ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lw::batch_persistent_kernel, lw::kWT, 0) !=
          cudaSuccess) {
    delete b;
    return LW_ECUDA;
  }
  b->grid = per_sm * sms;
  b->mode = coop != 0 && b->grid > 0 ? 1 : 0;
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    const size_t sz = align_up(make_layout(p[i]).total, 256);
    lbm_wenoc* h = nullptr;
    rc = lbm_wenoc_create(&p[i], b->ws + off, sz, cuda_stream, &h);
    if (rc != LW_OK || !h->wide) {
      if (h) lbm_wenoc_destroy(h);
      for (lbm_wenoc* q : b->inst) lbm_wenoc_destroy(q);
      delete b;
      return rc != LW_OK ? rc : LW_EINVAL;
    }
    b->inst.push_back(h);
    b->offsets.push_back(off);
    off += sz;
  }
  b->rows.assign(count, 0);
  b->tables_off = off;
  rc = batch_upload_tables(b);
  if (rc != LW_OK) {
    for (lbm_wenoc* q : b->inst) lbm_wenoc_destroy(q);
    delete b;
    return rc;
  }
  *out = b;
  return LW_OK;
}

lbm_wenoc* lbm_wenoc_batch_instance(lbm_wenoc_batch* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->inst.size()) return nullptr;
  return b->inst[i];
}

int lbm_wenoc_batch_step(lbm_wenoc_batch* b, int64_t nsteps) {
  NvtxRange range("lbm_wenoc_batch_step");
  if (!b) return LW_EINVAL;
  return batch_advance(b, nsteps, true);
}

int lbm_wenoc_batch_set_persistent(lbm_wenoc_batch* b, int32_t persistent) {
  if (!b || persistent < 0 || persistent > 2) return LW_EINVAL;
  int coop = 0;
  if (persistent && (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device) != cudaSuccess ||
                     !coop || b->grid <= 0))
    return LW_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LW_ECUDA;
  b->mode = persistent;
  batch_destroy_graphs(b);
  return LW_OK;
}

int lbm_wenoc_batch_set_wait_limit(lbm_wenoc_batch* b, int64_t cycles, int32_t skip_cta) {
  if (!b || cycles < 1 || skip_cta < -1 || skip_cta >= b->grid) return LW_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LW_ECUDA;
  if (cycles != b->wait_limit) batch_destroy_graphs(b);  // the limit is a kernel argument of the graphs
  b->wait_limit = cycles;
  b->skip_cta = skip_cta;
  return LW_OK;
}

int lbm_wenoc_batch_status(lbm_wenoc_batch* b) {
  if (!b) return LW_EINVAL;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LW_ECUDA;
  unsigned st = 0;
  if (cudaMemcpy(&st, b->tab.status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return LW_ECUDA;
  if (st & lw::kStatusTimeout) {  // reported once: the word is cleared for the next launches
    if (cudaMemset(b->tab.status, 0, sizeof(unsigned)) != cudaSuccess) return LW_ECUDA;
    return LW_ETIMEOUT;
  }
  for (lbm_wenoc* h : b->inst) {
    const int rc = sync_and_status(h);
    if (rc != LW_OK) return rc;
  }
  return LW_OK;
}

int lbm_wenoc_batch_autotune(lbm_wenoc_batch* b, int32_t steps_per_trial, int32_t* chosen_rows) {
  if (!b || steps_per_trial < 1) return LW_EINVAL;
  const int count = (int)b->inst.size();
  int rc = batch_trial_state(b);
  if (rc != LW_OK) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LW_ECUDA;
  // start from each instance's own heuristic, then one pass of coordinate descent over the
  // shape classes (instances of one lattice size share a segment height): try each
  // candidate height for the class with the whole batch timed, keep the fastest
  for (int i = 0; i < count; ++i) b->rows[i] = b->inst[i]->stage2d_rows;
  std::vector<std::pair<int, int>> shapes;
  for (lbm_wenoc* h : b->inst) {
    const std::pair<int, int> sh(h->p.nx, h->p.ny);
    if (std::find(shapes.begin(), shapes.end(), sh) == shapes.end()) shapes.push_back(sh);
  }
  const int candidates[] = {8, 12, 16, 20, 27, 32, 48, 64};
  float best_ms = 0.f;
  if ((rc = batch_upload_tables(b)) == LW_OK) rc = batch_time(b, steps_per_trial, e0, e1, &best_ms);
  for (size_t c = 0; c < shapes.size() && rc == LW_OK; ++c) {
    std::vector<int> keep = b->rows;
    for (int H : candidates) {
      if (H > shapes[c].second) break;
      bool same = true;
      for (int i = 0; i < count; ++i)
        if (b->inst[i]->p.nx == shapes[c].first && b->inst[i]->p.ny == shapes[c].second) {
          same = same && keep[i] == H;
          b->rows[i] = H;
        }
      if (same) continue;
      float ms = 0.f;
      if ((rc = batch_upload_tables(b)) != LW_OK || (rc = batch_time(b, steps_per_trial, e0, e1, &ms)) != LW_OK)
        break;
      if (ms < best_ms) {
        best_ms = ms;
        keep = b->rows;
      }
    }
    b->rows = keep;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LW_OK) return rc;
  rc = batch_upload_tables(b);
  for (lbm_wenoc* h : b->inst) h->initialised = false;  // trial state is not a user state
  if (chosen_rows)
    for (int i = 0; i < count; ++i) chosen_rows[i] = b->rows[i];
  return rc;
}

int64_t lbm_wenoc_batch_launch_count(const lbm_wenoc_batch* b) { return b ? b->launches : -1; }

void lbm_wenoc_batch_destroy(lbm_wenoc_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_destroy_graphs(b);
  for (lbm_wenoc* h : b->inst) lbm_wenoc_destroy(h);
  delete b;
}

}  // extern "C"

// ------------------------------------------------------------------------------------
// Gradient of the deposited mass by checkpoint-and-recompute and the adjoint kernels.
//
// Adjoint workspace: a checkpoint (populations + c, the handle's layout from g to c) at the
// start of every segment but the last; two segments of step records (c before the step,
// then the step's c1, c2, u and rho, which the recording steps write there directly);
// lambda of the populations (two buffers, natural layout); mu, lc2, lc1, lc, lambda(u);
// lambda(Vs) and its per-CTA partials; the face derivative records of one stage.

namespace {

bool gradient_params_ok(const lbm_wenoc* h) {
  return h && h->p.dim == 2 && h->walls && !h->frozen && !h->sweep && !h->sugar &&
         !(h->p.flags & (LW_WENO3 | LW_SIGN_SPLIT)) && h->ncls == 1 && h->p.lf_alpha > 0.0;
}

struct GradLayout {
  size_t ckpt, rec, lg0, lg1, mu, lc2, lc1, lc, lu, vs, vs_part, faces, total;
  size_t ckpt_bytes, field_bytes, rec_bytes;  // one checkpoint, one field, one step record
  int rec_sets;                               // record sets (segments in flight)
  int32_t segment;
  int nparts;                                 // per-CTA dJ/dVs partials of the face kernel
  int64_t nseg;
};

GradLayout grad_layout(const lbm_wenoc_params& p, int64_t nsteps, int32_t segment) {
  const Layout L = make_layout(p);
  const size_t n = (size_t)p.nx * p.ny;
  const size_t es = (p.flags & LW_FP64) ? 8 : 4;
  GradLayout G{};
  G.nseg = (nsteps + segment - 1) / segment;
  G.segment = segment;
  G.ckpt_bytes = align_up(L.c + n * es - L.g, 256);
  G.field_bytes = align_up(n * es, 256);
  G.rec_bytes = 6 * G.field_bytes;  // c, c1, c2, u (2), rho
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  G.ckpt = take(G.ckpt_bytes * (size_t)(G.nseg - 1));  // the last segment is recorded directly
  G.rec_sets = G.nseg > 1 ? 2 : 1;  // the recompute of a segment overlaps the reverse of the next
  G.rec = take(G.rec_bytes * (size_t)segment * G.rec_sets);
  G.lg0 = take(9 * n * es);
  G.lg1 = take(9 * n * es);
  G.mu = take(n * es);
  G.lc2 = take(n * es);
  G.lc1 = take(n * es);
  G.lc = take(n * es);
  G.lu = take(2 * n * es);
  G.vs = take(sizeof(double) * 4);
  G.nparts = ((p.nx + lw::kAdjThreads - 1) / lw::kAdjThreads) * p.ny;
  G.vs_part = take(sizeof(double) * (size_t)G.nparts);
  G.faces = take(24 * n * es);
  G.total = off;
  return G;
}

int copy_d2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? LW_OK : LW_ECUDA;
}

template <typename T>
struct StepRecord {
  T *c, *c1, *c2, *u, *rho;
};

// Record of step k of a segment whose records live in set `set`.
template <typename T>
StepRecord<T> step_record(unsigned char* aw, const GradLayout& G, int set, int64_t k) {
  unsigned char* r = aw + G.rec + ((size_t)set * (size_t)G.segment + (size_t)k) * G.rec_bytes;
  StepRecord<T> R;
  R.c = reinterpret_cast<T*>(r);
  R.c1 = reinterpret_cast<T*>(r + G.field_bytes);
  R.c2 = reinterpret_cast<T*>(r + 2 * G.field_bytes);
  R.u = reinterpret_cast<T*>(r + 3 * G.field_bytes);  // u[d*n + node], d = 0, 1
  R.rho = reinterpret_cast<T*>(r + 5 * G.field_bytes);
  return R;
}

// One forward step that records what its adjoint needs: c^n is copied into the record,
// and the step writes c1, c2, u and rho there instead of the handle's buffers.
template <typename T>
int record_step(lbm_wenoc* h, const StepRecord<T>& R) {
  cudaStream_t s = h->stream;
  const size_t n = (size_t)h->n;
  if (copy_d2d(R.c, h->ws + h->L.c, n * sizeof(T), s) != LW_OK) return LW_ECUDA;
  Args<T> a = make_args<T>(h);
  a.c1 = R.c1;
  a.c2 = R.c2;
  a.u = R.u;
  const dim3 blk(kLbmThreads), grd((a.nx + kLbmThreads - 1) / kLbmThreads, a.ny, 1);
  launch(h, K_LBM, [&] {
    if (h->parity == 0)
      lw::lbm_d2q9_record_kernel<T, 0><<<grd, blk, 0, s>>>(a, R.rho);
    else
      lw::lbm_d2q9_record_kernel<T, 1><<<grd, blk, 0, s>>>(a, R.rho);
  });
  enqueue_transport<D2Q9, T>(h, a);
  h->parity ^= 1;
  h->steps += 1;
  return cudaGetLastError() == cudaSuccess ? LW_OK : LW_ECUDA;
}

// Reverse step over record R: mu = lambda(c^{n+1}) in, lambda(c^n) out; lam_next /
// lam_out = lambda of the populations of steps n+1 / n.
template <typename T>
int adjoint_step(lbm_wenoc* h, const StepRecord<T>& R, const lw::AdjFields<T>& f, const lw::FaceRecords<T>& fr,
                 const T* lam_next, T* lam_out) {
  Args<T> a = make_args<T>(h);
  a.c = R.c;
  a.c1 = R.c1;
  a.c2 = R.c2;
  a.u = R.u;
  cudaStream_t s = h->stream;
  const dim3 blk(kLbmThreads), grd((a.nx + kLbmThreads - 1) / kLbmThreads, a.ny, 1);
  launch(h, K_ADJ_FACES, [&] { lw::adj_faces_kernel<T, 3><<<grd, blk, 0, s>>>(a, f, fr); });
  launch(h, K_ADJ_GATHER, [&] { lw::adj_gather_kernel<T, 3><<<grd, blk, 0, s>>>(a, f, fr); });
  launch(h, K_ADJ_FACES, [&] { lw::adj_faces_kernel<T, 2><<<grd, blk, 0, s>>>(a, f, fr); });
  launch(h, K_ADJ_GATHER, [&] { lw::adj_gather_kernel<T, 2><<<grd, blk, 0, s>>>(a, f, fr); });
  launch(h, K_ADJ_FACES, [&] { lw::adj_faces_kernel<T, 1><<<grd, blk, 0, s>>>(a, f, fr); });
  launch(h, K_ADJ_FLUID,
         [&] { lw::adj_gather_fluid_kernel<T><<<grd, blk, 0, s>>>(a, f, fr, R.rho, lam_next, lam_out); });
  return cudaGetLastError() == cudaSuccess ? LW_OK : LW_ECUDA;
}

// The streams of the reverse sweep: `rev`, at the device's greatest stream priority, runs
// the reverse steps (the critical path); `s`, at the default (least) priority, the
// recompute of the next segment, which then only takes the SMs the reverse kernels leave.
struct RecomputeStream {
  cudaStream_t s = nullptr;
  cudaStream_t rev = nullptr;
  cudaEvent_t rec_done[2] = {nullptr, nullptr};  // records of set i written
  cudaEvent_t rev_done[2] = {nullptr, nullptr};  // records of set i no longer read
  cudaEvent_t join[2] = {nullptr, nullptr};      // caller's stream -> rev, rev -> caller's stream
  bool ok = false;
  RecomputeStream() {
    int least = 0, greatest = 0;
    ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithPriority(&rev, cudaStreamNonBlocking, greatest) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i)
      ok = cudaEventCreateWithFlags(&rec_done[i], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&rev_done[i], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess;
  }
  ~RecomputeStream() {
    if (s) cudaStreamSynchronize(s);
    if (rev) cudaStreamSynchronize(rev);
    for (int i = 0; i < 2; ++i) {
      if (rec_done[i]) cudaEventDestroy(rec_done[i]);
      if (rev_done[i]) cudaEventDestroy(rev_done[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (s) cudaStreamDestroy(s);
    if (rev) cudaStreamDestroy(rev);
  }
};

template <typename T>
int deposit_gradient_impl(lbm_wenoc* h, const void* c0, int64_t nsteps, int32_t segment, unsigned char* aw,
                          const GradLayout& G, void* grad_c0, double* dJ_dVs, double* J) {
  int rc = lbm_wenoc_init(h, c0, nullptr);
  if (rc != LW_OK) return rc;
  cudaStream_t s = h->stream;
  const Layout& L = h->L;
  unsigned char* state = h->ws + L.g;
  const size_t n = (size_t)h->n;
  auto seg_len = [&](int64_t sg) { return std::min<int64_t>(segment, nsteps - sg * segment); };
  auto set_of = [&](int64_t sg) { return G.rec_sets > 1 ? (int)(sg & 1) : 0; };
  auto record_segment = [&](int64_t sg) -> int {
    for (int64_t k = 0; k < seg_len(sg); ++k) {
      const int r = record_step<T>(h, step_record<T>(aw, G, set_of(sg), k));
      if (r != LW_OK) return r;
    }
    return LW_OK;
  };
  // forward, keeping the state at the start of every segment; the last segment is
  // recorded on the way (it is the first one the reverse sweep needs)
  std::vector<int> ck_parity((size_t)G.nseg);
  for (int64_t sg = 0; sg < G.nseg; ++sg) {
    ck_parity[(size_t)sg] = h->parity;
    if (sg == G.nseg - 1) {
      rc = record_segment(sg);
    } else {
      rc = copy_d2d(aw + G.ckpt + (size_t)sg * G.ckpt_bytes, state, G.ckpt_bytes, s);
      if (rc == LW_OK) rc = lbm_wenoc_step(h, seg_len(sg));
    }
    if (rc != LW_OK) return rc;
  }
  if ((rc = lbm_wenoc_deposited_mass(h, J)) != LW_OK) return rc;  // synchronises
  lw::AdjFields<T> f;
  f.mu = reinterpret_cast<T*>(aw + G.mu);
  f.lc2 = reinterpret_cast<T*>(aw + G.lc2);
  f.lc1 = reinterpret_cast<T*>(aw + G.lc1);
  f.lc = reinterpret_cast<T*>(aw + G.lc);
  f.lam_u = reinterpret_cast<T*>(aw + G.lu);
  f.lam_vs = reinterpret_cast<double*>(aw + G.vs);
  f.vs_part = reinterpret_cast<double*>(aw + G.vs_part);
  const int nparts = G.nparts;
  lw::FaceRecords<T> fr;
  fr.dcx = reinterpret_cast<T*>(aw + G.faces);
  fr.dwx = fr.dcx + 6 * n;
  fr.dcy = fr.dcx + 12 * n;
  fr.dwy = fr.dcx + 18 * n;
  T* lg[2] = {reinterpret_cast<T*>(aw + G.lg0), reinterpret_cast<T*>(aw + G.lg1)};
  if (cudaMemsetAsync(lg[0], 0, 9 * n * sizeof(T), s) != cudaSuccess) return LW_ECUDA;
  launch(h, K_OTHER, [&] {
    lw::adj_init_kernel<T><<<(unsigned)((std::max<size_t>(n, (size_t)nparts) + 255) / 256), 256, 0, s>>>(
        f, (long long)n, nparts);
  });
  // Reverse sweep over the segments, last first.  Segment sg's records sit in set sg & 1;
  // while the reverse of sg runs on the handle's stream, the recompute of sg - 1 runs on a
  // second stream into the other set, after the reverse of sg + 1 has released it.
  RecomputeStream rs;
  if (!rs.ok) return LW_ECUDA;
  // the reverse steps run on rs.rev after everything queued so far on the caller's stream
  if (cudaEventRecord(rs.join[0], s) != cudaSuccess || cudaStreamWaitEvent(rs.rev, rs.join[0], 0) != cudaSuccess)
    return LW_ECUDA;
  auto recompute = [&](int64_t sg) -> int {
    h->stream = rs.s;
    int r = LW_OK;
    // set sg & 1 was last read by the reverse of segment sg + 2
    if (sg + 2 <= G.nseg - 1 && cudaStreamWaitEvent(rs.s, rs.rev_done[set_of(sg)], 0) != cudaSuccess) r = LW_ECUDA;
    if (r == LW_OK) r = copy_d2d(state, aw + G.ckpt + (size_t)sg * G.ckpt_bytes, G.ckpt_bytes, rs.s);
    if (r == LW_OK) {
      h->parity = ck_parity[(size_t)sg];
      h->cur = 0;
      r = record_segment(sg);
    }
    if (r == LW_OK && cudaEventRecord(rs.rec_done[set_of(sg)], rs.s) != cudaSuccess) r = LW_ECUDA;
    h->stream = rs.rev;
    return r;
  };
  int cur = 0;
  h->stream = rs.rev;
  std::vector<cudaGraphExec_t> rev_full(4, nullptr), rev_tail(4, nullptr);
  struct GraphsGuard {  // destroys the segment graphs once the reverse stream has drained
    std::vector<cudaGraphExec_t>* v[2];
    cudaStream_t rev;
    ~GraphsGuard() {
      cudaStreamSynchronize(rev);
      for (auto* g : v)
        for (cudaGraphExec_t e : *g)
          if (e) cudaGraphExecDestroy(e);
    }
  } graphs_guard{{&rev_full, &rev_tail}, rs.rev};
  for (int64_t sg = G.nseg - 1; sg >= 0; --sg) {
    if (sg >= 1 && (rc = recompute(sg - 1)) != LW_OK) break;
    if (sg != G.nseg - 1 && cudaStreamWaitEvent(rs.rev, rs.rec_done[set_of(sg)], 0) != cudaSuccess) {
      rc = LW_ECUDA;
      break;
    }
    // the segment's reverse steps: replayed from a CUDA graph captured once per (record
    // set, lambda buffer, length) -- six launches a step with no host gaps between them --
    // or launched one by one while the per-kernel timing is on
    const int64_t len = seg_len(sg);
    if (h->use_graphs && !h->profiling) {
      const int key = set_of(sg) * 2 + cur;
      std::vector<cudaGraphExec_t>& cache = len == segment ? rev_full : rev_tail;
      if (!cache[key]) {
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
          rc = LW_ECUDA;
          break;
        }
        cudaGraph_t gr = nullptr;
        h->stream = cap;
        const int64_t saved = h->launches;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int c2 = cur;
        for (int64_t k = len - 1; k >= 0 && e == cudaSuccess && rc == LW_OK; --k) {
          rc = adjoint_step<T>(h, step_record<T>(aw, G, set_of(sg), k), f, fr, lg[c2], lg[c2 ^ 1]);
          c2 ^= 1;
        }
        const cudaError_t e2 = cudaStreamEndCapture(cap, &gr);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&cache[key], gr, 0);
        if (gr) cudaGraphDestroy(gr);
        cudaStreamDestroy(cap);
        h->stream = rs.rev;
        h->launches = saved;
        if (e != cudaSuccess && rc == LW_OK) rc = LW_ECUDA;
        if (rc != LW_OK) break;
      }
      if (cudaGraphLaunch(cache[key], rs.rev) != cudaSuccess) {
        rc = LW_ECUDA;
        break;
      }
      h->launches += 6 * len;
      if (len & 1) cur ^= 1;
    } else {
      for (int64_t k = len - 1; k >= 0 && rc == LW_OK; --k) {
        rc = adjoint_step<T>(h, step_record<T>(aw, G, set_of(sg), k), f, fr, lg[cur], lg[cur ^ 1]);
        cur ^= 1;
      }
    }
    if (rc != LW_OK) break;
    if (G.nseg > 1 && cudaEventRecord(rs.rev_done[set_of(sg)], rs.rev) != cudaSuccess) {
      rc = LW_ECUDA;
      break;
    }
  }
  // back on the caller's stream, after the reverse sweep
  h->stream = s;
  if (cudaEventRecord(rs.join[1], rs.rev) != cudaSuccess || cudaStreamWaitEvent(s, rs.join[1], 0) != cudaSuccess)
    return LW_ECUDA;
  if (rc != LW_OK) return rc;
  // mu now holds lambda(c^0)
  launch(h, K_OTHER, [&] { lw::adj_vs_finish_kernel<<<1, 256, 0, s>>>(f.vs_part, nparts, f.lam_vs); });
  cudaMemcpyKind k = is_device_pointer(grad_c0) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (cudaMemcpyAsync(grad_c0, f.mu, n * sizeof(T), k, s) != cudaSuccess) return LW_ECUDA;
  if (cudaMemcpyAsync(dJ_dVs, f.lam_vs, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LW_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LW_ECUDA;
  h->initialised = false;  // the handle holds a recomputed intermediate state
  return sync_and_status(h);
}

}  // namespace

extern "C" {

int lbm_wenoc_gradient_workspace_bytes(const lbm_wenoc_params* p, int64_t nsteps, int32_t segment, size_t* bytes) {
  if (!p || !bytes || nsteps < 1 || segment < 1) return LW_EINVAL;
  if (check_params(p) != LW_OK || p->dim != 2) return LW_EINVAL;
  segment = (int32_t)std::min<int64_t>(segment, nsteps);
  *bytes = grad_layout(*p, nsteps, segment).total;
  return LW_OK;
}

int lbm_wenoc_deposit_gradient(lbm_wenoc* h, const void* c0, int64_t nsteps, int32_t segment, void* adj_workspace,
                               size_t bytes, void* grad_c0, double* dJ_dVs, double* J) {
  NvtxRange range("lbm_wenoc_deposit_gradient");
  if (!h || !c0 || !grad_c0 || !dJ_dVs || !J || nsteps < 1 || segment < 1 || !adj_workspace) return LW_EINVAL;
  if (!gradient_params_ok(h)) return LW_EINVAL;
  if (24.0 * (double)h->n >= 2147483647.0) return LW_EINVAL;  // 32-bit offsets of the face records
  if ((reinterpret_cast<uintptr_t>(adj_workspace) & 255u) != 0) return LW_EINVAL;
  segment = (int32_t)std::min<int64_t>(segment, nsteps);
  const GradLayout G = grad_layout(h->p, nsteps, segment);
  if (bytes < G.total) return LW_ENOMEM;
  unsigned char* aw = static_cast<unsigned char*>(adj_workspace);
  if (h->fp64) return deposit_gradient_impl<double>(h, c0, nsteps, segment, aw, G, grad_c0, dJ_dVs, J);
  return deposit_gradient_impl<float>(h, c0, nsteps, segment, aw, G, grad_c0, dJ_dVs, J);
}

}  // extern "C"
