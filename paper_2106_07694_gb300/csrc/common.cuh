// Shared device-side argument block and small helpers of the lbm_wenoc kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lw {

// Status bits ORed by kernels into the device status word.
constexpr unsigned kStatusUnstable = 1u;  // non-finite value or |u_d| > u_cap
constexpr unsigned kStatusTimeout = 2u;   // a bounded wait gave up

template <typename T>
struct Args {
  T* g;    // populations stored as g_i = f_i - w_i, SoA: g[i*n + node]
  T* c;    // concentration c^n (updated in place by the last RK stage)
  T* c1;   // RK stage 1 field
  T* c2;   // RK stage 2 field
  T* u;    // transport velocity of the current step, u[d*n + node]
  double* partials;  // per-block FP64 partial sums (fixed-order reductions)
  double* scalars;   // [0] deposit, [1] reduction result
  unsigned* status;  // status word
  unsigned* ticket;  // last-block ticket of the reductions
  int nx, ny, nz;    // extents (nz = 1 in 2D)
  long long n;       // nodes
  int walls;         // 1 = no-slip floor and lid, 0 = periodic vertical
  T omega;           // 1/tau
  T guo;             // 1 - 1/(2 tau)
  T A;               // gravity * density_contrast
  T bf[3];           // body force
  T vs;              // settling velocity
  T kappa;           // diffusivity
  T alpha;           // Lax-Friedrichs split speed
  T inv_alpha;
  T u_cap;
  // sugar (the paper's density-altering scalar), null S when off
  const T* S;  // S of step n
  T* S2;       // S of step n + 1
  T gS;        // gravity * sugar_contrast (S*): force -gS S (1 - phi0 c) along the vertical
  T phi0;      // particle volume fraction at c = 1
  T ks;        // settling velocity Vs (1 - ks S)
  T Ds;        // sugar diffusivity
  int scheme;  // flux variant bits (kSchemeWeno3, kSchemeSignSplit); 0 = WENO5, Lax-Friedrichs
};

// Global-load policies.  LoadNC reads through the non-coherent (read-only) path, for data
// no thread writes while the kernel runs; LoadL2 reads at L2 (ld.global.cg: no L1 line is
// kept), for a kernel that reads what other CTAs wrote earlier in the same launch, after
// a grid barrier; LoadPlain is an ordinary load.
struct LoadNC {
  static __device__ __forceinline__ float s(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ double s(const double* p) { return __ldg(p); }
  static __device__ __forceinline__ float4 v4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
};
struct LoadL2 {
  static __device__ __forceinline__ float s(const float* p) { return __ldcg(p); }
  static __device__ __forceinline__ double s(const double* p) { return __ldcg(p); }
  static __device__ __forceinline__ float4 v4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
};
struct LoadPlain {
  static __device__ __forceinline__ float s(const float* p) { return *p; }
  static __device__ __forceinline__ double s(const double* p) { return *p; }
  static __device__ __forceinline__ float4 v4(const float* p) { return *reinterpret_cast<const float4*>(p); }
};

constexpr int kSchemeWeno3 = 1;
constexpr int kSchemeSignSplit = 2;

// Settling velocity at node m: Vs, or Vs (1 - ks S_m) with sugar.
template <typename T>
__device__ __forceinline__ T settling_at(const Args<T>& a, long long m) {
  return a.S ? a.vs * (T(1) - a.ks * a.S[m]) : a.vs;
}

// Asynchronous 16-byte global -> shared copy at L2 (cp.async.cg: no L1 line, so it also
// sees what other SMs wrote earlier in the same launch); groups of copies are committed
// and waited for per thread.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// fused multiply-add of the kernel's precision (fmaf for FP32, fma for FP64)
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ int wrap_dec(int a, int n) { return a < 0 ? a + n : a; }
__device__ __forceinline__ int wrap_inc(int a, int n) { return a >= n ? a - n : a; }
__device__ __forceinline__ int wrap_any(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

template <typename T>
__device__ __forceinline__ bool finite_val(T v) { return isfinite(v); }

// Flag a bad value once per warp (no trap, no assert: the host reads the word).
__device__ __forceinline__ unsigned lane_id() {
  unsigned l;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}

__device__ __forceinline__ void report_status(unsigned* status, bool bad) {
  unsigned m = __ballot_sync(__activemask(), bad);
  if (m != 0u && lane_id() == (unsigned)(__ffs(m) - 1)) atomicOr(status, kStatusUnstable);
}

}  // namespace lw
