// cmc_potential_static: the shell potential of cmc_potential for callers
// that may not allocate device memory.
//
// Some callers cannot let a library allocate: real-time loops that forbid
// any allocation after start-up (an allocation can block, synchronise or
// fail), programs that hand all device memory to their own pool, and
// plug-ins whose host application owns the allocator.  This entry point needs nothing from the allocator: its
// only scratch, the per-tile sums of the scan, lives in a fixed array in
// the library's own device memory, reserved when the library is loaded and
// kept by every GPU that loads it until the process exits.
//
// The scan is cmc_potential's (same tiles, M_k and S_k from the tiles before
// and after in a fixed order) with summation orders of its own inside a
// tile: the two entry points agree to rounding, and each repeats its own
// results bit for bit.
#include <mutex>

#include "cmc_host.hpp"
#include "../../include/cmc.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPer = cmc::kTile / kThreads;
constexpr int64_t kMaxTiles = CMC_STATIC_MAX_STARS / cmc::kTile;
static_assert(CMC_STATIC_MAX_STARS % cmc::kTile == 0, "whole tiles");

// [0, kMaxTiles): mass per tile; [kMaxTiles, 2 kMaxTiles): sum of m/r per tile
static __device__ __align__(256) double g_tile_scratch[2 * kMaxTiles];

__device__ __forceinline__ double sum256(double v, double* s) {
  s[threadIdx.x] = v;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] = s[threadIdx.x] + s[threadIdx.x + w];
    __syncthreads();
  }
  double r = s[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void scans256(double vm, double vs, double* s1, double* s2,
                                         double& pre_m, double& suf_s) {
  const int t = threadIdx.x;
  s1[t] = vm;
  s2[t] = vs;
  __syncthreads();
  for (int o = 1; o < kThreads; o <<= 1) {
    double a = t >= o ? s1[t - o] : 0.0;
    double b = t + o < kThreads ? s2[t + o] : 0.0;
    __syncthreads();
    if (t >= o) s1[t] = a + s1[t];
    if (t + o < kThreads) s2[t] = s2[t] + b;
    __syncthreads();
  }
  pre_m = t > 0 ? s1[t - 1] : 0.0;
  suf_s = t + 1 < kThreads ? s2[t + 1] : 0.0;
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_static_tile_sums(int64_t n, const double* r,
                                                               const double* m,
                                                               double* scratch) {
  __shared__ double s[kThreads];
  const int64_t begin = (int64_t)blockIdx.x * cmc::kTile;
  const int64_t b = begin + (int64_t)threadIdx.x * kPer;
  double am = 0.0, ax = 0.0;
  for (int i = 0; i < kPer; ++i) {
    int64_t p = b + i;
    if (p < n) {
      double mm = m[p];
      am = am + mm;
      ax = ax + mm * (1.0 / r[p]);
    }
  }
  double tm = sum256(am, s);
  double tx = sum256(ax, s);
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = tm;
    scratch[kMaxTiles + blockIdx.x] = tx;
  }
}

__global__ void __launch_bounds__(kThreads) k_static_potential(int64_t n, int64_t n_tiles,
                                                               const double* r,
                                                               const double* m,
                                                               const double* scratch,
                                                               double* phi, double* Mout) {
  __shared__ double s1[kThreads], s2[kThreads];
  const int64_t lt = blockIdx.x;
  double pm = 0.0, ps = 0.0;
  for (int64_t j = threadIdx.x; j < n_tiles; j += kThreads) {
    if (j < lt) pm = pm + scratch[j];
    if (j > lt) ps = ps + scratch[kMaxTiles + j];
  }
  const double Mbefore = sum256(pm, s1);
  const double Safter = sum256(ps, s1);
  const int64_t b = lt * cmc::kTile + (int64_t)threadIdx.x * kPer;
  double mm[kPer], xx[kPer];
  double am = 0.0, ax = 0.0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    int64_t p = b + i;
    bool ok = p < n;
    mm[i] = ok ? m[p] : 0.0;
    xx[i] = ok ? 1.0 / r[p] : 0.0;
    am = am + mm[i];
    ax = ax + mm[i] * xx[i];
  }
  double pre_m, suf_s;
  scans256(am, ax, s1, s2, pre_m, suf_s);
  double Mk[kPer], Sk[kPer];
  double run = 0.0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    run = run + mm[i];
    Mk[i] = (Mbefore + pre_m) + run;
  }
  double suf = 0.0;
#pragma unroll
  for (int i = kPer - 1; i >= 0; --i) {
    Sk[i] = (Safter + suf_s) + suf;
    suf = suf + mm[i] * xx[i];
  }
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    int64_t p = b + i;
    if (p >= n) break;
    phi[p] = -(Mk[i] * xx[i] + Sk[i]);
    if (Mout) Mout[p] = Mk[i];
  }
}

// device address of g_tile_scratch, resolved once per device and kept for
// the life of the process (a device reset would invalidate it)
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" {

cmc_status cmc_potential_static(int64_t n, const double* r, const double* m, double* phi,
                                double* M, void* stream) {
  if (n < 0 || (n > 0 && (!r || !m || !phi))) return CMC_EINVAL;
  // more stars than the fixed scratch has tiles for
  if (n > (int64_t)CMC_STATIC_MAX_STARS) return CMC_EINVAL;
  if (n == 0) return CMC_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e || dev < 0 || dev >= kMaxDevices) return CMC_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      // host code cannot name the array's device address directly; ask the
      // runtime for it once, with this device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_tile_scratch);
      if (e != cudaSuccess || !p) return CMC_ECUDA;
      g_addr[dev] = (double*)p;
    }
    scratch = g_addr[dev];
  }
  const int64_t n_tiles = (n + cmc::kTile - 1) / cmc::kTile;
  cudaStream_t st = (cudaStream_t)stream;
  k_static_tile_sums<<<(unsigned)n_tiles, kThreads, 0, st>>>(n, r, m, scratch);
  k_static_potential<<<(unsigned)n_tiles, kThreads, 0, st>>>(n, n_tiles, r, m, scratch, phi,
                                                             M);
  // peek: an error left by someone else's earlier work is reported, not
  // cleared
  return cudaPeekAtLastError() == cudaSuccess ? CMC_OK : CMC_ECUDA;
}

}  // extern "C"
