// Shell potential (section 2.1 step 1, Eqs. 1-5), the energy correction of
// section 2.1 step 6, the diagnostics, and the data movement around the
// sort (payload gather).
//
// The potential is Eq. 1 in scan form, Phi_k = -G (M_k / r_k + S_k) with
// M_k = sum_{i<=k} m_i and S_k = sum_{i>k} m_i / r_i, over the bound stars
// of each segment.  The scan is reduce-then-scan on fixed tiles: one kernel
// writes per-tile sums, the next combines, per tile, the sums of the tiles
// before it (for M) and after it (for S) in a fixed order and scans inside
// the tile.  Every sum is therefore evaluated in the same order on every
// run, so a cluster gives the same bits whether it is advanced alone or in
// an ensemble, and a resumed run repeats an uninterrupted one exactly.
#include <cmath>

#include "cmc_host.hpp"

namespace cmc {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = kTile / kThreads;  // 16 consecutive elements per thread

__device__ __forceinline__ int64_t nb_eff(const int64_t* nb, const int64_t* esc, int c,
                                          bool sub) {
  int64_t v = nb[c];
  if (sub) v -= esc[c];
  return v;
}

// fixed-shape block reduction of one double per thread (256 threads)
__device__ __forceinline__ double block_sum(double v, double* s) {
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

// fixed-shape inclusive scans of one double per thread (Hillis-Steele on
// shared memory): forward for vm, backward for vs; returns the exclusive
// values (sum over lower threads, sum over higher threads)
__device__ __forceinline__ void block_scans(double vm, double vs, double* s1, double* s2,
                                            double& pre_m, double& suf_s) {
  // inclusive forward scan of vm, inclusive backward scan of vs
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

struct TR {
  int seg;
  int64_t lt, nt, seg_begin, begin, end, bound_end;
};

__device__ __forceinline__ TR tile_of(const Seg& S, const int64_t* esc, int64_t t, bool sub) {
  TR R;
  R.seg = seg_find(S.tile_off, S.n_seg, t);
  int64_t t0 = __ldg(S.tile_off + R.seg);
  R.lt = t - t0;
  R.nt = __ldg(S.tile_off + R.seg + 1) - t0;
  R.seg_begin = __ldg(S.off + R.seg);
  int64_t se = __ldg(S.off + R.seg + 1);
  R.begin = R.seg_begin + R.lt * kTile;
  R.end = R.begin + kTile < se ? R.begin + kTile : se;
  R.bound_end = R.seg_begin + nb_eff(S.nb, esc, R.seg, sub);
  return R;
}

// --------------------------------------------------------------- gather
__global__ void k_make_keys(int64_t n, const double* r, const double* vr, const double* vt,
                            const double* m, const uint32_t* id, uint64_t* keys,
                            Payload* pay) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double rr = r[p];
  uint32_t ii = id[p];
  keys[p] = radius_key(rr, ii);
  if (!pay) return;
  Payload P;
  P.vr = vr[p]; P.vt = vt[p]; P.m = m[p]; P.r_old = rr; P.c = 0.0; P.id = ii; P.pad = 0;
  pay[p] = P;
}

__global__ void k_id_keys(int64_t n, const uint32_t* id, uint64_t* keys) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) keys[p] = (uint64_t)id[p];
}

__global__ void k_rekey_radius(int64_t n, const uint32_t* perm, const double* r,
                               const uint32_t* id, uint64_t* keys) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint32_t q = perm[p];
  keys[p] = radius_key(r[q], id[q]);
}

__global__ void k_gather(int64_t n, const uint64_t* __restrict__ keys,
                         const uint32_t* __restrict__ vals, const Payload* __restrict__ pay,
                         double* r, double* x, double* vr, double* vt, double* m,
                         uint32_t* id, double* r_old, double* c) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint64_t k = keys[p];
  const uint32_t v = vals[p];
  if ((int64_t)v >= n) return;  // only after a reported sort failure
  const Payload P = pay[v];
  double rr, xx;
  if (key_is_escaper(k)) { rr = __longlong_as_double(0x7FF0000000000000ll); xx = 0.0; }
  else { rr = __longlong_as_double((long long)k); xx = div_rn(1.0, rr); }
  r[p] = rr; x[p] = xx; vr[p] = P.vr; vt[p] = P.vt; m[p] = P.m; id[p] = P.id;
  if (r_old) r_old[p] = P.r_old;
  if (c) c[p] = P.c;
}

// The gather of one tile with the potential's per-tile sums of m and m x
// (k_tile_sums over the bound stars after the orbit step) taken from the
// values it has just written: the same striped element order and tree, so
// the same sums, without reading m and x back.
__global__ void __launch_bounds__(kThreads) k_gather_sums(
    Seg S, const int64_t* esc, int64_t n, const uint64_t* __restrict__ keys,
    const uint32_t* __restrict__ vals, const Payload* __restrict__ pay, double* r, double* x,
    double* vr, double* vt, double* m, uint32_t* id, double* r_old, double* c, double* tile_m,
    double* tile_mx, const double* Rp, double* Rout, const double* Ap, double* Aout,
    bool packed) {
  __shared__ double s[kThreads];
  TR R = tile_of(S, esc, blockIdx.x, true);
  double am = 0.0, ax = 0.0;
#pragma unroll 4
  for (int i = 0; i < kPer; ++i) {
    const int64_t p = R.begin + (int64_t)i * kThreads + threadIdx.x;
    if (p >= R.end) continue;
    uint64_t k = keys[p];
    // packed keys: the star's index in the segment in the low 24 bits
    const int64_t v = packed ? R.seg_begin + (int64_t)(k & kPackMask) : (int64_t)vals[p];
    if (v >= n) continue;  // only after a reported sort failure
    const Payload P = pay[v];
    if (packed) k = (k & ~kPackMask) | (uint64_t)P.pad;
    double rr, xx;
    if (key_is_escaper(k)) { rr = __longlong_as_double(0x7FF0000000000000ll); xx = 0.0; }
    else { rr = __longlong_as_double((long long)k); xx = div_rn(1.0, rr); }
    r[p] = rr; x[p] = xx; vr[p] = P.vr; vt[p] = P.vt; m[p] = P.m; id[p] = P.id;
    r_old[p] = P.r_old;
    c[p] = P.c;
    if (Rout) Rout[p] = Rp[v];
    if (Aout) Aout[p] = Ap[v];
    if (p < R.bound_end) {
      am = am + P.m;
      ax = ax + P.m * xx;
    }
  }
  double tm = block_sum(am, s);
  double tx = block_sum(ax, s);
  if (threadIdx.x == 0) { tile_m[blockIdx.x] = tm; tile_mx[blockIdx.x] = tx; }
}

// Double -> float rounding to nearest even with integer operations: the
// conversion instruction runs on the FP64 pipe, which the potential kernel
// otherwise keeps busy with its scans.  For 2^-60 <= |v| < 2^126 (both
// parts below normal floats) the top 24 significand bits are rounded by the
// 29 bits below them; the remainder v - hi is then exact in those 29 bits
// and rounded the same way.  Other values take the conversions.
struct F32Pair {
  float hi, lo;
};

__device__ __forceinline__ F32Pair f32_pair(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned ex = (unsigned)(u >> 52) & 0x7FFu;
  F32Pair r;
  if (ex - 963u > 186u) {  // outside [963, 1149]
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
  }
  const unsigned sg = (unsigned)(u >> 32) & 0x80000000u;
  const unsigned top = ((ex - 896u) << 23) | ((unsigned)(u >> 29) & 0x7FFFFFu);
  const unsigned rest = (unsigned)u & 0x1FFFFFFFu;  // the 29 bits below
  const bool up = rest > 0x10000000u || (rest == 0x10000000u && (top & 1u));
  r.hi = __uint_as_float(sg | (top + (up ? 1u : 0u)));  // a carry moves the exponent
  // v - hi = (rest - (up ? 2^29 : 0)) 2^(ex - 1075), |.| <= 2^28
  const int rem = (int)rest - (up ? (1 << 29) : 0);
  if (rem == 0) {
    r.lo = 0.0f;
    return r;
  }
  const unsigned a = (unsigned)(rem < 0 ? -rem : rem);
  const int lz = __clz((int)a);            // >= 3
  const int pb = 31 - lz;                  // top bit of a
  const unsigned n = a << lz;              // top bit at 31
  unsigned m = n >> 8;                     // 24 bits with the leading one
  const unsigned low = n & 0xFFu;
  m += (low > 0x80u || (low == 0x80u && (m & 1u))) ? 1u : 0u;
  // a 2^(ex - 1075) = (m / 2^23) 2^(ex - 1075 + pb); a carry to 2^24 bumps
  // the exponent through the addition below
  const unsigned fe = ex - 1075u + 127u + (unsigned)pb;  // in [15, 229]
  const unsigned sl = (rem < 0 ? sg ^ 0x80000000u : sg);
  r.lo = __uint_as_float(sl | ((fe << 23) + (m - 0x800000u)));
  return r;
}

// (hi, lo) float pairs of 1/r and Phi: hi the float nearest, lo the float
// nearest the remainder (together ~48 bits)
__device__ __forceinline__ float4 float_pairs(double x, double ph) {
  const F32Pair a = f32_pair(x), b = f32_pair(ph);
  return make_float4(a.hi, a.lo, b.hi, b.lo);
}

// ------------------------------------------------------------ potential
// per-tile sums of m and m x (striped, coalesced loads; fixed tree)
__global__ void __launch_bounds__(kThreads) k_tile_sums(Seg S, const int64_t* esc, bool sub,
                                                        const double* x, const double* m,
                                                        double* tile_m, double* tile_mx) {
  __shared__ double s[kThreads];
  TR R = tile_of(S, esc, blockIdx.x, sub);
  // all 32 loads issued before the sums, which still run in element order
  double mv[kPer], xv[kPer];
  unsigned ok = 0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    const int64_t p = R.begin + (int64_t)i * kThreads + threadIdx.x;
    const bool in = p < R.end && p < R.bound_end;
    ok |= (unsigned)in << i;
    mv[i] = in ? __ldg(m + p) : 0.0;
    xv[i] = in ? __ldg(x + p) : 0.0;
  }
  double am = 0.0, ax = 0.0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    if ((ok >> i) & 1u) {
      am = am + mv[i];
      ax = ax + mv[i] * xv[i];
    }
  }
  double tm = block_sum(am, s);
  double tx = block_sum(ax, s);
  if (threadIdx.x == 0) { tile_m[blockIdx.x] = tm; tile_mx[blockIdx.x] = tx; }
}

// The potential kernel runs 512 threads on a tile, 8 consecutive elements
// each, so that two tiles' worth of warps (32) share an SM; its shared
// arrays pad one double per 8 (a thread's run of 8 sits 9 words from its
// neighbour's, free of bank conflicts within each half-warp).
constexpr int kPotThreads = 512;
constexpr int kPotPer = kTile / kPotThreads;
constexpr int kPotWarps = kPotThreads / 32;
__device__ __forceinline__ int pad8(int e) { return e + (e >> 3); }
constexpr int kPad8N = kTile + kTile / 8;

// fixed-order block sum over kPotThreads threads: a tree in each warp, then
// a tree over the warp totals in the first warp (w17: kPotWarps + 1 slots)
__device__ __forceinline__ double block_sum_pot(double v, double* w17) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = v + __shfl_down_sync(0xFFFFFFFFu, v, o);
  if (lane == 0) w17[w] = v;
  __syncthreads();
  if (w == 0) {
    double u = lane < kPotWarps ? w17[lane] : 0.0;
#pragma unroll
    for (int o = kPotWarps / 2; o > 0; o >>= 1) u = u + __shfl_down_sync(0xFFFFFFFFu, u, o);
    if (lane == 0) w17[kPotWarps] = u;
  }
  __syncthreads();
  const double r = w17[kPotWarps];
  __syncthreads();
  return r;
}

// Fixed point for the sums inside a tile: v >= 0 as round(v 2^S) in 64
// bits, S = 49 - (the largest unbiased exponent among the tile's values),
// so that a sum of 4096 values stays below 2^62; the largest values keep
// 50 significant bits, the sums are then exact (and independent of their
// order), and only the conversion back rounds.  Integer instructions only:
// the FP64 pipe is left to the products.
__device__ __forceinline__ int exp_of(double v) {  // biased exponent (0 for zero)
  return (int)((ubits(v) >> 52) & 0x7FFull);
}

__device__ __forceinline__ long long fix_of(double v, int S) {
  const unsigned long long u = ubits(v);
  const int e = (int)((u >> 52) & 0x7FFull);
  if (e == 0) return 0;  // zero (and subnormals, far below any sum here)
  const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = e - 1075 + S;  // v = mant 2^(e - 1075); sh <= -3 for the largest
  if (sh >= 0) return (long long)(mant << sh);
  if (sh < -60) return 0;
  const int d = -sh;
  // round to nearest, ties to even
  const unsigned long long q = mant >> d, rem = mant & ((1ull << d) - 1ull),
                           half = 1ull << (d - 1);
  return (long long)(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
}

// V 2^-S (V >= 0) as the nearest double, ties to even
__device__ __forceinline__ double dbl_of_fix(long long V, int S) {
  if (V <= 0) return 0.0;
  const unsigned long long a = (unsigned long long)V;
  int top = 63 - __clzll((long long)a);
  unsigned long long m;
  if (top <= 52) {
    m = a << (52 - top);
  } else {
    const int d = top - 52;
    m = a >> d;
    const unsigned long long rem = a & ((1ull << d) - 1ull), half = 1ull << (d - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m >> 53) {
      m >>= 1;
      ++top;
    }
  }
  return __longlong_as_double(
      (long long)(((unsigned long long)(top - S + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// the largest of one int per thread over kPotThreads threads
__device__ __forceinline__ int block_max_pot(int v, int* w17) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)v);
  if (lane == 0) w17[w] = v;
  __syncthreads();
  int r = 0;
#pragma unroll
  for (int i = 0; i < kPotWarps; ++i) r = w17[i] > r ? w17[i] : r;
  __syncthreads();
  return r;
}

// exclusive forward scan of vm and backward scan of vs (64-bit integers)
// over kPotThreads threads: inclusive scans inside each warp by shuffles,
// the 16 warp totals scanned by one warp, then (totals of the warps before
// or after) + (lanes before or after in the warp)
__device__ __forceinline__ void block_scans_fix(long long vm, long long vs, long long* wm,
                                                long long* ws, long long& pre_m,
                                                long long& suf_s) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long a = vm, b = vs;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long ua = __shfl_up_sync(0xFFFFFFFFu, a, o);
    const long long db = __shfl_down_sync(0xFFFFFFFFu, b, o);
    if (lane >= o) a = ua + a;
    if (lane + o < 32) b = b + db;
  }
  const long long ea = __shfl_up_sync(0xFFFFFFFFu, a, 1);
  const long long eb = __shfl_down_sync(0xFFFFFFFFu, b, 1);
  if (lane == 31) wm[w] = a;
  if (lane == 0) ws[w] = b;
  __syncthreads();
  if (w == 0) {
    long long ta = lane < kPotWarps ? wm[lane] : 0ll;
    long long tb = lane < kPotWarps ? ws[lane] : 0ll;
#pragma unroll
    for (int o = 1; o < kPotWarps; o <<= 1) {
      const long long ua = __shfl_up_sync(0xFFFFFFFFu, ta, o);
      const long long db = __shfl_down_sync(0xFFFFFFFFu, tb, o);
      if (lane >= o) ta = ua + ta;
      if (lane + o < kPotWarps) tb = tb + db;
    }
    const long long xa = __shfl_up_sync(0xFFFFFFFFu, ta, 1);
    const long long xb = __shfl_down_sync(0xFFFFFFFFu, tb, 1);
    __syncwarp();
    if (lane < kPotWarps) {
      wm[lane] = lane > 0 ? xa : 0ll;
      ws[lane] = lane + 1 < kPotWarps ? xb : 0ll;
    }
  }
  __syncthreads();
  pre_m = lane > 0 ? wm[w] + ea : wm[w];
  suf_s = lane < 31 ? ws[w] + eb : ws[w];
  __syncthreads();
}

// Phi_k = -(M_k x_k + S_k) over one tile.  The tile's m and x are staged in
// shared memory with coalesced loads; each thread scans its 8 consecutive
// elements (local suffix sums of m x kept in registers), the per-thread
// totals are scanned across the block, and the results (Phi, M_k, the
// float tables, the node records) leave through shared memory with
// coalesced stores.
__global__ void __launch_bounds__(kPotThreads) k_potential(Seg S, const int64_t* esc, bool sub,
                                                           const double* r, const double* x,
                                                           const double* m, const double* tile_m,
                                                           const double* tile_mx, double* phi,
                                                           float2* t32, double* Mout,
                                                           double4_32a* node, float4* tdf,
                                                           bool slopes, TableOut T) {
  extern __shared__ double smem[];
  double* s_m = smem;               // m, then M_k
  double* s_x = smem + kPad8N;      // x
  double* s_p = smem + 2 * kPad8N;  // Phi
  __shared__ double wm[kPotWarps + 1], ws[kPotWarps];
  __shared__ long long wq[kPotWarps], wr[kPotWarps];
  __shared__ int we[kPotWarps];
  TR R = tile_of(S, esc, blockIdx.x, sub);
  const int64_t t0 = blockIdx.x - R.lt;
  const int t = threadIdx.x;
  // tiles before (M) and after (S) this one, in a fixed order
  double pm = 0.0, ps = 0.0;
  for (int64_t j = t; j < R.nt; j += kPotThreads) {
    if (j < R.lt) pm = pm + tile_m[t0 + j];
    if (j > R.lt) ps = ps + tile_mx[t0 + j];
  }
  const double Mbefore = block_sum_pot(pm, wm);
  const double Safter = block_sum_pot(ps, wm);
#pragma unroll
  for (int i = 0; i < kPotPer; ++i) {
    const int e = i * kPotThreads + t;
    const int64_t p = R.begin + e;
    const bool ok = p < R.end && p < R.bound_end;
    s_m[pad8(e)] = ok ? __ldg(m + p) : 0.0;
    s_x[pad8(e)] = ok ? __ldg(x + p) : 0.0;
  }
  __syncthreads();
  const int e0 = t * kPotPer;
  // the tile's sums of m and m x in fixed point (exact inside the tile):
  // the scales from the largest exponents, then the thread's run of 8
  double mx[kPotPer];
  int em = 0, ex = 0;
#pragma unroll
  for (int i = 0; i < kPotPer; ++i) {
    const int q = pad8(e0 + i);
    mx[i] = s_m[q] * s_x[q];
    const int a = exp_of(s_m[q]), b = exp_of(mx[i]);
    em = a > em ? a : em;
    ex = b > ex ? b : ex;
  }
  const int Sm = 49 - (block_max_pot(em, we) - 1023);
  const int Sx = 49 - (block_max_pot(ex, we) - 1023);
  // exclusive suffix of m x along the thread's run, and its total
  long long suf[kPotPer];
  long long ax = 0;
#pragma unroll
  for (int i = kPotPer - 1; i >= 0; --i) {
    suf[i] = ax;
    ax = ax + fix_of(mx[i], Sx);
  }
  long long am = 0;
#pragma unroll
  for (int i = 0; i < kPotPer; ++i) am = am + fix_of(s_m[pad8(e0 + i)], Sm);
  long long pre_m, suf_s;
  block_scans_fix(am, ax, wq, wr, pre_m, suf_s);
  long long run = pre_m;
#pragma unroll
  for (int i = 0; i < kPotPer; ++i) {
    const int q = pad8(e0 + i);
    run = run + fix_of(s_m[q], Sm);
    const double Mk = Mbefore + dbl_of_fix(run, Sm);
    const double Sk = Safter + dbl_of_fix(suf_s + suf[i], Sx);
    const double ph = -(Mk * s_x[q] + Sk);
    s_m[q] = Mk;
    s_p[q] = ph;
  }
  __syncthreads();
#pragma unroll 4
  for (int i = 0; i < kPotPer; ++i) {
    const int e = i * kPotThreads + t;
    const int64_t p = R.begin + e;
    if (p >= R.end) break;
    const bool bound = p < R.bound_end;
    const int q = pad8(e);
    const double ph = bound ? s_p[q] : 0.0;
    phi[p] = ph;
    if (t32) t32[p] = make_float2(f32_pair(s_x[q]).hi, f32_pair(ph).hi);
    // the enclosed mass M_k, or with `slopes` the slope of Eq. 6 in 1/r
    // across shell k, (Phi_{k+1} - Phi_k) / (x_k - x_{k+1}) with Phi = 0 at
    // 1/r = 0 beyond the last bound star (the FP64 orbit step's shell
    // parameter); a tile's last star, whose neighbour is in the next tile,
    // gets its slope from k_slope_seams
    double w = bound ? s_m[q] : 0.0;
    if (slopes) {
      w = 0.0;
      if (bound) {
        if (p + 1 >= R.bound_end) w = div_rn(0.0 - ph, s_x[q] - 0.0);
        else if (e + 1 < kTile) {
          const int q1 = pad8(e + 1);
          w = div_rn(s_p[q1] - ph, s_x[q] - s_x[q1]);
        }
      }
    }
    if (Mout) Mout[p] = w;
    if (node) node[p] = make_double4_32a(r[p], s_x[q], ph, w);
    if (tdf) tdf[p] = float_pairs(s_x[q], ph);
    if (T.start && bound) {
      // the orbit step's index tables, star by star: bucket starts (from the
      // float keys of 1/r of this star and its predecessor, as t32 holds
      // them) and the grid cells between 1/r of this star and the next
      const int c = R.seg;
      const int64_t k = p - R.seg_begin, nb = R.bound_end - R.seg_begin;
      const int4 pr = T.prm[c];
      if (k >= pr.z && k <= pr.w) {
        const double xm1 = e > 0 ? s_x[pad8(e - 1)] : (k > 0 ? __ldg(x + p - 1) : 0.0);
        bucket_starts_of(k, nb, pr, T.base[c], __float_as_uint(f32_pair(s_x[q]).hi),
                         k > pr.z ? __float_as_uint(f32_pair(xm1).hi) : 0u,
                         T.start + T.boff[c], T.boff[c + 1] - T.boff[c]);
      }
      const double xk1 = k + 1 < nb ? (e + 1 < kTile ? s_x[pad8(e + 1)] : __ldg(x + p + 1)) : 0.0;
      grid_shells_of(k, nb, s_x[q], xk1, T.gprm[c], T.gshell + T.goff[c]);
    }
  }
}

// The slopes k_potential leaves to the seams between tiles: the last star
// of every tile whose next star (in the next tile) is bound.
__global__ void k_slope_seams(Seg S, const int64_t* esc, bool sub, const double* r,
                              const double* x, const double* phi, double* M,
                              double4_32a* node, int64_t n_tiles) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  TR R = tile_of(S, esc, t, sub);
  const int64_t p = R.end - 1;
  if (p < R.begin || p + 1 >= R.bound_end) return;
  const double xj = x[p], pj = phi[p], xj1 = x[p + 1], pj1 = phi[p + 1];
  const double w = div_rn(pj1 - pj, xj - xj1);
  if (M) M[p] = w;
  node[p] = make_double4_32a(r[p], xj, pj, w);
}

// ---------------------------------------------------- energy correction
// T' = T + 1/2 [(Phi_new(r_old) - Phi_new(r_new)) - (Phi_old(r_old) -
// Phi_old(r_new))], clamped at 0; both components scaled by sqrt(T'/T).
__global__ void k_correction(Seg S, const int64_t* esc, bool sub, const double* r,
                             const double* x, const double* phi, double* vr, double* vt,
                             const double* r_old, const double* cc, const double* m,
                             int64_t n) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool active = p < n;
  int c = 0;
  int64_t k = 0, nbc = 0, sb = 0;
  if (active) {
    c = seg_find(S.off, S.n_seg, p);
    sb = __ldg(S.off + c);
    k = p - sb;
    nbc = nb_eff(S.nb, esc, c, sub);
    active = k < nbc;
  }
  unsigned long long clamp = 0;
  if (active) {
    Table64 T{r + sb, x + sb, phi + sb, nbc};
    double a = vr[p], b = vt[p];
    double Tk = scale_down<1>(a * a + b * b);
    double dnew = phi_of_r(T, r_old[p]) - phi[p];
    double Tp = Tk + scale_down<1>(dnew - cc[p]);
    if (Tp < 0.0) {
      if (m) clamp_energy_add(S.stats, c, m[p], Tp);
      Tp = 0.0;
      clamp = 1;
    }
    if (Tk > 0.0) {
      double f = sqrt_rn(div_rn(Tp, Tk));
      vr[p] = a * f;
      vt[p] = b * f;
    }
  }
  if (clamp) stat_add(S.stats, c, kStClamps, 1ull);
}

// ---------------------------------------------------------- diagnostics
__global__ void __launch_bounds__(kThreads) k_energy_tiles(Seg S, const double* r,
                                                           const double* vr, const double* vt,
                                                           const double* m,
                                                           const double* tile_m,
                                                           double* tile_k, double* tile_w,
                                                           double* Mout) {
  __shared__ double s1[kThreads], s2[kThreads];
  TR R = tile_of(S, nullptr, blockIdx.x, false);
  const int64_t t0 = blockIdx.x - R.lt;
  double pm = 0.0;
  for (int64_t j = threadIdx.x; j < R.lt; j += kThreads) pm = pm + tile_m[t0 + j];
  double Mbefore = block_sum(pm, s1);
  const int64_t b = R.begin + (int64_t)threadIdx.x * kPer;
  double mm[kPer];
  double am = 0.0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    int64_t p = b + i;
    mm[i] = (p < R.end && p < R.bound_end) ? m[p] : 0.0;
    am = am + mm[i];
  }
  double pre_m, dummy;
  block_scans(am, 0.0, s1, s2, pre_m, dummy);
  double run = 0.0, ak = 0.0, aw = 0.0;
#pragma unroll
  for (int i = 0; i < kPer; ++i) {
    int64_t p = b + i;
    if (p < R.end && p < R.bound_end) {
      double Mex = (Mbefore + pre_m) + run;  // mass strictly inside star p
      double a = vr[p], bb = vt[p];
      ak = ak + mm[i] * (a * a + bb * bb);
      aw = aw + mm[i] * Mex / r[p];
      run = run + mm[i];
      if (Mout) Mout[p] = (Mbefore + pre_m) + run;
    } else if (p < R.end && Mout) {
      Mout[p] = 0.0;
    }
  }
  double tk = block_sum(ak, s1);
  double tw = block_sum(aw, s1);
  if (threadIdx.x == 0) { tile_k[blockIdx.x] = tk; tile_w[blockIdx.x] = tw; }
}

// Core diagnostics (section 4.2, Eq. 19): per bound star k with three
// neighbours on each side, the 6th-order density estimate in the radial
// order, rho_k = (m_{k-2} + ... + m_{k+2}) / (4 pi / 3 (r_{k+3}^3 - r_{k-3}^3));
// per tile the sums of rho, rho^2, rho r and the number of estimates, each
// in a fixed order (runs of 16 per thread, then a fixed tree).
__global__ void __launch_bounds__(kThreads) k_core_tiles(Seg S, const double* r, const double* m,
                                                         double* tile_s1, double* tile_s2,
                                                         double* tile_sr, double* tile_n) {
  __shared__ double s[kThreads];
  TR R = tile_of(S, nullptr, blockIdx.x, false);
  const int64_t b = R.begin + (int64_t)threadIdx.x * kPer;
  const double c43 = (4.0 * kPi) / 3.0;
  double a1 = 0.0, a2 = 0.0, ar = 0.0, an = 0.0;
  for (int i = 0; i < kPer; ++i) {
    const int64_t p = b + i;
    const int64_t k = p - R.seg_begin;
    if (p >= R.end || k < 3 || p + 3 >= R.bound_end) continue;
    const double ro = r[p + 3], ri = r[p - 3];
    const double vol = c43 * (ro * ro * ro - ri * ri * ri);
    if (!pos_num(vol)) continue;
    const double mass = (((m[p - 2] + m[p - 1]) + m[p]) + m[p + 1]) + m[p + 2];
    const double rho = mass / vol;
    a1 = a1 + rho;
    a2 = a2 + rho * rho;
    ar = ar + rho * r[p];
    an = an + 1.0;
  }
  const double t1 = block_sum(a1, s), t2 = block_sum(a2, s), tr = block_sum(ar, s),
               tn = block_sum(an, s);
  if (threadIdx.x == 0) {
    tile_s1[blockIdx.x] = t1;
    tile_s2[blockIdx.x] = t2;
    tile_sr[blockIdx.x] = tr;
    tile_n[blockIdx.x] = tn;
  }
}

// per cluster: rho_c = sum rho^2 / sum rho, r_c = sum rho r / sum rho and the
// number of estimates (3 doubles per cluster)
__global__ void __launch_bounds__(kThreads) k_core_final(Seg S, const double* tile_s1,
                                                         const double* tile_s2,
                                                         const double* tile_sr,
                                                         const double* tile_n, double* out3) {
  __shared__ double s[kThreads];
  const int c = blockIdx.x;
  const int64_t t0 = S.tile_off[c], t1 = S.tile_off[c + 1];
  double a1 = 0.0, a2 = 0.0, ar = 0.0, an = 0.0;
  for (int64_t j = t0 + threadIdx.x; j < t1; j += kThreads) {
    a1 = a1 + tile_s1[j];
    a2 = a2 + tile_s2[j];
    ar = ar + tile_sr[j];
    an = an + tile_n[j];
  }
  const double S1 = block_sum(a1, s), S2 = block_sum(a2, s), SR = block_sum(ar, s),
               SN = block_sum(an, s);
  if (threadIdx.x == 0) {
    out3[3 * c + 0] = S1 > 0.0 ? S2 / S1 : 0.0;
    out3[3 * c + 1] = S1 > 0.0 ? SR / S1 : 0.0;
    out3[3 * c + 2] = SN;
  }
}

__global__ void __launch_bounds__(kThreads) k_energy_final(Seg S, const double* tile_k,
                                                           const double* tile_w,
                                                           double* out3) {
  __shared__ double s[kThreads];
  const int c = blockIdx.x;
  int64_t t0 = S.tile_off[c], t1 = S.tile_off[c + 1];
  double ak = 0.0, aw = 0.0;
  for (int64_t j = t0 + threadIdx.x; j < t1; j += kThreads) {
    ak = ak + tile_k[j];
    aw = aw + tile_w[j];
  }
  double K = block_sum(ak, s);
  double W = block_sum(aw, s);
  if (threadIdx.x == 0) {
    out3[3 * c + 0] = 0.5 * K;
    out3[3 * c + 1] = -W;
    out3[3 * c + 2] = 0.5 * K - W;
  }
}

__global__ void k_lagrange(Seg S, const double* r, const double* M, const double* fracs,
                           int nf, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S.n_seg * nf) return;
  int c = i / nf, q = i % nf;
  int64_t sb = S.off[c], nbc = S.nb[c];
  if (nbc <= 0) { out[i] = 0.0; return; }
  double target = fracs[q] * M[sb + nbc - 1];
  int64_t lo = -1, hi = nbc - 1;  // first k with M_k >= target (M[nb-1] qualifies)
  while (hi - lo > 1) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (M[sb + mid] >= target) hi = mid; else lo = mid;
  }
  out[i] = r[sb + hi];
}

__global__ void k_validate(int64_t n, const double* r, const double* vr, const double* vt,
                           const double* m, bool allow_inf, uint32_t* err) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double rr = r[p], a = vr[p], b = vt[p], mm = m[p];
  bool rok = (rr > 0.0) && (isfinite(rr) || (allow_inf && isinf(rr)));
  bool ok = rok && isfinite(a) && isfinite(b) && (b >= 0.0) && isfinite(mm) && (mm >= 0.0);
  if (!ok) set_err(err, kErrInput);
}

__global__ void k_check_ids(int64_t n, const int64_t* off, int n_seg, const uint64_t* ids,
                            uint32_t* err) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p + 1 >= n) return;
  int c = seg_find(off, n_seg, p);
  if (p + 1 < off[c + 1] && ids[p] == ids[p + 1]) set_err(err, kErrInput);
}

// Whether the staged stars are already in (r, id) order within every
// segment (bit patterns of positive or infinite r order like the values),
// flag bit 0 set otherwise, and the largest id of each segment.
__global__ void k_order_check(int64_t n, const int64_t* off, int n_seg, const double* r,
                              const uint32_t* id, uint32_t* flag, unsigned int* maxid) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < n;
  int c = 0;
  uint32_t ip = 0;
  if (live) {
    c = seg_find(off, n_seg, p);
    ip = id[p];
    if (p + 1 < off[c + 1]) {
      const unsigned long long a = ubits(r[p]), b = ubits(r[p + 1]);
      if (!(a < b || (a == b && ip < id[p + 1]))) atomicOr(flag, 1u);
    }
  }
  // one atomic per segment present in the warp
  const unsigned full = __activemask();
  const unsigned peers = __match_any_sync(full, live ? c : -1);
  const unsigned mx = __reduce_max_sync(peers, ip);
  if (live && (threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(maxid + c, mx);
}

// Duplicate ids of sorted input: bit bitoff[c] + id of a bitmap per star;
// a bit found set already is a duplicate (error)
__global__ void k_ids_bitmap(int64_t n, const int64_t* off, int n_seg, const uint32_t* id,
                             const unsigned long long* bitoff, unsigned long long* bitmap,
                             uint32_t* err) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c = seg_find(off, n_seg, p);
  const unsigned long long b = bitoff[c] + id[p];
  const unsigned long long bit = 1ull << (b & 63ull);
  if (atomicOr(bitmap + (b >> 6), bit) & bit) set_err(err, kErrInput);
}

// One 256-thread block per segment.  The stars that escaped in this step
// are the escaped range's entries with a finite r_old (earlier escapers
// carry r_old = inf); their mass and energy m_k e_k (e_k in c) are summed
// in a fixed order and added to the segment's budget (section 4.2).
__global__ void __launch_bounds__(256) k_step_end(Seg S, int64_t* esc, uint64_t* dt_last,
                                                  uint32_t* step, const double* r_old,
                                                  const double* e, const double* m,
                                                  double* esc_me) {
  __shared__ double s_m[256], s_e[256];
  const int c = blockIdx.x, t = threadIdx.x;
  const int64_t ne = esc[c];
  const int64_t nb_new = S.nb[c] - ne;
  double dm = 0.0, de = 0.0;
  if (ne > 0)
    for (int64_t p = S.off[c] + nb_new + t; p < S.off[c + 1]; p += 256)
      if (isfinite(r_old[p])) {
        dm += m[p];
        de += m[p] * e[p];
      }
  s_m[t] = dm;
  s_e[t] = de;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) {
      s_m[t] += s_m[t + w];
      s_e[t] += s_e[t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    if (ne > 0) {
      esc_me[2 * c] += s_m[0];
      esc_me[2 * c + 1] += s_e[0];
    }
    dt_last[c] = S.dt_bits[c];
    S.nb[c] = nb_new;
    // the stars merged away in this step (sticky spheres) left with the
    // escapers; they are counted as collisions, not as escapes
    unsigned long long* st = S.stats + (size_t)c * kStStride;
    const unsigned long long merged = st[kStCollisions] - st[kStCollisionsSeen];
    st[kStCollisionsSeen] = st[kStCollisions];
    st[kStEscaped] += (unsigned long long)ne - merged;
    esc[c] = 0;
    S.dt_bits[c] = 0x7FF0000000000000ull;
    if (c == 0) *step += 1u;
  }
}

// one record of the diagnostics ring per segment, after the step end (the
// step counter already advanced): slot (step - 1) mod cap
__global__ void k_diag_ring(Seg S, const double* out3, const uint64_t* dt_last,
                            const double* esc_me, const uint32_t* step, const uint32_t* err,
                            double* ring, int cap) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= S.n_seg) return;
  const uint32_t stp = *step;
  double* rec = ring + ((size_t)c * cap + (stp - 1u) % (uint32_t)cap) * kDiagFields;
  const double K = out3[3 * c], W = out3[3 * c + 1];
  rec[0] = (double)stp;
  rec[1] = __longlong_as_double((long long)dt_last[c]);
  rec[2] = (double)S.nb[c];
  rec[3] = K;
  rec[4] = W;
  rec[5] = (K + W) + esc_me[2 * c + 1];
  rec[6] = esc_me[2 * c];
  rec[7] = esc_me[2 * c + 1];
  rec[8] = (double)S.stats[(size_t)c * kStStride + kStTrials];
  rec[9] = (double)*err;
}

__global__ void k_nb_from_keys(Seg S, const uint64_t* keys) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= S.n_seg) return;
  int64_t sb = S.off[c], se = S.off[c + 1];
  int64_t lo = sb - 1, hi = se;  // first escaper key in [sb, se)
  while (hi - lo > 1) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (key_is_escaper(keys[mid])) hi = mid; else lo = mid;
  }
  S.nb[c] = hi - sb;
}

__global__ void k_recip(int64_t n, const double* r, double* x) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) x[p] = 1.0 / r[p];
}

__global__ void k_make_t32(int64_t n, const double* x, const double* phi, float2* t32) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) t32[p] = make_float2((float)x[p], (float)phi[p]);
}

__global__ void k_make_nodes(int64_t n, const double* r, const double* x, const double* phi,
                             const double* M, double4_32a* node, float4* tdf) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  node[p] = make_double4_32a(r[p], x[p], phi[p], M[p]);
  tdf[p] = float_pairs(x[p], phi[p]);
}

__global__ void k_unpack_orbit(int64_t n, const uint64_t* keys, const Payload* pay,
                               double* r_new, double* vr_new, double* vt_new) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint64_t k = keys[p];
  r_new[p] = key_is_escaper(k) ? __longlong_as_double(0x7FF0000000000000ll)
                               : __longlong_as_double((long long)k);
  if (vr_new) vr_new[p] = pay[p].vr;
  if (vt_new) vt_new[p] = pay[p].vt;
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void launch_nb_from_keys(const SegLayout& L, const uint64_t* keys, cudaStream_t st) {
  k_nb_from_keys<<<blocks_for(L.n_seg, 128), 128, 0, st>>>(L.dev(), keys);
}

void launch_recip(int64_t n, const double* r, double* x, cudaStream_t st) {
  if (n > 0) k_recip<<<blocks_for(n, 256), 256, 0, st>>>(n, r, x);
}

void launch_make_t32(int64_t n, const double* x, const double* phi, float2* t32,
                     cudaStream_t st) {
  if (n > 0) k_make_t32<<<blocks_for(n, 256), 256, 0, st>>>(n, x, phi, t32);
}

void launch_make_nodes(int64_t n, const double* r, const double* x, const double* phi,
                       const double* M, double4_32a* node, float4* tdf, cudaStream_t st) {
  if (n > 0) k_make_nodes<<<blocks_for(n, 256), 256, 0, st>>>(n, r, x, phi, M, node, tdf);
}

void launch_unpack_orbit(int64_t n, const uint64_t* keys, const Payload* pay, double* r_new,
                         double* vr_new, double* vt_new, cudaStream_t st) {
  if (n > 0)
    k_unpack_orbit<<<blocks_for(n, 256), 256, 0, st>>>(n, keys, pay, r_new, vr_new, vt_new);
}

// ------------------------------------------------------------------ host
cudaError_t alloc_layout(SegLayout& L, const std::vector<int64_t>& sizes,
                         const std::vector<uint64_t>& seeds, const std::vector<double>& lnL,
                         int bin_size, cudaStream_t st) {
  L.n_seg = (int)sizes.size();
  L.bin_size = bin_size;
  L.h_off.assign(L.n_seg + 1, 0);
  L.h_tile_off.assign(L.n_seg + 1, 0);
  L.h_pair_off.assign(L.n_seg + 1, 0);
  L.h_bin_off.assign(L.n_seg + 1, 0);
  L.max_tiles_per_seg = 0;
  for (int c = 0; c < L.n_seg; ++c) {
    int64_t nc = sizes[c];
    int64_t nt = (nc + kTile - 1) / kTile;
    L.h_off[c + 1] = L.h_off[c] + nc;
    L.h_tile_off[c + 1] = L.h_tile_off[c] + nt;
    L.h_pair_off[c + 1] = L.h_pair_off[c] + nc / 2;
    L.h_bin_off[c + 1] = L.h_bin_off[c] + (nc + bin_size - 1) / bin_size;
    if (nt > L.max_tiles_per_seg) L.max_tiles_per_seg = nt;
  }
  L.n = L.h_off[L.n_seg];
  L.n_tiles = L.h_tile_off[L.n_seg];
  L.n_pairs = L.h_pair_off[L.n_seg];
  L.n_bins = L.h_bin_off[L.n_seg];
  size_t s1 = sizeof(int64_t) * (L.n_seg + 1);
  cudaError_t e;
#define CMC_A(ptr, bytes) \
  if ((e = cudaMallocAsync((void**)&(ptr), (bytes), st))) return e;
  CMC_A(L.off, s1);
  CMC_A(L.tile_off, s1);
  CMC_A(L.pair_off, s1);
  CMC_A(L.bin_off, s1);
  CMC_A(L.seed, sizeof(uint64_t) * L.n_seg);
  CMC_A(L.lnL, sizeof(double) * L.n_seg);
  CMC_A(L.nb, sizeof(int64_t) * L.n_seg);
  CMC_A(L.esc_step, sizeof(int64_t) * L.n_seg);
  CMC_A(L.dt_bits, sizeof(uint64_t) * L.n_seg);
  CMC_A(L.dt_last, sizeof(uint64_t) * L.n_seg);
  CMC_A(L.stats, sizeof(unsigned long long) * kStStride * L.n_seg);
  CMC_A(L.esc_me, sizeof(double) * 2 * L.n_seg);
  CMC_A(L.dt_cap, sizeof(double) * L.n_seg);
#undef CMC_A
  cudaMemcpyAsync(L.off, L.h_off.data(), s1, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.tile_off, L.h_tile_off.data(), s1, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.pair_off, L.h_pair_off.data(), s1, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.bin_off, L.h_bin_off.data(), s1, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.seed, seeds.data(), sizeof(uint64_t) * L.n_seg, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.lnL, lnL.data(), sizeof(double) * L.n_seg, cudaMemcpyHostToDevice, st);
  std::vector<int64_t> nb(sizes.begin(), sizes.end());
  cudaMemcpyAsync(L.nb, nb.data(), sizeof(int64_t) * L.n_seg, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(L.esc_step, 0, sizeof(int64_t) * L.n_seg, st);
  std::vector<uint64_t> inf(L.n_seg, 0x7FF0000000000000ull);
  cudaMemcpyAsync(L.dt_bits, inf.data(), sizeof(uint64_t) * L.n_seg, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(L.dt_last, inf.data(), sizeof(uint64_t) * L.n_seg, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(L.stats, 0, sizeof(unsigned long long) * kStStride * L.n_seg, st);
  cudaMemsetAsync(L.esc_me, 0, sizeof(double) * 2 * L.n_seg, st);
  cudaMemsetAsync(L.dt_cap, 0, sizeof(double) * L.n_seg, st);
  // the host vectors above must outlive the copies
  return cudaStreamSynchronize(st);
}

void free_layout(SegLayout& L, cudaStream_t st) {
  void* ps[] = {L.off, L.tile_off, L.pair_off, L.bin_off, L.seed, L.lnL,
                L.nb, L.esc_step, L.dt_bits, L.dt_last, L.stats, L.esc_me, L.dt_cap};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, st);
  L = SegLayout();
}

void launch_make_keys(const SegLayout& L, const double* r, const double* vr,
                      const double* vt, const double* m, const uint32_t* id,
                      uint64_t* keys, Payload* pay, cudaStream_t st) {
  if (L.n) k_make_keys<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, r, vr, vt, m, id, keys, pay);
}

void launch_id_keys(const SegLayout& L, const uint32_t* id, uint64_t* keys, cudaStream_t st) {
  if (L.n) k_id_keys<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, id, keys);
}

void launch_rekey_radius(const SegLayout& L, const uint32_t* perm, const double* r,
                         const uint32_t* id, uint64_t* keys, cudaStream_t st) {
  if (L.n) k_rekey_radius<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, perm, r, id, keys);
}

void launch_gather(const SegLayout& L, const uint64_t* keys, const uint32_t* vals,
                   const Payload* pay, double* r, double* x, double* vr, double* vt,
                   double* m, uint32_t* id, double* r_old, double* c, cudaStream_t st,
                   double* tile_m, double* tile_mx, const double* Rp, double* Rout,
                   const double* Ap, double* Aout, bool packed) {
  if (!L.n) return;
  if (tile_m && tile_mx && r_old && c && L.n_tiles)
    k_gather_sums<<<(unsigned)L.n_tiles, kThreads, 0, st>>>(L.dev(), L.esc_step, L.n, keys, vals,
                                                            pay, r, x, vr, vt, m, id, r_old, c,
                                                            tile_m, tile_mx, Rp, Rout, Ap,
                                                            Aout, packed);
  else
    k_gather<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, keys, vals, pay, r, x, vr, vt, m, id,
                                                  r_old, c);
}

constexpr size_t kPotentialSmem = sizeof(double) * 3 * kPad8N;

void potential_prepare() {
  cudaFuncSetAttribute(k_potential, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kPotentialSmem);
}

void launch_potential(const SegLayout& L, const double* r, const double* x, const double* m,
                      double* tile_m, double* tile_mx, double* phi, float2* t32,
                      double* Mout, bool nb_sub, cudaStream_t st, double4_32a* node,
                      float4* tdf, bool sums_ready, bool slopes, const TableOut* tables) {
  if (!L.n_tiles) return;
  Seg S = L.dev();
  if (!sums_ready)
    k_tile_sums<<<(unsigned)L.n_tiles, kThreads, 0, st>>>(S, L.esc_step, nb_sub, x, m, tile_m,
                                                         tile_mx);
  k_potential<<<(unsigned)L.n_tiles, kPotThreads, kPotentialSmem, st>>>(
      S, L.esc_step, nb_sub, r, x, m, tile_m, tile_mx, phi, t32, Mout, node, tdf, slopes,
      tables ? *tables : TableOut());
  // with the tables, the seams' slopes come with the grid's values
  if (slopes && node && !tables)
    k_slope_seams<<<blocks_for(L.n_tiles, 128), 128, 0, st>>>(S, L.esc_step, nb_sub, r, x, phi,
                                                              Mout, node, L.n_tiles);
}

void launch_correction(const SegLayout& L, const double* r, const double* x,
                       const double* phi, double* vr, double* vt, const double* r_old,
                       const double* c, bool nb_sub, uint32_t* err, cudaStream_t st,
                       const double* m) {
  (void)err;
  if (!L.n) return;
  k_correction<<<blocks_for(L.n, 128), 128, 0, st>>>(L.dev(), L.esc_step, nb_sub, r, x, phi,
                                                    vr, vt, r_old, c, m, L.n);
}

void launch_energy(const SegLayout& L, const double* r, const double* vr, const double* vt,
                   const double* m, double* tile_m, double* tile_k, double* tile_w,
                   double* Mbuf, double* out3, cudaStream_t st) {
  if (!L.n_tiles) return;
  Seg S = L.dev();
  k_tile_sums<<<(unsigned)L.n_tiles, kThreads, 0, st>>>(S, L.esc_step, false, r, m, tile_m,
                                                       tile_k);
  k_energy_tiles<<<(unsigned)L.n_tiles, kThreads, 0, st>>>(S, r, vr, vt, m, tile_m, tile_k,
                                                          tile_w, Mbuf);
  k_energy_final<<<(unsigned)L.n_seg, kThreads, 0, st>>>(S, tile_k, tile_w, out3);
}

void launch_diag_ring(const SegLayout& L, const double* out3, const uint32_t* step,
                      const uint32_t* err, double* ring, int cap, cudaStream_t st) {
  if (!L.n_seg || cap <= 0) return;
  k_diag_ring<<<(unsigned)((L.n_seg + 127) / 128), 128, 0, st>>>(L.dev(), out3, L.dt_last,
                                                                L.esc_me, step, err, ring, cap);
}

void launch_core(const SegLayout& L, const double* r, const double* m, double* tiles4,
                 double* out3, cudaStream_t st) {
  if (!L.n_tiles) return;
  Seg S = L.dev();
  const int64_t t = L.n_tiles;
  k_core_tiles<<<(unsigned)t, kThreads, 0, st>>>(S, r, m, tiles4, tiles4 + t, tiles4 + 2 * t,
                                                  tiles4 + 3 * t);
  k_core_final<<<(unsigned)L.n_seg, kThreads, 0, st>>>(S, tiles4, tiles4 + t, tiles4 + 2 * t,
                                                       tiles4 + 3 * t, out3);
}

void launch_lagrange(const SegLayout& L, const double* r, const double* M,
                     const double* fracs, int nf, double* out, cudaStream_t st) {
  int n = L.n_seg * nf;
  if (n) k_lagrange<<<blocks_for(n, 128), 128, 0, st>>>(L.dev(), r, M, fracs, nf, out);
}

void launch_validate(const SegLayout& L, const double* r, const double* vr,
                     const double* vt, const double* m, bool allow_inf, uint32_t* err,
                     cudaStream_t st) {
  if (L.n) k_validate<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, r, vr, vt, m, allow_inf, err);
}

void launch_order_check(const SegLayout& L, const double* r, const uint32_t* id, uint32_t* flag,
                        unsigned int* maxid, cudaStream_t st) {
  if (L.n) k_order_check<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, L.off, L.n_seg, r, id, flag,
                                                               maxid);
}

void launch_ids_bitmap(const SegLayout& L, const uint32_t* id, const unsigned long long* bitoff,
                       unsigned long long* bitmap, uint32_t* err, cudaStream_t st) {
  if (L.n) k_ids_bitmap<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, L.off, L.n_seg, id, bitoff,
                                                              bitmap, err);
}

void launch_check_ids(const SegLayout& L, const uint64_t* sorted_ids, uint32_t* err,
                      cudaStream_t st) {
  if (L.n > 1)
    k_check_ids<<<blocks_for(L.n, 256), 256, 0, st>>>(L.n, L.off, L.n_seg, sorted_ids, err);
}

void launch_step_end(const SegLayout& L, uint32_t* step, const double* r_old, const double* c,
                     const double* m, cudaStream_t st) {
  k_step_end<<<L.n_seg, 256, 0, st>>>(L.dev(), L.esc_step, L.dt_last, step, r_old, c, m,
                                      L.esc_me);
}

CMC_DEBUG_SITE_ACCESSOR

}  // namespace cmc
