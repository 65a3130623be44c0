// Device-side building blocks shared by the kernels of the Henon Monte Carlo
// timestep (Pattabiraman et al., section 2.1): counter-based random numbers,
// the segment (cluster) layout, error flags, and the shell potential of
// Eqs. 1 and 6 evaluated from the sorted table.
//
// Every kernel is compiled with --fmad=false: each floating-point operation
// is one IEEE-754 round-to-nearest operation in the order written, so the
// FP64 path reproduces an independent FP64 statement of the same method bit
// for bit.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cmc {

// ---------------------------------------------------------------- sizes
constexpr int kTile = 4096;          // elements per tile (sort, gather, scans)
constexpr int kBins = 256;           // radix digits per pass (8 bits)
constexpr double kPi = 3.14159265358979323846;

// stream tags (third counter word of the per-star random stream)
constexpr uint32_t kTagPsi = 0;      // relaxation: azimuth of star 2's v_t
constexpr uint32_t kTagPhi = 1;      // relaxation: azimuth of the deflection
constexpr uint32_t kTagRej = 2;      // orbit: rejection trials
constexpr uint32_t kTagSgn = 3;      // orbit: sign of the new v_r
constexpr uint32_t kTagCol = 4;      // relaxation pair: sticky-sphere collision draw

// escaped stars sort after every finite radius, by id: key 0x7FF0...0 | id
// << 20, above every finite radius (the timestep's sort orders by the top
// 40 bits and puts runs equal in them -- escapers whose ids differ only in
// their low 4 bits -- in (key, id) order, which for these keys is id order)
constexpr uint64_t kEscKeyBase = 0x7FF0000000000000ull;

// Debug builds (-DCMC_DEBUG, libcmc_debug.so): index checks at the table
// probes and scatters that a wrong bracket, bucket or segment offset would
// send out of range.  A failed check records the first failing site of its
// translation unit (CMC_TU x 100000 + source line) in that unit's
// g_debug_site, and the access is skipped; release builds compile the
// checks to nothing.
#ifndef CMC_TU
#define CMC_TU 0
#endif
#ifdef CMC_DEBUG
static __device__ unsigned int g_debug_site = 0u;
__device__ __forceinline__ bool debug_in(unsigned long long i, unsigned long long n,
                                         unsigned site) {
  if (i < n) return true;
  atomicCAS(&g_debug_site, 0u, site);
  return false;
}
#define CMC_IN(i, n) \
  ::cmc::debug_in((unsigned long long)(i), (unsigned long long)(n), CMC_TU * 100000u + __LINE__)
#else
#define CMC_IN(i, n) true
#endif

// error bits (fatal: they poison the context)
enum : uint32_t {
  kErrTimeout = 1u << 0,   // a bounded device wait gave up
  kErrTies = 1u << 1,      // a run of equal radii too long to order by id
  kErrInput = 1u << 2,     // invalid input state
  kErrNonFinite = 1u << 3, // a non-finite velocity appeared
};

// per-segment statistics (64-bit counters)
enum : int {
  kStEscaped = 0, kStDegenerate, kStCapHits, kStTrials, kStViolations,
  kStClamps, kStAngleFails, kStTies, kStFp64Trials, kStClampEnergy, kStCollisions,
  kStCollisionEnergy, kStEnvelope64, kStCount
};
// (slot 15: the collision count at the last step end, to tell this step's
// merged-away stars from its escapers)
constexpr int kStCollisionsSeen = 15;
constexpr int kStStride = 16;        // counters reserved per segment
constexpr int kDiagFields = 10;      // doubles per diagnostics record

// ------------------------------------------------------- segment layout
// Clusters of an ensemble are stored back to back.  Segment c owns global
// positions [off[c], off[c+1]); its bound stars are the first nb[c].
struct Seg {
  const int64_t* off;      // n_seg + 1 offsets (device)
  const int64_t* tile_off; // n_seg + 1 tile offsets (device)
  const int64_t* pair_off; // n_seg + 1 pair offsets (by capacity, device)
  const int64_t* bin_off;  // n_seg + 1 bin offsets (by capacity, device)
  const uint64_t* seed;    // per segment
  const double* lnL;       // ln(gamma N_c), per segment
  int64_t* nb;             // bound stars per segment (device, changes)
  uint64_t* dt_bits;       // timestep per segment as double bits
  const double* dt_cap;    // per segment: an outside bound on the timestep (0: none)
  unsigned long long* stats;  // kStStride counters per segment
  uint4* taus;             // combined-Tausworthe streams, one per id slot (or null)
  const int64_t* taus_base;  // per segment: first stream slot (slot = base + id)
  int n_seg;
};

// largest c with a[c] <= v, for a sorted array of n+1 offsets (a[0] = 0)
__device__ __forceinline__ int seg_find(const int64_t* a, int n, int64_t v) {
  int lo = 0, hi = n;  // invariant a[lo] <= v < a[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------- exact operations on bit patterns
// The FP64 pipe of this GPU issues two lanes per SM and clock, and most of
// the timestep's kernels are bound by it.  Operations that need no FP64
// arithmetic -- comparisons, rounding to float, scaling by 1/2 or 1/4 --
// run on the integer pipes from the bit patterns; each gives the IEEE-754
// result of the FP64 operation it replaces (NaN, infinities, zeros and
// subnormals included, by the bit tests or by falling back to the FP64
// operation where the shortcut does not hold).
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;
constexpr unsigned long long kSignBit = 0x8000000000000000ull;

__device__ __forceinline__ unsigned long long ubits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}
// v < 0.0
__device__ __forceinline__ bool lt0(double v) {
  const unsigned long long u = ubits(v);
  return u > kSignBit && u <= (kSignBit | kInfBits);
}
// v > 0.0 (+Inf included)
__device__ __forceinline__ bool pos_num(double v) { return ubits(v) - 1ull < kInfBits; }
// v >= 0.0 (-0 included)
__device__ __forceinline__ bool ge0(double v) {
  const unsigned long long u = ubits(v);
  return u <= kInfBits || u == kSignBit;
}
// v < +Inf
__device__ __forceinline__ bool lt_inf(double v) {
  const unsigned long long u = ubits(v);
  return (u & ~kSignBit) <= kInfBits && u != kInfBits;
}
// v <= 1.0
__device__ __forceinline__ bool le1(double v) {
  const unsigned long long u = ubits(v);
  return (u & ~kSignBit) <= kInfBits && (u >= kSignBit || u <= 0x3FF0000000000000ull);
}
// v >= rj for rj > 0
__device__ __forceinline__ bool ge_pos(double v, double rj) {
  const unsigned long long u = ubits(v);
  return u >= ubits(rj) && u <= kInfBits;
}
// a > b for a > 0 (b any value but NaN)
__device__ __forceinline__ bool gt_pos(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}
// v 2^-k for k = 1, 2: the exponent field lowered by k when the result stays
// normal, else the FP64 product
template <int k>
__device__ __forceinline__ double scale_down(double v) {
  const unsigned long long u = ubits(v);
  const unsigned f = (unsigned)(u >> 52) & 0x7FFu;
  if (f > (unsigned)k && f < 0x7FFu) return __longlong_as_double((long long)(u - ((unsigned long long)k << 52)));
  return v * (k == 1 ? 0.5 : 0.25);
}
// v 2^k for k = 1, 2: the exponent field raised by k when v and the result
// are normal, else the FP64 product
template <int k>
__device__ __forceinline__ double scale_up(double v) {
  const unsigned long long u = ubits(v);
  const unsigned f = (unsigned)(u >> 52) & 0x7FFu;
  if (f - 1u < 2046u - (unsigned)k) return __longlong_as_double((long long)(u + ((unsigned long long)k << 52)));
  return v * (k == 1 ? 2.0 : 4.0);
}
// (float)v: the top 24 significand bits rounded to nearest even by the 29
// bits below them, for doubles whose float is normal (2^-126 <= |v| <
// 2^126); others by the conversion
__device__ __forceinline__ float f32_rn(double v) {
  const unsigned long long u = ubits(v);
  const unsigned ex = (unsigned)(u >> 52) & 0x7FFu;
  if (ex - 897u > 252u) return (float)v;  // outside [897, 1149]
  const unsigned top = ((ex - 896u) << 23) | ((unsigned)(u >> 29) & 0x7FFFFFu);
  const unsigned rest = (unsigned)u & 0x1FFFFFFFu;
  const bool up = rest > 0x10000000u || (rest == 0x10000000u && (top & 1u));
  return __uint_as_float(((unsigned)(u >> 32) & 0x80000000u) | (top + (up ? 1u : 0u)));
}

// Correctly rounded FP64 product, quotient and square root from 64-bit
// integer arithmetic on the significands, for normal operands with a normal
// result (anything else: the FP64 operation).  On this GPU an FP64 division
// or square root takes several FP64 issues; these take none, and the FP64
// pipe is left to the additions.  Each returns the IEEE-754 round-to-
// nearest-even result exactly (checked bit for bit against the FP64
// operations on 3 x 2^28 operand pairs per operation: random bit patterns,
// random values over 81 binades, and significands with random runs of
// trailing zeros, which give exact results and ties).
//
// The significands are integers in [2^52, 2^53); the result's significand Q
// is an integer in the same range, its exponent follows from the operands'.
// A result assembled as sign + ((e - 1) << 52) + Q lets a significand that
// rounds up to 2^53 carry into the exponent.
__device__ __forceinline__ unsigned long long significand(unsigned long long u) {
  return (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
}

// a b: the 106-bit product of the significands, its top 53 bits rounded to
// nearest even by the bits below them.
__device__ __forceinline__ double mul_rn(double a, double b) {
  const unsigned long long ua = ubits(a), vb = ubits(b);
  const unsigned ea = (unsigned)(ua >> 52) & 0x7FFu, eb = (unsigned)(vb >> 52) & 0x7FFu;
  const int e = (int)ea + (int)eb - 1023;  // the result's biased exponent, before a carry
  if (ea - 1u < 2046u && eb - 1u < 2046u && (unsigned)(e - 2) < 2043u) {
    const unsigned long long ma = significand(ua), mb = significand(vb);
    const unsigned long long hi = __umul64hi(ma, mb), lo = ma * mb;
    const unsigned c = (unsigned)(hi >> 41);  // product >= 2^105
    const unsigned long long m = (hi << (12 - c)) | (lo >> (52 + c));
    const unsigned long long rest = lo << (12 - c);  // the dropped bits, left-aligned
    const unsigned long long up = (rest >> 63) & ((rest << 1) != 0ull ? 1ull : (m & 1ull));
    return __longlong_as_double((long long)(((ua ^ vb) & kSignBit) +
                                            ((unsigned long long)(e - 1 + (int)c) << 52) + m + up));
  }
  return a * b;
}

// a / b: Q = floor(N / d) for N = m_a 2^(63 + s), d = m_b 2^11 (s = 1 when
// m_a < m_b, so that Q has 53 bits).  The reciprocal v ~ 2^128 / d - 2^64
// is seeded from the float reciprocal of d's top 24 bits (~22 bits) and
// refined by two Newton-Raphson steps in fixed point, R' = R + R (2^128 -
// d R) / 2^128 with R = 2^64 + v (quadratic convergence: ~44, then ~64
// bits; Newton division as in Knuth, TAOCP vol. 2, 4.3.3, and Brent and
// Zimmermann, Modern Computer Arithmetic, 3.4).  The quotient estimate
// floor(N R / 2^128) is then corrected by one step either way from the
// exact remainder N - Q d, and rounded by comparing twice the remainder
// with d (ties to even).  If the remainder still lies outside [0, d), the
// FP64 division is used.
// The fixed-point reciprocal of a normalised divisor d in [2^63, 2^64):
// v ~ 2^128 / d - 2^64 (so R = 2^64 + v), seeded by the float reciprocal
// of d's top 24 bits and refined by two Newton steps.
__device__ __forceinline__ unsigned long long recip_fixed(unsigned long long d) {
  // the float of d's top 24 bits, from its bits (2^23 <= d >> 40 < 2^24)
  const float f = __uint_as_float(0x4B000000u | ((unsigned)(d >> 40) & 0x7FFFFFu));
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
  const unsigned yb = __float_as_uint(y);
  // 2^88 y - 2^64 for y in [2^-24, 2^-23); y = 2^-23 (d = 2^63) saturates
  unsigned long long v =
      ((yb >> 23) & 0xFFu) == 103u ? (unsigned long long)(yb & 0x7FFFFFu) << 41 : ~0ull;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    // d R - 2^128 = T 2^64 + pl (T signed, small); E = floor((2^128 - d R) / 2^64)
    const unsigned long long pl = d * v, ph = __umul64hi(d, v);
    const long long T = (long long)(ph + d);
    const long long E = -T - (pl != 0ull ? 1 : 0);
    const unsigned long long aE = E < 0 ? (unsigned long long)(-E) : (unsigned long long)E;
    const unsigned long long c = __umul64hi(v, aE);  // v |E| / 2^64
    v = E < 0 ? v + (unsigned long long)E - c : v + (unsigned long long)E + c;
  }
  return v;
}

// a / b from the reciprocal v of d = m_b 2^11 (b normal): false where the
// quotient needs the FP64 division (a not normal, a result out of the
// normal range, or a remainder still out of range after the correction).
__device__ __forceinline__ bool div_by_recip(unsigned long long ua, unsigned long long vb,
                                             unsigned long long d, unsigned long long v,
                                             double& out) {
  const unsigned ea = (unsigned)(ua >> 52) & 0x7FFu, eb = (unsigned)(vb >> 52) & 0x7FFu;
  const unsigned long long ma = significand(ua), mb = significand(vb);
  const unsigned s = ma < mb ? 1u : 0u;
  const int e = (int)ea - (int)eb + 1023 - (int)s;
  if (!(ea - 1u < 2046u && (unsigned)(e - 1) < 2045u)) return false;
  // N = u1 2^64 + u0
  const unsigned long long u1 = s ? ma : ma >> 1, u0 = s ? 0ull : (ma & 1ull) << 63;
  const unsigned long long ql = v * u1, qh = __umul64hi(v, u1);
  const unsigned long long q0 = ql + u0;
  unsigned long long Q = qh + u1 + (q0 < ql ? 1ull : 0ull);
  // remainder N - Q d as rh 2^64 + rl (rh signed)
  const unsigned long long pl = Q * d, ph = __umul64hi(Q, d);
  unsigned long long rl = u0 - pl;
  long long rh = (long long)(u1 - ph - (u0 < pl ? 1ull : 0ull));
  if (rh < 0) {
    const unsigned long long t = rl + d;
    rh += t < rl ? 1 : 0;
    rl = t;
    --Q;
  } else if (rh > 0 || rl >= d) {
    const unsigned long long t = rl - d;
    rh -= rl < d ? 1 : 0;
    rl = t;
    ++Q;
  }
  if (rh == 0 && rl < d) {
    const unsigned long long r2 = rl << 1;
    const bool up = (rl >> 63) != 0ull || r2 > d || (r2 == d && (Q & 1ull));
    out = __longlong_as_double((long long)(((ua ^ vb) & kSignBit) +
                                           ((unsigned long long)(e - 1) << 52) + Q +
                                           (up ? 1ull : 0ull)));
    return true;
  }
  return false;
}

__device__ __forceinline__ double div_rn(double a, double b) {
  const unsigned long long ua = ubits(a), vb = ubits(b);
  const unsigned eb = (unsigned)(vb >> 52) & 0x7FFu;
  if (eb - 1u < 2046u) {
    const unsigned long long d = significand(vb) << 11;  // [2^63, 2^64)
    double q;
    if (div_by_recip(ua, vb, d, recip_fixed(d), q)) return q;
  }
  return a / b;
}

// sqrt(x): Q = floor(sqrt(N)) for N = m_x 2^(52 + p), p = 1 when x's
// unbiased exponent is even (so that Q has 53 bits).  The reciprocal square
// root Y ~ 2^94 / sqrt(w) of w = m_x 2^(10 + p) in [2^62, 2^64) is seeded
// from the float reciprocal square root of w's top 24 bits and refined by
// two Newton steps Y' = Y (3 - w Y^2 / 2^188) / 2 in fixed point (Brent and
// Zimmermann, Modern Computer Arithmetic, 3.5); Q ~ N Y / 2^115 is then
// corrected by one step either way from the exact remainder N - Q^2 in [0,
// 2Q], and rounded up when the remainder exceeds Q (sqrt(N) >= Q + 1/2; an
// exact tie cannot occur).  Negative, zero, subnormal and non-finite x:
// the FP64 square root.
__device__ __forceinline__ double sqrt_rn(double x) {
  const unsigned long long ux = ubits(x);
  const unsigned ex = (unsigned)(ux >> 52);  // sign included: negative x falls back
  if (ex - 1u < 2046u) {
    const unsigned long long ma = significand(ux);
    const unsigned p = (ex & 1u) ^ 1u;
    const unsigned long long w = ma << (10 + p);
    // the float of w / 2^40, from its bits (2^22 <= w / 2^40 < 2^24)
    const float f = p ? __uint_as_float(0x4B000000u | ((unsigned)(w >> 40) & 0x7FFFFFu))
                      : __uint_as_float(0x4A800000u | ((unsigned)(w >> 39) & 0x7FFFFFu));
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
    const unsigned yb = __float_as_uint(y);
    const int ye = (int)((yb >> 23) & 0xFFu) - 127;  // y in [2^ye, 2^(ye + 1)), ye in {-12, -11}
    unsigned long long Y = (unsigned long long)((yb & 0x7FFFFFu) | 0x800000u) << (51 + ye);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      // E = floor((2^124 - w sh) / 2^64), sh = Y^2 / 2^64; Y' = Y + Y E / 2^61
      const unsigned long long sh = __umul64hi(Y, Y);
      const unsigned long long ml = w * sh, mh = __umul64hi(w, sh);
      const long long E = (long long)((1ull << 60) - mh) - (ml != 0ull ? 1 : 0);
      const unsigned long long aE = E < 0 ? (unsigned long long)(-E) : (unsigned long long)E;
      const unsigned long long h = __umul64hi(Y, aE), l = Y * aE;
      const unsigned long long c = (h << 3) | (l >> 61);
      Y = E < 0 ? Y - c : Y + c;
    }
    const unsigned long long lo = ma * Y, hi = __umul64hi(ma, Y);
    unsigned long long Q = p ? (hi << 2) | (lo >> 62) : (hi << 1) | (lo >> 63);
    // remainder N - Q^2 as rh 2^64 + rl (rh signed), N = u1 2^64 + u0
    const unsigned long long u1 = ma >> (12 - p), u0 = ma << (52 + p);
    const unsigned long long ql = Q * Q, qh = __umul64hi(Q, Q);
    unsigned long long rl = u0 - ql;
    long long rh = (long long)(u1 - qh - (u0 < ql ? 1ull : 0ull));
    if (rh < 0) {  // (Q - 1)^2 = Q^2 - (2Q - 1)
      const unsigned long long t = 2 * Q - 1, n = rl + t;
      rh += n < rl ? 1 : 0;
      rl = n;
      --Q;
    } else if (rh > 0 || rl > 2 * Q) {  // (Q + 1)^2 = Q^2 + 2Q + 1
      const unsigned long long t = 2 * Q + 1, n = rl - t;
      rh -= rl < t ? 1 : 0;
      rl = n;
      ++Q;
    }
    if (rh == 0 && rl <= 2 * Q) {
      const int er = ((int)ex - 1127 - (int)p) / 2 + 1075;
      return __longlong_as_double(
          (long long)(((unsigned long long)(er - 1) << 52) + Q + (rl > Q ? 1ull : 0ull)));
    }
  }
  return sqrt(x);
}

// ------------------------------------------------- counter-based RNG
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 bit products and xors, keys bumped by the Weyl constants.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint64_t seed) {
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// (2k + 1) 2^-53 from the top 52 bits k of (hi:lo): exact, inside (0, 1)
__device__ __forceinline__ double u01(uint32_t lo, uint32_t hi) {
  // (2k + 1) 2^-53 is exact: its bits are assembled with integer operations
  // (leading-zero count, shift, exponent) instead of an int -> double
  // conversion and a multiply on the FP64 pipe
  const uint64_t k = ((((uint64_t)hi) << 32) | lo) >> 12;
  const uint64_t mo = 2ull * k + 1ull;  // odd, < 2^53
  const int lz = __clzll((long long)mo) - 11;
  const uint64_t mm = mo << lz;  // top bit at 52
  return __longlong_as_double(
      (long long)(((uint64_t)(1022 - lz) << 52) | (mm & 0x000FFFFFFFFFFFFFull)));
}

// 2 X - 1 for X = u01(lo, hi) equals U 2^-52 exactly, U = 2k + 1 - 2^52 (odd,
// |U| < 2^52); sym_int gives U, sym_double the double
__device__ __forceinline__ int64_t sym_int(uint32_t lo, uint32_t hi) {
  const uint64_t k = ((((uint64_t)hi) << 32) | lo) >> 12;
  return (int64_t)(2ull * k + 1ull) - (int64_t)(1ull << 52);
}
__device__ __forceinline__ double sym_double(int64_t U) {
  const uint64_t a = U < 0 ? (uint64_t)(-U) : (uint64_t)U;
  const int lz = __clzll((long long)a) - 11;
  const uint64_t aa = a << lz;
  return __longlong_as_double((long long)((U < 0 ? 0x8000000000000000ull : 0ull) |
                                          ((uint64_t)(1023 - lz) << 52) |
                                          (aa & 0x000FFFFFFFFFFFFFull)));
}

// ------------------------------------------- combined Tausworthe streams
// The paper's generator as an option (section 3.6; L'Ecuyer 1999): four
// LFSR words with (k, q, s) = (31, 6, 18), (29, 2, 2), (28, 13, 7),
// (25, 3, 13); a step of a word z is b = ((z << q) ^ z) >> (k - s),
// z = ((z & m_k) << s) ^ b (m_k clears the low 32 - k bits); the output is
// the xor of the four words.
template <int k, int q, int s>
__device__ __forceinline__ uint32_t taus_word(uint32_t z) {
  const uint32_t b = ((z << q) ^ z) >> (k - s);
  return ((z & (0xFFFFFFFFu << (32 - k))) << s) ^ b;
}
__device__ __forceinline__ uint32_t taus_next(uint4& z) {
  z.x = taus_word<31, 6, 18>(z.x);
  z.y = taus_word<29, 2, 2>(z.y);
  z.z = taus_word<28, 13, 7>(z.z);
  z.w = taus_word<25, 3, 13>(z.w);
  return z.x ^ z.y ^ z.z ^ z.w;
}

// A star's random blocks of four words.  Counter mode (kTaus false):
// Philox4x32-10 at (id, step, tag, trial).  Stream mode: the next four
// outputs of the star's own stream; the method asks for each star's blocks
// in a fixed order (relaxation trials, orbit trials, the v_r sign), so the
// tag and the trial are implied by the order.
template <bool kTaus>
struct Draws {
  uint64_t seed;
  uint32_t id, step;
  uint4 z;
  __device__ __forceinline__ U4 block(uint32_t tag, uint32_t t) {
    if (!kTaus) return philox(id, step, tag, t, seed);
    U4 w;
    w.x = taus_next(z);
    w.y = taus_next(z);
    w.z = taus_next(z);
    w.w = taus_next(z);
    return w;
  }
  // pass over n blocks (stream mode)
  __device__ __forceinline__ void skip(uint32_t n) {
    if (kTaus)
      for (uint32_t i = 0; i < 4u * n; ++i) taus_next(z);
  }
};

template <bool kTaus>
__device__ __forceinline__ Draws<kTaus> draws_of(const Seg& S, int c, uint32_t id,
                                                 uint32_t step) {
  Draws<kTaus> d;
  d.seed = S.seed[c];
  d.id = id;
  d.step = step;
  if (kTaus) d.z = S.taus[__ldg(S.taus_base + c) + id];
  return d;
}

template <bool kTaus>
__device__ __forceinline__ void draws_keep(const Seg& S, int c, const Draws<kTaus>& d) {
  if (kTaus) S.taus[__ldg(S.taus_base + c) + d.id] = d.z;
}

// Non-inlined copies of div_rn and sqrt_rn for kernels with many call
// sites: each inlined copy is ~150 instructions, and a kernel holding a
// dozen of them no longer fits the instruction cache (ncu: instruction
// fetch the relaxation kernel's largest stall); one shared body costs a
// call per use instead (measured: relaxation 1.46 -> 1.06 ms at N = 1e7).
static __device__ __noinline__ double div_rn_nl(double a, double b) { return div_rn(a, b); }
static __device__ __noinline__ double sqrt_rn_nl(double x) { return sqrt_rn(x); }

// uniform planar direction (cos a, sin a) by rejection of a point in the
// unit disk; the doubled angle gives cos = (u^2 - v^2)/q, sin = 2uv/q.
//
// The draw (u, v) = (U, V) 2^-52 is accepted when the FP64 value of
// u u + v v is <= 1.  That value is within 2^-51 of the exact sum (both
// below 2), so outside a band of 2^54 around 2^104 the exact integer test
// U^2 + V^2 <= 2^104 (128-bit) gives the same answer; inside the band the
// FP64 expression decides.  The loop is integer work only; the FP64
// arithmetic of the accepted draw runs once, after it.  Not inlined: one
// copy serves both of the relaxation's angles (code size, as for div_rn_nl).
template <bool kTaus>
__device__ __noinline__ bool disk_angle(Draws<kTaus>& g, uint32_t tag, double& c, double& s) {
  int64_t Ua = 0, Va = 0;
  bool ok = false;
  for (uint32_t t = 0; t < 64u; ++t) {
    U4 w = g.block(tag, t);
    const int64_t U = sym_int(w.x, w.y), V = sym_int(w.z, w.w);
    const uint64_t A = U < 0 ? (uint64_t)(-U) : (uint64_t)U;
    const uint64_t B = V < 0 ? (uint64_t)(-V) : (uint64_t)V;
    const uint64_t l1 = A * A, l2 = B * B;
    const uint64_t lo = l1 + l2;
    const uint64_t hi = __umul64hi(A, A) + __umul64hi(B, B) + (lo < l1 ? 1ull : 0ull);
    // S = hi 2^64 + lo against 2^104 -+ 2^54
    const uint64_t H = 1ull << 40, band = 1ull << 54;
    bool in = hi < H - 1 || (hi == H - 1 && lo <= 0ull - band);
    const bool out = hi > H || (hi == H && lo >= band);
    if (!in && !out) {
      const double u = sym_double(U), v = sym_double(V);
      const double uu = u * u, vv = v * v;
      in = uu + vv <= 1.0;
    }
    if (in) {
      Ua = U;
      Va = V;
      ok = true;
      break;
    }
  }
  if (!ok) {
    c = 1.0;
    s = 0.0;
    return false;
  }
  const double u = sym_double(Ua), v = sym_double(Va);
  const double uu = u * u, vv = v * v, q = uu + vv;
  c = div_rn_nl(uu - vv, q);
  s = div_rn_nl(scale_up<1>(u) * v, q);
  return true;
}

// ------------------------------------------------------------ sort keys
__device__ __forceinline__ uint64_t radius_key(double r, uint32_t id) {
  uint64_t b = (uint64_t)__double_as_longlong(r);
  return (b >= 0x7FF0000000000000ull) ? kEscKeyBase | ((uint64_t)id << 20) : b;
}
__device__ __forceinline__ bool key_is_escaper(uint64_t k) {
  return k >= 0x7FF0000000000000ull;
}

// --------------------------------------------- shell potential (Eq. 6)
// Table of one segment: sorted radii r[0..nb), x = 1/r, Phi.  Node nb is
// the virtual star at 1/r = 0 with Phi = 0 (Eq. 2); inside r[0] Phi is
// the constant Phi_0 (Eq. 1 with nothing enclosed).
struct Table64 {
  const double* r;
  const double* x;
  const double* phi;
  int64_t nb;
};

// Radii are positive, and positive doubles order like their 64-bit
// patterns read as signed integers: comparing the patterns gives the same
// answer as the floating-point comparison without using the FP64 pipe.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }

// largest i in [0, nb) with r[i] <= q, else -1 (unique for sorted r)
__device__ __forceinline__ int64_t shell_of(const Table64& t, double q) {
  if (!(q >= 0.0)) return -1;  // (NaN: no radius compares <= it)
  const long long qb = dbits(q);
  const long long* rb = reinterpret_cast<const long long*>(t.r);
  int64_t lo = -1, hi = t.nb;
  while (hi - lo > 1) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(rb + mid) <= qb) lo = mid; else hi = mid;
  }
  return lo;
}

// Eq. 6 inside shell i (i = -1: central constant)
__device__ __forceinline__ double phi_in_shell(const Table64& t, int64_t i, double q) {
  if (i < 0) return __ldg(t.phi);
  double x = div_rn(1.0, q);
  double xj = __ldg(t.x + i), pj = __ldg(t.phi + i), xj1, pj1;
  if (i + 1 < t.nb) { xj1 = __ldg(t.x + i + 1); pj1 = __ldg(t.phi + i + 1); }
  else { xj1 = 0.0; pj1 = 0.0; }
  double den = xj - xj1;
  if (!(den > 0.0)) return pj;
  return pj + div_rn(xj - x, den) * (pj1 - pj);
}

__device__ __forceinline__ double phi_of_r(const Table64& t, double q) {
  return phi_in_shell(t, shell_of(t, q), q);
}

// Cube root by Newton's method, y <- y - (y^3 - v) / (3 y^2), eight steps
// from 2^floor(e/3) (e the binary exponent of v): the merged radius of two
// sticky spheres; the same operations in the same order as the FP64
// statement of the method, so the same bits; 0 for v <= 0.
__device__ __forceinline__ double cbrt_newton(double v) {
  if (!(v > 0.0)) return 0.0;
  const int e = (int)((ubits(v) >> 52) & 0x7FFu) - 1023;
  const int k = e >= 0 ? e / 3 : -((-e + 2) / 3);  // floor(e / 3)
  double y = __longlong_as_double((long long)((unsigned long long)(k + 1023) << 52));
#pragma unroll 1
  for (int i = 0; i < 8; ++i) y = y - (y * y * y - v) / (3.0 * (y * y));
  return y;
}

// ----------------------------------------------------- small utilities
__device__ __forceinline__ void set_err(uint32_t* err, uint32_t bit) {
  atomicOr(err, bit);
}

__device__ __forceinline__ void stat_add(unsigned long long* st, int seg, int which,
                                         unsigned long long v) {
  if (v) atomicAdd(st + (size_t)seg * kStStride + which, v);
}

// The energy a clamp of T' < 0 to 0 adds, m |T'|, into the segment's
// counter as a fixed-point integer in units of 2^-62 (integer sums do not
// depend on their order).
__device__ __forceinline__ void clamp_energy_add(unsigned long long* st, int seg, double m,
                                                double Tp) {
  const double e = -(m * Tp) * 4611686018427387904.0;  // 2^62
  if (e > 0.0) stat_add(st, seg, kStClampEnergy, __double2ull_rn(e));
}

// ------------------------------------------- the orbit step's index tables
// Both are written star by star, in one pass over the sorted stars (by the
// potential kernel, or by stand-alone kernels for a given potential).
// Bucket index of a segment (prm: shift, bucket count, first and last
// indexed node; base: float key bits of 1/r at the first indexed node):
// star k writes start[b] = k for the buckets from its predecessor's bucket
// (exclusive) to its own; the last indexed star closes the table with nb.
// key_k, key_km1: float bits of 1/r of stars k and k - 1.
__device__ __forceinline__ void bucket_starts_of(int64_t k, int64_t nb, int4 prm, uint32_t base,
                                                 uint32_t key_k, uint32_t key_km1, int* st,
                                                 int64_t cap) {
  if (k < prm.z || k > prm.w) return;
  const int sh = prm.x, nbk = prm.y;
  const long long bk = (long long)((base - key_k) >> sh);
  const long long bp = k == prm.z ? -1ll : (long long)((base - key_km1) >> sh);
  for (long long b = bp + 1; b <= bk && b < nbk; ++b)
    if (CMC_IN(b, cap)) st[b] = (int)k;
  if (k == prm.w)
    for (long long b = bk + 1; b <= nbk; ++b) st[b] = (int)nb;
}

// The potential grid's key shells (pr: key0, sh, cells): star k owns the
// keys in (1/r_{k+1}, 1/r_k], i.e. the cells from gmax(k + 1) + 1 to
// gmax(k), gmax(k) = the last cell whose key is <= 1/r_k.  A key (a
// positive float) is <= 1/r_k exactly when its bits are <= those of 1/r_k
// rounded down to a float.  The outermost star also owns the cells below
// it, the innermost one the cells above it (shell -1).
__device__ __forceinline__ int64_t grid_last_cell(double xk, int4 pr) {
  const uint32_t kb = __float_as_uint(__double2float_rd(xk));
  if (kb < (uint32_t)pr.x) return -1;
  const int64_t g = (int64_t)((kb - (uint32_t)pr.x) >> pr.y);
  return g < pr.z - 1 ? g : (int64_t)pr.z - 1;
}

__device__ __forceinline__ void grid_shells_of(int64_t k, int64_t nb, double xk, double xk1,
                                               int4 pr, int* sh) {
  if (pr.z <= 0) return;
  const int64_t hi = grid_last_cell(xk, pr);
  const int64_t lo = k + 1 < nb ? grid_last_cell(xk1, pr) + 1 : 0;
  for (int64_t g = lo; g <= hi; ++g)
    if (CMC_IN(g, pr.z)) sh[g] = (int)k;
  if (k == 0)
    for (int64_t g = hi + 1; g < pr.z; ++g) sh[g] = -1;
}

}  // namespace cmc
