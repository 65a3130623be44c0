// New orbits (section 2.1 step 5, Eqs. 12-15; Appendix A's bisection and
// rejection kernels, fused): one thread per star.
//
//   E = Phi_k + (v_r^2 + v_t^2)/2,  J = r_k v_t;  E >= 0: the star escapes.
//   r_max, r_min: bisection over the star nodes for the sign change of
//   Q(r) = 2E - 2 Phi(r) - J^2/r^2 (Eq. 12), then the root of Q inside the
//   shell, where Eq. 6 makes Phi = A - B/r.
//   New radius: von Neumann rejection (Eqs. 14-15) in the variable s of
//   r(s) = (rmax+rmin)/2 + (rmax-rmin)/4 (3s - s^3), whose density
//   g(s) = (dr/ds)/sqrt(Q) stays finite at both turning points; the bound
//   is F = 1.2 max_j g(s_j) on s_j = -1 + (j + 1/2)/10.5, j = 0..20.
//   v_t = J/r_new, v_r = +-sqrt(Q(r_new)).
//
// precision 0 (FP64): every operation is the FP64 operation of the
// method's statement, in the same order, so results are bit-identical to
// it.  precision 1 (mixed): the bisections, the bound F and the accept
// tests run in FP32 on an interleaved float2 (1/r, Phi) table, the F
// samples and trials located through a radius-bucket index; the brackets
// are then verified (and moved if needed) in FP64, the turning points are
// the FP64 shell roots with the shell slope taken from the enclosed mass,
// and the accepted radius, its potential and the velocities are
// recomputed in FP64.  A mixed result matches the FP64 result to rounding
// whenever both accept the same trial.
#include "cmc_host.hpp"

namespace cmc {

namespace {

struct Star {
  double E, J;
  int64_t k;
};

// Q = 2 (E - Phi) - (J x)^2 from node values, as Q_node64 evaluates it
__device__ __forceinline__ double Qv(const Star& s, double x, double p) {
  const double L = s.J * x;
  return 2.0 * (s.E - p) - L * L;
}

__device__ __forceinline__ double Q_node64(const Table64& T, const Star& s, int64_t i) {
  double L = s.J * __ldg(T.x + i);
  return scale_up<1>(s.E - __ldg(T.phi + i)) - L * L;
}

// root of Q inside shell j (nodes j, j+1; node nb is 1/r = 0, Phi = 0)
__device__ __forceinline__ double shell_root64(const Table64& T, const Star& s, int64_t j,
                                               bool outer) {
  const double rj = __ldg(T.r + j), xj = __ldg(T.x + j), pj = __ldg(T.phi + j);
  double rj1, xj1, pj1;
  const bool has_next = j + 1 < T.nb;
  if (has_next) { rj1 = __ldg(T.r + j + 1); xj1 = __ldg(T.x + j + 1); pj1 = __ldg(T.phi + j + 1); }
  else { rj1 = __longlong_as_double(0x7FF0000000000000ll); xj1 = 0.0; pj1 = 0.0; }
  if (!(xj - xj1 > 0.0)) return rj;
  const double B = div_rn(pj1 - pj, xj - xj1);
  const double A = pj + B * xj;
  double D = B * B + scale_up<1>(s.J * s.J) * (s.E - A);
  if (!(D > 0.0)) D = 0.0;
  const double sD = sqrt_rn(D);
  double root = outer ? div_rn(B + sD, scale_up<1>(A - s.E)) : div_rn(s.J * s.J, B + sD);
  if (!(root >= rj)) root = rj;
  if (has_next && root > rj1) root = rj1;
  return root;
}

// The same root with the slope of shell j taken from the enclosed mass:
// across shell j, (Phi_{j+1} - Phi_j)/(x_j - x_{j+1}) = G M_j exactly
// (Eqs. 1-5; for the outermost shell M_j is the bound mass), so
// Phi = Phi_j + M_j (x_j - x) needs no division (mixed mode).  The cores
// take the node values, so that values loaded ahead and the table give
// the same arithmetic.  The clamps are the FP64 comparisons restated on
// the bit patterns (radii are positive).  Their quotients go to the integer
// pipes through the shared body and their square roots stay on the FP64
// pipe: that balance measured fastest in this FP64-bound kernel (turning
// points 1.39 -> 1.36 ms at N = 10^7; both on the integer pipes, inlined or
// shared, 0.04-0.05 ms slower).
__device__ __forceinline__ double rmax_core(const Star& s, double rj, double xj, double pj,
                                            double Mj, bool has_next, double rj1) {
  const double B = Mj;
  const double A = pj + B * xj;
  const double em = s.E - A;
  double D = B * B + scale_up<1>(s.J * s.J) * em;
  if (!pos_num(D)) D = 0.0;
  const double sD = sqrt(D);
  // 2 (A - E) = -(2 (E - A)) exactly
  double root = div_rn_nl(B + sD, -scale_up<1>(em));
  if (!ge_pos(root, rj)) root = rj;
  if (has_next && ubits(root) > ubits(rj1)) root = rj1;
  return root;
}

// r_min in mixed mode: the shell root, or inside the innermost node
// (central, where Phi = Phi_0) J / sqrt(2 (E - Phi_0)) as central_root64
// computes it; both take one square root and one division, so the two
// cases share them (B = 0 makes B + sqrt(D) the bare root) and a warp
// holding both kinds of star runs them once.  Central: node values of
// node 0 and rj = r_0.
__device__ __forceinline__ double rmin_core(const Star& s, bool central, double rj, double xj,
                                            double pj, double Mj, bool has_next, double rj1) {
  const double B = central ? 0.0 : Mj;
  double D, num;
  if (central) {
    D = scale_up<1>(s.E - pj);
    num = s.J;
  } else {
    const double A = pj + B * xj;
    D = B * B + scale_up<1>(s.J * s.J) * (s.E - A);
    if (!pos_num(D)) D = 0.0;
    num = s.J * s.J;
  }
  double root = div_rn_nl(num, B + sqrt(D));
  if (central) {
    // root >= 0 (-0 included, NaN not), then root <= r_0
    const unsigned long long u = ubits(root);
    if (!(u <= kInfBits || u == 0x8000000000000000ull)) root = 0.0;
    if (__double_as_longlong(root) > __double_as_longlong(rj)) root = rj;
  } else {
    if (!ge_pos(root, rj)) root = rj;
    if (has_next && ubits(root) > ubits(rj1)) root = rj1;
  }
  return root;
}

// The FP64 shell of q (largest i with r_i <= q, -1 if none; integer
// compares of the radii's bits) from a guess i by a bounded walk, then a
// bisection, on the node records; a receives that shell's record (node 0's
// for -1).  The records of the guess and its successor are loaded together.
__device__ __forceinline__ int64_t fix_shell_nodes(const double4_32a* __restrict__ nd, int64_t nb,
                                                   int64_t i, double q, double4_32a& a) {
  if (!ge0(q)) {
    a = nd[0];
    return -1;
  }
  if (i < -1) i = -1;
  if (i >= nb) i = nb - 1;
  const long long qb = dbits(q);
  if (!CMC_IN(i < 0 ? 0 : i, nb)) i = -1;
  a = nd[i < 0 ? 0 : i];
  double4_32a b = i + 1 < nb ? nd[i + 1] : a;
  for (int w = 0; w < 64; ++w) {
    if (i + 1 < nb && dbits(b.x) <= qb) {
      ++i;
      a = b;
      if (i + 1 < nb) b = nd[i + 1];
      continue;
    }
    if (i >= 0 && dbits(a.x) > qb) {
      --i;
      b = a;
      a = nd[i < 0 ? 0 : i];
      continue;
    }
    return i;
  }
  int64_t lo = -1, hi = nb;
  while (hi - lo > 1) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (dbits(nd[mid].x) <= qb) lo = mid; else hi = mid;
  }
  a = nd[lo < 0 ? 0 : lo];
  return lo;
}

__device__ __forceinline__ double central_root64(const Table64& T, const Star& s) {
  double rmin = div_rn(s.J, sqrt_rn(scale_up<1>(s.E - __ldg(T.phi))));
  if (!(rmin >= 0.0)) rmin = 0.0;
  const double r0 = __ldg(T.r);
  if (rmin > r0) rmin = r0;
  return rmin;
}

__device__ __forceinline__ int64_t bisect_rmax64(const Table64& T, const Star& s) {
  int64_t lo = s.k, hi = T.nb;
  while (hi - lo > 1) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (Q_node64(T, s, mid) < 0.0) hi = mid; else lo = mid;
  }
  return lo;
}

__device__ __forceinline__ int64_t bisect_rmin64(const Table64& T, const Star& s) {
  int64_t lo = -1, hi = s.k;
  while (hi - lo > 1) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (Q_node64(T, s, mid) < 0.0) lo = mid; else hi = mid;
  }
  return lo;
}

// g(s) with Phi from the FP64 table
__device__ __forceinline__ double g64(const Table64& T, const Star& st, double c0, double c1,
                                      double s, double& rs, double& ph, double& Q) {
  rs = c0 + c1 * (s * (3.0 - s * s));
  const double drds = (3.0 * c1) * (1.0 - s * s);
  ph = phi_of_r(T, rs);
  const double L = div_rn(st.J, rs);
  Q = scale_up<1>(st.E - ph) - L * L;
  if (!(Q > 0.0)) return 0.0;
  return div_rn(drds, sqrt_rn(Q));
}

// ------------------------------------------------------------ FP32 side
// sample points of the bound F: s_j = -1 + (j + 1/2)/10.5 (IEEE double,
// evaluated at compile time), and their float roundings
#define CMC_SJ(j) (-1.0 + ((double)(j) + 0.5) / 10.5)
#define CMC_SJ21(f) f(0), f(1), f(2), f(3), f(4), f(5), f(6), f(7), f(8), f(9), f(10), \
    f(11), f(12), f(13), f(14), f(15), f(16), f(17), f(18), f(19), f(20)
__constant__ double c_s64[21] = {CMC_SJ21(CMC_SJ)};
// for the FP32 envelope: s_j (3 - s_j^2) and 3 (1 - s_j^2), rounded to float
#define CMC_SJA(j) ((float)(CMC_SJ(j) * (3.0 - CMC_SJ(j) * CMC_SJ(j))))
#define CMC_SJB(j) ((float)(3.0 * (1.0 - CMC_SJ(j) * CMC_SJ(j))))
__constant__ float c_sa32[21] = {CMC_SJ21(CMC_SJA)};
__constant__ float c_sb32[21] = {CMC_SJ21(CMC_SJB)};

// ---- FP32 searches run in lockstep: K independent searches per thread,
// each round issues K independent loads before any of them is needed.
__device__ __forceinline__ int search_rounds(int nb) { return 32 - __clz(nb); }

// Radius-bucket index of one segment's float table.  It covers the nodes
// lo..hi, all but the sparse 1/1024 at each end (where a bucket resolution
// fine enough for the core would leave long runs of empty buckets).
// Bucket of a key x > 0: (base - bits(x)) >> shift, base = bits(x_lo).
// Positive floats order like their bit patterns, so buckets are
// non-decreasing along the (non-increasing) keys.  start[b] is the first
// node whose bucket is >= b, start[nbk] = nb.  A node before start[b] has a
// key above any query of bucket b, a node from start[b+1] on (within lo..hi)
// a key below it, so the answer of a query of bucket b lies in
// [start[b] - 1, start[b+1] - 1]; queries above x_lo search [-1, lo),
// queries below x_hi search [hi, nb).
struct Buckets {
  const int* start;
  uint32_t base;
  int shift, nbk, lo, hi;
};

// largest i with x_i >= xq[q], else -1, for K queries (lockstep).
// The bucket of a query gives the bracket (start[b] - 1, start[b+1]); the
// keys inside one bucket are close to uniform, so the query's position in
// its bucket predicts the shell.  Each round loads 4 nodes per unfinished
// query at once: the first round around the prediction, later rounds
// evenly over the bracket (a bucket of up to 16 nodes takes at most 2
// rounds, a prediction that is right 1).  Queries in the tails outside the
// index search their tail the same way.  Any probe keeps the bracket
// valid (x falls with i), so the answer is the unique one of a bisection.
//
// The keys probed are those of a table adaptor: the float keys (1/r as a
// float, the high part of a float pair: FloatKeys) or the FP64 1/r of the
// node records compared on their bit patterns (NodeKeys; positive doubles
// order like their patterns).  Probing the table that the caller reads next
// (the float pairs of the bracket walks, the node record of the shell)
// brings its lines into the cache with the search.
struct FloatKeys {
  const float* p;  // key i at p[i * stride]
  int stride;
  using V = float;
  __device__ __forceinline__ V load(int i) const { return __ldg(p + (size_t)i * stride); }
  __device__ __forceinline__ V key(float q) const { return q; }
};
struct NodeKeys {
  const double4_32a* nd;
  using V = long long;
  __device__ __forceinline__ V load(int i) const { return dbits(nd[i].y); }
  // the query widened to FP64 exactly, as bits (queries are positive, finite)
  __device__ __forceinline__ V key(float q) const { return dbits((double)q); }
};

template <int K, class Tab>
__device__ __forceinline__ void shells32_bk(const Tab& tab, int nb, const Buckets& B,
                                            const float (&xq)[K], int (&out)[K]) {
  typename Tab::V kq[K];
#pragma unroll
  for (int q = 0; q < K; ++q) kq[q] = tab.key(xq[q]);
  int lo[K], hi[K], pred[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    pred[q] = -2;  // no prediction
    const long long d = (long long)B.base - (long long)__float_as_uint(xq[q]);
    if (d < 0) { lo[q] = -1; hi[q] = B.lo; continue; }           // inner tail
    const long long b = d >> B.shift;
    if (b >= B.nbk) { lo[q] = B.hi; hi[q] = nb; continue; }      // outer tail
    if (!CMC_IN(b + 1, B.nbk + 1)) { lo[q] = -1; hi[q] = nb; continue; }
    const int s0 = __ldg(B.start + b), s1 = __ldg(B.start + b + 1);
    lo[q] = s0 - 1;
    hi[q] = s1;
    const int frac = (int)(d & ((1ll << B.shift) - 1));
    pred[q] = s0 - 1 + (int)(((long long)(s1 - s0) * frac + (1ll << (B.shift - 1 > 0 ? B.shift - 1 : 0))) >> B.shift);
  }
  bool more = true;
  while (more) {
    more = false;
    int m[K][4];
    typename Tab::V v[K][4];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int c = hi[q] - lo[q] - 1;  // candidates lo+1 .. hi-1
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int mj;
        if (pred[q] >= -1) mj = pred[q] - 1 + j;
        else mj = lo[q] + 1 + (int)(((long long)(c > 0 ? c - 1 : 0) * j) / 3);
        mj = mj < lo[q] + 1 ? lo[q] + 1 : mj;
        mj = mj > hi[q] - 1 ? hi[q] - 1 : mj;
        m[q][j] = mj;
        v[q][j] = c > 0 && CMC_IN(mj, nb) ? tab.load(mj) : typename Tab::V(0);
      }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      if (hi[q] - lo[q] > 1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (v[q][j] >= kq[q]) lo[q] = m[q][j] > lo[q] ? m[q][j] : lo[q];
          else hi[q] = m[q][j] < hi[q] ? m[q][j] : hi[q];
        }
        pred[q] = -2;
        more |= hi[q] - lo[q] > 1;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = lo[q];
}

// The potential grid of one segment (see BucketArgs): Phi (float) at the
// float keys key0 + g 2^sh of 1/r.  Inside a binade a float's key is linear
// in its value, so on a binade-aligned grid Phi, linear in 1/r between
// stars, is interpolated linearly in the key up to the kinks of the stars
// inside one cell (relative error ~2e-7 at 1024 cells per binade).
struct Grid {
  const float* phi;
  uint32_t key0, kmax;
  int sh, cells;
  float phi0, mb, x0, err;  // err: relative bound on the interpolation error
};

__device__ __forceinline__ Grid grid_of(const BucketArgs& B, int c) {
  Grid G;
  const int4 pr = B.gprm[c];
  const float4 au = B.gaux[c];
  G.phi = B.gphi + B.goff[c];
  G.key0 = (uint32_t)pr.x;
  G.sh = pr.y;
  G.cells = pr.z;
  G.kmax = (uint32_t)pr.w;
  G.phi0 = au.x;
  G.mb = au.y;
  G.x0 = au.z;
  G.err = au.w;
  return G;
}

__device__ __forceinline__ float grid_phi(const Grid& G, float xq) {
  const uint32_t key = __float_as_uint(xq);
  if (key >= G.kmax) return G.phi0;                               // inside the first star
  if (key < G.key0) return __ldg(G.phi) + G.mb * (G.x0 - xq);     // beyond the last
  const uint32_t d = key - G.key0;
  const int g = (int)(d >> G.sh);
  if (!CMC_IN(g + 1, G.cells)) return G.phi0;
  // f = (d mod 2^sh) 2^-sh, exact: 1 + f assembled from its bits, minus 1
  const float f =
      __uint_as_float(0x3F800000u | ((d & ((1u << G.sh) - 1u)) << (23 - G.sh))) - 1.0f;
  const float a = __ldg(G.phi + g), b = __ldg(G.phi + g + 1);
  return a + f * (b - a);
}

// g(s_j) = (dr/ds) / sqrt(Q) at envelope sample j in FP32 with Phi from the
// grid (sa = s(3 - s^2), sb = 3 (1 - s^2) from the tables).  The envelope
// F = 1.2 max_j g(s_j) only has to bound g: the reciprocal and the inverse
// square root are the one-instruction approximations (relative errors
// below 2^-22), far inside the factor 1.2.
__device__ __forceinline__ float g32_grid(const Grid& G, float E, float J, float c0, float c1,
                                          float sa, float sb) {
  const float rs = c0 + c1 * sa;
  const float drds = c1 * sb;
  float xq, rq;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(xq) : "f"(rs));
  const float ph = grid_phi(G, xq);
  const float L = J * xq;
  const float Q = 2.0f * (E - ph) - L * L;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rq) : "f"(Q));
  return Q > 0.0f ? drds * rq : 0.0f;
}

// the FP32 shell (bucket index) of the point r(s), the start of the FP64
// shell walk of an accepted or edge point
__device__ __forceinline__ int shell32_of(const double4_32a* __restrict__ nd, int nb,
                                          const Buckets& B, float c0, float c1, float sv) {
  const float rs = c0 + c1 * (sv * (3.0f - sv * sv));
  const float xq[1] = {1.0f / rs};
  int sh[1];
  shells32_bk<1>(NodeKeys{nd}, nb, B, xq, sh);
  return sh[0];
}

// Mixed mode: the orbit point r(s) in FP64 from an FP32 shell index sh
// (moved to the exact shell), Phi from the enclosed-mass slope of its
// shell (Eq. 6: Phi = Phi_i + M_i (1/r_i - 1/r)), L = J / r and Q.
__device__ __forceinline__ void point64(const double4_32a* __restrict__ nd, int64_t nb,
                                        const Star& st, double c0, double c1, double sv, int sh,
                                        double& rs, double& xs, double& ph, double& L,
                                        double& Q) {
  rs = c0 + c1 * (sv * (3.0 - sv * sv));
  double4_32a a;
  const int64_t i64 = fix_shell_nodes(nd, nb, sh, rs, a);
  xs = div_rn(1.0, rs);
  ph = i64 < 0 ? a.z : a.z + a.w * (a.y - xs);
  L = st.J * xs;
  Q = scale_up<1>(st.E - ph) - L * L;
}


// FP64 mode: the orbit point r(s) in FP64 from an FP32 shell guess sh
// (moved to the exact shell), Phi by Eq. 6's division form (the FP64
// statement of the method, as phi_in_shell), L = J / r and Q.  Its
// quotients go through the shared bodies (div_rn_nl): measured faster in
// the long kernels that use it.
// sa = s (3 - s^2), the factor of c1 in r(s) (a table entry at the
// envelope's samples)
__device__ __forceinline__ void point64_div_sa(const double4_32a* __restrict__ nd, int64_t nb,
                                               const Star& st, double c0, double c1, double sa,
                                               int sh, double& rs, double& ph, double& Q,
                                               double& L) {
  rs = c0 + c1 * sa;
  double4_32a a;
  const int64_t i = fix_shell_nodes(nd, nb, sh, rs, a);
  if (i < 0) {
    ph = a.z;  // node 0's Phi: the central constant
  } else {
    const double xq = div_rn_nl(1.0, rs);
    double xj1 = 0.0, pj1 = 0.0;
    if (i + 1 < nb) {
      const double4_32a b = nd[i + 1];
      xj1 = b.y;
      pj1 = b.z;
    }
    const double den = a.y - xj1;
    ph = !(den > 0.0) ? a.z : a.z + div_rn_nl(a.y - xq, den) * (pj1 - a.z);
  }
  L = div_rn_nl(st.J, rs);
  Q = scale_up<1>(st.E - ph) - L * L;
}

__device__ __forceinline__ void point64_div(const double4_32a* __restrict__ nd, int64_t nb,
                                            const Star& st, double c0, double c1, double sv,
                                            int sh, double& rs, double& ph, double& Q,
                                            double& L) {
  point64_div_sa(nd, nb, st, c0, c1, sv * (3.0 - sv * sv), sh, rs, ph, Q, L);
}

// g(s) of FP64 mode at the point of point64_div, sb = 1 - s^2
__device__ __forceinline__ double g_of_point_sb(double c1, double sb, double Q) {
  if (!(Q > 0.0)) return 0.0;
  return div_rn_nl((3.0 * c1) * sb, sqrt_rn_nl(Q));
}

__device__ __forceinline__ double g_of_point(double c1, double sv, double Q) {
  return g_of_point_sb(c1, 1.0 - sv * sv, Q);
}

// (2k + 1) 2^-24 from the top 23 bits of a word: exact in float, in (0, 1)
__device__ __forceinline__ float u01f(uint32_t hi) {
  // 1 + k 2^-23 assembled from its bits, minus 1 (exact), plus 2^-24
  // (exact): no int -> float conversion
  return (__uint_as_float(0x3F800000u | (hi >> 9)) - 1.0f) + 0x1p-24f;
}

// ------------------------------------------- double-float (float pairs)
// A value as hi + lo with two floats (~48 bits), from the error-free sum of
// two floats (Knuth's two-sum; every operation rounds once, no contraction)
// and product (the fused multiply-add gives the product's error exactly).
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_of(double v) {
  DF d;
  d.hi = (float)v;
  d.lo = (float)(v - (double)d.hi);
  return d;
}

// The same split from the bit pattern with integer operations (hi: the top
// 24 significand bits of v, lo: the next 24 of the remaining 29, both
// truncated, together within 2^-46 |v|), for 2^-60 <= |v| < 2^100 where both
// are normal floats; other values (zero included) by the conversions.
__device__ __forceinline__ DF df_split(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned ex = (unsigned)(u >> 52) & 0x7FFu;
  if (ex < 1023u - 60u || ex >= 1023u + 100u) return df_of(v);
  const unsigned sg = (unsigned)(u >> 32) & 0x80000000u;
  DF d;
  d.hi = __uint_as_float(sg | ((ex - 896u) << 23) | ((unsigned)(u >> 29) & 0x7FFFFFu));
  const unsigned ml = (unsigned)u & 0x1FFFFFFFu;
  if (ml == 0u) {
    d.lo = 0.0f;
    return d;
  }
  const int lz = __clz((int)ml);  // 3 .. 31
  // ml 2^(ex - 1075) = 1.f 2^(ex - 1075 + 31 - lz); exponent field in [15, 202]
  const unsigned fe = ex - 1075u + 127u + (unsigned)(31 - lz);
  const unsigned mant = ((ml << lz) << 1) >> 9;  // the 23 bits after the leading one
  d.lo = __uint_as_float(sg | (fe << 23) | mant);
  return d;
}

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  DF d;
  d.hi = s;
  d.lo = (a - (s - bb)) + (b - bb);
  return d;
}

__device__ __forceinline__ DF df_norm(float hi, float lo) {
  const float s = hi + lo;
  DF d;
  d.hi = s;
  d.lo = lo - (s - hi);
  return d;
}

__device__ __forceinline__ DF df_sub(DF a, DF b) {
  const DF s = two_sum(a.hi, -b.hi);
  return df_norm(s.hi, s.lo + (a.lo - b.lo));
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  return df_norm(p, e + (a.hi * b.lo + a.lo * b.hi));
}

// Q = 2 (E - Phi) - (J x)^2 at a node from the float pairs, and whether its
// sign is certain.  The pairs hold E, J (truncated or rounded) within
// 2^-46 and 1/r, Phi within 2^-48; each pair sum adds at most 2^-46 of its
// operands' magnitudes and each pair product 2^-45 of its result, so L^2
// is within 2^-42.9 and Q within 2^-42.7 of S = |E| + |Phi| + L^2.  The
// FP64 evaluation 2 (E - Phi) - (J x) (J x) from the doubles is within
// 2^-50 S.  Beyond 2^-40 S both therefore have the sign of the exact Q.
__device__ __forceinline__ float node_q_df(const float4* __restrict__ tdf, DF E, DF J, int i,
                                           bool& sure) {
  const float4 t = __ldg(tdf + i);
  const DF x{t.x, t.y}, ph{t.z, t.w};
  const DF d = df_sub(E, ph);
  const DF L = df_mul(J, x);
  const DF L2 = df_mul(L, L);
  const DF q = df_sub(DF{2.0f * d.hi, 2.0f * d.lo}, L2);
  const float qv = q.hi != 0.0f ? q.hi : q.lo;
  sure = fabsf(qv) > 0x1p-40f * ((fabsf(E.hi) + fabsf(ph.hi)) + L2.hi);
  return qv;
}

// Q in FP32 at grid point g (1/r from the grid key, Phi from the grid)
__device__ __forceinline__ float grid_q(const Grid& G, float E, float J, int g, float& xg) {
  xg = __uint_as_float(G.key0 + ((uint32_t)g << G.sh));
  const float L = J * xg;
  return 2.0f * (E - __ldg(G.phi + g)) - L * L;
}

__device__ __forceinline__ float node_q(const float4* __restrict__ tdf, float E, float J, int i) {
  const float4 n = __ldg(tdf + i);  // (1/r, Phi) as the float pairs' high parts
  const float L = J * n.x;
  return 2.0f * (E - n.z) - L * L;
}

// FP32 node brackets of both turning points from the potential grid: the
// sign changes of Q on the grid points (bisections on the L1-resident grid,
// in lockstep), the root inside the cell by linear interpolation in 1/r,
// its node through the bucket index, then a short walk over neighbouring
// nodes to where Q32 changes sign (r_max: node j with Q32 >= 0, j + 1 with
// Q32 < 0 or the virtual node nb; r_min: j with Q32 < 0 or -1, j + 1 with
// Q32 >= 0 or the star).  Returns false when a walk exceeds its bound.
__device__ __forceinline__ bool grid_brackets(const Grid& G, const float4* __restrict__ tdf,
                                              const Buckets& BK, float E, float J, DF Ed, DF Jd,
                                              int nb, int k, int& jmax, int& jmin, bool& cert1,
                                              bool& cert2) {
  const float xk = __ldg(&tdf[k].x);
  const uint32_t kk = __float_as_uint(xk);
  cert1 = cert2 = false;
  if (G.cells < 2 || kk < G.key0) return false;
  int gk = (int)((kk - G.key0) >> G.sh);  // grid points 0..gk lie at or outside the star
  if (gk > G.cells - 1) gk = G.cells - 1;
  // r_max: last grid point in [0, gk] with Q < 0 (-1: none; Q -> 2E < 0 as 1/r -> 0)
  // r_min: first grid point in [gk + 1, cells) with Q < 0 (cells: none)
  int alo = -1, ahi = gk + 1, blo = gk, bhi = G.cells;
  float xa_lo = 0.0f, qa_lo = 0.0f, xb_hi = 0.0f, qb_hi = 0.0f;
  float xa_hi = xk, qa_hi = 0.0f, xb_lo = xk, qb_lo = 0.0f;
  while (ahi - alo > 1 || bhi - blo > 1) {
    const bool ra = ahi - alo > 1, rb = bhi - blo > 1;
    const int ma = ra ? (alo + ahi) >> 1 : 0, mb = rb ? (blo + bhi) >> 1 : 0;
    float xa, xb;
    const float qa = grid_q(G, E, J, ma, xa), qb = grid_q(G, E, J, mb, xb);
    if (ra) {
      if (qa < 0.0f) { alo = ma; xa_lo = xa; qa_lo = qa; }
      else { ahi = ma; xa_hi = xa; qa_hi = qa; }
    }
    if (rb) {
      if (qb < 0.0f) { bhi = mb; xb_hi = xb; qb_hi = qb; }
      else { blo = mb; xb_lo = xb; qb_lo = qb; }
    }
  }
  // the star's own end of each bracket: Q32 at the star
  const float qk = node_q(tdf, E, J, k);
  if (ahi == gk + 1) qa_hi = qk;
  if (blo == gk) qb_lo = qk;
  float xq[2];
  // root estimates (Q linear in 1/r across a cell up to ~(cell width)^2)
  xq[0] = alo < 0 ? 0.0f : xa_lo + (xa_hi - xa_lo) * (qa_lo / (qa_lo - qa_hi));
  xq[1] = bhi >= G.cells ? 0.0f : xb_lo + (xb_hi - xb_lo) * (qb_lo / (qb_lo - qb_hi));
  int sh[2];
  shells32_bk<2>(FloatKeys{&tdf[0].x, 4}, nb, BK, xq, sh);
  int j1 = alo < 0 ? nb - 1 : sh[0];
  int j2 = bhi >= G.cells ? -1 : sh[1];
  j1 = j1 < k ? k : (j1 > nb - 1 ? nb - 1 : j1);
  j2 = j2 < -1 ? -1 : (j2 > k - 1 ? k - 1 : j2);
  // walks; at the stop the sign tests that ended each walk are the FP64
  // walk's own stopping tests, and when every one of them is certain the
  // FP64 walk from this bracket would stop at once (cert)
  bool d1 = false, d2 = false, s1a = true, s2a = true;
  for (int w = 0; w < 64 && !(d1 && d2); ++w) {
    if (!d1) {
      bool su = true, sd = true;
      if (j1 + 1 < nb && !(node_q_df(tdf, Ed, Jd, j1 + 1, su) < 0.0f)) {
        ++j1;
      } else if (j1 > k && node_q_df(tdf, Ed, Jd, j1, sd) < 0.0f) {
        --j1;
      } else {
        d1 = true;
        s1a = su && sd;
      }
    }
    if (!d2) {
      bool su = true, sd = true;
      if (j2 + 1 < k && node_q_df(tdf, Ed, Jd, j2 + 1, su) < 0.0f) {
        ++j2;
      } else if (j2 >= 0 && !(node_q_df(tdf, Ed, Jd, j2, sd) < 0.0f)) {
        --j2;
      } else {
        d2 = true;
        s2a = su && sd;
      }
    }
  }
  jmax = j1;
  jmin = j2;
  cert1 = d1 && d2 && s1a;
  cert2 = d1 && d2 && s2a;
  return d1 && d2;
}

// verify_rmax / verify_rmin on the node records: the same walks (a bounded
// walk from the FP32 bracket, then the full bisection), returning the
// records of the bracket's node (a; node 0 for r_min's -1) and of the node
// after it (b)
__device__ __forceinline__ int64_t verify_rmax_nodes(const Table64& T,
                                                     const double4_32a* __restrict__ nd,
                                                     const Star& s, int64_t j, double4_32a& a,
                                                     double4_32a& b) {
  const int64_t nb = T.nb;
  if (j < s.k) j = s.k;
  if (j > nb - 1) j = nb - 1;
  a = nd[j];
  b = j + 1 < nb ? nd[j + 1] : a;
  for (int w = 0; w < 64; ++w) {
    if (j + 1 < nb && !(Qv(s, b.y, b.z) < 0.0)) {
      ++j;
      a = b;
      b = j + 1 < nb ? nd[j + 1] : a;
      continue;
    }
    if (j > s.k && Qv(s, a.y, a.z) < 0.0) {
      --j;
      b = a;
      a = nd[j];
      continue;
    }
    return j;
  }
  j = bisect_rmax64(T, s);
  a = nd[j];
  b = j + 1 < nb ? nd[j + 1] : a;
  return j;
}

__device__ __forceinline__ int64_t verify_rmin_nodes(const Table64& T,
                                                     const double4_32a* __restrict__ nd,
                                                     const Star& s, int64_t j, double4_32a& a,
                                                     double4_32a& b) {
  if (j < -1) j = -1;
  if (j > s.k - 1) j = s.k - 1;
  a = nd[j < 0 ? 0 : j];
  b = nd[j + 1];
  for (int w = 0; w < 64; ++w) {
    if (j + 1 < s.k && Qv(s, b.y, b.z) < 0.0) {
      ++j;
      a = b;
      b = nd[j + 1];
      continue;
    }
    if (j >= 0 && !(Qv(s, a.y, a.z) < 0.0)) {
      --j;
      b = a;
      a = nd[j < 0 ? 0 : j];
      continue;
    }
    return j;
  }
  j = bisect_rmin64(T, s);
  a = nd[j < 0 ? 0 : j];
  b = nd[j + 1];
  return j;
}

// Mixed mode, turning points of one bound star with E < 0: both node
// bisections in FP32 in lockstep on the float table (r_max over [k, nb],
// r_min over [-1, k]), each bracket verified in FP64 by a bounded walk,
// then the FP64 roots inside the bracketing shells (Eq. 12).
__device__ __forceinline__ void turning_mixed(const Table64& T,
                                              const float4* __restrict__ tdf,
                                              const double4_32a* __restrict__ nd, const Grid& G,
                                              const Buckets& BK, const Star& s, double& rmin,
                                              double& rmax) {
  // E and J as float pairs; their high parts serve the FP32 searches
  const DF Ed = df_split(s.E), Jd = df_split(s.J);
  const float E32 = Ed.hi, J32 = Jd.hi;
  const int nb32 = (int)T.nb, k32 = (int)s.k;
  int lo1, lo2;
  bool cert1, cert2;
  if (!grid_brackets(G, tdf, BK, E32, J32, Ed, Jd, nb32, k32, lo1, lo2, cert1, cert2)) {
    // both node bisections in FP32, in lockstep; their brackets are not
    // certified (the FP64 walks run from them)
    cert1 = cert2 = false;
    lo1 = k32, lo2 = -1;
    int hi1 = nb32, hi2 = k32;
    const int rounds = search_rounds(nb32);
    for (int it = 0; it < rounds; ++it) {
      const bool a1 = hi1 - lo1 > 1, a2 = hi2 - lo2 > 1;
      const int m1 = a1 ? lo1 + ((hi1 - lo1) >> 1) : k32;
      const int m2 = a2 ? lo2 + ((hi2 - lo2) >> 1) : k32;
      const float4 e1 = __ldg(tdf + m1), e2 = __ldg(tdf + m2);
      const float L1 = J32 * e1.x, L2 = J32 * e2.x;
      const bool n1 = 2.0f * (E32 - e1.z) - L1 * L1 < 0.0f;
      const bool n2 = 2.0f * (E32 - e2.z) - L2 * L2 < 0.0f;
      if (a1) { if (n1) hi1 = m1; else lo1 = m1; }
      if (a2) { if (n2) lo2 = m2; else hi2 = m2; }
    }
  }
  // A certified bracket is the one the FP64 walk stops at; otherwise that
  // walk runs from it.  Then the FP64 roots in the bracketing shells.
  const int64_t nb = T.nb;
  double4_32a a1, b1, a2, b2;
  int64_t jmax, jmin;
  if (cert1) {
    jmax = lo1;
    a1 = nd[jmax];
    b1 = jmax + 1 < nb ? nd[jmax + 1] : a1;
  } else {
    jmax = verify_rmax_nodes(T, nd, s, lo1, a1, b1);
  }
  if (cert2) {
    jmin = lo2;
    a2 = nd[jmin < 0 ? 0 : jmin];
    b2 = nd[jmin + 1];
  } else {
    jmin = verify_rmin_nodes(T, nd, s, lo2, a2, b2);
  }
  rmax = rmax_core(s, a1.x, a1.y, a1.z, a1.w, jmax + 1 < nb, b1.x);
  rmin = rmin_core(s, jmin < 0, a2.x, a2.y, a2.z, jmin < 0 ? 0.0 : a2.w, jmin >= 0, b2.x);
}

// First kernel of the mixed-mode orbit step: the turning points of every
// bound star with E < 0, into tp_min / tp_max (split from the sampling
// kernel so that each runs with fewer registers and more warps).
template <int kMinB>
__global__ void __launch_bounds__(256, kMinB) k_turning_mixed(
    Seg S, const double* r, const double* x, const double* phi,
    const double* Menc, const double* vr, const double* vt, BucketArgs BA, double* tp_min,
    double* tp_max, double4_32a* orb, int64_t n) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c = seg_find(S.off, S.n_seg, p);
  const int64_t sb = S.off[c];
  const int64_t nbc = S.nb[c];
  const int64_t k = p - sb;
  if (k >= nbc) return;
  const Table64 T{r + sb, x + sb, phi + sb, nbc};
  const double rk = r[p], vrk = vr[p], vtk = vt[p];
  Star s;
  s.k = k;
  s.E = __ldg(T.phi + k) + scale_down<1>(vrk * vrk + vtk * vtk);
  s.J = rk * vtk;
  // E < 0 on the bit pattern (negative, nonzero, not NaN); otherwise an
  // escaper, which the sampling kernel handles
  const unsigned long long eb = ubits(s.E);
  if (!(eb > 0x8000000000000000ull && eb <= 0xFFF0000000000000ull)) {
    orb[p] = make_double4_32a(s.E, s.J, 0.0, 0.0);
    return;
  }
  double rmin, rmax;
  Buckets BK;
  const int4 pr = BA.prm[c];
  BK.start = BA.start + BA.off[c];
  BK.base = BA.base[c];
  BK.shift = pr.x;
  BK.nbk = pr.y;
  BK.lo = pr.z;
  BK.hi = pr.w;
  turning_mixed(T, BA.tdf + sb, BA.node + sb, grid_of(BA, c), BK, s, rmin, rmax);
  if (tp_min) {
    tp_min[p] = rmin;
    tp_max[p] = rmax;
  }
  // the orbit's record for the sampling kernels: E, J, c0 = (r_max + r_min)
  // / 2 and c1 = (r_max - r_min) / 4 (c1 > 0 exactly when r_max > r_min:
  // radii are far from the underflow range)
  orb[p] = make_double4_32a(s.E, s.J, scale_down<1>(rmax + rmin), scale_down<2>(rmax - rmin));
}

// One trial's accept test in FP32 with a bound on its error: +1 accepted,
// 0 rejected, -1 undecided (the trial is then taken in FP64).  The test is
// F X' < g(s), g = (dr/ds) / sqrt(Q), at the FP64 point s (52 bits) and
// X' (53 bits); the float values use 23 bits of each, so |s32 - s| and
// |X'32 - X'| are at most 2^-23 and 2^-24.  Bounds (u = 2^-24):
//   r(s):  |r32 - r| <= 3|c1| (1 - s^2 + 2^-21) 2^-23 + 8u (|c0| + 2|c1|)
//          + 2^-22 |r|                         1/r by the approximate reciprocal
//   Q:     16u (|E| + |Phi| + L^2)             float operations and inputs
//          + (2 err_grid + 4u) |Phi|           grid interpolation and values
//          + 1.5 * 2 (M x + L^2) |dr| / r      Q's slope in r, M <= M_bound
//   g:     1.5 * (1/2) dQ / Q + 6|c1| 2^-23 / (dr/ds) + 16u
//          + 2^-21                             the approximate 1/sqrt(Q)
// Close to a turning point Q is within a few dQ of zero and the trial is
// left undecided; elsewhere the FP32 answer is the FP64 one.
// kExact (FP64 mode): F is the float of the FP64 envelope, and a trial
// whose g might lie on either side of F is left undecided too, so that the
// count of g > F (violations) is the FP64 one.
template <bool kExact>
__device__ __forceinline__ int accept32(const Grid& G, float E, float J, float c0, float c1,
                                        float F, float sv, float xp,
                                        unsigned long long& viol) {
  const float ss = sv * sv;
  const float rs = c0 + c1 * (sv * (3.0f - ss));
  const float drds = (3.0f * c1) * (1.0f - ss);
  // the one-instruction reciprocal and inverse square root (relative
  // errors below 2^-22): the reciprocal's error counts as an error in r (in
  // dr), the inverse square root's in eg (2^-21), and eg, computed with them,
  // is taken 2^-16 larger
  float xq;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(xq) : "f"(rs));
  const float ph = grid_phi(G, xq);
  const float L = J * xq, L2 = L * L;
  const float Q = 2.0f * (E - ph) - L2;
  const float ac1 = fabsf(c1), aph = fabsf(ph);
  const float dr = 3.0f * ac1 * ((1.0f - ss) + 0x1p-21f) * 0x1p-23f +
                   0x1p-21f * (fabsf(c0) + 2.0f * ac1) + 0x1p-22f * fabsf(rs);
  const float qerr = 0x1p-20f * (fabsf(E) + aph + L2) + (2.0f * G.err + 0x1p-22f) * aph +
                     3.0f * (G.mb * xq + L2) * (dr * xq);
  if (!(Q > 4.0f * qerr) || !(drds > 0x1p-100f)) return -1;
  float rq, rd;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rq) : "f"(Q));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(drds));
  const float g = drds * rq;
  const float eg = ((0.75f * qerr) * (rq * rq) + (6.0f * ac1 * 0x1p-23f) * rd + 0x1p-20f +
                    0x1p-21f) * (1.0f + 0x1p-16f);
  if (!(eg < 0.25f)) return -1;
  if (kExact) {
    const bool above = g * (1.0f - eg) > F * (1.0f + 0x1p-22f);
    const bool below = g * (1.0f + eg) < F * (1.0f - 0x1p-22f);
    if (!above && !below) return -1;
  }
  const float a = F * xp, da = F * 0x1p-22f;
  if (a + da < g * (1.0f - eg)) {
    if (g > F) ++viol;
    return 1;
  }
  if (a - da > g * (1.0f + eg)) {
    if (g > F) ++viol;
    return 0;
  }
  return -1;
}

// g(s) in FP32 at an envelope sample with the error bound of accept32
// (the sample's float s is within 2^-25 of the FP64 one): 1 with g and its
// relative bound eg, 0 when Q < 0 for certain (g = 0), -1 when FP32 cannot
// tell.  The reciprocal and the inverse square root are the one-instruction
// approximations (relative errors below 2^-22): the reciprocal's error is an
// error in r (added to dr, as r's own), the inverse square root's goes into
// eg (2^-21), and eg itself, computed with them, is taken 2^-16 larger.
__device__ __forceinline__ int g32_bounded(const Grid& G, float E, float J, float c0, float c1,
                                           float sv, float& g, float& eg) {
  const float ss = sv * sv;
  const float rs = c0 + c1 * (sv * (3.0f - ss));
  const float drds = (3.0f * c1) * (1.0f - ss);
  float xq;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(xq) : "f"(rs));
  const float ph = grid_phi(G, xq);
  const float L = J * xq, L2 = L * L;
  const float Q = 2.0f * (E - ph) - L2;
  const float ac1 = fabsf(c1), aph = fabsf(ph);
  const float dr = 3.0f * ac1 * ((1.0f - ss) + 0x1p-21f) * 0x1p-23f +
                   0x1p-21f * (fabsf(c0) + 2.0f * ac1) + 0x1p-22f * fabsf(rs);
  const float qerr = 0x1p-20f * (fabsf(E) + aph + L2) + (2.0f * G.err + 0x1p-22f) * aph +
                     3.0f * (G.mb * xq + L2) * (dr * xq);
  if (Q < -4.0f * qerr) return 0;
  if (!(Q > 4.0f * qerr) || !(drds > 0x1p-100f)) return -1;
  float rq, rd;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rq) : "f"(Q));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rd) : "f"(drds));
  g = drds * rq;
  eg = ((0.75f * qerr) * (rq * rq) + (6.0f * ac1 * 0x1p-23f) * rd + 0x1p-20f + 0x1p-21f) *
       (1.0f + 0x1p-16f);
  if (!(eg < 0.25f)) return -1;
  return 1;
}

// the envelope samples s_j as floats (within 2^-25 of the FP64 ones)
#define CMC_SJF(j) ((float)CMC_SJ(j))
__constant__ float c_s32[21] = {CMC_SJ21(CMC_SJF)};

// FP64 mode's envelope F = 1.2 max_j g(s_j) over the 21 samples, the FP64
// value (Eq. 6's division form, as the FP64 statement of the method):
// every g(s_j) is first bounded in FP32 (g32_bounded); only the samples
// whose upper bound reaches the largest lower bound, and those FP32 cannot
// bound, can hold the maximum, and only they are evaluated in FP64.  Nearly
// circular orbits have a flat g and FP32 bounds too loose to rank their
// samples, so the candidates per star range from 1 to 21 (about 1.1 on
// average).  Two kernels: k_env_screen bounds the samples and lists the
// candidate (star, sample) pairs; k_env_eval evaluates them one pair per
// thread (whole warps busy, where one warp pooling its own stars' pairs
// left most lanes idle in its last round), the maximum per star kept in
// gmax as bits (g >= 0 orders as its bits).  gmax = 0 for stars without an
// orbit to sample (r_max <= r_min: every g is 0 or negative there); the
// readers take F = 1.2 gmax.
constexpr int kEnvThreads = 128;
constexpr uint64_t kEnvNone = ~0ull;  // a list slot left empty

// s_j (3 - s_j^2) and 1 - s_j^2 at the 21 samples, computed once on the
// device with the operations of point64_div and g_of_point (k_env_tables)
__device__ double g_env_sa[21], g_env_sb[21];

__global__ void k_env_tables() {
  const int j = threadIdx.x;
  if (j >= 21) return;
  const double sv = c_s64[j];
  g_env_sa[j] = sv * (3.0 - sv * sv);
  g_env_sb[j] = 1.0 - sv * sv;
}

// FP64 g at sample j of a star (the noinline quotients keep this copy small)
__device__ __noinline__ double g64_sample(const double4_32a* __restrict__ nd, int64_t nb,
                                          const Buckets& BK, double E, double J, double c0,
                                          double c1, int j) {
  Star s;
  s.k = 0;
  s.E = E;
  s.J = J;
  const float c0f = f32_rn(c0), c1f = f32_rn(c1);
  double rs, ph, Q, L;
  point64_div_sa(nd, nb, s, c0, c1, g_env_sa[j],
                 shell32_of(nd, (int)nb, BK, c0f, c1f, c_s32[j]), rs, ph, Q, L);
  return g_of_point_sb(c1, g_env_sb[j], Q);
}

__device__ __forceinline__ Buckets buckets_of(const BucketArgs& BA, int c) {
  Buckets BK;
  const int4 pr = BA.prm[c];
  BK.start = BA.start + BA.off[c];
  BK.base = BA.base[c];
  BK.shift = pr.x;
  BK.nbk = pr.y;
  BK.lo = pr.z;
  BK.hi = pr.w;
  return BK;
}

// E, J and the orbit's c0 = (r_max + r_min) / 2, c1 = (r_max - r_min) / 4
// of star p (segment c) from the turning-point kernel's record; false where
// there is no orbit to sample
__device__ __forceinline__ bool env_star(const Seg& S, const double4_32a* orb, int64_t p,
                                         int& c, double& E, double& J, double& c0, double& c1) {
  c = seg_find(S.off, S.n_seg, p);
  const int64_t nbc = S.nb[c], k = p - S.off[c];
  if (!(k < nbc)) return false;
  const double4_32a o = orb[p];
  E = o.x;
  J = o.y;
  c0 = o.z;
  c1 = o.w;
  return lt0(E) && gt_pos(c1, 0.0);
}

__global__ void __launch_bounds__(kEnvThreads) k_env_screen(Seg S, BucketArgs BA,
                                                            const double4_32a* orb, EnvWork W,
                                                            int64_t n) {
  __shared__ float s_hi[21][kEnvThreads];  // upper bounds of the samples
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int c = -1;
  unsigned cand = 0u;
  if (p < n) {
    double E, J, c0, c1;
    if (env_star(S, orb, p, c, E, J, c0, c1)) {
      // the star's values for the evaluation of its pairs
      W.star[p] = make_double4_32a(E, J, c0, c1);
      const float c0f = f32_rn(c0), c1f = f32_rn(c1), E32 = f32_rn(E), J32 = f32_rn(J);
      const Grid GD = grid_of(BA, c);
      unsigned pos = 0u;
      float lo_max = 0.0f;
      // one copy of the sample code (not unrolled: code size), the upper
      // bounds kept in shared memory
#pragma unroll 1
      for (int jj = 0; jj < 21; ++jj) {
        float g = 0.0f, eg = 0.0f;
        const int st = g32_bounded(GD, E32, J32, c0f, c1f, c_s32[jj], g, eg);
        float h = 0.0f;
        if (st > 0) {
          const float lo = g * (1.0f - eg);
          h = g * (1.0f + eg);
          lo_max = lo > lo_max ? lo : lo_max;
          pos |= 1u << jj;
        } else if (st < 0) {
          cand |= 1u << jj;
        }
        s_hi[jj][threadIdx.x] = h;
      }
#pragma unroll 1
      for (int jj = 0; jj < 21; ++jj)
        if (((pos >> jj) & 1u) && s_hi[jj][threadIdx.x] >= lo_max) cand |= 1u << jj;
    }
    W.gmax[p] = 0.0;
  }
  // the warp's pairs go to the list in lane order, with one atomic
  const unsigned cnt = (unsigned)__popc(cand);
  unsigned incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  if (total) {
    unsigned long long base = 0ull;
    if (lane == 0) base = atomicAdd(W.cnt, (unsigned long long)total);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    const unsigned long long cap = (unsigned long long)W.cap;
    if (base + total <= cap) {
      unsigned long long at = base + (incl - cnt);
      for (unsigned m = cand; m; m &= m - 1u)
        W.list[at++] = ((uint64_t)p << 5) | (uint64_t)(__ffs(m) - 1);
    } else {
      // the list is full: its slots reserved here stay empty, and the
      // stars go to the spill list (one entry per star, never full)
      for (unsigned long long e = base + lane; e < base + total && e < cap; e += 32)
        W.list[e] = kEnvNone;
      if (cnt) {
        const unsigned long long at = atomicAdd(W.cnt + 1, 1ull);
        W.spill[at] = ((uint64_t)p << 21) | (uint64_t)cand;
      }
    }
  }
  // FP64 evaluations: one atomic per segment present in the warp
  const unsigned am = __ballot_sync(0xFFFFFFFFu, p < n);
  if (p < n) {
    const unsigned peers = __match_any_sync(am, c);
    const unsigned tot = __reduce_add_sync(peers, cnt);
    if (lane == __ffs(peers) - 1) stat_add(S.stats, c, kStEnvelope64, tot);
  }
}

// FP64 g of one listed pair into its star's maximum (E, J, c0, c1 from the
// screening kernel's record of the star)
__device__ __forceinline__ void env_pair(const Seg& S, const BucketArgs& BA, const EnvWork& W,
                                         int64_t p, int jj) {
  const int c = seg_find(S.off, S.n_seg, p);
  const double4_32a v = W.star[p];
  const int64_t sb = S.off[c];
  const Buckets BK = buckets_of(BA, c);
  double* gmax = W.gmax;
  const double g = g64_sample(BA.node + sb, S.nb[c], BK, v.x, v.y, v.z, v.w, jj);
  if (g > 0.0) atomicMax((unsigned long long*)(gmax + p), (unsigned long long)__double_as_longlong(g));
}

__global__ void __launch_bounds__(kEnvThreads) k_env_eval(Seg S, BucketArgs BA, EnvWork W) {
  const unsigned long long cap = (unsigned long long)W.cap;
  const unsigned long long np = W.cnt[0] < cap ? W.cnt[0] : cap;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < np;
       e += stride) {
    const uint64_t w = W.list[e];
    if (w == kEnvNone) continue;
    env_pair(S, BA, W, (int64_t)(w >> 5), (int)(w & 31u));
  }
  // spilled stars: 32 at a time per warp, each warp pooling their pairs
  const unsigned long long ns = W.cnt[1];
  const int lane = threadIdx.x & 31;
  const unsigned long long warps = stride / 32;
  for (unsigned long long w0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) / 32 * 32;
       w0 < ns; w0 += warps * 32) {
    const unsigned long long i = w0 + lane;
    const uint64_t w = i < ns ? W.spill[i] : 0ull;
    const unsigned cand = (unsigned)(w & 0x1FFFFFu);
    const int64_t ps = (int64_t)(w >> 21);
    const unsigned cnt = (unsigned)__popc(cand);
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    for (unsigned t0 = 0; t0 < total; t0 += 32) {
      const unsigned t = t0 + (unsigned)lane;
      // owner: the first lane whose inclusive count exceeds t
      int own = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const unsigned v = __shfl_sync(0xFFFFFFFFu, incl, own + step - 1);
        if (v <= t) own += step;
      }
      const unsigned o_incl = __shfl_sync(0xFFFFFFFFu, incl, own);
      const unsigned o_cnt = __shfl_sync(0xFFFFFFFFu, cnt, own);
      const unsigned o_cand = __shfl_sync(0xFFFFFFFFu, cand, own);
      const long long o_p = __shfl_sync(0xFFFFFFFFu, (long long)ps, own);
      if (t < total) {
        const int rank = (int)(t - (o_incl - o_cnt));  // which of the owner's pairs
        env_pair(S, BA, W, (int64_t)o_p, (int)__fns(o_cand, 0u, rank + 1));
      }
    }
  }
}

// Result of the FP32 sampler in a star's key slot: bits 0-29 the trial
// index, 30-31 the status, 32-63 the bits of F (float)
enum : uint32_t { kSmpAccepted = 0, kSmpPending = 1, kSmpDegenerate = 2, kSmpCap = 3 };

// Second kernel of the mixed-mode orbit step (after k_turning_mixed): the
// envelope F = 1.2 max g over the 21 samples with Phi from the potential
// grid, then the FP32 trials (accept32) up to the first one that is
// accepted (kSmpAccepted) or that FP32 cannot decide (kSmpPending:
// k_pending64 takes it and the rest of the sequence in FP64).  Only
// float state is live in the loop, so the kernel runs at full occupancy
// without spilling.  F only has to bound g: 1.2 max g over these FP32
// samples is as valid an envelope as the FP64 one (it differs from it by up
// to ~1e-4 at the outer samples, so the two modes draw different, equally
// exact, accept sequences).
// kExact (FP64 mode): F is FP64 mode's envelope, 1.2 Fx (Fx from k_env_eval),
// and a trial is decided here only where the FP64 decision and violation
// count are certain.
template <int kMinB, bool kTaus, bool kExact>
__global__ void __launch_bounds__(256, kMinB) k_sample32(Seg S, int max_trials,
                                                  const uint32_t* id,
                                                  const uint32_t* step_p, BucketArgs BA,
                                                  const double4_32a* orb,
                                                  uint64_t* keys, uint32_t* plist,
                                                  uint32_t* pcount, int64_t n, const double* Fx) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long viol = 0;
  bool pend = false;
  int c = -1;  // lanes past the end form their own group below
  if (p < n) {
    c = seg_find(S.off, S.n_seg, p);
    const int64_t k = p - S.off[c];
    // E, J, c0, c1 from the turning-point kernel
    const double4_32a o = k < S.nb[c] ? orb[p] : make_double4_32a(0.0, 0.0, 0.0, 0.0);
    const double E = o.x;
    if (k < S.nb[c] && lt0(E)) {
      const double J = o.y, c0 = o.z, c1 = o.w;
      const float c0f = f32_rn(c0), c1f = f32_rn(c1), E32 = f32_rn(E), J32 = f32_rn(J);
      const Grid GD = grid_of(BA, c);
      float F32;
      bool degenerate;
      if (kExact) {
        const double F64 = 1.2 * __ldg(Fx + p);
        F32 = f32_rn(F64);
        degenerate = !gt_pos(c1, 0.0) || !(F64 > 0.0);
      } else {
        float gmax = 0.0f;
#pragma unroll 3
        for (int j = 0; j < 21; ++j) {
          const float g = g32_grid(GD, E32, J32, c0f, c1f, c_sa32[j], c_sb32[j]);
          gmax = g > gmax ? g : gmax;
        }
        F32 = 1.2f * gmax;
        degenerate = !gt_pos(c1, 0.0) || !(F32 > 0.0f);
      }
      uint32_t st = kSmpCap;
      int t = 0;
      if (degenerate) {
        st = kSmpDegenerate;
      } else {
        Draws<kTaus> g = draws_of<kTaus>(S, c, id[p], *step_p);
        for (; t < max_trials; ++t) {
          const U4 w = g.block(kTagRej, (uint32_t)t);
          const int d = accept32<kExact>(GD, E32, J32, c0f, c1f, F32, 2.0f * u01f(w.y) - 1.0f,
                                 u01f(w.w), viol);
          if (d == 0) continue;
          st = d > 0 ? kSmpAccepted : kSmpPending;
          break;
        }
      }
      keys[p] = ((uint64_t)__float_as_uint(F32) << 32) | ((uint64_t)st << 30) |
                (uint64_t)(t & 0x3FFFFFFF);
      pend = st == kSmpPending;
    }
  }
  // pending stars onto the list of k_pending64 (one atomic per warp)
  const unsigned pm = __ballot_sync(__activemask(), pend);
  if (pm) {
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == __ffs(pm) - 1) base = atomicAdd(pcount, (uint32_t)__popc(pm));
    base = __shfl_sync(__activemask(), base, __ffs(pm) - 1);
    if (pend) plist[base + __popc(pm & ((1u << lane) - 1u))] = (uint32_t)p;
  }
  // violations: one atomic per segment present in the warp
  const unsigned full = __activemask();
  const unsigned peers = __match_any_sync(full, c);
  const unsigned vi = __reduce_add_sync(peers, (unsigned)viol);
  if ((threadIdx.x & 31) == __ffs(peers) - 1 && c >= 0) stat_add(S.stats, c, kStViolations, vi);
}

// Third kernel of the mixed-mode orbit step: every star the FP32 sampler
// left pending (a trial whose accept test FP32 could not decide, mostly
// close to a turning point, where Q vanishes like (1 - |s|)^2) takes that
// trial and the rest of its sequence in FP64; its key slot then holds
// kSmpAccepted and the accepted trial, or kSmpCap.  Most threads find no
// pending star and leave at once.
// one pending star (p = n: an idle lane); counts go to the statistics
// kExact (FP64 mode): F = 1.2 Fx, the points and g as FP64 mode's
template <bool kTaus, bool kExact>
__device__ __forceinline__ void pending_star(Seg S, int max_trials, const uint32_t* id,
                                             const uint32_t* step_p, BucketArgs BA,
                                             const double4_32a* orb, uint64_t* keys, int64_t p,
                                             int64_t n, const double* Fx) {
  unsigned long long viol = 0;
  unsigned int n64 = 0;
  int c = -1;
  if (p < n) {
    c = seg_find(S.off, S.n_seg, p);
    const int64_t sb = S.off[c], nbc = S.nb[c], k = p - sb;
    if (k < nbc) {
      const uint64_t res = keys[p];
      const double4_32a o = orb[p];  // E, J, c0, c1 from the turning-point kernel
      Star s;
      s.k = k;
      s.E = o.x;
      s.J = o.y;
      if (lt0(s.E) && ((uint32_t)(res >> 30) & 3u) == kSmpPending) {
        Buckets BK;
        const int4 pr = BA.prm[c];
        BK.start = BA.start + BA.off[c];
        BK.base = BA.base[c];
        BK.shift = pr.x;
        BK.nbk = pr.y;
        BK.lo = pr.z;
        BK.hi = pr.w;
        const double c0 = o.z, c1 = o.w;
        const float c0f = f32_rn(c0), c1f = f32_rn(c1);
        const double F =
            kExact ? 1.2 * __ldg(Fx + p) : (double)__uint_as_float((uint32_t)(res >> 32));
        uint32_t st = kSmpCap;
        int t = (int)(res & 0x3FFFFFFFull);
        // stream mode: the blocks of trials 0 .. t-1 were the FP32 sampler's
        Draws<kTaus> g = draws_of<kTaus>(S, c, id[p], *step_p);
        g.skip((uint32_t)t);
        for (; t < max_trials; ++t) {
          const U4 w = g.block(kTagRej, (uint32_t)t);
          const double sv = sym_double(sym_int(w.x, w.y));
          const int guess =
              shell32_of(BA.node + sb, (int)nbc, BK, c0f, c1f, 2.0f * u01f(w.y) - 1.0f);
          double g64v;
          if (kExact) {
            double rs, ph, Q, L;
            point64_div(BA.node + sb, nbc, s, c0, c1, sv, guess, rs, ph, Q, L);
            g64v = g_of_point(c1, sv, Q);
          } else {
            double rs, xs, ph, L, Q;
            point64(BA.node + sb, nbc, s, c0, c1, sv, guess, rs, xs, ph, L, Q);
            g64v = pos_num(Q) ? div_rn((3.0 * c1) * (1.0 - sv * sv), sqrt_rn(Q)) : 0.0;
          }
          ++n64;
          if (g64v > F) ++viol;
          if (F * u01(w.z, w.w) < g64v) { st = kSmpAccepted; break; }
        }
        if (t >= max_trials) t = max_trials;
        keys[p] = (res & 0xFFFFFFFF00000000ull) | ((uint64_t)st << 30) |
                  (uint64_t)(t & 0x3FFFFFFF);
      }
    }
  }
  const unsigned full = __activemask();
  const unsigned peers = __match_any_sync(full, c);
  const unsigned vi = __reduce_add_sync(peers, (unsigned)viol);
  const unsigned nf = __reduce_add_sync(peers, n64);
  if ((threadIdx.x & 31) == __ffs(peers) - 1 && c >= 0) {
    stat_add(S.stats, c, kStViolations, vi);
    stat_add(S.stats, c, kStFp64Trials, nf);
  }
}

template <bool kTaus, bool kExact>
__global__ void __launch_bounds__(128) k_pending64(Seg S, int max_trials, const uint32_t* id,
                                                   const uint32_t* step_p, BucketArgs BA,
                                                   const double4_32a* orb, uint64_t* keys,
                                                   const uint32_t* plist,
                                                   const uint32_t* pcount, int64_t n,
                                                   const double* Fx) {
  const uint32_t np = *pcount;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < np; i0 += gridDim.x * blockDim.x) {
    pending_star<kTaus, kExact>(S, max_trials, id, step_p, BA, orb, keys,
                                i0 + threadIdx.x < np ? (int64_t)plist[i0 + threadIdx.x] : n, n,
                                Fx);
  }
}

// the star's sort key and payload record; packed: the key's low 24 bits go
// to the record and the star's index in the segment takes their place
__device__ __forceinline__ void put_key(uint64_t* keys, Payload* pay, Payload& P, int64_t p,
                                        int64_t sb, uint64_t key, bool packed) {
  if (packed) {
    P.pad = (uint32_t)(key & kPackMask);
    key = (key & ~kPackMask) | (uint64_t)(p - sb);
  }
  keys[p] = key;
  pay[p] = P;
}

// kPrec: 0 FP64 by bisection (Appendix A's kernels: brackets, envelope and
// trials all on the FP64 table), 1 mixed (turning points from
// k_turning_mixed in tp_min, tp_max, FP32 sampler result from k_sample32 /
// k_pending64 in the key slot), 2 FP64 through the mixed kernels (their
// FP64 turning points, FP64 mode's envelope 1.2 Fx (Fx from k_env_eval), the
// accepted point as FP64 mode computes it).  kMinB: resident 256-thread
// blocks to fit (caps registers; 1 = no cap).
template <int kPrec, int kMinB, bool kTaus>
__global__ void __launch_bounds__(256, kMinB) k_orbit(Seg S, int max_trials, const double* r,
                                               const double* x, const double* phi,
                                               const double* Menc, const double* vr,
                                               const double* vt, const double* m,
                                               const uint32_t* id, const uint32_t* step_p,
                                               uint64_t* keys, Payload* pay, int64_t* esc,
                                               OrbitStageOut dbg, BucketArgs BA,
                                               const double* tp_min, const double* tp_max,
                                               const double4_32a* orb,
                                               int64_t n, const double* Rv, double* Rp,
                                               const double* Fx, const double* Av,
                                               double* Ap, bool packed) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c = seg_find(S.off, S.n_seg, p);
  const int64_t sb = S.off[c];
  const int64_t nbc = S.nb[c];
  const int64_t k = p - sb;
  const double rk = r[p], vrk = vr[p], vtk = vt[p];
  const uint32_t idk = id[p];
  Payload P;
  P.vr = vrk; P.vt = vtk; P.m = m[p]; P.r_old = rk; P.c = 0.0; P.id = idk; P.pad = 0;
  double r_new = rk, rmin = rk, rmax = rk, F = 0.0;
  int code = 0, trials = 0;
  unsigned long long viol = 0;
  bool escaped = false;

  if (Rp) Rp[p] = Rv[p];  // the stellar radius goes with the star
  if (Ap) Ap[p] = Av[p];  // and the binary's semi-major axis
  if (k >= nbc) {
    // escaped in an earlier step: stays at the end, ordered by id
    put_key(keys, pay, P, p, sb, radius_key(rk, idk), packed);
    if (dbg.code) dbg.code[p] = 1;
    return;
  }
  if (Rv && lt0(Rv[p])) {
    // merged into its partner in this step (sticky spheres): it leaves
    // with no mass, draws nothing, and carries off no energy
    put_key(keys, pay, P, p, sb, radius_key(__longlong_as_double(0x7FF0000000000000ll), idk),
            packed);
    if (dbg.code) dbg.code[p] = 1;
    const unsigned full = __activemask();
    const unsigned peers = __match_any_sync(full, c);
    if ((threadIdx.x & 31) == __ffs(peers) - 1)
      atomicAdd((unsigned long long*)(esc + c), (unsigned long long)__popc(peers));
    return;
  }
  const Table64 T{r + sb, x + sb, phi + sb, nbc};
  Star s;
  s.k = k;
  double c0o = 0.0, c1o = 0.0;
  if (kPrec >= 1) {
    // E, J, c0, c1 from the turning-point kernel
    const double4_32a o = orb[p];
    s.E = o.x;
    s.J = o.y;
    c0o = o.z;
    c1o = o.w;
  } else {
    s.E = __ldg(T.phi + k) + scale_down<1>(vrk * vrk + vtk * vtk);
    s.J = rk * vtk;
  }
  Draws<kTaus> g = draws_of<kTaus>(S, c, idk, *step_p);
  double ph_new = __ldg(T.phi + k);

  if (!lt0(s.E)) {
    escaped = true;
    code = 1;
    r_new = __longlong_as_double(0x7FF0000000000000ll);
    // energy carried off: the star's energy in the field of the others
    P.c = __ldg(T.phi + k) + div_rn(P.m, rk) + scale_down<1>(vrk * vrk + vtk * vtk);
  } else {
    int64_t jmax, jmin;
    Buckets BK;
    if (kPrec >= 1) {
      const int4 pr = BA.prm[c];
      BK.start = BA.start + BA.off[c];
      BK.base = BA.base[c];
      BK.shift = pr.x;
      BK.nbk = pr.y;
      BK.lo = pr.z;
      BK.hi = pr.w;
    }
    if (kPrec == 0) {
      jmax = bisect_rmax64(T, s);
      jmin = bisect_rmin64(T, s);
    } else if (dbg.rmin) {
      // turning points from k_turning_mixed (for the stage outputs)
      rmin = __ldg(tp_min + p);
      rmax = __ldg(tp_max + p);
    }
    if (kPrec == 0) {
      rmax = shell_root64(T, s, jmax, true);
      rmin = jmin < 0 ? central_root64(T, s) : shell_root64(T, s, jmin, false);
    }
    const double c0 = kPrec == 0 ? scale_down<1>(rmax + rmin) : c0o;
    const double c1 = kPrec == 0 ? scale_down<2>(rmax - rmin) : c1o;
    if (kPrec == 0) {
      double gmax = 0.0;
      for (int j = 0; j <= 20; ++j) {
        double rs, ph, Q;
        double g = g64(T, s, c0, c1, c_s64[j], rs, ph, Q);
        if (g > gmax) gmax = g;
      }
      F = 1.2 * gmax;
      if (!(rmax > rmin) || !(F > 0.0)) {
        code = 2;
      } else {
        code = 3;
        double rs_a = 0.0, ph_a = 0.0, Q_a = 0.0;
        for (int t = 0; t < max_trials; ++t) {
          U4 w = g.block(kTagRej, (uint32_t)t);
          const double Xp = u01(w.z, w.w);
          const double sv = sym_double(sym_int(w.x, w.y));  // 2 X - 1, exact
          double rs, ph, Q;
          const double g = g64(T, s, c0, c1, sv, rs, ph, Q);
          if (g > F) ++viol;
          if (F * Xp < g) {
            rs_a = rs;
            ph_a = ph;
            Q_a = Q;
            code = 0;
            trials = t + 1;
            break;
          }
        }
        if (code == 3) {
          trials = max_trials;
          draws_keep(S, c, g);
        } else {
          // the accepted point's velocities once the warp's lanes are done
          const double sq = sqrt_rn(Q_a);
          U4 sg = g.block(kTagSgn, 0u);
          draws_keep(S, c, g);
          r_new = rs_a;
          P.vr = (sg.x & 1u) ? -sq : sq;
          P.vt = div_rn(s.J, rs_a);
          P.c = __ldg(T.phi + k) - ph_a;
          ph_new = ph_a;
        }
      }
    } else {
      // the FP32 sampler's result (k_sample32); a pending star continues
      // its trial sequence here in FP64 from the trial near a turning point
      const uint64_t res = keys[p];
      const uint32_t st = (uint32_t)(res >> 30) & 3u;
      int t = (int)(res & 0x3FFFFFFFull);
      F = kPrec == 2 ? 1.2 * __ldg(Fx + p) : (double)__uint_as_float((uint32_t)(res >> 32));
      if (st == kSmpDegenerate) {
        code = 2;
      } else if (st == kSmpCap) {
        code = 3;
        trials = max_trials;
        g.skip((uint32_t)max_trials);
        draws_keep(S, c, g);
      } else {
        const float c0f = f32_rn(c0), c1f = f32_rn(c1);
        const int nb32 = (int)nbc;
        // (k_pending64 has resolved every pending star to accepted or cap)
        const bool acc = st == kSmpAccepted;
        if (!acc) {
          code = 3;
          trials = max_trials;
          g.skip((uint32_t)max_trials);
          draws_keep(S, c, g);
        } else {
          code = 0;
          trials = t + 1;
          // the accepted point in FP64 from the full 53-bit X, once per
          // star, with the warp's lanes together
          g.skip((uint32_t)t);  // stream mode: the rejected trials' blocks
          const U4 w = g.block(kTagRej, (uint32_t)t);
          const double sv = sym_double(sym_int(w.x, w.y));
          const int guess = shell32_of(BA.node + sb, nb32, BK, c0f, c1f, 2.0f * u01f(w.y) - 1.0f);
          double rs, ph, Q, vtn;
          if (kPrec == 2) {
            point64_div(BA.node + sb, nbc, s, c0, c1, sv, guess, rs, ph, Q, vtn);  // v_t = J / r
          } else {
            double xs;
            point64(BA.node + sb, nbc, s, c0, c1, sv, guess, rs, xs, ph, vtn, Q);
          }
          if (!pos_num(Q)) Q = 0.0;
          const double sq = sqrt_rn(Q);
          U4 sg = g.block(kTagSgn, 0u);
          draws_keep(S, c, g);
          r_new = rs;
          P.vr = (sg.x & 1u) ? -sq : sq;
          P.vt = vtn;
          P.c = __ldg(T.phi + k) - ph;
          ph_new = ph;
        }
      }
    }
  }
  put_key(keys, pay, P, p, sb, radius_key(r_new, idk), packed);

  // statistics: one atomic per counter per segment present in the warp
  const unsigned full = __activemask();
  const unsigned peers = __match_any_sync(full, c);
  const int lane = threadIdx.x & 31;
  const unsigned tr = __reduce_add_sync(peers, (unsigned)trials);
  const unsigned vi = __reduce_add_sync(peers, (unsigned)viol);
  const unsigned es = __reduce_add_sync(peers, escaped ? 1u : 0u);
  const unsigned dg = __reduce_add_sync(peers, code == 2 ? 1u : 0u);
  const unsigned cp = __reduce_add_sync(peers, code == 3 ? 1u : 0u);
  if (lane == __ffs(peers) - 1) {
    stat_add(S.stats, c, kStTrials, tr);
    stat_add(S.stats, c, kStViolations, vi);
    stat_add(S.stats, c, kStDegenerate, dg);
    stat_add(S.stats, c, kStCapHits, cp);
    if (es) atomicAdd((unsigned long long*)(esc + c), (unsigned long long)es);
  }
  if (dbg.phi_new) dbg.phi_new[p] = ph_new;
  if (dbg.rmin) dbg.rmin[p] = rmin;
  if (dbg.rmax) dbg.rmax[p] = rmax;
  if (dbg.F) dbg.F[p] = F;
  if (dbg.code) dbg.code[p] = code;
  if (dbg.trials) dbg.trials[p] = trials;
}

// Energy correction (section 2.1 step 6) in mixed mode, after the new
// potential and its bucket index: the shell of r_old in the new table from
// the index (FP32 1/r, moved to the exact FP64 shell by integer compares of
// the radii), Phi_new(r_old) = Phi_i + M_i (1/r_i - 1/r_old) from the
// enclosed mass of that shell (Eq. 6 without its division), then
// T' = T + 1/2 [(Phi_new(r_old) - Phi_new,k) - c] clamped at 0 and both
// velocity components scaled by sqrt(T'/T), as in the FP64 kernel.
// kDiv (FP64 mode): Phi_new(r_old) by Eq. 6's division form and the FP64
// kernel's comparisons, as the FP64 statement computes them, the shell found
// the same way (the shell of a radius is unique).
template <bool kDiv>
__global__ void __launch_bounds__(128, 12) k_correction_mixed(Seg S, const int64_t* esc,
                                                          const double* r, const double* x,
                                                          const double* phi,
                                                          const double* Menc, BucketArgs BA,
                                                          double* vr, double* vt,
                                                          const double* r_old, const double* cc,
                                                          const double* m, int64_t n) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c = seg_find(S.off, S.n_seg, p);
  const int64_t sb = __ldg(S.off + c);
  const int64_t nbc = S.nb[c] - esc[c];
  if (p - sb >= nbc) return;
  const double ro = r_old[p];
  const double xo = div_rn(1.0, ro);
  Buckets BK;
  const int4 pr = BA.prm[c];
  BK.start = BA.start + BA.off[c];
  BK.base = BA.base[c];
  BK.shift = pr.x;
  BK.nbk = pr.y;
  BK.lo = pr.z;
  BK.hi = pr.w;
  const float xq[1] = {f32_rn(xo)};
  int sh[1];
  shells32_bk<1>(NodeKeys{BA.node + sb}, (int)nbc, BK, xq, sh);
  double4_32a nd;
  const int64_t i = fix_shell_nodes(BA.node + sb, nbc, sh[0], ro, nd);
  double pn;
  if (!kDiv) {
    pn = i < 0 ? nd.z : nd.z + nd.w * (nd.y - xo);
  } else if (i < 0) {
    pn = nd.z;
  } else {
    double xj1 = 0.0, pj1 = 0.0;
    if (i + 1 < nbc) {
      const double4_32a nx = BA.node[sb + i + 1];
      xj1 = nx.y;
      pj1 = nx.z;
    }
    const double den = nd.y - xj1;
    pn = !(den > 0.0) ? nd.z : nd.z + div_rn(nd.y - xo, den) * (pj1 - nd.z);
  }
  const double a = vr[p], b = vt[p];
  const double Tk = scale_down<1>(a * a + b * b);
  const double dnew = pn - phi[p];
  double Tp = Tk + scale_down<1>(dnew - cc[p]);
  bool clamp = false;
  if (kDiv ? Tp < 0.0 : lt0(Tp)) {
    clamp_energy_add(S.stats, c, m[p], Tp);
    Tp = 0.0;
    clamp = true;
  }
  if (kDiv ? Tk > 0.0 : pos_num(Tk)) {
    const double f = sqrt_rn(div_rn(Tp, Tk));
    vr[p] = a * f;
    vt[p] = b * f;
  }
  if (clamp) stat_add(S.stats, c, kStClamps, 1ull);
}

// ------------------------------------------------------ potential grid
// Grid cells per segment: twice the stars, between 512 and 2^15.
int64_t grid_capacity(int64_t nc) {
  int64_t g = 2 * nc;
  if (g < 512) g = 512;  // p = 0 (a cell per binade) always fits
  if (g > (1 << 15)) g = 1 << 15;
  return g;
}

// per segment: the key range of 1/r over the bound stars, the finest 2^p
// cells per binade (p <= 10) that fit the capacity, Phi_0 and the bound
// mass (Phi = Phi_0 inside the first star; outside the last one Phi falls
// by M_bound per unit of 1/r)
__global__ void k_grid_params(Seg S, const int64_t* esc, bool sub, const double* x,
                              const double* phi, const double* Menc, const int64_t* goff,
                              int4* gprm, float4* gaux) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= S.n_seg) return;
  int64_t nb = S.nb[c];
  if (sub) nb -= esc[c];
  if (nb <= 0) { gprm[c] = make_int4(0, 0, 0, 0); gaux[c] = make_float4(0.f, 0.f, 0.f, 0.f); return; }
  const int64_t sb = S.off[c];
  const uint32_t klo = __float_as_uint((float)x[sb + nb - 1]);
  const uint32_t khi = __float_as_uint((float)x[sb]);
  const int64_t cap = goff[c + 1] - goff[c];
  int p = 10;
  while (p > 0 && (int64_t)((khi >> (23 - p)) - (klo >> (23 - p))) + 2 > cap) --p;
  const int sh = 23 - p;
  const uint32_t key0 = (klo >> sh) << sh;
  const int cells = (int)((khi - key0) >> sh) + 2;
  gprm[c] = make_int4((int)key0, sh, cells, (int)khi);
  gaux[c] = make_float4((float)phi[sb], (float)Menc[sb + nb - 1], __uint_as_float(key0), 0.f);
}

// The shell of every grid key, largest i with 1/r_i >= key (-1 when none),
// written by the stars (grid_shells_of) in one pass over stars and cells.
__global__ void k_grid_shells(Seg S, const int64_t* esc, bool sub, const double* x,
                              BucketArgs B, int* gshell, int64_t n) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c = seg_find(S.off, S.n_seg, p);
  int64_t nb = S.nb[c];
  if (sub) nb -= esc[c];
  const int64_t sb = S.off[c], k = p - sb;
  if (k >= nb) return;
  grid_shells_of(k, nb, __ldg(x + p), k + 1 < nb ? __ldg(x + p + 1) : 0.0, B.gprm[c],
                 gshell + B.goff[c]);
}

// Phi at every grid key from the FP64 table: Phi = Phi_i + M_i (1/r_i - 1/r)
// in the key's shell i (Eq. 6 with the enclosed-mass slope), Phi_0 inside
// the first star, rounded to float
// fused (launch_potential_tables): the slopes at the tile seams, which the
// potential kernel leaves, are computed here by n_tiles more threads (and
// locally where a cell needs one), and each segment's cell 0 fills Phi_0 and
// the bound mass into gaux
__global__ void k_grid_build(Seg S, const int64_t* esc, bool sub, const double* x,
                             const double* phi, double* Menc, BucketArgs B,
                             const int* gshell, float* gphi, float4* gaux, int64_t total,
                             bool fused, const double* r, double4_32a* node, int64_t n_tiles) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned am = __ballot_sync(0xFFFFFFFFu, p < total);
  if (p >= total) {
    const int64_t t = p - total;
    if (!fused || t >= n_tiles) return;
    const int cs = seg_find(S.tile_off, S.n_seg, t);
    const int64_t sbs = S.off[cs], nbs = S.nb[cs] - (sub ? esc[cs] : 0);
    const int64_t k = (t - S.tile_off[cs]) * kTile + kTile - 1;  // the tile's last star
    if (k + 1 >= nbs) return;
    const int64_t q = sbs + k;
    const double xj = x[q], pj = phi[q];
    const double w = div_rn(phi[q + 1] - pj, xj - x[q + 1]);
    Menc[q] = w;
    node[q] = make_double4_32a(r[q], xj, pj, w);
    return;
  }
  const int c = seg_find(B.goff, S.n_seg, p);
  const int4 pr = B.gprm[c];
  const int g = (int)(p - B.goff[c]);
  const int64_t sb = S.off[c];
  const int64_t nb = S.nb[c] - (sub ? esc[c] : 0);
  // shell i's slope (a seam's computed as the seam threads do)
  auto slope = [&](int64_t i) {
    if (fused && i % kTile == kTile - 1 && i + 1 < nb)
      return div_rn(__ldg(phi + sb + i + 1) - __ldg(phi + sb + i),
                    __ldg(x + sb + i) - __ldg(x + sb + i + 1));
    return __ldg(Menc + sb + i);
  };
  float rel = 0.0f;
  if (g < pr.z) {
    if (fused && g == 0) {
      gaux[c].x = (float)__ldg(phi + sb);
      gaux[c].y = (float)__ldg(Menc + sb + nb - 1);
    }
    const double xg = (double)__uint_as_float((uint32_t)pr.x + ((uint32_t)g << pr.y));
    const double xn = (double)__uint_as_float((uint32_t)pr.x + ((uint32_t)(g + 1) << pr.y));
    const int64_t lo = gshell[p];
    const double ph = lo < 0 ? __ldg(phi + sb)
                             : __ldg(phi + sb + lo) + slope(lo) * (__ldg(x + sb + lo) - xg);
    gphi[p] = (float)ph;
    // Phi is convex in 1/r (its slope -M(1/r) rises with 1/r), so inside the
    // cell [xg, xn] it lies below the chord by at most (xn - xg) dM / 4, dM
    // the mass of the stars in the cell; relative to |Phi(xg)|, the smallest
    // |Phi| of the cell, the largest over the segment's cells bounds the
    // grid's interpolation error (gaux.w; floats >= 0 order as their bits)
    if (g + 1 < pr.z && ph < 0.0) {
      const int64_t lo2 = gshell[p + 1];
      const double Ma = lo < 0 ? 0.0 : slope(lo);
      const double Mb = lo2 < 0 ? 0.0 : slope(lo2);
      const double dM = Ma - Mb;
      rel = (float)(((xn - xg) * (dM > 0.0 ? dM : 0.0) * 0.25) / -ph);
    }
  }
  // one atomic per segment present in the warp
  const unsigned grp = __match_any_sync(am, c);
  const unsigned mx = __reduce_max_sync(grp, __float_as_uint(rel));
  if ((threadIdx.x & 31) == (unsigned)(__ffs(grp) - 1) && mx)
    atomicMax(reinterpret_cast<unsigned int*>(&gaux[c].w), mx);
}

// Both tables' per-segment parameters from 1/r alone (before the potential
// kernel writes the tables): as k_bucket_params (its float keys are the
// floats nearest 1/r, as t32 holds them) and k_grid_params, with Phi_0 and
// the bound mass left to k_grid_build (fused)
__global__ void k_table_params(Seg S, const int64_t* esc, bool sub, const double* x,
                               const int64_t* boff, uint32_t* base, int4* prm,
                               const int64_t* goff, int4* gprm, float4* gaux) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= S.n_seg) return;
  int64_t nb = S.nb[c];
  if (sub) nb -= esc[c];
  if (nb <= 0) {
    base[c] = 0;
    prm[c] = make_int4(0, 0, 0, -1);
    gprm[c] = make_int4(0, 0, 0, 0);
    gaux[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int64_t sb = S.off[c];
  // buckets
  const int tail = nb >= 4096 ? (int)(nb >> 10) : 0;
  const int lo = tail, hi = (int)nb - 1 - tail;
  const uint32_t b0 = __float_as_uint(f32_rn(x[sb + lo]));
  const uint32_t b1 = __float_as_uint(f32_rn(x[sb + hi]));
  const uint32_t span = b0 >= b1 ? b0 - b1 : 0u;
  const int64_t bcap = boff[c + 1] - boff[c] - 1;
  int bs = 0;
  while ((int64_t)(span >> bs) + 1 > bcap) ++bs;
  base[c] = b0;
  prm[c] = make_int4(bs, (int)((span >> bs) + 1), lo, hi);
  // grid
  const uint32_t klo = __float_as_uint((float)x[sb + nb - 1]);
  const uint32_t khi = __float_as_uint((float)x[sb]);
  const int64_t gcap = goff[c + 1] - goff[c];
  int gp = 10;
  while (gp > 0 && (int64_t)((khi >> (23 - gp)) - (klo >> (23 - gp))) + 2 > gcap) --gp;
  const int sh = 23 - gp;
  const uint32_t key0 = (klo >> sh) << sh;
  const int cells = (int)((khi - key0) >> sh) + 2;
  gprm[c] = make_int4((int)key0, sh, cells, (int)khi);
  gaux[c] = make_float4(0.f, 0.f, __uint_as_float(key0), 0.f);
}

// per segment: the indexed node range lo..hi, base = bits(x_lo), the
// smallest shift that fits the key range into the segment's capacity, and
// the bucket count
__global__ void k_bucket_params(Seg S, const int64_t* esc, bool sub, const float2* t32,
                                BucketArgs B, uint32_t* base, int4* prm) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= S.n_seg) return;
  int64_t nb = S.nb[c];
  if (sub) nb -= esc[c];
  if (nb <= 0) { base[c] = 0; prm[c] = make_int4(0, 0, 0, -1); return; }
  const int64_t sb = S.off[c];
  const int tail = nb >= 4096 ? (int)(nb >> 10) : 0;
  const int lo = tail, hi = (int)nb - 1 - tail;
  const uint32_t b0 = __float_as_uint(t32[sb + lo].x);
  const uint32_t b1 = __float_as_uint(t32[sb + hi].x);
  const uint32_t span = b0 >= b1 ? b0 - b1 : 0u;
  const int64_t cap = B.off[c + 1] - B.off[c] - 1;  // buckets that fit
  int sh = 0;
  while ((int64_t)(span >> sh) + 1 > cap) ++sh;
  base[c] = b0;
  prm[c] = make_int4(sh, (int)((span >> sh) + 1), lo, hi);
}

// one thread per indexed star: it writes start[b] for the buckets between
// its predecessor's bucket and its own; the last one closes the table
__global__ void k_bucket_build(Seg S, const int64_t* esc, bool sub, const float2* t32,
                               BucketArgs B, int* start, int64_t n) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c = seg_find(S.off, S.n_seg, p);
  int64_t nb = S.nb[c];
  if (sub) nb -= esc[c];
  const int4 pr = B.prm[c];
  const int64_t k = p - S.off[c];
  if (k < pr.z || k > pr.w) return;
  bucket_starts_of(k, nb, pr, B.base[c], __float_as_uint(t32[p].x),
                   k == pr.z ? 0u : __float_as_uint(t32[p - 1].x), start + B.off[c],
                   B.off[c + 1] - B.off[c]);
}

// slope of Phi in 1/r across each shell of one table, for callers that
// have the potential but not the masses: (Phi_{k+1} - Phi_k)/(x_k - x_{k+1}),
// with Phi = 0 at 1/r = 0 beyond the last node
__global__ void k_slopes(int64_t n, const double* x, const double* phi, double* M) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double xj = x[k], pj = phi[k];
  const double xj1 = k + 1 < n ? x[k + 1] : 0.0, pj1 = k + 1 < n ? phi[k + 1] : 0.0;
  M[k] = div_rn(pj1 - pj, xj - xj1);
}

}  // namespace

void launch_slopes(int64_t n, const double* x, const double* phi, double* Menc,
                   cudaStream_t st) {
  if (n > 0) k_slopes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, phi, Menc);
}

cudaError_t alloc_buckets(BucketWork& B, const SegLayout& L, cudaStream_t st) {
  std::vector<int64_t> off(L.n_seg + 1, 0), goff(L.n_seg + 1, 0);
  for (int c = 0; c < L.n_seg; ++c) {
    const int64_t nc = L.h_off[c + 1] - L.h_off[c];
    off[c + 1] = off[c] + nc / 2 + 2;  // about two stars per bucket
    goff[c + 1] = goff[c] + grid_capacity(nc);
  }
  B.gcells = goff[L.n_seg];
  cudaError_t e;
  if ((e = cudaMallocAsync((void**)&B.start, sizeof(int) * off[L.n_seg], st))) return e;
  if ((e = cudaMallocAsync((void**)&B.off, sizeof(int64_t) * (L.n_seg + 1), st))) return e;
  if ((e = cudaMallocAsync((void**)&B.base, sizeof(uint32_t) * L.n_seg, st))) return e;
  if ((e = cudaMallocAsync((void**)&B.prm, sizeof(int4) * L.n_seg, st))) return e;
  if ((e = cudaMallocAsync((void**)&B.gphi, sizeof(float) * B.gcells, st))) return e;
  if ((e = cudaMallocAsync((void**)&B.gshell, sizeof(int) * B.gcells, st))) return e;
  if ((e = cudaMallocAsync((void**)&B.goff, sizeof(int64_t) * (L.n_seg + 1), st))) return e;
  if ((e = cudaMallocAsync((void**)&B.gprm, sizeof(int4) * L.n_seg, st))) return e;
  if ((e = cudaMallocAsync((void**)&B.gaux, sizeof(float4) * L.n_seg, st))) return e;
  if ((e = cudaMallocAsync((void**)&B.node, sizeof(double4_32a) * (L.n > 0 ? L.n : 1), st))) return e;
  if ((e = cudaMallocAsync((void**)&B.tdf, sizeof(float4) * (L.n > 0 ? L.n : 1), st))) return e;
  e = cudaMemcpyAsync(B.off, off.data(), sizeof(int64_t) * (L.n_seg + 1),
                      cudaMemcpyHostToDevice, st);
  if (!e)
    e = cudaMemcpyAsync(B.goff, goff.data(), sizeof(int64_t) * (L.n_seg + 1),
                        cudaMemcpyHostToDevice, st);
  if (e) return e;
  return cudaStreamSynchronize(st);  // off, goff live on this stack
}

void free_buckets(BucketWork& B, cudaStream_t st) {
  void* ps[] = {B.start, B.off, B.base, B.prm, B.gphi, B.gshell, B.goff, B.gprm, B.gaux, B.node,
                B.tdf};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, st);
  B = BucketWork();
}

void launch_grid(const SegLayout& L, const double* x, const double* phi, const double* Menc,
                 bool nb_sub, BucketWork& B, cudaStream_t st) {
  if (!L.n || !B.gcells) return;
  k_grid_params<<<(unsigned)((L.n_seg + 127) / 128), 128, 0, st>>>(
      L.dev(), L.esc_step, nb_sub, x, phi, Menc, B.goff, B.gprm, B.gaux);
  k_grid_shells<<<(unsigned)((L.n + 255) / 256), 256, 0, st>>>(L.dev(), L.esc_step, nb_sub, x,
                                                              B.args(), B.gshell, L.n);
  k_grid_build<<<(unsigned)((B.gcells + 255) / 256), 256, 0, st>>>(
      L.dev(), L.esc_step, nb_sub, x, phi, const_cast<double*>(Menc), B.args(), B.gshell,
      B.gphi, B.gaux, B.gcells, false, nullptr, nullptr, 0);
}

void launch_potential_tables(const SegLayout& L, const double* r, const double* x,
                             const double* m, double* tile_m, double* tile_mx, double* phi,
                             float2* t32, double* Menc, bool nb_sub, bool sums_ready,
                             BucketWork& B, cudaStream_t st) {
  if (!L.n) return;
  k_table_params<<<(unsigned)((L.n_seg + 127) / 128), 128, 0, st>>>(
      L.dev(), L.esc_step, nb_sub, x, B.off, B.base, B.prm, B.goff, B.gprm, B.gaux);
  TableOut T;
  T.start = B.start;
  T.boff = B.off;
  T.base = B.base;
  T.prm = B.prm;
  T.gshell = B.gshell;
  T.goff = B.goff;
  T.gprm = B.gprm;
  launch_potential(L, r, x, m, tile_m, tile_mx, phi, t32, Menc, nb_sub, st, B.node, B.tdf,
                   sums_ready, true, &T);
  const int64_t threads = B.gcells + L.n_tiles;
  k_grid_build<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      L.dev(), L.esc_step, nb_sub, x, phi, Menc, B.args(), B.gshell, B.gphi, B.gaux, B.gcells,
      true, r, B.node, L.n_tiles);
}

void launch_buckets(const SegLayout& L, const float2* t32, bool nb_sub, BucketWork& B,
                    cudaStream_t st) {
  if (!L.n) return;
  k_bucket_params<<<(unsigned)((L.n_seg + 127) / 128), 128, 0, st>>>(
      L.dev(), L.esc_step, nb_sub, t32, B.args(), B.base, B.prm);
  k_bucket_build<<<(unsigned)((L.n + 255) / 256), 256, 0, st>>>(L.dev(), L.esc_step, nb_sub,
                                                               t32, B.args(), B.start, L.n);
}

cudaError_t alloc_env(EnvWork& W, int64_t n, cudaStream_t st) {
  const int64_t m = n > 0 ? n : 1;
  W.cap = 2 * m + 1024;  // the pairs: 1.1 per star measured on Plummer models
  cudaError_t e = cudaMallocAsync((void**)&W.gmax, sizeof(double) * m, st);
  if (!e) e = cudaMallocAsync((void**)&W.star, sizeof(double4_32a) * m, st);
  if (!e) e = cudaMallocAsync((void**)&W.list, sizeof(uint64_t) * W.cap, st);
  if (!e) e = cudaMallocAsync((void**)&W.spill, sizeof(uint64_t) * m, st);
  if (!e) e = cudaMallocAsync((void**)&W.cnt, 2 * sizeof(unsigned long long), st);
  if (!e) {
    k_env_tables<<<1, 32, 0, st>>>();
    e = cudaGetLastError();
  }
  return e;
}

void free_env(EnvWork& W, cudaStream_t st) {
  void* ps[] = {W.gmax, W.star, W.list, W.spill, W.cnt};
  for (void* q : ps)
    if (q) cudaFreeAsync(q, st);
  W = EnvWork();
}

void launch_correction_mixed(const SegLayout& L, const double* r, const double* x,
                             const double* phi, const double* Menc,
                             const BucketArgs& ba, double* vr, double* vt, const double* r_old,
                             const double* c, const double* m, cudaStream_t st,
                             bool div_form) {
  if (!L.n) return;
  if (div_form)
    k_correction_mixed<true><<<(unsigned)((L.n + 127) / 128), 128, 0, st>>>(
        L.dev(), L.esc_step, r, x, phi, Menc, ba, vr, vt, r_old, c, m, L.n);
  else
    k_correction_mixed<false><<<(unsigned)((L.n + 127) / 128), 128, 0, st>>>(
        L.dev(), L.esc_step, r, x, phi, Menc, ba, vr, vt, r_old, c, m, L.n);
}

void launch_turning(const SegLayout& L, const double* r, const double* x, const double* phi,
                    const double* Menc, const double* vr, const double* vt,
                    const BucketArgs& ba, double* tp_min, double* tp_max, double4_32a* orb,
                    int block, cudaStream_t st) {
  if (!L.n) return;
  if (block <= 0) block = 64;
  const unsigned grid = (unsigned)((L.n + block - 1) / block);
  k_turning_mixed<5><<<grid, block, 0, st>>>(L.dev(), r, x, phi, Menc, vr, vt, ba, tp_min,
                                             tp_max, orb, L.n);
}

void launch_orbit(const SegLayout& L, int precision, int max_trials, const double* r,
                  const double* x, const double* phi, const double* Menc,
                  const double* vr, const double* vt, const double* m, const uint32_t* id,
                  const uint32_t* step,
                  uint64_t* keys, Payload* pay, const OrbitStageOut* dbg, int block,
                  int variant, const BucketArgs& ba, double* tp_min, double* tp_max,
                  uint32_t* plist, uint32_t* pcount, cudaStream_t st, bool with_turning,
                  const double* Rv, double* Rp, const EnvWork* env, const double* Av,
                  double* Ap, double4_32a* orb, bool packed) {
  if (!L.n) return;
  OrbitStageOut d;
  EnvWork W;
  if (env) W = *env;
  double* Fx = W.gmax;
  // the envelope's pairs, about 1.1 per star: one thread each (a grid for
  // 1.25 per star, striding over any more)
  const unsigned egrid = (unsigned)((L.n + L.n / 4 + kEnvThreads - 1) / kEnvThreads);
  if (dbg) d = *dbg;
  if (block <= 0) block = 64;
  const unsigned grid = (unsigned)((L.n + block - 1) / block);
  // the pending list is short: a grid of a few blocks per SM walks it
  const unsigned pgrid = (unsigned)((L.n + 127) / 128 < 1216 ? (L.n + 127) / 128 : 1216);
  // precision 0: FP64 through the mixed kernels (kPrec 2); 1 mixed; 2 FP64
  // by bisection (kPrec 0)
  const bool exact = precision == 0;
#define CMC_TURN(B)                                                                          \
  k_turning_mixed<5><<<grid, block, 0, st>>>(L.dev(), r, x, phi, Menc, vr, vt, ba,      \
                                             tp_min, tp_max, orb, L.n)
#define CMC_ORBIT(P, B, T)                                                                  \
  k_orbit<P, B, T><<<grid, block, 0, st>>>(L.dev(), max_trials, r, x, phi, Menc, vr, vt, \
                                           m, id, step, keys, pay, L.esc_step, d, ba, tp_min, \
                                           tp_max, orb, L.n, Rv, Rp, Fx, Av, Ap, packed)
#define CMC_SAMPLED(B, T, X)                                                                \
  do {                                                                                      \
    if (with_turning) CMC_TURN(B);                                                          \
    if (X) {                                                                                \
      cudaMemsetAsync(W.cnt, 0, 2 * sizeof(unsigned long long), st);                        \
      k_env_screen<<<(unsigned)((L.n + kEnvThreads - 1) / kEnvThreads), kEnvThreads, 0, st>>>( \
          L.dev(), ba, orb, W, L.n);                                                         \
      k_env_eval<<<egrid, kEnvThreads, 0, st>>>(L.dev(), ba, W);                             \
    }                                                                                       \
    cudaMemsetAsync(pcount, 0, sizeof(uint32_t), st);                                      \
    k_sample32<B, T, X><<<grid, block, 0, st>>>(L.dev(), max_trials, id, step, ba, orb, keys, \
                                                plist, pcount, L.n, Fx);                    \
    k_pending64<T, X><<<pgrid, 128, 0, st>>>(L.dev(), max_trials, id, step, ba, orb, keys,  \
                                             plist, pcount, L.n, Fx);                       \
    CMC_ORBIT(X ? 2 : 1, 5, T);                                                             \
  } while (0)
#define CMC_VARIANTS(X)                                                                     \
  do {                                                                                      \
    if (variant == 1) CMC_SAMPLED(2, false, X);                                             \
    else if (variant == 2) CMC_SAMPLED(3, false, X);                                        \
    else if (variant == 3) CMC_SAMPLED(4, false, X);                                        \
    else if (variant == 4) CMC_SAMPLED(5, false, X);                                        \
    else if (variant == 5) CMC_SAMPLED(6, false, X);                                        \
    else if (variant == 6) CMC_SAMPLED(8, false, X);                                        \
    else CMC_SAMPLED(1, false, X);                                                          \
  } while (0)
  if (precision == 2) {
    if (L.taus) CMC_ORBIT(0, 1, true);
    else CMC_ORBIT(0, 1, false);
  } else if (L.taus) {
    // stream mode: one launch shape of the sampler
    if (exact) CMC_SAMPLED(5, true, true);
    else CMC_SAMPLED(5, true, false);
  } else if (exact) {
    CMC_VARIANTS(true);
  } else {
    CMC_VARIANTS(false);
  }
#undef CMC_VARIANTS
#undef CMC_SAMPLED
#undef CMC_TURN
#undef CMC_ORBIT
}

CMC_DEBUG_SITE_ACCESSOR

}  // namespace cmc
