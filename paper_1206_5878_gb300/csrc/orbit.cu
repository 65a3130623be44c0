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
// tests run in FP32 on an interleaved float2 (1/r, Phi) table; the
// brackets are then verified (and moved if needed) in FP64, the turning
// points are the FP64 shell roots, and the accepted radius, its potential
// and the velocities are recomputed in FP64.  A mixed result equals the
// FP64 result whenever both accept the same trial.
#include "cmc_host.hpp"

namespace cmc {

namespace {

struct Star {
  double E, J;
  int64_t k;
};

__device__ __forceinline__ double Q_node64(const Table64& T, const Star& s, int64_t i) {
  double L = s.J * __ldg(T.x + i);
  return 2.0 * (s.E - __ldg(T.phi + i)) - L * L;
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
  const double B = (pj1 - pj) / (xj - xj1);
  const double A = pj + B * xj;
  double D = B * B + 2.0 * (s.J * s.J) * (s.E - A);
  if (!(D > 0.0)) D = 0.0;
  const double sD = sqrt(D);
  double root = outer ? (B + sD) / (2.0 * (A - s.E)) : (s.J * s.J) / (B + sD);
  if (!(root >= rj)) root = rj;
  if (has_next && root > rj1) root = rj1;
  return root;
}

__device__ __forceinline__ double central_root64(const Table64& T, const Star& s) {
  double rmin = s.J / sqrt(2.0 * (s.E - __ldg(T.phi)));
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
  const double L = st.J / rs;
  Q = 2.0 * (st.E - ph) - L * L;
  if (!(Q > 0.0)) return 0.0;
  return drds / sqrt(Q);
}

// ------------------------------------------------------------ FP32 side
struct Table32 {
  const float2* t;  // (1/r, Phi) per node
  int64_t nb;
};

__device__ __forceinline__ float Q_node32(const Table32& T, float E, float J, int64_t i) {
  const float2 e = __ldg(T.t + i);
  const float L = J * e.x;
  return 2.0f * (E - e.y) - L * L;
}

// largest i with 1/r_i >= xq (FP32), else -1
__device__ __forceinline__ int64_t shell_of32(const Table32& T, float xq) {
  int64_t lo = -1, hi = T.nb;
  while (hi - lo > 1) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(&T.t[mid].x) >= xq) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ float phi_in_shell32(const Table32& T, int64_t i, float xq) {
  if (i < 0) return __ldg(&T.t[0].y);
  const float2 a = __ldg(T.t + i);
  float2 b = make_float2(0.0f, 0.0f);
  if (i + 1 < T.nb) b = __ldg(T.t + i + 1);
  const float den = a.x - b.x;
  if (!(den > 0.0f)) return a.y;
  return a.y + ((a.x - xq) / den) * (b.y - a.y);
}

__device__ __forceinline__ float g32(const Table32& T, float E, float J, float c0, float c1,
                                     float s, int64_t& shell) {
  const float rs = c0 + c1 * (s * (3.0f - s * s));
  const float drds = (3.0f * c1) * (1.0f - s * s);
  const float xq = 1.0f / rs;
  shell = shell_of32(T, xq);
  const float ph = phi_in_shell32(T, shell, xq);
  const float L = J * xq;
  const float Q = 2.0f * (E - ph) - L * L;
  if (!(Q > 0.0f)) return 0.0f;
  return drds / sqrtf(Q);
}

// move an approximate shell index to the exact FP64 one: largest i with
// r_i <= q (bounded walk, then plain bisection)
__device__ __forceinline__ int64_t fix_shell64(const Table64& T, int64_t i, double q) {
  if (i < -1) i = -1;
  if (i >= T.nb) i = T.nb - 1;
  for (int w = 0; w < 64; ++w) {
    if (i + 1 < T.nb && __ldg(T.r + i + 1) <= q) { ++i; continue; }
    if (i >= 0 && __ldg(T.r + i) > q) { --i; continue; }
    return i;
  }
  return shell_of(T, q);
}

// FP32 bracket -> FP64 bracket for r_max: node lo has Q >= 0 (or is the
// star), node lo+1 has Q < 0 (or is the virtual node nb)
__device__ __forceinline__ int64_t verify_rmax(const Table64& T, const Star& s, int64_t j) {
  if (j < s.k) j = s.k;
  if (j > T.nb - 1) j = T.nb - 1;
  for (int w = 0; w < 64; ++w) {
    if (j + 1 < T.nb && !(Q_node64(T, s, j + 1) < 0.0)) { ++j; continue; }
    if (j > s.k && Q_node64(T, s, j) < 0.0) { --j; continue; }
    return j;
  }
  return bisect_rmax64(T, s);
}

// r_min: node lo has Q < 0 (or is -1), node lo+1 has Q >= 0 (or is the star)
__device__ __forceinline__ int64_t verify_rmin(const Table64& T, const Star& s, int64_t j) {
  if (j < -1) j = -1;
  if (j > s.k - 1) j = s.k - 1;
  for (int w = 0; w < 64; ++w) {
    if (j + 1 < s.k && Q_node64(T, s, j + 1) < 0.0) { ++j; continue; }
    if (j >= 0 && !(Q_node64(T, s, j) < 0.0)) { --j; continue; }
    return j;
  }
  return bisect_rmin64(T, s);
}

template <int kPrec>
__global__ void __launch_bounds__(256) k_orbit(Seg S, int max_trials, const double* r,
                                               const double* x, const double* phi,
                                               const float2* t32, const double* vr,
                                               const double* vt, const double* m,
                                               const uint32_t* id, const uint32_t* step_p,
                                               uint64_t* keys, Payload* pay, int64_t* esc,
                                               OrbitStageOut dbg, int64_t n) {
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

  if (k >= nbc) {
    // escaped in an earlier step: stays at the end, ordered by id
    keys[p] = radius_key(rk, idk);
    pay[p] = P;
    if (dbg.code) dbg.code[p] = 1;
    return;
  }
  const Table64 T{r + sb, x + sb, phi + sb, nbc};
  Star s;
  s.k = k;
  s.E = __ldg(T.phi + k) + 0.5 * (vrk * vrk + vtk * vtk);
  s.J = rk * vtk;
  const uint64_t seed = S.seed[c];
  const uint32_t step = *step_p;
  double ph_new = __ldg(T.phi + k);

  if (!(s.E < 0.0)) {
    escaped = true;
    code = 1;
    r_new = __longlong_as_double(0x7FF0000000000000ll);
  } else {
    int64_t jmax, jmin;
    Table32 T32{t32 + sb, nbc};
    const float E32 = (float)s.E, J32 = (float)s.J;
    if (kPrec == 0) {
      jmax = bisect_rmax64(T, s);
      jmin = bisect_rmin64(T, s);
    } else {
      int64_t lo = k, hi = nbc;
      while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (Q_node32(T32, E32, J32, mid) < 0.0f) hi = mid; else lo = mid;
      }
      jmax = verify_rmax(T, s, lo);
      lo = -1; hi = k;
      while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (Q_node32(T32, E32, J32, mid) < 0.0f) lo = mid; else hi = mid;
      }
      jmin = verify_rmin(T, s, lo);
    }
    rmax = shell_root64(T, s, jmax, true);
    rmin = jmin < 0 ? central_root64(T, s) : shell_root64(T, s, jmin, false);
    const double c0 = 0.5 * (rmax + rmin);
    const double c1 = 0.25 * (rmax - rmin);
    if (kPrec == 0) {
      double gmax = 0.0;
      for (int j = 0; j <= 20; ++j) {
        double sj = -1.0 + ((double)j + 0.5) / 10.5, rs, ph, Q;
        double g = g64(T, s, c0, c1, sj, rs, ph, Q);
        if (g > gmax) gmax = g;
      }
      F = 1.2 * gmax;
      if (!(rmax > rmin) || !(F > 0.0)) {
        code = 2;
      } else {
        code = 3;
        for (int t = 0; t < max_trials; ++t) {
          U4 w = philox(idk, step, kTagRej, (uint32_t)t, seed);
          const double X = u01(w.x, w.y), Xp = u01(w.z, w.w);
          const double sv = 2.0 * X - 1.0;
          double rs, ph, Q;
          const double g = g64(T, s, c0, c1, sv, rs, ph, Q);
          if (g > F) ++viol;
          if (F * Xp < g) {
            const double sq = sqrt(Q);
            U4 sg = philox(idk, step, kTagSgn, 0u, seed);
            r_new = rs;
            P.vr = (sg.x & 1u) ? -sq : sq;
            P.vt = s.J / rs;
            P.c = __ldg(T.phi + k) - ph;
            ph_new = ph;
            code = 0;
            trials = t + 1;
            break;
          }
        }
        if (code == 3) trials = max_trials;
      }
    } else {
      const float c0f = (float)c0, c1f = (float)c1;
      float gmax = 0.0f;
      for (int j = 0; j <= 20; ++j) {
        const float sj = (float)(-1.0 + ((double)j + 0.5) / 10.5);
        int64_t sh;
        const float g = g32(T32, E32, J32, c0f, c1f, sj, sh);
        if (g > gmax) gmax = g;
      }
      const float F32 = 1.2f * gmax;
      F = (double)F32;
      if (!(rmax > rmin) || !(F32 > 0.0f)) {
        code = 2;
      } else {
        code = 3;
        for (int t = 0; t < max_trials; ++t) {
          U4 w = philox(idk, step, kTagRej, (uint32_t)t, seed);
          const double X = u01(w.x, w.y), Xp = u01(w.z, w.w);
          const double sv = 2.0 * X - 1.0;
          int64_t sh;
          const float g = g32(T32, E32, J32, c0f, c1f, (float)sv, sh);
          if (g > F32) ++viol;
          if (F32 * (float)Xp < g) {
            // recompute the accepted point in FP64
            const double rs = c0 + c1 * (sv * (3.0 - sv * sv));
            const int64_t i64 = fix_shell64(T, sh, rs);
            const double ph = phi_in_shell(T, i64, rs);
            const double L = s.J / rs;
            double Q = 2.0 * (s.E - ph) - L * L;
            if (!(Q > 0.0)) Q = 0.0;
            const double sq = sqrt(Q);
            U4 sg = philox(idk, step, kTagSgn, 0u, seed);
            r_new = rs;
            P.vr = (sg.x & 1u) ? -sq : sq;
            P.vt = s.J / rs;
            P.c = __ldg(T.phi + k) - ph;
            ph_new = ph;
            code = 0;
            trials = t + 1;
            break;
          }
        }
        if (code == 3) trials = max_trials;
      }
    }
  }
  keys[p] = radius_key(r_new, idk);
  pay[p] = P;

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

}  // namespace

void launch_orbit(const SegLayout& L, int precision, int max_trials, const double* r,
                  const double* x, const double* phi, const float2* t32, const double* vr,
                  const double* vt, const double* m, const uint32_t* id, const uint32_t* step,
                  uint64_t* keys, Payload* pay, const OrbitStageOut* dbg, int block,
                  cudaStream_t st) {
  if (!L.n) return;
  OrbitStageOut d;
  if (dbg) d = *dbg;
  if (block <= 0) block = 128;
  const unsigned grid = (unsigned)((L.n + block - 1) / block);
  if (precision == 1)
    k_orbit<1><<<grid, block, 0, st>>>(L.dev(), max_trials, r, x, phi, t32, vr, vt, m, id, step,
                                       keys, pay, L.esc_step, d, L.n);
  else
    k_orbit<0><<<grid, block, 0, st>>>(L.dev(), max_trials, r, x, phi, t32, vr, vt, m, id, step,
                                       keys, pay, L.esc_step, d, L.n);
}

}  // namespace cmc
