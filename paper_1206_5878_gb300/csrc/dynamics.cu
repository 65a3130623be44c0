// Relaxation timestep (Eq. 7 on fixed bins of consecutive stars, section
// 3.3) and two-body relaxation between radial neighbours (section 2.1 step
// 3(i)).  Both are FP64 and evaluate, operation for operation, the same
// expressions as the independent FP64 statement of the method.
#include "cmc_host.hpp"

namespace cmc {

namespace {

// One thread per bin slot.  Bin b of a segment covers sorted positions
// [b*bs, min((b+1)*bs, nb)).  For P >= 2 stars:
//   n = 3 (P-1) / (4 pi (r_last^3 - r_first^3))
//   <v_rel> = mean over pairs (2j, 2j+1) of sqrt(v1^2 + v2^2)
//   <(M1+M2)^2> = mean over the same pairs of (m1 + m2)^2
//   T_b = pref <v_rel>^3 / (lnL n <(M1+M2)^2>),  pref = (theta_max/(pi/2)) (pi/32)
// and the segment's timestep is the minimum of T_b.
__global__ void __launch_bounds__(256) k_bins(Seg S, int bs, double pref, const double* r,
                                              const double* vr, const double* vt,
                                              const double* m, double* nbin) {
  __shared__ unsigned long long s_min[8];
  __shared__ int s_seg0;
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b0 = (int64_t)blockIdx.x * blockDim.x;
  if (threadIdx.x == 0) s_seg0 = seg_find(S.bin_off, S.n_seg, b0);
  __syncthreads();
  unsigned long long tb = 0x7FF0000000000000ull;  // +inf
  int c = s_seg0;
  if (b < S.bin_off[S.n_seg]) {
    c = seg_find(S.bin_off, S.n_seg, b);
    const int64_t lb = b - S.bin_off[c];
    const int64_t sb = S.off[c];
    const int64_t nbc = S.nb[c];
    const int64_t first = lb * bs;
    double n = 0.0;
    if (first < nbc) {
      int64_t P = nbc - first < bs ? nbc - first : bs;
      if (P >= 2) {
        const int64_t g = sb + first;
        double rf = r[g], rl = r[g + P - 1];
        double vol = rl * rl * rl - rf * rf * rf;
        if (vol > 0.0) {
          n = div_rn(3.0 * (double)(P - 1), (4.0 * kPi) * vol);
          int64_t q = P / 2;
          double sv = 0.0, sm = 0.0;
          for (int64_t j = 0; j < q; ++j) {
            int64_t a = g + 2 * j;
            double va2 = vr[a] * vr[a] + vt[a] * vt[a];
            double vb2 = vr[a + 1] * vr[a + 1] + vt[a + 1] * vt[a + 1];
            double ms = m[a] + m[a + 1];
            sv = sv + sqrt_rn(va2 + vb2);
            sm = sm + ms * ms;
          }
          double v = div_rn(sv, (double)q);
          double msq = div_rn(sm, (double)q);
          double num = pref * (v * v * v);
          double den = (S.lnL[c] * n) * msq;
          if (den > 0.0) {
            double T = div_rn(num, den);
            if (T < __longlong_as_double(0x7FF0000000000000ll))
              tb = (unsigned long long)__double_as_longlong(T);
          }
        }
      }
    }
    nbin[b] = n;
    // an outside bound on the segment's timestep (Eq. 11's stellar-evolution
    // step, say), with its first bin
    if (lb == 0 && S.dt_cap) {
      const double cap = S.dt_cap[c];
      if (cap > 0.0 && cap < __longlong_as_double(0x7FF0000000000000ll)) {
        const unsigned long long cb = (unsigned long long)__double_as_longlong(cap);
        tb = cb < tb ? cb : tb;
      }
    }
  }
  // positive doubles order like their bit patterns: min over the block for
  // the block's first segment, direct atomics for any other segment
  unsigned long long mine = (c == s_seg0) ? tb : 0x7FF0000000000000ull;
  if (c != s_seg0 && tb != 0x7FF0000000000000ull)
    atomicMin((unsigned long long*)(S.dt_bits + c), tb);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long y = __shfl_down_sync(0xffffffffu, mine, o);
    mine = y < mine ? y : mine;
  }
  if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = mine;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long v = s_min[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = s_min[w] < v ? s_min[w] : v;
    if (v != 0x7FF0000000000000ull) atomicMin((unsigned long long*)(S.dt_bits + s_seg0), v);
  }
}

// One thread per pair slot: stars a = 2j and b = 2j + 1 of a segment.  The
// pair's random draws come from its first star (counters keyed by its id,
// or its stream, kept after the draws).  kMinB: resident 128-thread blocks
// to fit per SM (caps the registers; 1 = no cap), a launch shape only.
//
// With stellar radii (col.R) the pair may merge instead (sticky spheres,
// section 2.1 step 3(iii)): with probability n pi (R1 + R2)^2 (1 + 2 G
// (m1 + m2) / ((R1 + R2) |w|^2)) |w| dt, decided by one draw of the pair
// after the azimuth psi, star a takes the total mass, the pair's 3-D
// momentum and the radius (R1^3 + R2^3)^(1/3); star b gets mass 0 and
// radius -1 (it leaves in the orbit step).  The merger's change of K + W,
// -(m1 m2 / (m1 + m2)) |w|^2 / 2 + m_b (Phi_a - Phi_b) + m_a m_b / r_a,
// is counted (fixed point, 2^-62).
struct Collide {
  double* R = nullptr;        // stellar radii (null: no collisions)
  const double* r = nullptr;  // the current radii and potential
  const double* phi = nullptr;
};

template <bool kTaus, int kMinB, bool kCol>
__global__ void __launch_bounds__(128, kMinB) k_relax(Seg S, int bs, double* vr, double* vt,
                                               double* m, const uint32_t* id,
                                               const double* nbin, const uint32_t* step_p,
                                               Collide col) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= S.pair_off[S.n_seg]) return;
  const int c = seg_find(S.pair_off, S.n_seg, p);
  const int64_t j = p - S.pair_off[c];
  const int64_t la = 2 * j;
  if (la + 1 >= S.nb[c]) return;
  const int64_t a = S.off[c] + la, b = a + 1;
  if (!CMC_IN(S.bin_off[c] + la / bs, S.bin_off[c + 1])) return;
  const double n = nbin[S.bin_off[c] + la / bs];
  const double m1 = m[a], m2 = m[b];
  const double msum = m1 + m2;
  const double dt = __longlong_as_double((long long)S.dt_bits[c]);
  const double lnL = S.lnL[c];
  // no density, no mass, or no positive Coulomb logarithm: no deflection
  if (!pos_num(n) || !pos_num(msum) || !pos_num(lnL) || !lt_inf(dt)) return;
  Draws<kTaus> g = draws_of<kTaus>(S, c, id[a], *step_p);
  int fails = 0;
  double cpsi, spsi, cphi, sphi;
  if (!disk_angle(g, kTagPsi, cpsi, spsi)) ++fails;
  const double v1x = vr[a], v1y = vt[a], v1z = 0.0;
  const double v2x = vr[b], vtb = vt[b];
  const double v2y = vtb * cpsi, v2z = vtb * spsi;
  const double wx = v1x - v2x, wy = v1y - v2y, wz = v1z - v2z;
  const double w2 = (wx * wx + wy * wy) + wz * wz;
  if (!pos_num(w2)) {
    draws_keep(S, c, g);
    if (fails) stat_add(S.stats, c, kStAngleFails, (unsigned long long)fails);
    return;
  }
  const double w = sqrt_rn_nl(w2);
  if (kCol) {
    const double R1 = col.R[a], R2 = col.R[b];
    if (R1 + R2 > 0.0) {
      const double Rs = R1 + R2;
      const double focus = 1.0 + div_rn_nl(2.0 * msum, Rs * w2);
      const double sig = (kPi * (Rs * Rs)) * focus;
      const double Pc = ((sig * n) * w) * dt;
      const U4 cw = g.block(kTagCol, 0u);
      if (u01(cw.x, cw.y) < Pc) {
        const double vcx = div_rn_nl(m1 * v1x + m2 * v2x, msum);
        const double vcy = div_rn_nl(m1 * v1y + m2 * v2y, msum);
        const double vcz = div_rn_nl(m1 * v1z + m2 * v2z, msum);
        const double dW = m2 * (col.phi[a] - col.phi[b]) + div_rn_nl(m1 * m2, col.r[a]);
        const double dK = (0.5 * div_rn_nl(m1 * m2, msum)) * w2;
        draws_keep(S, c, g);
        vr[a] = vcx;
        vt[a] = sqrt_rn_nl(vcy * vcy + vcz * vcz);
        m[a] = m1 + m2;
        col.R[a] = cbrt_newton(R1 * R1 * R1 + R2 * R2 * R2);
        m[b] = 0.0;
        col.R[b] = -1.0;
        stat_add(S.stats, c, kStCollisions, 1ull);
        const long long e = __double2ll_rn((dW - dK) * 4611686018427387904.0);  // 2^62
        stat_add(S.stats, c, kStCollisionEnergy, (unsigned long long)e);
        if (fails) stat_add(S.stats, c, kStAngleFails, (unsigned long long)fails);
        return;
      }
    }
  }
  // sin^2(beta/2) = min(1, 2 pi G^2 (m1+m2)^2 n lnL dt / |w|^3)
  double num = (2.0 * kPi) * msum;
  num = num * msum;
  num = num * n;
  num = num * lnL;
  num = num * dt;
  double s2 = div_rn_nl(num, w2 * w);
  if (!le1(s2)) s2 = 1.0;
  // cos(beta) = 1 - 2 sin^2(beta/2), sin(beta) = 2 sin(beta/2) cos(beta/2)
  const double cosb = 1.0 - scale_up<1>(s2);
  const double sinb = scale_up<1>(sqrt_rn_nl(s2)) * sqrt_rn_nl(1.0 - s2);
  if (!disk_angle(g, kTagPhi, cphi, sphi)) ++fails;
  draws_keep(S, c, g);
  // e1 = (w x xhat)/|w x xhat| = (0, wz, -wy)/|.| (yhat for radial w);
  // u = w x e1 has length |w| and completes the frame perpendicular to w
  const double wp2 = wy * wy + wz * wz;
  double e1y, e1z;
  if (pos_num(wp2)) {
    const double wp = sqrt_rn_nl(wp2);
    e1y = div_rn_nl(wz, wp);
    e1z = div_rn_nl(-wy, wp);
  } else {
    e1y = 1.0;
    e1z = 0.0;
  }
  const double ux = wy * e1z - wz * e1y;
  const double uy = -(wx * e1z);
  const double uz = wx * e1y;
  const double a1 = w * cphi;
  // w' = w cos(beta) + sin(beta) (|w| cos(phi) e1 + sin(phi) u)
  const double wpx = wx * cosb + sinb * (sphi * ux);
  const double wpy = wy * cosb + sinb * (a1 * e1y + sphi * uy);
  const double wpz = wz * cosb + sinb * (a1 * e1z + sphi * uz);
  const double dwx = wpx - wx, dwy = wpy - wy, dwz = wpz - wz;
  // the mass ratios as quotients; these products on the integer pipes
  // balance the FP64 pipe's load against the integer pipes' (measured: all
  // of the kernel's products there made it a third slower, none of them 2%
  // slower)
  const double f1 = div_rn_nl(m2, msum), f2 = div_rn_nl(m1, msum);
  const double p1x = v1x + mul_rn(f1, dwx), p1y = v1y + mul_rn(f1, dwy), p1z = v1z + mul_rn(f1, dwz);
  const double p2x = v2x - mul_rn(f2, dwx), p2y = v2y - mul_rn(f2, dwy), p2z = v2z - mul_rn(f2, dwz);
  vr[a] = p1x;
  vt[a] = sqrt_rn_nl(p1y * p1y + p1z * p1z);
  vr[b] = p2x;
  vt[b] = sqrt_rn_nl(p2y * p2y + p2z * p2z);
  if (fails) stat_add(S.stats, c, kStAngleFails, (unsigned long long)fails);
}

// Starting states of the Tausworthe streams: slot e of segment c (id =
// e - base[c]) gets T^(id 2^80) of the segment's seeded words, T^(id 2^80)
// as the product of the matrices P_b = T^(2^(80 + b)) over the bits of id.
// P: [4 components][32 bits b][32 columns], a column = the image of one bit.
__global__ void k_taus_init(int64_t slots, int n_seg, const int64_t* base, const uint4* words,
                            const uint32_t* P, uint4* table) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= slots) return;
  const int c = seg_find(base, n_seg, e);
  const uint64_t idv = (uint64_t)(e - base[c]);
  const uint4 w = words[c];
  uint32_t v[4] = {w.x, w.y, w.z, w.w};
  for (int j = 0; j < 4; ++j)
    for (int b = 0; b < 32; ++b) {
      if (!((idv >> b) & 1ull)) continue;
      const uint32_t* col = P + ((size_t)j * 32 + b) * 32;
      uint32_t r = 0u;
      for (int i = 0; i < 32; ++i)
        if ((v[j] >> i) & 1u) r ^= __ldg(col + i);
      v[j] = r;
    }
  table[e] = make_uint4(v[0], v[1], v[2], v[3]);
}

// The timesteps over the innermost P = min(300, nb) bound stars of each
// segment (one thread per segment summing in star order, as the FP64
// statement of the method does), into the segment's timestep (the minimum
// with Eq. 7's).  With stellar radii R, Eq. 8's collision timestep
//   1 / T_coll = 16 sqrt(pi) n_s <R^2> sigma (1 + G <M R> / (2 sigma^2 <R^2>)),
// n_s = 3 (P - 1) / (4 pi (r_{P-1}^3 - r_0^3)), sigma^2 = <v_r^2 + v_t^2> / 3.
// With binaries (semi-major axes A > 0, the star's mass the binary's),
// Eqs. 9 and 10:
//   1 / T_bb = 16 sqrt(pi) n_b X_bb^2 <a^2> sigma (1 + G <M a> / (2 sigma^2 X_bb <a^2>))
//   1 / T_bs = 4 sqrt(pi) n_s X_bs^2 <a^2> sigma (1 + G <M> <a> / (sigma^2 X_bs <a^2>))
// with n_b, n_s the central density times the binaries' and singles' shares
// of the P stars, <a^2>, <M a>, <a> over the binaries, <M> over all P.
__global__ void k_tcentral(Seg S, const double* r, const double* vr, const double* vt,
                           const double* m, const double* R, const double* A, double x_bb,
                           double x_bs) {
  const int c = blockIdx.x;
  if (threadIdx.x != 0 || c >= S.n_seg) return;
  const int64_t nb = S.nb[c], sb = S.off[c];
  const int64_t P = nb < 300 ? nb : 300;
  if (P < 2) return;
  const double* rr = r + sb;
  const double vol = rr[P - 1] * rr[P - 1] * rr[P - 1] - rr[0] * rr[0] * rr[0];
  if (!(vol > 0.0)) return;
  const double ns = (3.0 * (double)(P - 1)) / ((4.0 * kPi) * vol);
  const double inf = __longlong_as_double(0x7FF0000000000000ll);
  double Tmin = inf;
  if (R) {
    double sv = 0.0, sr = 0.0, smr = 0.0;
    for (int64_t k = 0; k < P; ++k) {
      const int64_t p = sb + k;
      sv = sv + (vr[p] * vr[p] + vt[p] * vt[p]);
      sr = sr + R[p] * R[p];
      smr = smr + m[p] * R[p];
    }
    const double sig2 = (sv / (double)P) / 3.0;
    const double R2 = sr / (double)P;
    const double MR = smr / (double)P;
    if (R2 > 0.0 && sig2 > 0.0) {
      const double sig = sqrt(sig2);
      double inv = (((16.0 * sqrt(kPi)) * ns) * R2) * sig;
      inv = inv * (1.0 + MR / ((2.0 * sig2) * R2));
      const double T = 1.0 / inv;
      if (T < Tmin) Tmin = T;
    }
  }
  if (A) {
    int64_t nbin = 0;
    double sv = 0.0, sm = 0.0, sa = 0.0, sa2 = 0.0, sma = 0.0;
    for (int64_t k = 0; k < P; ++k) {
      const int64_t p = sb + k;
      sv = sv + (vr[p] * vr[p] + vt[p] * vt[p]);
      sm = sm + m[p];
      if (A[p] > 0.0) {
        nbin += 1;
        sa = sa + A[p];
        sa2 = sa2 + A[p] * A[p];
        sma = sma + m[p] * A[p];
      }
    }
    const double sig2 = (sv / (double)P) / 3.0;
    if (nbin > 0 && sig2 > 0.0) {
      const double sig = sqrt(sig2);
      const double a2 = sa2 / (double)nbin, ma = sma / (double)nbin, am = sa / (double)nbin;
      const double mm = sm / (double)P;
      const double nbd = ns * ((double)nbin / (double)P);
      const double nsd = ns * ((double)(P - nbin) / (double)P);
      if (nbin < P) {
        double inv = (((4.0 * sqrt(kPi)) * nsd) * ((x_bs * x_bs) * a2)) * sig;
        inv = inv * (1.0 + (mm * am) / ((sig2 * x_bs) * a2));
        const double T = 1.0 / inv;
        if (T < Tmin) Tmin = T;
      }
      double inv = (((16.0 * sqrt(kPi)) * nbd) * ((x_bb * x_bb) * a2)) * sig;
      inv = inv * (1.0 + ma / (((2.0 * sig2) * x_bb) * a2));
      const double T = 1.0 / inv;
      if (T < Tmin) Tmin = T;
    }
  }
  if (Tmin < inf)
    atomicMin((unsigned long long*)(S.dt_bits + c), (unsigned long long)__double_as_longlong(Tmin));
}

}  // namespace

void launch_taus_init(int64_t slots, int n_seg, const int64_t* base, const uint4* words,
                      const uint32_t* P, uint4* table, cudaStream_t st) {
  if (slots > 0)
    k_taus_init<<<(unsigned)((slots + 255) / 256), 256, 0, st>>>(slots, n_seg, base, words, P,
                                                                 table);
}

void launch_tcentral(const SegLayout& L, const double* r, const double* vr, const double* vt,
                     const double* m, const double* R, const double* A, double x_bb,
                     double x_bs, cudaStream_t st) {
  if (!L.n || (!R && !A)) return;
  k_tcentral<<<(unsigned)L.n_seg, 32, 0, st>>>(L.dev(), r, vr, vt, m, R, A, x_bb, x_bs);
}

void launch_bins(const SegLayout& L, const double* r, const double* vr, const double* vt,
                 const double* m, double* nbin, double pref, cudaStream_t st) {
  if (!L.n_bins) return;
  k_bins<<<(unsigned)((L.n_bins + 255) / 256), 256, 0, st>>>(L.dev(), L.bin_size, pref, r, vr,
                                                             vt, m, nbin);
}

template <int kMinB>
static void relax_shape(const SegLayout& L, double* vr, double* vt, double* m,
                        const uint32_t* id, const double* nbin, const uint32_t* step,
                        const Collide& col, cudaStream_t st) {
  const unsigned grid = (unsigned)((L.n_pairs + 127) / 128);
  // (the collision code only in the kernels that need it: it costs
  // registers)
  if (L.taus && col.R)
    k_relax<true, kMinB, true><<<grid, 128, 0, st>>>(L.dev(), L.bin_size, vr, vt, m, id, nbin,
                                                     step, col);
  else if (L.taus)
    k_relax<true, kMinB, false><<<grid, 128, 0, st>>>(L.dev(), L.bin_size, vr, vt, m, id, nbin,
                                                      step, col);
  else if (col.R)
    k_relax<false, kMinB, true><<<grid, 128, 0, st>>>(L.dev(), L.bin_size, vr, vt, m, id, nbin,
                                                      step, col);
  else
    k_relax<false, kMinB, false><<<grid, 128, 0, st>>>(L.dev(), L.bin_size, vr, vt, m, id,
                                                       nbin, step, col);
}

void launch_relax(const SegLayout& L, double* vr, double* vt, double* m, const uint32_t* id,
                  const double* nbin, const uint32_t* step, cudaStream_t st, int variant,
                  double* R, const double* r, const double* phi) {
  if (!L.n_pairs) return;
  Collide col;
  col.R = R;
  col.r = r;
  col.phi = phi;
  // variants: registers capped for 1 (no cap), 6 or 8 resident blocks per SM
  if (variant == 1) relax_shape<6>(L, vr, vt, m, id, nbin, step, col, st);
  else if (variant == 2) relax_shape<8>(L, vr, vt, m, id, nbin, step, col, st);
  else relax_shape<1>(L, vr, vt, m, id, nbin, step, col, st);
}


CMC_DEBUG_SITE_ACCESSOR

}  // namespace cmc
