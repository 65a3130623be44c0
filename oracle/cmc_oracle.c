/*
 * Oracle for the Henon Monte Carlo timestep (Pattabiraman et al.,
 * "A Parallel Monte Carlo Code for Simulating Collisional N-body Systems").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * FP64 statement of what one timestep computes.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header or constant table with
 * the CUDA library: both are written from the same paper and the same
 * readings of it.
 *
 * Build: gcc -O2 -std=c99 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * Every floating-point operation below is a single IEEE-754 round-to-nearest
 * operation (+ - * / sqrt) evaluated in the order written; no operation is
 * contracted into a fused multiply-add.
 *
 * Conventions
 *   Henon N-body units: G = 1, total mass 1.
 *   Stars are indexed 0..n-1 in sorted order (the paper counts from 1).
 *   The first nb stars are bound; escaped stars carry r = +inf and sit at
 *   the end of the arrays, ordered by id.
 *   x_k denotes 1/r_k (the variable in which the shell potential is linear).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* pi rounded to the nearest double */
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers.                                             */
/*                                                                           */
/* The paper needs independent, evenly distributed streams per star (section */
/* "Parallel Random Number Generation").  The oracle uses Philox4x32-10      */
/* (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random numbers: as easy as */
/* 1, 2, 3"): ten rounds of two 32x32->64 multiplies and xors, with a Weyl   */
/* key schedule.  Constants are the published Philox4x32 multipliers and    */
/* Weyl increments.                                                          */
/* ------------------------------------------------------------------------ */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

/* stream tags: the third counter word */
#define OR_TAG_PSI 0u  /* relaxation: azimuth of star 2's transverse velocity */
#define OR_TAG_PHI 1u  /* relaxation: azimuth of the deflection about w        */
#define OR_TAG_REJ 2u  /* orbit: rejection trials (X, X')                      */
#define OR_TAG_SGN 3u  /* orbit: sign of the new radial velocity               */
#define OR_TAG_COL 4u  /* relaxation pair: the sticky-sphere collision draw    */

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += OR_PHILOX_W0;
        k1 += OR_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double strictly inside (0,1) from two 32-bit words: the top 52
 * bits k of (hi:lo) give (2k+1) * 2^-53, which is exact. */
double or_u01(uint32_t lo, uint32_t hi)
{
    uint64_t x = ((uint64_t)hi << 32) | (uint64_t)lo;
    uint64_t k = x >> 12;
    return (double)(2u * k + 1u) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* The paper's generator, as an alternative (section 3.6, App. A.2): the    */
/* combined Tausworthe generator of L'Ecuyer (1999), period ~2^113, four    */
/* LFSR components with parameters (k, q, s) = (31, 6, 18), (29, 2, 2),     */
/* (28, 13, 7), (25, 3, 13).  A step of component (k, q, s) on its 32-bit   */
/* word z is b = ((z << q) ^ z) >> (k - s), z = ((z & m_k) << s) ^ b, m_k   */
/* clearing the low 32 - k bits; the output is the xor of the four words.   */
/* Every step is linear over GF(2), so T^D is a 32 x 32 bit matrix per      */
/* component: the jump functions.                                           */
/* ------------------------------------------------------------------------ */
static const int OR_TK[4] = {31, 29, 28, 25};
static const int OR_TQ[4] = {6, 2, 13, 3};
static const int OR_TS[4] = {18, 2, 7, 13};

static uint32_t or_taus_comp(uint32_t z, int j)
{
    uint32_t mask = 0xFFFFFFFFu << (32 - OR_TK[j]);
    uint32_t b = ((z << OR_TQ[j]) ^ z) >> (OR_TK[j] - OR_TS[j]);
    return ((z & mask) << OR_TS[j]) ^ b;
}

/* One output; advances the four words in place. */
uint32_t or_taus_next(uint32_t z[4])
{
    int j;
    for (j = 0; j < 4; ++j) z[j] = or_taus_comp(z[j], j);
    return z[0] ^ z[1] ^ z[2] ^ z[3];
}

/* 32 x 32 bit matrices as 32 columns: col[i] = image of bit i. */
static uint32_t or_gf2_apply(const uint32_t col[32], uint32_t v)
{
    uint32_t r = 0u;
    int i;
    for (i = 0; i < 32; ++i)
        if ((v >> i) & 1u) r ^= col[i];
    return r;
}

static void or_gf2_mul(const uint32_t a[32], const uint32_t b[32], uint32_t out[32])
{
    uint32_t t[32];
    int i;
    for (i = 0; i < 32; ++i) t[i] = or_gf2_apply(a, b[i]);
    for (i = 0; i < 32; ++i) out[i] = t[i];
}

/* T_j^(2^e): the one-step matrix of component j squared e times. */
void or_taus_pow2(int j, int e, uint32_t out[32])
{
    int i;
    for (i = 0; i < 32; ++i) out[i] = or_taus_comp(1u << i, j);
    for (i = 0; i < e; ++i) or_gf2_mul(out, out, out);
}

/* T_j^D by binary powers (D up to 2^64 - 1). */
void or_taus_pow(int j, uint64_t D, uint32_t out[32])
{
    uint32_t p[32];
    int i;
    for (i = 0; i < 32; ++i) out[i] = 1u << i;
    or_taus_pow2(j, 0, p);
    while (D) {
        if (D & 1u) or_gf2_mul(p, out, out);
        D >>= 1;
        if (D) or_gf2_mul(p, p, p);
    }
}

/* The words applied to a vector: out = M v, per component. */
uint32_t or_gf2_apply_pub(const uint32_t col[32], uint32_t v) { return or_gf2_apply(col, v); }

/* Splitmix64 (Steele, Lea & Flood 2014): the seed's mixer. */
static uint64_t or_splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Starting words of a cluster's sequence from its seed (reading): two
 * splitmix64 outputs, top bit of each word set (every component's state,
 * its top k bits, is then nonzero). */
void or_taus_seed(uint64_t seed, uint32_t z[4])
{
    uint64_t x = seed, a = or_splitmix64(&x), b = or_splitmix64(&x);
    z[0] = (uint32_t)a | 0x80000000u;
    z[1] = (uint32_t)(a >> 32) | 0x80000000u;
    z[2] = (uint32_t)b | 0x80000000u;
    z[3] = (uint32_t)(b >> 32) | 0x80000000u;
}

/* Streams of ids 0 .. n_ids-1, D = 2^80 apart (section 3.6's jump
 * displacement), as the paper builds them: the jump function T^D applied
 * repeatedly to the seeded words, each intermediate state starting the
 * next stream.  table: 4 words per id. */
void or_taus_streams(uint64_t seed, int64_t n_ids, uint32_t *table)
{
    uint32_t J[4][32], z[4];
    int j;
    int64_t i;
    or_taus_seed(seed, z);
    for (j = 0; j < 4; ++j) or_taus_pow2(j, 80, J[j]);
    for (i = 0; i < n_ids; ++i)
        for (j = 0; j < 4; ++j) {
            table[4 * i + j] = z[j];
            z[j] = or_gf2_apply(J[j], z[j]);
        }
}

/* The draws of the method: in the default mode a block of four words of
 * Philox4x32-10 at the counter (id, step, tag, trial); with a stream table
 * bound (or_taus_bind), the next four outputs of the stream of that id --
 * the method draws each star's blocks in a fixed order (relaxation trials,
 * then orbit trials, then the sign), so tag and trial are implied. */
static uint32_t *or_taus_table = 0;

void or_taus_bind(uint32_t *table) { or_taus_table = table; }

static void or_draw(uint64_t seed, uint32_t id, uint32_t step, uint32_t tag,
                    uint32_t trial, uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    if (or_taus_table) {
        uint32_t *z = or_taus_table + 4 * (size_t)id;
        int k;
        for (k = 0; k < 4; ++k) out[k] = or_taus_next(z);
        return;
    }
    ctr[0] = id; ctr[1] = step; ctr[2] = tag; ctr[3] = trial;
    key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, out);
}

/* Bulk interface for tests: n counters (4 words each) -> n blocks. */
void or_philox_bulk(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out)
{
    int64_t i;
    uint32_t key[2];
    key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32);
    for (i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* A uniformly distributed direction in the plane, as (cos a, sin a), drawn by
 * von Neumann rejection of a point in the unit disk: (u, v) uniform in the
 * square [-1,1]^2, accepted when u^2 + v^2 <= 1; then the doubled angle has
 * cos = (u^2 - v^2)/q and sin = 2uv/q.  Returns 0 on success, 1 when 64
 * trials all fail. */
static int or_disk_angle(uint64_t seed, uint32_t id, uint32_t step, uint32_t tag,
                         double *c, double *s)
{
    uint32_t t, w[4];
    for (t = 0; t < 64u; ++t) {
        double u, v, uu, vv, q;
        or_draw(seed, id, step, tag, t, w);
        u = 2.0 * or_u01(w[0], w[1]) - 1.0;
        v = 2.0 * or_u01(w[2], w[3]) - 1.0;
        uu = u * u;
        vv = v * v;
        q = uu + vv;
        if (q <= 1.0) {
            *c = (uu - vv) / q;
            *s = ((2.0 * u) * v) / q;
            return 0;
        }
    }
    *c = 1.0; *s = 0.0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Sort by radius (section 2.1 step 6).                                      */
/* Order: bound stars by increasing r, equal r by increasing id; escaped     */
/* stars (r = +inf) after all bound stars, by increasing id.                 */
/* ------------------------------------------------------------------------ */
static const double *or_sort_r;
static const uint32_t *or_sort_id;

static int or_sort_cmp(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    double ra = or_sort_r[a], rb = or_sort_r[b];
    int ia = isinf(ra) ? 1 : 0, ib = isinf(rb) ? 1 : 0;
    if (ia != ib) return ia - ib;
    if (!ia) {
        if (ra < rb) return -1;
        if (ra > rb) return 1;
    }
    if (or_sort_id[a] < or_sort_id[b]) return -1;
    if (or_sort_id[a] > or_sort_id[b]) return 1;
    return 0;
}

/* perm[j] = index (into the input arrays) of the star that goes to slot j. */
void or_sort_perm(int64_t n, const double *r, const uint32_t *id, int64_t *perm)
{
    int64_t i;
    for (i = 0; i < n; ++i) perm[i] = i;
    or_sort_r = r;
    or_sort_id = id;
    qsort(perm, (size_t)n, sizeof(int64_t), or_sort_cmp);
}

/* ------------------------------------------------------------------------ */
/* Shell potential (section 2.1 step 1).                                     */
/* ------------------------------------------------------------------------ */

/* Eqs. 2-5 exactly as written: Phi_{N+1} = 0, M_N = sum m, then downward
 * Phi_k = Phi_{k+1} - G M_k (1/r_k - 1/r_{k+1}), M_{k-1} = M_k - m_k, with
 * 1/r_{N+1} = 0. */
void or_potential_recursion(int64_t nb, const double *r, const double *m, double *phi)
{
    int64_t k;
    double M = 0.0, phi_next = 0.0, x_next = 0.0;
    for (k = 0; k < nb; ++k) M = M + m[k];
    for (k = nb - 1; k >= 0; --k) {
        double xk = 1.0 / r[k];
        phi[k] = phi_next - M * (xk - x_next);
        phi_next = phi[k];
        x_next = xk;
        M = M - m[k];
    }
}

/* Eq. 1 at the star positions by brute force over all pairs: the shell
 * theorem gives Phi_k = -G sum_i m_i / max(r_k, r_i), the own mass included
 * (it lies at r_k, inside "the sum over i <= k"). */
void or_potential_brute(int64_t nb, const double *r, const double *m, double *phi)
{
    int64_t k, i;
    for (k = 0; k < nb; ++k) {
        double s = 0.0;
        for (i = 0; i < nb; ++i) {
            double d = r[k] > r[i] ? r[k] : r[i];
            s = s + m[i] / d;
        }
        phi[k] = -s;
    }
}

/* --- double-double helpers (Dekker / Knuth error-free transformations) --- */
typedef struct { double hi, lo; } or_dd;

static or_dd or_two_sum(double a, double b)
{
    or_dd r;
    double s = a + b;
    double bb = s - a;
    r.hi = s;
    r.lo = (a - (s - bb)) + (b - bb);
    return r;
}

static void or_split(double a, double *hi, double *lo)
{
    double c = 134217729.0 * a; /* 2^27 + 1 */
    *hi = c - (c - a);
    *lo = a - *hi;
}

static or_dd or_two_prod(double a, double b)
{
    or_dd r;
    double ah, al, bh, bl;
    double p = a * b;
    or_split(a, &ah, &al);
    or_split(b, &bh, &bl);
    r.hi = p;
    r.lo = ((ah * bh - p) + ah * bl + al * bh) + al * bl;
    return r;
}

static or_dd or_dd_add(or_dd a, or_dd b)
{
    or_dd s = or_two_sum(a.hi, b.hi);
    double lo = s.lo + (a.lo + b.lo);
    return or_two_sum(s.hi, lo);
}

/* (a.hi + a.lo) / d to double-double accuracy */
static or_dd or_dd_div_d(or_dd a, double d)
{
    double q1 = a.hi / d;
    or_dd p = or_two_prod(q1, d);
    double rem = ((a.hi - p.hi) - p.lo) + a.lo;
    double q2 = rem / d;
    return or_two_sum(q1, q2);
}

/* Eq. 1 in scan form, Phi_k = -G (M_k / r_k + sum_{i>k} m_i / r_i), with
 * every sum and quotient carried in double-double and rounded once.  This
 * is the accuracy reference the GPU scan is compared with. */
void or_potential_dd(int64_t nb, const double *r, const double *m, double *phi)
{
    int64_t k;
    or_dd *M = (or_dd *)malloc(sizeof(or_dd) * (size_t)(nb > 0 ? nb : 1));
    or_dd acc, S;
    acc.hi = 0.0; acc.lo = 0.0;
    for (k = 0; k < nb; ++k) {
        or_dd t; t.hi = m[k]; t.lo = 0.0;
        acc = or_dd_add(acc, t);
        M[k] = acc;
    }
    S.hi = 0.0; S.lo = 0.0;
    for (k = nb - 1; k >= 0; --k) {
        or_dd mk, q, tot;
        mk.hi = m[k]; mk.lo = 0.0;
        tot = or_dd_add(or_dd_div_d(M[k], r[k]), S);
        phi[k] = -(tot.hi + tot.lo);
        q = or_dd_div_d(mk, r[k]);
        S = or_dd_add(S, q);
    }
    free(M);
}

/* Largest index i in [0, nb) with r_i <= rq, or -1 when rq < r_0.  Plain
 * bisection on the sorted radii. */
static int64_t or_shell_of(int64_t nb, const double *r, double rq)
{
    int64_t lo = -1, hi = nb;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (r[mid] <= rq) lo = mid; else hi = mid;
    }
    return lo;
}

/* Eq. 6: Phi(r) between two stars is linear in 1/r.  Inside the innermost
 * star Eq. 1 has no enclosed mass and Phi is the constant Phi_0; beyond the
 * outermost star the virtual node Phi_{N+1} = 0 at 1/r = 0 applies. */
double or_phi_of_r(int64_t nb, const double *r, const double *phi, double rq)
{
    int64_t i = or_shell_of(nb, r, rq);
    double x, xj, xj1, pj1, den;
    if (i < 0) return phi[0];
    x = 1.0 / rq;
    xj = 1.0 / r[i];
    if (i + 1 < nb) { xj1 = 1.0 / r[i + 1]; pj1 = phi[i + 1]; }
    else { xj1 = 0.0; pj1 = 0.0; }
    den = xj - xj1;
    if (!(den > 0.0)) return phi[i];
    return phi[i] + ((xj - x) / den) * (pj1 - phi[i]);
}

/* ------------------------------------------------------------------------ */
/* Relaxation timestep, Eq. 7, on fixed bins of bin_size consecutive stars  */
/* (section 3.3's replacement of the sliding average).                      */
/* pref = (theta_max / (pi/2)) * (pi/32); lnL = ln(gamma N).                 */
/* Bin b holds stars [b*bs, min((b+1)*bs, nb)).  For P >= 2 stars:           */
/*   n    = 3 (P-1) / (4 pi (r_last^3 - r_first^3))                          */
/*   <v_rel>      = mean over the bin's pairs (2j, 2j+1) of sqrt(v1^2+v2^2)  */
/*   <(M1+M2)^2>  = mean over the same pairs of (m1+m2)^2                    */
/*   T_b  = pref <v_rel>^3 / (lnL n <(M1+M2)^2>)                             */
/* A bin with fewer than 2 stars, no volume, or no pair mass has n = 0 and   */
/* T_b = +inf.  Returns dt = min_b T_b.                                      */
/* ------------------------------------------------------------------------ */
double or_timestep(int64_t nb, const double *r, const double *vr, const double *vt,
                   const double *m, int32_t bs, double pref, double lnL, double *nbin)
{
    int64_t nbins = (nb + bs - 1) / bs, b;
    double dt = INFINITY;
    for (b = 0; b < nbins; ++b) {
        int64_t first = b * bs;
        int64_t P = nb - first < bs ? nb - first : bs;
        int64_t q = P / 2, j;
        double rf, rl, vol, n, sv = 0.0, sm = 0.0, v, msq, num, den, T;
        nbin[b] = 0.0;
        if (P < 2) continue;
        rf = r[first];
        rl = r[first + P - 1];
        vol = rl * rl * rl - rf * rf * rf;
        if (!(vol > 0.0)) continue;
        n = (3.0 * (double)(P - 1)) / ((4.0 * OR_PI) * vol);
        for (j = 0; j < q; ++j) {
            int64_t a = first + 2 * j;
            double va2 = vr[a] * vr[a] + vt[a] * vt[a];
            double vb2 = vr[a + 1] * vr[a + 1] + vt[a + 1] * vt[a + 1];
            double ms = m[a] + m[a + 1];
            sv = sv + sqrt(va2 + vb2);
            sm = sm + ms * ms;
        }
        v = sv / (double)q;
        msq = sm / (double)q;
        nbin[b] = n;
        num = pref * (v * v * v);
        den = (lnL * n) * msq;
        if (!(den > 0.0)) continue;
        T = num / den;
        if (T < dt) dt = T;
    }
    return dt;
}

/* ------------------------------------------------------------------------ */
/* Two-body relaxation between radial neighbours (section 2.1 step 3(i);     */
/* pairs (2j, 2j+1) never straddle a bin because the bin size is even).      */
/* Representative encounter: star 1 moves along (v_r1, v_t1, 0), star 2's    */
/* transverse velocity has a random azimuth psi.  The relative velocity w is */
/* turned by the deflection angle beta,                                      */
/*   sin^2(beta/2) = min(1, 2 pi G^2 (m1+m2)^2 n lnL dt / |w|^3),            */
/* about w by a random azimuth phi; the centre-of-mass velocity is kept.    */
/* (4 sin^2(beta/2) ~ beta^2 is the mean squared deflection the relative    */
/* velocity gathers over dt from small-angle encounters, 8 pi G^2 (m1+m2)^2 */
/* n lnL dt / |w|^3; with it a Plummer sphere collapses at ~17-18 t_rh, as  */
/* in section 4.2, where half this rate takes ~34 t_rh.)                     */
/* Random numbers are keyed by the id of the pair's first star.             */
/* Returns the number of pairs whose angle draw failed (normally 0).        */
/* ------------------------------------------------------------------------ */
/* One representative encounter.  out[] (16 doubles):
 *   0-2 v1, 3-5 v2 (3-D, before), 6-8 v1', 9-11 v2' (after),
 *   12 sin^2(beta/2), 13 cos(beta), 14 |w|, 15 status
 * status: 0 deflected, 1 skipped (no density, no mass or w = 0).
 * Returns the number of failed angle draws (normally 0). */
/* Sticky spheres (section 2.1 step 3(iii): two bodies merge when their
 * radii touch).  Reading: with stellar radii R1, R2 the pair's
 * representative encounter is a collision with probability
 *   P = n sigma |w| dt,  sigma = pi (R1 + R2)^2 (1 + 2 G (m1 + m2) / ((R1 + R2) |w|^2))
 * (the geometric cross section with gravitational focusing, the pair's bin
 * density n, its 3-D relative speed |w|), decided by one uniform draw of
 * the pair (tag 4) taken after the azimuth psi; the merged star keeps the
 * pair's momentum (3-D centre-of-mass velocity) and total mass, and the
 * relative kinetic energy (m1 m2 / (m1 + m2)) |w|^2 / 2 is dissipated.
 * out[] (20 doubles): as or_encounter, with status 2 for a merger (6-8 the
 * merged star's velocity), 16 P, 17 the dissipated energy. */
static int or_encounter_col(double m1, double m2, double vr1, double vt1, double vr2,
                            double vt2, double R1, double R2, double n, double dt, double lnL,
                            uint64_t seed, uint32_t id, uint32_t step, double *out);

int or_encounter(double m1, double m2, double vr1, double vt1, double vr2, double vt2,
                 double n, double dt, double lnL, uint64_t seed, uint32_t id,
                 uint32_t step, double *out)
{
    double o[20];
    int i, fails = or_encounter_col(m1, m2, vr1, vt1, vr2, vt2, 0.0, 0.0, n, dt, lnL, seed, id,
                                    step, o);
    for (i = 0; i < 16; ++i) out[i] = o[i];
    return fails;
}

/* Test hook: the encounter with stellar radii (out: 20 doubles). */
int or_encounter_radii(double m1, double m2, double vr1, double vt1, double vr2, double vt2,
                       double R1, double R2, double n, double dt, double lnL, uint64_t seed,
                       uint32_t id, uint32_t step, double *out)
{
    return or_encounter_col(m1, m2, vr1, vt1, vr2, vt2, R1, R2, n, dt, lnL, seed, id, step, out);
}

static int or_encounter_col(double m1, double m2, double vr1, double vt1, double vr2,
                            double vt2, double R1, double R2, double n, double dt, double lnL,
                            uint64_t seed, uint32_t id, uint32_t step, double *out)
{
    double msum, cpsi = 1.0, spsi = 0.0, cphi, sphi;
    double v1x, v1y, v1z, v2x, v2y, v2z, wx, wy, wz, w2, w;
    double num, s2, sb, cosb, sinb, wp2, e1y, e1z;
    double ux, uy, uz, a1, wpx, wpy, wpz, dwx, dwy, dwz, f1, f2;
    int fails = 0, i;
    for (i = 0; i < 20; ++i) out[i] = 0.0;
    out[15] = 1.0;
    msum = m1 + m2;
    /* no density, no mass, or no positive Coulomb logarithm (ln(gamma N) <= 0
     * for N <= 1/gamma): no deflection */
    if (!(n > 0.0) || !(msum > 0.0) || !(lnL > 0.0) || !(dt < INFINITY)) {
        out[0] = vr1; out[1] = vt1; out[3] = vr2; out[4] = vt2;
        for (i = 0; i < 6; ++i) out[6 + i] = out[i];
        return 0;
    }
    fails += or_disk_angle(seed, id, step, OR_TAG_PSI, &cpsi, &spsi);
    v1x = vr1; v1y = vt1; v1z = 0.0;
    v2x = vr2; v2y = vt2 * cpsi; v2z = vt2 * spsi;
    out[0] = v1x; out[1] = v1y; out[2] = v1z;
    out[3] = v2x; out[4] = v2y; out[5] = v2z;
    for (i = 0; i < 6; ++i) out[6 + i] = out[i];
    wx = v1x - v2x; wy = v1y - v2y; wz = v1z - v2z;
    w2 = (wx * wx + wy * wy) + wz * wz;
    if (!(w2 > 0.0)) return fails;
    w = sqrt(w2);
    if (R1 + R2 > 0.0) {
        double Rs = R1 + R2, focus, sig, Pc, X;
        uint32_t cw[4];
        focus = 1.0 + (2.0 * msum) / (Rs * w2);
        sig = (OR_PI * (Rs * Rs)) * focus;
        Pc = ((sig * n) * w) * dt;
        or_draw(seed, id, step, OR_TAG_COL, 0u, cw);
        X = or_u01(cw[0], cw[1]);
        out[16] = Pc;
        if (X < Pc) {
            out[6] = (m1 * v1x + m2 * v2x) / msum;
            out[7] = (m1 * v1y + m2 * v2y) / msum;
            out[8] = (m1 * v1z + m2 * v2z) / msum;
            out[9] = 0.0; out[10] = 0.0; out[11] = 0.0;
            out[14] = w;
            out[15] = 2.0;
            out[17] = (0.5 * ((m1 * m2) / msum)) * w2;
            return fails;
        }
    }
    num = (2.0 * OR_PI) * msum;
    num = num * msum;
    num = num * n;
    num = num * lnL;
    num = num * dt;
    s2 = num / (w2 * w);
    if (!(s2 <= 1.0)) s2 = 1.0;
    /* cos(beta) = 1 - 2 sin^2(beta/2), sin(beta) = 2 sin(beta/2) cos(beta/2) */
    sb = sqrt(s2);
    cosb = 1.0 - 2.0 * s2;
    sinb = (2.0 * sb) * sqrt(1.0 - s2);
    fails += or_disk_angle(seed, id, step, OR_TAG_PHI, &cphi, &sphi);
    /* unit vector e1 = (w x xhat)/|w x xhat| = (0, wz, -wy)/|.|, or yhat when
     * w is radial; u = w x e1 has length |w| and completes the orthogonal
     * frame (e1, u/|w|) perpendicular to w. */
    wp2 = wy * wy + wz * wz;
    if (wp2 > 0.0) {
        double wp = sqrt(wp2);
        e1y = wz / wp;
        e1z = -wy / wp;
    } else {
        e1y = 1.0;
        e1z = 0.0;
    }
    ux = wy * e1z - wz * e1y;
    uy = -(wx * e1z);
    uz = wx * e1y;
    a1 = w * cphi;
    /* w' = w cos(beta) + sin(beta) (|w| cos(phi) e1 + sin(phi) u) */
    wpx = wx * cosb + sinb * (sphi * ux);
    wpy = wy * cosb + sinb * (a1 * e1y + sphi * uy);
    wpz = wz * cosb + sinb * (a1 * e1z + sphi * uz);
    dwx = wpx - wx; dwy = wpy - wy; dwz = wpz - wz;
    /* the centre of mass keeps its velocity: v1' = v1 + m2/(m1+m2) dw,
     * v2' = v2 - m1/(m1+m2) dw */
    f1 = m2 / msum;
    f2 = m1 / msum;
    out[6] = v1x + f1 * dwx; out[7] = v1y + f1 * dwy; out[8] = v1z + f1 * dwz;
    out[9] = v2x - f2 * dwx; out[10] = v2y - f2 * dwy; out[11] = v2z - f2 * dwz;
    out[12] = s2; out[13] = cosb; out[14] = w; out[15] = 0.0;
    return fails;
}

/* Cube root by Newton's method, y <- y - (y^3 - v) / (3 y^2), eight steps
 * from 2^floor(e/3) (e the binary exponent of v), every operation one IEEE
 * rounding in this order (so that the GPU, taking the same steps, gets the
 * same bits); within a few units in the last place of the cube root for
 * normal v > 0, and 0 for v <= 0. */
double or_cbrt(double v)
{
    uint64_t b;
    int e, k, i;
    double y;
    if (!(v > 0.0)) return 0.0;
    memcpy(&b, &v, sizeof b);
    e = (int)((b >> 52) & 0x7FF) - 1023;
    k = e >= 0 ? e / 3 : -((-e + 2) / 3);  /* floor(e / 3) */
    b = (uint64_t)(k + 1023) << 52;
    memcpy(&y, &b, sizeof y);
    for (i = 0; i < 8; ++i) y = y - (y * y * y - v) / (3.0 * (y * y));
    return y;
}

/* All pairs (2j, 2j+1) of the nb bound stars; the density of a pair is that
 * of its bin.  New v_r is the radial (x) component, new v_t the length of
 * the transverse (y, z) part.  With stellar radii R (may be NULL) a pair may
 * merge instead (sticky spheres): the first star takes the total mass, the
 * pair's momentum and the radius cbrt(R1^3 + R2^3) (volume kept), the second
 * gets mass 0 and radius -1 (it leaves in the orbit step); col[0] counts
 * the mergers, col[1] adds what they change of K + W: the relative kinetic
 * energy dissipated, -(m_a m_b / (m_a + m_b)) |w|^2 / 2, plus the change of
 * the shell-model W = -sum_{i<j} m_i m_j / max(r_i, r_j) when b's mass joins
 * a (a, b adjacent, r_a <= r_b): m_b (Phi_a - Phi_b) + m_a m_b / r_a (the
 * pair's own term leaves W, the stars inside r_a now bind b's mass at r_a);
 * r and phi (the current potential) may be NULL when col is. */
int64_t or_relax_col(int64_t nb, double *vr, double *vt, double *m, double *R,
                     const uint32_t *id, const double *nbin, int32_t bs, double dt, double lnL,
                     uint64_t seed, uint32_t step, double *col, const double *r,
                     const double *phi)
{
    int64_t j, npairs = nb / 2, fails = 0;
    for (j = 0; j < npairs; ++j) {
        int64_t a = 2 * j, b = a + 1;
        double o[20];
        fails += or_encounter_col(m[a], m[b], vr[a], vt[a], vr[b], vt[b], R ? R[a] : 0.0,
                                  R ? R[b] : 0.0, nbin[a / bs], dt, lnL, seed, id[a], step, o);
        if (o[15] == 2.0) {
            double R1 = R[a], R2 = R[b];
            if (col) {
                double dW = m[b] * (phi[a] - phi[b]) + (m[a] * m[b]) / r[a];
                col[0] += 1.0;
                col[1] += dW - o[17];
            }
            vr[a] = o[6];
            vt[a] = sqrt(o[7] * o[7] + o[8] * o[8]);
            m[a] = m[a] + m[b];
            R[a] = or_cbrt(R1 * R1 * R1 + R2 * R2 * R2);
            m[b] = 0.0;
            R[b] = -1.0;
            continue;
        }
        if (o[15] != 0.0) continue;
        vr[a] = o[6]; vt[a] = sqrt(o[7] * o[7] + o[8] * o[8]);
        vr[b] = o[9]; vt[b] = sqrt(o[10] * o[10] + o[11] * o[11]);
    }
    return fails;
}

int64_t or_relax(int64_t nb, double *vr, double *vt, const double *m, const uint32_t *id,
                 const double *nbin, int32_t bs, double dt, double lnL,
                 uint64_t seed, uint32_t step)
{
    return or_relax_col(nb, vr, vt, (double *)m, NULL, id, nbin, bs, dt, lnL, seed, step, NULL,
                        NULL, NULL);
}

/* The collision timestep (section 2.1 step 2, Eq. 8) over the innermost
 * P = min(300, nb) bound stars (the paper averages it over the central 300):
 *   1 / T_coll = 16 sqrt(pi) n_s <R^2> sigma (1 + G <M R> / (2 sigma^2 <R^2>))
 * with n_s = 3 (P - 1) / (4 pi (r_{P-1}^3 - r_0^3)) (the bins' estimator),
 * sigma^2 = <v_r^2 + v_t^2> / 3 the one-dimensional velocity dispersion, and
 * the means over the P stars in order.  +inf without radii (<R^2> = 0). */
double or_tcoll(int64_t nb, const double *r, const double *vr, const double *vt,
                const double *m, const double *R)
{
    int64_t P = nb < 300 ? nb : 300, k;
    double vol, ns, sv = 0.0, sr = 0.0, smr = 0.0, sig2, R2, MR, sig, inv;
    if (P < 2 || !R) return INFINITY;
    vol = r[P - 1] * r[P - 1] * r[P - 1] - r[0] * r[0] * r[0];
    if (!(vol > 0.0)) return INFINITY;
    ns = (3.0 * (double)(P - 1)) / ((4.0 * OR_PI) * vol);
    for (k = 0; k < P; ++k) {
        sv = sv + (vr[k] * vr[k] + vt[k] * vt[k]);
        sr = sr + R[k] * R[k];
        smr = smr + m[k] * R[k];
    }
    sig2 = (sv / (double)P) / 3.0;
    R2 = sr / (double)P;
    MR = smr / (double)P;
    if (!(R2 > 0.0) || !(sig2 > 0.0)) return INFINITY;
    sig = sqrt(sig2);
    inv = (((16.0 * sqrt(OR_PI)) * ns) * R2) * sig;
    inv = inv * (1.0 + MR / ((2.0 * sig2) * R2));
    return 1.0 / inv;
}

/* The binary timesteps (section 2.1 step 2, Eqs. 9 and 10) over the
 * innermost P = min(300, nb) bound stars, a star being a binary when its
 * semi-major axis A[k] > 0 (its mass m[k] the binary's total):
 *   1 / T_bb = 16 sqrt(pi) n_b X_bb^2 <a^2> sigma
 *              (1 + G <M a> / (2 sigma^2 X_bb <a^2>))
 *   1 / T_bs = 4 sqrt(pi) n_s X_bs^2 <a^2> sigma
 *              (1 + G <M> <a> / (sigma^2 X_bs <a^2>))
 * Readings: n_b and n_s are the central density of Eq. 8's estimator,
 * n = 3 (P - 1) / (4 pi (r_{P-1}^3 - r_0^3)), times the binaries' and the
 * single stars' shares of the P stars; <a^2>, <M a>, <a> are means over
 * the binaries among them, <M> the mean mass of all P, sigma as in Eq. 8.
 * +inf where there is no binary (or, for T_bs, no single star).  Returns
 * T_bb; *tbs = T_bs. */
double or_tbinary(int64_t nb, const double *r, const double *vr, const double *vt,
                  const double *m, const double *A, double x_bb, double x_bs, double *tbs)
{
    int64_t P = nb < 300 ? nb : 300, k, nbin = 0;
    double vol, n, sv = 0.0, sm = 0.0, sa = 0.0, sa2 = 0.0, sma = 0.0;
    double sig2, sig, a2, ma, am, mm, nbd, nsd, inv;
    *tbs = INFINITY;
    if (P < 2 || !A) return INFINITY;
    vol = r[P - 1] * r[P - 1] * r[P - 1] - r[0] * r[0] * r[0];
    if (!(vol > 0.0)) return INFINITY;
    n = (3.0 * (double)(P - 1)) / ((4.0 * OR_PI) * vol);
    for (k = 0; k < P; ++k) {
        sv = sv + (vr[k] * vr[k] + vt[k] * vt[k]);
        sm = sm + m[k];
        if (A[k] > 0.0) {
            nbin += 1;
            sa = sa + A[k];
            sa2 = sa2 + A[k] * A[k];
            sma = sma + m[k] * A[k];
        }
    }
    sig2 = (sv / (double)P) / 3.0;
    if (nbin == 0 || !(sig2 > 0.0)) return INFINITY;
    sig = sqrt(sig2);
    a2 = sa2 / (double)nbin;
    ma = sma / (double)nbin;
    am = sa / (double)nbin;
    mm = sm / (double)P;
    nbd = n * ((double)nbin / (double)P);
    nsd = n * ((double)(P - nbin) / (double)P);
    if (nbin < P) {
        inv = (((4.0 * sqrt(OR_PI)) * nsd) * ((x_bs * x_bs) * a2)) * sig;
        inv = inv * (1.0 + (mm * am) / ((sig2 * x_bs) * a2));
        *tbs = 1.0 / inv;
    }
    inv = (((16.0 * sqrt(OR_PI)) * nbd) * ((x_bb * x_bb) * a2)) * sig;
    inv = inv * (1.0 + ma / (((2.0 * sig2) * x_bb) * a2));
    return 1.0 / inv;
}

/* The stellar-evolution timestep (Eq. 11): T_se = 0.001 M T_prev / dm_se,
 * the step in which stellar evolution, losing dm_se in the previous step of
 * length T_prev, takes 0.1% of the cluster's mass M; +inf without loss. */
double or_tse(double M, double T_prev, double dm_se)
{
    if (!(dm_se > 0.0)) return INFINITY;
    return ((0.001 * M) * T_prev) / dm_se;
}

/* Test hook for the angle draw. */
int or_disk_angle_pub(uint64_t seed, uint32_t id, uint32_t step, uint32_t tag, double *cs)
{
    return or_disk_angle(seed, id, step, tag, &cs[0], &cs[1]);
}

/* ------------------------------------------------------------------------ */
/* New orbits (section 2.1 step 5).                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t nb;
    const double *r, *phi;
    double E, J;
} or_orb;

/* Eq. 12 at star node i: Q = 2E - 2 Phi_i - J^2 / r_i^2 */
static double or_Q_node(const or_orb *o, int64_t i)
{
    double L = o->J * (1.0 / o->r[i]);
    return 2.0 * (o->E - o->phi[i]) - L * L;
}

/* Inside shell j (nodes j and j+1, node nb being 1/r = 0, Phi = 0) Eq. 6
 * reads Phi = A - B/r with B = (Phi_{j+1} - Phi_j)/(x_j - x_{j+1}),
 * A = Phi_j + B x_j, so Q(x) = 2(E - A) + 2Bx - J^2 x^2.  Its roots are
 * x = (B -+ sqrt(D))/J^2 with D = B^2 + 2 J^2 (E - A); they are evaluated
 * in the cancellation-free forms r = (B + sqrt D)/(2(A - E)) (outer root,
 * smaller x) and r = J^2/(B + sqrt D) (inner root, larger x), then clamped
 * into the shell. */
static double or_shell_root(const or_orb *o, int64_t j, int outer)
{
    double rj = o->r[j], xj = 1.0 / rj, pj = o->phi[j];
    double xj1, pj1, rj1, B, A, D, sD, root;
    int has_next = (j + 1 < o->nb);
    if (has_next) { rj1 = o->r[j + 1]; xj1 = 1.0 / rj1; pj1 = o->phi[j + 1]; }
    else { rj1 = INFINITY; xj1 = 0.0; pj1 = 0.0; }
    if (!(xj - xj1 > 0.0)) return rj;
    B = (pj1 - pj) / (xj - xj1);
    A = pj + B * xj;
    D = B * B + 2.0 * (o->J * o->J) * (o->E - A);
    if (!(D > 0.0)) D = 0.0;
    sD = sqrt(D);
    if (outer) root = (B + sD) / (2.0 * (A - o->E));
    else root = (o->J * o->J) / (B + sD);
    if (!(root >= rj)) root = rj;
    if (has_next && root > rj1) root = rj1;
    return root;
}

/* The substitution r(s) = (rmax+rmin)/2 + (rmax-rmin)/4 (3s - s^3) removes
 * the 1/|v_r| singularities at both turning points (the "slightly modified"
 * rejection of section 2.1 step 5); g(s) = (dr/ds)/sqrt(Q(r(s))) is the
 * density of s.  Writes r(s) and Phi(r(s)); returns g (0 where Q <= 0). */
static double or_g_of_s(const or_orb *o, double c0, double c1, double s,
                        double *rs_out, double *phis_out, double *Q_out)
{
    double rs = c0 + c1 * (s * (3.0 - s * s));
    double drds = (3.0 * c1) * (1.0 - s * s);
    double ph = or_phi_of_r(o->nb, o->r, o->phi, rs);
    double L = o->J / rs;
    double Q = 2.0 * (o->E - ph) - L * L;
    *rs_out = rs;
    *phis_out = ph;
    *Q_out = Q;
    if (!(Q > 0.0)) return 0.0;
    return drds / sqrt(Q);
}

/* Per-star result of the orbit step.  out[] layout:
 *   0 r_new, 1 vr_new, 2 vt_new, 3 Phi_old(r_new), 4 rmin, 5 rmax, 6 F,
 *   7 trials used.
 * Return code: 0 moved, 1 escaped (E >= 0), 2 degenerate orbit (kept in
 * place), 3 rejection cap hit (kept in place).  *viol counts trials with
 * g(s) > F. */
static int or_orbit_star_F(int64_t k, int64_t nb, const double *r, const double *phi,
                           double vr, double vt, uint32_t id, uint64_t seed, uint32_t step,
                           int32_t max_trials, double F_in, double *out, int64_t *viol);

int or_orbit_star(int64_t k, int64_t nb, const double *r, const double *phi,
                  double vr, double vt, uint32_t id, uint64_t seed, uint32_t step,
                  int32_t max_trials, double *out, int64_t *viol)
{
    return or_orbit_star_F(k, nb, r, phi, vr, vt, id, seed, step, max_trials, 0.0, out, viol);
}

/* Test hook: the same orbit step with the rejection bound F given from
 * outside (F_in > 0) instead of 1.2 max g(s_j).  Any F >= max g gives the
 * same distribution of r_new (Eqs. 13-15); for a given F, the draws fix the
 * accepted trial.  This lets a sampler with an envelope of its own be
 * compared star by star. */
int or_orbit_star_env(int64_t k, int64_t nb, const double *r, const double *phi,
                      double vr, double vt, uint32_t id, uint64_t seed, uint32_t step,
                      int32_t max_trials, double F_in, double *out, int64_t *viol)
{
    return or_orbit_star_F(k, nb, r, phi, vr, vt, id, seed, step, max_trials, F_in, out, viol);
}

static int or_orbit_star_F(int64_t k, int64_t nb, const double *r, const double *phi,
                           double vr, double vt, uint32_t id, uint64_t seed, uint32_t step,
                           int32_t max_trials, double F_in, double *out, int64_t *viol)
{
    or_orb o;
    double rk = r[k], rmin, rmax, c0, c1, gmax, F;
    int64_t lo, hi, jmax, jmin;
    int32_t t;
    uint32_t w[4];
    int j;
    o.nb = nb; o.r = r; o.phi = phi;
    o.E = phi[k] + 0.5 * (vr * vr + vt * vt);
    o.J = rk * vt;
    out[0] = rk; out[1] = vr; out[2] = vt; out[3] = phi[k];
    out[4] = rk; out[5] = rk; out[6] = 0.0; out[7] = 0.0;
    if (!(o.E < 0.0)) {
        out[0] = INFINITY;
        return 1;
    }
    /* r_max: Q(node k) >= 0 by construction, Q at 1/r = 0 is 2E < 0 */
    lo = k; hi = nb;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (or_Q_node(&o, mid) < 0.0) hi = mid; else lo = mid;
    }
    jmax = lo;
    rmax = or_shell_root(&o, jmax, 1);
    /* r_min: the virtual node -1 (r = 0) counts as Q < 0 */
    lo = -1; hi = k;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (or_Q_node(&o, mid) < 0.0) lo = mid; else hi = mid;
    }
    jmin = lo;
    if (jmin < 0) {
        /* inside the innermost star Phi = Phi_0, so Q = 2(E - Phi_0) - J^2/r^2 */
        rmin = o.J / sqrt(2.0 * (o.E - phi[0]));
        if (!(rmin >= 0.0)) rmin = 0.0;
        if (rmin > r[0]) rmin = r[0];
    } else {
        rmin = or_shell_root(&o, jmin, 0);
    }
    out[4] = rmin; out[5] = rmax;
    c0 = 0.5 * (rmax + rmin);
    c1 = 0.25 * (rmax - rmin);
    /* bound F = 1.2 max g(s_j) over s_j = -1 + (j + 1/2)/10.5, j = 0..20 */
    gmax = 0.0;
    for (j = 0; j <= 20; ++j) {
        double s = -1.0 + ((double)j + 0.5) / 10.5, rs, ph, Q;
        double g = or_g_of_s(&o, c0, c1, s, &rs, &ph, &Q);
        if (g > gmax) gmax = g;
    }
    F = 1.2 * gmax;
    if (!(rmax > rmin) || !(F > 0.0)) {
        out[6] = F;
        return 2;
    }
    if (F_in > 0.0) F = F_in;
    out[6] = F;
    /* von Neumann rejection (Eqs. 14-15 in the variable s) */
    for (t = 0; t < max_trials; ++t) {
        double X, Xp, s, rs, ph, Q, g;
        or_draw(seed, id, step, OR_TAG_REJ, (uint32_t)t, w);
        X = or_u01(w[0], w[1]);
        Xp = or_u01(w[2], w[3]);
        s = 2.0 * X - 1.0;
        g = or_g_of_s(&o, c0, c1, s, &rs, &ph, &Q);
        if (g > F) *viol += 1;
        if (F * Xp < g) {
            double sq = sqrt(Q);
            or_draw(seed, id, step, OR_TAG_SGN, 0u, w);
            out[0] = rs;
            out[1] = (w[0] & 1u) ? -sq : sq;
            out[2] = o.J / rs;
            out[3] = ph;
            out[7] = (double)(t + 1);
            return 0;
        }
    }
    out[7] = (double)max_trials;
    return 3;
}

/* The orbit step over all bound stars of one sorted state (no sort after
 * it).  Per star: r_new, vr_new, vt_new, Phi_old(r_new), rmin, rmax, F and
 * the return code of or_orbit_star.  stats[] as in or_step (indices 0-4). */
void or_orbit_all(int64_t nb, const double *r, const double *phi, const double *vr,
                  const double *vt, const uint32_t *id, uint64_t seed, uint32_t step,
                  int32_t max_trials, double *r_new, double *vr_new, double *vt_new,
                  double *phi_new, double *rmin, double *rmax, double *F,
                  int32_t *code, int64_t *stats)
{
    int64_t k;
    memset(stats, 0, 5 * sizeof(int64_t));
    for (k = 0; k < nb; ++k) {
        double out[8];
        int64_t viol = 0;
        int rc = or_orbit_star(k, nb, r, phi, vr[k], vt[k], id[k], seed, step,
                               max_trials, out, &viol);
        r_new[k] = out[0]; vr_new[k] = out[1]; vt_new[k] = out[2];
        phi_new[k] = out[3]; rmin[k] = out[4]; rmax[k] = out[5]; F[k] = out[6];
        code[k] = rc;
        stats[3] += (int64_t)out[7];
        stats[4] += viol;
        if (rc == 1) stats[0] += 1;
        if (rc == 2) stats[1] += 1;
        if (rc == 3) stats[2] += 1;
    }
}

/* The orbit step of the stars at sorted positions ks[0..nk) only (the same
 * per-star work as or_orbit_all), for timing a sample of a large state:
 * r_new[i] receives star ks[i]'s new radius. */
void or_orbit_sample(int64_t nb, const double *r, const double *phi, const double *vr,
                     const double *vt, const uint32_t *id, int64_t nk, const int64_t *ks,
                     uint64_t seed, uint32_t step, int32_t max_trials, double *r_new)
{
    int64_t i;
    for (i = 0; i < nk; ++i) {
        double out[8];
        int64_t viol = 0, k = ks[i];
        or_orbit_star(k, nb, r, phi, vr[k], vt[k], id[k], seed, step, max_trials, out, &viol);
        r_new[i] = out[0];
    }
}

/* ------------------------------------------------------------------------ */
/* Energy correction (section 2.1 step 6): the orbit was drawn in the old    */
/* potential; the work done on the star by the changing potential is taken  */
/* by the trapezoid rule between its old and new position,                  */
/*   T' = T + 1/2 [(Phi_new - Phi_old)(r_old) - (Phi_new - Phi_old)(r_new)], */
/* and both velocity components are scaled by sqrt(T'/T), which keeps       */
/* v_r/v_t.  c_k = Phi_old(r_old) - Phi_old(r_new) comes from the orbit     */
/* step.  T' < 0 is clamped to 0.  Returns the number of clamps; Tp_out    */
/* (may be NULL) receives the requested T' of every star.                   */
/* ------------------------------------------------------------------------ */
int64_t or_energy_correction(int64_t nb, const double *r, const double *phi,
                             double *vr, double *vt, const double *r_old, const double *c,
                             double *Tp_out)
{
    int64_t k, clamps = 0;
    for (k = 0; k < nb; ++k) {
        double T = 0.5 * (vr[k] * vr[k] + vt[k] * vt[k]);
        double dnew = or_phi_of_r(nb, r, phi, r_old[k]) - phi[k];
        double Tp = T + 0.5 * (dnew - c[k]);
        if (Tp_out) Tp_out[k] = Tp;
        if (Tp < 0.0) { Tp = 0.0; clamps += 1; }
        if (T > 0.0) {
            double f = sqrt(Tp / T);
            vr[k] = vr[k] * f;
            vt[k] = vt[k] * f;
        }
    }
    return clamps;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics (section 2.1 step 6).                                         */
/* K = 1/2 sum m v^2; W = -G sum_{i<j} m_i m_j / max(r_i, r_j), which over   */
/* sorted stars is -G sum_k m_k M_{k-1} / r_k; E = K + W.                    */
/* ------------------------------------------------------------------------ */
void or_energy(int64_t nb, const double *r, const double *vr, const double *vt,
               const double *m, double out[3])
{
    int64_t k;
    double K = 0.0, W = 0.0, Min = 0.0;
    for (k = 0; k < nb; ++k) {
        K = K + m[k] * (vr[k] * vr[k] + vt[k] * vt[k]);
        W = W - m[k] * Min / r[k];
        Min = Min + m[k];
    }
    out[0] = 0.5 * K;
    out[1] = W;
    out[2] = 0.5 * K + W;
}

/* W by the O(N^2) pair sum, for pinning or_energy on small inputs. */
double or_energy_W_brute(int64_t nb, const double *r, const double *m)
{
    int64_t i, j;
    double W = 0.0;
    for (i = 0; i < nb; ++i)
        for (j = i + 1; j < nb; ++j) {
            double d = r[i] > r[j] ? r[i] : r[j];
            W = W - m[i] * m[j] / d;
        }
    return W;
}

/* Lagrangian radius for mass fraction f: r_k of the first k whose enclosed
 * mass M_k = sum_{i<=k} m_i reaches f * M_bound. */
void or_lagrange_radii(int64_t nb, const double *r, const double *m,
                       const double *fracs, int32_t nf, double *out)
{
    int32_t q;
    int64_t k;
    double Mb = 0.0;
    for (k = 0; k < nb; ++k) Mb = Mb + m[k];
    for (q = 0; q < nf; ++q) {
        double target = fracs[q] * Mb, M = 0.0;
        out[q] = nb > 0 ? r[nb - 1] : 0.0;
        for (k = 0; k < nb; ++k) {
            M = M + m[k];
            if (M >= target) { out[q] = r[k]; break; }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Core diagnostics (section 4.2, Eq. 19).  The paper's density around star */
/* i is the 6th-order estimator of Casertano & Hut (1985): the mass of j - 1 */
/* neighbours over the volume out to the j-th (j = 6).  The method keeps     */
/* radii only, so the estimator is taken in the radial order (reading): the  */
/* stars i - 3 and i + 3 bound a shell that holds the 5 stars i - 2 .. i + 2, */
/*   rho_i = (m_{i-2} + ... + m_{i+2}) / (4 pi / 3 (r_{i+3}^3 - r_{i-3}^3)), */
/* unbiased for a Poisson sample (the shell spans 6 exponential gaps in      */
/* volume); stars with fewer than 3 neighbours on a side, or a shell of no   */
/* volume, have no estimate.                                                 */
/*   rho_c = sum rho_i^2 / sum rho_i        (Eq. 19)                         */
/*   r_c   = sum rho_i r_i / sum rho_i      (the density-weighted radius)    */
/* out[0] = rho_c, out[1] = r_c, out[2] = number of estimates.               */
/* ------------------------------------------------------------------------ */
void or_core(int64_t nb, const double *r, const double *m, double *out)
{
    double s1 = 0.0, s2 = 0.0, sr = 0.0;
    int64_t i, cnt = 0;
    for (i = 3; i + 3 < nb; ++i) {
        double mass = m[i - 2] + m[i - 1] + m[i] + m[i + 1] + m[i + 2];
        double ro = r[i + 3], ri = r[i - 3];
        double vol = (4.0 * OR_PI / 3.0) * (ro * ro * ro - ri * ri * ri);
        double rho;
        if (!(vol > 0.0)) continue;
        rho = mass / vol;
        s1 = s1 + rho;
        s2 = s2 + rho * rho;
        sr = sr + rho * r[i];
        ++cnt;
    }
    out[0] = s1 > 0.0 ? s2 / s1 : 0.0;
    out[1] = s1 > 0.0 ? sr / s1 : 0.0;
    out[2] = (double)cnt;
}

/* The estimates rho_i themselves (0 where there is none), for the tests. */
void or_core_rho(int64_t nb, const double *r, const double *m, double *rho)
{
    int64_t i;
    for (i = 0; i < nb; ++i) {
        double vol;
        rho[i] = 0.0;
        if (i < 3 || i + 3 >= nb) continue;
        vol = (4.0 * OR_PI / 3.0) * (r[i + 3] * r[i + 3] * r[i + 3] - r[i - 3] * r[i - 3] * r[i - 3]);
        if (vol > 0.0) rho[i] = (m[i - 2] + m[i - 1] + m[i] + m[i + 1] + m[i + 2]) / vol;
    }
}

/* ------------------------------------------------------------------------ */
/* One full timestep of one cluster, in the order of section 3.3:            */
/* timestep -> relaxation -> new orbits -> sort -> potential -> energy       */
/* correction.  On entry the first *nb stars are bound and sorted, phi holds */
/* their potential; on exit the same holds for the new state.                */
/* stats[]: 0 escaped this step, 1 degenerate orbits, 2 rejection-cap hits,  */
/*          3 trials, 4 g > F violations, 5 T' clamps, 6 angle-draw fails.   */
/* Returns dt.  pot_mode: 0 = Eqs. 2-5 recursion, 1 = double-double scan.    */
/* esc_io (may be NULL) accumulates what the escapers carry off (the        */
/* energy budget of section 4.2): [0] += m_k, [1] += m_k e_k, with          */
/* e_k = Phi_k + m_k / r_k + (v_r^2 + v_t^2) / 2 the star's energy in the   */
/* field of the others (Phi_k includes the star's own mass), in star order. */
/* ------------------------------------------------------------------------ */
double or_step_col(int64_t n, int64_t *nb_io, double *r, double *vr, double *vt, double *m,
                   double *R, uint32_t *id, double *phi, uint64_t seed, uint32_t step,
                   int32_t bs, double pref, double lnL, int32_t max_trials, int32_t ecorr,
                   int32_t pot_mode, int64_t *stats, double *esc_io, double *col,
                   double *A, double x_bb, double x_bs, double dt_cap);

double or_step(int64_t n, int64_t *nb_io, double *r, double *vr, double *vt, double *m,
               uint32_t *id, double *phi, uint64_t seed, uint32_t step, int32_t bs,
               double pref, double lnL, int32_t max_trials, int32_t ecorr,
               int32_t pot_mode, int64_t *stats, double *esc_io)
{
    return or_step_col(n, nb_io, r, vr, vt, m, NULL, id, phi, seed, step, bs, pref, lnL,
                       max_trials, ecorr, pot_mode, stats, esc_io, NULL, NULL, 1.0, 1.0, 0.0);
}

/* The timestep with stellar radii R (may be NULL: or_step): the collision
 * timestep of Eq. 8 joins the minimum, relaxation pairs may merge (sticky
 * spheres), and a star merged away (radius -1, mass 0) leaves in the orbit
 * step (r = +inf, no energy carried off: it has no mass); R is permuted with
 * the stars; col[0] += mergers, col[1] += their change of K + W.  With the
 * binaries' semi-major axes A (may be NULL; permuted with the stars), T_bb
 * and T_bs of Eqs. 9 and 10 join the minimum; a positive finite dt_cap (an
 * outside bound such as Eq. 11's stellar-evolution step) joins it too. */
double or_step_col(int64_t n, int64_t *nb_io, double *r, double *vr, double *vt, double *m,
                   double *R, uint32_t *id, double *phi, uint64_t seed, uint32_t step,
                   int32_t bs, double pref, double lnL, int32_t max_trials, int32_t ecorr,
                   int32_t pot_mode, int64_t *stats, double *esc_io, double *col,
                   double *A, double x_bb, double x_bs, double dt_cap)
{
    int64_t nb = *nb_io, k;
    int64_t nbins = (nb + bs - 1) / bs;
    double dt;
    double *nbin = (double *)calloc((size_t)(nbins > 0 ? nbins : 1), sizeof(double));
    double *rn = (double *)malloc(sizeof(double) * (size_t)n);
    double *ro = (double *)malloc(sizeof(double) * (size_t)n);
    double *cc = (double *)malloc(sizeof(double) * (size_t)n);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    uint32_t *tid = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memset(stats, 0, 7 * sizeof(int64_t));

    dt = or_timestep(nb, r, vr, vt, m, bs, pref, lnL, nbin);
    if (R) {
        double tc = or_tcoll(nb, r, vr, vt, m, R);
        if (tc < dt) dt = tc;
    }
    if (A) {
        double tbs, tbb = or_tbinary(nb, r, vr, vt, m, A, x_bb, x_bs, &tbs);
        if (tbb < dt) dt = tbb;
        if (tbs < dt) dt = tbs;
    }
    if (dt_cap > 0.0 && dt_cap < dt) dt = dt_cap;
    stats[6] += or_relax_col(nb, vr, vt, m, R, id, nbin, bs, dt, lnL, seed, step, col, r, phi);

    for (k = 0; k < n; ++k) { rn[k] = r[k]; ro[k] = r[k]; cc[k] = 0.0; }
    for (k = 0; k < nb; ++k) {
        double out[8];
        int64_t viol = 0;
        int rc;
        if (R && R[k] < 0.0) {  /* merged into its partner in this step */
            rn[k] = INFINITY;
            continue;
        }
        rc = or_orbit_star(k, nb, r, phi, vr[k], vt[k], id[k], seed, step,
                           max_trials, out, &viol);
        stats[3] += (int64_t)out[7];
        stats[4] += viol;
        if (rc == 1) {
            stats[0] += 1;
            rn[k] = INFINITY;
            if (esc_io) {
                double e = phi[k] + m[k] / r[k] + 0.5 * (vr[k] * vr[k] + vt[k] * vt[k]);
                esc_io[0] += m[k];
                esc_io[1] += m[k] * e;
            }
            continue;
        }
        if (rc == 2) { stats[1] += 1; continue; }
        if (rc == 3) { stats[2] += 1; continue; }
        rn[k] = out[0];
        vr[k] = out[1];
        vt[k] = out[2];
        cc[k] = phi[k] - out[3];
    }

    or_sort_perm(n, rn, id, perm);
#define OR_PERMUTE(arr)                                              \
    do {                                                             \
        for (k = 0; k < n; ++k) tmp[k] = (arr)[perm[k]];             \
        memcpy((arr), tmp, sizeof(double) * (size_t)n);              \
    } while (0)
    OR_PERMUTE(vr);
    OR_PERMUTE(vt);
    OR_PERMUTE(m);
    if (R) OR_PERMUTE(R);
    if (A) OR_PERMUTE(A);
    OR_PERMUTE(ro);
    OR_PERMUTE(cc);
    for (k = 0; k < n; ++k) tmp[k] = rn[perm[k]];
    memcpy(r, tmp, sizeof(double) * (size_t)n);
    for (k = 0; k < n; ++k) tid[k] = id[perm[k]];
    memcpy(id, tid, sizeof(uint32_t) * (size_t)n);
#undef OR_PERMUTE

    nb = 0;
    while (nb < n && !isinf(r[nb])) ++nb;
    for (k = nb; k < n; ++k) phi[k] = 0.0;
    if (pot_mode == 1) or_potential_dd(nb, r, m, phi);
    else or_potential_recursion(nb, r, m, phi);
    if (ecorr) stats[5] += or_energy_correction(nb, r, phi, vr, vt, ro, cc, NULL);
    *nb_io = nb;

    free(nbin); free(rn); free(ro); free(cc); free(tmp); free(tid); free(perm);
    return dt;
}
