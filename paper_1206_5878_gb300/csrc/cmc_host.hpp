// Host-side internals of the CUDA library: the segment (cluster) layout on
// the device, scratch buffers, and the launchers of each kernel.  Nothing
// here is part of the C ABI (see include/cmc.h).
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "cmc_device.cuh"

namespace cmc {

// Device-resident description of the segments of one state.  Offsets are
// fixed at initialisation; nb, dt and the statistics change every step.
struct SegLayout {
  int n_seg = 0;
  int64_t n = 0;          // total stars
  int64_t n_tiles = 0;    // tiles of kTile elements, never straddling segments
  int64_t n_pairs = 0;    // pair slots (floor(n_c / 2) summed)
  int64_t n_bins = 0;     // bin slots (ceil(n_c / bin_size) summed)
  int bin_size = 20;
  std::vector<int64_t> h_off, h_tile_off, h_pair_off, h_bin_off;
  int64_t max_tiles_per_seg = 0;
  // device arrays
  int64_t* off = nullptr;
  int64_t* tile_off = nullptr;
  int64_t* pair_off = nullptr;
  int64_t* bin_off = nullptr;
  uint64_t* seed = nullptr;
  double* lnL = nullptr;
  int64_t* nb = nullptr;
  int64_t* esc_step = nullptr;      // stars escaped during the current step
  uint64_t* dt_bits = nullptr;
  uint64_t* dt_last = nullptr;      // timestep of the last completed step
  double* dt_cap = nullptr;         // outside bounds on the timestep (cmc_set_dt_cap; 0: none)
  unsigned long long* stats = nullptr;
  double* esc_me = nullptr;         // [n_seg][2]: mass, energy carried off by escapers
  uint4* taus = nullptr;            // combined-Tausworthe streams (stream mode only)
  int64_t* taus_base = nullptr;     // per segment: first stream slot
  int64_t taus_slots = 0;

  Seg dev() const {
    Seg s;
    s.off = off; s.tile_off = tile_off; s.pair_off = pair_off; s.bin_off = bin_off;
    s.seed = seed; s.lnL = lnL; s.nb = nb; s.dt_bits = dt_bits; s.dt_cap = dt_cap;
    s.stats = stats;
    s.taus = taus; s.taus_base = taus_base;
    s.n_seg = n_seg;
    return s;
  }
};

// Scratch of the radix sort (sized for a given layout).
struct SortWork {
  uint64_t* keys_alt = nullptr;
  uint32_t* vals_alt = nullptr;
  unsigned long long* desc = nullptr;   // [passes][n_tiles][256] look-back words
  uint32_t* hist = nullptr;             // [n_seg][passes][256]
  uint32_t* tickets = nullptr;          // [passes]
  uint32_t* done = nullptr;             // [n_seg] upsweep blocks finished
  size_t zero_bytes = 0;                // hist + tickets + done, then desc
  size_t zero_head = 0;                 // bytes before desc (zeroed with it per sort)
  void* zero_base = nullptr;
  int max_passes = 0;
  // shape of the digit passes: keys per thread (8 or 16) and multisplit
  // (0: __match_any_sync, 1: ballots); tiles of 256 * ipt keys
  int ipt = 16;
  int rank = 0;
  int64_t n_stiles = 0;
  int64_t* stile_off = nullptr;         // n_seg + 1 tile offsets of that shape
};

// choose the pass shape (host offsets are copied; not during stream capture)
cudaError_t sort_set_shape(const SegLayout& L, SortWork& W, int ipt, int rank,
                           cudaStream_t st);

// allocation helpers (stream-ordered); return cudaError_t
cudaError_t alloc_layout(SegLayout& L, const std::vector<int64_t>& sizes,
                         const std::vector<uint64_t>& seeds, const std::vector<double>& lnL,
                         int bin_size, cudaStream_t st);
void free_layout(SegLayout& L, cudaStream_t st);
cudaError_t alloc_sort(SortWork& W, const SegLayout& L, int max_passes, cudaStream_t st);
void free_sort(SortWork& W, cudaStream_t st);

// ------------------------------------------------------------- launchers
// Stable LSD radix sort of (keys, vals) within each segment over the 8-bit
// digits [first_pass, first_pass + passes).  When vals_identity is set the
// input values are taken to be the global positions.  After an even number
// of passes the result is in (keys, vals); after an odd number it is in the
// alternate buffers, which *keys_res / *vals_res then name when both are
// given (else it is copied back into keys, vals).
cudaError_t sort_segments(const SegLayout& L, SortWork& W, uint64_t* keys, uint32_t* vals,
                          int first_pass, int passes, bool vals_identity, uint32_t* err,
                          cudaStream_t st, uint64_t** keys_res = nullptr,
                          uint32_t** vals_res = nullptr, bool packed = false);

// Order every run of finite keys equal in their bits from `shift` up by
// (key, id of the element: ids_by_val[vals[p] * id_stride]), so that after
// a sort on those bits the (r, id) order holds (shift 0: runs of equal
// radii, ordered by id).
void launch_tiefix(const SegLayout& L, uint64_t* keys, uint32_t* vals,
                   const uint32_t* ids_by_val, int id_stride, uint32_t* err,
                   cudaStream_t st, int shift = 0);

void launch_philox(int64_t n, const uint32_t* ctr, uint64_t seed, uint32_t* out,
                   cudaStream_t st);

// One star between the orbit step and the sort (48 B).  c: for a bound
// star Phi_old(r_old) - Phi_old(r_new); for a star escaping in this step
// its energy in the field of the others, Phi_k + m_k / r_k + v^2 / 2.
struct Payload {
  double vr, vt, m, r_old, c;
  uint32_t id, pad;  // pad: with packed keys, the key's own low 24 bits
};

// Packed sort keys (every segment below 2^24 stars): a key's low 24 bits,
// which the timestep's radix passes do not sort, hold the star's index in
// its segment (the key's own low bits go to the payload), so that the
// passes move 8-byte keys and no values.
constexpr uint64_t kPackMask = 0xFFFFFFull;
constexpr int64_t kPackMax = (int64_t)1 << 24;
// the tie fix of packed keys (runs equal in bits 24-63 into (key, id) order)
void launch_tiefix_packed(const SegLayout& L, uint64_t* keys, const Payload* pay,
                          uint32_t* err, cudaStream_t st);

// keys of the current state (radius_key of r, id) and the payload (if pay)
void launch_make_keys(const SegLayout& L, const double* r, const double* vr,
                      const double* vt, const double* m, const uint32_t* id,
                      uint64_t* keys, Payload* pay, cudaStream_t st);

// keys = id (for the (r, id) order at initialisation), and radius keys of
// the stars in the order of a permutation
void launch_id_keys(const SegLayout& L, const uint32_t* id, uint64_t* keys, cudaStream_t st);
void launch_rekey_radius(const SegLayout& L, const uint32_t* perm, const double* r,
                         const uint32_t* id, uint64_t* keys, cudaStream_t st);

// sorted (keys, vals) + payload -> SoA state (r, x, vr, vt, m, id, r_old, c);
// with tile_m and tile_mx (and r_old, c) also the potential's per-tile sums
// over the bound stars after the orbit step (launch_potential with
// nb_sub and sums_ready then skips them)
void launch_gather(const SegLayout& L, const uint64_t* keys, const uint32_t* vals,
                   const Payload* pay, double* r, double* x, double* vr, double* vt,
                   double* m, uint32_t* id, double* r_old, double* c, cudaStream_t st,
                   double* tile_m = nullptr, double* tile_mx = nullptr,
                   const double* Rp = nullptr, double* Rout = nullptr,
                   const double* Ap = nullptr, double* Aout = nullptr,
                   bool packed = false);

// potential: per-tile sums then the tile-local scans (Eqs. 1-5 in scan
// form).  nb_sub: subtract esc_step from nb (after the orbit step).
// Optional outputs: t32 (float 1/r, Phi), Mout (M_k) and node (the record
// {r, 1/r, Phi, M_k} of every star: one 32-byte sector per node for the
// kernels that read a few nodes at random).  slopes: Mout and the records
// carry the slope of Eq. 6 across each shell instead of M_k (the shell
// parameter the FP64 orbit step takes).
// The orbit step's index tables as the potential kernel writes them beside
// Phi: the bucket starts and the grid's key shells (their per-segment
// parameters computed before it, from 1/r).
struct TableOut {
  int* start = nullptr;
  const int64_t* boff = nullptr;
  const uint32_t* base = nullptr;
  const int4* prm = nullptr;
  int* gshell = nullptr;
  const int64_t* goff = nullptr;
  const int4* gprm = nullptr;
};
void launch_potential(const SegLayout& L, const double* r, const double* x, const double* m,
                      double* tile_m, double* tile_mx, double* phi, float2* t32,
                      double* Mout, bool nb_sub, cudaStream_t st, double4_32a* node = nullptr,
                      float4* tdf = nullptr, bool sums_ready = false, bool slopes = false,
                      const TableOut* tables = nullptr);
// node records (and float-pair table) from the arrays (stage calls)
void launch_make_nodes(int64_t n, const double* r, const double* x, const double* phi,
                       const double* M, double4_32a* node, float4* tdf, cudaStream_t st);

void launch_correction(const SegLayout& L, const double* r, const double* x,
                       const double* phi, double* vr, double* vt, const double* r_old,
                       const double* c, bool nb_sub, uint32_t* err, cudaStream_t st,
                       const double* m = nullptr);

void launch_bins(const SegLayout& L, const double* r, const double* vr, const double* vt,
                 const double* m, double* nbin, double pref, cudaStream_t st);

// relaxation of the neighbour pairs; with stellar radii R (may be null)
// pairs may merge (sticky spheres; r and phi: the current table)
void launch_relax(const SegLayout& L, double* vr, double* vt, double* m, const uint32_t* id,
                  const double* nbin, const uint32_t* step, cudaStream_t st, int variant = 0,
                  double* R = nullptr, const double* r = nullptr, const double* phi = nullptr);
// The timesteps over the innermost 300 bound stars into the segments'
// timesteps: Eq. 8's collision step (R: stellar radii, may be null) and
// Eqs. 9-10's binary steps (A: semi-major axes, may be null)
void launch_tcentral(const SegLayout& L, const double* r, const double* vr, const double* vt,
                     const double* m, const double* R, const double* A, double x_bb,
                     double x_bs, cudaStream_t st);

struct OrbitStageOut {   // optional per-star outputs of the orbit stage
  double* phi_new = nullptr;
  double* rmin = nullptr;
  double* rmax = nullptr;
  double* F = nullptr;
  int32_t* code = nullptr;
  int32_t* trials = nullptr;
};

// Radius-bucket index of the float table of every segment (mixed mode):
// start[off[c] + b] = first node of segment c whose bucket is >= b.
//
// With it, a potential grid per segment: Phi (float) at the float keys
// key0 + g 2^sh of 1/r, sh = 23 - p for 2^p cells per binade, so that no
// cell straddles a power of two and Phi, linear in 1/r between stars, is
// close to linear in the key inside a cell.
struct BucketArgs {
  const int* start = nullptr;
  const int64_t* off = nullptr;
  const uint32_t* base = nullptr;
  const int4* prm = nullptr;  // shift, bucket count, first and last indexed node
  const float* gphi = nullptr;
  const int64_t* goff = nullptr;
  const int4* gprm = nullptr;    // key0, sh, cells, key of 1/r_0 (as int)
  const float4* gaux = nullptr;  // Phi_0, bound mass, 1/r at key0, interpolation bound
  const double4_32a* node = nullptr; // {r, 1/r, Phi, M} per star (potential kernel)
  const float4* tdf = nullptr;       // {1/r, Phi} per star as float pairs (hi, lo, hi, lo)
};

struct BucketWork {
  int* start = nullptr;
  int64_t* off = nullptr;
  uint32_t* base = nullptr;
  int4* prm = nullptr;
  float* gphi = nullptr;
  int* gshell = nullptr;  // shell of every grid key (scratch of the grid build)
  int64_t* goff = nullptr;
  int4* gprm = nullptr;
  float4* gaux = nullptr;
  int64_t gcells = 0;  // grid cells over all segments
  double4_32a* node = nullptr;
  float4* tdf = nullptr;
  BucketArgs args() const {
    BucketArgs a;
    a.start = start; a.off = off; a.base = base; a.prm = prm;
    a.gphi = gphi; a.goff = goff; a.gprm = gprm; a.gaux = gaux;
    a.node = node;
    a.tdf = tdf;
    return a;
  }
};

cudaError_t alloc_buckets(BucketWork& B, const SegLayout& L, cudaStream_t st);
void free_buckets(BucketWork& B, cudaStream_t st);
// build the index from t32 over the bound stars (nb - esc_step when nb_sub)
void launch_buckets(const SegLayout& L, const float2* t32, bool nb_sub, BucketWork& B,
                    cudaStream_t st);
// build the potential grid from the FP64 table (x, Phi, enclosed masses)
void launch_grid(const SegLayout& L, const double* x, const double* phi, const double* Menc,
                 bool nb_sub, BucketWork& B, cudaStream_t st);
// The potential with the orbit step's tables in three kernels: the
// segments' bucket and grid parameters (from 1/r), the potential writing Phi,
// the slopes, node records, float tables, bucket starts and grid key shells,
// then the grid's values with the slopes at the tile seams.  The same tables
// as launch_potential + launch_buckets + launch_grid (slopes mode).
void launch_potential_tables(const SegLayout& L, const double* r, const double* x,
                             const double* m, double* tile_m, double* tile_mx, double* phi,
                             float2* t32, double* Menc, bool nb_sub, bool sums_ready,
                             BucketWork& B, cudaStream_t st);

// Menc (precision 0 and 1): the slope of Phi in 1/r across shell k.
// precision 1 (mixed): launch_orbit runs four kernels (turning points,
// FP32 sampler, FP64 continuation of the pending stars, finishing) and
// needs n records orb (E, J, c0 = (r_max + r_min) / 2, c1 = (r_max -
// r_min) / 4, from the turning-point kernel, for the sampling kernels), a
// list of n uint32 (the pending stars) and one uint32 counter; tp_min,
// tp_max (n doubles each: the turning points) only with the stage outputs
// of dbg (rmin, rmax).
// precision 0 (FP64): the same kernels with FP64 mode's envelope (two more
// kernels, into an EnvWork) and FP64 mode's points, every decision the FP64
// one.  precision 2 (FP64 by bisection): one kernel on the FP64 table.
void launch_slopes(int64_t n, const double* x, const double* phi, double* Menc,
                   cudaStream_t st);
// one diagnostics record per segment (after the step end; K, W in out3)
void launch_diag_ring(const SegLayout& L, const double* out3, const uint32_t* step,
                      const uint32_t* err, double* ring, int cap, cudaStream_t st);
// FP64 mode's envelope F = 1.2 max_j g(s_j): gmax (n doubles) the maximum
// per star; star (n records) the values its evaluations share; the (star,
// sample) pairs that FP32 bounds cannot rule out, each
// evaluated in FP64 by one thread (list: cap entries p << 5 | j); the stars
// whose pairs found the list full (spill: n entries p << 21 | sample mask);
// cnt[0] pairs, cnt[1] spilled stars
struct EnvWork {
  double* gmax = nullptr;
  double4_32a* star = nullptr;  // E, J, c0, c1 of each star with pairs
  uint64_t* list = nullptr;
  uint64_t* spill = nullptr;
  unsigned long long* cnt = nullptr;
  int64_t cap = 0;
};
cudaError_t alloc_env(EnvWork& W, int64_t n, cudaStream_t st);
void free_env(EnvWork& W, cudaStream_t st);

void launch_orbit(const SegLayout& L, int precision, int max_trials, const double* r,
                  const double* x, const double* phi, const double* Menc,
                  const double* vr,
                  const double* vt, const double* m, const uint32_t* id, const uint32_t* step,
                  uint64_t* keys, Payload* pay, const OrbitStageOut* dbg, int block,
                  int variant, const BucketArgs& ba, double* tp_min, double* tp_max,
                  uint32_t* plist, uint32_t* pcount, cudaStream_t st,
                  bool with_turning = true, const double* Rv = nullptr, double* Rp = nullptr,
                  const EnvWork* env = nullptr, const double* Av = nullptr,
                  double* Ap = nullptr, double4_32a* orb = nullptr, bool packed = false);
// the turning-point kernel alone (mixed mode; launch_orbit(..., false)
// then runs the sampling kernel only)
void launch_turning(const SegLayout& L, const double* r, const double* x, const double* phi,
                    const double* Menc, const double* vr, const double* vt,
                    const BucketArgs& ba, double* tp_min, double* tp_max, double4_32a* orb,
                    int block, cudaStream_t st);
// mixed-mode orbit variants: register caps for 1 (none), 2, 3, 4, 5, 6 and
// 8 resident 256-thread blocks per SM (128, 80, 64, 48, 40 and 32
// registers; the kernel is latency-bound, and occupancy buys more than the
// spills cost)
constexpr int kOrbitVariants = 7;
constexpr int kRelaxVariants = 3;  // relaxation kernel register caps (launch_relax)

// commits the step: nb, escaper statistics and budget (from the gathered
// r_old and c of the escaped range), dt; resets the per-step counters
// energy correction in mixed mode: shell of r_old from the bucket index of
// the new table (nb - esc_step bound stars), Phi from the enclosed mass
void launch_correction_mixed(const SegLayout& L, const double* r, const double* x,
                             const double* phi, const double* Menc,
                             const BucketArgs& ba, double* vr, double* vt, const double* r_old,
                             const double* c, const double* m, cudaStream_t st,
                             bool div_form = false);

void launch_step_end(const SegLayout& L, uint32_t* step, const double* r_old, const double* c,
                     const double* m, cudaStream_t st);

// energy diagnostics: per-segment K, W_pair (Mbuf receives M_k)
void launch_energy(const SegLayout& L, const double* r, const double* vr, const double* vt,
                   const double* m, double* tile_m, double* tile_k, double* tile_w,
                   double* Mbuf, double* out3, cudaStream_t st);

// core diagnostics (Eq. 19) per cluster: out3 = {rho_c, r_c, estimates};
// tiles4: 4 * n_tiles doubles of scratch
void launch_core(const SegLayout& L, const double* r, const double* m, double* tiles4,
                 double* out3, cudaStream_t st);
void launch_lagrange(const SegLayout& L, const double* r, const double* M,
                     const double* fracs, int nf, double* out, cudaStream_t st);

void launch_validate(const SegLayout& L, const double* r, const double* vr,
                     const double* vt, const double* m, bool allow_inf, uint32_t* err,
                     cudaStream_t st);

// nb of every segment = position of its first escaper key (sorted keys)
void launch_nb_from_keys(const SegLayout& L, const uint64_t* keys, cudaStream_t st);
void launch_recip(int64_t n, const double* r, double* x, cudaStream_t st);
void launch_make_t32(int64_t n, const double* x, const double* phi, float2* t32,
                     cudaStream_t st);
void launch_unpack_orbit(int64_t n, const uint64_t* keys, const Payload* pay, double* r_new,
                         double* vr_new, double* vt_new, cudaStream_t st);
void sort_prepare();
// look-back polls and tie-fix moves before the sort's waits give up (<= 0:
// the defaults), on the current device
cudaError_t set_wait_limits(int spin_polls, long long tie_moves);
void potential_prepare();  // shared-memory limit of the potential kernel

// (r, id) order of staged stars (flag bit 0 set when not) and the largest id
// per segment (maxid: n_seg values, zeroed by the caller)
void launch_order_check(const SegLayout& L, const double* r, const uint32_t* id, uint32_t* flag,
                        unsigned int* maxid, cudaStream_t st);
// duplicate ids by a bitmap with bitoff[c] + id per star (kErrInput)
void launch_ids_bitmap(const SegLayout& L, const uint32_t* id, const unsigned long long* bitoff,
                       unsigned long long* bitmap, uint32_t* err, cudaStream_t st);
// starting states of the Tausworthe streams (dynamics.cu): slots of
// segment c from base[c] (n_seg + 1 offsets), words: the segment's seeded
// words, P: [4][32][32] jump matrices T^(2^(80 + b))
void launch_taus_init(int64_t slots, int n_seg, const int64_t* base, const uint4* words,
                      const uint32_t* P, uint4* table, cudaStream_t st);
void launch_check_ids(const SegLayout& L, const uint64_t* sorted_ids, uint32_t* err,
                      cudaStream_t st);

// The first failed index check of each translation unit of a debug build
// since the last call (0: none), cleared; 0 in a release build.
uint32_t debug_site_tu1();
uint32_t debug_site_tu2();
uint32_t debug_site_tu3();
uint32_t debug_site_tu4();
uint32_t debug_site_tu5();
#define CMC_CAT2(a, b) a##b
#define CMC_CAT(a, b) CMC_CAT2(a, b)
#ifdef CMC_DEBUG
#define CMC_DEBUG_SITE_ACCESSOR                                              \
  uint32_t CMC_CAT(debug_site_tu, CMC_TU)() {                                \
    unsigned int v = 0u, z = 0u;                                             \
    cudaMemcpyFromSymbol(&v, g_debug_site, sizeof(v));                       \
    cudaMemcpyToSymbol(g_debug_site, &z, sizeof(z));                         \
    return v;                                                                \
  }
#else
#define CMC_DEBUG_SITE_ACCESSOR \
  uint32_t CMC_CAT(debug_site_tu, CMC_TU)() { return 0u; }
#endif

}  // namespace cmc
