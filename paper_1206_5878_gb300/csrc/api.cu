// C ABI (include/cmc.h): the context that advances clusters timestep by
// timestep, and the stage functions that run one step of the hot path on
// caller arrays.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cmc_host.hpp"
#include "../../include/cmc.h"

using namespace cmc;

struct cmc_ctx {
  cmc_config cfg{};
  cudaStream_t stream = nullptr;      // caller's stream (may be the default)
  cudaStream_t cap = nullptr;         // private stream used to capture the graph
                                      // (and as a second stream by load_state)
  cudaEvent_t ev_rim = nullptr, ev_aux = nullptr;  // load_state's ordering
  int device = 0;
  SegLayout L;
  SortWork W;
  BucketWork bk;  // radius-bucket index, grid and node records (precision 0 and 1)
  double pref = 0.0;
  // state (sorted SoA)
  double *r = nullptr, *x = nullptr, *vr = nullptr, *vt = nullptr, *m = nullptr,
         *phi = nullptr;
  uint32_t* id = nullptr;
  float2* t32 = nullptr;
  // scratch
  uint64_t* keys = nullptr;
  uint32_t* vals = nullptr;
  Payload* pay = nullptr;
  double *r_old = nullptr, *cc = nullptr, *nbin = nullptr;
  double *tile_a = nullptr, *tile_b = nullptr, *tile_c = nullptr, *Mbuf = nullptr,
         *out3 = nullptr, *fr = nullptr, *lag = nullptr;
  uint32_t* err = nullptr;
  uint32_t* step = nullptr;
  uint32_t* pcount = nullptr;  // pending stars of the sampled orbit step
  EnvWork env;                 // FP64 mode's envelope (precision 0)
  double4_32a* orb = nullptr;  // E, J, c0, c1 of every star's orbit (precision 0 and 1)
  bool packed = false;         // the timestep sorts packed keys (cfg.sort_packed, clusters < 2^24)
  double* ring = nullptr;      // per-step diagnostics (cfg.diag_ring records per cluster)
  int64_t steps_taken = 0;
  cudaGraphExec_t exec = nullptr;
  bool poisoned = false;
  std::string last_error;
  int kernels_per_step = 0;
  int orbit_variant = 0;  // sampler kernel variant (see kOrbitVariants)
  int relax_variant = 0;  // relaxation kernel variant (see kRelaxVariants)
  // stellar radii (cfg.collisions): the state's, and their copy through the sort
  double *R = nullptr, *Rp = nullptr;
  // semi-major axes (cfg.binaries; 0 for single stars), likewise
  double *A = nullptr, *Ap = nullptr;
};

namespace {

thread_local std::string g_err;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

cmc_status fail(cmc_ctx* ctx, cmc_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  else g_err = msg;
  return s;
}

cmc_status cuda_fail(cmc_ctx* ctx, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(ctx, CMC_ENOMEM, msg);
  return fail(ctx, CMC_ECUDA, msg);
}

template <class T>
cudaError_t dalloc(T*& p, size_t count, cudaStream_t st) {
  return cudaMallocAsync((void**)&p, sizeof(T) * (count ? count : 1), st);
}

template <class T>
void dfree(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
}

double t_rel_prefactor(double theta_max) {
  return (theta_max / (kPi / 2)) * (kPi / 32);
}

cmc_status check_err_flags(cmc_ctx* ctx) {
  uint32_t e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, ctx->err, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                   ctx->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) {
    ctx->poisoned = true;
    return cuda_fail(ctx, ce, "device work");
  }
  if (e == 0) return CMC_OK;
  ctx->poisoned = true;
  std::string msg = "device error flags:";
  if (e & kErrTimeout) msg += " bounded wait expired in the sort look-back;";
  if (e & kErrTies) msg += " run of equal radii too long to order by id;";
  if (e & kErrInput) msg += " invalid input state;";
  if (e & kErrNonFinite) msg += " non-finite value;";
  if (e & kErrTimeout) return fail(ctx, CMC_ETIMEOUT, msg);
  if (e & kErrInput) {
    ctx->poisoned = false;  // nothing was changed on the device state yet
    return fail(ctx, CMC_EINVAL, msg);
  }
  return fail(ctx, CMC_ECUDA, msg);
}

// Whether the staged stars are already in (r, id) order in every segment
// with ids that fit a bitmap of the key scratch (64 bits per star): then
// bitoff receives each segment's first bit.  A state read back with
// cmc_get_state always qualifies.
bool staged_in_order(cmc_ctx* c, std::vector<unsigned long long>& bitoff, cudaStream_t st) {
  const SegLayout& L = c->L;
  unsigned int* d = nullptr;  // [0] order flag, [1 + s] largest id of segment s
  if (dalloc(d, (size_t)L.n_seg + 1, st)) return false;
  std::vector<unsigned int> h((size_t)L.n_seg + 1, 1u);
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned int) * h.size(), st);
  if (!e) {
    launch_order_check(L, c->r, c->id, d, d + 1, st);
    e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned int) * h.size(), cudaMemcpyDeviceToHost, st);
  }
  if (!e) e = cudaStreamSynchronize(st);
  dfree(d, st);
  if (e || h[0] != 0u) return false;
  bitoff.assign((size_t)L.n_seg, 0ull);
  unsigned long long total = 0;
  for (int s = 0; s < L.n_seg; ++s) {
    bitoff[s] = total;
    total += (unsigned long long)h[1 + s] + 1ull;
  }
  return total <= 64ull * (unsigned long long)L.n;
}

// Sort the staged stars in r, vr, vt, m, id by (r, id) per segment and
// compute nb and the potential.  Ids must be unique per segment.  Stars
// already in order (a state read back and set again) keep their places: the
// order was checked, the ids are checked with a bitmap, and both sorts and
// the gather are skipped.
// Stars already in (r, id) order: the ids checked with a bitmap, the keys
// and 1/r written in place (r and id only: no sort, no gather).  False when
// the bitmap's scratch could not be had.
bool order_in_place(cmc_ctx* c, const std::vector<unsigned long long>& bitoff,
                    cudaStream_t st) {
  const SegLayout& L = c->L;
  unsigned long long* dbo = nullptr;
  if (dalloc(dbo, bitoff.size(), st)) return false;
  cudaMemcpyAsync(dbo, bitoff.data(), sizeof(unsigned long long) * bitoff.size(),
                  cudaMemcpyHostToDevice, st);
  // the bitmap lives in the key scratch (64 bits per star)
  cudaMemsetAsync(c->keys, 0, sizeof(uint64_t) * (size_t)L.n, st);
  launch_ids_bitmap(L, c->id, dbo, reinterpret_cast<unsigned long long*>(c->keys), c->err, st);
  launch_make_keys(L, c->r, nullptr, nullptr, nullptr, c->id, c->keys, nullptr, st);
  launch_recip(L.n, c->r, c->x, st);
  cudaStreamSynchronize(st);  // bitoff lives on the caller's stack frame
  dfree(dbo, st);
  return true;
}

// N_bound from the keys, then the potential and the orbit step's tables
void finish_order(cmc_ctx* c, cudaStream_t st) {
  const SegLayout& L = c->L;
  launch_nb_from_keys(L, c->keys, st);
  cudaMemsetAsync(L.esc_step, 0, sizeof(int64_t) * L.n_seg, st);
  // the float tables, node records and indexes of the sampled orbit step
  // (precision 0 and 1)
  if (c->cfg.precision != 2)
    launch_potential_tables(L, c->r, c->x, c->m, c->tile_a, c->tile_b, c->phi, c->t32, c->Mbuf,
                            false, false, c->bk, st);
  else
    launch_potential(L, c->r, c->x, c->m, c->tile_a, c->tile_b, c->phi, nullptr, nullptr, false,
                     st);
}

void order_state(cmc_ctx* c, cudaStream_t st) {
  const SegLayout& L = c->L;
  std::vector<unsigned long long> bitoff;
  if (!(L.n > 0 && staged_in_order(c, bitoff, st) && order_in_place(c, bitoff, st))) {
    launch_id_keys(L, c->id, c->keys, st);
    sort_segments(L, c->W, c->keys, c->vals, 0, 4, true, c->err, st);
    launch_check_ids(L, c->keys, c->err, st);
    launch_rekey_radius(L, c->vals, c->r, c->id, c->keys, st);
    sort_segments(L, c->W, c->keys, c->vals, 0, 8, false, c->err, st);
    launch_make_keys(L, c->r, c->vr, c->vt, c->m, c->id, c->W.keys_alt, c->pay, st);
    launch_gather(L, c->keys, c->vals, c->pay, c->r, c->x, c->vr, c->vt, c->m, c->id, nullptr,
                  nullptr, st);
  }
  finish_order(c, st);
}

// stage names (cmc_step_profiled, NVTX ranges)
const char* const kStageName[CMC_NSTAGES] = {"timestep", "relax",     "turning",
                                             "orbit",    "sort",      "gather",
                                             "potential", "correction", "end"};

// The kernels of one timestep, in the order of section 3.3.  With ev, an
// event is recorded before the first stage and after every stage, and
// every stage is an NVTX range (for timeline tools).
void record_step(cmc_ctx* c, cudaStream_t st, cudaEvent_t* ev = nullptr) {
  const SegLayout& L = c->L;
  const bool mixed = c->cfg.precision == 1, tab = c->cfg.precision != 2;
  auto mark = [&](int i) {
    if (!ev) return;
    cudaEventRecord(ev[i], st);
    if (i > 0) nvtxRangePop();
    if (i < CMC_NSTAGES) nvtxRangePushA(kStageName[i]);
  };
  mark(0);
  launch_bins(L, c->r, c->vr, c->vt, c->m, c->nbin, c->pref, st);
  launch_tcentral(L, c->r, c->vr, c->vt, c->m, c->R, c->A, c->cfg.x_bb, c->cfg.x_bs, st);
  mark(1);
  launch_relax(L, c->vr, c->vt, c->m, c->id, c->nbin, c->step, st, c->relax_variant, c->R, c->r,
               c->phi);
  mark(2);
  // the turning points (as the orbit records), then sampling
  if (tab)
    launch_turning(L, c->r, c->x, c->phi, c->Mbuf, c->vr, c->vt, c->bk.args(), nullptr,
                   nullptr, c->orb, c->cfg.orbit_block, st);
  mark(3);
  launch_orbit(L, c->cfg.precision, c->cfg.max_trials, c->r, c->x, c->phi,
               tab ? c->Mbuf : nullptr, c->vr, c->vt, c->m, c->id,
               c->step, c->keys, c->pay, nullptr, c->cfg.orbit_block, c->orbit_variant,
               c->bk.args(), c->r_old, c->cc, c->vals, c->pcount, st, false, c->R, c->Rp,
               c->cfg.precision == 0 ? &c->env : nullptr, c->A, c->Ap, c->orb, c->packed);
  mark(4);
  // radix passes over bits 24-63 of the radius keys; runs equal in those
  // bits (radii within 2^-28 of each other, escapers whose ids differ in
  // their low 4 bits) are put in (key, id) order after
  uint64_t* sk = nullptr;
  uint32_t* sv = nullptr;
  sort_segments(L, c->W, c->keys, c->vals, 3, 5, true, c->err, st, &sk, &sv, c->packed);
  if (c->packed)
    launch_tiefix_packed(L, sk, c->pay, c->err, st);
  else
    launch_tiefix(L, sk, sv, &c->pay[0].id, (int)(sizeof(Payload) / sizeof(uint32_t)), c->err,
                  st, 24);
  mark(5);
  launch_gather(L, sk, sv, c->pay, c->r, c->x, c->vr, c->vt, c->m, c->id, c->r_old, c->cc, st,
                c->tile_a, c->tile_b, c->Rp, c->R, c->Ap, c->A, c->packed);
  mark(6);
  // the tables carry the shell slopes of the FP64 orbit step (not the
  // scan's enclosed masses): the sampled step's turning points and points
  // are then FP64 mode's
  if (tab)
    launch_potential_tables(L, c->r, c->x, c->m, c->tile_a, c->tile_b, c->phi, c->t32, c->Mbuf,
                            true, true, c->bk, st);
  else
    launch_potential(L, c->r, c->x, c->m, c->tile_a, c->tile_b, c->phi, nullptr, nullptr, true,
                     st, nullptr, nullptr, true);
  mark(7);
  if (c->cfg.energy_correction) {
    // with the tables (precision 0 and 1) the shell of r_old comes from the
    // bucket index; FP64 mode evaluates Phi in Eq. 6's division form
    if (tab)
      launch_correction_mixed(L, c->r, c->x, c->phi, c->Mbuf, c->bk.args(), c->vr, c->vt,
                              c->r_old, c->cc, c->m, st, !mixed);
    else
      launch_correction(L, c->r, c->x, c->phi, c->vr, c->vt, c->r_old, c->cc, true, c->err, st,
                        c->m);
  }
  mark(8);
  launch_step_end(L, c->step, c->r_old, c->cc, c->m, st);
  if (c->ring) {
    // K and W of the new state (r_old is free scratch now), then the record
    launch_energy(L, c->r, c->vr, c->vt, c->m, c->tile_a, c->tile_b, c->tile_c, c->r_old,
                  c->out3, st);
    launch_diag_ring(L, c->out3, c->step, c->err, c->ring, c->cfg.diag_ring, st);
  }
  mark(9);
}

int count_step_kernels(const cmc_ctx* c) {
  // bins, relax, orbit, upsweep (with the histograms' scans), 5 passes, tie fix, gather with
  // the tile sums, potential, [precision 0 and 1: turning points, FP32
  // sampler, FP64 continuation, the tables' parameters, the grid's values
  // with the seams' slopes; precision 0: the envelope's screen and
  // evaluation], [correction], step end
  const int p = c->cfg.precision;
  return 3 + ((c->R || c->A) ? 1 : 0) + (c->ring ? 4 : 0) + 1 + 5 + 1 + 1 + 1 +
         (p == 1 ? 5 : p == 0 ? 7 : 0) +
         (c->cfg.energy_correction ? 1 : 0) + 1;
}

void free_ctx(cmc_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  double** ds[] = {&c->r, &c->x, &c->vr, &c->vt, &c->m, &c->phi, &c->r_old, &c->cc, &c->nbin,
                   &c->tile_a, &c->tile_b, &c->tile_c, &c->Mbuf, &c->out3, &c->fr, &c->lag};
  for (double** p : ds) dfree(*p, st);
  dfree(c->id, st);
  dfree(c->R, st);
  dfree(c->Rp, st);
  dfree(c->A, st);
  dfree(c->Ap, st);
  dfree(c->t32, st);
  dfree(c->keys, st);
  dfree(c->vals, st);
  dfree(c->pay, st);
  dfree(c->err, st);
  dfree(c->step, st);
  dfree(c->pcount, st);
  free_env(c->env, st);
  dfree(c->orb, st);
  dfree(c->ring, st);
  free_sort(c->W, st);
  free_buckets(c->bk, st);
  dfree(c->L.taus, st);
  dfree(c->L.taus_base, st);
  free_layout(c->L, st);
  cudaStreamSynchronize(st);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->ev_rim) cudaEventDestroy(c->ev_rim);
  if (c->ev_aux) cudaEventDestroy(c->ev_aux);
  delete c;
}

// A state set from outside.  r, id and m are copied first: the order check,
// N_bound, the potential and its tables need only them, so on the second
// stream they run while v_r and v_t are still arriving (from host memory
// the copies are the longer part).  A state in (r, id) order keeps its
// places; validation (every array) follows once all have landed.  A state
// out of order is validated first (the sort needs finite keys), then
// sorted.
cmc_status load_state(cmc_ctx* c, const double* r, const double* vr, const double* vt,
                      const double* m, const uint32_t* id, int32_t ptr_kind, bool allow_inf,
                      int64_t step) {
  const SegLayout& L = c->L;
  const size_t n = (size_t)L.n;
  const cudaMemcpyKind k = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaStream_t st = c->stream, aux = c->cap;
  cudaMemsetAsync(c->err, 0, sizeof(uint32_t), st);
  uint32_t st32 = (uint32_t)step;
  cudaError_t e = cudaMemcpyAsync(c->step, &st32, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(c->r, r, n * sizeof(double), k, st);
  if (!e) e = cudaMemcpyAsync(c->id, id, n * sizeof(uint32_t), k, st);
  if (!e) e = cudaMemcpyAsync(c->m, m, n * sizeof(double), k, st);
  if (!e) e = cudaEventRecord(c->ev_rim, st);
  if (!e) e = cudaMemcpyAsync(c->vr, vr, n * sizeof(double), k, st);
  if (!e) e = cudaMemcpyAsync(c->vt, vt, n * sizeof(double), k, st);
  if (!e) e = cudaStreamWaitEvent(aux, c->ev_rim, 0);
  if (e) return cuda_fail(c, e, "copy in");
  std::vector<unsigned long long> bitoff;
  bool placed = false;
  if (L.n > 0 && staged_in_order(c, bitoff, aux) && order_in_place(c, bitoff, aux)) {
    finish_order(c, aux);
    placed = true;
  }
  e = cudaEventRecord(c->ev_aux, aux);
  if (!e) e = cudaStreamWaitEvent(st, c->ev_aux, 0);
  if (e) return cuda_fail(c, e, "ordering the state");
  launch_validate(c->L, c->r, c->vr, c->vt, c->m, allow_inf, c->err, st);
  cmc_status s = check_err_flags(c);
  if (s != CMC_OK) return s;
  if (!placed) {
    order_state(c, st);
    e = cudaGetLastError();
    if (e) return cuda_fail(c, e, "ordering the state");
    s = check_err_flags(c);
    if (s != CMC_OK) return s;
  }
  c->steps_taken = step;
  return CMC_OK;
}

// Time the shapes of the sort passes and of the orbit kernel on this state
// and keep the fastest.  The orbit kernel runs once as a dry run (it writes
// only keys and payload scratch) to give the sort realistic input; counters
// it touched are reset.  Results never depend on the shapes.
// ------------------------------------------------ Tausworthe streams (host)
// Components (k, q, s) of the combined generator (section 3.6; L'Ecuyer
// 1999) and one step of a component word; every step is linear over GF(2).
constexpr int kTausK[4] = {31, 29, 28, 25}, kTausQ[4] = {6, 2, 13, 3},
              kTausS[4] = {18, 2, 7, 13};

uint32_t taus_word_host(uint32_t z, int j) {
  const uint32_t b = ((z << kTausQ[j]) ^ z) >> (kTausK[j] - kTausS[j]);
  return ((z & (0xFFFFFFFFu << (32 - kTausK[j]))) << kTausS[j]) ^ b;
}

// 32 x 32 matrices over GF(2) as columns (the image of each bit)
uint32_t gf2_times(const uint32_t* col, uint32_t v) {
  uint32_t r = 0u;
  for (int i = 0; i < 32; ++i)
    if ((v >> i) & 1u) r ^= col[i];
  return r;
}

void gf2_square(uint32_t* m) {
  uint32_t t[32];
  for (int i = 0; i < 32; ++i) t[i] = gf2_times(m, m[i]);
  for (int i = 0; i < 32; ++i) m[i] = t[i];
}

// P[j][b] = T_j^(2^(80 + b)) for b = 0..31: T_j squared 80 times, then once
// more per b
std::vector<uint32_t> taus_jump_matrices() {
  std::vector<uint32_t> P(4 * 32 * 32);
  for (int j = 0; j < 4; ++j) {
    uint32_t m[32];
    for (int i = 0; i < 32; ++i) m[i] = taus_word_host(1u << i, j);
    for (int k = 0; k < 80; ++k) gf2_square(m);
    for (int b = 0; b < 32; ++b) {
      for (int i = 0; i < 32; ++i) P[((size_t)j * 32 + b) * 32 + i] = m[i];
      gf2_square(m);
    }
  }
  return P;
}

// seeded starting words of a cluster's sequence (reading): two splitmix64
// outputs (Steele, Lea & Flood 2014) of the cluster seed, the top bit of
// each word set so that every component state is nonzero
void taus_seed_words(uint64_t seed, uint32_t w[4]) {
  uint64_t x = seed, o[2];
  for (int i = 0; i < 2; ++i) {
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    o[i] = z ^ (z >> 31);
  }
  w[0] = (uint32_t)o[0] | 0x80000000u;
  w[1] = (uint32_t)(o[0] >> 32) | 0x80000000u;
  w[2] = (uint32_t)o[1] | 0x80000000u;
  w[3] = (uint32_t)(o[1] >> 32) | 0x80000000u;
}

// One stream slot per id of every cluster (slot = base + id), started at
// T^(id 2^80) of the cluster's seeded words.  Ids must stay below
// 4 N_c + 64 so that the slots stay within a few words per star.
cmc_status init_streams(cmc_ctx* c, const uint64_t* seeds) {
  SegLayout& L = c->L;
  cudaStream_t st = c->stream;
  unsigned int* d = nullptr;
  std::vector<unsigned int> h((size_t)L.n_seg + 1, 0u);
  cudaError_t e = dalloc(d, h.size(), st);
  if (!e) e = cudaMemsetAsync(d, 0, sizeof(unsigned int) * h.size(), st);
  if (!e) {
    launch_order_check(L, c->r, c->id, d, d + 1, st);
    e = cudaMemcpyAsync(h.data(), d, sizeof(unsigned int) * h.size(), cudaMemcpyDeviceToHost, st);
  }
  if (!e) e = cudaStreamSynchronize(st);
  dfree(d, st);
  if (e) return cuda_fail(c, e, "cmc_init: streams");
  std::vector<int64_t> base((size_t)L.n_seg + 1, 0);
  std::vector<uint32_t> words((size_t)4 * L.n_seg);
  for (int s = 0; s < L.n_seg; ++s) {
    const int64_t nc = L.h_off[s + 1] - L.h_off[s];
    if ((int64_t)h[1 + s] >= 4 * nc + 64)
      return fail(c, CMC_EINVAL, "cmc_init: the Tausworthe streams need ids below 4 N + 64");
    base[s + 1] = base[s] + (int64_t)h[1 + s] + 1;
    taus_seed_words(seeds[s], &words[4 * (size_t)s]);
  }
  const std::vector<uint32_t> P = taus_jump_matrices();
  uint32_t* dP = nullptr;
  uint4* dw = nullptr;
  L.taus_slots = base[L.n_seg];
  e = dalloc(L.taus, (size_t)L.taus_slots, st);
  if (!e) e = dalloc(L.taus_base, base.size(), st);
  if (!e) e = dalloc(dP, P.size(), st);
  if (!e) e = dalloc(dw, (size_t)L.n_seg, st);
  if (!e) e = cudaMemcpyAsync(L.taus_base, base.data(), sizeof(int64_t) * base.size(),
                              cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(dP, P.data(), sizeof(uint32_t) * P.size(), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(dw, words.data(), sizeof(uint32_t) * words.size(),
                              cudaMemcpyHostToDevice, st);
  if (!e) {
    launch_taus_init(L.taus_slots, L.n_seg, L.taus_base, dw, dP, L.taus, st);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(st);  // the host vectors live on this frame
  dfree(dP, st);
  dfree(dw, st);
  if (e) return cuda_fail(c, e, "cmc_init: streams");
  return CMC_OK;
}

cmc_status autotune(cmc_ctx* c) {
  const SegLayout& L = c->L;
  cudaStream_t st = c->stream;
  const bool tab = c->cfg.precision != 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // the dry runs draw from the streams: keep a copy to put back
  uint4* taus_saved = nullptr;
  if (L.taus) {
    cudaError_t es = dalloc(taus_saved, (size_t)L.taus_slots, st);
    if (!es) es = cudaMemcpyAsync(taus_saved, L.taus, sizeof(uint4) * L.taus_slots,
                                  cudaMemcpyDeviceToDevice, st);
    if (es) return cuda_fail(c, es, "autotune");
  }
  auto run_orbit = [&](int blk, int var) {
    launch_orbit(L, c->cfg.precision, c->cfg.max_trials, c->r, c->x, c->phi,
                 tab ? c->Mbuf : nullptr, c->vr, c->vt, c->m,
                 c->id, c->step, c->keys, c->pay, nullptr, blk, var, c->bk.args(), c->r_old,
                 c->cc, c->vals, c->pcount, st, true, nullptr, nullptr,
                 c->cfg.precision == 0 ? &c->env : nullptr, nullptr, nullptr, c->orb);
  };
  auto time_it = [&](auto&& fn) {
    float best = 3.4e38f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, st);
      fn();
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    return best;
  };
  // orbit block size and (sampled step) kernel variant
  const int n_var = tab ? kOrbitVariants : 1;
  int blk_best = c->cfg.orbit_block ? c->cfg.orbit_block : 64, var_best = c->orbit_variant;
  float tb = 3.4e38f;
  for (int var = 0; var < n_var; ++var)
    for (int blk : {64, 128, 256}) {
      if (c->cfg.orbit_block && blk != c->cfg.orbit_block) continue;
      if (tab && c->cfg.orbit_variant >= 0 && var != c->cfg.orbit_variant) continue;
      const float ms = time_it([&] { run_orbit(blk, var); });
      if (ms < tb) { tb = ms; blk_best = blk; var_best = var; }
    }
  c->cfg.orbit_block = blk_best;
  c->orbit_variant = var_best;
  // relaxation kernel variant: on copies of the velocities (r_old and cc
  // are free scratch here), after the bins of this state; the timestep the
  // bins leave is put back
  if (c->cfg.relax_variant < 0 && L.n_pairs) {
    uint64_t* dt_saved = reinterpret_cast<uint64_t*>(c->tile_c);
    cudaMemcpyAsync(dt_saved, L.dt_bits, sizeof(uint64_t) * L.n_seg, cudaMemcpyDeviceToDevice,
                    st);
    launch_bins(L, c->r, c->vr, c->vt, c->m, c->nbin, c->pref, st);
    float trb = 3.4e38f;
    int rv_best = 0;
    for (int rv = 0; rv < kRelaxVariants; ++rv) {
      const float ms = time_it([&] {
        cudaMemcpyAsync(c->r_old, c->vr, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(c->cc, c->vt, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, st);
        launch_relax(L, c->r_old, c->cc, c->m, c->id, c->nbin, c->step, st, rv);
      });
      if (ms < trb) { trb = ms; rv_best = rv; }
    }
    c->relax_variant = rv_best;
    cudaMemcpyAsync(L.dt_bits, dt_saved, sizeof(uint64_t) * L.n_seg, cudaMemcpyDeviceToDevice,
                    st);
  }
  run_orbit(blk_best, var_best);
  // sort shapes on copies of the keys the orbit step produced
  uint64_t* saved = reinterpret_cast<uint64_t*>(c->cc);  // scratch of the same size
  cudaMemcpyAsync(saved, c->keys, sizeof(uint64_t) * L.n, cudaMemcpyDeviceToDevice, st);
  int best_ipt = 16, best_rank = 0;
  float tbest = 3.4e38f;
  for (int ipt : {8, 16, 24, 32})
    for (int rank : {0, 1}) {
      // 24 and 32 keys per thread: packed keys only
      if (ipt > 16 && !c->packed) continue;
      if (sort_set_shape(L, c->W, ipt, rank, st)) continue;
      const float ms = time_it([&] {
        cudaMemcpyAsync(c->keys, saved, sizeof(uint64_t) * L.n, cudaMemcpyDeviceToDevice, st);
        sort_segments(L, c->W, c->keys, c->vals, 3, 5, true, c->err, st, nullptr, nullptr,
                      c->packed);
      });
      if (ms < tbest) { tbest = ms; best_ipt = ipt; best_rank = rank; }
    }
  cudaError_t e = sort_set_shape(L, c->W, best_ipt, best_rank, st);
  // undo the dry run's bookkeeping
  if (!e && taus_saved)
    e = cudaMemcpyAsync(L.taus, taus_saved, sizeof(uint4) * L.taus_slots,
                        cudaMemcpyDeviceToDevice, st);
  if (!e) e = cudaMemsetAsync(L.esc_step, 0, sizeof(int64_t) * L.n_seg, st);
  if (!e) e = cudaMemsetAsync(L.stats, 0, sizeof(unsigned long long) * kStStride * L.n_seg, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (taus_saved) dfree(taus_saved, st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!e) e = cudaGetLastError();
  if (e) return cuda_fail(c, e, "autotune");
  return check_err_flags(c);
}

// A per-star attribute of the sorted state (stellar radii, semi-major
// axes): set from, or read to, caller memory (ptr_kind 0 host, 1 device);
// host values must be finite and >= 0.
cmc_status attr_set(cmc_ctx* c, double* dst, const double* src, int32_t ptr_kind,
                    const char* call, const char* option) {
  const std::string who(call);
  if (!c || !src || (ptr_kind != 0 && ptr_kind != 1))
    return fail(c, CMC_EINVAL, who + ": bad arguments");
  if (c->poisoned) return fail(c, CMC_EPOISONED, who + ": context poisoned");
  if (!dst) return fail(c, CMC_EINVAL, who + ": the context has no " + option);
  if (ptr_kind == 0)
    for (int64_t i = 0; i < c->L.n; ++i)
      if (!(src[i] >= 0.0) || !(src[i] < INFINITY))
        return fail(c, CMC_EINVAL, who + ": values must be finite and >= 0");
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)c->L.n,
                                  ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, call);
  return CMC_OK;
}

cmc_status attr_get(cmc_ctx* c, const double* src, double* dst, int32_t ptr_kind,
                    const char* call, const char* option) {
  const std::string who(call);
  if (!c || !dst || (ptr_kind != 0 && ptr_kind != 1))
    return fail(c, CMC_EINVAL, who + ": bad arguments");
  if (c->poisoned) return fail(c, CMC_EPOISONED, who + ": context poisoned");
  if (!src) return fail(c, CMC_EINVAL, who + ": the context has no " + option);
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(dst, src, sizeof(double) * (size_t)c->L.n,
                                  ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, call);
  return CMC_OK;
}

}  // namespace

namespace cmc {
CMC_DEBUG_SITE_ACCESSOR
}  // namespace cmc

extern "C" {

void cmc_config_default(cmc_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->precision = 0;
  cfg->bin_size = 20;
  cfg->theta_max = kPi / 2;
  cfg->gamma = 0.1;
  cfg->max_trials = 1000;
  cfg->energy_correction = 1;
  cfg->orbit_block = 0;
  cfg->autotune = 1;
  cfg->orbit_variant = -1;
  cfg->rng = 0;
  cfg->relax_variant = -1;
  cfg->collisions = 0;
  cfg->diag_ring = 0;
  cfg->binaries = 0;
  cfg->x_bb = 1.0;
  cfg->x_bs = 1.0;
  cfg->sort_packed = 1;
}

cmc_status cmc_init(cmc_ctx** out, const cmc_config* cfg_in, int32_t n_clusters,
                    const int64_t* n_per_cluster, const uint64_t* seeds, const double* r,
                    const double* vr, const double* vt, const double* m, const uint32_t* id,
                    int32_t ptr_kind, void* stream) {
  if (out) *out = nullptr;
  if (!out || n_clusters < 1 || !n_per_cluster || !seeds || !r || !vr || !vt || !m || !id ||
      (ptr_kind != 0 && ptr_kind != 1))
    return fail(nullptr, CMC_EINVAL, "cmc_init: bad arguments");
  cmc_config cfg;
  if (cfg_in) cfg = *cfg_in;
  else cmc_config_default(&cfg);
  if (cfg.precision < 0 || cfg.precision > 2 || cfg.bin_size < 2 || (cfg.bin_size & 1) ||
      cfg.max_trials < 1 || cfg.max_trials > (1 << 24) || !(cfg.theta_max > 0.0) ||
      !(cfg.gamma > 0.0) || cfg.orbit_block < 0 || cfg.orbit_block > 256 ||
      (cfg.orbit_block % 32) || cfg.orbit_variant < -1 || cfg.orbit_variant >= kOrbitVariants ||
      (cfg.rng != 0 && cfg.rng != 1) || cfg.relax_variant < -1 ||
      cfg.relax_variant >= kRelaxVariants || (cfg.collisions != 0 && cfg.collisions != 1) ||
      cfg.diag_ring < 0 || cfg.diag_ring > (1 << 20) ||
      (cfg.binaries != 0 && cfg.binaries != 1) || !(cfg.x_bb > 0.0) || !(cfg.x_bb < INFINITY) ||
      !(cfg.x_bs > 0.0) || !(cfg.x_bs < INFINITY) ||
      (cfg.sort_packed != 0 && cfg.sort_packed != 1))
    return fail(nullptr, CMC_EINVAL, "cmc_init: bad configuration");
  std::vector<int64_t> sizes(n_per_cluster, n_per_cluster + n_clusters);
  std::vector<uint64_t> sd(seeds, seeds + n_clusters);
  std::vector<double> lnL(n_clusters);
  int64_t total = 0;
  for (int c = 0; c < n_clusters; ++c) {
    if (sizes[c] < 1) return fail(nullptr, CMC_EINVAL, "cmc_init: empty cluster");
    total += sizes[c];
    lnL[c] = std::log(cfg.gamma * (double)sizes[c]);
  }
  if (total >= (int64_t)1 << 31)
    return fail(nullptr, CMC_EINVAL, "cmc_init: more than 2^31 - 1 stars");

  cmc_ctx* c = new cmc_ctx();
  c->cfg = cfg;
  c->packed = cfg.sort_packed != 0;
  for (int k = 0; k < n_clusters; ++k)
    if (sizes[k] > kPackMax) c->packed = false;
  c->stream = (cudaStream_t)stream;
  c->pref = t_rel_prefactor(cfg.theta_max);
  cudaGetDevice(&c->device);
  cudaError_t e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
  if (!e) e = cudaEventCreateWithFlags(&c->ev_rim, cudaEventDisableTiming);
  if (!e) e = cudaEventCreateWithFlags(&c->ev_aux, cudaEventDisableTiming);
  if (e) { cmc_status s = cuda_fail(nullptr, e, "cmc_init"); free_ctx(c); return s; }
  cudaStream_t st = c->stream;
  e = alloc_layout(c->L, sizes, sd, lnL, cfg.bin_size, st);
  const size_t n = (size_t)total;
  SegLayout& L = c->L;
#define CMC_ALLOC(ptr, cnt) \
  if (!e) e = dalloc(ptr, cnt, st);
  CMC_ALLOC(c->r, n);
  CMC_ALLOC(c->x, n);
  CMC_ALLOC(c->vr, n);
  CMC_ALLOC(c->vt, n);
  CMC_ALLOC(c->m, n);
  CMC_ALLOC(c->phi, n);
  CMC_ALLOC(c->id, n);
  if (cfg.precision != 2) CMC_ALLOC(c->t32, n);
  if (!e && cfg.precision == 0) e = alloc_env(c->env, (int64_t)n, st);
  if (cfg.precision != 2) CMC_ALLOC(c->orb, n);
  if (cfg.diag_ring > 0) {
    CMC_ALLOC(c->ring, (size_t)n_clusters * cfg.diag_ring * kDiagFields);
    if (!e) e = cudaMemsetAsync(c->ring, 0, sizeof(double) * (size_t)n_clusters *
                                                cfg.diag_ring * kDiagFields, st);
  }
  CMC_ALLOC(c->keys, n);
  CMC_ALLOC(c->vals, n);
  CMC_ALLOC(c->pay, n);
  CMC_ALLOC(c->r_old, n);
  CMC_ALLOC(c->cc, n);
  CMC_ALLOC(c->Mbuf, n);
  CMC_ALLOC(c->nbin, (size_t)L.n_bins);
  CMC_ALLOC(c->tile_a, (size_t)L.n_tiles);
  CMC_ALLOC(c->tile_b, (size_t)L.n_tiles);
  CMC_ALLOC(c->tile_c, (size_t)L.n_tiles);
  CMC_ALLOC(c->out3, (size_t)3 * n_clusters);
  CMC_ALLOC(c->err, 1);
  CMC_ALLOC(c->step, 1);
  CMC_ALLOC(c->pcount, 1);
  if (cfg.collisions) {
    CMC_ALLOC(c->R, n);
    CMC_ALLOC(c->Rp, n);
    if (!e) e = cudaMemsetAsync(c->R, 0, sizeof(double) * n, st);
  }
  if (cfg.binaries) {
    CMC_ALLOC(c->A, n);
    CMC_ALLOC(c->Ap, n);
    if (!e) e = cudaMemsetAsync(c->A, 0, sizeof(double) * n, st);
  }
#undef CMC_ALLOC
  if (!e) e = alloc_sort(c->W, L, 8, st);
  if (!e && cfg.precision != 2) e = alloc_buckets(c->bk, L, st);
  if (e) { cmc_status s = cuda_fail(nullptr, e, "cmc_init: allocation"); free_ctx(c); return s; }
  sort_prepare();
  potential_prepare();
  cmc_status s = load_state(c, r, vr, vt, m, id, ptr_kind, false, 0);
  if (s != CMC_OK) {
    g_err = c->last_error;
    free_ctx(c);
    return s;
  }
  if (cfg.rng == 1) {
    s = init_streams(c, seeds);
    if (s != CMC_OK) {
      g_err = c->last_error;
      free_ctx(c);
      return s;
    }
  }
  c->orbit_variant = cfg.orbit_variant > 0 ? cfg.orbit_variant : 0;
  c->relax_variant = cfg.relax_variant > 0 ? cfg.relax_variant : 0;
  if (cfg.autotune) {
    s = autotune(c);
    if (s != CMC_OK) {
      g_err = c->last_error;
      free_ctx(c);
      return s;
    }
  }
  if (c->cfg.orbit_block == 0) c->cfg.orbit_block = 64;
  c->kernels_per_step = count_step_kernels(c);
  *out = c;
  return CMC_OK;
}

cmc_status cmc_step(cmc_ctx* c, int32_t n_steps) {
  if (!c || n_steps < 0) return fail(c, CMC_EINVAL, "cmc_step: bad arguments");
  if (c->poisoned) return fail(c, CMC_EPOISONED, c->last_error);
  if (n_steps == 0) return CMC_OK;
  DeviceGuard g(c->device);
  cudaError_t e;
  if (!c->exec) {
    cudaGraph_t graph;
    e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e) return cuda_fail(c, e, "cmc_step: begin capture");
    record_step(c, c->cap);
    e = cudaStreamEndCapture(c->cap, &graph);
    if (e) return cuda_fail(c, e, "cmc_step: capture");
    e = cudaGraphInstantiate(&c->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) { c->exec = nullptr; return cuda_fail(c, e, "cmc_step: instantiate"); }
  }
  nvtxRangePushA("cmc_step");
  for (int32_t i = 0; i < n_steps; ++i) {
    e = cudaGraphLaunch(c->exec, c->stream);
    if (e) { nvtxRangePop(); return cuda_fail(c, e, "cmc_step: launch"); }
  }
  c->steps_taken += n_steps;
  const cmc_status s = check_err_flags(c);
  nvtxRangePop();
  return s;
}

cmc_status cmc_step_profiled(cmc_ctx* c, int32_t n_steps, double* stage_ms) {
  if (!c || n_steps < 0 || !stage_ms) return fail(c, CMC_EINVAL, "cmc_step_profiled: bad arguments");
  if (c->poisoned) return fail(c, CMC_EPOISONED, c->last_error);
  DeviceGuard g(c->device);
  for (int i = 0; i < CMC_NSTAGES; ++i) stage_ms[i] = 0.0;
  std::vector<cudaEvent_t> ev((size_t)(CMC_NSTAGES + 1) * (n_steps > 0 ? n_steps : 1));
  for (auto& e : ev) cudaEventCreate(&e);
  for (int32_t i = 0; i < n_steps; ++i) record_step(c, c->stream, &ev[(size_t)i * (CMC_NSTAGES + 1)]);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (!e) {
    for (int32_t i = 0; i < n_steps; ++i)
      for (int sidx = 0; sidx < CMC_NSTAGES; ++sidx) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[(size_t)i * (CMC_NSTAGES + 1) + sidx],
                             ev[(size_t)i * (CMC_NSTAGES + 1) + sidx + 1]);
        stage_ms[sidx] += ms;
      }
  }
  for (auto& x : ev) cudaEventDestroy(x);
  if (e) return cuda_fail(c, e, "cmc_step_profiled");
  c->steps_taken += n_steps;
  return check_err_flags(c);
}

cmc_status cmc_energy(cmc_ctx* c, double* out) {
  if (!c || !out) return fail(c, CMC_EINVAL, "cmc_energy: bad arguments");
  if (c->poisoned) return fail(c, CMC_EPOISONED, c->last_error);
  DeviceGuard g(c->device);
  launch_energy(c->L, c->r, c->vr, c->vt, c->m, c->tile_a, c->tile_b, c->tile_c, c->r_old,
                c->out3, c->stream);
  cudaError_t e = cudaMemcpyAsync(out, c->out3, sizeof(double) * 3 * c->L.n_seg,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_energy");
  return CMC_OK;
}

cmc_status cmc_get_rng_state(cmc_ctx* c, uint32_t* out, int64_t* n_words) {
  if (!c || !n_words) return fail(c, CMC_EINVAL, "cmc_get_rng_state: bad arguments");
  if (!c->L.taus) return fail(c, CMC_EINVAL, "cmc_get_rng_state: counter mode has no streams");
  *n_words = 4 * c->L.taus_slots;
  if (!out) return CMC_OK;
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(out, c->L.taus, sizeof(uint4) * c->L.taus_slots,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_get_rng_state");
  return CMC_OK;
}

cmc_status cmc_set_rng_state(cmc_ctx* c, const uint32_t* in, int64_t n_words) {
  if (!c || !in) return fail(c, CMC_EINVAL, "cmc_set_rng_state: bad arguments");
  if (!c->L.taus) return fail(c, CMC_EINVAL, "cmc_set_rng_state: counter mode has no streams");
  if (n_words != 4 * c->L.taus_slots)
    return fail(c, CMC_EINVAL, "cmc_set_rng_state: wrong number of words");
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(c->L.taus, in, sizeof(uint4) * c->L.taus_slots,
                                  cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_set_rng_state");
  return CMC_OK;
}

cmc_status cmc_core(cmc_ctx* c, double* out) {
  if (!c || !out) return fail(c, CMC_EINVAL, "cmc_core: bad arguments");
  if (c->poisoned) return fail(c, CMC_EPOISONED, c->last_error);
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  double *tiles = nullptr, *dout = nullptr;
  cudaError_t e = dalloc(tiles, 4 * (size_t)(c->L.n_tiles > 0 ? c->L.n_tiles : 1), st);
  if (!e) e = dalloc(dout, 3 * (size_t)c->L.n_seg, st);
  if (!e) {
    launch_core(c->L, c->r, c->m, tiles, dout, st);
    e = cudaGetLastError();
  }
  if (!e) e = cudaMemcpyAsync(out, dout, sizeof(double) * 3 * c->L.n_seg, cudaMemcpyDeviceToHost,
                              st);
  if (!e) e = cudaStreamSynchronize(st);
  dfree(tiles, st);
  dfree(dout, st);
  if (e) return cuda_fail(c, e, "cmc_core");
  return CMC_OK;
}

cmc_status cmc_lagrange_radii(cmc_ctx* c, const double* fracs, int32_t nf, double* out) {
  if (!c || !fracs || !out || nf < 1 || nf > 4096)
    return fail(c, CMC_EINVAL, "cmc_lagrange_radii: bad arguments");
  for (int i = 0; i < nf; ++i)
    if (!(fracs[i] >= 0.0 && fracs[i] <= 1.0))
      return fail(c, CMC_EINVAL, "cmc_lagrange_radii: fraction outside [0, 1]");
  if (c->poisoned) return fail(c, CMC_EPOISONED, c->last_error);
  DeviceGuard g(c->device);
  cudaStream_t st = c->stream;
  double *dfr = nullptr, *dout = nullptr;
  cudaError_t e = dalloc(dfr, nf, st);
  if (!e) e = dalloc(dout, (size_t)nf * c->L.n_seg, st);
  if (!e) e = cudaMemcpyAsync(dfr, fracs, sizeof(double) * nf, cudaMemcpyHostToDevice, st);
  if (!e) {
    launch_energy(c->L, c->r, c->vr, c->vt, c->m, c->tile_a, c->tile_b, c->tile_c, c->r_old,
                  c->out3, st);
    launch_lagrange(c->L, c->r, c->r_old, dfr, nf, dout, st);
    e = cudaMemcpyAsync(out, dout, sizeof(double) * nf * c->L.n_seg, cudaMemcpyDeviceToHost,
                        st);
  }
  if (!e) e = cudaStreamSynchronize(st);
  dfree(dfr, st);
  dfree(dout, st);
  if (e) return cuda_fail(c, e, "cmc_lagrange_radii");
  return CMC_OK;
}

cmc_status cmc_get_state(cmc_ctx* c, double* r, double* vr, double* vt, double* m,
                         uint32_t* id, double* phi, int64_t* step, int32_t ptr_kind) {
  if (!c || (ptr_kind != 0 && ptr_kind != 1))
    return fail(c, CMC_EINVAL, "cmc_get_state: bad arguments");
  if (c->poisoned) return fail(c, CMC_EPOISONED, c->last_error);
  DeviceGuard g(c->device);
  const size_t n = (size_t)c->L.n;
  cudaMemcpyKind k = ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaStream_t st = c->stream;
  cudaError_t e = cudaSuccess;
  if (!e && r) e = cudaMemcpyAsync(r, c->r, n * sizeof(double), k, st);
  if (!e && vr) e = cudaMemcpyAsync(vr, c->vr, n * sizeof(double), k, st);
  if (!e && vt) e = cudaMemcpyAsync(vt, c->vt, n * sizeof(double), k, st);
  if (!e && m) e = cudaMemcpyAsync(m, c->m, n * sizeof(double), k, st);
  if (!e && id) e = cudaMemcpyAsync(id, c->id, n * sizeof(uint32_t), k, st);
  if (!e && phi) e = cudaMemcpyAsync(phi, c->phi, n * sizeof(double), k, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_fail(c, e, "cmc_get_state");
  if (step) *step = c->steps_taken;
  return CMC_OK;
}

cmc_status cmc_set_state(cmc_ctx* c, const double* r, const double* vr, const double* vt,
                         const double* m, const uint32_t* id, int64_t step, int32_t ptr_kind) {
  if (!c || !r || !vr || !vt || !m || !id || step < 0 || (ptr_kind != 0 && ptr_kind != 1))
    return fail(c, CMC_EINVAL, "cmc_set_state: bad arguments");
  DeviceGuard g(c->device);
  c->poisoned = false;
  // a new state drops the stellar radii and semi-major axes (they belong
  // to the old order)
  if (c->R) cudaMemsetAsync(c->R, 0, sizeof(double) * (size_t)c->L.n, c->stream);
  if (c->A) cudaMemsetAsync(c->A, 0, sizeof(double) * (size_t)c->L.n, c->stream);
  return load_state(c, r, vr, vt, m, id, ptr_kind, true, step);
}

cmc_status cmc_get_nbound(cmc_ctx* c, int64_t* out) {
  if (!c || !out) return fail(c, CMC_EINVAL, "cmc_get_nbound: bad arguments");
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(out, c->L.nb, sizeof(int64_t) * c->L.n_seg,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_get_nbound");
  return CMC_OK;
}

cmc_status cmc_get_dt(cmc_ctx* c, double* out) {
  if (!c || !out) return fail(c, CMC_EINVAL, "cmc_get_dt: bad arguments");
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(out, c->L.dt_last, sizeof(double) * c->L.n_seg,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_get_dt");
  return CMC_OK;
}

cmc_status cmc_get_stats(cmc_ctx* c, int64_t* out) {
  if (!c || !out) return fail(c, CMC_EINVAL, "cmc_get_stats: bad arguments");
  DeviceGuard g(c->device);
  std::vector<unsigned long long> h((size_t)kStStride * c->L.n_seg);
  cudaError_t e = cudaMemcpyAsync(h.data(), c->L.stats, sizeof(unsigned long long) * h.size(),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_get_stats");
  for (int s = 0; s < c->L.n_seg; ++s)
    for (int j = 0; j < CMC_NSTATS; ++j)
      out[(size_t)s * CMC_NSTATS + j] = (int64_t)h[(size_t)s * kStStride + j];
  return CMC_OK;
}

cmc_status cmc_get_escaped(cmc_ctx* c, double* out) {
  if (!c || !out) return fail(c, CMC_EINVAL, "cmc_get_escaped: bad arguments");
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(out, c->L.esc_me, sizeof(double) * 2 * c->L.n_seg,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_get_escaped");
  return CMC_OK;
}

cmc_status cmc_get_diagnostics(cmc_ctx* c, double* out, int32_t* n_records) {
  if (!c || !n_records) return fail(c, CMC_EINVAL, "cmc_get_diagnostics: bad arguments");
  if (!c->ring) return fail(c, CMC_EINVAL, "cmc_get_diagnostics: the ring is off (diag_ring 0)");
  const int cap = c->cfg.diag_ring;
  const int64_t steps = c->steps_taken;
  const int nrec = steps < cap ? (int)steps : cap;
  *n_records = nrec;
  if (!out || nrec == 0) return CMC_OK;
  DeviceGuard g(c->device);
  const size_t nseg = (size_t)c->L.n_seg;
  std::vector<double> h(nseg * cap * kDiagFields);
  cudaError_t e = cudaMemcpyAsync(h.data(), c->ring, sizeof(double) * h.size(),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_get_diagnostics");
  // the step counter of the newest record: slot (step - 1) mod cap
  const double* first = h.data();
  uint32_t newest = 0;
  for (int j = 0; j < cap; ++j) {
    const uint32_t s = (uint32_t)first[(size_t)j * kDiagFields];
    if (s > newest) newest = s;
  }
  for (size_t cl = 0; cl < nseg; ++cl)
    for (int i = 0; i < nrec; ++i) {
      const uint32_t stp = newest - (uint32_t)(nrec - 1 - i);
      const size_t slot = (stp - 1u) % (uint32_t)cap;
      std::memcpy(out + (cl * cap + i) * kDiagFields, h.data() + (cl * cap + slot) * kDiagFields,
                  sizeof(double) * kDiagFields);
    }
  return CMC_OK;
}

cmc_status cmc_debug_check(uint32_t* site) {
  if (!site) return fail(nullptr, CMC_EINVAL, "cmc_debug_check: bad arguments");
  const uint32_t v[5] = {cmc::debug_site_tu1(), cmc::debug_site_tu2(), cmc::debug_site_tu3(),
                         cmc::debug_site_tu4(), cmc::debug_site_tu5()};
  *site = 0u;
  for (uint32_t x : v)
    if (x && !*site) *site = x;
  return CMC_OK;
}

int32_t cmc_is_debug_build(void) {
#ifdef CMC_DEBUG
  return 1;
#else
  return 0;
#endif
}

cmc_status cmc_set_escaped(cmc_ctx* c, const double* in) {
  if (!c || !in) return fail(c, CMC_EINVAL, "cmc_set_escaped: bad arguments");
  for (int s = 0; s < 2 * c->L.n_seg; ++s)
    if (!std::isfinite(in[s])) return fail(c, CMC_EINVAL, "cmc_set_escaped: non-finite value");
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(c->L.esc_me, in, sizeof(double) * 2 * c->L.n_seg,
                                  cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_set_escaped");
  return CMC_OK;
}

int32_t cmc_kernels_per_step(const cmc_ctx* c) { return c ? c->kernels_per_step : 0; }

cmc_status cmc_set_radii(cmc_ctx* c, const double* R, int32_t ptr_kind) {
  return attr_set(c, c ? c->R : nullptr, R, ptr_kind, "cmc_set_radii", "collisions");
}

cmc_status cmc_get_radii(cmc_ctx* c, double* R, int32_t ptr_kind) {
  return attr_get(c, c ? c->R : nullptr, R, ptr_kind, "cmc_get_radii", "collisions");
}

cmc_status cmc_set_binaries(cmc_ctx* c, const double* a, int32_t ptr_kind) {
  return attr_set(c, c ? c->A : nullptr, a, ptr_kind, "cmc_set_binaries", "binaries");
}

cmc_status cmc_get_binaries(cmc_ctx* c, double* a, int32_t ptr_kind) {
  return attr_get(c, c ? c->A : nullptr, a, ptr_kind, "cmc_get_binaries", "binaries");
}

cmc_status cmc_set_dt_cap(cmc_ctx* c, const double* cap) {
  if (!c || !cap) return fail(c, CMC_EINVAL, "cmc_set_dt_cap: bad arguments");
  if (c->poisoned) return fail(c, CMC_EPOISONED, "cmc_set_dt_cap: context poisoned");
  for (int s = 0; s < c->L.n_seg; ++s)
    if (!(cap[s] >= 0.0) || !(cap[s] < INFINITY))
      return fail(c, CMC_EINVAL, "cmc_set_dt_cap: bounds must be finite and >= 0");
  DeviceGuard g(c->device);
  cudaError_t e = cudaMemcpyAsync(c->L.dt_cap, cap, sizeof(double) * c->L.n_seg,
                                  cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);  // cap lives in the caller's memory
  if (e) return cuda_fail(c, e, "cmc_set_dt_cap");
  return CMC_OK;
}

double cmc_tse(double M, double T_prev, double dm_se) {
  if (!(dm_se > 0.0)) return INFINITY;
  return ((0.001 * M) * T_prev) / dm_se;
}

cmc_status cmc_get_tuning(const cmc_ctx* c, int32_t* out) {
  if (!c || !out) return CMC_EINVAL;
  out[0] = c->cfg.orbit_block;
  out[1] = c->W.ipt;
  out[2] = c->W.rank;
  out[3] = c->orbit_variant;
  out[4] = c->relax_variant;
  return CMC_OK;
}

cmc_status cmc_set_stream(cmc_ctx* c, void* stream) {
  if (!c) return fail(c, CMC_EINVAL, "cmc_set_stream: bad arguments");
  DeviceGuard g(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e) return cuda_fail(c, e, "cmc_set_stream");
  c->stream = (cudaStream_t)stream;
  return CMC_OK;
}

const char* cmc_last_error(const cmc_ctx* c) {
  return c ? c->last_error.c_str() : g_err.c_str();
}

void cmc_destroy(cmc_ctx* c) { free_ctx(c); }

// ----------------------------------------------------------- stage API
namespace {

struct Stage {
  SegLayout L;
  cudaStream_t st;
  cudaError_t e = cudaSuccess;
  Stage(int64_t n, uint64_t seed, double lnL, int bin_size, cudaStream_t s) : st(s) {
    std::vector<int64_t> sizes{n};
    std::vector<uint64_t> sd{seed};
    std::vector<double> ll{lnL};
    e = alloc_layout(L, sizes, sd, ll, bin_size, st);
  }
  ~Stage() { free_layout(L, st); }
};

}  // namespace

cmc_status cmc_rng_philox(int64_t n, const uint32_t* ctr, uint64_t seed, uint32_t* out,
                          void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return fail(nullptr, CMC_EINVAL, "cmc_rng_philox");
  launch_philox(n, ctr, seed, out, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(nullptr, e, "cmc_rng_philox") : CMC_OK;
}

cmc_status cmc_set_wait_limits(int32_t lookback_polls, int64_t tie_moves) {
  cudaError_t e = set_wait_limits(lookback_polls, (long long)tie_moves);
  if (e) return cuda_fail(nullptr, e, "cmc_set_wait_limits");
  return CMC_OK;
}

cmc_status cmc_sort_radius(int64_t n, const double* r, const uint32_t* id, uint32_t* perm,
                           void* stream) {
  if (n < 0 || n >= ((int64_t)1 << 31) || (n > 0 && (!r || !id || !perm)))
    return fail(nullptr, CMC_EINVAL, "cmc_sort_radius: bad arguments");
  if (n == 0) return CMC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Stage S(n, 0, 0.0, 20, st);
  if (S.e) return cuda_fail(nullptr, S.e, "cmc_sort_radius");
  SortWork W;
  uint64_t* keys = nullptr;
  uint32_t* err = nullptr;
  cudaError_t e = alloc_sort(W, S.L, 8, st);
  uint32_t he = 0;
  if (!e) e = dalloc(keys, n, st);
  if (!e) e = dalloc(err, 1, st);
  if (!e) {
    sort_prepare();
    cudaMemsetAsync(err, 0, sizeof(uint32_t), st);
    launch_make_keys(S.L, r, nullptr, nullptr, nullptr, id, keys, nullptr, st);
    // as in the timestep: passes over bits 24-63, then runs equal in those
    // bits in (r, id) order
    sort_segments(S.L, W, keys, perm, 3, 5, true, err, st);
    launch_tiefix(S.L, keys, perm, id, 1, err, st, 24);
    e = cudaMemcpyAsync(&he, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (!e && (he & kErrTies)) {
      // runs of equal radii too long for the tie fix: order by id first,
      // then stably by radius
      launch_id_keys(S.L, id, keys, st);
      sort_segments(S.L, W, keys, perm, 0, 4, true, err, st);
      launch_rekey_radius(S.L, perm, r, id, keys, st);
      sort_segments(S.L, W, keys, perm, 0, 8, false, err, st);
      if (!e) e = cudaMemcpyAsync(&he, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
      if (!e) e = cudaStreamSynchronize(st);
    }
    if (!e) e = cudaGetLastError();
  }
  dfree(keys, st);
  dfree(err, st);
  free_sort(W, st);
  if (e) return cuda_fail(nullptr, e, "cmc_sort_radius");
  if (he & kErrTimeout)
    return fail(nullptr, CMC_ETIMEOUT, "cmc_sort_radius: bounded wait expired in the look-back");
  return CMC_OK;
}

cmc_status cmc_potential(int64_t n, const double* r, const double* m, double* phi, double* M,
                         void* stream) {
  if (n < 0 || (n > 0 && (!r || !m || !phi)))
    return fail(nullptr, CMC_EINVAL, "cmc_potential: bad arguments");
  if (n == 0) return CMC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Stage S(n, 0, 0.0, 20, st);
  if (S.e) return cuda_fail(nullptr, S.e, "cmc_potential");
  double *x = nullptr, *ta = nullptr, *tb = nullptr;
  cudaError_t e = dalloc(x, n, st);
  if (!e) e = dalloc(ta, (size_t)S.L.n_tiles, st);
  if (!e) e = dalloc(tb, (size_t)S.L.n_tiles, st);
  if (!e) {
    potential_prepare();
    launch_recip(n, r, x, st);
    launch_potential(S.L, r, x, m, ta, tb, phi, nullptr, M, false, st);
    e = cudaGetLastError();
  }
  dfree(x, st);
  dfree(ta, st);
  dfree(tb, st);
  return e ? cuda_fail(nullptr, e, "cmc_potential") : CMC_OK;
}

cmc_status cmc_timestep(int64_t n, const double* r, const double* vr, const double* vt,
                        const double* m, int32_t bin_size, double theta_max, double lnL,
                        double* nbin, double* dt, void* stream) {
  if (n < 0 || bin_size < 2 || (bin_size & 1) || (n > 0 && (!r || !vr || !vt || !m || !nbin)) ||
      !dt)
    return fail(nullptr, CMC_EINVAL, "cmc_timestep: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    const double inf = INFINITY;
    cudaError_t e = cudaMemcpyAsync(dt, &inf, sizeof(double), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaStreamSynchronize(st);
    return e ? cuda_fail(nullptr, e, "cmc_timestep") : CMC_OK;
  }
  Stage S(n, 0, lnL, bin_size, st);
  if (S.e) return cuda_fail(nullptr, S.e, "cmc_timestep");
  launch_bins(S.L, r, vr, vt, m, nbin, t_rel_prefactor(theta_max), st);
  cudaError_t e = cudaMemcpyAsync(dt, S.L.dt_bits, sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (!e) e = cudaGetLastError();
  return e ? cuda_fail(nullptr, e, "cmc_timestep") : CMC_OK;
}

cmc_status cmc_relax(int64_t n, double* vr, double* vt, const double* m, const uint32_t* id,
                     const double* nbin, int32_t bin_size, double dt, double lnL, uint64_t seed,
                     uint32_t step, void* stream) {
  if (n < 0 || bin_size < 2 || (bin_size & 1) || (n > 0 && (!vr || !vt || !m || !id || !nbin)))
    return fail(nullptr, CMC_EINVAL, "cmc_relax: bad arguments");
  if (n < 2) return CMC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Stage S(n, seed, lnL, bin_size, st);
  if (S.e) return cuda_fail(nullptr, S.e, "cmc_relax");
  uint32_t* dstep = nullptr;
  cudaError_t e = dalloc(dstep, 1, st);
  if (!e) e = cudaMemcpyAsync(S.L.dt_bits, &dt, sizeof(double), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(dstep, &step, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
  if (!e) {
    launch_relax(S.L, vr, vt, const_cast<double*>(m), id, nbin, dstep, st);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(st);  // dt and step live on this stack
  dfree(dstep, st);
  return e ? cuda_fail(nullptr, e, "cmc_relax") : CMC_OK;
}

cmc_status cmc_orbit(int64_t n, const double* r, const double* phi, const double* vr,
                     const double* vt, const uint32_t* id, uint64_t seed, uint32_t step,
                     int32_t max_trials, int32_t precision, double* r_new, double* vr_new,
                     double* vt_new, double* phi_new, double* rmin, double* rmax, double* F,
                     int32_t* code, void* stream) {
  if (n < 0 || max_trials < 1 || precision < 0 || precision > 2 ||
      (n > 0 && (!r || !phi || !vr || !vt || !id || !r_new)))
    return fail(nullptr, CMC_EINVAL, "cmc_orbit: bad arguments");
  if (n == 0) return CMC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Stage S(n, seed, 0.0, 20, st);
  if (S.e) return cuda_fail(nullptr, S.e, "cmc_orbit");
  double *x = nullptr, *mm = nullptr;
  float2* t32 = nullptr;
  uint64_t* keys = nullptr;
  Payload* pay = nullptr;
  uint32_t* dstep = nullptr;
  cudaError_t e = dalloc(x, n, st);
  if (!e) e = dalloc(mm, n, st);
  if (!e) e = dalloc(t32, n, st);
  if (!e) e = dalloc(keys, n, st);
  if (!e) e = dalloc(pay, n, st);
  if (!e) e = dalloc(dstep, 1, st);
  if (!e) e = cudaMemsetAsync(mm, 0, sizeof(double) * n, st);
  if (!e) e = cudaMemcpyAsync(dstep, &step, sizeof(uint32_t), cudaMemcpyHostToDevice, st);
  if (!e) {
    launch_recip(n, r, x, st);
    launch_make_t32(n, x, phi, t32, st);
    BucketWork bk;
    double* sl = nullptr;  // shell slopes (enclosed masses) from the potential
    const bool tab = precision != 2;
    if (tab) {
      e = alloc_buckets(bk, S.L, st);
      if (!e) e = dalloc(sl, n, st);
      if (!e) {
        launch_buckets(S.L, t32, false, bk, st);
        launch_slopes(n, x, phi, sl, st);
        launch_make_nodes(n, r, x, phi, sl, bk.node, bk.tdf, st);
        launch_grid(S.L, x, phi, sl, false, bk, st);
      }
    }
    OrbitStageOut d;
    d.phi_new = phi_new; d.rmin = rmin; d.rmax = rmax; d.F = F; d.code = code;
    double *tmin = nullptr, *tmax = nullptr;
    double4_32a* orb = nullptr;
    EnvWork env;
    uint32_t *plist = nullptr, *pcnt = nullptr;
    if (!e && tab) e = dalloc(tmin, n, st);
    if (!e && tab) e = dalloc(tmax, n, st);
    if (!e && tab) e = dalloc(orb, n, st);
    if (!e && tab) e = dalloc(plist, n, st);
    if (!e && tab) e = dalloc(pcnt, 1, st);
    if (!e && precision == 0) e = alloc_env(env, n, st);
    if (!e)
      launch_orbit(S.L, precision, max_trials, r, x, phi, sl, vr, vt, mm, id, dstep, keys,
                   pay, &d, 0, 0, bk.args(), tmin, tmax, plist, pcnt, st, true, nullptr,
                   nullptr, precision == 0 ? &env : nullptr, nullptr, nullptr, orb);
    free_buckets(bk, st);
    free_env(env, st);
    dfree(sl, st);
    dfree(tmin, st);
    dfree(tmax, st);
    dfree(orb, st);
    dfree(plist, st);
    dfree(pcnt, st);
    launch_unpack_orbit(n, keys, pay, r_new, vr_new, vt_new, st);
    e = cudaGetLastError();
  }
  if (!e) e = cudaStreamSynchronize(st);
  dfree(x, st);
  dfree(mm, st);
  dfree(t32, st);
  dfree(keys, st);
  dfree(pay, st);
  dfree(dstep, st);
  return e ? cuda_fail(nullptr, e, "cmc_orbit") : CMC_OK;
}

cmc_status cmc_energy_correction(int64_t n, const double* r, const double* phi, double* vr,
                                 double* vt, const double* r_old, const double* c,
                                 void* stream) {
  if (n < 0 || (n > 0 && (!r || !phi || !vr || !vt || !r_old || !c)))
    return fail(nullptr, CMC_EINVAL, "cmc_energy_correction: bad arguments");
  if (n == 0) return CMC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Stage S(n, 0, 0.0, 20, st);
  if (S.e) return cuda_fail(nullptr, S.e, "cmc_energy_correction");
  double* x = nullptr;
  uint32_t* err = nullptr;
  cudaError_t e = dalloc(x, n, st);
  if (!e) e = dalloc(err, 1, st);
  if (!e) {
    launch_recip(n, r, x, st);
    launch_correction(S.L, r, x, phi, vr, vt, r_old, c, false, err, st);
    e = cudaGetLastError();
  }
  dfree(x, st);
  dfree(err, st);
  return e ? cuda_fail(nullptr, e, "cmc_energy_correction") : CMC_OK;
}

}  // extern "C"
