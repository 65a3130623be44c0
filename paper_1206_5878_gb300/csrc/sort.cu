// Key-value sort of the stars by radius (section 2.1 step 6).
//
// A stable least-significant-digit radix sort over 8-bit digits of the
// 64-bit key, run independently inside every segment (cluster) of the
// state.  Each digit pass is a single "onesweep" kernel: a CTA takes the
// next tile by atomic ticket, ranks its keys with a stable warp-level
// multisplit, publishes its digit counts, and obtains the counts of all
// earlier tiles of its segment by decoupled look-back on those published
// words (integer sums, so the result does not depend on timing).  Tiles are
// taken in ticket order, so every tile a CTA waits on is already running;
// each wait is still bounded and reports a timeout instead of spinning
// forever.  The tile is reordered in shared memory so that the scatter
// writes contiguous runs.
//
// Two shape parameters are chosen at initialisation by timing them on the
// real keys: keys per thread (8 or 16, so tiles of 2048 or 4096) and the
// multisplit (one __match_any_sync per key, or eight __ballot_sync
// intersected bit by bit).
#include <utility>
#include <vector>

#include "cmc_host.hpp"

namespace cmc {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kCountMask = (1ull << 62) - 1;
// Bounds of the device waits, in the library's device memory so that a
// change reaches kernels already captured in a graph: polls of a look-back
// word before a tile gives up on it (and reports a timeout), and moves of
// the tie fix's insertion sort before it gives up on a run.
constexpr int kSpinCapDefault = 1 << 22;
constexpr long long kTieMoveCapDefault = 1ll << 22;
__device__ int g_spin_cap = kSpinCapDefault;
__device__ long long g_tie_move_cap = kTieMoveCapDefault;
constexpr int kMaxPasses = 8;
static_assert(kThreads == kBins, "one thread per digit");

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *(volatile const unsigned long long*)p;
}

struct TileRange {
  int seg;
  int64_t lt;        // tile index inside the segment
  int64_t seg_begin, begin, end;
};

__device__ __forceinline__ TileRange tile_range(const int64_t* off, const int64_t* tile_off,
                                                int n_seg, int64_t t, int tile) {
  TileRange R;
  R.seg = seg_find(tile_off, n_seg, t);
  R.lt = t - __ldg(tile_off + R.seg);
  R.seg_begin = __ldg(off + R.seg);
  R.begin = R.seg_begin + R.lt * tile;
  int64_t se = __ldg(off + R.seg + 1);
  R.end = R.begin + tile < se ? R.begin + tile : se;
  return R;
}

// block-wide exclusive scan of one value per thread (256 threads)
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kWarps ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kWarps) s_warp[lane] = w;
  }
  __syncthreads();
  uint32_t before = warp ? s_warp[warp - 1] : 0;
  return before + x - v;
}

// ---------------------------------------------------------------- upsweep
// Per-segment histogram of every pass digit over tiles of kTile keys.  Each
// warp counts into its own shared-memory histogram (collisions only among
// its 32 lanes); the warps' histograms are summed before one global atomic
// per bin.  The last block of a segment to finish (a counter per segment,
// no waiting) turns that segment's histograms into exclusive scans.
__global__ void __launch_bounds__(kThreads) k_upsweep(const int64_t* off, const int64_t* tile_off,
                                                      int n_seg, const uint64_t* keys,
                                                      int first_pass, int passes,
                                                      uint32_t* hist, uint32_t* done) {
  __shared__ uint32_t s_warp[kWarps];
  __shared__ bool s_last;
  extern __shared__ uint32_t h[];  // [kWarps][passes][kBins]
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * passes * kBins; i += kThreads) h[i] = 0;
  __syncthreads();
  TileRange R = tile_range(off, tile_off, n_seg, blockIdx.x, kTile);
  uint32_t* hw = h + (size_t)warp * passes * kBins;
  for (int64_t p = R.begin + threadIdx.x; p < R.end; p += kThreads) {
    const uint64_t k = __ldg(keys + p);
    for (int q = 0; q < passes; ++q)
      atomicAdd(&hw[q * kBins + (int)((k >> (8 * (first_pass + q))) & 0xFF)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kBins; i += kThreads) {
    uint32_t s = 0;
    for (int w = 0; w < kWarps; ++w) s += h[(size_t)w * passes * kBins + i];
    if (s) atomicAdd(&hist[((size_t)R.seg * passes) * kBins + i], s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's counts before its arrival
    const uint32_t tiles = (uint32_t)(tile_off[R.seg + 1] - tile_off[R.seg]);
    s_last = atomicAdd(&done[R.seg], 1u) == tiles - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();  // every block's counts, read past L1
  for (int q = 0; q < passes; ++q) {
    uint32_t* hq = hist + ((size_t)R.seg * passes + q) * kBins;
    const uint32_t v = __ldcg(hq + threadIdx.x);
    const uint32_t e = block_excl_scan_u32(v, s_warp);
    hq[threadIdx.x] = e;
    __syncthreads();  // s_warp is read by the scan's last step
  }
}

// kPacked: keys only (each key carries its star's index in its unsorted low
// bits), no values
template <int IPT, bool kPacked>
struct PassSmem {
  uint64_t key[kThreads * IPT];
  uint32_t val[kPacked ? 1 : kThreads * IPT];
  uint32_t whist[kWarps][kBins];
  int64_t gbase[kBins];
  uint32_t dstart[kBins];
  uint32_t s_warp[kWarps];
  int64_t tile;
};

// lanes of the warp that hold the same digit (digits 0..256, 256 = no key),
// from one ballot per digit bit
__device__ __forceinline__ unsigned peers_ballot(int d) {
  unsigned m = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const bool bit = (d >> b) & 1;
    const unsigned x = __ballot_sync(0xffffffffu, bit);
    m &= bit ? x : ~x;
  }
  return m;
}

constexpr int kRankMatch = 0;   // __match_any_sync
constexpr int kRankBallot = 1;  // nine __ballot_sync

// ------------------------------------------------------------- onesweep
template <bool kValIdentity, int IPT, int kRank, bool kPacked>
__global__ void __launch_bounds__(kThreads, (IPT <= 8 ? 6 : IPT <= 16 ? (kPacked ? 4 : 3) : 2))
    k_pass(const int64_t* off, const int64_t* tile_off, int n_seg, int64_t n_tiles,
           const uint64_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
           uint64_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int pass, int q,
           int passes, const uint32_t* base, unsigned long long* desc, uint32_t* tickets,
           uint32_t* err) {
  constexpr int kTileKeys = kThreads * IPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassSmem<IPT, kPacked>& S = *reinterpret_cast<PassSmem<IPT, kPacked>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int shift = 8 * pass;

  if (tid == 0) S.tile = (int64_t)atomicAdd(tickets + q, 1u);
  for (int i = tid; i < kWarps * kBins; i += kThreads) (&S.whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t t = S.tile;
  TileRange R = tile_range(off, tile_off, n_seg, t, kTileKeys);
  const int64_t n_items = R.end - R.begin;

  // warp-striped load: warp w owns elements [w*32*IPT, (w+1)*32*IPT)
  uint64_t k[IPT];
  uint32_t v[IPT];
  int dg[IPT];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    int64_t e = (int64_t)warp * (32 * IPT) + i * 32 + lane;
    int64_t p = R.begin + e;
    bool valid = e < n_items;
    k[i] = valid ? keys_in[p] : 0ull;
    v[i] = (valid && !kPacked) ? (kValIdentity ? (uint32_t)p : vals_in[p]) : 0u;
    dg[i] = valid ? (int)((k[i] >> shift) & 0xFF) : kBins;
  }

  // warp-level multisplit ranks (stable: slot order, then lane order).
  // The leader of each group of equal digits adds the group's size to the
  // warp's counter with a shared-memory atomic; the counts before (the
  // atomics' results) are read only after a group of slots has been
  // issued, so the round trips overlap.  A __syncwarp between slots orders
  // the updates of one counter by different leaders in slot order.
  uint32_t rank[IPT];
  const unsigned lt_mask = lanemask_lt();
  constexpr int kGrp = IPT < 4 ? IPT : 4;
#pragma unroll
  for (int i0 = 0; i0 < IPT; i0 += kGrp) {
    unsigned pe[kGrp];
    uint32_t old[kGrp];
#pragma unroll
    for (int j = 0; j < kGrp; ++j) {
      const int i = i0 + j;
      pe[j] = kRank == kRankMatch ? __match_any_sync(0xffffffffu, dg[i]) : peers_ballot(dg[i]);
      old[j] = 0;
      if (lane == __ffs(pe[j]) - 1 && dg[i] < kBins)
        old[j] = atomicAdd(&S.whist[warp][dg[i]], (uint32_t)__popc(pe[j]));
      __syncwarp();
    }
#pragma unroll
    for (int j = 0; j < kGrp; ++j) {
      const uint32_t o = __shfl_sync(0xffffffffu, old[j], __ffs(pe[j]) - 1);
      rank[i0 + j] = o + __popc(pe[j] & lt_mask);
    }
  }
  __syncthreads();

  // per digit: exclusive prefix over warps, tile count
  const int d = tid;
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    uint32_t c = S.whist[w][d];
    S.whist[w][d] = cnt;
    cnt += c;
  }

  // decoupled look-back over the earlier tiles of this segment
  unsigned long long* my = desc + ((size_t)q * n_tiles + t) * kBins + d;
  uint64_t excl = 0;
  if (R.lt == 0) {
    atomicExch(my, kFlagInc | (unsigned long long)cnt);
  } else {
    atomicExch(my, kFlagAgg | (unsigned long long)cnt);
    int64_t j = t - 1;
    const int64_t first = t - R.lt;
    const int spin_cap = g_spin_cap;
    int spins = 0;
    while (j >= first) {
      unsigned long long w = ld_volatile(desc + ((size_t)q * n_tiles + j) * kBins + d);
      if ((w & ~kCountMask) == 0) {
        if (++spins > spin_cap) {
          set_err(err, kErrTimeout);
          --j;
          spins = 0;
          continue;
        }
        if (spins > 32) __nanosleep(64);
        continue;
      }
      excl += (w & kCountMask);
      if ((w & ~kCountMask) == kFlagInc) break;
      --j;
    }
    atomicExch(my, kFlagInc | (unsigned long long)(excl + cnt));
  }

  uint32_t ds = block_excl_scan_u32(cnt, S.s_warp);
  S.dstart[d] = ds;
  S.gbase[d] = R.seg_begin + (int64_t)base[((size_t)R.seg * passes + q) * kBins + d] +
               (int64_t)excl - (int64_t)ds;
  __syncthreads();

  // reorder the tile in shared memory by digit
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    if (dg[i] < kBins) {
      uint32_t lp = S.dstart[dg[i]] + S.whist[warp][dg[i]] + rank[i];
      S.key[lp] = k[i];
      if (!kPacked) S.val[lp] = v[i];
    }
  }
  __syncthreads();

  // contiguous runs per digit go out coalesced; a destination outside the
  // segment (possible only after a timed-out look-back) is dropped
  const int64_t seg_end = __ldg(off + R.seg + 1);
  for (int lp = tid; lp < n_items; lp += kThreads) {
    uint64_t kk = S.key[lp];
    int dd = (int)((kk >> shift) & 0xFF);
    int64_t dest = S.gbase[dd] + lp;
    if (dest < R.seg_begin || dest >= seg_end) {
      set_err(err, kErrTimeout);
      continue;
    }
    keys_out[dest] = kk;
    if (!kPacked) vals_out[dest] = S.val[lp];
  }
}

// ------------------------------------------------------------- tie fix
// Runs of keys equal in their bits above `shift` are put in (key, id) order
// (insertion sort by one thread per run; a run that is already ordered
// costs one pass): finite radii in (r, id) order, escapers in id order.

__global__ void k_tiefix(const int64_t* off, int n_seg, int64_t n, uint64_t* keys,
                         uint32_t* vals, const uint32_t* ids_by_val, int id_stride, int shift,
                         uint32_t* err, unsigned long long* stats) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int c = seg_find(off, n_seg, p);
  int64_t sb = __ldg(off + c), se = __ldg(off + c + 1);
  const uint64_t kp = keys[p], hp = kp >> shift;
  if (p + 1 >= se || (keys[p + 1] >> shift) != hp) return;
  if (p > sb && (keys[p - 1] >> shift) == hp) return;  // not the start of the run
  int64_t e = p + 2;
  while (e < se && (keys[e] >> shift) == hp) ++e;
  for (int64_t i = p; i < e; ++i)
    if ((int64_t)vals[i] >= n) {
      set_err(err, kErrTimeout);
      return;
    }
  // insertion sort of the run by (key, id)
  const long long move_cap = g_tie_move_cap;
  long long moves = 0;
  bool equal = false;
  for (int64_t i = p + 1; i < e; ++i) {
    const uint64_t kv = keys[i];
    const uint32_t v = vals[i];
    const uint32_t idv = ids_by_val[(size_t)v * id_stride];
    int64_t j = i - 1;
    while (j >= p) {
      const uint64_t kj = keys[j];
      if (kj == kv) equal = true;
      if (!(kj > kv || (kj == kv && ids_by_val[(size_t)vals[j] * id_stride] > idv))) break;
      keys[j + 1] = kj;
      vals[j + 1] = vals[j];
      --j;
      if (++moves > move_cap) {
        set_err(err, kErrTies);
        keys[j + 1] = kv;
        vals[j + 1] = v;
        return;
      }
    }
    keys[j + 1] = kv;
    vals[j + 1] = v;
  }
  if (equal && stats) atomicAdd(stats + (size_t)c * kStStride + kStTies, 1ull);
}

// The same for packed keys: the low 24 bits of a sorted word hold its star's
// index in the segment, the key's own low 24 bits and the id are in the
// star's payload record (lo24 in pad); runs equal in bits 24-63 are put in
// (key, id) order by moving the words.
__device__ __forceinline__ void tiefix_packed_at(const int64_t* off, int n_seg, int64_t p,
                                                 uint64_t* keys, const Payload* pay,
                                                 uint32_t* err, unsigned long long* stats) {
  int c = seg_find(off, n_seg, p);
  int64_t sb = __ldg(off + c), se = __ldg(off + c + 1);
  const uint64_t hp = keys[p] >> 24;
  if (p + 1 >= se || (keys[p + 1] >> 24) != hp) return;
  if (p > sb && (keys[p - 1] >> 24) == hp) return;  // not the start of the run
  int64_t e = p + 2;
  while (e < se && (keys[e] >> 24) == hp) ++e;
  for (int64_t i = p; i < e; ++i)
    if ((int64_t)(keys[i] & 0xFFFFFFull) >= se - sb) {
      set_err(err, kErrTimeout);
      return;
    }
  const Payload* P = pay + sb;
  auto full = [&](uint64_t w) { return (w & ~0xFFFFFFull) | (uint64_t)P[w & 0xFFFFFFull].pad; };
  auto idof = [&](uint64_t w) { return P[w & 0xFFFFFFull].id; };
  const long long move_cap = g_tie_move_cap;
  long long moves = 0;
  bool equal = false;
  for (int64_t i = p + 1; i < e; ++i) {
    const uint64_t wv = keys[i];
    const uint64_t kv = full(wv);
    const uint32_t idv = idof(wv);
    int64_t j = i - 1;
    while (j >= p) {
      const uint64_t wj = keys[j];
      const uint64_t kj = full(wj);
      if (kj == kv) equal = true;
      if (!(kj > kv || (kj == kv && idof(wj) > idv))) break;
      keys[j + 1] = wj;
      --j;
      if (++moves > move_cap) {
        set_err(err, kErrTies);
        keys[j + 1] = wv;
        return;
      }
    }
    keys[j + 1] = wv;
  }
  if (equal && stats) atomicAdd(stats + (size_t)c * kStStride + kStTies, 1ull);
}

// four positions per thread: the keys read once (two 16-byte loads), a run
// start looked for only where two neighbours agree in bits 24-63 (a few per
// cent of them)
__global__ void k_tiefix_packed(const int64_t* off, int n_seg, int64_t n, uint64_t* keys,
                                const Payload* pay, uint32_t* err,
                                unsigned long long* stats) {
  const int64_t p0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (p0 >= n) return;
  uint64_t k[6];  // keys[p0 - 1 .. p0 + 4]
  if (p0 + 4 <= n) {
    const uint4 a = reinterpret_cast<const uint4*>(keys + p0)[0];
    const uint4 b = reinterpret_cast<const uint4*>(keys + p0)[1];
    k[1] = ((uint64_t)a.y << 32) | a.x;
    k[2] = ((uint64_t)a.w << 32) | a.z;
    k[3] = ((uint64_t)b.y << 32) | b.x;
    k[4] = ((uint64_t)b.w << 32) | b.z;
  } else {
    for (int i = 0; i < 4; ++i) k[1 + i] = p0 + i < n ? keys[p0 + i] : 0ull;
  }
  k[0] = p0 > 0 ? keys[p0 - 1] : 0ull;
  k[5] = p0 + 4 < n ? keys[p0 + 4] : 0ull;
  bool any = false;
  for (int i = 0; i < 4; ++i)
    any |= p0 + i + 1 < n && (k[1 + i] >> 24) == (k[2 + i] >> 24);
  if (!any) return;
  // the full test (segment bounds, run start) where a run may begin; the
  // keys are re-read there, after any earlier run in this thread moved them
  for (int i = 0; i < 4 && p0 + i < n; ++i)
    if (p0 + i + 1 < n && (k[1 + i] >> 24) == (k[2 + i] >> 24))
      tiefix_packed_at(off, n_seg, p0 + i, keys, pay, err, stats);
}

__global__ void k_philox(int64_t n, const uint32_t* ctr, uint64_t seed, uint32_t* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = reinterpret_cast<const uint4*>(ctr)[i];
  U4 w = philox(c.x, c.y, c.z, c.w, seed);
  reinterpret_cast<uint4*>(out)[i] = make_uint4(w.x, w.y, w.z, w.w);
}

template <bool kId, int IPT, int kRank, bool kPacked>
void set_pass_smem() {
  cudaFuncSetAttribute(k_pass<kId, IPT, kRank, kPacked>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(PassSmem<IPT, kPacked>));
}

template <int IPT, int kRank>
void launch_pass(const SegLayout& L, SortWork& W, bool id, const uint64_t* kin,
                 const uint32_t* vin, uint64_t* kout, uint32_t* vout, int pass, int q,
                 int passes, uint32_t* err, cudaStream_t st, bool packed) {
  const unsigned grid = (unsigned)W.n_stiles;
  if (packed) {
    k_pass<false, IPT, kRank, true><<<grid, kThreads, sizeof(PassSmem<IPT, true>), st>>>(
        L.off, W.stile_off, L.n_seg, W.n_stiles, kin, nullptr, kout, nullptr, pass, q, passes,
        W.hist, W.desc, W.tickets, err);
    return;
  }
  const size_t sm = sizeof(PassSmem<IPT, false>);
  if (id)
    k_pass<true, IPT, kRank, false><<<grid, kThreads, sm, st>>>(L.off, W.stile_off, L.n_seg,
                                                         W.n_stiles, kin, vin, kout, vout, pass,
                                                         q, passes, W.hist, W.desc, W.tickets,
                                                         err);
  else
    k_pass<false, IPT, kRank, false><<<grid, kThreads, sm, st>>>(L.off, W.stile_off, L.n_seg,
                                                          W.n_stiles, kin, vin, kout, vout,
                                                          pass, q, passes, W.hist, W.desc,
                                                          W.tickets, err);
}

// the larger tiles (24 or 32 keys per thread) of packed keys
template <int IPT>
void launch_packed_pass(const SegLayout& L, SortWork& W, const uint64_t* kin, uint64_t* kout,
                        int pass, int q, int passes, uint32_t* err, cudaStream_t st) {
  const unsigned grid = (unsigned)W.n_stiles;
  const size_t sm = sizeof(PassSmem<IPT, true>);
  if (W.rank == kRankMatch)
    k_pass<false, IPT, kRankMatch, true><<<grid, kThreads, sm, st>>>(
        L.off, W.stile_off, L.n_seg, W.n_stiles, kin, nullptr, kout, nullptr, pass, q, passes,
        W.hist, W.desc, W.tickets, err);
  else
    k_pass<false, IPT, kRankBallot, true><<<grid, kThreads, sm, st>>>(
        L.off, W.stile_off, L.n_seg, W.n_stiles, kin, nullptr, kout, nullptr, pass, q, passes,
        W.hist, W.desc, W.tickets, err);
}

}  // namespace

// ------------------------------------------------------------------ host
cudaError_t set_wait_limits(int spin_polls, long long tie_moves) {
  const int sp = spin_polls > 0 ? spin_polls : kSpinCapDefault;
  const long long tm = tie_moves > 0 ? tie_moves : kTieMoveCapDefault;
  cudaError_t e = cudaMemcpyToSymbol(g_spin_cap, &sp, sizeof(sp));
  if (!e) e = cudaMemcpyToSymbol(g_tie_move_cap, &tm, sizeof(tm));
  return e;
}

void sort_prepare() {
  set_pass_smem<true, 8, kRankMatch, false>();
  set_pass_smem<false, 8, kRankMatch, false>();
  set_pass_smem<true, 8, kRankBallot, false>();
  set_pass_smem<false, 8, kRankBallot, false>();
  set_pass_smem<true, 16, kRankMatch, false>();
  set_pass_smem<false, 16, kRankMatch, false>();
  set_pass_smem<true, 16, kRankBallot, false>();
  set_pass_smem<false, 16, kRankBallot, false>();
  set_pass_smem<false, 8, kRankMatch, true>();
  set_pass_smem<false, 8, kRankBallot, true>();
  set_pass_smem<false, 16, kRankMatch, true>();
  set_pass_smem<false, 16, kRankBallot, true>();
  set_pass_smem<false, 24, kRankMatch, true>();
  set_pass_smem<false, 24, kRankBallot, true>();
  set_pass_smem<false, 32, kRankMatch, true>();
  set_pass_smem<false, 32, kRankBallot, true>();
  cudaFuncSetAttribute(k_upsweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(uint32_t) * kWarps * kMaxPasses * kBins));
}

static std::vector<int64_t> sort_tile_offsets(const SegLayout& L, int tile) {
  std::vector<int64_t> o(L.n_seg + 1, 0);
  for (int c = 0; c < L.n_seg; ++c) {
    const int64_t nc = L.h_off[c + 1] - L.h_off[c];
    o[c + 1] = o[c] + (nc + tile - 1) / tile;
  }
  return o;
}

cudaError_t sort_set_shape(const SegLayout& L, SortWork& W, int ipt, int rank,
                           cudaStream_t st) {
  if ((ipt != 8 && ipt != 16 && ipt != 24 && ipt != 32) || (rank != 0 && rank != 1))
    return cudaErrorInvalidValue;
  std::vector<int64_t> o = sort_tile_offsets(L, kThreads * ipt);
  cudaError_t e = cudaMemcpyAsync(W.stile_off, o.data(), sizeof(int64_t) * o.size(),
                                  cudaMemcpyHostToDevice, st);
  if (!e) e = cudaStreamSynchronize(st);  // o lives on this stack
  if (e) return e;
  W.ipt = ipt;
  W.rank = rank;
  W.n_stiles = o[L.n_seg];
  return cudaSuccess;
}

cudaError_t alloc_sort(SortWork& W, const SegLayout& L, int max_passes, cudaStream_t st) {
  W.max_passes = max_passes;
  size_t n = (size_t)L.n;
  cudaError_t e;
  if ((e = cudaMallocAsync((void**)&W.keys_alt, sizeof(uint64_t) * (n ? n : 1), st))) return e;
  if ((e = cudaMallocAsync((void**)&W.vals_alt, sizeof(uint32_t) * (n ? n : 1), st))) return e;
  if ((e = cudaMallocAsync((void**)&W.stile_off, sizeof(int64_t) * (L.n_seg + 1), st)))
    return e;
  // look-back words for the smallest tiles (the most tiles)
  const int64_t max_tiles = sort_tile_offsets(L, kThreads * 8)[L.n_seg];
  size_t desc_b = sizeof(unsigned long long) * (size_t)max_passes * max_tiles * kBins;
  size_t hist_b = sizeof(uint32_t) * (size_t)L.n_seg * max_passes * kBins;
  size_t tick_b = sizeof(uint32_t) * 16;
  size_t done_b = sizeof(uint32_t) * (size_t)L.n_seg;
  // histograms, tickets and done counters first, then the look-back words:
  // a sort zeroes the counters and the words of its own passes and tiles
  const size_t head_b = (hist_b + tick_b + done_b + 255) / 256 * 256;
  W.zero_bytes = head_b + desc_b;
  W.zero_head = head_b;
  if ((e = cudaMallocAsync(&W.zero_base, W.zero_bytes, st))) return e;
  W.hist = (uint32_t*)W.zero_base;
  W.tickets = (uint32_t*)((char*)W.zero_base + hist_b);
  W.done = (uint32_t*)((char*)W.zero_base + hist_b + tick_b);
  W.desc = (unsigned long long*)((char*)W.zero_base + head_b);
  return sort_set_shape(L, W, 16, 0, st);
}

void free_sort(SortWork& W, cudaStream_t st) {
  if (W.keys_alt) cudaFreeAsync(W.keys_alt, st);
  if (W.vals_alt) cudaFreeAsync(W.vals_alt, st);
  if (W.stile_off) cudaFreeAsync(W.stile_off, st);
  if (W.zero_base) cudaFreeAsync(W.zero_base, st);
  W = SortWork();
}

cudaError_t sort_segments(const SegLayout& L, SortWork& W, uint64_t* keys, uint32_t* vals,
                          int first_pass, int passes, bool vals_identity, uint32_t* err,
                          cudaStream_t st, uint64_t** keys_res, uint32_t** vals_res,
                          bool packed) {
  if (keys_res) *keys_res = keys;
  if (vals_res) *vals_res = vals;
  if (passes <= 0 || passes > W.max_passes || L.n_tiles == 0) return cudaSuccess;
  // tiles of 24 or 32 keys per thread exist for packed keys only: a sort of
  // keys and values (a new state's ordering, outside any graph capture)
  // takes tiles of 16 and then restores the shape
  if (!packed && W.ipt > 16) {
    const int ipt = W.ipt, rank = W.rank;
    cudaError_t e = sort_set_shape(L, W, 16, rank, st);
    if (!e) e = sort_segments(L, W, keys, vals, first_pass, passes, vals_identity, err, st,
                              keys_res, vals_res, false);
    const cudaError_t e2 = sort_set_shape(L, W, ipt, rank, st);
    return e ? e : e2;
  }
  cudaMemsetAsync(W.zero_base, 0,
                  W.zero_head + sizeof(unsigned long long) * (size_t)passes *
                                    (size_t)W.n_stiles * kBins,
                  st);
  k_upsweep<<<(unsigned)L.n_tiles, kThreads, sizeof(uint32_t) * kWarps * passes * kBins, st>>>(
      L.off, L.tile_off, L.n_seg, keys, first_pass, passes, W.hist, W.done);
  uint64_t* kin = keys;
  uint32_t* vin = vals;
  uint64_t* kout = W.keys_alt;
  uint32_t* vout = W.vals_alt;
  for (int q = 0; q < passes; ++q) {
    const bool id = q == 0 && vals_identity;
    const int pass = first_pass + q;
    if (packed && W.ipt == 24)
      launch_packed_pass<24>(L, W, kin, kout, pass, q, passes, err, st);
    else if (packed && W.ipt == 32)
      launch_packed_pass<32>(L, W, kin, kout, pass, q, passes, err, st);
    else if (W.ipt == 8 && W.rank == kRankMatch)
      launch_pass<8, kRankMatch>(L, W, id, kin, vin, kout, vout, pass, q, passes, err, st,
                                 packed);
    else if (W.ipt == 8)
      launch_pass<8, kRankBallot>(L, W, id, kin, vin, kout, vout, pass, q, passes, err, st,
                                  packed);
    else if (W.rank == kRankMatch)
      launch_pass<16, kRankMatch>(L, W, id, kin, vin, kout, vout, pass, q, passes, err, st,
                                  packed);
    else
      launch_pass<16, kRankBallot>(L, W, id, kin, vin, kout, vout, pass, q, passes, err, st,
                                   packed);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  // after an odd number of passes the result is in the alternate buffers:
  // the caller takes them, or they are copied back
  if (kin != keys) {
    if (keys_res && vals_res) {
      *keys_res = kin;
      *vals_res = vin;
    } else {
      cudaMemcpyAsync(keys, kin, sizeof(uint64_t) * (size_t)L.n, cudaMemcpyDeviceToDevice, st);
      if (!packed)
        cudaMemcpyAsync(vals, vin, sizeof(uint32_t) * (size_t)L.n, cudaMemcpyDeviceToDevice,
                        st);
    }
  }
  return cudaGetLastError();
}

void launch_tiefix(const SegLayout& L, uint64_t* keys, uint32_t* vals,
                   const uint32_t* ids_by_val, int id_stride, uint32_t* err,
                   cudaStream_t st, int shift) {
  if (L.n == 0) return;
  k_tiefix<<<(unsigned)((L.n + 255) / 256), 256, 0, st>>>(
      L.off, L.n_seg, L.n, keys, vals, ids_by_val, id_stride, shift, err, L.stats);
}

void launch_tiefix_packed(const SegLayout& L, uint64_t* keys, const Payload* pay,
                          uint32_t* err, cudaStream_t st) {
  if (L.n == 0) return;
  const int64_t nt = (L.n + 3) / 4;
  k_tiefix_packed<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(L.off, L.n_seg, L.n, keys, pay,
                                                               err, L.stats);
}

void launch_philox(int64_t n, const uint32_t* ctr, uint64_t seed, uint32_t* out,
                   cudaStream_t st) {
  if (n <= 0) return;
  k_philox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ctr, seed, out);
}

CMC_DEBUG_SITE_ACCESSOR

}  // namespace cmc
