// Device code of the level passes, shared by the single-tree build
// (wt_build.cu) and the batched build (wt_batch.cu).  Everything here has
// internal linkage: each translation unit instantiates what it uses.
#pragma once
#include <cstdint>

#include "wt_dev.cuh"
#include "wt_internal.h"

using namespace wtk;

namespace {

constexpr uint32_t kHistSmemMaxBins = 8192;
constexpr uint32_t kScanThreads = 256;
constexpr uint32_t kScanItems = 8;
constexpr uint32_t kScanChunk = kScanThreads * kScanItems;
constexpr uint32_t kDefaultSpin = 1u << 22;

// ------------------------------------------------------------------ helpers
template <int SB>
__device__ __forceinline__ void load32(const uint8_t *g, uint32_t my0, uint32_t nv, uint32_t *u) {
  if (my0 + 32 <= nv) {
    const uint4 *src = reinterpret_cast<const uint4 *>(g);
#pragma unroll
    for (int c = 0; c < 2 * SB; ++c) {
      const uint4 v = __ldg(src + c);
      u[4 * c + 0] = v.x;
      u[4 * c + 1] = v.y;
      u[4 * c + 2] = v.z;
      u[4 * c + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8 * SB; ++i) u[i] = 0;
    for (uint32_t q = 0; q < 32 && my0 + q < nv; ++q) {
      uint32_t s;
      if (SB == 1) s = g[q];
      else if (SB == 2) s = reinterpret_cast<const uint16_t *>(g)[q];
      else s = reinterpret_cast<const uint32_t *>(g)[q];
      if (SB == 1) u[q >> 2] |= s << (8 * (q & 3));
      else if (SB == 2) u[q >> 1] |= s << (16 * (q & 1));
      else u[q] = s;
    }
  }
}

__device__ __forceinline__ uint32_t valid_mask(uint32_t my0, uint32_t nv) {
  if (my0 + 32 <= nv) return 0xFFFFFFFFu;
  if (my0 >= nv) return 0u;
  return (1u << (nv - my0)) - 1u;
}

template <int SB>
struct SymT;
template <>
struct SymT<1> { using type = uint8_t; };
template <>
struct SymT<2> { using type = uint16_t; };
template <>
struct SymT<4> { using type = uint32_t; };

// Outputs of one level: its bitmap row, directory row and zero count.
struct LevelOut {
  uint32_t *bits;
  unsigned long long *rank;
  unsigned long long *zeros;
};

// Write the level's bitmap word, the directory entries that fall in this
// thread's 32 positions, and (last tile) the level totals.  R = ones before
// the tile, excl = ones before this thread within the tile.
template <int THREADS>
__device__ __forceinline__ void write_level(const LevelOut &o, uint32_t tile, uint32_t NT,
                                            uint64_t start, uint32_t my0, uint32_t n, uint32_t NB,
                                            uint64_t W, uint32_t word, uint32_t R, uint32_t excl,
                                            uint32_t total) {
  const uint64_t widx = (uint64_t)tile * THREADS + threadIdx.x;
  if (widx < W) o.bits[widx] = word;
  if ((threadIdx.x & 15) == 0 && start + my0 < n) o.rank[(start + my0) >> 9] = R + excl;
  if (tile == NT - 1 && threadIdx.x == 0) {
    o.rank[NB] = R + total;
    *o.zeros = (unsigned long long)(n - (R + total));
  }
}

// ------------------------------------------------------------------ tile pipeline
// Every level pass runs persistent CTAs that take tiles of T = 32*THREADS
// symbols by ticket.  Tickets are fetched two tiles ahead, a tile's symbols
// are copied into shared memory by the TMA engine one tile ahead (double
// buffer), and the loads of a tile's count prefix are issued one tile ahead,
// so no round trip to memory sits between two tiles of a CTA.
// DEPTH 2: the copy of tile it+1 runs while tile it is processed (double
// buffer).  DEPTH 1: one buffer, the next tile is copied once the current one
// is done; the shared memory saved lets more CTAs share an SM, and their
// work covers the copy.
template <int SB, int THREADS, int DEPTH = 2, int WPT = 1>
struct TilePipe {
  static constexpr uint32_t T = 32 * WPT * THREADS;
  static constexpr uint32_t TB = T * SB;
  uint8_t *sIn0, *sIn1;
  uint64_t *bar;       // 2 mbarriers
  uint32_t *ring;      // 3 tickets
  const uint8_t *in;   // this level's symbols, 16-byte aligned
  int in_padded;       // in holds whole tiles -> copy whole tiles
  uint32_t n, NT;
  uint32_t *ticket;

  __device__ __forceinline__ void issue(uint32_t tile, int buf) const {
    const uint64_t start = (uint64_t)tile * T;
    const uint32_t nv = (uint32_t)umin64(T, n - start);
    const uint32_t bytes = in_padded ? TB : ((nv * SB) & ~15u);
    mbar_arrive_expect_tx(&bar[buf], bytes);
    if (bytes) bulk_g2s(buf ? sIn1 : sIn0, in + start * SB, bytes, &bar[buf]);
  }
  // thread 0, before the first __syncthreads
  __device__ __forceinline__ void prologue() const {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    const uint32_t t0 = atomicAdd(ticket, 1u);
    const uint32_t t1 = atomicAdd(ticket, 1u);
    ring[0] = t0;
    ring[1] = t1;
    if (t0 < NT) issue(t0, 0);
  }
  // thread 0 at the top of iteration `it`: fetch the ticket of tile it+2
  // (returned, stored at the end of the iteration) and start the copy of
  // tile it+1
  __device__ __forceinline__ uint32_t advance(uint32_t it, uint32_t nxt) const {
    const uint32_t nn = atomicAdd(ticket, 1u);
    if (DEPTH == 2 && nxt < NT) {
      fence_proxy_async_smem();
      issue(nxt, (it + 1) & 1);
    }
    return nn;
  }
  // DEPTH 1, thread 0 after the block barrier that ends tile it: start the
  // copy of tile it+1 into the (now free) buffer
  __device__ __forceinline__ void after_tile(uint32_t nxt) const {
    if (DEPTH == 1 && nxt < NT) {
      fence_proxy_async_smem();
      issue(nxt, 0);
    }
  }
  // all threads: wait for tile `it`'s symbols (bounded); false on timeout
  __device__ __forceinline__ bool wait(uint32_t it, uint32_t spin, int *err) const {
    if (DEPTH == 1) return mbar_wait_bounded(&bar[0], it & 1u, spin, err);
    return mbar_wait_bounded(&bar[it & 1], (it >> 1) & 1u, spin, err);
  }
  // after a timeout: wait (bounded) for the copies this CTA started
  __device__ __forceinline__ void drain(uint32_t it, uint32_t spin, int *err) const {
    if (threadIdx.x == 0) {
      if (DEPTH == 1) {
        mbar_wait_bounded(&bar[0], it & 1u, spin, err);
        return;
      }
      mbar_wait_bounded(&bar[it & 1], (it >> 1) & 1u, spin, err);
      if (ring[(it + 1) % 3] < NT) mbar_wait_bounded(&bar[(it + 1) & 1], ((it + 1) >> 1) & 1u, spin, err);
    }
  }
  __device__ __forceinline__ uint8_t *data(uint32_t it) const { return (DEPTH == 2 && (it & 1)) ? sIn1 : sIn0; }
  // tail bytes of an unpadded input that the bulk copy (multiple of 16 bytes) left out
  __device__ __forceinline__ bool fill_tail(uint8_t *sIn, uint64_t start, uint32_t nv) const {
    if (in_padded || ((nv * SB) & 15u) == 0) return false;
    for (uint32_t i = ((nv * SB) & ~15u) + threadIdx.x; i < nv * SB; i += THREADS)
      sIn[i] = in[start * SB + i];
    return true;
  }
};

// This thread's part of the count-prefix of `tile`, loads issued now and
// summed later (up to 3 terms per thread: tile < 2^20 and THREADS >= 128).
struct PrefixLoads {
  uint32_t v0, v1, v2;
  __device__ __forceinline__ uint32_t sum() const { return v0 + v1 + v2; }
};

template <int THREADS>
__device__ __forceinline__ PrefixLoads prefix_loads(const TileCounts &c, uint32_t tile, uint32_t NT) {
  PrefixLoads p{0, 0, 0};
  if (tile >= NT) return p;
  const uint32_t nt = prefix_terms(tile), j = threadIdx.x;
  if (j < nt) p.v0 = __ldcg(prefix_term(c, tile, j));
  if (j + THREADS < nt) p.v1 = __ldcg(prefix_term(c, tile, j + THREADS));
  if (j + 2 * THREADS < nt) p.v2 = __ldcg(prefix_term(c, tile, j + 2 * THREADS));
  return p;
}

template <int SB, int THREADS>
__device__ __forceinline__ void load_from_smem(const uint8_t *sIn, uint32_t my0, uint32_t *u) {
  const uint4 *src = reinterpret_cast<const uint4 *>(sIn + my0 * SB);
#pragma unroll
  for (int c = 0; c < 2 * SB; ++c) {
    const uint4 v = src[c];
    u[4 * c + 0] = v.x;
    u[4 * c + 1] = v.y;
    u[4 * c + 2] = v.z;
    u[4 * c + 3] = v.w;
  }
}

// Bit k of this thread's 32 symbols (positions my0..my0+31 of the tile held
// in sIn) as one word, symbol q -> bit q.  One-byte symbols: two 16-byte
// loads and SWAR packing per thread.  Wider symbols: the warp reads its
// 32 x 32 symbols row by row (lane i takes symbol 32c + i: consecutive
// addresses, no bank conflict) and the ballot of row c is the word of the
// thread that owns it; per-thread 16-byte loads of 64 or 128 consecutive
// bytes would serialise 4 or 8 ways on the shared-memory banks.
// Called by all threads of the warp.
// Bit k of the 32 * WPT consecutive 1-byte symbols at my0 (WPT words).  The
// thread reads its 2 * WPT 16-byte chunks in an order rotated by lane: the
// eight lanes of a quarter-warp, whose chunks lie 32 * WPT bytes apart,
// would otherwise meet in 2 (WPT = 1) or 4 (WPT = 2) of the eight 16-byte
// bank groups on every load; rotated, each load of the quarter-warp touches
// all eight once.  The packed bits are rotated back into place.
template <int WPT>
__device__ __forceinline__ void tile_words_1b(const uint8_t *sIn, uint32_t my0, uint32_t k, uint32_t (&w)[WPT]) {
  static_assert(WPT == 1 || WPT == 2, "one or two words per thread");
  constexpr uint32_t NC = 2 * WPT;                    // 16-byte chunks of the thread
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t r = (lane / (8 / NC)) & (NC - 1);    // rotation of the chunk order
  const uint4 *src = reinterpret_cast<const uint4 *>(sIn + my0);
  uint32_t p[NC];
#pragma unroll
  for (uint32_t j = 0; j < NC; ++j) {
    const uint4 v = src[(j + r) & (NC - 1)];
    const uint32_t q[4] = {v.x, v.y, v.z, v.w};
    uint32_t bits = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      // bit k of each byte to bit 0 of the byte, then gather the four bits
      // into the top nibble with one multiply (no carries between terms)
      const uint32_t x = (q[m] >> k) & 0x01010101u;
      bits |= ((x * 0x10204080u) >> 28) << (4 * m);
    }
    p[j] = bits;  // 16 bits: chunk (j + r) mod NC
  }
  if constexpr (WPT == 1) {
    w[0] = __funnelshift_l(p[0] | (p[1] << 16), p[0] | (p[1] << 16), 16 * r);  // rotate left by 16 r
  } else {
    // the 64-bit value with chunk (j + r) mod 4 at bits 16 j, rotated left by 16 r
    uint32_t lo = p[0] | (p[1] << 16), hi = p[2] | (p[3] << 16);
    if (r & 2u) {
      const uint32_t t = lo;
      lo = hi;
      hi = t;
    }
    const uint32_t sh = 16u * (r & 1u);
    w[0] = __funnelshift_l(hi, lo, sh);
    w[1] = __funnelshift_l(lo, hi, sh);
  }
}

template <int SB, int THREADS>
__device__ __forceinline__ uint32_t tile_word(const uint8_t *sIn, uint32_t my0, uint32_t k) {
  if (SB == 1) {
    uint32_t w[1];
    tile_words_1b<1>(sIn, my0, k, w);
    return w[0];
  } else {
    using Sym = typename SymT<SB>::type;
    const uint32_t lane = threadIdx.x & 31;
    const Sym *rows = reinterpret_cast<const Sym *>(sIn) + (my0 - 32 * lane);
    uint32_t word = 0;
#pragma unroll 8
    for (uint32_t c = 0; c < 32; ++c) {
      const uint32_t b = __ballot_sync(0xFFFFFFFFu, ((uint32_t)rows[32 * c + lane] >> k) & 1u);
      word = lane == c ? b : word;
    }
    return word;
  }
}

template <int SB, int THREADS>
constexpr uint32_t pipe_smem_bytes() {
  return 2u * 32u * THREADS * SB;
}

// ------------------------------------------------------------------ pre-pass
// Where the pre-pass keeps its symbol histogram: nowhere (the wavelet matrix
// needs none), in shared-memory bins, in global bins updated with
// warp-aggregated atomics, or (few bins) in shared memory with one copy of
// every bin per lane: bin v of lane i at v * 32 + i, so the 32 updates of a
// warp row always fall in 32 distinct banks (the copies are summed once per
// CTA, each thread reading its bin's copies in a rotated order).
// One more for tiles handled one at a time (the batched build), where no
// per-CTA histogram outlives the tile: kHistBallot (up to 16 bins) counts
// each row with one ballot per bin and adds every warp's counts to the
// global bins at the end of the tile (shared-memory atomics of a row would
// collide on so few bins).
enum HistMode : int { kHistNone = 0, kHistSmem = 1, kHistGlobal = 2, kHistLanes = 3, kHistBallot = 4 };
constexpr uint32_t kHistBallotMaxBins = 16;
constexpr uint32_t kHistLanesMaxBins = 256;
constexpr uint32_t kHotSlots = 1024;  // per-CTA table of hot bins for kHistGlobal
constexpr uint32_t kHotEmpty = 0xFFFFFFFFu;

__host__ __device__ constexpr uint32_t hist_smem_words(int mode, uint32_t nbins) {
  return mode == kHistSmem ? ((nbins + 1) & ~1u)
         : mode == kHistLanes ? nbins * 32
         : mode == kHistGlobal ? 2u * kHotSlots : 0u;
}

// Add c occurrences of bin v to a global histogram (one lane).  A bin that
// occurs more than once among a warp's 32 symbols of one step is likely hot
// (skewed inputs), and global atomics on one hot word serialise across the
// whole GPU: such bins are counted in `hot`, a per-CTA open-addressed table
// in shared memory (kHotSlots tags, then kHotSlots counts; a slot, once
// claimed, keeps its bin), which the caller flushes once.  Other bins, and
// hot bins that find no slot within four probes, go to global memory.
__device__ __forceinline__ void hist_add(uint32_t *ghist, uint32_t *hot, uint32_t v, uint32_t c) {
  if (hot && c > 1) {
    uint32_t slot = v & (kHotSlots - 1);
#pragma unroll 1
    for (int probe = 0; probe < 4; ++probe) {
      uint32_t t = *reinterpret_cast<volatile uint32_t *>(&hot[slot]);
      if (t == kHotEmpty) t = atomicCAS(&hot[slot], kHotEmpty, v);
      if (t == kHotEmpty || t == v) {
        atomicAdd(&hot[kHotSlots + slot], c);
        return;
      }
      slot = (slot + 1) & (kHotSlots - 1);
    }
  }
  atomicAdd(&ghist[v], c);
}

struct PrepassArgs {
  const uint8_t *in;  // S, 16-byte aligned
  int in_padded;
  uint32_t n, L, NT, sigma;
  uint32_t *hist;     // 2^L bins
  TileCounts cnt;     // level-0 ones per tile
  uint32_t *ticket;
  uint32_t spin_limit;
  int *err;
};

template <int SB, int THREADS>
constexpr uint32_t prepass_smem_bytes(uint32_t hist_words) {
  return pipe_smem_bytes<SB, THREADS>() + 4u * hist_words + 64u;
}

// One pre-pass tile: symbol histogram (per HIST), range check (into `bad`)
// and the level-0 ones of the tile.  Ends with a block barrier, after which thread 0
// has stored ring_value to *ring_slot (if non-null).
template <int SB, int THREADS, int HIST>
__device__ __forceinline__ void prepass_tile(const PrepassArgs &a, uint32_t tile, const uint8_t *sIn,
                                           uint32_t *s_hist, uint32_t *s_wt, uint32_t &bad,
                                           uint32_t *ring_slot, uint32_t ring_value) {
  constexpr uint32_t T = 32 * THREADS;
  constexpr uint32_t NW = THREADS / 32;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lmask = (1u << a.L) - 1u;
  const uint64_t start = (uint64_t)tile * T;
  const uint32_t nv = (uint32_t)umin64(T, a.n - start);
  const uint32_t my0 = 32 * tid;
  const uint32_t word = a.L ? tile_word<SB, THREADS>(sIn, my0, a.L - 1) & valid_mask(my0, nv) : 0u;
  // The warp walks its 1024 symbols row by row: lane i takes symbol 32c + i
  // of row c (consecutive shared-memory addresses, and the symbols of a row
  // are what the warp-wide aggregation below sees together).
  using Sym = typename SymT<SB>::type;
  const Sym *rows = reinterpret_cast<const Sym *>(sIn) + 1024 * warp;
  const uint32_t seg = 1024 * warp;
  const uint32_t nvw = nv > seg ? min(nv - seg, 1024u) : 0u;  // warp-uniform
  uint32_t bcnt = 0;  // kHistBallot: lane b's count of bin b in the warp's rows
  if (HIST == kHistNone) {
    // range check only, and only when the storage type can exceed sigma
    if (a.sigma < (SB == 4 ? 0xFFFFFFFFu : (1u << (8 * SB)))) {
      uint32_t mx = 0;
#pragma unroll 8
      for (uint32_t c = 0; c < 32; ++c)
        if (32 * c + lane < nvw) mx = max(mx, (uint32_t)rows[32 * c + lane]);
      bad |= (uint32_t)(mx >= a.sigma);
    }
  } else if (nvw == 1024) {
#pragma unroll 4
    for (uint32_t c = 0; c < 32; ++c) {
      const uint32_t s = rows[32 * c + lane];
      bad |= (uint32_t)(s >= a.sigma);
      const uint32_t v = s & lmask;
      if (HIST == kHistLanes) {
        atomicAdd(&s_hist[v * 32 + lane], 1u);
      } else if (HIST == kHistSmem) {
        atomicAdd(&s_hist[v], 1u);
      } else if (HIST == kHistBallot) {
        for (uint32_t b = 0; b < (1u << a.L); ++b) {
          const uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, v == b));
          bcnt += lane == b ? c : 0u;
        }
      } else {
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, v);
        if (lane == (uint32_t)(__ffs(peers) - 1)) hist_add(a.hist, s_hist, v, (uint32_t)__popc(peers));
      }
    }
  } else {
    for (uint32_t c = 0; c < 32; ++c) {
      const bool valid = 32 * c + lane < nvw;
      const uint32_t s = valid ? (uint32_t)rows[32 * c + lane] : 0u;
      bad |= (uint32_t)(s >= a.sigma);
      const uint32_t v = s & lmask;
      if (HIST == kHistLanes) {
        if (valid) atomicAdd(&s_hist[v * 32 + lane], 1u);
      } else if (HIST == kHistSmem) {
        if (valid) atomicAdd(&s_hist[v], 1u);
      } else if (HIST == kHistBallot) {
        for (uint32_t b = 0; b < (1u << a.L); ++b) {
          const uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, valid && v == b));
          bcnt += lane == b ? c : 0u;
        }
      } else {
        const uint32_t am = __ballot_sync(0xFFFFFFFFu, valid);
        if (valid) {
          const uint32_t peers = __match_any_sync(am, v);
          if (lane == (uint32_t)(__ffs(peers) - 1)) hist_add(a.hist, s_hist, v, (uint32_t)__popc(peers));
        }
      }
    }
  }
  if (HIST == kHistBallot && bcnt) atomicAdd(&a.hist[lane], bcnt);
  const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, __popc(word));
  if (lane == 0) s_wt[warp] = wsum;
  cta_sync<THREADS>();
  if (warp == 0 && a.L) {
    const uint32_t total = __reduce_add_sync(0xFFFFFFFFu, lane < NW ? s_wt[lane] : 0u);
    if (lane == 0) {
      a.cnt.c0[tile] = total;
      if (total) {
        atomicAdd(&a.cnt.c1[tile >> 6], total);
        atomicAdd(&a.cnt.c2[tile >> 12], total);
      }
    }
  }
  if (ring_slot) *ring_slot = ring_value;
  cta_sync<THREADS>();
}

// Reads S once: the 2^L-bin histogram (node sizes of every level; not for
// the wavelet matrix), the range check, and the level-0 ones of every tile.
template <int SB, int THREADS, int HIST>
__global__ void __launch_bounds__(THREADS) k_prepass(PrepassArgs a) {
  constexpr uint32_t T = 32 * THREADS;
  extern __shared__ __align__(128) uint8_t smem[];
  TilePipe<SB, THREADS> pipe;
  const uint32_t nbins = 1u << a.L;
  pipe.sIn0 = smem;
  pipe.sIn1 = smem + pipe.TB;
  uint32_t *const s_hist = reinterpret_cast<uint32_t *>(smem + 2 * pipe.TB);
  uint64_t *const bar = reinterpret_cast<uint64_t *>(s_hist + hist_smem_words(HIST, nbins));
  pipe.bar = bar;
  pipe.ring = reinterpret_cast<uint32_t *>(bar + 2);
  uint32_t *const s_wt = pipe.ring + 4;  // ones per warp
  pipe.in = a.in;
  pipe.in_padded = a.in_padded;
  pipe.n = a.n;
  pipe.NT = a.NT;
  pipe.ticket = a.ticket;
  const uint32_t tid = threadIdx.x;
  uint32_t bad = 0;
  for (uint32_t i = tid; i < hist_smem_words(HIST, nbins); i += THREADS)
    s_hist[i] = (HIST == kHistGlobal && i < kHotSlots) ? kHotEmpty : 0u;
  if (tid == 0) pipe.prologue();
  __syncthreads();

  for (uint32_t it = 0;; ++it) {
    const uint32_t tile = pipe.ring[it % 3];
    if (tile >= a.NT) break;
    const uint32_t nxt = pipe.ring[(it + 1) % 3];
    uint32_t nn = 0;
    if (tid == 0) nn = pipe.advance(it, nxt);
    const bool ok = pipe.wait(it, a.spin_limit, a.err);
    if (__syncthreads_or(!ok)) {
      pipe.drain(it, a.spin_limit, a.err);
      __syncthreads();
      break;
    }
    const uint64_t start = (uint64_t)tile * T;
    const uint32_t nv = (uint32_t)umin64(T, a.n - start);
    uint8_t *const sIn = pipe.data(it);
    if (pipe.fill_tail(sIn, start, nv)) __syncthreads();
    prepass_tile<SB, THREADS, HIST>(a, tile, sIn, s_hist, s_wt, bad,
                                         tid == 0 ? &pipe.ring[(it + 2) % 3] : nullptr, nn);
  }
  if (bad) latch_error(a.err, WT_ERR_SYMBOL);
  if (HIST == kHistSmem) {
    __syncthreads();
    for (uint32_t i = tid; i < nbins; i += THREADS)
      if (s_hist[i]) atomicAdd(&a.hist[i], s_hist[i]);
  } else if (HIST == kHistGlobal) {
    __syncthreads();
    for (uint32_t i = tid; i < kHotSlots; i += THREADS)
      if (s_hist[i] != kHotEmpty && s_hist[kHotSlots + i]) atomicAdd(&a.hist[s_hist[i]], s_hist[kHotSlots + i]);
  } else if (HIST == kHistLanes) {
    __syncthreads();
    for (uint32_t i = tid; i < nbins; i += THREADS) {
      uint32_t c = 0;
#pragma unroll 8
      for (uint32_t r = 0; r < 32; ++r) c += s_hist[i * 32 + ((r + i) & 31u)];
      if (c) atomicAdd(&a.hist[i], c);
    }
  }
}

// ------------------------------------------------------------------ last level
struct LeafArgs {
  const uint8_t *in;  // T_{L-1}, 16-byte aligned
  int in_padded;
  uint32_t n, L, NT, NB;
  uint64_t W;
  LevelOut out;
  TileCounts cnt;     // ones of this level per tile
  uint32_t *ticket;
  uint32_t spin_limit;
  int *err;
};

template <int SB, int THREADS>
constexpr uint32_t leaf_smem_bytes() {
  return pipe_smem_bytes<SB, THREADS>() + 8u * (THREADS / 32) + 64u;
}

// One tile of the last level: bits and directory.  share_part is this
// thread's part of the tile's ones-prefix.  Ends with a block barrier, after
// which thread 0 has stored ring_value to *ring_slot (if non-null).
template <int SB, int THREADS>
__device__ __forceinline__ void leaf_tile(const LeafArgs &a, uint32_t tile, const uint8_t *sIn,
                                          uint32_t share_part, uint2 *s_wt, uint32_t *ring_slot,
                                          uint32_t ring_value) {
  constexpr uint32_t T = 32 * THREADS;
  constexpr uint32_t NW = THREADS / 32;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t start = (uint64_t)tile * T;
  const uint32_t nv = (uint32_t)umin64(T, a.n - start);
  const uint32_t my0 = 32 * tid;
  const uint32_t word = tile_word<SB, THREADS>(sIn, my0, 0) & valid_mask(my0, nv);
  const uint32_t pc = __popc(word);
  uint32_t incl = pc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  const uint32_t share = __reduce_add_sync(0xFFFFFFFFu, share_part);
  if (lane == 31) s_wt[warp] = make_uint2(incl, share);
  cta_sync<THREADS>();
  const uint2 wv = lane < NW ? s_wt[lane] : make_uint2(0, 0);
  const uint32_t Pw = __reduce_add_sync(0xFFFFFFFFu, lane < warp ? wv.x : 0u);
  const uint32_t total = __reduce_add_sync(0xFFFFFFFFu, wv.x);
  const uint32_t R = __reduce_add_sync(0xFFFFFFFFu, wv.y);
  write_level<THREADS>(a.out, tile, a.NT, start, my0, a.n, a.NB, a.W, word, R, Pw + incl - pc, total);
  if (ring_slot) *ring_slot = ring_value;
  cta_sync<THREADS>();
}

// Level L-1 (and level 0 when L = 1): bits and directory; its nodes have
// range 2 and no children.
template <int SB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_leaf(LeafArgs a) {
  constexpr uint32_t T = 32 * THREADS;
  constexpr uint32_t NW = THREADS / 32;
  extern __shared__ __align__(128) uint8_t smem[];
  TilePipe<SB, THREADS> pipe;
  pipe.sIn0 = smem;
  pipe.sIn1 = smem + pipe.TB;
  uint2 *const s_wt = reinterpret_cast<uint2 *>(smem + 2 * pipe.TB);  // {ones, prefix share} per warp
  pipe.bar = reinterpret_cast<uint64_t *>(s_wt + NW);
  pipe.ring = reinterpret_cast<uint32_t *>(pipe.bar + 2);
  pipe.in = a.in;
  pipe.in_padded = a.in_padded;
  pipe.n = a.n;
  pipe.NT = a.NT;
  pipe.ticket = a.ticket;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) pipe.prologue();
  __syncthreads();
  PrefixLoads pre = prefix_loads<THREADS>(a.cnt, pipe.ring[0], a.NT);

  for (uint32_t it = 0;; ++it) {
    const uint32_t tile = pipe.ring[it % 3];
    if (tile >= a.NT) break;
    const uint32_t nxt = pipe.ring[(it + 1) % 3];
    uint32_t nn = 0;
    if (tid == 0) nn = pipe.advance(it, nxt);
    const PrefixLoads pre_next = prefix_loads<THREADS>(a.cnt, nxt, a.NT);
    const bool ok = pipe.wait(it, a.spin_limit, a.err);
    if (__syncthreads_or(!ok)) {
      pipe.drain(it, a.spin_limit, a.err);
      __syncthreads();
      break;
    }
    const uint64_t start = (uint64_t)tile * T;
    const uint32_t nv = (uint32_t)umin64(T, a.n - start);
    uint8_t *const sIn = pipe.data(it);
    if (pipe.fill_tail(sIn, start, nv)) __syncthreads();
    leaf_tile<SB, THREADS>(a, tile, sIn, pre.sum(), s_wt, tid == 0 ? &pipe.ring[(it + 2) % 3] : nullptr, nn);
    pre = pre_next;
  }
}

// ------------------------------------------------------------------ split pass
struct SplitArgs {
  const uint8_t *in;   // T_l, 16-byte aligned
  uint8_t *out;        // T_{l+1}
  int in_padded;       // in holds whole tiles (scratch buffer) -> copy whole tiles
  uint32_t n, L, level, NT, NB, log2T;
  uint64_t W;
  const uint2 *tab;    // this level's {O_l[p], E_{l+1}[2p+1] - O_l[p]}
  uint32_t pshift;     // node prefix = symbol >> pshift (L - level; L for the matrix)
  int count_table;     // one node whose table {0, zeros of the level} comes from the
                       // level's tile counts (wavelet matrix; tree level 0 with node counts)
  uint2 *tab_out;      // if set, CTA 0 also stores that one-node table there
  uint32_t *nones_next;  // if set, ones of level l+1 per child node (2p + bit) are added here
  // If node_ones is set (node counts, a level of at most one node per
  // thread), every CTA computes this level's table in shared memory from the
  // nodes' ones (node_ones), the previous level's table (tab_prev) and the
  // node starts (E), and CTA 0 also stores it to tab_w and the odd nodes'
  // starts to E -- what the node-table kernel would have done before the pass.
  const uint32_t *node_ones;
  const uint2 *tab_prev;
  uint2 *tab_w;
  unsigned long long *E;
  LevelOut lo;
  TileCounts cin;      // ones of level l per tile of T_l
  TileCounts cout;     // ones of level l+1 per tile of T_{l+1} (accumulated here)
  uint32_t *ticket;
  uint32_t spin_limit;
  int *err;
};

// Bit k1 of the symbols packed in a 32-bit word, counted.
template <int SB>
__device__ __forceinline__ uint32_t count_bit(uint32_t w, uint32_t k1) {
  if (SB == 1) return __popc((w >> k1) & 0x01010101u);
  if (SB == 2) return __popc((w >> k1) & 0x00010001u);
  return (w >> k1) & 1u;
}

// Copy one run of `len` bytes staged in shared memory at byte offset soff of
// `stage` to global byte offset g of `gout`; executed by one warp.  The run
// was staged so that soff = g (mod 16): every full 16-byte chunk is one
// aligned shared load and one aligned global store; the unaligned head and
// tail bytes are copied singly.  Bit k1 of the copied symbols is counted into
// cnt_a (symbol positions before split_at) and cnt_b (from split_at on).
// Writes past gend (n * SB) are dropped (reachable only after a device error).
template <int SB>
__device__ __forceinline__ void warp_copy_run(const uint8_t *stage, uint32_t soff, uint8_t *gout,
                                              uint64_t g, uint32_t len, uint64_t gend,
                                              uint32_t split_at, uint32_t mk1, uint32_t k1,
                                              uint32_t &cnt_a, uint32_t &cnt_b) {
  if (g >= gend) return;
  if (g + len > gend) len = (uint32_t)(gend - g);
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t head = min(len, (16u - ((uint32_t)g & 15u)) & 15u);
  const uint32_t nch = (len - head) >> 4;
  const uint32_t tail0 = head + (nch << 4);
  const uint32_t nb = head + (len - tail0);  // single bytes: head, then tail
  const uint32_t p0 = (uint32_t)(g / SB);    // symbol position of the run's first byte
  if (lane < nb) {
    const uint32_t o = lane < head ? lane : tail0 + (lane - head);
    gout[g + o] = stage[soff + o];
    if (o % SB == 0) {  // first byte of a symbol: count it
      uint32_t v;
      if (SB == 1) v = stage[soff + o];
      else if (SB == 2) v = *reinterpret_cast<const uint16_t *>(stage + soff + o);
      else v = *reinterpret_cast<const uint32_t *>(stage + soff + o);
      const uint32_t one = (v >> k1) & 1u;
      if (p0 + o / SB >= split_at) cnt_b += one;
      else cnt_a += one;
    }
  }
  const uint4 *src = reinterpret_cast<const uint4 *>(stage + soff + head);
  uint4 *dst = reinterpret_cast<uint4 *>(gout + g + head);
  const uint32_t pc0 = p0 + head / SB;  // symbol position of chunk 0
  for (uint32_t c = lane; c < nch; c += 32) {
    const uint4 v = src[c];
    dst[c] = v;
    const uint32_t ones = __popc(v.x & mk1) + __popc(v.y & mk1) + __popc(v.z & mk1) + __popc(v.w & mk1);
    if (pc0 + c * (16 / SB) >= split_at) cnt_b += ones;
    else cnt_a += ones;
  }
}


// The two runs of a warp that lies in one node (zeros, then ones), as
// warp_copy_run does them one after the other, but as one list of 16-byte
// chunks, two per lane loaded from shared memory before either is stored, so
// that the loads' latency overlaps (J: chunks per lane at most, 2 * WPT * SB
// for a warp segment of 1024 * WPT symbols, even).  Used at 1-byte symbols
// with two words per thread (0.6 % faster there; at 2-byte symbols the
// split pass was 4 % slower with it).  Run r's head and tail bytes
// are copied singly by lanes 0..; the counts are split at split_r as there.
template <int SB, int J>
__device__ __forceinline__ void warp_copy_runs2(const uint8_t *stage, uint8_t *gout, uint64_t gend, uint32_t mk1,
                                                uint32_t k1, uint32_t soff0, uint64_t g0, uint32_t len0,
                                                uint32_t split0, uint32_t soff1, uint64_t g1, uint32_t len1,
                                                uint32_t split1, uint32_t &c0a, uint32_t &c0b, uint32_t &c1a,
                                                uint32_t &c1b) {
  const uint32_t lane = threadIdx.x & 31;
  if (g0 >= gend) len0 = 0;
  else if (g0 + len0 > gend) len0 = (uint32_t)(gend - g0);
  if (g1 >= gend) len1 = 0;
  else if (g1 + len1 > gend) len1 = (uint32_t)(gend - g1);
  const uint32_t h0 = min(len0, (16u - ((uint32_t)g0 & 15u)) & 15u), n0 = (len0 - h0) >> 4;
  const uint32_t h1 = min(len1, (16u - ((uint32_t)g1 & 15u)) & 15u), n1 = (len1 - h1) >> 4;
  const uint32_t p0 = (uint32_t)(g0 / SB), p1 = (uint32_t)(g1 / SB);  // symbol positions of the runs
  const uint32_t N = n0 + n1;
  // head and tail bytes: run 0's, then run 1's
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const uint32_t len = r ? len1 : len0, h = r ? h1 : h0, nch = r ? n1 : n0;
    const uint32_t soff = r ? soff1 : soff0, pr = r ? p1 : p0, split_at = r ? split1 : split0;
    const uint64_t g = r ? g1 : g0;
    const uint32_t tail0 = h + (nch << 4);
    const uint32_t nb = h + (len - tail0);
    if (lane < nb) {
      const uint32_t o = lane < h ? lane : tail0 + (lane - h);
      const uint8_t byte = stage[soff + o];
      gout[g + o] = byte;
      if (o % SB == 0) {  // first byte of a symbol: count it
        uint32_t sv;
        if (SB == 1) sv = byte;
        else if (SB == 2) sv = *reinterpret_cast<const uint16_t *>(stage + soff + o);
        else sv = *reinterpret_cast<const uint32_t *>(stage + soff + o);
        const uint32_t one = (sv >> k1) & 1u;
        const bool after = pr + o / SB >= split_at;
        if (r) {
          c1b += after ? one : 0u;
          c1a += after ? 0u : one;
        } else {
          c0b += after ? one : 0u;
          c0a += after ? 0u : one;
        }
      }
    }
  }
  // the chunks, two per lane at a time: both loads before the stores
#pragma unroll
  for (int j0 = 0; j0 < J; j0 += 2) {
    uint4 v[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t q = lane + 32u * (j0 + u);
      if (q < N) {
        const bool r = q >= n0;
        const uint32_t c = r ? q - n0 : q;
        v[u] = *reinterpret_cast<const uint4 *>(stage + (r ? soff1 + h1 : soff0 + h0) + 16u * c);
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const uint32_t q = lane + 32u * (j0 + u);
      if (q < N) {
        const bool r = q >= n0;
        const uint32_t c = r ? q - n0 : q;
        *reinterpret_cast<uint4 *>(gout + (r ? g1 + h1 : g0 + h0) + 16u * c) = v[u];
        const uint32_t ones =
            __popc(v[u].x & mk1) + __popc(v[u].y & mk1) + __popc(v[u].z & mk1) + __popc(v[u].w & mk1);
        const uint32_t pos = (r ? p1 + h1 / SB : p0 + h0 / SB) + c * (16u / SB);
        const bool after = pos >= (r ? split1 : split0);
        if (r) {
          c1b += after ? ones : 0u;
          c1a += after ? 0u : ones;
        } else {
          c0b += after ? ones : 0u;
          c0a += after ? 0u : ones;
        }
      }
    }
  }
}

// Store v (the low SB bytes) at shared address oa if bit != 0, else at za,
// and advance that address by one symbol.  Predicated, branch-free.
template <int SB>
__device__ __forceinline__ void scatter_one(uint32_t bit, uint32_t &oa, uint32_t &za, uint32_t v) {
  if (SB == 1) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
        "@p st.shared.u8 [%0], %3;\n\t@!p st.shared.u8 [%1], %3;\n\t"
        "@p add.u32 %0, %0, 1;\n\t@!p add.u32 %1, %1, 1;\n\t}"
        : "+r"(oa), "+r"(za)
        : "r"(bit), "r"(v)
        : "memory");
  } else if (SB == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
        "@p st.shared.u16 [%0], %3;\n\t@!p st.shared.u16 [%1], %3;\n\t"
        "@p add.u32 %0, %0, 2;\n\t@!p add.u32 %1, %1, 2;\n\t}"
        : "+r"(oa), "+r"(za)
        : "r"(bit), "h"((unsigned short)v)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
        "@p st.shared.u32 [%0], %3;\n\t@!p st.shared.u32 [%1], %3;\n\t"
        "@p add.u32 %0, %0, 4;\n\t@!p add.u32 %1, %1, 4;\n\t}"
        : "+r"(oa), "+r"(za)
        : "r"(bit), "r"(v)
        : "memory");
  }
}

// per-warp staging: 1024 symbols plus room to align both runs to their
// global 16-byte phase
template <int SB, int WPT = 1>
__host__ __device__ constexpr uint32_t stage_bytes() { return 1024u * WPT * SB + 48u; }

// Level tables of up to this many nodes live in shared memory.  1-byte
// symbols have at most 2^7 nodes per split level (sigma <= 256).
template <int SB>
__host__ __device__ constexpr uint32_t tab_smem_nodes() { return SB == 1 ? 128u : 1024u; }

template <int SB, int THREADS, int DEPTH = 2, int WPT = 1>
constexpr uint32_t split_smem_bytes() {
  // DEPTH input tiles, per-warp staging, per-word {bit word, warp-local
  // ones-prefix}, two sets (tile parity) of per-warp {ones, prefix share},
  // the level table, mbarriers, tickets, run counters and run starts
  return DEPTH * 32u * WPT * THREADS * SB + (THREADS / 32) * stage_bytes<SB, WPT>() + 8u * WPT * THREADS +
         16u * (THREADS / 32) + 8u * tab_smem_nodes<SB>() + 192u + (SB == 1 ? 1024u : 0u);
}

// Phase C of a warp whose symbols span several nodes (the tile is not in
// one node either): each symbol goes to the zero or one range of its own
// node.  wWP is the warp's {bit word, ones before the word} array.
//   1-byte symbols: symbol by symbol (small alphabets have few multi-node
//     warps, and this form keeps the single-node path's registers intact).
//   wider symbols, at most 32 nodes in the warp: one run per node and part.
//   more nodes: symbol by symbol.
template <int SB, bool NC>
__device__ __forceinline__ void split_multi_node(uint8_t *out, uint32_t n, uint32_t log2T, uint32_t NT,
                                              TileCounts cout, uint32_t *nones_next, const uint2 *tab,
                                              const typename SymT<SB>::type *sInS,
                                              const typename SymT<SB>::type *stageS, const uint2 *wWP,
                                              uint32_t seg, uint32_t nvw, uint32_t nzw, uint32_t wpf,
                                              uint32_t wpl, uint32_t Zw, uint32_t Ow, uint32_t lmask,
                                              uint32_t pshift, uint32_t k1) {
  using Sym = typename SymT<SB>::type;
  const uint32_t lane = threadIdx.x & 31;
  if constexpr (SB == 1) {
    // Zeros (then ones) are staged in node order, so their destinations
    // rise monotonically: ones are counted per run of equal destination
    // tile, carried across groups, one flush per change of tile.  When the
    // warp spans at most 32 nodes their table entries are fetched once, one
    // per lane, and exchanged by shuffle.
    (void)sInS;
    (void)wWP;
    Sym *outS = reinterpret_cast<Sym *>(out);
    const uint32_t span = wpl - wpf + 1;
    const bool lanes_tab = wpl >= wpf && span <= 32;
    uint2 mytab = make_uint2(0u, 0u);
    if (lanes_tab && lane < span) mytab = tab[wpf + lane];
    uint32_t cdt = 0xFFFFFFFFu, ccnt = 0;  // running destination tile and its ones
    for (uint32_t base = 0; base < nvw; base += 32) {
      const uint32_t kk = base + lane;
      const bool valid = kk < nvw;
      const Sym sv = valid ? stageS[kk] : (Sym)0;
      const uint32_t p = ((uint32_t)sv & lmask) >> pshift;
      uint2 tb;
      if (lanes_tab) {
        const uint32_t src = valid ? p - wpf : 0u;
        tb.x = __shfl_sync(0xFFFFFFFFu, mytab.x, src);
        tb.y = __shfl_sync(0xFFFFFFFFu, mytab.y, src);
      } else {
        tb = valid ? tab[p] : make_uint2(0u, 0u);
      }
      uint32_t dt = 0xFFFFFFFFu, bit = 0;
      if (valid) {
        const uint32_t dest = kk < nzw ? tb.x + Zw + kk : tb.y + Ow + (kk - nzw);
        if (dest < n) {
          outS[dest] = sv;
          dt = dest >> log2T;
          bit = ((uint32_t)sv >> k1) & 1u;
        }
      }
      const uint32_t ones = __ballot_sync(0xFFFFFFFFu, bit);
      if (NC && nones_next) {  // ones of level l+1 per child node 2p + bit
        const uint32_t child = dt != 0xFFFFFFFFu ? 2 * p + (kk >= nzw ? 1u : 0u) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, child);
        const uint32_t c = __popc(ones & peers);
        if (child != 0xFFFFFFFFu && c && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&nones_next[child], c);
      }
      const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, dt, 1);
      uint32_t heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || dt != prev);
      while (heads) {  // warp-uniform: one step per run of equal dt
        const uint32_t h = __ffs(heads) - 1;
        heads &= heads - 1;
        const uint32_t sdt = __shfl_sync(0xFFFFFFFFu, dt, h);
        if (sdt == 0xFFFFFFFFu) continue;
        const uint32_t nx = heads ? (uint32_t)__ffs(heads) - 1 : 32u;
        const uint32_t seg_mask = (nx == 32 ? 0xFFFFFFFFu : (1u << nx) - 1u) & ~((1u << h) - 1u);
        const uint32_t c = __popc(ones & seg_mask);
        if (sdt == cdt) {
          ccnt += c;
        } else {
          if (lane == 0 && ccnt) counts_add(cout, cdt, ccnt);
          cdt = sdt;
          ccnt = c;
        }
      }
    }
    if (lane == 0 && ccnt) counts_add(cout, cdt, ccnt);
  } else if (wpl >= wpf && wpl - wpf < 32) {
    // Several nodes in the warp, at most 32: the staging holds, for each
    // node in order, its zeros, then (after all zeros) its ones; each
    // is one run with one destination.  Lane q finds where node wpf+q
    // starts in the warp's input (binary search over the input, which
    // is in node order) and, from the bit words, how many zeros and
    // ones precede it; then the warp copies the runs node by node.
    Sym *outS = reinterpret_cast<Sym *>(out);
    const uint32_t span = wpl - wpf + 1;
    auto zeros_before = [&](uint32_t x) -> uint32_t {  // zeros of the warp before input position x
      if (x >= nvw) return nzw;
      const uint2 wv = wWP[x >> 5];
      return x - (wv.y + __popc(wv.x & ((1u << (x & 31)) - 1u)));
    };
    uint32_t f = nvw;  // first input position of node wpf + lane
    if (lane < span) {
      uint32_t lo = 0, hi = nvw;
      if (lane == 0) hi = 0;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((((uint32_t)sInS[seg + mid] & lmask) >> pshift) < wpf + lane) lo = mid + 1;
        else hi = mid;
      }
      f = lo;
    }
    const uint32_t fnext = __shfl_down_sync(0xFFFFFFFFu, f, 1);
    const uint32_t fe = lane + 1 < span ? fnext : nvw;
    const uint32_t zs = zeros_before(f), ze = zeros_before(fe);
    const uint2 tb = lane < span ? tab[wpf + lane] : make_uint2(0u, 0u);
    const uint32_t gzq = tb.x + Zw + zs;         // destination of the node's zeros
    const uint32_t goq = tb.y + Ow + (f - zs);   // destination of the node's ones
    const uint32_t zrun = ze - zs, orun = (fe - ze) - (f - zs);
    // The runs, node by node and zeros before ones, go to children 2p, 2p+1,
    // 2p+2, ... of T_{l+1}: their destinations rise, so the next level's ones
    // are added up per destination tile and flushed once per change of tile.
    uint32_t cdt = 0xFFFFFFFFu, ccnt = 0;  // running destination tile and its ones (lane 0)
    auto tile_add = [&](uint32_t t, uint32_t c) {
      if (t == cdt) {
        ccnt += c;
      } else {
        if (ccnt && cdt < NT) counts_add(cout, cdt, ccnt);
        cdt = t;
        ccnt = c;
      }
    };
    for (uint32_t q = 0; q < span; ++q) {
#pragma unroll
      for (uint32_t part = 0; part < 2; ++part) {
        const uint32_t len = __shfl_sync(0xFFFFFFFFu, part ? orun : zrun, q);
        if (len == 0) continue;
        const uint32_t src = __shfl_sync(0xFFFFFFFFu, part ? nzw + (f - zs) : zs, q);
        const uint32_t dst = __shfl_sync(0xFFFFFFFFu, part ? goq : gzq, q);
        const uint32_t dt = dst >> log2T, bnd = (dt + 1) << log2T;
        uint32_t ca = 0, cb = 0;
        for (uint32_t e = lane; e < len; e += 32) {
          const Sym v = stageS[src + e];
          const uint32_t d = dst + e;
          if (d < n) {
            outS[d] = v;
            const uint32_t one = ((uint32_t)v >> k1) & 1u;
            if (d < bnd) ca += one;
            else cb += one;
          }
        }
        ca = __reduce_add_sync(0xFFFFFFFFu, ca);
        cb = __reduce_add_sync(0xFFFFFFFFu, cb);
        if (lane == 0) {
          if (ca) tile_add(dt, ca);
          if (cb) tile_add(dt + 1, cb);
          if (NC && nones_next && ca + cb) atomicAdd(&nones_next[2 * (wpf + q) + part], ca + cb);
        }
      }
    }
    if (lane == 0 && ccnt && cdt < NT) counts_add(cout, cdt, ccnt);
  } else {
    // More than 32 nodes in the warp: each symbol goes to the zero or
    // one range of its own node.  Zeros (then ones) are staged in node
    // order, so their destinations rise monotonically: ones are counted
    // per run of equal destination tile, carried across groups, one
    // flush per change of tile.
    Sym *outS = reinterpret_cast<Sym *>(out);
    uint32_t cdt = 0xFFFFFFFFu, ccnt = 0;  // running destination tile and its ones
    for (uint32_t base = 0; base < nvw; base += 32) {
      const uint32_t kk = base + lane;
      const bool valid = kk < nvw;
      const Sym sv = valid ? stageS[kk] : (Sym)0;
      const uint32_t p = ((uint32_t)sv & lmask) >> pshift;
      const uint2 tb = valid ? tab[p] : make_uint2(0u, 0u);
      uint32_t dt = 0xFFFFFFFFu, bit = 0;
      if (valid) {
        const uint32_t dest = kk < nzw ? tb.x + Zw + kk : tb.y + Ow + (kk - nzw);
        if (dest < n) {
          outS[dest] = sv;
          dt = dest >> log2T;
          bit = ((uint32_t)sv >> k1) & 1u;
        }
      }
      const uint32_t ones = __ballot_sync(0xFFFFFFFFu, bit);
      if (NC && nones_next) {  // ones of level l+1 per child node 2p + bit
        const uint32_t child = dt != 0xFFFFFFFFu ? 2 * p + (kk >= nzw ? 1u : 0u) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, child);
        const uint32_t c = __popc(ones & peers);
        if (child != 0xFFFFFFFFu && c && lane == (uint32_t)(__ffs(peers) - 1))
          atomicAdd(&nones_next[child], c);
      }
      const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, dt, 1);
      uint32_t heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || dt != prev);
      while (heads) {  // warp-uniform: one step per run of equal dt
        const uint32_t h = __ffs(heads) - 1;
        heads &= heads - 1;
        const uint32_t sdt = __shfl_sync(0xFFFFFFFFu, dt, h);
        if (sdt == 0xFFFFFFFFu) continue;
        const uint32_t nx = heads ? (uint32_t)__ffs(heads) - 1 : 32u;
        const uint32_t seg_mask = (nx == 32 ? 0xFFFFFFFFu : (1u << nx) - 1u) & ~((1u << h) - 1u);
        const uint32_t c = __popc(ones & seg_mask);
        if (sdt == cdt) {
          ccnt += c;
        } else {
          if (lane == 0 && ccnt) counts_add(cout, cdt, ccnt);
          cdt = sdt;
          ccnt = c;
        }
      }
    }
    if (lane == 0 && ccnt) counts_add(cout, cdt, ccnt);
  }
}

// Shared-memory working set of one split tile.
struct SplitShared {
  uint8_t *stage;  // per-warp staging areas
  uint2 *wp;       // per thread {bit word, warp-local ones-prefix}
  uint2 *wt;       // per warp {ones, prefix share}
  uint32_t *cnt;   // 4 run counters
  uint32_t *run;   // 2 run starts
  uint32_t *nc;    // node-count cache of thread 0: {node, ones of child 2 node, of child 2 node + 1}
  const uint32_t *perm = nullptr;  // 1-byte symbols: the 256 partition selectors (partition_selectors)
};

// Selectors of the stable partition of 8 bytes by an 8-bit mask m (bit j set:
// byte j is a one): the bytes whose bit is clear, in order, then those whose
// bit is set, in order.  Entry m holds two byte-permute selectors (output
// bytes 0-3 in its low half, 4-7 in its high half), each a nibble per output
// byte naming the source byte 0..7 of the pair (low word, high word).
// Filled by threads 0..THREADS-1.
template <int THREADS>
__device__ __forceinline__ void partition_selectors(uint32_t *perm) {
  for (uint32_t m = threadIdx.x; m < 256; m += THREADS) {
    uint32_t sel = 0, o = 0;
    for (uint32_t side = 0; side < 2; ++side)
      for (uint32_t j = 0; j < 8; ++j)
        if (((m >> j) & 1u) == side) sel |= j << (4 * o++);
    perm[m] = sel;
  }
}

// Per-thread results of pass A that the rest of the tile uses.
template <int WPT>
struct SplitPassA {
  uint32_t word[WPT];  // the thread's bitmap words
  uint32_t pw[WPT];    // ones before each word, within the warp
  uint32_t incl;       // ones through the thread's words, within the warp
};

// Pass A of a split tile: 32 * WPT consecutive symbols per thread -> WPT
// bitmap words; warp scan of the ones; the thread's words and prefixes to
// sWP, the warp's {ones, prefix share} to sWT.  The block barrier that makes
// sWT complete is the caller's.
template <int SB, int THREADS, int WPT>
__device__ __forceinline__ SplitPassA<WPT> split_pass_a(const SplitArgs &a, const uint8_t *sIn, uint32_t nv,
                                                        uint32_t share_part, uint2 *sWP, uint2 *sWT) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t k = a.L - 1 - a.level;
  const uint32_t my0 = 32 * WPT * tid;
  SplitPassA<WPT> r;
  uint32_t pc = 0;
  if constexpr (SB == 1) {
    tile_words_1b<WPT>(sIn, my0, k, r.word);
#pragma unroll
    for (int i = 0; i < WPT; ++i) {
      r.word[i] &= valid_mask(my0 + 32 * i, nv);
      pc += __popc(r.word[i]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < WPT; ++i) {
      r.word[i] = tile_word<SB, THREADS>(sIn, my0 + 32 * i, k) & valid_mask(my0 + 32 * i, nv);
      pc += __popc(r.word[i]);
    }
  }
  uint32_t incl = pc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  r.incl = incl;
  r.pw[0] = incl - pc;
#pragma unroll
  for (int i = 1; i < WPT; ++i) r.pw[i] = r.pw[i - 1] + __popc(r.word[i - 1]);
#pragma unroll
  for (int i = 0; i < WPT; ++i) sWP[WPT * tid + i] = make_uint2(r.word[i], r.pw[i]);
  const uint32_t share = __reduce_add_sync(0xFFFFFFFFu, share_part);
  if (lane == 31) sWT[warp] = make_uint2(incl, share);
  return r;
}

// The run counters of a finished single-node tile (node pf; 0xFFFFFFFF for
// a tile over several nodes, whose counts went to global memory directly):
// counters 0/1 belong to the zero run, 2/3 to the one run; threads 0..3 add
// them to the next level's tile counts and clear them.  With node counts,
// thread 0 also accumulates the node's ones (the zero run lies in child 2pf,
// the one run in child 2pf+1; a node spans many tiles at shallow levels, so
// the counts of the current node are kept in shared memory and flushed when
// the node changes).
template <bool NC>
__device__ __forceinline__ void split_flush_runs(const SplitArgs &a, uint32_t *cnt, const uint32_t *run,
                                                 uint32_t *nc, uint32_t pf) {
  const uint32_t tid = threadIdx.x;
  if (tid < 4 && pf != 0xFFFFFFFFu) {
    const uint32_t v = cnt[tid];
    if (NC && a.nones_next) {
      const uint32_t pair = v + __shfl_down_sync(0xFu, v, 1);
      const uint32_t p1 = __shfl_sync(0xFu, pair, 2);
      if (tid == 0) {
        if (nc[0] == pf) {
          nc[1] += pair;
          nc[2] += p1;
        } else {
          if (nc[0] != 0xFFFFFFFFu) {
            if (nc[1]) atomicAdd(&a.nones_next[2 * nc[0]], nc[1]);
            if (nc[2]) atomicAdd(&a.nones_next[2 * nc[0] + 1], nc[2]);
          }
          nc[0] = pf;
          nc[1] = pair;
          nc[2] = p1;
        }
      }
    }
    if (v) {
      cnt[tid] = 0;
      const uint32_t dt = (run[tid >> 1] >> a.log2T) + (tid & 1);
      if (dt < a.NT) counts_add(a.cout, dt, v);
    }
  }
}

// The rest of a split tile after pass A and the block barrier behind it:
// bits and directory of the level, stable split into T_{level+1}, next-level
// ones per destination tile.  sIn holds the tile's symbols; pa is this
// thread's pass-A result; sm.wt holds every warp's {ones, prefix share}.  A
// single-node tile leaves its run counts in sm.cnt / sm.run for
// split_flush_runs; the node of such a tile is returned (0xFFFFFFFF for a
// tile over several nodes).  WPT: words (of 32 symbols) per thread; a warp's
// segment is 1024 * WPT symbols (WPT > 1 only for 1-byte symbols).
template <int SB, int THREADS, bool NC, int WPT = 1>
__device__ __forceinline__ uint32_t split_tile_rest(const SplitArgs &a, const uint2 *tab, uint32_t tile,
                                                    const uint8_t *sIn, const SplitPassA<WPT> &pa,
                                                    const SplitShared &sm) {
  static_assert(WPT == 1 || SB == 1, "several words per thread only for 1-byte symbols");
  using Sym = typename SymT<SB>::type;
  constexpr uint32_t T = 32 * WPT * THREADS;
  constexpr uint32_t SPW = 1024 * WPT;  // symbols per warp
  constexpr uint32_t NW = THREADS / 32;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t k1 = a.L - 2 - a.level;  // bit of the next level (this level reads bit k1 + 1)
  const uint32_t pshift = a.pshift;       // node prefix = symbol >> pshift
  const uint32_t lmask = (1u << a.L) - 1u;
  uint8_t *const stage = sm.stage + warp * stage_bytes<SB, WPT>();
  Sym *const stageS = reinterpret_cast<Sym *>(stage);
  uint2 *const sWP = sm.wp;
  uint2 *const sWT = sm.wt;
  uint32_t *const sCnt = sm.cnt;
  uint32_t *const sRun = sm.run;
  const uint64_t start = (uint64_t)tile * T;
  const uint32_t nv = (uint32_t)umin64(T, a.n - start);
  const uint32_t my0 = 32 * WPT * tid;
  const uint32_t incl = pa.incl;

    const uint2 wv = lane < NW ? sWT[lane] : make_uint2(0, 0);
    const uint32_t Pw = __reduce_add_sync(0xFFFFFFFFu, lane < warp ? wv.x : 0u);  // ones before the warp
    const uint32_t total = __reduce_add_sync(0xFFFFFFFFu, wv.x);
    const uint32_t R = __reduce_add_sync(0xFFFFFFFFu, wv.y);                       // ones before the tile
    if (WPT == 1) {
      write_level<THREADS>(a.lo, tile, a.NT, start, my0, a.n, a.NB, a.W, pa.word[0], R, Pw + pa.pw[0], total);
    } else {
#pragma unroll
      for (int i = 0; i < WPT; ++i) {
        const uint64_t widx = (uint64_t)tile * (WPT * THREADS) + WPT * tid + i;
        if (widx < a.W) a.lo.bits[widx] = pa.word[i];
        if ((widx & 15) == 0 && start + my0 + 32 * i < a.n) a.lo.rank[(start + my0 + 32 * i) >> 9] = R + Pw + pa.pw[i];
      }
      if (tile == a.NT - 1 && tid == 0) {
        a.lo.rank[a.NB] = R + total;
        *a.lo.zeros = (unsigned long long)(a.n - (R + total));
      }
    }

    // Pass B: stable split of the warp's segment into its staging area,
    // zeros first.  In step s lane i holds the G symbols at 32*G*s + G*i
    // (one 64-bit shared load); their bits come from the bitmap word, the
    // ones before them from the word prefix plus a popcount.  In a tile that
    // lies in one node, each run is staged at the 16-byte phase of its
    // destination in T_{l+1}, so that it is written with aligned 16-byte
    // copies.
    const uint32_t seg = SPW * warp;
    const uint32_t nvw = nv > seg ? min(nv - seg, SPW) : 0u;    // symbols of this warp
    const uint32_t tw = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint32_t nzw = nvw - tw;                              // zeros of this warp
    const Sym *sInS = reinterpret_cast<const Sym *>(sIn);
    const uint32_t pf = ((uint32_t)sInS[0] & lmask) >> pshift;
    const uint32_t pl = ((uint32_t)sInS[nv - 1] & lmask) >> pshift;
    const uint32_t Zb = (uint32_t)start - R;  // zeros of level l before the tile
    const uint32_t Zw = Zb + seg - Pw;        // zeros of level l before the warp
    const uint32_t Ow = R + Pw;               // ones of level l before the warp
    const bool one_node = pf == pl;
    // nodes of the warp's first and last symbol (its segment is in node order)
    uint32_t wpf = pf, wpl = pf;
    if (!one_node && nvw) {
      wpf = ((uint32_t)sInS[seg] & lmask) >> pshift;
      wpl = ((uint32_t)sInS[seg + nvw - 1] & lmask) >> pshift;
    }
    const bool warp_one = one_node || wpf == wpl;  // the warp's symbols lie in one node
    uint32_t gz = 0, go = 0, zoff = 0, ooff = nzw * SB;  // destinations, staging offsets (bytes)
    if (warp_one && nvw) {
      const uint2 tb = tab[wpf];
      gz = tb.x + Zw;
      go = tb.y + Ow;
      zoff = (gz * SB) & 15u;
      ooff = ((zoff + nzw * SB + 15u) & ~15u) + ((go * SB) & 15u);
    }
    if (nvw) {
      constexpr uint32_t G8 = 8 / SB;     // symbols per lane per step
      constexpr uint32_t LPW8 = 32 / G8;  // lanes per bitmap word
      const uint32_t wsub = lane / LPW8;
      const uint32_t bo = (lane % LPW8) * G8;
      const uint32_t lowmask = (1u << bo) - 1u;
      const uint8_t *segIn = sIn + seg * SB;
      Sym *const zS = reinterpret_cast<Sym *>(stage + zoff);
      Sym *const oS = reinterpret_cast<Sym *>(stage + ooff);
      if (SB == 1 && sm.perm && nvw == SPW) {
        // 1-byte symbols: the lane partitions its 8 symbols in registers
        // (two byte permutes, selectors by the 8-bit pattern), so that its
        // zeros are bytes 0..nz-1 and its ones bytes nz..7, then stores
        // byte i at the zero pointer + i or the one pointer + i - nz: one
        // select and one store per symbol, no pointer updates.
        const uint32_t zbase = smem_addr(zS), obase = smem_addr(oS);
        const uint32_t mbyte = 0x4440u | (lane & 3u);  // byte-permute selector of byte lane % 4
#pragma unroll
        for (uint32_t s = 0; s < 32 * WPT / 8; ++s) {
          const uint32_t pos0 = 256 * s + 8 * lane;
          const uint2 wp = sWP[32 * WPT * warp + 8 * s + wsub];
          const uint2 grp = *reinterpret_cast<const uint2 *>(segIn + pos0);
          const uint32_t m = __byte_perm(wp.x, 0u, mbyte);    // the bits of the lane's 8 symbols
          const uint32_t sel = sm.perm[m];
          const uint32_t lo = __byte_perm(grp.x, grp.y, sel & 0xFFFFu);
          const uint32_t hi = __byte_perm(grp.x, grp.y, sel >> 16);
          const uint32_t nz = 8u - __popc(m);
          const uint32_t zm = (1u << nz) - 1u;                 // bit i set: byte i is a zero
          const uint32_t Rl = wp.y + __popc(wp.x & lowmask);  // ones before pos0 in the warp
          const uint32_t za = zbase + (pos0 - Rl);             // byte i < nz goes to za + i
          const uint32_t ob = obase + Rl - nz;                 // byte i >= nz goes to ob + i
#pragma unroll
          for (uint32_t i = 0; i < 8; ++i) {
            const uint32_t v = (i < 4 ? lo : hi) >> (8 * (i & 3));
            const uint32_t addr = ((zm & (1u << i)) ? za : ob) + i;
            asm volatile("st.shared.u8 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
          }
        }
      } else if (nvw == SPW) {
        // Each symbol goes to the running zero or one pointer of its lane:
        // one predicate, two predicated stores, two predicated increments --
        // no branch, whatever the bits.
        const uint32_t zbase = smem_addr(zS), obase = smem_addr(oS);
#pragma unroll
        for (uint32_t s = 0; s < 32 * WPT / G8; ++s) {
          const uint32_t pos0 = 32 * G8 * s + G8 * lane;
          const uint2 wp = sWP[32 * WPT * warp + G8 * s + wsub];
          const uint2 grp = *reinterpret_cast<const uint2 *>(segIn + pos0 * SB);
          const uint32_t bits = wp.x >> bo;
          const uint32_t Rl = wp.y + __popc(wp.x & lowmask);  // ones before pos0 in the warp
          uint32_t oa = obase + Rl * SB, za = zbase + (pos0 - Rl) * SB;
#pragma unroll
          for (uint32_t j = 0; j < G8; ++j) {
            const uint32_t w = j < G8 / 2 ? grp.x : grp.y;
            const uint32_t v = w >> (8 * SB * (j % (G8 / 2)));
            scatter_one<SB>(bits & (1u << j), oa, za, v);
          }
        }
      } else {
        for (uint32_t s = 0; s < 32 * WPT / G8; ++s) {
          const uint32_t pos0 = 32 * G8 * s + G8 * lane;
          const uint2 wp = sWP[32 * WPT * warp + G8 * s + wsub];
          const uint2 grp = *reinterpret_cast<const uint2 *>(segIn + pos0 * SB);
          const uint32_t bits = wp.x >> bo;
          const uint32_t Rl = wp.y + __popc(wp.x & lowmask);
          uint32_t o = Rl, z = pos0 - Rl;
          for (uint32_t j = 0; j < G8; ++j) {
            if (pos0 + j < nvw) {
              const uint32_t w = j < G8 / 2 ? grp.x : grp.y;
              const Sym v = (Sym)(w >> (8 * SB * (j % (G8 / 2))));
              const uint32_t b = (bits >> j) & 1u;
              Sym *const dst = b ? oS + o : zS + z;
              *dst = v;
              o += b;
              z += b ^ 1u;
            }
          }
        }
      }
      __syncwarp();

      // Phase 2: the warp writes its zeros and ones to T_{l+1}, counting the
      // next level's ones per destination tile.
      const uint32_t mk1 = (SB == 1 ? 0x01010101u : SB == 2 ? 0x00010001u : 1u) << k1;
      const uint64_t gend = (uint64_t)a.n * SB;
      if (one_node) {
        // the whole tile lies in one node: its zeros and ones are two runs,
        // counted per destination tile for the whole CTA
        const uint2 tb = tab[pf];
        const uint32_t r0 = tb.x + Zb, r1 = tb.y + R;  // where the tile's runs start
        const uint32_t s0 = ((r0 >> a.log2T) + 1) << a.log2T, s1 = ((r1 >> a.log2T) + 1) << a.log2T;
        uint32_t c0a = 0, c0b = 0, c1a = 0, c1b = 0;
        if constexpr (SB == 1 && WPT == 2) {
          warp_copy_runs2<SB, 2 * WPT * SB>(stage, a.out, gend, mk1, k1, zoff, (uint64_t)gz * SB, nzw * SB, s0,
                                            ooff, (uint64_t)go * SB, tw * SB, s1, c0a, c0b, c1a, c1b);
        } else {
          warp_copy_run<SB>(stage, zoff, a.out, (uint64_t)gz * SB, nzw * SB, gend, s0, mk1, k1, c0a, c0b);
          warp_copy_run<SB>(stage, ooff, a.out, (uint64_t)go * SB, tw * SB, gend, s1, mk1, k1, c1a, c1b);
        }
        const uint32_t v0 = __reduce_add_sync(0xFFFFFFFFu, c0a);
        const uint32_t v1 = __reduce_add_sync(0xFFFFFFFFu, c0b);
        const uint32_t v2 = __reduce_add_sync(0xFFFFFFFFu, c1a);
        const uint32_t v3 = __reduce_add_sync(0xFFFFFFFFu, c1b);
        if (lane == 0) {
          if (v0) atomicAdd(&sCnt[0], v0);
          if (v1) atomicAdd(&sCnt[1], v1);
          if (v2) atomicAdd(&sCnt[2], v2);
          if (v3) atomicAdd(&sCnt[3], v3);
          if (warp == 0) {
            sRun[0] = r0;
            sRun[1] = r1;
          }
        }
      } else if (warp_one) {
        // the warp's symbols lie in one node (the tile does not): two runs
        // of at most 1024 symbols, each crossing at most one tile boundary
        // of T_{l+1}; counted per warp
        const uint32_t t0 = gz >> a.log2T, t1 = go >> a.log2T;
        uint32_t c0a = 0, c0b = 0, c1a = 0, c1b = 0;
        if constexpr (SB == 1 && WPT == 2) {
          warp_copy_runs2<SB, 2 * WPT * SB>(stage, a.out, gend, mk1, k1, zoff, (uint64_t)gz * SB, nzw * SB,
                                            (t0 + 1) << a.log2T, ooff, (uint64_t)go * SB, tw * SB,
                                            (t1 + 1) << a.log2T, c0a, c0b, c1a, c1b);
        } else {
          warp_copy_run<SB>(stage, zoff, a.out, (uint64_t)gz * SB, nzw * SB, gend, (t0 + 1) << a.log2T, mk1,
                            k1, c0a, c0b);
          warp_copy_run<SB>(stage, ooff, a.out, (uint64_t)go * SB, tw * SB, gend, (t1 + 1) << a.log2T, mk1,
                            k1, c1a, c1b);
        }
        const uint32_t v0 = __reduce_add_sync(0xFFFFFFFFu, c0a);
        const uint32_t v1 = __reduce_add_sync(0xFFFFFFFFu, c0b);
        const uint32_t v2 = __reduce_add_sync(0xFFFFFFFFu, c1a);
        const uint32_t v3 = __reduce_add_sync(0xFFFFFFFFu, c1b);
        if (lane == 0) {
          if (v0 && t0 < a.NT) counts_add(a.cout, t0, v0);
          if (v1 && t0 + 1 < a.NT) counts_add(a.cout, t0 + 1, v1);
          if (v2 && t1 < a.NT) counts_add(a.cout, t1, v2);
          if (v3 && t1 + 1 < a.NT) counts_add(a.cout, t1 + 1, v3);
          if (NC && a.nones_next) {
            if (v0 + v1) atomicAdd(&a.nones_next[2 * wpf], v0 + v1);
            if (v2 + v3) atomicAdd(&a.nones_next[2 * wpf + 1], v2 + v3);
          }
        }
      } else {
        split_multi_node<SB, NC>(a.out, a.n, a.log2T, a.NT, a.cout, a.nones_next, tab, sInS, stageS,
                                 sWP + 32 * WPT * warp, seg, nvw, nzw, wpf, wpl, Zw, Ow, lmask, pshift, k1);
      }
    }
    return one_node ? pf : 0xFFFFFFFFu;
}

// One whole tile of the split pass (pass A, block barrier, the rest, block
// barrier, run counts): for callers that process one tile at a time.  Ends
// with thread 0 having stored ring_value to *ring_slot (if non-null).
template <int SB, int THREADS, bool NC, int WPT = 1>
__device__ __forceinline__ void split_tile(const SplitArgs &a, const uint2 *tab, uint32_t tile,
                                           const uint8_t *sIn, uint32_t share_part,
                                           const SplitShared &sm, uint32_t *ring_slot,
                                           uint32_t ring_value) {
  constexpr uint32_t T = 32 * WPT * THREADS;
  const uint32_t nv = (uint32_t)umin64(T, a.n - (uint64_t)tile * T);
  const SplitPassA<WPT> pa = split_pass_a<SB, THREADS, WPT>(a, sIn, nv, share_part, sm.wp, sm.wt);
  cta_sync<THREADS>();
  const uint32_t pf = split_tile_rest<SB, THREADS, NC, WPT>(a, tab, tile, sIn, pa, sm);
  if (ring_slot) *ring_slot = ring_value;
  cta_sync<THREADS>();
  split_flush_runs<NC>(a, sm.cnt, sm.run, sm.nc, pf);
}

// Resident CTAs per SM the split pass is compiled for: as many as shared
// memory allows, up to 48 warps per SM, but not so many that a thread gets
// fewer than 48 registers (below that the pass spills) -- except with
// 512-thread CTAs, where 3 per SM at 40 registers beat 2 at 64.
template <int SB, int THREADS, int DEPTH = 2, int WPT = 1>
constexpr int split_min_blocks() {
  constexpr uint32_t by_smem = 232448u / split_smem_bytes<SB, THREADS, DEPTH, WPT>();
  constexpr uint32_t by_warps = 1536u / THREADS;
  constexpr uint32_t by_regs = THREADS >= 512 ? by_warps : 65536u / (48u * THREADS);
  constexpr uint32_t m = by_smem < by_warps ? by_smem : by_warps;
  constexpr uint32_t r = m < by_regs ? m : by_regs;
  return (int)(r ? r : 1u);
}

// The level's node table from per-node counts, by one CTA of THREADS
// threads, node q by thread q (2^level <= THREADS), into sTab; CTA 0 also
// stores it and the odd nodes' starts (see SplitArgs::node_ones).  With s(q)
// = start of node q and c(q) its ones: O(q) = sum of c over nodes < q, and
// tab[q] = {O(q), s(q+1) - c(q) - O(q)}; an odd node starts where its
// parent's 1-child does, an even node where its parent does (written at an
// earlier level).  s_warp: 33 words of scratch.  Ends with threads of the
// CTA still to be synchronised before sTab is read.
template <int THREADS>
__device__ __forceinline__ void split_node_table(const SplitArgs &a, uint2 *sTab, uint32_t *s_warp) {
  const uint32_t q = threadIdx.x, cnt = 1u << a.level, sh = a.L - a.level;
  auto start_of = [&](uint32_t v) -> uint32_t {
    if (v >= cnt) return a.n;
    if (v & 1u) {
      const uint2 t = a.tab_prev[v >> 1];
      return t.x + t.y;
    }
    return (uint32_t)a.E[(uint64_t)v << sh];
  };
  const uint32_t c = q < cnt ? __ldcg(&a.node_ones[q]) : 0u;
  uint32_t total;
  const uint32_t O = block_exclusive_scan<THREADS>(c, s_warp, &total);
  if (q < cnt) {
    const uint2 tb = make_uint2(O, start_of(q + 1) - c - O);
    sTab[q] = tb;
    if (blockIdx.x == 0) {
      a.tab_w[q] = tb;
      if (q & 1u) a.E[(uint64_t)q << sh] = start_of(q);
    }
  }
  if (a.level == 1 && blockIdx.x == 0 && q == 0) {
    a.E[0] = 0;
    a.E[1ull << a.L] = a.n;
  }
}

// NC: the tree's node sizes come from node counts (a.nones_next set): the
// pass also counts the next level's ones per child node.  Compiled as a
// separate kernel so that the other builds carry none of that code.
template <int SB, int THREADS, bool NC, int DEPTH, int WPT = 1>
__global__ void __launch_bounds__(THREADS, split_min_blocks<SB, THREADS, DEPTH, WPT>()) k_split(SplitArgs a) {
  constexpr uint32_t T = 32 * WPT * THREADS;
  constexpr uint32_t NW = THREADS / 32;
  extern __shared__ __align__(128) uint8_t smem[];
  TilePipe<SB, THREADS, DEPTH, WPT> pipe;
  pipe.sIn0 = smem;
  pipe.sIn1 = smem + (DEPTH - 1) * pipe.TB;
  uint8_t *const sStage = smem + DEPTH * pipe.TB;
  uint2 *const sWP = reinterpret_cast<uint2 *>(sStage + NW * stage_bytes<SB, WPT>());  // {word, prefix}
  uint2 *const sWT = sWP + WPT * THREADS;            // per warp {ones, prefix share}, 2 sets
  uint2 *const sTab = sWT + 2 * NW;                  // level table (small levels)
  pipe.bar = reinterpret_cast<uint64_t *>(sTab + tab_smem_nodes<SB>());
  pipe.ring = reinterpret_cast<uint32_t *>(pipe.bar + 2);
  uint32_t *const sCnt = pipe.ring + 4;              // 2 x 4 run counters
  uint32_t *const sRun = sCnt + 8;                   // 2 x 2 run starts
  uint32_t *const sNc = sRun + 4;                    // node-count cache (3 words)
  uint32_t *const sPerm = sNc + 16;                  // 1-byte symbols: partition selectors
  pipe.in = a.in;
  pipe.in_padded = a.in_padded;
  pipe.n = a.n;
  pipe.NT = a.NT;
  pipe.ticket = a.ticket;

  const uint32_t tid = threadIdx.x;
  const uint32_t nodes = 1u << (a.L - a.pshift);
  const bool tab_smem = nodes <= tab_smem_nodes<SB>();
  const uint2 *const tab = tab_smem ? sTab : a.tab;

  if (a.count_table) {
    // One node (the wavelet matrix of Section 7, or level 0): its ones go
    // after all zeros of the level, which are n minus the level's ones,
    // summed from the top tier of the level's tile counts.
    if (tid < 32) {
      const uint32_t ones = counts_total_warp(a.cin, a.NT);
      if (tid == 0) {
        sTab[0] = make_uint2(0u, a.n - ones);
        if (a.tab_out && blockIdx.x == 0) a.tab_out[0] = sTab[0];
      }
    }
  } else if (a.node_ones) {
    split_node_table<THREADS>(a, sTab, reinterpret_cast<uint32_t *>(sStage));
  } else if (tab_smem) {
    for (uint32_t i = tid; i < nodes; i += THREADS) sTab[i] = __ldg(&a.tab[i]);
  }
  if (tid < 8) sCnt[tid] = 0;
  if (SB == 1) partition_selectors<THREADS>(sPerm);
  if (tid == 0) {
    sNc[0] = 0xFFFFFFFFu;
    pipe.prologue();
  }
  __syncthreads();
  PrefixLoads pre = prefix_loads<THREADS>(a.cin, pipe.ring[0], a.NT);

  if constexpr (DEPTH == 2) {
    // One block barrier per tile: the one that completes pass A.  What
    // warps share across that barrier is kept per tile parity (the warps'
    // pass-A sums, the run counters of single-node tiles), so that a warp
    // may finish tile it while another has begun tile it+1; no warp gets
    // further ahead, since the barrier of tile it+1 waits for all.  Behind
    // that barrier every warp is done with tile it-1, so thread 0 then
    // starts the copy of tile it+1 into that tile's buffer, and threads 0..3
    // add the run counts of tile it-1 to the next level's tile counts.
    uint32_t prev_pf = 0xFFFFFFFFu;  // node of the previous tile if it lay in one node
    uint32_t it = 0;
    for (;; ++it) {
      const uint32_t tile = pipe.ring[it % 3];
      if (tile >= a.NT) break;
      const uint32_t nxt = pipe.ring[(it + 1) % 3];
      uint32_t nn = 0;
      if (tid == 0) nn = atomicAdd(a.ticket, 1u);  // the ticket of tile it+2
      const PrefixLoads pre_next = prefix_loads<THREADS>(a.cin, nxt, a.NT);
      const bool ok = pipe.wait(it, a.spin_limit, a.err);
      const uint64_t start = (uint64_t)tile * T;
      const uint32_t nv = (uint32_t)umin64(T, a.n - start);
      uint8_t *const sIn = pipe.data(it);
      if (pipe.fill_tail(sIn, start, nv)) __syncthreads();
      const uint32_t par = it & 1u;
      const SplitShared sm{sStage, sWP, sWT + par * NW, sCnt + 4 * par, sRun + 2 * par, sNc,
                           SB == 1 ? sPerm : nullptr};
      const SplitPassA<WPT> pa = split_pass_a<SB, THREADS, WPT>(a, sIn, nv, pre.sum(), sWP, sm.wt);
      if (tid == 0) pipe.ring[(it + 2) % 3] = nn;
      if (__syncthreads_or(!ok)) {
        // the tile's copy did not land in time: wait once more (bounded)
        // for it, the only copy in flight, and stop
        if (tid == 0) mbar_wait_bounded(&pipe.bar[it & 1], (it >> 1) & 1u, a.spin_limit, a.err);
        __syncthreads();
        break;
      }
      if (tid == 0 && nxt < a.NT) {
        fence_proxy_async_smem();
        pipe.issue(nxt, (it + 1) & 1);
      }
      split_flush_runs<NC>(a, sCnt + 4 * (par ^ 1u), sRun + 2 * (par ^ 1u), sNc, prev_pf);
      prev_pf = split_tile_rest<SB, THREADS, NC, WPT>(a, tab, tile, sIn, pa, sm);
      pre = pre_next;
    }
    __syncthreads();
    const uint32_t lp = (it & 1u) ^ 1u;  // parity of the last tile processed
    split_flush_runs<NC>(a, sCnt + 4 * lp, sRun + 2 * lp, sNc, prev_pf);
  } else {
    for (uint32_t it = 0;; ++it) {
      const uint32_t tile = pipe.ring[it % 3];
      if (tile >= a.NT) break;
      const uint32_t nxt = pipe.ring[(it + 1) % 3];
      uint32_t nn = 0;
      if (tid == 0) nn = pipe.advance(it, nxt);
      const PrefixLoads pre_next = prefix_loads<THREADS>(a.cin, nxt, a.NT);
      const bool ok = pipe.wait(it, a.spin_limit, a.err);
      if (__syncthreads_or(!ok)) {
        pipe.drain(it, a.spin_limit, a.err);
        __syncthreads();
        break;
      }
      const uint64_t start = (uint64_t)tile * T;
      const uint32_t nv = (uint32_t)umin64(T, a.n - start);
      uint8_t *const sIn = pipe.data(it);
      if (pipe.fill_tail(sIn, start, nv)) __syncthreads();

      const SplitShared sm{sStage, sWP, sWT, sCnt, sRun, sNc, SB == 1 ? sPerm : nullptr};
      split_tile<SB, THREADS, NC, WPT>(a, tab, tile, sIn, pre.sum(), sm,
                                       tid == 0 ? &pipe.ring[(it + 2) % 3] : nullptr, nn);
      if (tid == 0) pipe.after_tile(nxt);
      pre = pre_next;
    }
  }
  if (NC && a.nones_next && tid == 0 && sNc[0] != 0xFFFFFFFFu) {  // the cached node's counts
    if (sNc[1]) atomicAdd(&a.nones_next[2 * sNc[0]], sNc[1]);
    if (sNc[2]) atomicAdd(&a.nones_next[2 * sNc[0] + 1], sNc[2]);
  }
}

// ------------------------------------------------------------------ last two levels in one pass
// Copy bits [src, src+len) of the tile bitmap w (w[0] and w[NWD+1] are zero
// pads, bit x at w[1 + x/32]) to bits [g, g+len) of `row`, by one warp.
// Words the run covers entirely are stored; the two end words are shared
// with other runs and are or-ed in (the row was zeroed before the pass).
__device__ __forceinline__ void warp_bit_run(const uint32_t *w, uint32_t src, uint32_t *row, uint64_t g,
                                             uint32_t len) {
  if (!len) return;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t w0 = g >> 5, w1 = (g + len - 1) >> 5;
  for (uint64_t ow = w0 + lane; ow <= w1; ow += 32) {
    const long long sp = (long long)src + (long long)(32 * ow) - (long long)g;  // >= src - 31
    const long long wi = sp >> 5;                                               // >= -1
    const uint32_t lo = w[1 + wi], hi = w[2 + wi];
    uint32_t val = __funnelshift_r(lo, hi, (uint32_t)(sp & 31));
    const uint64_t base = 32 * ow;
    const uint32_t qlo = g > base ? (uint32_t)(g - base) : 0u;
    const uint32_t qhi = (uint32_t)umin64(32, g + len - base);
    const uint32_t mask = (qhi == 32 ? ~0u : ((1u << qhi) - 1u)) & ~((1u << qlo) - 1u);
    val &= mask;
    if (mask == ~0u) row[ow] = val;
    else if (val) atomicOr(&row[ow], val);
  }
}

// The last two levels in one pass over T_{L-2} (no T_{L-1} is written).
// Level L-2's bits and directory are written as by the split pass.  Each
// symbol's bit of level L-1 belongs at the position the split would move
// the symbol to: within a warp lying in one node, the level-(L-1) bits of
// its zeros, in order, form one run that starts where its zeros would go,
// and those of its ones another.  So a thread compacts its words' level-
// (L-1) bits into those of its zeros and those of its ones (8 at a time, by
// the byte permutes of the split's stable partition), the warp assembles the two
// bit streams in shared memory, and writes them as bit runs (the row is
// zeroed before the pass; each run's end words are or-ed in).  A warp
// spanning several nodes writes each of its level-(L-1) one bits at its
// own position.  The directory of level L-1 is a separate pass.
struct LastPairArgs {
  SplitArgs s;          // as for the split pass over level L-2 (out, cout unused)
  uint32_t *row_next;   // bitmap row of level L-1 (zeroed)
};

template <int SB, int WPT>
__host__ __device__ constexpr uint32_t lastpair_stage_words() { return 2u * (32u * WPT + 2u); }

// Node counts of level L-1 are kept per block in shared memory for up to
// this many nodes of level L-2 (two counters each), and flushed once.
constexpr uint32_t kLastPairSmemNodes = 1024;

template <int SB, int THREADS, int WPT = 1>
constexpr uint32_t lastpair_smem_bytes() {
  // two input tiles, per warp two bit streams (with a zero pad word at each
  // end), per-word {bit word, prefix}, two sets of per-warp {ones, share},
  // the level table, the partition selectors, node counters, mbarriers and
  // tickets
  return 2u * 32u * WPT * THREADS * SB + (THREADS / 32) * lastpair_stage_words<SB, WPT>() * 4u +
         8u * WPT * THREADS + 16u * (THREADS / 32) + 8u * tab_smem_nodes<SB>() + 1024u +
         8u * kLastPairSmemNodes + 128u;
}

template <int SB, int THREADS, int WPT = 1>
constexpr int lastpair_min_blocks() {
  constexpr uint32_t by_smem = 232448u / (lastpair_smem_bytes<SB, THREADS, WPT>() + 1024u);
  constexpr uint32_t by_warps = 2048u / THREADS;
  constexpr uint32_t r = by_smem < by_warps ? by_smem : by_warps;
  return (int)(r > 5 ? 5 : (r ? r : 1u));
}

template <int SB, int THREADS, bool NC, int WPT = 1>
__global__ void __launch_bounds__(THREADS, lastpair_min_blocks<SB, THREADS, WPT>()) k_lastpair(LastPairArgs la) {
  using Sym = typename SymT<SB>::type;
  constexpr uint32_t T = 32 * WPT * THREADS;
  constexpr uint32_t NW = THREADS / 32;
  constexpr uint32_t SPW = 1024 * WPT;          // symbols per warp
  constexpr uint32_t SW = 32 * WPT + 2;         // words of one bit stream, with two pads
  const SplitArgs &a = la.s;
  extern __shared__ __align__(128) uint8_t smem[];
  TilePipe<SB, THREADS, 2, WPT> pipe;
  pipe.sIn0 = smem;
  pipe.sIn1 = smem + pipe.TB;
  uint32_t *const sStream = reinterpret_cast<uint32_t *>(smem + 2 * pipe.TB);  // per warp: zeros' bits, ones' bits
  uint2 *const sWP = reinterpret_cast<uint2 *>(sStream + NW * 2 * SW);
  uint2 *const sWT = sWP + WPT * THREADS;         // 2 sets
  uint2 *const sTab = sWT + 2 * NW;
  uint32_t *const sPerm = reinterpret_cast<uint32_t *>(sTab + tab_smem_nodes<SB>());  // partition selectors
  uint32_t *const sNC = sPerm + 256;  // ones of child 2p + bit at [2p + bit]
  pipe.bar = reinterpret_cast<uint64_t *>(sNC + 2 * kLastPairSmemNodes);
  pipe.ring = reinterpret_cast<uint32_t *>(pipe.bar + 2);
  pipe.in = a.in;
  pipe.in_padded = a.in_padded;
  pipe.n = a.n;
  pipe.NT = a.NT;
  pipe.ticket = a.ticket;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t nodes = 1u << (a.L - a.pshift);
  const bool tab_smem = nodes <= tab_smem_nodes<SB>();
  const uint2 *const tab = tab_smem ? sTab : a.tab;
  const uint32_t k = a.L - 1 - a.level, k1 = k - 1;
  const uint32_t lmask = (1u << a.L) - 1u;

  partition_selectors<THREADS>(sPerm);
  if (a.count_table) {
    if (tid < 32) {
      const uint32_t ones = counts_total_warp(a.cin, a.NT);
      if (tid == 0) {
        sTab[0] = make_uint2(0u, a.n - ones);
        if (a.tab_out && blockIdx.x == 0) a.tab_out[0] = sTab[0];
      }
    }
  } else if (a.node_ones) {
    // scratch: the pass-A words, unused before the barrier below (the
    // stream areas are cleared before it)
    split_node_table<THREADS>(a, sTab, reinterpret_cast<uint32_t *>(sWP));
  } else if (tab_smem) {
    for (uint32_t i = tid; i < nodes; i += THREADS) sTab[i] = __ldg(&a.tab[i]);
  }
  // the next level's ones per child node: in shared memory when the level
  // has few nodes (then every warp of a node adds to the same counters)
  const bool nc_smem = NC && a.nones_next && nodes <= kLastPairSmemNodes;
  if (nc_smem)
    for (uint32_t i = tid; i < 2 * nodes; i += THREADS) sNC[i] = 0;
  auto nc_add = [&](uint32_t child, uint32_t c) {
    if (nc_smem) atomicAdd(&sNC[child], c);
    else atomicAdd(&a.nones_next[child], c);
  };
  uint32_t *const zs = sStream + warp * 2 * SW;  // this warp's zeros' bits: bit x at zs[1 + x / 32]
  uint32_t *const os = zs + SW;                  // its ones' bits
  for (uint32_t i = lane; i < 2 * SW; i += 32) zs[i] = 0;
  if (tid == 0) pipe.prologue();
  __syncthreads();
  PrefixLoads pre = prefix_loads<THREADS>(a.cin, pipe.ring[0], a.NT);

  for (uint32_t it = 0;; ++it) {
    const uint32_t tile = pipe.ring[it % 3];
    if (tile >= a.NT) break;
    const uint32_t nxt = pipe.ring[(it + 1) % 3];
    uint32_t nn = 0;
    if (tid == 0) nn = atomicAdd(a.ticket, 1u);  // the ticket of tile it+2
    const PrefixLoads pre_next = prefix_loads<THREADS>(a.cin, nxt, a.NT);
    const bool ok = pipe.wait(it, a.spin_limit, a.err);
    const uint64_t start = (uint64_t)tile * T;
    const uint32_t nv = (uint32_t)umin64(T, a.n - start);
    uint8_t *const sIn = pipe.data(it);
    if (pipe.fill_tail(sIn, start, nv)) __syncthreads();
    const uint32_t par = it & 1u;
    uint2 *const wt = sWT + par * NW;
    const SplitPassA<WPT> pa = split_pass_a<SB, THREADS, WPT>(a, sIn, nv, pre.sum(), sWP, wt);
    if (tid == 0) pipe.ring[(it + 2) % 3] = nn;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) mbar_wait_bounded(&pipe.bar[it & 1], (it >> 1) & 1u, a.spin_limit, a.err);
      __syncthreads();
      break;
    }
    if (tid == 0 && nxt < a.NT) {
      fence_proxy_async_smem();
      pipe.issue(nxt, (it + 1) & 1);
    }
    // level L-2: bits and directory, as in the split pass
    const uint2 wv = lane < NW ? wt[lane] : make_uint2(0, 0);
    const uint32_t Pw = __reduce_add_sync(0xFFFFFFFFu, lane < warp ? wv.x : 0u);  // ones before the warp
    const uint32_t total = __reduce_add_sync(0xFFFFFFFFu, wv.x);
    const uint32_t R = __reduce_add_sync(0xFFFFFFFFu, wv.y);                       // ones before the tile
    const uint32_t my0 = 32 * WPT * tid;
#pragma unroll
    for (int i = 0; i < WPT; ++i) {
      const uint64_t widx = (uint64_t)tile * (WPT * THREADS) + WPT * tid + i;
      if (widx < a.W) a.lo.bits[widx] = pa.word[i];
      if ((widx & 15) == 0 && start + my0 + 32 * i < a.n) a.lo.rank[(start + my0 + 32 * i) >> 9] = R + Pw + pa.pw[i];
    }
    if (tile == a.NT - 1 && tid == 0) {
      a.lo.rank[a.NB] = R + total;
      *a.lo.zeros = (unsigned long long)(a.n - (R + total));
    }
    // level L-1: this thread's bits split into those of its zeros and of its
    // ones, each in order, appended to the warp's two streams
    const uint32_t seg = SPW * warp;
    const uint32_t nvw = nv > seg ? min(nv - seg, SPW) : 0u;
    const uint32_t tw = __shfl_sync(0xFFFFFFFFu, pa.incl, 31);  // ones of the warp
    const uint32_t nzw = nvw - tw;
    {
      unsigned long long zacc = 0, oacc = 0;
      uint32_t zf = 0, of = 0;
      uint32_t w1s[WPT];  // the thread's level-(L-1) bit words
      if constexpr (SB == 1) {
        tile_words_1b<WPT>(sIn, my0, k1, w1s);
      } else {
#pragma unroll
        for (int i = 0; i < WPT; ++i) w1s[i] = tile_word<SB, THREADS>(sIn, my0 + 32 * i, k1);
      }
      // Per byte (8 symbols): spread the 8 level-(L-1) bits to one per byte
      // (a multiply and a mask per 4 bits), reorder those bytes with the
      // stable partition of the split (byte permutes, selectors by the 8
      // level-(L-2) bits), and gather them back: the zeros' bits, then the
      // ones', each in order.  Positions past n are neither (their level-
      // (L-2) bit is 0, so they sort after the valid zeros and are masked off).
#pragma unroll
      for (int i = 0; i < WPT; ++i) {
        const uint32_t vm = valid_mask(my0 + 32 * i, nv);
        const uint32_t w1 = w1s[i];
        const uint32_t w0 = pa.word[i];
        uint32_t z32 = 0, o32 = 0, zn = 0, on = 0;  // this word's zeros' and ones' bits
#pragma unroll
        for (uint32_t b = 0; b < 4; ++b) {
          const uint32_t m = (w0 >> (8 * b)) & 0xFFu, v = (w1 >> (8 * b)) & 0xFFu;
          const uint32_t sel = sPerm[m];
          const uint32_t slo = ((v & 15u) * 0x00204081u) & 0x01010101u;  // bit j to byte j
          const uint32_t shi = ((v >> 4) * 0x00204081u) & 0x01010101u;
          const uint32_t plo = __byte_perm(slo, shi, sel & 0xFFFFu), phi = __byte_perm(slo, shi, sel >> 16);
          const uint32_t P = ((plo * 0x10204080u) >> 28) | (((phi * 0x10204080u) >> 28) << 4);  // byte j to bit j
          const uint32_t c1 = __popc(m), nzv = __popc((vm >> (8 * b)) & 0xFFu) - c1;
          z32 |= (P & ((1u << nzv) - 1u)) << zn;
          o32 |= (P >> (8u - c1)) << on;
          zn += nzv;
          on += c1;
        }
        zacc |= (unsigned long long)z32 << zf;
        oacc |= (unsigned long long)o32 << of;
        zf += zn;
        of += on;
      }
      // zeros before this thread within the warp: its position in the warp
      // minus the ones before it
      const uint32_t zb = 32 * WPT * lane - pa.pw[0], ob = pa.pw[0];
      auto put = [&](uint32_t *s, uint32_t at, unsigned long long bits, uint32_t len) {
        if (!len) return;
        const uint32_t w = at >> 5, sh = at & 31u;
        const uint32_t lo = (uint32_t)bits, hi = (uint32_t)(bits >> 32);
        atomicOr(&s[1 + w], lo << sh);
        if (sh + len > 32) atomicOr(&s[2 + w], __funnelshift_l(lo, hi, sh));
        if (sh + len > 64) atomicOr(&s[3 + w], hi >> (32 - sh));
      };
      if (nvw) {
        put(zs, zb, zacc, zf);
        put(os, ob, oacc, of);
      }
    }
    __syncwarp();
    // the warp's node range (its segment is in node order)
    const Sym *sInS = reinterpret_cast<const Sym *>(sIn);
    const uint32_t Zw = (uint32_t)start - R + seg - Pw;  // zeros of level L-2 before the warp
    const uint32_t Ow = R + Pw;                          // ones of level L-2 before the warp
    if (nvw) {
      const uint32_t wpf = ((uint32_t)sInS[seg] & lmask) >> a.pshift;
      const uint32_t wpl = ((uint32_t)sInS[seg + nvw - 1] & lmask) >> a.pshift;
      if (wpf == wpl) {
        const uint2 tb = tab[wpf];
        const uint64_t gz = (uint64_t)tb.x + Zw, go = (uint64_t)tb.y + Ow;
        if (nzw && gz + nzw <= a.n) warp_bit_run(zs, 0, la.row_next, gz, nzw);
        if (tw && go + tw <= a.n) warp_bit_run(os, 0, la.row_next, go, tw);
        if (NC && a.nones_next) {
          uint32_t cz = 0, co = 0;
          for (uint32_t i = lane; i < 32 * WPT; i += 32) {
            cz += __popc(zs[1 + i]);
            co += __popc(os[1 + i]);
          }
          cz = __reduce_add_sync(0xFFFFFFFFu, cz);
          co = __reduce_add_sync(0xFFFFFFFFu, co);
          if (lane == 0) {
            if (cz) nc_add(2 * wpf, cz);
            if (co) nc_add(2 * wpf + 1, co);
          }
        }
      } else {
        // several nodes: each level-(L-1) one bit to its own position
        for (uint32_t x = lane; x < nvw; x += 32) {
          const uint32_t wi = (seg + x) >> 5, bi = x & 31u;
          const uint2 wp = sWP[wi];
          const uint32_t onesb = wp.y + __popc(wp.x & ((1u << bi) - 1u));  // ones before x within the warp
          const uint32_t s = (uint32_t)sInS[seg + x];
          if ((s >> k1) & 1u) {
            const uint32_t p = (s & lmask) >> a.pshift;
            const uint2 tb = tab[p];
            const bool one = (wp.x >> bi) & 1u;
            const uint64_t d = one ? (uint64_t)tb.y + Ow + onesb : (uint64_t)tb.x + Zw + (x - onesb);
            if (d < a.n) atomicOr(&la.row_next[d >> 5], 1u << (d & 31u));
            if (NC && a.nones_next) nc_add(2 * p + (one ? 1u : 0u), 1u);
          }
        }
      }
    }
    __syncwarp();
    for (uint32_t i = lane; i < 2 * SW; i += 32) zs[i] = 0;  // the streams of the next tile
    pre = pre_next;
  }
  if (nc_smem) {
    __syncthreads();
    for (uint32_t i = tid; i < 2 * nodes; i += THREADS)
      if (sNC[i]) atomicAdd(&a.nones_next[i], sNC[i]);
  }
}

// ------------------------------------------------------------------ tables
struct ScanArgs {
  const uint32_t *hist;
  unsigned long long *E;  // 2^L + 1 entries
  uint32_t nbins, nblocks;
  uint32_t *ticket;
  Lookback lb;
};

// E[v] = sum of hist[0..v), E[nbins] = total.
__global__ void __launch_bounds__(kScanThreads) k_hist_scan(ScanArgs a) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_tile, s_P;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= a.nblocks) return;
  const uint32_t base = tile * kScanChunk + tid * kScanItems;
  uint32_t v[kScanItems];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < (int)kScanItems; ++i) {
    v[i] = base + i < a.nbins ? a.hist[base + i] : 0u;
    sum += v[i];
  }
  uint32_t total;
  const uint32_t excl = block_exclusive_scan<kScanThreads>(sum, s_warp, &total);
  if (tid < 32) {
    const uint32_t P = lookback(a.lb, tile, 0, total);
    if (tid == 0) s_P = P;
  }
  __syncthreads();
  uint32_t run = s_P + excl;
#pragma unroll
  for (int i = 0; i < (int)kScanItems; ++i) {
    if (base + i < a.nbins) a.E[base + i] = run;
    run += v[i];
  }
  if (tile == a.nblocks - 1 && tid == 0) a.E[a.nbins] = s_P + total;
}

struct TabArgs {
  const unsigned long long *E;
  uint2 *tab;
  uint32_t L, nblocks;
  uint32_t *ticket;
  Lookback lb;
};

// For levels l = 0..L-2 and prefixes p < 2^l:
//   c1(p) = E[(2p+2) << (L-l-1)] - E[(2p+1) << (L-l-1)]   (size of node 2p+1 on level l+1)
//   O_l(p) = sum of c1 over prefixes < p                     (ones of level l before node p)
//   tab[2^l - 1 + p] = {O_l(p), E[(2p+1) << (L-l-1)] - O_l(p)}
// Blocks are numbered level by level; each level is one look-back segment.
__global__ void __launch_bounds__(kScanThreads) k_level_tables(TabArgs a) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_tile, s_P;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= a.nblocks) return;
  uint32_t l = 0, first = 0;
  for (; l + 1 < a.L; ++l) {
    const uint32_t nb = ((1u << l) + kScanChunk - 1) / kScanChunk;
    if (tile < first + nb) break;
    first += nb;
  }
  const uint32_t cnt = 1u << l;
  const uint32_t sh = a.L - l - 1;
  const uint32_t base = (tile - first) * kScanChunk + tid * kScanItems;
  uint32_t c1[kScanItems];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < (int)kScanItems; ++i) {
    const uint32_t p = base + i;
    c1[i] = p < cnt ? (uint32_t)(a.E[(uint64_t)(2 * p + 2) << sh] - a.E[(uint64_t)(2 * p + 1) << sh])
                    : 0u;
    sum += c1[i];
  }
  uint32_t total;
  const uint32_t excl = block_exclusive_scan<kScanThreads>(sum, s_warp, &total);
  if (tid < 32) {
    const uint32_t P = lookback(a.lb, tile, first, total);
    if (tid == 0) s_P = P;
  }
  __syncthreads();
  uint32_t O = s_P + excl;
  uint2 *tl = a.tab + (cnt - 1);
#pragma unroll
  for (int i = 0; i < (int)kScanItems; ++i) {
    const uint32_t p = base + i;
    if (p < cnt) tl[p] = make_uint2(O, (uint32_t)a.E[(uint64_t)(2 * p + 1) << sh] - O);
    O += c1[i];
  }
}

struct NodeTabArgs {
  const uint32_t *ones;    // ones of level m per node (2^m counters)
  const uint2 *tab_prev;   // level m-1 table
  uint2 *tab;              // level m table (null for the last level: node starts only)
  unsigned long long *E;   // node starts, 2^L + 1 entries
  uint32_t L, m, n, nblocks;
  uint32_t *ticket;
  Lookback lb;
};

// Node tables of level m from per-node counts (no histogram).  With
// s(q) = start of node q of level m (= E[q << (L-m)]) and c(q) its ones:
//   O_m(q) = sum of c over nodes < q            (exclusive scan, look-back)
//   tab_m[q] = {O_m(q), s(q+1) - c(q) - O_m(q)}  (the 1-child of q starts at
//               s(q+1) - c(q): the node's ones come last)
// Node starts are not scanned: an even node starts where its parent does
// (written at a coarser level), an odd node q where the parent's 1-child
// does, tab_{m-1}[q/2].x + tab_{m-1}[q/2].y; the kernel writes
// E[q << (L-m)] for odd q.  Level 1 also writes E[0] = 0 and E[2^L] = n.
__global__ void __launch_bounds__(kScanThreads) k_node_tables(NodeTabArgs a) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_tile, s_P;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= a.nblocks) return;
  const uint32_t cnt = 1u << a.m, sh = a.L - a.m;
  const uint32_t base = tile * kScanChunk + tid * kScanItems;
  auto start_of = [&](uint32_t q) -> uint32_t {  // s(q), 0 <= q <= 2^m
    if (q >= cnt) return a.n;
    if (q & 1u) {
      const uint2 t = a.tab_prev[q >> 1];
      return t.x + t.y;
    }
    return (uint32_t)a.E[(uint64_t)q << sh];
  };
  uint32_t c[kScanItems];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < (int)kScanItems; ++i) {
    c[i] = base + i < cnt ? __ldcg(&a.ones[base + i]) : 0u;
    sum += c[i];
  }
  uint32_t total;
  const uint32_t excl = block_exclusive_scan<kScanThreads>(sum, s_warp, &total);
  if (tid < 32) {
    const uint32_t P = lookback(a.lb, tile, 0, total);
    if (tid == 0) s_P = P;
  }
  __syncthreads();
  uint32_t O = s_P + excl;
#pragma unroll
  for (int i = 0; i < (int)kScanItems; ++i) {
    const uint32_t q = base + i;
    if (q < cnt) {
      if (q & 1u) a.E[(uint64_t)q << sh] = start_of(q);
      if (a.tab) a.tab[q] = make_uint2(O, start_of(q + 1) - c[i] - O);
    }
    O += c[i];
  }
  if (a.m == 1 && tile == 0 && tid == 0) {
    a.E[0] = 0;
    a.E[1ull << a.L] = a.n;
  }
}

struct LeafStartArgs {
  const uint32_t *ones;   // ones of level L-1 per node
  const uint2 *tab_prev;  // level L-2 table
  unsigned long long *E;
  uint32_t L, n;
};

// Node starts of the last two levels from per-node counts: node q of level
// L-1 starts at E[2q] (odd q: where the 1-child of its parent starts), and
// its 1-child, the symbol value 2q+1, at s(q+1) - c(q).  Also E[0] = 0 and
// E[2^L] = n.
__global__ void k_leaf_starts(LeafStartArgs a) {
  const uint32_t cnt = 1u << (a.L - 1);
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
    uint32_t next;
    if (q + 1 >= cnt) {
      next = a.n;
    } else if ((q + 1) & 1u) {
      const uint2 t = a.tab_prev[(q + 1) >> 1];
      next = t.x + t.y;
    } else {
      next = (uint32_t)a.E[2ull * (q + 1)];
    }
    if (q & 1u) {
      const uint2 t = a.tab_prev[q >> 1];
      a.E[2ull * q] = t.x + t.y;
    }
    a.E[2ull * q + 1] = next - __ldcg(&a.ones[q]);
    if (q == 0) {  // the ends (also written at level 1 when there are more levels)
      a.E[0] = 0;
      a.E[1ull << a.L] = a.n;
    }
  }
}

}  // namespace

namespace {

// Node starts and level tables of one tree, computed by one CTA (used by the
// batched build, where each tree's tables are one work item):
//   E[v] = sum of hist[0..v) for v <= 2^L;
//   tab[2^l - 1 + p] = {O_l(p), E[(2p+1) << (L-l-1)] - O_l(p)} for l <= L-2,
//   O_l(p) = sum over p' < p of (E[(2p'+2) << (L-l-1)] - E[(2p'+1) << (L-l-1)]).
// Ends with a block barrier.
template <int THREADS>
__device__ void tables_one_cta(const uint32_t *hist, uint32_t L, unsigned long long *E, uint2 *tab,
                               uint32_t *s_warp) {
  constexpr uint32_t ITEMS = 8;
  constexpr uint32_t CH = THREADS * ITEMS;
  const uint32_t tid = threadIdx.x;
  const uint32_t nbins = 1u << L;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < nbins; base += CH) {
    const uint32_t i0 = base + tid * ITEMS;
    uint32_t v[ITEMS], sum = 0;
#pragma unroll
    for (uint32_t i = 0; i < ITEMS; ++i) {
      v[i] = i0 + i < nbins ? hist[i0 + i] : 0u;
      sum += v[i];
    }
    uint32_t total;
    uint32_t run = carry + block_exclusive_scan<THREADS>(sum, s_warp, &total);
#pragma unroll
    for (uint32_t i = 0; i < ITEMS; ++i) {
      if (i0 + i < nbins) E[i0 + i] = run;
      run += v[i];
    }
    carry += total;
    cta_sync<THREADS>();
  }
  if (tid == 0) E[nbins] = carry;
  cta_sync<THREADS>();
  for (uint32_t l = 0; l + 1 < L; ++l) {
    const uint32_t cnt = 1u << l, sh = L - l - 1;
    uint2 *tl = tab + (cnt - 1);
    carry = 0;
    for (uint32_t base = 0; base < cnt; base += CH) {
      const uint32_t p0 = base + tid * ITEMS;
      uint32_t c1[ITEMS], sum = 0;
#pragma unroll
      for (uint32_t i = 0; i < ITEMS; ++i) {
        const uint32_t p = p0 + i;
        c1[i] = p < cnt ? (uint32_t)(E[(uint64_t)(2 * p + 2) << sh] - E[(uint64_t)(2 * p + 1) << sh]) : 0u;
        sum += c1[i];
      }
      uint32_t total;
      uint32_t O = carry + block_exclusive_scan<THREADS>(sum, s_warp, &total);
#pragma unroll
      for (uint32_t i = 0; i < ITEMS; ++i) {
        const uint32_t p = p0 + i;
        if (p < cnt) tl[p] = make_uint2(O, (uint32_t)E[(uint64_t)(2 * p + 1) << sh] - O);
        O += c1[i];
      }
      carry += total;
      cta_sync<THREADS>();
    }
  }
}

}  // namespace
