// Device-side building blocks shared by the level passes: single-pass
// decoupled look-back, block scans, bit extraction, TMA bulk copies and
// mbarrier waits.  sm_103a only.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "wt.h"

namespace wtk {

// ---------------------------------------------------------------- look-back
// One 64-bit status word per tile: [flag:2][epoch:30][value:32].  The flag
// says whether `value` is the tile's own count (aggregate) or the inclusive
// prefix through the tile.  The epoch tags the pass that wrote it, so the
// array is reused across passes and builds without clearing: an entry from
// another pass reads as "not yet published".
constexpr uint32_t kFlagX = 0;  // nothing published for this pass
constexpr uint32_t kFlagA = 1;  // aggregate of this tile only
constexpr uint32_t kFlagP = 2;  // inclusive prefix through this tile
constexpr uint32_t kEpochMask = 0x3FFFFFFFu;

struct Lookback {
  unsigned long long *status;
  uint32_t epoch;       // this pass
  uint32_t spin_limit;  // polls before giving up
  uint32_t skip;        // test hook: 1 + tile that never publishes, 0 = off
  int *err;             // latched device error
};

__device__ __forceinline__ unsigned long long pack_status(uint32_t flag, uint32_t epoch,
                                                          uint32_t value) {
  return ((unsigned long long)flag << 62) |
         ((unsigned long long)(epoch & kEpochMask) << 32) | value;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void latch_error(int *err, int code) {
  atomicCAS(err, 0, code);
}

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Called by one whole warp after the tile's aggregate is published: walks
// back over the predecessors of `tile` in its segment (which starts at tile
// `first`), 32 at a time, and returns the tile's exclusive prefix (same value
// in every lane).  A window is used as soon as, counting from the nearest
// predecessor, every entry up to the first inclusive prefix is published
// (entries behind that prefix are not waited for); a window of aggregates
// only is summed and the walk moves on.  Every wait is bounded: after
// spin_limit polls the missing predecessors count as zero, WT_ERR_TIMEOUT is
// latched, and the pass runs to completion.
__device__ __forceinline__ uint32_t lookback_walk(const Lookback &lb, uint32_t tile, uint32_t first) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t exclusive = 0;
  long long pred = (long long)tile - 1;
  uint32_t spins = 0;
  bool timed_out = false;
  while (pred >= (long long)first) {
    const long long idx = pred - (long long)lane;
    uint32_t flag, val;
    for (;;) {
      if (idx >= (long long)first) {
        const unsigned long long s = ld_relaxed(&lb.status[idx]);
        const bool mine = ((uint32_t)(s >> 32) & kEpochMask) == (lb.epoch & kEpochMask);
        flag = mine ? (uint32_t)(s >> 62) : kFlagX;
        val = (uint32_t)s;
      } else {
        flag = kFlagP;  // before the segment: contributes nothing, stops the walk
        val = 0;
      }
      const uint32_t xm = __ballot_sync(0xFFFFFFFFu, flag == kFlagX);
      const uint32_t pm = __ballot_sync(0xFFFFFFFFu, flag == kFlagP);
      const uint32_t pk = pm & (0u - pm);  // nearest inclusive prefix
      if (pk ? (xm & (pk - 1u)) == 0u : xm == 0u) break;
      ++spins;
      // give up after spin_limit polls, or at once when another wait of this
      // build already gave up (bounds the total delay of a failed build)
      const bool give_up = spins > lb.spin_limit ||
                           ((spins & 63u) == 0 && *(volatile int *)lb.err == WT_ERR_TIMEOUT);
      if (__any_sync(0xFFFFFFFFu, give_up)) {
        timed_out = true;
        break;
      }
      __nanosleep(spins < 32 ? 32 : 256);
    }
    if (flag == kFlagX) {  // only after a timeout
      flag = kFlagP;
      val = 0;
    }
    const uint32_t pmask = __ballot_sync(0xFFFFFFFFu, flag == kFlagP);
    if (pmask) {
      const uint32_t k = __ffs(pmask) - 1;
      exclusive += warp_sum(lane <= k ? val : 0u);
      break;
    }
    exclusive += warp_sum(val);
    pred -= 32;
  }
  if (timed_out && lane == 0) latch_error(lb.err, WT_ERR_TIMEOUT);
  return exclusive;
}

// Publish `v` with `flag` for `tile` (one thread), unless the test hook
// withholds this tile.
__device__ __forceinline__ void lookback_publish(const Lookback &lb, uint32_t tile, uint32_t flag,
                                                 uint32_t v) {
  if ((lb.skip == 0) || (tile != lb.skip - 1)) st_relaxed(&lb.status[tile], pack_status(flag, lb.epoch, v));
}

// Called by one whole warp.  `tile` is this block's index in the status
// array, `first` the index of the first tile of its segment (that tile's
// exclusive prefix is 0).  Publishes the aggregate, walks back, publishes
// the inclusive prefix and returns the exclusive prefix.
__device__ __forceinline__ uint32_t lookback_inline(const Lookback &lb, uint32_t tile, uint32_t first,
                                                   uint32_t aggregate) {
  const uint32_t lane = threadIdx.x & 31;
  if (tile == first) {
    if (lane == 0) lookback_publish(lb, tile, kFlagP, aggregate);
    return 0;
  }
  if (lane == 0) lookback_publish(lb, tile, kFlagA, aggregate);
  const uint32_t exclusive = lookback_walk(lb, tile, first);
  if (lane == 0) lookback_publish(lb, tile, kFlagP, exclusive + aggregate);
  return exclusive;
}

// Out-of-line copy for kernels that call it once per tile.
static __device__ __noinline__ uint32_t lookback(const Lookback &lb, uint32_t tile, uint32_t first,
                                                 uint32_t aggregate) {
  return lookback_inline(lb, tile, first, aggregate);
}

// Barrier over the first THREADS threads of the block (named barrier 1,
// with the memory ordering of a block barrier).  In a kernel whose blocks
// have exactly THREADS threads it is a block barrier; the batched build's
// consumer warps use it without the block's producer warp.
template <int THREADS>
__device__ __forceinline__ void cta_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(THREADS) : "memory");
}

// The same barrier, returning whether p held in any of the THREADS threads.
template <int THREADS>
__device__ __forceinline__ bool cta_sync_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, s;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred s, 1, %2, q;\n\tselp.u32 %0, 1, 0, s;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)p), "n"(THREADS)
      : "memory");
  return r != 0;
}

// Block-wide exclusive scan of one uint32 per thread.  s_warp holds >= 33
// words.  Returns the thread's exclusive prefix; *total gets the block sum.
// Contains two barriers over the THREADS threads (cta_sync); callers must
// sync before reusing s_warp.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp,
                                                         uint32_t *total) {
  constexpr int NW = THREADS / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  cta_sync<THREADS>();
  if (warp == 0) {
    uint32_t w = lane < (uint32_t)NW ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    s_warp[lane] = w;  // inclusive over warps
  }
  cta_sync<THREADS>();
  *total = s_warp[NW - 1];
  return (warp ? s_warp[warp - 1] : 0u) + x - v;
}

// 64-bit variant: the low 32 bits carry per-thread counts whose exclusive
// prefix is wanted, the high 32 bits carry terms whose block total is wanted
// (no carry crosses from the low half: block sums stay below 2^32).
template <int THREADS>
__device__ __forceinline__ unsigned long long block_exclusive_scan64(unsigned long long v,
                                                                     unsigned long long *s_warp,
                                                                     unsigned long long *total) {
  constexpr int NW = THREADS / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  cta_sync<THREADS>();
  if (warp == 0) {
    unsigned long long w = lane < (uint32_t)NW ? s_warp[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
      if (lane >= (uint32_t)o) w += y;
    }
    s_warp[lane] = w;
  }
  cta_sync<THREADS>();
  *total = s_warp[NW - 1];
  return (warp ? s_warp[warp - 1] : 0ull) + x - v;
}

// ------------------------------------------------------------ tile counts
// Ones of one level per tile of T symbols, kept at three granularities (per
// tile, per 64 tiles, per 4096 tiles) so that the exclusive prefix of any
// tile t is a sum of (t >> 12) + ((t >> 6) & 63) + (t & 63) terms, loaded in
// parallel by the tile's threads.  The pass over level l adds the counts of
// level l+1 for the tiles of T_{l+1} its output lands in; the pass over level
// l+1 then needs no inter-tile wait at all.
struct TileCounts {
  uint32_t *c0, *c1, *c2;
};

__device__ __forceinline__ void counts_add(const TileCounts &c, uint32_t tile, uint32_t v) {
  if (v == 0) return;
  atomicAdd(&c.c0[tile], v);
  atomicAdd(&c.c1[tile >> 6], v);
  atomicAdd(&c.c2[tile >> 12], v);
}

__device__ __forceinline__ uint32_t prefix_terms(uint32_t t) {
  return (t >> 12) + ((t >> 6) & 63u) + (t & 63u);
}

__device__ __forceinline__ const uint32_t *prefix_term(const TileCounts &c, uint32_t t, uint32_t j) {
  const uint32_t n2 = t >> 12;
  if (j < n2) return c.c2 + j;
  j -= n2;
  const uint32_t n1 = (t >> 6) & 63u;
  if (j < n1) return c.c1 + ((t >> 12) << 6) + j;
  j -= n1;
  return c.c0 + ((t >> 6) << 6) + j;
}

// Total of a level's counts over all NT tiles, from the top tier (one warp).
__device__ __forceinline__ uint32_t counts_total_warp(const TileCounts &c, uint32_t NT) {
  uint32_t s = 0;
  for (uint32_t i = threadIdx.x & 31; i <= (NT - 1) >> 12; i += 32) s += __ldcg(&c.c2[i]);
  return __reduce_add_sync(0xFFFFFFFFu, s);
}

// This thread's share of the exclusive prefix of tile t (sum over threads).
template <int THREADS>
__device__ __forceinline__ uint32_t prefix_share(const TileCounts &c, uint32_t t) {
  const uint32_t nt = prefix_terms(t);
  uint32_t s = 0;
  for (uint32_t j = threadIdx.x; j < nt; j += THREADS) s += __ldcg(prefix_term(c, t, j));
  return s;
}

// ------------------------------------------------------------ bit packing
// A thread holds 32 consecutive symbols as 8*SB little-endian 32-bit words.
// Pack bit k of each symbol into one 32-bit word, symbol q -> bit q.
template <int SB>
__device__ __forceinline__ uint32_t pack_bits(const uint32_t *u, uint32_t k);

template <>
__device__ __forceinline__ uint32_t pack_bits<1>(const uint32_t *u, uint32_t k) {
  uint32_t w = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    // bit k of each byte to bit 0 of the byte, then gather the four bits
    // into the top nibble with one multiply (no carries between terms)
    const uint32_t x = (u[m] >> k) & 0x01010101u;
    w |= ((x * 0x10204080u) >> 28) << (4 * m);
  }
  return w;
}

template <>
__device__ __forceinline__ uint32_t pack_bits<2>(const uint32_t *u, uint32_t k) {
  uint32_t w = 0;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const uint32_t x = (u[m] >> k) & 0x00010001u;
    w |= ((x | (x >> 15)) & 3u) << (2 * m);
  }
  return w;
}

template <>
__device__ __forceinline__ uint32_t pack_bits<4>(const uint32_t *u, uint32_t k) {
  uint32_t w = 0;
#pragma unroll
  for (int m = 0; m < 32; ++m) w |= ((u[m] >> k) & 1u) << m;
  return w;
}

template <int SB>
__device__ __forceinline__ uint32_t symbol_at(const uint32_t *u, int q) {
  if (SB == 1) return (u[q >> 2] >> (8 * (q & 3))) & 0xFFu;
  if (SB == 2) return (u[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
  return u[q];
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ------------------------------------------------------- TMA bulk + mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Returns false (and latches
// WT_ERR_TIMEOUT) when the phase did not complete within `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit,
                                                  int *err) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 16) __nanosleep(64);
  }
  latch_error(err, WT_ERR_TIMEOUT);
  return false;
}

// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// 16 bytes from shared memory at an arbitrary byte offset of a 16-byte
// aligned word array (reads up to 4 bytes past the 16).
__device__ __forceinline__ uint4 lds16_unaligned(const uint32_t *base, uint32_t byte_off) {
  const uint32_t w = byte_off >> 2, sh = (byte_off & 3u) * 8u;
  const uint32_t a0 = base[w], a1 = base[w + 1], a2 = base[w + 2], a3 = base[w + 3];
  if (sh == 0) return make_uint4(a0, a1, a2, a3);
  const uint32_t a4 = base[w + 4];
  return make_uint4(__funnelshift_r(a0, a1, sh), __funnelshift_r(a1, a2, sh),
                    __funnelshift_r(a2, a3, sh), __funnelshift_r(a3, a4, sh));
}

}  // namespace wtk
