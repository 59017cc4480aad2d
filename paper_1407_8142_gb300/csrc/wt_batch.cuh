// Device side of the batched build (work-list kernel), shared by the batch
// API (wt_batch.cu) and the build server (wt_serve.cu).
#pragma once
#include <algorithm>
#include <cstring>
#include <vector>

#include "wt_kernels.cuh"

namespace {

struct BTree {
  const uint8_t *in;        // the sequence (16-byte aligned)
  uint8_t *buf[2];          // ping-pong T_l buffers, whole tiles
  uint32_t n, L, sigma, sb, NT, NB;
  uint64_t W;
  uint32_t *bits;
  unsigned long long *rank, *zeros, *node_start;
  uint2 *tab;
  uint32_t *hist;           // 2^L bins
  uint32_t *counts;         // per level: tile counts (three granularities)
  uint32_t counts_per_level;
  int *err;
  uint32_t *done;           // one completion counter per phase
  uint32_t phases;
  unsigned long long *t_done;  // global-timer stamp when the tree's last item completed
  // node counts instead of a 2^L-bin histogram (large alphabets): the split
  // of each level counts, per child node, the next level's ones into `hist`,
  // and a node-table phase turns them into that level's tables
  uint32_t nc;
  uint32_t chunk_shift;     // node-table chunks and leaf-start items cover 2^chunk_shift nodes
};

// What a phase of a tree does, and on which level.
enum BatchPhaseKind : uint32_t {
  kPhPrepass = 0, kPhTables = 1, kPhSplit = 2, kPhLeaf = 3, kPhNodeTables = 4, kPhLeafStarts = 5
};
struct PhaseInfo {
  uint32_t kind, level;
};

// Phases of a tree with a histogram: 0 pre-pass, 1 tables, 2..L split
// levels 0..L-2, L+1 last level.  With node counts (L >= 2): 0 pre-pass,
// 2m+1 split of level m (m <= L-2), 2m node tables of level m (1 <= m <=
// L-2), 2L-2 node starts of the last two levels, 2L-1 last level.
__host__ __device__ __forceinline__ PhaseInfo batch_phase(uint32_t nc, uint32_t L, uint32_t ph) {
  if (ph == 0) return {kPhPrepass, 0};
  if (!nc) {
    if (ph == 1) return {kPhTables, 0};
    const uint32_t lv = ph - 2;
    return {lv + 1 < L ? kPhSplit : kPhLeaf, lv};
  }
  if (ph == 2 * L - 1) return {kPhLeaf, L - 1};
  if (ph == 2 * L - 2) return {kPhLeafStarts, L - 1};
  if (ph & 1u) return {kPhSplit, (ph - 1) / 2};
  return {kPhNodeTables, ph / 2};
}

// Items of a phase: tiles, one table item, or node chunks.
__host__ __device__ __forceinline__ uint32_t batch_phase_items(uint32_t nc, uint32_t L, uint32_t NT,
                                                              uint32_t chunk_shift, uint32_t ph) {
  const PhaseInfo pi = batch_phase(nc, L, ph);
  if (pi.kind == kPhTables) return 1u;
  if (pi.kind == kPhNodeTables) return 1u;
  if (pi.kind == kPhLeafStarts) return (((1u << (L - 1)) - 1u) >> chunk_shift) + 1u;
  return NT;
}

struct BatchArgs {
  const BTree *trees;
  const uint32_t *grp_first;  // n_groups + 1: first item of every group
  const uint2 *grp;           // n_groups: {tree, phase}
  const uint32_t *hint;       // group of item i << hint_shift, for every such item
  uint32_t hint_shift;
  uint32_t chunk;             // consecutive items per ticket (1..kBatchChunk)
  uint32_t n_groups, n_items;
  uint32_t *ticket;
  uint32_t spin_limit;
  int *err;                   // batch-level error (timeouts of dependency waits)
  unsigned long long *t_start;  // global-timer stamp when the first item started
};

__device__ __forceinline__ unsigned long long global_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t phase_items(const BTree &t, uint32_t phase) {
  return batch_phase_items(t.nc, t.L, t.NT, t.chunk_shift, phase);
}

__device__ __forceinline__ TileCounts tree_counts(const BTree &t, uint32_t level) {
  uint32_t *base = t.counts + (uint64_t)level * t.counts_per_level;
  return TileCounts{base, base + t.NT, base + t.NT + (t.NT >> 6) + 1};
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The symbols an item of `phase` reads: S for the pre-pass, for level 0 and
// for the only level of a one-level tree; else the ping-pong buffer the
// previous level wrote (whole tiles).
__device__ __forceinline__ const uint8_t *item_input(const BTree &tr, uint32_t phase) {
  const PhaseInfo pi = batch_phase(tr.nc, tr.L, phase);
  if (pi.kind == kPhPrepass || pi.level == 0 || tr.L < 2) return tr.in;
  return tr.buf[(pi.level - 1) & 1];
}

// Whether an item of the phase reads a tile of symbols.
__device__ __forceinline__ bool phase_reads_tile(const BTree &tr, uint32_t phase) {
  const uint32_t k = batch_phase(tr.nc, tr.L, phase).kind;
  return k == kPhPrepass || k == kPhSplit || k == kPhLeaf;
}

// Input tiles in flight per block: three, or two when the batch holds
// 4-byte symbols (their tiles are large).
template <int MAXSB>
__host__ __device__ constexpr uint32_t batch_slots() { return MAXSB == 4 ? 2u : 3u; }

// One work item as the producer warp hands it to the consumer warps.
struct BatchSlot {
  BTree tr;            // the item's tree
  uint32_t phase, tile, flags;
  uint32_t prefix;     // ones of the item's level before its tile (split and last-level items)
};
constexpr uint32_t kSlotEnd = 1;   // no more items
constexpr uint32_t kSlotSkip = 2;  // the item's dependency wait ran out: skip its work

template <int THREADS, int MAXSB>
constexpr uint32_t batch_smem_bytes() {
  // the ring of input tiles (symbols of up to MAXSB bytes), per-warp staging
  // (also the shared histogram of the pre-pass), {word, prefix} per thread,
  // per-warp {ones, share}, slot descriptors, full and empty mbarriers,
  // split-run counters, the table scan's warp sums and the partition
  // selectors of 1-byte symbols
  return batch_slots<MAXSB>() * 32u * THREADS * MAXSB + (THREADS / 32) * stage_bytes<MAXSB>() + 8u * THREADS +
         8u * (THREADS / 32) + batch_slots<MAXSB>() * (uint32_t)sizeof(BatchSlot) + 16u * batch_slots<MAXSB>() +
         64u + 4u * 33u + 16u + 1024u;
}

constexpr uint32_t kBatchHistSmem = 8192;  // histograms up to this many bins in shared memory
// Word offset, from the split-run counters, of the 256 partition selectors
// (after the counters and the table scan's 33 warp sums).
constexpr uint32_t kBatchPermWord = 52;

// The work of one item (a tile of the pre-pass, of a split level or of the
// last level) by the consumer warps; sIn holds the tile's symbols.
template <int SB, int THREADS, int MAXSB>
__device__ void batch_tile(const BTree &tr, PhaseInfo pi, uint32_t tile, uint32_t share_part, uint8_t *sIn,
                           uint8_t *sStage, uint2 *sWP, uint2 *sWT, uint32_t *sMisc,
                           uint32_t spin_limit) {
  const uint32_t tid = threadIdx.x;
  const uint32_t L = tr.L;
  if (pi.kind == kPhPrepass) {
    PrepassArgs a;
    a.in = tr.in;
    a.in_padded = 0;
    a.n = tr.n;
    a.L = L;
    a.NT = tr.NT;
    a.sigma = tr.sigma;
    a.hist = tr.hist;
    a.cnt = tree_counts(tr, 0);
    a.ticket = nullptr;
    a.spin_limit = spin_limit;
    a.err = tr.err;
    uint32_t bad = 0;
    const uint32_t nbins = 1u << L;
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(sStage);
    if (tr.nc) {
      // node counts: no histogram, the range check and level 0's ones only
      prepass_tile<SB, THREADS, kHistNone>(a, tile, sIn, nullptr, sMisc, bad, nullptr, 0);
    } else if (nbins <= kHistBallotMaxBins) {
      // few bins: shared-memory atomics of a row would collide on them
      prepass_tile<SB, THREADS, kHistBallot>(a, tile, sIn, nullptr, sMisc, bad, nullptr, 0);
    } else if (nbins <= kBatchHistSmem && nbins * 4 <= (THREADS / 32) * stage_bytes<MAXSB>()) {
      for (uint32_t i = tid; i < nbins; i += THREADS) s_hist[i] = 0;
      cta_sync<THREADS>();
      prepass_tile<SB, THREADS, kHistSmem>(a, tile, sIn, s_hist, sMisc, bad, nullptr, 0);
      for (uint32_t i = tid; i < nbins; i += THREADS)
        if (s_hist[i]) atomicAdd(&tr.hist[i], s_hist[i]);
    } else {
      prepass_tile<SB, THREADS, kHistGlobal>(a, tile, sIn, nullptr, sMisc, bad, nullptr, 0);
    }
    if (bad) latch_error(tr.err, WT_ERR_SYMBOL);
    return;
  }
  const uint32_t level = pi.level;
  const LevelOut lo{tr.bits + (uint64_t)level * tr.W, tr.rank + (uint64_t)level * (tr.NB + 1),
                    tr.zeros + level};
  if (pi.kind == kPhSplit) {
    SplitArgs a;
    a.in = level == 0 ? tr.in : tr.buf[(level - 1) & 1];
    a.out = tr.buf[level & 1];
    a.in_padded = level != 0;
    a.n = tr.n;
    a.L = L;
    a.level = level;
    a.NT = tr.NT;
    a.NB = tr.NB;
    a.log2T = 5 + (uint32_t)__ffs(THREADS) - 1;
    a.W = tr.W;
    a.tab = tr.tab + ((1u << level) - 1);
    a.pshift = L - level;
    a.count_table = 0;
    a.tab_out = nullptr;
    a.nones_next = tr.nc ? tr.hist + ((2u << level) - 1) : nullptr;
    a.node_ones = nullptr;  // the level's table comes from its node-table phase
    a.tab_prev = nullptr;
    a.tab_w = nullptr;
    a.E = nullptr;
    a.lo = lo;
    a.cin = tree_counts(tr, level);
    a.cout = tree_counts(tr, level + 1);
    a.ticket = nullptr;
    a.spin_limit = spin_limit;
    a.err = tr.err;
    // sMisc: [0..3] run counters, [4..5] run starts, [6..7] the level-0
    // table of a node-count tree, [8..10] node-count cache
    uint2 *const sTab0 = reinterpret_cast<uint2 *>(sMisc + 6);
    uint32_t *const sNc = sMisc + 8;
    const SplitShared sm{sStage, sWP, sWT, sMisc, sMisc + 4, sNc, SB == 1 ? sMisc + kBatchPermWord : nullptr};
    if (tid < 4) sMisc[tid] = 0;
    if (tr.nc && level == 0 && tid < 32) {
      // one node: its ones go after all zeros of the level, which are n
      // minus the level's ones (the top tier of its tile counts)
      const uint32_t ones = counts_total_warp(a.cin, tr.NT);
      if (tid == 0) {
        *sTab0 = make_uint2(0u, tr.n - ones);
        if (tile == 0) tr.tab[0] = *sTab0;  // the node tables of level 1 read it
      }
    }
    if (tid == 0) sNc[0] = 0xFFFFFFFFu;
    cta_sync<THREADS>();
    const uint2 *tab = (tr.nc && level == 0) ? sTab0 : a.tab;
    if (tr.nc) {
      split_tile<SB, THREADS, true>(a, tab, tile, sIn, share_part, sm, nullptr, 0);
      if (tid == 0 && sNc[0] != 0xFFFFFFFFu) {  // the item's cached node counts
        if (sNc[1]) atomicAdd(&a.nones_next[2 * sNc[0]], sNc[1]);
        if (sNc[2]) atomicAdd(&a.nones_next[2 * sNc[0] + 1], sNc[2]);
      }
    } else {
      split_tile<SB, THREADS, false>(a, tab, tile, sIn, share_part, sm, nullptr, 0);
    }
  } else {
    LeafArgs a;
    a.in = L >= 2 ? tr.buf[(L - 2) & 1] : tr.in;
    a.in_padded = L >= 2;
    a.n = tr.n;
    a.L = L;
    a.NT = tr.NT;
    a.NB = tr.NB;
    a.W = tr.W;
    a.out = lo;
    a.cnt = tree_counts(tr, level);
    a.ticket = nullptr;
    a.spin_limit = spin_limit;
    a.err = tr.err;
    leaf_tile<SB, THREADS>(a, tile, sIn, share_part, sWT, nullptr, 0);
  }
}

// Node tables of level m of a node-count tree: the same tables as the
// single-tree build's node-table kernel, by one block, chunk by chunk
// (2^chunk_shift nodes, 8 per thread), the scan carried from chunk to
// chunk.  With s(q) = start of node q and c(q) its ones: O_m(q) = sum of c
// over nodes < q, tab_m[q] = {O_m(q), s(q+1) - c(q) - O_m(q)}; an odd node
// starts where its parent's 1-child does, an even node where its parent
// does (written before).  One item per level: chunks scanned by several
// blocks through a look-back each waited for a chunk that sat in another
// block's queue behind another tree's waiting chunk, and those waits
// chained from block to block (levels 12-14 of a 512-tree batch took 4, 8
// and 15 ms).
template <int THREADS>
__device__ void batch_node_tables(const BTree &tr, uint32_t m, uint32_t *s_warp) {
  constexpr uint32_t ITEMS = 8;
  const uint32_t tid = threadIdx.x;
  const uint32_t cnt = 1u << m, sh = tr.L - m;
  const uint32_t *ones = tr.hist + (cnt - 1);
  const uint2 *tab_prev = tr.tab + ((cnt >> 1) - 1);
  uint2 *tab = tr.tab + (cnt - 1);
  unsigned long long *E = tr.node_start;
  auto start_of = [&](uint32_t q) -> uint32_t {  // s(q), 0 <= q <= 2^m
    if (q >= cnt) return tr.n;
    if (q & 1u) {
      const uint2 t = tab_prev[q >> 1];
      return t.x + t.y;
    }
    return (uint32_t)E[(uint64_t)q << sh];
  };
  uint32_t carry = 0;  // ones of the nodes of the chunks before
  for (uint32_t base0 = 0; base0 < cnt; base0 += 1u << tr.chunk_shift) {
    const uint32_t base = base0 + tid * ITEMS;
    uint32_t c[ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t i = 0; i < ITEMS; ++i) {
      c[i] = base + i < cnt ? __ldcg(&ones[base + i]) : 0u;
      sum += c[i];
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan<THREADS>(sum, s_warp, &total);
    uint32_t O = carry + excl;
#pragma unroll
    for (uint32_t i = 0; i < ITEMS; ++i) {
      const uint32_t q = base + i;
      if (q < cnt) {
        if (q & 1u) E[(uint64_t)q << sh] = start_of(q);
        tab[q] = make_uint2(O, start_of(q + 1) - c[i] - O);
      }
      O += c[i];
    }
    carry += total;
    cta_sync<THREADS>();  // s_warp is reused by the next chunk's scan
  }
  if (m == 1 && tid == 0) {
    E[0] = 0;
    E[1ull << tr.L] = tr.n;
  }
}

// Node starts of the last two levels of a node-count tree, for the nodes of
// level L-1 in chunk `chunk`: node q starts at E[2q] (odd q: where its
// parent's 1-child starts) and its 1-child, symbol value 2q+1, at
// s(q+1) - c(q).  Also E[0] = 0 and E[2^L] = n.
template <int THREADS>
__device__ void batch_leaf_starts(const BTree &tr, uint32_t chunk) {
  // Every node's inputs were written by earlier phases, so a thread issues
  // the loads of G nodes before it uses any of them (node by node, each
  // node's loads waited for the previous node's stores: 37 us per item of
  // 1024 nodes in a config-4 batch).
  constexpr uint32_t G = THREADS >= 256 ? 2 : 1;  // nodes per thread whose loads are in flight together (registers)
  const uint32_t L = tr.L;
  const uint32_t cnt = 1u << (L - 1);
  const uint32_t *ones = tr.hist + (cnt - 1);
  const uint2 *tab_prev = tr.tab + ((cnt >> 1) - 1);
  unsigned long long *E = tr.node_start;
  const uint32_t q0 = chunk << tr.chunk_shift;
  const uint32_t q1 = min(cnt, q0 + (1u << tr.chunk_shift));
  for (uint32_t qb = q0 + threadIdx.x; qb < q1; qb += G * THREADS) {
    uint2 tp[G];
    uint32_t c1[G];
    uint32_t en[G];
#pragma unroll
    for (uint32_t i = 0; i < G; ++i) {
      const uint32_t q = qb + i * THREADS;
      if (q < q1) {
        tp[i] = tab_prev[q >> 1];  // q odd: its own start; q even: its 1-sibling's, where q ends
        c1[i] = __ldcg(&ones[q]);
        en[i] = ((q & 1u) && q + 1 < cnt) ? (uint32_t)E[2ull * (q + 1)] : 0u;  // an even node's start
      }
    }
#pragma unroll
    for (uint32_t i = 0; i < G; ++i) {
      const uint32_t q = qb + i * THREADS;
      if (q < q1) {
        const uint32_t sib = tp[i].x + tp[i].y;
        const uint32_t next = q + 1 >= cnt ? tr.n : (q & 1u) ? en[i] : sib;
        if (q & 1u) E[2ull * q] = sib;
        E[2ull * q + 1] = next - c1[i];
        if (q == 0) {
          E[0] = 0;
          E[1ull << L] = tr.n;
        }
      }
    }
  }
}

// Items a producer takes per ticket, at most: consecutive items mostly share
// a group (tree and phase), so one group search, one descriptor and one
// dependency wait serve several items.  batch_launch takes fewer (items /
// (8 x blocks), at least one) when the batch has few items per block, so
// that a phase of a small tree is spread over as many blocks as it has
// tiles.
constexpr uint32_t kBatchChunk = 4;

// Publish the completion of the item a slot held (one thread of the
// producer warp, after the consumers released the slot): the consumers'
// writes, ordered before their release of the slot, become visible to the
// whole GPU before the tree's phase counter that later phases wait for.
__device__ __forceinline__ void batch_publish(const BatchSlot &sl) {
  __threadfence();
  const uint32_t prev = atomicAdd(&sl.tr.done[sl.phase], 1u);
  if (sl.phase + 1 == sl.tr.phases && prev + 1 == phase_items(sl.tr, sl.phase)) *sl.tr.t_done = global_timer();
}

// The producer warp: takes a.chunk consecutive items per ticket, finds
// each item's group (a hint per 2^hint_shift items, then a warp-wide search
// of the next 32 group starts; consecutive items of one group reuse it),
// copies the tree's descriptor into the next free slot, waits (bounded)
// until the tree's previous phase is complete, sums the item's count prefix,
// and starts the tile's copy into the slot's buffer (TMA), whose completion
// the slot's full barrier counts.  It runs up to batch_slots() items ahead
// of the consumers, and it publishes every item's completion as soon as the
// consumers release its slot -- also while it waits for a dependency, so
// that no completion it holds can hold up another block.
template <int THREADS, int MAXSB>
__device__ __forceinline__ void batch_producer(const BatchArgs &a, uint8_t *sBuf, BatchSlot *sSlot,
                                               uint64_t *full, uint64_t *empty) {
  constexpr uint32_t T = 32 * THREADS;
  constexpr uint32_t TB = T * MAXSB;
  constexpr uint32_t R = batch_slots<MAXSB>();
  const uint32_t lane = threadIdx.x & 31;
  uint32_t item = 0, left = 0;               // the current chunk
  uint32_t next_chunk = 0;                   // lane 0: the ticket of the chunk after it (fetched early)
  if (lane == 0) next_chunk = atomicAdd(a.ticket, a.chunk);
  uint32_t g = 0, g_lo = 1, g_hi = 0;        // the current group and its items [g_lo, g_hi)
  uint32_t ready = 0xFFFFFFFFu;              // group whose dependency was seen complete
  // the previous split or last-level item: its group, tile, prefix and own count
  uint32_t pv_g = 0xFFFFFFFFu, pv_tile = 0, pv_prefix = 0, pv_c0 = 0;
  // lane 0: uses of each slot handed to the consumers and not yet published
  // (bit s), and the use index of each
  uint32_t pending = 0, use_of[R];
#pragma unroll
  for (uint32_t i = 0; i < R; ++i) use_of[i] = 0;
  // lane 0: publish every pending slot the consumers have released
  auto publish_released = [&]() {
#pragma unroll
    for (uint32_t i = 0; i < R; ++i)
      if ((pending >> i) & 1u)
        if (mbar_try_wait(&empty[i], (use_of[i] / R) & 1u)) {
          batch_publish(sSlot[i]);
          pending &= ~(1u << i);
        }
  };
  bool alive = true;
  for (uint32_t u = 0;; ++u) {
    const uint32_t s = u % R;
    if (u >= R) {
      // the consumers release slot s after its previous item; publish it
      uint32_t ok = 1;
      if (lane == 0 && ((pending >> s) & 1u)) {
        ok = mbar_wait_bounded(&empty[s], (use_of[s] / R) & 1u, a.spin_limit, a.err);
        if (ok) {
          batch_publish(sSlot[s]);
          pending &= ~(1u << s);
        }
      }
      if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) {
        alive = false;  // the consumers stop on their own bounded wait
        break;
      }
    }
    if (left == 0) {
      uint32_t t = 0;
      if (lane == 0) {
        t = next_chunk;
        if (t < a.n_items) next_chunk = atomicAdd(a.ticket, a.chunk);
      }
      item = __shfl_sync(0xFFFFFFFFu, t, 0);
      left = a.chunk;
    } else {
      ++item;
    }
    --left;
    if (item >= a.n_items) {
      if (lane == 0) {
        sSlot[s].flags = kSlotEnd;
        mbar_arrive(&full[s]);
      }
      break;
    }
    if (item == 0 && lane == 0) *a.t_start = global_timer();
    if (item < g_lo || item >= g_hi) {
      g = (item >= g_hi && item < g_hi + 32) ? g : __ldg(&a.hint[item >> a.hint_shift]);
      for (;;) {
        const uint32_t c = g + 1 + lane;
        const bool le = c < a.n_groups && __ldg(&a.grp_first[c]) <= item;  // group starts rise
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, le);
        g += __popc(bal);
        if (bal != 0xFFFFFFFFu) break;
      }
      g_lo = __ldg(&a.grp_first[g]);
      g_hi = __ldg(&a.grp_first[g + 1]);
    }
    const uint2 gp = __ldg(&a.grp[g]);
    const uint32_t phase = gp.y;
    const uint32_t tile = item - g_lo;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.trees + gp.x);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sSlot[s].tr);
    for (uint32_t w = lane; w < (uint32_t)(sizeof(BTree) / 4); w += 32) dst[w] = __ldg(src + w);
    __syncwarp();
    const BTree &tr = sSlot[s].tr;
    uint32_t flags = 0, fresh = 0;
    if (lane == 0 && phase > 0 && ready != g) {
      const uint32_t want = phase_items(tr, phase - 1);
      uint32_t spins = 0;
      while (ld_acquire(&tr.done[phase - 1]) < want) {
        publish_released();
        if (++spins > a.spin_limit) {
          flags = kSlotSkip;
          latch_error(a.err, WT_ERR_TIMEOUT);
          latch_error(tr.err, WT_ERR_TIMEOUT);
          break;
        }
        __nanosleep(spins < 64 ? 64 : 512);
      }
      if (!flags) {
        ready = g;
        fresh = 1;
      }
    }
    ready = __shfl_sync(0xFFFFFFFFu, ready, 0);
    flags = __shfl_sync(0xFFFFFFFFu, flags, 0);
    __syncwarp();  // the dependency seen complete before the count loads
    uint32_t prefix = 0;
    const PhaseInfo pi = batch_phase(tr.nc, tr.L, phase);
    if ((pi.kind == kPhSplit || pi.kind == kPhLeaf) && !flags) {
      // the tile's exclusive ones-prefix from the level's tile counts: the
      // previous tile's prefix plus its count when this item follows it,
      // else a sum of up to (tile >> 12) + 126 terms; the tile's own count
      // is loaded for the next item
      const TileCounts c = tree_counts(tr, pi.level);
      if (g == pv_g && tile == pv_tile + 1) {
        prefix = pv_prefix + pv_c0;
      } else {
        const uint32_t nt = prefix_terms(tile);
        for (uint32_t j = lane; j < nt; j += 32) prefix += __ldcg(prefix_term(c, tile, j));
        prefix = __reduce_add_sync(0xFFFFFFFFu, prefix);
      }
      pv_g = g;
      pv_tile = tile;
      pv_prefix = prefix;
      pv_c0 = tile + 1 < tr.NT ? __ldcg(&c.c0[tile]) : 0u;
    }
    if (lane == 0) {
      sSlot[s].phase = phase;
      sSlot[s].tile = tile;
      sSlot[s].flags = flags;
      sSlot[s].prefix = prefix;
      if (phase_reads_tile(tr, phase) && flags == 0) {
        const uint8_t *in = item_input(tr, phase);
        const uint64_t start = (uint64_t)tile * T;
        const uint32_t nv = (uint32_t)umin64(T, tr.n - start);
        const uint32_t bytes = in != tr.in ? T * tr.sb : ((nv * tr.sb) & ~15u);
        // the previous phase's generic writes (seen complete just now)
        // before the async-proxy read of the copy
        if (fresh) fence_proxy_async_global();
        mbar_arrive_expect_tx(&full[s], bytes);
        if (bytes) bulk_g2s(sBuf + s * TB, in + start * tr.sb, bytes, &full[s]);
      } else {
        mbar_arrive(&full[s]);
      }
      pending |= 1u << s;
      use_of[s] = u;
    }
    __syncwarp();
  }
  // publish what the consumers still finish
  if (lane == 0 && alive) {
#pragma unroll
    for (uint32_t i = 0; i < R; ++i)
      if ((pending >> i) & 1u) {
        if (!mbar_wait_bounded(&empty[i], (use_of[i] / R) & 1u, a.spin_limit, a.err)) break;
        batch_publish(sSlot[i]);
      }
  }
}

// Batched build: THREADS consumer threads and one producer warp per block.
// Consumers take the slots in order: wait for the slot's item (bounded), do
// its work, and, behind a barrier of the consumer warps, release the slot to
// the producer (which then publishes the item's completion).
// Resident blocks per SM the batched kernel is compiled for (its shared
// memory allows as many; registers are capped to match).
template <int THREADS, int MAXSB>
constexpr int batch_min_blocks() {
  return MAXSB == 4 ? (THREADS == 128 ? 4 : 2) : (THREADS == 128 ? 6 : 3);
}

template <int THREADS, int MAXSB>
__global__ void __launch_bounds__(THREADS + 32, batch_min_blocks<THREADS, MAXSB>()) k_batch(BatchArgs a) {
  constexpr uint32_t T = 32 * THREADS;
  constexpr uint32_t NW = THREADS / 32;
  constexpr uint32_t TB = T * MAXSB;
  constexpr uint32_t R = batch_slots<MAXSB>();
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t *const sBuf = smem;
  uint8_t *const sStage = smem + R * TB;
  uint2 *const sWP = reinterpret_cast<uint2 *>(sStage + NW * stage_bytes<MAXSB>());
  uint2 *const sWT = sWP + THREADS;
  BatchSlot *const sSlot = reinterpret_cast<BatchSlot *>(sWT + NW);
  uint64_t *const full = reinterpret_cast<uint64_t *>(sSlot + R);
  uint64_t *const empty = full + R;
  uint32_t *const sMisc = reinterpret_cast<uint32_t *>(empty + R);  // split-run counters, starts, ...
  uint32_t *const s_warp = sMisc + 16;                              // 33 words
  const uint32_t tid = threadIdx.x;
  if (tid < THREADS) partition_selectors<THREADS>(sMisc + kBatchPermWord);
  if (tid == 0) {
    for (uint32_t i = 0; i < R; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (tid >= THREADS) {
    batch_producer<THREADS, MAXSB>(a, sBuf, sSlot, full, empty);
    return;
  }
  for (uint32_t u = 0;; ++u) {
    const uint32_t s = u % R;
    const bool ok = mbar_wait_bounded(&full[s], (u / R) & 1u, a.spin_limit, a.err);
    if (cta_sync_or<THREADS>(!ok)) {
      // the slot's item or its copy did not arrive in time: wait once more
      // (bounded) for a copy that may still be in flight, and stop
      if (tid == 0) mbar_wait_bounded(&full[s], (u / R) & 1u, a.spin_limit, a.err);
      cta_sync<THREADS>();
      return;
    }
    const BatchSlot &sl = sSlot[s];
    if (sl.flags & kSlotEnd) return;
    const BTree &tr = sl.tr;
    const uint32_t phase = sl.phase, tile = sl.tile;
    const PhaseInfo pi = batch_phase(tr.nc, tr.L, phase);
    if (!(sl.flags & kSlotSkip)) {
      if (pi.kind == kPhTables) {
        tables_one_cta<THREADS>(tr.hist, tr.L, tr.node_start, tr.tab, s_warp);
      } else if (pi.kind == kPhNodeTables) {
        batch_node_tables<THREADS>(tr, pi.level, s_warp);
      } else if (pi.kind == kPhLeafStarts) {
        batch_leaf_starts<THREADS>(tr, tile);
      } else {
        uint8_t *const sIn = sBuf + s * TB;
        const uint8_t *in = item_input(tr, phase);
        const uint64_t start = (uint64_t)tile * T;
        const uint32_t nv = (uint32_t)umin64(T, tr.n - start);
        if (in == tr.in && ((nv * tr.sb) & 15u)) {  // tail bytes the bulk copy left out
          for (uint32_t i = ((nv * tr.sb) & ~15u) + tid; i < nv * tr.sb; i += THREADS)
            sIn[i] = in[start * tr.sb + i];
          cta_sync<THREADS>();
        }
        const uint32_t share = tid == 0 ? sl.prefix : 0u;
        switch (tr.sb) {
          case 1: batch_tile<1, THREADS, MAXSB>(tr, pi, tile, share, sIn, sStage, sWP, sWT, sMisc, a.spin_limit); break;
          case 2:
            if constexpr (MAXSB >= 2)
              batch_tile<2, THREADS, MAXSB>(tr, pi, tile, share, sIn, sStage, sWP, sWT, sMisc, a.spin_limit);
            break;
          default:
            if constexpr (MAXSB >= 4)
              batch_tile<4, THREADS, MAXSB>(tr, pi, tile, share, sIn, sStage, sWP, sWT, sMisc, a.spin_limit);
            break;
        }
      }
    }
    // release the slot; the producer publishes the item's completion
    cta_sync<THREADS>();
    if (tid == 0) mbar_arrive(&empty[s]);
  }
}

}  // namespace

namespace {

// ------------------------------------------------------------------ layout
// Sizes of one tree's regions in a batch (bytes, 256-aligned).
struct BatchGeo {
  uint64_t n, NB, W, NT, nbins, cpl;
  uint64_t bits, rank, zeros, ns, tab, buf, ctrl;
  uint32_t L, phases;
  bool nc;               // node counts instead of a histogram
  uint32_t chunk_shift;  // nodes per node-table chunk and leaf-start item: 2^chunk_shift
};

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

inline uint32_t batch_levels(uint32_t sigma) {
  uint32_t L = 0;
  while ((1ull << L) < sigma) ++L;
  return L;
}

// Geometry of one sequence; false when its description is invalid.
inline bool batch_geo(const wt_seq_desc &d, uint32_t threads, BatchGeo &g) {
  if (!(d.symbol_bytes == 1 || d.symbol_bytes == 2 || d.symbol_bytes == 4) || d.sigma == 0 ||
      (uint64_t)d.sigma > (1ull << (8 * d.symbol_bytes)) || d.n >= (1ull << 32) || d.n == 0)
    return false;
  const uint64_t T = 32ull * threads;
  g.L = batch_levels(d.sigma);
  if (g.L > kMaxLevels) return false;
  g.n = d.n;
  g.NB = (d.n + 511) / 512;
  g.W = 16 * g.NB;
  g.NT = (d.n + T - 1) / T;
  const uint64_t Lz = std::max<uint32_t>(g.L, 1);
  g.bits = al256(Lz * g.W * 4);
  g.rank = al256(Lz * (g.NB + 1) * 8);
  g.zeros = al256(Lz * 8);
  g.nbins = 1ull << g.L;
  g.ns = al256((g.nbins + 1) * 8);
  g.tab = al256(std::max<uint64_t>(1, g.nbins / 2) * 8);
  g.buf = g.L >= 2 ? al256(g.NT * T * d.symbol_bytes + 16) : 0;
  g.cpl = g.NT + (g.NT >> 6) + 1 + (g.NT >> 12) + 1;
  // large alphabets: per-node counts instead of the 2^L-bin histogram
  g.nc = g.L >= 2 && g.nbins > kBatchHistSmem;
  g.chunk_shift = 0;
  while ((1u << g.chunk_shift) < 8u * threads) ++g.chunk_shift;  // 8 nodes per consumer thread
  g.phases = g.nc ? 2 * g.L : (g.L >= 1 ? g.L + 2 : 2);
  // control block: error word, histogram (or node counts), tile counts,
  // phase counters, stamp
  g.ctrl = al256((1 + g.nbins + Lz * g.cpl + g.phases) * 4 + 16 + 8);
  return true;
}

inline uint64_t batch_mem_bytes(const BatchGeo &g) {
  return g.bits + g.rank + g.zeros + g.ns + g.tab + 2 * g.buf;
}

// Descriptor of one tree whose regions start at mem (outputs and scratch)
// and ctrl (control block, cleared before every build).
inline BTree batch_tree(const wt_seq_desc &d, const BatchGeo &g, unsigned char *mem,
                        unsigned char *ctrl) {
  BTree t;
  std::memset(&t, 0, sizeof(t));
  unsigned char *p = mem;
  t.bits = reinterpret_cast<uint32_t *>(p);
  p += g.bits;
  t.rank = reinterpret_cast<unsigned long long *>(p);
  p += g.rank;
  t.zeros = reinterpret_cast<unsigned long long *>(p);
  p += g.zeros;
  t.node_start = reinterpret_cast<unsigned long long *>(p);
  p += g.ns;
  t.tab = reinterpret_cast<uint2 *>(p);
  p += g.tab;
  t.buf[0] = g.buf ? p : nullptr;
  p += g.buf;
  t.buf[1] = g.buf ? p : nullptr;
  uint32_t *c = reinterpret_cast<uint32_t *>(ctrl);
  t.err = reinterpret_cast<int *>(c);
  t.hist = c + 1;
  t.counts = c + 1 + g.nbins;
  t.done = t.counts + std::max<uint32_t>(g.L, 1) * g.cpl;
  t.phases = g.phases;
  t.t_done = reinterpret_cast<unsigned long long *>(
      (reinterpret_cast<uintptr_t>(t.done + g.phases) + 7) & ~uintptr_t(7));
  t.nc = g.nc ? 1u : 0u;
  t.chunk_shift = g.chunk_shift;
  t.n = (uint32_t)g.n;
  t.L = g.L;
  t.sigma = d.sigma;
  t.sb = d.symbol_bytes;
  t.NT = (uint32_t)g.NT;
  t.NB = (uint32_t)g.NB;
  t.W = g.W;
  t.counts_per_level = (uint32_t)g.cpl;
  return t;
}

// Work list: groups (tree, phase), phase by phase across trees.
inline uint32_t batch_worklist(const std::vector<BatchGeo> &geo, std::vector<uint32_t> &first,
                               std::vector<uint2> &grp) {
  uint32_t max_phases = 0;
  for (const BatchGeo &g : geo) max_phases = std::max(max_phases, g.phases);
  first.clear();
  grp.clear();
  uint32_t items = 0;
  for (uint32_t ph = 0; ph < max_phases; ++ph)
    for (uint32_t i = 0; i < (uint32_t)geo.size(); ++i) {
      if (ph >= geo[i].phases) continue;
      first.push_back(items);
      grp.push_back(make_uint2(i, ph));
      items += batch_phase_items(geo[i].nc, geo[i].L, (uint32_t)geo[i].NT, geo[i].chunk_shift, ph);
    }
  first.push_back(items);
  return items;
}

// Hints for the producer's group search: hint[h] = the group of item
// h << shift.  shift >= 5, and larger when the table would exceed max_hints
// entries (the search then walks several windows of 32 groups per item).
inline uint32_t batch_hints(const std::vector<uint32_t> &first, uint32_t items, uint32_t max_hints,
                            std::vector<uint32_t> &hint) {
  uint32_t shift = 5;
  while (((uint64_t)items >> shift) + 1 > max_hints) ++shift;
  const uint32_t nh = (items >> shift) + 1;
  hint.assign(nh, 0);
  uint32_t g = 0;
  const uint32_t ng = (uint32_t)first.size() - 1;
  for (uint32_t h = 0; h < nh; ++h) {
    const uint64_t item = (uint64_t)h << shift;
    while (g + 1 < ng && first[g + 1] <= item) ++g;
    hint[h] = g;
  }
  return shift;
}

// Launch the batch kernel over a work list on `stream`: blocks of `threads`
// consumer threads plus a producer warp, tiles sized for max_sb-byte symbols.
inline cudaError_t batch_launch(const BatchArgs &a, uint32_t threads, uint32_t max_sb, int sms,
                                uint32_t ctas_per_sm, cudaStream_t st) {
  auto go = [&](auto kern, uint32_t th, size_t sm) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, th + 32, sm) != cudaSuccess) {
      (void)cudaGetLastError();
      occ = 1;
    }
    occ = std::max(occ, 1);
    if (ctas_per_sm) occ = std::min<int>(occ, (int)ctas_per_sm);
    const int grid = (int)std::min<uint64_t>((uint64_t)occ * sms, std::max<uint32_t>(a.n_items, 1));
    BatchArgs b = a;
    b.chunk = std::max<uint32_t>(1, std::min<uint32_t>(kBatchChunk, a.n_items / (8u * (uint32_t)grid)));
    kern<<<grid, th + 32, sm, st>>>(b);
    return cudaGetLastError();
  };
  if (threads == 128) {
    if (max_sb <= 1) return go(k_batch<128, 1>, 128, batch_smem_bytes<128, 1>());
    if (max_sb <= 2) return go(k_batch<128, 2>, 128, batch_smem_bytes<128, 2>());
    return go(k_batch<128, 4>, 128, batch_smem_bytes<128, 4>());
  }
  if (max_sb <= 1) return go(k_batch<256, 1>, 256, batch_smem_bytes<256, 1>());
  if (max_sb <= 2) return go(k_batch<256, 2>, 256, batch_smem_bytes<256, 2>());
  return go(k_batch<256, 4>, 256, batch_smem_bytes<256, 4>());
}

}  // namespace
