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
};

struct BatchArgs {
  const BTree *trees;
  const uint32_t *grp_first;  // n_groups + 1: first item of every group
  const uint2 *grp;           // n_groups: {tree, phase}
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
  return phase == 1 ? 1u : t.NT;
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

template <int THREADS>
constexpr uint32_t batch_smem_bytes() {
  // one input tile of up to 4-byte symbols, per-warp staging (also the
  // shared histogram of the pre-pass), {word, prefix} per thread, per-warp
  // {ones, share}, mbarrier and scratch words
  return 32u * THREADS * 4 + (THREADS / 32) * stage_bytes<4>() + 8u * THREADS + 8u * (THREADS / 32) +
         64u;
}

constexpr uint32_t kBatchHistSmem = 8192;  // histograms up to this many bins in shared memory

template <int SB, int THREADS>
__device__ void batch_tile(const BTree &tr, uint32_t phase, uint32_t tile, uint8_t *sIn,
                           uint8_t *sStage, uint2 *sWP, uint2 *sWT, uint32_t *sMisc,
                           uint32_t spin_limit) {
  constexpr uint32_t T = 32 * THREADS;
  const uint32_t tid = threadIdx.x;
  const uint32_t L = tr.L;
  const uint64_t start = (uint64_t)tile * T;
  const uint32_t nv = (uint32_t)umin64(T, tr.n - start);
  if (phase == 0) {
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
    if (nbins <= kBatchHistSmem && nbins * 4 <= (THREADS / 32) * stage_bytes<4>()) {
      for (uint32_t i = tid; i < nbins; i += THREADS) s_hist[i] = 0;
      __syncthreads();
      prepass_tile<SB, THREADS, kHistSmem>(a, tile, sIn, s_hist, sMisc, bad, nullptr, 0);
      for (uint32_t i = tid; i < nbins; i += THREADS)
        if (s_hist[i]) atomicAdd(&tr.hist[i], s_hist[i]);
    } else {
      prepass_tile<SB, THREADS, kHistGlobal>(a, tile, sIn, nullptr, sMisc, bad, nullptr, 0);
    }
    if (bad) latch_error(tr.err, WT_ERR_SYMBOL);
    return;
  }
  const uint32_t level = phase - 2;  // split level, or L-1 for the last level
  const PrefixLoads pre = prefix_loads<THREADS>(tree_counts(tr, level), tile, tr.NT);
  const LevelOut lo{tr.bits + (uint64_t)level * tr.W, tr.rank + (uint64_t)level * (tr.NB + 1),
                    tr.zeros + level};
  (void)nv;
  if (level + 1 < L) {
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
    a.nones_next = nullptr;
    a.lo = lo;
    a.cin = tree_counts(tr, level);
    a.cout = tree_counts(tr, level + 1);
    a.ticket = nullptr;
    a.spin_limit = spin_limit;
    a.err = tr.err;
    const SplitShared sm{sStage, sWP, sWT, sMisc, sMisc + 4};
    if (tid < 4) sMisc[tid] = 0;
    __syncthreads();
    split_tile<SB, THREADS, false>(a, a.tab, tile, sIn, pre.sum(), sm, nullptr, 0);
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
    leaf_tile<SB, THREADS>(a, tile, sIn, pre.sum(), sWT, nullptr, 0);
  }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_batch(BatchArgs a) {
  constexpr uint32_t T = 32 * THREADS;
  constexpr uint32_t NW = THREADS / 32;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t *const sIn = smem;
  uint8_t *const sStage = smem + T * 4;
  uint2 *const sWP = reinterpret_cast<uint2 *>(sStage + NW * stage_bytes<4>());
  uint2 *const sWT = sWP + THREADS;
  uint64_t *const bar = reinterpret_cast<uint64_t *>(sWT + NW);
  uint32_t *const sMisc = reinterpret_cast<uint32_t *>(bar + 1);  // item, and split counters
  __shared__ uint32_t s_item, s_ok;
  __shared__ uint32_t s_warp[33];
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity = 0;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= a.n_items) break;
    if (item == 0 && tid == 0) *a.t_start = global_timer();
    // group of this item: last g with grp_first[g] <= item
    uint32_t lo = 0, hi = a.n_groups - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (a.grp_first[mid] <= item) lo = mid;
      else hi = mid - 1;
    }
    const uint2 gp = a.grp[lo];
    const uint32_t phase = gp.y;
    const uint32_t tile = item - a.grp_first[lo];
    const BTree tr = a.trees[gp.x];
    // wait for the tree's previous phase (bounded)
    if (tid == 0) {
      uint32_t ok = 1;
      if (phase > 0) {
        const uint32_t want = phase_items(tr, phase - 1);
        uint32_t spins = 0;
        while (ld_acquire(&tr.done[phase - 1]) < want) {
          if (++spins > a.spin_limit) {
            ok = 0;
            latch_error(a.err, WT_ERR_TIMEOUT);
            latch_error(tr.err, WT_ERR_TIMEOUT);
            break;
          }
          __nanosleep(spins < 64 ? 64 : 512);
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
      if (phase == 1) {
        tables_one_cta<THREADS>(tr.hist, tr.L, tr.node_start, tr.tab, s_warp);
      } else {
        // the tile's symbols into shared memory (TMA), tail bytes by hand
        const uint32_t level = phase >= 2 ? phase - 2 : 0;
        const uint8_t *in = phase == 0 ? tr.in
                            : (level == 0 || (level + 1 == tr.L && tr.L < 2)) ? tr.in
                                                                              : tr.buf[(level - 1) & 1];
        const bool padded = in != tr.in;
        const uint64_t start = (uint64_t)tile * T;
        const uint32_t nv = (uint32_t)umin64(T, tr.n - start);
        const uint32_t bytes = padded ? T * tr.sb : ((nv * tr.sb) & ~15u);
        if (tid == 0) {
          fence_proxy_async_global();
          mbar_arrive_expect_tx(bar, bytes);
          if (bytes) bulk_g2s(sIn, in + start * tr.sb, bytes, bar);
        }
        const bool ok = mbar_wait_bounded(bar, parity, a.spin_limit, tr.err);
        parity ^= 1u;
        if (__syncthreads_or(!ok)) {
          // the copy did not land in time: wait once more (bounded) and stop
          if (tid == 0) mbar_wait_bounded(bar, parity ^ 1u, a.spin_limit, tr.err);
          __syncthreads();
          return;
        }
        if (!padded && ((nv * tr.sb) & 15u)) {
          for (uint32_t i = ((nv * tr.sb) & ~15u) + tid; i < nv * tr.sb; i += THREADS)
            sIn[i] = in[start * tr.sb + i];
          __syncthreads();
        }
        switch (tr.sb) {
          case 1: batch_tile<1, THREADS>(tr, phase, tile, sIn, sStage, sWP, sWT, sMisc, a.spin_limit); break;
          case 2: batch_tile<2, THREADS>(tr, phase, tile, sIn, sStage, sWP, sWT, sMisc, a.spin_limit); break;
          default: batch_tile<4, THREADS>(tr, phase, tile, sIn, sStage, sWP, sWT, sMisc, a.spin_limit); break;
        }
      }
    }
    // publish the item's completion
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const uint32_t prev = atomicAdd(&tr.done[phase], 1u);
      if (phase + 1 == tr.phases && prev + 1 == phase_items(tr, phase)) *tr.t_done = global_timer();
    }
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
  g.phases = g.L >= 1 ? g.L + 2 : 2;
  // control block: error word, histogram, tile counts, phase counters, stamp
  g.ctrl = al256((1 + g.nbins + Lz * g.cpl + g.phases) * 4 + 16);
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
      items += ph == 1 ? 1u : (uint32_t)geo[i].NT;
    }
  first.push_back(items);
  return items;
}

// Launch the batch kernel over a work list on `stream`.
inline cudaError_t batch_launch(const BatchArgs &a, uint32_t threads, int sms, uint32_t ctas_per_sm,
                                cudaStream_t st) {
  auto go = [&](auto kern, uint32_t th, size_t sm) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, th, sm) != cudaSuccess) {
      (void)cudaGetLastError();
      occ = 1;
    }
    occ = std::max(occ, 1);
    if (ctas_per_sm) occ = std::min<int>(occ, (int)ctas_per_sm);
    const int grid = (int)std::min<uint64_t>((uint64_t)occ * sms, std::max<uint32_t>(a.n_items, 1));
    kern<<<grid, th, sm, st>>>(a);
    return cudaGetLastError();
  };
  if (threads == 128) return go(k_batch<128>, 128, batch_smem_bytes<128>());
  return go(k_batch<256>, 256, batch_smem_bytes<256>());
}

}  // namespace
