// Batched levelWT: many independent trees built by one persistent launch.
//
// Work list: for every tree its phases -- pre-pass (one item per tile), node
// tables (one item), split pass per level l = 0..L-2 (one item per tile),
// last level (one item per tile) -- grouped phase by phase across trees, so
// that all items an item depends on (its own tree's previous phase) come
// earlier in the list.  CTAs take items in list order from one ticket
// counter; an item waits, bounded, until its tree's previous phase has
// completed all its items (per-tree, per-phase completion counters), then runs
// the same tile code as the single-tree passes.  No grid-wide barrier, no
// deadlock: every item waited on was taken earlier by a running CTA.
#include <algorithm>
#include <cstring>
#include <new>
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
      prepass_tile<SB, THREADS, true>(a, tile, sIn, s_hist, sMisc, bad, nullptr, 0);
      for (uint32_t i = tid; i < nbins; i += THREADS)
        if (s_hist[i]) atomicAdd(&tr.hist[i], s_hist[i]);
    } else {
      prepass_tile<SB, THREADS, false>(a, tile, sIn, s_hist, sMisc, bad, nullptr, 0);
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
    a.lo = lo;
    a.cin = tree_counts(tr, level);
    a.cout = tree_counts(tr, level + 1);
    a.ticket = nullptr;
    a.spin_limit = spin_limit;
    a.err = tr.err;
    const SplitShared sm{sStage, sWP, sWT, sMisc, sMisc + 4};
    if (tid < 4) sMisc[tid] = 0;
    __syncthreads();
    split_tile<SB, THREADS>(a, a.tab, tile, sIn, pre.sum(), sm, nullptr, 0);
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

// ------------------------------------------------------------------ host side
int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? WT_ERR_OOM : WT_ERR_CUDA; }

#define WT_CUDA(call)            \
  do {                           \
    cudaError_t e__ = (call);    \
    if (e__ != cudaSuccess) {    \
      (void)cudaGetLastError();  \
      return cuda_fail(e__);     \
    }                            \
  } while (0)

uint32_t levels_of_b(uint32_t sigma) {
  uint32_t L = 0;
  while ((1ull << L) < sigma) ++L;
  return L;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct wt_batch {
  uint32_t m = 0;
  uint32_t threads = 256;
  wt_config cfg{};
  std::vector<wt_tree *> views;
  std::vector<BTree> host_trees;
  BTree *d_trees = nullptr;
  uint32_t *d_grp_first = nullptr;
  uint2 *d_grp = nullptr;
  uint32_t n_groups = 0, n_items = 0;
  unsigned char *d_mem = nullptr;    // outputs + scratch of every tree
  uint32_t *d_ctrl = nullptr;        // cleared per build: ticket, error, per-tree control blocks and counters
  size_t ctrl_bytes = 0;
  bool inputs_set = false;
  cudaStream_t stream = nullptr;
  int sms = 0;
};

extern "C" {

int wt_batch_free(wt_batch *b) {
  if (!b) return WT_OK;
  cudaStreamSynchronize(b->stream);
  (void)cudaGetLastError();
  for (wt_tree *v : b->views) delete v;
  cudaFree(b->d_mem);
  cudaFree(b->d_ctrl);
  cudaFree(b->d_trees);
  cudaFree(b->d_grp_first);
  cudaFree(b->d_grp);
  delete b;
  return WT_OK;
}

int wt_batch_create(const wt_seq_desc *descs, uint32_t m, const wt_config *cfg, wt_batch **out) {
  if (!out || !descs || m == 0) return WT_ERR_ARG;
  *out = nullptr;
  wt_batch *b = new (std::nothrow) wt_batch();
  if (!b) return WT_ERR_OOM;
  if (cfg) b->cfg = *cfg;
  b->threads = (cfg && cfg->tile_threads == 128) ? 128 : 256;
  if (cfg && cfg->tile_threads && cfg->tile_threads != 128 && cfg->tile_threads != 256) {
    delete b;
    return WT_ERR_ARG;
  }
  b->m = m;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return WT_ERR_CUDA;
  }
  const uint64_t T = 32ull * b->threads;
  // sizes
  struct Geo {
    uint64_t n, NB, W, NT, bits, rank, zeros, ns, tab, buf, nbins, cpl, ctrl;
    uint32_t L, phases;
  };
  std::vector<Geo> geo(m);
  size_t mem = 0, ctrl = 16 * 4;  // [0] ticket, [1] batch error
  for (uint32_t i = 0; i < m; ++i) {
    const wt_seq_desc &d = descs[i];
    if (!(d.symbol_bytes == 1 || d.symbol_bytes == 2 || d.symbol_bytes == 4) || d.sigma == 0 ||
        (uint64_t)d.sigma > (1ull << (8 * d.symbol_bytes)) || d.n >= (1ull << 32) || d.n == 0) {
      delete b;
      return WT_ERR_ARG;
    }
    Geo &g = geo[i];
    g.L = levels_of_b(d.sigma);
    if (g.L > kMaxLevels) {
      delete b;
      return WT_ERR_ARG;
    }
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
    // control block: error word, histogram, tile counts, phase counters
    g.ctrl = al256((1 + g.nbins + Lz * g.cpl + g.phases) * 4 + 16);
    mem += g.bits + g.rank + g.zeros + g.ns + g.tab + 2 * g.buf;
    ctrl += g.ctrl;
  }
  cudaError_t e;
  auto fail = [&](cudaError_t err) {
    (void)cudaGetLastError();
    wt_batch_free(b);
    return cuda_fail(err);
  };
  if ((e = cudaMalloc(&b->d_mem, std::max<size_t>(mem, 256)))) return fail(e);
  if ((e = cudaMalloc(&b->d_ctrl, ctrl))) return fail(e);
  b->ctrl_bytes = ctrl;
  // carve, build descriptors and views
  b->host_trees.resize(m);
  b->views.assign(m, nullptr);
  size_t off = 0, coff = 16 * 4;
  uint32_t max_phases = 0;
  for (uint32_t i = 0; i < m; ++i) {
    const Geo &g = geo[i];
    BTree &t = b->host_trees[i];
    std::memset(&t, 0, sizeof(t));
    unsigned char *p = b->d_mem + off;
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
    p += g.buf;
    off = p - b->d_mem;
    uint32_t *c = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(b->d_ctrl) + coff);
    t.err = reinterpret_cast<int *>(c);
    t.hist = c + 1;
    t.counts = c + 1 + g.nbins;
    t.done = t.counts + std::max<uint32_t>(g.L, 1) * g.cpl;
    t.phases = g.phases;
    t.t_done = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(t.done + g.phases) + 7) & ~uintptr_t(7));
    coff += g.ctrl;
    t.n = (uint32_t)g.n;
    t.L = g.L;
    t.sigma = descs[i].sigma;
    t.sb = descs[i].symbol_bytes;
    t.NT = (uint32_t)g.NT;
    t.NB = (uint32_t)g.NB;
    t.W = g.W;
    t.counts_per_level = (uint32_t)g.cpl;
    max_phases = std::max(max_phases, g.phases);
    // view
    wt_tree *v = new (std::nothrow) wt_tree();
    if (!v) {
      wt_batch_free(b);
      return WT_ERR_OOM;
    }
    v->owner = b;
    v->n = g.n;
    v->sigma = t.sigma;
    v->sb = t.sb;
    v->L = g.L;
    v->W = g.W;
    v->NB = g.NB;
    v->threads = b->threads;
    v->T = T;
    v->NT = g.NT;
    v->sms = b->sms;
    v->d_bits = t.bits;
    v->d_rank = t.rank;
    v->d_zeros = t.zeros;
    v->d_node_start = t.node_start;
    v->d_ctrl = c - kCtrlErr;  // so that d_ctrl + kCtrlErr is this tree's error word
    b->views[i] = v;
  }
  // work list: groups (tree, phase) phase by phase
  std::vector<uint32_t> first;
  std::vector<uint2> grp;
  uint32_t items = 0;
  for (uint32_t ph = 0; ph < max_phases; ++ph)
    for (uint32_t i = 0; i < m; ++i) {
      if (ph >= geo[i].phases) continue;
      first.push_back(items);
      grp.push_back(make_uint2(i, ph));
      items += ph == 1 ? 1u : (uint32_t)geo[i].NT;
    }
  first.push_back(items);
  b->n_groups = (uint32_t)grp.size();
  b->n_items = items;
  if ((e = cudaMalloc(&b->d_grp_first, first.size() * 4))) return fail(e);
  if ((e = cudaMalloc(&b->d_grp, grp.size() * sizeof(uint2)))) return fail(e);
  if ((e = cudaMalloc(&b->d_trees, m * sizeof(BTree)))) return fail(e);
  if ((e = cudaMemcpy(b->d_grp_first, first.data(), first.size() * 4, cudaMemcpyHostToDevice))) return fail(e);
  if ((e = cudaMemcpy(b->d_grp, grp.data(), grp.size() * sizeof(uint2), cudaMemcpyHostToDevice))) return fail(e);
  *out = b;
  return WT_OK;
}

int wt_batch_set_inputs(wt_batch *b, const void *const *d_seqs) {
  if (!b || !d_seqs) return WT_ERR_ARG;
  for (uint32_t i = 0; i < b->m; ++i) {
    if (!d_seqs[i] || (reinterpret_cast<uintptr_t>(d_seqs[i]) & 15u)) return WT_ERR_ARG;
    b->host_trees[i].in = static_cast<const uint8_t *>(d_seqs[i]);
  }
  WT_CUDA(cudaMemcpy(b->d_trees, b->host_trees.data(), b->m * sizeof(BTree), cudaMemcpyHostToDevice));
  b->inputs_set = true;
  return WT_OK;
}

int wt_batch_build(wt_batch *b, void *stream) {
  if (!b || !b->inputs_set) return WT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  b->stream = st;
  for (wt_tree *v : b->views) {
    v->stream = st;
    v->sticky_error = 0;
  }
  WT_CUDA(cudaMemsetAsync(b->d_ctrl, 0, b->ctrl_bytes, st));
  BatchArgs a;
  a.trees = b->d_trees;
  a.grp_first = b->d_grp_first;
  a.grp = b->d_grp;
  a.n_groups = b->n_groups;
  a.n_items = b->n_items;
  a.ticket = b->d_ctrl;
  a.spin_limit = b->cfg.spin_limit ? b->cfg.spin_limit : (1u << 22);
  a.err = reinterpret_cast<int *>(b->d_ctrl + 1);
  a.t_start = reinterpret_cast<unsigned long long *>(b->d_ctrl + 2);
  auto launch = [&](auto kern, uint32_t threads, size_t sm) -> int {
    WT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, sm) != cudaSuccess) {
      (void)cudaGetLastError();
      occ = 1;
    }
    occ = std::max(occ, 1);
    if (b->cfg.ctas_per_sm) occ = std::min<int>(occ, (int)b->cfg.ctas_per_sm);
    const int grid = (int)std::min<uint64_t>((uint64_t)occ * b->sms, std::max<uint32_t>(b->n_items, 1));
    kern<<<grid, threads, sm, st>>>(a);
    WT_CUDA(cudaGetLastError());
    return WT_OK;
  };
  if (b->threads == 128) return launch(k_batch<128>, 128, batch_smem_bytes<128>());
  return launch(k_batch<256>, 256, batch_smem_bytes<256>());
}

int wt_batch_sync(wt_batch *b) {
  if (!b) return WT_ERR_ARG;
  WT_CUDA(cudaStreamSynchronize(b->stream));
  int first = 0;
  std::vector<int> errs(b->m);
  for (uint32_t i = 0; i < b->m; ++i) {
    int e = 0;
    WT_CUDA(cudaMemcpy(&e, b->host_trees[i].err, sizeof(int), cudaMemcpyDeviceToHost));
    b->views[i]->sticky_error = e;
    if (e && !first) first = e;
  }
  int be = 0;
  WT_CUDA(cudaMemcpy(&be, b->d_ctrl + 1, sizeof(int), cudaMemcpyDeviceToHost));
  return first ? first : be;
}

int wt_batch_latencies(wt_batch *b, uint64_t *ns) {
  if (!b || !ns) return WT_ERR_ARG;
  WT_CUDA(cudaStreamSynchronize(b->stream));
  unsigned long long t0 = 0;
  WT_CUDA(cudaMemcpy(&t0, b->d_ctrl + 2, 8, cudaMemcpyDeviceToHost));
  for (uint32_t i = 0; i < b->m; ++i) {
    unsigned long long t = 0;
    WT_CUDA(cudaMemcpy(&t, b->host_trees[i].t_done, 8, cudaMemcpyDeviceToHost));
    ns[i] = t >= t0 ? t - t0 : 0;
  }
  return WT_OK;
}

int wt_batch_tree(wt_batch *b, uint32_t i, wt_tree **tree) {
  if (!b || !tree || i >= b->m) return WT_ERR_ARG;
  *tree = b->views[i];
  return WT_OK;
}

int wt_build_batch(const wt_seq_desc *descs, const void *const *d_seqs, uint32_t m,
                   const wt_config *cfg, void *stream, wt_batch **out) {
  int rc = wt_batch_create(descs, m, cfg, out);
  if (rc) return rc;
  if ((rc = wt_batch_set_inputs(*out, d_seqs)) || (rc = wt_batch_build(*out, stream))) {
    wt_batch_free(*out);
    *out = nullptr;
  }
  return rc;
}

}  // extern "C"
