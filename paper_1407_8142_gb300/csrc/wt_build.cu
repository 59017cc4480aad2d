// levelWT construction on one GB300 (sm_103a).
//
// One build (Shun, "Parallel Wavelet Tree Construction", Section 4, Fig. 1,
// restated as global passes over each level's sequence T_l):
//   pre-pass   reads S once: the 2^L-bin symbol histogram, the range check,
//              and the ones of level 0 (bit L-1) per tile.
//   tables     node starts E[v] = #{S[j] < v} by an exclusive scan of the
//              histogram; per level l and node prefix p the ones before the
//              node, O_l[p], and the start of its 1-child.  These replace the
//              per-node prefix-sum totals X_s and the node list A of Fig. 1.
//   split(l)   l = 0..L-2: bits and directory of level l, the ones-before-
//              tile prefix from the tile counts of the previous pass (each
//              pass counts the next level's ones per destination tile), and
//              the stable split of every node into its 0-child and 1-child
//              ranges of T_{l+1} (Fig. 1's X_s + i - X[i] placement, with the
//              prefix sum taken over the whole level instead of per node).
//   leaf       level L-1: bits and directory only; its nodes have range 2 and
//              no children (the early stop of Fig. 1).
//
// Destinations.  For symbol s at position j of T_l, with node prefix
// p = s >> (L-l), bit beta = bit (L-1-l) of s and R(j) = ones of level l
// before j:  beta = 0 -> j - R(j) + O_l[p];  beta = 1 -> E_{l+1}[2p+1] +
// R(j) - O_l[p].  The tables store {O_l[p], E_{l+1}[2p+1] - O_l[p]}.
//
// Wavelet matrix (Section 7): the same passes without histogram and tables;
// every level is one node, so zeros go to j - R(j) and ones to Z_l + R(j),
// Z_l = zeros of level l = n minus the level's ones, which the previous pass
// (or the pre-pass, for level 0) has counted.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>

#include "wt_dev.cuh"
#include "wt_fused.h"
#include "wt_internal.h"

using namespace wtk;

#include "wt_kernels.cuh"

namespace {

// ------------------------------------------------------------------ host side
int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return WT_ERR_OOM;
  return WT_ERR_CUDA;
}

#define WT_CUDA(call)                         \
  do {                                        \
    cudaError_t e__ = (call);                 \
    if (e__ != cudaSuccess) {                 \
      (void)cudaGetLastError();               \
      return cuda_fail(e__);                  \
    }                                         \
  } while (0)

uint32_t levels_of(uint32_t sigma) {
  uint32_t L = 0;
  while ((1ull << L) < sigma) ++L;
  return L;
}

uint32_t tables_blocks(uint32_t L) {
  uint32_t nb = 0;
  for (uint32_t l = 0; l + 1 < L; ++l) nb += ((1u << l) + kScanChunk - 1) / kScanChunk;
  return nb;
}

uint32_t hist_blocks(uint32_t L) { return ((1u << L) + kScanChunk - 1) / kScanChunk; }

template <typename K>
int occupancy(K kernel, int threads, size_t smem, int sms, uint32_t cap) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    occ = 1;
  }
  occ = std::max(occ, 1);
  if (cap) occ = std::min<int>(occ, (int)cap);
  return occ * sms;
}

struct Launcher {
  wt_tree *t;
  cudaStream_t st;
  uint32_t epoch_base;
  uint32_t pass = 0;

  Lookback lb() const {
    Lookback l;
    l.status = t->d_status;
    l.epoch = epoch_base + pass;
    l.spin_limit = spin();
    l.skip = t->cfg.debug_skip_publish;
    l.err = err();
    return l;
  }
  uint32_t spin() const { return t->cfg.spin_limit ? t->cfg.spin_limit : kDefaultSpin; }
  int *err() const { return reinterpret_cast<int *>(t->d_ctrl + kCtrlErr); }
  uint32_t *ticket() const { return t->d_ctrl + pass; }
  TileCounts counts(uint32_t level) const {
    const uint64_t NT = t->NT;
    uint32_t *base = t->d_counts + (uint64_t)level * t->counts_per_level;
    return TileCounts{base, base + NT, base + NT + (NT >> 6) + 1};
  }
  LevelOut out(uint32_t level) const {
    return LevelOut{t->d_bits + (uint64_t)level * t->W, t->d_rank + (uint64_t)level * (t->NB + 1),
                    t->d_zeros + level};
  }

  void before(int kind) {
    if (t->profile && t->n_ev < (int)kMaxProfiled) {
      cudaEventRecord(t->ev[2 * t->n_ev], st);
      t->ev_kind[t->n_ev] = kind;
    }
  }
  void after() {
    if (t->profile && t->n_ev < (int)kMaxProfiled) {
      cudaEventRecord(t->ev[2 * t->n_ev + 1], st);
      ++t->n_ev;
    }
  }
};

template <typename K>
int set_smem(K kern, size_t bytes) {
  if (bytes > 48 * 1024)
    WT_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return WT_OK;
}

// Persistent launch: as many CTAs as fit on the GPU (capped by ctas_per_sm),
// never more than there are tiles.
template <typename K, typename A>
int launch_persistent(Launcher &ln, K kern, int threads, size_t smem, const A &args) {
  wt_tree *t = ln.t;
  if (int rc = set_smem(kern, smem)) return rc;
  const int grid = std::min<int>((int)t->NT, occupancy(kern, threads, smem, t->sms, t->cfg.ctas_per_sm));
  kern<<<std::max(grid, 1), threads, smem, ln.st>>>(args);
  return WT_OK;
}

template <int SB, int THREADS>
int launch_prepass(Launcher &ln, const uint8_t *in, bool in_padded) {
  wt_tree *t = ln.t;
  PrepassArgs a;
  a.in = in;
  a.in_padded = in_padded ? 1 : 0;
  a.n = (uint32_t)t->n;
  a.L = t->L;
  a.NT = (uint32_t)t->NT;
  a.sigma = t->sigma;
  a.hist = t->d_hist;
  a.cnt = ln.counts(0);
  a.ticket = ln.ticket();
  a.spin_limit = ln.spin();
  a.err = ln.err();
  const uint32_t nbins = 1u << t->L;
  ln.before(kPrepass);
  int rc;
  if (t->shape == WT_SHAPE_MATRIX || t->node_counts)
    rc = launch_persistent(ln, k_prepass<SB, THREADS, kHistNone>, THREADS, prepass_smem_bytes<SB, THREADS>(0), a);
  else if (nbins <= kHistLanesMaxBins)
    rc = launch_persistent(ln, k_prepass<SB, THREADS, kHistLanes>, THREADS,
                           prepass_smem_bytes<SB, THREADS>(hist_smem_words(kHistLanes, nbins)), a);
  else if (nbins <= kHistSmemMaxBins)
    rc = launch_persistent(ln, k_prepass<SB, THREADS, kHistSmem>, THREADS,
                           prepass_smem_bytes<SB, THREADS>(hist_smem_words(kHistSmem, nbins)), a);
  else
    rc = launch_persistent(ln, k_prepass<SB, THREADS, kHistGlobal>, THREADS,
                           prepass_smem_bytes<SB, THREADS>(hist_smem_words(kHistGlobal, nbins)), a);
  if (rc) return rc;
  ln.after();
  ++ln.pass;
  WT_CUDA(cudaGetLastError());
  return WT_OK;
}

template <int SB, int THREADS>
int launch_leaf(Launcher &ln, const uint8_t *in, bool in_padded, uint32_t level) {
  wt_tree *t = ln.t;
  LeafArgs a;
  a.in = in;
  a.in_padded = in_padded ? 1 : 0;
  a.n = (uint32_t)t->n;
  a.L = t->L;
  a.NT = (uint32_t)t->NT;
  a.NB = (uint32_t)t->NB;
  a.W = t->W;
  a.out = ln.out(level);
  a.cnt = ln.counts(level);
  a.ticket = ln.ticket();
  a.spin_limit = ln.spin();
  a.err = ln.err();
  auto kern = k_leaf<SB, THREADS>;
  constexpr size_t sm = leaf_smem_bytes<SB, THREADS>();
  if (int rc = set_smem(kern, sm)) return rc;
  const int grid = std::min<int>((int)t->NT, occupancy(kern, THREADS, sm, t->sms, t->cfg.ctas_per_sm));
  ln.before(kLeaf);
  kern<<<std::max(grid, 1), THREADS, sm, ln.st>>>(a);
  ln.after();
  ++ln.pass;
  WT_CUDA(cudaGetLastError());
  return WT_OK;
}

// Whether the pass over `level` computes that level's node table itself
// (SplitArgs::node_ones): node counts, one level per pass, and at most one
// node per thread of the pass's CTA with the table in shared memory (CTA
// and table sizes as chosen by launch_split and launch_lastpair); the
// node-table kernel of the level is then not launched.
bool tables_in_pass(const wt_tree *t, uint32_t level) {
  if (!t->node_counts || t->fuse_k != 1 || level == 0) return false;
  const uint32_t cta = (t->sb == 1 && t->threads == 512) ? 256u : t->threads;
  const uint32_t smem_nodes = t->sb == 1 ? 128u : 1024u;
  return (1ull << level) <= std::min(cta, smem_nodes);
}

// Set the node-table fields of a pass's arguments (none if the level's
// table comes from the node-table kernel or the level has one node).
void set_pass_tables(const wt_tree *t, uint32_t level, SplitArgs &a) {
  const bool own = tables_in_pass(t, level);
  a.node_ones = own ? t->d_hist + ((1u << level) - 1) : nullptr;
  a.tab_prev = own ? t->d_tab + ((1u << (level - 1)) - 1) : nullptr;
  a.tab_w = own ? t->d_tab + ((1u << level) - 1) : nullptr;
  a.E = own ? t->d_node_start : nullptr;
}

template <int SB, int THREADS>
int launch_split(Launcher &ln, const uint8_t *in, bool in_padded, uint8_t *out, uint32_t level) {
  wt_tree *t = ln.t;
  SplitArgs a;
  a.in = in;
  a.out = out;
  a.in_padded = in_padded ? 1 : 0;
  a.n = (uint32_t)t->n;
  a.L = t->L;
  a.level = level;
  a.NT = (uint32_t)t->NT;
  a.NB = (uint32_t)t->NB;
  a.log2T = 5 + (uint32_t)__builtin_ctz(THREADS);
  a.W = t->W;
  const bool matrix = t->shape == WT_SHAPE_MATRIX;
  // one node whose table comes from the tile counts: the matrix, and level 0
  // of a tree whose tables come from node counts
  const bool count_table = matrix || (t->node_counts && level == 0);
  a.tab = count_table ? nullptr : t->d_tab + ((1u << level) - 1);
  a.pshift = matrix ? t->L : t->L - level;
  a.count_table = count_table ? 1 : 0;
  a.tab_out = (t->node_counts && level == 0) ? t->d_tab : nullptr;
  a.nones_next = t->node_counts ? t->d_hist + ((2u << level) - 1) : nullptr;
  set_pass_tables(t, level, a);
  a.lo = ln.out(level);
  a.cin = ln.counts(level);
  a.cout = ln.counts(level + 1);
  a.ticket = ln.ticket();
  a.spin_limit = ln.spin();
  a.err = ln.err();
  // 4-byte symbols: one input buffer (see TilePipe), more CTAs per SM.
  // 1-byte symbols in tiles of 16384: 256 threads of 64 symbols each, so
  // that every warp's fixed per-tile work is spread over 2048 symbols.
  constexpr int DEPTH = SB == 4 ? 1 : 2;
  constexpr int WPT = (SB == 1 && THREADS == 512) ? 2 : 1;
  constexpr int CTA = THREADS / WPT;
  auto kern = t->node_counts ? k_split<SB, CTA, true, DEPTH, WPT> : k_split<SB, CTA, false, DEPTH, WPT>;
  constexpr uint32_t sm = split_smem_bytes<SB, CTA, DEPTH, WPT>();
  if (int rc = set_smem(kern, sm)) return rc;
  const int grid = std::min<int>((int)t->NT, occupancy(kern, CTA, sm, t->sms, t->cfg.ctas_per_sm));
  ln.before(kSplit);
  kern<<<std::max(grid, 1), CTA, sm, ln.st>>>(a);
  ln.after();
  ++ln.pass;
  WT_CUDA(cudaGetLastError());
  return WT_OK;
}

// Levels L-2 and L-1 in one pass over T_{L-2} (k_lastpair): the arguments
// of the split pass over level L-2, and level L-1's row, zeroed first.
template <int SB, int THREADS>
int launch_lastpair(Launcher &ln, const uint8_t *in, bool in_padded) {
  wt_tree *t = ln.t;
  const uint32_t level = t->L - 2;
  LastPairArgs la;
  SplitArgs &a = la.s;
  a.in = in;
  a.out = nullptr;
  a.in_padded = in_padded ? 1 : 0;
  a.n = (uint32_t)t->n;
  a.L = t->L;
  a.level = level;
  a.NT = (uint32_t)t->NT;
  a.NB = (uint32_t)t->NB;
  a.log2T = 5 + (uint32_t)__builtin_ctz(THREADS);
  a.W = t->W;
  const bool matrix = t->shape == WT_SHAPE_MATRIX;
  const bool count_table = matrix || (t->node_counts && level == 0);
  a.tab = count_table ? nullptr : t->d_tab + ((1u << level) - 1);
  a.pshift = matrix ? t->L : t->L - level;
  a.count_table = count_table ? 1 : 0;
  a.tab_out = (t->node_counts && level == 0) ? t->d_tab : nullptr;
  a.nones_next = t->node_counts ? t->d_hist + ((2u << level) - 1) : nullptr;
  set_pass_tables(t, level, a);
  a.lo = ln.out(level);
  a.cin = ln.counts(level);
  a.cout = ln.counts(level);  // unused: no T_{L-1}
  a.ticket = ln.ticket();
  a.spin_limit = ln.spin();
  a.err = ln.err();
  la.row_next = t->d_bits + (uint64_t)(level + 1) * t->W;
  WT_CUDA(cudaMemsetAsync(la.row_next, 0, t->W * 4, ln.st));
  constexpr int WPT = (SB == 1 && THREADS == 512) ? 2 : 1;
  constexpr int CTA = THREADS / WPT;
  auto kern = t->node_counts ? k_lastpair<SB, CTA, true, WPT> : k_lastpair<SB, CTA, false, WPT>;
  constexpr uint32_t sm = lastpair_smem_bytes<SB, CTA, WPT>();
  if (int rc = set_smem(kern, sm)) return rc;
  const int grid = std::min<int>((int)t->NT, occupancy(kern, CTA, sm, t->sms, t->cfg.ctas_per_sm));
  ln.before(kLastPair);
  kern<<<std::max(grid, 1), CTA, sm, ln.st>>>(la);
  ln.after();
  ++ln.pass;
  WT_CUDA(cudaGetLastError());
  return WT_OK;
}

// Whether the build takes its last two levels in one pass: when the nodes of
// level L-2 are long (64 Ki symbols on average), so that almost every warp
// lies in one node and writes its level-(L-1) bits as two runs.
bool use_lastpair(const wt_tree *t) {
  return t->fuse_k == 1 && t->L >= 2 && (t->n >> (t->L - 2)) >= (1ull << 16);
}

// Node starts E[v] = symbols whose top log2(nbins) bits are < v.
int launch_hist_scan(Launcher &ln, uint32_t nbins) {
  wt_tree *t = ln.t;
  ScanArgs a;
  a.hist = t->d_hist;
  a.E = t->d_node_start;
  a.nbins = nbins;
  a.nblocks = (nbins + kScanChunk - 1) / kScanChunk;
  a.ticket = ln.ticket();
  a.lb = ln.lb();
  ln.before(kHistScan);
  k_hist_scan<<<a.nblocks, kScanThreads, 0, ln.st>>>(a);
  ln.after();
  ++ln.pass;
  WT_CUDA(cudaGetLastError());
  return WT_OK;
}

// Level tables of every level from the node starts of level L.
int launch_level_tables(Launcher &ln) {
  wt_tree *t = ln.t;
  const uint32_t nb = tables_blocks(t->L);
  if (nb) {
    TabArgs a;
    a.E = t->d_node_start;
    a.tab = t->d_tab;
    a.L = t->L;
    a.nblocks = nb;
    a.ticket = ln.ticket();
    a.lb = ln.lb();
    ln.before(kTables);
    k_level_tables<<<nb, kScanThreads, 0, ln.st>>>(a);
    ln.after();
    WT_CUDA(cudaGetLastError());
  }
  ++ln.pass;
  return WT_OK;
}

int launch_tables(Launcher &ln) {
  if (int rc = launch_hist_scan(ln, 1u << ln.t->L)) return rc;
  return launch_level_tables(ln);
}

// Tables of level m (1 <= m <= L-2) from the node counts of the previous
// split pass; m = L-1: node starts of the last two levels only.
int launch_node_tables(Launcher &ln, uint32_t m) {
  wt_tree *t = ln.t;
  const uint32_t L = t->L;
  const uint2 *tab_prev = t->d_tab + ((1u << (m - 1)) - 1);
  const uint32_t *ones = t->d_hist + ((1u << m) - 1);
  if (m + 1 < L) {
    NodeTabArgs a;
    a.ones = ones;
    a.tab_prev = tab_prev;
    a.tab = t->d_tab + ((1u << m) - 1);
    a.E = t->d_node_start;
    a.L = L;
    a.m = m;
    a.n = (uint32_t)t->n;
    a.nblocks = ((1u << m) + kScanChunk - 1) / kScanChunk;
    a.ticket = ln.ticket();
    a.lb = ln.lb();
    ln.before(kTables);
    k_node_tables<<<a.nblocks, kScanThreads, 0, ln.st>>>(a);
  } else {
    LeafStartArgs a;
    a.ones = ones;
    a.tab_prev = tab_prev;
    a.E = t->d_node_start;
    a.L = L;
    a.n = (uint32_t)t->n;
    const uint32_t cnt = 1u << (L - 1);
    ln.before(kHistScan);
    k_leaf_starts<<<std::min<uint32_t>((cnt + 255) / 256, 4096u), 256, 0, ln.st>>>(a);
  }
  ln.after();
  ++ln.pass;
  WT_CUDA(cudaGetLastError());
  return WT_OK;
}

// k levels per pass (L >= 1).  No pre-pass: the first pass's count kernel
// checks the symbol range.  Per pass over T_l with K levels: the digit
// counts of its tiles and their scan; for the tree also the node counts of
// level l+K (gathered by the count kernel), their scan into node starts and
// the F tables of levels l+1..l+K; the zeroing of its inner rows, the
// k-level pass and the directories of its rows.  The tree's level tables
// (used by the queries) come last, from the node starts of level L.
template <int SB, int THREADS>
int run_build_fused(wt_tree *t, const uint8_t *seq, bool seq_padded, cudaStream_t st) {
  Launcher ln{t, st, (t->build_count * kPasses) & kEpochMask};
  int rc;
  const bool tree = t->shape == WT_SHAPE_TREE;
  const uint8_t *in = seq;
  bool padded = seq_padded;
  for (uint32_t l = 0, j = 0; l < t->L; ++j) {
    const uint32_t K = std::min(t->fuse_k, t->L - l);
    const uint32_t top = l + K;
    const bool last = top == t->L;
    if (tree) WT_CUDA(cudaMemsetAsync(t->d_hist, 0, (4ull << top), st));
    ln.before(kTileCount);
    if ((rc = fused_count(t, st, in, l, K, l == 0))) return rc;
    ln.after();
    ln.before(kTileScan);
    if ((rc = fused_scan(t, st, l, K))) return rc;
    ln.after();
    if (tree) {
      if ((rc = launch_hist_scan(ln, 1u << top))) return rc;
      const uint32_t m_hi = std::min(top, t->L - 1);
      if (m_hi >= l + 1) {
        ln.before(kTables);
        if ((rc = fused_tables(t, st, l + 1, m_hi, top, ln.lb(), ln.ticket()))) return rc;
        ln.after();
        ++ln.pass;
      }
    }
    if (K > 1) WT_CUDA(cudaMemsetAsync(t->d_bits + (uint64_t)(l + 1) * t->W, 0, (uint64_t)(K - 1) * t->W * 4, st));
    uint8_t *out = last ? nullptr : static_cast<uint8_t *>(t->d_buf[j & 1]);
    ln.before(kFused);
    if ((rc = fused_pass(t, st, in, padded, out, l, K, ln.ticket()))) return rc;
    ln.after();
    ++ln.pass;
    ln.before(kDirectory);
    if ((rc = fused_dir(t, st, l, K, ln.lb(), ln.ticket()))) return rc;
    ln.after();
    ++ln.pass;
    if (t->record_levels)
      for (uint32_t m = l; m < l + K; ++m) WT_CUDA(cudaEventRecord(t->level_ev[m], st));
    in = out;
    padded = true;
    l += K;
  }
  if (tree && (rc = launch_level_tables(ln))) return rc;
  return WT_OK;
}

template <int SB, int THREADS>
int run_build(wt_tree *t, const uint8_t *seq, bool seq_padded, cudaStream_t st) {
  if (t->fuse_k > 1 && t->L >= 1) return run_build_fused<SB, THREADS>(t, seq, seq_padded, st);
  Launcher ln{t, st, (t->build_count * kPasses) & kEpochMask};
  int rc;
  if ((rc = launch_prepass<SB, THREADS>(ln, seq, seq_padded))) return rc;
  if (t->shape == WT_SHAPE_TREE && !t->node_counts && (rc = launch_tables(ln))) return rc;
  if (t->L == 0) return WT_OK;
  const uint8_t *in = seq;
  bool padded = seq_padded;
  const bool pair = use_lastpair(t);
  const uint32_t last_split = pair ? t->L - 2 : t->L - 1;  // levels below it take one split pass each
  for (uint32_t l = 0; l < last_split; ++l) {
    // with node counts, the tables of level l come from the pass over l-1
    if (t->node_counts && l >= 1 && !tables_in_pass(t, l) && (rc = launch_node_tables(ln, l))) return rc;
    uint8_t *out = static_cast<uint8_t *>(t->d_buf[l & 1]);
    if ((rc = launch_split<SB, THREADS>(ln, in, padded, out, l))) return rc;
    if (t->record_levels) WT_CUDA(cudaEventRecord(t->level_ev[l], st));  // level l's rows are final
    in = out;
    padded = true;
  }
  if (pair) {
    const uint32_t m = t->L - 2;
    if (t->node_counts && m >= 1 && !tables_in_pass(t, m) && (rc = launch_node_tables(ln, m))) return rc;
    if ((rc = launch_lastpair<SB, THREADS>(ln, in, padded))) return rc;
    if (t->record_levels) WT_CUDA(cudaEventRecord(t->level_ev[m], st));
    if (t->node_counts && (rc = launch_node_tables(ln, t->L - 1))) return rc;
    ln.before(kDirectory);
    rc = fused_dir(t, st, t->L - 1, 1, ln.lb(), ln.ticket());
    ln.after();
    ++ln.pass;
    if (rc) return rc;
  } else {
    if (t->node_counts && (rc = launch_node_tables(ln, t->L - 1))) return rc;
    if ((rc = launch_leaf<SB, THREADS>(ln, in, padded, t->L - 1))) return rc;
  }
  if (t->record_levels) WT_CUDA(cudaEventRecord(t->level_ev[t->L - 1], st));
  return WT_OK;
}

template <int SB>
int run_build_sb(wt_tree *t, const uint8_t *seq, bool padded, cudaStream_t st) {
  switch (t->threads) {
    case 128: return run_build<SB, 128>(t, seq, padded, st);
    case 256: return run_build<SB, 256>(t, seq, padded, st);
    case 512: return run_build<SB, 512>(t, seq, padded, st);
  }
  return WT_ERR_ARG;
}

void release(wt_tree *t) {
  cudaFree(t->d_bits);
  cudaFree(t->d_rank);
  cudaFree(t->d_zeros);
  cudaFree(t->d_node_start);
  cudaFree(t->d_tab);
  cudaFree(t->d_ftab);
  cudaFree(t->d_fcount);
  cudaFree(t->d_ctrl);
  cudaFree(t->d_buf[0]);
  cudaFree(t->d_buf[1]);
  cudaFree(t->d_status);
  cudaFree(t->d_in_host);
  if (t->copy_stream) {
    cudaStreamSynchronize(t->copy_stream);
    cudaStreamDestroy(t->copy_stream);
    for (uint32_t l = 0; l < kMaxLevels; ++l)
      if (t->level_ev[l]) cudaEventDestroy(t->level_ev[l]);
    if (t->copy_done) cudaEventDestroy(t->copy_done);
  }
  if (t->ev) {
    for (uint32_t i = 0; i < 2 * kMaxProfiled; ++i)
      if (t->ev[i]) cudaEventDestroy(t->ev[i]);
    delete[] t->ev;
    delete[] t->ev_kind;
  }
}

uint32_t pick_threads(uint64_t n, uint32_t sb, int sms, uint32_t requested) {
  if (requested == 128 || requested == 256 || requested == 512) return requested;
  // the largest tile that still gives every SM two tiles; 128 threads below that
  for (uint32_t th : {512u, 256u}) {
    if (sb == 4 && th == 512) continue;  // 64 KB tiles leave one CTA per SM
    if ((n + 32ull * th - 1) / (32ull * th) >= 2ull * (uint64_t)sms) return th;
  }
  return 128;
}

// Levels per pass when the caller leaves the choice to the library, as
// measured on GB300: four for 4-byte symbols, at least 8 levels and
// n >= 2^22 (the one-level pass runs near the copy bandwidth there, so
// reading and writing the symbols once per four levels pays; config 3:
// tree 9.46 ms against 9.91 ms, wavelet matrix 7.37 ms against 7.90 ms);
// one everywhere else (at 1-byte symbols the one-level pass is bound by
// instruction issue, not by memory; short sequences are bound by launch
// latency, and a k-level pass takes six launches).
uint32_t auto_levels_per_pass(uint32_t shape, uint32_t symbol_bytes, uint32_t L, uint64_t n) {
  (void)shape;
  return (symbol_bytes == 4 && L >= 8 && n >= (1ull << 22)) ? 4u : 1u;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

}  // extern "C"

namespace wtk {

int tree_shape(wt_tree *t, uint64_t n, uint32_t sigma, uint32_t symbol_bytes, const wt_config *cfg,
               uint32_t shape) {
  if (!(symbol_bytes == 1 || symbol_bytes == 2 || symbol_bytes == 4)) return WT_ERR_ARG;
  if (sigma == 0 || (uint64_t)sigma > (1ull << (8 * symbol_bytes))) return WT_ERR_ARG;
  if (n >= (1ull << 32)) return WT_ERR_ARG;
  const uint32_t L = levels_of(sigma);
  if (L > kMaxLevels) return WT_ERR_ARG;
  if (cfg && cfg->tile_threads && !(cfg->tile_threads == 128 || cfg->tile_threads == 256 ||
                                    cfg->tile_threads == 512))
    return WT_ERR_ARG;
  if (cfg && cfg->levels_per_pass > kMaxLevelsPerPass) return WT_ERR_ARG;
  if (cfg) t->cfg = *cfg;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return WT_ERR_CUDA;
  }
  t->n = n;
  t->cap_n = n;
  t->sigma = sigma;
  t->sb = symbol_bytes;
  t->L = L;
  t->shape = shape;
  // per-node counts kept by the split passes replace the 2^L-bin histogram:
  // for large alphabets, whose global histogram atomics serialise on hot
  // symbols, and for long sequences, where the histogram's shared-memory
  // atomics cost the pre-pass more than one small table kernel per level
  // costs; short sequences of small alphabets keep it (fewer launches)
  t->fuse_k = t->cfg.levels_per_pass ? t->cfg.levels_per_pass : auto_levels_per_pass(shape, symbol_bytes, L, n);
  // the k-level passes of a tree take their tables from the histogram
  t->node_counts = shape == WT_SHAPE_TREE && L >= 2 && t->fuse_k == 1 &&
                   ((1ull << L) > kHistSmemMaxBins || n >= (1ull << 24));
  t->NB = (n + 511) / 512;
  t->W = 16 * t->NB;
  t->threads = pick_threads(n, symbol_bytes, t->sms, t->cfg.tile_threads);
  t->T = 32ull * t->threads;
  t->NT = std::max<uint64_t>(1, (n + t->T - 1) / t->T);
  t->tile_f = fused_tile_symbols(symbol_bytes);
  t->NTf = std::max<uint64_t>(1, (n + t->tile_f - 1) / t->tile_f);
  const bool tree = shape == WT_SHAPE_TREE;
  // histogram words: the tree's 2^L bins, or the matrix's digit counts of its k-level passes
  const uint64_t hist_words = tree ? 1ull << L : (t->fuse_k > 1 ? 256 : 0);
  const uint64_t Lz = std::max<uint32_t>(L, 1);
  t->counts_per_level = t->NT + (t->NT >> 6) + 1 + (t->NT >> 12) + 1;
  t->ctrl_words = kCtrlWords + hist_words + Lz * t->counts_per_level;
  // whole tiles of either schedule
  t->buf_bytes = std::max(t->NT * t->T, t->NTf * t->tile_f) * symbol_bytes + 16;
  t->status_n = std::max<uint64_t>({t->NT, (uint64_t)hist_blocks(L), (uint64_t)tables_blocks(L), 1});
  if (t->fuse_k > 1)
    t->status_n = std::max<uint64_t>({t->status_n, (uint64_t)fused_tables_blocks(L, t->fuse_k),
                                      (uint64_t)t->fuse_k * fused_dir_chunks(t->NB)});
  return WT_OK;
}

TreeLayout tree_layout(const wt_tree *t) {
  TreeLayout ly{};
  const bool tree = t->shape == WT_SHAPE_TREE;
  const uint64_t nbins = tree ? 1ull << t->L : 0;
  const size_t Lz = std::max<uint32_t>(t->L, 1);
  ly.bits = std::max<size_t>(4, Lz * t->W * 4);
  ly.rank = Lz * (t->NB + 1) * 8;
  ly.zeros = Lz * 8;
  if (tree) {
    ly.node_start = (nbins + 1) * 8;
    ly.tab = std::max<uint64_t>(1, nbins / 2) * sizeof(uint2);
    if (t->fuse_k > 1 && t->L >= 2) ly.ftab = nbins * 4;
  }
  if (t->fuse_k > 1) ly.fcount = (2 * t->NTf << t->fuse_k) * 4;
  ly.ctrl = t->ctrl_words * 4;
  ly.buf = t->L >= 2 ? t->buf_bytes : 0;
  ly.status = t->status_n * 8;
  return ly;
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

size_t tree_region_bytes(const TreeLayout &ly) {
  return al256(ly.bits) + al256(ly.rank) + al256(ly.zeros) + al256(ly.node_start) + al256(ly.tab) +
         al256(ly.ftab) + al256(ly.fcount) + al256(ly.ctrl) + 2 * al256(ly.buf) + al256(ly.status);
}

void tree_bind_derived(wt_tree *t) {
  const uint64_t hist_words = t->shape == WT_SHAPE_TREE ? 1ull << t->L : (t->fuse_k > 1 ? 256 : 0);
  t->d_hist = t->d_ctrl + kCtrlWords;
  t->d_counts = t->d_hist + hist_words;
}

void tree_bind(wt_tree *t, const TreeLayout &ly, unsigned char *base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> unsigned char * {
    if (!bytes) return nullptr;
    unsigned char *p = base + off;
    off += al256(bytes);
    return p;
  };
  t->d_bits = reinterpret_cast<uint32_t *>(take(ly.bits));
  t->d_rank = reinterpret_cast<unsigned long long *>(take(ly.rank));
  t->d_zeros = reinterpret_cast<unsigned long long *>(take(ly.zeros));
  t->d_node_start = reinterpret_cast<unsigned long long *>(take(ly.node_start));
  t->d_tab = reinterpret_cast<uint2 *>(take(ly.tab));
  t->d_ftab = reinterpret_cast<uint32_t *>(take(ly.ftab));
  t->d_fcount = reinterpret_cast<uint32_t *>(take(ly.fcount));
  t->d_ctrl = reinterpret_cast<uint32_t *>(take(ly.ctrl));
  t->d_buf[0] = take(ly.buf);
  t->d_buf[1] = take(ly.buf);
  t->d_status = reinterpret_cast<unsigned long long *>(take(ly.status));
  tree_bind_derived(t);
}

}  // namespace wtk

namespace {

int create_shape(uint64_t n, uint32_t sigma, uint32_t symbol_bytes, const wt_config *cfg,
                 uint32_t shape, wt_tree **out) {
  if (!out) return WT_ERR_ARG;
  *out = nullptr;
  wt_tree *t = new (std::nothrow) wt_tree();
  if (!t) return WT_ERR_OOM;
  if (int rc = tree_shape(t, n, sigma, symbol_bytes, cfg, shape)) {
    delete t;
    return rc;
  }
  auto fail = [&](cudaError_t e) {
    (void)cudaGetLastError();
    release(t);
    delete t;
    return cuda_fail(e);
  };
  const TreeLayout ly = tree_layout(t);
  cudaError_t e;
  if ((e = cudaMalloc(&t->d_bits, ly.bits))) return fail(e);
  if ((e = cudaMalloc(&t->d_rank, ly.rank))) return fail(e);
  if ((e = cudaMalloc(&t->d_zeros, ly.zeros))) return fail(e);
  if (ly.node_start && (e = cudaMalloc(&t->d_node_start, ly.node_start))) return fail(e);
  if (ly.tab && (e = cudaMalloc(&t->d_tab, ly.tab))) return fail(e);
  if (ly.ftab && (e = cudaMalloc(&t->d_ftab, ly.ftab))) return fail(e);
  if (ly.fcount && (e = cudaMalloc(&t->d_fcount, ly.fcount))) return fail(e);
  if ((e = cudaMalloc(&t->d_ctrl, ly.ctrl))) return fail(e);
  if (ly.buf) {
    if ((e = cudaMalloc(&t->d_buf[0], ly.buf))) return fail(e);
    if ((e = cudaMalloc(&t->d_buf[1], ly.buf))) return fail(e);
  }
  if ((e = cudaMalloc(&t->d_status, ly.status))) return fail(e);
  tree_bind_derived(t);
  if ((e = cudaMemset(t->d_status, 0, ly.status))) return fail(e);
  if ((e = cudaMemset(t->d_zeros, 0, ly.zeros))) return fail(e);
  if ((e = cudaMemset(t->d_rank, 0, ly.rank))) return fail(e);
  *out = t;
  return WT_OK;
}

}  // namespace

extern "C" {

int wt_create(uint64_t n, uint32_t sigma, uint32_t symbol_bytes, const wt_config *cfg,
              wt_tree **out) {
  return create_shape(n, sigma, symbol_bytes, cfg, WT_SHAPE_TREE, out);
}

int wt_matrix_create(uint64_t n, uint32_t sigma, uint32_t symbol_bytes, const wt_config *cfg,
                     wt_tree **out) {
  return create_shape(n, sigma, symbol_bytes, cfg, WT_SHAPE_MATRIX, out);
}

int wt_rebuild(wt_tree *t, const void *d_seq, void *stream) {
  if (!t || (!d_seq && t->n) || t->owner) return WT_ERR_ARG;
  return wtk::tree_rebuild(t, d_seq, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace wtk {

int tree_rebuild(wt_tree *t, const void *d_seq, cudaStream_t st) {
  if (!t || (!d_seq && t->n)) return WT_ERR_ARG;
  t->stream = st;
  t->sticky_error = 0;
  ++t->build_count;
  const uint64_t nbins = 1ull << t->L;
  WT_CUDA(cudaMemsetAsync(t->d_ctrl, 0, t->ctrl_words * 4, st));
  const uint8_t *seq = static_cast<const uint8_t *>(d_seq);
  bool padded = false;
  if (t->n && (reinterpret_cast<uintptr_t>(seq) & 15u)) {
    // TMA and vector loads need 16-byte alignment: stage the input.
    void *dst = t->L >= 2 ? t->d_buf[1] : nullptr;
    if (!dst) {
      if (!t->d_in_host) WT_CUDA(cudaMalloc(&t->d_in_host, t->buf_bytes));
      dst = t->d_in_host;
    }
    WT_CUDA(cudaMemcpyAsync(dst, seq, t->n * t->sb, cudaMemcpyDeviceToDevice, st));
    seq = static_cast<const uint8_t *>(dst);
    padded = true;  // scratch buffers hold whole tiles
  }
  if (seq == t->d_in_host) padded = true;
  if (t->n == 0) {
    // nothing to scan: zero bits/directories are already in place; node
    // starts are all zero
    if (t->d_node_start) WT_CUDA(cudaMemsetAsync(t->d_node_start, 0, (nbins + 1) * 8, st));
    return WT_OK;
  }
  switch (t->sb) {
    case 1: return run_build_sb<1>(t, seq, padded, st);
    case 2: return run_build_sb<2>(t, seq, padded, st);
    case 4: return run_build_sb<4>(t, seq, padded, st);
  }
  return WT_ERR_ARG;
}

}  // namespace wtk

extern "C" {

int wt_build_ex(const void *d_seq, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
                const wt_config *cfg, void *stream, wt_tree **out) {
  int rc = wt_create(n, sigma, symbol_bytes, cfg, out);
  if (rc) return rc;
  rc = wt_rebuild(*out, d_seq, stream);
  if (rc) {
    wt_free(*out);
    *out = nullptr;
  }
  return rc;
}

int wt_build(const void *d_seq, uint64_t n, uint32_t sigma, uint32_t symbol_bytes, void *stream,
             wt_tree **out) {
  return wt_build_ex(d_seq, n, sigma, symbol_bytes, nullptr, stream, out);
}

int wt_matrix_build(const void *d_seq, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
                    const wt_config *cfg, void *stream, wt_tree **out) {
  int rc = wt_matrix_create(n, sigma, symbol_bytes, cfg, out);
  if (rc) return rc;
  rc = wt_rebuild(*out, d_seq, stream);
  if (rc) {
    wt_free(*out);
    *out = nullptr;
  }
  return rc;
}

int wt_sync(wt_tree *t) {
  if (!t) return WT_ERR_ARG;
  WT_CUDA(cudaStreamSynchronize(t->stream));
  int err = 0;
  WT_CUDA(cudaMemcpy(&err, t->d_ctrl + kCtrlErr, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) t->sticky_error = err;
  return t->sticky_error;
}

int wt_build_host_async(wt_tree *t, const void *h_seq, uint32_t *h_bits, uint64_t *h_rank,
                        void *stream) {
  if (!t || (!h_seq && t->n) || t->owner) return WT_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!t->d_in_host) WT_CUDA(cudaMalloc(&t->d_in_host, t->buf_bytes));
  const uint32_t L = t->L;
  const bool copy_out = t->n && L && (h_bits || h_rank);
  if (copy_out && !t->copy_stream) {
    WT_CUDA(cudaStreamCreateWithFlags(&t->copy_stream, cudaStreamNonBlocking));
    WT_CUDA(cudaEventCreateWithFlags(&t->copy_done, cudaEventDisableTiming));
    for (uint32_t l = 0; l < L; ++l) WT_CUDA(cudaEventCreateWithFlags(&t->level_ev[l], cudaEventDisableTiming));
  }
  if (t->n) WT_CUDA(cudaMemcpyAsync(t->d_in_host, h_seq, t->n * t->sb, cudaMemcpyHostToDevice, st));
  // each level's bitmap and directory rows are copied out while the later
  // levels are still being built
  t->record_levels = copy_out;
  int rc = wt_rebuild(t, t->d_in_host, stream);
  t->record_levels = false;
  if (rc) return rc;
  if (copy_out) {
    for (uint32_t l = 0; l < L; ++l) {
      WT_CUDA(cudaStreamWaitEvent(t->copy_stream, t->level_ev[l], 0));
      if (h_bits && t->W)
        WT_CUDA(cudaMemcpyAsync(h_bits + (uint64_t)l * t->W, t->d_bits + (uint64_t)l * t->W, t->W * 4,
                                cudaMemcpyDeviceToHost, t->copy_stream));
      if (h_rank)
        WT_CUDA(cudaMemcpyAsync(h_rank + (uint64_t)l * (t->NB + 1), t->d_rank + (uint64_t)l * (t->NB + 1),
                                (t->NB + 1) * 8, cudaMemcpyDeviceToHost, t->copy_stream));
    }
    // later work on `stream` (the next build, wt_sync) waits for the copies
    WT_CUDA(cudaEventRecord(t->copy_done, t->copy_stream));
    WT_CUDA(cudaStreamWaitEvent(st, t->copy_done, 0));
  }
  return WT_OK;
}

int wt_build_host(wt_tree *t, const void *h_seq, uint32_t *h_bits, uint64_t *h_rank,
                  void *stream) {
  const int rc = wt_build_host_async(t, h_seq, h_bits, h_rank, stream);
  if (rc) return rc;
  return wt_sync(t);
}

int wt_resize(wt_tree *t, uint64_t n) {
  if (!t || t->owner || n > t->cap_n) return WT_ERR_ARG;
  // every size below grows with n at a fixed tile size, so the buffers
  // allocated for cap_n hold them; the schedule chosen at creation (tile
  // size, levels per pass, node counts) is kept: it builds any n
  t->n = n;
  t->NB = (n + 511) / 512;
  t->W = 16 * t->NB;
  t->NT = std::max<uint64_t>(1, (n + t->T - 1) / t->T);
  t->NTf = std::max<uint64_t>(1, (n + t->tile_f - 1) / t->tile_f);
  t->counts_per_level = t->NT + (t->NT >> 6) + 1 + (t->NT >> 12) + 1;
  const bool tree = t->shape == WT_SHAPE_TREE;
  const uint64_t hist_words = tree ? (1ull << t->L) : (t->fuse_k > 1 ? 256 : 0);
  const uint64_t Lz = std::max<uint32_t>(t->L, 1);
  t->ctrl_words = kCtrlWords + hist_words + Lz * t->counts_per_level;
  ++t->build_count;  // the contents (and any query index) belong to the old n
  t->sticky_error = 0;
  if (n == 0) {
    // an empty build leaves the directories as they are: they must read 0
    WT_CUDA(cudaMemset(t->d_rank, 0, Lz * 8));
    WT_CUDA(cudaMemset(t->d_zeros, 0, Lz * 8));
  }
  return WT_OK;
}

int wt_info(const wt_tree *t, wt_info_t *info) {
  if (!t || !info) return WT_ERR_ARG;
  info->n = t->n;
  info->sigma = t->sigma;
  info->symbol_bytes = t->sb;
  info->levels = t->L;
  info->shape = t->shape;
  info->words_per_level = t->W;
  info->blocks = t->NB;
  info->d_bits = t->d_bits;
  info->d_rank = reinterpret_cast<uint64_t *>(t->d_rank);
  info->d_zeros = reinterpret_cast<uint64_t *>(t->d_zeros);
  info->d_node_start = reinterpret_cast<uint64_t *>(t->d_node_start);
  info->levels_per_pass = t->fuse_k;
  return WT_OK;
}

int wt_profile(wt_tree *t, int enable) {
  if (!t) return WT_ERR_ARG;
  if (enable && !t->ev) {
    t->ev = new (std::nothrow) cudaEvent_t[2 * kMaxProfiled]();
    t->ev_kind = new (std::nothrow) int32_t[kMaxProfiled]();
    if (!t->ev || !t->ev_kind) return WT_ERR_OOM;
    for (uint32_t i = 0; i < 2 * kMaxProfiled; ++i) WT_CUDA(cudaEventCreate(&t->ev[i]));
  }
  t->profile = enable != 0;
  t->n_ev = 0;
  return WT_OK;
}

int wt_profile_read(wt_tree *t, float *ms, int32_t *kind, int32_t cap) {
  if (!t) return WT_ERR_ARG;
  if (!t->ev) return 0;
  const int n = t->n_ev;
  for (int i = 0; i < n && i < cap; ++i) {
    float v = 0.f;
    if (cudaEventElapsedTime(&v, t->ev[2 * i], t->ev[2 * i + 1]) != cudaSuccess) {
      (void)cudaGetLastError();
      v = -1.f;
    }
    if (ms) ms[i] = v;
    if (kind) kind[i] = t->ev_kind[i];
  }
  return n;
}

int wt_kernels_per_build(const wt_tree *t) {
  if (!t) return WT_ERR_ARG;
  if (t->n == 0) return 0;
  if (t->fuse_k > 1 && t->L >= 1) {
    int k = 0;
    for (uint32_t l = 0; l < t->L; l += t->fuse_k) {
      k += 4;  // counts, their scan, the k-level pass, directories
      if (t->shape == WT_SHAPE_TREE) k += 1 + (std::min(l + t->fuse_k, t->L - 1) >= l + 1 ? 1 : 0);  // node starts, F tables
    }
    if (t->shape == WT_SHAPE_TREE && t->L >= 2) k += 1;  // level tables
    return k;
  }
  int k = 1;                                              // pre-pass
  if (t->node_counts) {  // node tables of levels 1..L-2 (unless the pass over the level makes
                         // its own) and the node starts of the last level
    for (uint32_t l = 1; l + 1 < t->L; ++l) k += tables_in_pass(t, l) ? 0 : 1;
    k += 1;
  }
  else if (t->shape == WT_SHAPE_TREE) k += 1 + (tables_blocks(t->L) ? 1 : 0);  // histogram scan, tables
  if (t->L >= 1) k += (int)(t->L - 1) + 1;    // splits + last level
  return k;
}

int wt_free(wt_tree *t) {
  if (!t) return WT_OK;
  if (t->owner) return WT_ERR_ARG;  // a view owned by a batch: free the batch
  cudaStreamSynchronize(t->stream);
  (void)cudaGetLastError();
  release(t);
  delete t;
  return WT_OK;
}

}  // extern "C"

// ============================================================ allocation-free build
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured with a capture mode that forbids allocation, hosts whose
// allocator is owned by another runtime or pinned at start-up, and real-time
// loops that must not enter the driver's allocator.  wt_build_noalloc serves
// them: the caller passes the input and every output buffer, and all scratch
// the build needs (ping-pong symbol buffers, histogram, tile counts, node
// tables, look-back state) is carved from one file-scope device array of
// fixed size.  Every GPU that loads this library holds that array until the
// process exits.
#include <atomic>
#include <mutex>

namespace {

constexpr uint64_t kStaticMaxSymbolBytes = 1ull << 21;  // n * symbol_bytes
constexpr uint32_t kStaticMaxLevels = 16;               // sigma <= 65536
constexpr size_t kStaticScratchBytes = 5ull << 20;      // 5 MiB
constexpr int kStaticMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

std::mutex g_static_mu;
unsigned char *g_static_ptr[kStaticMaxDevices] = {};
std::atomic<uint32_t> g_static_builds{0};

// Device address of g_static_scratch for the current device.  The name of
// the array in host code is only a host-side stand-in; the device address is
// looked up once per device, with that device current.
int static_scratch(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) {
    (void)cudaGetLastError();
    return WT_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return WT_ERR_CUDA;
    }
    g_static_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_static_ptr[dev];
  return WT_OK;
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int wt_build_noalloc(const void *d_seq, uint64_t n, uint32_t sigma,
                                uint32_t symbol_bytes, uint32_t *d_bits, uint64_t *d_rank,
                                uint64_t *d_zeros, uint64_t *d_node_start, int32_t *d_status,
                                void *stream) {
  if (!(symbol_bytes == 1 || symbol_bytes == 2 || symbol_bytes == 4)) return WT_ERR_ARG;
  // size limit first, written so that no product can wrap (n < 2^21 here,
  // hence also n < 2^32 as for wt_create)
  if (n > kStaticMaxSymbolBytes / symbol_bytes) return WT_ERR_ARG;
  if (sigma == 0 || (uint64_t)sigma > (1ull << (8 * symbol_bytes))) return WT_ERR_ARG;
  const uint32_t L = levels_of(sigma);
  if (L > kStaticMaxLevels) return WT_ERR_ARG;
  if (n && !d_seq) return WT_ERR_ARG;
  if (!d_node_start || (L && (!d_bits || !d_rank || !d_zeros))) return WT_ERR_ARG;

  unsigned char *base = nullptr;
  if (int rc = static_scratch(&base)) return rc;

  wt_tree t;  // on the stack: describes the build, owns nothing
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&t.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return WT_ERR_CUDA;
  }
  t.n = n;
  t.sigma = sigma;
  t.sb = symbol_bytes;
  t.L = L;
  t.NB = (n + 511) / 512;
  t.W = 16 * t.NB;
  t.threads = pick_threads(n, symbol_bytes, t.sms, 0);
  t.T = 32ull * t.threads;
  t.NT = std::max<uint64_t>(1, (n + t.T - 1) / t.T);
  t.d_bits = d_bits;
  t.d_rank = reinterpret_cast<unsigned long long *>(d_rank);
  t.d_zeros = reinterpret_cast<unsigned long long *>(d_zeros);
  t.d_node_start = reinterpret_cast<unsigned long long *>(d_node_start);

  // carve the scratch
  const uint64_t nbins = 1ull << L;
  const uint32_t Lz = std::max<uint32_t>(L, 1);
  t.counts_per_level = t.NT + (t.NT >> 6) + 1 + (t.NT >> 12) + 1;
  t.ctrl_words = kCtrlWords + nbins + (uint64_t)Lz * t.counts_per_level;
  t.status_n = std::max<uint64_t>({t.NT, (uint64_t)hist_blocks(L), (uint64_t)tables_blocks(L), 1});
  t.buf_bytes = t.NT * t.T * symbol_bytes + 16;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char *p = base + off;
    off += round256(bytes);
    return p;
  };
  t.d_buf[0] = take(t.buf_bytes);
  t.d_buf[1] = take(t.buf_bytes);
  t.d_tab = reinterpret_cast<uint2 *>(take(std::max<uint64_t>(1, nbins / 2) * sizeof(uint2)));
  t.d_ctrl = reinterpret_cast<uint32_t *>(take(t.ctrl_words * 4));
  t.d_hist = t.d_ctrl + kCtrlWords;
  t.d_counts = t.d_hist + nbins;
  t.d_status = reinterpret_cast<unsigned long long *>(take(t.status_n * 8));
  if (off > kStaticScratchBytes) return WT_ERR_ARG;
  // every build also tags its look-back entries with a new epoch
  t.build_count = g_static_builds.fetch_add(1) + 1;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // tickets, error word, histogram and tile counts must start at zero.  The
  // look-back status words sit at an offset that depends on this call's
  // sizes, so an earlier call with other sizes may have left symbol bytes
  // there that happen to decode as a published entry of this build's epoch:
  // they are cleared on every call (a few KB).
  WT_CUDA(cudaMemsetAsync(t.d_ctrl, 0, t.ctrl_words * 4, st));
  WT_CUDA(cudaMemsetAsync(t.d_status, 0, t.status_n * 8, st));
  if (n == 0) {
    if (L) {
      WT_CUDA(cudaMemsetAsync(d_rank, 0, (size_t)L * 8, st));
      WT_CUDA(cudaMemsetAsync(d_zeros, 0, (size_t)L * 8, st));
    }
    WT_CUDA(cudaMemsetAsync(d_node_start, 0, (nbins + 1) * 8, st));
    if (d_status) WT_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int32_t), st));
    return WT_OK;
  }
  const uint8_t *seq = static_cast<const uint8_t *>(d_seq);
  bool padded = false;
  if (reinterpret_cast<uintptr_t>(seq) & 15u) {
    // stage an unaligned input in the buffer the first pass does not write
    void *dst = L >= 2 ? t.d_buf[1] : t.d_buf[0];
    WT_CUDA(cudaMemcpyAsync(dst, seq, n * symbol_bytes, cudaMemcpyDeviceToDevice, st));
    seq = static_cast<const uint8_t *>(dst);
    padded = true;
  }
  int rc = WT_ERR_ARG;
  switch (symbol_bytes) {
    case 1: rc = run_build_sb<1>(&t, seq, padded, st); break;
    case 2: rc = run_build_sb<2>(&t, seq, padded, st); break;
    case 4: rc = run_build_sb<4>(&t, seq, padded, st); break;
  }
  if (rc == WT_OK && d_status)
    WT_CUDA(cudaMemcpyAsync(d_status, t.d_ctrl + kCtrlErr, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return rc;
}

