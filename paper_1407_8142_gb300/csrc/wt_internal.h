// Host-side tree object shared by the build and query translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "wt.h"

namespace wtk {

constexpr uint32_t kMaxLevels = 26;     // 2^L histogram bins must fit comfortably
constexpr uint32_t kPasses = 64;        // ticket counters per build (passes <= 2L + 3)
constexpr uint32_t kCtrlWords = 128;    // [0,64) tickets, [64] error, rest reserved
constexpr uint32_t kCtrlErr = 64;
constexpr uint32_t kMaxProfiled = 2048;  // kernel launches recorded per profiling window

enum KernelKind : int32_t {
  kPrepass = 0, kHistScan = 1, kTables = 2, kSplit = 3, kLeaf = 4, kFused = 5, kDirectory = 6,
  kTileCount = 7, kTileScan = 8, kLastPair = 9
};

}  // namespace wtk

struct wt_tree {
  uint64_t n = 0;
  uint64_t cap_n = 0;             // the n the buffers were sized for (wt_resize keeps n <= cap_n)
  uint32_t sigma = 0, sb = 0, L = 0;
  uint32_t shape = WT_SHAPE_TREE;  // WT_SHAPE_TREE or WT_SHAPE_MATRIX
  // tree with a large alphabet: node sizes come from per-node counts kept by
  // the split passes instead of a 2^L-bin histogram of the input
  bool node_counts = false;
  // levels per pass: 1 = one split pass per level; k > 1 = passes that each
  // build k levels (their F tables in d_ftab, tiles of tile_f symbols)
  uint32_t fuse_k = 1;
  uint64_t tile_f = 0, NTf = 0;
  uint64_t W = 0, NB = 0;
  uint32_t threads = 0;         // CTA size of the level passes
  uint64_t T = 0;               // symbols per tile
  uint64_t NT = 0;              // tiles per level
  wt_config cfg{};
  int sms = 0;

  // outputs
  uint32_t *d_bits = nullptr;
  unsigned long long *d_rank = nullptr;
  unsigned long long *d_zeros = nullptr;
  unsigned long long *d_node_start = nullptr;
  // scratch
  uint2 *d_tab = nullptr;       // per level l (heap offset 2^l - 1): {O_l[p], E_{l+1}[2p+1]-O_l[p]}
  uint32_t *d_ftab = nullptr;   // k-level passes of a tree: F_m at offset 2^m - 2, m = 1..L-1
  uint32_t *d_fcount = nullptr; // k-level passes: per-tile digit counts, then their prefixes
  uint32_t *d_ctrl = nullptr;   // kCtrlWords control words, then 2^L words: the histogram
                                // (tree) or the per-node ones counters (node_counts)
  uint32_t *d_hist = nullptr;
  uint32_t *d_counts = nullptr;   // per level: ones per tile, per 64 tiles, per 4096 tiles
  uint64_t counts_per_level = 0;
  uint64_t ctrl_words = 0;        // control words + histogram + tile counts (cleared per build)
  void *d_buf[2] = {nullptr, nullptr};
  size_t buf_bytes = 0;
  unsigned long long *d_status = nullptr;
  size_t status_n = 0;
  void *d_in_host = nullptr;    // device staging of wt_build_host input (lazy)

  uint32_t build_count = 0;
  cudaStream_t stream = nullptr;
  int sticky_error = 0;
  void *owner = nullptr;          // set for views of trees owned by a batch or a server

  // query index: sampled select positions per level (built on first select
  // after a build, owned by the tree object itself, also for views)
  uint32_t *d_sel = nullptr;
  uint64_t sel_stride = 0;        // entries per (level, bit value)
  uint32_t sel_for = 0;           // build_count + 1 the index was built for (0 = none)

  // host-buffer builds: each level's rows are copied out on copy_stream as
  // soon as the pass that writes them is done (level_ev, recorded after it)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t level_ev[wtk::kMaxLevels] = {};
  cudaEvent_t copy_done = nullptr;  // recorded after the last copy out
  bool record_levels = false;

  bool profile = false;
  cudaEvent_t *ev = nullptr;      // 2 * kMaxProfiled events, created on first use
  int32_t *ev_kind = nullptr;
  int n_ev = 0;                   // launches recorded since wt_profile(tree, 1)

  ~wt_tree() {
    if (d_sel) cudaFree(d_sel);
  }
};

namespace wtk {

// Device buffers of a tree (bytes; 0 = not needed), from its shape fields.
struct TreeLayout {
  size_t bits, rank, zeros, node_start, tab, ftab, fcount, ctrl, buf, status;
};

// Check the arguments and fill the shape fields of t (schedule, tile sizes,
// buffer sizes) as wt_create / wt_matrix_create do, without allocating.
int tree_shape(wt_tree *t, uint64_t n, uint32_t sigma, uint32_t symbol_bytes, const wt_config *cfg,
               uint32_t shape);
TreeLayout tree_layout(const wt_tree *t);
// All of a tree's buffers in one region (256-byte aligned pieces).
size_t tree_region_bytes(const TreeLayout &ly);
// Point t's buffers into the region at base (tree_region_bytes bytes).
void tree_bind(wt_tree *t, const TreeLayout &ly, unsigned char *base);
// The pointers derived from d_ctrl (histogram, tile counts).
void tree_bind_derived(wt_tree *t);
// Enqueue a build of t from d_seq on st (wt_rebuild without its ownership check).
int tree_rebuild(wt_tree *t, const void *d_seq, cudaStream_t st);

}  // namespace wtk
