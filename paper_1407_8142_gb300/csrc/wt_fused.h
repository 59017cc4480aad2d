// Launchers of the k-level schedule (wt_fused.cu), called by the build
// orchestration in wt_build.cu.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "wt_dev.cuh"
#include "wt_internal.h"

namespace wtk {

constexpr uint32_t kMaxLevelsPerPass = 4;

// Symbols per tile of a k-level pass (a multiple of 512).
uint32_t fused_tile_symbols(uint32_t symbol_bytes);

// Blocks of the F-table kernel and of the directory kernel (per row).
uint32_t fused_tables_blocks(uint32_t L, uint32_t K);
uint32_t fused_dir_chunks(uint64_t NB);

// Digit counts of every tile of T_level (K levels: 2^K digits), checking
// the symbols against sigma when `check` is set, and for the tree the node
// counts of level level+K into d_hist (zeroed by the caller); then their
// exclusive scan over the tiles (and, for the matrix, the digit totals).
int fused_count(wt_tree *t, cudaStream_t st, const uint8_t *in, uint32_t level, uint32_t K, bool check);
int fused_scan(wt_tree *t, cudaStream_t st, uint32_t level, uint32_t K);

// One pass over T_level: bits of levels level..level+K-1 and, unless `out`
// is null (last pass), T_{level+K}.  Rows level+1..level+K-1 of the bitmaps
// must be zero; the tile counts and prefixes of this level must be in place.
int fused_pass(wt_tree *t, cudaStream_t st, const uint8_t *in, bool in_padded, uint8_t *out,
               uint32_t level, uint32_t K, uint32_t *ticket);

// F tables of levels m_lo..m_hi (tree only) from E = d_node_start, the
// exclusive scan of the node counts of level Ltop (m_hi <= Ltop).
int fused_tables(wt_tree *t, cudaStream_t st, uint32_t m_lo, uint32_t m_hi, uint32_t Ltop, const Lookback &lb,
                 uint32_t *ticket);
uint32_t fused_tables_blocks_range(uint32_t m_lo, uint32_t m_hi, uint32_t K);

// Directories and zero counts of rows level0..level0+levels-1.
int fused_dir(wt_tree *t, cudaStream_t st, uint32_t level0, uint32_t levels, const Lookback &lb,
              uint32_t *ticket);

}  // namespace wtk
