/*
 * wt.h -- C ABI of the GB300 levelwise wavelet-tree library (libwt.so).
 *
 * Construction follows levelWT (Shun, "Parallel Wavelet Tree Construction",
 * Section 4, Fig. 1): the tree is built one level at a time; on level l every
 * symbol contributes bit (L-1-l) to the level bitmap and is moved, stably, to
 * the 0-child or 1-child range of its node for level l+1.  Each level carries
 * a popcount rank directory (Section 6).  Access, rank and select (defined in
 * Section 2) are provided as batched device calls for validation.
 *
 * Conventions shared by every call:
 *   - All d_* pointers are device pointers (cudaMalloc'd or equivalent).
 *     h_* pointers are host pointers (page-locked memory gives the fastest
 *     copies, pageable memory also works).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that take a stream only enqueue work on it and return at once,
 *     unless stated otherwise.
 *   - Symbols are unsigned little-endian integers of symbol_bytes = 1, 2 or 4
 *     bytes; sigma is the alphabet size, 1 <= sigma <= min(2^(8*symbol_bytes), 2^26);
 *     every symbol must be < sigma.  n < 2^32.
 *   - L = ceil(log2 sigma) levels (L = 0 when sigma = 1).  Level 0 reads the
 *     most significant of the L bits ("mask = 2^(L-(l+1))", Fig. 1).
 *   - Return value: WT_OK (0) or a negative WT_ERR_* code.  Errors detected
 *     on the host are returned at once and nothing is enqueued.  Errors
 *     detected by the device (a symbol >= sigma, a wait that timed out) are
 *     latched in the tree and returned by wt_sync and by later calls on it;
 *     after WT_ERR_SYMBOL the tree's contents are unspecified.
 *   - The library never allocates or frees caller memory; every buffer it
 *     allocates is owned by the tree and released by wt_free.
 */
#ifndef WT_H_
#define WT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WT_OK 0
#define WT_ERR_ARG (-1)     /* invalid argument (host-side check) */
#define WT_ERR_OOM (-2)     /* device allocation failed */
#define WT_ERR_CUDA (-3)    /* a CUDA runtime call failed */
#define WT_ERR_SYMBOL (-4)  /* the input holds a symbol >= sigma (device-side check) */
#define WT_ERR_TIMEOUT (-5) /* a bounded device-side wait ran out (device-side check) */

typedef struct wt_tree wt_tree; /* opaque, library-owned */

/* What a wt_tree object holds (wt_info_t.shape). */
#define WT_SHAPE_TREE 0   /* levelwise wavelet tree (Sections 2 and 4) */
#define WT_SHAPE_MATRIX 1 /* wavelet matrix (Section 7) */

/*
 * Output layout, read through wt_info.  All pointers are device pointers
 * owned by the tree; callers read them and must not free them.
 *
 *   d_bits       uint32[L][W], W = words_per_level = 16*ceil(n/512).  Position
 *                j of level l is bit (j & 31) of d_bits[l*W + (j >> 5)]
 *                (LSB-first; the paper leaves the bit order open).  Bits past
 *                n are 0.  Level l holds bit (L-1-l) of the symbols in the
 *                order T_l of that level (T_0 = S; T_{l+1} is T_l stably
 *                split, node by node, into 0-children then 1-children).
 *   d_rank       uint64[L][NB+1], NB = blocks = ceil(n/512).  d_rank[l*(NB+1)+k]
 *                = number of 1 bits of level l before position 512k (first
 *                level of the Jacobson directory, Section 6, with 512-bit
 *                blocks); entry NB is the level's total number of 1 bits.
 *   d_zeros      uint64[L]: number of 0 bits of each level.
 *   d_node_start uint64[2^L + 1]: d_node_start[v] = #{j : S[j] < v}.  The
 *                node of prefix p on level l (Fig. 1's Nodes[2^l - 1 + p])
 *                starts at d_node_start[p << (L-l)] in that level's bitmap and
 *                has length d_node_start[(p+1) << (L-l)] - d_node_start[p << (L-l)].
 *                NULL for a wavelet matrix.
 *
 * A wavelet matrix (shape WT_SHAPE_MATRIX, Section 7) has the same d_bits,
 * d_rank and d_zeros layout; only the order T_l differs: T_{l+1} is the
 * whole of T_l stably split by bit (L-1-l), all zeros first, and
 * d_zeros[l] is the Z_l that the matrix's queries add to a 1-bit position.
 */
typedef struct {
  uint64_t n;
  uint32_t sigma;
  uint32_t symbol_bytes;
  uint32_t levels;
  uint32_t shape; /* WT_SHAPE_TREE or WT_SHAPE_MATRIX */
  uint64_t words_per_level;
  uint64_t blocks;
  uint32_t *d_bits;
  uint64_t *d_rank;
  uint64_t *d_zeros;
  uint64_t *d_node_start;
  uint32_t levels_per_pass; /* the schedule the builds use (see wt_config) */
} wt_info_t;

/*
 * Launch configuration.  Zero-initialise and set what you need; zero fields
 * take the library's choice.
 *   tile_threads   threads per CTA of the level passes: 128, 256 or 512.  A
 *                  tile is 32*tile_threads symbols (a multiple of 512).
 *   ctas_per_sm    cap on resident CTAs per SM for the persistent passes.
 *   spin_limit     polls before a look-back wait gives up (WT_ERR_TIMEOUT).
 *   debug_skip_publish
 *                  test hook: 1 + the tile index (of every pass) that never
 *                  publishes its look-back status, so that its successor's
 *                  bounded wait runs out.  0 = off.
 *   levels_per_pass
 *                  1: one split pass per level (Fig. 1's level loop).
 *                  2..4: passes that each build that many levels (the
 *                  multiary bucketing of Section 7 applied to the level
 *                  passes): one pass reads T_l once, writes the bitmaps of
 *                  levels l..l+k-1 and T_{l+k}, and a directory pass
 *                  follows.  0 = the library's choice.  Above 4: WT_ERR_ARG.
 */
typedef struct {
  uint32_t tile_threads;
  uint32_t ctas_per_sm;
  uint32_t spin_limit;
  uint32_t debug_skip_publish;
  uint32_t levels_per_pass;
} wt_config;

/*
 * Allocate a tree for sequences of n symbols over [0, sigma) stored in
 * symbol_bytes bytes each.  Allocates device memory (cudaMalloc) for the
 * outputs and for scratch: two ping-pong buffers of n*symbol_bytes bytes
 * (rounded up to whole tiles), a 2^L-bin histogram, per-level tables and the
 * look-back state.  No kernel runs.  cfg may be NULL.
 * Errors: WT_ERR_ARG, WT_ERR_OOM, WT_ERR_CUDA.
 */
int wt_create(uint64_t n, uint32_t sigma, uint32_t symbol_bytes, const wt_config *cfg,
              wt_tree **out);

/*
 * Enqueue the construction of `tree` from d_seq[0..n) on `stream` (levelWT,
 * Fig. 1): a pre-pass that histograms the symbols, checks their range and
 * counts level 0's ones per tile, the node tables, one split pass per level
 * l = 0..L-2 (bits, directory and the stable split into T_{l+1}), and a last
 * pass for level L-1 (bits and directory).  For sigma > 2^13 and for
 * n >= 2^24 the pre-pass builds no histogram: each split pass counts, per
 * child node, the ones of the next level, and these counts become that
 * level's node tables and node starts -- in the prologue of the pass over
 * the level when it has at most one node per thread of the pass's blocks,
 * else in a small kernel before it.  When the nodes of level L-2 average
 * 2^16 symbols or more, levels L-2 and L-1 are one pass that moves no
 * symbols (level L-1's bits are compacted straight to their positions),
 * followed by a directory kernel for level L-1.  With levels_per_pass =
 * k > 1 (see wt_config; the library's choice for 4-byte symbols, at least 8
 * levels and n >= 2^22) each pass builds k levels, after a kernel that
 * counts every tile's k-bit digits (and the node sizes of level l+k, which
 * give that pass's tables) and a scan of those counts; a directory kernel
 * follows each pass.  Every size is known on the host, so the call has no host
 * synchronisation and may be captured into a CUDA graph.
 * d_seq is read-only; it must stay valid until the stream work completes.
 * A d_seq that is not 16-byte aligned is first copied into tree scratch.
 * Errors: WT_ERR_ARG, WT_ERR_CUDA; device errors are reported by wt_sync.
 */
int wt_rebuild(wt_tree *tree, const void *d_seq, void *stream);

/*
 * Re-target `tree` to sequences of n symbols, n <= the n it was created
 * with, reusing its device memory: a caller that builds many sequences of
 * different lengths over one alphabet allocates one tree for the longest
 * and resizes it before each wt_rebuild, with no cudaMalloc per sequence.
 * The output layout follows the new n (wt_info); the contents of earlier
 * builds are invalid afterwards.  The schedule chosen at creation (tile
 * size, levels per pass, node counts) is kept; it builds any n.  Host-side
 * only and immediate, except that n = 0 clears the directories with a
 * synchronous cudaMemset.  The tree's last build must be complete (wt_sync)
 * before the call.  Not for views (WT_ERR_ARG).
 * Errors: WT_ERR_ARG (n above the creation size, NULL or a view), WT_ERR_CUDA.
 */
int wt_resize(wt_tree *tree, uint64_t n);

/* wt_create followed by wt_rebuild. */
int wt_build(const void *d_seq, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
             void *stream, wt_tree **out);

/* Same, with a launch configuration (may be NULL). */
int wt_build_ex(const void *d_seq, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
                const wt_config *cfg, void *stream, wt_tree **out);

/*
 * Host-memory path: copy h_seq[0..n) to the device, build, and copy the
 * bitmaps (L*W uint32) into h_bits and the directory (L*(NB+1) uint64) into
 * h_rank (either may be NULL to skip that copy).  Each level's rows are
 * copied on a stream of the tree's own as soon as the pass that writes them
 * has finished, overlapping the copies with the later passes (page-locked
 * host buffers make the copies asynchronous).  Synchronises before
 * returning and returns the build status (as wt_sync).  The tree must have
 * been created for this n, sigma and symbol_bytes; not for views.
 */
int wt_build_host(wt_tree *tree, const void *h_seq, uint32_t *h_bits, uint64_t *h_rank,
                  void *stream);

/*
 * wt_build_host without the final synchronisation: enqueues the copy in, the
 * build and the copies out, and returns.  Work enqueued later on `stream`
 * (including the next build of this tree) runs after the copies out;
 * wt_sync(tree) waits for all of it and returns the build status.  h_seq,
 * h_bits and h_rank must stay valid until then.  Builds of different trees
 * on different streams overlap: one build's copies with another's kernels.
 * Errors: as wt_build_host, but device-side errors only through wt_sync.
 */
int wt_build_host_async(wt_tree *tree, const void *h_seq, uint32_t *h_bits, uint64_t *h_rank,
                        void *stream);

/*
 * Wavelet matrix (Section 7).  Allocates like wt_create, without the
 * histogram, node tables and d_node_start, for a wt_tree of shape
 * WT_SHAPE_MATRIX.  Every other call taking a wt_tree (wt_rebuild,
 * wt_build_host, wt_sync, wt_info, the queries, wt_profile, wt_free,
 * wt_kernels_per_build) works on it unchanged.  Its construction is one
 * pre-pass (range check, level-0 ones per tile), then per level
 * l = 0..L-2 the split pass of the tree with a single node: zeros go to
 * j - R(j), ones to Z_l + R(j), where Z_l is the level's zero count, known
 * before the pass from the previous pass's tile counts.  The last level
 * writes bits and directory only.  With levels_per_pass = k > 1 (the
 * library's choice for 4-byte symbols and at least 8 levels) each pass
 * builds k levels: a class of i bits goes to the start of its class in
 * T_{l+i} (the classes ordered by their bits read from the last level to
 * the first) plus the symbols of that class before it; no pre-pass runs.
 * Errors: as wt_create / wt_rebuild.
 */
int wt_matrix_create(uint64_t n, uint32_t sigma, uint32_t symbol_bytes, const wt_config *cfg,
                     wt_tree **out);

/* wt_matrix_create followed by wt_rebuild.  cfg may be NULL. */
int wt_matrix_build(const void *d_seq, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
                    const wt_config *cfg, void *stream, wt_tree **out);

/* Wait for the tree's last enqueued work and return its status. */
int wt_sync(wt_tree *tree);

/* Describe the tree's outputs (see wt_info_t).  Does not synchronise. */
int wt_info(const wt_tree *tree, wt_info_t *info);

/*
 * Batched queries over a built tree or matrix (Section 2 definitions), one
 * result per query, enqueued on `stream`.  The build must be complete in
 * stream order (same stream, or synchronised).  Queries walk the levels with
 * rank on the bitmaps; node ranges are derived by rank, so the node table is
 * not used.  On a matrix, a position moves to rank0 on a 0 bit and to
 * d_zeros[l] + rank1 on a 1 bit (Section 7).
 *   wt_access: d_out[q] = S[d_i[q]]; UINT32_MAX when d_i[q] >= n.
 *   wt_rank:   d_out[q] = #{j <= d_i[q] : S[j] = d_c[q]} (inclusive);
 *              UINT64_MAX when d_i[q] >= n or d_c[q] >= sigma.
 *   wt_select: d_out[q] = position of the d_k[q]-th occurrence of d_c[q]
 *              (k counted from 1), so that select_c(rank_c(i)) = i when
 *              S[i] = c; UINT64_MAX when k = 0, k exceeds the number of
 *              occurrences, or d_c[q] >= sigma.
 * m = 0 is valid and does nothing.  Errors: WT_ERR_ARG, WT_ERR_CUDA.
 */
int wt_access(const wt_tree *tree, const uint64_t *d_i, uint64_t m, uint32_t *d_out,
              void *stream);
int wt_rank(const wt_tree *tree, const uint32_t *d_c, const uint64_t *d_i, uint64_t m,
            uint64_t *d_out, void *stream);
int wt_select(const wt_tree *tree, const uint32_t *d_c, const uint64_t *d_k, uint64_t m,
              uint64_t *d_out, void *stream);

/*
 * Per-kernel timing of the following builds of `tree` (measurement support).
 * wt_profile(tree, 1) starts a recording window: every later wt_rebuild
 * records a CUDA event pair on its stream around each kernel it launches (up
 * to 2048 launches per window).  wt_profile_read, after wt_sync, returns the
 * number of launches recorded in the window and fills up to `cap` entries of
 * ms[] with each launch's duration and kind[] with its kind: 0 pre-pass,
 * 1 node starts (histogram scan, or the last two levels' starts from node
 * counts), 2 node tables, 3 split pass, 4 last-level pass, 5 k-level pass,
 * 6 directories, 7 digit counts, 8 their scan, 9 the last two levels in one
 * pass.
 * wt_profile(tree, 0) stops recording.
 */
int wt_profile(wt_tree *tree, int enable);
int wt_profile_read(wt_tree *tree, float *ms, int32_t *kind, int32_t cap);

/* Release everything the tree owns.  Synchronises the tree's last stream. */
int wt_free(wt_tree *tree);

/* Number of kernels one wt_rebuild of this tree launches. */
int wt_kernels_per_build(const wt_tree *tree);

/*
 * Batched construction of many independent trees (one persistent launch).
 *
 * The trees of a batch are built by a single persistent kernel over a work
 * list of (tree, phase, tile) items -- pre-pass tiles, one node-table item,
 * split-pass tiles per level, last-level tiles -- ordered phase by phase
 * across trees.  An item waits (bounded) only on its own tree's previous
 * phase, through a per-tree completion counter; there is no grid-wide
 * barrier.  Each tree gets exactly the outputs of wt_build (same layout,
 * identical bits); parallelism across trees is the paper's observation that
 * independent constructions are embarrassingly parallel, and inside a tree
 * the passes are those of levelWT (Fig. 1).
 *
 *   wt_seq_desc        n, sigma, symbol_bytes of one sequence (limits as
 *                      for wt_create).
 *   wt_batch_create    allocate outputs and scratch for m sequences (one
 *                      device allocation) and the work list.  cfg may be
 *                      NULL; cfg->tile_threads (128 or 256) selects the CTA
 *                      size of the batch kernel.
 *   wt_batch_set_inputs
 *                      record the m device input pointers (host array of
 *                      pointers, each 16-byte aligned, else WT_ERR_ARG);
 *                      synchronous copy of the pointer table.
 *   wt_batch_build     enqueue the build of every tree: one memset and one
 *                      kernel launch on `stream`; capturable in a CUDA graph.
 *   wt_batch_sync      wait; returns 0 or the first device error of any tree.
 *   wt_batch_latencies per-tree completion times of the last build.
 *   wt_batch_tree      tree i as a wt_tree view for wt_info / wt_sync /
 *                      wt_access / wt_rank / wt_select; owned by the batch
 *                      (wt_free on a view returns WT_ERR_ARG).
 *   wt_batch_free      release the batch and its views.
 *   wt_build_batch     create + set_inputs + build.
 */
typedef struct {
  uint64_t n;
  uint32_t sigma;
  uint32_t symbol_bytes;
} wt_seq_desc;

typedef struct wt_batch wt_batch; /* opaque, library-owned */

int wt_batch_create(const wt_seq_desc *descs, uint32_t m, const wt_config *cfg, wt_batch **out);
int wt_batch_set_inputs(wt_batch *batch, const void *const *d_seqs);
int wt_batch_build(wt_batch *batch, void *stream);
int wt_batch_sync(wt_batch *batch);
int wt_batch_tree(wt_batch *batch, uint32_t i, wt_tree **tree);
/* Measurement: after a build, ns[i] = time from the start of the batch's
 * first item to the completion of tree i's last item (GPU global timer),
 * for i < m.  Synchronises the batch's stream. */
int wt_batch_latencies(wt_batch *batch, uint64_t *ns);
int wt_batch_free(wt_batch *batch);
int wt_build_batch(const wt_seq_desc *descs, const void *const *d_seqs, uint32_t m,
                   const wt_config *cfg, void *stream, wt_batch **out);

/*
 * Build server: continuous batching of build requests under an HBM budget.
 *
 * A worker thread admits queued requests in arrival order as soon as a
 * request's footprint (its input copy, outputs, scratch and control block)
 * fits in a device arena of `budget_bytes` (allocated once at creation) and
 * one of `max_inflight` streams is free; the requests admissible at that
 * moment with fewer than 2^20 symbols and sigma <= 2^13 form one batch (one
 * launch of the batched build kernel); every other request is built alone
 * with the single-tree schedule of wt_build (the library's choice of tile
 * size and levels per pass), its buffers in its arena region.  Work on
 * different streams overlaps on the device, so requests that arrive while
 * others run start as soon as memory and a stream free up.  Results stay in
 * the arena until released.  Each result is bit-identical to a wt_build of
 * the same input.  A completed result holds its memory until it is
 * released, so a client that keeps results must release them for queued
 * requests to be admitted.
 *
 *   wt_server_create   budget_bytes >= 1 MiB, 1 <= max_inflight <= 64; cfg may
 *                      be NULL (tile_threads 128 or 256).  Uses the current
 *                      device.
 *   wt_server_submit   queue a build of h_seq[0..n) (host memory; page-locked
 *                      memory copies asynchronously).  h_seq must stay valid
 *                      until the request completes.  A request larger than
 *                      the budget returns WT_ERR_ARG.
 *   wt_server_poll     ids (and latencies, seconds from submit to completion
 *                      on the device) of requests completed since the last
 *                      poll, up to cap; *count gets their number.
 *   wt_server_tree     the result of a completed request as a wt_tree view
 *                      (owned by the server); returns its device status.
 *   wt_server_release  free a completed request's memory (its view dies).
 *   wt_server_drain    wait until every submitted request has completed;
 *                      WT_ERR_OOM when nothing is running and the next queued
 *                      request cannot fit because completed results still hold
 *                      the memory (release them and drain again).
 *   wt_server_stats    out[0..5] = batches launched, requests admitted, peak
 *                      arena bytes in use, bytes in use, budget, queued.
 *   wt_server_free     stop the worker and release everything.
 */
typedef struct wt_server wt_server; /* opaque, library-owned */

int wt_server_create(uint64_t budget_bytes, uint32_t max_inflight, const wt_config *cfg,
                     wt_server **out);
int wt_server_submit(wt_server *server, const void *h_seq, uint64_t n, uint32_t sigma,
                     uint32_t symbol_bytes, uint64_t *id);
int wt_server_poll(wt_server *server, uint64_t *ids, double *latency_s, uint32_t cap,
                   uint32_t *count);
int wt_server_tree(wt_server *server, uint64_t id, wt_tree **tree);
int wt_server_release(wt_server *server, uint64_t id);
int wt_server_drain(wt_server *server);
int wt_server_stats(wt_server *server, uint64_t *out, uint32_t cap);
int wt_server_free(wt_server *server);

/*
 * Allocation-free build.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they run --
 * code inside a CUDA graph capture whose mode forbids allocation, hosts whose
 * device allocator belongs to another runtime, and loops with a fixed memory
 * footprint.  It builds the same outputs as wt_build (identical bits) but
 * allocates nothing: the caller passes the input and every output, laid out
 * as in wt_info_t (d_bits L*W uint32, d_rank L*(NB+1) uint64, d_zeros L
 * uint64, d_node_start 2^L+1 uint64), and all scratch comes from one
 * file-scope device array of 5 MiB that every GPU loading this library keeps
 * until the process exits.
 *   Limits: n * symbol_bytes <= 2^21 bytes and sigma <= 2^16; larger
 *   problems return WT_ERR_ARG.
 *   d_status (may be NULL) receives, in stream order, the device-detected
 *   status of the build (0, WT_ERR_SYMBOL or WT_ERR_TIMEOUT).
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   All calls share the scratch array: calls whose work overlaps on the GPU
 *   (different streams, or different host threads) race and corrupt each
 *   other.  Serialise them on one stream.
 * Errors: WT_ERR_ARG, WT_ERR_CUDA.
 */
int wt_build_noalloc(const void *d_seq, uint64_t n, uint32_t sigma, uint32_t symbol_bytes,
                     uint32_t *d_bits, uint64_t *d_rank, uint64_t *d_zeros,
                     uint64_t *d_node_start, int32_t *d_status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WT_H_ */
