/*
 * serialWT: the sequential wavelet-tree construction, used as the ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library; the two are compared on the same seeded inputs.
 *
 * What it computes (Shun, "Parallel Wavelet Tree Construction"):
 *   - The levelwise wavelet tree of Section 2: the root covers symbols
 *     [0, 2^L) with L = ceil(log2 sigma); a node's bitmap holds, for each of
 *     its symbols in sequence order, 0 if the symbol lies in the lower half of
 *     the node's range and 1 otherwise; children take the two halves; the
 *     recursion ends at ranges of size 2 or less.  Level l therefore reads bit
 *     (L-1-l) of every symbol ("mask = 2^(L-(l+1))", Fig. 1).
 *   - The construction is levelWT (Fig. 1, Section 4) with every parallel
 *     loop run as a plain sequential loop; a serial run of that algorithm is
 *     the paper's serialWT (Section 5, "Implementations").  Per node: count
 *     the symbols that go left (the total X_s of the prefix sum), then place
 *     left symbols at start + (lefts so far) and right symbols at
 *     start + X_s + (rights so far), which is the paper's X_s + i - X[i].
 *     Children are appended only when non-empty, in node order, so the node
 *     list of the next level is the filtered A'.
 *   - One bitmap of n bits per level shared by all nodes of that level
 *     (Section 4 and Section 5, "levelwise representation").  Bits are packed
 *     LSB-first into 32-bit words: position i of level l is bit (i & 31) of
 *     word l*W + (i >> 5), W = 16*ceil(n/512); padding bits are 0.  The paper
 *     omits the bit arithmetic (footnote to Fig. 1); LSB-first is the reading
 *     adopted by this project.
 *   - A rank directory per level (Section 6, first-level Jacobson directory,
 *     blocks of 512 bits as in the practical variants the paper cites):
 *     rank[l*(NB+1) + k] = number of 1 bits of level l in positions
 *     [0, 512k), k = 0..NB, NB = ceil(n/512).  Counted naively.
 *   - zeros[l] = n - (number of 1 bits of level l).
 *   - The node table of Fig. 1 (Nodes[id] = bitmap offset, length), with the
 *     heap ids 2id+1 / 2id+2 for the children.
 *   - The wavelet matrix of Section 7 (wto_matrix_build): per level, the
 *     bitmap of bit (L-1-l) of the level's sequence and its zero count; the
 *     next level's sequence is the stable reordering of the current one by
 *     that bit, zeros first.  Same bit, directory and zero-count layout.
 *   - Queries by their definitions (Section 2): access(i) = S[i];
 *     rank_c(i) = #{j <= i : S[j] = c}; select_c(k) = position of the k-th
 *     occurrence of c (k counted from 1), by naive scans over S.
 *
 * Readings where the paper is silent: n = 0 is valid (empty bitmaps, a
 * directory of one 0 entry per level); sigma = 1 gives L = 0 (no levels);
 * a symbol >= sigma is an error (WTO_ERR_SYMBOL); an out-of-range query
 * returns the all-ones value of its output type.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define WTO_OK 0
#define WTO_ERR_ARG (-1)
#define WTO_ERR_OOM (-2)
#define WTO_ERR_SYMBOL (-4)

static uint32_t sym_at(const void *S, uint64_t i, uint32_t b) {
  if (b == 1) return ((const uint8_t *)S)[i];
  if (b == 2) return ((const uint16_t *)S)[i];
  return ((const uint32_t *)S)[i];
}

/* L = ceil(log2 sigma); 0 for sigma <= 1. */
uint32_t wto_levels(uint64_t sigma) {
  uint32_t L = 0;
  while ((1ull << L) < sigma) ++L;
  return L;
}

uint64_t wto_words_per_level(uint64_t n) { return 16ull * ((n + 511) / 512); }

uint64_t wto_blocks(uint64_t n) { return (n + 511) / 512; }

/* Rank directory and zero counts of every level, naively from the packed
 * bits: rank[l*(NB+1) + k] = ones of level l before position 512k (k < NB),
 * rank[l*(NB+1) + NB] = ones of level l, zeros[l] = n - ones of level l. */
static void wto_directory(const uint32_t *bits, uint64_t n, uint32_t L, uint64_t *rank,
                          uint64_t *zeros) {
  const uint64_t W = wto_words_per_level(n);
  const uint64_t NB = wto_blocks(n);
  for (uint32_t l = 0; l < L; ++l) {
    const uint32_t *B = bits + (uint64_t)l * W;
    uint64_t *D = rank + (uint64_t)l * (NB + 1);
    uint64_t ones = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if ((i & 511) == 0) D[i >> 9] = ones;
      ones += (B[i >> 5] >> (i & 31)) & 1u;
    }
    D[NB] = ones;
    zeros[l] = n - ones;
  }
}

/* One entry of the node list A of Fig. 1: (start, len, id, range). */
typedef struct {
  uint64_t start, len, id, range;
} wto_node;

/*
 * Build the levelwise wavelet tree of S[0..n) over alphabet [0, sigma).
 *   bits : L*W uint32 words, must be zeroed by the caller.
 *   rank : L*(NB+1) uint64.
 *   zeros: L uint64.
 *   node_id/node_start/node_len: capacity node_cap entries; *n_nodes gets the
 *     number written (every node Fig. 1 creates, level by level).
 */
int wto_build(const void *S, uint64_t n, uint64_t sigma, uint32_t b,
              uint32_t *bits, uint64_t *rank, uint64_t *zeros,
              uint64_t *node_id, uint64_t *node_start, uint64_t *node_len,
              uint64_t node_cap, uint64_t *n_nodes) {
  if (!(b == 1 || b == 2 || b == 4) || sigma == 0) return WTO_ERR_ARG;
  if (sigma > (1ull << (8 * b))) return WTO_ERR_ARG;
  for (uint64_t i = 0; i < n; ++i)
    if (sym_at(S, i, b) >= sigma) return WTO_ERR_SYMBOL;

  const uint32_t L = wto_levels(sigma);
  const uint64_t W = wto_words_per_level(n);
  *n_nodes = 0;
  if (L == 0) return WTO_OK;

  uint32_t *cur = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  uint32_t *nxt = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  /* A level has at most min(2^l, n) non-empty nodes (+1 for an empty root). */
  const uint64_t acap = (n < (1ull << L) ? n : (1ull << L)) + 1;
  wto_node *A = (wto_node *)malloc(acap * sizeof(wto_node));
  wto_node *A2 = (wto_node *)malloc(acap * sizeof(wto_node));
  if (!cur || !nxt || !A || !A2) {
    free(cur); free(nxt); free(A); free(A2);
    return WTO_ERR_OOM;
  }
  for (uint64_t i = 0; i < n; ++i) cur[i] = sym_at(S, i, b);

  uint64_t na = 1;
  A[0].start = 0; A[0].len = n; A[0].id = 0; A[0].range = 1ull << L;

  for (uint32_t l = 0; l < L; ++l) {
    const uint32_t mask = 1u << (L - (l + 1));
    uint32_t *B = bits + (uint64_t)l * W;
    uint64_t na2 = 0;
    for (uint64_t j = 0; j < na; ++j) {
      const uint64_t start = A[j].start, len = A[j].len, id = A[j].id, r = A[j].range;
      if (*n_nodes < node_cap) {
        node_id[*n_nodes] = id;
        node_start[*n_nodes] = start;
        node_len[*n_nodes] = len;
      }
      ++*n_nodes;
      if (r <= 2) {
        /* No children: only this node's bits. */
        for (uint64_t i = 0; i < len; ++i)
          if (cur[start + i] & mask) B[(start + i) >> 5] |= 1u << ((start + i) & 31);
        continue;
      }
      /* X_s: how many of the node's symbols go to the left child. */
      uint64_t xs = 0;
      for (uint64_t i = 0; i < len; ++i)
        if ((cur[start + i] & mask) == 0) ++xs;
      uint64_t lefts = 0, rights = 0;
      for (uint64_t i = 0; i < len; ++i) {
        const uint32_t s = cur[start + i];
        if (s & mask) {
          B[(start + i) >> 5] |= 1u << ((start + i) & 31);
          nxt[start + xs + rights] = s;
          ++rights;
        } else {
          nxt[start + lefts] = s;
          ++lefts;
        }
      }
      if (xs > 0) {
        A2[na2].start = start; A2[na2].len = xs;
        A2[na2].id = 2 * id + 1; A2[na2].range = r / 2;
        ++na2;
      }
      if (len - xs > 0) {
        A2[na2].start = start + xs; A2[na2].len = len - xs;
        A2[na2].id = 2 * id + 2; A2[na2].range = r / 2;
        ++na2;
      }
    }
    /* A = filtered A'; swap(S, S'). */
    wto_node *tA = A; A = A2; A2 = tA; na = na2;
    uint32_t *t = cur; cur = nxt; nxt = t;
  }

  wto_directory(bits, n, L, rank, zeros);
  free(cur); free(nxt); free(A); free(A2);
  return WTO_OK;
}

/*
 * The wavelet matrix of S (Section 7, after Claude and Navarro): level l's
 * bitmap holds bit (L-1-l) of the symbols in the order T_l, where T_0 = S
 * and T_{l+1} lists the symbols of T_l whose bit (L-1-l) is 0, in their T_l
 * order, followed by those whose bit is 1, in their T_l order (the stable
 * reordering by that bit).  zeros[l] is the number of 0 bits of level l;
 * bits, rank and zeros have the layout of wto_build.  Plain sequential
 * loops, one level after the other.
 */
int wto_matrix_build(const void *S, uint64_t n, uint64_t sigma, uint32_t b,
                     uint32_t *bits, uint64_t *rank, uint64_t *zeros) {
  if (!(b == 1 || b == 2 || b == 4) || sigma == 0) return WTO_ERR_ARG;
  if (sigma > (1ull << (8 * b))) return WTO_ERR_ARG;
  for (uint64_t i = 0; i < n; ++i)
    if (sym_at(S, i, b) >= sigma) return WTO_ERR_SYMBOL;
  const uint32_t L = wto_levels(sigma);
  const uint64_t W = wto_words_per_level(n);
  if (L == 0) return WTO_OK;
  uint32_t *cur = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  uint32_t *nxt = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  if (!cur || !nxt) {
    free(cur); free(nxt);
    return WTO_ERR_OOM;
  }
  for (uint64_t i = 0; i < n; ++i) cur[i] = sym_at(S, i, b);
  for (uint32_t l = 0; l < L; ++l) {
    const uint32_t mask = 1u << (L - (l + 1));
    uint32_t *B = bits + (uint64_t)l * W;
    uint64_t z = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (cur[i] & mask) B[i >> 5] |= 1u << (i & 31);
      else ++z;
    }
    /* zeros keep their order at the front, ones keep theirs behind them */
    uint64_t lefts = 0, rights = 0;
    for (uint64_t i = 0; i < n; ++i) {
      if (cur[i] & mask) nxt[z + rights++] = cur[i];
      else nxt[lefts++] = cur[i];
    }
    uint32_t *t = cur; cur = nxt; nxt = t;
  }
  wto_directory(bits, n, L, rank, zeros);
  free(cur); free(nxt);
  return WTO_OK;
}

/* access(i) = S[i]; UINT32_MAX when i >= n. */
void wto_access(const void *S, uint64_t n, uint32_t b, const uint64_t *idx,
                uint64_t m, uint32_t *out) {
  for (uint64_t q = 0; q < m; ++q) out[q] = idx[q] < n ? sym_at(S, idx[q], b) : UINT32_MAX;
}

/* rank_c(i) = #{j <= i : S[j] = c}; UINT64_MAX when i >= n or c >= sigma. */
void wto_rank(const void *S, uint64_t n, uint64_t sigma, uint32_t b,
              const uint32_t *c, const uint64_t *idx, uint64_t m, uint64_t *out) {
  for (uint64_t q = 0; q < m; ++q) {
    if (idx[q] >= n || c[q] >= sigma) { out[q] = UINT64_MAX; continue; }
    uint64_t cnt = 0;
    for (uint64_t j = 0; j <= idx[q]; ++j) cnt += sym_at(S, j, b) == c[q];
    out[q] = cnt;
  }
}

/* select_c(k) = position of the k-th occurrence of c, k >= 1; UINT64_MAX when
 * k = 0, k exceeds the number of occurrences, or c >= sigma. */
void wto_select(const void *S, uint64_t n, uint64_t sigma, uint32_t b,
                const uint32_t *c, const uint64_t *k, uint64_t m, uint64_t *out) {
  for (uint64_t q = 0; q < m; ++q) {
    out[q] = UINT64_MAX;
    if (k[q] == 0 || c[q] >= sigma) continue;
    uint64_t seen = 0;
    for (uint64_t j = 0; j < n; ++j) {
      if (sym_at(S, j, b) == c[q] && ++seen == k[q]) { out[q] = j; break; }
    }
  }
}
