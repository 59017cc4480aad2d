// k levels per pass (Shun, "Parallel Wavelet Tree Construction": the
// multiary tree of Section 7 sorts log d bits at a time; here that bucketing
// is applied to levelWT's global passes).
//
// A pass over T_l builds the bitmaps of levels l .. l+K-1 and writes
// T_{l+K}, reading and writing the symbols once instead of K times.  Let the
// digit of a symbol be its K bits below the node prefix (the bits of levels
// l..l+K-1, level l's bit most significant), and a class of granularity i
// (1 <= i <= K) the first i of those bits.  For the symbol at position j of
// T_l, node p (its top l bits) and class c of granularity i, with
// G_c(j) = symbols of class c before j (over the whole level, every node):
//
//   tree:    position in T_{l+i} = F_{l+i}[p*2^i + c] + G_c(j),
//            F_m[q] = E_m[q] - (symbols of class c in nodes p' < p),
//            E_m[q] = start of node q of level m  (Section 4's node starts;
//            the symbols of node q before j are G_c(j) - G_c(start of p))
//   matrix:  position in T_{l+i} = B_i[c] + G_c(j), where B_i[c] counts the
//            symbols whose class precedes c in the order of the bits read
//            from the last level to the first (Section 7: each level is a
//            stable split of the whole previous level)
//
// G_c(tile start) comes from two small kernels before each k-level pass:
// k_tilecount counts every tile's digits (reading T_l once) and k_tilescan
// scans those counts over the tiles (coarser classes are sums of digits).
// The k-level pass itself then has no dependence between tiles.  Inside a
// tile the K stable 2-way splits run in shared memory: round i splits the
// tile's image by the bit of level l+i, so that after round i the image
// holds the tile's symbols ordered by class (bits read from the last to the
// first) and, within a class, in T_l order.  Round i's ballot words are
// level l+i's bits of the tile in image order: each class is one run of bits
// that belongs at position F (or B) + G_c(tile start) of row l+i.  The last
// image is written to T_{l+K} the same way.  Level l's own bits are the
// tile's first ballot words, in place.
//
// A tile whose symbols lie in one node (all tiles of the matrix) writes one
// run per class.  A tile over a few nodes counts its symbols per (node,
// digit) and writes one run per class and node (within a class the nodes'
// symbols follow each other in T_l order).  A tile over many nodes writes,
// per row of 32 image positions, one run per stretch of consecutive
// destinations, with F looked up per symbol.
//
// Directories are a separate pass over the finished rows (k_dir).
#include <algorithm>

#include "wt_dev.cuh"
#include "wt_fused.h"
#include "wt_internal.h"

using namespace wtk;

#include "wt_kernels.cuh"

namespace {

constexpr uint32_t kFThreads = 256;
constexpr uint32_t kFWarps = kFThreads / 32;

template <int SB>
struct FGeom {
  // 4-byte symbols: one tile buffer, copied after each tile (the smaller
  // footprint lets four CTAs share an SM, and their work covers the copy);
  // narrower symbols: two, the next tile's copy overlapping this one
  static constexpr int DEPTH = SB == 4 ? 1 : 2;
  static constexpr uint32_t V = 32;  // rows per warp = symbols per thread (tiles of 8192)
  static constexpr uint32_t TS = kFThreads * V;       // symbols per tile
  static constexpr uint32_t NWD = TS / 32;            // bit words per tile and level
};

constexpr uint32_t kFewNodes = 16;  // tree tiles over fewer nodes write per-(class, node) runs

template <int SB, int K, bool MATRIX>
__host__ __device__ constexpr uint32_t fused_smem_bytes() {
  using G = FGeom<SB>;
  return G::DEPTH * G::TS * SB          // tile buffers (TMA); the rounds run in place
         + 4u * (G::NWD + 2)             // round bits, a zero word at each end
         + 8u * G::NWD                   // per row: {bit word, ones before it within its warp}
         + 4u * kFWarps                  // ones per warp
         + 4u * 6u * (2u << K)           // per class: count, offset, start, prefix, matrix base, start - offset
         + (MATRIX ? 0u : 4u * kFewNodes * ((1u << K) * 2u + (2u << K) * 3u))  // per node: digit counts,
                                         // start - offset; per (class, node) run: length, offset, start
         + 4u * 8u                       // zeros per round, flags
         + 72u;                          // mbarriers, tickets
}

struct FusedArgs {
  const uint8_t *in;   // T_l (S for level 0), 16-byte aligned
  int in_padded;       // in holds whole tiles
  uint8_t *out;        // T_{l+K}; null on the last pass
  uint32_t n, L, level, NT;
  uint64_t W;
  uint32_t *bits;      // bitmaps, row m at bits + m * W; rows level+1.. are zero on entry
  int matrix;          // wavelet matrix (one node per level) or tree
  const uint32_t *F;   // tree: F_m at F + 2^m - 2 (1 <= m <= L-1)
  const uint32_t *mtot;  // matrix: symbols per digit (2^K)
  const uint32_t *tcnt;  // symbols per digit and tile: digit d of tile t at tcnt[d * NT + t]
  const uint32_t *tpre;  // exclusive prefix of tcnt over the tiles, same layout
  uint32_t *ticket;
  uint32_t spin_limit;
  int *err;
};

// Class index helpers: heap slot h = 2^i - 1 + c for class c of granularity i.
__device__ __forceinline__ uint32_t gran_of(uint32_t h) { return 31u - __clz(h + 1u); }
__device__ __forceinline__ uint32_t rev_bits(uint32_t c, uint32_t i) { return i ? __brev(c) >> (32u - i) : 0u; }

// Phase 1 of a round: this warp's V rows of the image into v[] (masked to
// L bits on the first round, MASK), and the ballot of bit `sh` of each row,
// which lane 0 stores at words[r]; lane r returns row r's word.  Positions
// at or past nv read as 0 (bit 0).
template <typename Sym, uint32_t V, bool FULL, bool MASK>
__device__ __forceinline__ uint32_t round_bits(const Sym *X, uint32_t x0, uint32_t nv, uint32_t sh,
                                               uint32_t mask, uint32_t *words, uint32_t (&v)[V]) {
  static_assert(V == 32, "one row word per lane");
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t bm = 1u << sh;
#pragma unroll
  for (uint32_t r = 0; r < V; ++r) {
    const uint32_t x = x0 + 32 * r;
    uint32_t s = (FULL || x < nv) ? (uint32_t)X[x] : 0u;
    if (MASK) s &= mask;
    v[r] = s;
    const uint32_t b = __ballot_sync(0xFFFFFFFFu, (s & bm) != 0u);
    if (lane == 0) words[r] = b;
  }
  __syncwarp();
  return words[lane];
}

// Phase 2 of a round: the stable 2-way split of the image in place.  Row r's
// {bit word, ones before it within the warp} is wp[r]; a symbol with t ones
// before it in the warp goes to one_base + t (bit 1) or zero_base - t
// (bit 0), where the bases fold in the warp's offset.
template <typename Sym, uint32_t V, uint32_t TS, bool FULL>
__device__ __forceinline__ void round_split(Sym *X, const uint2 *wp, uint32_t x0, uint32_t nv,
                                            uint32_t one_base, uint32_t zero_base, const uint32_t (&v)[V]) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (uint32_t r = 0; r < V; ++r) {
    const uint2 w = wp[r];
    const uint32_t t = w.y + __popc(w.x & lt);
    const uint32_t dest = (w.x & (1u << lane)) ? one_base + t : zero_base + 32 * r - t;
    if (FULL) X[dest & (TS - 1)] = (Sym)v[r];
    else if (x0 + 32 * r < nv && dest < nv) X[dest] = (Sym)v[r];
  }
}

template <int SB, int K, bool MATRIX>
__global__ void __launch_bounds__(kFThreads, SB == 4 ? 4 : 3) k_fused(FusedArgs a) {
  using G = FGeom<SB>;
  using Sym = typename SymT<SB>::type;
  constexpr uint32_t V = G::V, TS = G::TS, NWD = G::NWD;
  constexpr uint32_t D = 1u << K, NH = 2u << K, SP = kFewNodes;
  extern __shared__ __align__(128) uint8_t smem[];
  TilePipe<SB, TS / 32, G::DEPTH> pipe;  // tiles of TS symbols, tickets two ahead
  pipe.sIn0 = smem;
  pipe.sIn1 = smem + (G::DEPTH - 1) * TS * SB;
  uint32_t *const sBits = reinterpret_cast<uint32_t *>(smem + G::DEPTH * TS * SB);
  uint2 *const sWP = reinterpret_cast<uint2 *>(sBits + NWD + 2);  // NWD + 2 words: 8-byte aligned
  uint32_t *const sWarpOnes = reinterpret_cast<uint32_t *>(sWP + NWD);
  uint32_t *const sCnt = sWarpOnes + kFWarps;  // per heap slot
  uint32_t *const sOff = sCnt + NH;
  uint32_t *const sGb = sOff + NH;
  uint32_t *const sGx = sGb + NH;
  uint32_t *const sMb = sGx + NH;
  uint32_t *const sDelta = sMb + NH;  // digit d: start of its run in T_{l+K} minus its offset in the tile
  // tiles over a few nodes (tree only): node j = node - first node of the tile
  uint32_t *const sCntN = sDelta + NH;                        // [j][digit] symbols
  uint32_t *const sDeltaN = sCntN + (MATRIX ? 0 : SP * D);    // [j][digit] start - offset in T_{l+K}
  uint32_t *const sRunLen = sDeltaN + (MATRIX ? 0 : SP * D);  // [class][j] run of node j in the class
  uint32_t *const sRunOff = sRunLen + (MATRIX ? 0 : NH * SP);
  uint32_t *const sRunG = sRunOff + (MATRIX ? 0 : NH * SP);
  uint32_t *const sZt = sRunG + (MATRIX ? 0 : NH * SP);       // K words
  uint32_t *const sFlag = sZt + 4;  // [0] nodes of the tile: 1, few (< SP) = 2, more = 0; [1] first node; [2] span
  pipe.bar = reinterpret_cast<uint64_t *>(smem + ((fused_smem_bytes<SB, K, MATRIX>() - 72u + 7u) & ~7u));
  pipe.ring = reinterpret_cast<uint32_t *>(pipe.bar + 2);
  pipe.in = a.in;
  pipe.in_padded = a.in_padded;
  pipe.n = a.n;
  pipe.NT = a.NT;
  pipe.ticket = a.ticket;

  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lmask = (1u << a.L) - 1u;  // L <= 26
  const uint32_t ps = a.L - a.level;        // node of a symbol: its top l bits
  if (tid == 0) {
    sBits[0] = 0;
    sBits[NWD + 1] = 0;
  }
  if (MATRIX && tid < NH - 1) {
    // start of each class of granularity >= 1 in T_{l+i}: the classes whose
    // bits, read from the last to the first, are smaller come first
    const uint32_t h = tid, i = gran_of(h), c = h + 1 - (1u << i);
    uint32_t b = 0;
    if (i) {
      const uint32_t rc = rev_bits(c, i), span = 1u << (K - i);
      for (uint32_t c2 = 0; c2 < (1u << i); ++c2)
        if (rev_bits(c2, i) < rc)
          for (uint32_t d = c2 * span; d < (c2 + 1) * span; ++d) b += __ldg(&a.mtot[d]);
    }
    sMb[h] = b;
  }
  if (tid == 0) pipe.prologue();
  __syncthreads();
  // thread d < D: the count of digit d in a tile; D <= thread < 2D: its prefix
  auto tile_word = [&](uint32_t t) -> uint32_t {
    if (t >= a.NT || tid >= 2 * D) return 0u;
    return tid < D ? __ldcg(&a.tcnt[(uint64_t)tid * a.NT + t]) : __ldcg(&a.tpre[(uint64_t)(tid - D) * a.NT + t]);
  };
  uint32_t pre = tile_word(pipe.ring[0]);

  const uint32_t xw = warp * 32 * V;  // this warp's first image position
  for (uint32_t it = 0;; ++it) {
    const uint32_t tile = pipe.ring[it % 3];
    if (tile >= a.NT) break;
    const uint32_t nxt = pipe.ring[(it + 1) % 3];
    uint32_t nn = 0;
    if (tid == 0) nn = pipe.advance(it, nxt);
    const uint32_t pre_next = tile_word(nxt);
    const bool ok = pipe.wait(it, a.spin_limit, a.err);
    if (__syncthreads_or(!ok)) {
      pipe.drain(it, a.spin_limit, a.err);
      __syncthreads();
      break;
    }
    const uint64_t start = (uint64_t)tile * TS;
    const uint32_t nv = (uint32_t)umin64(TS, a.n - start);
    uint8_t *const buf = pipe.data(it);
    if (!a.in_padded && ((nv * SB) & 15u)) {  // tail bytes the bulk copy left out
      for (uint32_t i = ((nv * SB) & ~15u) + tid; i < nv * SB; i += kFThreads) buf[i] = a.in[start * SB + i];
      __syncthreads();
    }
    Sym *const X = reinterpret_cast<Sym *>(buf);

    // ---- class tables of the tile
    if (tid < D) sCnt[D - 1 + tid] = pre;
    else if (tid < 2 * D) sGx[D - 1 + (tid - D)] = pre;
    if (!MATRIX) {
      for (uint32_t i = tid; i < SP * D; i += kFThreads) sCntN[i] = 0;
      if (tid == 2 * D) {
        // nodes of the tile (T_l is ordered by node)
        uint32_t kind = 1, node = 0, span = 0;
        if (a.level) {
          node = ((uint32_t)X[0] & lmask) >> ps;
          span = (((uint32_t)X[nv - 1] & lmask) >> ps) - node;
          kind = span == 0 ? 1u : span < SP ? 2u : 0u;
        }
        sFlag[0] = kind;
        sFlag[1] = node;
        sFlag[2] = span;
      }
    }
    __syncthreads();
    const uint32_t kind = MATRIX ? 1u : sFlag[0];
    const bool single = kind == 1, few = kind == 2;
    const uint32_t p0 = MATRIX ? 0u : sFlag[1], span = MATRIX ? 0u : sFlag[2];
    if (few) {  // digits of every node of the tile
      const uint32_t dsh = a.L - a.level - K;
      for (uint32_t x = tid; x < nv; x += kFThreads) {
        const uint32_t v = (uint32_t)X[x] & lmask;
        atomicAdd(&sCntN[((v >> ps) - p0) * D + ((v >> dsh) & (D - 1))], 1u);
      }
    }
    if (tid < D - 1) {  // coarser classes: sums over their digits
      const uint32_t h = tid, gi = gran_of(h), c = h + 1 - (1u << gi), sp = 1u << (K - gi);
      uint32_t cn = 0, gx = 0;
      for (uint32_t d = c * sp; d < (c + 1) * sp; ++d) {
        cn += sCnt[D - 1 + d];
        gx += sGx[D - 1 + d];
      }
      sCnt[h] = cn;
      sGx[h] = gx;
    }
    __syncthreads();
    if (tid < NH - 1) {
      const uint32_t h = tid, gi = gran_of(h), c = h + 1 - (1u << gi);
      uint32_t off = 0;
      if (gi) {
        const uint32_t rc = rev_bits(c, gi);
        for (uint32_t c2 = 0; c2 < (1u << gi); ++c2)
          if (rev_bits(c2, gi) < rc) off += sCnt[(1u << gi) - 1 + c2];
      }
      sOff[h] = off;
      uint32_t gb = 0;
      if (gi && (gi < K || a.out)) {  // the last pass writes no T_{l+K}
        if (MATRIX) gb = sMb[h] + sGx[h];
        else if (single) gb = __ldg(&a.F[(1u << (a.level + gi)) - 2u + ((p0 << gi) | c)]) + sGx[h];
      }
      sGb[h] = gb;
      if (gi == K) sDelta[c] = gb - off;
    }
    if (few) {  // symbols of node j in class h (granularity >= 1)
      for (uint32_t t = tid; t < (NH - 2) * (span + 1); t += kFThreads) {
        const uint32_t h = 1 + t / (span + 1), j = t % (span + 1);
        const uint32_t gi = gran_of(h), c = h + 1 - (1u << gi), sp = 1u << (K - gi);
        uint32_t cn = 0;
        for (uint32_t d = c * sp; d < (c + 1) * sp; ++d) cn += sCntN[j * D + d];
        sRunLen[h * SP + j] = cn;
      }
    }
    if (tid < K) {  // zeros of round tid: classes of the next granularity ending in 0
      uint32_t z = 0;
      for (uint32_t c = 0; c < (1u << tid); ++c) z += sCnt[(2u << tid) - 1 + 2 * c];
      sZt[tid] = z;
    }
    __syncthreads();
    if (few) {
      // node j's run of class h starts after the runs of nodes < j in the
      // class segment; its symbols go to F of node j's child plus G of the
      // class plus their place in the class segment
      for (uint32_t t = tid; t < (NH - 2) * (span + 1); t += kFThreads) {
        const uint32_t h = 1 + t / (span + 1), j = t % (span + 1);
        const uint32_t gi = gran_of(h), c = h + 1 - (1u << gi);
        uint32_t before = 0;
        for (uint32_t j2 = 0; j2 < j; ++j2) before += sRunLen[h * SP + j2];
        sRunOff[h * SP + j] = sOff[h] + before;
        uint32_t g = 0;
        if (sRunLen[h * SP + j] && (gi < K || a.out)) {
          const uint32_t f = __ldg(&a.F[(1u << (a.level + gi)) - 2u + (((p0 + j) << gi) | c)]) + sGx[h];
          g = f + before;
          if (gi == K) sDeltaN[j * D + c] = f - sOff[h];
        }
        sRunG[h * SP + j] = g;
      }
      __syncthreads();
    }

    const bool full = nv == TS;
    uint32_t v[V];
#pragma unroll 1
    for (uint32_t i = 0; i < K; ++i) {
      const uint32_t sh = a.L - 1 - a.level - i;  // bit of level l+i
      // ---- phase 1: this round's bit of every symbol, as ballot words (the
      // first round masks the symbols to L bits; later rounds hold masked ones)
      uint32_t *const words = sBits + 1 + warp * V;
      uint32_t mine;
      if (i == 0)
        mine = full ? round_bits<Sym, V, true, true>(X, xw + lane, nv, sh, lmask, words, v)
                    : round_bits<Sym, V, false, true>(X, xw + lane, nv, sh, lmask, words, v);
      else
        mine = full ? round_bits<Sym, V, true, false>(X, xw + lane, nv, sh, lmask, words, v)
                    : round_bits<Sym, V, false, false>(X, xw + lane, nv, sh, lmask, words, v);
      const uint32_t pc = __popc(mine);
      uint32_t incl = pc;
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
      }
      sWP[warp * V + lane] = make_uint2(mine, incl - pc);
      if (lane == 31) sWarpOnes[warp] = incl;
      __syncthreads();

      // ---- phase 2: bits out, then the stable split of the image
      uint32_t Pw = 0;
      for (uint32_t w2 = 0; w2 < warp; ++w2) Pw += sWarpOnes[w2];
      const uint32_t m = a.level + i;
      uint32_t *const row = a.bits + (uint64_t)m * a.W;
      if (i == 0) {
        const uint64_t widx = (uint64_t)tile * NWD + tid;
        if (tid < NWD && widx < a.W) row[widx] = sBits[1 + tid];
      } else if (single) {
        for (uint32_t c = warp; c < (1u << i); c += kFWarps) {
          const uint32_t h = (1u << i) - 1 + c;
          const uint32_t len = sCnt[h];
          if (len && sGb[h] + (uint64_t)len <= a.n) warp_bit_run(sBits, sOff[h], row, sGb[h], len);
        }
      } else if (few) {
        // one run per (class, node)
        const uint32_t runs = (1u << i) * (span + 1);
        for (uint32_t t = warp; t < runs; t += kFWarps) {
          const uint32_t h = (1u << i) - 1 + t / (span + 1), j = t % (span + 1);
          const uint32_t len = sRunLen[h * SP + j], g = sRunG[h * SP + j];
          if (len && g + (uint64_t)len <= a.n) warp_bit_run(sBits, sRunOff[h * SP + j], row, g, len);
        }
      } else if (!MATRIX) {
        // a tile over many nodes: destinations of each row in T_{l+i}, one
        // run per stretch of consecutive destinations
#pragma unroll
        for (uint32_t r = 0; r < V; ++r) {
          const uint32_t x = xw + 32 * r + lane;
          const bool valid = x < nv;
          const uint32_t word = sBits[1 + warp * V + r];
          uint32_t gpos = 0;
          if (valid) {
            const uint32_t q = v[r] >> (a.L - m);
            const uint32_t h = (1u << i) - 1 + (q & ((1u << i) - 1u));
            gpos = __ldg(&a.F[(1u << m) - 2u + q]) + sGx[h] + (x - sOff[h]);
          }
          const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, gpos, 1);
          const bool st = valid && (lane == 0 || prev + 1u != gpos);
          const uint32_t starts = __ballot_sync(0xFFFFFFFFu, st);
          const uint32_t vm = __ballot_sync(0xFFFFFFFFu, valid);
          if (st && gpos < a.n) {
            const uint32_t later = starts & ~((2u << lane) - 1u);
            const uint32_t end = later ? (uint32_t)__ffs(later) - 1u : (uint32_t)__popc(vm);
            const uint32_t len = end - lane;
            const uint32_t b = (word >> lane) & (len >= 32 ? ~0u : ((1u << len) - 1u));
            if (b) {
              const uint32_t s = gpos & 31u;
              atomicOr(&row[gpos >> 5], b << s);
              if (s && s + len > 32u && (gpos >> 5) + 1u < a.W) {
                const uint32_t hb = b >> (32u - s);
                if (hb) atomicOr(&row[(gpos >> 5) + 1], hb);
              }
            }
          }
        }
      }
      if ((i + 1 < K) || a.out != nullptr) {
        const uint32_t one_base = sZt[i] + Pw, zero_base = xw + lane - Pw;
        if (full) round_split<Sym, V, TS, true>(X, sWP + warp * V, xw + lane, nv, one_base, zero_base, v);
        else round_split<Sym, V, TS, false>(X, sWP + warp * V, xw + lane, nv, one_base, zero_base, v);
      }
      __syncthreads();
    }

    // ---- T_{l+K}: the final image, class by class
    if (a.out) {
      Sym *const out = reinterpret_cast<Sym *>(a.out);
      const uint32_t m = a.level + K;
      const uint32_t shK = a.L - m;
      if (single || few) {
        // the class (and node) of a symbol gives its destination: x + (start - offset)
        const uint32_t *delta = single ? sDelta : sDeltaN;
        for (uint32_t x = tid; x < nv; x += kFThreads) {
          const uint32_t s = X[x];
          const uint32_t j = few ? (s >> ps) - p0 : 0u;
          const uint32_t dest = x + delta[j * D + ((s >> shK) & (D - 1))];
          if (dest < a.n) out[dest] = (Sym)s;
        }
      } else if (!MATRIX) {
        for (uint32_t x = tid; x < nv; x += kFThreads) {
          const uint32_t s = X[x];
          const uint32_t h = D - 1 + ((s >> shK) & (D - 1));
          const uint32_t dest = __ldg(&a.F[(1u << m) - 2u + (s >> shK)]) + sGx[h] + (x - sOff[h]);
          if (dest < a.n) out[dest] = (Sym)s;
        }
      }
    }
    if (tid == 0) pipe.ring[(it + 2) % 3] = nn;
    __syncthreads();
    if (G::DEPTH == 1 && tid == 0) pipe.after_tile(nxt);
    pre = pre_next;
  }
}

// ------------------------------------------------------------------ digit counts
struct CountArgs {
  const uint8_t *in;   // T_l, 16-byte aligned
  uint32_t n, L, level, NT;
  uint32_t sigma;      // range check of the input symbols (first pass), 0 = none
  uint32_t *tcnt;      // digit d of tile t at tcnt[d * NT + t]
  uint32_t *ncount;    // tree: symbols per node of level level+K (zeroed), else null;
                       // tile t adds to copy t & rep_mask (2^top counters each)
  uint32_t rep_mask, top;
  int *err;
};

constexpr uint32_t kSpanKeyed = 32;  // tiles over fewer nodes count them in shared memory

// Count one symbol of a tile that spans nodes into its node of level l+K:
// in shared memory (key = node offset from the tile's first node, digit)
// when the tile spans fewer than kSpanKeyed nodes, else straight to global
// memory (such tiles hold many small nodes, so there is no hot counter).
template <uint32_t K>
__device__ __forceinline__ void count_node(const CountArgs &a, uint32_t *nc, uint32_t *sNC, uint32_t v,
                                           uint32_t p0, bool keyed) {
  const uint32_t q = v >> (a.L - a.level - K);
  if (keyed) atomicAdd(&sNC[q - (p0 << K)], 1u);
  else atomicAdd(&nc[q], 1u);
}

// Symbols of each digit in each tile of T_l (tiles of the k-level pass).
// One CTA per tile; per-thread counters in shared memory (thread t owns
// column t, so there are no bank conflicts and no atomics).  For the tree
// the kernel also counts the symbols of every node of level l+K, which the
// pass's tables need: a tile within one node adds its digit counts to that
// node's 2^K children.
template <int SB, int K>
__global__ void __launch_bounds__(kFThreads) k_tilecount(CountArgs a) {
  using G = FGeom<SB>;
  using Sym = typename SymT<SB>::type;
  constexpr uint32_t TS = G::TS, D = 1u << K;
  __shared__ uint32_t sH[D * kFThreads];
  __shared__ uint32_t sNC[kSpanKeyed * D];
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = blockIdx.x;
  const uint64_t start = (uint64_t)tile * TS;
  const uint32_t nv = (uint32_t)umin64(TS, a.n - start);
  const uint32_t lmask = (1u << a.L) - 1u, dsh = a.L - a.level - K;
#pragma unroll
  for (uint32_t d = 0; d < D; ++d) sH[d * kFThreads + tid] = 0;
  const uint8_t *base = a.in + start * SB;
  const Sym *syms = reinterpret_cast<const Sym *>(base);
  // the tile's nodes of level l (T_l is ordered by node)
  const uint32_t ps = a.L - a.level;
  const bool tree_node = a.ncount != nullptr && a.level != 0;
  const uint32_t p0 = tree_node ? (((uint32_t)syms[0] & lmask) >> ps) : 0u;
  const uint32_t p1 = tree_node ? (((uint32_t)syms[nv - 1] & lmask) >> ps) : 0u;
  const bool nodes = a.ncount != nullptr && p0 != p1;  // count nodes per symbol
  // this tile's copy of the node counters: the tiles of one large node
  // would otherwise all add to the same 2^K counters
  uint32_t *const nc = a.ncount ? a.ncount + ((size_t)(tile & a.rep_mask) << a.top) : nullptr;
  const bool keyed = p1 - p0 < kSpanKeyed;
  if (nodes && keyed)
    for (uint32_t i = tid; i < kSpanKeyed * D; i += kFThreads) sNC[i] = 0;
  if (nodes) __syncthreads();
  const uint32_t full = (nv * SB) >> 4;  // whole 16-byte chunks
  uint32_t mx = 0;
  // all of this thread's loads are issued before any is counted
  constexpr uint32_t CH = TS * SB / 16 / kFThreads;
  uint4 w[CH];
#pragma unroll
  for (uint32_t c = 0; c < CH; ++c) {
    const uint32_t q = tid + c * kFThreads;
    w[c] = q < full ? __ldg(reinterpret_cast<const uint4 *>(base) + q) : make_uint4(0, 0, 0, 0);
  }
#pragma unroll
  for (uint32_t c = 0; c < CH; ++c) {
    if (tid + c * kFThreads >= full) break;
    const uint32_t words[4] = {w[c].x, w[c].y, w[c].z, w[c].w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int e = 0; e < 4 / SB; ++e) {
        const uint32_t raw = SB == 4 ? words[k] : (words[k] >> (8 * SB * e)) & ((1u << (8 * SB)) - 1u);
        mx = max(mx, raw);
        sH[(((raw & lmask) >> dsh) & (D - 1)) * kFThreads + tid] += 1u;
        if (nodes) count_node<K>(a, nc, sNC, raw & lmask, p0, keyed);
      }
    }
  }
  for (uint32_t x = full * (16 / SB) + tid; x < nv; x += kFThreads) {
    const uint32_t raw = syms[x];
    mx = max(mx, raw);
    sH[(((raw & lmask) >> dsh) & (D - 1)) * kFThreads + tid] += 1u;
    if (nodes) count_node<K>(a, nc, sNC, raw & lmask, p0, keyed);
  }
  if (a.sigma && mx >= a.sigma) latch_error(a.err, WT_ERR_SYMBOL);
  __syncthreads();
  for (uint32_t d = warp; d < D; d += kFWarps) {
    uint32_t s = 0;
    for (uint32_t k = lane; k < kFThreads; k += 32) s += sH[d * kFThreads + k];
    s = __reduce_add_sync(0xFFFFFFFFu, s);
    if (lane == 0) {
      a.tcnt[(uint64_t)d * a.NT + tile] = s;
      if (a.ncount && !nodes && s) atomicAdd(&nc[(p0 << K) | d], s);  // one node
    }
  }
  if (nodes && keyed) {
    for (uint32_t i = tid; i < kSpanKeyed * D && (i >> K) <= p1 - p0; i += kFThreads)
      if (sNC[i]) atomicAdd(&nc[(p0 << K) + i], sNC[i]);
  }
}

struct TileScanArgs {
  const uint32_t *tcnt;
  uint32_t *tpre;      // exclusive prefix over the tiles, per digit
  uint32_t *tot;       // symbols per digit (may be null)
  uint32_t NT;
  uint32_t *ncount;    // tree: rep copies of nwords node counters, summed into the first
  uint32_t rep, nwords;
};

// One CTA per digit: exclusive scan of its NT tile counts.  The CTAs also
// sum the copies of the node counters into the first copy.
__global__ void __launch_bounds__(1024) k_tilescan(TileScanArgs a) {
  constexpr uint32_t ITEMS = 4, CH = 1024 * ITEMS;
  __shared__ uint32_t s_warp[33];
  const uint32_t d = blockIdx.x, tid = threadIdx.x;
  if (a.ncount && a.rep > 1)
    for (uint32_t i = d * 1024 + tid; i < a.nwords; i += gridDim.x * 1024) {
      uint32_t s = 0;
      for (uint32_t r = 0; r < a.rep; ++r) s += __ldcg(&a.ncount[(size_t)r * a.nwords + i]);
      a.ncount[i] = s;
    }
  const uint32_t *c = a.tcnt + (uint64_t)d * a.NT;
  uint32_t *p = a.tpre + (uint64_t)d * a.NT;
  uint32_t carry = 0;
  for (uint32_t base = 0; base < a.NT; base += CH) {
    const uint32_t i0 = base + tid * ITEMS;
    uint32_t v[ITEMS], sum = 0;
#pragma unroll
    for (uint32_t i = 0; i < ITEMS; ++i) {
      v[i] = i0 + i < a.NT ? __ldcg(&c[i0 + i]) : 0u;
      sum += v[i];
    }
    uint32_t total;
    uint32_t run = carry + block_exclusive_scan<1024>(sum, s_warp, &total);
#pragma unroll
    for (uint32_t i = 0; i < ITEMS; ++i) {
      if (i0 + i < a.NT) p[i0 + i] = run;
      run += v[i];
    }
    carry += total;
    __syncthreads();
  }
  if (tid == 0 && a.tot) a.tot[d] = carry;
}

// ------------------------------------------------------------------ directories
struct DirArgs {
  const uint32_t *bits;        // first row
  unsigned long long *rank;    // its directory row
  unsigned long long *zeros;   // its zero count
  uint32_t levels, n, NB, nchunks;
  uint64_t W;
  uint32_t *ticket;
  Lookback lb;
};

// D[b] = ones of the row before bit 512 b, D[NB] = all ones, zeros = n - D[NB];
// one look-back segment per row.  A CTA takes kScanChunk blocks: thread t
// counts blocks t, t + kScanThreads, ... (adjacent threads read adjacent
// 64-byte blocks), the counts are regrouped in shared memory so that thread
// t scans the kScanItems consecutive blocks from kScanItems t on, and the
// entries go back out in the loading order.  (Each thread reading its own
// kScanItems consecutive blocks put the lanes of a load 512 bytes apart.)
__global__ void __launch_bounds__(kScanThreads) k_dir(DirArgs a) {
  static_assert(kScanItems == 8, "two 16-byte shared words per thread");
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_tile, s_P;
  __shared__ __align__(16) uint32_t s_c[kScanChunk];  // counts, then entries minus the chunk's prefix
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= a.levels * a.nchunks) return;
  const uint32_t lvl = tile / a.nchunks, chunk = tile - lvl * a.nchunks;
  const uint32_t *rowp = a.bits + (uint64_t)lvl * a.W;
  const uint32_t cb = chunk * kScanChunk;  // the chunk's first block
#pragma unroll
  for (uint32_t i = 0; i < kScanItems; ++i) {
    const uint32_t b = cb + i * kScanThreads + tid;
    uint32_t c = 0;
    if (b < a.NB) {
      const uint4 *p = reinterpret_cast<const uint4 *>(rowp + 16ull * b);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 w = __ldg(p + q);
        c += __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
      }
    }
    s_c[i * kScanThreads + tid] = c;
  }
  __syncthreads();
  uint4 *const s_c4 = reinterpret_cast<uint4 *>(s_c);
  const uint4 c0 = s_c4[2 * tid], c1 = s_c4[2 * tid + 1];  // blocks cb + 8 tid .. cb + 8 tid + 7
  const uint32_t sum = c0.x + c0.y + c0.z + c0.w + c1.x + c1.y + c1.z + c1.w;
  uint32_t total;
  const uint32_t excl = block_exclusive_scan<kScanThreads>(sum, s_warp, &total);
  if (tid < 32) {
    const uint32_t P = lookback(a.lb, tile, lvl * a.nchunks, total);
    if (tid == 0) s_P = P;
  }
  uint4 e0, e1;
  e0.x = excl;
  e0.y = e0.x + c0.x;
  e0.z = e0.y + c0.y;
  e0.w = e0.z + c0.z;
  e1.x = e0.w + c0.w;
  e1.y = e1.x + c1.x;
  e1.z = e1.y + c1.y;
  e1.w = e1.z + c1.z;
  s_c4[2 * tid] = e0;  // this thread's own words: read above by it alone
  s_c4[2 * tid + 1] = e1;
  __syncthreads();
  const uint32_t P = s_P;
  unsigned long long *rk = a.rank + (uint64_t)lvl * (a.NB + 1);
#pragma unroll
  for (uint32_t i = 0; i < kScanItems; ++i) {
    const uint32_t b = cb + i * kScanThreads + tid;
    if (b < a.NB) rk[b] = P + s_c[i * kScanThreads + tid];
  }
  if (chunk == a.nchunks - 1 && tid == 0) {
    rk[a.NB] = P + total;
    a.zeros[lvl] = (unsigned long long)(a.n - (P + total));
  }
}

// ------------------------------------------------------------------ F tables
struct FTabArgs {
  const unsigned long long *E;  // E[v] = symbols whose top Ltop bits are < v, 2^Ltop + 1 entries
  uint32_t *F;                  // F_m at F + 2^m - 2
  uint32_t L, K, Ltop, m_lo, m_hi, nblocks;
  uint32_t *ticket;
  Lookback lb;
};

// Level m (m_lo <= m <= m_hi, m_hi <= Ltop) is built by the pass starting at
// l = K floor((m-1)/K), as granularity i = m - l.  For node q = p 2^i + c
// of level m:
//   F_m[q] = E[q << (Ltop-m)] - sum over p' < p of |node p' 2^i + c|.
// Blocks walk levels, then classes c, then chunks of p; every (m, c) is one
// look-back segment.
__global__ void __launch_bounds__(kScanThreads) k_fuse_tables(FTabArgs a) {
  __shared__ uint32_t s_warp[33];
  __shared__ uint32_t s_tile, s_P;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= a.nblocks) return;
  uint32_t first = 0, m = a.m_lo, l = 0, i = 1, nch = 1;
  for (; m <= a.m_hi; ++m) {
    l = a.K * ((m - 1) / a.K);
    i = m - l;
    nch = ((1u << l) + kScanChunk - 1) / kScanChunk;
    if (tile < first + (nch << i)) break;
    first += nch << i;
  }
  const uint32_t c = (tile - first) / nch, chunk = (tile - first) - c * nch;
  const uint32_t seg_first = first + c * nch;
  const uint32_t sh = a.Ltop - m, cntp = 1u << l;
  const uint32_t p0 = chunk * kScanChunk + tid * kScanItems;
  uint32_t sz[kScanItems];
  uint32_t sum = 0;
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k) {
    const uint32_t p = p0 + k;
    const uint64_t q = ((uint64_t)p << i) | c;
    sz[k] = p < cntp ? (uint32_t)(a.E[(q + 1) << sh] - a.E[q << sh]) : 0u;
    sum += sz[k];
  }
  uint32_t total;
  const uint32_t excl = block_exclusive_scan<kScanThreads>(sum, s_warp, &total);
  if (tid < 32) {
    const uint32_t P = lookback(a.lb, tile, seg_first, total);
    if (tid == 0) s_P = P;
  }
  __syncthreads();
  uint32_t run = s_P + excl;
  uint32_t *Fm = a.F + (1u << m) - 2u;
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k) {
    const uint32_t p = p0 + k;
    if (p < cntp) {
      const uint64_t q = ((uint64_t)p << i) | c;
      Fm[q] = (uint32_t)a.E[q << sh] - run;
    }
    run += sz[k];
  }
}

int cuda_err(cudaError_t e) {
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? WT_ERR_OOM : WT_ERR_CUDA;
}

int last_error() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WT_OK : cuda_err(e);
}

template <int SB, int K, bool MATRIX>
int launch_k(wt_tree *t, cudaStream_t st, const FusedArgs &a) {
  auto kern = k_fused<SB, K, MATRIX>;
  constexpr uint32_t sm = fused_smem_bytes<SB, K, MATRIX>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return cuda_err(e);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kFThreads, sm) != cudaSuccess) {
    (void)cudaGetLastError();
    occ = 1;
  }
  occ = std::max(occ, 1);
  if (t->cfg.ctas_per_sm) occ = std::min<int>(occ, (int)t->cfg.ctas_per_sm);
  const int grid = std::max(1, std::min<int>((int)a.NT, occ * t->sms));
  kern<<<grid, kFThreads, sm, st>>>(a);
  return last_error();
}

template <int SB, bool MATRIX>
int launch_shape(wt_tree *t, cudaStream_t st, const FusedArgs &a, uint32_t K) {
  switch (K) {
    case 1: return launch_k<SB, 1, MATRIX>(t, st, a);
    case 2: return launch_k<SB, 2, MATRIX>(t, st, a);
    case 3: return launch_k<SB, 3, MATRIX>(t, st, a);
    case 4: return launch_k<SB, 4, MATRIX>(t, st, a);
  }
  return WT_ERR_ARG;
}

template <int SB>
int launch_sb(wt_tree *t, cudaStream_t st, const FusedArgs &a, uint32_t K) {
  return a.matrix ? launch_shape<SB, true>(t, st, a, K) : launch_shape<SB, false>(t, st, a, K);
}

template <int SB>
int launch_count_sb(cudaStream_t st, const CountArgs &a, uint32_t K) {
  switch (K) {
    case 1: k_tilecount<SB, 1><<<a.NT, kFThreads, 0, st>>>(a); break;
    case 2: k_tilecount<SB, 2><<<a.NT, kFThreads, 0, st>>>(a); break;
    case 3: k_tilecount<SB, 3><<<a.NT, kFThreads, 0, st>>>(a); break;
    case 4: k_tilecount<SB, 4><<<a.NT, kFThreads, 0, st>>>(a); break;
    default: return WT_ERR_ARG;
  }
  return last_error();
}

}  // namespace

namespace wtk {

uint32_t fused_tile_symbols(uint32_t symbol_bytes) {
  return symbol_bytes == 4 ? FGeom<4>::TS : symbol_bytes == 2 ? FGeom<2>::TS : FGeom<1>::TS;
}

uint32_t fused_tables_blocks(uint32_t L, uint32_t K) { return L >= 2 ? fused_tables_blocks_range(1, L - 1, K) : 0u; }

uint32_t fused_tables_blocks_range(uint32_t m_lo, uint32_t m_hi, uint32_t K) {
  uint32_t nb = 0;
  for (uint32_t m = m_lo; m <= m_hi && m >= 1; ++m) {
    const uint32_t l = K * ((m - 1) / K), i = m - l;
    nb += (((1u << l) + kScanChunk - 1) / kScanChunk) << i;
  }
  return nb;
}

uint32_t fused_dir_chunks(uint64_t NB) { return (uint32_t)((NB + kScanChunk - 1) / kScanChunk); }

// Copies of the tree's node counters of level `top`: as many as fit in the
// 2^L-word counter array, at most 256.
uint32_t node_copies(const wt_tree *t, uint32_t top) {
  return t->shape == WT_SHAPE_TREE ? std::min<uint32_t>(256u, 1u << (t->L - top)) : 1u;
}

int fused_count(wt_tree *t, cudaStream_t st, const uint8_t *in, uint32_t level, uint32_t K, bool check) {
  CountArgs a;
  a.in = in;
  a.n = (uint32_t)t->n;
  a.L = t->L;
  a.level = level;
  a.NT = (uint32_t)t->NTf;
  a.sigma = check ? t->sigma : 0u;
  a.tcnt = t->d_fcount;
  a.ncount = t->shape == WT_SHAPE_TREE ? t->d_hist : nullptr;
  a.top = level + K;
  const uint32_t rep = node_copies(t, a.top);
  a.rep_mask = rep - 1;
  a.err = reinterpret_cast<int *>(t->d_ctrl + kCtrlErr);
  if (a.ncount && rep > 1) {
    const cudaError_t e = cudaMemsetAsync(a.ncount, 0, ((size_t)rep << a.top) * 4, st);
    if (e != cudaSuccess) return cuda_err(e);
  }
  switch (t->sb) {
    case 1: return launch_count_sb<1>(st, a, K);
    case 2: return launch_count_sb<2>(st, a, K);
    case 4: return launch_count_sb<4>(st, a, K);
  }
  return WT_ERR_ARG;
}

int fused_scan(wt_tree *t, cudaStream_t st, uint32_t level, uint32_t K) {
  TileScanArgs a;
  a.tcnt = t->d_fcount;
  a.tpre = t->d_fcount + ((uint64_t)t->NTf << t->fuse_k);
  a.tot = t->shape == WT_SHAPE_MATRIX ? t->d_hist : nullptr;
  a.NT = (uint32_t)t->NTf;
  a.ncount = t->shape == WT_SHAPE_TREE ? t->d_hist : nullptr;
  a.rep = node_copies(t, level + K);
  a.nwords = 1u << (level + K);
  k_tilescan<<<1u << K, 1024, 0, st>>>(a);
  return last_error();
}

int fused_pass(wt_tree *t, cudaStream_t st, const uint8_t *in, bool in_padded, uint8_t *out,
               uint32_t level, uint32_t K, uint32_t *ticket) {
  FusedArgs a;
  a.in = in;
  a.in_padded = in_padded ? 1 : 0;
  a.out = out;
  a.n = (uint32_t)t->n;
  a.L = t->L;
  a.level = level;
  a.NT = (uint32_t)t->NTf;
  a.W = t->W;
  a.bits = t->d_bits;
  const bool matrix = t->shape == WT_SHAPE_MATRIX;
  a.matrix = matrix ? 1 : 0;
  a.F = matrix ? nullptr : t->d_ftab;
  a.mtot = matrix ? t->d_hist : nullptr;
  a.tcnt = t->d_fcount;
  a.tpre = t->d_fcount + ((uint64_t)t->NTf << t->fuse_k);
  a.ticket = ticket;
  a.spin_limit = t->cfg.spin_limit ? t->cfg.spin_limit : kDefaultSpin;
  a.err = reinterpret_cast<int *>(t->d_ctrl + kCtrlErr);
  switch (t->sb) {
    case 1: return launch_sb<1>(t, st, a, K);
    case 2: return launch_sb<2>(t, st, a, K);
    case 4: return launch_sb<4>(t, st, a, K);
  }
  return WT_ERR_ARG;
}

int fused_tables(wt_tree *t, cudaStream_t st, uint32_t m_lo, uint32_t m_hi, uint32_t Ltop, const Lookback &lb,
                 uint32_t *ticket) {
  FTabArgs a;
  a.E = t->d_node_start;
  a.F = t->d_ftab;
  a.L = t->L;
  a.K = t->fuse_k;
  a.Ltop = Ltop;
  a.m_lo = m_lo;
  a.m_hi = m_hi;
  a.nblocks = m_hi >= m_lo ? fused_tables_blocks_range(m_lo, m_hi, t->fuse_k) : 0;
  a.ticket = ticket;
  a.lb = lb;
  if (!a.nblocks) return WT_OK;
  k_fuse_tables<<<a.nblocks, kScanThreads, 0, st>>>(a);
  return last_error();
}

int fused_dir(wt_tree *t, cudaStream_t st, uint32_t level0, uint32_t levels, const Lookback &lb,
              uint32_t *ticket) {
  DirArgs a;
  a.bits = t->d_bits + (uint64_t)level0 * t->W;
  a.rank = t->d_rank + (uint64_t)level0 * (t->NB + 1);
  a.zeros = t->d_zeros + level0;
  a.levels = levels;
  a.n = (uint32_t)t->n;
  a.NB = (uint32_t)t->NB;
  a.nchunks = fused_dir_chunks(t->NB);
  a.W = t->W;
  a.ticket = ticket;
  a.lb = lb;
  k_dir<<<a.levels * a.nchunks, kScanThreads, 0, st>>>(a);
  return last_error();
}

}  // namespace wtk
