// Batched access / rank / select over a built levelwise wavelet tree or
// wavelet matrix, one thread per query.  Definitions from Section 2 of the
// paper.
//
// Tree.  A position j of level l in node p (prefix p = top l bits) moves to
// level l+1 exactly as the build moved its symbol (Fig. 1's X_s + i - X[i]
// placement): to O_l[p] + j - R_l(j) on a 0 bit and to
// E_{l+1}[2p+1] - O_l[p] + R_l(j) on a 1 bit, R_l(j) = ones of level l before
// j; the build's node tables hold exactly {O_l[p], E_{l+1}[2p+1] - O_l[p]}
// for l <= L-2.  So every level costs one rank (access, rank) or one select
// (select, walking back up), with no node bounds.  The last level has no
// table: its node start is E[2p] (node starts) and the ones before it one
// extra rank.
//
// Matrix (Section 7).  A position moves to rank0(j) on a 0 bit and to
// Z_l + rank1(j) on a 1 bit, Z_l the zeros of level l.
//
// rank1 reads the block's cumulative count and at most four 16-byte loads of
// the block's bits; select finds the block by binary search between two
// sampled positions of the query index (every 4096-th one and every 4096-th
// zero of each level, built on the first select after a build), then scans
// the block's words.
#include <algorithm>
#include <cstdint>

#include "wt_dev.cuh"
#include "wt_internal.h"

using namespace wtk;

namespace {

constexpr uint32_t kSelSample = 4096;  // one sampled position per 4096 wanted bits

struct QTree {
  const uint32_t *bits;
  const unsigned long long *rank;
  const unsigned long long *zeros;
  const uint2 *tab;                 // tree: heap layout 2^l - 1 + p, levels 0..L-2
  const unsigned long long *E;      // tree: node starts, 2^L + 1 entries
  const uint32_t *sel;              // [L][2][sel_stride] sampled blocks (may be null)
  uint64_t W, NB, sel_stride;
  uint32_t n, L, sigma;
};

// Ones of level l in positions [0, i), 0 <= i <= n; *bit = bit i (0 when i = n).
__device__ uint32_t rank1(const QTree &t, uint32_t l, uint32_t i, uint32_t *bit = nullptr) {
  const unsigned long long *D = t.rank + (uint64_t)l * (t.NB + 1);
  const uint32_t blk = i >> 9;
  uint32_t r = (uint32_t)__ldg(&D[blk]);
  if (bit) *bit = 0;
  if (i >= t.n) return i == t.n ? (uint32_t)__ldg(&D[t.NB]) : r;
  const uint4 *q = reinterpret_cast<const uint4 *>(t.bits + (uint64_t)l * t.W + (uint64_t)blk * 16);
  const uint32_t w = (i >> 5) & 15u;  // word of i within the block
  const uint32_t lowmask = (1u << (i & 31)) - 1u;
#pragma unroll
  for (uint32_t c = 0; c < 4; ++c) {
    if (4 * c > w) break;
    const uint4 v = __ldg(q + c);
    const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) {
      const uint32_t idx = 4 * c + k;
      if (idx < w) r += __popc(x[k]);
      else if (idx == w) {
        r += __popc(x[k] & lowmask);
        if (bit) *bit = (x[k] >> (i & 31)) & 1u;
      }
    }
  }
  return r;
}

// Position of the bit with 0-based rank g among the ones (want = 1) or the
// zeros (want = 0) of level l; g must exist.
__device__ uint32_t select_bit(const QTree &t, uint32_t l, uint32_t g, uint32_t want) {
  const uint32_t *B = t.bits + (uint64_t)l * t.W;
  const unsigned long long *D = t.rank + (uint64_t)l * (t.NB + 1);
  auto before = [&](uint32_t blk) -> uint32_t {  // wanted bits before block blk
    const uint32_t ones = (uint32_t)__ldg(&D[blk]);
    return want ? ones : (uint32_t)umin64((uint64_t)blk * 512, t.n) - ones;
  };
  // largest block whose prefix is <= g, between two samples when indexed
  uint32_t lo = 0, hi = (uint32_t)t.NB;  // invariant: before(lo) <= g
  if (t.sel) {
    const uint32_t *S = t.sel + ((uint64_t)l * 2 + want) * t.sel_stride;
    const uint32_t j = g / kSelSample;
    lo = __ldg(&S[j]);
    hi = __ldg(&S[j + 1]);
  }
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (before(mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  uint32_t cnt = before(lo);
  for (uint32_t w = lo * 16; w < (uint32_t)t.W; ++w) {
    const uint32_t word = want ? __ldg(&B[w]) : ~__ldg(&B[w]);
    const uint32_t pc = __popc(word);
    if (cnt + pc > g) {
      uint32_t m = word;
      for (uint32_t need = g - cnt; need; --need) m &= m - 1;  // drop the lower set bits
      return w * 32 + (__ffs(m) - 1);
    }
    cnt += pc;
  }
  return 0xFFFFFFFFu;  // not reached for a valid g
}

// Sampled select index: S[l][b][j] = the block holding the (4096 j)-th bit of
// value b of level l (0-based), S[l][b][last + 1] = NB - 1.  One thread per
// (level, block); a block holds at most 512 < 4096 bits, so at most one
// sample of each value starts in it.
__global__ void k_sel_index(QTree t, uint32_t *sel) {
  const uint64_t per_level = t.NB;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < (uint64_t)t.L * per_level;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t l = (uint32_t)(x / per_level), k = (uint32_t)(x % per_level);
    const unsigned long long *D = t.rank + (uint64_t)l * (t.NB + 1);
    const uint32_t o0 = (uint32_t)D[k], o1 = (uint32_t)D[k + 1];
    const uint32_t z0 = (uint32_t)umin64((uint64_t)k * 512, t.n) - o0;
    const uint32_t z1 = (uint32_t)umin64((uint64_t)(k + 1) * 512, t.n) - o1;
    uint32_t *S0 = sel + ((uint64_t)l * 2 + 0) * t.sel_stride;
    uint32_t *S1 = sel + ((uint64_t)l * 2 + 1) * t.sel_stride;
    const uint32_t jz = (z0 + kSelSample - 1) / kSelSample, jo = (o0 + kSelSample - 1) / kSelSample;
    if ((uint64_t)jz * kSelSample < z1) S0[jz] = k;
    if ((uint64_t)jo * kSelSample < o1) S1[jo] = k;
    if (k + 1 == per_level) {  // sentinels after the last sample
      S0[(z1 ? (z1 - 1) / kSelSample : 0) + 1] = k;
      S1[(o1 ? (o1 - 1) / kSelSample : 0) + 1] = k;
      if (z1 == 0) S0[0] = k;
      if (o1 == 0) S1[0] = k;
    }
  }
}

// ----------------------------------------------------------------- tree
__global__ void k_access(QTree t, const uint64_t *idx, uint64_t m, uint32_t *out) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = idx[q];
    if (i0 >= t.n) {
      out[q] = 0xFFFFFFFFu;
      continue;
    }
    uint32_t j = (uint32_t)i0, p = 0;
    for (uint32_t l = 0; l < t.L; ++l) {
      uint32_t b;
      const uint32_t r = rank1(t, l, j, &b);
      if (l + 1 < t.L) {
        const uint2 tb = __ldg(&t.tab[(1u << l) - 1 + p]);
        j = b ? tb.y + r : tb.x + j - r;
      }
      p = 2 * p + b;
    }
    out[q] = p;
  }
}

__global__ void k_rank(QTree t, const uint32_t *cs, const uint64_t *idx, uint64_t m,
                       unsigned long long *out) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = idx[q];
    const uint32_t c = cs[q];
    if (i0 >= t.n || c >= t.sigma) {
      out[q] = ~0ull;
      continue;
    }
    // `end` = number of positions of the current node's level before the
    // image of position i0 + 1, in the order of that level
    uint32_t end = (uint32_t)i0 + 1, p = 0, res = 0;
    for (uint32_t l = 0; l < t.L; ++l) {
      const uint32_t b = (c >> (t.L - 1 - l)) & 1u;
      const uint32_t r = rank1(t, l, end);
      if (l + 1 < t.L) {
        const uint2 tb = __ldg(&t.tab[(1u << l) - 1 + p]);
        end = b ? tb.y + r : tb.x + end - r;
      } else {
        // last level: count c's bit inside node p = [s, end)
        const uint32_t s = (uint32_t)__ldg(&t.E[2 * p]);
        const uint32_t rs = rank1(t, l, s);
        res = b ? r - rs : (end - s) - (r - rs);
      }
      p = 2 * p + b;
    }
    out[q] = t.L ? res : (uint32_t)i0 + 1;
  }
}

__global__ void k_select(QTree t, const uint32_t *cs, const uint64_t *ks, uint64_t m,
                         unsigned long long *out) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ks[q];
    const uint32_t c = cs[q];
    if (k == 0 || c >= t.sigma) {
      out[q] = ~0ull;
      continue;
    }
    const uint64_t e0 = __ldg(&t.E[c]), e1 = __ldg(&t.E[c + 1]);
    if (k > e1 - e0) {
      out[q] = ~0ull;
      continue;
    }
    if (t.L == 0) {
      out[q] = k - 1;
      continue;
    }
    // last level: the (k-1)-th bit of value c&1 inside node c>>1
    const uint32_t L = t.L, pl = c >> 1, bl = c & 1u;
    const uint32_t s = (uint32_t)__ldg(&t.E[2 * pl]);
    const uint32_t rs = rank1(t, L - 1, s);
    uint32_t pos = select_bit(t, L - 1, (bl ? rs : s - rs) + (uint32_t)k - 1, bl);
    for (int l = (int)L - 2; l >= 0; --l) {
      const uint32_t p = c >> (L - l), b = (c >> (L - 1 - l)) & 1u;
      const uint2 tb = __ldg(&t.tab[(1u << l) - 1 + p]);
      pos = b ? select_bit(t, l, pos - tb.y, 1) : select_bit(t, l, pos - tb.x, 0);
    }
    out[q] = pos;
  }
}

// ----------------------------------------------------------- wavelet matrix
__global__ void k_maccess(QTree t, const uint64_t *idx, uint64_t m, uint32_t *out) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = idx[q];
    if (i0 >= t.n) {
      out[q] = 0xFFFFFFFFu;
      continue;
    }
    uint32_t i = (uint32_t)i0, code = 0;
    for (uint32_t l = 0; l < t.L; ++l) {
      uint32_t bit;
      const uint32_t r1 = rank1(t, l, i, &bit);
      i = bit ? (uint32_t)__ldg(&t.zeros[l]) + r1 : i - r1;
      code = 2 * code + bit;
    }
    out[q] = code;
  }
}

__global__ void k_mrank(QTree t, const uint32_t *cs, const uint64_t *idx, uint64_t m,
                        unsigned long long *out) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = idx[q];
    const uint32_t c = cs[q];
    if (i0 >= t.n || c >= t.sigma) {
      out[q] = ~0ull;
      continue;
    }
    // [s, e) holds the symbols of S[0..i] that share c's top l bits
    uint32_t s = 0, e = (uint32_t)i0 + 1;
    for (uint32_t l = 0; l < t.L; ++l) {
      const uint32_t rs = rank1(t, l, s), re = rank1(t, l, e);
      if ((c >> (t.L - 1 - l)) & 1u) {
        const uint32_t z = (uint32_t)__ldg(&t.zeros[l]);
        s = z + rs;
        e = z + re;
      } else {
        s -= rs;
        e -= re;
      }
    }
    out[q] = e - s;
  }
}

__global__ void k_mselect(QTree t, const uint32_t *cs, const uint64_t *ks, uint64_t m,
                          unsigned long long *out) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ks[q];
    const uint32_t c = cs[q];
    if (k == 0 || c >= t.sigma) {
      out[q] = ~0ull;
      continue;
    }
    uint32_t s = 0, e = t.n;  // all occurrences of c's top l bits
    for (uint32_t l = 0; l < t.L; ++l) {
      const uint32_t rs = rank1(t, l, s), re = rank1(t, l, e);
      if ((c >> (t.L - 1 - l)) & 1u) {
        const uint32_t z = (uint32_t)__ldg(&t.zeros[l]);
        s = z + rs;
        e = z + re;
      } else {
        s -= rs;
        e -= re;
      }
    }
    if (k > (uint64_t)(e - s)) {
      out[q] = ~0ull;
      continue;
    }
    uint32_t pos = s + (uint32_t)k - 1;  // in the order after the last level
    for (int l = (int)t.L - 1; l >= 0; --l) {
      if ((c >> (t.L - 1 - l)) & 1u) pos = select_bit(t, l, pos - (uint32_t)__ldg(&t.zeros[l]), 1);
      else pos = select_bit(t, l, pos, 0);
    }
    out[q] = pos;
  }
}

QTree qtree(const wt_tree *t) {
  QTree q;
  q.bits = t->d_bits;
  q.rank = t->d_rank;
  q.zeros = t->d_zeros;
  q.tab = t->d_tab;
  q.E = t->d_node_start;
  q.sel = (t->d_sel && t->sel_for == t->build_count + 1) ? t->d_sel : nullptr;
  q.sel_stride = t->sel_stride;
  q.W = t->W;
  q.NB = t->NB;
  q.n = (uint32_t)t->n;
  q.L = t->L;
  q.sigma = t->sigma;
  return q;
}

int grid_for(uint64_t m) {
  const uint64_t g = (m + 255) / 256;
  return (int)(g < 65535 * 16 ? g : 65535 * 16);
}

int check_launch() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

// Build the sampled select index of the tree's current contents on `st`
// (once per build).  The index is optional: without memory for it select
// falls back to a binary search over the whole directory.
int ensure_sel_index(wt_tree *t, cudaStream_t st) {
  if (t->n == 0 || t->L == 0 || t->sel_for == t->build_count + 1) return WT_OK;
  // sized for the largest n the tree can be resized to, so that the index
  // stays valid across wt_resize
  const uint64_t stride = (std::max(t->n, t->cap_n) / kSelSample) + 2;
  if (!t->d_sel) {
    if (cudaMalloc(&t->d_sel, (uint64_t)t->L * 2 * stride * 4) != cudaSuccess) {
      (void)cudaGetLastError();
      t->d_sel = nullptr;
      return WT_OK;
    }
    t->sel_stride = stride;
  }
  QTree q = qtree(t);
  q.sel_stride = t->sel_stride;
  const uint64_t items = (uint64_t)t->L * t->NB;
  k_sel_index<<<grid_for(items), 256, 0, st>>>(q, t->d_sel);
  if (int rc = check_launch()) return rc;
  t->sel_for = t->build_count + 1;
  return WT_OK;
}

}  // namespace

extern "C" {

int wt_access(const wt_tree *t, const uint64_t *d_i, uint64_t m, uint32_t *d_out, void *stream) {
  if (!t || (m && (!d_i || !d_out))) return WT_ERR_ARG;
  if (t->sticky_error) return t->sticky_error;
  if (!m) return WT_OK;
  auto kern = t->shape == WT_SHAPE_MATRIX ? k_maccess : k_access;
  kern<<<grid_for(m), 256, 0, static_cast<cudaStream_t>(stream)>>>(qtree(t), d_i, m, d_out);
  return check_launch();
}

int wt_rank(const wt_tree *t, const uint32_t *d_c, const uint64_t *d_i, uint64_t m,
            uint64_t *d_out, void *stream) {
  if (!t || (m && (!d_c || !d_i || !d_out))) return WT_ERR_ARG;
  if (t->sticky_error) return t->sticky_error;
  if (!m) return WT_OK;
  auto kern = t->shape == WT_SHAPE_MATRIX ? k_mrank : k_rank;
  kern<<<grid_for(m), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      qtree(t), d_c, d_i, m, reinterpret_cast<unsigned long long *>(d_out));
  return check_launch();
}

int wt_select(const wt_tree *t, const uint32_t *d_c, const uint64_t *d_k, uint64_t m,
              uint64_t *d_out, void *stream) {
  if (!t || (m && (!d_c || !d_k || !d_out))) return WT_ERR_ARG;
  if (t->sticky_error) return t->sticky_error;
  if (!m) return WT_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the index is a cache of the tree's contents, not part of its value
  if (int rc = ensure_sel_index(const_cast<wt_tree *>(t), st)) return rc;
  auto kern = t->shape == WT_SHAPE_MATRIX ? k_mselect : k_select;
  kern<<<grid_for(m), 256, 0, st>>>(qtree(t), d_c, d_k, m, reinterpret_cast<unsigned long long *>(d_out));
  return check_launch();
}

}  // extern "C"
