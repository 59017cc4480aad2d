// Batched access / rank / select over a built levelwise wavelet tree or
// wavelet matrix, one thread per query (validation path).  Definitions from
// Section 2 of the paper.  Tree walks derive node ranges by rank on the
// level bitmaps (the child of [s, e) on level l is [s, s+z) or [s+z, e) on
// level l+1, z the zeros of B_l[s, e)), so no node table is needed.  Matrix
// walks (Section 7) move a position to rank0(i) on a 0 bit and to
// Z_l + rank1(i) on a 1 bit, Z_l the zeros of level l.
#include <cstdint>

#include "wt_dev.cuh"
#include "wt_internal.h"

using namespace wtk;

namespace {

struct QTree {
  const uint32_t *bits;
  const unsigned long long *rank;
  const unsigned long long *zeros;
  uint64_t W, NB;
  uint32_t n, L, sigma;
};

// ones of level l in positions [0, i), 0 <= i <= n
__device__ uint32_t rank1(const QTree &t, uint32_t l, uint32_t i) {
  const uint32_t *B = t.bits + (uint64_t)l * t.W;
  const unsigned long long *D = t.rank + (uint64_t)l * (t.NB + 1);
  const uint32_t blk = i >> 9;
  uint32_t r = (uint32_t)D[blk];
  const uint32_t w = i >> 5;
  for (uint32_t x = blk * 16; x < w; ++x) r += __popc(B[x]);
  if (i & 31) r += __popc(B[w] & ((1u << (i & 31)) - 1u));
  return r;
}

__device__ __forceinline__ uint32_t bit_at(const QTree &t, uint32_t l, uint32_t i) {
  return (t.bits[(uint64_t)l * t.W + (i >> 5)] >> (i & 31)) & 1u;
}

// position of the bit with 0-based rank g among the ones (want = 1) or the
// zeros (want = 0) of level l; g must exist inside [0, n)
__device__ uint32_t select_bit(const QTree &t, uint32_t l, uint32_t g, uint32_t want) {
  const uint32_t *B = t.bits + (uint64_t)l * t.W;
  const unsigned long long *D = t.rank + (uint64_t)l * (t.NB + 1);
  auto before = [&](uint32_t blk) -> uint32_t {  // wanted bits before block blk
    const uint32_t ones = (uint32_t)D[blk];
    return want ? ones : (uint32_t)umin64((uint64_t)blk * 512, t.n) - ones;
  };
  // largest block whose prefix is <= g
  uint32_t lo = 0, hi = (uint32_t)t.NB;  // invariant: before(lo) <= g
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (before(mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  uint32_t cnt = before(lo);
  for (uint32_t w = lo * 16; w < (uint32_t)t.W; ++w) {
    const uint32_t word = want ? B[w] : ~B[w];
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

__global__ void k_access(QTree t, const uint64_t *idx, uint64_t m, uint32_t *out) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < m;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i0 = idx[q];
    if (i0 >= t.n) {
      out[q] = 0xFFFFFFFFu;
      continue;
    }
    uint32_t i = (uint32_t)i0, s = 0, e = t.n, code = 0;
    for (uint32_t l = 0; l < t.L; ++l) {
      const uint32_t rs = rank1(t, l, s), re = rank1(t, l, e), ri = rank1(t, l, i);
      const uint32_t z = (e - s) - (re - rs);
      const uint32_t bit = bit_at(t, l, i);
      if (bit == 0) {
        i = s + (i - s) - (ri - rs);
        e = s + z;
      } else {
        i = s + z + (ri - rs);
        s = s + z;
      }
      code = 2 * code + bit;
    }
    out[q] = code;
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
    uint32_t s = 0, e = t.n, p = (uint32_t)i0 + 1;
    for (uint32_t l = 0; l < t.L; ++l) {
      const uint32_t bit = (c >> (t.L - 1 - l)) & 1u;
      const uint32_t rs = rank1(t, l, s), re = rank1(t, l, e), rp = rank1(t, l, p);
      const uint32_t z = (e - s) - (re - rs);
      if (bit == 0) {
        p = s + (p - s) - (rp - rs);
        e = s + z;
      } else {
        p = s + z + (rp - rs);
        s = s + z;
      }
    }
    out[q] = p - s;
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
    uint32_t S[kMaxLevels + 1], E[kMaxLevels + 1];
    uint32_t s = 0, e = t.n;
    for (uint32_t l = 0; l < t.L; ++l) {
      S[l] = s;
      E[l] = e;
      const uint32_t rs = rank1(t, l, s), re = rank1(t, l, e);
      const uint32_t z = (e - s) - (re - rs);
      if (((c >> (t.L - 1 - l)) & 1u) == 0) e = s + z;
      else s = s + z;
    }
    if (k > (uint64_t)(e - s)) {
      out[q] = ~0ull;
      continue;
    }
    uint32_t pos = s + (uint32_t)k - 1;
    for (int l = (int)t.L - 1; l >= 0; --l) {
      const uint32_t sl = S[l], el = E[l];
      const uint32_t rs = rank1(t, l, sl), re = rank1(t, l, el);
      const uint32_t z = (el - sl) - (re - rs);
      if (((c >> (t.L - 1 - l)) & 1u) == 0) {
        const uint32_t j = pos - sl;            // j-th zero of the node
        pos = select_bit(t, l, (sl - rs) + j, 0);
      } else {
        const uint32_t j = pos - (sl + z);      // j-th one of the node
        pos = select_bit(t, l, rs + j, 1);
      }
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
      const uint32_t bit = bit_at(t, l, i);
      const uint32_t r1 = rank1(t, l, i);
      i = bit ? (uint32_t)t.zeros[l] + r1 : i - r1;
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
        const uint32_t z = (uint32_t)t.zeros[l];
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
        const uint32_t z = (uint32_t)t.zeros[l];
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
      if ((c >> (t.L - 1 - l)) & 1u) pos = select_bit(t, l, pos - (uint32_t)t.zeros[l], 1);
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
  auto kern = t->shape == WT_SHAPE_MATRIX ? k_mselect : k_select;
  kern<<<grid_for(m), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      qtree(t), d_c, d_k, m, reinterpret_cast<unsigned long long *>(d_out));
  return check_launch();
}

}  // extern "C"
