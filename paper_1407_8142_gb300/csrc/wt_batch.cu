// Batched levelWT: many independent trees built by one persistent launch.
// The device side (work-list kernel) is in wt_batch.cuh; see include/wt.h.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "wt_batch.cuh"

namespace {

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? WT_ERR_OOM : WT_ERR_CUDA; }

#define WT_CUDA(call)            \
  do {                           \
    cudaError_t e__ = (call);    \
    if (e__ != cudaSuccess) {    \
      (void)cudaGetLastError();  \
      return cuda_fail(e__);     \
    }                            \
  } while (0)

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
  uint32_t *d_hint = nullptr;
  uint32_t hint_shift = 5;
  uint32_t max_sb = 1;               // widest symbol of the batch (sizes the kernel's tiles)
  uint32_t n_groups = 0, n_items = 0;
  unsigned char *d_mem = nullptr;    // outputs + scratch of every tree
  uint32_t *d_ctrl = nullptr;        // cleared per build: ticket, error, stamp, per-tree control blocks
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
  cudaFree(b->d_hint);
  delete b;
  return WT_OK;
}

int wt_batch_create(const wt_seq_desc *descs, uint32_t m, const wt_config *cfg, wt_batch **out) {
  if (!out || !descs || m == 0) return WT_ERR_ARG;
  *out = nullptr;
  if (cfg && cfg->tile_threads && cfg->tile_threads != 128 && cfg->tile_threads != 256) return WT_ERR_ARG;
  wt_batch *b = new (std::nothrow) wt_batch();
  if (!b) return WT_ERR_OOM;
  if (cfg) b->cfg = *cfg;
  b->threads = (cfg && cfg->tile_threads == 128) ? 128 : 256;
  b->m = m;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return WT_ERR_CUDA;
  }
  std::vector<BatchGeo> geo(m);
  size_t mem = 0, ctrl = 16 * 4;  // [0] ticket, [1] batch error, [2..3] start stamp
  for (uint32_t i = 0; i < m; ++i) {
    if (!batch_geo(descs[i], b->threads, geo[i])) {
      delete b;
      return WT_ERR_ARG;
    }
    mem += batch_mem_bytes(geo[i]);
    ctrl += geo[i].ctrl;
    b->max_sb = std::max(b->max_sb, descs[i].symbol_bytes);
  }
  auto fail = [&](cudaError_t err) {
    (void)cudaGetLastError();
    wt_batch_free(b);
    return cuda_fail(err);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_mem, std::max<size_t>(mem, 256)))) return fail(e);
  if ((e = cudaMalloc(&b->d_ctrl, ctrl))) return fail(e);
  b->ctrl_bytes = ctrl;
  b->host_trees.resize(m);
  b->views.assign(m, nullptr);
  size_t off = 0, coff = 16 * 4;
  for (uint32_t i = 0; i < m; ++i) {
    const BatchGeo &g = geo[i];
    BTree &t = b->host_trees[i];
    t = batch_tree(descs[i], g, b->d_mem + off, reinterpret_cast<unsigned char *>(b->d_ctrl) + coff);
    off += batch_mem_bytes(g);
    coff += g.ctrl;
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
    v->T = 32ull * b->threads;
    v->NT = g.NT;
    v->sms = b->sms;
    v->d_bits = t.bits;
    v->d_rank = t.rank;
    v->d_zeros = t.zeros;
    v->d_node_start = t.node_start;
    v->d_tab = t.tab;
    v->d_ctrl = reinterpret_cast<uint32_t *>(t.err) - kCtrlErr;  // d_ctrl + kCtrlErr is the tree's error word
    b->views[i] = v;
  }
  std::vector<uint32_t> first;
  std::vector<uint2> grp;
  b->n_items = batch_worklist(geo, first, grp);
  b->n_groups = (uint32_t)grp.size();
  std::vector<uint32_t> hint;
  b->hint_shift = batch_hints(first, b->n_items, 0xFFFFFFFFu, hint);
  if ((e = cudaMalloc(&b->d_hint, hint.size() * 4))) return fail(e);
  if ((e = cudaMemcpy(b->d_hint, hint.data(), hint.size() * 4, cudaMemcpyHostToDevice))) return fail(e);
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
    ++v->build_count;  // invalidates a query index built for the previous contents
  }
  WT_CUDA(cudaMemsetAsync(b->d_ctrl, 0, b->ctrl_bytes, st));
  BatchArgs a;
  a.trees = b->d_trees;
  a.grp_first = b->d_grp_first;
  a.grp = b->d_grp;
  a.hint = b->d_hint;
  a.hint_shift = b->hint_shift;
  a.n_groups = b->n_groups;
  a.n_items = b->n_items;
  a.ticket = b->d_ctrl;
  a.spin_limit = b->cfg.spin_limit ? b->cfg.spin_limit : (1u << 22);
  a.err = reinterpret_cast<int *>(b->d_ctrl + 1);
  a.t_start = reinterpret_cast<unsigned long long *>(b->d_ctrl + 2);
  WT_CUDA(batch_launch(a, b->threads, b->max_sb, b->sms, b->cfg.ctas_per_sm, st));
  return WT_OK;
}

int wt_batch_sync(wt_batch *b) {
  if (!b) return WT_ERR_ARG;
  WT_CUDA(cudaStreamSynchronize(b->stream));
  int first = 0;
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
