// Build server: continuous batching of wavelet-tree build requests under an
// HBM budget.
//
// A worker thread owns the GPU side.  Requests (host sequences) queue in
// arrival order; the worker admits the head of the queue as soon as its
// footprint (input copy, outputs, scratch, control block) fits in the
// arena -- one device allocation of the budget made at creation, managed by
// a first-fit free list -- and gathers every admissible request into one
// batch: input copies, descriptors and one launch of the batch kernel
// (wt_batch.cuh) on one of `max_inflight` streams.  Batches on different
// streams overlap on the device; requests that arrive while others run are
// admitted as soon as a stream and memory are free.  A request is complete
// when its batch's event has fired; its outputs stay in the arena (a
// wt_tree view) until the client releases it.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "wt_batch.cuh"

namespace {

constexpr uint32_t kSlotMaxTrees = 1024;   // requests per batch
constexpr uint32_t kSlotMaxGroups = kSlotMaxTrees * (kMaxLevels + 2);
constexpr uint32_t kSlotMaxHints = 1u << 20;  // group hints per batch (coarser for larger batches)
// Requests of at least this many symbols, and requests whose alphabet the
// batched kernel would build with node counts (2L phases whose hand-offs
// dominate a short tree's latency), are built alone, with the single-tree
// schedule (whole-GPU passes, levels per pass as the library chooses) in
// their own arena region; the others share batched launches.
constexpr uint64_t kSingleMinSymbols = 1ull << 20;

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing; 256-byte granules.
class Arena {
 public:
  void init(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t &off) {
    bytes = al256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        off = it->first;
        const size_t rest = it->second - bytes;
        const size_t roff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[roff] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Request {
  const void *h_seq = nullptr;
  wt_seq_desc d{};
  BatchGeo geo{};
  size_t off = 0, bytes = 0;  // arena region: input | outputs + scratch | control block
  double t_submit = 0, t_done = 0;
  int state = 0;              // 0 queued, 1 in flight, 2 done
  int status = 0;
  bool single = false;        // built alone with the single-tree schedule
  wt_tree *view = nullptr;    // the result; for a single build also the tree that builds it
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  std::vector<uint64_t> ids;
  // device: batch control words, descriptors, work list (fixed capacity)
  uint32_t *d_ctrl = nullptr;
  BTree *d_trees = nullptr;
  uint32_t *d_first = nullptr;
  uint2 *d_grp = nullptr;
  uint32_t *d_hint = nullptr;
  // pinned host staging of the same
  BTree *h_trees = nullptr;
  uint32_t *h_first = nullptr;
  uint2 *h_grp = nullptr;
  uint32_t *h_hint = nullptr;
};

}  // namespace

struct wt_server {
  int device = 0;
  int sms = 0;
  uint32_t threads = 256;
  wt_config cfg{};
  unsigned char *d_arena = nullptr;
  size_t budget = 0;
  Arena arena;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<uint64_t> completed;
  uint64_t next_id = 1;
  uint64_t in_flight = 0;
  bool stop = false;
  bool blocked = false;   // nothing runs and the head of the queue does not fit
  int fatal = 0;
  std::thread worker;
  // statistics
  uint64_t batches = 0, admitted = 0;
  size_t peak_used = 0;
};

namespace {

// Launch one request built alone on slot s: its input and the tree's
// buffers in its arena region, the single-tree schedule on the slot's stream.
int launch_single(wt_server *srv, Slot &s, Request &r) {
  unsigned char *base = srv->d_arena + r.off;
  const size_t in_bytes = al256(r.d.n * r.d.symbol_bytes);
  wt_tree *v = r.view;
  const TreeLayout ly = tree_layout(v);
  tree_bind(v, ly, base + in_bytes);
  v->owner = srv;
  v->sticky_error = 0;
  if (cudaMemcpyAsync(base, r.h_seq, r.d.n * r.d.symbol_bytes, cudaMemcpyHostToDevice, s.st) != cudaSuccess ||
      cudaMemsetAsync(v->d_status, 0, ly.status, s.st) != cudaSuccess ||
      cudaMemsetAsync(v->d_rank, 0, ly.rank, s.st) != cudaSuccess ||
      cudaMemsetAsync(v->d_zeros, 0, ly.zeros, s.st) != cudaSuccess)
    return WT_ERR_CUDA;
  if (int rc = tree_rebuild(v, base, s.st)) return rc;
  if (cudaEventRecord(s.ev, s.st) != cudaSuccess) return WT_ERR_CUDA;
  s.busy = true;
  ++srv->batches;
  return WT_OK;
}

// Launch one batch of admitted requests on slot s (worker thread, lock held).
int launch_slot(wt_server *srv, Slot &s) {
  const uint32_t m = (uint32_t)s.ids.size();
  if (m == 1 && srv->reqs[s.ids[0]].single) return launch_single(srv, s, srv->reqs[s.ids[0]]);
  std::vector<BatchGeo> geo(m);
  for (uint32_t i = 0; i < m; ++i) geo[i] = srv->reqs[s.ids[i]].geo;
  std::vector<uint32_t> first;
  std::vector<uint2> grp;
  const uint32_t items = batch_worklist(geo, first, grp);
  std::vector<uint32_t> hint;
  const uint32_t hint_shift = batch_hints(first, items, kSlotMaxHints, hint);
  uint32_t max_sb = 1;
  for (uint32_t i = 0; i < m; ++i) max_sb = std::max(max_sb, srv->reqs[s.ids[i]].d.symbol_bytes);
  for (uint32_t i = 0; i < m; ++i) {
    Request &r = srv->reqs[s.ids[i]];
    unsigned char *base = srv->d_arena + r.off;
    const size_t in_bytes = al256(r.d.n * r.d.symbol_bytes);
    unsigned char *mem = base + in_bytes;
    unsigned char *ctrl = mem + batch_mem_bytes(r.geo);
    BTree t = batch_tree(r.d, r.geo, mem, ctrl);
    t.in = base;
    s.h_trees[i] = t;
    if (cudaMemcpyAsync(base, r.h_seq, r.d.n * r.d.symbol_bytes, cudaMemcpyHostToDevice, s.st) != cudaSuccess ||
        cudaMemsetAsync(ctrl, 0, r.geo.ctrl, s.st) != cudaSuccess)
      return WT_ERR_CUDA;
    // the result view
    wt_tree *v = r.view;
    v->owner = srv;
    v->n = r.geo.n;
    v->sigma = r.d.sigma;
    v->sb = r.d.symbol_bytes;
    v->L = r.geo.L;
    v->W = r.geo.W;
    v->NB = r.geo.NB;
    v->threads = srv->threads;
    v->T = 32ull * srv->threads;
    v->NT = r.geo.NT;
    v->sms = srv->sms;
    v->d_bits = t.bits;
    v->d_rank = t.rank;
    v->d_zeros = t.zeros;
    v->d_node_start = t.node_start;
    v->d_tab = t.tab;
    v->d_ctrl = reinterpret_cast<uint32_t *>(t.err) - kCtrlErr;
    v->stream = s.st;
    v->sticky_error = 0;
  }
  std::memcpy(s.h_first, first.data(), first.size() * 4);
  std::memcpy(s.h_grp, grp.data(), grp.size() * sizeof(uint2));
  std::memcpy(s.h_hint, hint.data(), hint.size() * 4);
  if (cudaMemcpyAsync(s.d_trees, s.h_trees, m * sizeof(BTree), cudaMemcpyHostToDevice, s.st) != cudaSuccess ||
      cudaMemcpyAsync(s.d_hint, s.h_hint, hint.size() * 4, cudaMemcpyHostToDevice, s.st) != cudaSuccess ||
      cudaMemcpyAsync(s.d_first, s.h_first, first.size() * 4, cudaMemcpyHostToDevice, s.st) != cudaSuccess ||
      cudaMemcpyAsync(s.d_grp, s.h_grp, grp.size() * sizeof(uint2), cudaMemcpyHostToDevice, s.st) != cudaSuccess ||
      cudaMemsetAsync(s.d_ctrl, 0, 64, s.st) != cudaSuccess)
    return WT_ERR_CUDA;
  BatchArgs a;
  a.trees = s.d_trees;
  a.grp_first = s.d_first;
  a.grp = s.d_grp;
  a.hint = s.d_hint;
  a.hint_shift = hint_shift;
  a.n_groups = (uint32_t)grp.size();
  a.n_items = items;
  a.ticket = s.d_ctrl;
  a.spin_limit = srv->cfg.spin_limit ? srv->cfg.spin_limit : (1u << 22);
  a.err = reinterpret_cast<int *>(s.d_ctrl + 1);
  a.t_start = reinterpret_cast<unsigned long long *>(s.d_ctrl + 2);
  if (batch_launch(a, srv->threads, max_sb, srv->sms, srv->cfg.ctas_per_sm, s.st) != cudaSuccess) return WT_ERR_CUDA;
  if (cudaEventRecord(s.ev, s.st) != cudaSuccess) return WT_ERR_CUDA;
  s.busy = true;
  ++srv->batches;
  return WT_OK;
}

void worker_main(wt_server *srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop) {
    bool progress = false;
    // completions
    for (Slot &s : srv->slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.ev);
      if (q == cudaErrorNotReady) continue;
      const double t = now_s();
      for (uint64_t id : s.ids) {
        Request &r = srv->reqs[id];
        // device-side status (symbol range, timeouts) is read on demand by
        // wt_server_tree / wt_sync on the view
        r.status = q == cudaSuccess ? 0 : WT_ERR_CUDA;
        r.state = 2;
        r.t_done = t;
        srv->completed.push_back(id);
        --srv->in_flight;
      }
      (void)cudaGetLastError();
      s.ids.clear();
      s.busy = false;
      progress = true;
    }
    // admission: FIFO, as long as the head fits and a stream is free
    Slot *free_slot = nullptr;
    for (Slot &s : srv->slots)
      if (!s.busy) {
        free_slot = &s;
        break;
      }
    if (free_slot && !srv->queue.empty()) {
      while (!srv->queue.empty() && free_slot->ids.size() < kSlotMaxTrees) {
        Request &r = srv->reqs[srv->queue.front()];
        // a single-schedule request is launched alone (it waits for the next
        // slot when this one already holds batched requests)
        if (!free_slot->ids.empty() && (r.single || srv->reqs[free_slot->ids[0]].single)) break;
        size_t off;
        if (!srv->arena.alloc(r.bytes, off)) break;  // wait for memory to free up
        r.off = off;
        r.state = 1;
        free_slot->ids.push_back(srv->queue.front());
        srv->queue.pop_front();
        ++srv->admitted;
      }
      srv->peak_used = std::max(srv->peak_used, srv->arena.used());
      bool any_busy = false;
      for (const Slot &s2 : srv->slots) any_busy |= s2.busy;
      srv->blocked = free_slot->ids.empty() && !any_busy && !srv->queue.empty();
      if (!free_slot->ids.empty()) {
        const int rc = launch_slot(srv, *free_slot);
        if (rc) srv->fatal = rc;
        progress = true;
      }
    }
    srv->cv.notify_all();
    if (!progress) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

}  // namespace

extern "C" {

int wt_server_free(wt_server *srv) {
  if (!srv) return WT_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  if (srv->worker.joinable()) srv->worker.join();
  for (Slot &s : srv->slots) {
    if (s.st) cudaStreamSynchronize(s.st);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.st) cudaStreamDestroy(s.st);
    cudaFree(s.d_ctrl);
    cudaFree(s.d_trees);
    cudaFree(s.d_first);
    cudaFree(s.d_grp);
    cudaFree(s.d_hint);
    cudaFreeHost(s.h_trees);
    cudaFreeHost(s.h_first);
    cudaFreeHost(s.h_grp);
    cudaFreeHost(s.h_hint);
  }
  for (auto &kv : srv->reqs) delete kv.second.view;
  cudaFree(srv->d_arena);
  (void)cudaGetLastError();
  delete srv;
  return WT_OK;
}

int wt_server_create(uint64_t budget_bytes, uint32_t max_inflight, const wt_config *cfg,
                     wt_server **out) {
  if (!out || budget_bytes < (1u << 20) || max_inflight == 0 || max_inflight > 64) return WT_ERR_ARG;
  if (cfg && cfg->tile_threads && cfg->tile_threads != 128 && cfg->tile_threads != 256) return WT_ERR_ARG;
  *out = nullptr;
  wt_server *srv = new (std::nothrow) wt_server();
  if (!srv) return WT_ERR_OOM;
  if (cfg) srv->cfg = *cfg;
  srv->threads = (cfg && cfg->tile_threads == 128) ? 128 : 256;
  auto fail = [&](int rc) {
    (void)cudaGetLastError();
    wt_server_free(srv);
    return rc;
  };
  if (cudaGetDevice(&srv->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&srv->sms, cudaDevAttrMultiProcessorCount, srv->device) != cudaSuccess)
    return fail(WT_ERR_CUDA);
  srv->budget = budget_bytes;
  if (cudaMalloc(&srv->d_arena, budget_bytes) != cudaSuccess) return fail(WT_ERR_OOM);
  srv->arena.init(budget_bytes);
  srv->slots.resize(max_inflight);
  for (Slot &s : srv->slots) {
    if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&s.d_ctrl, 64) != cudaSuccess ||
        cudaMalloc(&s.d_trees, kSlotMaxTrees * sizeof(BTree)) != cudaSuccess ||
        cudaMalloc(&s.d_first, (kSlotMaxGroups + 1) * 4) != cudaSuccess ||
        cudaMalloc(&s.d_grp, kSlotMaxGroups * sizeof(uint2)) != cudaSuccess ||
        cudaMalloc(&s.d_hint, kSlotMaxHints * 4) != cudaSuccess ||
        cudaMallocHost(&s.h_trees, kSlotMaxTrees * sizeof(BTree)) != cudaSuccess ||
        cudaMallocHost(&s.h_first, (kSlotMaxGroups + 1) * 4) != cudaSuccess ||
        cudaMallocHost(&s.h_grp, kSlotMaxGroups * sizeof(uint2)) != cudaSuccess ||
        cudaMallocHost(&s.h_hint, kSlotMaxHints * 4) != cudaSuccess)
      return fail(WT_ERR_OOM);
  }
  srv->worker = std::thread(worker_main, srv);
  *out = srv;
  return WT_OK;
}

int wt_server_submit(wt_server *srv, const void *h_seq, uint64_t n, uint32_t sigma,
                     uint32_t symbol_bytes, uint64_t *id) {
  if (!srv || !h_seq || !id) return WT_ERR_ARG;
  Request r;
  r.h_seq = h_seq;
  r.d = wt_seq_desc{n, sigma, symbol_bytes};
  if (!batch_geo(r.d, srv->threads, r.geo)) return WT_ERR_ARG;
  r.view = new (std::nothrow) wt_tree();
  if (!r.view) return WT_ERR_OOM;
  r.single = n >= kSingleMinSymbols || r.geo.nc;
  if (r.single) {
    wt_config c{};
    c.spin_limit = srv->cfg.spin_limit;
    if (int rc = tree_shape(r.view, n, sigma, symbol_bytes, &c, WT_SHAPE_TREE)) {
      delete r.view;
      return rc;
    }
    r.bytes = al256(n * symbol_bytes) + tree_region_bytes(tree_layout(r.view));
  } else {
    r.bytes = al256(n * symbol_bytes) + batch_mem_bytes(r.geo) + r.geo.ctrl;
  }
  if (r.bytes > srv->budget) {  // can never be admitted
    delete r.view;
    return WT_ERR_ARG;
  }
  r.t_submit = now_s();
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->fatal) {
    delete r.view;
    return srv->fatal;
  }
  const uint64_t rid = srv->next_id++;
  srv->reqs.emplace(rid, r);
  srv->queue.push_back(rid);
  srv->blocked = false;
  ++srv->in_flight;
  *id = rid;
  return WT_OK;
}

int wt_server_poll(wt_server *srv, uint64_t *ids, double *latency_s, uint32_t cap, uint32_t *count) {
  if (!srv || !count || (cap && !ids)) return WT_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  uint32_t k = 0;
  while (k < cap && !srv->completed.empty()) {
    const uint64_t id = srv->completed.front();
    srv->completed.pop_front();
    const Request &r = srv->reqs[id];
    ids[k] = id;
    if (latency_s) latency_s[k] = r.t_done - r.t_submit;
    ++k;
  }
  *count = k;
  return srv->fatal;
}

int wt_server_tree(wt_server *srv, uint64_t id, wt_tree **tree) {
  if (!srv || !tree) return WT_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(id);
  if (it == srv->reqs.end() || it->second.state != 2) return WT_ERR_ARG;
  *tree = it->second.view;
  if (it->second.status) return it->second.status;
  int e = 0;
  if (cudaMemcpy(&e, it->second.view->d_ctrl + kCtrlErr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    (void)cudaGetLastError();
    return WT_ERR_CUDA;
  }
  it->second.view->sticky_error = e;
  return e;
}

int wt_server_release(wt_server *srv, uint64_t id) {
  if (!srv) return WT_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(id);
  if (it == srv->reqs.end() || it->second.state != 2) return WT_ERR_ARG;
  srv->arena.release(it->second.off, it->second.bytes);
  delete it->second.view;
  srv->reqs.erase(it);
  srv->blocked = false;  // memory freed: the worker re-evaluates admission
  return WT_OK;
}

int wt_server_drain(wt_server *srv) {
  if (!srv) return WT_ERR_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  srv->cv.wait(lk, [&] { return srv->in_flight == 0 || srv->fatal || srv->blocked; });
  if (srv->fatal) return srv->fatal;
  // queued requests cannot be admitted until completed results are released
  return srv->in_flight ? WT_ERR_OOM : WT_OK;
}

int wt_server_stats(wt_server *srv, uint64_t *out, uint32_t cap) {
  if (!srv || !out) return WT_ERR_ARG;
  std::lock_guard<std::mutex> lk(srv->mu);
  const uint64_t v[6] = {srv->batches, srv->admitted, srv->peak_used, srv->arena.used(), srv->budget,
                         (uint64_t)srv->queue.size()};
  for (uint32_t i = 0; i < cap && i < 6; ++i) out[i] = v[i];
  return WT_OK;
}

}  // extern "C"
