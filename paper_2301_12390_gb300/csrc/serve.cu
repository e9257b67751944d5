// serve.cu — a request server with continuous batching over the C ABI.
//
// Requests (graphs) arrive at any time through louvain_server_submit and wait
// in arrival order.  Each worker slot owns one engine context on its own
// stream, so the slots' device work overlaps.  A free slot takes the oldest
// waiting request together with every request behind it while their entries
// fit the batch limit, and runs them as one batched launch sequence
// (louvain_load_batch: every graph keeps its own M, iterations and passes, so
// each result equals the graph's result alone).  A slot's device arena stays
// resident between runs and is reused when the next batch fits; admission
// keeps the arenas of all slots within the device-memory budget, a slot that
// cannot grow waits for memory that other slots release, and a request that
// cannot fit even alone is answered with LOUVAIN_ERR_OOM.
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <iterator>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/louvain.h"

namespace {

// Pinned host memory for request graphs, reused from request to request
// (block sizes recur): a request's device load is then a DMA instead of a
// copy staged through the driver's buffers.  At most cap bytes are pinned;
// past that a request keeps pageable memory.
class PinnedPool {
 public:
  explicit PinnedPool(size_t cap) : cap_(cap) {}
  ~PinnedPool() {
    for (auto& kv : free_) cudaFreeHost(kv.second);
  }
  void* get(size_t bytes, size_t* got) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = free_.lower_bound(bytes);
    if (it != free_.end() && it->first <= 2 * bytes + (1u << 20)) {
      void* p = it->second;
      *got = it->first;
      free_.erase(it);
      return p;
    }
    const size_t sz = (bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
    while (held_ + sz > cap_ && !free_.empty()) {   // give back free blocks, largest first
      auto e = std::prev(free_.end());
      cudaFreeHost(e->second);
      held_ -= e->first;
      free_.erase(e);
    }
    if (held_ + sz > cap_) return nullptr;
    void* p = nullptr;
    if (cudaMallocHost(&p, sz) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    held_ += sz;
    *got = sz;
    return p;
  }
  void put(void* p, size_t bytes) {
    std::lock_guard<std::mutex> lk(mu_);
    free_.emplace(bytes, p);
  }

 private:
  std::mutex mu_;
  std::multimap<size_t, void*> free_;
  size_t held_ = 0, cap_;
};

// A block of the pool, returned to it when its owner goes away.
struct PinnedBlock {
  PinnedPool* pool = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  PinnedBlock() = default;
  PinnedBlock(const PinnedBlock&) = delete;
  PinnedBlock& operator=(const PinnedBlock&) = delete;
  PinnedBlock(PinnedBlock&& o) noexcept : pool(o.pool), p(o.p), bytes(o.bytes) { o.p = nullptr; }
  PinnedBlock& operator=(PinnedBlock&& o) noexcept {
    if (this != &o) {
      release();
      pool = o.pool;
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
    }
    return *this;
  }
  ~PinnedBlock() { release(); }
  void release() {
    if (p && pool) pool->put(p, bytes);
    p = nullptr;
  }
};

struct Request {
  int64_t id = 0;
  int64_t n = 0, nnz = 0;
  PinnedBlock pin;              // the graph's arrays, pinned
  std::vector<char> heap;       // or pageable, when the pool is full
  const int64_t* off = nullptr;
  const int32_t* col = nullptr;
  const int32_t* w = nullptr;
  double submit_s = 0;
};

struct Slot {
  louvain_ctx* ctx = nullptr;
  int64_t reserved = 0;   // device bytes its arena holds
  bool busy = false;
};

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct louvain_server {
  PinnedPool pinned{(size_t)8 << 30};   // destroyed last: queued requests return their blocks first
  louvain_options opt;
  louvain_server_config cfg;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_mem, cv_done;
  std::deque<Request> queue;
  std::deque<louvain_server_result> done;
  std::unordered_map<int64_t, std::vector<int32_t>> memberships;
  std::vector<Slot> slots;
  std::vector<std::thread> threads;
  int64_t reserved_total = 0, peak_reserved = 0;
  int64_t submitted = 0, finished = 0, runs = 0;
  double t_assemble = 0, t_load = 0, t_run = 0, t_fetch = 0;   // seconds summed over runs (all slots)
  bool stopping = false;
  std::string err;
};

namespace {

louvain_server_result make_result(const Request& r, int status, double submit_s, double start_s, double done_s,
                                  int batch) {
  louvain_server_result x;
  memset(&x, 0, sizeof(x));
  x.request_id = r.id;
  x.status = status;
  x.batch_size = batch;
  x.n = r.n;
  x.submit_s = submit_s;
  x.start_s = start_s;
  x.done_s = done_s;
  return x;
}

// Run a batch on a slot's context: one graph with louvain_load_csr, several
// with louvain_load_batch.  Fills results and memberships.
int run_batch(louvain_server* S, Slot& slot, std::vector<Request>& batch, double start_s,
              std::vector<louvain_server_result>& res, std::vector<std::vector<int32_t>>& membs) {
  const int64_t G = (int64_t)batch.size();
  int64_t N = 0, E = 0;
  for (auto& r : batch) { N += r.n; E += r.nnz; }
  const double t0 = now_s(S->t0);
  // no host-side concatenation: one request loads from its own arrays, a
  // batch is copied graph by graph to its place on the device
  std::vector<int64_t> vo(G + 1, 0), ns(G), nnzs(G);
  std::vector<const int64_t*> offs(G);
  std::vector<const int32_t*> cols(G), ws(G);
  for (int64_t g = 0; g < G; ++g) {
    const Request& r = batch[g];
    vo[g + 1] = vo[g] + r.n;
    ns[g] = r.n;
    nnzs[g] = r.nnz;
    offs[g] = r.off;
    cols[g] = r.col;
    ws[g] = r.w;
  }
  const double t1 = now_s(S->t0);
  int rc = G == 1 ? louvain_load_csr(slot.ctx, N, E, offs[0], cols[0], ws[0], LOUVAIN_PTR_HOST)
                  : louvain_load_parts(slot.ctx, G, ns.data(), nnzs.data(), offs.data(), cols.data(), ws.data());
  const double t2 = now_s(S->t0);
  if (!rc) rc = louvain_run(slot.ctx);
  const double t3 = now_s(S->t0);
  std::vector<int32_t> memb(N);
  std::vector<double> q(G, 0.0);
  std::vector<int64_t> hi(G, 0), M(G, 0);
  std::vector<uint64_t> lo(G, 0);
  if (!rc) rc = louvain_get_membership(slot.ctx, memb.data(), N, LOUVAIN_PTR_HOST);
  if (!rc) rc = louvain_batch_get_modularity(slot.ctx, q.data(), hi.data(), lo.data(), M.data());
  const double done_s = now_s(S->t0);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->t_assemble += t1 - t0;
    S->t_load += t2 - t1;
    S->t_run += t3 - t2;
    S->t_fetch += done_s - t3;
  }
  for (int64_t g = 0; g < G; ++g) {
    louvain_server_result x = make_result(batch[g], rc, batch[g].submit_s, start_s, done_s, (int)G);
    if (!rc) {
      x.q = q[g];
      x.num_hi = hi[g];
      x.num_lo = lo[g];
      x.M = M[g];
      int64_t info[4];
      if (louvain_batch_get_graph_info(slot.ctx, g, info) == 0) x.communities = info[2];
      membs.emplace_back(memb.begin() + vo[g], memb.begin() + vo[g + 1]);
    } else {
      membs.emplace_back();
    }
    res.push_back(x);
  }
  return rc;
}

void worker(louvain_server* S, int k) {
  cudaSetDevice(S->device);
  Slot& slot = S->slots[k];
  for (;;) {
    std::vector<Request> batch;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_work.wait(lk, [&] { return S->stopping || !S->queue.empty(); });
    if (S->queue.empty()) break;   // stopping and nothing left
    // continuous batching: the oldest request and the ones behind it that fit
    int64_t N = 0, E = 0;
    do {
      Request& r = S->queue.front();
      N += r.n;
      E += r.nnz;
      batch.push_back(std::move(r));
      S->queue.pop_front();
    } while (!S->queue.empty() && S->cfg.batch_max_entries > 0 &&
             E + S->queue.front().nnz <= S->cfg.batch_max_entries &&
             (int64_t)batch.size() < S->cfg.batch_max_graphs);
    // admission by device memory: shrink the batch until its arena fits the
    // budget (the rest goes back to the head of the queue, in order)
    int64_t need = 0;
    louvain_arena_bytes(N, E, &need);
    while (batch.size() > 1 && need > S->cfg.hbm_budget_bytes) {
      N -= batch.back().n;
      E -= batch.back().nnz;
      S->queue.push_front(std::move(batch.back()));
      batch.pop_back();
      louvain_arena_bytes(N, E, &need);
    }
    if (need > S->cfg.hbm_budget_bytes) {
      // too large even alone: answer it now
      const double t = now_s(S->t0);
      louvain_server_result x = make_result(batch[0], LOUVAIN_ERR_OOM, batch[0].submit_s, t, t, 1);
      S->done.push_back(x);
      S->memberships[x.request_id];
      S->finished++;
      S->cv_done.notify_all();
      S->cv_work.notify_all();
      continue;
    }
    for (;;) {
      if (need <= slot.reserved) break;   // the slot's arena already holds it
      const int64_t growth = need - slot.reserved;
      if (S->reserved_total + growth <= S->cfg.hbm_budget_bytes) {
        S->reserved_total += growth;
        slot.reserved = need;
        if (S->reserved_total > S->peak_reserved) S->peak_reserved = S->reserved_total;
        break;
      }
      bool others_busy = false;
      for (auto& o : S->slots)
        if (&o != &slot && o.busy) others_busy = true;
      if (!others_busy) {
        // only idle slots hold the rest: take their arenas back, then retry
        for (auto& o : S->slots)
          if (&o != &slot && o.reserved > 0) {
            louvain_destroy(o.ctx);
            o.ctx = nullptr;
            louvain_create(&o.ctx, &S->opt, S->device, nullptr);
            S->reserved_total -= o.reserved;
            o.reserved = 0;
          }
        continue;   // now reserved_total == slot.reserved and need <= budget: admitted next round
      }
      S->cv_mem.wait(lk);   // a busy slot will finish and notify
    }
    slot.busy = true;
    S->runs++;
    lk.unlock();
    const double start_s = now_s(S->t0);
    std::vector<louvain_server_result> res;
    std::vector<std::vector<int32_t>> membs;
    run_batch(S, slot, batch, start_s, res, membs);
    int64_t bytes = 0;
    louvain_get_device_bytes(slot.ctx, &bytes);
    lk.lock();
    // the arena may have been kept larger than this batch needed
    S->reserved_total += bytes - slot.reserved;
    slot.reserved = bytes;
    slot.busy = false;
    for (size_t i = 0; i < res.size(); ++i) {
      S->memberships[res[i].request_id] = std::move(membs[i]);
      S->done.push_back(res[i]);
    }
    S->finished += (int64_t)res.size();
    S->cv_done.notify_all();
    S->cv_mem.notify_all();
  }
}

}  // namespace

extern "C" {

int louvain_server_default_config(louvain_server_config* cfg) {
  if (!cfg) return LOUVAIN_ERR_INVALID_ARG;
  memset(cfg, 0, sizeof(*cfg));
  cfg->slots = 2;
  cfg->hbm_budget_bytes = 0;
  cfg->batch_max_entries = 256ll << 20;   // measured best of 16M-1G on the 10,000-request stream
  cfg->batch_max_graphs = 1024;
  return 0;
}

int louvain_server_create(louvain_server** out, const louvain_options* opt, const louvain_server_config* cfg,
                          int device) {
  if (!out) return LOUVAIN_ERR_INVALID_ARG;
  *out = nullptr;
  louvain_server* S = new louvain_server();
  if (opt) S->opt = *opt; else louvain_default_options(&S->opt);
  if (cfg) S->cfg = *cfg; else louvain_server_default_config(&S->cfg);
  if (S->cfg.slots < 1 || S->cfg.slots > 64 || S->cfg.batch_max_entries < 0 || S->cfg.batch_max_graphs < 1 ||
      S->cfg.hbm_budget_bytes < 0 || S->cfg.borrow_inputs < 0 || S->cfg.borrow_inputs > 1) {
    delete S;
    return LOUVAIN_ERR_INVALID_ARG;
  }
  S->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete S; return LOUVAIN_ERR_CUDA; }
  if (S->cfg.hbm_budget_bytes == 0) {
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) { delete S; return LOUVAIN_ERR_CUDA; }
    S->cfg.hbm_budget_bytes = (int64_t)(0.9 * (double)freeb);
  }
  S->t0 = std::chrono::steady_clock::now();
  S->slots.resize(S->cfg.slots);
  for (auto& sl : S->slots) {
    int rc = louvain_create(&sl.ctx, &S->opt, device, nullptr);
    if (rc) {
      for (auto& o : S->slots)
        if (o.ctx) louvain_destroy(o.ctx);
      delete S;
      return rc;
    }
  }
  for (int k = 0; k < S->cfg.slots; ++k) S->threads.emplace_back(worker, S, k);
  *out = S;
  return 0;
}

int louvain_server_submit(louvain_server* S, int64_t request_id, int64_t n, int64_t nnz, const int64_t* offsets,
                          const int32_t* cols, const int32_t* weights) {
  if (!S || n < 0 || nnz < 0 || !offsets || (nnz > 0 && (!cols || !weights))) return LOUVAIN_ERR_INVALID_ARG;
  if (offsets[0] != 0 || offsets[n] != nnz) return LOUVAIN_ERR_BAD_CSR;
  Request r;
  r.id = request_id;
  r.n = n;
  r.nnz = nnz;
  if (S->cfg.borrow_inputs) {   // the caller keeps the arrays until the result is polled
    r.off = offsets;
    r.col = cols;
    r.w = weights;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return LOUVAIN_ERR_STATE;
    if (S->memberships.count(request_id)) return LOUVAIN_ERR_INVALID_ARG;   // id still holds a result
    r.submit_s = now_s(S->t0);
    S->queue.push_back(std::move(r));
    S->submitted++;
    S->cv_work.notify_one();
    return 0;
  }
  // one block: offsets, then columns and weights (16-byte aligned)
  const size_t b_off = (size_t)(n + 1) * sizeof(int64_t);
  const size_t at_col = (b_off + 15) & ~(size_t)15;
  const size_t at_w = at_col + (((size_t)nnz * sizeof(int32_t) + 15) & ~(size_t)15);
  const size_t total = at_w + (size_t)nnz * sizeof(int32_t);
  size_t got = 0;
  char* base = (char*)S->pinned.get(total, &got);
  if (base) {
    r.pin.pool = &S->pinned;
    r.pin.p = base;
    r.pin.bytes = got;
  } else {
    r.heap.resize(total + 16);
    base = (char*)(((uintptr_t)r.heap.data() + 15) & ~(uintptr_t)15);
  }
  memcpy(base, offsets, b_off);
  if (nnz) {
    memcpy(base + at_col, cols, (size_t)nnz * sizeof(int32_t));
    memcpy(base + at_w, weights, (size_t)nnz * sizeof(int32_t));
  }
  r.off = (const int64_t*)base;
  r.col = (const int32_t*)(base + at_col);
  r.w = (const int32_t*)(base + at_w);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return LOUVAIN_ERR_STATE;
    if (S->memberships.count(request_id)) return LOUVAIN_ERR_INVALID_ARG;   // id still holds a result
    r.submit_s = now_s(S->t0);
    S->queue.push_back(std::move(r));
    S->submitted++;
  }
  S->cv_work.notify_one();
  return 0;
}

int louvain_server_poll(louvain_server* S, louvain_server_result* out, int64_t cap, int64_t* count, int32_t wait_ms) {
  if (!S || !count || (cap > 0 && !out)) return LOUVAIN_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && wait_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
  int64_t k = 0;
  while (k < cap && !S->done.empty()) {
    out[k++] = S->done.front();
    S->done.pop_front();
  }
  *count = k;
  return 0;
}

int louvain_server_membership(louvain_server* S, int64_t request_id, int32_t* out, int64_t n) {
  if (!S) return LOUVAIN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->memberships.find(request_id);
  if (it == S->memberships.end()) return LOUVAIN_ERR_STATE;
  if ((int64_t)it->second.size() != n || (n > 0 && !out)) return LOUVAIN_ERR_INVALID_ARG;
  if (n) memcpy(out, it->second.data(), n * sizeof(int32_t));
  S->memberships.erase(it);
  return 0;
}

int louvain_server_stats(louvain_server* S, int64_t out[8]) {
  if (!S || !out) return LOUVAIN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = S->submitted;
  out[1] = S->finished;
  out[2] = S->runs;
  out[3] = (int64_t)S->queue.size();
  out[4] = S->reserved_total;
  out[5] = S->peak_reserved;
  out[6] = S->cfg.hbm_budget_bytes;
  out[7] = S->cfg.slots;
  return 0;
}

int louvain_server_timings(louvain_server* S, double out[4]) {
  if (!S || !out) return LOUVAIN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = S->t_assemble;
  out[1] = S->t_load;
  out[2] = S->t_run;
  out[3] = S->t_fetch;
  return 0;
}

void louvain_server_destroy(louvain_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;   // workers finish what is queued, then exit
  }
  S->cv_work.notify_all();
  S->cv_mem.notify_all();
  for (auto& t : S->threads) t.join();
  for (auto& sl : S->slots)
    if (sl.ctx) louvain_destroy(sl.ctx);
  delete S;
}

}  // extern "C"
