// Serving: a request loop that keeps many graphs' sketches resident on the
// device and answers interleaved update batches and Connected queries
// (App. A.2, Problem 2: queries are answered on the graph defined by the
// updates submitted before them).
//
// Continuous batching: one worker thread runs cycles. In each cycle it
//   - admits waiting graphs while their workspace fits the memory cap
//     (workspaces are carved from one device arena allocated up front);
//   - completes finished requests (event polling) and wakes waiters;
//   - takes, from every resident graph with no request in flight, its next
//     request: consecutive update requests of a graph are joined into one
//     batch (exact: sketch addition is XOR), and the joined batches of all
//     those graphs go to the device in one cupc_batcher launch sequence
//     (replayed CUDA graph); a query runs on one of several query streams
//     (recovery + answers), so queries of different graphs overlap with each
//     other and with the update launches.
// A graph has at most one request in flight, so its requests complete in
// submission order and the result of each request is the same as when the
// graph is served alone. Request payloads are copied at submission into a
// pinned pool owned by the server.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

using namespace cupc;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit range allocator over [0, size) with coalescing frees.
class RangeAlloc {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  bool alloc(size_t bytes, size_t align, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      const size_t a = (it->first + align - 1) / align * align;
      if (a + bytes <= it->first + it->second) {
        const size_t start = it->first, end = it->first + it->second;
        free_.erase(it);
        if (a > start) free_[start] = a - start;
        if (a + bytes < end) free_[a + bytes] = end - (a + bytes);
        *off = a;
        used_[a] = bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t start = off, len = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(start);
    if (next != free_.end() && next->first == start + len) {
      len += next->second;
      free_.erase(next);
    }
    auto prev = free_.lower_bound(start);
    if (prev != free_.begin()) {
      --prev;
      if (prev->first + prev->second == start) {
        start = prev->first;
        len += prev->second;
        free_.erase(prev);
      }
    }
    free_[start] = len;
  }

 private:
  std::map<size_t, size_t> free_, used_;
};

enum Kind { K_UPDATE = 0, K_QUERY = 1, K_CLOSE = 2 };

struct Request {
  uint64_t ticket;
  int kind;
  size_t n;          // edges or pairs
  size_t pin_off;    // payload in the pinned pool
  size_t pin_bytes;
  uint8_t* user_out; // query answers go here on completion
  Clock::time_point t_submit;
};

struct Ticket {
  bool done = false;
  cupc_status status = CUPC_OK;
  double latency_us = 0.0;
};

struct Instance {
  uint64_t id;
  uint32_t V;
  uint64_t seed;
  cupc_graph* g = nullptr;
  size_t ws_off = 0, ws_bytes = 0;
  uint32_t slot = 0;  // status word index while resident
  bool resident = false, busy = false, closed = false;
  std::deque<Request> q;
};

struct Inflight {
  std::vector<Request> reqs;  // completed together
  std::vector<uint64_t> insts;
  cudaEvent_t ev;
  int kind;
  int qslot;
  size_t m;
  uint8_t* pinned_out;
};

}  // namespace

struct cupc_server {
  cupc_server_config cfg;
  int device = 0;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  RangeAlloc arena_alloc;
  uint8_t* pinned = nullptr;
  size_t pinned_bytes = 0;
  RangeAlloc pin_alloc;
  // one pinned status word per resident graph (its slot; a graph has at
  // most one request in flight)
  uint32_t* stat_words = nullptr;
  std::vector<uint32_t> free_slots;
  // updates run on one stream at the lowest priority, queries on streams at
  // the highest: when a kernel ends, a waiting query's kernels start before
  // the next update's, so a query waits at most for the update kernel running
  // when it arrives
  cudaStream_t upd_stream = nullptr;
  int prio_low = 0, prio_high = 0;
  std::vector<cudaStream_t> q_streams;
  std::vector<uint32_t*> q_pairs;  // device staging per query stream
  std::vector<uint8_t*> q_out;
  std::vector<bool> q_busy;
  cupc_batcher* batcher = nullptr;
  std::vector<cudaEvent_t> event_pool;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
  uint64_t next_id = 1, next_ticket = 1;
  std::unordered_map<uint64_t, Instance> inst;
  std::deque<uint64_t> admit_q;
  std::unordered_map<uint64_t, Ticket> tickets;
  std::vector<Inflight> inflight;
  uint64_t stat[8] = {0};  // updates, queries, update launches, joined requests, admissions, waits for memory
};

namespace {

cudaEvent_t take_event(cupc_server* s) {
  if (!s->event_pool.empty()) {
    cudaEvent_t e = s->event_pool.back();
    s->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  return e;
}

void finish_ticket(cupc_server* s, const Request& r, cupc_status st, Clock::time_point now) {
  Ticket& t = s->tickets[r.ticket];
  t.done = true;
  t.status = st;
  t.latency_us = std::chrono::duration<double, std::micro>(now - r.t_submit).count();
  if (r.pin_bytes) s->pin_alloc.release(r.pin_off);
}

// Stream-ordered capture of a graph's sticky error word after its work:
// copied into pinned memory, then cleared, so each request reports the
// errors its own batch or pairs raised (as cupc_sync would).
void capture_status(cupc_graph* g, uint32_t* pinned_word, cudaStream_t st) {
  cudaMemcpyAsync(pinned_word, g->gc + GC_ERR, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  cudaMemsetAsync(g->gc + GC_ERR, 0, sizeof(uint32_t), st);
}

cupc_status status_of(uint32_t err) {
  if (!err) return CUPC_OK;
  return (err & kErrTimeout) ? CUPC_ETIMEOUT : CUPC_EINVAL;
}

void admit(cupc_server* s) {
  while (!s->admit_q.empty()) {
    Instance& in = s->inst[s->admit_q.front()];
    cupc_params p{0, 0, 0, s->cfg.max_batch};
    const size_t bytes = cupc_workspace_bytes(in.V, &p);
    size_t off = 0;
    if (s->free_slots.empty()) return;
    if (!bytes || !s->arena_alloc.alloc(bytes, 256, &off)) {
      s->stat[5]++;
      return;  // wait for memory
    }
    cupc_graph* g = nullptr;
    const cupc_status st = cupc_init(in.V, in.seed, &p, (char*)s->arena + off, s->upd_stream, &g);
    if (st != CUPC_OK) {
      // the graph cannot be created: finish its queued requests with that
      // status and refuse later ones, so the graphs behind it still admit
      s->arena_alloc.release(off);
      s->admit_q.pop_front();
      in.closed = true;
      while (!in.q.empty()) {
        finish_ticket(s, in.q.front(), st, Clock::now());
        in.q.pop_front();
      }
      s->cv_done.notify_all();
      continue;
    }
    in.g = g;
    in.slot = s->free_slots.back();
    s->free_slots.pop_back();
    in.ws_off = off;
    in.ws_bytes = bytes;
    in.resident = true;
    s->admit_q.pop_front();
    s->stat[4]++;
  }
}

// Edges one multi-graph update launch joins at most, and how long the worker
// keeps polling after its last activity before it sleeps.
constexpr size_t kLaunchEdges = (size_t)1 << 18;
constexpr int kIdleSpinUs = 500;

void worker_loop(cupc_server* s) {
  cudaSetDevice(s->device);
  Clock::time_point last_busy = Clock::now();
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (s->stop && s->inflight.empty()) break;
    admit(s);
    // completions
    const auto now = Clock::now();
    bool completed = false;
    for (size_t i = 0; i < s->inflight.size();) {
      Inflight& f = s->inflight[i];
      if (cudaEventQuery(f.ev) != cudaSuccess) {
        ++i;
        continue;
      }
      const auto t_done = Clock::now();
      for (size_t j = 0; j < f.reqs.size(); j++) {
        Instance& in = s->inst[f.insts[j]];
        cupc_status st = status_of(s->stat_words[in.slot]);
        if (st == CUPC_OK && s->tickets[f.reqs[j].ticket].status != CUPC_OK) st = s->tickets[f.reqs[j].ticket].status;
        if (f.kind == K_QUERY && f.reqs[j].user_out) memcpy(f.reqs[j].user_out, f.pinned_out, f.m);
        finish_ticket(s, f.reqs[j], st, t_done);
        in.busy = false;
      }
      if (f.kind == K_QUERY) s->q_busy[f.qslot] = false;
      s->event_pool.push_back(f.ev);
      s->inflight[i] = s->inflight.back();
      s->inflight.pop_back();
      completed = true;
    }
    if (completed) s->cv_done.notify_all();
    (void)now;

    // gather: next request of every idle resident graph; one update launch
    // joins at most kLaunchEdges edges over its graphs (a single larger
    // request goes alone), which bounds how long a query can wait for it
    std::vector<uint64_t> upd_insts;
    std::vector<std::vector<Request>> upd_reqs;
    std::vector<size_t> upd_n;
    size_t launch_edges = 0;
    for (auto& kv : s->inst) {
      Instance& in = kv.second;
      if (!in.resident || in.busy || in.q.empty()) continue;
      Request& head = in.q.front();
      if (head.kind == K_CLOSE) {
        Request r = head;
        in.q.pop_front();
        cupc_destroy(in.g);
        in.g = nullptr;
        s->arena_alloc.release(in.ws_off);
        s->free_slots.push_back(in.slot);
        in.resident = false;
        in.closed = true;
        finish_ticket(s, r, CUPC_OK, Clock::now());
        completed = true;
        continue;
      }
      if (head.kind == K_QUERY) {
        int slot = -1;
        for (size_t k = 0; k < s->q_busy.size(); k++)
          if (!s->q_busy[k]) {
            slot = (int)k;
            break;
          }
        if (slot < 0 || head.n > s->cfg.max_batch) {
          if (head.n > s->cfg.max_batch) {
            Request r = head;
            in.q.pop_front();
            finish_ticket(s, r, CUPC_EINVAL, Clock::now());
            completed = true;
          }
          continue;
        }
        Request r = head;
        in.q.pop_front();
        in.busy = true;
        s->q_busy[slot] = true;
        cudaStream_t qs = s->q_streams[slot];
        const uint8_t* payload = s->pinned + r.pin_off;
        cudaMemcpyAsync(s->q_pairs[slot], payload, r.n * 8, cudaMemcpyHostToDevice, qs);
        cupc_status st = cupc_query(in.g, s->q_pairs[slot], r.n, s->q_out[slot], (cupc_stream)qs);
        uint8_t* pout = s->pinned + r.pin_off;  // answers reuse the payload space
        cudaMemcpyAsync(pout, s->q_out[slot], r.n, cudaMemcpyDeviceToHost, qs);
        Inflight f;
        capture_status(in.g, s->stat_words + in.slot, qs);
        f.kind = K_QUERY;
        f.qslot = slot;
        f.m = r.n;
        f.pinned_out = pout;
        f.ev = take_event(s);
        cudaEventRecord(f.ev, qs);
        f.reqs.push_back(r);
        f.insts.push_back(in.id);
        if (st != CUPC_OK) s->tickets[r.ticket].status = st;
        s->inflight.push_back(f);
        s->stat[1] += r.n;
        continue;
      }
      // join consecutive updates (up to max_batch edges, and up to the
      // launch's remaining budget unless this graph would be its first)
      if (in.q.front().n <= s->cfg.max_batch && !upd_insts.empty() &&
          launch_edges + in.q.front().n > kLaunchEdges)
        continue;  // the next launch takes it
      std::vector<Request> joined;
      size_t n = 0;
      while (!in.q.empty() && in.q.front().kind == K_UPDATE && n + in.q.front().n <= s->cfg.max_batch &&
             (joined.empty() || launch_edges + n + in.q.front().n <= kLaunchEdges)) {
        n += in.q.front().n;
        joined.push_back(in.q.front());
        in.q.pop_front();
      }
      launch_edges += n;
      if (joined.empty()) {  // a single request above max_batch: reject it
        Request r = in.q.front();
        in.q.pop_front();
        finish_ticket(s, r, CUPC_EINVAL, Clock::now());
        completed = true;
        continue;
      }
      in.busy = true;
      upd_insts.push_back(in.id);
      upd_reqs.push_back(std::move(joined));
      upd_n.push_back(n);
    }
    if (completed) s->cv_done.notify_all();
    if (!upd_insts.empty()) {
      std::vector<cupc_graph*> gs;
      std::vector<const uint32_t*> es;
      std::vector<const int8_t*> os;
      for (size_t i = 0; i < upd_insts.size(); i++) {
        Instance& in = s->inst[upd_insts[i]];
        size_t at = 0;
        for (const Request& r : upd_reqs[i]) {  // payload: edges then ops
          const uint8_t* p = s->pinned + r.pin_off;
          cudaMemcpyAsync(in.g->stage_edges + 2 * at, p, r.n * 8, cudaMemcpyHostToDevice, s->upd_stream);
          cudaMemcpyAsync(in.g->stage_ops + at, p + r.n * 8, r.n, cudaMemcpyHostToDevice, s->upd_stream);
          at += r.n;
        }
        gs.push_back(in.g);
        es.push_back(in.g->stage_edges);
        os.push_back(in.g->stage_ops);
        s->stat[0] += upd_n[i];
        s->stat[3] += upd_reqs[i].size();
      }
      // one graph: its own launch sequence (a plan over many CTAs); several:
      // one multi-graph launch
      if (gs.size() == 1)
        cupc_update_batch(gs[0], es[0], os[0], upd_n[0], (cupc_stream)s->upd_stream);
      else
        cupc_batcher_update(s->batcher, gs.data(), es.data(), os.data(), upd_n.data(), (uint32_t)gs.size(),
                            (cupc_stream)s->upd_stream);
      s->stat[2]++;
      Inflight f;
      f.kind = K_UPDATE;
      f.qslot = -1;
      f.m = 0;
      f.pinned_out = nullptr;
      for (size_t i = 0; i < gs.size(); i++)
        capture_status(gs[i], s->stat_words + s->inst[upd_insts[i]].slot, s->upd_stream);
      f.ev = take_event(s);
      cudaEventRecord(f.ev, s->upd_stream);
      for (size_t i = 0; i < upd_insts.size(); i++)
        for (const Request& r : upd_reqs[i]) {
          f.reqs.push_back(r);
          f.insts.push_back(upd_insts[i]);
        }
      s->inflight.push_back(f);
    }
    // wait for work or completions: poll while busy and for a short while
    // after (a request arriving then is picked up at once), then sleep
    if (!s->inflight.empty() || !upd_insts.empty()) last_busy = Clock::now();
    if (s->inflight.empty() && Clock::now() - last_busy > std::chrono::microseconds(kIdleSpinUs)) {
      s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    } else {
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    }
  }
}

uint64_t submit(cupc_server* s, uint64_t id, Request r, cupc_status* st) {
  auto it = s->inst.find(id);
  if (it == s->inst.end() || it->second.closed) {
    *st = CUPC_EINVAL;
    return 0;
  }
  r.ticket = s->next_ticket++;
  s->tickets[r.ticket] = Ticket();
  it->second.q.push_back(r);
  *st = CUPC_OK;
  s->cv_work.notify_one();
  return r.ticket;
}

}  // namespace

extern "C" {

cupc_status cupc_server_create(const cupc_server_config* cfg, cupc_server** out) {
  if (!out || !cfg || !cfg->mem_bytes || !cfg->max_graphs) return CUPC_EINVAL;
  *out = nullptr;
  cupc_server* s = new (std::nothrow) cupc_server();
  if (!s) return CUPC_ENOMEM;
  s->cfg = *cfg;
  if (!s->cfg.max_batch) s->cfg.max_batch = 1u << 20;
  if (!s->cfg.query_streams) s->cfg.query_streams = 4;
  if (!s->cfg.pinned_bytes) s->cfg.pinned_bytes = (size_t)256 << 20;
  bool ok = cudaGetDevice(&s->device) == cudaSuccess && cudaMalloc(&s->arena, cfg->mem_bytes) == cudaSuccess &&
            cudaMallocHost((void**)&s->pinned, s->cfg.pinned_bytes) == cudaSuccess &&
            cudaMallocHost((void**)&s->stat_words, 4 * (size_t)cfg->max_graphs) == cudaSuccess &&
            cudaDeviceGetStreamPriorityRange(&s->prio_low, &s->prio_high) == cudaSuccess &&
            cudaStreamCreateWithPriority(&s->upd_stream, cudaStreamNonBlocking, s->prio_low) == cudaSuccess &&
            cupc_batcher_create(cfg->max_graphs, 1, &s->batcher) == CUPC_OK;
  for (uint32_t i = 0; ok && i < s->cfg.query_streams; i++) {
    cudaStream_t qs;
    uint32_t* qp = nullptr;
    uint8_t* qo = nullptr;
    ok = cudaStreamCreateWithPriority(&qs, cudaStreamNonBlocking, s->prio_high) == cudaSuccess &&
         cudaMalloc((void**)&qp, (size_t)s->cfg.max_batch * 8) == cudaSuccess &&
         cudaMalloc((void**)&qo, s->cfg.max_batch) == cudaSuccess;
    if (ok) {
      s->q_streams.push_back(qs);
      s->q_pairs.push_back(qp);
      s->q_out.push_back(qo);
      s->q_busy.push_back(false);
    }
  }
  if (!ok) {
    cudaGetLastError();
    cupc_server_destroy(s);
    return CUPC_ENOMEM;
  }
  s->arena_bytes = cfg->mem_bytes;
  s->arena_alloc.reset(cfg->mem_bytes);
  s->pinned_bytes = s->cfg.pinned_bytes;
  s->pin_alloc.reset(s->pinned_bytes);
  for (uint32_t i = cfg->max_graphs; i-- > 0;) s->free_slots.push_back(i);
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return CUPC_OK;
}

cupc_status cupc_server_open(cupc_server* s, uint32_t V, uint64_t seed, uint64_t* id) {
  if (!s || !id || V < 2) return CUPC_EINVAL;
  cupc_params p{0, 0, 0, s->cfg.max_batch};
  const size_t bytes = cupc_workspace_bytes(V, &p);
  if (!bytes || bytes > s->arena_bytes) return CUPC_ENOMEM;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->inst.size() >= s->cfg.max_graphs) {
    size_t live = 0;
    for (auto& kv : s->inst) live += !kv.second.closed;
    if (live >= s->cfg.max_graphs) return CUPC_ENOMEM;
  }
  Instance in;
  in.id = s->next_id++;
  in.V = V;
  in.seed = seed;
  s->inst[in.id] = in;
  s->admit_q.push_back(in.id);
  *id = in.id;
  s->cv_work.notify_one();
  return CUPC_OK;
}

cupc_status cupc_server_update(cupc_server* s, uint64_t id, const uint32_t* edges, const int8_t* ops, size_t n,
                               uint64_t* ticket) {
  if (!s || !ticket || (n && (!edges || !ops))) return CUPC_EINVAL;
  Request r{};
  r.kind = K_UPDATE;
  r.n = n;
  r.pin_bytes = n * 9;
  r.t_submit = Clock::now();  // latency counts from here, the payload copy included
  if (r.pin_bytes) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->pin_alloc.alloc(r.pin_bytes, 16, &r.pin_off)) return CUPC_ENOMEM;
  }
  if (n) {  // the range is this request's: copy without holding the server lock
    memcpy(s->pinned + r.pin_off, edges, n * 8);
    memcpy(s->pinned + r.pin_off + n * 8, ops, n);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  cupc_status st;
  *ticket = submit(s, id, r, &st);
  if (st != CUPC_OK && r.pin_bytes) s->pin_alloc.release(r.pin_off);
  return st;
}

cupc_status cupc_server_query(cupc_server* s, uint64_t id, const uint32_t* pairs, size_t m, uint8_t* out,
                              uint64_t* ticket) {
  if (!s || !ticket || !m || !pairs || !out) return CUPC_EINVAL;
  Request r{};
  r.kind = K_QUERY;
  r.n = m;
  r.pin_bytes = m * 8;
  r.user_out = out;
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->pin_alloc.alloc(r.pin_bytes, 16, &r.pin_off)) return CUPC_ENOMEM;
  }
  memcpy(s->pinned + r.pin_off, pairs, m * 8);
  std::lock_guard<std::mutex> lk(s->mu);
  cupc_status st;
  *ticket = submit(s, id, r, &st);
  if (st != CUPC_OK) s->pin_alloc.release(r.pin_off);
  return st;
}

cupc_status cupc_server_close(cupc_server* s, uint64_t id, uint64_t* ticket) {
  if (!s || !ticket) return CUPC_EINVAL;
  Request r{};
  r.kind = K_CLOSE;
  r.t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  cupc_status st;
  *ticket = submit(s, id, r, &st);
  if (st == CUPC_OK) s->inst[id].closed = true;  // no further requests
  return st;
}

cupc_status cupc_server_wait(cupc_server* s, uint64_t ticket, uint32_t timeout_ms, double* latency_us) {
  if (!s) return CUPC_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return CUPC_EINVAL;
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  while (!s->tickets[ticket].done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !s->tickets[ticket].done)
      return CUPC_ETIMEOUT;
  }
  Ticket t = s->tickets[ticket];
  s->tickets.erase(ticket);
  if (latency_us) *latency_us = t.latency_us;
  return t.status;
}

cupc_status cupc_server_export(cupc_server* s, uint64_t id, void* dst, size_t bytes) {
  if (!s) return CUPC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->inst.find(id);
  if (it == s->inst.end() || !it->second.resident || it->second.busy || !it->second.q.empty()) return CUPC_EINVAL;
  return cupc_export_sketches(it->second.g, dst, bytes, (cupc_stream)s->upd_stream);
}

cupc_status cupc_server_stats(cupc_server* s, uint64_t* out8) {
  if (!s || !out8) return CUPC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  for (int i = 0; i < 8; i++) out8[i] = s->stat[i];
  size_t resident = 0;
  for (auto& kv : s->inst) resident += kv.second.resident;
  out8[6] = resident;
  out8[7] = s->admit_q.size();
  return CUPC_OK;
}

void cupc_server_destroy(cupc_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->inst)
    if (kv.second.g) cupc_destroy(kv.second.g);
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  if (s->batcher) cupc_batcher_destroy(s->batcher);
  for (size_t i = 0; i < s->q_streams.size(); i++) {
    cudaStreamSynchronize(s->q_streams[i]);
    cudaStreamDestroy(s->q_streams[i]);
    cudaFree(s->q_pairs[i]);
    cudaFree(s->q_out[i]);
  }
  if (s->upd_stream) {
    cudaStreamSynchronize(s->upd_stream);
    cudaStreamDestroy(s->upd_stream);
  }
  if (s->pinned) cudaFreeHost(s->pinned);
  if (s->stat_words) cudaFreeHost(s->stat_words);
  if (s->arena) cudaFree(s->arena);
  delete s;
}

}  // extern "C"
