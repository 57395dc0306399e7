// sp_server.cu -- serving runtime over libsp handles (host code).
//
// A request loop over several graphs: worker slots (threads) take the oldest
// runnable request whose graph is not already in use, so requests of one
// graph keep their order while requests of different graphs run at the same
// time on their own CUDA streams.  Graphs are admitted under an HBM budget,
// by an upper bound of their footprint (sp_footprint_bound, with the batch
// buffers reserved for the largest batch a request may carry): before a
// non-resident graph is loaded, idle resident graphs are evicted in
// least-recently-used order (their edge set and their distances and parents
// are exported to host memory and the handle destroyed); a reloaded graph is
// rebuilt from that checkpoint and its distances restored (sp_set_dist
// checks that they are exact) instead of recomputed.  No request starts
// while the resident graphs are over the budget.  Each graph's cooperative
// kernels use a share of the SMs (sp_set_loop_blocks), each block an SM of
// its own, so that the grids of all slots are resident together.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sp.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t id = 0;
  int32_t graph = 0;
  int kind = 0;  // 0 batch, 1 query
  std::vector<int32_t> ds, dd, as, ad, aw, qv, qout;
  sp_request_info info{};
  bool done = false;
};

// A host array for checkpoints: page-locked (cudaMallocHost) so that the
// copies of an eviction and a reload run at full link speed, or ordinary
// memory if page-locked memory is not to be had.  Page-locking is slow, so
// an array keeps its memory between checkpoints of its graph (with a quarter
// to spare for growth) and holds data only while `valid`.
template <typename T>
struct HostArr {
  T *p = nullptr;
  size_t cap = 0;
  bool pinned = false;
  bool valid = false;
  HostArr() = default;
  HostArr(const HostArr &) = delete;
  HostArr &operator=(const HostArr &) = delete;
  ~HostArr() { free_all(); }
  bool empty() const { return !valid; }
  T *data() { return p; }
  bool alloc(size_t count) {
    valid = false;
    if (p && cap >= count) {
      valid = true;
      return true;
    }
    free_all();
    const size_t want = std::max<size_t>(count + count / 4, 1);
    if (cudaMallocHost((void **)&p, want * sizeof(T)) == cudaSuccess) {
      pinned = true;
    } else {
      cudaGetLastError();
      p = (T *)std::malloc(want * sizeof(T));
      pinned = false;
    }
    cap = p ? want : 0;
    valid = p != nullptr;
    return valid;
  }
  void release() { valid = false; }   // the data is stale; the memory stays
  void free_all() {
    if (p) {
      if (pinned) cudaFreeHost(p);
      else std::free(p);
    }
    p = nullptr;
    cap = 0;
    valid = false;
  }
};

struct GEnt {
  int32_t id = 0;
  int32_t n = 0;
  int32_t source = 0;
  sp_graph *g = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};   // device interval of a request
  HostArr<int64_t> ro;      // checkpoint of the edge set while not resident
  HostArr<int32_t> col, w;
  HostArr<int32_t> ck_dist, ck_parent;   // and of the distances (if valid)
  int64_t ck_m = 0;          // edges in the checkpoint
  int64_t bound = 0;        // footprint bound of the checkpointed graph
  int64_t charge = 0;       // bytes counted in `resident` while resident
  bool busy = false;        // a worker holds it (request, load or eviction)
  std::deque<Req *> pending;
  int64_t last_used = 0;
};

}  // namespace

struct sp_server {
  sp_server_config cfg{};
  int device = 0;
  int num_sms = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::unique_ptr<GEnt>> graphs;
  std::map<int64_t, std::unique_ptr<Req>> reqs;
  std::vector<std::thread> workers;
  bool stop = false;
  int64_t next_id = 1, use_counter = 0, inflight = 0, loading = 0;
  int64_t resident = 0, max_resident = 0, loads = 0, evictions = 0;
  int64_t batches = 0, queries = 0, updates = 0;
  std::atomic<int64_t> recovered{0};
  int64_t restores = 0;       // reloads that restored distances (no recompute)
  double load_ms = 0, evict_ms = 0;   // host time in loads / evictions (under mu)
  Clock::time_point t0 = Clock::now();
  cudaStream_t ref_stream = nullptr;
  cudaEvent_t ref_ev = nullptr;   // the device clock's origin for request intervals

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }
  void worker(int slot);
  sp_status make_room(std::unique_lock<std::mutex> &lk, int64_t need, bool wait,
                      const GEnt *self = nullptr);
  sp_status load(GEnt *ge);
  sp_status evict(GEnt *ge);
};

// Build a handle from the checkpoint (mu not held): batch buffers reserved
// for the largest batch, distances restored from the checkpoint when it
// holds them (checked exact on the device), else computed from the source.
sp_status sp_server::load(GEnt *ge) {
  sp_graph *g = nullptr;
  const int64_t m = ge->ck_m;
  sp_status rc = sp_graph_create(ge->n, m, ge->ro.data(), ge->col.data(), ge->w.data(), 0,
                                 cfg.slack, nullptr, ge->stream, &g);
  if (rc != SP_OK) return rc;
  int lb = cfg.loop_blocks > 0 ? cfg.loop_blocks : std::max(1, num_sms / std::max(1, cfg.n_slots));
  sp_set_loop_blocks(g, lb);
  sp_set_push_delta(g, cfg.delta);
  rc = sp_reserve(g, cfg.max_batch_updates);
  bool restored = false;
  if (rc == SP_OK && !ge->ck_dist.empty())
    restored = sp_set_dist(g, ge->source, ge->ck_dist.data(), ge->ck_parent.data(), 0) == SP_OK;
  if (rc == SP_OK && !restored) rc = sp_sssp_init(g, ge->source, nullptr);
  if (rc != SP_OK) {
    sp_graph_destroy(g);
    return rc;
  }
  sp_graph_info info{};
  sp_graph_info_get(g, &info);
  if (info.device_bytes > cfg.hbm_budget_bytes) {   // cannot fit even alone
    sp_graph_destroy(g);
    return SP_ENOMEM_BUDGET;
  }
  ge->g = g;
  ge->charge = std::max<int64_t>(ge->bound, info.device_bytes);
  if (restored) ++restores;
  ge->ro.release();   // the checkpoint is stale from here on
  ge->col.release();
  ge->w.release();
  ge->ck_dist.release();
  ge->ck_parent.release();
  return SP_OK;
}

// Checkpoint the edge set, the distances and the parents to host memory and
// release the handle.
sp_status sp_server::evict(GEnt *ge) {
  int64_t m = 0;
  sp_status rc = sp_graph_num_edges(ge->g, &m);
  if (rc != SP_OK) return rc;
  if (!ge->ro.alloc((size_t)ge->n + 1) || !ge->col.alloc((size_t)m) || !ge->w.alloc((size_t)m))
    return SP_ENOMEM;
  rc = sp_export_csr(ge->g, 0, ge->ro.data(), ge->col.data(), ge->w.data(), 0);
  if (rc != SP_OK) return rc;
  ge->ck_m = m;
  if (!ge->ck_dist.alloc((size_t)ge->n) || !ge->ck_parent.alloc((size_t)ge->n) ||
      sp_get_dist(ge->g, ge->ck_dist.data(), ge->ck_parent.data(), 0) != SP_OK) {
    ge->ck_dist.release();   // no valid distances: recompute on load
    ge->ck_parent.release();
  }
  int64_t b = 0;
  ge->bound = sp_footprint_bound(ge->n, m, cfg.slack, cfg.max_batch_updates, &b) == SP_OK
                  ? b : ge->charge;
  sp_graph_destroy(ge->g);
  ge->g = nullptr;
  return SP_OK;
}

// Evict idle resident graphs, least recently used first, until `need` more
// bytes fit the budget (mu held; released around each eviction).  `self` is
// the graph the caller holds (never a victim, and not counted as running).
// When every other resident graph is running, wait for one to finish if
// `wait`, else stop there (SP_OK: the caller re-checks before its next
// request).  SP_ENOMEM_BUDGET when nothing is left to evict or wait for.
sp_status sp_server::make_room(std::unique_lock<std::mutex> &lk, int64_t need, bool wait,
                               const GEnt *self) {
  while (resident + need > cfg.hbm_budget_bytes) {
    GEnt *victim = nullptr;
    for (auto &g : graphs)
      if (g->g && !g->busy && (!victim || g->last_used < victim->last_used)) victim = g.get();
    if (!victim) {
      // graphs being loaded or running a request (not those waiting for
      // admission, which hold nothing yet)
      bool running = loading > 0;
      for (auto &g : graphs) running |= (g.get() != self && g->g && g->busy);
      if (!wait) return SP_OK;
      if (!running) return SP_ENOMEM_BUDGET;
      cv_done.wait(lk);
      continue;
    }
    victim->busy = true;
    lk.unlock();
    const double t_ev = now_ms();
    const sp_status rc = evict(victim);
    const double dt_ev = now_ms() - t_ev;
    lk.lock();
    evict_ms += dt_ev;
    if (rc == SP_OK) {
      resident -= victim->charge;
      victim->charge = 0;
      ++evictions;
    }
    victim->busy = false;
    cv_work.notify_all();
    cv_done.notify_all();
    if (rc != SP_OK) return rc;
  }
  return SP_OK;
}

void sp_server::worker(int slot) {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    GEnt *ge = nullptr;
    int64_t oldest = INT64_MAX;
    for (auto &g : graphs)
      if (!g->busy && !g->pending.empty() && g->pending.front()->id < oldest) {
        oldest = g->pending.front()->id;
        ge = g.get();
      }
    if (!ge) {
      if (stop) break;
      cv_work.wait(lk);
      continue;
    }
    ge->busy = true;
    Req *r = ge->pending.front();
    ge->pending.pop_front();
    r->info.start_ms = now_ms();
    r->info.slot = slot;
    r->info.gpu_start_ms = r->info.gpu_done_ms = -1.0;
    sp_status rc = SP_OK;
    if (!ge->g) {
      // admission: evict idle resident graphs (LRU) until the footprint
      // bound of this one fits
      rc = make_room(lk, ge->bound, true, ge);
      if (rc == SP_OK) {
        resident += ge->bound;
        max_resident = std::max(max_resident, resident);
        ++loading;
        lk.unlock();
        const double t_ld = now_ms();
        rc = load(ge);
        const double dt_ld = now_ms() - t_ld;
        lk.lock();
        load_ms += dt_ld;
        --loading;
        if (rc == SP_OK) {
          resident += ge->charge - ge->bound;   // the measured size, if above the bound
          ++loads;
          r->info.loaded = 1;
        } else {
          resident -= ge->bound;
        }
        max_resident = std::max(max_resident, resident);
      }
    } else if (resident > cfg.hbm_budget_bytes) {
      // a graph outgrew its bound (its spare pool grew): no request starts
      // until the others make room
      rc = make_room(lk, 0, true, ge);
    }
    lk.unlock();
    if (rc == SP_OK) {
      cudaEventRecord(ge->ev[0], ge->stream);
      if (r->kind == 0) {
        rc = sp_apply_batch(ge->g, (int64_t)r->ds.size(), r->ds.data(), r->dd.data(),
                            (int64_t)r->as.size(), r->as.data(), r->ad.data(), r->aw.data(), 0,
                            nullptr);
        if (rc == SP_ETIMEOUT) {
          // a device bound stopped the repair: recompute the distances from
          // the source (exact), once
          rc = sp_sssp_init(ge->g, ge->source, nullptr);
          if (rc == SP_OK) ++recovered;
        }
      } else {
        r->qout.assign(r->qv.size(), 0);
        rc = sp_query(ge->g, (int32_t)r->qv.size(), r->qv.data(), r->qout.data(), 0);
      }
      cudaEventRecord(ge->ev[1], ge->stream);
      float t0 = 0.f, t1 = 0.f;
      if (cudaEventSynchronize(ge->ev[1]) == cudaSuccess &&
          cudaEventElapsedTime(&t0, ref_ev, ge->ev[0]) == cudaSuccess &&
          cudaEventElapsedTime(&t1, ref_ev, ge->ev[1]) == cudaSuccess) {
        r->info.gpu_start_ms = t0;
        r->info.gpu_done_ms = t1;
      }
      cudaGetLastError();
    }
    sp_graph_info info{};
    if (ge->g) sp_graph_info_get(ge->g, &info);
    lk.lock();
    if (ge->g && info.device_bytes > ge->charge) {   // the spare pool grew
      resident += info.device_bytes - ge->charge;
      ge->charge = info.device_bytes;
      max_resident = std::max(max_resident, resident);
      if (resident > cfg.hbm_budget_bytes) (void)make_room(lk, 0, false, ge);
    }
    r->info.status = rc;
    r->info.done_ms = now_ms();
    r->done = true;
    if (r->kind == 0) {
      ++batches;
      updates += r->info.updates;
    } else {
      ++queries;
    }
    ge->busy = false;
    ge->last_used = ++use_counter;
    --inflight;
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

sp_status sp_server_create(const sp_server_config *cfg, sp_server **out) {
  if (!cfg || !out || cfg->n_slots < 1 || cfg->n_slots > 64 || cfg->hbm_budget_bytes <= 0 ||
      cfg->loop_blocks < 0 || cfg->delta < 0 || !(cfg->slack >= 0.f) || cfg->slack > 16.f ||
      cfg->max_batch_updates < 0 || cfg->max_batch_updates > (1LL << 30))
    return SP_EINVAL;
  *out = nullptr;
  sp_server *s = new (std::nothrow) sp_server();
  if (!s) return SP_ENOMEM;
  s->cfg = *cfg;
  if (s->cfg.max_batch_updates == 0) s->cfg.max_batch_updates = 1 << 20;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device) !=
          cudaSuccess ||
      cudaStreamCreateWithFlags(&s->ref_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&s->ref_ev) != cudaSuccess || cudaEventRecord(s->ref_ev, s->ref_stream) !=
      cudaSuccess || cudaEventSynchronize(s->ref_ev) != cudaSuccess) {
    cudaGetLastError();
    if (s->ref_ev) cudaEventDestroy(s->ref_ev);
    if (s->ref_stream) cudaStreamDestroy(s->ref_stream);
    delete s;
    return SP_ECUDA;
  }
  for (int i = 0; i < cfg->n_slots; ++i) s->workers.emplace_back(&sp_server::worker, s, i);
  *out = s;
  return SP_OK;
}

sp_status sp_server_destroy(sp_server *s) {
  if (!s) return SP_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [s] { return s->inflight == 0; });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->workers) t.join();
  for (auto &g : s->graphs) {
    if (g->g) sp_graph_destroy(g->g);
    for (auto &e : g->ev)
      if (e) cudaEventDestroy(e);
    if (g->stream) cudaStreamDestroy(g->stream);
  }
  cudaEventDestroy(s->ref_ev);
  cudaStreamDestroy(s->ref_stream);
  delete s;
  return SP_OK;
}

sp_status sp_server_add_graph(sp_server *s, int32_t n, int64_t m, const int64_t *row_off,
                              const int32_t *col, const int32_t *w, int32_t source,
                              int32_t *graph_id) {
  if (!s || !graph_id || n <= 0 || m < 0 || !row_off || (m > 0 && (!col || !w)) || source < 0 ||
      source >= n || row_off[n] != m)
    return SP_EINVAL;
  auto ge = std::make_unique<GEnt>();
  ge->n = n;
  ge->source = source;
  if (!ge->ro.alloc((size_t)n + 1) || !ge->col.alloc((size_t)m) || !ge->w.alloc((size_t)m))
    return SP_ENOMEM;
  std::copy(row_off, row_off + n + 1, ge->ro.data());
  std::copy(col, col + m, ge->col.data());
  std::copy(w, w + m, ge->w.data());
  ge->ck_m = m;
  // admitted by an upper bound of its footprint, batch buffers included
  sp_status rc = sp_footprint_bound(n, m, s->cfg.slack, s->cfg.max_batch_updates, &ge->bound);
  if (rc != SP_OK) return rc;
  if (ge->bound > s->cfg.hbm_budget_bytes) return SP_ENOMEM_BUDGET;
  if (cudaStreamCreateWithFlags(&ge->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&ge->ev[0]) != cudaSuccess || cudaEventCreate(&ge->ev[1]) != cudaSuccess) {
    cudaGetLastError();
    for (auto &e : ge->ev)
      if (e) cudaEventDestroy(e);
    if (ge->stream) cudaStreamDestroy(ge->stream);
    return SP_ECUDA;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  ge->id = (int32_t)s->graphs.size();
  *graph_id = ge->id;
  s->graphs.push_back(std::move(ge));
  return SP_OK;
}

static sp_status submit(sp_server *s, int32_t graph_id, std::unique_ptr<Req> r,
                        int64_t *request_id) {
  std::lock_guard<std::mutex> lk(s->mu);
  if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) return SP_EINVAL;
  r->id = s->next_id++;
  r->graph = graph_id;
  r->info.graph = graph_id;
  r->info.kind = r->kind;
  r->info.submit_ms = s->now_ms();
  r->info.status = 1;  // pending
  *request_id = r->id;
  s->graphs[graph_id]->pending.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  ++s->inflight;
  s->cv_work.notify_one();
  return SP_OK;
}

sp_status sp_server_submit_batch(sp_server *s, int32_t graph_id, int64_t n_del,
                                 const int32_t *del_src, const int32_t *del_dst, int64_t n_add,
                                 const int32_t *add_src, const int32_t *add_dst,
                                 const int32_t *add_w, int64_t *request_id) {
  if (!s || !request_id || n_del < 0 || n_add < 0 || (n_del && (!del_src || !del_dst)) ||
      (n_add && (!add_src || !add_dst || !add_w)) || n_del + n_add > s->cfg.max_batch_updates)
    return SP_EINVAL;
  auto r = std::make_unique<Req>();
  r->kind = 0;
  r->ds.assign(del_src, del_src + n_del);
  r->dd.assign(del_dst, del_dst + n_del);
  r->as.assign(add_src, add_src + n_add);
  r->ad.assign(add_dst, add_dst + n_add);
  r->aw.assign(add_w, add_w + n_add);
  r->info.updates = n_del + n_add;
  return submit(s, graph_id, std::move(r), request_id);
}

sp_status sp_server_submit_query(sp_server *s, int32_t graph_id, int32_t k,
                                 const int32_t *vertices, int64_t *request_id) {
  if (!s || !request_id || k < 0 || (k && !vertices)) return SP_EINVAL;
  auto r = std::make_unique<Req>();
  r->kind = 1;
  r->qv.assign(vertices, vertices + k);
  return submit(s, graph_id, std::move(r), request_id);
}

sp_status sp_server_wait(sp_server *s, int64_t request_id, sp_request_info *info,
                         int32_t *dist_out, int32_t timeout_ms) {
  if (!s) return SP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return SP_EINVAL;
  Req *r = it->second.get();
  auto ready = [r] { return r->done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return SP_ETIMEOUT;
  }
  if (info) *info = r->info;
  if (dist_out && r->kind == 1) std::copy(r->qout.begin(), r->qout.end(), dist_out);
  s->reqs.erase(it);
  return SP_OK;
}

sp_status sp_server_drain(sp_server *s) {
  if (!s) return SP_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [s] { return s->inflight == 0; });
  return SP_OK;
}

sp_status sp_server_stats_get(sp_server *s, sp_server_stats *out) {
  if (!s || !out) return SP_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->resident_bytes = s->resident;
  out->max_resident_bytes = s->max_resident;
  out->loads = s->loads;
  out->evictions = s->evictions;
  out->batches = s->batches;
  out->queries = s->queries;
  out->updates = s->updates;
  out->registered_graphs = (int32_t)s->graphs.size();
  int32_t res = 0;
  for (auto &g : s->graphs) res += g->g ? 1 : 0;
  out->resident_graphs = res;
  out->recoveries = s->recovered.load();
  out->restores = s->restores;
  out->load_ms = s->load_ms;
  out->evict_ms = s->evict_ms;
  return SP_OK;
}

sp_status sp_server_get_dist(sp_server *s, int32_t graph_id, int32_t *dist) {
  if (!s || !dist) return SP_EINVAL;
  int32_t n;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) return SP_EINVAL;
    n = s->graphs[graph_id]->n;
  }
  std::vector<int32_t> all((size_t)n);
  std::iota(all.begin(), all.end(), 0);
  int64_t id = 0;
  sp_status rc = sp_server_submit_query(s, graph_id, n, all.data(), &id);
  if (rc != SP_OK) return rc;
  sp_request_info info{};
  rc = sp_server_wait(s, id, &info, dist, -1);
  return rc == SP_OK ? (sp_status)info.status : rc;
}

}  // extern "C"
