// sp_api.cu -- the C ABI (include/sp.h): handle lifetime, argument checks,
// buffer management and the order of launches for one call.
//
// One sp_apply_batch is one stream-ordered sequence of kernels with a single
// device-to-host copy of the control block at the end (the paper's CUDA
// backend instead copies a `finished` flag to the host every fixedPoint
// iteration, Section 5.3).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sp_graph.cuh"

using sp::Ctl;
using sp::u32;
using sp::u64;

namespace sp {

void *Alloc::get(size_t bytes) {
  if (bytes == 0) bytes = 256;
  void *p = nullptr;
  if (has_user) {
    p = user.alloc(user.ctx, bytes, (void *)stream);
  } else if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) bytes_held += (long long)bytes;
  return p;
}

void Alloc::put(void *p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  if (has_user) user.free(user.ctx, p, bytes, (void *)stream);
  else cudaFreeAsync(p, stream);
  bytes_held -= (long long)bytes;
}

sp_status csr_validate(sp_graph *g, const long long *row_off_d, const int *col_d,
                       const int *w_d, long long m, int *launches);

}  // namespace sp

namespace {

// Frontier edge ranges are 32-bit (a frontier holds each vertex at most once,
// so its edges never exceed m); graphs stay below 2^31 edges.
constexpr long long kMaxEdges = (1LL << 31) - 1;

// Buffers sized by the batch: grown (never shrunk) when a larger batch comes.
// Grow the per-call buffers to ni items (and nb_host staged host inputs).
// New buffers are allocated before the old ones are released, so a failed
// allocation (SP_ENOMEM) leaves every buffer as it was.
sp_status ensure_batch_buffers(sp_graph *g, long long ni, long long nb_host) {
  sp::BatchBufs &b = g->bb;
  auto &al = g->al;
  const long long want = std::max<long long>(ni + 1, 1024);
  if (want > b.cap_items) {
    const long long c = std::max(want, b.cap_items * 2);
    const size_t tmp_bytes = std::max({sp::sort_tmp_bytes(c), sp::scan_tmp_bytes(c),
                                       sp::batch_sort_tmp_bytes(g->sort_blocks)}) + 1024;
    void *p[10];
    const size_t sz[10] = {(size_t)c * 8, (size_t)c * 8, (size_t)c * 4, (size_t)c * 4,
                           (size_t)c,     (size_t)c * 8, (size_t)c * 4,
                           (size_t)c * sizeof(sp::Seg), tmp_bytes, (size_t)c * 8};
    bool ok = true;
    for (int i = 0; i < 10; ++i) {
      p[i] = ok ? al.get(sz[i]) : nullptr;
      ok = ok && p[i];
    }
    if (!ok) {
      for (int i = 0; i < 10; ++i) al.put(p[i], sz[i]);
      return SP_ENOMEM;
    }
    const long long old = b.cap_items;
    al.put(b.keys, old * 8); al.put(b.keys_alt, old * 8);
    al.put(b.vals, old * 4); al.put(b.vals_alt, old * 4);
    al.put(b.flags, old); al.put(b.item_pref, old * 8);
    al.put(b.opos, old * 4);
    al.put(b.seg, old * sizeof(sp::Seg));
    al.put(b.tmp, b.tmp_bytes);
    al.put(b.srch, old * 8);
    b.keys = (u64 *)p[0]; b.keys_alt = (u64 *)p[1];
    b.vals = (u32 *)p[2]; b.vals_alt = (u32 *)p[3];
    b.flags = (unsigned char *)p[4];
    b.item_pref = (u64 *)p[5];
    b.opos = (u32 *)p[6];
    b.seg = (sp::Seg *)p[7];
    b.tmp = p[8];
    b.tmp_bytes = tmp_bytes;
    b.srch = (u64 *)p[9];
    b.cap_items = c;
    ++g->gen;
  }
  if (nb_host > b.cap_in) {
    const long long c = std::max(nb_host, b.cap_in * 2);
    int *p[5];
    bool ok = true;
    for (int i = 0; i < 5; ++i) {
      p[i] = ok ? (int *)al.get((size_t)c * 4) : nullptr;
      ok = ok && p[i];
    }
    if (!ok) {
      for (int i = 0; i < 5; ++i) al.put(p[i], (size_t)c * 4);
      return SP_ENOMEM;
    }
    const long long old = b.cap_in;
    al.put(b.in_del_src, old * 4); al.put(b.in_del_dst, old * 4);
    al.put(b.in_add_src, old * 4); al.put(b.in_add_dst, old * 4); al.put(b.in_add_w, old * 4);
    b.in_del_src = p[0]; b.in_del_dst = p[1];
    b.in_add_src = p[2]; b.in_add_dst = p[3];
    b.in_add_w = p[4];
    b.cap_in = c;
    ++g->gen;
  }
  // merge strips: at most (old entries of touched rows) / 256 + one per row
  const long long sneed = (2 * g->m) / 256 + ni + 64;
  if (sneed > b.strips_cap) {
    const long long c = std::max(sneed, 2 * b.strips_cap);
    int2 *ns = (int2 *)al.get((size_t)c * 8);
    if (!ns) return SP_ENOMEM;
    al.put(b.strips, (size_t)b.strips_cap * 8);
    b.strips = ns;
    b.strips_cap = c;
    ++g->gen;
  }
  return SP_OK;
}

void fill_stats(sp_graph *g, const Ctl &c, sp_batch_stats *st, int launches, int regrows,
                long long ni, bool timed, bool fold = false) {
  if (!st) return;
  st->n_del_applied = (int64_t)c.del_applied;
  st->n_del_absent = (int64_t)c.del_absent;
  st->n_add_applied = (int64_t)c.add_applied;
  st->n_add_present = (int64_t)c.add_present;
  st->affected = (int64_t)c.affected;
  st->seeds = (int64_t)c.seeds;
  st->relaxed_edges = (int64_t)c.relaxed;
  st->improved = (int64_t)c.improved;
  st->rows_touched = (int64_t)c.rows_touched;
  st->rows_relocated = (int64_t)c.rows_relocated;
  st->rounds_inval = (int32_t)c.rounds_inval;
  st->rounds_push = (int32_t)c.rounds_push;
  st->n_launches = launches;
  st->regrows = regrows;
  // Algorithmic bytes: what each phase must move, counted from what it did.
  const int passes = (2 * g->bits + 2 + 7) / 8;
  const long long nb = ni / 2;
  // the sort phase also holds the old-row searches that run beside the sort
  // (inputs 10 per item on average, the row's meta 16, the result 8)
  st->alg_bytes[SP_PH_SORT] =
      ni ? (int64_t)(nb * 20 + ni * 12 + (long long)passes * ni * 24 + ni * 34) : 0;
  // key 8, number 4 and search result 8 read; opos 4, flags 1, weight 4 and
  // prefix 8 written per item; 16 per touched row
  st->alg_bytes[SP_PH_COUNT] = (int64_t)(ni * 37 + (long long)c.rows_touched * 16);
  st->alg_bytes[SP_PH_MERGE] = (int64_t)(c.merge_slots * 8 + c.rows_touched * 32 + ni * 21);
  st->alg_bytes[SP_PH_INVAL] =
      (int64_t)(c.affected * (16 + 8 + 8 + 4) + c.inval_edges * 16);
  // the pull and OnAdd run inside the push loop's launch (its first stage),
  // so their bytes count with the push phase
  st->alg_bytes[SP_PH_PULL] = 0;
  st->alg_bytes[SP_PH_ADD] = 0;
  st->alg_bytes[SP_PH_PUSH] =
      (int64_t)(c.push_vertices * (4 + 16 + 8) + c.relaxed * 16 + c.improved * 8 +
                c.enqueued * (4 + 4 + 4)) +
      (int64_t)(c.affected * 16 + c.pull_edges * 16 + c.seeds * 20) +
      (int64_t)(c.add_applied * (12 + 16));
  st->alg_bytes[SP_PH_FINISH] = (int64_t)sizeof(Ctl);
  for (int i = 0; i < SP_NPHASE; ++i) st->ms_phase[i] = 0.f;
  st->ms_total = 0.f;
  if (timed) {
    // fold: a batch pipeline, whose pull and OnAdd run inside the push launch;
    // it records no events 5 and 6, and its push phase spans events 4..7
    for (int i = 0; i < SP_NPHASE; ++i) {
      if (fold && (i == SP_PH_PULL || i == SP_PH_ADD)) continue;
      const cudaEvent_t from = fold && i == SP_PH_PUSH ? g->ev[SP_PH_PULL] : g->ev[i];
      if (cudaEventElapsedTime(&st->ms_phase[i], from, g->ev[i + 1]) != cudaSuccess)
        st->ms_phase[i] = 0.f;
    }
    // an invalidation beside the store update: its own duration (it overlaps
    // the count and merge phases, so the phases add up to more than the total)
    if (g->last_beside &&
        cudaEventElapsedTime(&st->ms_phase[SP_PH_INVAL], g->ev_inval[0], g->ev_inval[1]) !=
            cudaSuccess)
      st->ms_phase[SP_PH_INVAL] = 0.f;
    if (cudaEventElapsedTime(&st->ms_total, g->ev[0], g->ev[SP_NPHASE]) != cudaSuccess)
      st->ms_total = 0.f;
    cudaGetLastError();
  }
}

// Phase boundary i of a batch: records timing event i.  While the pipeline
// is being captured the record becomes a node of the graph, so a replay
// times its phases too.
void rec(sp_graph *g, bool timed, int i) {
  if (!timed) return;
  if (g->capturing >= 0)
    cudaEventRecordWithFlags(g->ev[i], g->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(g->ev[i], g->stream);
}

void drop_batch_graphs(sp_graph *g) {
  if (g->bg_exec) cudaGraphExecDestroy(g->bg_exec);
  if (g->bg_graph) cudaGraphDestroy(g->bg_graph);
  g->bg_exec = nullptr;
  g->bg_graph = nullptr;
  g->bg_sort = g->bg_inval = g->bg_search = nullptr;
  g->bg_ready = false;
}

// Pointer jumping reads only the parents in s, so the invalidation can run
// beside the store update; frontier rounds walk the forward store and wait
// for the merge.
bool inval_beside(const sp_graph *g) { return g->side && g->lim.jump_round == 0; }

// The kernel nodes of the captured batch graph that read the batch inputs:
// the batch sort and the old-row searches (every input array) and the
// invalidation loop (the deletions).  Every other kernel reads the sorted items.
bool find_input_nodes(sp_graph *g) {
  g->bg_sort = g->bg_inval = g->bg_search = nullptr;
  size_t nn = 0;
  if (cudaGraphGetNodes(g->bg_graph, nullptr, &nn) != cudaSuccess) return false;
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn && cudaGraphGetNodes(g->bg_graph, nodes.data(), &nn) != cudaSuccess) return false;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams p = {};
    if (cudaGraphKernelNodeGetParams(nd, &p) != cudaSuccess) return false;
    if (p.func == sp::batch_sort_fn()) g->bg_sort = nd;
    else if (p.func == sp::inval_fn()) g->bg_inval = nd;
    else if (p.func == sp::search_fn()) g->bg_search = nd;
  }
  return g->bg_sort != nullptr && g->bg_search != nullptr;
}

cudaError_t retarget_input_nodes(sp_graph *g, const int *ds, const int *dd, long long nd,
                                 const int *as, const int *ad, const int *aw, long long na) {
  cudaError_t e = sp::retarget_batch_sort(g, g->bg_exec, g->bg_sort, ds, dd, nd, as, ad, aw, na);
  if (e == cudaSuccess)
    e = sp::retarget_search(g, g->bg_exec, g->bg_search, ds, dd, nd, as, ad, aw, na);
  if (e == cudaSuccess && g->bg_inval)
    e = sp::retarget_inval(g, g->bg_exec, g->bg_inval, ds, dd, nd, inval_beside(g) ? 1 : 0);
  return e;
}

// The control block of the call, on the host.  mirrored: the call ended
// with k_finish, which wrote it into the pinned copy already.
sp_status read_ctl(sp_graph *g, bool mirrored = false) {
  if (!mirrored)
    cudaMemcpyAsync(g->ctl_host, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, g->stream);
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
    cudaGetLastError();
    return SP_ECUDA;
  }
  return SP_OK;
}

void set_limits(sp_graph *g) {
  // Bellman-Ford bound n + 1; near-far ordering adds split rounds, so the
  // default cap is then 4 (n + 1)
  const long long bf = (long long)g->n + 1;
  const long long cap = g->delta_user > 0 ? 4 * bf : bf;
  g->lim.max_rounds = g->max_rounds_user > 0 ? (u32)g->max_rounds_user
                                             : (u32)std::min<long long>(cap, 0x7fffffffLL);
  g->lim.wait_ns = g->wait_ns_user > 0 ? (u64)g->wait_ns_user : 2000000000ull;
  g->lim.delta = (u32)std::max(0, g->delta_user);
  g->lim.jump_round = g->jump_round_user;
  g->lim.local_edges = (u32)g->local_edges_user;
  g->lim.small_deg = (u32)g->small_deg_user;
  g->lim.pool_rounds = (u32)g->pool_rounds_user;
  g->lim.miss_site = (u32)g->miss_site_user;
  ++g->gen;
}

sp_status status_of_repair(sp_graph *g, const Ctl &c) {
  if (c.bad) {
    g->state = 2;
    return SP_ECUDA;
  }
  if (c.timeout) {
    g->state = 2;
    return SP_ETIMEOUT;
  }
  if (c.range_err) {
    g->state = 2;
    return SP_ERANGE;
  }
  return SP_OK;
}

// Timing event i (0 start, 1 end) of an invalidation on the side stream.
void rec_side(sp_graph *g, bool timed, int i) {
  if (!timed) return;
  if (g->capturing >= 0)
    cudaEventRecordWithFlags(g->ev_inval[i], g->side, cudaEventRecordExternal);
  else
    cudaEventRecord(g->ev_inval[i], g->side);
}

// How a batch's invalidation runs.
enum InvalMode {
  kInvalAfter = 0,    // after the merge, on the graph's stream
  kInvalBeside = 1,   // on the side stream, beside the count and the merge
  kInvalKept = 2,     // a rerun after a pool grow: the first attempt's stands
};

// The kernel sequence of one batch (no host synchronisation).
cudaError_t enqueue_batch(sp_graph *g, const int *ds, const int *dd, long long n_del,
                          const int *as, const int *ad, const int *aw, long long n_add,
                          bool timed, int *launches, int mode = kInvalAfter) {
  const long long ni = 2 * (n_del + n_add);
  sp::launch_ctl_reset(g, mode == kInvalKept ? 2 : 0, launches);
  // the items' searches in their old rows run beside the batch sort (on the
  // SMs the sort leaves free; they read only the inputs and the old stores)
  cudaError_t e = cudaSuccess;
  if (g->side) {
    cudaEventRecord(g->fork0_ev, g->stream);
    cudaStreamWaitEvent(g->side, g->fork0_ev, 0);
    e = sp::launch_search(g, ds, dd, n_del, as, ad, aw, n_add, launches, g->side);
    cudaEventRecord(g->search_ev, g->side);
  } else {
    e = sp::launch_search(g, ds, dd, n_del, as, ad, aw, n_add, launches, g->stream);
  }
  const cudaError_t es = sp::launch_batch_sort(g, ds, dd, n_del, as, ad, aw, n_add, launches);
  if (e == cudaSuccess) e = es;
  rec(g, timed, 1);
  if (g->side) cudaStreamWaitEvent(g->stream, g->search_ev, 0);
  const bool beside = mode == kInvalBeside && n_del > 0;
  g->last_beside = beside && timed;
  // fork: the invalidation runs beside the count pass and the merge once the
  // batch is validated.  Two cooperative grids side by side are safe only if
  // neither can hold SMs the other's blocks wait for: the invalidation's
  // blocks each need a whole SM, so the count's grid is capped to what the
  // other SMs hold and is resident in full whichever is placed first.  With
  // a block share (several handles at once) the invalidation waits for the
  // count instead, so each handle runs one cooperative grid at a time.
  const bool share = g->loop_blocks_user > 0;
  auto fork = [&]() {
    cudaEventRecord(g->fork_ev, g->stream);
    cudaStreamWaitEvent(g->side, g->fork_ev, 0);
    rec_side(g, timed, 0);
    const cudaError_t ei = sp::launch_inval(g, ds, dd, n_del, launches, 1, g->side);
    if (e == cudaSuccess) e = ei;
    rec_side(g, timed, 1);
    cudaEventRecord(g->join_ev, g->side);
  };
  if (beside && !share) fork();
  sp::launch_count(g, ni, launches, beside && !share ? sp::inval_beside_blocks(g) : 0);
  rec(g, timed, 2);
  if (beside && share) fork();
  sp::launch_merge(g, ni, launches);
  rec(g, timed, 3);
  if (beside) cudaStreamWaitEvent(g->stream, g->join_ev, 0);   // join
  else if (mode == kInvalAfter && e == cudaSuccess && n_del > 0)
    e = sp::launch_inval(g, ds, dd, n_del, launches);
  rec(g, timed, 4);
  // the pull and OnAdd run as the first stage of the push loop's launch: the
  // push phase spans events 4..7 (fill_stats with `fold`), and events 5 and 6
  // are not recorded (each timing event is one more node of a captured graph)
  if (e == cudaSuccess) e = sp::launch_push(g, launches, n_del > 0 ? 1 : 0, ni);
  rec(g, timed, 7);
  // the degree share that picks the pool kernel of the next call
  if (g->lim.pool_rounds > 0) sp::launch_deg_mid(g, launches);
  sp::launch_finish(g, launches);
  rec(g, timed, 8);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

// A batch that stops before its merge (the store could not grow) leaves the
// edge set as it was.  If its invalidation already ran beside the store
// update (touched), the distances are recomputed from the sources of the
// last init, which allocates nothing; if that fails too the handle needs
// sp_sssp_init (SP_ESTATE).  Returns rc, the batch's own status.
sp_status restore_after(sp_graph *g, bool touched, sp_status rc) {
  if (!touched) return rc;
  int launches = 0;
  sp::launch_ctl_reset(g, 0, &launches);
  if (g->n_src == 1 && g->source >= 0) sp::launch_init(g, g->source, &launches);
  else if (g->n_src > 1 && g->src_dev) sp::launch_init_multi(g, g->src_dev, g->n_src, &launches);
  else {
    g->state = 2;
    return rc;
  }
  cudaError_t e = sp::launch_push(g, &launches);
  sp::launch_finish(g, &launches);
  if (e != cudaSuccess || read_ctl(g, true) != SP_OK ||
      status_of_repair(g, *g->ctl_host) != SP_OK) {
    cudaGetLastError();
    g->state = 2;
  }
  return rc;
}

// The device address of a page-locked host array that is mapped into the
// device's address space (cudaHostAlloc, torch's pinned memory), or nullptr
// for any other pointer.  Kernels read and write such arrays directly across
// the host link (NVLink-C2C on Grace machines), with no copy-engine transfer.
const void *mapped_host(const void *p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// A device array the graph's kernels may write: memory of the graph's device
// (or managed memory).  Host pointers passed as device outputs are refused
// before anything is launched.
bool device_out(const sp_graph *g, const void *p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice && at.device == g->device) ||
         at.type == cudaMemoryTypeManaged;
}

// Buffers big enough for an asynchronous batch of ni items?
bool reserved_for(const sp_graph *g, long long ni) {
  const sp::BatchBufs &b = g->bb;
  return ni + 1 <= b.cap_items && (2 * g->m) / 256 + ni + 64 <= b.strips_cap;
}

}  // namespace

struct sp_exec {
  sp_graph *g = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

const char *sp_status_str(sp_status s) {
  switch (s) {
    case SP_OK: return "SP_OK";
    case SP_EINVAL: return "SP_EINVAL: invalid argument";
    case SP_ENOMEM: return "SP_ENOMEM: allocation failed";
    case SP_ERANGE: return "SP_ERANGE: a distance does not fit below SP_INF";
    case SP_ESTATE: return "SP_ESTATE: no valid distances (call sp_sssp_init)";
    case SP_ECUDA: return "SP_ECUDA: CUDA runtime error";
    case SP_ETIMEOUT: return "SP_ETIMEOUT: device-side round cap or wait bound hit";
    case SP_ENOMEM_BUDGET: return "SP_ENOMEM_BUDGET: over the memory budget";
  }
  return "unknown sp_status";
}

const char *sp_version(void) { return "0.1.0"; }

sp_status sp_graph_destroy(sp_graph *g) {
  if (!g) return SP_OK;
  if (g->side) cudaStreamSynchronize(g->side);
  cudaStreamSynchronize(g->stream);
  auto &al = g->al;
  auto &b = g->bb;
  const long long n = g->n;
  long long c = b.cap_items;
  al.put(b.keys, c * 8); al.put(b.keys_alt, c * 8);
  al.put(b.vals, c * 4); al.put(b.vals_alt, c * 4);
  al.put(b.flags, c); al.put(b.item_pref, c * 8);
  al.put(b.opos, c * 4);
  al.put(b.seg, c * sizeof(sp::Seg));
  al.put(b.strips, (size_t)b.strips_cap * 8);
  al.put(b.tmp, b.tmp_bytes);
  al.put(b.srch, c * 8);
  c = b.cap_in;
  al.put(b.in_del_src, c * 4); al.put(b.in_del_dst, c * 4);
  al.put(b.in_add_src, c * 4); al.put(b.in_add_dst, c * 4); al.put(b.in_add_w, c * 4);
  al.put(g->fwd.row, n * sizeof(sp::RowMeta));
  al.put(g->fwd.alt, n * sizeof(long long));
  al.put(g->rev.alt, n * sizeof(long long));
  al.put(g->fwd.adj, (size_t)g->fwd.slots * sizeof(int2));
  al.put(g->rev.row, n * sizeof(sp::RowMeta));
  al.put(g->rev.adj, (size_t)g->rev.slots * sizeof(int2));
  al.put(g->s, n * 8);
  al.put(g->qflag, n * 4);
  al.put(g->asv, n * 4);
  for (int b = 0; b < 3; ++b) {
    al.put(g->qent[b], n * 8);
    al.put(g->qsv[b], n * 4);
    al.put(g->fq[b], n * 4);
    al.put(g->qown[b], (size_t)g->own_cap * 4);
  }
  al.put(g->aent, n * 8);
  al.put(g->ftag, n * 4);
  al.put(g->jmp, n * 4);
  al.put(g->cut, n * 4);
  al.put(g->aown, (size_t)g->own_cap * 4);
  al.put(g->out_dist, n * 4); al.put(g->out_parent, n * 4);
  al.put(g->pr[0], n * 4); al.put(g->pr[1], n * 4);
  al.put(g->prc[0], n * 4); al.put(g->prc[1], n * 4);
  al.put(g->pracc, n * 4); al.put(g->prflag, n * 4);
  al.put(g->ctl, sizeof(Ctl));
  if (g->src_dev) al.put(g->src_dev, (size_t)g->n_src * 4);
  drop_batch_graphs(g);
  if (g->ctl_host) cudaFreeHost(g->ctl_host);
  for (auto &e : g->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : g->ev_inval)
    if (e) cudaEventDestroy(e);
  if (g->fork_ev) cudaEventDestroy(g->fork_ev);
  if (g->join_ev) cudaEventDestroy(g->join_ev);
  if (g->fork0_ev) cudaEventDestroy(g->fork0_ev);
  if (g->search_ev) cudaEventDestroy(g->search_ev);
  if (g->side) cudaStreamDestroy(g->side);
  cudaStreamSynchronize(g->stream);
  delete g;
  return SP_OK;
}

sp_status sp_graph_create(int32_t n, int64_t m, const int64_t *row_off, const int32_t *col,
                          const int32_t *w, int inputs_on_device, float slack,
                          const sp_allocator *alloc, void *cuda_stream, sp_graph **out) {
  if (!out) return SP_EINVAL;
  *out = nullptr;
  if (n <= 0 || m < 0 || !row_off || (m > 0 && (!col || !w)) || !(slack >= 0.f) || slack > 16.f)
    return SP_EINVAL;
  if (m > kMaxEdges) return SP_EINVAL;
  if (alloc && (!alloc->alloc || !alloc->free)) return SP_EINVAL;
  sp_graph *g = new (std::nothrow) sp_graph();
  if (!g) return SP_ENOMEM;
  g->n = n;
  g->bits = sp::id_bits(n);
  g->slack = slack;
  g->stream = (cudaStream_t)cuda_stream;
  g->al.stream = g->stream;
  if (alloc) {
    g->al.user = *alloc;
    g->al.has_user = true;
  }
  if (cudaGetDevice(&g->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) !=
          cudaSuccess) {
    cudaGetLastError();
    delete g;
    return SP_ECUDA;
  }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
  g->loop_blocks_push = sp::loop_blocks(0, g->num_sms);
  g->loop_blocks_inval = sp::loop_blocks(1, g->num_sms);
  g->loop_blocks_pool = std::min(sp::loop_blocks(3, g->num_sms), sp::loop_blocks(4, g->num_sms));
  g->sort_blocks = sp::batch_sort_blocks(g->num_sms);
  g->count_blocks = sp::count_blocks(g->num_sms);
  if (!coop || g->loop_blocks_push <= 0 || g->loop_blocks_inval <= 0 ||
      g->loop_blocks_pool <= 0 || g->sort_blocks <= 0 || g->count_blocks <= 0) {
    delete g;
    return SP_ECUDA;
  }
  for (auto &e : g->ev)
    if (cudaEventCreate(&e) != cudaSuccess) {
      sp_graph_destroy(g);
      return SP_ECUDA;
    }
  for (auto &e : g->ev_inval)
    if (cudaEventCreate(&e) != cudaSuccess) {
      sp_graph_destroy(g);
      return SP_ECUDA;
    }
  // the side stream of the invalidation; without it (or on the legacy
  // default stream) the invalidation runs after the merge
  if (g->stream &&
      (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess ||
       cudaEventCreateWithFlags(&g->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&g->join_ev, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&g->fork0_ev, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&g->search_ev, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    sp_graph_destroy(g);
    return SP_ECUDA;
  }
  if (cudaMallocHost(&g->ctl_host, sizeof(Ctl)) != cudaSuccess) {
    cudaGetLastError();
    g->ctl_host = nullptr;
    sp_graph_destroy(g);
    return SP_ENOMEM;
  }
  g->ctl = (Ctl *)g->al.get(sizeof(Ctl));
  const size_t nn = (size_t)n;
  g->s = (u64 *)g->al.get(nn * 8);
  g->qflag = (u32 *)g->al.get(nn * 4);
  bool bufs_ok = true;
  for (int b = 0; b < 3; ++b) {
    g->qent[b] = (int2 *)g->al.get(nn * 8);
    g->qsv[b] = (u32 *)g->al.get(nn * 4);
    g->fq[b] = (u32 *)g->al.get(nn * 4);
    bufs_ok = bufs_ok && g->qent[b] && g->qsv[b] && g->fq[b];
  }
  g->asv = (u32 *)g->al.get(nn * 4);
  bufs_ok = bufs_ok && g->asv;
  g->aent = (int2 *)g->al.get(nn * 8);
  g->ftag = (u32 *)g->al.get(nn * 4);
  g->jmp = (u32 *)g->al.get(nn * 4);
  g->cut = (u32 *)g->al.get(nn * 4);
  g->out_dist = (int *)g->al.get(nn * 4);
  g->out_parent = (int *)g->al.get(nn * 4);
  if (!g->ctl || !g->s || !g->qflag || !bufs_ok || !g->aent || !g->ftag || !g->jmp || !g->cut ||
      !g->out_dist || !g->out_parent) {
    sp_graph_destroy(g);
    return SP_ENOMEM;
  }
  cudaMemsetAsync(g->ctl, 0, sizeof(Ctl), g->stream);
  cudaMemsetAsync(g->qflag, 0, nn * 4, g->stream);
  cudaMemsetAsync(g->ftag, 0, nn * 4, g->stream);
  int launches = 0;
  sp::launch_ctl_reset(g, 1, &launches);

  // inputs on the device
  const long long *ro_d = (const long long *)row_off;
  const int *col_d = col, *w_d = w;
  void *tmp_in = nullptr;
  size_t tmp_in_bytes = 0;
  if (!inputs_on_device) {
    tmp_in_bytes = (nn + 1) * 8 + (size_t)std::max<int64_t>(m, 1) * 8 + 512;
    tmp_in = g->al.get(tmp_in_bytes);
    if (!tmp_in) {
      sp_graph_destroy(g);
      return SP_ENOMEM;
    }
    long long *ro = (long long *)tmp_in;
    int *cc = (int *)(((uintptr_t)(ro + nn + 1) + 255) & ~(uintptr_t)255);
    int *ww = cc + std::max<int64_t>(m, 1);
    cudaMemcpyAsync(ro, row_off, (nn + 1) * 8, cudaMemcpyHostToDevice, g->stream);
    if (m > 0) {
      cudaMemcpyAsync(cc, col, (size_t)m * 4, cudaMemcpyHostToDevice, g->stream);
      cudaMemcpyAsync(ww, w, (size_t)m * 4, cudaMemcpyHostToDevice, g->stream);
    }
    ro_d = ro;
    col_d = cc;
    w_d = ww;
  }
  sp_status rc = sp::csr_validate(g, ro_d, col_d, w_d, m, &launches);
  if (rc == SP_OK) rc = sp::store_build(g, &g->fwd, ro_d, col_d, w_d, m, 0, &launches);
  if (rc == SP_OK) rc = sp::store_build(g, &g->rev, ro_d, col_d, w_d, m, 1, &launches);
  if (rc == SP_OK) rc = sp::ensure_owner_tables(g);
  if (tmp_in) g->al.put(tmp_in, tmp_in_bytes);
  unsigned long long deg_mid = 0;
  if (rc == SP_OK) {   // the degree share that picks the pool kernel
    sp::launch_deg_mid(g, &launches);
    cudaMemcpyAsync(&deg_mid, &g->ctl->deg_mid, sizeof(deg_mid), cudaMemcpyDeviceToHost,
                    g->stream);
  }
  if (rc == SP_OK && cudaStreamSynchronize(g->stream) != cudaSuccess) rc = SP_ECUDA;
  g->pool_wide = sp::pool_wide_for((long long)deg_mid, g->n);
  if (rc != SP_OK) {
    cudaGetLastError();
    sp_graph_destroy(g);
    return rc;
  }
  g->m = m;
  set_limits(g);
  *out = g;
  return SP_OK;
}

sp_status sp_set_limits(sp_graph *g, int32_t max_rounds, int64_t wait_ns) {
  if (!g || max_rounds < 0 || wait_ns < 0) return SP_EINVAL;
  g->max_rounds_user = max_rounds;
  g->wait_ns_user = wait_ns;
  set_limits(g);
  return SP_OK;
}

sp_status sp_set_push_delta(sp_graph *g, int32_t delta) {
  if (!g || delta < 0) return SP_EINVAL;
  g->delta_user = delta;
  set_limits(g);
  return SP_OK;
}

sp_status sp_loop_counters(const sp_graph *g, int64_t *out, int32_t k) {
  if (!g || !out || k < 0 || k > 16) return SP_EINVAL;
  const Ctl &c = *g->ctl_host;
  const int64_t v[16] = {c.rounds_push, c.local_rounds, c.local_episodes, c.splits,
                         (int64_t)c.far_moves, c.rounds_inval, c.jumps,
                         (int64_t)c.local_ns, (int64_t)c.push_ns, c.timeout,
                         c.to_site, c.to_info, (int64_t)c.pool_sub, (int64_t)c.pool_in,
                         (int64_t)c.pool_ns, (int64_t)c.pool_sub0};
  for (int i = 0; i < k; ++i) out[i] = v[i];
  return SP_OK;
}

sp_status sp_set_local_rounds(sp_graph *g, int32_t max_edges) {
  if (!g || max_edges < 0) return SP_EINVAL;
  g->local_edges_user = std::min<int32_t>(max_edges, (int32_t)sp::kLocalRoundCap);
  set_limits(g);
  return SP_OK;
}

sp_status sp_set_schedule(sp_graph *g, int32_t small_deg, int32_t pool_rounds) {
  if (!g || small_deg < 0 || small_deg > 64 || pool_rounds < 0 || pool_rounds > 16384)
    return SP_EINVAL;
  g->small_deg_user = small_deg;
  g->pool_rounds_user = pool_rounds;
  set_limits(g);
  return SP_OK;
}

sp_status sp_inject_missed_arrival(sp_graph *g, int32_t site) {
  if (!g || !(site == 0 || site == 2 || site == 4 || site == 5)) return SP_EINVAL;
  g->miss_site_user = site;
  set_limits(g);
  return SP_OK;
}

sp_status sp_set_inval_switch(sp_graph *g, int32_t rounds) {
  if (!g) return SP_EINVAL;
  g->jump_round_user = rounds < 0 ? -1 : rounds;
  set_limits(g);
  return SP_OK;
}

sp_status sp_sssp_init(sp_graph *g, int32_t source, sp_batch_stats *stats) {
  if (!g) return SP_EINVAL;
  if (source < 0 || source >= g->n) return SP_EINVAL;
  const bool timed = stats != nullptr;
  int launches = 0;
  for (int i = 0; i < SP_NPHASE; ++i) rec(g, timed, i);   // empty phases
  sp::launch_ctl_reset(g, 0, &launches);
  sp::launch_init(g, source, &launches);
  cudaError_t e = sp::launch_push(g, &launches);
  rec(g, timed, SP_NPHASE - 1);
  sp::launch_finish(g, &launches);
  rec(g, timed, SP_NPHASE);
  if (e != cudaSuccess) {
    g->last_err = (int)e;
    cudaGetLastError();
    cudaStreamSynchronize(g->stream);
    g->state = 2;
    return SP_ECUDA;
  }
  sp_status rc = read_ctl(g, true);
  if (rc != SP_OK) {
    g->state = 2;
    return rc;
  }
  const Ctl &c = *g->ctl_host;
  fill_stats(g, c, stats, launches, 0, 0, timed);
  if (stats) {
    // an init has only the push phase
    for (int i = 0; i < SP_NPHASE; ++i)
      if (i != SP_PH_PUSH) stats->alg_bytes[i] = 0;
    stats->alg_bytes[SP_PH_PUSH] += (int64_t)g->n * 8;  // the reset of all states
  }
  rc = status_of_repair(g, c);
  g->source = source;
  if (g->src_dev) g->al.put(g->src_dev, (size_t)g->n_src * 4);
  g->src_dev = nullptr;
  g->n_src = 1;
  if (rc == SP_OK) g->state = 1;
  return rc;
}

}  // extern "C"

namespace {

// Where a batch call writes the distances (and parents) after the repair:
// device addresses for the unpack kernel, or the graph's unpack buffers and
// a copy to pageable host arrays behind it.  want = false: no read-out.
struct DistOut {
  bool want = false;
  int32_t *dist_d = nullptr, *parent_d = nullptr;   // unpack targets
  int32_t *dist_h = nullptr, *parent_h = nullptr;   // pageable host copies (or null)
};

sp_status resolve_out(sp_graph *g, int32_t *dist, int32_t *parent, int out_on_device,
                      DistOut *o) {
  o->want = true;
  if (out_on_device) {
    if (!device_out(g, dist) || (parent && !device_out(g, parent))) return SP_EINVAL;
    o->dist_d = dist;
    o->parent_d = parent;
    return SP_OK;
  }
  int32_t *md = (int32_t *)mapped_host(dist);
  int32_t *mp = parent ? (int32_t *)mapped_host(parent) : nullptr;
  if (md && (!parent || mp)) {   // page-locked and mapped: written in place
    o->dist_d = md;
    o->parent_d = mp;
    return SP_OK;
  }
  o->dist_d = g->out_dist;
  o->parent_d = parent ? g->out_parent : nullptr;
  o->dist_h = dist;
  o->parent_h = parent;
  return SP_OK;
}

void enqueue_out(sp_graph *g, const DistOut &o, int *launches) {
  if (!o.want) return;
  sp::launch_unpack(g, o.dist_d, o.parent_d, launches);
  if (o.dist_h)
    cudaMemcpyAsync(o.dist_h, o.dist_d, (size_t)g->n * 4, cudaMemcpyDeviceToHost, g->stream);
  if (o.parent_h)
    cudaMemcpyAsync(o.parent_h, o.parent_d, (size_t)g->n * 4, cudaMemcpyDeviceToHost,
                    g->stream);
}

sp_status apply_batch(sp_graph *g, int64_t n_del, const int32_t *del_src,
                      const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                      const int32_t *add_dst, const int32_t *add_w, int inputs_on_device,
                      sp_batch_stats *stats, const DistOut &out);

}  // namespace

extern "C" {

sp_status sp_apply_batch(sp_graph *g, int64_t n_del, const int32_t *del_src,
                         const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                         const int32_t *add_dst, const int32_t *add_w, int inputs_on_device,
                         sp_batch_stats *stats) {
  return apply_batch(g, n_del, del_src, del_dst, n_add, add_src, add_dst, add_w,
                     inputs_on_device, stats, DistOut());
}

sp_status sp_apply_batch_get(sp_graph *g, int64_t n_del, const int32_t *del_src,
                             const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                             const int32_t *add_dst, const int32_t *add_w,
                             int inputs_on_device, int32_t *dist, int32_t *parent,
                             int out_on_device, sp_batch_stats *stats) {
  if (!g || !dist) return SP_EINVAL;
  DistOut o;
  sp_status rc = resolve_out(g, dist, parent, out_on_device, &o);
  if (rc != SP_OK) return rc;
  return apply_batch(g, n_del, del_src, del_dst, n_add, add_src, add_dst, add_w,
                     inputs_on_device, stats, o);
}

}  // extern "C"

namespace {

sp_status apply_batch(sp_graph *g, int64_t n_del, const int32_t *del_src,
                      const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                      const int32_t *add_dst, const int32_t *add_w, int inputs_on_device,
                      sp_batch_stats *stats, const DistOut &out) {
  if (!g) return SP_EINVAL;
  if (n_del < 0 || n_add < 0) return SP_EINVAL;
  if ((n_del > 0 && (!del_src || !del_dst)) || (n_add > 0 && (!add_src || !add_dst || !add_w)))
    return SP_EINVAL;
  if (n_del + n_add > (1LL << 30)) return SP_EINVAL;
  if (g->m + n_add > kMaxEdges) return SP_EINVAL;
  if (g->state != 1) return SP_ESTATE;
  const long long nb = n_del + n_add, ni = 2 * nb;
  const bool timed = stats != nullptr;
  // the same batch shape twice in a row: the pipeline runs as a cached CUDA
  // graph (one launch instead of seven), its input-reading nodes pointed at
  // this call's arrays
  const bool repeat = n_del == g->last_nd && n_add == g->last_na && (int)timed == g->last_timed;
  g->last_nd = n_del;
  g->last_na = n_add;
  g->last_timed = (int)timed;
  const bool use_graph = g->batch_graphs && g->stream && nb > 0 && repeat;
  const int *ds = del_src, *dd = del_dst, *as = add_src, *ad = add_dst, *aw = add_w;
  // host arrays in page-locked, mapped memory are gathered into the staging
  // buffers by one kernel (16-byte loads across the host link); any other
  // host array is copied there by the copy engine
  const void *m[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool mapped = false;
  if (!inputs_on_device) {
    mapped = true;
    if (n_del) {
      m[0] = mapped_host(del_src);
      m[1] = mapped_host(del_dst);
      mapped = m[0] && m[1];
    }
    if (n_add && mapped) {
      m[2] = mapped_host(add_src);
      m[3] = mapped_host(add_dst);
      m[4] = mapped_host(add_w);
      mapped = m[2] && m[3] && m[4];
    }
  }
  sp_status rc = ensure_batch_buffers(g, ni, inputs_on_device ? 0 : std::max(n_del, n_add));
  if (rc != SP_OK) return rc;
  auto &b = g->bb;
  rec(g, timed, 0);
  int staged = 0;
  if (mapped) {
    const int *src[5] = {(const int *)m[0], (const int *)m[1], (const int *)m[2],
                         (const int *)m[3], (const int *)m[4]};
    int *const dst[5] = {b.in_del_src, b.in_del_dst, b.in_add_src, b.in_add_dst, b.in_add_w};
    const long long cnt[5] = {n_del, n_del, n_add, n_add, n_add};
    sp::launch_stage_inputs(g, src, dst, cnt, &staged);
    ds = b.in_del_src; dd = b.in_del_dst; as = b.in_add_src; ad = b.in_add_dst; aw = b.in_add_w;
  } else if (!inputs_on_device) {
    cudaStream_t s = g->stream;
    const cudaMemcpyKind kind = inputs_on_device ? cudaMemcpyDeviceToDevice
                                                 : cudaMemcpyHostToDevice;
    if (n_del) {
      cudaMemcpyAsync(b.in_del_src, del_src, n_del * 4, kind, s);
      cudaMemcpyAsync(b.in_del_dst, del_dst, n_del * 4, kind, s);
    }
    if (n_add) {
      cudaMemcpyAsync(b.in_add_src, add_src, n_add * 4, kind, s);
      cudaMemcpyAsync(b.in_add_dst, add_dst, n_add * 4, kind, s);
      cudaMemcpyAsync(b.in_add_w, add_w, n_add * 4, kind, s);
    }
    ds = b.in_del_src; dd = b.in_del_dst; as = b.in_add_src; ad = b.in_add_dst; aw = b.in_add_w;
  }
  int launches = 0, regrows = 0;
  // the first attempt runs the invalidation beside the store update; a rerun
  // after a pool grow keeps what it found (it already changed the distances)
  const int mode0 = inval_beside(g) ? kInvalBeside : kInvalAfter;
  for (int attempt = 0;; ++attempt) {
    launches = 0;
    if (attempt) rec(g, timed, 0);
    cudaError_t e = cudaSuccess;
    bool replayed = false;
    if (use_graph && attempt == 0) {
      if (!(g->bg_ready && g->bg_gen == g->gen && g->bg_nd == n_del && g->bg_na == n_add &&
            g->bg_timed == (int)timed)) {
        drop_batch_graphs(g);
        int cl = 0;
        if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
          g->capturing = 0;
          const cudaError_t ce = enqueue_batch(g, ds, dd, n_del, as, ad, aw, n_add, timed, &cl,
                                               mode0);
          g->capturing = -1;
          cudaGraph_t gr = nullptr;
          bool ok = cudaStreamEndCapture(g->stream, &gr) == cudaSuccess && ce == cudaSuccess && gr;
          g->bg_graph = gr;
          ok = ok && cudaGraphInstantiate(&g->bg_exec, g->bg_graph, 0) == cudaSuccess;
          ok = ok && find_input_nodes(g);
          if (ok) {
            g->bg_ready = true;
            g->bg_gen = g->gen;
            g->bg_nd = n_del;
            g->bg_na = n_add;
            g->bg_timed = (int)timed;
            g->bg_launches = cl;
          } else {
            drop_batch_graphs(g);
          }
        }
        g->capturing = -1;
        cudaGetLastError();
      }
      // a replay reads this call's inputs: the two nodes that read them are
      // pointed at them (no copy of the batch)
      if (g->bg_ready && retarget_input_nodes(g, ds, dd, n_del, as, ad, aw, n_add) != cudaSuccess) {
        cudaGetLastError();
        drop_batch_graphs(g);
      }
      if (g->bg_ready) {
        e = cudaGraphLaunch(g->bg_exec, g->stream);
        launches = g->bg_launches;
        replayed = true;
      }
    }
    if (!replayed)
      e = enqueue_batch(g, ds, dd, n_del, as, ad, aw, n_add, timed, &launches,
                        attempt == 0 ? mode0 : (mode0 == kInvalBeside ? kInvalKept : kInvalAfter));
    if (e != cudaSuccess) {
      g->last_err = (int)e;
      cudaGetLastError();
      cudaStreamSynchronize(g->stream);
      g->state = 2;
      return SP_ECUDA;
    }
    // the read-out follows the batch on the stream (a rerun repeats it)
    enqueue_out(g, out, &launches);
    rc = read_ctl(g, true);   // the batch ends with k_finish, replayed or not
    if (rc != SP_OK) {
      g->state = 2;
      return rc;
    }
    const Ctl &c = *g->ctl_host;
    // the edge set is as it was: the merge did not run.  A bound hit in the
    // batch sort or the count pass (SP_ETIMEOUT) may have let the
    // invalidation beside them change distances, which then need sp_sssp_init
    if (c.status != 0) {
      if (c.status == SP_ETIMEOUT) g->state = 2;
      return (sp_status)c.status;
    }
    if (c.need_grow == 0) break;
    // the merge did not run either; a shortfall that cannot be grown leaves
    // the edge set as it was and the distances are restored
    const bool touched = mode0 == kInvalBeside && n_del > 0;
    if (attempt >= 6) return restore_after(g, touched, SP_ENOMEM);
    ++regrows;
    if (c.need_grow & sp::kGrowPoolFwd) {
      rc = sp::store_grow_pool(g, &g->fwd, (long long)c.pool_need[0] + 1024);
      if (rc != SP_OK) return restore_after(g, touched, rc);
    }
    if (c.need_grow & sp::kGrowPoolRev) {
      rc = sp::store_grow_pool(g, &g->rev, (long long)c.pool_need[1] + 1024);
      if (rc != SP_OK) return restore_after(g, touched, rc);
    }
    if (c.need_grow & (sp::kGrowPoolFwd | sp::kGrowPoolRev)) {
      rc = sp::ensure_owner_tables(g);
      if (rc != SP_OK) return restore_after(g, touched, rc);
    }

  }
  const Ctl &c = *g->ctl_host;
  g->m += (long long)c.add_applied - (long long)c.del_applied;
  if (c.add_applied + c.del_applied > 0) {
    g->pr_state = 0;   // ranks no longer hold
    g->tc_state = 0;   // nor does the triangle count
  }
  fill_stats(g, c, stats, launches + staged, regrows, ni, timed, true);
  if (g->lim.pool_rounds > 0) {   // a changed choice of pool kernel recaptures the graph
    const bool wide = sp::pool_wide_for((long long)c.deg_mid, g->n);
    if (wide != g->pool_wide) {
      g->pool_wide = wide;
      ++g->gen;
    }
  }
  return status_of_repair(g, c);
}

}  // namespace

extern "C" {

sp_status sp_sssp_init_multi(sp_graph *g, const int32_t *sources, int32_t k,
                             int sources_on_device, sp_batch_stats *stats) {
  if (!g || !sources || k < 1) return SP_EINVAL;
  std::vector<int32_t> hs((size_t)k);
  if (sources_on_device) {
    if (cudaMemcpy(hs.data(), sources, (size_t)k * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return SP_ECUDA;
    }
  } else {
    std::copy(sources, sources + k, hs.begin());
  }
  for (int32_t v : hs)
    if (v < 0 || v >= g->n) return SP_EINVAL;
  int *src_d = (int *)g->al.get((size_t)k * 4);
  if (!src_d) return SP_ENOMEM;
  const bool timed = stats != nullptr;
  int launches = 0;
  for (int i = 0; i < SP_NPHASE; ++i) rec(g, timed, i);
  cudaMemcpyAsync(src_d, hs.data(), (size_t)k * 4, cudaMemcpyHostToDevice, g->stream);
  sp::launch_ctl_reset(g, 0, &launches);
  sp::launch_init_multi(g, src_d, k, &launches);
  cudaError_t e = sp::launch_push(g, &launches);
  rec(g, timed, SP_NPHASE - 1);
  sp::launch_finish(g, &launches);
  rec(g, timed, SP_NPHASE);
  sp_status rc = read_ctl(g, true);
  // the list stays with the handle (a failed batch restores from it)
  if (g->src_dev) g->al.put(g->src_dev, (size_t)g->n_src * 4);
  g->src_dev = src_d;
  g->n_src = k;
  if (e != cudaSuccess) {
    g->last_err = (int)e;
    cudaGetLastError();
    g->state = 2;
    return SP_ECUDA;
  }
  if (rc != SP_OK) {
    g->state = 2;
    return rc;
  }
  const Ctl &c = *g->ctl_host;
  fill_stats(g, c, stats, launches, 0, 0, timed);
  rc = status_of_repair(g, c);
  g->source = hs[0];
  if (rc == SP_OK) g->state = 1;
  return rc;
}

sp_status sp_reserve(sp_graph *g, int64_t max_updates) {
  if (!g || max_updates < 0 || max_updates > (1LL << 30)) return SP_EINVAL;
  return ensure_batch_buffers(g, 2 * max_updates, 0);
}

size_t sp_async_result_bytes(void) { return sizeof(Ctl); }

sp_status sp_apply_batch_async(sp_graph *g, int64_t n_del, const int32_t *del_src,
                               const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                               const int32_t *add_dst, const int32_t *add_w, void *result) {
  if (!g || !result || n_del < 0 || n_add < 0) return SP_EINVAL;
  if ((n_del > 0 && (!del_src || !del_dst)) || (n_add > 0 && (!add_src || !add_dst || !add_w)))
    return SP_EINVAL;
  if (g->state != 1) return SP_ESTATE;
  const long long ni = 2 * (n_del + n_add);
  if (!reserved_for(g, ni)) return SP_ENOMEM;
  int launches = 0;
  cudaError_t e = enqueue_batch(g, del_src, del_dst, n_del, add_src, add_dst, add_w, n_add,
                                false, &launches);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(result, g->ctl, sizeof(Ctl), cudaMemcpyDefault, g->stream);
  if (e != cudaSuccess) {
    g->last_err = (int)e;
    cudaGetLastError();
    return SP_ECUDA;
  }
  g->async_ni = ni;
  g->async_launches = launches + 1;
  g->pr_state = 0;   // the edge set may change: ranks and counts no longer hold
  g->tc_state = 0;
  return SP_OK;
}

sp_status sp_apply_batch_finish(sp_graph *g, const void *result_host, sp_batch_stats *stats) {
  if (!g || !result_host) return SP_EINVAL;
  const Ctl &c = *(const Ctl *)result_host;
  if (c.status != 0) {   // the edge set did not change
    if (c.status == SP_ETIMEOUT) g->state = 2;
    return (sp_status)c.status;
  }
  if (c.need_grow) return SP_ENOMEM;               // nothing changed: use sp_apply_batch
  g->m += (long long)c.add_applied - (long long)c.del_applied;
  fill_stats(g, c, stats, g->async_launches, 0, g->async_ni, false);
  return status_of_repair(g, c);
}

sp_status sp_capture_apply(sp_graph *g, int64_t n_del, const int32_t *del_src,
                           const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                           const int32_t *add_dst, const int32_t *add_w, void *result,
                           sp_exec **out) {
  if (!g || !out) return SP_EINVAL;
  *out = nullptr;
  if (!g->stream) return SP_EINVAL;   // the legacy default stream cannot be captured
  if (g->state != 1) return SP_ESTATE;
  if (!reserved_for(g, 2 * (n_del + n_add))) return SP_ENOMEM;
  sp_exec *x = new (std::nothrow) sp_exec();
  if (!x) return SP_ENOMEM;
  x->g = g;
  if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    delete x;
    return SP_ECUDA;
  }
  sp_status rc = sp_apply_batch_async(g, n_del, del_src, del_dst, n_add, add_src, add_dst,
                                      add_w, result);
  cudaError_t e = cudaStreamEndCapture(g->stream, &x->graph);
  if (rc == SP_OK && e == cudaSuccess)
    e = cudaGraphInstantiate(&x->exec, x->graph, 0);
  if (rc != SP_OK || e != cudaSuccess) {
    cudaGetLastError();
    if (x->graph) cudaGraphDestroy(x->graph);
    delete x;
    return rc != SP_OK ? rc : SP_ECUDA;
  }
  *out = x;
  return SP_OK;
}

sp_status sp_exec_launch(sp_exec *x) {
  if (!x || !x->exec) return SP_EINVAL;
  if (cudaGraphLaunch(x->exec, x->g->stream) != cudaSuccess) {
    cudaGetLastError();
    return SP_ECUDA;
  }
  return SP_OK;
}

sp_status sp_exec_destroy(sp_exec *x) {
  if (!x) return SP_OK;
  if (x->exec) cudaGraphExecDestroy(x->exec);
  if (x->graph) cudaGraphDestroy(x->graph);
  delete x;
  return SP_OK;
}

// ---- PageRank (appendix listing "Dynamic PR") ------------------------------

namespace {

// One DynPR phase on the device: flags from `dst` spread along out-edges
// (propagateNodeFlags), the phase's updates merged into both stores
// (updateCSRDel or updateCSRAdd), then Jacobi steps over the flagged
// vertices (Decremental or Incremental).  Grows the spare pools and
// repeats the phase when a merge runs out of room (nothing has changed
// then).  Adds the phase's counters to acc.
sp_status pr_phase(sp_graph *g, const int *ds, const int *dd, long long nd, const int *as,
                   const int *ad, const int *aw, long long na, const int *flag_dst,
                   long long n_flag, Ctl &acc, int *launches, int *regrows) {
  const long long ni = 2 * (nd + na);
  if (ni == 0) return SP_OK;
  sp_status rc = SP_OK;
  for (int attempt = 0;; ++attempt) {
    ++g->prtag;
    sp::launch_ctl_reset(g, 0, launches);
    cudaError_t e = cudaSuccess;
    if (n_flag > 0) e = sp::launch_flag(g, flag_dst, n_flag, launches);
    const cudaError_t eq = sp::launch_search(g, ds, dd, nd, as, ad, aw, na, launches, g->stream);
    if (e == cudaSuccess) e = eq;
    const cudaError_t es = sp::launch_batch_sort(g, ds, dd, nd, as, ad, aw, na, launches);
    if (e == cudaSuccess) e = es;
    sp::launch_count(g, ni, launches);
    sp::launch_merge(g, ni, launches);
    sp::launch_finish(g, launches);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      g->last_err = (int)e;
      cudaGetLastError();
      cudaStreamSynchronize(g->stream);
      return SP_ECUDA;
    }
    rc = read_ctl(g, true);
    if (rc != SP_OK) return rc;
    const Ctl &c = *g->ctl_host;
    if (c.status != 0) return (sp_status)c.status;
    if (c.bad) return SP_ECUDA;
    if (c.timeout) return SP_ETIMEOUT;
    if (c.need_grow == 0) break;
    if (attempt >= 6) return SP_ENOMEM;
    ++*regrows;
    if (c.need_grow & sp::kGrowPoolFwd) {
      rc = sp::store_grow_pool(g, &g->fwd, (long long)c.pool_need[0] + 1024);
      if (rc != SP_OK) return rc;
    }
    if (c.need_grow & sp::kGrowPoolRev) {
      rc = sp::store_grow_pool(g, &g->rev, (long long)c.pool_need[1] + 1024);
      if (rc != SP_OK) return rc;
    }
    rc = sp::ensure_owner_tables(g);
    if (rc != SP_OK) return rc;
  }
  {
    const Ctl &c = *g->ctl_host;
    g->m += (long long)c.add_applied - (long long)c.del_applied;
    acc.del_applied += c.del_applied;
    acc.del_absent += c.del_absent;
    acc.add_applied += c.add_applied;
    acc.add_present += c.add_present;
    acc.affected += c.affected;
    acc.rows_touched += c.rows_touched;
    acc.rows_relocated += c.rows_relocated;
    acc.inval_edges += c.inval_edges;
    acc.merge_slots += c.merge_slots;
    acc.rounds_inval += c.rounds_inval;
  }
  if (n_flag == 0) return SP_OK;   // nothing flagged: every rank stays
  sp::launch_pr_select(g, 0, launches);
  cudaError_t e = sp::launch_pr(g, launches);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    g->last_err = (int)e;
    cudaGetLastError();
    cudaStreamSynchronize(g->stream);
    return SP_ECUDA;
  }
  rc = read_ctl(g);
  if (rc != SP_OK) return rc;
  const Ctl &c = *g->ctl_host;
  acc.pull_edges += c.pull_edges;
  acc.rounds_push += c.pr_iters;
  if (c.bad) return SP_ECUDA;
  if (c.timeout) return SP_ETIMEOUT;
  return SP_OK;
}

void pr_stats(sp_graph *g, const Ctl &c, sp_batch_stats *st, int launches, int regrows,
              float ms) {
  if (!st) return;
  std::memset(st, 0, sizeof(*st));
  st->n_del_applied = (int64_t)c.del_applied;
  st->n_del_absent = (int64_t)c.del_absent;
  st->n_add_applied = (int64_t)c.add_applied;
  st->n_add_present = (int64_t)c.add_present;
  st->affected = (int64_t)c.affected;          // vertices flagged, both phases
  st->relaxed_edges = (int64_t)c.pull_edges;   // in-edges pulled, all Jacobi steps
  st->rows_touched = (int64_t)c.rows_touched;
  st->rows_relocated = (int64_t)c.rows_relocated;
  st->rounds_inval = (int32_t)c.rounds_inval;  // flag-propagation rounds
  st->rounds_push = (int32_t)c.rounds_push;    // Jacobi steps
  st->n_launches = launches;
  st->regrows = regrows;
  // algorithmic bytes: flag propagation (as a frontier walk), the merge, and
  // per pulled in-edge its source id (4), rank (4) and out-degree (4)
  st->alg_bytes[SP_PH_INVAL] = (int64_t)(c.affected * 16 + c.inval_edges * 12);
  st->alg_bytes[SP_PH_MERGE] = (int64_t)(c.merge_slots * 8 + c.rows_touched * 32);
  st->alg_bytes[SP_PH_PULL] = (int64_t)(c.pull_edges * 12);
  st->ms_total = ms;
  (void)g;
}

}  // namespace

sp_status sp_pr_init(sp_graph *g, float damping, float beta, int32_t max_iter,
                     sp_batch_stats *stats) {
  if (!g || !(damping >= 0.f && damping <= 1.f) || !(beta >= 0.f) || max_iter < 1)
    return SP_EINVAL;
  const size_t nn = (size_t)g->n;
  if (!g->pr[0]) {
    g->pr[0] = (float *)g->al.get(nn * 4);
    g->pr[1] = (float *)g->al.get(nn * 4);
    g->prc[0] = (float *)g->al.get(nn * 4);
    g->prc[1] = (float *)g->al.get(nn * 4);
    g->pracc = (float *)g->al.get(nn * 4);
    g->prflag = (u32 *)g->al.get(nn * 4);
    if (!g->pr[0] || !g->pr[1] || !g->prc[0] || !g->prc[1] || !g->pracc || !g->prflag)
      return SP_ENOMEM;
    cudaMemsetAsync(g->prflag, 0, nn * 4, g->stream);
    g->prtag = 0;
    if (sp::loop_blocks(2, g->num_sms) <= 0) return SP_ECUDA;
  }
  g->pr_damping = damping;
  g->pr_beta = beta;
  g->pr_max_iter = max_iter;
  int launches = 0;
  rec(g, true, 0);
  sp::launch_ctl_reset(g, 0, &launches);
  sp::launch_pr_fill(g, 1.0f / (float)g->n, &launches);
  sp::launch_pr_select(g, 1, &launches);
  cudaError_t e = sp::launch_pr(g, &launches);
  rec(g, true, SP_NPHASE);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    g->last_err = (int)e;
    cudaGetLastError();
    cudaStreamSynchronize(g->stream);
    g->pr_state = 0;
    return SP_ECUDA;
  }
  sp_status rc = read_ctl(g);
  if (rc != SP_OK) return rc;
  const Ctl &c = *g->ctl_host;
  if (c.bad || c.timeout) {
    g->pr_state = 0;
    return c.bad ? SP_ECUDA : SP_ETIMEOUT;
  }
  g->pr_state = 1;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, g->ev[0], g->ev[SP_NPHASE]);
  Ctl acc{};
  acc.pull_edges = c.pull_edges;
  acc.rounds_push = c.pr_iters;
  acc.affected = (u64)g->n;
  pr_stats(g, acc, stats, launches, 0, ms);
  return SP_OK;
}

sp_status sp_pr_apply_batch(sp_graph *g, int64_t n_del, const int32_t *del_src,
                            const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                            const int32_t *add_dst, const int32_t *add_w, int inputs_on_device,
                            sp_batch_stats *stats) {
  if (!g) return SP_EINVAL;
  if (n_del < 0 || n_add < 0) return SP_EINVAL;
  if ((n_del > 0 && (!del_src || !del_dst)) || (n_add > 0 && (!add_src || !add_dst || !add_w)))
    return SP_EINVAL;
  if (n_del + n_add > (1LL << 30)) return SP_EINVAL;
  if (g->m + n_add > kMaxEdges) return SP_EINVAL;
  if (g->pr_state != 1) return SP_ESTATE;
  const long long nb = n_del + n_add;
  sp_status rc = ensure_batch_buffers(g, 2 * nb, inputs_on_device ? 0 : std::max(n_del, n_add));
  if (rc != SP_OK) return rc;
  auto &b = g->bb;
  const int *ds = del_src, *dd = del_dst, *as = add_src, *ad = add_dst, *aw = add_w;
  rec(g, true, 0);
  if (!inputs_on_device) {
    cudaStream_t s = g->stream;
    if (n_del) {
      cudaMemcpyAsync(b.in_del_src, del_src, n_del * 4, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(b.in_del_dst, del_dst, n_del * 4, cudaMemcpyHostToDevice, s);
    }
    if (n_add) {
      cudaMemcpyAsync(b.in_add_src, add_src, n_add * 4, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(b.in_add_dst, add_dst, n_add * 4, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(b.in_add_w, add_w, n_add * 4, cudaMemcpyHostToDevice, s);
    }
    ds = b.in_del_src; dd = b.in_del_dst; as = b.in_add_src; ad = b.in_add_dst; aw = b.in_add_w;
  }
  int launches = 0, regrows = 0;
  // the whole batch is checked before the first phase changes anything
  sp::launch_ctl_reset(g, 0, &launches);
  sp::launch_check_batch(g, ds, dd, n_del, as, ad, aw, n_add, &launches);
  rc = read_ctl(g);
  if (rc != SP_OK) return rc;
  if (g->ctl_host->status != 0) return (sp_status)g->ctl_host->status;
  Ctl acc{};
  // deletions: OnDelete flags, propagateNodeFlags, updateCSRDel, Decremental
  rc = pr_phase(g, ds, dd, n_del, nullptr, nullptr, nullptr, 0, dd, n_del, acc, &launches,
                &regrows);
  // insertions: OnAdd flags, propagateNodeFlags, updateCSRAdd, Incremental
  if (rc == SP_OK)
    rc = pr_phase(g, nullptr, nullptr, 0, as, ad, aw, n_add, ad, n_add, acc, &launches,
                  &regrows);
  rec(g, true, SP_NPHASE);
  if (acc.del_applied + acc.add_applied > 0) {
    g->state = 0;      // distances no longer hold
    g->tc_state = 0;   // nor does the triangle count
  }
  if (rc != SP_OK) {
    g->pr_state = 0;
    return rc;
  }
  float ms = 0.f;
  cudaEventSynchronize(g->ev[SP_NPHASE]);
  cudaEventElapsedTime(&ms, g->ev[0], g->ev[SP_NPHASE]);
  pr_stats(g, acc, stats, launches, regrows, ms);
  return SP_OK;
}

// ---- triangle count (appendix listing "Dynamic TC") ---------------------------

sp_status sp_tc_init(sp_graph *g, int64_t *count) {
  if (!g || !count) return SP_EINVAL;
  int launches = 0;
  sp::launch_ctl_reset(g, 0, &launches);
  sp::launch_tc_sym_check(g, &launches);
  sp_status rc = read_ctl(g);
  if (rc != SP_OK) return rc;
  if (g->ctl_host->status != 0) {
    g->tc_state = 0;
    return (sp_status)g->ctl_host->status;
  }
  sp::launch_tc_static(g, &launches);
  if (cudaGetLastError() != cudaSuccess) {
    cudaStreamSynchronize(g->stream);
    return SP_ECUDA;
  }
  rc = read_ctl(g);
  if (rc != SP_OK) return rc;
  g->tc_count = (long long)g->ctl_host->tc_static;
  g->tc_state = 1;
  *count = g->tc_count;
  return SP_OK;
}

sp_status sp_tc_apply_batch(sp_graph *g, int64_t n_del, const int32_t *del_src,
                            const int32_t *del_dst, int64_t n_add, const int32_t *add_src,
                            const int32_t *add_dst, const int32_t *add_w, int inputs_on_device,
                            int64_t *count, sp_batch_stats *stats) {
  if (!g || !count) return SP_EINVAL;
  if (n_del < 0 || n_add < 0) return SP_EINVAL;
  if ((n_del > 0 && (!del_src || !del_dst)) || (n_add > 0 && (!add_src || !add_dst || !add_w)))
    return SP_EINVAL;
  if (n_del + n_add > (1LL << 30)) return SP_EINVAL;
  if (g->m + n_add > kMaxEdges) return SP_EINVAL;
  if (g->tc_state != 1) return SP_ESTATE;
  const long long nb = n_del + n_add, ni = 2 * nb;
  sp_status rc = ensure_batch_buffers(g, ni, inputs_on_device ? 0 : std::max(n_del, n_add));
  if (rc != SP_OK) return rc;
  auto &b = g->bb;
  const int *ds = del_src, *dd = del_dst, *as = add_src, *ad = add_dst, *aw = add_w;
  rec(g, true, 0);
  if (!inputs_on_device) {
    cudaStream_t s = g->stream;
    if (n_del) {
      cudaMemcpyAsync(b.in_del_src, del_src, n_del * 4, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(b.in_del_dst, del_dst, n_del * 4, cudaMemcpyHostToDevice, s);
    }
    if (n_add) {
      cudaMemcpyAsync(b.in_add_src, add_src, n_add * 4, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(b.in_add_dst, add_dst, n_add * 4, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(b.in_add_w, add_w, n_add * 4, cudaMemcpyHostToDevice, s);
    }
    ds = b.in_del_src; dd = b.in_del_dst; as = b.in_add_src; ad = b.in_add_dst; aw = b.in_add_w;
  }
  int launches = 0, regrows = 0;
  for (int attempt = 0;; ++attempt) {
    sp::launch_ctl_reset(g, 0, &launches);
    const cudaError_t eq =
        sp::launch_search(g, ds, dd, n_del, as, ad, aw, n_add, &launches, g->stream);
    cudaError_t es = sp::launch_batch_sort(g, ds, dd, n_del, as, ad, aw, n_add, &launches);
    if (es == cudaSuccess) es = eq;
    rec(g, true, 1);
    sp::launch_count(g, ni, &launches);
    sp::launch_tc_batch_sym(g, nb, &launches);     // before anything changes
    rec(g, true, 2);
    sp::launch_tc_delta(g, nb, 0, &launches);      // Decremental, old graph
    rec(g, true, 3);
    sp::launch_merge(g, ni, &launches);            // updateCSRDel + updateCSRAdd
    rec(g, true, 4);
    sp::launch_tc_delta(g, nb, 1, &launches);      // Incremental, new graph
    rec(g, true, 5);
    sp::launch_finish(g, &launches);
    for (int i = 6; i <= SP_NPHASE; ++i) rec(g, true, i);
    if (es != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      cudaStreamSynchronize(g->stream);
      g->tc_state = 0;
      return SP_ECUDA;
    }
    rc = read_ctl(g, true);
    if (rc != SP_OK) return rc;
    const Ctl &c = *g->ctl_host;
    if (c.status != 0) return (sp_status)c.status;   // nothing changed
    if (c.bad) {
      g->tc_state = 0;
      return SP_ECUDA;
    }
    if (c.need_grow == 0) break;
    if (attempt >= 6) return SP_ENOMEM;
    ++regrows;
    if (c.need_grow & sp::kGrowPoolFwd) {
      rc = sp::store_grow_pool(g, &g->fwd, (long long)c.pool_need[0] + 1024);
      if (rc != SP_OK) return rc;
    }
    if (c.need_grow & sp::kGrowPoolRev) {
      rc = sp::store_grow_pool(g, &g->rev, (long long)c.pool_need[1] + 1024);
      if (rc != SP_OK) return rc;
    }
    rc = sp::ensure_owner_tables(g);
    if (rc != SP_OK) return rc;
  }
  const Ctl &c = *g->ctl_host;
  g->m += (long long)c.add_applied - (long long)c.del_applied;
  if (c.add_applied + c.del_applied > 0) {
    g->state = 0;      // distances no longer hold
    g->pr_state = 0;   // nor do ranks
  }
  const u64 *d = c.tc_del, *a = c.tc_ins;
  if (d[0] % 2 || d[1] % 4 || d[2] % 6 || a[0] % 2 || a[1] % 4 || a[2] % 6) {
    g->tc_state = 0;   // cannot happen on a symmetric graph and batch
    return SP_ECUDA;
  }
  g->tc_count += (long long)(a[0] / 2 + a[1] / 4 + a[2] / 6) -
                 (long long)(d[0] / 2 + d[1] / 4 + d[2] / 6);
  *count = g->tc_count;
  fill_stats(g, c, stats, launches, regrows, ni, true);
  if (stats) {
    stats->affected = (int64_t)(d[0] + d[1] + d[2] + a[0] + a[1] + a[2]);   // sightings
    stats->rounds_inval = stats->rounds_push = 0;
  }
  return SP_OK;
}

sp_status sp_pr_get(const sp_graph *g, float *pr, int out_on_device) {
  if (!g || !pr) return SP_EINVAL;
  if (g->pr_state != 1) return SP_ESTATE;
  const cudaError_t e = cudaMemcpyAsync(pr, g->pr[0], (size_t)g->n * 4,
                                        out_on_device ? cudaMemcpyDeviceToDevice
                                                      : cudaMemcpyDeviceToHost,
                                        g->stream);
  if (e != cudaSuccess || cudaStreamSynchronize(g->stream) != cudaSuccess) {
    cudaGetLastError();
    return SP_ECUDA;
  }
  return SP_OK;
}

sp_status sp_query(sp_graph *g, int32_t k, const int32_t *vertices, int32_t *dist_out,
                   int on_device) {
  if (!g || k < 0 || (k > 0 && (!vertices || !dist_out))) return SP_EINVAL;
  if (g->state != 1) return SP_ESTATE;
  if (k == 0) return SP_OK;
  int launches = 0;
  const int *vs = vertices;
  int *out = dist_out;
  void *buf = nullptr;
  const size_t bytes = (size_t)k * 8 + 256;
  if (!on_device) {
    buf = g->al.get(bytes);
    if (!buf) return SP_ENOMEM;
    int *vd = (int *)buf;
    out = vd + k;
    cudaMemcpyAsync(vd, vertices, (size_t)k * 4, cudaMemcpyHostToDevice, g->stream);
    vs = vd;
  }
  sp::launch_ctl_reset(g, 0, &launches);
  sp::launch_gather(g, vs, k, out, &launches);
  if (!on_device)
    cudaMemcpyAsync(dist_out, out, (size_t)k * 4, cudaMemcpyDeviceToHost, g->stream);
  sp_status rc = read_ctl(g);
  if (buf) g->al.put(buf, bytes);
  if (rc != SP_OK) return rc;
  return g->ctl_host->status != 0 ? (sp_status)g->ctl_host->status : SP_OK;
}

sp_status sp_set_loop_blocks(sp_graph *g, int32_t blocks) {
  if (!g || blocks < 0) return SP_EINVAL;
  g->loop_blocks_user = blocks;
  ++g->gen;
  return SP_OK;
}

const char *sp_last_cuda_error(const sp_graph *g) {
  if (!g) return "invalid handle";
  return cudaGetErrorName((cudaError_t)g->last_err);
}

sp_status sp_set_batch_graphs(sp_graph *g, int32_t on) {
  if (!g || on < 0 || on > 1) return SP_EINVAL;
  g->batch_graphs = on;
  return SP_OK;
}

sp_status sp_sync(sp_graph *g) {
  if (!g) return SP_EINVAL;
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
    cudaGetLastError();
    return SP_ECUDA;
  }
  return SP_OK;
}

sp_status sp_get_dist(sp_graph *g, int32_t *dist, int32_t *parent, int out_on_device) {
  if (!g || !dist) return SP_EINVAL;
  if (g->state != 1) return SP_ESTATE;
  int launches = 0;
  if (out_on_device && (!device_out(g, dist) || (parent && !device_out(g, parent))))
    return SP_EINVAL;
  // a page-locked, mapped host destination is written in place
  int32_t *mdist = out_on_device ? nullptr : (int32_t *)mapped_host(dist);
  int32_t *mparent = out_on_device || !parent ? nullptr : (int32_t *)mapped_host(parent);
  if (out_on_device) {
    sp::launch_unpack(g, dist, parent, &launches);
  } else if (mdist && (!parent || mparent)) {
    sp::launch_unpack(g, mdist, mparent, &launches);
  } else {
    sp::launch_unpack(g, g->out_dist, parent ? g->out_parent : nullptr, &launches);
    cudaMemcpyAsync(dist, g->out_dist, (size_t)g->n * 4, cudaMemcpyDeviceToHost, g->stream);
    if (parent)
      cudaMemcpyAsync(parent, g->out_parent, (size_t)g->n * 4, cudaMemcpyDeviceToHost, g->stream);
  }
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
    cudaGetLastError();
    return SP_ECUDA;
  }
  return SP_OK;
}

sp_status sp_set_dist(sp_graph *g, int32_t source, const int32_t *dist, const int32_t *parent,
                      int in_on_device) {
  if (!g || !dist || !parent || source < 0 || source >= g->n) return SP_EINVAL;
  const int *dd = dist, *pd = parent;
  if (!in_on_device) {   // staged in the unpack buffers
    cudaMemcpyAsync(g->out_dist, dist, (size_t)g->n * 4, cudaMemcpyHostToDevice, g->stream);
    cudaMemcpyAsync(g->out_parent, parent, (size_t)g->n * 4, cudaMemcpyHostToDevice, g->stream);
    dd = g->out_dist;
    pd = g->out_parent;
  }
  int launches = 0;
  sp::launch_ctl_reset(g, 0, &launches);
  sp::launch_state_check(g, dd, pd, source, &launches);
  sp_status rc = read_ctl(g);
  if (rc != SP_OK) return rc;
  if (g->ctl_host->status != 0) return SP_EINVAL;   // not the exact solution: nothing changed
  sp::launch_state_pack(g, dd, pd, &launches);
  if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
    cudaGetLastError();
    g->state = 2;
    return SP_ECUDA;
  }
  g->source = source;
  if (g->src_dev) g->al.put(g->src_dev, (size_t)g->n_src * 4);
  g->src_dev = nullptr;
  g->n_src = 1;
  g->state = 1;
  return SP_OK;
}

sp_status sp_footprint_bound(int32_t n, int64_t m, float slack, int64_t max_updates,
                             int64_t *bytes) {
  if (!bytes || n <= 0 || m < 0 || m > kMaxEdges || !(slack >= 0.f) || slack > 16.f ||
      max_updates < 0 || max_updates > (1LL << 30))
    return SP_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SP_ECUDA;
  }
  const double N = (double)n, M = (double)m;
  // a row of deg edges gets round4(deg + max(slack * deg, 4)) <= (1 + slack) deg + 8
  // slots per region (the float product rounded up), two regions per row
  const double main_slots = 2.0 * ((1.0 + (double)slack * (1.0 + 1e-6)) * M + 9.0 * N);
  const double pool = std::max(main_slots / 4.0 + 4.0, 65536.0);
  const double slots = main_slots + pool;
  double b = 0;
  b += (double)sizeof(Ctl) + 92.0 * N;                   // state, queues, lists, tags
  b += 2.0 * (24.0 * N + 8.0 * slots);                   // two stores: row, alt, adj
  b += 16.0 * (slots / sp::kChunk + 64.0);               // chunk-owner tables
  const long long c = std::max<long long>(2 * max_updates + 1, 1024);
  const int sblocks = sp::batch_sort_blocks(sms);
  const size_t tmp = std::max({sp::sort_tmp_bytes(c), sp::scan_tmp_bytes(c),
                               sp::batch_sort_tmp_bytes(sblocks)}) + 1024;
  b += (double)c * (8 + 8 + 4 + 4 + 1 + 8 + 4 + sizeof(sp::Seg) + 8) + (double)tmp;
  b += 8.0 * (2.0 * M / 256.0 + 2.0 * (double)max_updates + 64.0);   // merge strips
  b += 20.0 * (double)max_updates;                       // staged host inputs
  *bytes = (int64_t)std::ceil(b) + 64 * 256;             // allocation slack
  return SP_OK;
}

sp_status sp_graph_num_edges(const sp_graph *g, int64_t *m) {
  if (!g || !m) return SP_EINVAL;
  *m = g->m;
  return SP_OK;
}

sp_status sp_export_csr(sp_graph *g, int reverse, int64_t *row_off, int32_t *col, int32_t *w,
                        int out_on_device) {
  if (!g || !row_off || (g->m > 0 && (!col || !w))) return SP_EINVAL;
  int launches = 0;
  const sp::Store *st = reverse ? &g->rev : &g->fwd;
  if (out_on_device) {
    if (!device_out(g, row_off) || (g->m > 0 && (!device_out(g, col) || !device_out(g, w))))
      return SP_EINVAL;
    return sp::store_export(g, st, (long long *)row_off, col, w, &launches);
  }
  const size_t nn = (size_t)g->n, mm = (size_t)std::max<long long>(g->m, 1);
  size_t bytes = (nn + 1) * 8 + 2 * mm * 4 + 512;
  char *buf = (char *)g->al.get(bytes);
  if (!buf) return SP_ENOMEM;
  long long *ro = (long long *)buf;
  int *cc = (int *)(((uintptr_t)(ro + nn + 1) + 255) & ~(uintptr_t)255);
  int *ww = cc + mm;
  sp_status rc = sp::store_export(g, st, ro, cc, ww, &launches);
  if (rc == SP_OK) {
    cudaMemcpyAsync(row_off, ro, (nn + 1) * 8, cudaMemcpyDeviceToHost, g->stream);
    if (g->m > 0) {
      cudaMemcpyAsync(col, cc, (size_t)g->m * 4, cudaMemcpyDeviceToHost, g->stream);
      cudaMemcpyAsync(w, ww, (size_t)g->m * 4, cudaMemcpyDeviceToHost, g->stream);
    }
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) rc = SP_ECUDA;
  }
  g->al.put(buf, bytes);
  return rc;
}

sp_status sp_graph_info_get(const sp_graph *g, sp_graph_info *info) {
  if (!g || !info) return SP_EINVAL;
  info->n = g->n;
  info->source = g->source;
  info->m = g->m;
  info->cap_fwd = g->fwd.slots;
  info->cap_rev = g->rev.slots;
  Ctl c{};
  if (cudaMemcpy(&c, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return SP_ECUDA;
  }
  info->pool_used_fwd = (int64_t)c.pool_used[0];
  info->pool_used_rev = (int64_t)c.pool_used[1];
  info->device_bytes = g->al.bytes_held;
  info->state = g->state;
  info->num_sms = g->num_sms;
  info->pool_step = g->pool_wide ? 5 : 4;
  info->reserved = 0;
  return SP_OK;
}

}  // extern "C"
