// sp_frontier.cu -- distance repair on the device.
//
// The paper's Incremental and Decremental functions (Section 3.3 and the
// Appendix SSSP listings) sweep every vertex each iteration with a
// `modified` filter and copy a `finished` flag to the host per iteration
// (Section 5.3).  Here the same fixed points run over explicit frontier
// queues inside one cooperative launch per loop:
//   * invalidation (Decremental, first loop): the OnDelete mark seeds the
//     queue with vertices whose parent edge was deleted; each round walks the
//     out-edges of the frontier and takes every child whose parent is the
//     frontier vertex, setting it to INF / parent -1;
//   * pull (Decremental, second loop, one pass): every invalidated vertex
//     takes the minimum over its in-edges of dist[x] + w;
//   * OnAdd: every inserted edge is relaxed directly;
//   * push (Incremental fixedPoint): rounds of Min relaxations over the
//     out-edges of the frontier until no distance changes.
// Rounds are separated by a grid barrier whose waits are bounded; the round
// count is capped (Bellman-Ford bound n + 1 by default).
//
// Work balance: a vertex entering a frontier reserves a contiguous range of
// that frontier's edge space (one packed 64-bit atomic per warp), and the
// round is processed as chunks of kChunk edges, one warp per chunk and
// kEdgesPerLane consecutive edges per lane, so a 40,000-edge hub and a
// 2-edge vertex cost the same per edge.  Each lane issues the loads of all
// its edges before it uses any of them.
#include <algorithm>

#include "sp_graph.cuh"

namespace sp {

namespace {

constexpr int kOpPush = 0, kOpInval = 1;
constexpr int K = kEdgesPerLane;
constexpr u32 kNoEdge = 0xFFFFFFFFu;
constexpr u32 kFull = 0xffffffffu;

__device__ __forceinline__ u32 warp_incl_scan(u32 x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u32 y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ u64 shfl64(u64 x, int src) {
  u32 lo = __shfl_sync(kFull, (u32)x, src), hi = __shfl_sync(kFull, (u32)(x >> 32), src);
  return ((u64)hi << 32) | lo;
}
__device__ __forceinline__ u64 shfl64_down(u64 x, int d) {
  u32 lo = __shfl_down_sync(kFull, (u32)x, d), hi = __shfl_down_sync(kFull, (u32)(x >> 32), d);
  return ((u64)hi << 32) | lo;
}

// Grid barrier: the last block to arrive runs `hook` (thread 0 only), then
// releases the others.  Every wait is bounded by lim.wait_ns; a wait that runs
// out sets ctl->timeout = 2 and returns, and every later wait returns at once.
template <class Hook>
__device__ __forceinline__ void grid_barrier(Ctl *c, const Limits &lim, Hook hook) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const u32 gen = ld_acquire_u32(&c->bar_gen);
    __threadfence();
    const u32 arrived = atomicAdd(&c->bar_arrive, 1u);
    if (arrived == gridDim.x - 1) {
      __threadfence();
      atomicExch(&c->bar_arrive, 0u);
      hook();
      __threadfence();
      st_release_u32(&c->bar_gen, gen + 1);
    } else {
      const u64 t0 = globaltimer_ns();
      u32 nap = 20;
      while (ld_acquire_u32(&c->bar_gen) == gen) {
        if (ld_cg_i32(&c->timeout) != 0) break;
        if (globaltimer_ns() - t0 > lim.wait_ns) {
          atomicCAS(&c->timeout, 0, 2);
          break;
        }
        __nanosleep(nap);
        if (nap < 320) nap += nap >> 1;
      }
    }
  }
  __syncthreads();
}

__device__ __forceinline__ volatile u64 *qcnt_of(volatile Ctl *c, u32 b) {
  return b ? &c->qcnt1 : &c->qcnt0;
}

// Serial step between rounds (runs in one thread).  `first` is the step
// before round 0, when the producers have filled frontier buffer `cur`.
__device__ void serial_advance(Ctl *cc, const Limits &lim, bool first, int op) {
  volatile Ctl *c = cc;
  u32 cur = c->cur;
  if (first) {
    c->round = 0;
    c->done = 0;
  } else {
    cur ^= 1u;
    c->cur = cur;
    c->round = c->round + 1;
  }
  *qcnt_of(c, cur ^ 1u) = 0ull;          // the buffer this round fills
  const u64 q = *qcnt_of(c, cur);
  const u32 ne = (u32)(q >> 32), edges = (u32)q;
  c->n_ent = ne;
  c->n_edges = edges;
  c->n_chunks = (edges + kChunk - 1) / kChunk;
  c->epoch = c->epoch + 1;
  bool done = false;
  if (edges == 0) {
    done = true;
  } else if (c->round >= lim.max_rounds) {
    c->timeout = 1;
    done = true;
  }
  if (done) {
    c->done = 1;
    if (op == kOpPush) c->rounds_push = c->round;
    else c->rounds_inval = c->round;
    c->cur = 0;                          // leave the frontier empty
    c->qcnt0 = 0ull;
    c->qcnt1 = 0ull;
    c->epoch = c->epoch + 1;
  }
}

// Append up to K vertices per lane to queue q (warp-collective).  Each kept
// vertex (want and degree > 0 in `row`) reserves deg slots of the queue's
// edge space; the chunk-owner table gets its slot for every chunk whose first
// edge falls in that range.
__device__ __forceinline__ void enqueue(const Queue &q, const RowMeta *row, const u32 *x,
                                        const bool *want, int kk, u64 &n_enq) {
  const int lane = threadIdx.x & 31;
  int d[K];
  u32 cnt = 0, sum = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    d[k] = (k < kk && want[k]) ? __ldg(&row[x[k]].deg) : 0;
    if (d[k] > 0) {
      ++cnt;
      sum += (u32)d[k];
    }
  }
  if (!__ballot_sync(kFull, cnt > 0)) return;
  const u32 ci = warp_incl_scan(cnt), si = warp_incl_scan(sum);
  const u32 ctot = __shfl_sync(kFull, ci, 31), stot = __shfl_sync(kFull, si, 31);
  u64 base = 0;
  if (lane == 0) base = atomicAdd(q.cnt, ((u64)ctot << 32) | (u64)stot);
  base = shfl64(base, 0);
  u32 slot = (u32)(base >> 32) + ci - cnt;
  u32 eb = (u32)base + si - sum;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (d[k] > 0) {
      q.ent[slot] = make_int2((int)x[k], (int)eb);
      const u32 c0 = (eb + kChunk - 1) / kChunk, c1 = (eb + (u32)d[k] - 1) / kChunk;
      for (u32 ch = c0; ch <= c1; ++ch) q.owner[ch] = slot;
      ++slot;
      eb += (u32)d[k];
    }
  }
  n_enq += cnt;
}

// --- edge operations ------------------------------------------------------
//
// Each op provides vdata(v) (a per-source datum read once per queue entry),
// load(e) (the state word an edge needs) and run(...) (the updates of one
// lane's edges followed by the warp-collective enqueue of what they queue).

// Incremental fixedPoint body: <dist, parent>[x] = <Min(dist[x], dist[v] + w), v>
// as one packed atomicMin; an improved x joins the next frontier once.
struct PushOp {
  u64 *s;
  u32 *qflag;
  u32 tag;
  Queue next;
  const RowMeta *row;
  u64 n_edges = 0, n_imp = 0, n_enq = 0;
  int range_err = 0;

  __device__ __forceinline__ u32 vdata(u32 v) { return dist_of(ld_cg_u64(s + v)); }
  __device__ __forceinline__ u64 load(int2 e) { return ld_cg_u64(s + e.x); }
  __device__ __forceinline__ void run(const bool *act, const u32 *ov, const u32 *od,
                                      const int2 *ed, const u64 *sx) {
    u32 tx[K];
    bool want[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      want[k] = false;
      tx[k] = (u32)ed[k].x;
      if (act[k]) {
        ++n_edges;
        if (od[k] < kInf) {
          const u32 nd = od[k] + (u32)ed[k].y;
          if (nd >= kInf) {
            range_err = 1;
          } else {
            const u64 cand = pack(nd, ov[k]);
            if (cand < sx[k]) {
              const u64 old = atomicMin((unsigned long long *)(s + ed[k].x), cand);
              if (cand < old) {
                ++n_imp;
                want[k] = atomicExch(qflag + ed[k].x, tag) != tag;
              }
            }
          }
        }
      }
    }
    enqueue(next, row, tx, want, K, n_enq);
  }
};

// Decremental first loop body: a child x of v (parent[x] == v) loses its
// distance and parent, joins the next frontier (its out-edges) and the
// affected list A (its in-edges, for the pull).
struct InvalOp {
  u64 *s;
  Queue next, alist;
  const RowMeta *row, *rrow;
  u64 n_edges = 0, n_enq = 0, n_aff = 0;
  int range_err = 0;

  __device__ __forceinline__ u32 vdata(u32) { return 0; }
  __device__ __forceinline__ u64 load(int2 e) { return ld_cg_u64(s + e.x); }
  __device__ __forceinline__ void run(const bool *act, const u32 *ov, const u32 *,
                                      const int2 *ed, const u64 *sx) {
    u32 tx[K];
    bool want[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      tx[k] = (u32)ed[k].x;
      want[k] = act[k] && parent_of(sx[k]) == ov[k];
      if (act[k]) ++n_edges;
      if (want[k]) {
        __stcg((unsigned long long *)(s + ed[k].x), kInfPack);
        ++n_aff;
      }
    }
    enqueue(next, row, tx, want, K, n_enq);
    u64 dummy = 0;
    enqueue(alist, rrow, tx, want, K, dummy);
  }
};

// Decremental second loop body, one pass over the reverse store: an
// invalidated v takes min over in-edges x -> v of (dist[x] + w, x).  The
// minimum is formed per lane and then per warp before one atomicMin per
// (warp, vertex); v joins the first push frontier once if it improved.
struct PullOp {
  u64 *s;
  u32 *qflag;
  u32 tag;
  Queue next;
  const RowMeta *row;
  u64 n_edges = 0, n_enq = 0;
  int range_err = 0;

  __device__ __forceinline__ u32 vdata(u32) { return 0; }
  __device__ __forceinline__ u64 load(int2 e) { return ld_cg_u64(s + e.x); }
  __device__ __forceinline__ bool offer(u32 v, u64 best) {
    if (best == ~0ull || best >= ld_cg_u64(s + v)) return false;
    const u64 old = atomicMin((unsigned long long *)(s + v), best);
    return best < old && atomicExch(qflag + v, tag) != tag;
  }
  __device__ __forceinline__ void run(const bool *act, const u32 *ov, const u32 *,
                                      const int2 *ed, const u64 *sx) {
    const int lane = threadIdx.x & 31;
    u32 tx[K];
    bool want[K];
    int nw = 0;
    u32 bv = kNoEdge;
    u64 best = ~0ull;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      want[k] = false;
      tx[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (act[k]) {
        ++n_edges;
        u64 cand = ~0ull;
        const u32 dx = dist_of(sx[k]);
        if (dx < kInf) {
          const u32 nd = dx + (u32)ed[k].y;
          if (nd >= kInf) range_err = 1;
          else cand = pack(nd, (u32)ed[k].x);
        }
        if (ov[k] != bv) {           // owner changed inside this lane's run
          if (bv != kNoEdge && offer(bv, best)) {
            tx[nw] = bv;
            want[nw] = true;
            ++nw;
          }
          bv = ov[k];
          best = ~0ull;
        }
        if (cand < best) best = cand;
      }
    }
    // segmented minimum over the lanes that end on the same vertex
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = shfl64_down(best, o);
      const u32 yv = __shfl_down_sync(kFull, bv, o);
      if (lane + o < 32 && yv == bv && y < best) best = y;
    }
    const u32 pv = __shfl_up_sync(kFull, bv, 1);
    const bool head = bv != kNoEdge && (lane == 0 || pv != bv);
    if (head && nw < K && offer(bv, best)) {
      tx[nw] = bv;
      want[nw] = true;
      ++nw;
    }
    enqueue(next, row, tx, want, K, n_enq);
  }
};

// --- chunk expansion --------------------------------------------------------

// Expand edge chunk `chunk` of a frontier (ent/own, n_ent entries, n_edges
// edges) over store `st`: lane L takes edges [e0 + K*L, e0 + K*L + K).
template <class Op>
__device__ __forceinline__ void process_chunk(Op &op, const int2 *ent, const u32 *own, u32 n_ent,
                                              u32 n_edges, u32 chunk, const Store &st, int n,
                                              Ctl *c) {
  const int lane = threadIdx.x & 31;
  const u32 e0 = chunk * kChunk;
  const u32 e_end = e0 + kChunk < n_edges ? e0 + kChunk : n_edges;
  const u32 jw = __ldcg(own + chunk);
  // window: the 32 entries from the one holding e0
  const u32 wj = jw + lane;
  u32 wv = 0, web = kNoEdge, wdeg = 0, wd = 0;
  long long wstart = 0;
  if (wj < n_ent) {
    const int2 en = __ldcg(ent + wj);
    wv = (u32)en.x;
    web = (u32)en.y;
    if (wv < (u32)n) {
      const RowMeta rm = st.row[wv];
      wdeg = (u32)rm.deg;
      wstart = rm.start;
      wd = op.vdata(wv);
    } else {                             // never expected: record and skip
      atomicExch(&c->bad, 1);
      wv = 0;
      web = kNoEdge;
    }
  }
  const u32 l31 = __shfl_sync(kFull, web == kNoEdge ? kNoEdge : web + wdeg, 31);
  const u32 wend = l31 == kNoEdge ? n_edges : l31;
  const u32 ebeg = e0 + (u32)(K * lane);
  // owner of ebeg inside the window: last lane whose first edge <= ebeg
  int o = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const u32 ebc = __shfl_sync(kFull, web, (o + step) & 31);
    if (o + step < 32 && ebc <= ebeg) o += step;
  }
  u32 slot = jw + (u32)o;
  u32 v = __shfl_sync(kFull, wv, o), eb = __shfl_sync(kFull, web, o);
  u32 deg = __shfl_sync(kFull, wdeg, o), dv = __shfl_sync(kFull, wd, o);
  long long start = (long long)shfl64((u64)wstart, o);
  if (ebeg < e_end && ebeg >= wend) {
    // beyond the window (many tiny rows in one chunk): search the queue
    u32 lo = jw, hi = n_ent - 1;
    while (lo < hi) {
      const u32 mid = (lo + hi + 1) >> 1;
      if ((u32)__ldcg(&ent[mid].y) <= ebeg) lo = mid; else hi = mid - 1;
    }
    slot = lo;
    const int2 en = __ldcg(ent + slot);
    v = (u32)en.x;
    eb = (u32)en.y;
    const RowMeta rm = st.row[v];
    deg = (u32)rm.deg;
    start = rm.start;
    dv = op.vdata(v);
    o = 32;
  }
  bool act[K];
  u32 ov[K], od[K];
  int2 ed[K];
  u64 sx[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const u32 e = ebeg + (u32)k;
    act[k] = e < e_end;
    const int nl = (o + 1) & 31;
    const u32 nv = __shfl_sync(kFull, wv, nl), neb = __shfl_sync(kFull, web, nl);
    const u32 ndeg = __shfl_sync(kFull, wdeg, nl), nd = __shfl_sync(kFull, wd, nl);
    const long long nstart = (long long)shfl64((u64)wstart, nl);
    if (act[k] && e >= eb + deg) {  // next entry (entries are contiguous in edge space)
      ++slot;
      if (o + 1 < 32) {
        ++o;
        v = nv; eb = neb; deg = ndeg; dv = nd; start = nstart;
      } else {
        const int2 en = __ldcg(ent + slot);
        v = (u32)en.x;
        eb = (u32)en.y;
        const RowMeta rm = st.row[v];
        deg = (u32)rm.deg;
        start = rm.start;
        dv = op.vdata(v);
        o = 32;
      }
    }
    ov[k] = v;
    od[k] = dv;
    ed[k] = act[k] ? __ldg(st.adj + start + (e - eb)) : make_int2(0, 0);
  }
#pragma unroll
  for (int k = 0; k < K; ++k) sx[k] = act[k] ? op.load(ed[k]) : 0ull;
  op.run(act, ov, od, ed, sx);
}

__device__ __forceinline__ bool repair_enabled(Ctl *c) {
  return ld_cg_i32(&c->status) == 0 && ld_cg_i32(&c->need_grow) == 0 &&
         ld_cg_i32(&c->timeout) == 0 && ld_cg_i32(&c->bad) == 0;
}

__device__ __forceinline__ Queue make_queue(int2 *ent, u32 *own, u64 *cnt) {
  Queue q;
  q.ent = ent;
  q.owner = own;
  q.cnt = (unsigned long long *)cnt;
  return q;
}

// --- persistent loop ------------------------------------------------------

template <int OP>
__global__ void __launch_bounds__(kLoopThreads, 2) k_loop(LoopArgs a) {
  Ctl *c = a.ctl;
  if (!repair_enabled(c)) return;
  const int lane = threadIdx.x & 31;
  const u32 gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  u64 n_edges = 0, n_imp = 0, n_enq = 0, n_aff = 0;
  int range_err = 0;

  if (OP == kOpInval && a.n_del > 0) {
    // OnDelete: a deleted edge u -> v that is v's parent edge invalidates v.
    const Queue q0 = make_queue(a.qent[0], a.qown[0], &c->qcnt0);
    const Queue qa = make_queue(a.aent, a.aown, &c->acnt);
    for (long long base = (long long)gw * 32; base < a.n_del; base += (long long)nw * 32) {
      const long long i = base + lane;
      bool hit[K] = {};
      u32 v[K] = {};
      if (i < a.n_del) {
        const u32 u = (u32)a.del_src[i];
        v[0] = (u32)a.del_dst[i];
        const u64 sv = ld_cg_u64(a.s + v[0]);
        if (parent_of(sv) == u)
          hit[0] = atomicCAS((unsigned long long *)(a.s + v[0]), sv, kInfPack) == sv;
      }
      n_aff += hit[0];
      enqueue(q0, a.fwd.row, v, hit, 1, n_enq);
      u64 dummy = 0;
      enqueue(qa, a.rev.row, v, hit, 1, dummy);
    }
  }

  grid_barrier(c, a.lim, [&] { serial_advance(c, a.lim, true, OP); });
  for (;;) {
    if (ld_cg_u32(&c->done) || ld_cg_i32(&c->timeout)) break;
    const u32 cur = ld_cg_u32(&c->cur), nxt = cur ^ 1u;
    const u32 ne = ld_cg_u32(&c->n_ent), nedge = ld_cg_u32(&c->n_edges);
    const u32 nch = ld_cg_u32(&c->n_chunks);
    const u32 tag = ld_cg_u32(&c->epoch);
    const Queue qn = make_queue(a.qent[nxt], a.qown[nxt], nxt ? &c->qcnt1 : &c->qcnt0);
    if (OP == kOpPush) {
      PushOp op{a.s, a.qflag, tag, qn, a.fwd.row};
      for (u32 ch = gw; ch < nch; ch += nw)
        process_chunk(op, a.qent[cur], a.qown[cur], ne, nedge, ch, a.fwd, a.n, c);
      n_edges += op.n_edges;
      n_imp += op.n_imp;
      n_enq += op.n_enq;
      range_err |= op.range_err;
    } else {
      InvalOp op{a.s, qn, make_queue(a.aent, a.aown, &c->acnt), a.fwd.row, a.rev.row};
      for (u32 ch = gw; ch < nch; ch += nw)
        process_chunk(op, a.qent[cur], a.qown[cur], ne, nedge, ch, a.fwd, a.n, c);
      n_edges += op.n_edges;
      n_enq += op.n_enq;
      n_aff += op.n_aff;
    }
    grid_barrier(c, a.lim, [&] { serial_advance(c, a.lim, false, OP); });
  }
  n_edges = warp_sum(n_edges);
  n_imp = warp_sum(n_imp);
  n_enq = warp_sum(n_enq);
  n_aff = warp_sum(n_aff);
  range_err = __any_sync(kFull, range_err);
  if (lane == 0) {
    if (OP == kOpPush) {
      if (n_edges) atomicAdd(&c->relaxed, n_edges);
      if (n_imp) atomicAdd(&c->improved, n_imp);
      if (n_enq) atomicAdd(&c->enqueued, n_enq);
    } else {
      if (n_edges) atomicAdd(&c->inval_edges, n_edges);
      if (n_aff) atomicAdd(&c->affected, n_aff);
    }
    if (range_err) atomicExch(&c->range_err, 1);
  }
}

// --- pull (one pass over A) -----------------------------------------------

__global__ void __launch_bounds__(kLoopThreads) k_pull(LoopArgs a) {
  Ctl *c = a.ctl;
  if (!repair_enabled(c)) return;
  const int lane = threadIdx.x & 31;
  const u64 ac = ld_cg_u64(&c->acnt);
  const u32 ne = (u32)(ac >> 32), nedge = (u32)ac;
  const u32 nch = (nedge + kChunk - 1) / kChunk;
  const u32 tag = ld_cg_u32(&c->epoch);
  PullOp op{a.s, a.qflag, tag, make_queue(a.qent[0], a.qown[0], &c->qcnt0), a.fwd.row};
  const u32 gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  for (u32 ch = gw; ch < nch; ch += nw)
    process_chunk(op, a.aent, a.aown, ne, nedge, ch, a.rev, a.n, c);
  u64 e = warp_sum(op.n_edges), q = warp_sum(op.n_enq);
  int re = __any_sync(kFull, op.range_err);
  if (lane == 0) {
    if (e) atomicAdd(&c->pull_edges, e);
    if (q) atomicAdd(&c->seeds, q);
    if (re) atomicExch(&c->range_err, 1);
  }
}

// --- OnAdd: relax every applied insertion ---------------------------------

struct AddArgs {
  LoopArgs la;
  const u64 *keys;
  const u32 *vals;
  const unsigned char *flags;
  long long n_items;
  int bits;
};

__global__ void __launch_bounds__(kLoopThreads) k_add(AddArgs a) {
  Ctl *c = a.la.ctl;
  if (!repair_enabled(c)) return;
  const int lane = threadIdx.x & 31;
  const u32 tag = ld_cg_u32(&c->epoch);
  const Queue q0 = make_queue(a.la.qent[0], a.la.qown[0], &c->qcnt0);
  const u64 cmask = (1ull << a.bits) - 1;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  int range_err = 0;
  u64 n_enq = 0;
  for (long long base = gw * 32; base < a.n_items; base += nw * 32) {
    const long long i = base + lane;
    bool want[K] = {};
    u32 v[K] = {};
    if (i < a.n_items) {
      const u64 key = a.keys[i];
      // forward-store insertion that the merge applied
      if ((key >> (2 * a.bits + 1)) == 0 && (key & 1) && (a.flags[i] & 1)) {
        const u32 u = (u32)((key >> (a.bits + 1)) & cmask);
        v[0] = (u32)((key >> 1) & cmask);
        const u32 du = dist_of(ld_cg_u64(a.la.s + u));
        if (du < kInf) {
          const u32 nd = du + a.vals[i];
          if (nd >= kInf) {
            range_err = 1;
          } else {
            const u64 cand = pack(nd, u);
            if (cand < ld_cg_u64(a.la.s + v[0])) {
              const u64 old = atomicMin((unsigned long long *)(a.la.s + v[0]), cand);
              if (cand < old) want[0] = atomicExch(a.la.qflag + v[0], tag) != tag;
            }
          }
        }
      }
    }
    enqueue(q0, a.la.fwd.row, v, want, 1, n_enq);
  }
  u64 q = warp_sum(n_enq);
  int re = __any_sync(kFull, range_err);
  if (lane == 0) {
    if (q) atomicAdd(&c->seeds, q);
    if (re) atomicExch(&c->range_err, 1);
  }
}

// --- from-scratch init, unpack ----------------------------------------------

__global__ void k_init(u64 *s, int n, int src, Ctl *c, u32 *qflag, int2 *qent, u32 *qown,
                       const RowMeta *row) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    s[v] = v == src ? pack(0, kNoParent) : kInfPack;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    qflag[src] = c->epoch;
    const int d = row[src].deg;
    if (d > 0) {
      qent[0] = make_int2(src, 0);
      for (u32 ch = 0; ch <= (u32)(d - 1) / kChunk; ++ch) qown[ch] = 0;
      c->qcnt0 = (1ull << 32) | (u64)d;
    }
    c->seeds = 1;
  }
}

__global__ void k_unpack(const u64 *__restrict__ s, int n, int *dist, int *parent) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const u64 x = s[v];
    dist[v] = (int)dist_of(x);
    if (parent) parent[v] = (int)parent_of(x);
  }
}

LoopArgs make_args(sp_graph *g) {
  LoopArgs a;
  a.ctl = g->ctl;
  a.lim = g->lim;
  a.fwd = g->fwd;
  a.rev = g->rev;
  a.s = g->s;
  a.qflag = g->qflag;
  a.qent[0] = g->qent[0];
  a.qent[1] = g->qent[1];
  a.qown[0] = g->qown[0];
  a.qown[1] = g->qown[1];
  a.aent = g->aent;
  a.aown = g->aown;
  a.n = g->n;
  a.del_src = nullptr;
  a.del_dst = nullptr;
  a.n_del = 0;
  return a;
}

}  // namespace

int loop_blocks(int which, int num_sms) {
  int per_sm = 0;
  const void *fn = which == kOpPush ? (const void *)k_loop<kOpPush> : (const void *)k_loop<kOpInval>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kLoopThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return 0;
  return per_sm * num_sms;
}

void launch_init(sp_graph *g, int source, int *launches) {
  k_init<<<(unsigned)std::max(1, g->num_sms * 8), 256, 0, g->stream>>>(
      g->s, g->n, source, g->ctl, g->qflag, g->qent[0], g->qown[0], g->fwd.row);
  ++*launches;
}

static cudaError_t launch_loop(sp_graph *g, int op, LoopArgs &a, int *launches) {
  int blocks = op == kOpPush ? g->loop_blocks_push : g->loop_blocks_inval;
  void *args[] = {&a};
  const void *fn = op == kOpPush ? (const void *)k_loop<kOpPush> : (const void *)k_loop<kOpInval>;
  ++*launches;
  return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kLoopThreads), args, 0, g->stream);
}

cudaError_t launch_inval(sp_graph *g, const int *ds, const int *dd, long long nd, int *launches) {
  LoopArgs a = make_args(g);
  a.del_src = ds;
  a.del_dst = dd;
  a.n_del = nd;
  return launch_loop(g, kOpInval, a, launches);
}

void launch_pull(sp_graph *g, int *launches) {
  LoopArgs a = make_args(g);
  k_pull<<<(unsigned)std::max(1, g->num_sms * 4), kLoopThreads, 0, g->stream>>>(a);
  ++*launches;
}

void launch_add(sp_graph *g, long long n_items, int *launches) {
  if (n_items == 0) return;
  AddArgs a;
  a.la = make_args(g);
  a.keys = g->bb.keys;
  a.vals = g->bb.vals;
  a.flags = g->bb.flags;
  a.n_items = n_items;
  a.bits = g->bits;
  long long blocks = (n_items + kLoopThreads - 1) / kLoopThreads;
  blocks = std::min<long long>(std::max<long long>(blocks, 1), g->num_sms * 8);
  k_add<<<(unsigned)blocks, kLoopThreads, 0, g->stream>>>(a);
  ++*launches;
}

cudaError_t launch_push(sp_graph *g, int *launches) {
  LoopArgs a = make_args(g);
  return launch_loop(g, kOpPush, a, launches);
}

void launch_unpack(sp_graph *g, int *dist_d, int *parent_d, int *launches) {
  k_unpack<<<(unsigned)std::max(1, g->num_sms * 8), 256, 0, g->stream>>>(g->s, g->n, dist_d,
                                                                        parent_d);
  ++*launches;
}

}  // namespace sp
