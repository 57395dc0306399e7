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
#include <algorithm>

#include "sp_graph.cuh"

namespace sp {

namespace {

constexpr int kWarps = kLoopThreads / 32;
constexpr u64 kMask40 = (1ull << 40) - 1;
constexpr int kOpPush = 0, kOpInval = 1;

struct WarpSmem {
  u32 excl[32];
  u32 v[32];
  u32 d[32];
  long long start[32];
};

__device__ __forceinline__ u32 warp_incl_scan(u32 x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u32 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
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
      while (ld_acquire_u32(&c->bar_gen) == gen) {
        if (ld_cg_i32(&c->timeout) != 0) break;
        if (globaltimer_ns() - t0 > lim.wait_ns) {
          atomicCAS(&c->timeout, 0, 2);
          break;
        }
        __nanosleep(32);
      }
    }
  }
  __syncthreads();
}

// Serial step between rounds (runs in one thread).  `first` is the step
// before round 0, when the producers have filled queue `cur`.
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
  c->light_cnt[cur ^ 1u] = 0;
  c->heavy_cnt[cur ^ 1u] = 0;
  const u32 nl = c->light_cnt[cur];
  const u64 hv = c->heavy_cnt[cur];
  const u32 hc = (u32)(hv & kMask40);
  c->n_heavy = (u32)(hv >> 40);
  c->n_light_groups = (nl + 31) / 32;
  c->work_total = c->n_light_groups + hc;
  c->work_next = 0;
  c->epoch = c->epoch + 1;
  bool done = false;
  if (nl == 0 && hc == 0) {
    done = true;
  } else if (c->round >= lim.max_rounds) {
    c->timeout = 1;
    done = true;
  }
  if (done) {
    c->done = 1;
    if (op == kOpPush) c->rounds_push = c->round;
    else c->rounds_inval = c->round;
    // leave the queues empty for the next producer
    c->cur = 0;
    c->light_cnt[0] = c->light_cnt[1] = 0;
    c->heavy_cnt[0] = c->heavy_cnt[1] = 0;
    c->epoch = c->epoch + 1;
  }
}

// Position of the owner of edge k among the 32 lanes of a group: the last
// lane whose exclusive degree prefix is <= k (lanes with no edges are skipped
// because the next lane has the same prefix).
__device__ __forceinline__ int find_owner(const u32 *excl, u32 k) {
  int o = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1)
    if (o + step < 32 && excl[o + step] <= k) o += step;
  return o;
}

// Append x to the next frontier (warp-collective: every lane calls).  Light
// vertices go to the light queue, 32 per warp later; heavy ones get one queue
// entry plus ceil(deg / kChunk) chunk ids for the next round.
struct Enqueuer {
  Ctl *c;
  u32 *ql;
  int2 *qh;
  u32 *lcnt;
  u64 *hcnt;
  const RowMeta *row;   // forward rows (degree decides light/heavy)
  u32 *alist;           // also append to A (invalidation only)
  u64 n_enq = 0;

  __device__ __forceinline__ void push(bool want, u32 x) {
    const int lane = threadIdx.x & 31;
    int dx = 0;
    if (want) dx = __ldg(&row[x].deg);
    const bool heavy = want && dx > kHeavyDeg;
    const bool light = want && !heavy;
    const u32 lm = __ballot_sync(0xffffffffu, light);
    if (lm) {
      const int leader = __ffs(lm) - 1;
      u32 base = 0;
      if (lane == leader) base = atomicAdd(lcnt, (u32)__popc(lm));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (light) ql[base + __popc(lm & lanemask_lt())] = x;
    }
    if (heavy) {
      const u64 ch = (u64)((dx + kChunk - 1) / kChunk);
      const u64 old = atomicAdd((unsigned long long *)hcnt, (1ull << 40) | ch);
      qh[old >> 40] = make_int2((int)x, (int)(old & kMask40));
    }
    if (alist) {
      const u32 am = __ballot_sync(0xffffffffu, want);
      if (am) {
        const int leader = __ffs(am) - 1;
        u32 base = 0;
        if (lane == leader) base = atomicAdd(&c->a_count, (u32)__popc(am));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (want) alist[base + __popc(am & lanemask_lt())] = x;
      }
    }
    if (want) ++n_enq;
  }
};

// --- edge operations ------------------------------------------------------

// Incremental fixedPoint body: <dist, parent>[x] = <Min(dist[x], dist[v] + w), v>
// as one packed atomicMin; an improved x joins the next frontier once.
struct PushOp {
  u64 *s;
  u32 *qflag;
  u32 tag;
  Enqueuer enq;
  Ctl *c;
  int n;
  u64 n_vert = 0, n_edges = 0, n_imp = 0;
  int range_err = 0;

  __device__ __forceinline__ bool vertex(u32 v, u32 &d) {
    d = dist_of(ld_cg_u64(s + v));
    ++n_vert;
    return d < kInf;
  }
  __device__ __forceinline__ void edge(bool act, u32 v, u32 dv, int x, int w) {
    bool want = false;
    if (act) {
      ++n_edges;
      const u32 nd = dv + (u32)w;
      if (nd >= kInf) {
        range_err = 1;
      } else {
        const u64 cand = pack(nd, v);
        if (cand < ld_cg_u64(s + x)) {
          const u64 old = atomicMin((unsigned long long *)(s + x), cand);
          if (cand < old) {
            ++n_imp;
            want = atomicExch(qflag + x, tag) != tag;
          }
        }
      }
    }
    enq.push(want, (u32)x);
  }
};

// Decremental first loop body: a child x of v (parent[x] == v) loses its
// distance and parent and joins the next frontier and the affected list A.
struct InvalOp {
  u64 *s;
  Enqueuer enq;
  Ctl *c;
  int n;
  u64 n_vert = 0, n_edges = 0;

  __device__ __forceinline__ bool vertex(u32, u32 &d) {
    d = 0;
    ++n_vert;
    return true;
  }
  __device__ __forceinline__ void edge(bool act, u32 v, u32, int x, int) {
    bool hit = false;
    if (act) {
      ++n_edges;
      const u64 sx = ld_cg_u64(s + x);
      if (parent_of(sx) == v) {
        __stcg((unsigned long long *)(s + x), kInfPack);
        hit = true;
      }
    }
    enq.push(hit, (u32)x);
  }
};

// Decremental second loop body, one pass over the reverse store: an
// invalidated v takes min over in-edges x -> v of (dist[x] + w, x).  v joins
// the first push frontier once if it got a finite distance.
struct PullOp {
  u64 *s;
  u32 *qflag;
  u32 tag;
  Enqueuer enq;
  Ctl *c;
  int n;
  int2 *defer_q;       // heavy in-degree rows, chunked by a second kernel
  u64 *defer_cnt;
  u64 n_vert = 0, n_edges = 0;
  int range_err = 0;

  __device__ __forceinline__ bool vertex(u32, u32 &d) {
    d = 0;
    ++n_vert;
    return true;
  }
  __device__ __forceinline__ void defer(u32 v, int deg) {
    const u64 ch = (u64)((deg + kChunk - 1) / kChunk);
    const u64 old = atomicAdd((unsigned long long *)defer_cnt, (1ull << 40) | ch);
    defer_q[old >> 40] = make_int2((int)v, (int)(old & kMask40));
  }
  __device__ __forceinline__ void edge(bool act, u32 v, u32, int x, int w) {
    bool want = false;
    if (act) {
      ++n_edges;
      const u32 dx = dist_of(ld_cg_u64(s + x));
      if (dx < kInf) {
        const u32 nd = dx + (u32)w;
        if (nd >= kInf) {
          range_err = 1;
        } else {
          const u64 cand = pack(nd, (u32)x);
          if (cand < ld_cg_u64(s + v)) {
            const u64 old = atomicMin((unsigned long long *)(s + v), cand);
            if (cand < old) want = atomicExch(qflag + v, tag) != tag;
          }
        }
      }
    }
    enq.push(want, v);
  }
};

// --- frontier expansion ---------------------------------------------------

// One warp expands up to 32 queued vertices: a warp scan of their degrees
// maps the concatenated edge lists onto lanes 32 edges at a time, so rows of
// any length up to kHeavyDeg share the warp without divergence.
template <class Op, bool kDefer>
__device__ __forceinline__ void expand_group(Op &op, const u32 *q, u32 count, u32 group,
                                             const Store &st, WarpSmem &ws) {
  const int lane = threadIdx.x & 31;
  const u32 idx = group * 32 + lane;
  u32 v = 0, dv = 0;
  int deg = 0;
  long long start = 0;
  if (idx < count) {
    v = ld_cg_u32(q + idx);
    if (v >= (u32)op.n) {  // never expected: record and skip
      atomicExch(&op.c->bad, 1);
      v = 0;
    }
    const RowMeta rm = st.row[v];
    if (op.vertex(v, dv)) {
      deg = rm.deg;
      start = rm.start;
    }
    if constexpr (kDefer) {
      if (deg > kHeavyDeg) {
        op.defer(v, deg);
        deg = 0;
      }
    }
  }
  const u32 incl = warp_incl_scan((u32)deg);
  const u32 total = __shfl_sync(0xffffffffu, incl, 31);
  ws.excl[lane] = incl - (u32)deg;
  ws.v[lane] = v;
  ws.d[lane] = dv;
  ws.start[lane] = start;
  __syncwarp();
  for (u32 e = 0; e < total; e += 32) {
    const u32 k = e + lane;
    const bool act = k < total;
    int o = 0;
    int2 ed = make_int2(0, 0);
    if (act) {
      o = find_owner(ws.excl, k);
      ed = __ldg(st.adj + ws.start[o] + (k - ws.excl[o]));
    }
    op.edge(act, ws.v[o], ws.d[o], ed.x, ed.y);
  }
  __syncwarp();
}

// One warp expands chunk `chunk` (kChunk edges) of a heavy queue entry.
template <class Op>
__device__ __forceinline__ void expand_chunk(Op &op, const int2 *hq, u32 nheavy, u32 chunk,
                                             const Store &st) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = (int)nheavy - 1;  // last entry whose first chunk <= chunk
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((u32)__ldcg(&hq[mid].y) <= chunk) lo = mid; else hi = mid - 1;
  }
  const int2 h = __ldcg(hq + lo);
  u32 v = (u32)h.x;
  if (nheavy == 0 || v >= (u32)op.n) {  // never expected: record and skip
    atomicExch(&op.c->bad, 1);
    return;
  }
  const long long e0 = (long long)(chunk - (u32)h.y) * kChunk;
  const RowMeta rm = st.row[v];
  u32 dv = 0;
  long long cnt = 0;
  if (op.vertex(v, dv)) {
    cnt = (long long)rm.deg - e0;
    if (cnt > kChunk) cnt = kChunk;
  }
#pragma unroll 2
  for (int t = 0; t < kChunk; t += 32) {
    const int kk = t + lane;
    const bool act = kk < cnt;
    int2 ed = make_int2(0, 0);
    if (act) ed = __ldg(st.adj + rm.start + e0 + kk);
    op.edge(act, v, dv, ed.x, ed.y);
  }
}

__device__ __forceinline__ bool repair_enabled(Ctl *c) {
  return ld_cg_i32(&c->status) == 0 && ld_cg_i32(&c->need_grow) == 0 &&
         ld_cg_i32(&c->timeout) == 0 && ld_cg_i32(&c->bad) == 0;
}

// --- persistent loop ------------------------------------------------------

template <int OP>
__global__ void __launch_bounds__(kLoopThreads) k_loop(LoopArgs a) {
  __shared__ WarpSmem ws[kWarps];
  Ctl *c = a.ctl;
  if (!repair_enabled(c)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 n_vert = 0, n_edges = 0, n_imp = 0, n_enq = 0;
  int range_err = 0;

  if (OP == kOpInval && a.n_del > 0) {
    // OnDelete: a deleted edge u -> v that is v's parent edge invalidates v.
    Enqueuer enq{c, a.qlight[0], a.qheavy[0], &c->light_cnt[0], &c->heavy_cnt[0], a.fwd.row,
                 a.alist};
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = gw * 32; base < a.n_del; base += nw * 32) {
      const long long i = base + lane;
      bool hit = false;
      u32 v = 0;
      if (i < a.n_del) {
        const u32 u = (u32)a.del_src[i];
        v = (u32)a.del_dst[i];
        const u64 sv = ld_cg_u64(a.s + v);
        if (parent_of(sv) == u)
          hit = atomicCAS((unsigned long long *)(a.s + v), sv, kInfPack) == sv;
      }
      enq.push(hit, v);
    }
    n_enq += enq.n_enq;
  }

  grid_barrier(c, a.lim, [&] { serial_advance(c, a.lim, true, OP); });
  for (;;) {
    if (ld_cg_u32(&c->done) || ld_cg_i32(&c->timeout)) break;
    const u32 cur = ld_cg_u32(&c->cur), nxt = cur ^ 1u;
    const u32 nl = ld_cg_u32(&c->light_cnt[cur]);
    const u32 nlg = ld_cg_u32(&c->n_light_groups);
    const u32 tot = ld_cg_u32(&c->work_total);
    const u32 nh = ld_cg_u32(&c->n_heavy);
    const u32 tag = ld_cg_u32(&c->epoch);
    Enqueuer enq{c, a.qlight[nxt], a.qheavy[nxt], &c->light_cnt[nxt], &c->heavy_cnt[nxt],
                 a.fwd.row, OP == kOpInval ? a.alist : nullptr};
    if (OP == kOpPush) {
      PushOp op{a.s, a.qflag, tag, enq, c, a.n};
      for (;;) {
        u32 item = 0;
        if (lane == 0) item = atomicAdd(&c->work_next, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= tot) break;
        if (item < nlg) expand_group<PushOp, false>(op, a.qlight[cur], nl, item, a.fwd, ws[warp]);
        else expand_chunk(op, a.qheavy[cur], nh, item - nlg, a.fwd);
      }
      n_vert += op.n_vert; n_edges += op.n_edges; n_imp += op.n_imp;
      n_enq += op.enq.n_enq; range_err |= op.range_err;
    } else {
      InvalOp op{a.s, enq, c, a.n};
      for (;;) {
        u32 item = 0;
        if (lane == 0) item = atomicAdd(&c->work_next, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= tot) break;
        if (item < nlg) expand_group<InvalOp, false>(op, a.qlight[cur], nl, item, a.fwd, ws[warp]);
        else expand_chunk(op, a.qheavy[cur], nh, item - nlg, a.fwd);
      }
      n_vert += op.n_vert; n_edges += op.n_edges; n_enq += op.enq.n_enq;
    }
    grid_barrier(c, a.lim, [&] { serial_advance(c, a.lim, false, OP); });
  }
  n_vert = warp_sum(n_vert);
  n_edges = warp_sum(n_edges);
  n_imp = warp_sum(n_imp);
  n_enq = warp_sum(n_enq);
  range_err = __any_sync(0xffffffffu, range_err);
  if (lane == 0) {
    if (OP == kOpPush) {
      if (n_vert) atomicAdd(&c->push_vertices, n_vert);
      if (n_edges) atomicAdd(&c->relaxed, n_edges);
      if (n_imp) atomicAdd(&c->improved, n_imp);
      if (n_enq) atomicAdd(&c->enqueued, n_enq);
    } else {
      if (n_edges) atomicAdd(&c->inval_edges, n_edges);
      if (n_enq) atomicAdd(&c->affected, n_enq);
    }
    if (range_err) atomicExch(&c->range_err, 1);
  }
}

// --- pull (one pass over A) -----------------------------------------------

__global__ void __launch_bounds__(kLoopThreads) k_pull(LoopArgs a) {
  __shared__ WarpSmem ws[kWarps];
  Ctl *c = a.ctl;
  if (!repair_enabled(c)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 na = ld_cg_u32(&c->a_count);
  const u32 groups = (na + 31) / 32;
  const u32 tag = ld_cg_u32(&c->epoch);
  Enqueuer enq{c, a.qlight[0], a.qheavy[0], &c->light_cnt[0], &c->heavy_cnt[0], a.fwd.row,
               nullptr};
  PullOp op{a.s, a.qflag, tag, enq, c, a.n, a.qheavy[1], &c->pull_heavy};
  const u32 gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  for (u32 g = gw; g < groups; g += nw)
    expand_group<PullOp, true>(op, a.alist, na, g, a.rev, ws[warp]);
  u64 e = warp_sum(op.n_edges), q = warp_sum(op.enq.n_enq);
  int re = __any_sync(0xffffffffu, op.range_err);
  if (lane == 0) {
    if (e) atomicAdd(&c->pull_edges, e);
    if (q) atomicAdd(&c->seeds, q);
    if (re) atomicExch(&c->range_err, 1);
  }
}

__global__ void __launch_bounds__(kLoopThreads) k_pull_heavy(LoopArgs a) {
  Ctl *c = a.ctl;
  if (!repair_enabled(c)) return;
  const int lane = threadIdx.x & 31;
  const u64 hv = ld_cg_u64(&c->pull_heavy);
  const u32 nh = (u32)(hv >> 40), chunks = (u32)(hv & kMask40);
  if (chunks == 0) return;
  const u32 tag = ld_cg_u32(&c->epoch);
  Enqueuer enq{c, a.qlight[0], a.qheavy[0], &c->light_cnt[0], &c->heavy_cnt[0], a.fwd.row,
               nullptr};
  PullOp op{a.s, a.qflag, tag, enq, c, a.n, nullptr, nullptr};
  const u32 gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  for (u32 ch = gw; ch < chunks; ch += nw) expand_chunk(op, a.qheavy[1], nh, ch, a.rev);
  u64 e = warp_sum(op.n_edges), q = warp_sum(op.enq.n_enq);
  int re = __any_sync(0xffffffffu, op.range_err);
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
  Enqueuer enq{c, a.la.qlight[0], a.la.qheavy[0], &c->light_cnt[0], &c->heavy_cnt[0],
               a.la.fwd.row, nullptr};
  const u64 cmask = (1ull << a.bits) - 1;
  const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  int range_err = 0;
  for (long long base = gw * 32; base < a.n_items; base += nw * 32) {
    const long long i = base + lane;
    bool want = false;
    u32 v = 0;
    if (i < a.n_items) {
      const u64 key = a.keys[i];
      // forward-store insertion that the merge applied
      if ((key >> (2 * a.bits + 1)) == 0 && (key & 1) && (a.flags[i] & 1)) {
        const u32 u = (u32)((key >> (a.bits + 1)) & cmask);
        v = (u32)((key >> 1) & cmask);
        const u32 du = dist_of(ld_cg_u64(a.la.s + u));
        if (du < kInf) {
          const u32 nd = du + a.vals[i];
          if (nd >= kInf) {
            range_err = 1;
          } else {
            const u64 cand = pack(nd, u);
            if (cand < ld_cg_u64(a.la.s + v)) {
              const u64 old = atomicMin((unsigned long long *)(a.la.s + v), cand);
              if (cand < old) want = atomicExch(a.la.qflag + v, tag) != tag;
            }
          }
        }
      }
    }
    enq.push(want, v);
  }
  u64 q = warp_sum(enq.n_enq);
  int re = __any_sync(0xffffffffu, range_err);
  if (lane == 0) {
    if (q) atomicAdd(&c->seeds, q);
    if (re) atomicExch(&c->range_err, 1);
  }
}

// --- from-scratch init, unpack ----------------------------------------------

__global__ void k_init(u64 *s, int n, int src, Ctl *c, u32 *qflag, u32 *ql, int2 *qh,
                       const RowMeta *row) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    s[v] = v == src ? pack(0, kNoParent) : kInfPack;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const u32 tag = c->epoch;
    qflag[src] = tag;
    const int d = row[src].deg;
    if (d > kHeavyDeg) {
      qh[0] = make_int2(src, 0);
      c->heavy_cnt[0] = (1ull << 40) | (u64)((d + kChunk - 1) / kChunk);
    } else {
      ql[0] = (u32)src;
      c->light_cnt[0] = 1;
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
  a.qlight[0] = g->qlight[0];
  a.qlight[1] = g->qlight[1];
  a.qheavy[0] = g->qheavy[0];
  a.qheavy[1] = g->qheavy[1];
  a.alist = g->alist;
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
      g->s, g->n, source, g->ctl, g->qflag, g->qlight[0], g->qheavy[0], g->fwd.row);
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
  const unsigned grid = (unsigned)std::max(1, g->num_sms * 8);
  k_pull<<<grid, kLoopThreads, 0, g->stream>>>(a);
  k_pull_heavy<<<grid, kLoopThreads, 0, g->stream>>>(a);
  *launches += 2;
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
  blocks = std::min<long long>(std::max<long long>(blocks, 1), g->num_sms * 16);
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
