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

// kOpPool: the push fixedPoint with block-local relaxation (pool schedule)
constexpr int kOpPush = 0, kOpInval = 1, kOpFlag = 2, kOpPool = 3, kOpPoolWide = 4;
// the two pool kernels differ only in the edges a lane relaxes per step
__host__ __device__ constexpr bool is_pool(int op) { return op == kOpPool || op == kOpPoolWide; }
constexpr int K = kEdgesPerLane;
// block stages of the persistent loops (dynamic shared memory)
constexpr u32 kStageQ = 4096, kStageQS = 12288, kStageA = 2048, kStageAS = 4096, kStageF = 4096;
constexpr size_t kLoopSmem =
    (2 * kStageQ + kStageQS + 2 * kStageA + kStageAS + kStageF) * sizeof(u32);
// the pool schedule's two entry lists follow the stages
constexpr size_t kLoopSmemPool = kLoopSmem + 2 * kPoolCap * sizeof(uint4);
constexpr u32 kStageK = 1024;    // stages of the one-pass kernels (static)
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

// Grid barrier over a monotone arrival count: barrier k of a launch waits
// for k * gridDim.x arrivals (the count is zeroed at the start of every
// call).  Every wait is bounded by lim.wait_ns; a wait that runs out sets
// ctl->timeout = 2 and returns, and every later wait returns at once.
__device__ __forceinline__ u64 ld_acquire_u64(const u64 *p) {
  u64 v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

//
// Returns whether a timeout has been raised (the same answer in every thread
// of the block, so that loops leave in step and no __syncthreads is left
// waiting for threads that have gone).
// With `src`, thread 0 also reads the next round's frontier counters once
// the wait is over and hands them to the block in *out: one read per block
// instead of one per warp, all of them at the same line.
struct RoundCounts {
  u64 q;        // next frontier: entries << 32 | edges
  u32 ns;       // its small list
  u32 nf, fm;   // far pile: count and smallest distance (0, ~0 without one)
};
struct CountSrc {
  const u64 *q;
  const u32 *ns, *nf, *fm;   // nf, fm null without a far pile
};

__device__ __forceinline__ bool grid_sync(u64 *bar, u64 target, Ctl *c, const Limits &lim,
                                          const CountSrc *src = nullptr,
                                          RoundCounts *out = nullptr) {
  __shared__ int s_stop;
  __shared__ RoundCounts s_rc;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    // the count before this arrival says whether it was the last one; the
    // wait polls the count alone and looks at the timeout flag and the
    // clock every 16th poll
    // (the test hook lim.miss_site == 2: block 0 does not arrive)
    const bool miss = lim.miss_site == 2u && blockIdx.x == 0;
    const u64 arrived = miss ? ld_acquire_u64(bar) : atomicAdd((unsigned long long *)bar, 1ull) + 1;
    if (arrived < target) {
      const u64 t0 = globaltimer_ns();
      u32 polls = 0;
      while (ld_acquire_u64(bar) < target) {
        if ((++polls & 15u) == 0) {
          if (ld_cg_i32(&c->timeout) != 0) break;
          if (globaltimer_ns() - t0 > lim.wait_ns || polls > kMaxPolls) {
            raise_timeout(c, 2, 2, (u32)(target / gridDim.x));
            break;
          }
        }
        __nanosleep(64);
      }
    }
    s_stop = ld_cg_i32(&c->timeout) != 0;
    if (src) {
      s_rc.q = ld_cg_u64(src->q);
      s_rc.ns = ld_cg_u32(src->ns);
      s_rc.nf = src->nf ? ld_cg_u32(src->nf) : 0u;
      s_rc.fm = src->fm ? ld_cg_u32(src->fm) : 0xFFFFFFFFu;
    }
  }
  __syncthreads();
  if (src) *out = s_rc;
  return s_stop != 0;
}

__device__ __forceinline__ u64 *qcnt_ptr(Ctl *c, u32 b) {
  return b == 0 ? &c->qcnt0 : (b == 1 ? &c->qcnt1 : &c->qcnt2);
}
__device__ __forceinline__ u32 *fcnt_ptr(Ctl *c, u32 b) {
  return b == 0 ? &c->fcnt0 : (b == 1 ? &c->fcnt1 : &c->fcnt2);
}
__device__ __forceinline__ u32 *fmin_ptr(Ctl *c, u32 b) {
  return b == 0 ? &c->fmin0 : (b == 1 ? &c->fmin1 : &c->fmin2);
}
__device__ __forceinline__ u32 *jcnt_ptr(Ctl *c, u32 b) {
  return b == 0 ? &c->jcnt0 : (b == 1 ? &c->jcnt1 : &c->jcnt2);
}
__device__ __forceinline__ u32 next3(u32 b) { return b == 2 ? 0u : b + 1u; }

// Pointer-jumping words: an ancestor id (< n), or one of two final states.
constexpr u32 kJumpCut = 0xFFFFFFFFu;    // a cut vertex lies on the path
constexpr u32 kJumpRoot = 0xFFFFFFFEu;   // the path reached the root uncut
constexpr u32 kMaxJumps = 40;            // > log2 of any tree depth

__device__ __forceinline__ u32 sat_add(u32 a, u32 b) {
  const u64 x = (u64)a + b;
  return x > 0xFFFFFFFFull ? 0xFFFFFFFFu : (u32)x;
}

// Reserve `cnt` slots of a block stage (lane 0 only); false if it is full.
__device__ __forceinline__ bool stage_reserve(Stage *st, u32 cnt, u32 &pos) {
  u32 old = *(volatile u32 *)&st->n;
  while (old + cnt <= st->cap) {
    const u32 prev = atomicCAS(&st->n, old, old + cnt);
    if (prev == old) {
      pos = old;
      return true;
    }
    old = prev;
  }
  return false;
}

// Append up to K vertices per lane to queue q (warp-collective), given
// their out-degrees (0: not appended).  A vertex with 1..q.small edges goes
// to the small list; a larger one reserves deg slots of the queue's edge
// space, and the chunk-owner table gets its slot for every chunk whose first
// edge falls in that range.  With block stages the vertices wait there and
// are published when the block flushes.
__device__ __forceinline__ void enqueue_d(const Queue &q, const u32 *x, const int *dk, int kk,
                                          u64 &n_enq) {
  const int lane = threadIdx.x & 31;
  int d[K];
  u32 cnt = 0, sum = 0, scount = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    d[k] = k < kk ? dk[k] : 0;
    if (d[k] > (int)q.small) {
      ++cnt;
      sum += (u32)d[k];
    } else if (d[k] > 0) {
      ++scount;
    }
  }
  const u32 any = __ballot_sync(kFull, cnt > 0), sany = __ballot_sync(kFull, scount > 0);
  if (!any && !sany) return;
  n_enq += cnt + scount;
  if (sany) {   // small list
    const u32 si = warp_incl_scan(scount), stot = __shfl_sync(kFull, si, 31);
    u32 pos = 0;
    bool ok = false;
    if (lane == 0) ok = q.sst && stage_reserve(q.sst, stot, pos);
    ok = __shfl_sync(kFull, ok, 0);
    u32 *dst;
    if (ok) {
      dst = q.sst->v;
    } else {
      if (lane == 0) pos = atomicAdd(q.scnt, stot);
      dst = q.sv;
    }
    u32 p = __shfl_sync(kFull, pos, 0) + si - scount;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (d[k] > 0 && d[k] <= (int)q.small) dst[p++] = x[k];
  }
  if (!any) return;
  const u32 ci = warp_incl_scan(cnt), si = warp_incl_scan(sum);
  const u32 ctot = __shfl_sync(kFull, ci, 31), stot = __shfl_sync(kFull, si, 31);
  if (q.st) {
    u32 pos = 0;
    bool ok = false;
    if (lane == 0) ok = stage_reserve(q.st, ctot, pos);
    if (__shfl_sync(kFull, ok, 0)) {
      u32 p = __shfl_sync(kFull, pos, 0) + ci - cnt;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (d[k] > (int)q.small) {
          q.st->v[p] = x[k];
          q.st->d[p] = (u32)d[k];
          ++p;
        }
      }
      return;
    }
  }
  u64 base = 0;
  if (lane == 0) base = atomicAdd(q.cnt, ((u64)ctot << 32) | (u64)stot);
  base = shfl64(base, 0);
  u32 slot = (u32)(base >> 32) + ci - cnt;
  u32 eb = (u32)base + si - sum;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (d[k] > (int)q.small) {
      q.ent[slot] = make_int2((int)x[k], (int)eb);
      const u32 c0 = (eb + kChunk - 1) / kChunk, c1 = (eb + (u32)d[k] - 1) / kChunk;
      for (u32 ch = c0; ch <= c1; ++ch) q.owner[ch] = slot;
      ++slot;
      eb += (u32)d[k];
    }
  }
}

// The same, reading the out-degree of every wanted vertex.
__device__ __forceinline__ void enqueue(const Queue &q, const RowMeta *row, const u32 *x,
                                        const bool *want, int kk, u64 &n_enq) {
  int d[K];
#pragma unroll
  for (int k = 0; k < K; ++k) d[k] = (k < kk && want[k]) ? __ldg(&row[x[k]].deg) : 0;
  enqueue_d(q, x, d, kk, n_enq);
}

// Block scan helper: exclusive prefix of one value per thread; the block
// total goes to *total (smem scratch of 33 words).
__device__ __forceinline__ u32 block_excl_scan(u32 x, u32 *scratch, u32 *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const u32 incl = warp_incl_scan(x);
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    u32 v = lane < nwarps ? scratch[lane] : 0u;
    v = warp_incl_scan(v);
    if (lane < nwarps) scratch[lane] = v;
  }
  __syncthreads();
  const u32 r = (warp ? scratch[warp - 1] : 0u) + incl - x;
  *total = scratch[nwarps - 1];
  __syncthreads();
  return r;
}

// Publish a block's staged appends (block-collective): up to two queues
// (entries with their chunk owners, and small lists) and one far pile.
// Every list takes one global atomic, each issued by its own thread and all
// of them together, so the block waits for one round trip instead of one per
// list; then the entries are written out.  scratch needs 39 words and the
// block more than 128 threads.
__device__ __forceinline__ void flush_stages(const Queue *q1, const Queue *q2, Stage *fst,
                                          u32 *pile, u32 *pcnt, u32 *pmin, u32 *scratch) {
  __syncthreads();
  const Queue *qs[2] = {q1, q2};
  const u32 t = threadIdx.x;
  u32 n[2], ns[2], b[2], e[2], run[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    n[j] = qs[j] && qs[j]->st ? *(volatile u32 *)&qs[j]->st->n : 0u;
    ns[j] = qs[j] && qs[j]->sst ? *(volatile u32 *)&qs[j]->sst->n : 0u;
    b[j] = e[j] = run[j] = 0;
    if (n[j]) {   // block-uniform
      const Stage *st = qs[j]->st;
      const u32 per = (n[j] + blockDim.x - 1) / blockDim.x;
      b[j] = min(t * per, n[j]);
      e[j] = min(b[j] + per, n[j]);
      u32 sum = 0;
      for (u32 i = b[j]; i < e[j]; ++i) sum += st->d[i];
      u32 total;
      run[j] = block_excl_scan(sum, scratch, &total);
      if (t == 64u * j) {
        const u64 base = atomicAdd(qs[j]->cnt, ((u64)n[j] << 32) | (u64)total);
        scratch[32 + 3 * j] = (u32)(base >> 32);
        scratch[33 + 3 * j] = (u32)base;
      }
    }
    if (ns[j] && t == 64u * j + 32u) scratch[34 + 3 * j] = atomicAdd(qs[j]->scnt, ns[j]);
  }
  const u32 nf = fst ? *(volatile u32 *)&fst->n : 0u;
  if (nf && t == 128u) {
    scratch[38] = atomicAdd(pcnt, nf);
    atomicMin(pmin, *(volatile u32 *)&fst->vmin);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (n[j]) {
      const Queue &q = *qs[j];
      u32 slot = scratch[32 + 3 * j] + b[j];
      u32 eb = scratch[33 + 3 * j] + run[j];
      for (u32 i = b[j]; i < e[j]; ++i) {
        const u32 d = q.st->d[i];
        q.ent[slot] = make_int2((int)q.st->v[i], (int)eb);
        const u32 c0 = (eb + kChunk - 1) / kChunk, c1 = (eb + d - 1) / kChunk;
        for (u32 ch = c0; ch <= c1; ++ch) q.owner[ch] = slot;
        ++slot;
        eb += d;
      }
    }
    if (ns[j]) {
      const u32 base = scratch[34 + 3 * j];
      for (u32 i = t; i < ns[j]; i += blockDim.x) qs[j]->sv[base + i] = qs[j]->sst->v[i];
    }
  }
  if (nf) {
    const u32 base = scratch[38];
    for (u32 i = t; i < nf; i += blockDim.x) pile[base + i] = fst->v[i];
  }
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (qs[j] && qs[j]->st) qs[j]->st->n = 0;
      if (qs[j] && qs[j]->sst) qs[j]->sst->n = 0;
    }
    if (fst) {
      fst->n = 0;
      fst->vmin = 0xFFFFFFFFu;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void flush_queue(const Queue &q, u32 *scratch) {
  flush_stages(&q, nullptr, nullptr, nullptr, nullptr, nullptr, scratch);
}

// Append each lane's wanted vertices to a far pile (warp-collective) and
// lower far_min to the smallest distance appended (through the block stage
// when there is one).
__device__ __forceinline__ void far_append(u32 *pile, u32 *cnt, u32 *far_min, Stage *st,
                                           const u32 *x, const bool *want, int kk,
                                           u32 lane_min) {
  const int lane = threadIdx.x & 31;
  u32 n = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) n += (k < kk && want[k]) ? 1u : 0u;
  if (!__ballot_sync(kFull, n > 0)) return;
  const u32 ni = warp_incl_scan(n), tot = __shfl_sync(kFull, ni, 31);
  u32 mn = lane_min;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u32 y = __shfl_xor_sync(kFull, mn, o);
    mn = y < mn ? y : mn;
  }
  if (st) {
    u32 pos = 0;
    bool ok = false;
    if (lane == 0) {
      ok = stage_reserve(st, tot, pos);
      if (ok) atomicMin(&st->vmin, mn);
    }
    if (__shfl_sync(kFull, ok, 0)) {
      u32 p = __shfl_sync(kFull, pos, 0) + ni - n;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (k < kk && want[k]) st->v[p++] = x[k];
      return;
    }
  }
  u32 base = 0;
  if (lane == 0) {
    base = atomicAdd(cnt, tot);
    atomicMin(far_min, mn);
  }
  base = __shfl_sync(kFull, base, 0);
  u32 slot = base + ni - n;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (k < kk && want[k]) pile[slot++] = x[k];
}

// Publish a block's staged far-pile entries (block-collective).
__device__ __forceinline__ void flush_far(Stage *st, u32 *pile, u32 *cnt, u32 *far_min,
                                          u32 *scratch) {
  flush_stages(nullptr, nullptr, st, pile, cnt, far_min, scratch);
}

// --- block-local relaxation (pool schedule of the push loop) ----------------
//
// On a high-diameter graph a push round advances the frontier by one edge,
// and a grid barrier per edge of the deepest shortest path costs more than
// the relaxations.  With the pool schedule every block keeps the vertices it
// improved below the near threshold in a pool in shared memory and expands
// them itself, in sub-rounds ended by block barriers, before it meets the
// other blocks at the grid barrier.  A wave then crosses many edges per grid
// round.  Blocks relax any vertex, not a partition of their own: two blocks
// that reach one vertex race through the packed atomicMin, and only the
// winner's entry survives.  Correctness rests on the same invariant as the
// frontier rounds: every vertex improved below the threshold is expanded
// with its final distance, here from the pool of the block that improved it
// last, or from the global frontier when its degree or a full pool sends it
// there.

constexpr u32 kPoolUnknown = 0xFFFFFFFFu;   // entry degree not read yet
// Pool edges per lane and step: four (kOpPool) or five (kOpPoolWide).  A warp
// takes as many steps as its largest entry needs, and each step is one more
// dependent round trip, so on a grid where batches gave many vertices a fifth
// edge the wide steps win; where almost every vertex has at most four, the
// narrow steps issue fewer instructions per sub-round and win.
constexpr int kPoolWideShare = 64;   // wide when >= 1/64 of the vertices have 5..8 out-edges

// Fetch a line toward L2 without waiting for it: a pool entry's next use is
// one sub-round later, by then its row is on chip.
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Append each lane's improved near targets to pool list b (warp-collective).
// A target with 1..kPoolDeg out-edges becomes an entry (x, nd, start / 4,
// deg); with kMeta false the row is not known yet and the entry carries
// kPoolUnknown instead (the drain reads it).  A target without out-edges
// needs nothing; a larger one, or one that finds the list full, comes back
// in rest[] for the global frontier.
template <bool kMeta>
__device__ __forceinline__ void pool_push(Pool *pl, u32 b, const u32 *x, const u32 *nd,
                                          const bool *want, int kk, const u32 *ms4,
                                          const int *mdg, bool *rest, u64 &n_in,
                                          const RowMeta *row, const int2 *adj) {
  const int lane = threadIdx.x & 31;
  bool take[K];
  u32 cnt = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    rest[k] = false;
    take[k] = false;
    if (k < kk && want[k]) {
      if (!kMeta || (mdg[k] > 0 && mdg[k] <= kPoolDeg)) {
        take[k] = true;
        ++cnt;
      } else if (mdg[k] > kPoolDeg) {
        rest[k] = true;
      }
    }
  }
  if (!__ballot_sync(kFull, cnt > 0)) return;
  const u32 ci = warp_incl_scan(cnt), tot = __shfl_sync(kFull, ci, 31);
  u32 base = 0;
  if (lane == 31) base = atomicAdd(&pl->n[b], tot);
  base = __shfl_sync(kFull, base, 31) + ci - cnt;
  uint4 *E = pl->e[b];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (take[k]) {
      if (base < kPoolCap) {
        E[base] = kMeta ? make_uint4(x[k], nd[k], ms4[k], (u32)mdg[k])
                        : make_uint4(x[k], nd[k], 0u, kPoolUnknown);
        // what the entry's expansion reads first: its edges (or its row)
        if (kMeta) {
          const int2 *e0 = adj + ((long long)ms4[k] << 2);
          prefetch_l2(e0);
          prefetch_l2(e0 + mdg[k] - 1);
        } else {
          prefetch_l2(row + x[k]);
        }
        ++n_in;
      } else {
        rest[k] = true;
      }
      ++base;
    }
  }
}

struct PoolCounters {
  u64 n_edges = 0, n_imp = 0, n_enq = 0, n_in = 0, ns = 0;
  u32 subs = 0;
  int range_err = 0;
};

// Sub-rounds over the block's pool (block-collective, every thread of the
// block), starting from list 0, until the pool is empty or lim.pool_rounds
// sub-rounds have run; then the entries left go to the global frontier qn.
// An entry whose vertex holds a smaller distance by now is skipped (the
// improvement that lowered it appended its own entry).  Each lane expands
// one entry, kPU edges per step, with every edge's load, packed atomicMin and
// (speculative) read of the target's row in flight together, so that a
// target it improves enters the other list with its row already known.
// Improved targets at or above thresh go to the far pile (pile != nullptr).
template <int kPU>
__device__ __forceinline__ void pool_drain(const LoopArgs &a, Pool *pl, u32 thresh, u32 tag,
                                           u32 phase, const Queue &qn, u32 *pile, u32 *pcnt,
                                           u32 *pmin, Stage *sf, PoolCounters &pc) {
  const int lane = threadIdx.x & 31;
  const u32 bs = blockDim.x;
  const RowMeta *row = a.fwd.row;
  const u64 t_in = globaltimer_ns();
  u32 p = 0, sub = 0;
  for (;;) {
    __syncthreads();
    const u32 nraw = *(volatile u32 *)&pl->n[p];
    const u32 n = nraw < kPoolCap ? nraw : kPoolCap;
    if (n == 0 || sub >= a.lim.pool_rounds) break;   // block-uniform
    const u32 q = p ^ 1;
    const uint4 *E = pl->e[p];
    for (u32 base = threadIdx.x & ~31u; base < n; base += bs) {
      const u32 i = base + lane;
      uint4 en = make_uint4(0u, 0u, 0u, 0u);
      if (i < n) en = E[i];
      const u32 v = en.x, d = en.y;
      u32 deg = en.w;
      long long start = (long long)en.z << 2;
      u64 sv = 0ull;
      if (deg != 0 && (v >= (u32)a.n ||
                       (deg != kPoolUnknown && start + (long long)deg > a.fwd.slots))) {
        atomicExch(&a.ctl->bad, 1);   // never expected: record and skip
        deg = 0;
      }
      if (deg == kPoolUnknown) {     // appended by the round's frontier expansion
        const int4 r = __ldg((const int4 *)(row + v));
        sv = ld_cg_u64(a.s + v);
        start = (long long)(((u64)(u32)r.y << 32) | (u32)r.x);
        deg = (u32)r.z;
      } else if (deg) {
        sv = ld_cg_u64(a.s + v);
      }
      // the first step's edges load together with the state word, before
      // anything waits for either
      int2 ed0[kPU];
#pragma unroll
      for (int k = 0; k < kPU; ++k)
        ed0[k] = (u32)k < deg && deg <= (u32)kPoolDeg ? __ldg(a.fwd.adj + start + k)
                                                       : make_int2(0, 0);
      // a vertex with more out-edges than a lane takes goes to the frontier
      bool big[K] = {};
      u32 bx[K] = {};
      big[0] = deg > (u32)kPoolDeg && dist_of(sv) == d;
      bx[0] = v;
      if (big[0]) big[0] = atomicExch(a.qflag + v, tag) != tag;
      enqueue(qn, row, bx, big, 1, pc.n_enq);
      if (deg > (u32)kPoolDeg) deg = 0;
      u32 steps = (deg + kPU - 1) / kPU;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const u32 y = __shfl_xor_sync(kFull, steps, o);
        steps = y > steps ? y : steps;
      }
      bool live = false;
      for (u32 t = 0; t < steps; ++t) {
        int2 ed[kPU];
#pragma unroll
        for (int k = 0; k < kPU; ++k) {
          const u32 e = t * kPU + (u32)k;
          ed[k] = t == 0 ? ed0[k] : (e < deg ? __ldg(a.fwd.adj + start + e) : make_int2(0, 0));
        }
        if (t == 0) live = deg > 0 && dist_of(sv) == d;
        // per edge: target, candidate distance, the target's old state (from
        // the atomicMin) and its row (start / 4, degree), read together
        u32 tx[K], nd[K], ms4[K];
        int mdg[K];
        u64 old[K];
        bool act[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const u32 e = t * kPU + (u32)k;
          act[k] = k < kPU && live && e < deg;
          tx[k] = k < kPU ? (u32)ed[k < kPU ? k : 0].x : 0u;
          nd[k] = k < kPU ? d + (u32)ed[k < kPU ? k : 0].y : kInf;
          if (act[k]) {
            ++pc.n_edges;
            if (nd[k] >= kInf) {
              pc.range_err = 1;
              act[k] = false;
            }
          }
          old[k] = act[k] ? atomicMin((unsigned long long *)(a.s + tx[k]), pack(nd[k], v)) : 0ull;
          ms4[k] = 0;
          mdg[k] = 0;
          if (act[k]) {
            const int4 r = __ldg((const int4 *)(row + tx[k]));
            ms4[k] = (u32)((((u64)(u32)r.y << 32) | (u32)r.x) >> 2);
            mdg[k] = r.z;
          }
        }
        bool near[K], far[K];
        u32 fmin = 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          near[k] = far[k] = false;
          if (act[k] && pack(nd[k], v) < old[k]) {
            ++pc.n_imp;
            if (nd[k] < thresh) {
              near[k] = true;
            } else if (pile) {
              far[k] = atomicExch(a.ftag + tx[k], phase) != phase;
              if (far[k] && nd[k] < fmin) fmin = nd[k];
            }
          }
        }
        bool rest[K], want[K];
        pool_push<true>(pl, q, tx, nd, near, kPU, ms4, mdg, rest, pc.n_in, row, a.fwd.adj);
#pragma unroll
        for (int k = 0; k < K; ++k)
          want[k] = k < kPU && rest[k] && atomicExch(a.qflag + tx[k], tag) != tag;
        enqueue(qn, row, tx, want, kPU, pc.n_enq);
        if (pile) far_append(pile, pcnt, pmin, sf, tx, far, kPU, fmin);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) pl->n[p] = 0u;
    p = q;
    ++sub;
  }
  pc.subs += sub;
  if (sub) pc.ns += globaltimer_ns() - t_in;
  // entries left when the budget ran out: to the global frontier
  {
    const u32 nraw = *(volatile u32 *)&pl->n[p];
    const u32 n = nraw < kPoolCap ? nraw : kPoolCap;
    const uint4 *E = pl->e[p];
    for (u32 base = threadIdx.x & ~31u; base < n; base += bs) {
      const u32 i = base + lane;
      bool want[K] = {};
      u32 x[K] = {};
      if (i < n) {
        x[0] = E[i].x;
        want[0] = atomicExch(a.qflag + x[0], tag) != tag;
      }
      enqueue(qn, row, x, want, 1, pc.n_enq);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) pl->n[0] = pl->n[1] = 0u;
}

// --- edge operations ------------------------------------------------------
//
// Each op provides vdata(v) (a per-source datum read once per queue entry),
// load(e) (the state word an edge needs) and run(...) (the updates of one
// lane's edges followed by the warp-collective enqueue of what they queue).

// Incremental fixedPoint body: <dist, parent>[x] = <Min(dist[x], dist[v] + w), v>
// as one packed atomicMin; an improved x joins the next frontier once, or,
// under near-far ordering with a distance >= thresh, the far pile once per
// phase.
struct PushOp {
  u64 *s;
  u32 *qflag;
  u32 tag;
  Queue next;
  const RowMeta *row;
  u32 thresh;
  u32 *pile, *pcnt, *far_min, *ftag;
  u32 phase;
  Stage *fst;
  Pool *pool;              // pool schedule: near improvements go to list 0
  u64 n_edges = 0, n_imp = 0, n_enq = 0, n_in = 0;
  int range_err = 0;

  __device__ __forceinline__ u32 vdata(u32 v) { return dist_of(ld_cg_u64(s + v)); }
  __device__ __forceinline__ u64 load(int2 e) { return ld_cg_u64(s + e.x); }
  __device__ __forceinline__ void run(const bool *act, const u32 *ov, const u32 *od,
                                      const int2 *ed, const u64 *sx) {
    // every atomicMin of the lane is issued before any result is used, then
    // every dedupe exchange: two round trips per lane instead of up to 2K
    u32 tx[K], nd[K];
    u64 cand[K], old[K];
    bool want[K], far[K], tried[K];
    u32 fmin = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      want[k] = false;
      far[k] = false;
      tx[k] = (u32)ed[k].x;
      nd[k] = od[k] + (u32)ed[k].y;
      cand[k] = pack(nd[k], ov[k]);
      tried[k] = false;
      if (act[k]) {
        ++n_edges;
        if (od[k] < kInf) {
          if (nd[k] >= kInf) range_err = 1;
          else tried[k] = cand[k] < sx[k];
        }
      }
    }
    // Frontier rounds issue the dedupe exchange of a near candidate and the
    // read of its out-degree together with its atomicMin, not after it.  A
    // candidate below the distance read this round that loses its atomicMin
    // lost to an improvement made this round, whose own candidate is smaller,
    // so also near and exchanged: whichever exchange comes first enqueues the
    // vertex, which is then enqueued exactly when it was improved.
    bool spec[K];
    u32 ex[K];
    int dg[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      spec[k] = pool == nullptr && tried[k] && nd[k] < thresh;
      old[k] = tried[k] ? atomicMin((unsigned long long *)(s + ed[k].x), cand[k]) : 0ull;
      ex[k] = spec[k] ? atomicExch(qflag + ed[k].x, tag) : tag;
      dg[k] = spec[k] ? __ldg(&row[tx[k]].deg) : 0;
    }
    bool pw[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      pw[k] = false;
      if (tried[k] && cand[k] < old[k]) {
        ++n_imp;
        if (nd[k] >= thresh) far[k] = atomicExch(ftag + ed[k].x, phase) != phase;
        else if (pool) pw[k] = true;
      }
      want[k] = spec[k] && ex[k] != tag;
      if (!want[k]) dg[k] = 0;
    }
    if (pool) {
      bool rest[K];
      pool_push<false>(pool, 0, tx, nd, pw, K, nullptr, nullptr, rest, n_in, row, nullptr);
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (rest[k]) want[k] = atomicExch(qflag + tx[k], tag) != tag;
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (far[k] && nd[k] < fmin) fmin = nd[k];
    if (pool) enqueue(next, row, tx, want, K, n_enq);
    else enqueue_d(next, tx, dg, K, n_enq);
    if (pile) far_append(pile, pcnt, far_min, fst, tx, far, K, fmin);
  }
};

// Decremental first loop body: a child x of v (parent[x] == v) loses its
// distance and parent, joins the next frontier (its out-edges) and the
// cut list (its in-edges are pulled later).
struct InvalOp {
  u64 *s;
  Queue next;
  const RowMeta *row;
  u32 *cut, *ccnt, *cmin;   // cut-vertex list and its block stage
  Stage *cst;
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
    far_append(cut, ccnt, cmin, cst, tx, want, K, 0u);
  }
};

// propagateNodeFlags body (PageRank): every vertex reachable from a flagged
// one is flagged once (prflag[x] = ptag) and joins the next frontier.
struct FlagOp {
  u32 *flag;
  u32 ptag;
  Queue next;
  const RowMeta *row;
  u64 n_edges = 0, n_enq = 0, n_aff = 0;
  int range_err = 0;

  __device__ __forceinline__ u32 vdata(u32) { return 0; }
  __device__ __forceinline__ u64 load(int2 e) { return __ldcg(flag + e.x); }
  __device__ __forceinline__ void run(const bool *act, const u32 *, const u32 *,
                                      const int2 *ed, const u64 *sx) {
    u32 tx[K], prev[K];
    bool want[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {   // every exchange in flight before any is read
      tx[k] = (u32)ed[k].x;
      n_edges += act[k];
      prev[k] = act[k] && (u32)sx[k] != ptag ? atomicExch(flag + ed[k].x, ptag) : ptag;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      want[k] = prev[k] != ptag;
      n_aff += want[k];
    }
    enqueue(next, row, tx, want, K, n_enq);
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
  u32 *seed_min;
  u64 n_edges = 0, n_enq = 0;
  int range_err = 0;

  __device__ __forceinline__ u32 vdata(u32) { return 0; }
  __device__ __forceinline__ u64 load(int2 e) { return ld_cg_u64(s + e.x); }
  __device__ __forceinline__ void run(const bool *act, const u32 *ov, const u32 *,
                                      const int2 *ed, const u64 *sx) {
    const int lane = threadIdx.x & 31;
    // the lane's candidates: a run of edges of one vertex that ends inside
    // the lane is kept in the slot of the edge that ended it (slot 0 never
    // ends a run, so it takes the lane's last run once the warp has combined
    // it with the lanes that end on the same vertex); every offer's load,
    // atomicMin and dedupe exchange then goes out together
    u32 cv[K];
    u64 cb[K];
    bool has[K];
    u32 bv = kNoEdge;
    u64 best = ~0ull;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      has[k] = false;
      cv[k] = 0;
      cb[k] = ~0ull;
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
          if (bv != kNoEdge && best != ~0ull) {
            cv[k] = bv;
            cb[k] = best;
            has[k] = true;
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
    if (head && best != ~0ull) {
      cv[0] = bv;
      cb[0] = best;
      has[0] = true;
    }
    u64 cur[K], old[K];
    bool imp[K], want[K];
#pragma unroll
    for (int k = 0; k < K; ++k) cur[k] = has[k] ? ld_cg_u64(s + cv[k]) : 0ull;
    // the exchange and the out-degree read go with the atomicMin, as in the
    // push rounds: a candidate that loses its atomicMin lost to a smaller one
    // of this stage, which exchanges too
    u32 pr[K];
    int dg[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      has[k] = has[k] && cb[k] < cur[k];
      old[k] = has[k] ? atomicMin((unsigned long long *)(s + cv[k]), cb[k]) : 0ull;
      pr[k] = has[k] ? atomicExch(qflag + cv[k], tag) : tag;
      dg[k] = has[k] ? __ldg(&row[cv[k]].deg) : 0;
    }
    u32 mind = kInf;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      imp[k] = has[k] && cb[k] < old[k];
      if (imp[k] && dist_of(cb[k]) < mind) mind = dist_of(cb[k]);
      want[k] = has[k] && pr[k] != tag;
      if (!want[k]) dg[k] = 0;
    }
    if (mind < kInf) atomicMin(seed_min, mind);
    enqueue_d(next, cv, dg, K, n_enq);
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

// The batch passed validation (one answer for the whole block).
__device__ __forceinline__ bool batch_valid_block(Ctl *c) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = ld_cg_i32(&c->status) == 0 ? 1 : 0;
  __syncthreads();
  return s_ok != 0;
}

// The same test with one answer for the whole block (kernels with barriers).
__device__ __forceinline__ bool repair_enabled_block(Ctl *c) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = repair_enabled(c) ? 1 : 0;
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ Queue make_queue(int2 *ent, u32 *own, u64 *cnt, u32 *sv, u32 *scnt,
                                            Stage *st = nullptr, Stage *sst = nullptr,
                                            u32 small = kSmallDeg) {
  Queue q;
  q.small = small;
  q.ent = ent;
  q.owner = own;
  q.cnt = (unsigned long long *)cnt;
  q.sv = sv;
  q.scnt = scnt;
  q.st = st;
  q.sst = sst;
  return q;
}

__device__ __forceinline__ u32 *scnt_ptr(Ctl *c, u32 b) {
  return b == 0 ? &c->scnt0 : (b == 1 ? &c->scnt1 : &c->scnt2);
}

// Expand up to 32 small-list vertices, one lane each, K edges per step (the
// warp takes as many steps as its largest vertex needs).
template <class Op>
__device__ __forceinline__ void process_small(Op &op, const u32 *sv, u32 n_small, u32 group,
                                              const Store &st, int n, Ctl *c) {
  const int lane = threadIdx.x & 31;
  const u32 idx = group * 32 + lane;
  u32 v = 0, dv = 0;
  int deg = 0;
  long long start = 0;
  if (idx < n_small) {
    v = __ldcg(sv + idx);
    if (v < (u32)n) {
      const RowMeta rm = st.row[v];
      deg = rm.deg;
      start = rm.start;
      dv = op.vdata(v);
    } else {                             // never expected: record and skip
      atomicExch(&c->bad, 1);
      v = 0;
    }
  }
  int steps = (deg + K - 1) / K;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int y = __shfl_xor_sync(kFull, steps, o);
    steps = y > steps ? y : steps;
  }
  for (int t = 0; t < steps; ++t) {
    bool act[K];
    u32 ov[K], od[K];
    int2 ed[K];
    u64 sx[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int e = t * K + k;
      act[k] = e < deg;
      ov[k] = v;
      od[k] = dv;
      ed[k] = act[k] ? __ldg(st.adj + start + e) : make_int2(0, 0);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) sx[k] = act[k] ? op.load(ed[k]) : 0ull;
    op.run(act, ov, od, ed, sx);
  }
}

// --- persistent loop ------------------------------------------------------
//
// Every block keeps the loop state (current buffer, round, threshold, far
// pile, phase) in registers and derives it from the same counters after each
// barrier, so a round costs one barrier and no serial step.  Buffers rotate
// over three slots: round r reads frontier slot r%3, appends to (r+1)%3, and
// block 0 zeroes (r+2)%3, which nobody touches until round r+1.  Far piles
// rotate the same way: a split round reads pile f, keeps entries in f+1 and
// zeroes f+2.

// Pointer-jumping tail of the invalidation (block-collective, every block).
// jmp[v] starts as kJumpCut for a vertex without a distance (cut by
// OnDelete, reached by the frontier rounds, or unreachable), kJumpRoot for
// the source, else its parent.  A pass replaces every ancestor word by the
// ancestor's own word, which doubles the path it covers; a cut anywhere on
// the path reaches v as kJumpCut.  Passes read words that other threads may
// have advanced already, which only skips further up the same path.
struct JumpState {
  u64 target, n_aff;
  u32 jumps, capped;
};

__device__ __forceinline__ JumpState jump_phase(const LoopArgs &a, u64 *bar, u64 target,
                                             u32 *scratch, Stage *cst) {
  Ctl *c = a.ctl;
  u32 jumps = 0;
  bool capped = false;
  u64 n_aff = 0;
  const int lane = threadIdx.x & 31;
  const u32 gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  const u32 n = (u32)a.n;
  const u32 gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  // every sweep below takes K vertices per thread at a time and issues all
  // their loads before it stores anything, so their latencies overlap
  for (u32 v0 = gt; v0 < n; v0 += nt * K) {
    u64 sv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const u32 v = v0 + (u32)k * nt;
      sv[k] = v < n ? ld_cg_u64(a.s + v) : 0ull;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const u32 v = v0 + (u32)k * nt;
      const u32 p = parent_of(sv[k]);
      if (v < n)
        __stcg(a.jmp + v, dist_of(sv[k]) >= kInf ? kJumpCut : (p == kNoParent ? kJumpRoot : p));
    }
  }
  target += gridDim.x;
  bool stop = grid_sync(bar, target, c, a.lim);
  for (;;) {
    if (stop) break;
    if (jumps > 0 && ld_cg_u32(jcnt_ptr(c, (jumps - 1) % 3)) == 0) break;
    if (jumps >= kMaxJumps) {
      capped = true;
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *(volatile u32 *)jcnt_ptr(c, (jumps + 1) % 3) = 0u;
    // a vertex whose word turns into kJumpCut in this pass had a distance
    // (its word was an ancestor) and a cut lies on its tree path: it loses
    // the distance and joins the cut list here, exactly once
    u32 act = 0;
    for (u32 w0 = gw * 32 * K; w0 < n; w0 += nw * 32 * K) {
      u32 v[K], j[K], ja[K];
      bool hit[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        v[k] = w0 + lane + 32 * k;
        j[k] = v[k] < n ? __ldcg(a.jmp + v[k]) : kJumpRoot;
      }
#pragma unroll
      for (int k = 0; k < K; ++k) ja[k] = j[k] < kJumpRoot ? __ldcg(a.jmp + j[k]) : j[k];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        hit[k] = false;
        if (j[k] < kJumpRoot) {
          __stcg(a.jmp + v[k], ja[k]);
          act += ja[k] < kJumpRoot ? 1u : 0u;
          if (ja[k] == kJumpCut) {
            a.s[v[k]] = kInfPack;
            hit[k] = true;
            ++n_aff;
          }
        }
      }
      far_append(a.cut, &c->ccnt, &c->cmin, cst, v, hit, K, 0u);
    }
    u32 total;
    block_excl_scan(act, scratch, &total);
    if (threadIdx.x == 0 && total) atomicAdd(jcnt_ptr(c, jumps % 3), total);
    ++jumps;
    target += gridDim.x;
    stop = grid_sync(bar, target, c, a.lim);
  }
  flush_far(cst, a.cut, &c->ccnt, &c->cmin, scratch);
  JumpState out;
  out.target = target;
  out.n_aff = n_aff;
  out.jumps = jumps;
  out.capped = capped ? 1u : 0u;
  return out;
}

// Single-block rounds of the push loop.  While the frontier is small a round
// is mostly latency (a chain of dependent loads and atomics) plus the grid
// barrier, and one block can do the work: block 0 keeps the frontier in
// shared memory, ends each round with __syncthreads, and the other blocks
// wait.  A frontier entry carries its vertex, the vertex's out-degree and
// the distance it was improved to, so a round needs no global read before
// its edges: a block scan of the degrees assigns kLocalUnroll edges to each
// thread, and every edge's (col, w) load, packed atomicMin and (speculative)
// read of the target's degree are in flight together.  Entries are not
// deduplicated: every improvement appends its target with the new distance,
// so the entry with a vertex's current distance is always present and stale
// ones only repeat relaxations that cannot win.  The next frontier thus
// holds at most one entry per edge of this one, and a round runs here only
// if its frontier has at most lim.local_edges (<= kLocalCap) edges.  On exit
// the frontier goes to queue slot next3(cur), which is empty, and slot
// next3(next3(cur)) is cleared for the round after.
constexpr u32 kLocalCap = kStageQ;
constexpr int kLocalUnroll = (kLocalRoundCap + kPersistThreads - 1) / kPersistThreads;
static_assert(kLocalUnroll <= K, "far appends go K at a time");
static_assert(kLocalRoundCap <= (int)kLocalCap, "single-block frontier lists too small");
// shared-memory words used: two lists of (vertex, degree, distance) and the
// edge offsets; the far-pile stage starts after the other stages
static_assert(7 * kLocalCap <= 2 * kStageQ + kStageQS + 2 * kStageA + kStageAS,
              "single-block round arrays overlap the far-pile stage");

struct LocalState {      // what an episode hands back to the loop
  u32 cur, round, capped, stop;
  u64 n_edges, n_imp, n_enq;
  int range_err;
  // the counters the loop decides on next (frontier slot cur, far pile f),
  // as block 0 left them: every block takes the same decision even though
  // block 0 may already be changing them in its next episode
  u64 q;
  u32 nsmall, n_far, fmin;
};

// Block 0 only (block-collective).  smem: 7 * kLocalCap words that no other
// stage of the push loop uses while the episode runs.
__device__ __forceinline__ LocalState local_rounds(const LoopArgs &a, u32 cur, u32 round, u32 thresh,
                                                u32 f, u32 phase, bool nf, u32 *smem,
                                                Stage *sf, u32 *scratch) {
  LocalState out{};
  Ctl *c = a.ctl;
  const int lane = threadIdx.x & 31;
  const u32 tid = threadIdx.x, bs = blockDim.x;
  u32 *lx[2] = {smem, smem + kLocalCap};
  u32 *ldeg[2] = {smem + 2 * kLocalCap, smem + 3 * kLocalCap};
  u32 *ld[2] = {smem + 4 * kLocalCap, smem + 5 * kLocalCap};
  u32 *soff = smem + 6 * kLocalCap;    // exclusive prefix of the entries' out-degrees
  __shared__ u32 s_n[2], s_stop;
  {
    const u64 q = ld_cg_u64(qcnt_ptr(c, cur));
    const u32 ne = (u32)(q >> 32), ns = ld_cg_u32(scnt_ptr(c, cur));
    for (u32 i = tid; i < ne + ns; i += bs) {
      const u32 v = i < ne ? (u32)__ldcg(&a.qent[cur][i].x) : __ldcg(a.qsv[cur] + (i - ne));
      lx[0][i] = v;
      ld[0][i] = dist_of(ld_cg_u64(a.s + v));
      ldeg[0][i] = (u32)__ldg(&a.fwd.row[v].deg);
    }
    if (tid == 0) {
      s_n[0] = ne + ns;
      s_n[1] = 0;
      s_stop = 0;
    }
  }
  __syncthreads();
  u32 p = 0;
  for (;;) {
    const u32 nl = s_n[p];
    if (nl == 0) break;
    if (round >= a.lim.max_rounds) {
      out.capped = 1;
      break;
    }
    const u32 *Lx = lx[p], *Ld = ld[p], *Ldeg = ldeg[p];
    u32 *Nx = lx[p ^ 1], *Nd = ld[p ^ 1], *Ndeg = ldeg[p ^ 1];
    // (A) edge offsets: a block scan of the degrees (a contiguous run of
    // entries per thread)
    const u32 per = (nl + bs - 1) / bs;
    const u32 b0 = tid * per < nl ? tid * per : nl;
    const u32 b1 = b0 + per < nl ? b0 + per : nl;
    u32 sum = 0;
    for (u32 i = b0; i < b1; ++i) sum += Ld[i] < kInf ? Ldeg[i] : 0u;
    u32 total;
    u32 run = block_excl_scan(sum, scratch, &total);
    if (total > a.lim.local_edges) break;   // the next frontier might not fit
    for (u32 i = b0; i < b1; ++i) {
      soff[i] = run;
      run += Ld[i] < kInf ? Ldeg[i] : 0u;
    }
    __syncthreads();
    // (B) edges: kLocalUnroll per thread, all in flight together
    u32 x[kLocalUnroll], nd[kLocalUnroll], vv[kLocalUnroll], dx[kLocalUnroll];
    u64 cand[kLocalUnroll], old[kLocalUnroll];
#pragma unroll
    for (int k = 0; k < kLocalUnroll; ++k) {
      const u32 e = (u32)k * bs + tid;
      x[k] = 0;
      nd[k] = kInf;
      vv[k] = 0;
      if (e < total) {
        u32 lo = 0, hi = nl - 1;   // entry owning edge e: last offset <= e
        while (lo < hi) {
          const u32 mid = (lo + hi + 1) >> 1;
          if (soff[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const u32 v = Lx[lo];
        const long long st = __ldg(&a.fwd.row[v].start);
        const int2 ed = a.fwd.adj[st + (e - soff[lo])];
        vv[k] = v;
        x[k] = (u32)ed.x;
        nd[k] = Ld[lo] + (u32)ed.y;
      }
    }
#pragma unroll
    for (int k = 0; k < kLocalUnroll; ++k) {
      cand[k] = ~0ull;
      old[k] = 0ull;
      dx[k] = 0;
      if ((u32)k * bs + tid < total) {
        ++out.n_edges;
        if (nd[k] >= kInf) {
          out.range_err = 1;
        } else {
          cand[k] = pack(nd[k], vv[k]);
          old[k] = atomicMin((unsigned long long *)(a.s + x[k]), cand[k]);
          // speculative: the degree is needed only if the edge improves x
          dx[k] = (u32)__ldg(&a.fwd.row[x[k]].deg);
        }
      }
    }
    bool want[kLocalUnroll], far[kLocalUnroll];
    u32 fmin = 0xFFFFFFFFu, cnt = 0;
#pragma unroll
    for (int k = 0; k < kLocalUnroll; ++k) {
      want[k] = far[k] = false;
      if (cand[k] < old[k]) {
        ++out.n_imp;
        if (nd[k] < thresh) {
          want[k] = dx[k] > 0;
          cnt += want[k] ? 1u : 0u;
        } else {
          far[k] = atomicExch(a.ftag + x[k], phase) != phase;
          if (far[k] && nd[k] < fmin) fmin = nd[k];
        }
      }
    }
    // append the improved targets (warp-aggregated)
    {
      const u32 inc = warp_incl_scan(cnt);
      u32 base = 0;
      if (lane == 31 && inc) base = atomicAdd(&s_n[p ^ 1], inc);
      base = __shfl_sync(kFull, base, 31) + inc - cnt;
#pragma unroll
      for (int k = 0; k < kLocalUnroll; ++k) {
        if (want[k]) {
          Nx[base] = x[k];
          Nd[base] = nd[k];
          Ndeg[base] = dx[k];
          ++base;
        }
      }
      out.n_enq += cnt;
    }
    if (nf) {
      bool fw[K];
      u32 fx[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        fw[k] = k < kLocalUnroll ? far[k] : false;
        fx[k] = k < kLocalUnroll ? x[k] : 0u;
      }
      far_append(a.fq[f], fcnt_ptr(c, f), fmin_ptr(c, f), sf, fx, fw, K, fmin);
    }
    __syncthreads();
    if (tid == 0) {
      s_n[p] = 0;
      if ((round & 63u) == 0) {   // heartbeat for the waiting blocks
        *(volatile u64 *)&c->lbeat = globaltimer_ns();
        s_stop = ld_cg_i32(&c->timeout) != 0 ? 1u : 0u;
      }
    }
    ++round;
    p ^= 1;
    __syncthreads();
    if (s_stop) {
      out.stop = 1;
      break;
    }
  }
  // hand the frontier back through the global queue (duplicates are fine:
  // the distributed rounds read each vertex's distance when they expand it)
  const u32 nxt = next3(cur);
  const Queue qn =
      make_queue(a.qent[nxt], a.qown[nxt], qcnt_ptr(c, nxt), a.qsv[nxt], scnt_ptr(c, nxt));
  u64 dummy = 0;
  const u32 nl = s_n[p];
  const u32 *Lx = lx[p];
  for (u32 base = (threadIdx.x >> 5) * 32; base < nl; base += bs) {
    const u32 i = base + lane;
    bool want[K] = {};
    u32 xx[K] = {};
    if (i < nl) {
      xx[0] = Lx[i];
      want[0] = true;
    }
    enqueue(qn, a.fwd.row, xx, want, 1, dummy);
  }
  if (tid == 0) {
    *(volatile u64 *)qcnt_ptr(c, next3(nxt)) = 0ull;
    *(volatile u32 *)scnt_ptr(c, next3(nxt)) = 0u;
  }
  if (nf) flush_far(sf, a.fq[f], fcnt_ptr(c, f), fmin_ptr(c, f), scratch);
  __syncthreads();
  out.cur = nxt;
  out.round = round;
  return out;
}

// One episode of single-block rounds (block-collective, every block): block 0
// runs them and hands the loop state back through the control block; the
// others wait for it, bounded by block 0's heartbeat.  Counters in the
// result are this thread's.
__device__ __forceinline__ LocalState local_episode(const LoopArgs &a, u32 lep, u32 cur, u32 round,
                                                 u32 thresh, u32 f, u32 phase, bool nf,
                                                 u32 *smem, Stage *sf, u32 *scratch) {
  Ctl *c = a.ctl;
  LocalState out{};
  __shared__ u64 s_q;
  __shared__ u32 s_sn, s_fn, s_fm;
  if (blockIdx.x == 0) {
    const u64 t_in = globaltimer_ns();
    out = local_rounds(a, cur, round, thresh, f, phase, nf, smem, sf, scratch);
    if (threadIdx.x == 0) {
      c->local_ns += globaltimer_ns() - t_in;
      const u64 q = ld_cg_u64(qcnt_ptr(c, out.cur));
      const u32 sn = ld_cg_u32(scnt_ptr(c, out.cur));
      const u32 fn = nf ? ld_cg_u32(fcnt_ptr(c, f)) : 0u;
      const u32 fm = nf ? ld_cg_u32(fmin_ptr(c, f)) : kInf;
      *(volatile u32 *)&c->lcur = out.cur;
      *(volatile u32 *)&c->lround = out.round;
      *(volatile u32 *)&c->lcap = out.capped;
      *(volatile u64 *)&c->lq = q;
      *(volatile u32 *)&c->lsn = sn;
      *(volatile u32 *)&c->lfn = fn;
      *(volatile u32 *)&c->lfm = fm;
      c->local_episodes += 1;
      c->local_rounds += out.round - round;
      __threadfence();
      st_release_u32(&c->lres, lep);
      scratch[39] = (out.stop || ld_cg_i32(&c->timeout) != 0) ? 1u : 0u;
      s_q = q;
      s_sn = sn;
      s_fn = fn;
      s_fm = fm;
    }
    __syncthreads();
    out.stop = scratch[39];
    out.q = s_q;
    out.nsmall = s_sn;
    out.n_far = s_fn;
    out.fmin = s_fm;
    __syncthreads();
  } else {
    if (threadIdx.x == 0) {
      // bounded wait: block 0 refreshes a heartbeat every round
      const u64 t0 = globaltimer_ns();
      u32 nap = 32, polls = 0;
      while (ld_acquire_u32(&c->lres) < lep) {
        if (ld_cg_i32(&c->timeout) != 0) break;
        if (++polls > kMaxPolls) {
          raise_timeout(c, 2, 3, lep);
          break;
        }
        // the heartbeat is block 0's clock, read after this block's: it can
        // be the later of the two, and then nothing has run out yet
        const u64 beat = ld_cg_u64(&c->lbeat), now = globaltimer_ns();
        const u64 since = beat > t0 ? beat : t0;
        if (now > since && now - since > a.lim.wait_ns) {
          raise_timeout(c, 2, 3, lep);
          break;
        }
        __nanosleep(nap);
        if (nap < 1024) nap += nap >> 1;
      }
      scratch[36] = ld_cg_u32(&c->lcur);
      scratch[37] = ld_cg_u32(&c->lround);
      scratch[38] = ld_cg_u32(&c->lcap);
      scratch[39] = ld_cg_i32(&c->timeout) != 0 ? 1u : 0u;
      s_q = ld_cg_u64(&c->lq);
      s_sn = ld_cg_u32(&c->lsn);
      s_fn = ld_cg_u32(&c->lfn);
      s_fm = ld_cg_u32(&c->lfm);
    }
    __syncthreads();
    out.cur = scratch[36];
    out.round = scratch[37];
    out.capped = scratch[38];
    out.stop = scratch[39];
    out.q = s_q;
    out.nsmall = s_sn;
    out.n_far = s_fn;
    out.fmin = s_fm;
    __syncthreads();
  }
  return out;
}

__device__ __forceinline__ void cut_to_a(const LoopArgs &a, Stage *sa, Stage *sas, u32 *scratch);
__device__ __forceinline__ void pull_stage(const LoopArgs &a, Stage *st, Stage *sst, u32 *scratch);
__device__ __forceinline__ void add_stage(const LoopArgs &a, Stage *st, Stage *sst, u32 *scratch);

template <int OP>
__global__ void __launch_bounds__(is_pool(OP) ? kPoolThreads : kPersistThreads, 1)
    k_loop(LoopArgs a) {
  extern __shared__ __align__(16) u32 dsm[];
  __shared__ Stage sq, sqs, sa, sas, sf;
  __shared__ Pool pool;
  constexpr bool kPushOp = OP == kOpPush || is_pool(OP);
  __shared__ u32 scratch[40];
  Ctl *c = a.ctl;
  // beside the store update the invalidation starts once the batch is
  // validated and does not wait for the merge's pool check: a rerun after a
  // pool grow keeps what it found
  if (OP == kOpInval && a.concurrent) {
    if (!batch_valid_block(c)) return;
  } else if (!repair_enabled_block(c)) {
    return;
  }
  if (threadIdx.x == 0) {
    u32 *p = dsm;
    sq.n = 0; sq.cap = kStageQ; sq.vmin = kInf; sq.v = p; sq.d = p + kStageQ; p += 2 * kStageQ;
    sqs.n = 0; sqs.cap = kStageQS; sqs.vmin = kInf; sqs.v = p; sqs.d = nullptr; p += kStageQS;
    sa.n = 0; sa.cap = kStageA; sa.vmin = kInf; sa.v = p; sa.d = p + kStageA; p += 2 * kStageA;
    sas.n = 0; sas.cap = kStageAS; sas.vmin = kInf; sas.v = p; sas.d = nullptr; p += kStageAS;
    sf.n = 0; sf.cap = kStageF; sf.vmin = 0xFFFFFFFFu; sf.v = p; sf.d = nullptr;
    if (is_pool(OP)) {
      pool.e[0] = (uint4 *)(dsm + kLoopSmem / sizeof(u32));
      pool.e[1] = pool.e[0] + kPoolCap;
      pool.n[0] = pool.n[1] = 0u;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const u64 t_start = globaltimer_ns();
  // warp ids interleaved across blocks, so that a round with few chunks
  // still spreads over every SM
  const u32 gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  u64 n_edges = 0, n_imp = 0, n_enq = 0, n_aff = 0, moved = 0;
  int range_err = 0;
  u64 *bar = kPushOp ? &c->bar_push : &c->bar_inval;
  PoolCounters pc;
  u64 target = 0;

  if (OP == kOpInval && a.n_del > 0) {
    // OnDelete: a deleted edge u -> v that is v's parent edge invalidates v;
    // v joins the cut list and, for frontier rounds, the first frontier
    // (beside the store update there are none: the tree walk is jumping)
    const Queue q0 = make_queue(a.qent[0], a.qown[0], &c->qcnt0, a.qsv[0], &c->scnt0, &sq, &sqs);
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
      if (!a.concurrent) enqueue(q0, a.fwd.row, v, hit, 1, n_enq);
      far_append(a.cut, &c->ccnt, &c->cmin, &sf, v, hit, 1, 0u);
    }
    flush_stages(a.concurrent ? nullptr : &q0, nullptr, &sf, a.cut, &c->ccnt, &c->cmin, scratch);
  }
  if (OP == kOpFlag && a.n_del > 0) {
    // the phase's destinations are the flags' seeds
    const Queue q0 = make_queue(a.qent[0], a.qown[0], &c->qcnt0, a.qsv[0], &c->scnt0, &sq, &sqs);
    for (long long base = (long long)gw * 32; base < a.n_del; base += (long long)nw * 32) {
      const long long i = base + lane;
      bool hit[K] = {};
      u32 v[K] = {};
      if (i < a.n_del) {
        v[0] = (u32)a.del_dst[i];
        hit[0] = atomicExch(a.prflag + v[0], a.ptag) != a.ptag;
      }
      n_aff += hit[0];
      enqueue(q0, a.fwd.row, v, hit, 1, n_enq);
    }
    flush_queue(q0, scratch);
  }

  if (kPushOp) {   // a batch's seeds: OnAdd, and the pull over A
    // (the cut list becomes A while OnAdd runs; the pull needs all of A)
    if (a.seed_pull) cut_to_a(a, &sa, &sas, scratch);
    if (a.n_items > 0) add_stage(a, &sq, &sqs, scratch);
    if (a.seed_pull || a.n_items > 0) {   // both stages' appends in one flush
      const Queue qa = make_queue(a.aent, a.aown, &c->acnt, a.asv, &c->ascnt, &sa, &sas);
      const Queue q0 =
          make_queue(a.qent[0], a.qown[0], &c->qcnt0, a.qsv[0], &c->scnt0, &sq, &sqs);
      flush_stages(a.seed_pull ? &qa : nullptr, a.n_items > 0 ? &q0 : nullptr, nullptr,
                   nullptr, nullptr, nullptr, scratch);
    }
    if (a.seed_pull) {
      target += gridDim.x;
      if (!grid_sync(bar, target, c, a.lim)) pull_stage(a, &sq, &sqs, scratch);
    }
  }

  // state shared by all blocks (read before the first barrier; only block 0
  // writes it back, after the last barrier)
  const u32 tag0 = ld_cg_u32(&c->epoch);
  const u32 phase0 = ld_cg_u32(&c->phase);
  const bool nf = kPushOp && a.lim.delta > 0;
  target += gridDim.x;
  RoundCounts rc;
  CountSrc csrc{qcnt_ptr(c, 0), scnt_ptr(c, 0), nf ? fcnt_ptr(c, 0) : nullptr,
                nf ? fmin_ptr(c, 0) : nullptr};
  bool stop = grid_sync(bar, target, c, a.lim, &csrc, &rc);

  u32 thresh = 0xFFFFFFFFu;
  if (nf) {
    const u32 sm = ld_cg_u32(&c->seed_min);
    thresh = sat_add(sm < kInf ? sm : 0u, a.lim.delta);
  }
  u32 cur = 0, f = 0, round = 0, splits = 0, jumps = 0, lep = 0;
  bool capped = false, jump = false;
  // after a single-block episode the loop decides on block 0's snapshot
  bool snap = false;
  u64 snap_q = 0;
  u32 snap_sn = 0, snap_fn = 0, snap_fm = 0;
  // beside the store update the subtree walk is pointer jumping only (it
  // reads the parents in s, never a store)
  if (OP == kOpInval && a.concurrent && !stop) jump = ld_cg_u32(&c->ccnt) > 0;
  for (;;) {
    if (stop || (OP == kOpInval && a.concurrent)) break;
    if (round >= a.lim.max_rounds) {
      capped = true;
      break;
    }
    const u64 q = snap ? snap_q : rc.q;
    const u32 ne = (u32)(q >> 32), nedge = (u32)q;
    const u32 nsmall = snap ? snap_sn : rc.ns;
    const bool from_snap = snap;
    snap = false;
    const u32 sgroups = (nsmall + 31) / 32;
    const u32 items = sgroups + (nedge + kChunk - 1) / kChunk;
    bool split = false;
    u32 n_far = 0;
    if (OP == kOpInval && items > 0 && a.lim.jump_round >= 0 &&
        round >= (u32)a.lim.jump_round) {
      jump = true;   // the remaining levels by pointer jumping
      break;
    }
    if (kPushOp && items > 0 && ne + nsmall <= a.lim.local_edges &&
        (u64)nedge + (u64)a.lim.small_deg * nsmall <= a.lim.local_edges) {
      // small frontier: block 0 runs rounds alone until it grows or empties
      ++lep;
      const LocalState ls = local_episode(a, lep, cur, round, thresh, f, phase0 + 1u + splits,
                                          nf, dsm, &sf, scratch);
      cur = ls.cur;
      round = ls.round;
      capped = ls.capped != 0;
      stop = ls.stop != 0;
      snap = true;
      snap_q = ls.q;
      snap_sn = ls.nsmall;
      snap_fn = ls.n_far;
      snap_fm = ls.fmin;
      n_edges += ls.n_edges;
      n_imp += ls.n_imp;
      n_enq += ls.n_enq;
      range_err |= ls.range_err;
      if (capped) break;
      continue;
    }
    if (items == 0) {
      if (nf) n_far = from_snap ? snap_fn : rc.nf;
      if (n_far == 0) break;                       // fixed point reached
      split = true;
      const u32 fm = from_snap ? snap_fm : rc.fm;
      thresh = sat_add(thresh > fm ? thresh : fm, a.lim.delta);
    }
    const u32 nxt = next3(cur);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      *(volatile u64 *)qcnt_ptr(c, next3(nxt)) = 0ull;
      *(volatile u32 *)scnt_ptr(c, next3(nxt)) = 0u;
      if (split) {
        const u32 fz = next3(next3(f));
        *(volatile u32 *)fcnt_ptr(c, fz) = 0u;
        *(volatile u32 *)fmin_ptr(c, fz) = kInf;
      }
    }
    const u32 tag = tag0 + 1u + round;
    const u32 phase = phase0 + 1u + splits;
    const Queue qn = make_queue(a.qent[nxt], a.qown[nxt], qcnt_ptr(c, nxt), a.qsv[nxt],
                                scnt_ptr(c, nxt), &sq, &sqs,
                                kPushOp ? a.lim.small_deg : (u32)kSmallDeg);
    const u32 fk = next3(f);
    if (kPushOp) {
      if (split) {
        // far entries below thresh go back to the near frontier, the rest
        // move to the next pile.  An entry whose vertex was expanded since it
        // was piled is expanded again: skipping it would need the distance
        // every chunk of that expansion used, and chunks of one vertex can
        // read different distances within a round.
        const u32 *pin = a.fq[f];
        for (u32 base = gw * 32; base < n_far; base += nw * 32) {
          const u32 i = base + lane;
          bool near[K] = {}, keep[K] = {};
          u32 x[K] = {};
          u32 kmin = 0xFFFFFFFFu;
          u32 dx[K] = {};
          if (i < n_far) {
            x[0] = __ldcg(pin + i);
            dx[0] = dist_of(ld_cg_u64(a.s + x[0]));
            if (dx[0] < kInf) {
              if (dx[0] < thresh) {
                near[0] = is_pool(OP) || atomicExch(a.qflag + x[0], tag) != tag;
              } else {
                keep[0] = true;
                a.ftag[x[0]] = phase + 1u;
                kmin = dx[0];
              }
            }
          }
          moved += near[0];
          if (is_pool(OP)) {   // into the pool; what does not fit to the frontier
            bool rest[K];
            pool_push<false>(&pool, 0, x, dx, near, 1, nullptr, nullptr, rest, pc.n_in,
                             a.fwd.row, nullptr);
            near[0] = rest[0] && atomicExch(a.qflag + x[0], tag) != tag;
          }
          enqueue(qn, a.fwd.row, x, near, 1, n_enq);
          far_append(a.fq[fk], fcnt_ptr(c, fk), fmin_ptr(c, fk), &sf, x, keep, 1, kmin);
        }
      } else {
        PushOp op{a.s, a.qflag, tag, qn, a.fwd.row, thresh,
                  nf ? a.fq[f] : nullptr, fcnt_ptr(c, f), fmin_ptr(c, f), a.ftag,
                  phase, &sf, is_pool(OP) ? &pool : nullptr};
        for (u32 it = gw; it < items; it += nw) {
          if (it < sgroups) process_small(op, a.qsv[cur], nsmall, it, a.fwd, a.n, c);
          else process_chunk(op, a.qent[cur], a.qown[cur], ne, nedge, it - sgroups, a.fwd, a.n, c);
        }
        n_edges += op.n_edges;
        n_imp += op.n_imp;
        n_enq += op.n_enq;
        pc.n_in += op.n_in;
        range_err |= op.range_err;
      }
      if (is_pool(OP)) {
        // the block relaxes what it improved below thresh before the barrier;
        // its far appends belong to the phase that follows this round's split
        const u32 fp = split ? fk : f;
        pool_drain<OP == kOpPoolWide ? 5 : 4>(a, &pool, thresh, tag, split ? phase + 1u : phase, qn,
                   nf ? a.fq[fp] : nullptr, fcnt_ptr(c, fp), fmin_ptr(c, fp), &sf, pc);
      }
    } else if (OP == kOpFlag) {
      FlagOp op{a.prflag, a.ptag, qn, a.fwd.row};
      for (u32 it = gw; it < items; it += nw) {
        if (it < sgroups) process_small(op, a.qsv[cur], nsmall, it, a.fwd, a.n, c);
        else process_chunk(op, a.qent[cur], a.qown[cur], ne, nedge, it - sgroups, a.fwd, a.n, c);
      }
      n_edges += op.n_edges;
      n_enq += op.n_enq;
      n_aff += op.n_aff;
    } else {
      InvalOp op{a.s, qn, a.fwd.row, a.cut, &c->ccnt, &c->cmin, &sf};
      for (u32 it = gw; it < items; it += nw) {
        if (it < sgroups) process_small(op, a.qsv[cur], nsmall, it, a.fwd, a.n, c);
        else process_chunk(op, a.qent[cur], a.qown[cur], ne, nedge, it - sgroups, a.fwd, a.n, c);
      }
      n_edges += op.n_edges;
      n_enq += op.n_enq;
      n_aff += op.n_aff;
    }
    // publish this block's staged appends before the barrier: the next
    // frontier and the far pile (the invalidation's: the cut list)
    if (OP == kOpInval) {
      flush_stages(&qn, nullptr, &sf, a.cut, &c->ccnt, &c->cmin, scratch);
    } else if (nf) {
      const u32 fp = split ? fk : f;
      flush_stages(&qn, nullptr, &sf, a.fq[fp], fcnt_ptr(c, fp), fmin_ptr(c, fp), scratch);
    } else {
      flush_queue(qn, scratch);
    }
    if (split) {
      f = next3(f);
      ++splits;
    }
    cur = nxt;
    ++round;
    target += gridDim.x;
    csrc = CountSrc{qcnt_ptr(c, cur), scnt_ptr(c, cur), nf ? fcnt_ptr(c, f) : nullptr,
                    nf ? fmin_ptr(c, f) : nullptr};
    stop = grid_sync(bar, target, c, a.lim, &csrc, &rc);
  }
  if (OP == kOpInval && jump) {
    const JumpState js = jump_phase(a, bar, target, scratch, &sf);
    target = js.target;
    jumps = js.jumps;
    capped = capped || js.capped != 0;
    n_aff += js.n_aff;
  }
  n_edges = warp_sum(n_edges);
  n_imp = warp_sum(n_imp);
  n_enq = warp_sum(n_enq);
  n_aff = warp_sum(n_aff);
  moved = warp_sum(moved);
  range_err = __any_sync(kFull, range_err | pc.range_err);
  if (is_pool(OP)) {
    n_edges += warp_sum(pc.n_edges);
    n_imp += warp_sum(pc.n_imp);
    n_enq += warp_sum(pc.n_enq);
    const u64 pin = warp_sum(pc.n_in);
    if (lane == 0 && pin) atomicAdd(&c->pool_in, pin);
    if (threadIdx.x == 0 && pc.subs) {
      atomicAdd(&c->pool_sub, (u64)pc.subs);
      if (blockIdx.x == 0) {
        c->pool_ns = pc.ns;
        c->pool_sub0 = pc.subs;
      }
    }
  }
  if (lane == 0) {
    if (kPushOp) {
      if (n_edges) atomicAdd(&c->relaxed, n_edges);
      if (n_imp) atomicAdd(&c->improved, n_imp);
      if (n_enq) atomicAdd(&c->enqueued, n_enq);
      if (moved) atomicAdd(&c->far_moves, moved);
    } else {
      if (n_edges) atomicAdd(&c->inval_edges, n_edges);
      if (n_aff) atomicAdd(&c->affected, n_aff);
    }
    if (range_err) atomicExch(&c->range_err, 1);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // every block has read the counters of the final round: leave the
    // frontier slots empty for the next producer and publish the tags
    volatile Ctl *vc = c;
    vc->epoch = tag0 + round + 2u;
    vc->phase = phase0 + splits + 2u;
    vc->qcnt0 = 0ull;
    vc->qcnt1 = 0ull;
    vc->qcnt2 = 0ull;
    vc->scnt0 = 0u;
    vc->scnt1 = 0u;
    vc->scnt2 = 0u;
    if (kPushOp) {
      vc->rounds_push = round;
      vc->splits = splits;
      vc->push_ns = globaltimer_ns() - t_start;
    } else {
      vc->rounds_inval = round + jumps;
      vc->jumps = jumps;
    }
    if (capped) raise_timeout(c, 1, 1, round + jumps);
  }
}

// --- pull (one pass over A) -----------------------------------------------

// Seeding stages of the push launch (block-collective).  cut_to_a: the
// invalidation's cut vertices become the affected list A, sized by their
// in-degrees in the updated reverse store (the invalidation may have run
// beside the store update, so it could not size them).  pull_stage (after a
// grid barrier): every vertex of A takes the minimum over its in-edges, and
// the improved ones join the push loop's first frontier (queue slot 0).
__device__ __forceinline__ void cut_to_a(const LoopArgs &a, Stage *sa, Stage *sas, u32 *scratch) {
  Ctl *c = a.ctl;
  const int lane = threadIdx.x & 31;
  {
    const Queue qa = make_queue(a.aent, a.aown, &c->acnt, a.asv, &c->ascnt, sa, sas);
    const u32 ncut = ld_cg_u32(&c->ccnt);
    const u32 gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const u32 nw = (gridDim.x * blockDim.x) >> 5;
    u64 dummy = 0;
    for (u32 base = gw * 32 * K; base < ncut; base += nw * 32 * K) {
      u32 v[K];
      bool want[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const u32 i = base + lane + 32 * k;
        want[k] = i < ncut;
        v[k] = want[k] ? __ldcg(a.cut + i) : 0u;
      }
      enqueue(qa, a.rev.row, v, want, K, dummy);
    }
    // published by the caller, together with OnAdd's appends
  }
}

__device__ __forceinline__ void pull_stage(const LoopArgs &a, Stage *st, Stage *sst, u32 *scratch) {
  Ctl *c = a.ctl;
  const int lane = threadIdx.x & 31;
  const u64 ac = ld_cg_u64(&c->acnt);
  const u32 ne = (u32)(ac >> 32), nedge = (u32)ac;
  const u32 nsmall = ld_cg_u32(&c->ascnt);
  const u32 sgroups = (nsmall + 31) / 32;
  const u32 items = sgroups + (nedge + kChunk - 1) / kChunk;
  const u32 tag = ld_cg_u32(&c->epoch);
  const Queue q0 =
      make_queue(a.qent[0], a.qown[0], &c->qcnt0, a.qsv[0], &c->scnt0, st, sst, a.lim.small_deg);
  PullOp op{a.s, a.qflag, tag, q0, a.fwd.row, &c->seed_min};
  const u32 gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;   // interleaved over blocks
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  for (u32 it = gw; it < items; it += nw) {
    if (it < sgroups) process_small(op, a.asv, nsmall, it, a.rev, a.n, c);
    else process_chunk(op, a.aent, a.aown, ne, nedge, it - sgroups, a.rev, a.n, c);
  }
  flush_queue(q0, scratch);
  u64 e = warp_sum(op.n_edges), q = warp_sum(op.n_enq);
  int re = __any_sync(kFull, op.range_err);
  if (lane == 0) {
    if (e) atomicAdd(&c->pull_edges, e);
    if (q) atomicAdd(&c->seeds, q);
    if (re) atomicExch(&c->range_err, 1);
  }
}

// --- OnAdd: relax every applied insertion ---------------------------------

// OnAdd stage (block-collective): every applied insertion (u, v, w) is
// relaxed; an improved v joins the push loop's first frontier (slot 0).
__device__ __forceinline__ void add_stage(const LoopArgs &a, Stage *st, Stage *sst, u32 *scratch) {
  Ctl *c = a.ctl;
  const int lane = threadIdx.x & 31;
  const u32 tag = ld_cg_u32(&c->epoch);
  const Queue q0 =
      make_queue(a.qent[0], a.qown[0], &c->qcnt0, a.qsv[0], &c->scnt0, st, sst, a.lim.small_deg);
  const u64 cmask = (1ull << a.bits) - 1;
  const long long gw = (long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  int range_err = 0;
  u64 n_enq = 0;
  // the forward-store items are the first half of the sorted batch (the
  // store bit is the key's top bit)
  const long long nfw = a.n_items / 2;
  for (long long base = gw * 32; base < nfw; base += nw * 32) {
    const long long i = base + lane;
    bool want[K] = {};
    u32 v[K] = {};
    int dg[K] = {};
    if (i < nfw) {
      const u64 key = a.keys[i];
      const unsigned char fl = a.flags[i];
      const u32 w = a.vals[i];
      const u32 u = (u32)((key >> (a.bits + 1)) & cmask);
      v[0] = (u32)((key >> 1) & cmask);
      // forward-store insertion that the merge applied
      if ((key & 1) && (fl & 1)) {
        const u64 su = ld_cg_u64(a.s + u), sv = ld_cg_u64(a.s + v[0]);
        const u32 du = dist_of(su);
        if (du < kInf) {
          const u32 nd = du + w;
          if (nd >= kInf) {
            range_err = 1;
          } else {
            const u64 cand = pack(nd, u);
            if (cand < sv) {
              // exchange and out-degree with the atomicMin (a candidate that
              // loses it lost to a smaller insertion of this stage, which
              // exchanges too)
              const u64 old = atomicMin((unsigned long long *)(a.s + v[0]), cand);
              want[0] = atomicExch(a.qflag + v[0], tag) != tag;
              dg[0] = __ldg(&a.fwd.row[v[0]].deg);
              if (cand < old) atomicMin(&c->seed_min, nd);
              if (!want[0]) dg[0] = 0;
            }
          }
        }
      }
    }
    enqueue_d(q0, v, dg, 1, n_enq);
  }
  // published by the caller, together with the cut list's
  u64 q = warp_sum(n_enq);
  int re = __any_sync(kFull, range_err);
  if (lane == 0) {
    if (q) atomicAdd(&c->seeds, q);
    if (re) atomicExch(&c->range_err, 1);
  }
}

// --- from-scratch init, unpack ----------------------------------------------

__global__ void k_init(u64 *s, int n, int src, Ctl *c, u32 *qflag, int2 *qent, u32 *qown,
                       u32 *qsv, const RowMeta *row) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    s[v] = v == src ? pack(0, kNoParent) : kInfPack;
  if (src >= 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    qflag[src] = c->epoch;
    const int d = row[src].deg;
    if (d > kSmallDeg) {
      qent[0] = make_int2(src, 0);
      for (u32 ch = 0; ch <= (u32)(d - 1) / kChunk; ++ch) qown[ch] = 0;
      c->qcnt0 = (1ull << 32) | (u64)d;
    } else if (d > 0) {
      qsv[0] = (u32)src;
      c->scnt0 = 1;
    }
    c->seeds = 1;
    c->seed_min = 0;
  }
}

// Multi-source init, second step (after every state is INF): each source
// gets distance 0 and parent -1 and joins the first frontier once.
__global__ void k_seed_sources(u64 *s, const int *src, int k, Ctl *c, u32 *qflag, int2 *qent,
                               u32 *qown, u32 *qsv, const RowMeta *row) {
  const Queue q0 = make_queue(qent, qown, &c->qcnt0, qsv, &c->scnt0);
  const u32 tag = ld_cg_u32(&c->epoch);
  u64 n_enq = 0;
  for (int base = blockIdx.x * blockDim.x; base < k; base += gridDim.x * blockDim.x) {
    const int i = base + (int)threadIdx.x;
    bool want[K] = {};
    u32 v[K] = {};
    if (i < k) {
      v[0] = (u32)src[i];
      s[v[0]] = pack(0, kNoParent);
      want[0] = atomicExch(qflag + v[0], tag) != tag;
    }
    enqueue(q0, row, v, want, 1, n_enq);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->seed_min = 0;
    c->seeds = (u64)k;
  }
}

__global__ void k_gather_dist(const u64 *__restrict__ s, int n, const int *__restrict__ vs, int k,
                              int *out, Ctl *c) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const int v = vs[i];
    if (v >= 0 && v < n) out[i] = (int)dist_of(s[v]);
    else atomicCAS(&c->status, 0, SP_EINVAL);
  }
}

// Distances (and parents) out of the packed state.  Four vertices per thread
// with 16-byte stores when the outputs are 16-byte aligned (fewer, larger
// transactions when they are host memory written across the host link).
__global__ void k_unpack(const u64 *__restrict__ s, int n, int *dist, int *parent) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  const bool vec = ((((unsigned long long)dist) | ((unsigned long long)parent)) & 15) == 0;
  const long long nv = vec ? n / 4 : 0;
  for (long long i = tid; i < nv; i += nt) {
    const ulonglong2 x0 = __ldg((const ulonglong2 *)s + 2 * i);
    const ulonglong2 x1 = __ldg((const ulonglong2 *)s + 2 * i + 1);
    ((int4 *)dist)[i] = make_int4((int)dist_of(x0.x), (int)dist_of(x0.y), (int)dist_of(x1.x),
                                  (int)dist_of(x1.y));
    if (parent)
      ((int4 *)parent)[i] = make_int4((int)parent_of(x0.x), (int)parent_of(x0.y),
                                      (int)parent_of(x1.x), (int)parent_of(x1.y));
  }
  for (long long v = 4 * nv + tid; v < n; v += nt) {
    const u64 x = s[v];
    dist[v] = (int)dist_of(x);
    if (parent) parent[v] = (int)parent_of(x);
  }
}

// --- restoring exported distances -----------------------------------------
//
// A (dist, parent) pair exported by sp_get_dist is installed again only if
// it is the exact shortest-path solution of the current edge set from
// `src`: dist[src] = 0 with parent -1; every other finite dist[v] has a
// parent p with an edge p -> v of weight dist[v] - dist[p] (w >= 1 makes
// the parent chains strictly decreasing, so they are acyclic and end at the
// source: every finite distance is realised by a path); every infinite one
// has parent -1; and no edge u -> x offers dist[u] + w < dist[x].  Together
// these say that dist equals the shortest-path distances (the problem of
// Section 3.2), so a restore gives the same answer as a recompute.  A
// violation sets the status (SP_EINVAL) and nothing is installed.

__global__ void k_state_vertices(const int *__restrict__ dist, const int *__restrict__ parent,
                                 int n, int src, Store fwd, Ctl *c) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int d = dist[v], p = parent[v];
    bool ok;
    if (v == src) {
      ok = d == 0 && p == -1;
    } else if (d < 0 || d > (int)kInf) {
      ok = false;
    } else if (d == (int)kInf) {
      ok = p == -1;
    } else if (p < 0 || p >= n || p == (int)v) {
      ok = false;
    } else {
      const int dp = dist[p];
      ok = false;
      if (dp >= 0 && dp < d) {   // the parent edge p -> v: a search in p's sorted row
        const RowMeta rm = fwd.row[p];
        long long lo = rm.start, hi = rm.start + rm.deg;
        while (lo < hi) {
          const long long mid = (lo + hi) >> 1;
          if (__ldg(&fwd.adj[mid].x) < (int)v) lo = mid + 1; else hi = mid;
        }
        ok = lo < rm.start + rm.deg && __ldg(&fwd.adj[lo].x) == (int)v &&
             (long long)dp + __ldg(&fwd.adj[lo].y) == (long long)d;
      }
    }
    if (!ok) atomicCAS(&c->status, 0, SP_EINVAL);
  }
}

// Every edge: no shorter way into its head (one warp per row).
__global__ void k_state_edges(const int *__restrict__ dist, int n, Store fwd, Ctl *c) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  for (long long u = w0; u < n; u += nw) {
    const int du = dist[u];
    if (du >= (int)kInf) continue;
    const RowMeta rm = fwd.row[u];
    for (int e = lane; e < rm.deg; e += 32) {
      const int2 ed = __ldg(&fwd.adj[rm.start + e]);
      if ((long long)du + ed.y < (long long)dist[ed.x]) bad = true;
    }
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicCAS(&c->status, 0, SP_EINVAL);
}

__global__ void k_state_pack(const int *__restrict__ dist, const int *__restrict__ parent,
                             int n, u64 *s) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    s[v] = pack((u32)dist[v], (u32)parent[v]);
}

// --- PageRank (appendix listing "Dynamic PR") ---------------------------------

// Select the vertices of a Jacobi phase into the list A (entries over the
// reverse store): every vertex (staticPR) or those flagged in this phase.
// Selected vertices without in-edges go to a plain list (zlist, zcnt): their
// new rank is the constant term.
__global__ void __launch_bounds__(kLoopThreads) k_pr_select(LoopArgs a, int all) {
  __shared__ u32 sv[kStageK], sd[kStageK], ssv[kStageK];
  __shared__ Stage st, sst;
  __shared__ u32 scratch[40];
  Ctl *c = a.ctl;
  if (!repair_enabled(c)) return;
  if (threadIdx.x == 0) {
    st.n = 0; st.cap = kStageK; st.vmin = kInf; st.v = sv; st.d = sd;
    sst.n = 0; sst.cap = kStageK; sst.vmin = kInf; sst.v = ssv; sst.d = nullptr;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const Queue qa = make_queue(a.aent, a.aown, &c->acnt, a.asv, &c->ascnt, &st, &sst);
  u64 dummy = 0;
  const u32 n = (u32)a.n;
  const u32 step = gridDim.x * blockDim.x;
  for (u32 base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += step) {
    const u32 v = base + lane;
    bool want[K] = {};
    u32 x[K] = {};
    x[0] = v;
    if (v < n) want[0] = all || __ldcg(a.prflag + v) == a.ptag;
    const bool z = want[0] && __ldg(&a.rev.row[v].deg) == 0;
    const u32 bal = __ballot_sync(kFull, z);
    if (bal) {
      u32 zb = 0;
      if (lane == 0) zb = atomicAdd(&c->zcnt, (u32)__popc(bal));
      zb = __shfl_sync(kFull, zb, 0);
      if (z) a.jmp[zb + __popc(bal & lanemask_lt())] = v;
    }
    enqueue(qa, a.rev.row, x, want, 1, dummy);
  }
  flush_queue(qa, scratch);
}

__global__ void k_pr_fill(float *p0, float *p1, float *acc, int n, float value) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    p0[v] = value;
    p1[v] = value;
    acc[v] = 0.0f;
  }
}

// Pull body of a Jacobi step: each lane adds the terms pr[u] / outdeg(u)
// (kept per vertex in `contrib`, rounded exactly as a division per edge
// would be) over its run of in-edges u -> v in slot order and adds the run's
// sum to acc[v].  A vertex with at most kSmallDeg in-edges is one lane's
// single run, so its sum is formed in in-neighbour order, as a sequential
// loop would.
struct PrOp {
  const float *contrib;
  float *acc;
  u64 n_edges = 0, n_enq = 0;
  int range_err = 0;

  __device__ __forceinline__ u32 vdata(u32) { return 0; }
  __device__ __forceinline__ u64 load(int2 e) { return __float_as_uint(__ldcg(contrib + e.x)); }
  __device__ __forceinline__ void run(const bool *act, const u32 *ov, const u32 *,
                                      const int2 *, const u64 *sx) {
    u32 bv = kNoEdge;
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (act[k]) {
        ++n_edges;
        if (ov[k] != bv) {
          if (bv != kNoEdge) atomicAdd(acc + bv, sum);
          bv = ov[k];
          sum = 0.0f;
        }
        sum = __fadd_rn(sum, __uint_as_float((u32)sx[k]));
      }
    }
    if (bv != kNoEdge) atomicAdd(acc + bv, sum);
  }
};

struct PrArgs {
  LoopArgs la;
  float *pr[2];
  float *contrib[2];   // pr / outdeg, kept beside each rank buffer
  float *acc;
  float base, damping;
  double beta;
  int max_iter;
};

// Jacobi steps over the list A (persistent, cooperative): pass 1 pulls the
// in-edge sums into acc, pass 2 forms pr' = base + damping * acc, adds
// |pr' - pr| to the step's difference and clears acc; a step ends when the
// difference is at most beta or max_iter steps have run.  The result is left
// in both rank buffers.
__device__ __forceinline__ double *prd_ptr(Ctl *c, u32 b) {
  return b == 0 ? &c->prd0 : (b == 1 ? &c->prd1 : &c->prd2);
}

__global__ void __launch_bounds__(kPersistThreads, 1) k_pr(PrArgs p) {
  const LoopArgs &a = p.la;
  Ctl *c = a.ctl;
  if (!repair_enabled_block(c)) return;
  __shared__ double s_sum[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const u32 nw = (gridDim.x * blockDim.x) >> 5;
  const u64 ac = ld_cg_u64(&c->acnt);
  const u32 ne = (u32)(ac >> 32), nedge = (u32)ac;
  const u32 ns = ld_cg_u32(&c->ascnt);
  const u32 nz = ld_cg_u32(&c->zcnt);
  const u32 sgroups = (ns + 31) / 32;
  const u32 items = sgroups + (nedge + kChunk - 1) / kChunk;
  u64 *bar = &c->bar_push;
  u64 target = 0;
  u64 n_edges = 0;
  u32 it = 0, cur = 0;
  bool stop = false;
  {
    // the terms of every vertex (out-degrees may have changed since the
    // last phase); both rank buffers agree here
    const u32 gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (u32 v = gt; v < (u32)a.n; v += nt) {
      const int deg = __ldg(&a.fwd.row[v].deg);
      const float t = deg > 0 ? __fdiv_rn(__ldcg(p.pr[0] + v), (float)deg) : 0.0f;
      p.contrib[0][v] = t;
      p.contrib[1][v] = t;
    }
    target += gridDim.x;
    stop = grid_sync(bar, target, c, a.lim);
  }
  for (;;) {
    if (stop) break;
    // pass 1: in-edge sums
    PrOp op{p.contrib[cur], p.acc};
    for (u32 i = gw; i < items; i += nw) {
      if (i < sgroups) process_small(op, a.asv, ns, i, a.rev, a.n, c);
      else process_chunk(op, a.aent, a.aown, ne, nedge, i - sgroups, a.rev, a.n, c);
    }
    n_edges += op.n_edges;
    target += gridDim.x;
    stop = grid_sync(bar, target, c, a.lim);
    if (stop) break;
    // pass 2: new ranks and the step's difference
    const float *pc = p.pr[cur];
    float *pn = p.pr[cur ^ 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) *(volatile double *)prd_ptr(c, (it + 1) % 3) = 0.0;
    double diff = 0.0;
    const u32 gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (u32 i = gt; i < ns + ne + nz; i += nt) {
      const u32 v = i < ns ? __ldcg(a.asv + i)
                           : (i < ns + ne ? (u32)__ldcg(&a.aent[i - ns].x) : __ldcg(a.jmp + (i - ns - ne)));
      const float val = __fadd_rn(p.base, __fmul_rn(p.damping, __ldcg(p.acc + v)));
      diff += fabs((double)val - (double)__ldcg(pc + v));
      pn[v] = val;
      const int deg = __ldg(&a.fwd.row[v].deg);
      p.contrib[cur ^ 1][v] = deg > 0 ? __fdiv_rn(val, (float)deg) : 0.0f;
      p.acc[v] = 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) diff += __shfl_xor_sync(kFull, diff, o);
    if (lane == 0) s_sum[warp] = diff;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_sum[w];
      if (t != 0.0) atomicAdd(prd_ptr(c, it % 3), t);
    }
    target += gridDim.x;
    stop = grid_sync(bar, target, c, a.lim);
    if (stop) break;
    const double d = *(volatile double *)prd_ptr(c, it % 3);
    ++it;
    cur ^= 1;
    if (!(d > p.beta) || it >= (u32)p.max_iter) break;
  }
  // leave the result in both buffers
  if (!stop) {
    const float *src = p.pr[cur];
    float *dst = p.pr[cur ^ 1];
    const u32 gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    for (u32 i = gt; i < ns + ne + nz; i += nt) {
      const u32 v = i < ns ? __ldcg(a.asv + i)
                           : (i < ns + ne ? (u32)__ldcg(&a.aent[i - ns].x) : __ldcg(a.jmp + (i - ns - ne)));
      dst[v] = __ldcg(src + v);
    }
  }
  n_edges = warp_sum(n_edges);
  if (lane == 0 && n_edges) atomicAdd(&c->pull_edges, n_edges);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    volatile Ctl *vc = c;
    vc->pr_iters = it;
    vc->rounds_push = it;
    vc->acnt = 0ull;
    vc->ascnt = 0u;
    vc->zcnt = 0u;
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
  for (int b = 0; b < 3; ++b) {
    a.qent[b] = g->qent[b];
    a.qown[b] = g->qown[b];
    a.qsv[b] = g->qsv[b];
    a.fq[b] = g->fq[b];
  }
  a.asv = g->asv;
  a.aent = g->aent;
  a.aown = g->aown;
  a.ftag = g->ftag;
  a.jmp = g->jmp;
  a.n = g->n;
  a.del_src = nullptr;
  a.del_dst = nullptr;
  a.n_del = 0;
  a.prflag = g->prflag;
  a.ptag = g->prtag;
  a.cut = g->cut;
  a.concurrent = 0;
  a.seed_pull = 0;
  a.keys = g->bb.keys;
  a.vals = g->bb.vals_alt;   // the batch's weights in sorted order (the count pass's)
  a.flags = g->bb.flags;
  a.n_items = 0;
  a.bits = g->bits;
  return a;
}

}  // namespace

int loop_blocks(int which, int num_sms) {
  int per_sm = 0;
  const void *fn = which == kOpPush       ? (const void *)k_loop<kOpPush>
                   : which == kOpInval    ? (const void *)k_loop<kOpInval>
                   : which == kOpPool     ? (const void *)k_loop<kOpPool>
                   : which == kOpPoolWide ? (const void *)k_loop<kOpPoolWide>
                                          : (const void *)k_loop<kOpFlag>;
  const size_t smem = is_pool(which) ? kLoopSmemPool : kLoopSmem;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, fn, is_pool(which) ? kPoolThreads : kPersistThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return 0;
  return per_sm * num_sms;
}

void launch_init_multi(sp_graph *g, const int *src_d, int k, int *launches) {
  k_init<<<(unsigned)std::max(1, g->num_sms * 8), 256, 0, g->stream>>>(
      g->s, g->n, -1, g->ctl, g->qflag, g->qent[0], g->qown[0], g->qsv[0], g->fwd.row);
  k_seed_sources<<<(unsigned)std::max(1, (k + 255) / 256), 256, 0, g->stream>>>(
      g->s, src_d, k, g->ctl, g->qflag, g->qent[0], g->qown[0], g->qsv[0], g->fwd.row);
  *launches += 2;
}

void launch_init(sp_graph *g, int source, int *launches) {
  k_init<<<(unsigned)std::max(1, g->num_sms * 8), 256, 0, g->stream>>>(
      g->s, g->n, source, g->ctl, g->qflag, g->qent[0], g->qown[0], g->qsv[0], g->fwd.row);
  ++*launches;
}

// Blocks of a persistent loop; an invalidation beside the store update
// takes a quarter of the SMs and leaves the rest to the count and merge.
static int loop_grid(const sp_graph *g, int op, int concurrent) {
  int blocks = op == kOpPush   ? g->loop_blocks_push
               : is_pool(op)   ? g->loop_blocks_pool
                               : g->loop_blocks_inval;
  if (g->loop_blocks_user > 0 && g->loop_blocks_user < blocks) blocks = g->loop_blocks_user;
  if (concurrent) blocks = std::max(1, std::min(blocks, g->num_sms / 4));
  return blocks;
}

static cudaError_t launch_loop(sp_graph *g, int op, LoopArgs &a, int *launches,
                               cudaStream_t stream) {
  const int blocks = loop_grid(g, op, a.concurrent);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(is_pool(op) ? kPoolThreads : kPersistThreads);
  cfg.dynamicSmemBytes = is_pool(op) ? kLoopSmemPool : kLoopSmem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++*launches;
  if (op == kOpPush) return cudaLaunchKernelEx(&cfg, k_loop<kOpPush>, a);
  if (op == kOpPool) return cudaLaunchKernelEx(&cfg, k_loop<kOpPool>, a);
  if (op == kOpPoolWide) return cudaLaunchKernelEx(&cfg, k_loop<kOpPoolWide>, a);
  if (op == kOpInval) return cudaLaunchKernelEx(&cfg, k_loop<kOpInval>, a);
  return cudaLaunchKernelEx(&cfg, k_loop<kOpFlag>, a);
}

const void *inval_fn() { return (const void *)k_loop<kOpInval>; }

int inval_beside_blocks(const sp_graph *g) { return loop_grid(g, kOpInval, 1); }

cudaError_t retarget_inval(sp_graph *g, cudaGraphExec_t ex, cudaGraphNode_t node, const int *ds,
                           const int *dd, long long nd, int concurrent) {
  LoopArgs a = make_args(g);
  a.del_src = ds;
  a.del_dst = dd;
  a.n_del = nd;
  a.concurrent = concurrent;
  const int blocks = loop_grid(g, kOpInval, concurrent);
  void *args[1] = {&a};
  cudaKernelNodeParams p = {};
  p.func = (void *)k_loop<kOpInval>;
  p.gridDim = dim3((unsigned)blocks);
  p.blockDim = dim3(kPersistThreads);
  p.sharedMemBytes = (unsigned)kLoopSmem;
  p.kernelParams = args;
  return cudaGraphExecKernelNodeSetParams(ex, node, &p);
}

cudaError_t launch_inval(sp_graph *g, const int *ds, const int *dd, long long nd, int *launches,
                         int concurrent, cudaStream_t stream) {
  LoopArgs a = make_args(g);
  a.del_src = ds;
  a.del_dst = dd;
  a.n_del = nd;
  a.concurrent = concurrent;
  return launch_loop(g, kOpInval, a, launches, concurrent && stream ? stream : g->stream);
}

cudaError_t launch_push(sp_graph *g, int *launches, int pull, long long n_items) {
  LoopArgs a = make_args(g);
  a.seed_pull = pull;
  a.n_items = n_items;
  // pool entries carry a row's start / 4 in 32 bits
  if (g->fwd.slots >= (1LL << 34)) a.lim.pool_rounds = 0;
  // a single-block round covers kLocalUnroll edges per thread
  if (a.lim.pool_rounds > 0)
    a.lim.local_edges = std::min<u32>(a.lim.local_edges, (u32)(kLocalUnroll * kPoolThreads));
  const int op = a.lim.pool_rounds == 0 ? kOpPush : g->pool_wide ? kOpPoolWide : kOpPool;
  return launch_loop(g, op, a, launches, g->stream);
}

// Vertices whose out-degree is 5..8 (the share that picks the pool kernel),
// into ctl->deg_mid (zeroed by the control reset).
__global__ void k_deg_mid(const RowMeta *__restrict__ row, int n, Ctl *c) {
  u64 k = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const int d = row[v].deg;
    k += d >= 5 && d <= 8;
  }
  k = warp_sum(k);
  if ((threadIdx.x & 31) == 0 && k) atomicAdd((unsigned long long *)&c->deg_mid, k);
}

void launch_deg_mid(sp_graph *g, int *launches) {
  k_deg_mid<<<(unsigned)std::max(1, g->num_sms * 4), 256, 0, g->stream>>>(g->fwd.row, g->n, g->ctl);
  ++*launches;
}

bool pool_wide_for(long long deg_mid, int n) { return deg_mid * kPoolWideShare >= (long long)n; }

void launch_gather(sp_graph *g, const int *vs_d, int k, int *out_d, int *launches) {
  k_gather_dist<<<(unsigned)std::max(1, std::min(g->num_sms * 4, (k + 255) / 256)), 256, 0,
                  g->stream>>>(g->s, g->n, vs_d, k, out_d, g->ctl);
  ++*launches;
}

cudaError_t launch_flag(sp_graph *g, const int *dst, long long n, int *launches) {
  LoopArgs a = make_args(g);
  a.del_dst = dst;
  a.n_del = n;
  return launch_loop(g, kOpFlag, a, launches, g->stream);
}

void launch_pr_fill(sp_graph *g, float value, int *launches) {
  k_pr_fill<<<(unsigned)std::max(1, g->num_sms * 8), 256, 0, g->stream>>>(
      g->pr[0], g->pr[1], g->pracc, g->n, value);
  ++*launches;
}

void launch_pr_select(sp_graph *g, int all, int *launches) {
  LoopArgs a = make_args(g);
  k_pr_select<<<(unsigned)std::max(1, g->num_sms), kLoopThreads, 0, g->stream>>>(a, all);
  ++*launches;
}

cudaError_t launch_pr(sp_graph *g, int *launches) {
  PrArgs p;
  p.la = make_args(g);
  p.pr[0] = g->pr[0];
  p.pr[1] = g->pr[1];
  p.contrib[0] = g->prc[0];
  p.contrib[1] = g->prc[1];
  p.acc = g->pracc;
  p.base = (1.0f - g->pr_damping) / (float)g->n;
  p.damping = g->pr_damping;
  p.beta = (double)g->pr_beta;
  p.max_iter = g->pr_max_iter;
  int blocks = g->num_sms;
  if (g->loop_blocks_user > 0 && g->loop_blocks_user < blocks) blocks = g->loop_blocks_user;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = g->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++*launches;
  return cudaLaunchKernelEx(&cfg, k_pr, p);
}

void launch_state_check(sp_graph *g, const int *dist_d, const int *parent_d, int src,
                        int *launches) {
  const unsigned grid = (unsigned)std::max(1, g->num_sms * 8);
  k_state_vertices<<<grid, 256, 0, g->stream>>>(dist_d, parent_d, g->n, src, g->fwd, g->ctl);
  k_state_edges<<<grid, 256, 0, g->stream>>>(dist_d, g->n, g->fwd, g->ctl);
  *launches += 2;
}

void launch_state_pack(sp_graph *g, const int *dist_d, const int *parent_d, int *launches) {
  k_state_pack<<<(unsigned)std::max(1, g->num_sms * 8), 256, 0, g->stream>>>(dist_d, parent_d,
                                                                            g->n, g->s);
  ++*launches;
}

void launch_unpack(sp_graph *g, int *dist_d, int *parent_d, int *launches) {
  k_unpack<<<(unsigned)std::max(1, g->num_sms * 8), 256, 0, g->stream>>>(g->s, g->n, dist_d,
                                                                        parent_d);
  ++*launches;
}

}  // namespace sp
