// sp_internal.cuh -- device data layout and helpers shared by libsp's
// translation units.  Nothing here is part of the ABI (include/sp.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sp.h"

namespace sp {

typedef unsigned long long u64;
typedef unsigned int u32;

// ---------------------------------------------------------------------------
// Packed per-vertex state: s[v] = dist << 32 | (u32)parent.
// A 64-bit atomicMin on the packed word realises the paper's
// <dist, parent> = <Min(dist, cand), v> multi-assignment (Incremental listing,
// Section 3.3) as one atomic, so a parent always belongs to the distance
// stored next to it.  Ties on distance pick the smaller parent id.
// ---------------------------------------------------------------------------
constexpr u32 kInf = SP_INF;                     // INT_MAX/2
constexpr u32 kNoParent = 0xFFFFFFFFu;           // parent -1
constexpr u64 kInfPack = ((u64)kInf << 32) | kNoParent;

__host__ __device__ __forceinline__ u64 pack(u32 d, u32 p) {
  return ((u64)d << 32) | (u64)p;
}
__host__ __device__ __forceinline__ u32 dist_of(u64 s) { return (u32)(s >> 32); }
__host__ __device__ __forceinline__ u32 parent_of(u64 s) { return (u32)s; }

// ---------------------------------------------------------------------------
// Slack CSR.  Row r owns two regions of cap slots: the active one,
// adj[start, start+cap), whose first deg slots hold (col, w) pairs sorted by
// col, and an alternate one at alt[r].  A batch merge reads the active region
// and writes the alternate one, then the two swap roles.  Row regions start
// at multiples of 4 slots (32 B, one DRAM sector).  Rows that outgrow their
// capacity move to a fresh pair of regions in the spare pool at the end of
// adj.
struct __align__(16) RowMeta {
  long long start;
  int deg;
  int cap;
};

struct Store {
  RowMeta *row = nullptr;   // [n]
  long long *alt = nullptr; // [n] start of each row's alternate region
  int2 *adj = nullptr;      // [slots]  (x = col, y = w)
  long long main_slots = 0; // end of the per-row region
  long long slots = 0;      // total = main + pool
};

// ---------------------------------------------------------------------------
// Control block in device memory.  One per graph; the host reads it back at
// the end of every call (one small D2H copy).
// ---------------------------------------------------------------------------
enum : int {
  kGrowPoolFwd = 1,
  kGrowPoolRev = 2,
};

// Fields that many SMs hit at once (barrier words, queue counters) sit on
// cache lines of their own so that polling one does not slow the others.
struct Ctl {
  int status;            // sp_status of the running call (0 = ok)
  int need_grow;         // kGrow* bits: a buffer was too small, nothing changed
  int range_err;         // a candidate distance reached SP_INF
  int timeout;           // 1 = round cap, 2 = barrier wait bound
  int bad;               // an internal bounds check failed (write skipped)
  u32 to_site;           // the wait that raised timeout: 1 round cap, 2 loop barrier,
                         // 3 single-block episode, 4 batch-sort barrier
  u32 to_info;           // its round, barrier index or episode
  // grid barriers of the two persistent loops (monotone arrival counts)
  alignas(128) u64 bar_inval;
  alignas(128) u64 bar_push;
  alignas(128) u64 bar_sort;       // the batch sort's grid barrier
  alignas(128) u64 bar_count;      // the count pass's grid barrier
  // loop bookkeeping shared across launches
  alignas(128) u32 epoch;          // dedupe tag of the last frontier built
  u32 phase;                       // far dedupe tag of the last phase
  u32 call;                        // call id (tags the per-vertex expanded distance)
  // frontier counters (atomics), triple-buffered: count << 32 | edges
  alignas(128) u64 qcnt0;
  alignas(128) u64 qcnt1;
  alignas(128) u64 qcnt2;
  alignas(128) u64 acnt;           // affected list A (reverse-store edges)
  // small-degree lists (one lane per vertex), triple-buffered, and A's
  alignas(128) u32 scnt0;
  alignas(128) u32 scnt1;
  alignas(128) u32 scnt2;
  alignas(128) u32 ascnt;
  // far piles of the near-far push, triple-buffered
  alignas(128) u32 fcnt0;
  alignas(128) u32 fcnt1;
  alignas(128) u32 fcnt2;
  alignas(128) u32 fmin0;
  alignas(128) u32 fmin1;
  alignas(128) u32 fmin2;
  alignas(128) u32 seed_min;       // smallest distance seeded into the push
  // single-block rounds of the push loop: episodes ended by block 0 (the
  // other blocks wait for it), the loop state it hands back, its heartbeat
  alignas(128) u32 lres;
  u32 lcur, lround, lcap;
  u64 lbeat;
  // what the loop decides on after an episode, as block 0 left it: the
  // counters of the current frontier slot and of the current far pile
  u64 lq;
  u32 lsn, lfn, lfm;
  // PageRank: sum |pr' - pr| of each Jacobi step (rotating) and the steps run
  alignas(128) double prd0;
  alignas(128) double prd1;
  alignas(128) double prd2;
  u32 pr_iters;
  u32 zcnt;              // selected vertices without in-edges (PageRank)
  // triangle count: staticTC, and the sightings of the deletions' and the
  // insertions' corrections by number of updated edges (1, 2, 3)
  alignas(128) u64 tc_static;
  u64 tc_del[3], tc_ins[3];
  // the invalidation's cut vertices (a plain list: the pull stage of the
  // push launch turns them into the affected list A)
  alignas(128) u32 ccnt;
  u32 cmin;              // unused minimum of the cut list's appends
  // vertices still jumping after each pointer-jumping pass, triple-buffered
  alignas(128) u32 jcnt0;
  alignas(128) u32 jcnt1;
  alignas(128) u32 jcnt2;
  // batch bookkeeping
  alignas(128) u64 mcnt;           // merge elements: segments << 32 | elements
  alignas(128) u32 bstrips;        // 256-entry strips of big rows
  alignas(128) u32 mpos;           // strips handed out by the merge so far
  alignas(128) u32 sstrips;        // small rows, merged eight to a warp
  alignas(128) u32 spos;           // groups of small rows handed out so far
  alignas(128) u32 n_seg;          // touched (dir,row) segments
  u64 pool_used[2];      // spare slots taken (fwd, rev), persistent
  u64 pool_need[2];      // demand seen by the last count pass
  // counters of the call
  alignas(128) u64 del_applied;
  u64 del_absent, add_applied, add_present;
  u64 affected, seeds, relaxed, improved, rows_touched, rows_relocated;
  u64 inval_edges, pull_edges, push_vertices, enqueued;
  u64 merge_slots;       // old + new slots of all merged rows
  u64 far_moves;         // far-pile entries moved back to near
  u32 rounds_inval, rounds_push, splits;
  u32 local_episodes, local_rounds, jumps;
  u64 local_ns, push_ns;   // block 0's time in single-block rounds / in the push loop
  u64 pool_sub;            // block-local sub-rounds, summed over blocks
  u64 pool_in;             // entries appended to the block pools
  u64 pool_ns;             // block 0's time in block-local sub-rounds
  u64 pool_sub0;           // block 0's block-local sub-rounds
  u64 deg_mid;             // vertices with 5..8 out-edges, when the call counts them
};

// Launch-time limits and knobs.
struct Limits {
  u32 max_rounds;        // per fixedPoint loop
  u64 wait_ns;           // per barrier wait
  u32 delta;             // near-far bucket width of the push loop (0 = off)
  u32 local_edges;       // push rounds with at most this many frontier edges
                         // run in one block (0 = never)
  int jump_round;        // frontier rounds of the invalidation before it
                         // switches to pointer jumping (< 0: never)
  u32 small_deg;         // push frontiers: vertices with at most this many
                         // out-edges are expanded one lane each, larger ones
                         // as edge chunks spread over warps
  u32 pool_rounds;       // block-local relaxation: block sub-rounds per push
                         // round (0 = off, plain frontier rounds)
  u32 miss_site;         // test hook: block 0 does not arrive at the grid
                         // barriers of this wait site (0 = none), so that
                         // their bounded waits run out
};

// Every barrier wait also ends after this many polls, whatever the clock
// says (a poll sleeps 64 ns and reads one word: seconds in all).
constexpr u32 kMaxPolls = 1u << 24;

// ---------------------------------------------------------------------------
// Small device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 ld_cg_u64(const u64 *p) {
  return __ldcg((const unsigned long long *)p);
}
__device__ __forceinline__ u32 ld_cg_u32(const u32 *p) { return __ldcg(p); }
__device__ __forceinline__ int ld_cg_i32(const int *p) { return __ldcg(p); }

__device__ __forceinline__ u32 ld_acquire_u32(const u32 *p) {
  u32 v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(u32 *p, u32 v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Raise the call's timeout (kind 1 = a cap, 2 = a wait bound) and, for
// the first raiser only, record where it happened.
__device__ __forceinline__ void raise_timeout(Ctl *c, int kind, u32 site, u32 info) {
  if (atomicCAS(&c->timeout, 0, kind) == 0) {
    c->to_site = site;
    c->to_info = info;
  }
}

__device__ __forceinline__ u64 globaltimer_ns() {
  u64 t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ u64 ld_acquire_u64_(const u64 *p) {
  u64 v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch on a monotone arrival count (zeroed
// when the call starts): barrier k waits for k * gridDim.x arrivals.  Used by
// the batch sort (site 4) and the count pass (site 5), which run before the
// merge changes anything.  A wait is bounded by wait_ns (and kMaxPolls); the
// first one that runs out sets the call's status to SP_ETIMEOUT and records
// its site (over a loop's earlier record: the site then says that the store
// update stopped, and the edge set is as it was).  Every wait also ends when
// the status is set (the kernel's other blocks failed, or the batch was
// invalid), so all blocks leave together.  A timeout of another kernel (the
// invalidation beside the store update) does not stop these barriers.
// Returns whether the kernel must stop, the same in every thread.
__device__ __forceinline__ bool coop_barrier(u64 *bar, u64 target, Ctl *c, u64 wait_ns,
                                             u32 site, u32 miss_site = 0) {
  __shared__ int s_stop;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    // the count before this arrival says whether it was the last one; the
    // wait polls the count alone and looks at the status and the clock every
    // 16th poll.  (miss_site: block 0 does not arrive, and every wait of the
    // barrier runs out.)
    const bool miss = miss_site == site && blockIdx.x == 0;
    const u64 arrived = miss ? ld_acquire_u64_(bar) : atomicAdd((unsigned long long *)bar, 1ull) + 1;
    if (arrived < target) {
      const u64 t0 = globaltimer_ns();
      u32 polls = 0;
      while (ld_acquire_u64_(bar) < target) {
        if ((++polls & 15u) == 0) {
          if (ld_cg_i32(&c->status) != 0) break;
          if (globaltimer_ns() - t0 > wait_ns || polls > kMaxPolls) {
            if (atomicCAS(&c->status, 0, SP_ETIMEOUT) == 0) {
              atomicExch(&c->timeout, 2);
              c->to_site = site;
              c->to_info = (u32)(target / gridDim.x);
            }
            break;
          }
        }
        __nanosleep(64);
      }
    }
    s_stop = ld_cg_i32(&c->status) != 0;
  }
  __syncthreads();
  return s_stop != 0;
}

__device__ __forceinline__ u32 lanemask_lt() {
  u32 m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__host__ __device__ __forceinline__ long long round_up4(long long x) {
  return (x + 3) & ~3LL;
}

// Capacity given to a row of `deg` edges: deg plus max(slack*deg, 4) spare
// slots, rounded up to a multiple of 4.
__host__ __device__ __forceinline__ int row_capacity(long long deg, float slack) {
  long long extra = (long long)(slack * (float)deg + 0.999f);
  if (extra < 4) extra = 4;
  return (int)round_up4(deg + extra);
}

// Number of bits needed for vertex ids in [0, n).
__host__ __device__ __forceinline__ int id_bits(long long n) {
  int b = 1;
  while ((1LL << b) < n) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// Host-side helpers implemented in the .cu files.
// ---------------------------------------------------------------------------
struct Alloc {
  sp_allocator user{};
  bool has_user = false;
  cudaStream_t stream = nullptr;
  long long bytes_held = 0;
  void *get(size_t bytes);
  void put(void *p, size_t bytes);
};

// Device-wide exclusive scans (sp_scan.cu).  `tmp` needs scan_tmp_bytes(n).
size_t scan_tmp_bytes(long long n);
void scan_exclusive_u32(const u32 *in, u32 *out, long long n, void *tmp,
                        cudaStream_t st, int *launches);
void scan_exclusive_u64(const u64 *in, u64 *out, long long n, void *tmp,
                        cudaStream_t st, int *launches);

// LSD radix sort of (u64 key, u32 value) pairs on the low `key_bits` bits
// (sp_sort.cu).  Sorts keys/vals in place using alt buffers of the same size
// and `tmp` of sort_tmp_bytes(n).  Stable.
size_t sort_tmp_bytes(long long n);
void sort_pairs(u64 *keys, u32 *vals, u64 *keys_alt, u32 *vals_alt, long long n,
                int key_bits, void *tmp, cudaStream_t st, int *launches);

}  // namespace sp
