// sp_store.cu -- the slack CSR: building it, exporting it, and merging a
// sorted batch into it.
//
// The paper keeps deletions as an infinity sentinel inside the CSR and puts
// insertions into vacant slots or a per-batch diff-CSR (Section 3.5,
// "Modified Graph Representation: diff-CSR").  Here every row keeps spare
// slots instead and stays sorted and compact: the batch is sorted by
// (store, row, col), and each touched row of the forward and the reverse
// store is rewritten once by a merge (updateCSRDel + updateCSRAdd of the
// DynSSSP driver in one pass).  A row that outgrows its capacity moves to a
// spare pool at the end of the slot array.
#include <algorithm>
#include <cstddef>

#include "sp_graph.cuh"

namespace sp {

namespace {

constexpr int kThreads = 256;
constexpr u32 kFull = 0xffffffffu;

inline unsigned blocks_for(long long work, int per_block, int cap) {
  long long b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

__device__ __forceinline__ void set_status(Ctl *c, int st) { atomicCAS(&c->status, 0, st); }

// Add per-thread counters into global ones with one atomic per block.
__device__ __forceinline__ void block_add(u64 v, u64 *sm, u64 *global) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd((unsigned long long *)sm, v);
  __syncthreads();
  if (threadIdx.x == 0 && *sm) atomicAdd((unsigned long long *)global, *sm);
}

// --------------------------------------------------------------------------
// building a store from a CSR
// --------------------------------------------------------------------------

// One item per input edge: key = row << bits | col (reverse: col << bits | row).
__global__ void k_edge_items(const long long *__restrict__ row_off, const int *__restrict__ col,
                             const int *__restrict__ w, int n, long long m, int bits, int reverse,
                             u64 *keys, u32 *vals) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = n - 1;  // last row u with row_off[u] <= i
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (row_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    u64 u = (u64)lo, v = (u64)(unsigned)col[i];
    keys[i] = reverse ? (v << bits) | u : (u << bits) | v;
    vals[i] = (u32)w[i];
  }
}

__global__ void k_validate_csr(const long long *__restrict__ row_off, const int *__restrict__ col,
                               const int *__restrict__ w, int n, long long m, int *bad) {
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long u = tid; u <= n; u += stride) {
    long long r = row_off[u];
    if ((u == 0 && r != 0) || (u == n && r != m) || r < 0 || r > m ||
        (u > 0 && row_off[u - 1] > r))
      atomicExch(bad, 1);
  }
  for (long long i = tid; i < m; i += stride) {
    int v = col[i], ww = w[i];
    if (v < 0 || v >= n || ww < 1 || ww > SP_WMAX) atomicExch(bad, 1);
  }
}

// flag[0] |= 1 if keys are not strictly increasing (unsorted or duplicate).
__global__ void k_check_order(const u64 *__restrict__ keys, long long m, int *flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x + 1; i < m;
       i += (long long)gridDim.x * blockDim.x)
    if (keys[i - 1] >= keys[i]) atomicOr(flag, keys[i - 1] == keys[i] ? 2 : 1);
}

__global__ void k_row_bounds(const u64 *__restrict__ keys, long long m, int bits,
                             long long *first, long long *last) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    u64 r = keys[i] >> bits;
    if (i == 0 || (keys[i - 1] >> bits) != r) first[r] = i;
    if (i == m - 1 || (keys[i + 1] >> bits) != r) last[r] = i + 1;
  }
}

__global__ void k_row_caps(const long long *__restrict__ first, const long long *__restrict__ last,
                           int n, float slack, u64 *cap_out) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x)
    cap_out[r] = 2ull * (u64)row_capacity(last[r] - first[r], slack);   // two regions
}

__global__ void k_row_meta(const long long *__restrict__ first, const long long *__restrict__ last,
                           const u64 *__restrict__ cap_scan, int n, float slack, RowMeta *row,
                           long long *alt) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    long long d = last[r] - first[r];
    RowMeta rm;
    rm.start = (long long)cap_scan[r];
    rm.deg = (int)d;
    rm.cap = row_capacity(d, slack);
    row[r] = rm;
    alt[r] = rm.start + rm.cap;
  }
}

__global__ void k_fill_adj(const u64 *__restrict__ keys, const u32 *__restrict__ vals, long long m,
                           int bits, const long long *__restrict__ first,
                           const RowMeta *__restrict__ row, int2 *adj) {
  const u64 mask = (1ull << bits) - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    u64 k = keys[i];
    u64 r = k >> bits;
    adj[row[r].start + (i - first[r])] = make_int2((int)(k & mask), (int)vals[i]);
  }
}

// --------------------------------------------------------------------------
// exporting a store
// --------------------------------------------------------------------------

__global__ void k_row_degs(const RowMeta *__restrict__ row, int n, u64 *deg) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r <= n;
       r += (long long)gridDim.x * blockDim.x)
    deg[r] = r < n ? (u64)row[r].deg : 0ull;
}

__global__ void k_export_rows(const RowMeta *__restrict__ row, const int2 *__restrict__ adj, int n,
                              const u64 *__restrict__ off, long long *row_off, int *col, int *w) {
  const int lane = threadIdx.x & 31;
  long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r <= n; r += nwarps) {
    if (lane == 0) row_off[r] = (long long)off[r];
    if (r == n) continue;
    RowMeta rm = row[r];
    long long o = (long long)off[r];
    for (int j = lane; j < rm.deg; j += 32) {
      int2 e = adj[rm.start + j];
      col[o + j] = e.x;
      w[o + j] = e.y;
    }
  }
}

__global__ void k_copy_slots(const int2 *__restrict__ src, int2 *dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// --------------------------------------------------------------------------
// batch: control reset, validation, items
// --------------------------------------------------------------------------

// full: 0 a new call, 1 a new graph, 2 a call rerun after a pool grow,
// which keeps what the first attempt's invalidation found (it ran beside
// the store update, changed the distances, and does not run again)
__global__ void k_ctl_reset(Ctl *c, int full) {
  const bool keep = full == 2;
  c->status = 0;
  c->need_grow = 0;
  c->range_err = 0;
  if (!keep) {
    c->timeout = 0;
    c->to_site = c->to_info = 0;
    c->ccnt = 0;
    c->affected = 0;
    c->inval_edges = 0;
    c->rounds_inval = 0;
    c->jumps = 0;
  }
  c->cmin = 0xFFFFFFFFu;
  c->bad = 0;
  c->bar_inval = 0;
  c->bar_push = 0;
  c->bar_sort = 0;
  c->bar_count = 0;
  c->qcnt0 = c->qcnt1 = c->qcnt2 = c->acnt = 0;
  c->scnt0 = c->scnt1 = c->scnt2 = c->ascnt = 0;
  c->fcnt0 = c->fcnt1 = c->fcnt2 = 0;
  c->fmin0 = c->fmin1 = c->fmin2 = kInf;
  c->seed_min = kInf;
  c->jcnt0 = c->jcnt1 = c->jcnt2 = 0;
  c->prd0 = c->prd1 = c->prd2 = 0.0;
  c->pr_iters = 0;
  c->zcnt = 0;
  c->tc_static = 0;
  c->tc_del[0] = c->tc_del[1] = c->tc_del[2] = 0;
  c->tc_ins[0] = c->tc_ins[1] = c->tc_ins[2] = 0;
  c->lres = c->lcur = c->lround = c->lcap = 0;
  c->lbeat = 0;
  c->mcnt = 0;
  c->bstrips = 0;
  c->mpos = 0;
  c->sstrips = 0;
  c->spos = 0;
  c->n_seg = 0;
  c->pool_need[0] = c->pool_used[0];
  c->pool_need[1] = c->pool_used[1];
  c->del_applied = c->del_absent = c->add_applied = c->add_present = 0;
  c->seeds = c->relaxed = c->improved = 0;
  c->rows_touched = c->rows_relocated = 0;
  c->pull_edges = c->push_vertices = c->enqueued = 0;
  c->merge_slots = 0;
  c->far_moves = 0;
  c->rounds_push = c->splits = 0;
  c->local_episodes = c->local_rounds = 0;
  c->local_ns = c->push_ns = 0;
  c->pool_sub = c->pool_in = 0;
  c->pool_ns = c->pool_sub0 = 0;
  c->deg_mid = 0;
  c->call = c->call + 1;
  if (full == 1) {
    c->epoch = 1;
    c->phase = 1;
    c->call = 1;
    c->pool_used[0] = c->pool_used[1] = 0;
    c->pool_need[0] = c->pool_need[1] = 0;
  }
}

// Validation only (ids and weights), for callers that apply a batch in
// several steps and must reject it before the first one.
__global__ void k_check_batch(const int *__restrict__ ds, const int *__restrict__ dd, long long nd,
                              const int *__restrict__ as, const int *__restrict__ ad,
                              const int *__restrict__ aw, long long na, int n, Ctl *ctl) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd + na;
       i += (long long)gridDim.x * blockDim.x) {
    bool ok;
    if (i < nd) {
      ok = ds[i] >= 0 && ds[i] < n && dd[i] >= 0 && dd[i] < n;
    } else {
      const long long j = i - nd;
      ok = as[j] >= 0 && as[j] < n && ad[j] >= 0 && ad[j] < n && aw[j] >= 1 && aw[j] <= SP_WMAX;
    }
    if (!ok) set_status(ctl, SP_EINVAL);
  }
}

// --------------------------------------------------------------------------
// batch: count pass (which updates apply, new row sizes, where rows go)
// --------------------------------------------------------------------------


struct CountArgs {
  Ctl *ctl;
  long long strips_cap;  // small rows are listed from the end of strips
  const u64 *keys;
  const u32 *vals;       // each sorted item's number in the batch's own order
  const u64 *srch;       // by that number: weight << 32 | present << 31 | position
  u32 *wts;              // out: the weights in sorted order (merge, OnAdd)
  Seg *seg;
  unsigned char *flags;
  u64 *item_pref;      // exclusive prefix of the applied (ins << 32 | dels), n_items + 1
  u32 *opos;
  int2 *strips;
  u64 *tab;            // per-block totals of the prefix
  Store st[2];
  int bits;
  float slack;
  u32 n_items;
  u32 chunk;           // items per block
  int n;
  u64 wait_ns;
  u32 miss_site;         // test hook of the bounded waits (Limits::miss_site)
};

// The merge works on strips of kStrip old entries of a row, one warp each,
// and on groups of kGroup small rows (at most kSmallRow old entries and
// kSmallItems items each), one warp per group: lane j takes entry j of every
// row of the group.
constexpr int kStrip = 256;
constexpr int kGroup = 8;
constexpr int kSmallRow = 32;
constexpr int kSmallItems = 16;

constexpr int kCT = 256;              // threads per block of the count pass
constexpr int kCI = 4;                // items per thread per sub-tile
constexpr int kCS = 4;                // touched rows per thread and pass (third step)
static_assert(offsetof(Seg, first) == 0 && offsetof(Seg, end) == 4 && offsetof(Seg, row) == 8 &&
                  offsetof(Seg, dir) == 12 && alignof(Seg) == 8 && sizeof(Seg) % 8 == 0,
              "the count pass reads a Seg's first four fields as two 8-byte words");
constexpr int kCTile = kCT * kCI;

__device__ __forceinline__ u64 warp_incl_scan_u64(u64 x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 lo = __shfl_up_sync(kFull, (u32)x, o), hi = __shfl_up_sync(kFull, (u32)(x >> 32), o);
    if (lane >= o) x += ((u64)hi << 32) | lo;
  }
  return x;
}

// Block-wide exclusive prefix of one u64 per thread; the block total goes to
// *total.  ws holds one word per warp.
__device__ __forceinline__ u64 block_excl_scan_u64(u64 x, u64 *ws, u64 *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const u64 incl = warp_incl_scan_u64(x);
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    u64 v = lane < nwarps ? ws[lane] : 0ull;
    v = warp_incl_scan_u64(v);
    if (lane < nwarps) ws[lane] = v;
  }
  __syncthreads();
  const u64 r = (warp ? ws[warp - 1] : 0ull) + incl - x;
  *total = ws[nwarps - 1];
  __syncthreads();
  return r;
}

// The count pass in one cooperative launch; block b owns items
// [b*chunk, (b+1)*chunk).
//  1. Items.  A deletion applies if the edge is in the row and it is the
//     first deletion of that edge in the batch; among the insertions of one
//     edge the smallest weight is the candidate (first on ties), and it
//     applies if the edge is absent after the deletions.  Every item also
//     records where its col falls in the old row (opos: the old entries with
//     a smaller col) and whether the edge was there (flags bit 1), which is
//     all the merge needs to place it, and its weight in sorted order.  The
//     searches that find those ran beside the batch sort (k_search); an item
//     reads its result through the number the sort carried as its value.
//  2. The exclusive prefix of the applied (ins << 32 | dels) over all items
//     (block scans, then the block bases after a grid barrier).
//  3. One thread per touched row (after a second barrier): new size,
//     destination (the row's alternate region, or a fresh pair of regions in
//     the spare pool when the row outgrows its capacity), and the row's
//     strips of kStrip old entries (one strip for a row with fewer), the
//     merge's units.
__global__ void __launch_bounds__(kCT, 3) k_count(CountArgs a) {
  __shared__ u32 scratch[40];
  __shared__ u64 ws64[kCT / 32];
  __shared__ u64 s_run;
  __shared__ u64 sums[7];
  Ctl *c = a.ctl;
  if (ld_cg_i32(&c->status) != 0) return;   // the same answer in every block
  const u32 G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const u32 ni = a.n_items;
  const u32 cb = min(b * a.chunk, ni), ce = min(cb + a.chunk, ni);
  u64 *bar = &c->bar_count;
  u64 del_ok = 0, del_abs = 0, add_ok = 0, add_pres = 0;
  if (t == 0) s_run = 0;
  if (t < 7) sums[t] = 0;
  __syncthreads();

  for (u32 tb = cb; tb < ce; tb += kCTile) {
    u64 key[kCI], pk[kCI], nk[kCI], sr[kCI];
    int dir[kCI];
    u32 orig[kCI];
    bool val[kCI];
#pragma unroll
    for (int k = 0; k < kCI; ++k) {
      const u32 i = tb + k * kCT + t;
      val[k] = i < ce;
      key[k] = val[k] ? a.keys[i] : 0ull;
      pk[k] = val[k] && i > 0 ? a.keys[i - 1] : ~0ull;
      nk[k] = val[k] && i + 1 < ni ? a.keys[i + 1] : ~0ull;
      orig[k] = val[k] ? a.vals[i] : 0u;
    }
    // the item's search in its old row ran beside the batch sort (k_search)
#pragma unroll
    for (int k = 0; k < kCI; ++k) {
      dir[k] = (int)(key[k] >> (2 * a.bits + 1));
      sr[k] = val[k] && orig[k] < ni ? __ldcg(a.srch + orig[k]) : 0ull;
    }
    u64 iv[kCI];
#pragma unroll
    for (int k = 0; k < kCI; ++k) {
      iv[k] = 0;
      if (!val[k]) continue;
      const u32 i = tb + k * kCT + t;
      const bool present = (sr[k] >> 31) & 1;
      const unsigned char pbit = present ? 2 : 0;
      a.opos[i] = (u32)sr[k] & 0x7FFFFFFFu;
      a.wts[i] = (u32)(sr[k] >> 32);
      if ((key[k] & 1) == 0) {
        const bool applied = present && pk[k] != key[k];
        a.flags[i] = (applied ? 1 : 0) | pbit;
        iv[k] = applied ? 1ull : 0ull;
        if (dir[k] == 0) { applied ? ++del_ok : ++del_abs; }
      } else {
        // the run of insertions of this edge (almost always this item alone)
        u32 first = i, last = i;
        bool best = true;
        if (pk[k] == key[k] || nk[k] == key[k]) {
          while (first > 0 && a.keys[first - 1] == key[k]) --first;
          while (last + 1 < ni && a.keys[last + 1] == key[k]) ++last;
          u32 bi = first, bw = (u32)(__ldcg(a.srch + a.vals[first]) >> 32);
          for (u32 q = first + 1; q <= last; ++q) {
            const u32 w2 = (u32)(__ldcg(a.srch + a.vals[q]) >> 32);
            if (w2 < bw) { bw = w2; bi = q; }
          }
          best = bi == i;
        }
        const u64 before = first == i ? pk[k] : (first > 0 ? a.keys[first - 1] : ~0ull);
        const bool del_exists = first > 0 && before == (key[k] ^ 1ull);
        const bool run_applies = !present || del_exists;
        const bool applied = best && run_applies;
        a.flags[i] = (applied ? 1 : 0) | pbit;
        iv[k] = applied ? (1ull << 32) : 0ull;
        if (dir[k] == 0 && i == first) {
          add_ok += run_applies;
          add_pres += (u64)(last - first + 1) - (run_applies ? 1 : 0);
        }
      }
    }
    // prefix of the applied over this block's items so far
#pragma unroll
    for (int k = 0; k < kCI; ++k) {
      u64 tot;
      const u64 ex = block_excl_scan_u64(iv[k], ws64, &tot);
      const u32 i = tb + k * kCT + t;
      if (i < ce) a.item_pref[i] = s_run + ex;
      __syncthreads();
      if (t == 0) s_run += tot;
      __syncthreads();
    }
  }
  if (t == 0) __stcg(a.tab + b, s_run);
  if (coop_barrier(bar, (u64)G, c, a.wait_ns, 5, a.miss_site)) return;
  {   // this block's base: the totals of the blocks before it
    u64 part = 0;
    for (u32 q = t; q < b; q += kCT) part += __ldcg(a.tab + q);
    u64 all;
    block_excl_scan_u64(part, ws64, &all);
    for (u32 i = cb + t; i < ce; i += kCT) a.item_pref[i] += all;
    if (b == G - 1 && t == 0) a.item_pref[ni] = all + s_run;
  }
  if (coop_barrier(bar, 2ull * G, c, a.wait_ns, 5, a.miss_site)) return;

  const u32 nseg = ld_cg_u32(&c->n_seg);
  u64 touched = 0, relocated = 0, slots = 0;
  // kCS segments per thread, their loads in flight together: the grid holds
  // kCT * kCS segments per block and at least one item per segment, so a
  // batch normally needs one pass
  for (u32 base = b * kCT * kCS; base < nseg; base += G * kCT * kCS) {
    u32 f[kCS], e[kCS];
    int row[kCS], dir[kCS];
    bool ok[kCS];
#pragma unroll
    for (int j = 0; j < kCS; ++j) {
      const u32 si = base + (u32)j * kCT + t;
      ok[j] = si < nseg;
      f[j] = e[j] = 0;
      row[j] = dir[j] = 0;
      if (ok[j]) {
        // first, end, row, dir: two 8-byte loads (a Seg is 8-byte aligned)
        const int2 *hp = (const int2 *)(a.seg + si);
        const int2 h0 = __ldcg(hp), h1 = __ldcg(hp + 1);
        f[j] = (u32)h0.x;
        e[j] = (u32)h0.y;
        row[j] = h1.x;
        dir[j] = h1.y;
        if (f[j] >= e[j] || e[j] > a.n_items || row[j] < 0 || row[j] >= a.n || dir[j] < 0 ||
            dir[j] > 1) {  // never expected: record and skip
          atomicExch(&c->bad, 1);
          ok[j] = false;
        }
      }
    }
    RowMeta rm[kCS];
    u64 pf[kCS], pe[kCS], key[kCS];
#pragma unroll
    for (int j = 0; j < kCS; ++j) {
      rm[j].start = 0;
      rm[j].deg = rm[j].cap = 0;
      pf[j] = pe[j] = key[j] = 0;
      if (ok[j]) {
        rm[j] = a.st[dir[j]].row[row[j]];
        pf[j] = __ldcg(a.item_pref + f[j]);
        pe[j] = __ldcg(a.item_pref + e[j]);
        key[j] = a.keys[f[j]];
      }
    }
    u32 nstr[kCS], nsmall[kCS];
    u64 want = 0;   // this thread's strips (low word) and small rows (high word)
#pragma unroll
    for (int j = 0; j < kCS; ++j) {
      nstr[j] = nsmall[j] = 0;
      if (!ok[j]) continue;
      const Store &st = a.st[dir[j]];
      const u64 p = pe[j] - pf[j];
      const int new_deg = rm[j].deg - (int)(u32)p + (int)(u32)(p >> 32);
      Seg &sg = a.seg[base + (u32)j * kCT + t];
      sg.old_start = rm[j].start;
      sg.old_deg = rm[j].deg;
      sg.new_deg = new_deg;
      sg.pad = 0;
      sg.prefix = key[j] & ~((2ull << a.bits) - 1);
      sg.base_pref = pf[j];
      if (new_deg > rm[j].cap) {
        long long nc = row_capacity(new_deg, a.slack);
        const long long dbl = round_up4(2LL * rm[j].cap);
        if (dbl > nc) nc = dbl;
        const u64 off = atomicAdd(&c->pool_need[dir[j]], (u64)(2 * nc));
        if ((long long)(off + 2 * nc) > st.slots - st.main_slots)
          atomicOr(&c->need_grow, dir[j] ? kGrowPoolRev : kGrowPoolFwd);
        sg.dest = st.main_slots + (long long)off;
        sg.new_alt = st.main_slots + (long long)off + nc;
        sg.new_cap = (int)nc;
        ++relocated;
      } else {
        sg.dest = st.alt[row[j]];
        sg.new_alt = rm[j].start;
        sg.new_cap = rm[j].cap;
      }
      if (rm[j].deg <= kSmallRow && e[j] - f[j] <= (u32)kSmallItems)
        nsmall[j] = 1;
      else
        nstr[j] = rm[j].deg > kStrip ? (u32)((rm[j].deg + kStrip - 1) / kStrip) : 1u;
      want += (u64)nstr[j] | ((u64)nsmall[j] << 32);
      ++touched;
      slots += (u64)rm[j].deg + (u64)new_deg;
    }
    {   // reserve the strips (from the front) and the small rows (from the
        // back of the same array): one scan and one atomic each per block
      u64 tot;
      const u64 ex = block_excl_scan_u64(want, ws64, &tot);
      const u32 stot = (u32)tot, smtot = (u32)(tot >> 32);
      if (t == 0) scratch[35] = stot ? atomicAdd(&c->bstrips, stot) : 0u;
      if (t == 32) scratch[36] = smtot ? atomicAdd(&c->sstrips, smtot) : 0u;
      __syncthreads();
      u32 sb = scratch[35] + (u32)ex, smb = scratch[36] + (u32)(ex >> 32);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kCS; ++j) {
        const int si = (int)(base + (u32)j * kCT + t);
        for (u32 k = 0; k < nstr[j]; ++k) a.strips[sb + k] = make_int2(si, (int)(k * kStrip));
        sb += nstr[j];
        if (nsmall[j]) a.strips[a.strips_cap - 1 - smb++] = make_int2(si, 0);
      }
    }
  }
  block_add(del_ok, &sums[0], &c->del_applied);
  block_add(del_abs, &sums[1], &c->del_absent);
  block_add(add_ok, &sums[2], &c->add_applied);
  block_add(add_pres, &sums[3], &c->add_present);
  block_add(touched, &sums[4], &c->rows_touched);
  block_add(relocated, &sums[5], &c->rows_relocated);
  block_add(slots, &sums[6], &c->merge_slots);
}

// --------------------------------------------------------------------------
// batch: the old-row searches, beside the batch sort
// --------------------------------------------------------------------------

struct SearchArgs {
  const int *ds, *dd, *as, *ad, *aw;
  long long nd, na;
  Store st[2];
  u64 *srch;
  int n;
  u32 n_items;
};

// Item i of the batch in the batch sort's own numbering (update j < nd is
// deletion j, then the insertions; item j is its forward item, nb + j its
// reverse one): the binary search of its col in its old row, as the count
// pass needs it (position = old entries with a smaller col, and whether the
// edge is there), and its weight, into srch[i].  The stores do not change
// before the merge, so this runs beside the sort; ids out of range (the sort
// rejects the batch) get 0.  Each thread advances kCI searches in lockstep.
__global__ void __launch_bounds__(kCT) k_search(SearchArgs a) {
  const long long nb = a.nd + a.na;
  const u32 ni = a.n_items;
  for (u32 tb = blockIdx.x * (u32)kCTile; tb < ni; tb += gridDim.x * (u32)kCTile) {
    int col[kCI], lo[kCI], hi[kCI], deg[kCI];
    u32 w[kCI];
    const int2 *old[kCI];
    bool val[kCI];
#pragma unroll
    for (int k = 0; k < kCI; ++k) {   // every input load first
      const u32 i = tb + (u32)(k * kCT) + threadIdx.x;
      val[k] = i < ni;
      int u = 0, v = 0;
      w[k] = 0;
      const bool rev = (long long)i >= nb;
      const long long j = rev ? (long long)i - nb : (long long)i;
      if (val[k]) {
        if (j < a.nd) {
          u = __ldg(a.ds + j);
          v = __ldg(a.dd + j);
        } else {
          u = __ldg(a.as + (j - a.nd));
          v = __ldg(a.ad + (j - a.nd));
          w[k] = (u32)__ldg(a.aw + (j - a.nd));
        }
      }
      const bool ok = val[k] && u >= 0 && u < a.n && v >= 0 && v < a.n;
      const int row = rev ? v : u;
      col[k] = rev ? u : v;
      RowMeta rm;
      rm.start = 0;
      rm.deg = 0;
      if (ok) rm = a.st[rev ? 1 : 0].row[row];
      old[k] = a.st[rev ? 1 : 0].adj + rm.start;
      lo[k] = 0;
      hi[k] = deg[k] = rm.deg;
    }
    for (;;) {   // binary searches in lockstep: every load of a step in flight together
      bool act = false;
      int mid[kCI], x[kCI];
#pragma unroll
      for (int k = 0; k < kCI; ++k) {
        act |= lo[k] < hi[k];
        mid[k] = (lo[k] + hi[k]) >> 1;
        x[k] = lo[k] < hi[k] ? __ldg(&old[k][mid[k]].x) : 0;
      }
      if (!act) break;
#pragma unroll
      for (int k = 0; k < kCI; ++k)
        if (lo[k] < hi[k]) {
          if (x[k] < col[k]) lo[k] = mid[k] + 1; else hi[k] = mid[k];
        }
    }
#pragma unroll
    for (int k = 0; k < kCI; ++k) {
      const int cl = lo[k] < deg[k] ? __ldg(&old[k][lo[k]].x) : -1;
      if (val[k]) {
        const u32 i = tb + (u32)(k * kCT) + threadIdx.x;
        a.srch[i] = ((u64)w[k] << 32) | (cl == col[k] ? 0x80000000ull : 0ull) | (u32)lo[k];
      }
    }
  }
}

SearchArgs search_args(sp_graph *g, const int *ds, const int *dd, long long nd, const int *as,
                       const int *ad, const int *aw, long long na) {
  SearchArgs a;
  a.ds = ds; a.dd = dd; a.as = as; a.ad = ad; a.aw = aw;
  a.nd = nd; a.na = na;
  a.st[0] = g->fwd;
  a.st[1] = g->rev;
  a.srch = g->bb.srch;
  a.n = g->n;
  a.n_items = (u32)(2 * (nd + na));
  return a;
}

// One block of 256 threads per SM at most: beside it an SM still holds a
// block of the batch sort (512 threads, 90-116 KB of shared memory, about
// 45k registers), so the search never delays the sort's cooperative grid.
unsigned search_grid(const sp_graph *g, long long ni) {
  return blocks_for(ni, kCTile, std::max(1, g->num_sms));
}

// --------------------------------------------------------------------------
// batch: merge pass (rewrite each touched row into its other region)
// --------------------------------------------------------------------------

struct MergeArgs {
  Ctl *ctl;
  const u64 *keys;
  const u32 *vals;
  const unsigned char *flags;
  const u64 *item_pref;   // exclusive prefix of the applied updates, n_items + 1 entries
  const Seg *seg;
  const u32 *opos;
  const int2 *strips;
  long long strips_cap;   // small rows are listed from the end of strips
  Store st[2];
  int bits;
  u32 n_items;
};

__device__ __forceinline__ bool merge_enabled(Ctl *c) {
  return ld_cg_i32(&c->status) == 0 && ld_cg_i32(&c->need_grow) == 0 &&
         ld_cg_i32(&c->bad) == 0;
}

// The merged row holds the kept old entries and the applied insertions in
// col order, so every element knows its output slot from prefix counts:
//   old entry j (col c):   j - #applied deletions with col < c
//                            + #applied insertions with col < c
//   applied insertion i:   opos[i] + present[i] - #applied deletions before i
//                            + #applied insertions before i
// (opos = old entries with a smaller col; when the edge was present, its
// deletion is among the deletions before i and its old entry is not).
// Items are sorted by (col, deletion before insertion) and opos is
// non-decreasing along a row's items.
//
// One warp per strip of kStrip old entries.  The strip owns the items with
// opos in [j0, jl) (the last strip also those past the end), so every item
// of the row belongs to exactly one strip, and every item of an earlier
// strip has a smaller col than every old entry of this one.  A warp takes
// kMergeGrab strips at a time and finds all their item ranges at once (one
// lane per range end, binary searches in lockstep; none for a row of one
// strip).  Per strip it loads its old entries (eight coalesced 256-byte
// loads), stages its items in shared memory, and places both from there:
// the dependent global loads per strip are one round of item loads.
constexpr int kStripItems = 128;   // items staged per warp
constexpr int kMergeGrab = 8;      // strips a warp takes at a time
struct StripItems {
  u64 pre[kStripItems];            // applied (ins << 32 | dels) of the row before the item
  u32 col[kStripItems];
  u32 w[kStripItems];
  u32 opos[kStripItems];
  unsigned char fl[kStripItems];   // bit0 applied, bit1 present, bit2 insertion
  Seg seg[kMergeGrab];             // the grabbed strips' segments
  int2 sp[kMergeGrab];             // ... and strip records
  u32 ilo[kMergeGrab], ihi[kMergeGrab];   // ... their item ranges
  u64 pend[kMergeGrab];            // ... and applied updates before their range's end
  u64 gpend[kGroup];               // small-row groups: applied updates of each row
  u32 goff[kGroup + 1];            // ... and where each row's items are staged
};
static_assert(kGroup <= kMergeGrab && kGroup * kSmallItems <= kStripItems,
              "a small-row group's records and items fit the warp's stage");

__global__ void __launch_bounds__(kThreads, 4) k_merge(MergeArgs a) {
  __shared__ StripItems sitems[kThreads / 32];
  Ctl *c = a.ctl;
  if (!__shfl_sync(kFull, (int)merge_enabled(c), 0)) return;   // warp-uniform
  const int lane = threadIdx.x & 31;
  StripItems &S = sitems[threadIdx.x >> 5];
  const u32 nstrips = ld_cg_u32(&c->bstrips);
  const u64 cmask = (1ull << a.bits) - 1;
  bool bad = false;
  // warps take strips kMergeGrab at a time from a global counter, so blocks
  // that start late (SMs busy with the invalidation beside the merge) find
  // only the work that is left
  u32 grab = 0, gend = 0, g0 = 0;
  for (;;) {
    if (grab == gend) {
      u32 b0 = 0;
      if (lane == 0) b0 = atomicAdd(&c->mpos, (u32)kMergeGrab);
      grab = g0 = __shfl_sync(kFull, b0, 0);
      gend = min(grab + (u32)kMergeGrab, nstrips);
      if (grab >= nstrips) break;
      // the grabbed strips' records and segments in one round of loads
      // each, one lane per strip (the later strips' old entries are
      // prefetched toward L2 a strip ahead)
      __syncwarp();   // every lane is done with the previous grab's records
      if (lane < (int)(gend - grab)) {
        const int2 q = __ldcg(a.strips + grab + lane);
        S.sp[lane] = q;
        S.seg[lane] = a.seg[q.x];
      }
      __syncwarp();
      // the grabbed strips' item ranges: lane l < ng finds the first item of
      // strip l, lane kMergeGrab + l its end, every binary search in lockstep
      // with the others (a row of one strip needs none)
      const u32 ng = gend - grab;
      if (lane < 2 * kMergeGrab) {
        const u32 l = (u32)lane & (kMergeGrab - 1);
        const bool hi_q = lane >= kMergeGrab;
        u32 r = 0;
        if (l < ng) {
          const Seg &sq = S.seg[l];
          const int jb = S.sp[l].y + (hi_q ? kStrip : 0);
          u32 lo = sq.first, hi = sq.end;
          if (jb <= 0) hi = lo;                 // the row's first strip starts at its first item
          else if (jb >= sq.old_deg) lo = hi;   // its last strip ends at its last
          while (lo < hi) {
            const u32 mid = (lo + hi) >> 1;
            if (__ldg(a.opos + mid) < (u32)jb) lo = mid + 1; else hi = mid;
          }
          r = lo;
          if (hi_q) S.ihi[l] = r; else S.ilo[l] = r;
        }
        if (hi_q && l < ng) S.pend[l] = a.item_pref[r] - S.seg[l].base_pref;
      }
      __syncwarp();
    }
    const u32 sidx = grab++;
    const int2 sp = S.sp[sidx - g0];
    const Seg sg = S.seg[sidx - g0];
    if (grab < gend && lane < kStrip * 8 / 128) {   // the next strip's old entries
      const Seg &nx = S.seg[grab - g0];
      const int nj = S.sp[grab - g0].y + lane * (128 / 8);
      if (nj < nx.old_deg) {
        const int2 *p = a.st[nx.dir].adj + nx.old_start + nj;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
      }
    }
    const Store &st = a.st[sg.dir];
    const int2 *old = st.adj + sg.old_start;
    int2 *dst = st.adj + sg.dest;
    const int j0 = sp.y;
    const int jl = j0 + kStrip < sg.old_deg ? j0 + kStrip : sg.old_deg;
    int2 en[kStrip / 32];
#pragma unroll
    for (int t = 0; t < kStrip / 32; ++t) {
      const int j = j0 + lane + 32 * t;
      en[t] = j < jl ? old[j] : make_int2(0, 0);
    }
    if (j0 == 0 && lane == 0) {
      RowMeta nm;
      nm.start = sg.dest;
      nm.deg = sg.new_deg;
      nm.cap = sg.new_cap;
      st.row[sg.row] = nm;
      st.alt[sg.row] = sg.new_alt;
    }
    const u32 ilo = S.ilo[sidx - g0], ihi = S.ihi[sidx - g0];
    const u32 k = ihi - ilo;
    const u64 pend = S.pend[sidx - g0];
    if (k <= (u32)kStripItems) {
      for (u32 q = lane; q < k; q += 32) {
        const u32 i = ilo + q;
        const u64 key = a.keys[i];
        S.pre[q] = a.item_pref[i] - sg.base_pref;
        S.col[q] = (u32)((key >> 1) & cmask);
        S.w[q] = a.vals[i];
        S.opos[q] = a.opos[i];
        S.fl[q] = (unsigned char)((a.flags[i] & 3) | ((key & 1) ? 4 : 0));
      }
      __syncwarp();
      // first staged item with col >= cj: a lane's entries rise in col, so
      // each search starts where the lane's previous one ended; a short walk
      // when the strip has few items (the common case), else a binary search
      u32 lo = 0;
#pragma unroll
      for (int t = 0; t < kStrip / 32; ++t) {
        const int j = j0 + lane + 32 * t;
        if (j < jl) {
          const u32 cj = (u32)en[t].x;
          if (k <= 16u) {
            while (lo < k && S.col[lo] < cj) ++lo;
          } else {
            u32 hi = k;
            while (lo < hi) {
              const u32 mid = (lo + hi) >> 1;
              if (S.col[mid] < cj) lo = mid + 1; else hi = mid;
            }
          }
          const bool del = lo < k && S.col[lo] == cj && (S.fl[lo] & 5) == 1;
          if (!del) {
            const u64 pp = lo < k ? S.pre[lo] : pend;
            const int pos = j - (int)(u32)pp + (int)(u32)(pp >> 32);
            if (pos >= 0 && pos < sg.new_deg) dst[pos] = en[t];
            else bad = true;
          }
        }
      }
      for (u32 q = lane; q < k; q += 32) {
        if ((S.fl[q] & 5) == 5) {   // applied insertion
          const u64 pp = S.pre[q];
          const int pos = (int)S.opos[q] + ((S.fl[q] >> 1) & 1) - (int)(u32)pp +
                          (int)(u32)(pp >> 32);
          if (pos >= 0 && pos < sg.new_deg) dst[pos] = make_int2((int)S.col[q], (int)S.w[q]);
          else bad = true;
        }
      }
      __syncwarp();
    } else {
      // more items than the stage holds: the same placement, searching the
      // batch arrays in global memory
#pragma unroll
      for (int t = 0; t < kStrip / 32; ++t) {
        const int j = j0 + lane + 32 * t;
        if (j < jl) {
          const u64 kc = sg.prefix | ((u64)(unsigned)en[t].x << 1);
          u32 lo = ilo, hi = ihi;
          while (lo < hi) {
            const u32 mid = (lo + hi) >> 1;
            if (a.keys[mid] < kc) lo = mid + 1; else hi = mid;
          }
          const bool del = lo < ihi && a.keys[lo] == kc && (a.flags[lo] & 1);
          if (!del) {
            const u64 pp = a.item_pref[lo] - sg.base_pref;
            const int pos = j - (int)(u32)pp + (int)(u32)(pp >> 32);
            if (pos >= 0 && pos < sg.new_deg) dst[pos] = en[t];
            else bad = true;
          }
        }
      }
      for (u32 i = ilo + lane; i < ihi; i += 32) {
        const u64 key = a.keys[i];
        const unsigned char f = a.flags[i];
        if ((key & 1) && (f & 1)) {
          const u64 pp = a.item_pref[i] - sg.base_pref;
          const int pos = (int)a.opos[i] + ((f >> 1) & 1) - (int)(u32)pp + (int)(u32)(pp >> 32);
          if (pos >= 0 && pos < sg.new_deg)
            dst[pos] = make_int2((int)((key >> 1) & cmask), (int)a.vals[i]);
          else bad = true;
        }
      }
    }
  }
  // Groups of small rows (at most kSmallRow old entries and kSmallItems
  // items each): a warp merges kGroup of them at once, lane j taking old
  // entry j of every row, so the dependent loads of eight rows are in flight
  // together.  The placement is the strips' (prefix counts of the applied
  // updates before each element).
  const u32 nsmall = ld_cg_u32(&c->sstrips);
  const u32 ngroups = (nsmall + kGroup - 1) / kGroup;
  for (;;) {
    u32 g0 = 0;
    if (lane == 0) g0 = atomicAdd(&c->spos, 1u);
    g0 = __shfl_sync(kFull, g0, 0);
    if (g0 >= ngroups) break;
    const u32 s0 = g0 * kGroup;
    const u32 cnt = min(s0 + (u32)kGroup, nsmall) - s0;
    __syncwarp();   // every lane is done with the previous group's stage
    u32 kt = 0;
    if ((u32)lane < cnt) {
      const int2 q = __ldcg(a.strips + (a.strips_cap - 1 - (long long)(s0 + lane)));
      const Seg sg = a.seg[q.x];
      S.seg[lane] = sg;
      kt = sg.end - sg.first;
      S.gpend[lane] = a.item_pref[sg.end] - sg.base_pref;
      if (sg.old_deg > kSmallRow || kt > (u32)kSmallItems) {   // never expected
        bad = true;
        kt = 0;
      }
    }
    bad = __any_sync(kFull, bad);
    if (bad) break;   // warp-uniform; the flag below makes the call fail
    // where each row's items go in the stage: exclusive prefix of kt
    {
      const u32 inc = (u32)warp_incl_scan_u64(kt);
      const u32 tot = __shfl_sync(kFull, inc, cnt - 1);
      if ((u32)lane < cnt) S.goff[lane] = inc - kt;
      if (lane == 0) S.goff[cnt] = tot;
    }
    __syncwarp();
    const u32 ktot = S.goff[cnt];
    int2 en[kGroup];
#pragma unroll
    for (int t = 0; t < kGroup; ++t) {
      en[t] = make_int2(0, 0);
      if ((u32)t < cnt) {
        const Seg &sg = S.seg[t];
        if (lane < sg.old_deg) en[t] = a.st[sg.dir].adj[sg.old_start + lane];
      }
    }
    for (u32 q = lane; q < ktot; q += 32) {
      u32 t = 0;
      while (t + 1 < cnt && S.goff[t + 1] <= q) ++t;
      const Seg &sg = S.seg[t];
      const u32 i = sg.first + (q - S.goff[t]);
      const u64 key = a.keys[i];
      S.pre[q] = a.item_pref[i] - sg.base_pref;
      S.col[q] = (u32)((key >> 1) & cmask);
      S.w[q] = a.vals[i];
      S.opos[q] = a.opos[i];
      S.fl[q] = (unsigned char)((a.flags[i] & 3) | ((key & 1) ? 4 : 0));
    }
    if ((u32)lane < cnt) {   // the rows' new places
      const Seg &sg = S.seg[lane];
      RowMeta nm;
      nm.start = sg.dest;
      nm.deg = sg.new_deg;
      nm.cap = sg.new_cap;
      a.st[sg.dir].row[sg.row] = nm;
      a.st[sg.dir].alt[sg.row] = sg.new_alt;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kGroup; ++t) {
      if ((u32)t < cnt) {
        const Seg &sg = S.seg[t];
        if (lane < sg.old_deg) {
          const u32 cj = (u32)en[t].x;
          const u32 o0 = S.goff[t], o1 = S.goff[t + 1];
          u32 lo = o0;
          while (lo < o1 && S.col[lo] < cj) ++lo;
          const bool del = lo < o1 && S.col[lo] == cj && (S.fl[lo] & 5) == 1;
          if (!del) {
            const u64 pp = lo < o1 ? S.pre[lo] : S.gpend[t];
            const int pos = lane - (int)(u32)pp + (int)(u32)(pp >> 32);
            if (pos >= 0 && pos < sg.new_deg) a.st[sg.dir].adj[sg.dest + pos] = en[t];
            else bad = true;
          }
        }
      }
    }
    for (u32 q = lane; q < ktot; q += 32) {
      if ((S.fl[q] & 5) == 5) {   // applied insertion
        u32 t = 0;
        while (t + 1 < cnt && S.goff[t + 1] <= q) ++t;
        const Seg &sg = S.seg[t];
        const u64 pp = S.pre[q];
        const int pos = (int)S.opos[q] + ((S.fl[q] >> 1) & 1) - (int)(u32)pp +
                        (int)(u32)(pp >> 32);
        if (pos >= 0 && pos < sg.new_deg)
          a.st[sg.dir].adj[sg.dest + pos] = make_int2((int)S.col[q], (int)S.w[q]);
        else bad = true;
      }
    }
  }
  if (bad) atomicExch(&c->bad, 1);
}

// The call's bookkeeping, then the whole control block into the host's
// pinned copy (mapped memory), so the host needs no copy of its own.
__global__ void k_finish(Ctl *c, Ctl *host) {
  if (threadIdx.x == 0 && c->status == 0 && c->need_grow == 0) {
    c->pool_used[0] = c->pool_need[0];
    c->pool_used[1] = c->pool_need[1];
  }
  __syncthreads();
  if (host) {
    const u32 *src = (const u32 *)c;
    u32 *dst = (u32 *)host;
    for (u32 i = threadIdx.x; i < sizeof(Ctl) / 4; i += blockDim.x) dst[i] = __ldcg(src + i);
  }
}

}  // namespace

// ==========================================================================
// host side
// ==========================================================================

sp_status store_build(sp_graph *g, Store *st, const long long *row_off_d, const int *col_d,
                      const int *w_d, long long m, int reverse, int *launches) {
  cudaStream_t s = g->stream;
  const int n = g->n, bits = g->bits;
  const unsigned grid = (unsigned)std::max(1, g->num_sms * 8);
  // edge items
  long long mm = std::max(m, 1LL);
  size_t tmpb = std::max(sort_tmp_bytes(mm), scan_tmp_bytes((long long)n + 1)) + 64;
  size_t need = (size_t)mm * (2 * sizeof(u64) + 2 * sizeof(u32)) + 2 * (size_t)(n + 1) * 8 +
                (size_t)(n + 1) * 8 + tmpb + 16 * 256;
  char *buf = (char *)g->al.get(need);
  if (!buf) return SP_ENOMEM;
  auto carve = [&](size_t bytes) {
    char *p = buf;
    buf += (bytes + 255) & ~(size_t)255;
    return (void *)p;
  };
  char *base = buf;
  u64 *keys = (u64 *)carve((size_t)mm * 8);
  u64 *keys_alt = (u64 *)carve((size_t)mm * 8);
  u32 *vals = (u32 *)carve((size_t)mm * 4);
  u32 *vals_alt = (u32 *)carve((size_t)mm * 4);
  long long *first = (long long *)carve((size_t)(n + 1) * 8);
  long long *last = (long long *)carve((size_t)(n + 1) * 8);
  u64 *caps = (u64 *)carve((size_t)(n + 1) * 8);
  int *flag = (int *)carve(256);
  void *tmp = carve(tmpb);
  (void)keys_alt;
  sp_status rc = SP_OK;
  int hflag = 0;
  if (m > 0) {
    k_edge_items<<<grid, kThreads, 0, s>>>(row_off_d, col_d, w_d, n, m, bits, reverse, keys, vals);
    ++*launches;
    bool need_sort = reverse != 0;
    if (!need_sort) {
      cudaMemsetAsync(flag, 0, sizeof(int), s);
      k_check_order<<<grid, kThreads, 0, s>>>(keys, m, flag);
      ++*launches;
      cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) rc = SP_ECUDA;
      need_sort = hflag != 0;
    }
    if (rc == SP_OK && need_sort) {
      sort_pairs(keys, vals, keys_alt, vals_alt, m, 2 * bits, tmp, s, launches);
      cudaMemsetAsync(flag, 0, sizeof(int), s);
      k_check_order<<<grid, kThreads, 0, s>>>(keys, m, flag);
      ++*launches;
      cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) rc = SP_ECUDA;
      else if (hflag != 0) rc = SP_EINVAL;  // duplicate edges
    }
  }
  if (rc == SP_OK) {
    cudaMemsetAsync(first, 0, (size_t)(n + 1) * 8, s);
    cudaMemsetAsync(last, 0, (size_t)(n + 1) * 8, s);
    if (m > 0) {
      k_row_bounds<<<grid, kThreads, 0, s>>>(keys, m, bits, first, last);
      ++*launches;
    }
    k_row_caps<<<grid, kThreads, 0, s>>>(first, last, n, g->slack, caps);
    cudaMemsetAsync(caps + n, 0, 8, s);
    scan_exclusive_u64(caps, caps, (long long)n + 1, tmp, s, launches);
    ++*launches;
    u64 main_slots = 0;
    cudaMemcpyAsync(&main_slots, caps + n, 8, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = SP_ECUDA;
    if (rc == SP_OK) {
      long long pool = std::max<long long>(round_up4((long long)main_slots / 4), 1LL << 16);
      st->main_slots = (long long)main_slots;
      st->slots = st->main_slots + pool;
      st->row = (RowMeta *)g->al.get((size_t)n * sizeof(RowMeta));
      st->alt = (long long *)g->al.get((size_t)n * sizeof(long long));
      st->adj = (int2 *)g->al.get((size_t)st->slots * sizeof(int2));
      if (!st->row || !st->alt || !st->adj) rc = SP_ENOMEM;
    }
    if (rc == SP_OK) {
      k_row_meta<<<grid, kThreads, 0, s>>>(first, last, caps, n, g->slack, st->row, st->alt);
      ++*launches;
      if (m > 0) {
        k_fill_adj<<<grid, kThreads, 0, s>>>(keys, vals, m, bits, first, st->row, st->adj);
        ++*launches;
      }
      if (cudaStreamSynchronize(s) != cudaSuccess) rc = SP_ECUDA;
    }
  }
  g->al.put(base, need);
  return rc;
}

sp_status csr_validate(sp_graph *g, const long long *row_off_d, const int *col_d,
                       const int *w_d, long long m, int *launches) {
  cudaStream_t s = g->stream;
  int *flag = (int *)g->al.get(256);
  if (!flag) return SP_ENOMEM;
  const unsigned grid = (unsigned)std::max(1, g->num_sms * 8);
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  k_validate_csr<<<grid, kThreads, 0, s>>>(row_off_d, col_d, w_d, g->n, m, flag);
  ++*launches;
  int h = 0;
  cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  sp_status rc = cudaStreamSynchronize(s) == cudaSuccess ? SP_OK : SP_ECUDA;
  g->al.put(flag, 256);
  if (rc == SP_OK && h) rc = SP_EINVAL;
  return rc;
}

sp_status store_export(sp_graph *g, const Store *st, long long *row_off_d, int *col_d, int *w_d,
                       int *launches) {
  cudaStream_t s = g->stream;
  const int n = g->n;
  const unsigned grid = (unsigned)std::max(1, g->num_sms * 8);
  size_t tmpb = scan_tmp_bytes((long long)n + 1) + 256;
  size_t need = 2 * (size_t)(n + 1) * 8 + tmpb + 512;
  char *buf = (char *)g->al.get(need);
  if (!buf) return SP_ENOMEM;
  u64 *deg = (u64 *)buf;
  u64 *off = deg + (n + 1);
  void *tmp = (void *)(((uintptr_t)(off + n + 1) + 255) & ~(uintptr_t)255);
  k_row_degs<<<grid, kThreads, 0, s>>>(st->row, n, deg);
  scan_exclusive_u64(deg, off, (long long)n + 1, tmp, s, launches);
  k_export_rows<<<grid, kThreads, 0, s>>>(st->row, st->adj, n, off, row_off_d, col_d, w_d);
  *launches += 2;
  sp_status rc = cudaStreamSynchronize(s) == cudaSuccess ? SP_OK : SP_ECUDA;
  g->al.put(buf, need);
  return rc;
}

sp_status store_grow_pool(sp_graph *g, Store *st, long long min_pool_slots) {
  ++g->gen;
  long long pool = st->slots - st->main_slots;
  long long np = std::max(2 * pool, round_up4(min_pool_slots));
  long long slots = st->main_slots + np;
  int2 *adj = (int2 *)g->al.get((size_t)slots * sizeof(int2));
  if (!adj) return SP_ENOMEM;
  const unsigned grid = (unsigned)std::max(1, g->num_sms * 8);
  k_copy_slots<<<grid, kThreads, 0, g->stream>>>(st->adj, adj, st->slots);
  g->al.put(st->adj, (size_t)st->slots * sizeof(int2));
  st->adj = adj;
  st->slots = slots;
  return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

// Chunk-owner tables sized for the stores' slots.  The new tables are
// allocated before the old ones are released: on SP_ENOMEM the old ones
// stay (they still cover the edge set, which did not change).
sp_status ensure_owner_tables(sp_graph *g) {
  const long long slots = std::max(g->fwd.slots, g->rev.slots);
  const long long need = slots / kChunk + 64;
  if (need <= g->own_cap && g->qown[0]) return SP_OK;
  const long long c = std::max(need, g->own_cap * 2);
  u32 *p[4];
  bool ok = true;
  for (int b = 0; b < 4; ++b) {
    p[b] = ok ? (u32 *)g->al.get((size_t)c * 4) : nullptr;
    ok = ok && p[b];
  }
  if (!ok) {
    for (int b = 0; b < 4; ++b) g->al.put(p[b], (size_t)c * 4);
    return SP_ENOMEM;
  }
  for (int b = 0; b < 3; ++b) {
    g->al.put(g->qown[b], (size_t)g->own_cap * 4);
    g->qown[b] = p[b];
  }
  g->al.put(g->aown, (size_t)g->own_cap * 4);
  g->aown = p[3];
  ++g->gen;
  g->own_cap = c;
  return SP_OK;
}

void launch_ctl_reset(sp_graph *g, int full, int *launches) {
  k_ctl_reset<<<1, 1, 0, g->stream>>>(g->ctl, full);
  ++*launches;
}

int count_blocks(int num_sms) {
  int per_sm = 0;
  if (cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kExclusiveSmem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count, kCT, 0) != cudaSuccess ||
      per_sm < 1)
    return 0;
  return per_sm * num_sms;
}

void launch_count(sp_graph *g, long long ni, int *launches, int avoid_sms) {
  if (ni == 0) return;
  BatchBufs &b = g->bb;
  CountArgs a;
  a.ctl = g->ctl;
  a.keys = b.keys;
  a.vals = b.vals;
  a.srch = b.srch;
  a.wts = b.vals_alt;   // free once the sort has ended (its output is keys / vals)
  a.seg = b.seg;
  a.flags = b.flags;
  a.item_pref = b.item_pref;
  a.opos = b.opos;
  a.strips = b.strips;
  a.strips_cap = b.strips_cap;
  a.tab = (u64 *)b.tmp;   // the batch sort's table is free again
  a.st[0] = g->fwd;
  a.st[1] = g->rev;
  a.bits = g->bits;
  a.slack = g->slack;
  a.n_items = (u32)ni;
  a.n = g->n;
  a.wait_ns = g->lim.wait_ns;
  a.miss_site = g->lim.miss_site;
  int G = (int)std::min<long long>((ni + kCTile - 1) / kCTile, g->count_blocks);
  // a block share: at most that many blocks, each holding an SM alone
  const bool share = g->loop_blocks_user > 0;
  if (share && g->loop_blocks_user < G) G = g->loop_blocks_user;
  // beside a cooperative grid that holds avoid_sms whole SMs: at most what
  // the other SMs hold, so the count is resident in full whichever grid the
  // GPU places first
  if (avoid_sms > 0) {
    const int per_sm = std::max(1, g->count_blocks / std::max(1, g->num_sms));
    G = std::min(G, per_sm * std::max(1, g->num_sms - avoid_sms));
  }
  if (G < 1) G = 1;
  a.chunk = (u32)((ni + G - 1) / G);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = share ? kExclusiveSmem : 0;
  cfg.stream = g->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_count, a);
  *launches += 1;
}

void launch_merge(sp_graph *g, long long ni, int *launches) {
  if (ni == 0) return;
  BatchBufs &b = g->bb;
  MergeArgs a;
  a.ctl = g->ctl;
  a.keys = b.keys;
  a.vals = b.vals_alt;   // the weights in sorted order (written by the count pass)
  a.flags = b.flags;
  a.item_pref = b.item_pref;
  a.seg = b.seg;
  a.opos = b.opos;
  a.strips = b.strips;
  a.strips_cap = b.strips_cap;
  a.st[0] = g->fwd;
  a.st[1] = g->rev;
  a.bits = g->bits;
  a.n_items = (u32)ni;
  // exactly the resident blocks: every warp starts at once and the strips
  // spread evenly over them
  static int per_sm = 0;
  if (per_sm == 0 &&
      (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge, kThreads, 0) !=
           cudaSuccess ||
       per_sm < 1))
    per_sm = 4;
  k_merge<<<(unsigned)std::max(1, g->num_sms * per_sm), kThreads, 0, g->stream>>>(a);
  *launches += 1;
}

void launch_check_batch(sp_graph *g, const int *ds, const int *dd, long long nd, const int *as,
                        const int *ad, const int *aw, long long na, int *launches) {
  if (nd + na == 0) return;
  k_check_batch<<<blocks_for(nd + na, kThreads, g->num_sms * 16), kThreads, 0, g->stream>>>(
      ds, dd, nd, as, ad, aw, na, g->n, g->ctl);
  ++*launches;
}

// A batch's five arrays from page-locked host memory (device addresses of
// the mapped arrays) into the device staging buffers: one launch with
// 16-byte loads across the host link wherever both sides are 16-byte
// aligned, so that the batch sort then reads device memory.
struct StageArgs {
  const int *src[5];
  int *dst[5];
  long long cnt[5];
};

__global__ void k_stage_inputs(StageArgs a) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  long long nv[5], most = 0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const bool vec =
        ((((unsigned long long)a.src[q]) | ((unsigned long long)a.dst[q])) & 15) == 0;
    nv[q] = vec ? a.cnt[q] / 4 : 0;
    most = nv[q] > most ? nv[q] : most;
  }
  // a thread's loads of all five arrays are in flight together (one
  // round trip across the link), then its stores
  for (long long i = tid; i < most; i += nt) {
    int4 v[5];
#pragma unroll
    for (int q = 0; q < 5; ++q)
      if (i < nv[q]) v[q] = __ldg((const int4 *)a.src[q] + i);
#pragma unroll
    for (int q = 0; q < 5; ++q)
      if (i < nv[q]) ((int4 *)a.dst[q])[i] = v[q];
  }
#pragma unroll
  for (int q = 0; q < 5; ++q)   // tails, and arrays that are not 16-byte aligned
    for (long long i = 4 * nv[q] + tid; i < a.cnt[q]; i += nt) a.dst[q][i] = __ldg(a.src[q] + i);
}

void launch_stage_inputs(sp_graph *g, const int *const src[5], int *const dst[5],
                         const long long cnt[5], int *launches) {
  StageArgs a;
  long long most = 0;
  for (int q = 0; q < 5; ++q) {
    a.src[q] = src[q];
    a.dst[q] = dst[q];
    a.cnt[q] = src[q] ? cnt[q] : 0;
    most = std::max(most, (a.cnt[q] + 3) / 4);
  }
  if (most == 0) return;
  k_stage_inputs<<<blocks_for(most, kThreads, g->num_sms * 8), kThreads, 0, g->stream>>>(a);
  ++*launches;
}

cudaError_t launch_search(sp_graph *g, const int *ds, const int *dd, long long nd,
                          const int *as, const int *ad, const int *aw, long long na,
                          int *launches, cudaStream_t stream) {
  const long long ni = 2 * (nd + na);
  if (ni == 0) return cudaSuccess;
  k_search<<<search_grid(g, ni), kCT, 0, stream>>>(search_args(g, ds, dd, nd, as, ad, aw, na));
  ++*launches;
  return cudaGetLastError();
}

const void *search_fn() { return (const void *)k_search; }

cudaError_t retarget_search(sp_graph *g, cudaGraphExec_t ex, cudaGraphNode_t node,
                            const int *ds, const int *dd, long long nd, const int *as,
                            const int *ad, const int *aw, long long na) {
  SearchArgs a = search_args(g, ds, dd, nd, as, ad, aw, na);
  void *args[1] = {&a};
  cudaKernelNodeParams p = {};
  p.func = (void *)k_search;
  p.gridDim = dim3(search_grid(g, 2 * (nd + na)));
  p.blockDim = dim3(kCT);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  return cudaGraphExecKernelNodeSetParams(ex, node, &p);
}

void launch_finish(sp_graph *g, int *launches) {
  k_finish<<<1, 256, 0, g->stream>>>(g->ctl, g->ctl_host);
  ++*launches;
}

}  // namespace sp
