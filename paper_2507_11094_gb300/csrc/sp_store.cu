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

#include "sp_graph.cuh"

namespace sp {

namespace {

constexpr int kThreads = 256;
constexpr int kSmallRow = 256;     // rows merged by one warp: deg <= this
constexpr int kSmallItems = 256;   // ... and at most this many batch items
constexpr int kPerLane = kSmallRow / 32;

inline unsigned blocks_for(long long work, int per_block, int cap) {
  long long b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

__device__ __forceinline__ void set_status(Ctl *c, int st) { atomicCAS(&c->status, 0, st); }

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
    cap_out[r] = (u64)row_capacity(last[r] - first[r], slack);
}

__global__ void k_row_meta(const long long *__restrict__ first, const long long *__restrict__ last,
                           const u64 *__restrict__ cap_scan, int n, float slack, RowMeta *row) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    long long d = last[r] - first[r];
    RowMeta rm;
    rm.start = (long long)cap_scan[r];
    rm.deg = (int)d;
    rm.cap = row_capacity(d, slack);
    row[r] = rm;
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

__global__ void k_ctl_reset(Ctl *c, int full) {
  c->status = 0;
  c->need_grow = 0;
  c->range_err = 0;
  c->timeout = 0;
  c->bad = 0;
  c->bar_arrive = 0;
  c->cur = 0;
  c->round = 0;
  c->done = 0;
  c->n_ent = c->n_edges = c->n_chunks = 0;
  c->qcnt0 = c->qcnt1 = c->acnt = 0;
  c->n_seg = c->n_small = c->n_medium = 0;
  c->large_pack = c->copy_pack = 0;
  c->pool_need[0] = c->pool_used[0];
  c->pool_need[1] = c->pool_used[1];
  c->scratch_used = 0;
  c->del_applied = c->del_absent = c->add_applied = c->add_present = 0;
  c->affected = c->seeds = c->relaxed = c->improved = 0;
  c->rows_touched = c->rows_relocated = 0;
  c->inval_edges = c->pull_edges = c->push_vertices = c->enqueued = 0;
  c->merge_slots = 0;
  c->rounds_inval = c->rounds_push = 0;
  if (full) {
    c->bar_gen = 0;
    c->epoch = 1;
    c->pool_used[0] = c->pool_used[1] = 0;
    c->pool_need[0] = c->pool_need[1] = 0;
  }
}

// Items of the batch: for update i, a forward item (row u, col v) at i and a
// reverse item (row v, col u) at nb + i; the low key bit is 0 for a deletion
// and 1 for an insertion, so a deletion sorts before an insertion of the
// same edge (deletions first, DynSSSP driver).
__global__ void k_prep(const int *__restrict__ ds, const int *__restrict__ dd, long long nd,
                       const int *__restrict__ as, const int *__restrict__ ad,
                       const int *__restrict__ aw, long long na, int n, int bits, u64 *keys,
                       u32 *vals, Ctl *ctl) {
  const long long nb = nd + na;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
       i += (long long)gridDim.x * blockDim.x) {
    int u, v, w = 0;
    u64 kind;
    bool ok;
    if (i < nd) {
      u = ds[i]; v = dd[i]; kind = 0;
      ok = u >= 0 && u < n && v >= 0 && v < n;
    } else {
      long long j = i - nd;
      u = as[j]; v = ad[j]; w = aw[j]; kind = 1;
      ok = u >= 0 && u < n && v >= 0 && v < n && w >= 1 && w <= SP_WMAX;
    }
    if (!ok) {
      set_status(ctl, SP_EINVAL);
      u = 0; v = 0;
    }
    keys[i] = ((u64)u << (bits + 1)) | ((u64)v << 1) | kind;
    keys[nb + i] = (1ull << (2 * bits + 1)) | ((u64)v << (bits + 1)) | ((u64)u << 1) | kind;
    vals[i] = (u32)w;
    vals[nb + i] = (u32)w;
  }
}

// --------------------------------------------------------------------------
// batch: segments (one per touched (store, row))
// --------------------------------------------------------------------------

__global__ void k_seg_heads(const u64 *__restrict__ keys, long long ni, int bits, u32 *head) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ni;
       i += (long long)gridDim.x * blockDim.x)
    head[i] = (i == 0 || (keys[i] >> (bits + 1)) != (keys[i - 1] >> (bits + 1))) ? 1u : 0u;
}

__global__ void k_seg_emit(const u64 *__restrict__ keys, const u32 *__restrict__ head,
                           const u32 *__restrict__ head_scan, long long ni, int bits, Seg *seg,
                           Ctl *ctl) {
  const u64 rmask = (1ull << bits) - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ni;
       i += (long long)gridDim.x * blockDim.x) {
    const u32 s = head_scan[i] + head[i] - 1;   // segment holding item i
    if (head[i]) {
      u64 rk = keys[i] >> (bits + 1);
      seg[s].first = (u32)i;
      seg[s].row = (int)(rk & rmask);
      seg[s].dir = (int)(rk >> bits);
    }
    if (i == ni - 1 || head[i + 1]) seg[s].end = (u32)(i + 1);
    if (i == ni - 1) ctl->n_seg = s + 1;
  }
}

// --------------------------------------------------------------------------
// batch: count pass (which updates apply, new row sizes, where rows go)
// --------------------------------------------------------------------------

constexpr int kMedRow = 4096;      // rows merged in place by one block
constexpr int kMedThreads = 512;
constexpr int kMedPer = kMedRow / kMedThreads;
constexpr int kLargeChunk = 4096;  // elements per block in the chunked tier
constexpr u64 kMask40 = (1ull << 40) - 1;

// First slot j in [0, deg) of a sorted row with row[j].x >= c.
__device__ __forceinline__ int row_lower_bound(const int2 *row, int deg, int c) {
  int lo = 0, hi = deg;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(&row[mid].x) < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// First item index in [lo, hi) whose key >= k.
__device__ __forceinline__ u32 items_lower_bound(const u64 *keys, u32 lo, u32 hi, u64 k) {
  while (lo < hi) {
    u32 mid = (lo + hi) >> 1;
    if (keys[mid] < k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct CountArgs {
  Ctl *ctl;
  const u64 *keys;
  const u32 *vals;
  Seg *seg;
  unsigned char *flags;
  u64 *itemv;
  const u64 *item_pref;
  u32 *small_list, *medium_list, *large_list, *large_cb, *copy_list, *copy_cb;
  Store st[2];
  int bits;
  float slack;
  long long scratch_cap;
  u32 n_items;
  int n;
};

// One thread per batch item: does this deletion / insertion apply?
//  - a deletion applies if the edge is in the row and it is the first
//    deletion of that edge in the batch;
//  - among the insertions of one edge the smallest weight is the candidate
//    (first on ties); it applies if the edge is absent after the deletions.
__global__ void __launch_bounds__(kThreads) k_count_items(CountArgs a) {
  Ctl *c = a.ctl;
  if (ld_cg_i32(&c->status) != 0) return;
  const int lane = threadIdx.x & 31;
  const u64 cmask = (1ull << a.bits) - 1;
  u64 del_ok = 0, del_abs = 0, add_ok = 0, add_pres = 0;
  const long long ni = a.n_items;
  for (long long base = blockIdx.x * (long long)blockDim.x; base < ni;
       base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    if (i < ni) {
      const u64 key = a.keys[i];
      const int dir = (int)(key >> (2 * a.bits + 1));
      const int row = (int)((key >> (a.bits + 1)) & cmask);
      const int col = (int)((key >> 1) & cmask);
      const Store &st = a.st[dir];
      const RowMeta rm = st.row[row];
      const int2 *old = st.adj + rm.start;
      const int j = row_lower_bound(old, rm.deg, col);
      const bool present = j < rm.deg && __ldg(&old[j].x) == col;
      if ((key & 1) == 0) {
        const bool applied = present && !(i > 0 && a.keys[i - 1] == key);
        a.flags[i] = applied ? 1 : 0;
        a.itemv[i] = applied ? 1ull : 0ull;
        if (dir == 0) { applied ? ++del_ok : ++del_abs; }
      } else if (i == 0 || a.keys[i - 1] != key) {  // first insertion of this edge
        long long j2 = i + 1, best = i;
        u32 bw = a.vals[i];
        while (j2 < ni && a.keys[j2] == key) {
          const u32 w2 = a.vals[j2];
          if (w2 < bw) { bw = w2; best = j2; }
          ++j2;
        }
        const bool del_exists = i > 0 && a.keys[i - 1] == (key ^ 1ull);
        const bool applied = !present || del_exists;
        for (long long t = i; t < j2; ++t) {
          const bool on = applied && t == best;
          a.flags[t] = on ? 1 : 0;
          a.itemv[t] = on ? (1ull << 32) : 0ull;
        }
        if (dir == 0) {
          add_ok += applied;
          add_pres += (u64)(j2 - i) - (applied ? 1 : 0);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    del_ok += __shfl_xor_sync(0xffffffffu, del_ok, o);
    del_abs += __shfl_xor_sync(0xffffffffu, del_abs, o);
    add_ok += __shfl_xor_sync(0xffffffffu, add_ok, o);
    add_pres += __shfl_xor_sync(0xffffffffu, add_pres, o);
  }
  if (lane == 0) {
    if (del_ok) atomicAdd(&c->del_applied, del_ok);
    if (del_abs) atomicAdd(&c->del_absent, del_abs);
    if (add_ok) atomicAdd(&c->add_applied, add_ok);
    if (add_pres) atomicAdd(&c->add_present, add_pres);
  }
}

// One thread per touched row: new size (from the item prefix counts), merge
// tier, destination (in place, or a fresh spare-pool segment when the row
// outgrows its capacity), scratch and chunk reservations.
__global__ void __launch_bounds__(kThreads) k_count_segs(CountArgs a) {
  Ctl *c = a.ctl;
  if (ld_cg_i32(&c->status) != 0) return;
  const int lane = threadIdx.x & 31;
  const u32 nseg = ld_cg_u32(&c->n_seg);
  u64 touched = 0, relocated = 0, slots = 0;
  for (u32 base = blockIdx.x * blockDim.x; base < nseg; base += gridDim.x * blockDim.x) {
    const u32 si = base + threadIdx.x;
    if (si >= nseg) continue;
    Seg sg = a.seg[si];
    if (sg.first >= sg.end || sg.end > a.n_items || sg.row < 0 || sg.row >= a.n ||
        sg.dir < 0 || sg.dir > 1) {  // never expected: record and skip
      atomicExch(&c->bad, 1);
      continue;
    }
    const Store &st = a.st[sg.dir];
    const RowMeta rm = st.row[sg.row];
    const u64 p = a.item_pref[sg.end] - a.item_pref[sg.first];
    const int new_deg = rm.deg - (int)(u32)p + (int)(u32)(p >> 32);
    const int nitems = (int)(sg.end - sg.first);
    sg.old_start = rm.start;
    sg.old_deg = rm.deg;
    sg.new_deg = new_deg;
    sg.scratch = -1;
    sg.tier = (rm.deg <= kSmallRow && nitems <= kSmallItems) ? 0
            : (rm.deg <= kMedRow && nitems <= kMedRow) ? 1 : 2;
    const bool reloc = new_deg > rm.cap;
    if (reloc) {
      long long nc = row_capacity(new_deg, a.slack);
      const long long dbl = round_up4(2LL * rm.cap);
      if (dbl > nc) nc = dbl;
      const u64 off = atomicAdd(&c->pool_need[sg.dir], (u64)nc);
      if ((long long)(off + nc) > st.slots - st.main_slots)
        atomicOr(&c->need_grow, sg.dir ? kGrowPoolRev : kGrowPoolFwd);
      sg.dest = st.main_slots + (long long)off;
      sg.new_cap = (int)nc;
      ++relocated;
    } else {
      sg.dest = rm.start;
      sg.new_cap = rm.cap;
    }
    if (sg.tier == 0) {
      a.small_list[atomicAdd(&c->n_small, 1u)] = si;
    } else if (sg.tier == 1) {
      a.medium_list[atomicAdd(&c->n_medium, 1u)] = si;
    } else {
      if (!reloc && new_deg > 0) {  // written to scratch, then copied back
        const u64 off = atomicAdd(&c->scratch_used, (u64)new_deg);
        if ((long long)(off + new_deg) > a.scratch_cap) atomicOr(&c->need_grow, kGrowScratch);
        sg.scratch = (long long)off;
        const u64 nch = (u64)((new_deg + kLargeChunk - 1) / kLargeChunk);
        const u64 o2 = atomicAdd((unsigned long long *)&c->copy_pack, (1ull << 40) | nch);
        a.copy_list[o2 >> 40] = si;
        a.copy_cb[o2 >> 40] = (u32)(o2 & kMask40);
      }
      const u64 nch = (u64)((rm.deg + nitems + kLargeChunk - 1) / kLargeChunk);
      const u64 o = atomicAdd((unsigned long long *)&c->large_pack, (1ull << 40) | nch);
      a.large_list[o >> 40] = si;
      a.large_cb[o >> 40] = (u32)(o & kMask40);
    }
    a.seg[si] = sg;
    ++touched;
    slots += (u64)rm.deg + (u64)new_deg;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    touched += __shfl_xor_sync(0xffffffffu, touched, o);
    relocated += __shfl_xor_sync(0xffffffffu, relocated, o);
    slots += __shfl_xor_sync(0xffffffffu, slots, o);
  }
  if (lane == 0) {
    if (touched) atomicAdd(&c->rows_touched, touched);
    if (relocated) atomicAdd(&c->rows_relocated, relocated);
    if (slots) atomicAdd(&c->merge_slots, slots);
  }
}

// --------------------------------------------------------------------------
// batch: merge pass (rewrite each touched row)
// --------------------------------------------------------------------------

struct MergeArgs {
  Ctl *ctl;
  const u64 *keys;
  const u32 *vals;
  const unsigned char *flags;
  const u64 *item_pref;   // exclusive scan of itemv, n_items + 1 entries
  const Seg *seg;
  const u32 *list, *list_cb;
  Store st[2];
  int2 *scratch;
  int bits;
};

__device__ __forceinline__ bool merge_enabled(Ctl *c) {
  return ld_cg_i32(&c->status) == 0 && ld_cg_i32(&c->need_grow) == 0 &&
         ld_cg_i32(&c->bad) == 0;
}

// Output slot of old entry j (col c) of a row, or -1 if the batch deletes it.
// Items with col < c are [first, i); the new row holds the kept old entries
// and the applied insertions in col order.
__device__ __forceinline__ int old_entry_pos(const MergeArgs &a, const Seg &sg, u64 prefix,
                                             u64 base_pref, int j, int c) {
  const u64 k = prefix | ((u64)(unsigned)c << 1);
  const u32 i = items_lower_bound(a.keys, sg.first, sg.end, k);
  if (i < sg.end && a.keys[i] == k && (a.flags[i] & 1)) return -1;  // applied deletion
  const u64 p = a.item_pref[i] - base_pref;
  return j - (int)(u32)p + (int)(u32)(p >> 32);
}

// Output slot of applied insertion item i (col c).
__device__ __forceinline__ int add_entry_pos(const MergeArgs &a, const Seg &sg, u64 prefix,
                                             u64 base_pref, const int2 *old, int deg, u32 i,
                                             int c) {
  const int pos_old = row_lower_bound(old, deg, c);
  const u32 i0 = items_lower_bound(a.keys, sg.first, i, prefix | ((u64)(unsigned)c << 1));
  const u64 p0 = a.item_pref[i0] - base_pref;
  const u64 pi = a.item_pref[i] - base_pref;
  return pos_old - (int)(u32)p0 + (int)(u32)(pi >> 32);
}

__device__ __forceinline__ void write_meta(const Store &st, const Seg &sg) {
  RowMeta nm;
  nm.start = sg.dest;
  nm.deg = sg.new_deg;
  nm.cap = sg.new_cap;
  st.row[sg.row] = nm;
}

// Tier 0: one warp per row with deg <= 256 and <= 256 items.  All reads go to
// registers before any write, so the row is rewritten in place.
__global__ void __launch_bounds__(kThreads) k_merge_small(MergeArgs a) {
  Ctl *c = a.ctl;
  if (!merge_enabled(c)) return;
  const int lane = threadIdx.x & 31;
  const u32 nlist = ld_cg_u32(&c->n_small);
  const u32 warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const u32 nwarps = (gridDim.x * blockDim.x) >> 5;
  const u64 cmask = (1ull << a.bits) - 1;
  for (u32 li = warp0; li < nlist; li += nwarps) {
    const Seg sg = a.seg[a.list[li]];
    const Store &st = a.st[sg.dir];
    const int2 *old = st.adj + sg.old_start;
    const u64 prefix = a.keys[sg.first] & ~((2ull << a.bits) - 1);
    const u64 base_pref = a.item_pref[sg.first];
    int2 ent[kPerLane];
    int pos[kPerLane];
#pragma unroll
    for (int t = 0; t < kPerLane; ++t) {
      const int j = lane + 32 * t;
      pos[t] = -1;
      if (j < sg.old_deg) {
        ent[t] = old[j];
        pos[t] = old_entry_pos(a, sg, prefix, base_pref, j, ent[t].x);
      }
    }
    int2 aent[kPerLane];
    int apos[kPerLane];
#pragma unroll
    for (int t = 0; t < kPerLane; ++t) {
      const u32 i = sg.first + lane + 32 * t;
      apos[t] = -1;
      if (i < sg.end && (a.keys[i] & 1) && (a.flags[i] & 1)) {
        const int col = (int)((a.keys[i] >> 1) & cmask);
        aent[t] = make_int2(col, (int)a.vals[i]);
        apos[t] = add_entry_pos(a, sg, prefix, base_pref, old, sg.old_deg, i, col);
      }
    }
    __syncwarp();
    int2 *dst = st.adj + sg.dest;
    bool bad = false;
#pragma unroll
    for (int t = 0; t < kPerLane; ++t) {
      if (pos[t] >= 0) {
        if (pos[t] < sg.new_deg) dst[pos[t]] = ent[t]; else bad = true;
      }
      if (apos[t] >= 0) {
        if (apos[t] < sg.new_deg) dst[apos[t]] = aent[t]; else bad = true;
      }
    }
    if (bad) atomicExch(&c->bad, 1);
    if (lane == 0) write_meta(st, sg);
    __syncwarp();
  }
}

// Tier 1: one block per row with deg <= 4096 and <= 4096 items, rewritten in
// place: every thread holds its entries in registers across a block barrier.
__global__ void __launch_bounds__(kMedThreads) k_merge_medium(MergeArgs a) {
  Ctl *c = a.ctl;
  if (!merge_enabled(c)) return;
  const u32 nlist = ld_cg_u32(&c->n_medium);
  const u64 cmask = (1ull << a.bits) - 1;
  for (u32 li = blockIdx.x; li < nlist; li += gridDim.x) {
    const Seg sg = a.seg[a.list[li]];
    const Store &st = a.st[sg.dir];
    const int2 *old = st.adj + sg.old_start;
    const u64 prefix = a.keys[sg.first] & ~((2ull << a.bits) - 1);
    const u64 base_pref = a.item_pref[sg.first];
    int2 ent[kMedPer];
    int pos[kMedPer];
#pragma unroll
    for (int t = 0; t < kMedPer; ++t) {
      const int j = threadIdx.x + kMedThreads * t;
      pos[t] = -1;
      if (j < sg.old_deg) {
        ent[t] = old[j];
        pos[t] = old_entry_pos(a, sg, prefix, base_pref, j, ent[t].x);
      }
    }
    int2 aent[kMedPer];
    int apos[kMedPer];
#pragma unroll
    for (int t = 0; t < kMedPer; ++t) {
      const u32 i = sg.first + threadIdx.x + kMedThreads * t;
      apos[t] = -1;
      if (i < sg.end && (a.keys[i] & 1) && (a.flags[i] & 1)) {
        const int col = (int)((a.keys[i] >> 1) & cmask);
        aent[t] = make_int2(col, (int)a.vals[i]);
        apos[t] = add_entry_pos(a, sg, prefix, base_pref, old, sg.old_deg, i, col);
      }
    }
    __syncthreads();
    int2 *dst = st.adj + sg.dest;
    bool bad = false;
#pragma unroll
    for (int t = 0; t < kMedPer; ++t) {
      if (pos[t] >= 0) {
        if (pos[t] < sg.new_deg) dst[pos[t]] = ent[t]; else bad = true;
      }
      if (apos[t] >= 0) {
        if (apos[t] < sg.new_deg) dst[apos[t]] = aent[t]; else bad = true;
      }
    }
    if (bad) atomicExch(&c->bad, 1);
    if (threadIdx.x == 0) write_meta(st, sg);
    __syncthreads();
  }
}

// Slot in a packed (count << 40 | chunks) list owning chunk `ch`.
__device__ __forceinline__ u32 chunk_owner(const u32 *cb, u32 count, u32 ch) {
  u32 lo = 0, hi = count - 1;
  while (lo < hi) {
    const u32 mid = (lo + hi + 1) >> 1;
    if (__ldcg(cb + mid) <= ch) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Tier 2: rows too large for one block, split into chunks of 4096 elements
// (old entries, then batch items) over all blocks.  Output goes out of place:
// to the row's new pool segment, or to scratch and then back (k_merge_copy),
// so no chunk reads a slot another chunk has rewritten.
__global__ void __launch_bounds__(kThreads) k_merge_large(MergeArgs a) {
  Ctl *c = a.ctl;
  if (!merge_enabled(c)) return;
  const u64 pk = ld_cg_u64(&c->large_pack);
  const u32 nlist = (u32)(pk >> 40), nch = (u32)(pk & kMask40);
  const u64 cmask = (1ull << a.bits) - 1;
  for (u32 ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const u32 slot = chunk_owner(a.list_cb, nlist, ch);
    const Seg sg = a.seg[__ldcg(a.list + slot)];
    const Store &st = a.st[sg.dir];
    const int2 *old = st.adj + sg.old_start;
    const u64 prefix = a.keys[sg.first] & ~((2ull << a.bits) - 1);
    const u64 base_pref = a.item_pref[sg.first];
    int2 *target = sg.scratch >= 0 ? a.scratch + sg.scratch : st.adj + sg.dest;
    const long long e0 = (long long)(ch - __ldcg(a.list_cb + slot)) * kLargeChunk;
    const long long ne = (long long)sg.old_deg + (sg.end - sg.first);
    const long long e1 = e0 + kLargeChunk < ne ? e0 + kLargeChunk : ne;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      if (e < sg.old_deg) {
        const int j = (int)e;
        const int2 en = old[j];
        const int p = old_entry_pos(a, sg, prefix, base_pref, j, en.x);
        if (p >= sg.new_deg) atomicExch(&c->bad, 1);
        else if (p >= 0) target[p] = en;
      } else {
        const u32 i = sg.first + (u32)(e - sg.old_deg);
        if ((a.keys[i] & 1) && (a.flags[i] & 1)) {
          const int col = (int)((a.keys[i] >> 1) & cmask);
          const int p = add_entry_pos(a, sg, prefix, base_pref, old, sg.old_deg, i, col);
          if (p < 0 || p >= sg.new_deg) atomicExch(&c->bad, 1);
          else target[p] = make_int2(col, (int)a.vals[i]);
        }
      }
    }
  }
}

// Tier 2, second pass: copy scratch back into rows merged in place, and
// publish the new row metadata of every tier-2 row.
__global__ void __launch_bounds__(kThreads) k_merge_copy(MergeArgs a, const u32 *large_list) {
  Ctl *c = a.ctl;
  if (!merge_enabled(c)) return;
  const u64 pk = ld_cg_u64(&c->copy_pack);
  const u32 nlist = (u32)(pk >> 40), nch = (u32)(pk & kMask40);
  for (u32 ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const u32 slot = chunk_owner(a.list_cb, nlist, ch);
    const Seg sg = a.seg[__ldcg(a.list + slot)];
    const int2 *src = a.scratch + sg.scratch;
    int2 *dst = a.st[sg.dir].adj + sg.dest;
    const long long e0 = (long long)(ch - __ldcg(a.list_cb + slot)) * kLargeChunk;
    const long long e1 = e0 + kLargeChunk < sg.new_deg ? e0 + kLargeChunk : sg.new_deg;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) dst[e] = __ldcg(src + e);
  }
  const u32 nl = (u32)(ld_cg_u64(&c->large_pack) >> 40);
  for (u32 li = blockIdx.x * blockDim.x + threadIdx.x; li < nl; li += gridDim.x * blockDim.x) {
    const Seg sg = a.seg[__ldcg(large_list + li)];
    write_meta(a.st[sg.dir], sg);
  }
}

__global__ void k_finish(Ctl *c) {
  if (c->status == 0 && c->need_grow == 0) {
    c->pool_used[0] = c->pool_need[0];
    c->pool_used[1] = c->pool_need[1];
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
      st->adj = (int2 *)g->al.get((size_t)st->slots * sizeof(int2));
      if (!st->row || !st->adj) rc = SP_ENOMEM;
    }
    if (rc == SP_OK) {
      k_row_meta<<<grid, kThreads, 0, s>>>(first, last, caps, n, g->slack, st->row);
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

sp_status ensure_owner_tables(sp_graph *g) {
  const long long slots = std::max(g->fwd.slots, g->rev.slots);
  const long long need = slots / kChunk + 64;
  if (need <= g->own_cap && g->qown[0]) return SP_OK;
  const long long c = std::max(need, g->own_cap * 2);
  g->al.put(g->qown[0], (size_t)g->own_cap * 4);
  g->al.put(g->qown[1], (size_t)g->own_cap * 4);
  g->al.put(g->aown, (size_t)g->own_cap * 4);
  g->qown[0] = (u32 *)g->al.get((size_t)c * 4);
  g->qown[1] = (u32 *)g->al.get((size_t)c * 4);
  g->aown = (u32 *)g->al.get((size_t)c * 4);
  g->own_cap = c;
  return (g->qown[0] && g->qown[1] && g->aown) ? SP_OK : SP_ENOMEM;
}

void launch_ctl_reset(sp_graph *g, int full, int *launches) {
  k_ctl_reset<<<1, 1, 0, g->stream>>>(g->ctl, full);
  ++*launches;
}

void launch_prep(sp_graph *g, const int *ds, const int *dd, long long nd, const int *as,
                 const int *ad, const int *aw, long long na, int *launches) {
  long long nb = nd + na;
  if (nb == 0) return;
  k_prep<<<blocks_for(nb, kThreads, g->num_sms * 16), kThreads, 0, g->stream>>>(
      ds, dd, nd, as, ad, aw, na, g->n, g->bits, g->bb.keys, g->bb.vals, g->ctl);
  ++*launches;
}

void launch_segments(sp_graph *g, long long ni, int *launches) {
  if (ni == 0) return;
  BatchBufs &b = g->bb;
  sort_pairs(b.keys, b.vals, b.keys_alt, b.vals_alt, ni, 2 * g->bits + 2, b.tmp, g->stream,
             launches);
  unsigned gb = blocks_for(ni, kThreads, g->num_sms * 16);
  k_seg_heads<<<gb, kThreads, 0, g->stream>>>(b.keys, ni, g->bits, b.head);
  scan_exclusive_u32(b.head, b.head_scan, ni, b.tmp, g->stream, launches);
  k_seg_emit<<<gb, kThreads, 0, g->stream>>>(b.keys, b.head, b.head_scan, ni, g->bits, b.seg,
                                             g->ctl);
  *launches += 2;
}

void launch_count(sp_graph *g, long long ni, int *launches) {
  if (ni == 0) return;
  BatchBufs &b = g->bb;
  CountArgs a;
  a.ctl = g->ctl;
  a.keys = b.keys;
  a.vals = b.vals;
  a.seg = b.seg;
  a.flags = b.flags;
  a.itemv = b.itemv;
  a.item_pref = b.item_pref;
  a.small_list = b.small_list;
  a.medium_list = b.medium_list;
  a.large_list = b.large_list;
  a.large_cb = b.large_cb;
  a.copy_list = b.copy_list;
  a.copy_cb = b.copy_cb;
  a.st[0] = g->fwd;
  a.st[1] = g->rev;
  a.bits = g->bits;
  a.slack = g->slack;
  a.scratch_cap = b.scratch_cap;
  a.n_items = (u32)ni;
  a.n = g->n;
  const unsigned grid = blocks_for(ni, kThreads, g->num_sms * 16);
  k_count_items<<<grid, kThreads, 0, g->stream>>>(a);
  // item prefix counts (n_items + 1 entries; itemv[ni] is 0)
  cudaMemsetAsync(b.itemv + ni, 0, sizeof(u64), g->stream);
  scan_exclusive_u64(b.itemv, b.item_pref, ni + 1, b.tmp, g->stream, launches);
  k_count_segs<<<grid, kThreads, 0, g->stream>>>(a);
  *launches += 2;
}

void launch_merge(sp_graph *g, long long ni, int *launches) {
  if (ni == 0) return;
  BatchBufs &b = g->bb;
  MergeArgs a;
  a.ctl = g->ctl;
  a.keys = b.keys;
  a.vals = b.vals;
  a.flags = b.flags;
  a.item_pref = b.item_pref;
  a.seg = b.seg;
  a.st[0] = g->fwd;
  a.st[1] = g->rev;
  a.scratch = b.scratch;
  a.bits = g->bits;
  a.list = b.small_list;
  a.list_cb = nullptr;
  k_merge_small<<<blocks_for(ni * 32, kThreads, g->num_sms * 16), kThreads, 0, g->stream>>>(a);
  a.list = b.medium_list;
  k_merge_medium<<<(unsigned)std::max(1, g->num_sms * 2), kMedThreads, 0, g->stream>>>(a);
  a.list = b.large_list;
  a.list_cb = b.large_cb;
  k_merge_large<<<(unsigned)std::max(1, g->num_sms * 8), kThreads, 0, g->stream>>>(a);
  a.list = b.copy_list;
  a.list_cb = b.copy_cb;
  k_merge_copy<<<(unsigned)std::max(1, g->num_sms * 8), kThreads, 0, g->stream>>>(
      a, b.large_list);
  *launches += 4;
}

void launch_finish(sp_graph *g, int *launches) {
  k_finish<<<1, 1, 0, g->stream>>>(g->ctl);
  ++*launches;
}

}  // namespace sp
