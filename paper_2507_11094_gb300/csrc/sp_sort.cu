// sp_sort.cu -- stable LSD radix sort of (u64 key, u32 value) pairs.
//
// Groups a batch's updates by (store, row, col) so that each touched row is
// merged once (updateCSRDel / updateCSRAdd of the DynSSSP driver, done as a
// sort-merge), and orders graph edges when a store is built.
//
// Per 9-bit digit:
//   k_hist       per-tile digit counts (count table is digit-major), for the
//                first digit only;
//   k_digit_scan one block per digit: prefix of its counts over the tiles,
//                and the digit's total; it also clears the other count table;
//   k_scatter    digit bases from the totals (block scan), then a stable
//                in-tile rank with warp match_any + per-warp digit counters;
//                every item it places also counts the next digit for the
//                output tile it lands in (into the other table), which
//                replaces the next pass's k_hist.
#include "sp_graph.cuh"

#include <algorithm>

namespace sp {

namespace {

constexpr int kBits = 9;
constexpr int kBins = 1 << kBits;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 4;
constexpr int kTile = kThreads * kItems;
constexpr int kBinsPerThread = kBins / kThreads;

__global__ void __launch_bounds__(kThreads)
k_hist(const u64 *__restrict__ keys, long long n, int shift, u32 *__restrict__ counts,
       u32 tiles) {
  __shared__ u32 h[kBins];
#pragma unroll
  for (int j = 0; j < kBinsPerThread; ++j) h[threadIdx.x + j * kThreads] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTile;
  u32 d[kItems];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {   // all loads first, then the counts
    long long i = base + k * kThreads + threadIdx.x;
    d[k] = i < n ? (u32)((keys[i] >> shift) & (kBins - 1)) : 0xFFFFFFFFu;
  }
#pragma unroll
  for (int k = 0; k < kItems; ++k)
    if (d[k] != 0xFFFFFFFFu) atomicAdd(&h[d[k]], 1u);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kBinsPerThread; ++j) {
    const int b = threadIdx.x + j * kThreads;
    counts[(long long)b * tiles + blockIdx.x] = h[b];
  }
}

__device__ __forceinline__ u32 warp_incl_scan(u32 x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ u32 block_excl_scan(u32 x, u32 *ws, u32 *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 incl = warp_incl_scan(x);
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    u32 v = lane < kWarps ? ws[lane] : 0u;
    v = warp_incl_scan(v);
    if (lane < kWarps) ws[lane] = v;
  }
  __syncthreads();
  const u32 r = (warp ? ws[warp - 1] : 0u) + incl - x;
  *total = ws[kWarps - 1];
  __syncthreads();
  return r;
}

// Block d: exclusive prefix of counts[d][0..tiles) in place, total to
// totals[d]; clears row d of `clear` (the next pass's table) when given.
__global__ void __launch_bounds__(kThreads)
k_digit_scan(u32 *__restrict__ counts, u32 tiles, u32 *__restrict__ totals,
             u32 *__restrict__ clear) {
  __shared__ u32 ws[kWarps];
  u32 *row = counts + (long long)blockIdx.x * tiles;
  if (clear) {
    u32 *crow = clear + (long long)blockIdx.x * tiles;
    for (u32 i = threadIdx.x; i < tiles; i += kThreads) crow[i] = 0;
  }
  const u32 per = (tiles + kThreads - 1) / kThreads;
  const u32 b = threadIdx.x * per < tiles ? threadIdx.x * per : tiles;
  const u32 e = b + per < tiles ? b + per : tiles;
  u32 sum = 0;
  for (u32 i = b; i < e; ++i) sum += row[i];
  u32 total;
  u32 run = block_excl_scan(sum, ws, &total);
  for (u32 i = b; i < e; ++i) {
    const u32 x = row[i];
    row[i] = run;
    run += x;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads)
k_scatter(const u64 *__restrict__ keys, const u32 *__restrict__ vals, long long n, int shift,
          const u32 *__restrict__ offs, const u32 *__restrict__ totals, u32 tiles,
          u64 *__restrict__ keys_out, u32 *__restrict__ vals_out, u32 *__restrict__ next_counts,
          int next_shift) {
  __shared__ u32 s_off[kBins];
  __shared__ u32 s_run[kBins];
  __shared__ u32 s_cnt[2][kWarps][kBins];
  __shared__ u32 ws[kWarps];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const long long base = (long long)blockIdx.x * kTile;
  u64 rk[kItems];
  u32 rv[kItems];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {   // the whole tile is in flight at once
    const long long i = base + k * kThreads + t;
    rk[k] = i < n ? keys[i] : 0ull;
    rv[k] = i < n ? vals[i] : 0u;
  }
  // digit bases: exclusive scan of the digit totals (each thread owns
  // kBinsPerThread consecutive digits)
  {
    u32 tot[kBinsPerThread], sum = 0;
#pragma unroll
    for (int j = 0; j < kBinsPerThread; ++j) {
      tot[j] = totals[t * kBinsPerThread + j];
      sum += tot[j];
    }
    u32 all;
    u32 run = block_excl_scan(sum, ws, &all);
#pragma unroll
    for (int j = 0; j < kBinsPerThread; ++j) {
      const int dgt = t * kBinsPerThread + j;
      s_off[dgt] = run + offs[(long long)dgt * tiles + blockIdx.x];
      run += tot[j];
      s_run[dgt] = 0;
    }
  }
#pragma unroll
  for (int j = 0; j < kBinsPerThread; ++j)
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s_cnt[0][w][t + j * kThreads] = 0;
  __syncthreads();
  const u32 lt = lanemask_lt();
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int p = k & 1;
    const long long i = base + k * kThreads + t;
    const bool valid = i < n;
    const u64 key = rk[k];
    const u32 val = rv[k];
    u32 d = valid ? (u32)((key >> shift) & (kBins - 1)) : (u32)(kBins + lane);
    u32 peers = __match_any_sync(0xffffffffu, d);
    u32 rank = __popc(peers & lt);
    if (valid && rank == 0) s_cnt[p][warp][d] = __popc(peers);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBinsPerThread; ++j) {   // digit-owners: scan over warps
      const int dgt = t + j * kThreads;
      u32 run = s_run[dgt];
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        u32 c = s_cnt[p][w][dgt];
        s_cnt[p][w][dgt] = run;
        run += c;
        s_cnt[p ^ 1][w][dgt] = 0;
      }
      s_run[dgt] = run;
    }
    __syncthreads();
    if (valid) {
      u32 pos = s_off[d] + s_cnt[p][warp][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
      if (next_counts) {
        const u32 nd = (u32)((key >> next_shift) & (kBins - 1));
        atomicAdd(next_counts + (long long)nd * tiles + pos / kTile, 1u);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The batch sort: one cooperative launch builds the items of a batch, sorts
// them by (store, row, col, kind) and emits one segment per touched
// (store, row) -- the grouping that lets every touched row be merged once
// (updateCSRDel + updateCSRAdd of the DynSSSP driver as one sort-merge).
//
// Block b owns the contiguous chunk [b*C, (b+1)*C) of item positions.  Per
// 9-bit digit pass:
//   1. the block counts the digit over its chunk and writes the counts as
//      row b of a table (chunk-major);                     -- grid barrier
//   2. thread d reads column d (coalesced across the warp): the digit's
//      total and its count in earlier chunks; a block scan of the totals
//      gives the digit bases;
//   3. per sub-tile of kBTile items (warp w holds items w*256 .. w*256+255,
//      eight per lane): each warp ranks its items with match_any against
//      warp-private digit counters, one scan over the warps per digit
//      turns those into offsets, the items are staged in shared memory in
//      digit order and written out so that consecutive threads store
//      consecutive positions of a digit's run.             -- grid barrier
// A chunk of one sub-tile keeps its items in registers from the count to
// the scatter.  Data other blocks wrote is read through L2 (.cg), and
// loads are issued in unrolled batches so that their latencies overlap.
// ---------------------------------------------------------------------------
constexpr int kBT = 512;                  // threads per block (one digit each)
constexpr int kBW = kBT / 32;
constexpr int kBItems = 8;
constexpr int kBTile = kBT * kBItems;     // items per sub-tile
constexpr int kBWarpItems = 32 * kBItems; // items per warp and sub-tile
static_assert(kBT == kBins, "one digit per thread");
// dynamic shared memory: staged keys and values, per-warp digit counters,
// four per-digit arrays
constexpr size_t kBSmem =
    (size_t)kBTile * (sizeof(u64) + sizeof(u32)) + (size_t)(kBW * kBins + 4 * kBins) * 4;

struct BatchSortArgs {
  const int *ds, *dd, *as, *ad, *aw;
  long long nd, na;
  int n, bits, passes;
  u64 *kbuf[2];
  u32 *vbuf[2];
  u32 *tab;          // [G][kBins] digit counts per chunk
  Seg *seg;
  Ctl *ctl;
  unsigned long long wait_ns;
  u32 miss_site;         // test hook of the bounded waits (Limits::miss_site)
  u32 n_items, chunk;
};

// Block-wide exclusive scan over kBT threads.
__device__ __forceinline__ u32 bscan512(u32 x, u32 *ws, u32 *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u32 incl = warp_incl_scan(x);
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    u32 v = lane < kBW ? ws[lane] : 0u;
    v = warp_incl_scan(v);
    if (lane < kBW) ws[lane] = v;
  }
  __syncthreads();
  const u32 r = (warp ? ws[warp - 1] : 0u) + incl - x;
  *total = ws[kBW - 1];
  __syncthreads();
  return r;
}

// Lanes of the warp whose valid item has the same 9-bit digit (the answer of
// a match_any, built from one ballot per digit bit).
__device__ __forceinline__ u32 digit_peers(u32 d, bool valid) {
  u32 peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int bb = 0; bb < kBits; ++bb) {
    const bool on = (d >> bb) & 1;
    const u32 bal = __ballot_sync(0xffffffffu, on);
    peers &= on ? bal : ~bal;
  }
  return peers;
}

__device__ __forceinline__ u64 shfl64_up1(u64 x) {
  const u32 lo = __shfl_up_sync(0xffffffffu, (u32)x, 1);
  const u32 hi = __shfl_up_sync(0xffffffffu, (u32)(x >> 32), 1);
  return ((u64)hi << 32) | lo;
}

// Position of item k of this thread in its sub-tile.
__device__ __forceinline__ u32 sub_pos(int k) {
  return (threadIdx.x >> 5) * kBWarpItems + k * 32 + (threadIdx.x & 31);
}

__global__ void __launch_bounds__(kBT) k_batch_sort(BatchSortArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  u64 *s_key = (u64 *)smraw;                         // [kBTile]
  u32 *s_val = (u32 *)(s_key + kBTile);              // [kBTile]
  u32 *s_wc = s_val + kBTile;                        // [kBW][kBins] per-warp digit counts
  u32 *s_off = s_wc + kBW * kBins;                   // global start of digit (next sub-tile)
  u32 *s_run = s_off + kBins;
  u32 *s_loc = s_run + kBins;                        // sub-tile start of digit
  u32 *s_hist = s_loc + kBins;                       // digit counts
  __shared__ u32 ws[kBW];
  Ctl *c = a.ctl;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const u32 G = gridDim.x, b = blockIdx.x;
  const u32 cb = min(b * a.chunk, a.n_items), ce = min(cb + a.chunk, a.n_items);
  const bool one = ce - cb <= (u32)kBTile;           // the chunk is one sub-tile
  u64 *bar = &c->bar_sort;
  u64 nbar = 0;
  const long long nb = a.nd + a.na;
  const int bits = a.bits;
  const u32 lt = lanemask_lt();
  u64 rk[kBItems];
  u32 rv[kBItems];

  // the items (forward item of update i at i, reverse item at nb + i; the
  // low key bit is 0 for a deletion and 1 for an insertion, so a deletion
  // sorts before an insertion of the same edge) with the first digit's
  // counts; an invalid id or weight raises SP_EINVAL (nothing will change)
  s_hist[t] = 0;
  __syncthreads();
  for (u32 tb = cb; tb < ce; tb += kBTile) {
    int u[kBItems], v[kBItems], w[kBItems];
#pragma unroll
    for (int k = 0; k < kBItems; ++k) {   // every load first
      const u32 i = tb + sub_pos(k);
      u[k] = 0; v[k] = 0; w[k] = 0;
      if (i < ce) {
        const long long j = (long long)i >= nb ? (long long)i - nb : (long long)i;
        if (j < a.nd) {
          u[k] = __ldg(a.ds + j); v[k] = __ldg(a.dd + j); w[k] = 0;
        } else {
          const long long q = j - a.nd;
          u[k] = __ldg(a.as + q); v[k] = __ldg(a.ad + q); w[k] = __ldg(a.aw + q);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kBItems; ++k) {
      const u32 i = tb + sub_pos(k);
      rk[k] = 0;
      rv[k] = 0;
      if (i < ce) {
        const bool rev = (long long)i >= nb;
        const long long j = rev ? (long long)i - nb : (long long)i;
        const u64 kind = j < a.nd ? 0 : 1;
        const bool ok = u[k] >= 0 && u[k] < a.n && v[k] >= 0 && v[k] < a.n &&
                        (kind == 0 || (w[k] >= 1 && w[k] <= SP_WMAX));
        if (!ok) {
          atomicCAS(&c->status, 0, SP_EINVAL);
          u[k] = 0; v[k] = 0;
        }
        rk[k] = rev ? (1ull << (2 * bits + 1)) | ((u64)v[k] << (bits + 1)) | ((u64)u[k] << 1) | kind
                    : ((u64)u[k] << (bits + 1)) | ((u64)v[k] << 1) | kind;
        rv[k] = i;   // the item's own number: its search result and weight (k_search)
      }
    }
#pragma unroll
    for (int k = 0; k < kBItems; ++k) {
      const u32 i = tb + sub_pos(k);
      if (i < ce) {
        a.kbuf[0][i] = rk[k];
        a.vbuf[0][i] = rv[k];
        atomicAdd(&s_hist[rk[k] & (kBins - 1)], 1u);
      }
    }
  }
  __syncthreads();
  a.tab[(size_t)b * kBins + t] = s_hist[t];

  for (int p = 0; p < a.passes; ++p) {
    if (coop_barrier(bar, ++nbar * G, c, a.wait_ns, 4, a.miss_site)) return;
    const int shift = p * kBits;
    // digit bases of this chunk: thread t sums digits 4*(t % 128) .. +3 over
    // the rows q = t / 128 (mod 4) with 16-byte loads; the four partial sums
    // of each digit meet in shared memory (s_loc holds the totals, s_run the
    // counts of earlier chunks)
    {
      const u32 dq = (u32)(t & 127) * 4, rg = (u32)t >> 7;
      uint4 tot = make_uint4(0u, 0u, 0u, 0u), pre = tot;
      for (u32 q0 = rg; q0 < G; q0 += 4 * 8) {
        uint4 x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const u32 q = q0 + 4 * u;
          x[u] = q < G ? __ldcg((const uint4 *)(a.tab + (size_t)q * kBins + dq))
                       : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool before = q0 + 4 * u < b;
          tot.x += x[u].x; tot.y += x[u].y; tot.z += x[u].z; tot.w += x[u].w;
          if (before) { pre.x += x[u].x; pre.y += x[u].y; pre.z += x[u].z; pre.w += x[u].w; }
        }
      }
      s_loc[t] = 0;
      s_run[t] = 0;
      __syncthreads();
      atomicAdd(&s_loc[dq], tot.x); atomicAdd(&s_loc[dq + 1], tot.y);
      atomicAdd(&s_loc[dq + 2], tot.z); atomicAdd(&s_loc[dq + 3], tot.w);
      atomicAdd(&s_run[dq], pre.x); atomicAdd(&s_run[dq + 1], pre.y);
      atomicAdd(&s_run[dq + 2], pre.z); atomicAdd(&s_run[dq + 3], pre.w);
      __syncthreads();
      u32 all;
      const u32 base = bscan512(s_loc[t], ws, &all);
      s_off[t] = base + s_run[t];
    }
    const u64 *kin = a.kbuf[p & 1];
    const u32 *vin = a.vbuf[p & 1];
    u64 *kout = a.kbuf[(p + 1) & 1];
    u32 *vout = a.vbuf[(p + 1) & 1];
    for (u32 tb = cb; tb < ce; tb += kBTile) {
      if (!one) {   // this sub-tile's items and digit counts
#pragma unroll
        for (int k = 0; k < kBItems; ++k) {
          const u32 i = tb + sub_pos(k);
          rk[k] = i < ce ? __ldcg(kin + i) : 0ull;
          rv[k] = i < ce ? __ldcg(vin + i) : 0u;
        }
        s_hist[t] = 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kBItems; ++k)
          if (tb + sub_pos(k) < ce) atomicAdd(&s_hist[(rk[k] >> shift) & (kBins - 1)], 1u);
        __syncthreads();
      }
      {
        u32 all;
        s_loc[t] = bscan512(s_hist[t], ws, &all);
#pragma unroll
        for (int w = 0; w < kBW; ++w) s_wc[w * kBins + t] = 0;
      }
      __syncthreads();
      // stable rank within the warp's items (rows k, then lanes)
      u32 lr[kBItems];
      u32 *wc = s_wc + warp * kBins;
#pragma unroll
      for (int k = 0; k < kBItems; ++k) {
        const bool valid = tb + sub_pos(k) < ce;
        const u32 d = (u32)((rk[k] >> shift) & (kBins - 1));
        const u32 peers = digit_peers(d, valid);
        const u32 rank = __popc(peers & lt);
        const u32 before = valid ? wc[d] : 0u;
        __syncwarp();
        if (valid && rank == 0) wc[d] = before + __popc(peers);
        __syncwarp();
        lr[k] = before + rank;
      }
      __syncthreads();
      {   // digit t: offsets of the warps
        u32 run = 0;
#pragma unroll
        for (int w = 0; w < kBW; ++w) {
          const u32 x = s_wc[w * kBins + t];
          s_wc[w * kBins + t] = run;
          run += x;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kBItems; ++k) {
        if (tb + sub_pos(k) < ce) {
          const u32 d = (u32)((rk[k] >> shift) & (kBins - 1));
          const u32 lp = s_loc[d] + wc[d] + lr[k];
          s_key[lp] = rk[k];
          s_val[lp] = rv[k];
        }
      }
      __syncthreads();
      // write out in digit order: a digit's items are consecutive in both
#pragma unroll
      for (int k = 0; k < kBItems; ++k) {
        const u32 j = k * kBT + t;
        if (tb + j < ce) {
          const u64 key = s_key[j];
          const u32 d = (u32)((key >> shift) & (kBins - 1));
          const u32 pos = s_off[d] + (j - s_loc[d]);
          kout[pos] = key;
          vout[pos] = s_val[j];
        }
      }
      __syncthreads();
      s_off[t] += s_hist[t];
      __syncthreads();
    }
    if (coop_barrier(bar, ++nbar * G, c, a.wait_ns, 4, a.miss_site)) return;
    if (p + 1 < a.passes) {   // the next digit's counts over this chunk
      const int nshift = shift + kBits;
      s_hist[t] = 0;
      __syncthreads();
      for (u32 tb = cb; tb < ce; tb += kBTile) {
#pragma unroll
        for (int k = 0; k < kBItems; ++k) {
          const u32 i = tb + sub_pos(k);
          rk[k] = i < ce ? __ldcg(kout + i) : 0ull;
          if (one) rv[k] = i < ce ? __ldcg(vout + i) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kBItems; ++k)
          if (tb + sub_pos(k) < ce) atomicAdd(&s_hist[(rk[k] >> nshift) & (kBins - 1)], 1u);
      }
      __syncthreads();
      a.tab[(size_t)b * kBins + t] = s_hist[t];
    }
  }

  // segments: a head is an item whose (store, row) differs from its
  // predecessor's.  Items sit as in the passes (warp w, row k, lane), so a
  // predecessor is one lane back (or the previous row's last lane); heads
  // become ballot masks, a segment ends at the next head -- in the same
  // row, a later row, a later warp of the block (a minimum over the warps),
  // or, only for a row of the graph that runs past the sub-tile, where a
  // galloping search finds it.
  const u64 *keys = a.kbuf[a.passes & 1];
  const u32 n = a.n_items;
  const int hs = bits + 1;
  for (u32 tb = cb; tb < ce; tb += kBTile) {
    const u32 te = tb + kBTile < ce ? tb + kBTile : ce;
    u64 pf[kBItems];
    u32 hm[kBItems];
#pragma unroll
    for (int k = 0; k < kBItems; ++k) {
      const u32 i = tb + sub_pos(k);
      pf[k] = i < te ? __ldcg(keys + i) >> hs : 0ull;
    }
    const u32 w0 = tb + (u32)warp * kBWarpItems;   // the warp's first position
    const u64 before0 = (w0 > 0 && w0 < te) ? __ldcg(keys + w0 - 1) >> hs : ~0ull;
    u32 nh = 0;
#pragma unroll
    for (int k = 0; k < kBItems; ++k) {
      const u32 i = tb + sub_pos(k);
      u64 pred = shfl64_up1(pf[k]);
      const u64 last_prev = __shfl_sync(0xffffffffu, (u32)(k ? pf[k - 1] : before0), 31) |
                            ((u64)__shfl_sync(0xffffffffu, (u32)((k ? pf[k - 1] : before0) >> 32), 31) << 32);
      if (lane == 0) pred = k ? last_prev : before0;
      const bool head = i < te && (i == 0 || pf[k] != pred);
      hm[k] = __ballot_sync(0xffffffffu, head);
      nh += __popc(hm[k]);
    }
    // the warp's first head, its head count, then the block's prefix
    u32 first = 0xFFFFFFFFu;
#pragma unroll
    for (int k = kBItems - 1; k >= 0; --k)
      if (hm[k]) first = w0 + (u32)k * 32 + (u32)(__ffs(hm[k]) - 1);
    if (lane == 0) {
      s_hist[warp] = nh;
      s_loc[warp] = first;
    }
    __syncthreads();
    if (t == 0) {
      u32 tot = 0;
      for (int w = 0; w < kBW; ++w) {
        const u32 x = s_hist[w];
        s_hist[w] = tot;
        tot += x;
      }
      s_run[0] = tot ? atomicAdd(&c->n_seg, tot) : 0u;
    }
    u32 after = 0xFFFFFFFFu;   // first head of a later warp
    for (int w = warp + 1; w < kBW; ++w) after = min(after, s_loc[w]);
    __syncthreads();
    u32 sidx = s_run[0] + s_hist[warp];
#pragma unroll
    for (int k = 0; k < kBItems; ++k) {
      const u32 mine = hm[k] & lt;
      if ((hm[k] >> lane) & 1) {
        const u32 i = tb + sub_pos(k);
        const u64 pfx = pf[k];
        u32 end = 0xFFFFFFFFu;
        const u32 above = hm[k] & ~((2u << lane) - 1);   // later heads in this row
        if (above) {
          end = w0 + (u32)k * 32 + (u32)(__ffs(above) - 1);
        } else {
#pragma unroll
          for (int k2 = k + 1; k2 < kBItems; ++k2)
            if (end == 0xFFFFFFFFu && hm[k2]) end = w0 + (u32)k2 * 32 + (u32)(__ffs(hm[k2]) - 1);
        }
        if (end == 0xFFFFFFFFu) end = after;
        if (end == 0xFFFFFFFFu) {   // the row runs past the sub-tile
          u32 lo = te, step = 1;
          u32 hi = lo;
          while (hi < n && (__ldcg(keys + hi) >> hs) == pfx) {
            lo = hi + 1;
            hi = lo + step < n ? lo + step : n;
            step <<= 1;
          }
          while (lo < hi) {   // first item of another (store, row) in [lo, hi]
            const u32 mid = (lo + hi) >> 1;
            if ((__ldcg(keys + mid) >> hs) == pfx) lo = mid + 1; else hi = mid;
          }
          end = lo;
        }
        Seg &sg = a.seg[sidx + __popc(mine)];
        sg.first = i;
        sg.end = end;
        sg.row = (int)(pfx & ((1ull << bits) - 1));
        sg.dir = (int)(pfx >> bits);
      }
      sidx += __popc(hm[k]);
    }
    __syncthreads();
  }
}

}  // namespace

size_t sort_tmp_bytes(long long n) {
  long long tiles = (n + kTile - 1) / kTile;
  long long cnt = tiles * kBins;
  return (size_t)(2 * cnt + kBins + 64) * sizeof(u32) + 256;
}

int batch_sort_blocks(int num_sms) {
  int per_sm = 0;
  if (cudaFuncSetAttribute(k_batch_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)std::max(kBSmem, kExclusiveSmem)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_sort, kBT, kBSmem) !=
          cudaSuccess ||
      per_sm < 1)
    return 0;
  return per_sm * num_sms;
}

size_t batch_sort_tmp_bytes(int max_blocks) {
  return (size_t)kBins * std::max(max_blocks, 1) * sizeof(u32) + 256;
}

namespace {

// Dynamic shared memory of a launch: a handle with a block share gives each
// block an SM of its own (kExclusiveSmem).
size_t sort_smem(const sp_graph *g) {
  return g->loop_blocks_user > 0 ? std::max(kBSmem, kExclusiveSmem) : kBSmem;
}

// Arguments and grid of the batch sort for these inputs.
int batch_sort_args(sp_graph *g, const int *ds, const int *dd, long long nd, const int *as,
                    const int *ad, const int *aw, long long na, BatchSortArgs &a) {
  const long long ni = 2 * (nd + na);
  BatchBufs &bb = g->bb;
  int G = (int)std::min<long long>((ni + kBTile - 1) / kBTile, g->sort_blocks);
  if (g->loop_blocks_user > 0 && g->loop_blocks_user < G) G = g->loop_blocks_user;
  if (G < 1) G = 1;
  a.ds = ds; a.dd = dd; a.as = as; a.ad = ad; a.aw = aw;
  a.nd = nd; a.na = na;
  a.n = g->n;
  a.bits = g->bits;
  const int key_bits = 2 * g->bits + 2;
  a.passes = (key_bits + kBits - 1) / kBits;
  // the last pass writes keys/vals
  const int odd = a.passes & 1;
  a.kbuf[0] = odd ? bb.keys_alt : bb.keys;
  a.kbuf[1] = odd ? bb.keys : bb.keys_alt;
  a.vbuf[0] = odd ? bb.vals_alt : bb.vals;
  a.vbuf[1] = odd ? bb.vals : bb.vals_alt;
  a.tab = (u32 *)bb.tmp;
  a.seg = bb.seg;
  a.ctl = g->ctl;
  a.wait_ns = g->lim.wait_ns;
  a.miss_site = g->lim.miss_site;
  a.n_items = (u32)ni;
  a.chunk = (u32)((ni + G - 1) / G);
  return G;
}

}  // namespace

const void *batch_sort_fn() { return (const void *)k_batch_sort; }

cudaError_t launch_batch_sort(sp_graph *g, const int *ds, const int *dd, long long nd,
                              const int *as, const int *ad, const int *aw, long long na,
                              int *launches) {
  if (nd + na == 0) return cudaSuccess;
  BatchSortArgs a;
  const int G = batch_sort_args(g, ds, dd, nd, as, ad, aw, na, a);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = sort_smem(g);
  cfg.stream = g->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++*launches;
  return cudaLaunchKernelEx(&cfg, k_batch_sort, a);
}

cudaError_t retarget_batch_sort(sp_graph *g, cudaGraphExec_t ex, cudaGraphNode_t node,
                                const int *ds, const int *dd, long long nd, const int *as,
                                const int *ad, const int *aw, long long na) {
  BatchSortArgs a;
  const int G = batch_sort_args(g, ds, dd, nd, as, ad, aw, na, a);
  void *args[1] = {&a};
  cudaKernelNodeParams p = {};
  p.func = (void *)k_batch_sort;
  p.gridDim = dim3((unsigned)G);
  p.blockDim = dim3(kBT);
  p.sharedMemBytes = (unsigned)sort_smem(g);
  p.kernelParams = args;
  return cudaGraphExecKernelNodeSetParams(ex, node, &p);
}

void sort_pairs(u64 *keys, u32 *vals, u64 *keys_alt, u32 *vals_alt, long long n,
                int key_bits, void *tmp, cudaStream_t st, int *launches) {
  if (n <= 1 || key_bits <= 0) return;
  const u32 tiles = (u32)((n + kTile - 1) / kTile);
  const long long cnt = (long long)tiles * kBins;
  u32 *counts[2] = {(u32 *)tmp, (u32 *)tmp + cnt};
  u32 *totals = counts[1] + cnt;
  u64 *kin = keys, *kout = keys_alt;
  u32 *vin = vals, *vout = vals_alt;
  int passes = (key_bits + kBits - 1) / kBits;
  k_hist<<<tiles, kThreads, 0, st>>>(kin, n, 0, counts[0], tiles);
  if (launches) *launches += 1;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kBits;
    const bool more = pass + 1 < passes;
    u32 *cur = counts[pass & 1], *nxt = more ? counts[(pass + 1) & 1] : nullptr;
    k_digit_scan<<<kBins, kThreads, 0, st>>>(cur, tiles, totals, nxt);
    k_scatter<<<tiles, kThreads, 0, st>>>(kin, vin, n, shift, cur, totals, tiles, kout, vout, nxt,
                                          shift + kBits);
    if (launches) *launches += 2;
    u64 *tk = kin; kin = kout; kout = tk;
    u32 *tv = vin; vin = vout; vout = tv;
  }
  if (kin != keys) {
    cudaMemcpyAsync(keys, kin, (size_t)n * sizeof(u64), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vals, vin, (size_t)n * sizeof(u32), cudaMemcpyDeviceToDevice, st);
  }
}

}  // namespace sp
