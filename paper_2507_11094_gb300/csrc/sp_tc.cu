// sp_tc.cu -- dynamic triangle count (paper, appendix listing "Dynamic TC
// coded in StarPlat DSL": staticTC, Decremental, Incremental, DynTC).
//
// The graph is read as undirected: every edge is stored in both directions
// (checked).  staticTC counts, for every vertex v, the pairs of neighbours
// u < v < w with u -> w an edge: every triangle once, at its middle vertex.
// A batch changes the count by the listing's corrections.  For every
// applied update (v1, v2) (each pair appears in both directions) and every
// common neighbour v3 of v1 and v2, the triangle {v1, v2, v3} is seen once
// per updated edge it contains and per direction, so with k of its three
// edges updated it is seen 2k times: the correction is
//     count1 / 2 + count2 / 4 + count3 / 6
// where count_k counts the sightings with k updated edges.  Deletions are
// counted on the graph before the merge (Decremental) and subtracted,
// insertions on the graph after it (Incremental) and added.  The common
// neighbours are found by walking the shorter of the two sorted rows and
// binary-searching the other, which finds the same set as the listing's
// walk over v1's row.
#include "sp_graph.cuh"

namespace sp {

namespace {

constexpr int kThreads = 256;
constexpr u32 kFull = 0xffffffffu;

__device__ __forceinline__ bool row_has(const int2 *row, int deg, int x) {
  int lo = 0, hi = deg;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&row[mid].x) < x) lo = mid + 1; else hi = mid;
  }
  return lo < deg && __ldg(&row[lo].x) == x;
}

__device__ __forceinline__ int row_lower(const int2 *row, int deg, int x) {
  int lo = 0, hi = deg;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&row[mid].x) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ u64 warp_sum64(u64 x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Every edge u -> v has its reverse v -> u (a warp per vertex).
__global__ void __launch_bounds__(kThreads) k_tc_sym_check(Store st, int n, Ctl *c) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = w0; u < n; u += nw) {
    const RowMeta ru = st.row[u];
    for (int e = lane; e < ru.deg; e += 32) {
      const int v = __ldg(&st.adj[ru.start + e].x);
      const RowMeta rv = st.row[v];
      if (!row_has(st.adj + rv.start, rv.deg, (int)u)) atomicCAS(&c->status, 0, SP_EINVAL);
    }
  }
}

// staticTC (a warp per vertex v): for every neighbour u < v, count the
// neighbours w > v of v that are neighbours of u.
__global__ void __launch_bounds__(kThreads) k_tc_static(Store st, int n, Ctl *c) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  u64 cnt = 0;
  for (long long v = w0; v < n; v += nw) {
    const RowMeta rv = st.row[v];
    const int2 *row = st.adj + rv.start;
    const int lo_end = row_lower(row, rv.deg, (int)v);        // neighbours < v
    int up = lo_end;
    if (up < rv.deg && __ldg(&row[up].x) == (int)v) ++up;     // skip a self-loop
    const int nup = rv.deg - up;                               // neighbours > v
    if (nup == 0) continue;
    for (int a = 0; a < lo_end; ++a) {
      const int u = __ldg(&row[a].x);
      const RowMeta ru = st.row[u];
      const int2 *urow = st.adj + ru.start;
      if (nup <= ru.deg) {
        for (int b = lane; b < nup; b += 32) cnt += row_has(urow, ru.deg, __ldg(&row[up + b].x));
      } else {
        // walk u's neighbours above v, search v's upper part
        const int s = row_lower(urow, ru.deg, (int)v + 1);
        for (int b = s + lane; b < ru.deg; b += 32)
          cnt += row_has(row + up, nup, __ldg(&urow[b].x));
      }
    }
  }
  cnt = warp_sum64(cnt);
  if (lane == 0 && cnt) atomicAdd(&c->tc_static, cnt);
}

// Is (x, y) an applied update of `kind` in the sorted forward items [0, nb)?
__device__ __forceinline__ bool item_applied(const u64 *keys, const unsigned char *flags,
                                             long long nb, int bits, u32 x, u32 y, u32 kind) {
  const u64 key = ((u64)x << (bits + 1)) | ((u64)y << 1) | kind;
  long long lo = 0, hi = nb;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if (__ldg(&keys[mid]) < key) lo = mid + 1; else hi = mid;
  }
  // equal keys (repeated updates): the applied one may be any of them
  for (long long i = lo; i < nb && __ldg(&keys[i]) == key; ++i)
    if (__ldg(&flags[i]) & 1) return true;
  return false;
}

// Every forward item has its reverse among the forward items (a thread per
// item); checked before anything changes.
__global__ void __launch_bounds__(kThreads) k_tc_batch_sym(const u64 *keys, long long nb, int bits,
                                                           Ctl *c) {
  const u64 cmask = (1ull << bits) - 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nb;
       i += (long long)gridDim.x * blockDim.x) {
    const u64 k = __ldg(&keys[i]);
    const u32 u = (u32)((k >> (bits + 1)) & cmask), v = (u32)((k >> 1) & cmask);
    const u64 r = ((u64)v << (bits + 1)) | ((u64)u << 1) | (k & 1);
    long long lo = 0, hi = nb;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (__ldg(&keys[mid]) < r) lo = mid + 1; else hi = mid;
    }
    if (lo >= nb || __ldg(&keys[lo]) != r) atomicCAS(&c->status, 0, SP_EINVAL);
  }
}

// The listing's correction for the applied forward items of `kind` (a warp
// per item): sightings of common neighbours v3 by the number of updated
// edges of the triangle, into cnt[0..2].
__global__ void __launch_bounds__(kThreads) k_tc_delta(const u64 *keys, const unsigned char *flags,
                                                       long long nb, int bits, u32 kind, Store st,
                                                       Ctl *c, int second) {
  if (ld_cg_i32(&c->status) != 0 || ld_cg_i32(&c->need_grow) != 0) return;
  const int lane = threadIdx.x & 31;
  const u64 cmask = (1ull << bits) - 1;
  const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  u64 k1 = 0, k2 = 0, k3 = 0;
  for (long long i = w0; i < nb; i += nw) {
    const u64 key = __ldg(&keys[i]);
    if ((key & 1) != kind || !(__ldg(&flags[i]) & 1)) continue;
    const u32 v1 = (u32)((key >> (bits + 1)) & cmask), v2 = (u32)((key >> 1) & cmask);
    if (v1 == v2) continue;
    const RowMeta r1 = st.row[v1], r2 = st.row[v2];
    const bool walk1 = r1.deg <= r2.deg;
    const int2 *wrow = st.adj + (walk1 ? r1.start : r2.start);
    const int wdeg = walk1 ? r1.deg : r2.deg;
    const int2 *srow = st.adj + (walk1 ? r2.start : r1.start);
    const int sdeg = walk1 ? r2.deg : r1.deg;
    for (int b = lane; b < wdeg; b += 32) {
      const u32 v3 = (u32)__ldg(&wrow[b].x);
      if (v3 == v1 || v3 == v2) continue;
      if (!row_has(srow, sdeg, (int)v3)) continue;
      const int k = 1 + item_applied(keys, flags, nb, bits, v1, v3, kind) +
                    item_applied(keys, flags, nb, bits, v2, v3, kind);
      k1 += k == 1;
      k2 += k == 2;
      k3 += k == 3;
    }
  }
  k1 = warp_sum64(k1);
  k2 = warp_sum64(k2);
  k3 = warp_sum64(k3);
  if (lane == 0) {
    u64 *dst = second ? c->tc_ins : c->tc_del;
    if (k1) atomicAdd(&dst[0], k1);
    if (k2) atomicAdd(&dst[1], k2);
    if (k3) atomicAdd(&dst[2], k3);
  }
}

inline unsigned grid_for(long long work, int per_block, int cap) {
  long long b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

}  // namespace

void launch_tc_sym_check(sp_graph *g, int *launches) {
  k_tc_sym_check<<<grid_for((long long)g->n * 32, kThreads, g->num_sms * 16), kThreads, 0,
                   g->stream>>>(g->fwd, g->n, g->ctl);
  ++*launches;
}

void launch_tc_static(sp_graph *g, int *launches) {
  k_tc_static<<<grid_for((long long)g->n * 32, kThreads, g->num_sms * 16), kThreads, 0,
                g->stream>>>(g->fwd, g->n, g->ctl);
  ++*launches;
}

void launch_tc_batch_sym(sp_graph *g, long long nb, int *launches) {
  if (nb == 0) return;
  k_tc_batch_sym<<<grid_for(nb, kThreads, g->num_sms * 16), kThreads, 0, g->stream>>>(
      g->bb.keys, nb, g->bits, g->ctl);
  ++*launches;
}

void launch_tc_delta(sp_graph *g, long long nb, int kind, int *launches) {
  if (nb == 0) return;
  k_tc_delta<<<grid_for(nb * 32, kThreads, g->num_sms * 16), kThreads, 0, g->stream>>>(
      g->bb.keys, g->bb.flags, nb, g->bits, (u32)kind, g->fwd, g->ctl, kind);
  ++*launches;
}

}  // namespace sp
