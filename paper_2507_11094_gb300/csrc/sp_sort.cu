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
#include "sp_internal.cuh"

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

}  // namespace

size_t sort_tmp_bytes(long long n) {
  long long tiles = (n + kTile - 1) / kTile;
  long long cnt = tiles * kBins;
  return (size_t)(2 * cnt + kBins + 64) * sizeof(u32) + 256;
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
