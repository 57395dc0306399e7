// sp_sort.cu -- stable LSD radix sort of (u64 key, u32 value) pairs.
//
// Groups a batch's updates by (store, row, col) so that each touched row is
// merged once (updateCSRDel / updateCSRAdd of the DynSSSP driver, done as a
// sort-merge), and orders graph edges when a store is built.
//
// Per 8-bit digit: a histogram kernel (per-tile digit counts), a device-wide
// scan of the digit-major count table, and a scatter kernel that ranks keys
// stably inside the tile with warp match_any + per-warp digit counters.
#include "sp_internal.cuh"

namespace sp {

namespace {

constexpr int kBits = 8;
constexpr int kBins = 1 << kBits;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

__global__ void __launch_bounds__(kThreads)
k_hist(const u64 *__restrict__ keys, long long n, int shift, u32 *__restrict__ counts,
       u32 tiles) {
  __shared__ u32 h[kBins];
  h[threadIdx.x] = 0;
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
  counts[(long long)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads)
k_scatter(const u64 *__restrict__ keys, const u32 *__restrict__ vals, long long n, int shift,
          const u32 *__restrict__ offs, u32 tiles, u64 *__restrict__ keys_out,
          u32 *__restrict__ vals_out) {
  __shared__ u32 s_off[kBins];
  __shared__ u32 s_run[kBins];
  __shared__ u32 s_cnt[2][kWarps][kBins];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  s_off[t] = offs[(long long)t * tiles + blockIdx.x];
  s_run[t] = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s_cnt[0][w][t] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTile;
  const u32 lt = lanemask_lt();
  u64 rk[kItems];
  u32 rv[kItems];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {   // the whole tile is in flight at once
    const long long i = base + k * kThreads + t;
    rk[k] = i < n ? keys[i] : 0ull;
    rv[k] = i < n ? vals[i] : 0u;
  }
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
    {  // thread t owns digit t: exclusive scan over warps, carry across k
      u32 run = s_run[t];
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        u32 c = s_cnt[p][w][t];
        s_cnt[p][w][t] = run;
        run += c;
        s_cnt[p ^ 1][w][t] = 0;
      }
      s_run[t] = run;
    }
    __syncthreads();
    if (valid) {
      u32 pos = s_off[d] + s_cnt[p][warp][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
  }
}

}  // namespace

size_t sort_tmp_bytes(long long n) {
  long long tiles = (n + kTile - 1) / kTile;
  long long cnt = tiles * kBins;
  return (size_t)(2 * cnt + 64) * sizeof(u32) + scan_tmp_bytes(cnt) + 256;
}

void sort_pairs(u64 *keys, u32 *vals, u64 *keys_alt, u32 *vals_alt, long long n,
                int key_bits, void *tmp, cudaStream_t st, int *launches) {
  if (n <= 1 || key_bits <= 0) return;
  const u32 tiles = (u32)((n + kTile - 1) / kTile);
  const long long cnt = (long long)tiles * kBins;
  u32 *counts = (u32 *)tmp;
  u32 *offs = counts + cnt;
  void *scan_tmp = (void *)(((uintptr_t)(offs + cnt) + 255) & ~(uintptr_t)255);
  u64 *kin = keys, *kout = keys_alt;
  u32 *vin = vals, *vout = vals_alt;
  int passes = (key_bits + kBits - 1) / kBits;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kBits;
    k_hist<<<tiles, kThreads, 0, st>>>(kin, n, shift, counts, tiles);
    scan_exclusive_u32(counts, offs, cnt, scan_tmp, st, launches);
    k_scatter<<<tiles, kThreads, 0, st>>>(kin, vin, n, shift, offs, tiles, kout, vout);
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
