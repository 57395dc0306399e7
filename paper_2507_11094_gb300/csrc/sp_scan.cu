// sp_scan.cu -- device-wide exclusive prefix sums (u32, u64).
//
// Reduce-then-scan: each 2048-element tile is reduced to one sum, the tile
// sums are scanned (recursively), then every tile is scanned again with its
// offset.  Used for CSR layout (row starts from capacities), segment lists
// and per-item counters of the batch merge.
#include "sp_internal.cuh"

namespace sp {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) >= o) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread across the block; returns the
// block total through *total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T *total) {
  __shared__ T warp_sums[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = warp_incl_scan(x);
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T v = lane < kThreads / 32 ? warp_sums[lane] : T(0);
    v = warp_incl_scan(v);
    if (lane < kThreads / 32) warp_sums[lane] = v;
  }
  __syncthreads();
  T warp_off = warp ? warp_sums[warp - 1] : T(0);
  *total = warp_sums[kThreads / 32 - 1];
  __syncthreads();
  return warp_off + incl - x;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_tile_reduce(const T *in, T *sums, long long n) {
  const long long base = (long long)blockIdx.x * kTile;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    long long i = base + k * kThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  T total;
  block_excl_scan(acc, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Scan each tile; add offsets[tile] (or 0 when offsets == nullptr).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const T *in, T *out, long long n,
                                                        const T *offsets) {
  __shared__ T buf[kTile];
  const long long base = (long long)blockIdx.x * kTile;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    long long i = base + k * kThreads + threadIdx.x;
    buf[k * kThreads + threadIdx.x] = i < n ? in[i] : T(0);
  }
  __syncthreads();
  T v[kItems];
  T acc = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = buf[threadIdx.x * kItems + k];
    acc += v[k];
  }
  T total;
  T run = block_excl_scan(acc, &total);
  if (offsets) run += offsets[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    buf[threadIdx.x * kItems + k] = run;
    run += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    long long i = base + k * kThreads + threadIdx.x;
    if (i < n) out[i] = buf[k * kThreads + threadIdx.x];
  }
}

// One block of 1024 threads scans up to kOneBlockMax elements: each thread
// takes a contiguous run, the run totals are scanned across the block, and
// every thread rescans its run with its offset.  One launch instead of three
// for the mid-sized arrays (sort digit tables, segment heads) of a batch.
constexpr int kOneThreads = 1024;
constexpr long long kOneBlockMax = 8192;

template <typename T>
__global__ void __launch_bounds__(kOneThreads) k_scan_one_block(const T *in, T *out,
                                                                long long n) {
  __shared__ T warp_sums[kOneThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const long long per = (n + kOneThreads - 1) / kOneThreads;
  const long long b = t * per, e = b + per < n ? b + per : n;
  T acc = 0;
  for (long long i = b; i < e; ++i) acc += in[i];
  T incl = warp_incl_scan(acc);
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T v = warp_sums[lane];
    v = warp_incl_scan(v);
    warp_sums[lane] = v;
  }
  __syncthreads();
  T run = (warp ? warp_sums[warp - 1] : T(0)) + incl - acc;
  for (long long i = b; i < e; ++i) {
    const T x = in[i];
    out[i] = run;
    run += x;
  }
}

template <typename T>
void scan_rec(const T *in, T *out, long long n, T *tmp, cudaStream_t st, int *launches) {
  if (n <= 0) return;
  long long tiles = (n + kTile - 1) / kTile;
  if (tiles > 1 && n <= kOneBlockMax) {
    k_scan_one_block<T><<<1, kOneThreads, 0, st>>>(in, out, n);
    if (launches) ++*launches;
    return;
  }
  if (tiles == 1) {
    k_tile_scan<T><<<1, kThreads, 0, st>>>(in, out, n, nullptr);
    if (launches) ++*launches;
    return;
  }
  T *sums = tmp;
  T *rest = tmp + tiles;
  k_tile_reduce<T><<<(unsigned)tiles, kThreads, 0, st>>>(in, sums, n);
  scan_rec<T>(sums, sums, tiles, rest, st, launches);
  k_tile_scan<T><<<(unsigned)tiles, kThreads, 0, st>>>(in, out, n, sums);
  if (launches) *launches += 2;
}

}  // namespace

size_t scan_tmp_bytes(long long n) {
  size_t total = 0;
  long long t = n;
  while (t > kTile) {
    t = (t + kTile - 1) / kTile;
    total += (size_t)t;
  }
  return (total + 64) * sizeof(u64);
}

void scan_exclusive_u32(const u32 *in, u32 *out, long long n, void *tmp,
                        cudaStream_t st, int *launches) {
  scan_rec<u32>(in, out, n, (u32 *)tmp, st, launches);
}

void scan_exclusive_u64(const u64 *in, u64 *out, long long n, void *tmp,
                        cudaStream_t st, int *launches) {
  scan_rec<u64>(in, out, n, (u64 *)tmp, st, launches);
}

}  // namespace sp
