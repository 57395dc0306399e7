// sp_noalloc.cu -- sp_export_csr_noalloc: the device-side CSR export without
// any memory allocation.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example a serving process that snapshots a live graph into buffers it
// reserved at start-up (an allocation at that moment could fail under its
// memory budget, or stall behind the allocator's synchronisation), or code
// that runs with a fixed device-memory footprint.  sp_export_csr allocates a
// temporary degree/offset array and scan buffers for every call; this variant
// writes the degrees into the caller's row_off array, prefix-sums them in
// place, and keeps the scan's only temporary (per-tile partial sums) in a
// fixed array compiled into the library.
//
// The fixed array is a file-scope __device__ array: every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits.  Host code
// cannot pass the symbol itself to a kernel -- on the host it is only a
// stand-in, and a kernel given it would fault or, where the GPU can reach host
// memory, silently use the wrong memory -- so the device address is looked up
// once per device with cudaGetSymbolAddress (the first call on each device
// does that look-up; make that first call before any stream capture).  The
// address is cached for the life of the process; it would be stale after a
// reset of the device's primary context, so the library is not to be used on
// a device again after cudaDeviceReset.  All calls share the array: two
// calls whose work overlaps on the GPU (e.g. two graphs exported
// concurrently on different streams) race on it.  The scan writes every
// partial sum it reads, so nothing in the array has to start at zero and a
// call never depends on what an earlier call left there.  A call returns
// after its work on the graph's stream has completed.
#include <mutex>

#include "sp_graph.cuh"

namespace sp {

namespace {

constexpr int kMaxDevices = 64;
constexpr long long kNoAllocMaxVertices = 1LL << 26;             // 67,108,864
constexpr size_t kNoAllocScratchBytes = 512 * 1024;              // scan partials

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` (which must be current).
sp_status scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return SP_ECUDA;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SP_ECUDA;
    }
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return SP_OK;
}

// Row degrees into row_off (as unsigned 64-bit), with row_off[n] = 0 so that
// the exclusive scan leaves the edge count there.
__global__ void k_nx_degrees(const RowMeta *__restrict__ row, int n, u64 *row_off) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r <= n;
       r += (long long)gridDim.x * blockDim.x)
    row_off[r] = r < n ? (u64)row[r].deg : 0ull;
}

// Copy every row to its offset; one warp per row.
__global__ void k_nx_rows(const RowMeta *__restrict__ row, const int2 *__restrict__ adj, int n,
                          const long long *__restrict__ row_off, int *col, int *w) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < n; r += nwarps) {
    const RowMeta rm = row[r];
    const long long o = row_off[r];
    for (int j = lane; j < rm.deg; j += 32) {
      const int2 e = adj[rm.start + j];
      col[o + j] = e.x;
      w[o + j] = e.y;
    }
  }
}

}  // namespace

}  // namespace sp

extern "C" sp_status sp_export_csr_noalloc(sp_graph *g, int reverse, int64_t *row_off,
                                           int32_t *col, int32_t *w) {
  if (!g || !row_off || (g->m > 0 && (!col || !w))) return SP_EINVAL;
  if ((long long)g->n > sp::kNoAllocMaxVertices) return SP_EINVAL;   // beyond the fixed scratch
  if (sp::scan_tmp_bytes((long long)g->n + 1) > sp::kNoAllocScratchBytes) return SP_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device) {
    cudaGetLastError();
    return SP_EINVAL;   // the graph's device must be current
  }
  void *scratch = nullptr;
  sp_status rc = sp::scratch_address(dev, &scratch);
  if (rc != SP_OK) return rc;
  const sp::Store &st = reverse ? g->rev : g->fwd;
  const unsigned grid = (unsigned)(g->num_sms > 0 ? g->num_sms * 8 : 1);
  int launches = 0;
  sp::k_nx_degrees<<<grid, 256, 0, g->stream>>>(st.row, g->n, (sp::u64 *)row_off);
  sp::scan_exclusive_u64((const sp::u64 *)row_off, (sp::u64 *)row_off, (long long)g->n + 1,
                         scratch, g->stream, &launches);
  sp::k_nx_rows<<<grid, 256, 0, g->stream>>>(st.row, st.adj, g->n, (const long long *)row_off,
                                             col, w);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(g->stream) != cudaSuccess) {
    cudaGetLastError();
    return SP_ECUDA;
  }
  return SP_OK;
}
